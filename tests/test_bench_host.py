"""Host logic of the benchmark's multi-rank path, on CPU (gloo, world size 2).

`bench.py --gpus N` runs N independent replicas (weak scaling, no collective on the data path):
every rank times its own steps, the job's time is the slowest rank's (max over ranks), and the
job's throughput counts the units of all ranks.  Under torchrun the reference arm runs on rank 0
only; the other ranks exit 0 without work."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench = load_bench()
    t = 1.5 + rank          # rank 1 is the slow one
    tmax = bench.max_over_ranks(t, ws, "cpu")
    value = bench.job_throughput(ws, 1000, 10, tmax)
    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"tmax": tmax, "value": value}, f)


def test_max_over_ranks_and_job_throughput_two_gloo_ranks(tmp_path):
    ws = 2
    torch.multiprocessing.spawn(_rank_main, args=(ws, free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(ws)]
    for r in res:
        assert r["tmax"] == 2.5                       # every rank sees the slowest rank's time
        assert r["value"] == pytest.approx(2 * 1000 * 10 / 2.5)


def test_single_rank_needs_no_process_group():
    bench = load_bench()
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_throughput(1, 1003520, 100, 0.42) == pytest.approx(1003520 * 100 / 0.42)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_workload_names_agree_between_arms():
    bench = load_bench()
    assert bench.workload_name(224, 10).startswith("dome-100k-tri-x10: ")
    assert "1003520 wedges" in bench.workload_name(224, 10)


def test_traffic_record_hash_follows_code_not_comments(tmp_path):
    """The DRAM-traffic record of the headline kernel is reported only while the kernel's code is
    the one it was captured from: a comment edit keeps the hash, a code edit changes it."""
    import shutil
    bench = load_bench()
    csrc = os.path.join("paper_2204_04321_b300", "csrc")
    os.makedirs(tmp_path / csrc)
    for name in ("bp_column.cuh", "bp_internal.cuh"):
        shutil.copy(os.path.join(ROOT, csrc, name), tmp_path / csrc / name)
    bench.ROOT = str(tmp_path)
    h0 = bench.kernel_hash()
    col = tmp_path / csrc / "bp_column.cuh"
    src = col.read_text()
    i = src.index("\n", src.index("constexpr int MODE_RES")) + 1  # inside the hashed part
    col.write_text(src[:i] + "// an added comment line\n/* and a block\n   comment */\n\n" + src[i:] +
                   "\n// trailing note\n")
    assert bench.kernel_hash() == h0
    col.write_text(src.replace("TL(0.5) * yy", "TL(0.25) * yy", 1))
    assert bench.kernel_hash() != h0
