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


def test_reference_arm_prints_the_gpu_arms_config():
    """Both arms name the same workload dict, so the two lines compare like for like."""
    import argparse
    bench = load_bench()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0"),
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 1
    assert line["config"] == bench.bench_config(argparse.Namespace(mesh_m=224, layers=10), 1)
    assert line["e2e"]["value"] == line["value"] == line["cpu_baseline"]["value"]


def test_headline_is_short_and_last():
    """The line's last key carries the nested sections' key figures in a short tail."""
    bench = load_bench()
    solve = {"s": 0.0214, "converged": True, "newton_iters": 12, "krylov_iters": 138}
    kinds = ["f64", "mixed_f32", "f64_accurate_double_single", "mixed_f32_double_single",
             "mixed_f32_double_single_value32_until_1e-4"] + [f"mixed_f32_value32_until_{t}" for t in
                                                               ("0.01", "0.001", "0.0001", "1e-05")] + \
        ["f64_mdsc", "mixed_f32_mdsc", "mixed_f32_mdsc_amg", "mixed_f32_gmres50"]
    dome = {k: dict(solve) for k in kinds}
    dome["learned_start_mixed"] = {"unseen_beta_fields": {"seeds": 40, "speedup_learned_picard_vs_sia": 1.0881,
                                                          "ci99": [1.0264, 1.1534]}}
    line = {"roofline": {"kernel_ms": 3.5654, "frac": 0.8012},
            "secondary": {"residual_only": {"ms": 0.774}, "jacobian_f32_lanes": {"ms": 0.893},
                          "jacobian_paired_lanes_double_single_values": {"ms": 2.54},
                          "jacobian_f32_lanes_double_single_values": {"ms": 0.68}},
            "newton": {"dome-100k-tri-x10": dome,
                       "dome-400k-tri-x10": {k: dict(solve) for k in kinds[:6]},
                       "marine-100k-tri-x10": {k: dict(solve) for k in kinds[:4]}},
            "ensemble": {"value": 2.75e8}, "mlp": {"inference": {"ms": 0.023}, "train_step": {"ms": 0.17}}}
    h = bench.headline(line)
    assert len(json.dumps(h)) < 1500
    assert h["learned_picard_vs_sia"] == {"seeds": 40, "speedup": 1.088, "ci99": [1.026, 1.153]}
    assert h["newton_1M_ms"]["mixed_f32_double_single_value32_until_1e-4"] == 21.4
    assert h["assembly_ms"]["f64x2_ds"] == 2.54 and h["roofline_frac"] == 0.801
    assert bench.headline({}) == {"assembly_ms": {k: None for k in ("f64", "f64x2_ds", "f32_ds", "f32_lanes",
                                                                     "residual")}, "roofline_frac": None}


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
