"""Changepoint detection of performance time series (paper Sec. 4.5, Algorithm 1), on CPU.

Pinned against library statistics (scipy's two-sample t-test and Student-t quantiles), seeded
synthetic series with known steps, and the coverage of the 99 % interval."""
import json
import math

import numpy as np
import pytest
from scipy import stats

from paper_2204_04321_b300 import perftrack as pt


def test_t_statistic_is_the_pooled_two_sample_t_test():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.normal(0.0, 1.0, rng.integers(2, 30))
        b = rng.normal(0.3, 1.5, rng.integers(2, 30))
        ref = stats.ttest_ind(b, a, equal_var=True).statistic
        assert pt.t_statistic(a, b) == pytest.approx(ref, rel=1e-12)


def test_mad_clean_removes_gross_outliers_but_at_most_ten_percent():
    x = 0.01 * stats.norm.ppf(np.linspace(0.02, 0.98, 40))   # normal quantiles, all within 2.1 sd
    np.random.default_rng(1).shuffle(x)
    y = x.copy()
    y[[3, 17]] = [1.0, -2.0]
    c = pt.mad_clean(y)
    assert c.size == 38 and np.all(np.abs(c) < 0.1)
    z = x.copy()
    z[:10] = 5.0            # a quarter of the data far off: only 10 % may go
    assert pt.mad_clean(z).size == 36


def step_series(n=80, at=40, step=0.10, sd=0.02, seed=2):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, sd, n)
    x[at:] += step
    return x


def test_single_detection_finds_the_step():
    x = step_series()
    C, S = pt.changepoints(x)
    assert C and max(C, key=lambda nu: abs(S[nu])) == 40
    assert S[40] > 0     # the level went up


def test_critical_value_is_the_bonferroni_student_quantile():
    """A split whose |t| lies just below t*(n - 2, 1 - alpha / 2k) is rejected, just above accepted."""
    n, alpha, k = 30, 0.005, 10
    tcrit = stats.t.ppf(1 - alpha / (2 * k), n - 2)
    base = np.tile([-1.0, 1.0], n // 2) * 0.01     # alternating noise, one clean jump below
    for factor, expect in ((0.999, False), (1.001, True)):
        # choose the step so that the t statistic of the split at 15 equals factor * tcrit
        x = base.copy()
        a, b = x[:15], x[15:]
        se = math.sqrt(((a - a.mean()) ** 2).sum() + ((b - b.mean()) ** 2).sum()) / math.sqrt(n - 2) * math.sqrt(2 / 15)
        step = factor * tcrit * se - (b.mean() - a.mean())
        x[15:] += step
        C, S = pt.changepoints(x, alpha, k, clean=False)
        assert (15 in C) == expect, (factor, S)


def test_stationary_series_has_no_changepoint():
    rng = np.random.default_rng(3)
    for seed in range(5):
        x = np.random.default_rng(seed).normal(0.0, 0.03, 60)
        assert pt.changepoints(x)[0] == []


def test_sequential_tracking_confirms_after_m_runs_and_ignores_an_outlier():
    x = step_series(n=70, at=40, step=0.15, sd=0.02, seed=4)
    x[20] += 0.5                                   # one bad night
    series = np.exp(x) * 10.0
    res = pt.track(series)
    assert [r["index"] for r in res] == [40]
    assert 40 + pt.M_CONSECUTIVE - 1 <= res[0]["confirmed_at"] <= 40 + pt.M_CONSECUTIVE + 3
    lo, hi = res[0]["ci99"]
    assert lo < math.exp(0.15) < hi and lo > 1.0   # a slowdown of 16 %, significant


def test_two_steps_are_both_found_in_order():
    x = step_series(n=100, at=30, step=-0.2, sd=0.02, seed=5)
    x[65:] += 0.3
    res = pt.track(np.exp(x))
    assert [r["index"] for r in res] == [30, 65]
    assert res[0]["ratio"] < 1 < res[1]["ratio"]


def test_ratio_interval_coverage_is_about_99_percent():
    rng = np.random.default_rng(6)
    true = 0.05
    hits = 0
    trials = 400
    for _ in range(trials):
        a = rng.normal(0.0, 0.03, 20)
        b = rng.normal(true, 0.03, 15)
        _, (lo, hi) = pt.ratio_ci(a, b)
        hits += lo < math.exp(true) < hi
    assert hits / trials >= 0.97


def test_command_line_reads_benchmark_lines(tmp_path, capsys):
    x = np.exp(step_series(n=50, at=25, step=0.2, sd=0.02, seed=7)) * 2.4e8
    files = []
    for i, v in enumerate(x):
        p = tmp_path / f"bench_{i:03d}.json"
        p.write_text("log line\n" + json.dumps({"metric": "wedges/s", "value": float(v)}) + "\n")
        files.append(str(p))
    pt.main(files)
    out = json.loads(capsys.readouterr().out)
    assert out["runs"] == 50 and [c["index"] for c in out["changepoints"]] == [25]
    assert out["changepoints"][0]["kind"] == "improvement"
