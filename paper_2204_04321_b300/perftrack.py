"""Changepoint detection for performance time series (paper Sec. 4.5, Algorithm 1 and the
sequential multiple-changepoint method described after it).

A performance metric recorded run after run (wall time, wedges/s, ...) is log-transformed (the paper
finds a log-normal fit slightly better) and scanned for abrupt level changes:

* single detection (Algorithm 1): the k largest jumps between consecutive samples are the candidate
  split points nu; each is tested with a two-sample t-test of the samples before and after it; a
  candidate is a changepoint when |t| exceeds the Student-t critical value for n - 2 degrees of
  freedom at level alpha / (2 k) (Bonferroni over the k tests);
* outliers: in every t-test each sample is cleaned with the median absolute deviation (threshold
  equivalent to three standard deviations), removing at most 10 % of it;
* sequential use: the series is traversed run by run; each test sees at most the last w samples
  since the last confirmed changepoint; a changepoint is confirmed once the same index has been the
  strongest detection m runs in a row, and data before it are then disregarded;
* quantification: between confirmed changepoints, the 99 % confidence interval of the difference
  of mean log values (Student t) is transformed back into a ratio (Eq. mean-transform).

Readings where the paper is silent: the t-test is the pooled-variance (Student) test, whose degrees
of freedom n1 + n2 - 2 match the n - 2 of the algorithm's critical value; a split needs at least
three samples on each side (t-tests on two samples at the Bonferroni level alpha / 2k are dominated
by chance, and the paper notes that a change typically takes three runs to detect); the strongest
changepoint of a window is the one with the largest |t|.

    python -m paper_2204_04321_b300.perftrack bench_*.json [--key value] [--lower-is-better]
"""
from __future__ import annotations

import argparse
import json
import math
from dataclasses import dataclass, field

import numpy as np
from scipy import stats

ALPHA = 0.005
K_LARGEST = 10
M_CONSECUTIVE = 3
LOOKBACK = 30
MAD_SIGMAS = 3.0
MAD_TO_SD = 1.4826           # sd / MAD of a normal distribution
MAX_OUTLIER_FRACTION = 0.10
MIN_SIDE = 3                 # samples required on each side of a split


def mad_clean(x: np.ndarray) -> np.ndarray:
    """Drop the samples farther than three (MAD-estimated) standard deviations from the median,
    the farthest first, at most 10 % of the sample."""
    x = np.asarray(x, dtype=np.float64)
    if x.size < 3:
        return x
    med = np.median(x)
    sd = MAD_TO_SD * np.median(np.abs(x - med))
    if sd == 0.0:
        return x
    dev = np.abs(x - med)
    far = np.nonzero(dev > MAD_SIGMAS * sd)[0]
    limit = int(math.floor(MAX_OUTLIER_FRACTION * x.size))
    drop = far[np.argsort(dev[far])[::-1][:limit]]
    keep = np.ones(x.size, dtype=bool)
    keep[drop] = False
    return x[keep]


def t_statistic(a: np.ndarray, b: np.ndarray) -> float:
    """Pooled-variance two-sample t statistic of mean(b) - mean(a)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    na, nb = a.size, b.size
    ssa = np.sum((a - a.mean()) ** 2)
    ssb = np.sum((b - b.mean()) ** 2)
    sp2 = (ssa + ssb) / (na + nb - 2)
    se = math.sqrt(sp2 * (1.0 / na + 1.0 / nb))
    diff = b.mean() - a.mean()
    if se == 0.0:
        return 0.0 if diff == 0.0 else math.copysign(math.inf, diff)
    return diff / se


def changepoints(x, alpha: float = ALPHA, k: int = K_LARGEST, clean: bool = True):
    """Single changepoint detection (Algorithm 1) on the series x (already log-transformed).
    Returns (C, S): the accepted split indices nu (x[:nu] before, x[nu:] after) in the order the
    candidates were tested, and their t statistics."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    C, S = [], {}
    if n < 2 * MIN_SIDE:
        return C, S
    tcrit = stats.t.ppf(1.0 - alpha / (2.0 * k), n - 2)
    jumps = np.abs(np.diff(x))                      # jump i sits between x[i] and x[i + 1]
    order = np.argsort(jumps, kind="stable")[::-1]  # largest jumps first
    for i in order[:k]:
        nu = int(i) + 1
        if nu < MIN_SIDE or n - nu < MIN_SIDE:
            continue
        a, b = x[:nu], x[nu:]
        if clean:
            a, b = mad_clean(a), mad_clean(b)
        t = t_statistic(a, b)
        if abs(t) > tcrit:
            C.append(nu)
            S[nu] = t
    return C, S


@dataclass
class Tracker:
    """Sequential multiple-changepoint detection over a growing series."""

    alpha: float = ALPHA
    k: int = K_LARGEST
    m: int = M_CONSECUTIVE
    w: int = LOOKBACK
    values: list = field(default_factory=list)
    confirmed: list = field(default_factory=list)    # [(index, run at which it was confirmed)]
    _streak: tuple = (None, 0)                       # (candidate index, consecutive detections)

    def add(self, x: float):
        """Append one (log-transformed) sample; returns a newly confirmed index or None."""
        self.values.append(float(x))
        n = len(self.values)
        start = self.confirmed[-1][0] if self.confirmed else 0
        lo = max(start, n - self.w)
        C, S = changepoints(np.array(self.values[lo:]), self.alpha, self.k)
        if not C:
            self._streak = (None, 0)
            return None
        best = lo + max(C, key=lambda nu: abs(S[nu]))
        cand, count = self._streak
        count = count + 1 if cand == best else 1
        self._streak = (best, count)
        if count >= self.m:
            self.confirmed.append((best, n - 1))
            self._streak = (None, 0)
            return best
        return None


def ratio_ci(before, after, level: float = 0.99):
    """Relative change exp(mean(after) - mean(before)) of log values with its confidence interval
    (pooled-variance Student t), as in Eq. mean-transform."""
    a = np.asarray(before, dtype=np.float64)
    b = np.asarray(after, dtype=np.float64)
    na, nb = a.size, b.size
    diff = b.mean() - a.mean()
    sp2 = (np.sum((a - a.mean()) ** 2) + np.sum((b - b.mean()) ** 2)) / (na + nb - 2)
    half = stats.t.ppf(0.5 + level / 2.0, na + nb - 2) * math.sqrt(sp2 * (1.0 / na + 1.0 / nb))
    return math.exp(diff), (math.exp(diff - half), math.exp(diff + half))


def track(series, **kw):
    """Run the sequential detection over a whole series of positive metric values; returns the
    confirmed changepoints with the ratio (after / before) and its 99 % interval per segment pair."""
    logs = np.log(np.asarray(series, dtype=np.float64))
    tr = Tracker(**kw)
    for v in logs:
        tr.add(v)
    idx = [c for c, _ in tr.confirmed]
    bounds = [0] + idx + [logs.size]
    out = []
    for j, (c, run) in enumerate(tr.confirmed):
        before, after = logs[bounds[j]:c], logs[c:bounds[j + 2]]
        r, (lo, hi) = ratio_ci(before, after)
        out.append({"index": c, "confirmed_at": run, "ratio": r, "ci99": [lo, hi]})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("files", nargs="+", help="benchmark JSON lines, one run per file or line, in run order")
    ap.add_argument("--key", default="value", help="metric key of the JSON line (dotted path allowed)")
    ap.add_argument("--lower-is-better", action="store_true")
    args = ap.parse_args(argv)
    series = []
    for path in args.files:
        with open(path) as f:
            for line in f:
                line = line.strip()
                if not line.startswith("{"):
                    continue
                d = json.loads(line)
                for part in args.key.split("."):
                    d = d.get(part) if isinstance(d, dict) else None
                if isinstance(d, (int, float)) and d > 0:
                    series.append(float(d))
    res = track(series)
    for r in res:
        better = (r["ratio"] < 1) if args.lower_is_better else (r["ratio"] > 1)
        r["kind"] = "improvement" if better else "regression"
    print(json.dumps({"runs": len(series), "changepoints": res}, indent=1))


if __name__ == "__main__":
    main()
