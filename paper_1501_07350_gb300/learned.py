"""Learned choice of an execution candidate (the run-time tuning of Sec. 3.2.3).

The paper's tuner runs every communication method twice during
initialisation and keeps the fastest.  Here that exhaustive timing becomes the
dataset writer and the reference of the regret: ``collect`` times every candidate of many
problems (``openfft_tune_times``), ``train`` fits the cost model on the GPU with
the library's own kernels (``openfft_mlp_train``), and ``evaluate`` reports,
per held-out problem, the regret t(learned pick) / t(exhaustive best) - 1, the
speed-up over the default candidate (tuning switched off) and the tuning time
the learned pick avoids.

Usage (on a GPU machine):
    python -m paper_1501_07350_gb300.learned collect --out timings.json
    python -m paper_1501_07350_gb300.learned train --data timings.json --out model.json
    python -m paper_1501_07350_gb300.learned families --data timings.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

from . import openfft as of
from . import synth

HIDDEN = 32
HERE = os.path.dirname(os.path.abspath(__file__))
DATA_DIR = os.path.join(HERE, "data")
TIMINGS_FILE = os.path.join(DATA_DIR, "tuning_timings_gb300.json")
MODEL_FILE = os.path.join(DATA_DIR, "cost_model_gb300.json")

# the five benchmark configurations, held out of training
HELD_OUT = [((32, 32, 32), 4, "f64"), ((256, 256, 256), 16, "f64"), ((256, 256, 256), 64, "f64"),
            ((256, 256, 256), 256, "f64"), ((256, 256, 256), 64, "f32"), ((120, 144, 160), 32, "f64"),
            ((120, 144, 160), 32, "f32"), ((512, 512, 512), 64, "f64"), ((512, 512, 512), 128, "f64"),
            ((512, 512, 512), 256, "f64"), ((512, 512, 512), 512, "f64"), ((512, 512, 512), 1024, "f64")]


def default_problems():
    """Training problems: cubes, mixed-radix and non-cubic shapes, both dtypes, several P."""
    probs = []
    for dt in ("f64", "f32"):
        for n, Ps in ((32, (1, 8)), (64, (4, 32)), (128, (8, 128)), (256, (4, 1024))):
            for P in Ps:
                probs.append(((n, n, n), P, dt))
        for shape, P in (((48, 48, 48), 8), ((96, 96, 96), 8), ((100, 108, 120), 8), ((64, 128, 256), 16),
                         ((256, 128, 64), 32), ((160, 144, 120), 20), ((36, 40, 30), 12), ((200, 100, 50), 10),
                         ((60, 90, 150), 15), ((24, 250, 30), 6), ((128, 64, 32), 64), ((144, 144, 144), 48),
                         ((512, 128, 128), 64), ((80, 80, 80), 5), ((192, 96, 48), 24), ((320, 160, 64), 40),
                         ((512, 256, 128), 32), ((256, 512, 256), 64), ((512, 512, 128), 128), ((512, 64, 64), 8),
                         ((384, 96, 96), 24), ((16, 16, 16), 4), ((32, 64, 32), 16), ((48, 64, 40), 8),
                         ((96, 200, 64), 16), ((64, 64, 512), 32), ((128, 512, 64), 16), ((256, 256, 128), 8),
                         ((128, 128, 128), 2), ((32, 32, 64), 32), ((64, 32, 32), 1), ((160, 160, 160), 80)):
            probs.append((shape, P, dt))
    probs.append(((512, 512, 512), 32, "f32"))
    probs.append(((512, 512, 256), 16, "f64"))
    probs.append(((512, 256, 512), 2048, "f64"))
    return probs


def _dtype(name: str) -> int:
    return of.C2C_F64 if name == "f64" else of.C2C_F32


def collect(problems, stream=None, log=None, passes=3):
    """Exhaustive timings of every candidate of every problem (the dataset).

    Each pass times every candidate twice (the tuner's protocol); the dataset
    keeps the fastest of all passes, which damps the noise of a shared GPU."""
    rows = []
    for shape, P, dt in problems:
        h = of.openfft_plan(shape[0], shape[1], shape[2], P, _dtype(dt))
        try:
            if stream is not None:
                of.openfft_set_stream(h, stream)
            ms = of.openfft_tune_times(h)
            for _ in range(passes - 1):
                ms = np.where((ms < 0) | (ms == 0), ms, np.minimum(ms, of.openfft_tune_times(h)))
            nc = of.openfft_num_candidates(h)
            rows.append({"shape": list(shape), "P": P, "dtype": dt,
                         "candidates": [of.openfft_candidate(h, i) for i in range(nc)],
                         "features": [of.openfft_candidate_features(h, i).tolist() for i in range(nc)],
                         "ms": [float(t) for t in ms]})
            if log:
                log("%s P=%d %s: best %.4f ms (candidate %d), default %.4f ms" % (
                    shape, P, dt, min(t for t in ms if t >= 0), int(np.argmin(np.where(ms >= 0, ms, 1e30))), ms[0]))
        finally:
            of.openfft_destroy(h)
    return rows


def save(obj, path):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as fh:
        json.dump(obj, fh)


def load_rows(path=TIMINGS_FILE):
    with open(path) as fh:
        return json.load(fh)["rows"]


def _key(row):
    return (tuple(row["shape"]), row["P"], row["dtype"])


def _has_factor(n: int, primes) -> bool:
    return any(n % q == 0 for q in primes)


# Held-out shape families: the benchmark problems of a family are evaluated
# by a model trained without ANY problem of that family, so that a near-twin
# in the training set cannot stand in for generalisation.
FAMILIES = {
    "512-point axes": (lambda shape: 512 in shape,
                       [k for k in HELD_OUT if 512 in k[0]]),
    "axes with a factor 3 or 5": (lambda shape: any(_has_factor(n, (3, 5)) for n in shape),
                                  [k for k in HELD_OUT if any(_has_factor(n, (3, 5)) for n in k[0])]),
}


def family_split(rows, family):
    """(training rows: no problem of the family and no benchmark problem;
    the family's benchmark rows)."""
    member, bench = FAMILIES[family]
    keys = {(tuple(s), P, dt) for s, P, dt in bench}
    every = {(tuple(s), P, dt) for s, P, dt in HELD_OUT}
    return ([r for r in rows if not member(tuple(r["shape"])) and _key(r) not in every],
            [r for r in rows if _key(r) in keys])


def evaluate_families(rows, steps=8000):
    """Per family: train without the family, evaluate on its benchmark problems."""
    out = {}
    for fam in FAMILIES:
        tr, te = family_split(rows, fam)
        ps, _ = train(tr, steps=steps)
        ev = evaluate(te, ps)
        out[fam] = {"train_problems": len(tr), "summary": summary(ev), "problems": ev}
    return out


def split(rows, held_out=HELD_OUT):
    ho = {(tuple(s), P, dt) for s, P, dt in held_out}
    train_rows = [r for r in rows if _key(r) not in ho]
    test_rows = [r for r in rows if _key(r) in ho]
    return train_rows, test_rows


TARGET_CAP = 1.0
ENSEMBLE = 5


def arrays(rows):
    """Features and targets of every candidate that ran.

    The target is log(t / t_best of the problem), capped at TARGET_CAP: only
    the order of a problem's candidates matters to the pick, the problem's
    own scale (three decades) is removed, and candidates more than e times
    slower than the best are all just "slow", so the fit spends its capacity
    on the candidates near the top."""
    X, y = [], []
    for r in rows:
        best = math.log(min(t for t in r["ms"] if t > 0))
        for f, t in zip(r["features"], r["ms"]):
            if t > 0:
                X.append(f)
                y.append(min(math.log(t) - best, TARGET_CAP))
    return np.asarray(X, dtype=np.float32), np.asarray(y, dtype=np.float32)


def init_params(d: int, hidden: int, seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases, from the seeded SplitMix64 stream."""
    u = synth.uniform01(seed, d * hidden + hidden * hidden + hidden)
    p = np.zeros(of.openfft_mlp_num_params(d, hidden), dtype=np.float64)
    o = k = 0
    for fan_in, fan_out in ((d, hidden), (hidden, hidden)):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        cnt = fan_in * fan_out
        p[o:o + cnt] = (2.0 * u[k:k + cnt] - 1.0) * a
        o += cnt + fan_out
        k += cnt
    a = math.sqrt(6.0 / (hidden + 1))
    p[o:o + hidden] = (2.0 * u[k:k + hidden] - 1.0) * a
    return p.astype(np.float32)


def train(rows, hidden=HIDDEN, steps=8000, lr=3e-3, seed=150107355, members=ENSEMBLE):
    """Fit an ensemble of cost models on the GPU (the library's forward /
    backward / Adam kernels), one per seed; returns (list of params, losses of
    the first member)."""
    X, y = arrays(rows)
    d = X.shape[1]
    params, first = [], None
    for k in range(members):
        p0 = init_params(d, hidden, seed + k)
        p, losses = of.openfft_mlp_train(d, hidden, X, y, steps, lr, p0)
        params.append(p)
        first = losses if first is None else first
    return params, first


def pick(params, features, hidden=HIDDEN, ms=None):
    """Candidate of lowest mean predicted time over the ensemble (skipping
    candidates known not to run)."""
    F = np.asarray(features, dtype=np.float32)
    if not isinstance(params, (list, tuple)):
        params = [params]
    pred = np.mean([of.openfft_mlp_predict(F.shape[1], hidden, p, F) for p in params], axis=0)
    if ms is not None:
        pred = np.where(np.asarray(ms) > 0, pred, np.inf)
    return int(np.argmin(pred)), pred


def install(path=MODEL_FILE):
    """Install the committed ensemble for OPENFFT_TUNE_LEARNED."""
    with open(path) as fh:
        m = json.load(fh)
    flat = np.concatenate([np.asarray(p, dtype=np.float32) for p in m["params"]])
    of.openfft_set_cost_model(m["d"], m["hidden"], flat, count=len(m["params"]))
    return m


def evaluate(rows, params, hidden=HIDDEN):
    """Per problem: regret of the learned pick, speed-up over the default, tuning cost avoided."""
    out = []
    for r in rows:
        ms = np.asarray(r["ms"], dtype=np.float64)
        ok = ms > 0
        best = float(ms[ok].min())
        i, _ = pick(params, r["features"], hidden, r["ms"])
        t_pick = float(ms[i]) if ms[i] > 0 else float("inf")
        out.append({"shape": r["shape"], "P": r["P"], "dtype": r["dtype"], "pick": i,
                    "best": int(np.argmin(np.where(ok, ms, np.inf))),
                    "t_pick_ms": t_pick, "t_best_ms": best, "t_default_ms": float(ms[0]),
                    "regret": t_pick / best - 1.0, "speedup_vs_default": float(ms[0]) / t_pick,
                    "tuning_cost_ms": float(2.0 * ms[ok].sum())})
    return out


def summary(ev):
    reg = [e["regret"] for e in ev]
    # the problems where tuning matters: the default candidate is not the best
    hard = [e for e in ev if e["best"] != 0]
    return {"problems": len(ev), "mean_regret": float(np.mean(reg)), "max_regret": float(np.max(reg)),
            "geomean_speedup_vs_default": float(np.exp(np.mean([math.log(e["speedup_vs_default"]) for e in ev]))),
            "default_not_best": len(hard),
            "geomean_speedup_vs_default_where_default_not_best":
                float(np.exp(np.mean([math.log(e["speedup_vs_default"]) for e in hard]))) if hard else None,
            "tuning_cost_avoided_ms": float(sum(e["tuning_cost_ms"] for e in ev))}


def main(argv=None):
    ap = argparse.ArgumentParser(description="timings dataset and cost model of the learned tuner")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("--out", default=TIMINGS_FILE)
    c.add_argument("--held-out-only", action="store_true")
    t = sub.add_parser("train")
    t.add_argument("--data", default=TIMINGS_FILE)
    t.add_argument("--out", default=MODEL_FILE)
    t.add_argument("--steps", type=int, default=8000)
    f = sub.add_parser("families")
    f.add_argument("--data", default=TIMINGS_FILE)
    f.add_argument("--steps", type=int, default=8000)
    args = ap.parse_args(argv)
    if args.cmd == "collect":
        import torch
        probs = [(s, P, dt) for s, P, dt in HELD_OUT]
        if not args.held_out_only:
            probs = default_problems() + probs
        rows = collect(probs, stream=torch.cuda.current_stream(), log=lambda m: print(m, file=sys.stderr))
        save({"device": torch.cuda.get_device_name(0), "rows": rows}, args.out)
        print(args.out)
    elif args.cmd == "families":
        fam = evaluate_families(load_rows(args.data), steps=args.steps)
        print(json.dumps({k: {"train_problems": v["train_problems"], "summary": v["summary"],
                              "regrets": [round(e["regret"], 4) for e in v["problems"]]} for k, v in fam.items()}))
    else:
        rows = load_rows(args.data)
        tr, te = split(rows)
        ps, losses = train(tr, steps=args.steps)
        ev = evaluate(te, ps)
        save({"hidden": HIDDEN, "d": len(tr[0]["features"][0]), "params": [[float(v) for v in p] for p in ps],
              "target_cap": TARGET_CAP, "train_loss": [float(losses[0]), float(losses[-1])],
              "held_out": summary(ev), "held_out_problems": ev}, args.out)
        print(json.dumps(summary(ev)))


if __name__ == "__main__":
    main()
