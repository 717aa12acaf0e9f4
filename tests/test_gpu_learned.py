"""Learned tuner: the CUDA training/inference kernels against the FP64 oracle,
the LEARNED tuning mode, and the regret of the trained cost model.

- gradients of openfft_mlp_loss_grad (FP32, GPU) vs oracle/mlp.py (FP64):
  max abs difference <= 1e-4 of the largest gradient component;
- a training trajectory (GPU Adam, graph-replayed steps) vs the oracle's Adam;
- OPENFFT_TUNE_LEARNED picks a candidate of the lowest predicted time;
- trained on the committed timing dataset, the model's picks on the held-out
  problems (the benchmark configurations) are within 5 % of exhaustive tuning
  on average, and avoid the exhaustive tuning time;
- trained without any problem that has a 512-point axis, its picks on the
  512^3 benchmark problems are within 5 % of exhaustive tuning too.
"""
import os

import numpy as np
import pytest

from oracle import mlp
from paper_1501_07350_gb300 import learned
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1501_07350_gb300 import _build
    _build.build()
    return of.load()


def _data(n, d, seed):
    X = synth.uniform01(seed, n * d).reshape(n, d)
    y = np.log(0.1 + X @ np.linspace(0.1, 1.0, d)) + 0.3 * np.sin(3 * X[:, 0])
    return X.astype(np.float32), y.astype(np.float32)


def test_gradients_match_fp64_oracle(lib):
    d, H, n = 17, 32, 96
    X, y = _data(n, d, 1)
    p = learned.init_params(d, H, 2)
    p[d * H:d * H + H] = 0.05 * synth.uniform_pm1(3, H)
    L, g = of.openfft_mlp_loss_grad(d, H, p, X, y)
    L_ref, g_ref = mlp.loss_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64), d, H)
    assert abs(L - L_ref) <= 1e-5 * max(1.0, L_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref))


def test_predict_matches_fp64_oracle(lib):
    d, H, n = 17, 32, 40
    X, _ = _data(n, d, 4)
    p = learned.init_params(d, H, 5)
    yhat = of.openfft_mlp_predict(d, H, p, X)
    ref, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64), d, H)
    assert np.max(np.abs(yhat - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_training_trajectory_matches_fp64_adam(lib):
    d, H, n = 17, 16, 64
    X, y = _data(n, d, 6)
    p0 = learned.init_params(d, H, 7)
    steps, lr = 25, 1e-2
    p_gpu, losses_gpu = of.openfft_mlp_train(d, H, X, y, steps, lr, p0)
    p_ref, losses_ref = mlp.train(p0.astype(np.float64), X.astype(np.float64), y.astype(np.float64), d, H, steps, lr)
    assert np.max(np.abs(losses_gpu - losses_ref) / losses_ref) < 1e-3
    assert np.max(np.abs(p_gpu - p_ref)) < 1e-3 * max(1.0, np.max(np.abs(p_ref)))
    assert losses_gpu[-1] < losses_gpu[0]


def test_learned_mode_follows_the_model(lib):
    d, H = of.openfft_num_features(), 4
    p = np.zeros(of.openfft_mlp_num_params(d, H), dtype=np.float32)
    # yhat = -tanh(tanh(2 f14)): lowest for the tile-family candidates (feature 14)
    W1 = np.zeros((d, H), np.float32); W1[14, 0] = 2.0
    W2 = np.zeros((H, H), np.float32); W2[0, 0] = 1.0
    o = 0
    p[o:o + d * H] = W1.ravel(); o += d * H + H
    p[o:o + H * H] = W2.ravel(); o += H * H + H
    p[o] = -1.0
    of.openfft_set_cost_model(d, H, p, count=1)
    try:
        h = of.openfft_plan(48, 64, 40, 8, of.C2C_F64)
        try:
            of.openfft_set_tuning(h, of.TUNE_LEARNED)
            assert of.openfft_candidate(h, of.openfft_current_candidate(h))["kernel"] == of.KERNEL_TILE
        finally:
            of.openfft_destroy(h)
    finally:
        of.openfft_set_cost_model(d, H, None)
    h = of.openfft_plan(48, 64, 40, 8, of.C2C_F64)
    try:
        of.openfft_set_tuning(h, of.TUNE_LEARNED)          # no model installed: the default
        assert of.openfft_current_candidate(h) == 0
    finally:
        of.openfft_destroy(h)


@pytest.mark.skipif(not os.path.exists(learned.TIMINGS_FILE), reason="no committed timing dataset")
def test_trained_model_regret_on_held_out_problems(lib):
    rows = learned.load_rows()
    train_rows, test_rows = learned.split(rows)
    assert len(test_rows) == len(learned.HELD_OUT)
    ps, losses = learned.train(train_rows)
    assert losses[-1] < 0.05 * losses[0]
    ev = learned.evaluate(test_rows, ps)
    s = learned.summary(ev)
    assert s["mean_regret"] <= 0.05, s
    assert s["geomean_speedup_vs_default"] >= 0.97, s
    assert s["tuning_cost_avoided_ms"] > 0
    # family hold-out: no training problem with a 512-point axis when the 512^3
    # benchmark problems are evaluated (the headline configuration)
    fam = learned.evaluate_families(rows)
    f512 = fam["512-point axes"]
    assert f512["summary"]["problems"] == 5
    assert f512["summary"]["mean_regret"] <= 0.05, f512["summary"]
    assert fam["axes with a factor 3 or 5"]["summary"]["problems"] == 2
    # the committed ensemble, installed, drives OPENFFT_TUNE_LEARNED
    learned.install()
    try:
        h = of.openfft_plan(256, 256, 256, 64, of.C2C_F64)
        try:
            of.openfft_set_tuning(h, of.TUNE_LEARNED)
            c = of.openfft_candidate(h, of.openfft_current_candidate(h))
            assert c["variant"] == of.VARIANT_FUSED
        finally:
            of.openfft_destroy(h)
    finally:
        of.openfft_set_cost_model(0, 0, None)
