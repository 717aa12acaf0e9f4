"""Element-wise parity of the kernel instantiations the benchmark times.

Every comparison here is over a whole output array against the FP64 oracle
(oracle.fft3d, the paper's steps (1)-(6) of Sec. 3.1.1 computed literally),
element by element through the relative L2 norm, at the bars of the other
GPU tests: 1e-12 for the complex128 plans (double-float and native FP64),
1e-5 for complex64 (FP32) against the oracle on the same input upcast.

  * Shapes with a 256- or 512-point axis in each stage position drive the
    power-of-two warp-per-line stage kernels (n = 256 with 4 or 8 lines per
    CTA, n = 512 with 8) and every other candidate of the plan, both
    directions.
  * 256^3 at P = 16, 64 and 256: the default candidate and the exhaustively
    tuned one, both directions, FP64-accurate and FP32, plus the
    host-buffer entry points (openfft_exec_c2c_host_async).
  * 512^3 at P = 64, 256 and 1024, tuned, both directions (the oracle needs
    about 12 GB of host memory and half a minute per direction).
  * The 64-transform batch of the benchmark (sizes drawn from its seed), every
    transform against the oracle.

The oracle's result does not depend on P (every rank transforms whole lines,
and the transposes move values unchanged), so one oracle run serves all P of
a shape; the decomposition itself is checked bit-exactly elsewhere.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.C2C_F64: 1e-12, of.C2C_F32: 1e-5}
_REF = {}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _ref(key, fn):
    if key not in _REF:
        _REF[key] = fn()
    return _REF[key]


def _dev(torch, x, dtype):
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(device="cuda", dtype=tdt)


def _exec(torch, plan, xd, direction):
    yd = torch.full_like(xd, float("nan"))
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_c2c(plan, xd, yd, direction)
    of.openfft_sync(plan)
    return yd.cpu().numpy().astype(np.complex128)


def _rounded(x, dtype):
    """The input as the plan sees it (complex64 plans round it once)."""
    return x if dtype == of.C2C_F64 else x.astype(np.complex64).astype(np.complex128)


# ------------------------------------- 256- and 512-point axes, every candidate --

AXIS_SHAPES = [((256, 256, 32), 16), ((32, 256, 256), 16), ((256, 32, 256), 64),
               ((512, 64, 32), 64), ((32, 512, 64), 64), ((64, 32, 512), 1024)]


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
@pytest.mark.parametrize("shape,P", AXIS_SHAPES)
def test_long_power_of_two_axes_every_candidate(torch, shape, P, dtype):
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=Na * 7 + Nb * 11 + Nc * 13)
    xin = _rounded(x, dtype)
    ref_f = oracle.fft3d(xin, Na, Nb, Nc, P, oracle.FORWARD)
    ref_b = oracle.fft3d(xin, Na, Nb, Nc, P, oracle.BACKWARD)     # x read as a cba spectrum
    xd = _dev(torch, x, dtype)
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        for c in range(of.openfft_num_candidates(plan)):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            cand = of.openfft_candidate(plan, c)
            e_f = oracle.rel_l2(_exec(torch, plan, xd, of.FORWARD), ref_f)
            e_b = oracle.rel_l2(_exec(torch, plan, xd, of.BACKWARD), ref_b)
            assert e_f < TOL[dtype] and e_b < TOL[dtype], (shape, P, cand, e_f, e_b)
    finally:
        of.openfft_destroy(plan)


# Ragged tiles of the asynchronous-output kernels: the grouped line count is
# not a multiple of the tile (4 / 8 lines complex128, 8 / 16 complex64), so
# the last tile's tensor store is clipped at the output's edge, and the
# per-line contiguous store leaves its missing lines out.  (6, 256, 7):
# forward stage 2 grouped over 6 lines, backward stage 2 over 7;
# (5, 6, 512): forward stage 1 over 30; (512, 5, 6): backward stage 1 over 5
# and the contiguous forward stage 3.
RAGGED_SHAPES = [((6, 256, 7), 6), ((5, 6, 512), 5), ((512, 5, 6), 3)]


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
@pytest.mark.parametrize("shape,P", RAGGED_SHAPES)
def test_async_output_ragged_tiles_every_candidate(torch, shape, P, dtype):
    test_long_power_of_two_axes_every_candidate(torch, shape, P, dtype)


# ------------------------------------------------------------- 256^3 ------

def _x256():
    return synth.complex_field((256, 256, 256), seed=synth.config_seed(2), dist="normal")


def _y256():
    # an independent cba-ordered spectrum for the backward direction
    return synth.complex_field((256 ** 3,), seed=synth.config_seed(2) + 1000, dist="normal")


def _ref256(dtype, direction):
    def run():
        x = _x256() if direction == oracle.FORWARD else _y256()
        return oracle.fft3d(_rounded(x, dtype), 256, 256, 256, 16, direction)
    return _ref(("256", dtype, direction), run)


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
@pytest.mark.parametrize("P", [16, 64, 256])
def test_256cubed_whole_output_default_and_tuned(torch, P, dtype):
    n = 256
    xd = _dev(torch, _x256(), dtype)
    yd = _dev(torch, _y256(), dtype)
    ref_f = _ref256(dtype, oracle.FORWARD)
    ref_b = _ref256(dtype, oracle.BACKWARD)
    plan = of.openfft_plan(n, n, n, P, dtype)
    try:
        picks = []
        for mode in (of.TUNE_DEFAULT, of.TUNE_EXHAUSTIVE):
            of.openfft_set_tuning(plan, mode)
            picks.append(of.openfft_current_candidate(plan))
            cand = of.openfft_candidate(plan, picks[-1])
            e_f = oracle.rel_l2(_exec(torch, plan, xd, of.FORWARD), ref_f)
            e_b = oracle.rel_l2(_exec(torch, plan, yd, of.BACKWARD), ref_b)
            assert e_f < TOL[dtype] and e_b < TOL[dtype], (P, mode, cand, e_f, e_b)
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
def test_256cubed_host_buffers_whole_output(torch, dtype):
    """The host-buffer path the end-to-end figure times: page-locked buffers,
    the asynchronous call on shared copy streams, then openfft_sync."""
    n, P = 256, 64
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    hx = torch.from_numpy(_x256().reshape(-1)).to(tdt).pin_memory()
    hy = torch.from_numpy(_y256()).to(tdt).pin_memory()
    out_f = torch.full_like(hx, float("nan")).pin_memory()
    out_b = torch.full_like(hx, float("nan")).pin_memory()
    h2d = torch.cuda.Stream()
    d2h = torch.cuda.Stream()
    plan = of.openfft_plan(n, n, n, P, dtype)
    try:
        of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
        of.openfft_set_copy_streams(plan, h2d, d2h)
        of.openfft_exec_c2c_host_async(plan, hx.numpy(), out_f.numpy(), of.FORWARD)
        of.openfft_exec_c2c_host_async(plan, hy.numpy(), out_b.numpy(), of.BACKWARD)
        of.openfft_sync(plan)
        e_f = oracle.rel_l2(out_f.numpy().astype(np.complex128), _ref256(dtype, oracle.FORWARD))
        e_b = oracle.rel_l2(out_b.numpy().astype(np.complex128), _ref256(dtype, oracle.BACKWARD))
        assert e_f < TOL[dtype] and e_b < TOL[dtype], (e_f, e_b)
    finally:
        of.openfft_destroy(plan)


# ------------------------------------------------------------- 512^3 ------

def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def _x512():
    return synth.complex_field((512, 512, 512), seed=synth.config_seed(5))


def _y512():
    return synth.complex_field((512 ** 3,), seed=synth.config_seed(5) + 1000)


def test_512cubed_whole_output_tuned(torch):
    """512^3 complex128 at P = 64, 256 and 1024, exhaustively tuned, both
    directions, every element against the oracle."""
    if _mem_available_gb() < 40:
        pytest.skip("512^3 oracle needs about 12 GB of free host memory beyond the arrays")
    n = 512
    x = _x512()
    ref_f = oracle.fft3d(x, n, n, n, 64, oracle.FORWARD)
    xd = _dev(torch, x, of.C2C_F64)
    del x
    outs = {}
    for P in (64, 256, 1024):
        plan = of.openfft_plan(n, n, n, P, of.C2C_F64)
        try:
            of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
            outs[P] = (of.openfft_candidate(plan, of.openfft_current_candidate(plan)),
                       oracle.rel_l2(_exec(torch, plan, xd, of.FORWARD), ref_f))
        finally:
            of.openfft_destroy(plan)
    del ref_f
    for P, (cand, e) in outs.items():
        assert e < TOL[of.C2C_F64], ("forward", P, cand, e)
    y = _y512()
    ref_b = oracle.fft3d(y, n, n, n, 64, oracle.BACKWARD)
    yd = _dev(torch, y, of.C2C_F64)
    del y
    for P in (64, 256, 1024):
        plan = of.openfft_plan(n, n, n, P, of.C2C_F64)
        try:
            of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
            cand = of.openfft_candidate(plan, of.openfft_current_candidate(plan))
            e = oracle.rel_l2(_exec(torch, plan, yd, of.BACKWARD), ref_b)
            assert e < TOL[of.C2C_F64], ("backward", P, cand, e)
        finally:
            of.openfft_destroy(plan)


# --------------------------------------------- the benchmark's 64-transform batch --

def test_batch_of_the_benchmark_every_transform(torch):
    """The 64 uneven complex64 transforms of the benchmark, drawn from its seed,
    in one persistent launch: each output against the oracle on its own input."""
    count = 64
    shapes = synth.batch_shapes(synth.config_seed(4), count)
    Ps = [8] * count
    xs = [synth.complex_field((a * b * c,), seed=synth.config_seed(4) + 1 + i)
          for i, (a, b, c) in enumerate(shapes)]
    xd = [_dev(torch, x, of.C2C_F32) for x in xs]
    yd = [torch.full_like(x, float("nan")) for x in xd]
    plan = of.openfft_plan_many(shapes, Ps, of.C2C_F32)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        of.openfft_exec_many(plan, xd, yd, of.FORWARD)
        of.openfft_sync(plan)
        for i, ((Na, Nb, Nc), x, y) in enumerate(zip(shapes, xs, yd)):
            ref = oracle.fft3d(_rounded(x, of.C2C_F32), Na, Nb, Nc, 8, oracle.FORWARD)
            e = oracle.rel_l2(y.cpu().numpy().astype(np.complex128), ref)
            assert e < TOL[of.C2C_F32], (i, (Na, Nb, Nc), e)
        zd = [torch.full_like(x, float("nan")) for x in xd]
        of.openfft_exec_many(plan, yd, zd, of.BACKWARD)
        of.openfft_sync(plan)
        for i, ((Na, Nb, Nc), y, z) in enumerate(zip(shapes, yd, zd)):
            yin = y.cpu().numpy().astype(np.complex128)
            ref = oracle.fft3d(yin, Na, Nb, Nc, 8, oracle.BACKWARD)
            e = oracle.rel_l2(z.cpu().numpy().astype(np.complex128), ref)
            assert e < TOL[of.C2C_F32], ("backward", i, (Na, Nb, Nc), e)
    finally:
        of.openfft_destroy(plan)
