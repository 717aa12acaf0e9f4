"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bars (fixed before the first GPU run):
  - transposes: bit-exact (they move bytes);
  - FP64 plans (native and double-float arithmetic): relative L2 <= 1e-12;
  - FP32 plans: relative L2 <= 1e-5 against the FP64 oracle on the same input.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _run(torch, plan, x, direction, dtype):
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(device="cuda", dtype=tdt)
    yd = torch.empty_like(xd)
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_c2c(plan, xd, yd, direction)
    of.openfft_sync(plan)
    out = yd.cpu().numpy()
    # the input must be left unchanged (out of place)
    assert np.array_equal(xd.cpu().numpy(), x.reshape(-1).astype(out.dtype))
    return out.astype(np.complex128)


def _all_candidates(plan):
    return range(of.openfft_num_candidates(plan))


# ---------------------------------------------------- 32^3, P = 4 ------

def test_32cubed_p4_every_candidate(torch):
    Na = Nb = Nc = 32
    x = synth.complex_field((Na, Nb, Nc), seed=synth.config_seed(1))
    ref = oracle.fft3d(x, Na, Nb, Nc, 4, oracle.FORWARD)
    back_ref = x.reshape(-1)
    plan = of.openfft_plan(Na, Nb, Nc, 4, of.C2C_F64)
    try:
        for c in _all_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
            assert oracle.rel_l2(y, ref) < TOL_F64, (c, of.openfft_candidate(plan, c))
            z = _run(torch, plan, y, of.BACKWARD, of.C2C_F64)
            assert oracle.rel_l2(z, back_ref) < TOL_F64, (c, of.openfft_candidate(plan, c))
    finally:
        of.openfft_destroy(plan)


# ------------------------------------------ small and ragged shapes -----

SMALL = [((1, 1, 1), 1), ((1, 8, 1), 1), ((2, 3, 5), 2), ((4, 6, 5), 3), ((8, 3, 5), 5), ((5, 4, 3), 12),
         ((12, 10, 9), 30), ((9, 25, 14), 7), ((36, 40, 30), 64), ((7, 49, 6), 42), ((3, 1, 2), 2),
         ((16, 16, 16), 256), ((64, 48, 100), 33)]


@pytest.mark.parametrize("shape,P", SMALL)
def test_small_shapes_f64_every_candidate(torch, shape, P):
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=Na * 1000 + Nb * 10 + Nc)
    ref = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
    refb = oracle.fft3d(x, Na, Nb, Nc, P, oracle.BACKWARD)      # x read as a cba spectrum
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        for c in _all_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
            assert oracle.rel_l2(y, ref) < TOL_F64, (shape, P, of.openfft_candidate(plan, c))
            z = _run(torch, plan, x, of.BACKWARD, of.C2C_F64)
            assert oracle.rel_l2(z, refb) < TOL_F64, (shape, P, of.openfft_candidate(plan, c))
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("shape,P", [((32, 32, 32), 4), ((12, 10, 9), 30), ((36, 40, 30), 64), ((5, 4, 3), 12)])
def test_small_shapes_f32_every_candidate(torch, shape, P):
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=77).astype(np.complex64)
    ref = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, P, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F32)
    try:
        for c in _all_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, of.C2C_F32)
            assert oracle.rel_l2(y, ref) < TOL_F32, (shape, P, of.openfft_candidate(plan, c))
            z = _run(torch, plan, y.astype(np.complex64), of.BACKWARD, of.C2C_F32)
            assert oracle.rel_l2(z, x.reshape(-1).astype(np.complex128)) < TOL_F32
    finally:
        of.openfft_destroy(plan)


# ----------------------------------------------- 120 x 144 x 160, P = 32 --

def test_mixed_radix_120x144x160(torch):
    Na, Nb, Nc = 120, 144, 160
    x = synth.complex_field((Na, Nb, Nc), seed=synth.config_seed(3))
    ref = oracle.fft3d(x, Na, Nb, Nc, 32, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, 32, of.C2C_F64)
    try:
        for c in _all_candidates(plan):
            cand = of.openfft_candidate(plan, c)
            if cand["variant"] != of.VARIANT_FUSED and cand["lines_per_cta"] != 8:
                continue
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
            assert oracle.rel_l2(y, ref) < TOL_F64, cand
    finally:
        of.openfft_destroy(plan)
    plan = of.openfft_plan(Na, Nb, Nc, 32, of.C2C_F32)
    try:
        y = _run(torch, plan, x.astype(np.complex64), of.FORWARD, of.C2C_F32)
        assert oracle.rel_l2(y, ref) < TOL_F32
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("k0", [(0, 0, 0), (1, 2, 3), (59, 71, 79), (119, 143, 159)])
def test_plane_waves_120x144x160(torch, k0):
    Na, Nb, Nc = 120, 144, 160
    N = Na * Nb * Nc
    x = synth.plane_wave(Na, Nb, Nc, k0)
    exact = np.zeros((Na, Nb, Nc), complex)
    exact[k0] = N
    exact = oracle.abc_to_cba(exact)
    for dtype, tol in [(of.C2C_F64, 1e-14), (of.C2C_F32, 1e-6)]:
        plan = of.openfft_plan(Na, Nb, Nc, 32, dtype)
        try:
            xx = x if dtype == of.C2C_F64 else x.astype(np.complex64)
            y = _run(torch, plan, xx, of.FORWARD, dtype)
            assert np.linalg.norm(y - exact) / (N * np.sqrt(N)) < tol
        finally:
            of.openfft_destroy(plan)


# --------------------------------------------------- transposes alone ----

REDIST = [((4, 3, 2), 3), ((4, 3, 2), 6), ((8, 6, 10), 40), ((12, 10, 9), 30), ((5, 7, 3), 15),
          ((16, 16, 16), 64), ((32, 32, 32), 4), ((20, 18, 15), 7), ((8, 8, 8), 16), ((7, 1, 5), 5),
          ((16, 16, 16), 100), ((12, 10, 16), 97)]


@pytest.mark.parametrize("shape,P", REDIST)
def test_transposes_bit_exact(torch, shape, P):
    Na, Nb, Nc = shape
    N = Na * Nb * Nc
    src = synth.complex_field((N,), seed=N + P)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        for which, code in [("abc->cab", 1), ("cab->cba", 2), ("cba->cab", -2), ("cab->abc", -1)]:
            ref, C = oracle.redistribute(Na, Nb, Nc, P, which, src)
            assert np.array_equal(of.openfft_counts(plan, code, P), C)
            for variant in sorted(of.METHODS.values()):           # the six methods of Sec. 3.2.1 and fused
                xd = torch.from_numpy(src).cuda()
                yd = torch.full_like(xd, float("nan"))
                of.openfft_redistribute(plan, code, variant, xd, yd)
                of.openfft_sync(plan)
                got = yd.cpu().numpy()
                assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (which, variant)
    finally:
        of.openfft_destroy(plan)


# --------------------------------------------- full sizes, sampled ------

def _sample_lines(x, y_cba, Na, Nb, Nc, picks):
    for kb, kc in picks:
        ref = oracle.dft3d_line(x, kb, kc, oracle.FORWARD)
        got = y_cba[(kc * Nb + kb) * Na:(kc * Nb + kb + 1) * Na]
        assert oracle.rel_l2(got, ref) < TOL_F64, (kb, kc)


@pytest.mark.parametrize("P", [16, 64, 256])
def test_256cubed_default_plan_sampled(torch, P):
    n = 256
    x = synth.complex_field((n, n, n), seed=synth.config_seed(2), dist="normal")
    plan = of.openfft_plan(n, n, n, P, of.C2C_F64)
    try:
        y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
        _sample_lines(x, y, n, n, n, [(0, 0), (1, 2), (255, 128), (77, 200)])
        N = n ** 3
        assert abs(np.sum(np.abs(y) ** 2) / (N * np.sum(np.abs(x) ** 2)) - 1.0) < 1e-13   # Parseval
        z = _run(torch, plan, y, of.BACKWARD, of.C2C_F64)
        assert oracle.rel_l2(z, x.reshape(-1)) < TOL_F64
    finally:
        of.openfft_destroy(plan)


def test_512cubed_sampled(torch):
    n = 512
    x = synth.complex_field((n, n, n), seed=synth.config_seed(5))
    plan = of.openfft_plan(n, n, n, 1024, of.C2C_F64)
    try:
        y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
        _sample_lines(x, y, n, n, n, [(3, 5), (511, 256)])
        z = _run(torch, plan, y, of.BACKWARD, of.C2C_F64)
        assert oracle.rel_l2(z, x.reshape(-1)) < TOL_F64
    finally:
        of.openfft_destroy(plan)


# ---------------------------------------- double-float value range ------

@pytest.mark.parametrize("scale", [1e-25, 1e-8, 1.0, 3e7, 1e22])
def test_double_float_range(torch, scale):
    """The double-float arithmetic keeps FP64 accuracy across its documented
    input range (|x| in [2^-100, 2^90]), including mixed magnitudes."""
    Na, Nb, Nc = 24, 40, 30
    x = synth.complex_field((Na, Nb, Nc), seed=13) * scale
    x.reshape(-1)[::7] *= 1e-6          # a spread of exponents inside one array
    ref = oracle.fft3d(x, Na, Nb, Nc, 6, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, 6, of.C2C_F64)
    try:
        for c in _all_candidates(plan):
            cand = of.openfft_candidate(plan, c)
            if cand["arith"] != of.ARITH_DOUBLE_FLOAT:
                continue
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, of.C2C_F64)
            assert oracle.rel_l2(y, ref) < TOL_F64, (scale, cand)
            z = _run(torch, plan, y, of.BACKWARD, of.C2C_F64)
            assert oracle.rel_l2(z, x.reshape(-1)) < TOL_F64, (scale, cand)
    finally:
        of.openfft_destroy(plan)


def _df_candidates(plan):
    return [c for c in _all_candidates(plan) if of.openfft_candidate(plan, c)["arith"] == of.ARITH_DOUBLE_FLOAT]


@pytest.mark.parametrize("k", [-40, 40])
def test_double_float_power_of_two_scaling_is_exact(torch, k):
    """Every double-float operation commutes with scaling by 2^k while no hi or lo
    part leaves the float range, so the outputs for 2^k x are exactly 2^k times
    those for x: a bit-exact check of the exponent handling of the double ->
    double-float split and the join back, both directions."""
    Na, Nb, Nc, P = 20, 36, 32, 5
    x = synth.complex_field((Na, Nb, Nc), seed=17)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        for c in _df_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            for direction in (of.FORWARD, of.BACKWARD):
                y1 = _run(torch, plan, x, direction, of.C2C_F64)
                y2 = _run(torch, plan, np.ldexp(x.real, k) + 1j * np.ldexp(x.imag, k), direction, of.C2C_F64)
                want = np.ldexp(y1.real, k) + 1j * np.ldexp(y1.imag, k)
                assert np.array_equal(y2, want), (k, direction, of.openfft_candidate(plan, c))
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("bad", [float("inf"), float("nan"), 1e300])
def test_double_float_non_finite_and_out_of_range_inputs(torch, bad):
    """An infinity, a NaN, or a finite value beyond the float exponent range in the
    input makes every output of the double-float forms non-finite in its real or
    its imaginary part (each output depends on every input): never a finite wrong
    number."""
    Na, Nb, Nc, P = 12, 10, 16, 4
    x = synth.complex_field((Na, Nb, Nc), seed=19)
    x[3, 4, 5] = complex(bad, 0.0)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        for c in _df_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            xd = torch.from_numpy(x.reshape(-1)).cuda()
            yd = torch.empty_like(xd)
            of.openfft_set_stream(plan, torch.cuda.current_stream())
            of.openfft_exec_c2c(plan, xd, yd, of.FORWARD)
            of.openfft_sync(plan)
            y = yd.cpu().numpy()
            assert (~np.isfinite(y.real) | ~np.isfinite(y.imag)).all(), (bad, of.openfft_candidate(plan, c))
    finally:
        of.openfft_destroy(plan)


# ------------------------------------------------------------ errors ----

def test_argument_errors(torch):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_plan(11, 8, 8, 2, of.C2C_F64)
    assert ei.value.status == of.ERR_UNSUPPORTED_RADIX
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_plan(8, 8, 8, 65, of.C2C_F64)
    assert ei.value.status == of.ERR_P_TOO_LARGE
    plan = of.openfft_plan(8, 8, 8, 2, of.C2C_F64)
    try:
        x = torch.zeros(512, dtype=torch.complex128, device="cuda")
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_c2c(plan, x, x, of.FORWARD)
        assert ei.value.status == of.ERR_ALIAS
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_c2c(plan, x, torch.zeros_like(x), 0)
        assert ei.value.status == of.ERR_INVALID_ARG
    finally:
        of.openfft_destroy(plan)


def test_host_exec_and_tuning(torch):
    Na, Nb, Nc = 48, 64, 40
    x = synth.complex_field((Na, Nb, Nc), seed=4)
    ref = oracle.fft3d(x, Na, Nb, Nc, 8, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, 8, of.C2C_F64)
    try:
        of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
        y = np.empty(Na * Nb * Nc, np.complex128)
        of.openfft_exec_c2c_host(plan, np.ascontiguousarray(x.reshape(-1)), y, of.FORWARD)
        assert oracle.rel_l2(y, ref) < TOL_F64
        of.openfft_set_timing(plan, True)
        of.openfft_exec_c2c_host(plan, np.ascontiguousarray(x.reshape(-1)), y, of.FORWARD)
        t = of.openfft_get_timing(plan)
        assert t["exec"]["launches"] == 1 and t["fft"]["launches"] == 3
        assert t["fft"]["ms"] > 0
    finally:
        of.openfft_destroy(plan)


# --------------------------------------------- the longest supported axes --

@pytest.mark.parametrize("shape,P", [((2048, 2, 3), 2), ((3, 2048, 2), 3), ((2, 3, 2048), 2),
                                     ((1792, 4, 3), 6), ((5, 1000, 2), 4)])
@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
def test_longest_axes_every_candidate(torch, shape, P, dtype):
    """Axes at the 2048 limit (and 1792 = 2^8 7, 1000 = 2^3 5^3) on each axis position."""
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=Na + 7 * Nb + 31 * Nc)
    if dtype == of.C2C_F32:
        x = x.astype(np.complex64)
    ref = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, P, oracle.FORWARD)
    tol = TOL_F64 if dtype == of.C2C_F64 else TOL_F32
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        for c in _all_candidates(plan):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _run(torch, plan, x, of.FORWARD, dtype)
            assert oracle.rel_l2(y, ref) < tol, (shape, P, of.openfft_candidate(plan, c))
            z = _run(torch, plan, y.astype(x.dtype), of.BACKWARD, dtype)
            assert oracle.rel_l2(z, x.reshape(-1).astype(np.complex128)) < 2 * tol
    finally:
        of.openfft_destroy(plan)


def test_axes_beyond_the_limit_are_refused(torch):
    for shape in [(4096, 2, 2), (2, 2, 4096), (2, 2049, 2), (2, 2, 2 * 11 * 13)]:
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_plan(*shape, 2, of.C2C_F64)
        assert ei.value.status == of.ERR_UNSUPPORTED_RADIX, shape


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
def test_host_exec_page_locked_buffers(torch, dtype):
    """Host-buffer execution with page-locked and with pageable buffers, for the
    default and two explicit candidates, both directions: matches the oracle."""
    Na, Nb, Nc, P = 64, 48, 40, 12
    x = synth.complex_field((Na, Nb, Nc), seed=91)
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    tol = TOL_F64 if dtype == of.C2C_F64 else TOL_F32
    ref = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
    refb = oracle.fft3d(x, Na, Nb, Nc, P, oracle.BACKWARD)
    hx = torch.from_numpy(x.reshape(-1)).to(tdt).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    assert hx.is_pinned() and hy.is_pinned()
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        for c in [0] + [i for i in range(of.openfft_num_candidates(plan))
                        if of.openfft_candidate(plan, i)["variant"] != of.VARIANT_FUSED][:2]:
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            hy.fill_(float("nan"))
            of.openfft_exec_c2c_host(plan, hx.numpy(), hy.numpy(), of.FORWARD)
            assert oracle.rel_l2(hy.numpy().astype(np.complex128), ref) < tol, of.openfft_candidate(plan, c)
            of.openfft_exec_c2c_host(plan, hx.numpy(), hy.numpy(), of.BACKWARD)
            assert oracle.rel_l2(hy.numpy().astype(np.complex128), refb) < tol, of.openfft_candidate(plan, c)
        assert np.array_equal(hx.numpy(), x.reshape(-1).astype(hx.numpy().dtype))     # input untouched
        # pageable buffers: the copy path
        y = np.empty(Na * Nb * Nc, dtype=hx.numpy().dtype)
        of.openfft_set_tuning(plan, of.TUNE_USER, 0)
        of.openfft_exec_c2c_host(plan, x.reshape(-1).astype(y.dtype), y, of.FORWARD)
        assert oracle.rel_l2(y.astype(np.complex128), ref) < tol
    finally:
        of.openfft_destroy(plan)
