"""The transform over several devices (paper_1501_07350_gb300/dist.py and the
openfft_dist_* host functions), on CPU processes over gloo.

Device g of G holds the logical ranks [floor(g P / G), floor((g+1) P / G)).
Each transpose is pack (Sec. 3.1.1 step (4)), one all-to-all with variable
counts among the devices (step 5, the Alltoallv method of Sec. 3.2.1, here
torch.distributed over gloo) and unpack (step 6).  Checked bit for bit
against the oracle's literal redistribution (oracle.redistribute), for slab
and pencil decompositions, on 2 and 4 processes; the full transform, with the
oracle's own 1-D FFT as the line-local stages, against oracle.fft3d bit for
bit in both directions.  The device count matrix is the P x P count matrix
summed over each device pair's ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (shape, P): slabs in every ordering, pencils in every ordering, mixed
CASES = [((8, 6, 10), 4), ((8, 6, 10), 40), ((12, 10, 9), 30), ((5, 7, 3), 15), ((16, 16, 16), 100),
         ((7, 1, 5), 5), ((6, 8, 4), 6)]


@pytest.fixture(scope="module")
def lib():
    from paper_1501_07350_gb300 import _build
    from paper_1501_07350_gb300 import openfft as of
    _build.build()
    of.load()
    import oracle
    oracle.build()
    return of


@pytest.mark.parametrize("shape,P", CASES)
@pytest.mark.parametrize("G", [1, 2, 3, 4])
def test_device_counts_and_slices(lib, shape, P, G):
    of = lib
    Na, Nb, Nc = shape
    if G > P:
        pytest.skip("every device holds a rank")
    N = Na * Nb * Nc
    r0 = [(P * g) // G for g in range(G + 1)]
    for exchange in (1, 2, -2, -1):
        C = of.openfft_decomp_counts(Na, Nb, Nc, P, exchange)
        D = of.openfft_dist_counts(Na, Nb, Nc, P, G, exchange)
        want = np.array([[C[r0[g]:r0[g + 1], r0[h]:r0[h + 1]].sum() for h in range(G)] for g in range(G)])
        assert np.array_equal(D, want), exchange
        assert D.sum() == N
    for layout in (0, 1, 2):
        nxt = 0
        for g in range(G):
            off, cnt = of.openfft_dist_rows(Na, Nb, Nc, P, G, layout, g)
            assert off == nxt
            # the slice is the union of the device's ranks' boxes (Eqs. 3-4)
            first = of.openfft_decomp_box(Na, Nb, Nc, P, layout, r0[g])[2]
            assert off == first
            nxt = off + cnt
        assert nxt == N


def test_argument_errors(lib):
    of = lib
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_dist_counts(8, 8, 8, 4, 5, 1)           # more devices than ranks
    assert ei.value.status == of.ERR_INVALID_ARG
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_dist_rows(8, 8, 8, 65, 2, 0, 0)          # P beyond Eq. 2
    assert ei.value.status == of.ERR_P_TOO_LARGE
    with pytest.raises(of.OpenFFTError):
        of.openfft_dist_counts(8, 8, 8, 4, 2, 3)            # no such exchange


# ------------------------------------------------------------ gloo ranks --

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class HostOps:
    """Test-side operations of one device on CPU tensors: the library's host
    pack / unpack, and the oracle's own 1-D FFT for the line-local stages."""

    def __init__(self, of, oracle, Na, Nb, Nc, P, G, g, fft=True):
        self.of, self.oracle = of, oracle
        self.dims = (Na, Nb, Nc, P, G, g)
        self.fft = fft

    def pack(self, exchange, src, send):
        Na, Nb, Nc, P, G, g = self.dims
        self.of.openfft_dist_pack_host(Na, Nb, Nc, P, G, exchange, g, src.numpy(), send.numpy())

    def unpack(self, exchange, recv, dst):
        Na, Nb, Nc, P, G, g = self.dims
        self.of.openfft_dist_unpack_host(Na, Nb, Nc, P, G, exchange, g, recv.numpy(), dst.numpy())

    def stage(self, stage, direction, src, dst):
        Na, Nb, Nc, P, G, g = self.dims
        fwd = direction == self.of.FORWARD
        n = [Nc, Nb, Na][stage - 1] if fwd else [Na, Nb, Nc][stage - 1]
        x = src.numpy().reshape(-1, n) if n else src.numpy()
        y = np.empty_like(x)
        for i in range(x.shape[0]):
            y[i] = self.oracle.fft1d(x[i], self.oracle.FORWARD if fwd else self.oracle.BACKWARD) if self.fft else x[i]
        if not fwd and stage == 3 and self.fft:
            # the oracle's 1/N: each real component divided by N
            scaled = np.empty_like(y)
            scaled.real = y.real / float(Na * Nb * Nc)
            scaled.imag = y.imag / float(Na * Nb * Nc)
            y = scaled
        dst.numpy()[:] = y.reshape(-1)


def _worker(rank, world, port, shape, P, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1501_07350_gb300 import dist as pdist
        from paper_1501_07350_gb300 import openfft as of
        from paper_1501_07350_gb300 import synth
        Na, Nb, Nc = shape
        N = Na * Nb * Nc
        x = synth.complex_field((N,), seed=N + P + 7)
        failures = []
        # the four transposes alone (no FFT): bit-exact against the oracle
        plain = pdist.DistFFT(Na, Nb, Nc, P, of.C2C_F64, ops=HostOps(of, oracle, Na, Nb, Nc, P, world, rank, fft=False))
        layouts = {1: (0, 1, "abc->cab"), 2: (1, 2, "cab->cba"), -2: (2, 1, "cba->cab"), -1: (1, 0, "cab->abc")}
        for exchange, (src_l, dst_l, which) in layouts.items():
            ref, _ = oracle.redistribute(Na, Nb, Nc, P, which, x)
            off, cnt = plain.rows[src_l]
            src = torch.from_numpy(x[off:off + cnt].copy())
            got = plain.transpose(exchange, src).numpy()
            doff, dcnt = plain.rows[dst_l]
            if got.shape != (dcnt,) or not np.array_equal(got.view(np.uint64), ref[doff:doff + dcnt].view(np.uint64)):
                failures.append(("transpose", exchange))
        # the whole transform with the oracle's 1-D FFT as the stages
        full = pdist.DistFFT(Na, Nb, Nc, P, of.C2C_F64, ops=HostOps(of, oracle, Na, Nb, Nc, P, world, rank))
        ref_f = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
        ref_b = oracle.fft3d(x, Na, Nb, Nc, P, oracle.BACKWARD)
        off, cnt = full.rows[0]
        y = full.forward(torch.from_numpy(x[off:off + cnt].copy())).numpy()
        yoff, ycnt = full.rows[2]
        if not np.array_equal(y.view(np.uint64), ref_f[yoff:yoff + ycnt].view(np.uint64)):
            failures.append(("forward",))
        z = full.backward(torch.from_numpy(x[yoff:yoff + ycnt].copy())).numpy()
        if not np.array_equal(z.view(np.uint64), ref_b[off:off + cnt].view(np.uint64)):
            failures.append(("backward",))
        q.put((rank, failures))
    except Exception as e:          # reported to the parent
        q.put((rank, [("exception", repr(e))]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("shape,P", [((8, 6, 10), 4), ((8, 6, 10), 40), ((12, 10, 9), 30), ((16, 16, 16), 100)])
def test_gloo_ranks_transposes_and_transform_bit_exact(lib, world, shape, P):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shape, P, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, failures in sorted(res):
        assert not failures, (rank, failures)
