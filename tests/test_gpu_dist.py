"""The transform over several devices on one GPU (openfft_dist_* kernels).

A single GPU cannot host several communicating processes whose kernels wait
on one another, so the G devices are emulated in one process: G device plans
(device g of G each) run their stages, pack and unpack kernels on slices of
one GPU's memory, and the all-to-all-v between them (Sec. 3.1.1 step (5)) is
done with plain copies of the send segments into the receive buffers, after
every device has packed.  No kernel waits on another.  Checked against the
oracle: the transposes alone bit for bit (oracle.redistribute), the whole
transform within the bars of the other GPU tests (1e-12 relative L2 for
complex128, 1e-5 for complex64).  Then one real process group of one rank
over NCCL runs DistFFT.forward / backward end to end.
"""
import socket

import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import dist as pdist
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.C2C_F64: 1e-12, of.C2C_F32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _devices(Na, Nb, Nc, P, G, dtype):
    return [pdist.DistFFT(Na, Nb, Nc, P, dtype, G=G, g=g) for g in range(G)]


def _exchange(devs, exchange, sends):
    """Step (5) among the emulated devices: segment g -> h copied into h's
    receive buffer at g's receive displacement."""
    import torch
    G = len(devs)
    recvs = []
    for h in range(G):
        parts = []
        for g in range(G):
            sc = devs[g].send_counts[exchange]
            off = sum(sc[:h])
            parts.append(sends[g][off:off + sc[h]])
        recvs.append(torch.cat(parts) if parts else sends[h][:0])
        assert recvs[-1].numel() == sum(devs[h].recv_counts[exchange])
    return recvs


def _transpose_all(devs, exchange, slices):
    sends = [d.pack(exchange, s) for d, s in zip(devs, slices)]
    return [d.unpack(exchange, r) for d, r in zip(devs, _exchange(devs, exchange, sends))]


def _run(devs, xs, direction):
    import torch
    fwd = direction == of.FORWARD
    xr = [torch.empty_like(x) for x in xs]
    for d, x, y in zip(devs, xs, xr):
        d.ops.stage(1, direction, x, y)
    b = _transpose_all(devs, pdist.R1 if fwd else pdist.R2_INV, xr)
    for d, v in zip(devs, b):
        d.ops.stage(2, direction, v, v)
    c = _transpose_all(devs, pdist.R2 if fwd else pdist.R1_INV, b)
    for d, v in zip(devs, c):
        d.ops.stage(3, direction, v, v)
    return c


CASES = [((8, 6, 10), 4, 2), ((8, 6, 10), 40, 4), ((12, 10, 9), 30, 3), ((16, 16, 16), 100, 4),
         ((64, 48, 40), 12, 3), ((128, 64, 32), 256, 4)]


@pytest.mark.parametrize("shape,P,G", CASES)
def test_emulated_devices_transposes_bit_exact(torch, shape, P, G):
    Na, Nb, Nc = shape
    N = Na * Nb * Nc
    x = synth.complex_field((N,), seed=N + 3 * P + G)
    devs = _devices(Na, Nb, Nc, P, G, of.C2C_F64)
    try:
        src_dst = {1: (0, 1, "abc->cab"), 2: (1, 2, "cab->cba"), -2: (2, 1, "cba->cab"), -1: (1, 0, "cab->abc")}
        for exchange, (sl, dl, which) in src_dst.items():
            ref, _ = oracle.redistribute(Na, Nb, Nc, P, which, x)
            slices = []
            for d in devs:
                off, cnt = d.rows[sl]
                slices.append(torch.from_numpy(x[off:off + cnt].copy()).cuda())
            outs = _transpose_all(devs, exchange, slices)
            torch.cuda.synchronize()
            got = np.concatenate([o.cpu().numpy() for o in outs])
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), (which, G)
    finally:
        for d in devs:
            d.close()


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
@pytest.mark.parametrize("shape,P,G", CASES)
def test_emulated_devices_transform(torch, shape, P, G, dtype):
    Na, Nb, Nc = shape
    N = Na * Nb * Nc
    x = synth.complex_field((N,), seed=N + P)
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    xin = x if dtype == of.C2C_F64 else x.astype(np.complex64).astype(np.complex128)
    devs = _devices(Na, Nb, Nc, P, G, dtype)
    try:
        for direction, src_l in ((of.FORWARD, 0), (of.BACKWARD, 2)):
            ref = oracle.fft3d(xin, Na, Nb, Nc, P, direction)
            xs = []
            for d in devs:
                off, cnt = d.rows[src_l]
                xs.append(torch.from_numpy(x[off:off + cnt].copy()).to("cuda", tdt))
            outs = _run(devs, xs, direction)
            torch.cuda.synchronize()
            got = np.concatenate([o.cpu().numpy().astype(np.complex128) for o in outs])
            assert oracle.rel_l2(got, ref) < TOL[dtype], (shape, P, G, direction)
    finally:
        for d in devs:
            d.close()


def test_one_rank_nccl_group_end_to_end(torch):
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        Na, Nb, Nc, P = 64, 40, 48, 16
        x = synth.complex_field((Na * Nb * Nc,), seed=31)
        plan = pdist.DistFFT(Na, Nb, Nc, P, of.C2C_F64)
        try:
            y = plan.forward(torch.from_numpy(x).cuda())
            z = plan.backward(y)
            torch.cuda.synchronize()
            assert oracle.rel_l2(y.cpu().numpy(), oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)) < 1e-12
            assert oracle.rel_l2(z.cpu().numpy(), x) < 1e-12
        finally:
            plan.close()
    finally:
        dist.destroy_process_group()
