"""The 3-D transform over several devices, one process per device.

Device g of G (its rank in the torch.distributed group) holds the logical
ranks [floor(g P / G), floor((g+1) P / G)) of the decomposition, which is one
contiguous slice of each ordering (abc, cab, cba).  A transform runs the
paper's execution flow (Duy & Ozaki, Sec. 3.1.1): the line-local FFT stages
of steps (1)-(3) on each device, and each transpose as pack (step 4), one
all-to-all with variable counts among the devices (step 5, the Alltoallv
method of Sec. 3.2.1) and unpack (step 6).  The stages, pack and unpack are
the library's kernels (openfft_dist_* of the C ABI); step 5 is
torch.distributed.all_to_all_single (NCCL between GPUs), which delivers the
remote segments into this device's memory before the unpack kernel reads
them.  This module only marshals arguments and sequences the calls.

Between the stages the buffers hold the library's internal element format
(double-float pairs for complex128 plans), 16 or 8 bytes per element, carried
in complex128 / complex64 tensors; pack and unpack move them unchanged.
"""
from __future__ import annotations

from . import openfft as of

ABC, CAB, CBA = 0, 1, 2
R1, R2, R2_INV, R1_INV = 1, 2, -2, -1


class DeviceOps:
    """The library's kernels on this process's CUDA device (the default)."""

    def __init__(self, plan: int):
        self.plan = plan

    def stage(self, stage, direction, src, dst):
        of.openfft_dist_stage(self.plan, stage, direction, src, dst)

    def pack(self, exchange, src, send):
        of.openfft_dist_pack(self.plan, exchange, src, send)

    def unpack(self, exchange, recv, dst):
        of.openfft_dist_unpack(self.plan, exchange, recv, dst)


class DistFFT:
    """Distributed plan of this process (device g of G).

    forward(x): x = this device's slice of the abc array -> its slice of the
    cba spectrum.  backward(y): cba slice -> abc slice, divided by N.
    `group` is the torch.distributed group of the G devices (default: the
    world); `ops` replaces the per-device operations (tests drive the same
    sequence with host-side operations on CPU tensors)."""

    def __init__(self, Na, Nb, Nc, P, dtype=of.C2C_F64, group=None, ops=None, G=None, g=None, exchange=None):
        import torch.distributed as dist
        self.Na, self.Nb, self.Nc, self.P, self.dtype = Na, Nb, Nc, P, dtype
        self.group = group
        self.G = G if G is not None else dist.get_world_size(group)
        self.g = g if g is not None else dist.get_rank(group)
        self.plan = None
        if ops is None:
            import torch
            self.plan = of.openfft_dist_plan(Na, Nb, Nc, P, self.G, self.g, dtype)
            of.openfft_dist_set_stream(self.plan, torch.cuda.current_stream())
            ops = DeviceOps(self.plan)
        self.ops = ops
        self._exchange = exchange or self._all_to_all
        counts = {x: of.openfft_dist_counts(Na, Nb, Nc, P, self.G, x) for x in (R1, R2, R2_INV, R1_INV)}
        self.send_counts = {x: [int(v) for v in c[self.g, :]] for x, c in counts.items()}
        self.recv_counts = {x: [int(v) for v in c[:, self.g]] for x, c in counts.items()}
        self.rows = {L: of.openfft_dist_rows(Na, Nb, Nc, P, self.G, L, self.g) for L in (ABC, CAB, CBA)}

    def close(self):
        if self.plan:
            of.openfft_dist_destroy(self.plan)
            self.plan = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def local_size(self, layout: int) -> int:
        """Elements of this device's slice of an ordering."""
        return self.rows[layout][1]

    def _all_to_all(self, send, send_counts, recv_counts):
        import torch
        import torch.distributed as dist
        recv = torch.empty(sum(recv_counts), dtype=send.dtype, device=send.device)
        # dim-0 splits of the (n, 2) real views are element counts
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), recv_counts, send_counts,
                               group=self.group)
        return recv

    def pack(self, exchange: int, src):
        """Step (4): the send buffer of this device, segments by destination."""
        import torch
        send = torch.empty(sum(self.send_counts[exchange]), dtype=src.dtype, device=src.device)
        self.ops.pack(exchange, src, send)
        return send

    def unpack(self, exchange: int, recv):
        """Step (6): this device's slice of the destination ordering."""
        import torch
        dst = torch.empty(sum(self.recv_counts[exchange]), dtype=recv.dtype, device=recv.device)
        self.ops.unpack(exchange, recv, dst)
        return dst

    def transpose(self, exchange: int, src):
        """One transpose of this device's slice (steps (4)-(6))."""
        send = self.pack(exchange, src)
        recv = self._exchange(send, self.send_counts[exchange], self.recv_counts[exchange])
        return self.unpack(exchange, recv)

    def forward(self, x):
        """abc slice -> cba slice (unnormalised, exp(-2 pi i ...))."""
        import torch
        a = torch.empty_like(x)
        self.ops.stage(1, of.FORWARD, x, a)          # c-lines of abc
        b = self.transpose(R1, a)                    # abc -> cab
        self.ops.stage(2, of.FORWARD, b, b)          # b-lines of cab
        c = self.transpose(R2, b)                    # cab -> cba
        self.ops.stage(3, of.FORWARD, c, c)          # a-lines of cba
        return c

    def backward(self, y):
        """cba slice -> abc slice (exp(+2 pi i ...), divided by N)."""
        import torch
        a = torch.empty_like(y)
        self.ops.stage(1, of.BACKWARD, y, a)         # a-lines of cba
        b = self.transpose(R2_INV, a)                # cba -> cab
        self.ops.stage(2, of.BACKWARD, b, b)         # b-lines of cab
        c = self.transpose(R1_INV, b)                # cab -> abc
        self.ops.stage(3, of.BACKWARD, c, c)         # c-lines of abc
        return c
