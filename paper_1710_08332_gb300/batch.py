"""Batches of uneven dot and GEMV instances in one persistent launch.

``Batch`` packs the instances (every instance at a 128-byte aligned offset,
GEMV rows padded to a multiple of 4 floats), gives each instance its own
reduction strategy from a policy, has the library build the plan (host C++),
keeps a device copy of it and the workspace, and launches the batched forward
and backward kernels. ``per_launch_*`` run the same instances with one
single-instance call each (the baseline the batch is measured against; with
the same strategies its results are bit-identical).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N
from . import ops
from .strategy import ReduceStrategy

ALIGN = 32  # elements: 128-byte instance offsets


def _round(v: int, m: int) -> int:
    return (v + m - 1) // m * m


@dataclass(frozen=True)
class BatchPolicy:
    """How instance strategies are chosen from their sizes (what the autotuner varies)."""
    threads: int = 256
    dot_split_cap: int = 8192      # dot split = the length rounded up to threads*4, capped
    dot_second: str = "tree"
    gemv_split_cap: int = 4096     # GEMV row split = N rounded up to 128, capped
    row_split: int = 256           # backward dx rows per chunk
    schedule: int = 0              # 0: longest first, round robin; 1: contiguous equal-cost runs;
    #                                2: longest first, forward round robin, each backward warp
    #                                   takes the next item when it is free

    def dot_strategy(self, n: int) -> ReduceStrategy:
        q = self.threads * 4
        s = min(max(_round(max(n, 1), q), q), _round(self.dot_split_cap, q))
        return ReduceStrategy(split=s, threads=self.threads, vec=4, second=self.dot_second,
                              threads2=min(self.threads, 256), pad=True)

    def gemv_strategy(self, N_: int) -> ReduceStrategy:
        s = min(_round(N_, 128), _round(self.gemv_split_cap, 128))
        return ReduceStrategy(split=s, threads=self.threads, vec=4, map_level="warp", pad=True)


class Batch:
    def __init__(self, dot_lengths, gemv_shapes, device="cuda", policy: BatchPolicy | None = None,
                 row_align: int = 32):
        """row_align: each GEMV matrix's rows start every round_up(N, row_align) floats
        (32, the default: rows on 128-byte lines, so that no two pieces of a row that
        different items read share a line; 4: 16-byte rows, the least the vector loads
        need)."""
        if row_align < 4 or row_align % 4:
            raise ValueError("row_align must be a positive multiple of 4 floats")
        self.device = torch.device(device)
        self.policy = policy or BatchPolicy()
        P = self.policy
        self.dot_lengths = [int(n) for n in dot_lengths]
        self.gemv_shapes = [(int(m), int(n)) for m, n in gemv_shapes]
        # packed layout
        self.dot_offs, off = [], 0
        for n in self.dot_lengths:
            self.dot_offs.append(off)
            off += _round(max(n, 1), ALIGN)
        self.xs_len = max(off, ALIGN)
        self.a_offs, self.gx_offs, self.gy_offs, self.ldas = [], [], [], []
        aoff = xoff = yoff = 0
        for M, N_ in self.gemv_shapes:
            lda = _round(N_, row_align)
            self.a_offs.append(aoff)
            self.gx_offs.append(xoff)
            self.gy_offs.append(yoff)
            self.ldas.append(lda)
            aoff += _round(M * lda, ALIGN)
            xoff += _round(N_, ALIGN)
            yoff += _round(max(M, 1), ALIGN)
        self.as_len, self.gx_len, self.gy_len = max(aoff, ALIGN), max(xoff, ALIGN), max(yoff, ALIGN)
        # instances and plan
        self.dot_st = [P.dot_strategy(n) for n in self.dot_lengths]
        self.gemv_st = [P.gemv_strategy(n) for _, n in self.gemv_shapes]
        nd, ng = len(self.dot_lengths), len(self.gemv_shapes)
        dots = (N.DotInstanceC * max(nd, 1))()
        for i, (o, n, st) in enumerate(zip(self.dot_offs, self.dot_lengths, self.dot_st)):
            dots[i] = N.DotInstanceC(o, n, st.to_c())
        gemvs = (N.GemvInstanceC * max(ng, 1))()
        for i, ((M, N_), st) in enumerate(zip(self.gemv_shapes, self.gemv_st)):
            gemvs[i] = N.GemvInstanceC(self.a_offs[i], self.gx_offs[i], self.gy_offs[i], M, N_, self.ldas[i],
                                       st.to_c(), P.row_split)
        L = N.lib()
        opt = ctypes.byref(N.BatchOptionsC(P.threads, P.schedule))
        nbytes = L.dpia_batch_plan_size(nd, dots, ng, gemvs, opt)
        if nbytes == 0:
            raise N.DPIAError(N.ERR_STRATEGY, L.dpia_last_error_message().decode())
        self._plan_host = (ctypes.c_char * nbytes)()
        N.check(L.dpia_batch_plan(nd, dots, ng, gemvs, opt, self._plan_host, nbytes), "dpia_batch_plan")
        host = torch.frombuffer(bytearray(self._plan_host.raw), dtype=torch.uint8)
        self.plan_dev = host.to(self.device)
        self.ws = torch.zeros(L.dpia_batch_workspace_size(self._plan_host), dtype=torch.uint8, device=self.device)

    # --- packing helpers ---------------------------------------------------
    def pack_vectors(self, vecs, length, offs):
        out = torch.zeros(length, dtype=torch.float32, device=self.device)
        for o, v in zip(offs, vecs):
            out[o:o + v.numel()] = v
        return out

    def dot_view(self, packed, i):
        o = self.dot_offs[i]
        return packed[o:o + self.dot_lengths[i]]

    def a_view(self, packed, i):
        M, N_ = self.gemv_shapes[i]
        o = self.a_offs[i]
        return packed[o:o + M * self.ldas[i]].view(M, self.ldas[i])[:, :N_]

    def gx_view(self, packed, i):
        o = self.gx_offs[i]
        return packed[o:o + self.gemv_shapes[i][1]]

    def gy_view(self, packed, i):
        o = self.gy_offs[i]
        return packed[o:o + self.gemv_shapes[i][0]]

    # --- launches ----------------------------------------------------------
    def forward(self, xs, ys, dot_out, As, gx, gy, grid=0, stream=None):
        """dot_out[i] = dot_i, gy_i = A_i gx_i: one persistent launch."""
        p = ops._ptr
        N.check(N.lib().dpia_batch_forward_f32(p(self.plan_dev), self._plan_host, p(xs), p(ys), p(dot_out), p(As),
                                               p(gx), p(gy), p(self.ws), self.ws.numel(), int(grid),
                                               ops._stream(stream)), "dpia_batch_forward_f32")

    def backward(self, xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx, grid=0, stream=None):
        """dxs_i = g_i y_i, dys_i = g_i x_i, dA_i = dy_i x_i^T, dgx_i = A_i^T dy_i: one launch."""
        p = ops._ptr
        N.check(N.lib().dpia_batch_backward_f32(p(self.plan_dev), self._plan_host, p(xs), p(ys), p(dot_g), p(dxs),
                                                p(dys), p(As), p(gx), p(gdy), p(dAs), p(dgx), p(self.ws),
                                                self.ws.numel(), int(grid), ops._stream(stream)),
                "dpia_batch_backward_f32")

    # --- the per-launch baseline ---------------------------------------------
    def per_launch_forward(self, xs, ys, dot_out, As, gx, gy, ws=None):
        """The same instances, one dpia_dot_f32 / dpia_gemv_f32 call each."""
        L = N.lib()
        p = ops._ptr
        s = ops._stream()
        if ws is None:
            ws = self.per_launch_workspace()
        wsb = ws.numel()
        for i, n in enumerate(self.dot_lengths):
            o = self.dot_offs[i] * 4
            st = self.dot_st[i].to_c()
            N.check(L.dpia_dot_f32(ctypes.c_void_p(xs.data_ptr() + o), ctypes.c_void_p(ys.data_ptr() + o), n,
                                   ctypes.byref(st), ctypes.c_void_p(dot_out.data_ptr() + 4 * i), p(ws), wsb, s),
                    "dpia_dot_f32")
        for i, (M, N_) in enumerate(self.gemv_shapes):
            st = self.gemv_st[i].to_c()
            N.check(L.dpia_gemv_f32(ctypes.c_void_p(As.data_ptr() + 4 * self.a_offs[i]), M, N_, self.ldas[i],
                                    ctypes.c_void_p(gx.data_ptr() + 4 * self.gx_offs[i]),
                                    ctypes.c_void_p(gy.data_ptr() + 4 * self.gy_offs[i]), ctypes.byref(st), s),
                    "dpia_gemv_f32")

    def per_launch_workspace(self):
        n = max([ops.dpia_dot_workspace_size(n, st) for n, st in zip(self.dot_lengths, self.dot_st)] + [128])
        return torch.zeros(n, dtype=torch.uint8, device=self.device)

    def per_launch_backward(self, xs, ys, dot_g, dxs, dys, As, gx, gdy, dAs, dgx, ws_list=None):
        L = N.lib()
        s = ops._stream()
        for i, n in enumerate(self.dot_lengths):
            o = self.dot_offs[i] * 4
            N.check(L.dpia_dot_bwd_f32(ctypes.c_void_p(xs.data_ptr() + o), ctypes.c_void_p(ys.data_ptr() + o),
                                       ctypes.c_void_p(dot_g.data_ptr() + 4 * i), n,
                                       ctypes.c_void_p(dxs.data_ptr() + o), ctypes.c_void_p(dys.data_ptr() + o), s),
                    "dpia_dot_bwd_f32")
        if ws_list is None:
            ws_list = self.per_launch_bwd_workspaces()
        for i, (M, N_) in enumerate(self.gemv_shapes):
            ws = ws_list[i]
            N.check(L.dpia_gemv_bwd_f32(ctypes.c_void_p(As.data_ptr() + 4 * self.a_offs[i]), M, N_, self.ldas[i],
                                        ctypes.c_void_p(gx.data_ptr() + 4 * self.gx_offs[i]),
                                        ctypes.c_void_p(gdy.data_ptr() + 4 * self.gy_offs[i]),
                                        ctypes.c_void_p(dgx.data_ptr() + 4 * self.gx_offs[i]),
                                        ctypes.c_void_p(dAs.data_ptr() + 4 * self.a_offs[i]), self.ldas[i],
                                        self.policy.row_split, ctypes.c_void_p(ws.data_ptr()), ws.numel(), s),
                    "dpia_gemv_bwd_f32")

    def per_launch_bwd_workspaces(self):
        """One zeroed workspace per GEMV shape (a GEMV backward's counters depend on its shape)."""
        return [torch.zeros(ops.dpia_gemv_bwd_workspace_size(M, N_, self.policy.row_split), dtype=torch.uint8,
                            device=self.device) for M, N_ in self.gemv_shapes]
