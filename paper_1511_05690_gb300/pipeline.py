"""Host-buffer products with copy / compute overlap.

For a sequence of independent products whose inputs and outputs live in
pinned host memory, ``HostPipeline`` overlaps the host->device copies of the
next product, the p-norm product of the current one, and the device->host copy
of the previous one, on three CUDA streams with double-buffered device
staging.  Only stream events order the work (no device-side waits).  Every
product still performs its own copies and its own full call of the C ABI.
"""
from __future__ import annotations

import torch

from . import maxprod_pnorm


class HostPipeline:
    """Pipelined ``C_i = maxprod_pnorm(A_i, B_i)`` for pinned host tensors.

    All products share the shapes (M, K) x (K, N) given here.  ``run`` takes an
    iterable of (A_host, B_host, C_host) triples, returns when every C_host is
    written, and forwards the keyword options to ``maxprod_pnorm``.
    """

    def __init__(self, M, N, K, device="cuda", **opts):
        self.opts = dict(opts)
        self.opts.setdefault("want_psel", False)
        self.opts.setdefault("want_ssel", False)
        self.opts["check"] = False
        dev = torch.device(device)
        self.A = [torch.empty((M, K), dtype=torch.float32, device=dev) for _ in range(2)]
        self.B = [torch.empty((K, N), dtype=torch.float32, device=dev) for _ in range(2)]
        self.C = [torch.empty((M, N), dtype=torch.float32, device=dev) for _ in range(2)]
        self.s_in = torch.cuda.Stream(device=dev)
        self.s_comp = torch.cuda.Stream(device=dev)
        self.s_out = torch.cuda.Stream(device=dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]  # noqa: E731
        self.ev_in, self.ev_done, self.ev_out = ev(), ev(), ev()
        self.h2d_bytes = 4 * (M * K + K * N)
        self.d2h_bytes = 4 * M * N

    def run(self, items, ev_start=None, ev_end=None):
        """ev_start / ev_end (optional torch.cuda.Event with timing) are recorded
        before the first copy in and after the last copy out."""
        used = [False, False]
        if ev_start is not None:
            ev_start.record(self.s_in)
        for i, (Ah, Bh, Ch) in enumerate(items):
            b = i & 1
            if used[b]:  # buffer b was last used two products ago
                self.s_in.wait_event(self.ev_done[b])
                self.s_comp.wait_event(self.ev_out[b])
            with torch.cuda.stream(self.s_in):
                self.A[b].copy_(Ah, non_blocking=True)
                self.B[b].copy_(Bh, non_blocking=True)
                self.ev_in[b].record(self.s_in)
            self.s_comp.wait_event(self.ev_in[b])
            with torch.cuda.stream(self.s_comp):
                maxprod_pnorm(self.A[b], self.B[b], out=self.C[b], stream=self.s_comp, **self.opts)
                self.ev_done[b].record(self.s_comp)
            self.s_out.wait_event(self.ev_done[b])
            with torch.cuda.stream(self.s_out):
                Ch.copy_(self.C[b], non_blocking=True)
                self.ev_out[b].record(self.s_out)
            used[b] = True
        self.s_out.wait_stream(self.s_in)
        self.s_out.wait_stream(self.s_comp)
        if ev_end is not None:
            ev_end.record(self.s_out)
        self.s_out.synchronize()
