"""Host-buffer products with copy / compute overlap.

For a sequence of independent products whose inputs and outputs live in
pinned host memory, ``HostPipeline`` overlaps the host->device copies of the
next product, the p-norm product of the current one, and the device->host copy
of the previous one, with double-buffered device staging.  Each direction
can be split over several streams (copy_streams); one stream per direction
measured best on GB300 (about 209 GB/s in and 190 GB/s out, concurrently).
Only stream events order the work (no device-side waits).  Every product
still performs its own copies and its own full call of the C ABI.
"""
from __future__ import annotations

import torch

from . import maxprod_pnorm


class HostPipeline:
    """Pipelined ``C_i = maxprod_pnorm(A_i, B_i)`` for pinned host tensors.

    All products share the shapes (M, K) x (K, N) given here.  ``run`` takes an
    iterable of (A_host, B_host, C_host) triples, returns when every C_host is
    written, and forwards the keyword options to ``maxprod_pnorm``.  Copies are
    split over ``copy_streams`` streams per direction.
    """

    def __init__(self, M, N, K, device="cuda", copy_streams=1, **opts):
        self.opts = dict(opts)
        self.opts.setdefault("want_psel", False)
        self.opts.setdefault("want_ssel", False)
        self.opts["check"] = False
        dev = torch.device(device)
        self.A = [torch.empty((M, K), dtype=torch.float32, device=dev) for _ in range(2)]
        self.B = [torch.empty((K, N), dtype=torch.float32, device=dev) for _ in range(2)]
        self.C = [torch.empty((M, N), dtype=torch.float32, device=dev) for _ in range(2)]
        ns = max(1, int(copy_streams))
        self.s_in = [torch.cuda.Stream(device=dev) for _ in range(ns)]
        self.s_out = [torch.cuda.Stream(device=dev) for _ in range(ns)]
        self.s_comp = torch.cuda.Stream(device=dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]  # noqa: E731
        self.ev_done = ev()
        self.ev_in = [ev() for _ in range(ns)]
        self.ev_out = [ev() for _ in range(ns)]
        self.h2d_bytes = 4 * (M * K + K * N)
        self.d2h_bytes = 4 * M * N

    @staticmethod
    def _rows(t, i, parts):
        """Row block i of `parts` nearly equal blocks of the 2-D tensor t."""
        n = t.shape[0]
        step = (n + parts - 1) // parts
        return t[min(n, i * step):min(n, (i + 1) * step)]

    def run(self, items, ev_start=None, ev_end=None, stages=None):
        """ev_start / ev_end (optional torch.cuda.Event with timing) are recorded
        before the first copy in and after the last copy out.  stages (optional
        list) receives, per product, timing events around its copy in (first
        input stream), its product and its copy out (first output stream):
        (in_begin, in_end, comp_begin, comp_end, out_begin, out_end)."""
        ns = len(self.s_in)
        used = [False, False]

        def tev():
            return torch.cuda.Event(enable_timing=True)
        if ev_start is not None:
            ev_start.record(self.s_in[0])
            for s in self.s_in[1:]:
                s.wait_stream(self.s_in[0])
        for i, (Ah, Bh, Ch) in enumerate(items):
            b = i & 1
            st = [tev() for _ in range(6)] if stages is not None else None
            for c in range(ns):
                if used[b]:  # buffer b was last used two products ago
                    self.s_in[c].wait_event(self.ev_done[b])
                with torch.cuda.stream(self.s_in[c]):
                    if st is not None and c == 0:
                        st[0].record(self.s_in[0])
                    self._rows(self.A[b], c, ns).copy_(self._rows(Ah, c, ns), non_blocking=True)
                    self._rows(self.B[b], c, ns).copy_(self._rows(Bh, c, ns), non_blocking=True)
                    if st is not None and c == 0:
                        st[1].record(self.s_in[0])
                    self.ev_in[c][b].record(self.s_in[c])
                self.s_comp.wait_event(self.ev_in[c][b])
                if used[b]:
                    self.s_comp.wait_event(self.ev_out[c][b])
            with torch.cuda.stream(self.s_comp):
                if st is not None:
                    st[2].record(self.s_comp)
                maxprod_pnorm(self.A[b], self.B[b], out=self.C[b], stream=self.s_comp, **self.opts)
                if st is not None:
                    st[3].record(self.s_comp)
                self.ev_done[b].record(self.s_comp)
            for c in range(ns):
                self.s_out[c].wait_event(self.ev_done[b])
                with torch.cuda.stream(self.s_out[c]):
                    if st is not None and c == 0:
                        st[4].record(self.s_out[0])
                    self._rows(Ch, c, ns).copy_(self._rows(self.C[b], c, ns), non_blocking=True)
                    if st is not None and c == 0:
                        st[5].record(self.s_out[0])
                    self.ev_out[c][b].record(self.s_out[c])
            if st is not None:
                stages.append(st)
            used[b] = True
        last = self.s_out[0]
        for s in self.s_out[1:] + self.s_in + [self.s_comp]:
            last.wait_stream(s)
        if ev_end is not None:
            ev_end.record(last)
        last.synchronize()


def stage_summary(stages, h2d_bytes, d2h_bytes):
    """Mean milliseconds of each pipeline stage over the products (events from
    HostPipeline.run, after it returned), with the copy rates in GB/s."""
    if not stages:
        return {}
    n = len(stages)
    cin = sum(s[0].elapsed_time(s[1]) for s in stages) / n
    comp = sum(s[2].elapsed_time(s[3]) for s in stages) / n
    cout = sum(s[4].elapsed_time(s[5]) for s in stages) / n
    return {"h2d_ms": cin, "compute_ms": comp, "d2h_ms": cout,
            "h2d_gbs": h2d_bytes / (cin / 1e3) / 1e9, "d2h_gbs": d2h_bytes / (cout / 1e3) / 1e9}
