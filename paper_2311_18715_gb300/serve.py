"""Serving loop: many hybrid simulations on one GPU at once (continuous batching).

Each request is one simulation of the hybrid FOM/ROM workflow (Sec. 2.1 of the paper): it
streams its snapshots into an online DMD of its own size and rank cap, then asks for
predictions at some horizons past its last snapshot.  The server

* admits requests in arrival order as device memory allows: the workspace a model needs is
  known before anything is allocated (``footprint``, the C ABI's odmd_footprint), so
  admission by HBM footprint is exact;
* keeps every admitted model resident (basis, operator and eigen-cache stay on the GPU);
* advances all streaming requests together, one snapshot each per round, with one
  ``update_batch`` call (each model on its own CUDA stream, so their kernels overlap), and
  answers the queries of the requests that finished streaming with one ``predict_batch``;
* frees a request's memory as soon as its answers are read back, so waiting requests can
  take its place while others are still running.

Snapshots come from a caller-supplied source per request (for the benchmark, a synthetic
stream drawn on the device); the server only moves them into the models.  Every step runs
in the library's kernels; this module is scheduling only.
"""
from __future__ import annotations

import ctypes as C
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import torch

from ._lib import PREC, OdmdConfig, check, load_library
from .odmd import OnlineDMD, predict_batch, update_batch


def footprint(n: int, r_max: int, prec: str = "fp64", slack: int = 16) -> int:
    """Device bytes of the workspace a model of this shape needs (odmd_footprint)."""
    lib = load_library()
    cfg = OdmdConfig()
    check(lib, lib.odmd_config_default(C.byref(cfg), int(n), int(r_max)))
    cfg.prec = PREC[prec]
    cfg.slack = int(slack)
    nb = C.c_size_t()
    check(lib, lib.odmd_footprint(C.byref(cfg), C.byref(nb)))
    return int(nb.value)


@dataclass
class Request:
    rid: int
    arrival: float                      # seconds after the trace starts
    n: int
    r_max: int
    snapshots: int                      # snapshots streamed before the queries
    horizons: Sequence[float]           # predict u(t) at t = snapshots - 1 + h for each h
    source: Callable[[int, torch.Tensor], None]  # writes snapshot k into the (device) tensor
    prec: str = "fp64"
    slack: int = 16
    source_bytes: int = 0               # device memory the source itself holds
    keep: bool = False                  # copy the predictions to the host in the result


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    updates: int
    predictions: Optional[torch.Tensor] = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Session:
    req: Request
    model: OnlineDMD
    buf: torch.Tensor
    admitted: float
    bytes: int
    k: int = 0
    out: Optional[torch.Tensor] = None


@dataclass
class Server:
    device: torch.device = field(default_factory=lambda: torch.device("cuda", torch.cuda.current_device()))
    hbm_budget: Optional[int] = None    # bytes the server may hand out (default: 90% of free memory)
    max_active: int = 64

    def _need(self, r: Request) -> int:
        elt = 8 if r.prec == "fp64" else 4
        return footprint(r.n, r.r_max, r.prec, r.slack) + r.n * elt + r.source_bytes

    def run(self, requests: Sequence[Request]) -> list[Result]:
        """Serve the trace in real time (arrivals are seconds after the call starts)."""
        pending = deque(sorted(requests, key=lambda q: q.arrival))
        budget = self.hbm_budget
        if budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget = int(0.9 * free)
        for r in pending:
            if self._need(r) > budget:
                raise ValueError(f"request {r.rid} needs more device memory than the budget")
        waiting: deque[Request] = deque()
        active: list[_Session] = []
        used = 0
        results: list[Result] = []
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or waiting or active:
            now = clock()
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # admission in arrival order, by exact footprint
            while waiting and len(active) < self.max_active:
                r = waiting[0]
                need = self._need(r)
                if used + need > budget:
                    break
                waiting.popleft()
                dt = torch.float64 if r.prec == "fp64" else torch.float32
                model = OnlineDMD(r.n, r.r_max, prec=r.prec, slack=r.slack, device=self.device,
                                  stream=torch.cuda.Stream(self.device))
                buf = torch.empty(r.n, dtype=dt, device=self.device)
                active.append(_Session(r, model, buf, clock(), need))
                used += need
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)))
                continue
            # one snapshot for every streaming session, all models updated in one call
            streaming = [s for s in active if s.k < s.req.snapshots]
            if streaming:
                for s in streaming:
                    with torch.cuda.stream(s.model.stream):
                        s.req.source(s.k, s.buf)
                update_batch([s.model for s in streaming], [s.buf for s in streaming])
                for s in streaming:
                    s.k += 1
            # queries of the sessions that have all their snapshots
            done = [s for s in active if s.k >= s.req.snapshots]
            if done:
                ts = [[float(s.req.snapshots - 1 + h) for h in s.req.horizons] for s in done]
                outs = predict_batch([s.model for s in done], ts)
                for s, o in zip(done, outs):
                    s.model.sync()
                    keep = o.cpu() if s.req.keep else None
                    results.append(Result(s.req.rid, s.req.arrival, s.admitted, clock(), s.k, keep))
                    s.model.close()
                    used -= s.bytes
                active = [s for s in active if s.k < s.req.snapshots]
                del done, outs
        return results
