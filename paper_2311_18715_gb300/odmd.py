"""Python face of libodmd: torch tensors in, C ABI calls out.

torch provides device memory (the workspace, outputs) and streams; every step of the
online DMD runs in the CUDA kernels behind include/odmd.h.  There is no CPU path: if
the library is missing or no GPU is present, construction fails.
"""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import torch

from ._lib import PREC, OdmdConfig, check, load_library

_SNAP_DTYPE = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.float32}


class OnlineDMD:
    """Online DMD of a snapshot stream on one GPU (Sec. 2.3 of the paper).

    update(x) appends u^k; predict(ts) returns u(t) = Re(Phi Lambda^t Phi^+ u^0) for the
    step counts in ts (rows of the result); check(t, x_fom) is the relative-L2
    credibility test of the hybrid FOM/ROM loop (Sec. 2.2).  tensor_cores=False keeps
    rollouts and compactions on the CUDA cores (ODMD_CUDA_CORES); pipeline=False runs each
    update to its end before the next (ODMD_NO_PIPELINE), with bitwise the same results.
    """

    def __init__(self, n: int, r_max: int, prec: str = "fp64", slack: int = 16,
                 trunc_tol: float = 1e-10, check_tol: float = 1e-5, refine_every: int = 0,
                 stream: torch.cuda.Stream | None = None, device: torch.device | int | None = None,
                 tensor_cores: bool = True, pipeline: bool = True):
        if prec not in PREC:
            raise ValueError(f"prec must be one of {sorted(PREC)}")
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("OnlineDMD needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.n, self.r_max, self.prec = int(n), int(r_max), prec
        self.dtype = _SNAP_DTYPE[prec]
        cfg = OdmdConfig()
        check(self._lib, self._lib.odmd_config_default(C.byref(cfg), self.n, self.r_max))
        cfg.slack = int(slack)
        cfg.trunc_tol = float(trunc_tol)
        cfg.check_tol = float(check_tol)
        cfg.prec = PREC[prec]
        cfg.refine_every = int(refine_every)
        cfg.flags = (0 if tensor_cores else 1) | (0 if pipeline else 2)  # ODMD_CUDA_CORES, ODMD_NO_PIPELINE
        self.cfg = cfg
        nbytes = C.c_size_t()
        check(self._lib, self._lib.odmd_footprint(C.byref(cfg), C.byref(nbytes)))
        self.footprint = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(self.footprint, dtype=torch.uint8, device=self.device)
            h = C.c_void_p()
            check(self._lib, self._lib.odmd_create(C.byref(cfg), C.c_void_p(self.workspace.data_ptr()),
                                                   self.footprint, C.c_void_p(self.stream.cuda_stream),
                                                   C.byref(h)))
        self._h = h

    # ------------------------------------------------------------------ helpers
    def _ck(self, status: int) -> None:
        check(self._lib, status, self._h)

    def _snap(self, x: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(x, torch.Tensor) or x.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if x.dtype != self.dtype or x.numel() != self.n or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of {self.n} elements")
        if self.stream != torch.cuda.current_stream(self.device):
            x.record_stream(self.stream)
        return x

    # ------------------------------------------------------------------ API
    def update(self, x: torch.Tensor) -> None:
        x = self._snap(x, "x")
        self._ck(self._lib.odmd_update(self._h, C.c_void_p(x.data_ptr())))

    def predict(self, ts: Sequence[float], out: torch.Tensor | None = None) -> torch.Tensor:
        """Return a (len(ts), n) tensor whose row j is u(t_j)."""
        ts = [float(t) for t in ts]
        k = len(ts)
        if out is None:
            out = torch.empty((k, self.n), dtype=self.dtype, device=self.device)
        elif out.shape != (k, self.n) or out.dtype != self.dtype or not out.is_contiguous():
            raise ValueError("out must be a contiguous (k, n) tensor of the snapshot dtype")
        arr = (C.c_double * max(k, 1))(*ts)
        self._ck(self._lib.odmd_predict(self._h, arr, k, C.c_void_p(out.data_ptr()), self.n))
        return out

    def check(self, t: float, x_fom: torch.Tensor, tol: float = 0.0) -> tuple[float, bool]:
        x_fom = self._snap(x_fom, "x_fom")
        err = C.c_double()
        ok = C.c_int32()
        self._ck(self._lib.odmd_check(self._h, float(t), C.c_void_p(x_fom.data_ptr()), float(tol),
                                      C.byref(err), C.byref(ok)))
        return float(err.value), bool(ok.value)

    def hybrid_step(self, x_fom: torch.Tensor, tol: float = 0.0,
                    out: torch.Tensor | None = None) -> tuple[torch.Tensor, bool, float]:
        """One step of the hybrid FOM/ROM loop (odmd_hybrid_step): returns the state taken
        (the ROM prediction if it passes the credibility test against x_fom, else x_fom),
        whether the prediction was accepted, and the relative error measured."""
        x_fom = self._snap(x_fom, "x_fom")
        if out is None:
            out = torch.empty(self.n, dtype=self.dtype, device=self.device)
        out = self._snap(out, "out")
        acc = C.c_int32()
        err = C.c_double()
        self._ck(self._lib.odmd_hybrid_step(self._h, C.c_void_p(x_fom.data_ptr()), float(tol),
                                            C.c_void_p(out.data_ptr()), C.byref(acc), C.byref(err)))
        return out, bool(acc.value), float(err.value)

    def refine(self) -> None:
        """odmd_refine: restore L^T L = I now (needs refine_every > 0 at construction)."""
        self._ck(self._lib.odmd_refine(self._h))

    def _callbacks(self, residual, fom, failure):
        from ._lib import FOM_FN, RESIDUAL_FN

        def _res(user, step, u, rr, bb, stream):
            try:
                with torch.cuda.stream(self.stream):
                    residual(int(step))
                return 0
            except Exception as e:  # reported to the library as a failed callback
                failure.append(e)
                return 1

        def _fom(user, step, u, stream):
            try:
                with torch.cuda.stream(self.stream):
                    fom(int(step))
                return 0
            except Exception as e:
                failure.append(e)
                return 1

        return RESIDUAL_FN(_res), FOM_FN(_fom)

    def _check_bufs(self, *tensors):
        for tns in tensors:
            if tns.shape != (self.n,) or tns.dtype != self.dtype or not tns.is_contiguous():
                raise ValueError("state buffers must be contiguous (n,) tensors of the snapshot dtype")

    def hybrid_run(self, residual, fom, state_out: torch.Tensor, prev: torch.Tensor, r: torch.Tensor,
                   b: torch.Tensor, t_final: int, tol: float = 0.0, check_every: int = 10, conv_checks: int = 3,
                   conv_tol: float = 1e-8) -> dict:
        """odmd_hybrid_run: hybrid steps up to t_final with the convergence exit (callbacks as
        in hybrid_step_residual; prev holds the state taken at the previous step, refreshed by
        the library after every step).  Returns the run report as a dict."""
        from ._lib import RunReport
        self._check_bufs(state_out, prev, r, b)
        failure = []
        cres, cfom = self._callbacks(residual, fom, failure)
        rep = RunReport()
        st = self._lib.odmd_hybrid_run(self._h, cres, cfom, None, float(tol), int(t_final), int(check_every),
                                       int(conv_checks), float(conv_tol), C.c_void_p(state_out.data_ptr()),
                                       C.c_void_p(prev.data_ptr()), C.c_void_p(r.data_ptr()),
                                       C.c_void_p(b.data_ptr()), C.byref(rep))
        if failure:
            raise failure[0]
        self._ck(st)
        return {f: getattr(rep, f) for f, _ in RunReport._fields_ if f != "pad"}

    def hybrid_step_residual(self, residual, fom, state_out: torch.Tensor, r: torch.Tensor, b: torch.Tensor,
                             tol: float = 0.0) -> tuple[bool, float]:
        """odmd_hybrid_step_residual: one hybrid step with the residual credibility test.

        residual(step) must fill r with b - A u and b with the right-hand side of the FOM's
        step for the predicted state held in state_out; fom(step) must write the FOM's state
        of that step into state_out.  Both run on this model's stream (torch work inside
        them is enqueued there).  Returns (accepted, relative residual)."""
        self._check_bufs(state_out, r, b)
        failure = []
        cres, cfom = self._callbacks(residual, fom, failure)
        acc, rel = C.c_int32(), C.c_double()
        st = self._lib.odmd_hybrid_step_residual(self._h, cres, cfom, None, float(tol),
                                                 C.c_void_p(state_out.data_ptr()), C.c_void_p(r.data_ptr()),
                                                 C.c_void_p(b.data_ptr()), C.byref(acc), C.byref(rel))
        if failure:
            raise failure[0]
        self._ck(st)
        return bool(acc.value), float(rel.value)

    def update_host(self, X: torch.Tensor) -> None:
        """odmd_update_host: append the rows of a host (CPU) tensor X (count x n, the snapshot
        dtype) as snapshots; the copies overlap the updates when X is in pinned memory, which
        must then stay alive until sync()."""
        if X.device.type != "cpu" or X.dtype != self.dtype or X.dim() != 2 or X.shape[1] != self.n:
            raise ValueError("X must be a CPU (count, n) tensor of the snapshot dtype")
        if X.stride(1) != 1:
            raise ValueError("X rows must be contiguous")
        self._ck(self._lib.odmd_update_host(self._h, C.c_void_p(X.data_ptr()), X.shape[0], X.stride(0)))

    def save(self) -> bytes:
        """odmd_save: the model's whole state as a host checkpoint (synchronises)."""
        nb = C.c_size_t()
        self._ck(self._lib.odmd_checkpoint_size(self._h, C.byref(nb)))
        buf = C.create_string_buffer(nb.value)
        self._ck(self._lib.odmd_save(self._h, buf, nb.value))
        return buf.raw

    def load(self, checkpoint: bytes) -> None:
        """odmd_load: continue from a checkpoint of a handle with the same n, r_max,
        precision and slack."""
        buf = C.create_string_buffer(bytes(checkpoint), len(checkpoint))
        self._ck(self._lib.odmd_load(self._h, buf, len(checkpoint)))

    def sync(self) -> None:
        self._ck(self._lib.odmd_sync(self._h))

    @property
    def rank(self) -> int:
        r = C.c_int32()
        self._ck(self._lib.odmd_get_rank(self._h, C.byref(r)))
        return int(r.value)

    def singular_values(self) -> list[float]:
        buf = (C.c_double * self.r_max)()
        r = C.c_int32()
        self._ck(self._lib.odmd_get_singular_values(self._h, buf, self.r_max, C.byref(r)))
        return [buf[i] for i in range(r.value)]

    def eigs(self) -> tuple[list[complex], list[float]]:
        """DMD eigenvalues and mode amplitudes |b_i| ||Phi e_i||."""
        re = (C.c_double * self.r_max)()
        im = (C.c_double * self.r_max)()
        amp = (C.c_double * self.r_max)()
        r = C.c_int32()
        self._ck(self._lib.odmd_get_eigs(self._h, re, im, amp, self.r_max, C.byref(r)))
        return [complex(re[i], im[i]) for i in range(r.value)], [amp[i] for i in range(r.value)]

    def basis(self) -> torch.Tensor:
        """The orthonormal basis L = L0 Q as an (r, n) tensor (row i = column i of L)."""
        out = torch.empty((self.r_max, self.n), dtype=self.dtype, device=self.device)
        r = C.c_int32()
        self._ck(self._lib.odmd_get_basis(self._h, C.c_void_p(out.data_ptr()), self.n, C.byref(r)))
        return out[: r.value]

    def counts(self) -> tuple[int, int]:
        s = C.c_int64()
        c = C.c_int64()
        self._ck(self._lib.odmd_get_counts(self._h, C.byref(s), C.byref(c)))
        return int(s.value), int(c.value)

    def set_row_shards(self, shards: int) -> None:
        """odmd_set_row_shards: run the passes that end in a reduction as `shards` row shards."""
        self._ck(self._lib.odmd_set_row_shards(self._h, int(shards)))

    def row_blocks(self) -> list[int]:
        """odmd_get_row_blocks: the B + 1 row boundaries of the row blocks."""
        b = C.c_int32()
        self._ck(self._lib.odmd_get_row_blocks(self._h, C.byref(b), None, 0))
        rows = (C.c_int64 * (b.value + 1))()
        self._ck(self._lib.odmd_get_row_blocks(self._h, C.byref(b), rows, b.value + 1))
        return [int(x) for x in rows]

    def profile(self, enable: bool = True) -> None:
        """Start (or stop) per-kernel-class event timing; resets the accumulators."""
        self._ck(self._lib.odmd_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{class: (ms_total, kernels_launched)} plus 'mean_r0' of the profiled pass-A launches."""
        from ._lib import KERNEL_CLASSES
        nk = len(KERNEL_CLASSES)
        ms = (C.c_double * nk)()
        nl = (C.c_int64 * nk)()
        r0 = C.c_double()
        self._ck(self._lib.odmd_profile_read(self._h, ms, nl, nk, C.byref(r0)))
        out = {KERNEL_CLASSES[i]: (ms[i], int(nl[i])) for i in range(nk)}
        out["mean_r0"] = r0.value
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._ck(self._lib.odmd_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_noalloc(pred: torch.Tensor, x_fom: torch.Tensor, tol: float = 0.0,
                  stream: torch.cuda.Stream | None = None) -> tuple[float, bool]:
    """Relative L2 credibility check of a prediction the caller already holds, through
    odmd_check_noalloc: no handle, no workspace, and no device allocation in the library.

    For callers that must not allocate device memory (a callback inside a solver's time
    loop whose memory belongs to the solver's pool, a process under a device-memory cap).
    pred and x_fom: contiguous float64 CUDA tensors of the same length (at most
    33,554,432 elements).  Calls whose GPU work overlaps share one scratch array and race.
    """
    lib = load_library()
    for name, t in (("pred", pred), ("x_fom", x_fom)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if pred.numel() != x_fom.numel() or pred.device != x_fom.device:
        raise ValueError("pred and x_fom must have the same length and device")
    err = C.c_double()
    ok = C.c_int32()
    with torch.cuda.device(pred.device):
        s = stream if stream is not None else torch.cuda.current_stream(pred.device)
        check(lib, lib.odmd_check_noalloc(C.c_void_p(pred.data_ptr()), C.c_void_p(x_fom.data_ptr()),
                                          pred.numel(), float(tol), C.c_void_p(s.cuda_stream),
                                          C.byref(err), C.byref(ok)))
    return float(err.value), bool(ok.value)


def update_batch(models: Sequence[OnlineDMD], xs: Sequence[torch.Tensor]) -> None:
    """odmd_update_batch: append xs[i] to models[i] for every i in one call; instances on
    different streams run concurrently."""
    if len(models) != len(xs):
        raise ValueError("models and xs differ in length")
    lib = load_library()
    xs = [m._snap(x, f"xs[{i}]") for i, (m, x) in enumerate(zip(models, xs))]
    k = len(models)
    hs = (C.c_void_p * max(k, 1))(*[m._h for m in models])
    ps = (C.c_void_p * max(k, 1))(*[x.data_ptr() for x in xs])
    check(lib, lib.odmd_update_batch(hs, ps, k))


def batch_split(models: Sequence[OnlineDMD]) -> int:
    """odmd_get_batch_split: the sub-batch split the tuner chose for this set of models (0
    while it is still timing, -1 if the set has not run as one group)."""
    lib = load_library()
    k = len(models)
    hs = (C.c_void_p * max(k, 1))(*[m._h for m in models])
    out = C.c_int32()
    check(lib, lib.odmd_get_batch_split(hs, k, C.byref(out)))
    return int(out.value)


def predict_batch(models: Sequence[OnlineDMD], ts: Sequence[Sequence[float]]) -> list[torch.Tensor]:
    """odmd_predict_batch: predictions of every model at its own step counts."""
    if len(models) != len(ts):
        raise ValueError("models and ts differ in length")
    lib = load_library()
    k = len(models)
    outs = [torch.empty((len(t), m.n), dtype=m.dtype, device=m.device) for m, t in zip(models, ts)]
    tarrs = [(C.c_double * max(len(t), 1))(*[float(v) for v in t]) for t in ts]
    hs = (C.c_void_p * max(k, 1))(*[m._h for m in models])
    tp = (C.POINTER(C.c_double) * max(k, 1))(*[C.cast(a, C.POINTER(C.c_double)) for a in tarrs])
    ks = (C.c_int32 * max(k, 1))(*[len(t) for t in ts])
    op = (C.c_void_p * max(k, 1))(*[o.data_ptr() for o in outs])
    lds = (C.c_int64 * max(k, 1))(*[m.n for m in models])
    check(lib, lib.odmd_predict_batch(hs, tp, ks, op, lds, k))
    return outs


class OnlineDMDPairs:
    """Online DMD fed (x, y) snapshot pairs that need not be contiguous: the hybrid loop of
    Sec. 2 (Fig. 1) in the reading where only FOM steps update the model (y = FOM(x), x the
    state the FOM started from, a DMD state whenever the step before it was accepted).

    update(x, y) appends the pair; predict(u, ts) returns L A~^t L^T u for integer step
    counts t after the state u (rows of the result).  FP64 accuracy; double tensors.
    """

    def __init__(self, n: int, r_max: int, trunc_tol: float = 1e-10,
                 stream: torch.cuda.Stream | None = None, device: torch.device | int | None = None):
        from ._lib import check_pairs

        self._check = check_pairs
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("OnlineDMDPairs needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.n, self.r_max = int(n), int(r_max)
        nbytes = C.c_size_t()
        check_pairs(self._lib, self._lib.odmd_pairs_footprint(self.n, self.r_max, C.byref(nbytes)))
        self.footprint = int(nbytes.value)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(self.footprint, dtype=torch.uint8, device=self.device)
            h = C.c_void_p()
            check_pairs(self._lib, self._lib.odmd_pairs_create(
                self.n, self.r_max, float(trunc_tol), C.c_void_p(self.workspace.data_ptr()), self.footprint,
                C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def _vec(self, x: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(x, torch.Tensor) or x.device != self.device:
            raise ValueError(f"{name} must be a tensor on {self.device}")
        if x.dtype != torch.float64 or x.numel() != self.n or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor of {self.n} elements")
        if self.stream != torch.cuda.current_stream(self.device):
            x.record_stream(self.stream)
        return x

    def update(self, x: torch.Tensor, y: torch.Tensor) -> None:
        """odmd_pairs_update: X gains x, Y gains y."""
        x, y = self._vec(x, "x"), self._vec(y, "y")
        self._check(self._lib, self._lib.odmd_pairs_update(self._h, C.c_void_p(x.data_ptr()),
                                                           C.c_void_p(y.data_ptr())), self._h)

    def predict(self, u: torch.Tensor, ts: Sequence[float], out: torch.Tensor | None = None) -> torch.Tensor:
        """odmd_pairs_predict: row j is L A~^{t_j} L^T u (integer t_j >= 0, at most 64)."""
        u = self._vec(u, "u")
        ts = [float(t) for t in ts]
        k = len(ts)
        if out is None:
            out = torch.empty((k, self.n), dtype=torch.float64, device=self.device)
        if out.shape != (k, self.n) or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous (len(ts), n) float64 tensor")
        tarr = (C.c_double * max(k, 1))(*ts)
        self._check(self._lib, self._lib.odmd_pairs_predict(self._h, C.c_void_p(u.data_ptr()), tarr, k,
                                                            C.c_void_p(out.data_ptr()), self.n), self._h)
        return out

    def hybrid_step_residual(self, residual, fom, step: int, state: torch.Tensor, nxt: torch.Tensor,
                             r: torch.Tensor, b: torch.Tensor, tol: float = 0.0) -> tuple[bool, float]:
        """odmd_pairs_hybrid_step_residual: one step of the FOM-only hybrid loop.  residual(step)
        fills r and b for the prediction in nxt (state still holds the previous state);
        fom(step) advances nxt in place from the previous state.  Returns (accepted, relative
        residual)."""
        from ._lib import FOM_FN, RESIDUAL_FN

        for t, name in ((state, "state"), (nxt, "next"), (r, "r"), (b, "b")):
            self._vec(t, name)
        failure = []

        def _res(user, st, u, rr, bb, stream):
            try:
                with torch.cuda.stream(self.stream):
                    residual(int(st))
                return 0
            except Exception as e:
                failure.append(e)
                return 1

        def _fom(user, st, u, stream):
            try:
                with torch.cuda.stream(self.stream):
                    fom(int(st))
                return 0
            except Exception as e:
                failure.append(e)
                return 1

        cres, cfom = RESIDUAL_FN(_res), FOM_FN(_fom)
        acc, rel = C.c_int32(), C.c_double()
        st = self._lib.odmd_pairs_hybrid_step_residual(
            self._h, cres, cfom, None, float(tol), int(step), C.c_void_p(state.data_ptr()),
            C.c_void_p(nxt.data_ptr()), C.c_void_p(r.data_ptr()), C.c_void_p(b.data_ptr()), C.byref(acc), C.byref(rel))
        if failure:
            raise failure[0]
        self._check(self._lib, st, self._h)
        return bool(acc.value), float(rel.value)

    def singular_values(self) -> list[float]:
        buf = (C.c_double * self.r_max)()
        r = C.c_int32()
        self._check(self._lib, self._lib.odmd_pairs_get_singular_values(self._h, buf, self.r_max, C.byref(r)),
                    self._h)
        return [buf[i] for i in range(r.value)]

    @property
    def rank(self) -> int:
        return len(self.singular_values())

    @property
    def pairs(self) -> int:
        n = C.c_int64()
        self._check(self._lib, self._lib.odmd_pairs_get_count(self._h, C.byref(n)), self._h)
        return int(n.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._check(self._lib, self._lib.odmd_pairs_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
