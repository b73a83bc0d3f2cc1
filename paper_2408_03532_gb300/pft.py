"""Thin Python binding over the C ABI in include/pft.h (argument marshalling only).

Every computation runs in the CUDA library ``lib/libpft_gb300.so``; this module
only passes device pointers, sizes and the current CUDA stream. It raises if
the library has not been built (``python -m paper_2408_03532_gb300.build`` or
``__graft_entry__.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpft_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pft.h")

PFT_OK = 0
PATH_AUTO, PATH_FACTORISED, PATH_DIRECT = 0, 1, 2
PREC_FP32 = 0
PREC_SPLIT_BF16 = 1
TRANSFORM_PFT, TRANSFORM_FULL = 0, 1
MODE_COLOURED, MODE_BATCHED = 0, 1
LAUNCH_PER_COLOUR, LAUNCH_PERSISTENT, LAUNCH_DATAFLOW = 0, 1, 2
PROBE_STEP_NORMALISED, PROBE_STEP_SCALAR = 0, 1
TEST_WAIT_NONE, TEST_WAIT_GRID_BARRIER, TEST_WAIT_DATAFLOW = 0, 1, 2
_ERRORS = {-1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "OOM"}


class PftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"PFT_ERR_{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("n1", "n2", "M1", "M2", "p1", "p2", "q1", "q2", "r1", "r2")] + [
        ("xi1", ctypes.c_double), ("xi2", ctypes.c_double), ("eps", ctypes.c_double),
        ("path", ctypes.c_int), ("precision", ctypes.c_int)]


class PieProblem(ctypes.Structure):
    _fields_ = [("obj_h", ctypes.c_int), ("obj_w", ctypes.c_int), ("n", ctypes.c_int), ("npos", ctypes.c_int),
                ("M", ctypes.c_int), ("p", ctypes.c_int), ("eps", ctypes.c_double), ("mode", ctypes.c_int),
                ("path", ctypes.c_int), ("delta_rel", ctypes.c_double), ("autotune", ctypes.c_int)]


class PieCtxInfo(ctypes.Structure):
    _fields_ = [("ncolours", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int), ("r", ctypes.c_int),
                ("cluster_pft", ctypes.c_int), ("cluster_full", ctypes.c_int),
                ("sweep_ms_pft", ctypes.c_double), ("sweep_ms_full", ctypes.c_double),
                ("persistent_pft", ctypes.c_int), ("persistent_full", ctypes.c_int)]


class PieStats(ctypes.Structure):
    _fields_ = [("phi", ctypes.c_double), ("rel_change", ctypes.c_double)]


class PieSchedule(ctypes.Structure):
    _fields_ = [("beta_pft", ctypes.c_double), ("beta_full", ctypes.c_double), ("tol_pft", ctypes.c_double),
                ("tol_full", ctypes.c_double), ("max_pft", ctypes.c_int), ("max_full", ctypes.c_int),
                ("tv_pft", ctypes.c_double), ("tv_full", ctypes.c_double), ("tv_eps", ctypes.c_double),
                ("pft_batched", ctypes.c_int)]


class PieTrace(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int), ("phi", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("nrmse", ctypes.c_double), ("seconds", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def declared_functions() -> list[str]:
    """Names of the functions declared in include/pft.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(\w+)\s*\(", txt, flags=re.M)))


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "pft_last_error": (ctypes.c_char_p, []),
        "pft_version": (ctypes.c_int, []),
        "pft_design_coefficients": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, _P, _P, _P]),
        "pft_choose_r": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P]),
        "pft_plan_create": (ctypes.c_int, [_P] + [ctypes.c_int] * 6 + [ctypes.c_double] + [ctypes.c_int] * 4),
        "pft_plan_destroy": (ctypes.c_int, [_P]),
        "pft_plan_info_get": (ctypes.c_int, [_P, _P]),
        "pft_plan_tables": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
        "pft_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
        "pft_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P]),
        "pft_fft2": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int, _P]),
        "pft_fft_crop": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P]),
        "pie_ctx_create": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "pie_ctx_destroy": (ctypes.c_int, [_P]),
        "pie_ctx_colours": (ctypes.c_int, [_P, _P, _P]),
        "pie_ctx_info_get": (ctypes.c_int, [_P, _P]),
        "pie_iteration": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, _P, _P]),
        "pie_iteration_mode": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P]),
        "pie_iteration_blind": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               _P, _P]),
        "pie_ctx_probe": (ctypes.c_int, [_P, _P, _P]),
        "pie_ctx_set_probe": (ctypes.c_int, [_P, _P, _P]),
        "warm_start_then_refine": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
        "pie_nrmse": (ctypes.c_int, [_P, _P, _P, _P, _P]),
        "pie_tv_step": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double, _P]),
        "pie_ctx_set_order": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "pie_ctx_set_persistent": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
        "pie_ctx_test_unreachable_wait": (ctypes.c_int, [_P, ctypes.c_int]),
        "pie_ctx_set_cluster": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
        "pie_amp_loss_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
        "pie_nrmse_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
        "pie_lf_create": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
        "pie_lf_destroy": (ctypes.c_int, [_P]),
        "pie_lf_iteration": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P]),
        "pie_lf_colours": (ctypes.c_int, [_P, _P, _P]),
        "pie_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
        "pie_batch_destroy": (ctypes.c_int, [_P]),
        "pie_batch_iteration": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, _P, _P]),
        "pie_batch_classes": (ctypes.c_int, [_P, _P, _P]),
        "pie_batch_set_launch": (ctypes.c_int, [_P, ctypes.c_int]),
        "pie_scan_schedule": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                             ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int64, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != PFT_OK:
        raise PftError(rc, load().pft_last_error().decode())


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _need(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape[-len(shape):]) != tuple(shape):
        raise ValueError(f"{name}: trailing shape {tuple(t.shape)} != {shape}")


# ------------------------------------------------------------ offline phase
def design_coefficients(eps: float, r: int) -> tuple[float, np.ndarray, float]:
    """(xi(eps, r), a (w_j = i^j a_j), uniform error) from the host designer."""
    lib = load()
    xi, err = ctypes.c_double(), ctypes.c_double()
    a = np.zeros(r, dtype=np.float64)
    _check(lib.pft_design_coefficients(eps, r, ctypes.byref(xi), a.ctypes.data, ctypes.byref(err)))
    return xi.value, a, err.value


def choose_r(eps: float, ratio: float) -> int:
    r = ctypes.c_int()
    _check(load().pft_choose_r(eps, ratio, ctypes.byref(r)))
    return r.value


# ------------------------------------------------------------------- plans
class Plan:
    """A PFT plan (Algorithm 4): n1 x n2 frames -> centred M1 x M2 outputs.

    Plan(n, M) is square; n2, M2, p2 (default: as axis 1) make it rectangular
    (PREC_FP32; each axis has its own p, q, r and tables)."""

    def __init__(self, n: int, M: int, p: int = 0, eps: float = 1e-7, r: int = 0,
                 path: int = PATH_AUTO, precision: int = PREC_FP32, n2: int | None = None,
                 M2: int | None = None, p2: int | None = None):
        lib = load()
        h = ctypes.c_void_p()
        n2 = n if n2 is None else n2
        M2 = M if M2 is None else M2
        p2 = p if p2 is None else p2
        _check(lib.pft_plan_create(ctypes.byref(h), n, n2, M, M2, p, p2, eps, r, r, path, precision))
        self._h = h
        info = PlanInfo()
        _check(lib.pft_plan_info_get(h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in PlanInfo._fields_}
        self.n, self.M = n, M
        self.n2, self.M2 = n2, M2

    def tables(self, axis: int = 0) -> tuple[np.ndarray, np.ndarray]:
        ax = "2" if axis else "1"
        q, r, M = self.info["q" + ax], self.info["r" + ax], self.M2 if axis else self.M
        B = np.zeros((q, r), dtype=np.float32)
        W = np.zeros((M, r), dtype=np.complex64)
        _check(load().pft_plan_tables(self._h, axis, B.ctypes.data, W.ctypes.data))
        return B, W

    def forward(self, x, out=None, stream=None):
        import torch
        _need(x, torch.complex64, (self.n, self.n2), "x")
        lead = x.shape[:-2]
        if out is None:
            out = torch.empty(*lead, self.M, self.M2, dtype=torch.complex64, device=x.device)
        batch = int(np.prod(lead)) if len(lead) else 1
        _check(load().pft_forward(self._h, _ptr(x), _ptr(out), batch, _stream(stream)))
        return out

    def adjoint(self, y, out=None, stream=None):
        import torch
        _need(y, torch.complex64, (self.M, self.M2), "y")
        lead = y.shape[:-2]
        if out is None:
            out = torch.empty(*lead, self.n, self.n2, dtype=torch.complex64, device=y.device)
        batch = int(np.prod(lead)) if len(lead) else 1
        _check(load().pft_adjoint(self._h, _ptr(y), _ptr(out), batch, _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().pft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft2(x, inverse: bool = False, out=None, stream=None):
    """Unnormalised full 2-D DFT of n x n frames (inverse: its conjugate transpose)."""
    import torch
    _need(x, torch.complex64, None, "x")
    n = x.shape[-1]
    out = torch.empty_like(x) if out is None else out
    batch = int(np.prod(x.shape[:-2])) if x.dim() > 2 else 1
    _check(load().pft_fft2(_ptr(x), _ptr(out), n, batch, int(inverse), _stream(stream)))
    return out


def fft_crop(x, M: int, out=None, stream=None):
    """Full 2-D FFT then the centred M x M crop (baseline)."""
    import torch
    _need(x, torch.complex64, None, "x")
    n = x.shape[-1]
    lead = x.shape[:-2]
    if out is None:
        out = torch.empty(*lead, M, M, dtype=torch.complex64, device=x.device)
    batch = int(np.prod(lead)) if len(lead) else 1
    _check(load().pft_fft_crop(_ptr(x), _ptr(out), n, M, batch, _stream(stream)))
    return out


def nrmse_noalloc(obj, truth, mask=None, stream=None) -> float:
    """Phase-aligned error of obj against truth over mask (uint8, or None for
    all elements), computed without any device allocation: for callers that
    cannot call cudaMalloc when they need the error (a framework that owns all
    device memory through its own pool, or a latency-critical loop where an
    allocation can synchronise the device). The library keeps the partial sums
    in one fixed device array, so calls must not overlap on the GPU; the call
    synchronises its stream before returning."""
    import torch
    _need(obj, torch.complex64, None, "obj")
    _need(truth, torch.complex64, tuple(obj.shape), "truth")
    if mask is not None:
        _need(mask, torch.uint8, None, "mask")
        if mask.numel() != obj.numel():
            raise ValueError("mask must have one byte per element")
    out = ctypes.c_double()
    _check(load().pie_nrmse_noalloc(_ptr(obj), _ptr(truth), _ptr(mask), obj.numel(), ctypes.byref(out),
                                    _stream(stream)))
    return out.value


# --------------------------------------------------------------------- PIE
def pie_scan_schedule(positions, n: int, obj_shape, order=None, sequential: bool = False) -> dict:
    """The order a coloured sweep visits the positions in (host only, no GPU):
    greedy colours (or, with `sequential`, one colour per position in visiting
    order), the colour-major schedule and each schedule item's dataflow
    predecessors (schedule indices). Returns a dict with ncolours, colour,
    sched, dep_off and dep (numpy int32 arrays)."""
    lib = load()
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(-1, 2))
    N = len(pos)
    o = None if order is None else np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    if o is not None and o.shape != (N,):
        raise ValueError("order must be a permutation of the positions")
    h, w = obj_shape
    ncol, ndep = ctypes.c_int(), ctypes.c_int64()
    _check(lib.pie_scan_schedule(pos.ctypes.data, N, int(n), int(h), int(w), None if o is None else o.ctypes.data,
                                 int(sequential), ctypes.byref(ncol), None, None, None, None, 0, ctypes.byref(ndep)))
    colour, sched = np.empty(N, np.int32), np.empty(N, np.int32)
    dep_off, dep = np.empty(N + 1, np.int32), np.empty(max(1, ndep.value), np.int32)
    _check(lib.pie_scan_schedule(pos.ctypes.data, N, int(n), int(h), int(w), None if o is None else o.ctypes.data,
                                 int(sequential), ctypes.byref(ncol), colour.ctypes.data, sched.ctypes.data, dep_off.ctypes.data,
                                 dep.ctypes.data, len(dep), ctypes.byref(ndep)))
    return {"ncolours": ncol.value, "colour": colour, "sched": sched, "dep_off": dep_off, "dep": dep[:ndep.value]}


@dataclass
class Schedule:
    beta_pft: float = 1.0
    beta_full: float = 1.0
    tol_pft: float = 1e-2
    tol_full: float = 5e-4
    max_pft: int = 50
    max_full: int = 100
    tv_pft: float = 0.0
    tv_full: float = 0.0
    tv_eps: float = 1e-3
    pft_batched: bool = False


class PieContext:
    """One ptychography problem resident on the GPU (probe, scan, amplitudes, plans)."""

    def __init__(self, obj_shape, probe, positions, intensities, M: int, p: int = 0, eps: float = 1e-7,
                 mode: int = MODE_COLOURED, delta_rel: float = 1e-3, autotune: bool = True, stream=None):
        import torch
        n = probe.shape[-1]
        _need(probe, torch.complex64, (n, n), "probe")
        _need(intensities, torch.float32, (n, n), "intensities")
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(-1, 2))
        prob = PieProblem(int(obj_shape[0]), int(obj_shape[1]), n, len(pos), M, p, eps, mode, PATH_AUTO, delta_rel,
                          int(autotune))
        h = ctypes.c_void_p()
        _check(load().pie_ctx_create(ctypes.byref(h), ctypes.byref(prob), _ptr(probe), pos.ctypes.data,
                                     _ptr(intensities), _stream(stream)))
        self._h = h
        self.shape = (int(obj_shape[0]), int(obj_shape[1]))
        self.n, self.M, self.npos = n, M, len(pos)

    def info(self) -> dict:
        i = PieCtxInfo()
        _check(load().pie_ctx_info_get(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in PieCtxInfo._fields_}

    def colours(self) -> np.ndarray:
        nc = ctypes.c_int()
        col = np.zeros(self.npos, dtype=np.int32)
        _check(load().pie_ctx_colours(self._h, ctypes.byref(nc), col.ctypes.data))
        return col

    def _obj(self, obj, name="object"):
        import torch
        _need(obj, torch.complex64, self.shape, name)

    def iteration(self, obj, transform: int = TRANSFORM_PFT, beta: float = 1.0, stats: bool = True, stream=None,
                  mode: int | None = None):
        """One sweep; `mode` (MODE_COLOURED / MODE_BATCHED) overrides the context's."""
        self._obj(obj)
        st = PieStats()
        sp = ctypes.byref(st) if stats else None
        if mode is None:
            _check(load().pie_iteration(self._h, _ptr(obj), transform, beta, sp, _stream(stream)))
        else:
            _check(load().pie_iteration_mode(self._h, _ptr(obj), transform, mode, beta, sp, _stream(stream)))
        return {"phi": st.phi, "rel_change": st.rel_change} if stats else None

    def tv_step(self, obj, lam: float, eps: float = 1e-3, stream=None):
        """One total-variation gradient step on obj, in place."""
        self._obj(obj)
        _check(load().pie_tv_step(self._h, _ptr(obj), lam, eps, _stream(stream)))

    def set_order(self, order=None, sequential: bool = False):
        """Visit the positions in `order` (a permutation; None = index order):
        greedy colours in that order, swept colour-major, or with `sequential`
        one colour per position, so sweeps follow `order` exactly."""
        if order is None:
            _check(load().pie_ctx_set_order(self._h, None, int(sequential)))
            return
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        if o.shape != (self.npos,):
            raise ValueError("order must be a permutation of the positions")
        _check(load().pie_ctx_set_order(self._h, o.ctypes.data, int(sequential)))

    def set_persistent(self, transform: int, persistent=True):
        """Launch form of the coloured sweeps of `transform`: LAUNCH_PER_COLOUR
        (or False), LAUNCH_PERSISTENT (or True: one cooperative launch, grid
        barrier between colours) or LAUNCH_DATAFLOW (one cooperative launch,
        per-position waits on overlapping predecessors)."""
        form = int(persistent) if not isinstance(persistent, bool) else (1 if persistent else 0)
        _check(load().pie_ctx_set_persistent(self._h, transform, form))

    def set_cluster(self, transform: int, cluster: int):
        """CTAs per position (1, 2, 4, 8) for `transform`'s sweeps in every
        launch form; 0 returns to the built-in choice."""
        _check(load().pie_ctx_set_cluster(self._h, transform, int(cluster)))

    def test_unreachable_wait(self, kind: int):
        """Test hook: TEST_WAIT_GRID_BARRIER / TEST_WAIT_DATAFLOW make every
        wait of that launch form unreachable, so the next such sweep runs its
        bounded timeout and reports PFT_ERR_TIMEOUT; TEST_WAIT_NONE turns it off."""
        _check(load().pie_ctx_test_unreachable_wait(self._h, int(kind)))

    def iteration_blind(self, obj, transform: int = TRANSFORM_FULL, beta: float = 1.0, gamma: float = 1.0,
                        stats: bool = True, stream=None, probe_step: int = 0):
        """One blind sweep (object and probe updated; coloured mode).
        probe_step: PROBE_STEP_NORMALISED (pixel-wise, per colour) or
        PROBE_STEP_SCALAR (Eq. epie_probe_update's scalar gamma)."""
        self._obj(obj)
        st = PieStats()
        _check(load().pie_iteration_blind(self._h, _ptr(obj), transform, beta, gamma, int(probe_step),
                                          ctypes.byref(st) if stats else None, _stream(stream)))
        return {"phi": st.phi, "rel_change": st.rel_change} if stats else None

    def probe(self, stream=None):
        import torch
        out = torch.empty(self.n, self.n, dtype=torch.complex64, device="cuda")
        _check(load().pie_ctx_probe(self._h, _ptr(out), _stream(stream)))
        return out

    def set_probe(self, probe, stream=None):
        import torch
        _need(probe, torch.complex64, (self.n, self.n), "probe")
        _check(load().pie_ctx_set_probe(self._h, _ptr(probe), _stream(stream)))

    def nrmse(self, obj, truth, stream=None) -> float:
        self._obj(obj)
        self._obj(truth, "truth")
        out = ctypes.c_double()
        _check(load().pie_nrmse(self._h, _ptr(obj), _ptr(truth), ctypes.byref(out), _stream(stream)))
        return out.value

    def warm_start_then_refine(self, obj, schedule: Schedule, truth=None, stream=None) -> list[dict]:
        self._obj(obj)
        if truth is not None:
            self._obj(truth, "truth")
        s = PieSchedule(schedule.beta_pft, schedule.beta_full, schedule.tol_pft, schedule.tol_full,
                        schedule.max_pft, schedule.max_full, schedule.tv_pft, schedule.tv_full, schedule.tv_eps,
                        int(schedule.pft_batched))
        cap = max(1, schedule.max_pft + schedule.max_full)
        tr = (PieTrace * cap)()
        cnt = ctypes.c_int()
        _check(load().warm_start_then_refine(self._h, _ptr(obj), ctypes.byref(s), _ptr(truth), tr,
                                             ctypes.byref(cnt), _stream(stream)))
        return [{"phase": "pft" if t.phase == TRANSFORM_PFT else "full", "phi": t.phi,
                 "rel_change": t.rel_change, "nrmse": t.nrmse, "seconds": t.seconds} for t in tr[:cnt.value]]

    def amp_loss_grad(self, obj, probe, need_probe_grad: bool = True, stream=None):
        import torch
        self._obj(obj)
        _need(probe, torch.complex64, (self.n, self.n), "probe")
        g_obj = torch.empty_like(obj)
        g_probe = torch.empty_like(probe) if need_probe_grad else None
        loss = ctypes.c_double()
        _check(load().pie_amp_loss_grad(self._h, _ptr(obj), _ptr(probe), _ptr(g_obj), _ptr(g_probe),
                                        ctypes.byref(loss), _stream(stream)))
        return loss.value, g_obj, g_probe

    def close(self):
        if getattr(self, "_h", None):
            load().pie_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LargeFramePie:
    """PFT sweeps of PIE over large frames (n = 2048 ... 16384, M = 128): each
    colour's positions are one batch of the split-BF16 large-frame transforms."""

    def __init__(self, obj_shape, probe, positions, intensities, M: int = 128, p: int = 0, eps: float = 1e-7,
                 stream=None):
        import torch
        n = probe.shape[-1]
        _need(probe, torch.complex64, (n, n), "probe")
        _need(intensities, torch.float32, (n, n), "intensities")
        pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int32).reshape(-1, 2))
        prob = PieProblem(int(obj_shape[0]), int(obj_shape[1]), n, len(pos), M, p, eps, MODE_COLOURED, PATH_AUTO,
                          1e-3, 0)
        h = ctypes.c_void_p()
        _check(load().pie_lf_create(ctypes.byref(h), ctypes.byref(prob), _ptr(probe), pos.ctypes.data,
                                    _ptr(intensities), _stream(stream)))
        self._h = h
        self.shape = (int(obj_shape[0]), int(obj_shape[1]))
        self.n, self.M, self.npos = n, M, len(pos)

    def colours(self) -> tuple[int, int]:
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().pie_lf_colours(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def iteration(self, obj, beta: float = 1.0, stats: bool = True, stream=None):
        """One PFT sweep over all positions, in place on obj."""
        import torch
        _need(obj, torch.complex64, self.shape, "object")
        st = PieStats()
        _check(load().pie_lf_iteration(self._h, _ptr(obj), beta, ctypes.byref(st) if stats else None,
                                       _stream(stream)))
        return {"phi": st.phi, "rel_change": st.rel_change} if stats else None

    def close(self):
        if getattr(self, "_h", None):
            load().pie_lf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PieBatch:
    """Independent PIE problems of different sizes swept together (one graph per sweep).

    Each instance is a dict with keys obj_shape, probe (CUDA complex64 [n, n]),
    positions (int32 [N, 2]), intensities (CUDA float32 [N, n, n]), M and
    optionally p and eps.
    """

    def __init__(self, instances: list[dict], mode: int = MODE_COLOURED, delta_rel: float = 1e-3, stream=None):
        import torch
        cnt = len(instances)
        probs = (PieProblem * cnt)()
        self._keep = []
        probes = (ctypes.c_void_p * cnt)()
        poss = (ctypes.c_void_p * cnt)()
        ints = (ctypes.c_void_p * cnt)()
        self.shapes = []
        for i, inst in enumerate(instances):
            n = inst["probe"].shape[-1]
            _need(inst["probe"], torch.complex64, (n, n), "probe")
            _need(inst["intensities"], torch.float32, (n, n), "intensities")
            pos = np.ascontiguousarray(np.asarray(inst["positions"], dtype=np.int32).reshape(-1, 2))
            self._keep.append(pos)
            h, w = inst["obj_shape"]
            probs[i] = PieProblem(int(h), int(w), n, len(pos), int(inst["M"]), int(inst.get("p", 0)),
                                  float(inst.get("eps", 1e-7)), mode, PATH_AUTO, delta_rel, 0)
            probes[i] = _ptr(inst["probe"])
            poss[i] = pos.ctypes.data
            ints[i] = _ptr(inst["intensities"])
            self.shapes.append((int(h), int(w)))
        hnd = ctypes.c_void_p()
        _check(load().pie_batch_create(ctypes.byref(hnd), cnt, probs, probes, poss, ints, _stream(stream)))
        self._h = hnd
        self.count = cnt

    def classes(self) -> tuple[int, int]:
        nc, nl = ctypes.c_int(), ctypes.c_int()
        _check(load().pie_batch_classes(self._h, ctypes.byref(nc), ctypes.byref(nl)))
        return nc.value, nl.value

    def set_launch(self, form: int):
        """Coloured batches: LAUNCH_PER_COLOUR (one launch per class and
        colour, the default) or LAUNCH_DATAFLOW (one launch per class and sweep)."""
        _check(load().pie_batch_set_launch(self._h, int(form)))

    def iteration(self, objects, transform: int = TRANSFORM_PFT, beta: float = 1.0, stats: bool = True,
                  stream=None):
        import torch
        if len(objects) != self.count:
            raise ValueError("one object per instance")
        ptrs = (ctypes.c_void_p * self.count)()
        for i, o in enumerate(objects):
            _need(o, torch.complex64, self.shapes[i], f"object {i}")
            ptrs[i] = _ptr(o)
        phi = (ctypes.c_double * self.count)() if stats else None
        _check(load().pie_batch_iteration(self._h, ptrs, transform, beta, phi, _stream(stream)))
        return list(phi) if stats else None

    def close(self):
        if getattr(self, "_h", None):
            load().pie_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
