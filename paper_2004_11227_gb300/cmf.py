"""Thin ctypes binding of libcmf (include/cmf.h).

Argument marshalling only: torch tensors become device pointers, the current
torch CUDA stream becomes the cudaStream_t, and the C-ABI does all the work.
Importing this module never falls back to anything: if libcmf.so is missing
or was built without CUDA, every call raises.

Planes are row-major (H, pitch) float tensors; ``alloc_binary`` /
``alloc_potts`` allocate correctly pitched state and workspace tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, NOT_CONVERGED = range(6)
PADMM, RPADMM_FG, RPADMM_EB, RPDRQ, TY, CP = range(6)
F32, F16, BF16 = range(3)
FUSED, PLAIN = range(2)
ALGO_NAMES = {PADMM: "pADMMI", RPADMM_FG: "rpADMMI", RPADMM_EB: "rpADMMII", RPDRQ: "rPDRQ",
              TY: "pADMM-TY", CP: "ALG1"}
_TORCH_DTYPE = {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16}


class CmfError(RuntimeError):
    pass


class Params(ctypes.Structure):
    """Mirror of cmf_params."""
    _fields_ = [
        ("algo", ctypes.c_int), ("storage", ctypes.c_int), ("impl", ctypes.c_int),
        ("aniso", ctypes.c_int), ("sweeps", ctypes.c_int), ("max_iter", ctypes.c_int),
        ("check_every", ctypes.c_int), ("warm_start", ctypes.c_int),
        ("use_graph", ctypes.c_int), ("variant", ctypes.c_int),
        ("c", ctypes.c_double), ("a", ctypes.c_double), ("a1", ctypes.c_double),
        ("a2", ctypes.c_double), ("rho", ctypes.c_double), ("r", ctypes.c_double),
        ("sigma", ctypes.c_double), ("tau", ctypes.c_double), ("tol_gap", ctypes.c_double),
        ("costs", ctypes.c_int),
        ("rho_schedule", ctypes.POINTER(ctypes.c_double)), ("rho_schedule_len", ctypes.c_int),
        ("phase_storage", ctypes.c_int), ("phase_gap", ctypes.c_double),
        ("tune_step", ctypes.c_int), ("batch_rows", ctypes.c_int),
    ]

    def set_rho_schedule(self, rhos) -> "Params":
        """Relaxation sequence rho_0, rho_1, ... for the first len(rhos)
        iterations of each iterate / solve call (rpADMMII, rPDRQ); rho after.
        The array is kept alive by this object."""
        arr = np.ascontiguousarray(np.asarray(rhos, dtype=np.float64).ravel())
        self._rho_keep = arr
        if arr.size == 0:
            self.rho_schedule = None
        else:
            self.rho_schedule = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.rho_schedule_len = int(arr.size)
        return self


class Instance(ctypes.Structure):
    """Mirror of cmf_instance (one problem of a batch)."""
    _fields_ = [
        ("model", ctypes.c_int), ("L", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
        ("pitch", ctypes.c_int), ("d_cost", ctypes.c_void_p), ("d_alpha", ctypes.c_void_p),
        ("alpha0", ctypes.c_float), ("d_u", ctypes.c_void_p), ("d_qx", ctypes.c_void_p),
        ("d_qy", ctypes.c_void_p), ("d_p", ctypes.c_void_p), ("d_ps", ctypes.c_void_p),
        ("iters", ctypes.c_int), ("status", ctypes.c_int), ("energy", ctypes.c_double),
        ("dual", ctypes.c_double), ("gap", ctypes.c_double), ("res", ctypes.c_double),
    ]


_lib = None
_SIGS = {
    "cmf_default_params": [ctypes.c_int, ctypes.c_int, ctypes.c_void_p],
    "cmf_status_str": [ctypes.c_int],
    "cmf_workspace_bytes": [ctypes.c_int] * 4 + [ctypes.c_void_p],
    "cmf_init_binary": [ctypes.c_void_p] * 2 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 7,
    "cmf_iterate_binary": [ctypes.c_void_p] * 3 + [ctypes.c_float] + [ctypes.c_int] * 3 +
                          [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6 +
                          [ctypes.c_size_t, ctypes.c_void_p],
    "cmf_eval_binary": [ctypes.c_void_p] * 3 + [ctypes.c_float] + [ctypes.c_int] * 3 +
                       [ctypes.c_void_p] * 8 + [ctypes.c_size_t, ctypes.c_void_p],
    "cmf_eval_binary_noalloc": [ctypes.c_void_p] * 3 + [ctypes.c_float] + [ctypes.c_int] * 3 +
                               [ctypes.c_void_p] * 8,
    "cmf_solve_binary": [ctypes.c_void_p] * 3 + [ctypes.c_float] + [ctypes.c_int] * 3 +
                        [ctypes.c_void_p] * 7 + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_size_t, ctypes.c_void_p],
    "cmf_init_potts": [ctypes.c_void_p] + [ctypes.c_int] * 4 + [ctypes.c_void_p] * 7,
    "cmf_iterate_potts": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_float] +
                         [ctypes.c_int] * 3 + [ctypes.c_void_p, ctypes.c_int] +
                         [ctypes.c_void_p] * 6 + [ctypes.c_size_t, ctypes.c_void_p],
    "cmf_eval_potts": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_float] +
                      [ctypes.c_int] * 3 + [ctypes.c_void_p] * 8 +
                      [ctypes.c_size_t, ctypes.c_void_p],
    "cmf_solve_potts": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_float] +
                       [ctypes.c_int] * 3 + [ctypes.c_void_p] * 7 +
                       [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                        ctypes.c_void_p],
    "cmf_autotune_binary": [ctypes.c_void_p] * 3 + [ctypes.c_float] + [ctypes.c_int] * 3 +
                           [ctypes.c_void_p] * 7 + [ctypes.c_size_t] + [ctypes.c_void_p] * 3,
    "cmf_autotune_potts": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_float] +
                          [ctypes.c_int] * 3 + [ctypes.c_void_p] * 7 + [ctypes.c_size_t] +
                          [ctypes.c_void_p] * 3,
    "cmf_release_graphs": [],
    "cmf_batch_workspace_bytes": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "cmf_solve_batch": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_size_t, ctypes.c_void_p],
    "cmf_autotune_batch": [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 +
                          [ctypes.c_size_t, ctypes.c_void_p],
}
EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libcmf.so (it must have been built: ``_build.build()``)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise CmfError(f"libcmf.so not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.cmf_status_str.restype = ctypes.c_char_p
        L.cmf_workspace_bytes.restype = ctypes.c_size_t
        L.cmf_batch_workspace_bytes.restype = ctypes.c_size_t
        _lib = L
    return _lib


def _check(status: int, what: str, allow=(OK,)) -> int:
    if status not in allow:
        msg = lib().cmf_status_str(status).decode()
        raise CmfError(f"{what}: {msg} (status {status})")
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise CmfError("expected a CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def default_params(algo: int, L: int = 2, **kw) -> Params:
    p = Params()
    _check(lib().cmf_default_params(algo, L, ctypes.byref(p)), "cmf_default_params")
    for k, v in kw.items():
        if k == "rho_schedule":
            p.set_rho_schedule(v)
            continue
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def cmf_release_graphs() -> None:
    """Destroy the solve graphs kept for reuse by cmf_solve_* (see cmf.h)."""
    _check(lib().cmf_release_graphs(), "cmf_release_graphs")


def cmf_workspace_bytes(H: int, W: int, L: int, pitch: int, p: Params) -> int:
    return int(lib().cmf_workspace_bytes(H, W, L, pitch, ctypes.byref(p)))


def pitch_for(W: int) -> int:
    """Row stride in elements: W rounded up to a multiple of 32."""
    return (W + 31) // 32 * 32


# --- state containers --------------------------------------------------------------

class Binary:
    """Device buffers of one binary problem (costs, alpha, state, workspace)."""

    def __init__(self, Cs, Ct, alpha, params: Params, device="cuda"):
        Cs = np.asarray(Cs, dtype=np.float32)
        Ct = np.asarray(Ct, dtype=np.float32)
        self.H, self.W = Cs.shape
        self.pitch = pitch_for(self.W)
        self.params = params
        self.device = device
        self.Cs = _pitched(Cs, self.pitch, device)
        self.Ct = _pitched(Ct, self.pitch, device)
        if np.isscalar(alpha):
            self.alpha, self.alpha0 = None, float(alpha)
        else:
            self.alpha, self.alpha0 = _pitched(np.asarray(alpha, np.float32), self.pitch,
                                               device), 0.0
        sd = _TORCH_DTYPE[params.storage]
        shp = (self.H, self.pitch)
        self.u = torch.zeros(shp, dtype=torch.float32, device=device)
        self.qx = torch.zeros(shp, dtype=sd, device=device)
        self.qy = torch.zeros(shp, dtype=sd, device=device)
        self.ps = torch.zeros(shp, dtype=sd, device=device)
        self.pt = torch.zeros(shp, dtype=sd, device=device)
        nb = cmf_workspace_bytes(self.H, self.W, 2, self.pitch, params)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=device)

    def state(self) -> dict:
        """Host float64 copies of (u, qx, qy, ps, pt) without padding."""
        W = self.W
        return {k: getattr(self, k)[:, :W].float().cpu().double().numpy()
                for k in ("u", "qx", "qy", "ps", "pt")}

    def load_state(self, st: dict) -> None:
        W = self.W
        for k in ("u", "qx", "qy", "ps", "pt"):
            t = getattr(self, k)
            t[:, :W] = torch.as_tensor(np.asarray(st[k]), device=self.device).to(t.dtype)

    def _common(self):
        return (_ptr(self.Cs), _ptr(self.Ct), _ptr(self.alpha), self.alpha0, self.H, self.W,
                self.pitch, ctypes.byref(self.params))

    def _state_ptrs(self):
        return (_ptr(self.u), _ptr(self.qx), _ptr(self.qy), _ptr(self.ps), _ptr(self.pt))


class Potts:
    """Device buffers of one Potts problem with L labels."""

    def __init__(self, C, alpha, params: Params, device="cuda"):
        C = np.asarray(C, dtype=np.float32)
        self.L, self.H, self.W = C.shape
        self.pitch = pitch_for(self.W)
        self.params = params
        self.device = device
        # costs = 2: the cost planes are stored as float16 (rounded once here)
        cdt = torch.float16 if params.costs == 2 else torch.float32
        self.C = _pitched(C, self.pitch, device, cdt)
        if np.isscalar(alpha):
            self.alpha, self.alpha0 = None, float(alpha)
        else:
            self.alpha, self.alpha0 = _pitched(np.asarray(alpha, np.float32), self.pitch,
                                               device), 0.0
        sd = _TORCH_DTYPE[params.storage]
        shp = (self.L, self.H, self.pitch)
        self.u = torch.zeros(shp, dtype=torch.float32, device=device)
        self.qx = torch.zeros(shp, dtype=sd, device=device)
        self.qy = torch.zeros(shp, dtype=sd, device=device)
        self.p = torch.zeros(shp, dtype=sd, device=device)
        # the source flow p_s (one plane shared by the labels) is float32 for
        # every flow storage
        self.ps = torch.zeros((self.H, self.pitch), dtype=torch.float32, device=device)
        nb = cmf_workspace_bytes(self.H, self.W, self.L, self.pitch, params)
        self.ws = torch.empty(nb, dtype=torch.uint8, device=device)

    def state(self) -> dict:
        W = self.W
        out = {k: getattr(self, k)[..., :W].float().cpu().double().numpy()
               for k in ("u", "qx", "qy", "p")}
        out["ps"] = self.ps[:, :W].float().cpu().double().numpy()
        return out

    def load_state(self, st: dict) -> None:
        W = self.W
        for k in ("u", "qx", "qy", "p", "ps"):
            t = getattr(self, k)
            t[..., :W] = torch.as_tensor(np.asarray(st[k]), device=self.device).to(t.dtype)

    def _common(self):
        return (_ptr(self.C), self.L, _ptr(self.alpha), self.alpha0, self.H, self.W,
                self.pitch, ctypes.byref(self.params))

    def _state_ptrs(self):
        return (_ptr(self.u), _ptr(self.qx), _ptr(self.qy), _ptr(self.p), _ptr(self.ps))


def _pitched(a: np.ndarray, pitch: int, device, dtype=torch.float32) -> torch.Tensor:
    shp = a.shape[:-1] + (pitch,)
    t = torch.zeros(shp, dtype=dtype, device=device)
    t[..., :a.shape[-1]] = torch.as_tensor(np.ascontiguousarray(a), device=device).to(dtype)
    return t


def alloc_binary(inst, params: Params, device="cuda") -> Binary:
    return Binary(inst.costs[0], inst.costs[1], inst.alpha, params, device)


def alloc_potts(inst, params: Params, device="cuda") -> Potts:
    return Potts(inst.costs, inst.alpha, params, device)


def alloc_potts_levels(I, levels, alpha, params: Params, device="cuda") -> Potts:
    """A Potts problem whose costs C_i = (I - levels[i])^2 the kernels compute
    where they read them: the returned object carries a copy of ``params``
    with costs = 1, and its cost buffer holds the image plane followed by the
    levels."""
    I = np.asarray(I, dtype=np.float32)
    lev = np.asarray(levels, dtype=np.float32)
    H, W = I.shape
    # a copy with costs = 1: the caller's params object is left as it was
    keep = getattr(params, "_rho_keep", None)
    params = Params.from_buffer_copy(params)
    if keep is not None:
        params._rho_keep = keep
    params.costs = 1
    # shape the container as an L-label problem, then replace its cost buffer
    pot = Potts(np.zeros((len(lev), H, W), np.float32), alpha, params, device)
    pitch = pot.pitch
    buf = torch.zeros(H * pitch + len(lev), dtype=torch.float32, device=device)
    buf[:H * pitch].view(H, pitch)[:, :W] = torch.as_tensor(I, device=device)
    buf[H * pitch:] = torch.as_tensor(lev, device=device)
    pot.C = buf
    return pot


# --- C-ABI calls (same names as include/cmf.h) --------------------------------------

def cmf_init_binary(b: Binary, stream=None) -> None:
    _check(lib().cmf_init_binary(_ptr(b.Cs), _ptr(b.Ct), b.H, b.W, b.pitch,
                                 ctypes.byref(b.params), *b._state_ptrs(), _stream(stream)),
           "cmf_init_binary")


def cmf_iterate_binary(b: Binary, n_iter: int, stream=None) -> None:
    _check(lib().cmf_iterate_binary(*b._common(), n_iter, *b._state_ptrs(), _ptr(b.ws),
                                    b.ws.numel(), _stream(stream)), "cmf_iterate_binary")


def cmf_eval_binary(b: Binary, stream=None):
    out = (ctypes.c_double * 4)()
    _check(lib().cmf_eval_binary(*b._common(), *b._state_ptrs(), out, _ptr(b.ws), b.ws.numel(),
                                 _stream(stream)), "cmf_eval_binary")
    return tuple(out)


def cmf_eval_binary_noalloc(b: Binary, stream=None):
    """Certificates of the binary state without a workspace (the library's
    static scratch; grids up to 4096 x 4096)."""
    out = (ctypes.c_double * 4)()
    _check(lib().cmf_eval_binary_noalloc(*b._common(), *b._state_ptrs(), out,
                                         _stream(stream)), "cmf_eval_binary_noalloc")
    return tuple(out)


def cmf_solve_binary(b: Binary, hist_cap: int = 4096, stream=None):
    """Returns (status, iterations, history array [n, 5])."""
    hist = np.zeros((hist_cap, 5))
    iters = ctypes.c_int(0)
    st = _check(lib().cmf_solve_binary(*b._common(), *b._state_ptrs(),
                                       hist.ctypes.data_as(ctypes.c_void_p), hist_cap,
                                       ctypes.byref(iters), _ptr(b.ws), b.ws.numel(),
                                       _stream(stream)),
                "cmf_solve_binary", allow=(OK, NOT_CONVERGED))
    n = int(np.count_nonzero(hist[:, 0]))
    return st, iters.value, hist[:n]


def cmf_init_potts(s: Potts, stream=None) -> None:
    _check(lib().cmf_init_potts(_ptr(s.C), s.L, s.H, s.W, s.pitch, ctypes.byref(s.params),
                                *s._state_ptrs(), _stream(stream)), "cmf_init_potts")


def cmf_iterate_potts(s: Potts, n_iter: int, stream=None) -> None:
    _check(lib().cmf_iterate_potts(*s._common(), n_iter, *s._state_ptrs(), _ptr(s.ws),
                                   s.ws.numel(), _stream(stream)), "cmf_iterate_potts")


def cmf_eval_potts(s: Potts, stream=None):
    out = (ctypes.c_double * 4)()
    _check(lib().cmf_eval_potts(*s._common(), *s._state_ptrs(), out, _ptr(s.ws), s.ws.numel(),
                                _stream(stream)), "cmf_eval_potts")
    return tuple(out)


def cmf_solve_potts(s: Potts, hist_cap: int = 4096, stream=None):
    hist = np.zeros((hist_cap, 5))
    iters = ctypes.c_int(0)
    st = _check(lib().cmf_solve_potts(*s._common(), *s._state_ptrs(),
                                      hist.ctypes.data_as(ctypes.c_void_p), hist_cap,
                                      ctypes.byref(iters), _ptr(s.ws), s.ws.numel(),
                                      _stream(stream)),
                "cmf_solve_potts", allow=(OK, NOT_CONVERGED))
    n = int(np.count_nonzero(hist[:, 0]))
    return st, iters.value, hist[:n]


class Batch:
    """The C instance table, the stacked binary costs and the workspace of a
    batch, built once so that repeated solves call only the library."""

    def __init__(self, items, params: Params):
        n = len(items)
        self.items, self.params = items, params
        self.insts = (Instance * n)()
        self.keep = []
        for i, it in enumerate(items):
            d = self.insts[i]
            if isinstance(it, Binary):
                cost = torch.stack([it.Cs, it.Ct]).contiguous()
                self.keep.append(cost)
                d.model, d.L = 0, 2
                d.d_p, d.d_ps = _ptr(it.pt), _ptr(it.ps)
            else:
                cost = it.C
                d.model, d.L = 1, it.L
                d.d_p, d.d_ps = _ptr(it.p), _ptr(it.ps)
            d.H, d.W, d.pitch = it.H, it.W, it.pitch
            d.d_cost = _ptr(cost)
            d.d_alpha = _ptr(it.alpha)
            d.alpha0 = it.alpha0
            d.d_u, d.d_qx, d.d_qy = _ptr(it.u), _ptr(it.qx), _ptr(it.qy)
        nb = int(lib().cmf_batch_workspace_bytes(self.insts, n, ctypes.byref(params)))
        if nb == 0:
            raise CmfError("cmf_batch_workspace_bytes: invalid batch or parameters")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=items[0].u.device)

    def solve(self, stream=None):
        st = _check(lib().cmf_solve_batch(self.insts, len(self.items), ctypes.byref(self.params),
                                          _ptr(self.ws), self.ws.numel(), _stream(stream)),
                    "cmf_solve_batch", allow=(OK, NOT_CONVERGED))
        res = [dict(iters=d.iters, status=d.status, energy=d.energy, dual=d.dual, gap=d.gap,
                    res=d.res) for d in self.insts]
        return st, res


def cmf_autotune_batch(items, params: Params, stream=None):
    """cmf_autotune_batch over a list of Binary / Potts containers (their
    state is overwritten).  Returns (best Params, milliseconds)."""
    q = Params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(params), ctypes.sizeof(Params))
    q.batch_rows = 12  # the workspace for the largest item tables
    b = Batch(items, q)
    best = Params()
    ms = ctypes.c_double(0.0)
    _check(lib().cmf_autotune_batch(b.insts, len(items), ctypes.byref(params), ctypes.byref(best),
                                    ctypes.byref(ms), _ptr(b.ws), b.ws.numel(), _stream(stream)),
           "cmf_autotune_batch")
    return best, ms.value


def cmf_solve_batch(items, params: Params, stream=None):
    """Solve a list of Binary / Potts containers as one batch.  Returns
    (status, [per-instance result dicts]); the containers' state tensors hold
    the solutions."""
    return Batch(items, params).solve(stream)


def cmf_autotune_binary(b: Binary, stream=None):
    """Launch-configuration search (see cmf.h); returns (best Params, ms)."""
    best = Params()
    ms = ctypes.c_double(0.0)
    _check(lib().cmf_autotune_binary(*b._common(), *b._state_ptrs(), _ptr(b.ws), b.ws.numel(),
                                     ctypes.byref(best), ctypes.byref(ms), _stream(stream)),
           "cmf_autotune_binary")
    best._rho_keep = getattr(b.params, "_rho_keep", None)  # the copied schedule pointer
    return best, ms.value


def cmf_autotune_potts(s: Potts, stream=None):
    best = Params()
    ms = ctypes.c_double(0.0)
    _check(lib().cmf_autotune_potts(*s._common(), *s._state_ptrs(), _ptr(s.ws), s.ws.numel(),
                                    ctypes.byref(best), ctypes.byref(ms), _stream(stream)),
           "cmf_autotune_potts")
    best._rho_keep = getattr(s.params, "_rho_keep", None)  # the copied schedule pointer
    return best, ms.value


def tuned_params(problem, cache_path: str | None = None) -> Params:
    """Autotuned parameters for a Binary / Potts container, cached in a JSON
    file keyed by (model, H, W, L, storage, algo, impl, tune_step, c,
    phase_storage, phase_gap, SM count, device)."""
    import json

    p = problem.params
    props = torch.cuda.get_device_properties(problem.u.device)
    key = "|".join(str(v) for v in (
        "binary" if isinstance(problem, Binary) else "potts", problem.H, problem.W,
        getattr(problem, "L", 2), p.storage, p.algo, p.impl, p.tune_step, p.c,
        p.phase_storage, p.phase_gap, props.multi_processor_count, props.name))
    path = cache_path or os.environ.get(
        "CMF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cmf_tune.json"))
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    q = Params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(Params))
    q._rho_keep = getattr(p, "_rho_keep", None)  # the copied schedule pointer
    if key in cache:
        q.variant, q.sweeps = cache[key]["variant"], cache[key]["sweeps"]
        q.c = cache[key].get("c", q.c)
        q.phase_gap = cache[key].get("phase_gap", q.phase_gap)
        return q
    if isinstance(problem, Binary):
        best, ms = cmf_autotune_binary(problem)
    else:
        best, ms = cmf_autotune_potts(problem)
    cache[key] = {"variant": best.variant, "sweeps": best.sweeps, "c": best.c,
                  "phase_gap": best.phase_gap, "ms_to_gap": ms}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    with open(path, "w") as f:
        json.dump(cache, f, indent=1)
    q.variant, q.sweeps, q.c, q.phase_gap = best.variant, best.sweeps, best.c, best.phase_gap
    return q
