"""FP64 CPU oracle for the continuous max-flow solvers (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this package.  The CUDA product path never imports it.  The arithmetic lives in
``cmf_oracle.c`` (plain C, double precision, one loop per step of the paper);
this module compiles it with gcc and wraps it with ctypes.

Algorithm codes: 0 pADMMI (Fortin-Glowinski with r = 1), 1 rpADMMI
(Fortin-Glowinski, Eq. rpADMMI), 2 rpADMMII (Eckstein-Bertsekas, Eq. rpADMMII),
3 rPDRQ (preconditioned Douglas-Rachford, Eq. iteration:quadratic:seg /
Eq. pdrq:4labels), 4 pADMM-TY (the classical multi-block ADMM, Eq. ADMM:Tai_yuan /
Eq. mADMM:Tai_yuan), 5 ALG1 (the Chambolle-Pock primal-dual method of the
Appendix, Eq. iteration:pd:seg / Eq. alg1:4labels).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

PADMM, RPADMM_FG, RPADMM_EB, RPDRQ, TY, CP = 0, 1, 2, 3, 4, 5
ALGO_NAMES = {PADMM: "pADMMI", RPADMM_FG: "rpADMMI", RPADMM_EB: "rpADMMII", RPDRQ: "rPDRQ",
              TY: "pADMM-TY", CP: "ALG1"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmf_oracle.c")
_LIB = os.path.join(_HERE, "libcmf_oracle.so")


class Params(ctypes.Structure):
    _fields_ = [
        ("algo", ctypes.c_int), ("aniso", ctypes.c_int), ("sweeps", ctypes.c_int),
        ("literal_potts_u", ctypes.c_int),
        ("c", ctypes.c_double), ("a", ctypes.c_double), ("a1", ctypes.c_double),
        ("a2", ctypes.c_double), ("rho", ctypes.c_double), ("r", ctypes.c_double),
        ("sigma", ctypes.c_double), ("tau", ctypes.c_double),
    ]


def default_params(algo: int, L: int = 2, **kw) -> Params:
    """The paper's settings (Sec. 4): c = 0.3, a = 8, a~ = a_1 = 2, a_2 = 2L,
    rho = 1.9, r = 1.618; rPDRQ sigma = 0.2, tau = 1.0 (two labels) or
    sigma = 5, tau = 0.4 (Potts); ALG1 sigma = 0.4, tau = 1/(L'^2 sigma) with
    L'^2 = 10 (two labels) or 9 + L; one sRBGS sweep."""
    sigma, tau = (0.2, 1.0) if L == 2 else (5.0, 0.4)
    if algo == CP:
        sigma = 0.4
        tau = 1.0 / ((10.0 if L == 2 else 9.0 + L) * sigma)
    p = Params(algo=algo, aniso=0, sweeps=1, literal_potts_u=0, c=0.3, a=8.0, a1=2.0,
               a2=2.0 * L, rho=1.9, r=1.618, sigma=sigma, tau=tau)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree),
    with OpenMP for its element-wise loops where the compiler has it (the
    results do not depend on the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                "-o", _LIB, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
    return _LIB


def set_threads(n: int) -> int:
    """Threads for the oracle's element-wise loops (n < 1 keeps the current
    setting); returns the count in use (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        L = _lib
        L.orc_grad.argtypes = [i, i, dp, dp, dp]
        L.orc_div.argtypes = [i, i, dp, dp, dp]
        L.orc_project_alpha.argtypes = [ctypes.c_size_t, dp, dp, dp, i]
        L.orc_srbgs.argtypes = [i, i, ctypes.c_double, ctypes.c_double, dp, dp, i]
        L.orc_set_threads.argtypes = [i]
        L.orc_set_threads.restype = i
        L.orc_simplex.argtypes = [i, dp, dp]
        L.orc_simplex.restype = i
        L.orc_binary_init.argtypes = [i, i, dp, dp, i, ctypes.c_double, dp, dp, dp, dp, dp]
        L.orc_binary_run.argtypes = [i, i, dp, dp, dp, ctypes.POINTER(Params), i, i,
                                     dp, dp, dp, dp, dp]
        L.orc_binary_run.restype = i
        L.orc_binary_eval.argtypes = [i, i, dp, dp, dp, i, i, ctypes.c_double,
                                      dp, dp, dp, dp, dp, dp]
        L.orc_potts_init.argtypes = [i, i, i, dp, i, ctypes.c_double, dp, dp, dp, dp, dp]
        L.orc_potts_run.argtypes = [i, i, i, dp, dp, ctypes.POINTER(Params), i, i,
                                    dp, dp, dp, dp, dp]
        L.orc_potts_run.restype = i
        L.orc_potts_eval.argtypes = [i, i, i, dp, dp, i, i, ctypes.c_double,
                                     dp, dp, dp, dp, dp, dp]
        L.orc_potts_eval.restype = i
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _alpha_field(alpha, H: int, W: int) -> np.ndarray:
    if np.isscalar(alpha):
        return np.full((H, W), float(np.float32(alpha)))
    return _f64(alpha)


# --- discrete operators -------------------------------------------------------

def grad(g):
    g = _f64(g)
    H, W = g.shape
    gx, gy = np.empty_like(g), np.empty_like(g)
    lib().orc_grad(H, W, _ptr(g), _ptr(gx), _ptr(gy))
    return gx, gy


def div(qx, qy):
    qx, qy = _f64(qx), _f64(qy)
    H, W = qx.shape
    d = np.empty_like(qx)
    lib().orc_div(H, W, _ptr(qx), _ptr(qy), _ptr(d))
    return d


def project_alpha(qx, qy, alpha, aniso: int = 0):
    qx, qy = _f64(qx).copy(), _f64(qy).copy()
    al = _alpha_field(alpha, *qx.shape)
    lib().orc_project_alpha(qx.size, _ptr(qx), _ptr(qy), _ptr(al), aniso)
    return qx, qy


def srbgs(b, u, kappa: float, st: float, sweeps: int = 1):
    b, u = _f64(b), _f64(u).copy()
    H, W = u.shape
    lib().orc_srbgs(H, W, kappa, st, _ptr(b), _ptr(u), sweeps)
    return u


def simplex(v):
    v = _f64(v)
    w = np.empty_like(v)
    if lib().orc_simplex(v.size, _ptr(v), _ptr(w)) != 0:
        raise ValueError("oracle: the simplex projection takes 1 to 64 entries")
    return w


# --- binary model -------------------------------------------------------------



def _run_scheduled(run, args, params: Params, n_iter: int, state, rho_schedule, k0: int):
    """Relaxed iterations with a sequence {rho_k} (the rho_k of Eq.
    update:two:sun:lag, Eq. rpADMMII and the relaxed Douglas-Rachford step,
    which Thm 1 and Thm 2 take non-decreasing in (0, 2)): iteration k0 + i uses
    rho_schedule[k0 + i] while the sequence covers it, params.rho after."""
    sched = np.asarray(rho_schedule, dtype=np.float64).ravel()
    i = 0
    while i < n_iter and k0 + i < sched.size:
        q = Params.from_buffer_copy(params)
        q.rho = float(sched[k0 + i])
        state = run(*args, q, 1, state)
        i += 1
    if i < n_iter or state is None:
        state = run(*args, params, n_iter - i, state)
    return state


def binary_run(Cs, Ct, alpha, params: Params, n_iter: int, state=None, rho_schedule=None,
               k0: int = 0) -> dict:
    """Run n_iter iterations.  state=None: cold start.  Returns the state dict
    (u, qx, qy, ps, pt); for rPDRQ the flow entries hold (qbar, pbar).
    rho_schedule: see _run_scheduled (k0 = index of the first iteration)."""
    if rho_schedule is not None:
        return _run_scheduled(binary_run, (Cs, Ct, alpha), params, n_iter, state,
                              rho_schedule, k0)
    Cs, Ct = _f64(Cs), _f64(Ct)
    H, W = Cs.shape
    al = _alpha_field(alpha, H, W)
    cold = state is None
    st = {k: (np.zeros((H, W)) if cold else _f64(state[k]).copy())
          for k in ("u", "qx", "qy", "ps", "pt")}
    rc = lib().orc_binary_run(H, W, _ptr(Cs), _ptr(Ct), _ptr(al), ctypes.byref(params), n_iter,
                              int(cold), *[_ptr(st[k]) for k in ("u", "qx", "qy", "ps", "pt")])
    if rc != 0:
        raise ValueError("oracle: bad parameters")
    return st


def binary_eval(Cs, Ct, alpha, state, params: Params):
    """(E, D, relative gap, conservation residual) of a binary state."""
    Cs, Ct = _f64(Cs), _f64(Ct)
    H, W = Cs.shape
    al = _alpha_field(alpha, H, W)
    out = np.zeros(4)
    arrs = [_f64(state[k]) for k in ("u", "qx", "qy", "ps", "pt")]
    lib().orc_binary_eval(H, W, _ptr(Cs), _ptr(Ct), _ptr(al), params.aniso,
                          int(params.algo == RPDRQ), params.tau, *[_ptr(a) for a in arrs],
                          _ptr(out))
    return tuple(float(x) for x in out)


# --- Potts model --------------------------------------------------------------

def potts_run(C, alpha, params: Params, n_iter: int, state=None, rho_schedule=None,
              k0: int = 0) -> dict:
    """State dict: u, qx, qy, p of shape (L, H, W) and ps of shape (H, W).
    rho_schedule: see _run_scheduled (k0 = index of the first iteration)."""
    if rho_schedule is not None:
        return _run_scheduled(potts_run, (C, alpha), params, n_iter, state, rho_schedule, k0)
    C = _f64(C)
    L, H, W = C.shape
    al = _alpha_field(alpha, H, W)
    cold = state is None
    st = {}
    for k in ("u", "qx", "qy", "p"):
        st[k] = np.zeros((L, H, W)) if cold else _f64(state[k]).copy()
    st["ps"] = np.zeros((H, W)) if cold else _f64(state["ps"]).copy()
    rc = lib().orc_potts_run(H, W, L, _ptr(C), _ptr(al), ctypes.byref(params), n_iter, int(cold),
                             *[_ptr(st[k]) for k in ("u", "qx", "qy", "p", "ps")])
    if rc != 0:
        raise ValueError("oracle: bad parameters")
    return st


def potts_eval(C, alpha, state, params: Params):
    C = _f64(C)
    L, H, W = C.shape
    al = _alpha_field(alpha, H, W)
    out = np.zeros(4)
    arrs = [_f64(state[k]) for k in ("u", "qx", "qy", "p", "ps")]
    rc = lib().orc_potts_eval(H, W, L, _ptr(C), _ptr(al), params.aniso,
                              int(params.algo == RPDRQ), params.tau, *[_ptr(a) for a in arrs],
                              _ptr(out))
    if rc != 0:
        raise ValueError("oracle: Potts certificates take 2 to 64 labels")
    return tuple(float(x) for x in out)


# --- labellings -------------------------------------------------------------------

def binary_labels(u) -> np.ndarray:
    """Thresholded labelling 1[u > 1/2] (any threshold in (0,1) is allowed by
    the thresholding result quoted after Eq. seg:chanvese)."""
    return (np.asarray(u) > 0.5).astype(np.uint8)


def potts_labels(u) -> np.ndarray:
    """argmax_i u_i, ties to the lowest index."""
    return np.argmax(np.asarray(u), axis=0).astype(np.int32)


def solve(inst, algo: int, tol: float = 1e-4, max_iter: int = 20000, check_every: int = 10,
          params: Params | None = None, rho_schedule=None):
    """Iterate until the relative primal-dual gap is <= tol (checked every
    check_every iterations).  Returns (state, iterations, history)."""
    if params is None:
        params = default_params(algo, inst.L)
    hist = []
    state = None
    it = 0
    while it < max_iter:
        k = min(check_every, max_iter - it)
        if inst.kind == "binary":
            state = binary_run(inst.costs[0], inst.costs[1], inst.alpha, params, k, state,
                               rho_schedule, it)
            ev = binary_eval(inst.costs[0], inst.costs[1], inst.alpha, state, params)
        else:
            state = potts_run(inst.costs, inst.alpha, params, k, state, rho_schedule, it)
            ev = potts_eval(inst.costs, inst.alpha, state, params)
        it += k
        hist.append((it,) + ev)
        if ev[2] <= tol:
            break
    return state, it, hist
