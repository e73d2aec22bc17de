"""GPU parity on the method's degenerate inputs, through every kernel family
(warp strips, two-iteration warp strips, TMA tiles, shared-memory tiles and
the plain one-kernel-per-step form), against the FP64 oracle:

* alpha = 0 everywhere: P_alpha(q) = 0 (Eq. projections read with alpha = 0),
  so the flows stay 0 and u stays the pointwise argmin of the data cost;
* alpha fields with exact zeros among positive weights;
* data costs with exact ties, where the cold start takes the first cheapest
  label (binary: u = 1 only where C_t < C_s) and the labelling must agree.

Tolerances as in the other parity tests: float32 state within 1e-4 of the
oracle after a fixed iteration count, certificates within 1e-5 relative."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu

ALGOS = [0, 1, 2, 3, 4, 5]
TOL_U = 1e-4
# (variant, impl): automatic choice, warp strips, two iterations per launch
# (binary ADMM; the others run as warp strips), TMA tiles of 16 rows (ADMM;
# rPDRQ falls back to shared-memory tiles), shared-memory tiles, plain form
PATHS = [(0, 0), (2, 0), (4, 0), (16, 0), (1, 0), (0, 1)]
PATH_IDS = ["auto", "strip", "strip2", "tma16", "tile", "plain"]


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _alpha_with_zeros(H, W, seed, base=0.4):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, base, size=(H, W)).astype(np.float32)
    a[rng.random((H, W)) < 0.35] = 0.0
    a[:, 5] = 0.0  # a whole column of zero weight
    return a


def _binary_cases():
    H, W = 38, 64  # even width: every kernel family applies
    rng = np.random.default_rng(41)
    tied = (rng.integers(0, 3, size=(2, H, W)) / 4.0).astype(np.float32)
    inst0 = synth.random_binary(H, W, seed=42, alpha=0.0)
    instz = synth.random_binary(H, W, seed=43, alpha=0.3)
    instz.alpha = _alpha_with_zeros(H, W, 44)
    instt = synth.random_binary(H, W, seed=45, alpha=0.3)
    instt.costs = tied
    return {"alpha0": inst0, "alpha_zeros": instz, "tied_costs": instt}


def _potts_cases():
    H, W, L = 34, 64, 4
    rng = np.random.default_rng(51)
    tied = (rng.integers(0, 3, size=(L, H, W)) / 4.0).astype(np.float32)
    inst0 = synth.random_potts(H, W, L, seed=52, alpha=0.0)
    instz = synth.random_potts(H, W, L, seed=53, alpha=0.3)
    instz.alpha = _alpha_with_zeros(H, W, 54, base=0.3)
    instt = synth.random_potts(H, W, L, seed=55, alpha=0.25)
    instt.costs = tied
    return {"alpha0": inst0, "alpha_zeros": instz, "tied_costs": instt}


def _binary_gpu(cmf, inst, algo, n, variant, impl):
    p = cmf.default_params(algo, 2, variant=variant, impl=impl)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    torch.cuda.synchronize()
    u0 = b.state()["u"]
    cmf.cmf_iterate_binary(b, n)
    torch.cuda.synchronize()
    return b, u0


def _potts_gpu(cmf, inst, algo, n, variant, impl):
    p = cmf.default_params(algo, inst.L, variant=variant, impl=impl)
    s = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(s)
    torch.cuda.synchronize()
    u0 = s.state()["u"]
    cmf.cmf_iterate_potts(s, n)
    torch.cuda.synchronize()
    return s, u0


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", ["alpha0", "alpha_zeros", "tied_costs"])
def test_binary_degenerate_inputs(cmf, case, algo, path):
    inst = _binary_cases()[case]
    Cs, Ct = inst.costs
    b, u0 = _binary_gpu(cmf, inst, algo, 30, *path)
    # cold start: u = 1 exactly where C_t < C_s (ties stay 0)
    np.testing.assert_array_equal(u0, (Ct < Cs).astype(np.float64))
    got = b.state()
    p = O.default_params(algo, 2)
    ref = O.binary_run(Cs, Ct, inst.alpha, p, 30)
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)
    if case == "alpha0" and algo != 3:
        # zero weight: the flows stay exactly zero and u at the argmin
        assert np.abs(got["qx"]).max() == 0.0 and np.abs(got["qy"]).max() == 0.0
        np.testing.assert_array_equal(O.binary_labels(got["u"]), (Ct < Cs).astype(np.uint8))
    if case == "alpha_zeros" and algo != 3:
        z = inst.alpha == 0.0
        assert np.abs(got["qx"][z]).max() == 0.0 and np.abs(got["qy"][z]).max() == 0.0
    E, D, gap, res = cmf.cmf_eval_binary(b)
    Eo, Do, gapo, reso = O.binary_eval(Cs, Ct, inst.alpha, got, p)
    assert abs(E - Eo) <= 1e-5 * abs(Eo) + 1e-9
    assert abs(D - Do) <= 1e-5 * abs(Eo) + 1e-9


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", ["alpha0", "alpha_zeros", "tied_costs"])
def test_potts_degenerate_inputs(cmf, case, algo, path):
    inst = _potts_cases()[case]
    C = inst.costs
    s, u0 = _potts_gpu(cmf, inst, algo, 24, *path)
    # cold start: u_i = 1 for the first cheapest label, also under ties
    first = np.argmin(C, axis=0)
    u_exp = (np.arange(inst.L)[:, None, None] == first[None]).astype(np.float64)
    np.testing.assert_array_equal(u0, u_exp)
    got = s.state()
    p = O.default_params(algo, inst.L)
    ref = O.potts_run(C, inst.alpha, p, 24)
    for k in ("u", "qx", "qy", "p", "ps"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)
    if case == "alpha0" and algo != 3:
        assert np.abs(got["qx"]).max() == 0.0 and np.abs(got["qy"]).max() == 0.0
        np.testing.assert_array_equal(O.potts_labels(got["u"]), first)
    if case == "alpha_zeros" and algo != 3:
        z = np.broadcast_to(inst.alpha == 0.0, got["qx"].shape)
        assert np.abs(got["qx"][z]).max() == 0.0 and np.abs(got["qy"][z]).max() == 0.0
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(C, inst.alpha, got, p)
    assert abs(E - Eo) <= 1e-5 * abs(Eo) + 1e-9
    assert abs(D - Do) <= 1e-5 * abs(Eo) + 1e-9


@pytest.mark.parametrize("model", ["binary", "potts"])
def test_alpha_zero_solve_is_the_argmin(cmf, model):
    """With alpha = 0 the cold start is already optimal: the solve stops at
    its first check with a gap of zero up to the float32 rounding of the
    per-pixel terms (the primal sums them per label, the dual per pixel)."""
    if model == "binary":
        inst = _binary_cases()["alpha0"]
        p = cmf.default_params(2, 2, tol_gap=1e-7, max_iter=200, check_every=10)
        b = cmf.alloc_binary(inst, p)
        status, iters, hist = cmf.cmf_solve_binary(b)
        expect = (inst.costs[1] < inst.costs[0]).astype(np.uint8)
        labels = O.binary_labels(b.state()["u"])
    else:
        inst = _potts_cases()["alpha0"]
        p = cmf.default_params(2, inst.L, tol_gap=1e-7, max_iter=200, check_every=10)
        b = cmf.alloc_potts(inst, p)
        status, iters, hist = cmf.cmf_solve_potts(b)
        expect = np.argmin(inst.costs, axis=0)
        labels = O.potts_labels(b.state()["u"])
    assert status == cmf.OK and iters == 10 and abs(hist[0, 3]) <= 1e-7
    np.testing.assert_array_equal(labels, expect)
