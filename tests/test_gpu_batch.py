"""Batched solve (many instances of uneven size and label count in one
device-driven loop) against the single-instance solver run with the same
kernels (warp strips for Potts instances of even width under the ADMM
algorithms, shared-memory tiles for the others): identical iteration counts
and states within float32 rounding, each instance certified by the FP64
oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _instances():
    return [
        synth.binary_shapes(97, 130, seed=101),
        synth.potts_shapes(64, 71, 3, seed=102),
        synth.binary_disk(40, 33, seed=103),
        synth.potts_shapes(120, 88, 8, seed=104),
        synth.potts_shapes(33, 150, 4, seed=105),
        synth.binary_shapes(150, 64, seed=106),
    ]


def _alloc(cmf, inst, p):
    return cmf.alloc_binary(inst, p) if inst.kind == "binary" else cmf.alloc_potts(inst, p)


@pytest.mark.parametrize("algo", [1, 2, 3, 5])
def test_batch_matches_single_solves(cmf, algo):
    insts = _instances()
    kw = dict(tol_gap=1e-4, max_iter=20000, check_every=10, variant=1)
    if algo == 5:  # one (sigma, tau) for the batch: the 8-label bound (9 + 8) sigma tau <= 1
        kw["tau"] = 1.0 / (17 * 0.4)
    p = cmf.default_params(algo, 2, **kw)
    items = [_alloc(cmf, i, p) for i in insts]
    status, res = cmf.cmf_solve_batch(items, p)
    assert status == cmf.OK, res
    iters = [r["iters"] for r in res]
    assert len(set(iters)) > 1  # instances converge at different iterations
    for inst, item, r in zip(insts, items, res):
        # the batch shares p (sigma, tau, c, ...) and takes a2 = max(a2, 2L)
        q = cmf.default_params(algo, 2, **kw)
        q.a2 = max(q.a2, 2.0 * inst.L)
        if inst.kind == "potts" and inst.W % 2 == 0 and algo != 3:
            q.variant = 2  # the batch runs this instance by warp strips
        single = _alloc(cmf, inst, q)
        if inst.kind == "binary":
            st, it, hist = cmf.cmf_solve_binary(single)
        else:
            st, it, hist = cmf.cmf_solve_potts(single)
        assert st == cmf.OK and it == r["iters"], (inst.kind, it, r["iters"])
        a, b = item.state(), single.state()
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= 1e-5, k
        assert abs(r["gap"] - hist[-1, 3]) <= 1e-7 + 1e-3 * abs(hist[-1, 3])
        po = O.default_params(algo, inst.L, sigma=q.sigma, tau=q.tau, a2=q.a2)
        if inst.kind == "binary":
            E, D, gap, _ = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, a, po)
        else:
            E, D, gap, _ = O.potts_eval(inst.costs, inst.alpha, a, po)
        assert gap <= 1.01e-4


def test_batch_max_iter_cap_and_float16(cmf):
    insts = _instances()[:3]
    kw = dict(tol_gap=1e-12, max_iter=40, check_every=10, storage=1)
    items = [_alloc(cmf, i, cmf.default_params(2, i.L, **kw)) for i in insts]
    status, res = cmf.cmf_solve_batch(items, cmf.default_params(2, 2, **kw))
    assert status == cmf.NOT_CONVERGED
    assert all(r["iters"] == 40 and r["status"] == cmf.NOT_CONVERGED for r in res)


def test_batch_rejects_bad_parameters(cmf):
    items = [_alloc(cmf, synth.binary_disk(16, 16), cmf.default_params(2, 2))]
    for bad in (dict(check_every=5), dict(impl=1), dict(max_iter=105, check_every=10)):
        p = cmf.default_params(2, 2, **bad)
        with pytest.raises(cmf.CmfError):
            cmf.cmf_solve_batch(items, p)


@pytest.mark.parametrize("storage", [0, 1])
def test_batch_strip_instances_float16(cmf, storage):
    """Even-width Potts instances run by warp strips inside the batch: the
    same iteration counts and states as single strip solves, in float32 and
    with float16 flows."""
    insts = [synth.potts_shapes(120, 88, 8, seed=104), synth.potts_shapes(33, 150, 4, seed=105),
             synth.potts_shapes(64, 64, 3, seed=107)]
    kw = dict(tol_gap=2e-3 if storage else 1e-4, max_iter=20000, check_every=10,
              storage=storage)
    p = cmf.default_params(2, 2, **kw)
    items = [cmf.alloc_potts(i, p) for i in insts]
    status, res = cmf.cmf_solve_batch(items, p)
    assert status == cmf.OK, res
    for inst, item, r in zip(insts, items, res):
        q = cmf.default_params(2, 2, variant=2, **kw)
        q.a2 = max(q.a2, 2.0 * inst.L)
        single = cmf.alloc_potts(inst, q)
        st, it, hist = cmf.cmf_solve_potts(single)
        assert st == cmf.OK and it == r["iters"], (it, r["iters"])
        a, b = item.state(), single.state()
        # the two kernels compile the same item arithmetic separately (their
        # coefficients come from registers or from the parameter bank), so
        # float32 results may differ in the last bit; float16 storage turns
        # that into a few units in the last place of the stored flows
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= (1e-5 if storage == 0 else 8e-3), k
        assert r["gap"] <= kw["tol_gap"] and hist[-1, 3] <= kw["tol_gap"]


@pytest.mark.parametrize("algo", [0, 2, 4, 5])
def test_batch_strip_odd_widths_match_oracle(cmf, algo):
    """Potts instances of odd width run by warp strips inside the batch (the
    last pair masked): after a fixed number of iterations every instance
    matches the FP64 oracle element by element (float32 state, 1e-4)."""
    insts = [synth.potts_shapes(37, 71, 3, seed=111), synth.potts_shapes(66, 129, 8, seed=112),
             synth.potts_shapes(45, 60, 4, seed=113), synth.config5(33, 181)]
    kw = dict(tol_gap=0.0, max_iter=40, check_every=10)
    if algo == 5:
        kw["tau"] = 1.0 / (25 * 0.4)
    p = cmf.default_params(algo, 2, **kw)
    items = [cmf.alloc_potts(i, p) for i in insts]
    status, res = cmf.cmf_solve_batch(items, p)
    assert status == cmf.NOT_CONVERGED and all(r["iters"] == 40 for r in res)
    for inst, item in zip(insts, items):
        q = O.default_params(algo, inst.L, a2=max(p.a2, 2.0 * inst.L), sigma=p.sigma, tau=p.tau)
        ref = O.potts_run(inst.costs, inst.alpha, q, 40)
        got = item.state()
        for k in ("u", "qx", "qy", "p", "ps"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-4, (inst.W, k)


@pytest.mark.parametrize("algo", [2, 3])
def test_batch_host_driven_loop_equals_graph(cmf, algo):
    """use_graph = 0 runs the batch's chunks host-driven: the same kernels in
    the same order, so the same iteration counts, certificates and states bit
    for bit as the device-driven graph."""
    insts = _instances() + [synth.potts_shapes(45, 61, 4, seed=114)]
    out = []
    for g in (1, 0):
        p = cmf.default_params(algo, 2, tol_gap=1e-4, max_iter=20000, check_every=10,
                               use_graph=g)
        items = [_alloc(cmf, i, p) for i in insts]
        status, res = cmf.cmf_solve_batch(items, p)
        assert status == cmf.OK, res
        out.append((res, [it.state() for it in items]))
    (r1, s1), (r0, s0) = out
    for a, b in zip(r1, r0):
        assert a["iters"] == b["iters"] and a["gap"] == b["gap"], (a, b)
    for a, b in zip(s1, s0):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("algo", [0, 2])
def test_batch_strip_odd_widths_ignore_the_padding_column(cmf, algo):
    """The padding column next to an odd width is read by the strip kernel's
    last pair but must not reach the grid: with NaN in every padding column
    of the costs, alpha and the caller's state, the batch still matches the
    FP64 oracle element by element and its certificates stay finite."""
    insts = [synth.potts_shapes(37, 71, 3, seed=111), synth.config5(33, 181)]
    kw = dict(tol_gap=0.0, max_iter=40, check_every=10)
    p = cmf.default_params(algo, 2, **kw)
    items = [cmf.alloc_potts(i, p) for i in insts]
    nan = float("nan")
    for it in items:
        assert it.W % 2 == 1 and it.pitch > it.W
        for t in (it.C, it.u, it.qx, it.qy, it.p, it.ps):
            t[..., it.W:] = nan
        if isinstance(it.alpha, torch.Tensor):
            it.alpha[..., it.W:] = nan
    status, res = cmf.cmf_solve_batch(items, p)
    assert status == cmf.NOT_CONVERGED and all(r["iters"] == 40 for r in res)
    assert all(np.isfinite(r["gap"]) for r in res), res
    for inst, item in zip(insts, items):
        q = O.default_params(algo, inst.L, a2=max(p.a2, 2.0 * inst.L))
        ref = O.potts_run(inst.costs, inst.alpha, q, 40)
        got = item.state()
        for k in ("u", "qx", "qy", "p", "ps"):
            assert np.abs(got[k] - ref[k]).max() <= 1e-4, (inst.W, k)


def test_batch_alg1_takes_each_instances_step_bound(cmf):
    """ALG1 without a hand-set tau: every instance of the batch runs with
    tau = min(p.tau, 1 / (bound(L) sigma)), the bound cmf_default_params takes
    for its label count, so it matches a single solve with its own defaults."""
    insts = _instances()
    kw = dict(tol_gap=1e-4, max_iter=20000, check_every=10, variant=1)
    p = cmf.default_params(5, 2, **kw)
    items = [_alloc(cmf, i, p) for i in insts]
    status, res = cmf.cmf_solve_batch(items, p)
    assert status == cmf.OK, res
    for inst, item, r in zip(insts, items, res):
        q = cmf.default_params(5, inst.L, **kw)
        q.a2 = max(p.a2, 2.0 * inst.L)
        assert q.tau == min(p.tau, 1.0 / ((10 if inst.L == 2 else 9 + inst.L) * q.sigma))
        if inst.kind == "potts" and inst.W % 2 == 0:
            q.variant = 2  # the batch runs this instance by warp strips
        single = _alloc(cmf, inst, q)
        if inst.kind == "binary":
            st, it, hist = cmf.cmf_solve_binary(single)
        else:
            st, it, hist = cmf.cmf_solve_potts(single)
        assert st == cmf.OK and it == r["iters"], (inst.kind, it, r["iters"])
        a, b = item.state(), single.state()
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= 1e-5, k


def test_batch_rows_give_the_same_solution(cmf):
    """params.batch_rows changes only how the strip instances are cut into
    work items: the same iterations and states bit for bit."""
    insts = [synth.potts_shapes(120, 88, 8, seed=104), synth.potts_shapes(67, 71, 3, seed=102),
             synth.binary_shapes(40, 50, seed=106)]
    out = []
    for rows in (24, 12, 8):
        p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=20000, check_every=10,
                               batch_rows=rows)
        items = [_alloc(cmf, i, p) for i in insts]
        status, res = cmf.cmf_solve_batch(items, p)
        assert status == cmf.OK, res
        out.append(([r["iters"] for r in res], [it.state() for it in items]))
    for iters, states in out[1:]:
        assert iters == out[0][0]
        for a, b in zip(states, out[0][1]):
            for k in a:
                assert np.array_equal(a[k], b[k]), k


def test_batch_autotune(cmf):
    """cmf_autotune_batch times the batch over check intervals and strip band
    heights and returns one whose instances all converge; solved with it,
    every instance is certified by the oracle."""
    insts = _instances()
    p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=20000, check_every=10)
    items = [_alloc(cmf, i, p) for i in insts]
    best, ms = cmf.cmf_autotune_batch(items, p)
    assert ms > 0 and best.check_every in (10, 20, 50) and best.batch_rows in (12, 16, 24)
    items = [_alloc(cmf, i, best) for i in insts]
    status, res = cmf.cmf_solve_batch(items, best)
    assert status == cmf.OK, res
    for inst, item in zip(insts, items):
        po = O.default_params(2, inst.L, a2=max(best.a2, 2.0 * inst.L))
        if inst.kind == "binary":
            gap = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, item.state(), po)[2]
        else:
            gap = O.potts_eval(inst.costs, inst.alpha, item.state(), po)[2]
        assert gap <= 1.01e-4
