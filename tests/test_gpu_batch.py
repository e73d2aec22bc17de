"""Batched solve (many instances of uneven size and label count in one
device-driven loop) against the single-instance solver run with the same
shared-memory tile kernels: identical iteration counts and states within
float32 rounding, each instance certified by the FP64 oracle."""
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
