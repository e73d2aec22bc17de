"""Reuse of the instantiated solve graphs (cmf_solve_* with use_graph = 1):
a replay gives what a freshly built graph and the host-driven loop give, for
repeated calls, alternating problems, changed parameters, warm starts,
relaxation schedules and after cmf_release_graphs."""
import numpy as np
import pytest
import torch

from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _solve(cmf, b):
    st, it, hist = cmf.cmf_solve_binary(b)
    return st, it, hist.copy(), b.state()


def _same(r1, r2):
    assert r1[0] == r2[0] and r1[1] == r2[1]
    np.testing.assert_array_equal(r1[2], r2[2])
    for k in r1[3]:
        np.testing.assert_array_equal(r1[3][k], r2[3][k])


@pytest.mark.parametrize("algo", [2, 3])
def test_repeated_solves_replay_the_graph(cmf, algo):
    cmf.cmf_release_graphs()
    inst = synth.config2(96, 128)
    p = cmf.default_params(algo, 2, tol_gap=1e-4, max_iter=4000, check_every=10)
    b = cmf.alloc_binary(inst, p)
    first = _solve(cmf, b)
    for _ in range(3):
        _same(first, _solve(cmf, b))
    q = cmf.default_params(algo, 2, tol_gap=1e-4, max_iter=4000, check_every=10, use_graph=0)
    h = cmf.alloc_binary(inst, q)
    _same(first, _solve(cmf, h))


def test_alternating_problems_and_parameters(cmf):
    cmf.cmf_release_graphs()
    a_inst, b_inst = synth.config2(64, 80, seed=12), synth.config2(72, 64, seed=13)
    pa = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=4000, check_every=10)
    pb = cmf.default_params(2, 2, tol_gap=1e-6, max_iter=4000, check_every=10)
    A, B = cmf.alloc_binary(a_inst, pa), cmf.alloc_binary(b_inst, pb)
    ra, rb = _solve(cmf, A), _solve(cmf, B)
    for _ in range(2):
        _same(ra, _solve(cmf, A))
        _same(rb, _solve(cmf, B))
    # a changed parameter is a new signature: the same buffers, a tighter gap
    A.params.tol_gap = 1e-6
    rt = _solve(cmf, A)
    assert rt[1] > ra[1] and rt[2][-1, 3] <= 1e-6
    A.params.tol_gap = 1e-4
    _same(ra, _solve(cmf, A))
    # more signatures than the cache keeps: evictions, results unchanged (check
    # intervals >= 10 keep the history within the workspace sized for 10)
    for ce in (12, 14, 16, 18, 20, 22, 24, 26, 28):
        A.params.check_every = ce
        st, it, hist = cmf.cmf_solve_binary(A)
        assert st == cmf.OK and it % ce == 0
    A.params.check_every = 10
    _same(ra, _solve(cmf, A))
    cmf.cmf_release_graphs()
    _same(rb, _solve(cmf, B))


def test_warm_start_and_schedule_with_a_kept_graph(cmf):
    cmf.cmf_release_graphs()
    inst = synth.config2(80, 96)
    out = []
    for use_graph in (1, 0):
        p = cmf.default_params(2, 2, tol_gap=1e-3, max_iter=4000, check_every=10,
                               use_graph=use_graph, rho_schedule=np.linspace(0.8, 1.9, 15))
        b = cmf.alloc_binary(inst, p)
        r1 = _solve(cmf, b)
        b.params.warm_start = 1
        b.params.tol_gap = 1e-5
        r2 = _solve(cmf, b)
        r3 = _solve(cmf, b)  # warm again: the graph of r2 is replayed
        out.append((r1, r2, r3))
    for g, h in zip(out[0], out[1]):
        _same(g, h)


def test_potts_repeated_solves(cmf):
    cmf.cmf_release_graphs()
    inst = synth.config3(64, 64)
    p = cmf.default_params(2, 4, tol_gap=1e-4, max_iter=4000, check_every=10)
    s = cmf.alloc_potts(inst, p)
    runs = []
    for _ in range(3):
        st, it, hist = cmf.cmf_solve_potts(s)
        runs.append((st, it, hist.copy(), s.state()))
    for r in runs[1:]:
        _same(runs[0], r)


@pytest.mark.parametrize("check_every,max_iter", [(10, 4000), (9, 3996), (7, 3997), (5, 4000),
                                                  (10, 30), (10, 40), (3, 30), (2, 4000)])
@pytest.mark.parametrize("model", ["binary", "binary_single", "potts"])
def test_graph_body_shapes_equal_host_loop(cmf, model, check_every, max_iter):
    """Chunks that end in the workspace buffers (an odd number of launches:
    5 pairs, or 4 pairs and a single, or an odd count of single launches)
    make the loop body two chunks with the second under an IF node; solves
    that stop after either half, or at max_iter, equal the host loop."""
    out = []
    tol = 1e-9 if max_iter < 100 else 1e-4  # the short runs stop at max_iter
    for use_graph in (1, 0):
        if model == "potts":
            inst = synth.config3(48, 64)
            p = cmf.default_params(2, 4, tol_gap=tol, max_iter=max_iter,
                                   check_every=check_every, use_graph=use_graph)
            s = cmf.alloc_potts(inst, p)
            st, it, hist = cmf.cmf_solve_potts(s)
            out.append((st, it, hist.copy(), s.state()))
        else:
            inst = synth.config2(80, 112)
            p = cmf.default_params(2, 2, tol_gap=tol, max_iter=max_iter,
                                   check_every=check_every, use_graph=use_graph,
                                   variant=2 if model == "binary_single" else 0)
            b = cmf.alloc_binary(inst, p)
            out.append(_solve(cmf, b))
    _same(out[0], out[1])
    if max_iter < 100:
        assert out[0][0] == cmf.NOT_CONVERGED and out[0][1] == max_iter
