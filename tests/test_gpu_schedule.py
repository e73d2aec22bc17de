"""GPU parity of relaxation schedules {rho_k} (rpADMMII, rPDRQ; Thm 1 and
Thm 2 take them non-decreasing in (0, 2)) against the FP64 oracle run with the
same schedule, in every kernel family (warp strips, shared-memory tiles, TMA
tiles, the plain form); and the solve driver: the scheduled iterations run
host-driven, the rest in the device-driven graph, with the same iterations,
history and state as an all-host loop.  Tolerances as for constant rho."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_U = 1e-4
SCHED = np.linspace(0.5, 1.8, 23)


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _close(got, ref, keys):
    for k in keys:
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


# kernel family -> params: 0 = automatic (warp strips on an even width),
# 1 = shared-memory tiles, 16 = TMA tiles (ADMM only), plain form
FAMILIES = {"auto": dict(variant=0), "tiles": dict(variant=1), "tma": dict(variant=16),
            "plain": dict(impl=1)}


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("algo", [2, 3])
@pytest.mark.parametrize("shape", [(48, 64), (37, 53)])
def test_binary_schedule_matches_oracle(cmf, algo, family, shape):
    if family == "tma" and algo == 3:
        pytest.skip("rPDRQ has no TMA kernel")
    inst = synth.config2(*shape)
    n = 40  # 23 scheduled iterations, 17 at rho
    p = cmf.default_params(algo, 2, rho_schedule=SCHED, **FAMILIES[family])
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, n)
    torch.cuda.synchronize()
    ref = O.binary_run(inst.costs[0], inst.costs[1], inst.alpha, O.default_params(algo, 2), n,
                       rho_schedule=SCHED)
    _close(b.state(), ref, ("u", "qx", "qy", "ps", "pt"))
    # the schedule matters: the constant-rho run differs
    const = O.binary_run(inst.costs[0], inst.costs[1], inst.alpha, O.default_params(algo, 2), n)
    assert np.abs(const["u"] - ref["u"]).max() > 100 * TOL_U


@pytest.mark.parametrize("family", list(FAMILIES))
@pytest.mark.parametrize("algo", [2, 3])
@pytest.mark.parametrize("inst_name", ["voronoi4_40x64", "L5_ragged_33x35"])
def test_potts_schedule_matches_oracle(cmf, algo, family, inst_name):
    if family == "tma" and algo == 3:
        pytest.skip("rPDRQ has no TMA kernel")
    inst = (synth.config3(40, 64) if inst_name == "voronoi4_40x64" else
            synth.random_potts(33, 35, 5, seed=24, alpha=0.25, field_alpha=True))
    n = 30
    p = cmf.default_params(algo, inst.L, rho_schedule=SCHED, **FAMILIES[family])
    s = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(s)
    cmf.cmf_iterate_potts(s, n)
    torch.cuda.synchronize()
    ref = O.potts_run(inst.costs, inst.alpha, O.default_params(algo, inst.L), n,
                      rho_schedule=SCHED)
    _close(s.state(), ref, ("u", "qx", "qy", "p", "ps"))


@pytest.mark.parametrize("algo", [2, 3])
@pytest.mark.parametrize("sched_len", [20, 25, 400])
def test_scheduled_solve_graph_equals_host_loop(cmf, algo, sched_len):
    """Schedules that end on a check, between checks, and past max_iter."""
    inst = synth.config2(80, 112)
    sched = np.linspace(0.6, 1.9, sched_len)
    out = []
    for use_graph in (1, 0):
        p = cmf.default_params(algo, 2, use_graph=use_graph, tol_gap=1e-4, max_iter=300,
                               check_every=10, rho_schedule=sched)
        b = cmf.alloc_binary(inst, p)
        out.append((cmf.cmf_solve_binary(b), b.state()))
    (s1, i1, h1), st1 = out[0]
    (s0, i0, h0), st0 = out[1]
    assert s1 == s0 and i1 == i0
    np.testing.assert_array_equal(h1, h0)
    assert h1[len(h1) - 1, 0] == i1 and np.all(np.diff(h1[:, 0]) == 10)
    for k in st0:
        np.testing.assert_array_equal(st1[k], st0[k])


def test_scheduled_potts_solve_certified(cmf):
    inst = synth.config3(64, 64)
    sched = np.linspace(0.5, 1.9, 60)
    out = []
    for use_graph in (1, 0):
        p = cmf.default_params(2, 4, use_graph=use_graph, tol_gap=1e-4, max_iter=4000,
                               check_every=10, rho_schedule=sched)
        s = cmf.alloc_potts(inst, p)
        st, it, hist = cmf.cmf_solve_potts(s)
        assert st == cmf.OK
        out.append((it, hist, s.state()))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    # certified by the oracle on the returned state
    E, D, gap, _ = O.potts_eval(inst.costs, inst.alpha, out[0][2], O.default_params(2, 4))
    assert gap <= 2e-4, gap
