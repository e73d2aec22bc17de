"""Pins of the oracle's relaxed iterations with a relaxation sequence {rho_k}
(Eq. update:two:sun:lag and Eq. rpADMMII take rho_k per iteration; Thm 1 and
Thm 2 assume {rho_k} non-decreasing in (0, 2)):

* the iterations are a map of the stored state alone, so n single iterations
  equal one call of n iterations (a schedule is then well defined);
* rho_k = 1 turns rpADMMII into pADMMI (no relaxation), so a schedule that
  starts with ones follows pADMMI exactly for that many iterations and
  rpADMMII(rho) from there, which also fixes that iteration k takes rho_k;
* a non-decreasing ramp converges (Thm 1, Thm 2) to the same optimal value as
  the constant rho."""
import numpy as np
import pytest

from paper_2004_11227_gb300 import synth


@pytest.mark.parametrize("algo", [2, 3])
def test_single_iterations_equal_one_call(orc, algo):
    inst = synth.config2(24, 30)
    Cs, Ct = inst.costs
    p = orc.default_params(algo, 2)
    whole = orc.binary_run(Cs, Ct, inst.alpha, p, 12)
    st = orc.binary_run(Cs, Ct, inst.alpha, p, 1)
    for _ in range(11):
        st = orc.binary_run(Cs, Ct, inst.alpha, p, 1, st)
    for k in whole:
        np.testing.assert_array_equal(whole[k], st[k])
    pot = synth.config3(14, 18)
    p = orc.default_params(algo, 4)
    whole = orc.potts_run(pot.costs, pot.alpha, p, 9)
    st = orc.potts_run(pot.costs, pot.alpha, p, 4)
    st = orc.potts_run(pot.costs, pot.alpha, p, 5, st)
    for k in whole:
        np.testing.assert_array_equal(whole[k], st[k])


def test_unit_prefix_follows_padmm_then_rpadmm(orc):
    inst = synth.config2(32, 40)
    Cs, Ct = inst.costs
    n, m = 17, 13
    eb = orc.default_params(2, 2)  # rho = 1.9 after the schedule
    got = orc.binary_run(Cs, Ct, inst.alpha, eb, n + m, rho_schedule=[1.0] * n)
    ref = orc.binary_run(Cs, Ct, inst.alpha, orc.default_params(0, 2), n)
    ref = orc.binary_run(Cs, Ct, inst.alpha, eb, m, ref)
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k])
    # one iteration more or less at rho = 1 gives a different state
    off = orc.binary_run(Cs, Ct, inst.alpha, eb, n + m, rho_schedule=[1.0] * (n + 1))
    assert np.abs(off["u"] - got["u"]).max() > 1e-6
    pot = synth.config3(20, 24)
    eb4 = orc.default_params(2, 4)
    got = orc.potts_run(pot.costs, pot.alpha, eb4, n + m, rho_schedule=[1.0] * n)
    ref = orc.potts_run(pot.costs, pot.alpha, orc.default_params(0, 4), n)
    ref = orc.potts_run(pot.costs, pot.alpha, eb4, m, ref)
    for k in ref:  # pADMMI and rpADMMII(rho = 1) associate the Potts sums differently
        np.testing.assert_allclose(got[k], ref[k], atol=1e-12, rtol=0)


def test_k0_offsets_the_schedule(orc):
    """A run split at iteration j with k0 = j equals the unsplit run."""
    inst = synth.config2(20, 26)
    Cs, Ct = inst.costs
    sched = np.linspace(0.6, 1.8, 25)
    p = orc.default_params(3, 2)
    whole = orc.binary_run(Cs, Ct, inst.alpha, p, 40, rho_schedule=sched)
    st = orc.binary_run(Cs, Ct, inst.alpha, p, 11, rho_schedule=sched)
    st = orc.binary_run(Cs, Ct, inst.alpha, p, 29, st, rho_schedule=sched, k0=11)
    for k in whole:
        np.testing.assert_array_equal(whole[k], st[k])


@pytest.mark.parametrize("kind,algo", [("binary", 2), ("binary", 3), ("potts", 2),
                                       ("potts", 3)])
def test_ramp_converges_to_the_same_value(orc, kind, algo):
    inst = synth.config2(28, 34) if kind == "binary" else synth.config3(22, 26)
    ramp = np.linspace(0.3, 1.9, 120)
    tol = 1e-9 if kind == "binary" else 1e-6
    out = []
    for sched in (None, ramp):
        p = orc.default_params(algo, inst.L)
        st, it, hist = orc.solve(inst, algo, tol=tol, max_iter=60000, check_every=20,
                                 params=p, rho_schedule=sched)
        assert hist[-1][3] <= tol, (sched is None, hist[-1])
        out.append(hist[-1][1])
    # weak duality: D <= E* <= E and E - D <= tol E, so each E is within tol E of E*
    assert abs(out[0] - out[1]) <= 1.001 * tol * max(out)
