"""Pins of the oracle's iterations against what the paper and the mathematics
fix: the alpha = 0 solution, strong duality at convergence (Eq. two-label-mf /
Eq. potts-mf vs their primal models), exactness of thresholding for the
anisotropic relaxation (brute force and an independent LP solver), weak
duality for arbitrary states, the Potts L = 2 / binary equivalence, the
rpADMMII(rho = 1) = rpADMMI(r = 1) identity, and grid symmetries."""
import itertools

import numpy as np
import pytest

from paper_2004_11227_gb300 import synth

ALGOS = [0, 1, 2, 3, 4, 5]


def _converge(orc, inst, algo, tol, max_iter=40000, **kw):
    p = orc.default_params(algo, inst.L, **kw)
    st, it, hist = orc.solve(inst, algo, tol=tol, max_iter=max_iter, check_every=20, params=p)
    assert hist[-1][3] <= tol, (algo, hist[-1])
    return st, hist[-1], p


# --- alpha = 0: pointwise argmin --------------------------------------------------

@pytest.mark.parametrize("algo", ALGOS)
def test_alpha_zero_binary_is_pointwise_argmin(orc, algo):
    inst = synth.random_binary(9, 7, seed=11, alpha=0.0)
    Cs, Ct = inst.costs
    p = orc.default_params(algo, 2)
    # warm start far from the answer: u = 1/2, zero flows
    st = {"u": np.full((9, 7), 0.5), "qx": np.zeros((9, 7)), "qy": np.zeros((9, 7)),
          "ps": np.zeros((9, 7)), "pt": np.zeros((9, 7))}
    for _ in range(100):
        st = orc.binary_run(Cs, Ct, 0.0, p, 20, st)
        if orc.binary_eval(Cs, Ct, 0.0, st, p)[2] < 1e-10:
            break
    np.testing.assert_array_equal(orc.binary_labels(st["u"]), (Ct < Cs).astype(np.uint8))
    assert np.abs(st["qx"]).max() == 0.0 and np.abs(st["qy"]).max() == 0.0 or algo == 3
    E, D, gap, res = orc.binary_eval(Cs, Ct, 0.0, st, p)
    assert abs(E - np.minimum(Cs, Ct).astype(np.float64).sum()) < 1e-8


@pytest.mark.parametrize("algo", ALGOS)
def test_alpha_zero_potts_is_pointwise_argmin(orc, algo):
    inst = synth.random_potts(6, 8, 4, seed=12, alpha=0.0)
    C = inst.costs
    p = orc.default_params(algo, 4)
    L, H, W = C.shape
    st = {"u": np.full((L, H, W), 1.0 / L), "qx": np.zeros((L, H, W)),
          "qy": np.zeros((L, H, W)), "p": np.zeros((L, H, W)), "ps": np.zeros((H, W))}
    for _ in range(200):
        st = orc.potts_run(C, 0.0, p, 20, st)
        if orc.potts_eval(C, 0.0, st, p)[2] < 1e-10:
            break
    np.testing.assert_array_equal(orc.potts_labels(st["u"]), np.argmin(C, axis=0))
    E = orc.potts_eval(C, 0.0, st, p)[0]
    assert abs(E - C.astype(np.float64).min(axis=0).sum()) < 1e-8


def test_cold_start_is_alpha_zero_fixed_point(orc):
    inst = synth.random_binary(5, 6, seed=13, alpha=0.0)
    for algo in ALGOS:
        p = orc.default_params(algo, 2)
        st = orc.binary_run(inst.costs[0], inst.costs[1], 0.0, p, 3)
        np.testing.assert_allclose(st["u"], (inst.costs[1] < inst.costs[0]).astype(float),
                                   atol=1e-12)


# --- strong duality ---------------------------------------------------------------

def test_strong_duality_binary_all_algorithms_config1(orc):
    inst = synth.config1()
    Es = []
    for algo in ALGOS:
        st, (it, E, D, gap, res), p = _converge(orc, inst, algo, tol=1e-10)
        assert res < 1e-3, (algo, res)
        Es.append(E)
    assert (max(Es) - min(Es)) / min(Es) < 1e-8


def test_strong_duality_potts_all_algorithms(orc):
    inst = synth.config3(16, 14)
    Es = []
    for algo in ALGOS:
        st, (it, E, D, gap, res), p = _converge(orc, inst, algo, tol=1e-7, max_iter=80000)
        Es.append(E)
    assert (max(Es) - min(Es)) / min(Es) < 2e-7


def test_conservation_residual_vanishes(orc):
    """Flow conservation div q - p_s + p_t = 0 holds at the limit."""
    inst = synth.config1()
    p = orc.default_params(2, 2)
    st = orc.binary_run(inst.costs[0], inst.costs[1], inst.alpha, p, 500)
    res0 = orc.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st, p)[3]
    st = orc.binary_run(inst.costs[0], inst.costs[1], inst.alpha, p, 7500, st)
    E, D, gap, res = orc.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st, p)
    assert res < res0 / 50 and gap < 1e-8


# --- weak duality for arbitrary states ----------------------------------------------

def test_weak_duality_random_states(orc):
    rng = np.random.default_rng(5)
    inst = synth.random_binary(7, 9, seed=14, alpha=0.4, field_alpha=True)
    Cs, Ct = inst.costs
    for algo in [0, 3]:
        p = orc.default_params(algo, 2)
        for _ in range(20):
            st = {k: rng.normal(size=(7, 9)) for k in ("u", "qx", "qy", "ps", "pt")}
            E, D, gap, res = orc.binary_eval(Cs, Ct, inst.alpha, st, p)
            assert E >= D - 1e-12
    instp = synth.random_potts(5, 6, 3, seed=15, alpha=0.3, field_alpha=True)
    for algo in [0, 3]:
        p = orc.default_params(algo, 3)
        for _ in range(20):
            st = {k: rng.normal(size=(3, 5, 6)) for k in ("u", "qx", "qy", "p")}
            st["ps"] = rng.normal(size=(5, 6))
            E, D, gap, res = orc.potts_eval(instp.costs, instp.alpha, st, p)
            assert E >= D - 1e-12


# --- exactness of thresholding (anisotropic TV) --------------------------------------

def _binary_aniso_energy_all(Cs, Ct, al):
    """Energy of every labelling u in {0,1}^(H x W) (rows of the result)."""
    H, W = Cs.shape
    N = H * W
    U = ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.float64)
    U = U.reshape(-1, H, W)
    data = ((1 - U) * Cs + U * Ct).reshape(len(U), -1).sum(1)
    tv = (al[:, :-1] * np.abs(U[:, :, 1:] - U[:, :, :-1])).reshape(len(U), -1).sum(1)
    tv += (al[:-1, :] * np.abs(U[:, 1:, :] - U[:, :-1, :])).reshape(len(U), -1).sum(1)
    return data + tv, U


@pytest.mark.parametrize("H,W,seed", [(4, 4, 21), (3, 4, 22), (4, 4, 23)])
@pytest.mark.parametrize("algo", ALGOS)
def test_brute_force_binary_anisotropic(orc, H, W, seed, algo):
    inst = synth.random_binary(H, W, seed=seed, alpha=0.35, field_alpha=True)
    Cs, Ct = inst.costs.astype(np.float64)
    al = inst.alpha.astype(np.float64)
    energies, U = _binary_aniso_energy_all(Cs, Ct, al)
    emin = energies.min()
    st, (it, E, D, gap, res), p = _converge(orc, inst, algo, tol=1e-11, aniso=1)
    assert abs(E - emin) <= 1e-8 * max(1.0, emin)
    assert abs(D - emin) <= 1e-8 * max(1.0, emin)
    lab = orc.binary_labels(st["u"]).astype(np.float64)
    e_lab = ((1 - lab) * Cs + lab * Ct).sum() + (al[:, :-1] * np.abs(np.diff(lab, axis=1))).sum() \
        + (al[:-1, :] * np.abs(np.diff(lab, axis=0))).sum()
    assert abs(e_lab - emin) <= 1e-8 * max(1.0, emin)


def _lp_binary_aniso(Cs, Ct, al):
    """min sum (1-u) Cs + u Ct + sum al (t1 + t2), t >= |forward differences|,
    0 <= u <= 1, by scipy's HiGHS LP solver."""
    from scipy.optimize import linprog
    from scipy.sparse import lil_matrix

    H, W = Cs.shape
    N = H * W
    idx = np.arange(N).reshape(H, W)
    pairs = [(idx[i, j], idx[i, j + 1]) for i in range(H) for j in range(W - 1)] + \
            [(idx[i, j], idx[i + 1, j]) for i in range(H - 1) for j in range(W)]
    wts = [al[i, j] for i in range(H) for j in range(W - 1)] + \
          [al[i, j] for i in range(H - 1) for j in range(W)]
    nP = len(pairs)
    cvec = np.concatenate([(Ct - Cs).ravel(), np.asarray(wts)])
    A = lil_matrix((2 * nP, N + nP))
    for k, (x, y) in enumerate(pairs):
        A[2 * k, y], A[2 * k, x], A[2 * k, N + k] = 1, -1, -1
        A[2 * k + 1, y], A[2 * k + 1, x], A[2 * k + 1, N + k] = -1, 1, -1
    res = linprog(cvec, A_ub=A.tocsr(), b_ub=np.zeros(2 * nP),
                  bounds=[(0, 1)] * N + [(0, None)] * nP, method="highs")
    assert res.status == 0
    return res.fun + Cs.sum()


def test_lp_binary_anisotropic_8x8(orc):
    pytest.importorskip("scipy")
    inst = synth.random_binary(8, 8, seed=31, alpha=0.3, field_alpha=True)
    Cs, Ct = inst.costs.astype(np.float64)
    e_lp = _lp_binary_aniso(Cs, Ct, inst.alpha.astype(np.float64))
    for algo in ALGOS:
        st, (it, E, D, gap, res), p = _converge(orc, inst, algo, tol=1e-11, aniso=1)
        assert abs(E - e_lp) <= 1e-7 * e_lp, (algo, E, e_lp)


def test_brute_force_potts_relaxation_bound(orc):
    """Potts L = 3 on 3x3 (3^9 labellings): relaxed optimum <= integer optimum."""
    inst = synth.random_potts(3, 3, 3, seed=41, alpha=0.25)
    C = inst.costs.astype(np.float64)
    L, H, W = C.shape
    best = np.inf
    for lab in itertools.product(range(L), repeat=H * W):
        lab = np.asarray(lab).reshape(H, W)
        U = np.stack([(lab == i).astype(float) for i in range(L)])
        e = (U * C).sum()
        for i in range(L):
            gx = np.zeros((H, W))
            gy = np.zeros((H, W))
            gx[:, :-1] = U[i][:, 1:] - U[i][:, :-1]
            gy[:-1, :] = U[i][1:, :] - U[i][:-1, :]
            e += 0.25 * np.sqrt(gx ** 2 + gy ** 2).sum()
        best = min(best, e)
    for algo in ALGOS:
        st, (it, E, D, gap, res), p = _converge(orc, inst, algo, tol=1e-10)
        assert E <= best + 1e-9
        assert E >= 0.9 * best  # the relaxation is not loose on this instance


# --- equivalences -------------------------------------------------------------------

def test_potts_two_labels_equals_binary_double_alpha(orc):
    """TV(u_1) + TV(1 - u_1) = 2 TV(u_1): Potts L = 2 with weight alpha has the
    optimum of the binary model with weight 2 alpha (C_s = C_1, C_t = C_2)."""
    pot = synth.random_potts(12, 10, 2, seed=51, alpha=0.2, field_alpha=True)
    binst = synth.Instance("binary", pot.image, pot.costs.copy(),
                           (2.0 * pot.alpha.astype(np.float64)))
    _, (_, Ep, _, _, _), _ = _converge(orc, pot, 2, tol=1e-11, max_iter=80000)
    st, (_, Eb, _, _, _), _ = _converge(orc, binst, 2, tol=1e-11, max_iter=80000)
    assert abs(Ep - Eb) <= 1e-8 * Eb


def test_eb_rho1_equals_fg_r1_equals_padmm(orc):
    inst = synth.config2(32, 40)
    Cs, Ct = inst.costs
    pa = orc.binary_run(Cs, Ct, inst.alpha, orc.default_params(0, 2), 50)
    fg = orc.binary_run(Cs, Ct, inst.alpha, orc.default_params(1, 2, r=1.0), 50)
    eb = orc.binary_run(Cs, Ct, inst.alpha, orc.default_params(2, 2, rho=1.0), 50)
    for k in pa:
        np.testing.assert_array_equal(pa[k], fg[k])
        np.testing.assert_array_equal(pa[k], eb[k])
    pot = synth.config3(20, 24)
    pa = orc.potts_run(pot.costs, pot.alpha, orc.default_params(0, 4), 50)
    fg = orc.potts_run(pot.costs, pot.alpha, orc.default_params(1, 4, r=1.0), 50)
    eb = orc.potts_run(pot.costs, pot.alpha, orc.default_params(2, 4, rho=1.0), 50)
    lit = orc.potts_run(pot.costs, pot.alpha, orc.default_params(2, 4, rho=1.0,
                                                                 literal_potts_u=1), 50)
    for k in pa:  # the paper's Potts formulas associate the sums differently
        np.testing.assert_array_equal(pa[k], fg[k])
        np.testing.assert_allclose(pa[k], eb[k], atol=1e-13, rtol=0)
        np.testing.assert_array_equal(eb[k], lit[k])


# --- symmetries ---------------------------------------------------------------------

@pytest.mark.parametrize("algo", ALGOS)
def test_transpose_symmetry_binary(orc, algo):
    inst = synth.random_binary(7, 11, seed=61, alpha=0.4, field_alpha=True)
    Cs, Ct = inst.costs
    p = orc.default_params(algo, 2)
    a = orc.binary_run(Cs, Ct, inst.alpha, p, 30)
    b = orc.binary_run(Cs.T, Ct.T, inst.alpha.T, p, 30)
    np.testing.assert_allclose(b["u"], a["u"].T, atol=1e-12)
    np.testing.assert_allclose(b["qx"], a["qy"].T, atol=1e-12)
    np.testing.assert_allclose(b["qy"], a["qx"].T, atol=1e-12)
    np.testing.assert_allclose(b["ps"], a["ps"].T, atol=1e-12)


@pytest.mark.parametrize("algo", ALGOS)
def test_label_permutation_potts(orc, algo):
    inst = synth.random_potts(6, 7, 4, seed=62, alpha=0.3, field_alpha=True)
    perm = np.array([2, 0, 3, 1])
    p = orc.default_params(algo, 4)
    a = orc.potts_run(inst.costs, inst.alpha, p, 30)
    b = orc.potts_run(inst.costs[perm], inst.alpha, p, 30)
    for k in ("u", "qx", "qy", "p"):
        np.testing.assert_allclose(b[k], a[k][perm], atol=1e-12)
    np.testing.assert_allclose(b["ps"], a["ps"], atol=1e-12)


def test_ty_p_steps_maximise_the_augmented_lagrangian(orc):
    """pADMM-TY (Eq. ADMM:Tai_yuan, Remark 1): p_s^{k+1} maximises the
    augmented Lagrangian of Eq. augfunc:twolabel over p_s <= C_s with p_t^k,
    q^{k+1}, u^k fixed; then p_t^{k+1} maximises it over p_t <= C_t with
    p_s^{k+1}; then u^{k+1} = u^k - c (p_t - p_s + div q)^{k+1}.  Checked per
    pixel with a bounded scalar optimiser on the Lagrangian as written."""
    from scipy.optimize import minimize_scalar

    rng = np.random.default_rng(7)
    inst = synth.random_binary(4, 5, seed=71, alpha=0.4)
    Cs, Ct = inst.costs.astype(np.float64)
    p = orc.default_params(orc.TY, 2)
    c = p.c
    st0 = {k: rng.normal(scale=0.3, size=(4, 5)) for k in ("u", "qx", "qy", "ps", "pt")}
    st1 = orc.binary_run(Cs, Ct, inst.alpha, p, 1, st0)
    d = orc.div(st1["qx"], st1["qy"])
    for i in range(4):
        for j in range(5):
            u0, pt0 = st0["u"][i, j], st0["pt"][i, j]

            def neg_ps(ps):  # -(p_s + u (p_t - p_s + div q) - c/2 (p_t - p_s + div q)^2)
                r = pt0 - ps + d[i, j]
                return -(ps + u0 * r - 0.5 * c * r * r)
            ps_best = minimize_scalar(neg_ps, bounds=(-50, Cs[i, j]), method="bounded",
                                      options={"xatol": 1e-12}).x
            assert abs(st1["ps"][i, j] - ps_best) < 1e-6
            ps1 = st1["ps"][i, j]

            def neg_pt(pt):
                r = pt - ps1 + d[i, j]
                return -(u0 * r - 0.5 * c * r * r)
            pt_best = minimize_scalar(neg_pt, bounds=(-50, Ct[i, j]), method="bounded",
                                      options={"xatol": 1e-12}).x
            assert abs(st1["pt"][i, j] - pt_best) < 1e-6
            u1 = u0 - c * (st1["pt"][i, j] - ps1 + d[i, j])
            assert abs(st1["u"][i, j] - u1) < 1e-12


def test_ty_potts_p_steps_maximise_the_augmented_lagrangian(orc):
    """Potts pADMM-TY (Eq. mADMM:Tai_yuan, with Eq. multi:aug:func): each p_i
    maximises over p_i <= C_i with p_s^k, then p_s maximises over p_s with
    the new p_i (the sequential order described after the equation)."""
    from scipy.optimize import minimize_scalar

    rng = np.random.default_rng(8)
    L = 3
    inst = synth.random_potts(3, 4, L, seed=72, alpha=0.3)
    C = inst.costs.astype(np.float64)
    p = orc.default_params(orc.TY, L)
    c = p.c
    st0 = {k: rng.normal(scale=0.3, size=(L, 3, 4)) for k in ("u", "qx", "qy", "p")}
    st0["ps"] = rng.normal(scale=0.3, size=(3, 4))
    st1 = orc.potts_run(C, inst.alpha, p, 1, st0)
    d = np.stack([orc.div(st1["qx"][i], st1["qy"][i]) for i in range(L)])
    for y in range(3):
        for x in range(4):
            ps0 = st0["ps"][y, x]
            for i in range(L):
                u0 = st0["u"][i, y, x]

                def neg_pi(pi):
                    r = d[i, y, x] + pi - ps0
                    return -(u0 * r - 0.5 * c * r * r)
                best = minimize_scalar(neg_pi, bounds=(-50, C[i, y, x]), method="bounded",
                                       options={"xatol": 1e-12}).x
                assert abs(st1["p"][i, y, x] - best) < 1e-6

            def neg_ps(ps):
                r = d[:, y, x] + st1["p"][:, y, x] - ps
                return -(ps + np.dot(st0["u"][:, y, x], r) - 0.5 * c * np.dot(r, r))
            best = minimize_scalar(neg_ps, bounds=(-50, 50), method="bounded",
                                   options={"xatol": 1e-12}).x
            assert abs(st1["ps"][y, x] - best) < 1e-6


# --- ALG1: the extrapolated multiplier is recovered from the state ------------------

def test_alg1_split_runs_equal_one_run(orc):
    """A run recovers ubar^k = 2u^k - u^{k-1} from u^k - tau (div q + p_t -
    p_s)^k; the explicit recursion inside a run and the recovery at the start
    of the next must agree, so splitting a run changes nothing (to rounding)."""
    inst = synth.config2(23, 31)
    Cs, Ct = inst.costs
    p = orc.default_params(5, 2)
    one = orc.binary_run(Cs, Ct, inst.alpha, p, 40)
    two = orc.binary_run(Cs, Ct, inst.alpha, p, 17)
    two = orc.binary_run(Cs, Ct, inst.alpha, p, 23, two)
    for k in one:
        np.testing.assert_allclose(two[k], one[k], atol=1e-12)
    instp = synth.config3(14, 17)
    p = orc.default_params(5, 4)
    one = orc.potts_run(instp.costs, instp.alpha, p, 30)
    two = orc.potts_run(instp.costs, instp.alpha, p, 11)
    two = orc.potts_run(instp.costs, instp.alpha, p, 19, two)
    for k in one:
        np.testing.assert_allclose(two[k], one[k], atol=1e-12)


@pytest.mark.parametrize("L", [2, 3, 4, 8])
def test_alg1_default_steps_satisfy_cp_condition(orc, L):
    """sigma tau ||K*K|| < 1 (the convergence condition the Appendix cites)
    for the default steps, with K*K assembled as a matrix on a small grid:
    binary K u = (-grad u, u, -u); Potts K*K = Diag(-Lap + I) + Ones(L, L)."""
    H, W = 5, 6
    n = H * W
    D = np.zeros((2 * n, n))
    for j in range(n):
        e = np.zeros((H, W))
        e.flat[j] = 1.0
        gx, gy = orc.grad(e)
        D[:n, j] = gx.ravel()
        D[n:, j] = gy.ravel()
    lap = -(D.T @ D)
    if L == 2:
        KK = -lap + 2.0 * np.eye(n)
    else:
        KK = np.kron(np.eye(L), -lap + np.eye(n)) + np.kron(np.ones((L, L)), np.eye(n))
    p = orc.default_params(5, L)
    lam = np.linalg.eigvalsh(KK).max()
    assert p.sigma * p.tau * lam < 1.0, (p.sigma, p.tau, lam)


# --- Potts cold start ---------------------------------------------------------

def _np_grad(g):
    """Forward differences with a zero far boundary (unit spacing), written
    out here independently of the oracle's operator."""
    gx = np.zeros_like(g)
    gy = np.zeros_like(g)
    gx[:, :-1] = g[:, 1:] - g[:, :-1]
    gy[:-1, :] = g[1:, :] - g[:-1, :]
    return gx, gy


def _tied_potts_costs(L, H, W, seed):
    """Costs on a coarse grid of values, so many pixels have exact ties for
    the cheapest label."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 3, size=(L, H, W)) / 4.0).astype(np.float32)


@pytest.mark.parametrize("algo", ALGOS)
def test_potts_cold_start_is_alpha_zero_saddle_point(orc, algo):
    """The cold start is the alpha = 0 saddle point: u_i = 1 for the FIRST
    cheapest label (ties included), q_i = 0, p_i = p_s = min_j C_j; rPDRQ
    stores ybar = y - tau K u of that point (Eq. pdrq:4labels: y is recovered
    as q_i = qbar_i - tau grad u_i, p_i = pbar_i + tau u_i,
    p_s = pbar_s - tau sum_i u_i).  With alpha = 0 every algorithm must leave
    it unchanged."""
    L, H, W = 5, 6, 7
    C = _tied_potts_costs(L, H, W, seed=31)
    first = np.argmin(C, axis=0)  # numpy returns the first minimiser
    assert (np.sort(C, axis=0)[0] == np.sort(C, axis=0)[1]).sum() > 5  # ties present
    m = C.astype(np.float64).min(axis=0)
    p = orc.default_params(algo, L)
    st0 = orc.potts_run(C, 0.0, p, 0)
    u_exp = (np.arange(L)[:, None, None] == first[None]).astype(np.float64)
    np.testing.assert_array_equal(st0["u"], u_exp)
    qx, qy, pp, ps = (st0[k].copy() for k in ("qx", "qy", "p", "ps"))
    if algo == 3:
        for i in range(L):
            gx, gy = _np_grad(u_exp[i])
            qx[i] -= p.tau * gx
            qy[i] -= p.tau * gy
            pp[i] += p.tau * u_exp[i]
        ps -= p.tau * u_exp.sum(axis=0)
    np.testing.assert_allclose(qx, 0.0, atol=1e-15)
    np.testing.assert_allclose(qy, 0.0, atol=1e-15)
    np.testing.assert_allclose(pp, np.broadcast_to(m, pp.shape), atol=1e-15)
    np.testing.assert_allclose(ps, m, atol=1e-15)
    st = orc.potts_run(C, 0.0, p, 4, st0)
    for k in ("u", "qx", "qy", "p", "ps"):
        np.testing.assert_allclose(st[k], st0[k], atol=1e-12, err_msg=k)
    E, D, gap, res = orc.potts_eval(C, 0.0, st, p)
    assert abs(E - m.sum()) < 1e-12 and abs(D - m.sum()) < 1e-12 and res < 1e-12


def test_potts_conservation_residual_vanishes(orc):
    """Flow conservation div q_i - p_s + p_i = 0 for every label holds at the
    limit (Eq. potts-mf)."""
    inst = synth.config3(16, 14)
    for algo in (2, 3):
        p = orc.default_params(algo, 4)
        st = orc.potts_run(inst.costs, inst.alpha, p, 200)
        res0 = orc.potts_eval(inst.costs, inst.alpha, st, p)[3]
        st = orc.potts_run(inst.costs, inst.alpha, p, 20000, st)
        E, D, gap, res = orc.potts_eval(inst.costs, inst.alpha, st, p)
        assert res < res0 / 1000 and res < 1e-7 and gap < 1e-8, (algo, res0, res, gap)


def test_potts_label_count_guard(orc):
    """The oracle's per-pixel label buffers hold 64 entries; more labels are
    refused instead of overrunning them."""
    C = np.zeros((65, 2, 2), dtype=np.float32)
    st = {k: np.zeros((65, 2, 2)) for k in ("u", "qx", "qy", "p")}
    st["ps"] = np.zeros((2, 2))
    with pytest.raises(ValueError):
        orc.potts_eval(C, 0.1, st, orc.default_params(2, 65))
    with pytest.raises(ValueError):
        orc.potts_run(C, 0.1, orc.default_params(2, 65), 1)
    with pytest.raises(ValueError):
        orc.simplex(np.zeros(65))
    np.testing.assert_allclose(orc.simplex(np.zeros(64)), np.full(64, 1.0 / 64))
