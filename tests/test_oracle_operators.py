"""Pins of the oracle's discrete operators and preconditioners against
mathematics the paper fixes (Thm 1, Thm 2, Lemma 1, the sRBGS preconditioner
of the rPDRQ steps) and against textbook constructions that share no code with
the oracle (networkx grid-graph Laplacian, explicit Gauss-Seidel matrices,
bisection for the simplex projection)."""
import itertools

import networkx as nx
import numpy as np
import pytest


def _grad_matrix(orc, H, W):
    """Columns: oracle grad applied to unit vectors -> (2N x N)."""
    N = H * W
    G = np.zeros((2 * N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        gx, gy = orc.grad(e.reshape(H, W))
        G[:N, k] = gx.ravel()
        G[N:, k] = gy.ravel()
    return G


def _div_matrix(orc, H, W):
    N = H * W
    D = np.zeros((N, 2 * N))
    for k in range(2 * N):
        e = np.zeros(2 * N)
        e[k] = 1.0
        D[:, k] = orc.div(e[:N].reshape(H, W), e[N:].reshape(H, W)).ravel()
    return D


def _grid_laplacian(H, W):
    """-Laplacian of the 4-neighbour grid graph (Neumann), row-major order."""
    g = nx.grid_2d_graph(H, W)
    nodes = [(i, j) for i in range(H) for j in range(W)]
    return nx.laplacian_matrix(g, nodelist=nodes).toarray().astype(float)


def test_gradient_of_ramp(orc):
    H, W = 5, 7
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    gx, gy = orc.grad(3.0 * jj + 5.0 * ii)
    ex = np.full((H, W), 3.0)
    ex[:, -1] = 0.0
    ey = np.full((H, W), 5.0)
    ey[-1, :] = 0.0
    np.testing.assert_array_equal(gx, ex)
    np.testing.assert_array_equal(gy, ey)


def test_div_is_minus_grad_adjoint(orc):
    rng = np.random.default_rng(0)
    for H, W in [(1, 6), (6, 1), (4, 5), (7, 3)]:
        g = rng.normal(size=(H, W))
        qx, qy = rng.normal(size=(H, W)), rng.normal(size=(H, W))
        qx[:, -1] = 0.0  # components grad never produces
        qy[-1, :] = 0.0
        gx, gy = orc.grad(g)
        lhs = np.sum(gx * qx + gy * qy)
        rhs = -np.sum(g * orc.div(qx, qy))
        assert abs(lhs - rhs) < 1e-12


@pytest.mark.parametrize("H,W", [(1, 5), (3, 3), (4, 6), (5, 5)])
def test_div_grad_is_grid_laplacian(orc, H, W):
    G = _grad_matrix(orc, H, W)
    D = _div_matrix(orc, H, W)
    np.testing.assert_allclose(-D @ G, _grid_laplacian(H, W), atol=0, rtol=0)


@pytest.mark.parametrize("H,W", [(3, 3), (4, 6), (6, 6), (10, 10)])
def test_thm1_div_norm_bound(orc, H, W):
    """Thm 1: 8 I >= div^* div, so a = 8 is admissible for N = a c I."""
    D = _div_matrix(orc, H, W)
    lam = np.linalg.eigvalsh(D.T @ D).max()
    assert lam <= 8.0 + 1e-12
    if H >= 10:
        assert lam > 7.5  # the bound is essentially tight


def test_thm1_two_block_bound():
    """Thm 1: 2 I_2 >= A^* A for A = [I, -I] (one pixel suffices)."""
    A = np.array([[1.0, -1.0]])
    assert np.linalg.eigvalsh(2.0 * np.eye(2) - A.T @ A).min() >= -1e-15


@pytest.mark.parametrize("L", [2, 3, 4, 8, 16])
def test_thm2_block_preconditioner(orc, L):
    """Thm 2: Diag[a1 I,...,a1 I, a2 I] >= A^* A with A = [I_n, -L_n], a1 = 2,
    a2 = 2n; a2 = 2n is also the smallest admissible value for a1 = 2."""
    p = orc.default_params(orc.RPADMM_EB, L)
    assert p.a1 == 2.0 and p.a2 == 2.0 * L
    A = np.hstack([np.eye(L), -np.ones((L, 1))])
    AtA = A.T @ A
    At = np.diag([p.a1] * L + [p.a2])
    assert np.linalg.eigvalsh(At - AtA).min() >= -1e-12
    At_small = np.diag([p.a1] * L + [p.a2 - 0.1])
    assert np.linalg.eigvalsh(At_small - AtA).min() < 0


@pytest.mark.parametrize("L", [2, 3, 4])
def test_lemma1_T0_dominates_KstarK(orc, L):
    """Lemma 1: T_0 = Diag[-Lap + (n+1) I] >= K^* K, and K^* K equals
    Diag[-Lap + I] + Ones(n, n) (the second form of the garbled identity)."""
    H, W = 3, 3
    N = H * W
    G = _grad_matrix(orc, H, W)
    # K u = (B^* u; A^* u): B^* = Diag[-grad], A^* u = (u_1..u_n, -sum u_i)
    Bs = np.kron(np.eye(L), -G)
    As = np.vstack([np.eye(L * N), -np.kron(np.ones((1, L)), np.eye(N))])
    K = np.vstack([Bs, As])
    KtK = K.T @ K
    lap = _grid_laplacian(H, W)
    expect = np.kron(np.eye(L), lap + np.eye(N)) + np.kron(np.ones((L, L)), np.eye(N))
    np.testing.assert_allclose(KtK, expect, atol=1e-12)
    T0 = np.kron(np.eye(L), lap + (L + 1) * np.eye(N))
    assert np.linalg.eigvalsh(T0 - KtK).min() >= -1e-10


def _sgs_matrices(H, W, kappa, st):
    lap = _grid_laplacian(H, W)
    T = st * (kappa * np.eye(H * W) + lap)
    red = [i * W + j for i in range(H) for j in range(W) if (i + j) % 2 == 0]
    black = [i * W + j for i in range(H) for j in range(W) if (i + j) % 2 == 1]
    perm = np.array(red + black)
    Tp = T[np.ix_(perm, perm)]
    Dg = np.diag(np.diag(Tp))
    Lo = -np.tril(Tp, -1)
    Up = -np.triu(Tp, 1)
    M = (Dg - Lo) @ np.linalg.inv(Dg) @ (Dg - Up)
    return T, Tp, M, perm


@pytest.mark.parametrize("H,W,kappa,st", [(4, 4, 2.0, 0.2), (5, 3, 5.0, 2.0), (1, 6, 3.0, 0.7)])
def test_srbgs_is_symmetric_gauss_seidel_preconditioner(orc, H, W, kappa, st):
    """One rPDRQ u-step u + M^{-1}(b - T u), M the symmetric red-black
    Gauss-Seidel preconditioner of T = st (kappa I - Lap), equals the oracle's
    red/black/red sweep; s sweeps equal s applications; M >= T."""
    T, Tp, M, perm = _sgs_matrices(H, W, kappa, st)
    rng = np.random.default_rng(1)
    b = rng.normal(size=H * W)
    u = rng.normal(size=H * W)
    Mi = np.linalg.inv(M)

    def step(v):
        vp, bp = v[perm], b[perm]
        out = np.empty_like(v)
        out[perm] = vp + Mi @ (bp - Tp @ vp)
        return out

    got1 = orc.srbgs(b.reshape(H, W), u.reshape(H, W), kappa, st, 1).ravel()
    np.testing.assert_allclose(got1, step(u), atol=1e-12)
    got2 = orc.srbgs(b.reshape(H, W), u.reshape(H, W), kappa, st, 2).ravel()
    np.testing.assert_allclose(got2, step(step(u)), atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (M + M.T) - Tp).min() >= -1e-10
    np.testing.assert_allclose(M, M.T, atol=1e-12)


def test_projection_alpha(orc):
    rng = np.random.default_rng(2)
    qx, qy = rng.normal(size=(6, 6)), rng.normal(size=(6, 6))
    al = rng.uniform(0.0, 1.5, size=(6, 6))
    al[0, 0] = 0.0
    px, py = orc.project_alpha(qx, qy, al, 0)
    n0 = np.hypot(qx, qy)
    n1 = np.hypot(px, py)
    assert np.all(n1 <= al + 1e-15)
    inside = n0 <= al
    np.testing.assert_array_equal(px[inside], qx[inside])
    out = ~inside & (al > 0)
    np.testing.assert_allclose(n1[out], al[out], rtol=1e-14)
    # direction preserved
    np.testing.assert_allclose(px[out] * qy[out] - py[out] * qx[out], 0.0, atol=1e-14)
    assert px[0, 0] == 0.0 and py[0, 0] == 0.0
    ax, ay = orc.project_alpha(qx, qy, al, 1)
    np.testing.assert_array_equal(ax, np.clip(qx, -al, al))
    np.testing.assert_array_equal(ay, np.clip(qy, -al, al))


def test_simplex_projection_matches_bisection(orc):
    rng = np.random.default_rng(3)
    for n in [2, 3, 4, 8, 16]:
        for _ in range(20):
            v = rng.normal(size=n) * rng.uniform(0.1, 3.0)
            w = orc.simplex(v)
            lo, hi = v.min() - 1.0, v.max()
            for _ in range(200):  # sum(max(v - t, 0)) = 1 by bisection
                t = 0.5 * (lo + hi)
                if np.maximum(v - t, 0).sum() > 1.0:
                    lo = t
                else:
                    hi = t
            np.testing.assert_allclose(w, np.maximum(v - 0.5 * (lo + hi), 0), atol=1e-12)
            assert abs(w.sum() - 1.0) < 1e-12 and w.min() >= 0.0
