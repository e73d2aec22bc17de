"""GPU parity of the Potts solver (through the C ABI) against the FP64
oracle on the same seeded inputs; tolerances as for the binary solver."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu

ALGOS = [0, 1, 2, 3, 4]
TOL_U = 1e-4


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _cases():
    return {
        "voronoi4_48x40": (synth.config3(48, 40), 60),
        "voronoi16_edge_45x70": (synth.config5(45, 70), 30),
        "L2_33x29": (synth.random_potts(33, 29, 2, seed=21, alpha=0.3, field_alpha=True), 40),
        "L3_1x50": (synth.random_potts(1, 50, 3, seed=22, alpha=0.3), 30),
        "L8_37x1": (synth.random_potts(37, 1, 8, seed=23, alpha=0.3), 30),
        "L5_ragged_67x35": (synth.random_potts(67, 35, 5, seed=24, alpha=0.25,
                                               field_alpha=True), 40),
    }


def _gpu_run(cmf, inst, algo, n, **kw):
    p = cmf.default_params(algo, inst.L, **kw)
    s = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(s)
    cmf.cmf_iterate_potts(s, n)
    torch.cuda.synchronize()
    return s


def _oracle_run(inst, algo, n, **kw):
    p = O.default_params(algo, inst.L, **kw)
    return O.potts_run(inst.costs, inst.alpha, p, n), p


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", list(_cases()))
def test_iterations_match_oracle_f32(cmf, case, algo, impl):
    inst, n = _cases()[case]
    s = _gpu_run(cmf, inst, algo, n, impl=impl)
    got = s.state()
    ref, _ = _oracle_run(inst, algo, n)
    for k in ("u", "qx", "qy", "p", "ps"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


@pytest.mark.parametrize("L", [17, 32])
def test_many_labels(cmf, L):
    inst = synth.random_potts(23, 37, L, seed=30 + L, alpha=0.2, field_alpha=True)
    for algo in [2, 3]:
        s = _gpu_run(cmf, inst, algo, 20)
        ref, _ = _oracle_run(inst, algo, 20)
        assert np.abs(s.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("algo", ALGOS)
def test_anisotropic_and_multisweep(cmf, algo):
    inst = synth.random_potts(31, 26, 4, seed=40, alpha=0.3, field_alpha=True)
    for aniso, sweeps in [(1, 1), (0, 2)]:
        s = _gpu_run(cmf, inst, algo, 30, aniso=aniso, sweeps=sweeps)
        ref, _ = _oracle_run(inst, algo, 30, aniso=aniso, sweeps=sweeps)
        assert np.abs(s.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("algo", ALGOS)
def test_certificates_match_oracle(cmf, algo):
    inst = synth.config3(64, 72)
    s = _gpu_run(cmf, inst, algo, 25)
    E, D, gap, res = cmf.cmf_eval_potts(s)
    st = s.state()
    Eo, Do, gapo, reso = O.potts_eval(inst.costs, inst.alpha, st, O.default_params(algo, 4))
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert abs(D - Do) <= 1e-5 * abs(Eo)
    assert abs(gap - gapo) <= 1e-6 + 1e-4 * abs(gapo)
    assert abs(res - reso) <= 1e-4 * reso + 1e-6


@pytest.mark.parametrize("storage,tol", [(1, 3e-3), (2, 3e-2)])
@pytest.mark.parametrize("algo", [1, 2, 3])
def test_half_storage_tracks_oracle(cmf, storage, tol, algo):
    inst = synth.config3(40, 48)
    s = _gpu_run(cmf, inst, algo, 30, storage=storage)
    ref, _ = _oracle_run(inst, algo, 30)
    assert np.abs(s.state()["u"] - ref["u"]).max() <= tol


@pytest.mark.parametrize("algo", ALGOS)
def test_solve_certified_by_oracle(cmf, algo):
    inst = synth.config3(96, 80)
    p = cmf.default_params(algo, 4, tol_gap=1e-4, max_iter=30000, check_every=10)
    s = cmf.alloc_potts(inst, p)
    status, iters, hist = cmf.cmf_solve_potts(s)
    assert status == cmf.OK and hist[-1, 3] <= 1e-4
    st = s.state()
    E, D, gap, res = O.potts_eval(inst.costs, inst.alpha, st, O.default_params(algo, 4))
    assert gap <= 1.01e-4
    ref, _, _ = O.solve(inst, algo, tol=1e-4, max_iter=60000, check_every=10)
    agree = np.mean(O.potts_labels(st["u"]) == O.potts_labels(ref["u"]))
    assert agree >= 0.999, agree
    opt, _, _ = O.solve(inst, algo, tol=1e-7, max_iter=60000)
    assert np.mean(O.potts_labels(st["u"]) == O.potts_labels(opt["u"])) >= 0.99


def _window_step_check(cmf, inst, algo, k_before, windows, margin=8, storage=0, tol=2e-5):
    p = cmf.default_params(algo, inst.L, storage=storage)
    s = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(s)
    cmf.cmf_iterate_potts(s, k_before)
    torch.cuda.synchronize()
    W = s.W
    keys = ("u", "qx", "qy", "p", "ps")
    before = {k: getattr(s, k)[..., :W].float().clone() for k in keys}
    cmf.cmf_iterate_potts(s, 1)
    torch.cuda.synchronize()
    after = {k: getattr(s, k)[..., :W].float().clone() for k in keys}
    po = O.default_params(algo, inst.L)
    alpha = inst.alpha_field()
    for (r0, c0, h, w) in windows:
        R0, C0 = max(r0 - margin, 0), max(c0 - margin, 0)
        R1, C1 = min(r0 + h + margin, s.H), min(c0 + w + margin, s.W)
        if (R0 + C0) % 2:  # keep the crop's red/black colouring that of the grid
            if R0 > 0:
                R0 -= 1
            else:
                C0 -= 1
        st = {k: v[..., R0:R1, C0:C1].cpu().double().numpy() for k, v in before.items()}
        res = O.potts_run(inst.costs[:, R0:R1, C0:C1], alpha[R0:R1, C0:C1], po, 1, st)
        ri0 = r0 - R0 if R0 > 0 else 0
        ci0 = c0 - C0 if C0 > 0 else 0
        for k in keys:
            got = after[k][..., r0:r0 + h, c0:c0 + w].cpu().double().numpy()
            ref = res[k][..., ri0:ri0 + h, ci0:ci0 + w]
            if storage:
                # the oracle step from the stored half-precision state, then
                # one rounding of the result to the storage type
                ref = torch.as_tensor(ref).to(getattr(s, k).dtype).double().numpy() \
                    if k != "u" else ref
            err = np.abs(got - ref).max()
            assert err <= tol, (k, (r0, c0), err)


@pytest.mark.parametrize("algo", [1, 2, 3])
def test_full_size_2048_L4_windows(cmf, algo):
    inst = synth.config3()
    wins = [(0, 0, 40, 40), (2048 - 37, 2048 - 45, 37, 45), (1000, 1500, 64, 64),
            (0, 1111, 33, 70)]
    _window_step_check(cmf, inst, algo, 23, wins)


@pytest.mark.parametrize("algo", [2, 3])
def test_graph_solve_equals_host_loop(cmf, algo):
    inst = synth.config3(72, 56)
    out = []
    for use_graph in (1, 0):
        p = cmf.default_params(algo, 4, use_graph=use_graph, tol_gap=1e-4, max_iter=8000,
                               check_every=10)
        s = cmf.alloc_potts(inst, p)
        out.append((cmf.cmf_solve_potts(s), s.state()))
    (s1, i1, h1), st1 = out[0]
    (s0, i0, h0), st0 = out[1]
    assert s1 == s0 == cmf.OK and i1 == i0
    np.testing.assert_array_equal(h1, h0)
    for k in st0:
        np.testing.assert_array_equal(st1[k], st0[k])


def test_full_size_4096_L16_f16_windows(cmf):
    """4096^2, 16 labels, float16 flow storage (the largest workload): one
    rpADMMII step from the stored state matches the oracle step on windows;
    float16 results are compared after rounding the oracle's to float16."""
    inst = synth.config5()
    wins = [(0, 0, 32, 32), (4096 - 29, 4096 - 40, 29, 40), (2001, 3007, 40, 40)]
    _window_step_check(cmf, inst, 2, 11, wins, storage=1, tol=2e-3)


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("variant", [8, 16, 32])
@pytest.mark.parametrize("L,shape", [(4, (70, 97)), (16, (33, 40)), (3, (5, 130))])
def test_tma_tiles_match_smem_tiles(cmf, storage, variant, L, shape):
    """The TMA-staged fused ADMM kernel computes what the shared-memory tile
    kernel computes (same formulas; only the staging differs)."""
    inst = synth.random_potts(*shape, L, seed=70 + L, alpha=0.3, field_alpha=True)
    a = _gpu_run(cmf, inst, 2, 7, storage=storage, variant=1).state()
    b = _gpu_run(cmf, inst, 2, 7, storage=storage, variant=variant).state()
    tol = 1e-6 if storage == 0 else 1e-2
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= tol, k
