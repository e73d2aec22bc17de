"""GPU parity of the Potts solver (through the C ABI) against the FP64
oracle on the same seeded inputs; tolerances as for the binary solver."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu

ALGOS = [0, 1, 2, 3, 4, 5]
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
        # wide enough for interior warp-strip items (no bounds predicates)
        # beside boundary ones, in both directions
        "voronoi16_mixed_130x256": (synth.config5(130, 256), 20),
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


@pytest.mark.parametrize("L", [31, 64])
def test_many_labels_strips(cmf, L):
    """Even width: the warp-strip kernels at large label counts (the rPDRQ
    kernel shares 31 labels out over 4 warps of 8 and 7 passes, 64 over 4
    warps of 16), against the oracle."""
    inst = synth.random_potts(23, 38, L, seed=40 + L, alpha=0.2, field_alpha=True)
    for algo in [2, 3]:
        s = _gpu_run(cmf, inst, algo, 20, variant=2)
        ref, _ = _oracle_run(inst, algo, 20)
        got = s.state()
        for k in ("u", "qx", "qy", "p", "ps"):
            assert np.abs(got[k] - ref[k]).max() <= TOL_U, (algo, k)


@pytest.mark.parametrize("algo", ALGOS)
def test_anisotropic_and_multisweep(cmf, algo):
    inst = synth.random_potts(31, 26, 4, seed=40, alpha=0.3, field_alpha=True)
    for aniso, sweeps in [(1, 1), (0, 2)]:
        s = _gpu_run(cmf, inst, algo, 30, aniso=aniso, sweeps=sweeps)
        ref, _ = _oracle_run(inst, algo, 30, aniso=aniso, sweeps=sweeps)
        assert np.abs(s.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("shape", [(64, 72), (64, 71), (1, 64), (131, 2), (300, 250)])
@pytest.mark.parametrize("algo", ALGOS)
def test_certificates_match_oracle(cmf, algo, shape):
    """Even widths go through the warp-strip certificate kernel, odd ones
    through the tile kernel; both against the oracle's evaluation."""
    inst = synth.config3(*shape)
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


def _window_step_check(cmf, inst, algo, k_before, windows, margin=8, storage=0, tol=2e-5,
                       variant=0):
    p = cmf.default_params(algo, inst.L, storage=storage, variant=variant)
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


# ---- warp-strip kernel (variant 2) ---------------------------------------------

STRIP_CASES = {
    "voronoi4_48x40": (synth.config3(48, 40), 60),
    "voronoi16_edge_45x64": (synth.config5(45, 64), 31),
    "L4_ragged_70x130": (synth.random_potts(70, 130, 4, seed=81, alpha=0.3,
                                            field_alpha=True), 25),
    "L3_1x50": (synth.random_potts(1, 50, 3, seed=22, alpha=0.3), 30),
    "L8_37x2": (synth.random_potts(37, 2, 8, seed=23, alpha=0.3), 30),
    "L2_tall_301x62": (synth.random_potts(301, 62, 2, seed=82, alpha=0.4,
                                          field_alpha=True), 17),
}


@pytest.mark.parametrize("algo", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("case", list(STRIP_CASES))
def test_strip_matches_oracle_f32(cmf, case, algo):
    """Warp-strip ADMM kernel against the oracle after a fixed number of
    iterations (odd and even counts: the result lands in either buffer set,
    and the multipliers are turned back from the w form at the end)."""
    inst, n = STRIP_CASES[case]
    s = _gpu_run(cmf, inst, algo, n, variant=2)
    got = s.state()
    ref, _ = _oracle_run(inst, algo, n)
    for k in ("u", "qx", "qy", "p", "ps"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


@pytest.mark.parametrize("algo", [1, 2])
def test_strip_anisotropic(cmf, algo):
    inst = synth.random_potts(31, 26, 4, seed=40, alpha=0.3, field_alpha=True)
    s = _gpu_run(cmf, inst, algo, 30, aniso=1, variant=2)
    ref, _ = _oracle_run(inst, algo, 30, aniso=1)
    assert np.abs(s.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("L,shape", [(4, (70, 98)), (16, (33, 40)), (3, (5, 130))])
def test_strip_matches_smem_tiles_half(cmf, storage, L, shape):
    """16-bit flow storage: the strip kernel computes what the shared-memory
    tile kernel computes, up to the storage rounding of close values."""
    inst = synth.random_potts(*shape, L, seed=70 + L, alpha=0.3, field_alpha=True)
    for algo in (2, 3):
        a = _gpu_run(cmf, inst, algo, 7, storage=storage, variant=1).state()
        b = _gpu_run(cmf, inst, algo, 7, storage=storage, variant=2).state()
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= 1e-2, (algo, k)


def test_strip_rejects_odd_width(cmf):
    inst = synth.random_potts(20, 33, 3, seed=83, alpha=0.3)
    p = cmf.default_params(2, 3, variant=2)
    s = cmf.alloc_potts(inst, p)
    with pytest.raises(cmf.CmfError):
        cmf.cmf_iterate_potts(s, 2)


def test_strip_iterate_then_solve_continues(cmf):
    """Calls chain: the state after cmf_iterate holds u (not the w form), so
    two calls of n iterations equal one call of 2n."""
    inst = synth.random_potts(40, 64, 4, seed=84, alpha=0.3, field_alpha=True)
    p = cmf.default_params(2, 4, variant=2)
    a = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(a)
    cmf.cmf_iterate_potts(a, 9)
    cmf.cmf_iterate_potts(a, 8)
    b = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(b)
    cmf.cmf_iterate_potts(b, 17)
    ga, gb = a.state(), b.state()
    for k in ga:
        assert np.abs(ga[k] - gb[k]).max() <= 1e-6, k


@pytest.mark.parametrize("algo", [2, 4])
def test_strip_full_size_2048_L4_windows(cmf, algo):
    inst = synth.config3()
    wins = [(0, 0, 40, 40), (2048 - 37, 2048 - 45, 37, 45), (1000, 1500, 64, 64),
            (0, 1111, 33, 70)]
    _window_step_check(cmf, inst, algo, 23, wins, variant=2)


def test_strip_full_size_4096_L16_f16_windows(cmf):
    inst = synth.config5()
    wins = [(0, 0, 32, 32), (4096 - 29, 4096 - 40, 29, 40), (2001, 3007, 40, 40)]
    _window_step_check(cmf, inst, 2, 11, wins, storage=1, tol=2e-3, variant=2)


def test_strip_matches_tma_full_size_2048_L4(cmf):
    """Every output of a few full-size iterations: strip kernel against the
    TMA tile kernel (many work items per warp, ragged last strip)."""
    inst = synth.config3()
    a = _gpu_run(cmf, inst, 2, 6, variant=16)
    b = _gpu_run(cmf, inst, 2, 6, variant=2)
    for k in ("u", "qx", "qy", "p", "ps"):
        err = (getattr(a, k).float() - getattr(b, k).float()).abs().max().item()
        assert err <= 1e-5, (k, err)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_strip_solve_certified(cmf, use_graph):
    """Solve to the gap with the strip kernel (checks between chunks see u,
    not the w form); the oracle certifies the returned state."""
    inst = synth.config3(96, 80)
    p = cmf.default_params(2, 4, tol_gap=1e-4, max_iter=30000, check_every=10, variant=2,
                           use_graph=use_graph)
    s = cmf.alloc_potts(inst, p)
    status, iters, hist = cmf.cmf_solve_potts(s)
    assert status == cmf.OK and hist[-1, 3] <= 1e-4
    E, D, gap, res = O.potts_eval(inst.costs, inst.alpha, s.state(), O.default_params(2, 4))
    assert gap <= 1.01e-4


@pytest.mark.parametrize("aniso", [0, 1])
@pytest.mark.parametrize("algo", [2, 3])
def test_strip_certificates_many_labels(cmf, algo, aniso):
    inst = synth.config5(70, 96)
    s = _gpu_run(cmf, inst, algo, 20, aniso=aniso)
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(inst.costs, inst.alpha, s.state(),
                                      O.default_params(algo, 16, aniso=aniso))
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert abs(D - Do) <= 1e-5 * abs(Eo)
    assert abs(res - reso) <= 1e-4 * reso + 1e-6


@pytest.mark.parametrize("storage", [1, 2])
def test_strip_certificates_half_storage(cmf, storage):
    inst = synth.config3(64, 96)
    s = _gpu_run(cmf, inst, 2, 25, storage=storage)
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(inst.costs, inst.alpha, s.state(), O.default_params(2, 4))
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert abs(D - Do) <= 1e-5 * abs(Eo)


def test_strip_certificates_full_size_2048_L4(cmf):
    inst = synth.config3()
    s = _gpu_run(cmf, inst, 2, 30)
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(inst.costs, inst.alpha, s.state(), O.default_params(2, 4))
    assert abs(E - Eo) <= 1e-6 * abs(Eo)
    assert abs(D - Do) <= 1e-6 * abs(Eo)
    assert abs(res - reso) <= 1e-5 * reso + 1e-6


@pytest.mark.parametrize("sweeps", [1, 2, 3, 4])
@pytest.mark.parametrize("aniso", [0, 1])
def test_strip_dr_sweeps(cmf, sweeps, aniso):
    """Potts rPDRQ with 1..4 red-black sweeps through the pipelined strip
    kernel against the oracle; several strips and bands, 5 labels."""
    inst = synth.random_potts(90, 130, 5, seed=93, alpha=0.3, field_alpha=True)
    s = _gpu_run(cmf, inst, 3, 13, variant=2, sweeps=sweeps, aniso=aniso)
    ref, _ = _oracle_run(inst, 3, 13, sweeps=sweeps, aniso=aniso)
    got = s.state()
    for k in ("u", "qx", "qy", "p", "ps"):
        assert np.abs(got[k] - ref[k]).max() <= TOL_U, k


def test_strip_dr_full_size_2048_L4_windows(cmf):
    inst = synth.config3()
    wins = [(0, 0, 40, 40), (2048 - 37, 2048 - 45, 37, 45), (1000, 1500, 64, 64)]
    _window_step_check(cmf, inst, 3, 23, wins, variant=2)


# ---- costs computed from (I, levels) where they are read (params.costs = 1) ---------

def _levels_inputs(inst):
    """float32 image and levels, and the float32 cost planes the kernels
    compute from them: (I - c_i)^2 with one rounding per operation."""
    I = inst.image.astype(np.float32)
    lev = np.asarray(inst.levels, dtype=np.float32)
    C = np.stack([(I - c) * (I - c) for c in lev]).astype(np.float32)
    return I, lev, C


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("shape", [(48, 40), (45, 71), (1, 64)])
def test_levels_costs_match_oracle(cmf, algo, shape):
    """Costs from the image and the levels (strip kernels for even widths,
    TMA or tile kernels for odd ones) against the oracle given the same
    float32 cost planes; certificates too."""
    inst = synth.config3(*shape)
    I, lev, C = _levels_inputs(inst)
    p = cmf.default_params(algo, 4)
    s = cmf.alloc_potts_levels(I, lev, inst.alpha, p)
    cmf.cmf_init_potts(s)
    cmf.cmf_iterate_potts(s, 27)
    got = s.state()
    ref = O.potts_run(C, inst.alpha, O.default_params(algo, 4), 27)
    for k in ("u", "qx", "qy", "p", "ps"):
        assert np.abs(got[k] - ref[k]).max() <= TOL_U, k
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(C, inst.alpha, got, O.default_params(algo, 4))
    assert abs(E - Eo) <= 1e-5 * abs(Eo) and abs(D - Do) <= 1e-5 * abs(Eo)


@pytest.mark.parametrize("algo,storage", [(2, 0), (2, 1), (3, 0)])
def test_levels_equal_planes_full_size(cmf, algo, storage):
    """Full-size 16-label recipe at 2048^2: computing the costs in the
    kernels gives the iterates of reading the same float32 cost planes."""
    inst = synth.config5(2048, 2048)
    I, lev, C = _levels_inputs(inst)
    p = cmf.default_params(algo, 16, storage=storage)
    a = cmf.alloc_potts_levels(I, lev, inst.alpha, p)
    cmf.cmf_init_potts(a)
    cmf.cmf_iterate_potts(a, 6)
    b = cmf.Potts(C, inst.alpha, cmf.default_params(algo, 16, storage=storage))
    cmf.cmf_init_potts(b)
    cmf.cmf_iterate_potts(b, 6)
    for k in ("u", "qx", "qy", "p", "ps"):
        err = (getattr(a, k).float() - getattr(b, k).float()).abs().max().item()
        assert err <= 1e-6, (k, err)


def test_levels_solve_certified(cmf):
    inst = synth.config3(96, 80)
    I, lev, C = _levels_inputs(inst)
    p = cmf.default_params(2, 4, tol_gap=1e-4, max_iter=30000, check_every=10)
    s = cmf.alloc_potts_levels(I, lev, inst.alpha, p)
    status, iters, hist = cmf.cmf_solve_potts(s)
    assert status == cmf.OK and hist[-1, 3] <= 1e-4
    E, D, gap, res = O.potts_eval(C, inst.alpha, s.state(), O.default_params(2, 4))
    assert gap <= 1.01e-4


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("shape", [(48, 40), (45, 71), (130, 256)])
def test_half_cost_planes_match_oracle(cmf, algo, shape):
    """costs = 2: the cost planes stored as float16.  The oracle is given the
    same rounded costs (upcast to float64), so both solve the same problem."""
    inst = synth.config5(*shape) if shape[1] > 200 else synth.config3(*shape)
    C16 = inst.costs.astype(np.float16).astype(np.float32)
    p = cmf.default_params(algo, inst.L, costs=2)
    s = cmf.alloc_potts(inst, p)
    assert s.C.dtype == torch.float16
    cmf.cmf_init_potts(s)
    cmf.cmf_iterate_potts(s, 21)
    got = s.state()
    po = O.default_params(algo, inst.L)
    ref = O.potts_run(C16, inst.alpha, po, 21)
    for k in ("u", "qx", "qy", "p", "ps"):
        assert np.abs(got[k] - ref[k]).max() <= TOL_U, k
    E, D, gap, res = cmf.cmf_eval_potts(s)
    Eo, Do, gapo, reso = O.potts_eval(C16, inst.alpha, got, po)
    assert abs(E - Eo) <= 1e-5 * abs(Eo) and abs(D - Do) <= 1e-5 * abs(Eo)


def _phase_one_stop(h, switch, check_every):
    """Row of a 16-bit solve's history at which the first phase of a
    two-phase solve stops: the first gap <= switch, or, tested every
    ceil(200 / check_every) checks from the first, a gap below 10 switch and
    above 0.7 times the gap at the previous tested check."""
    w = -(-200 // check_every)
    ref = None
    for n in range(len(h)):
        g = h[n, 3]
        if g <= switch:
            return n
        if n % w == 0:
            if n > 0 and g < 10 * switch and g > 0.7 * ref:
                return n
            ref = g
    return len(h) - 1


@pytest.mark.parametrize("phase_storage,switch", [(1, 2e-3), (2, 1e-2), (1, 1.2e-4)])
def test_two_phase_solve(cmf, phase_storage, switch):
    """phase_storage: the solve runs in 16-bit flows to the switch gap (or
    to where that storage's gap stalls), then in float32 from exactly that
    state.  Phase one equals the 16-bit solve row for row up to the row the
    switch rule picks; phase two equals a float32 warm start from that state
    row for row; the result is certified by the oracle.  A switch gap below
    the float16 floor (1.2e-4) ends phase one by the stall rule."""
    inst = synth.config5(96, 128)
    tol = 1e-4
    kw = dict(max_iter=20000, check_every=10)
    p16 = cmf.default_params(2, 16, storage=phase_storage, tol_gap=switch, **kw)
    a = cmf.alloc_potts(inst, p16)
    st_a, it_a, h_a = cmf.cmf_solve_potts(a)
    n_s = _phase_one_stop(h_a, switch, kw["check_every"])
    if switch < 2e-4:
        assert h_a[n_s, 3] > switch  # the stall rule, not the gap, ends phase one
    if n_s < len(h_a) - 1 or h_a[n_s, 3] > switch:
        # the state at the stalled check: the same 16-bit iterations, stopped there
        it_a = int(h_a[n_s, 0])
        q16 = cmf.default_params(2, 16, storage=phase_storage, tol_gap=0.0, max_iter=it_a,
                                 check_every=kw["check_every"])
        a = cmf.alloc_potts(inst, q16)
        st_s, it_s, h_s = cmf.cmf_solve_potts(a)
        assert it_s == it_a
        np.testing.assert_array_equal(h_s, h_a[:n_s + 1])
        h_a = h_s
    else:
        assert st_a == cmf.OK and h_a[-1, 3] <= switch
    p32 = cmf.default_params(2, 16, tol_gap=tol, warm_start=1, **kw)
    c = cmf.alloc_potts(inst, p32)
    c.load_state(a.state())  # 16-bit values are exact in float32
    st_c, it_c, h_c = cmf.cmf_solve_potts(c)
    p = cmf.default_params(2, 16, tol_gap=tol, phase_storage=phase_storage, phase_gap=switch, **kw)
    b = cmf.alloc_potts(inst, p)
    st_b, it_b, h_b = cmf.cmf_solve_potts(b)
    assert st_b == cmf.OK == st_c and it_b == it_a + it_c
    np.testing.assert_array_equal(h_b[:len(h_a)], h_a)
    np.testing.assert_array_equal(h_b[len(h_a):, 1:], h_c[:, 1:])
    np.testing.assert_array_equal(h_b[len(h_a):, 0], h_c[:, 0] + it_a)
    got = b.state()
    for k in ("u", "qx", "qy", "p", "ps"):
        np.testing.assert_array_equal(got[k], c.state()[k])
    E, D, gap, res = O.potts_eval(inst.costs, inst.alpha, got, O.default_params(2, 16))
    assert gap <= 1.001e-4
    # the host-driven loop takes the same decisions
    ph = cmf.default_params(2, 16, tol_gap=tol, phase_storage=phase_storage, phase_gap=switch,
                            use_graph=0, **kw)
    e = cmf.alloc_potts(inst, ph)
    st_e, it_e, h_e = cmf.cmf_solve_potts(e)
    assert st_e == cmf.OK and it_e == it_b
    np.testing.assert_array_equal(h_e, h_b)


def test_autotune_step_size(cmf, tmp_path):
    """tune_step = 1 adds the ADMM step sizes c, 2c, 4c, 8c to the search.  The
    tuned c is a parameter of the same method: the GPU iterates with it match
    the oracle run with the same c, and its solve is certified by the oracle."""
    inst = synth.config5(64, 96)
    p = cmf.default_params(2, 16, tol_gap=1e-4, max_iter=8000, check_every=10, tune_step=1)
    s = cmf.alloc_potts(inst, p)
    best, ms = cmf.cmf_autotune_potts(s)
    assert ms > 0 and any(abs(best.c - 0.3 * f) < 1e-12 for f in (1, 2, 4, 8))
    q = cmf.tuned_params(s, cache_path=str(tmp_path / "tune.json"))
    assert abs(q.c - best.c) < 1e-12
    g = _gpu_run(cmf, inst, 2, 25, c=best.c)
    ref, _ = _oracle_run(inst, 2, 25, c=best.c)
    for k in ("u", "qx", "qy", "p", "ps"):
        assert np.abs(g.state()[k] - ref[k]).max() <= TOL_U, k
    t = cmf.alloc_potts(inst, q)
    st, it, hist = cmf.cmf_solve_potts(t)
    assert st == cmf.OK
    E, D, gap, res = O.potts_eval(inst.costs, inst.alpha, t.state(), O.default_params(2, 16))
    assert gap <= 1.001e-4


def test_autotune_two_phase_switch(cmf, tmp_path):
    """tune_step = 1 on a two-phase solve also tries each step size with the
    switch left to the stall test (phase_gap = 1.5 tol_gap); the binding's
    cache carries the chosen switch gap, and the tuned solve is certified."""
    inst = synth.config5(64, 96)
    p = cmf.default_params(2, 16, tol_gap=1e-4, max_iter=8000, check_every=10, tune_step=1,
                           phase_storage=1, phase_gap=2e-3)
    s = cmf.alloc_potts(inst, p)
    best, ms = cmf.cmf_autotune_potts(s)
    assert ms > 0 and any(abs(best.c - 0.3 * f) < 1e-12 for f in (1, 2, 4, 8))
    assert best.phase_gap in (2e-3, 1.5 * p.tol_gap) and best.phase_storage == 1
    q = cmf.tuned_params(s, cache_path=str(tmp_path / "tune.json"))
    assert q.phase_gap == best.phase_gap and abs(q.c - best.c) < 1e-12
    q2 = cmf.tuned_params(s, cache_path=str(tmp_path / "tune.json"))  # from the cache
    assert q2.phase_gap == best.phase_gap and abs(q2.c - best.c) < 1e-12
    t = cmf.alloc_potts(inst, q)
    st, it, hist = cmf.cmf_solve_potts(t)
    assert st == cmf.OK
    E, D, gap, res = O.potts_eval(inst.costs, inst.alpha, t.state(), O.default_params(2, 16))
    assert gap <= 1.001e-4


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("L,shape", [(5, (301, 130)), (16, (140, 64)), (3, (9, 200))])
def test_rpdrq_strip_label_sum_plane_is_exact(cmf, storage, L, shape):
    """The rPDRQ strip kernel's later launches of a call read sum_i u_i from
    the plane the previous launch wrote; the first launch sums the u_i
    planes. Both sums are taken in label order, so seven iterations in one
    call equal seven calls of one iteration bit for bit (bands of several
    heights, label counts shared out over 3, 4 and 5 warps)."""
    H, W = shape
    inst = synth.random_potts(H, W, L, seed=90 + L, alpha=0.3, field_alpha=True)
    p = cmf.default_params(3, L, storage=storage, variant=2)
    a = cmf.alloc_potts(inst, p)
    b = cmf.alloc_potts(inst, p)
    cmf.cmf_init_potts(a)
    cmf.cmf_init_potts(b)
    cmf.cmf_iterate_potts(a, 7)
    for _ in range(7):
        cmf.cmf_iterate_potts(b, 1)
    torch.cuda.synchronize()
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("algo,shape", [(3, (64, 96)), (5, (64, 96)), (0, (64, 96)),
                                        (2, (63, 91))])
def test_two_phase_other_algorithms_and_tiles(cmf, algo, shape):
    """Two-phase solves of rPDRQ (its strip kernel's label-sum planes serve
    both phases), ALG1 and pADMMI, and of an odd width (tile kernels): the
    result is certified by the oracle, and the host-driven loop takes the
    same decisions as the device-driven one."""
    inst = synth.config5(*shape)
    kw = dict(tol_gap=1e-4, max_iter=30000, check_every=10, phase_storage=1, phase_gap=2e-3)
    p = cmf.default_params(algo, 16, **kw)
    s = cmf.alloc_potts(inst, p)
    st, it, hist = cmf.cmf_solve_potts(s)
    assert st == cmf.OK, (it, hist[-1])
    po = O.default_params(algo, 16, sigma=p.sigma, tau=p.tau)
    assert O.potts_eval(inst.costs, inst.alpha, s.state(), po)[2] <= 1.001e-4
    ph = cmf.default_params(algo, 16, use_graph=0, **kw)
    e = cmf.alloc_potts(inst, ph)
    st_e, it_e, h_e = cmf.cmf_solve_potts(e)
    assert st_e == cmf.OK and it_e == it
    np.testing.assert_array_equal(h_e, hist)


def test_two_phase_first_phase_uses_up_max_iter(cmf):
    """A first phase that reaches neither the switch gap nor a stall within
    max_iter: NOT_CONVERGED after max_iter iterations, the 16-bit state
    widened into the caller's buffers (equal to a 16-bit solve stopped there)."""
    inst = synth.config5(32, 64)
    kw = dict(max_iter=40, check_every=10)
    p = cmf.default_params(2, 16, tol_gap=1e-4, phase_storage=1, phase_gap=2e-3, **kw)
    s = cmf.alloc_potts(inst, p)
    st, it, hist = cmf.cmf_solve_potts(s)
    assert st == cmf.NOT_CONVERGED and it == 40 and len(hist) == 4
    q = cmf.default_params(2, 16, storage=1, tol_gap=2e-3, **kw)
    a = cmf.alloc_potts(inst, q)
    st_a, it_a, h_a = cmf.cmf_solve_potts(a)
    assert it_a == 40
    np.testing.assert_array_equal(hist, h_a)
    got, ref = s.state(), a.state()
    for k in got:
        np.testing.assert_array_equal(got[k], ref[k])
