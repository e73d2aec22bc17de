"""GPU parity of the binary solver (through the C ABI) against the FP64
oracle on the same seeded inputs.

Tolerances (float32 state, float32 arithmetic): max |u - u_oracle| <= 1e-4
and flows within 1e-4 after a fixed iteration count; certificates (E, D)
within 1e-5 relative and the relative gap within 1e-6 absolute of the
oracle's evaluation of the same state; a solve to gap 1e-4 is certified by the
oracle and its thresholded labelling agrees with the oracle's converged one
on >= 99.9% of pixels.  float16 / bfloat16 flow storage is checked with
tolerances derived from their unit roundoff (2^-11 and 2^-8)."""
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
        "disk64": (synth.config1(), 200),
        "shapes37x53": (synth.config2(37, 53), 60),
        "row1x67": (synth.random_binary(1, 67, seed=3, alpha=0.3), 40),
        "col45x1": (synth.random_binary(45, 1, seed=4, alpha=0.3), 40),
        "tiny2x3": (synth.random_binary(2, 3, seed=5, alpha=0.2, field_alpha=True), 30),
        "ragged70x33": (synth.random_binary(70, 33, seed=6, alpha=0.4, field_alpha=True), 50),
    }


def _gpu_run(cmf, inst, algo, n, **kw):
    p = cmf.default_params(algo, 2, **kw)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, n)
    torch.cuda.synchronize()
    return b


def _oracle_run(inst, algo, n, aniso=0, sweeps=1):
    p = O.default_params(algo, 2, aniso=aniso, sweeps=sweeps)
    return O.binary_run(inst.costs[0], inst.costs[1], inst.alpha, p, n), p


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("case", list(_cases()))
def test_iterations_match_oracle_f32(cmf, case, algo, impl):
    inst, n = _cases()[case]
    b = _gpu_run(cmf, inst, algo, n, impl=impl)
    got = b.state()
    ref, _ = _oracle_run(inst, algo, n)
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


@pytest.mark.parametrize("algo", ALGOS)
def test_anisotropic_and_multisweep(cmf, algo):
    inst = synth.random_binary(29, 41, seed=8, alpha=0.35, field_alpha=True)
    for aniso, sweeps in [(1, 1), (0, 3)]:
        b = _gpu_run(cmf, inst, algo, 40, aniso=aniso, sweeps=sweeps)
        ref, _ = _oracle_run(inst, algo, 40, aniso=aniso, sweeps=sweeps)
        assert np.abs(b.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("algo", ALGOS)
def test_fused_equals_plain(cmf, algo):
    inst = synth.config2(96, 80)
    a = _gpu_run(cmf, inst, algo, 30, impl=0).state()
    b = _gpu_run(cmf, inst, algo, 30, impl=1).state()
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= 1e-5, k


@pytest.mark.parametrize("shape", [(70, 90), (70, 91), (1, 64), (131, 2), (300, 250)])
@pytest.mark.parametrize("algo", ALGOS)
def test_certificates_match_oracle(cmf, algo, shape):
    """Even widths go through the warp-strip certificate kernel, odd ones
    through the tile kernel; both against the oracle's evaluation."""
    inst = synth.config2(*shape)
    b = _gpu_run(cmf, inst, algo, 25)
    E, D, gap, res = cmf.cmf_eval_binary(b)
    st = b.state()
    p = O.default_params(algo, 2)
    Eo, Do, gapo, reso = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st, p)
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert abs(D - Do) <= 1e-5 * abs(Eo)
    assert abs(gap - gapo) <= 1e-6 + 1e-4 * abs(gapo)
    assert abs(res - reso) <= 1e-4 * reso + 1e-6


@pytest.mark.parametrize("storage,tol", [(1, 3e-3), (2, 3e-2)])
@pytest.mark.parametrize("algo", [0, 2, 3])
def test_half_storage_tracks_oracle(cmf, storage, tol, algo):
    inst = synth.config1()
    b = _gpu_run(cmf, inst, algo, 30, storage=storage)
    ref, _ = _oracle_run(inst, algo, 30)
    assert np.abs(b.state()["u"] - ref["u"]).max() <= tol


@pytest.mark.parametrize("algo", ALGOS)
def test_solve_certified_by_oracle(cmf, algo):
    inst = synth.config2(160, 192)
    p = cmf.default_params(algo, 2, tol_gap=1e-4, max_iter=20000, check_every=10)
    b = cmf.alloc_binary(inst, p)
    status, iters, hist = cmf.cmf_solve_binary(b)
    assert status == cmf.OK and hist[-1, 3] <= 1e-4 and iters == int(hist[-1, 0])
    st = b.state()
    po = O.default_params(algo, 2)
    E, D, gap, res = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st, po)
    assert gap <= 1.01e-4
    # same algorithm and stopping rule in FP64: the labellings agree
    ref, it_ref, _ = O.solve(inst, algo, tol=1e-4, max_iter=40000, check_every=10)
    agree = np.mean(O.binary_labels(st["u"]) == O.binary_labels(ref["u"]))
    assert agree >= 0.999, agree
    # and both are close to the converged labelling
    opt, _, _ = O.solve(inst, algo, tol=1e-7, max_iter=40000)
    assert np.mean(O.binary_labels(st["u"]) == O.binary_labels(opt["u"])) >= 0.99


@pytest.mark.parametrize("storage", [1, 2])
def test_half_storage_solve_reaches_gap(cmf, storage):
    inst = synth.config2(128, 128)
    p = cmf.default_params(2, 2, storage=storage, tol_gap=1e-4, max_iter=20000)
    b = cmf.alloc_binary(inst, p)
    status, iters, hist = cmf.cmf_solve_binary(b)
    assert status == cmf.OK
    st = b.state()
    E, D, gap, res = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st,
                                   O.default_params(2, 2))
    assert gap <= 2e-4
    ref, _, _ = O.solve(inst, 2, tol=1e-4, max_iter=40000)
    assert np.mean(O.binary_labels(st["u"]) == O.binary_labels(ref["u"])) >= 0.999


def test_warm_start_split_equals_single_run(cmf):
    inst = synth.config2(64, 96)
    a = _gpu_run(cmf, inst, 2, 40).state()
    p = cmf.default_params(2, 2)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, 17)
    cmf.cmf_iterate_binary(b, 23)
    torch.cuda.synchronize()
    s = b.state()
    for k in a:
        np.testing.assert_array_equal(a[k], s[k])


def _window_step_check(cmf, inst, algo, k_before, windows, margin=8, variant=0):
    """Full-size state: GPU runs k_before iterations, then one more; the
    oracle runs that last iteration on cropped windows (with a margin that
    covers the iteration's stencil reach) and the window interiors must
    match element by element."""
    p = cmf.default_params(algo, 2, variant=variant)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, k_before)
    torch.cuda.synchronize()
    W = b.W
    before = {k: getattr(b, k)[:, :W].float().clone() for k in ("u", "qx", "qy", "ps", "pt")}
    cmf.cmf_iterate_binary(b, 1)
    torch.cuda.synchronize()
    after = {k: getattr(b, k)[:, :W].float().clone() for k in ("u", "qx", "qy", "ps", "pt")}
    po = O.default_params(algo, 2)
    alpha = inst.alpha_field()
    for (r0, c0, h, w) in windows:
        R0, C0 = max(r0 - margin, 0), max(c0 - margin, 0)
        R1, C1 = min(r0 + h + margin, b.H), min(c0 + w + margin, b.W)
        if (R0 + C0) % 2:  # keep the crop's red/black colouring that of the grid
            if R0 > 0:
                R0 -= 1
            else:
                C0 -= 1
        st = {k: v[R0:R1, C0:C1].cpu().double().numpy() for k, v in before.items()}
        res = O.binary_run(inst.costs[0][R0:R1, C0:C1], inst.costs[1][R0:R1, C0:C1],
                           alpha[R0:R1, C0:C1], po, 1, st)
        for k in res:
            # interior = the window, minus a margin wherever the crop is not the grid edge
            ri0 = r0 - R0 if R0 > 0 else 0
            ci0 = c0 - C0 if C0 > 0 else 0
            got = after[k][r0:r0 + h, c0:c0 + w].cpu().double().numpy()
            ref = res[k][ri0:ri0 + h, ci0:ci0 + w]
            err = np.abs(got - ref).max()
            assert err <= 2e-5, (k, (r0, c0), err)


@pytest.mark.parametrize("algo", ALGOS)
def test_full_size_1024_windows(cmf, algo):
    """1024^2 (the benchmark workload) in the benchmark's launch
    configuration: windows at corners, edges, the centre and a ragged spot."""
    inst = synth.config2()
    wins = [(0, 0, 48, 48), (0, 1024 - 40, 40, 40), (1024 - 33, 0, 33, 64),
            (1024 - 50, 1024 - 50, 50, 50), (500, 500, 64, 64), (257, 771, 31, 45)]
    _window_step_check(cmf, inst, algo, 37, wins)


@pytest.mark.parametrize("impl", [0, 1])
@pytest.mark.parametrize("algo", [0, 3])
def test_graph_solve_equals_host_loop(cmf, algo, impl):
    """The device-driven solve loop (graph with a conditional node) runs the
    same kernels in the same order as the host loop: identical state, history
    and iteration count; a max_iter cap yields NOT_CONVERGED on both paths."""
    inst = synth.config2(80, 112)
    out = []
    for use_graph in (1, 0):
        p = cmf.default_params(algo, 2, impl=impl, use_graph=use_graph, tol_gap=1e-4,
                               max_iter=4000, check_every=10)
        b = cmf.alloc_binary(inst, p)
        out.append((cmf.cmf_solve_binary(b), b.state()))
    (s1, i1, h1), st1 = out[0]
    (s0, i0, h0), st0 = out[1]
    assert s1 == s0 == cmf.OK and i1 == i0
    np.testing.assert_array_equal(h1, h0)
    for k in st0:
        np.testing.assert_array_equal(st1[k], st0[k])
    for use_graph in (1, 0):
        p = cmf.default_params(algo, 2, impl=impl, use_graph=use_graph, tol_gap=1e-12,
                               max_iter=40, check_every=10)
        b = cmf.alloc_binary(inst, p)
        st, it, hist = cmf.cmf_solve_binary(b)
        assert st == cmf.NOT_CONVERGED and it == 40 and len(hist) == 4


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("variant", [8, 16, 32])
@pytest.mark.parametrize("shape", [(70, 97), (5, 130), (131, 33)])
def test_tma_tiles_match_smem_tiles(cmf, storage, variant, shape):
    """The persistent TMA-staged fused ADMM kernel computes what the
    shared-memory tile kernel computes (only the staging differs)."""
    inst = synth.random_binary(*shape, seed=90, alpha=0.3, field_alpha=True)
    for algo in (0, 2):
        a = _gpu_run(cmf, inst, algo, 9, storage=storage, variant=1).state()
        b = _gpu_run(cmf, inst, algo, 9, storage=storage, variant=variant).state()
        tol = 1e-6 if storage == 0 else 1e-2
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= tol, k


def test_autotune_picks_a_converging_configuration(cmf, tmp_path):
    inst = synth.config2(200, 240)
    for algo in (2, 3):
        p = cmf.default_params(algo, 2, tol_gap=1e-4, max_iter=4000)
        b = cmf.alloc_binary(inst, p)
        best, ms = cmf.cmf_autotune_binary(b)
        assert ms > 0 and best.algo == algo
        assert best.variant in (1, 2, 4, 8, 16, 32) if algo != 3 else best.sweeps in (1, 2, 3)
        q = cmf.tuned_params(b, cache_path=str(tmp_path / "tune.json"))
        assert (tmp_path / "tune.json").exists()
        b2 = cmf.alloc_binary(inst, q)
        st, it, hist = cmf.cmf_solve_binary(b2)
        assert st == cmf.OK


# ---- warp-strip kernel (variant 2) ---------------------------------------------

STRIP_CASES = {
    "disk64": (synth.config1(), 200),
    "shapes37x54": (synth.config2(37, 54), 60),
    "row1x68": (synth.random_binary(1, 68, seed=3, alpha=0.3), 40),
    "col45x2": (synth.random_binary(45, 2, seed=4, alpha=0.3), 40),
    "ragged70x130": (synth.random_binary(70, 130, seed=6, alpha=0.4, field_alpha=True), 51),
    "tall301x62": (synth.random_binary(301, 62, seed=7, alpha=0.3, field_alpha=True), 17),
}


@pytest.mark.parametrize("algo", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("case", list(STRIP_CASES))
def test_strip_matches_oracle_f32(cmf, case, algo):
    inst, n = STRIP_CASES[case]
    b = _gpu_run(cmf, inst, algo, n, variant=2)
    got = b.state()
    ref, _ = _oracle_run(inst, algo, n)
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


@pytest.mark.parametrize("algo", [1, 2])
def test_strip_anisotropic(cmf, algo):
    inst = synth.random_binary(41, 36, seed=8, alpha=0.3, field_alpha=True)
    b = _gpu_run(cmf, inst, algo, 40, aniso=1, variant=2)
    ref, _ = _oracle_run(inst, algo, 40, aniso=1)
    assert np.abs(b.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("shape", [(70, 98), (5, 130), (130, 6)])
def test_strip_matches_smem_tiles_half(cmf, storage, shape):
    inst = synth.random_binary(*shape, seed=91, alpha=0.3, field_alpha=True)
    for algo in (0, 2, 3):
        a = _gpu_run(cmf, inst, algo, 9, storage=storage, variant=1).state()
        b = _gpu_run(cmf, inst, algo, 9, storage=storage, variant=2).state()
        for k in a:
            assert np.abs(a[k] - b[k]).max() <= 1e-2, k


def test_strip_rejects_odd_width(cmf):
    inst = synth.random_binary(20, 33, seed=9, alpha=0.3)
    p = cmf.default_params(2, 2, variant=2)
    b = cmf.alloc_binary(inst, p)
    with pytest.raises(cmf.CmfError):
        cmf.cmf_iterate_binary(b, 2)


@pytest.mark.parametrize("algo", [1, 2])
def test_strip_full_size_1024_windows(cmf, algo):
    inst = synth.config2()
    wins = [(0, 0, 48, 48), (0, 1024 - 40, 40, 40), (1024 - 33, 0, 33, 64),
            (1024 - 50, 1024 - 50, 50, 50), (500, 500, 64, 64), (257, 771, 31, 45)]
    _window_step_check(cmf, inst, algo, 37, wins, variant=2)


def test_strip_matches_tma_full_size_1024(cmf):
    inst = synth.config2()
    a = _gpu_run(cmf, inst, 2, 6, variant=16)
    b = _gpu_run(cmf, inst, 2, 6, variant=2)
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = (getattr(a, k).float() - getattr(b, k).float()).abs().max().item()
        assert err <= 1e-5, (k, err)


def test_strip_solve_certified(cmf):
    inst = synth.config2(256, 256)
    p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=20000, check_every=10, variant=2)
    b = cmf.alloc_binary(inst, p)
    status, iters, hist = cmf.cmf_solve_binary(b)
    assert status == cmf.OK and hist[-1, 3] <= 1e-4
    st = b.state()
    E, D, gap, res = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st,
                                   O.default_params(2, 2))
    assert gap <= 1.01e-4


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("algo", [2, 3])
def test_strip_certificates_half_storage(cmf, storage, algo):
    inst = synth.config2(64, 96)
    b = _gpu_run(cmf, inst, algo, 25, storage=storage)
    E, D, gap, res = cmf.cmf_eval_binary(b)
    Eo, Do, gapo, reso = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, b.state(),
                                       O.default_params(algo, 2))
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert abs(D - Do) <= 1e-5 * abs(Eo)


@pytest.mark.parametrize("aniso", [0, 1])
def test_strip_certificates_full_size(cmf, aniso):
    """1024^2 state after some iterations: strip certificates against the
    oracle's evaluation of the same state (FP64, whole grid)."""
    inst = synth.config2()
    b = _gpu_run(cmf, inst, 2, 30, aniso=aniso)
    E, D, gap, res = cmf.cmf_eval_binary(b)
    Eo, Do, gapo, reso = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, b.state(),
                                       O.default_params(2, 2, aniso=aniso))
    assert abs(E - Eo) <= 1e-6 * abs(Eo)
    assert abs(D - Do) <= 1e-6 * abs(Eo)
    assert abs(res - reso) <= 1e-5 * reso + 1e-6


@pytest.mark.parametrize("sweeps", [1, 2, 3, 4])
@pytest.mark.parametrize("aniso", [0, 1])
def test_strip_dr_sweeps(cmf, sweeps, aniso):
    """rPDRQ with 1..4 symmetric red-black sweeps per iteration through the
    pipelined strip kernel (1 + 2 sweeps half-sweep stages) against the
    oracle; the grid spans several strips and bands."""
    inst = synth.random_binary(150, 130, seed=92, alpha=0.35, field_alpha=True)
    b = _gpu_run(cmf, inst, 3, 21, variant=2, sweeps=sweeps, aniso=aniso)
    ref, _ = _oracle_run(inst, 3, 21, aniso=aniso, sweeps=sweeps)
    got = b.state()
    for k in ("u", "qx", "qy", "ps", "pt"):
        assert np.abs(got[k] - ref[k]).max() <= TOL_U, k
