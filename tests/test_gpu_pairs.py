"""GPU parity of the two-iterations-per-launch warp-strip kernel (binary ADMM,
variant 4) against the FP64 oracle and against single-iteration launches.

A launch makes iteration k+1 on chip and iteration k+2 from it, rounding the
intermediate state to the storage type exactly where a single launch stores
it, so its result equals two single launches up to float32 contraction
order; against the oracle the float32 tolerances of the single kernel hold."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2004_11227_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_U = 1e-4
ADMM = [0, 1, 2, 4, 5]


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2004_11227_gb300 import cmf as m

    return m


def _gpu_run(cmf, inst, algo, n, **kw):
    p = cmf.default_params(algo, 2, **kw)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, n)
    torch.cuda.synchronize()
    return b


CASES = {
    "disk64": (synth.config1(), 200),            # 100 pairs
    "shapes37x54": (synth.config2(37, 54), 61),  # 30 pairs and one single launch
    "row1x68": (synth.random_binary(1, 68, seed=3, alpha=0.3), 40),
    "col45x2": (synth.random_binary(45, 2, seed=4, alpha=0.3), 40),
    "ragged70x130": (synth.random_binary(70, 130, seed=6, alpha=0.4, field_alpha=True), 52),
    "tall301x62": (synth.random_binary(301, 62, seed=7, alpha=0.3, field_alpha=True), 18),
    "wide6x1000": (synth.random_binary(6, 1000, seed=10, alpha=0.3, field_alpha=True), 24),
}


@pytest.mark.parametrize("algo", ADMM)
@pytest.mark.parametrize("case", list(CASES))
def test_pairs_match_oracle_f32(cmf, case, algo):
    inst, n = CASES[case]
    b = _gpu_run(cmf, inst, algo, n, variant=4)
    ref = O.binary_run(inst.costs[0], inst.costs[1], inst.alpha, O.default_params(algo, 2), n)
    got = b.state()
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= TOL_U, (k, err)


@pytest.mark.parametrize("storage,tol", [(0, 2e-6), (1, 2e-3), (2, 1.6e-2)])
@pytest.mark.parametrize("shape", [(70, 98), (5, 130), (130, 6), (200, 226)])
def test_pairs_equal_single_launches(cmf, storage, tol, shape):
    """Up to contraction order (float32) or one unit in the last place of a
    rounded intermediate (float16, bfloat16)."""
    inst = synth.random_binary(*shape, seed=91, alpha=0.3, field_alpha=True)
    for algo in ADMM:
        a = _gpu_run(cmf, inst, algo, 12, storage=storage, variant=2).state()
        b = _gpu_run(cmf, inst, algo, 12, storage=storage, variant=4).state()
        for k in a:
            err = np.abs(a[k] - b[k]).max()
            assert err <= tol, (algo, k, err)


@pytest.mark.parametrize("algo", [1, 2])
def test_pairs_anisotropic(cmf, algo):
    inst = synth.random_binary(41, 36, seed=8, alpha=0.3, field_alpha=True)
    b = _gpu_run(cmf, inst, algo, 40, aniso=1, variant=4)
    ref = O.binary_run(inst.costs[0], inst.costs[1], inst.alpha,
                       O.default_params(algo, 2, aniso=1), 40)
    assert np.abs(b.state()["u"] - ref["u"]).max() <= TOL_U


@pytest.mark.parametrize("algo", [2, 5])
def test_pairs_full_size_1024_windows(cmf, algo):
    """1024^2 in the benchmark's launch configuration: 36 iterations, then two
    pair launches; the oracle runs those 4 iterations on cropped windows whose
    margin covers 4 iterations of stencil reach."""
    inst = synth.config2()
    p = cmf.default_params(algo, 2, variant=4)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    cmf.cmf_iterate_binary(b, 36)
    torch.cuda.synchronize()
    W = b.W
    keys = ("u", "qx", "qy", "ps", "pt")
    before = {k: getattr(b, k)[:, :W].float().clone() for k in keys}
    cmf.cmf_iterate_binary(b, 4)
    torch.cuda.synchronize()
    after = {k: getattr(b, k)[:, :W].float().clone() for k in keys}
    po = O.default_params(algo, 2)
    alpha = inst.alpha_field()
    margin = 16
    for (r0, c0, h, w) in [(0, 0, 48, 48), (0, 1024 - 40, 40, 40), (1024 - 33, 0, 33, 64),
                           (1024 - 50, 1024 - 50, 50, 50), (500, 500, 64, 64),
                           (257, 771, 31, 45), (100, 54, 20, 8)]:
        R0, C0 = max(r0 - margin, 0), max(c0 - margin, 0)
        R1, C1 = min(r0 + h + margin, b.H), min(c0 + w + margin, b.W)
        st = {k: v[R0:R1, C0:C1].cpu().double().numpy() for k, v in before.items()}
        res = O.binary_run(inst.costs[0][R0:R1, C0:C1], inst.costs[1][R0:R1, C0:C1],
                           alpha[R0:R1, C0:C1], po, 4, st)
        for k in keys:
            got = after[k][r0:r0 + h, c0:c0 + w].cpu().double().numpy()
            ref = res[k][r0 - R0:r0 - R0 + h, c0 - C0:c0 - C0 + w]
            err = np.abs(got - ref).max()
            assert err <= 4e-5, (k, (r0, c0), err)


def test_pairs_equal_single_full_size_1024(cmf):
    inst = synth.config2()
    a = _gpu_run(cmf, inst, 2, 8, variant=2)
    b = _gpu_run(cmf, inst, 2, 8, variant=4)
    for k in ("u", "qx", "qy", "ps", "pt"):
        err = (getattr(a, k).float() - getattr(b, k).float()).abs().max().item()
        assert err <= 2e-6, (k, err)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_pairs_solve_matches_single_launch_solve(cmf, use_graph):
    inst = synth.config2(256, 256)
    out = []
    for variant in (2, 4):
        p = cmf.default_params(2, 2, tol_gap=1e-4, max_iter=20000, check_every=10,
                               variant=variant, use_graph=use_graph)
        b = cmf.alloc_binary(inst, p)
        out.append((cmf.cmf_solve_binary(b), b.state()))
    (s2, i2, h2), st2 = out[0]
    (s4, i4, h4), st4 = out[1]
    assert s2 == s4 == cmf.OK and i2 == i4
    np.testing.assert_allclose(h4[:, 3], h2[:, 3], atol=1e-6, rtol=0)
    E, D, gap, res = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha, st4,
                                   O.default_params(2, 2))
    assert gap <= 1.01e-4


def test_pairs_with_schedule_match_oracle(cmf):
    """Scheduled iterations run as single launches, the rest as pairs."""
    inst = synth.config2(48, 64)
    sched = np.linspace(0.5, 1.8, 13)
    b = _gpu_run(cmf, inst, 2, 41, variant=4, rho_schedule=sched)
    ref = O.binary_run(inst.costs[0], inst.costs[1], inst.alpha, O.default_params(2, 2), 41,
                       rho_schedule=sched)
    got = b.state()
    for k in ("u", "qx", "qy", "ps", "pt"):
        assert np.abs(got[k] - ref[k]).max() <= TOL_U, k


@pytest.mark.parametrize("aniso", [0, 1])
@pytest.mark.parametrize("shape,algo", [((1024, 1024), 2), ((70, 98), 2), ((130, 6), 1),
                                        ((5, 130), 4), ((301, 62), 5), ((64, 64), 0)])
def test_fused_certificates_match_certificate_kernel(cmf, shape, algo, aniso):
    """A solve's check runs in the chunk's last two-iteration launch; its
    history row equals what the certificate kernel and the oracle compute
    for the state the solve returns (one check: max_iter = check_every)."""
    inst = synth.random_binary(*shape, seed=77, alpha=0.35, field_alpha=True)
    for use_graph in (1, 0):
        p = cmf.default_params(algo, 2, aniso=aniso, tol_gap=1e-12, max_iter=20,
                               check_every=20, use_graph=use_graph)
        b = cmf.alloc_binary(inst, p)
        st, it, hist = cmf.cmf_solve_binary(b)
        assert st == cmf.NOT_CONVERGED and it == 20 and len(hist) == 1
        E, D, gap, res = hist[0, 1:]
        Ek, Dk, gapk, resk = cmf.cmf_eval_binary(b)
        assert abs(E - Ek) <= 1e-7 * abs(Ek) and abs(D - Dk) <= 1e-7 * abs(Dk) + 1e-9
        assert abs(gap - gapk) <= 1e-7 and abs(res - resk) <= 1e-5 * resk + 1e-7
        Eo, Do, gapo, reso = O.binary_eval(inst.costs[0], inst.costs[1], inst.alpha,
                                           b.state(), O.default_params(algo, 2, aniso=aniso))
        assert abs(E - Eo) <= 1e-5 * abs(Eo) and abs(D - Do) <= 1e-5 * abs(Do) + 1e-6
