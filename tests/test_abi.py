"""The C-ABI library loads, exports every symbol include/cmf.h declares, and
rejects bad arguments with error codes before touching the GPU (these calls
run on a machine without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cmf():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2004_11227_gb300 import cmf as m

    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "cmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cmf_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree(cmf):
    assert _declared() == sorted(cmf.EXPORTED)


def test_every_declared_symbol_is_exported(cmf):
    lib = ctypes.CDLL(cmf.library_path())
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_params_are_the_papers(cmf):
    p = cmf.default_params(cmf.RPADMM_EB, 2)
    assert (p.c, p.a, p.a1, p.rho, p.r) == (0.3, 8.0, 2.0, 1.9, 1.618)
    assert (p.sigma, p.tau, p.sweeps) == (0.2, 1.0, 1)
    q = cmf.default_params(cmf.RPDRQ, 4)
    assert (q.sigma, q.tau, q.a2) == (5.0, 0.4, 8.0)
    with pytest.raises(cmf.CmfError):
        cmf.default_params(7, 2)


def test_workspace_bytes(cmf):
    p = cmf.default_params(cmf.RPADMM_EB, 2)
    n1 = cmf.cmf_workspace_bytes(64, 64, 2, 64, p)
    n2 = cmf.cmf_workspace_bytes(128, 64, 2, 64, p)
    assert n1 > 5 * 64 * 64 * 4 and n2 > n1
    p16 = cmf.default_params(cmf.RPADMM_EB, 2, storage=cmf.F16)
    assert cmf.cmf_workspace_bytes(64, 64, 2, 64, p16) < n1
    assert cmf.cmf_workspace_bytes(64, 64, 4, 64, p) > n1
    assert cmf.cmf_workspace_bytes(0, 64, 2, 64, p) == 0
    assert cmf.cmf_workspace_bytes(64, 64, 2, 32, p) == 0


def _fake(n=8):
    # host memory standing in for device pointers: the calls below must fail
    # validation before any pointer is dereferenced or any kernel launched
    buf = (ctypes.c_float * (n * 64 + 256))()
    addr = ctypes.cast(buf, ctypes.c_void_p).value
    return (addr + 255) // 256 * 256, buf


def test_bad_arguments_rejected_without_launch(cmf):
    lib = cmf.lib()
    p = cmf.default_params(cmf.RPADMM_EB, 2)
    ptr, keep = _fake()
    P = ctypes.byref(p)
    args = lambda H, W, pitch, n, ws_bytes: (ptr, ptr, None, 0.5, H, W, pitch, P, n,
                                              ptr, ptr, ptr, ptr, ptr, ptr, ws_bytes, None)
    assert lib.cmf_iterate_binary(*args(0, 8, 8, 1, 1 << 20)) == cmf.EINVAL
    assert lib.cmf_iterate_binary(*args(8, 8, 4, 1, 1 << 20)) == cmf.EINVAL
    assert lib.cmf_iterate_binary(*args(8, 8, 8, -1, 1 << 30)) == cmf.EINVAL
    assert lib.cmf_iterate_binary(*args(8, 8, 8, 1, 16)) == cmf.ENOMEM
    # negative constant alpha
    assert lib.cmf_iterate_binary(ptr, ptr, None, -1.0, 8, 8, 8, P, 1, ptr, ptr, ptr, ptr, ptr,
                                  ptr, 1 << 20, None) == cmf.EINVAL
    # NULL state pointer
    assert lib.cmf_iterate_binary(ptr, ptr, None, 0.5, 8, 8, 8, P, 1, None, ptr, ptr, ptr, ptr,
                                  ptr, 1 << 20, None) == cmf.EINVAL
    for bad in [dict(algo=9), dict(storage=5), dict(impl=3), dict(sweeps=0), dict(c=0.0),
                dict(rho=2.0), dict(rho=0.0), dict(check_every=0), dict(sweeps=5),
                dict(costs=1), dict(costs=2)]:
        q = cmf.default_params(cmf.RPADMM_EB, 2)
        for k, v in bad.items():
            setattr(q, k, v)
        assert lib.cmf_iterate_binary(ptr, ptr, None, 0.5, 8, 8, 8, ctypes.byref(q), 1, ptr,
                                      ptr, ptr, ptr, ptr, ptr, 1 << 20, None) == cmf.EINVAL, bad
    # Potts: unknown cost input (0 float32 planes, 1 image and levels, 2 float16 planes)
    for bad_costs in (3, -1):
        pc = cmf.default_params(cmf.RPADMM_EB, 4)
        pc.costs = bad_costs
        assert lib.cmf_iterate_potts(ptr, 4, None, 0.5, 8, 8, 8, ctypes.byref(pc), 1, ptr, ptr,
                                     ptr, ptr, ptr, ptr, 1 << 20, None) == cmf.EINVAL
    # Potts: L out of range
    pp = cmf.default_params(cmf.RPADMM_EB, 4)
    assert lib.cmf_iterate_potts(ptr, 1, None, 0.5, 8, 8, 8, ctypes.byref(pp), 1, ptr, ptr, ptr,
                                 ptr, ptr, ptr, 1 << 20, None) == cmf.EINVAL
    assert lib.cmf_iterate_potts(ptr, 65, None, 0.5, 8, 8, 8, ctypes.byref(pp), 1, ptr, ptr,
                                 ptr, ptr, ptr, ptr, 1 << 20, None) == cmf.EINVAL
    out = (ctypes.c_double * 4)()
    assert lib.cmf_eval_binary(ptr, ptr, None, 0.5, 8, 8, 8, P, ptr, ptr, ptr, ptr, ptr, None,
                               ptr, 1 << 20, None) == cmf.EINVAL
    assert lib.cmf_solve_binary(ptr, ptr, None, 0.5, 8, 8, 8, P, ptr, ptr, ptr, ptr, ptr, None,
                                -1, None, ptr, 1 << 20, None) == cmf.EINVAL
    del keep, out


def test_rho_schedule_rejected_without_launch(cmf):
    """A relaxation schedule must be non-decreasing in (0, 2), end at or below
    rho, and belong to rpADMMII or rPDRQ; batches take none."""
    lib = cmf.lib()
    ptr, keep = _fake()

    def call(algo=cmf.RPADMM_EB, sched=(1.0, 1.5), n=None, null=False, rho=1.9):
        q = cmf.default_params(algo, 2)
        q.rho = rho
        q.set_rho_schedule(sched)
        if n is not None:
            q.rho_schedule_len = n
        if null:
            q.rho_schedule = None
        return lib.cmf_iterate_binary(ptr, ptr, None, 0.5, 8, 8, 8, ctypes.byref(q), 1, ptr, ptr,
                                      ptr, ptr, ptr, ptr, 1 << 20, None)

    for bad in [dict(sched=(1.5, 1.2)), dict(sched=(1.0, 2.0)), dict(sched=(0.0, 1.0)),
                dict(sched=(1.0, 1.95)), dict(sched=(1.0, float("nan"))),
                dict(algo=cmf.PADMM), dict(algo=cmf.RPADMM_FG), dict(algo=cmf.TY),
                dict(algo=cmf.CP), dict(null=True), dict(n=-1)]:
        assert call(**bad) == cmf.EINVAL, bad
    q = cmf.default_params(cmf.RPADMM_EB, 4)
    q.set_rho_schedule([1.2, 1.1])
    assert lib.cmf_iterate_potts(ptr, 4, None, 0.5, 8, 8, 8, ctypes.byref(q), 1, ptr, ptr, ptr,
                                 ptr, ptr, ptr, 1 << 20, None) == cmf.EINVAL
    inst = cmf.Instance()
    q = cmf.default_params(cmf.RPADMM_EB, 2)
    q.set_rho_schedule([1.0])
    assert lib.cmf_batch_workspace_bytes(ctypes.byref(inst), 1, ctypes.byref(q)) == 0
    del keep


def test_release_graphs_with_nothing_kept(cmf):
    # no graph was built in this process: nothing to destroy, no CUDA call
    assert cmf.lib().cmf_release_graphs() == cmf.OK


def test_status_strings(cmf):
    lib = cmf.lib()
    for s in range(6):
        assert lib.cmf_status_str(s)
    assert b"unknown" in lib.cmf_status_str(42)


def test_product_path_does_not_touch_oracle():
    """The CUDA package never imports the test oracle."""
    pkg = os.path.join(ROOT, "paper_2004_11227_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "synth.py", f


def test_rho_schedule_binding_keeps_its_array(cmf):
    import gc

    p = cmf.default_params(cmf.RPADMM_EB, 2, rho_schedule=[0.5, 1.0, 1.5])
    gc.collect()  # the list is gone; the params object holds its own copy
    assert p.rho_schedule_len == 3
    assert [p.rho_schedule[i] for i in range(3)] == [0.5, 1.0, 1.5]
    p.set_rho_schedule([])
    assert p.rho_schedule_len == 0 and not p.rho_schedule
    q = cmf.default_params(cmf.RPDRQ, 4)
    assert q.rho_schedule_len == 0 and not q.rho_schedule


def test_levels_container_leaves_callers_params_alone(cmf):
    """alloc_potts_levels works on a copy of the parameters (costs = 1), so
    the caller's object keeps costs = 0 and its relaxation schedule."""
    import numpy as np

    p = cmf.default_params(cmf.RPADMM_EB, 3, rho_schedule=[1.0, 1.5])
    I = np.zeros((4, 6), np.float32)
    s = cmf.alloc_potts_levels(I, [0.1, 0.5, 0.9], 0.3, p, device="cpu")
    assert p.costs == 0 and s.params.costs == 1
    assert s.params.rho_schedule_len == 2 and s.params.rho_schedule[1] == 1.5
    assert s.C.numel() == 4 * s.pitch + 3


def test_params_mirror_has_the_c_size(cmf):
    """cmf_default_params clears sizeof(cmf_params) bytes: the bytes right after
    the ctypes mirror must stay untouched, and the last field must be set."""
    n = ctypes.sizeof(cmf.Params)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    assert cmf.lib().cmf_default_params(2, 4, ctypes.cast(buf, ctypes.c_void_p)) == cmf.OK
    assert bytes(buf[n:]) == b"\xab" * 64
    p = cmf.Params.from_buffer_copy(bytes(buf[:n]))
    assert p.phase_storage == 0 and p.phase_gap == 0.0 and p.a2 == 8.0


def test_two_phase_parameters_validated(cmf):
    """A two-phase solve needs float32 buffers, a 16-bit first phase, a switch
    gap above the tolerance, a cold start and no relaxation schedule; binary
    solves have no two-phase form."""
    lib = cmf.lib()
    ptr = ctypes.c_void_p(256)
    hist = (ctypes.c_double * 10)()
    it = ctypes.c_int(0)

    def potts(**kw):
        q = cmf.default_params(cmf.RPADMM_EB, 4, **kw)
        return lib.cmf_solve_potts(ptr, 4, None, 0.5, 8, 8, 8, ctypes.byref(q), ptr, ptr, ptr,
                                   ptr, ptr, hist, 2, ctypes.byref(it), ptr, 1 << 30, None)

    for bad in [dict(phase_storage=1, phase_gap=1e-4),            # not above tol_gap
                dict(phase_storage=1, phase_gap=2e-3, storage=1),  # buffers not float32
                dict(phase_storage=3, phase_gap=2e-3),
                dict(phase_storage=1, phase_gap=2e-3, warm_start=1),
                dict(phase_storage=2, phase_gap=2e-3, rho_schedule=[1.5])]:
        assert potts(**bad) == cmf.EINVAL, bad
    q = cmf.default_params(cmf.RPADMM_EB, 2, phase_storage=1, phase_gap=2e-3)
    assert lib.cmf_solve_binary(ptr, ptr, None, 0.5, 8, 8, 8, ctypes.byref(q), ptr, ptr, ptr,
                                ptr, ptr, hist, 2, ctypes.byref(it), ptr, 1 << 30,
                                None) == cmf.EINVAL
    # the workspace grows by the two 16-bit phase sets
    p0 = cmf.default_params(cmf.RPADMM_EB, 4)
    p1 = cmf.default_params(cmf.RPADMM_EB, 4, phase_storage=1, phase_gap=2e-3)
    assert cmf.cmf_workspace_bytes(64, 64, 4, 64, p1) > cmf.cmf_workspace_bytes(64, 64, 4, 64, p0)


def test_batch_rows_validated_and_sized(cmf):
    """params.batch_rows (the strip band height of a batch): 0 or 8..24; the
    workspace grows with the item table as the bands get shorter; the batch
    autotuner validates before any launch."""
    lib = cmf.lib()
    ptr, keep = _fake(64 * 64)
    inst = cmf.Instance()
    inst.model, inst.L, inst.H, inst.W, inst.pitch = 1, 4, 1024, 64, 64
    inst.d_cost = inst.d_u = inst.d_qx = inst.d_qy = inst.d_p = inst.d_ps = ptr
    inst.alpha0 = 0.3

    def nbytes(rows):
        q = cmf.default_params(cmf.RPADMM_EB, 2)
        q.batch_rows = rows
        return lib.cmf_batch_workspace_bytes(ctypes.byref(inst), 1, ctypes.byref(q))

    for bad in (7, 25, -1):
        assert nbytes(bad) == 0, bad
    assert nbytes(0) == nbytes(24) > 0
    assert nbytes(8) > nbytes(12) >= nbytes(24)
    q = cmf.default_params(cmf.RPADMM_EB, 2)
    q.batch_rows = 30
    best = cmf.Params()
    ms = ctypes.c_double(0.0)
    assert lib.cmf_autotune_batch(ctypes.byref(inst), 1, ctypes.byref(q), ctypes.byref(best),
                                  ctypes.byref(ms), ptr, 1 << 20, None) == cmf.EINVAL
    del keep
