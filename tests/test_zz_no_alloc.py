"""The allocation-free certificate entry point, cmf_eval_binary_noalloc.

It serves callers that cannot allocate device memory when they need a
certificate (for example a plug-in that only receives a stream and the
solver's buffers from a host application that owns every allocation).  Its
scratch is a static device array inside the library.  This file is collected last so that a failure here leaves every
other test already run; it passes alone in a fresh process and after the
other tests (the shared static array keeps nothing a later call depends on).
"""
import ctypes

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


@pytest.mark.parametrize("algo", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("W", [168, 171])  # even: warp-strip certificates; odd: tiles
def test_noalloc_matches_workspace_eval_two_calls(cmf, algo, storage, W):
    inst = synth.config2(200, W)
    p = cmf.default_params(algo, 2, storage=storage)
    b = cmf.alloc_binary(inst, p)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        cmf.cmf_init_binary(b, stream=side)
        for n in (9, 14):  # two calls in a row on two different states
            cmf.cmf_iterate_binary(b, n, stream=side)
            ref = cmf.cmf_eval_binary(b, stream=side)
            got = cmf.cmf_eval_binary_noalloc(b, stream=side)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_noalloc_refuses_a_capturing_stream(cmf):
    """Inside a stream capture the call returns CMF_EINVAL before launching
    anything, and the capture it was called in still instantiates and runs."""
    inst = synth.config2(64, 64)
    p = cmf.default_params(2, 2)
    b = cmf.alloc_binary(inst, p)
    cmf.cmf_init_binary(b)
    torch.cuda.synchronize()
    x = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    out = (ctypes.c_double * 4)()
    with torch.cuda.graph(g, stream=s):
        st = cmf.lib().cmf_eval_binary_noalloc(*b._common(), *b._state_ptrs(), out,
                                               s.cuda_stream)
        x.add_(1.0)
    assert st == cmf.EINVAL
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 2.0
    ref = cmf.cmf_eval_binary(b)
    np.testing.assert_allclose(cmf.cmf_eval_binary_noalloc(b), ref, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_grids_beyond_its_scratch(cmf):
    # 4097 x 4096 needs 129 x 128 > 16384 certificate blocks; validation
    # rejects it before any launch, so the pointers are never dereferenced
    p = cmf.default_params(2, 2)
    out = (ctypes.c_double * 4)()
    fake = torch.empty(1, device="cuda").data_ptr()
    st = cmf.lib().cmf_eval_binary_noalloc(fake, fake, None, 0.5, 4097, 4096, 4096,
                                           ctypes.byref(p), fake, fake, fake, fake, fake,
                                           out, None)
    assert st == cmf.EINVAL
