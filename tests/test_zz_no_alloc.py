"""qn_residual_noalloc: the residual entry point for callers that cannot
allocate device memory (their device memory belongs entirely to another
allocator or budget, or they are in a section that must not allocate). It
keeps its scratch in a fixed array inside libqn instead of a context.

Checked through the C-ABI against qn_residual (which uses a context's
workspace) on two calls in a row, so that the shared scratch left over from
the first call cannot leak into the second. The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_03611_gb300.inputs import random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn
    B.build()
    L = qn.load_library()
    L.qn_residual_noalloc.restype = ctypes.c_int
    L.qn_residual_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(qn.QnStats), ctypes.c_void_p]
    return L


@pytest.mark.parametrize("dim,n,lam,b", [(3, 65, 0.0, 1.0), (2, 100, 0.4, 2.0), (3, 255, 0.0, 1.0)])
def test_noalloc_residual_matches_context_residual(lib, dim, n, lam, b):
    import torch
    from paper_2502_03611_gb300 import qn
    ctx = qn.QnContext(dim, n, "fp64", lam=lam, b=b)
    N = n ** dim
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    R_ref = torch.empty(N, dtype=torch.float64, device="cuda")
    outs = []
    for call in range(2):
        # a different U each call, so a stale scratch value would show
        U = torch.from_numpy(random_field((N,), seed=10 + call + n)).cuda()
        f = torch.from_numpy(random_field((N,), seed=20 + call + n) * 30.0).cuda()
        want = qn.qn_residual(ctx, U, f, R_ref)
        R = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        st = qn.QnStats()
        rc = lib.qn_residual_noalloc(dim, n, lam, b, ctypes.c_void_p(U.data_ptr()),
                                     ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                     ctypes.byref(st), stream)
        assert rc == qn.QN_OK, qn.qn_last_error()
        got = st.as_dict()
        scale = float(R_ref.abs().max())
        assert float((R - R_ref).abs().max()) <= 1e-13 * scale
        for k in ("res_norm", "f_norm", "fu_min", "fu_max", "beta", "rel"):
            assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-300), k
        outs.append(got["res_norm"])
    assert outs[0] != outs[1]


def _call(lib, dim, n, lam, b, U, f, R, st, stream):
    return lib.qn_residual_noalloc(dim, n, lam, b, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(R.data_ptr()) if R is not None else None,
                                   ctypes.byref(st), stream)


def test_noalloc_without_output_and_without_allocating(lib):
    """R = NULL returns the statistics alone; after a first call (which loads the
    kernels and looks up the scratch address) further calls leave the device's
    free memory and torch's pool unchanged: the entry point allocates nothing."""
    import torch
    from paper_2502_03611_gb300 import qn
    dim, n, lam, b = 3, 96, 0.2, 1.5
    N = n ** dim
    ctx = qn.QnContext(dim, n, "fp64", lam=lam, b=b)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    U = torch.from_numpy(random_field((N,), seed=31)).cuda()
    f = torch.from_numpy(random_field((N,), seed=32) * 10.0).cuda()
    want = qn.qn_residual(ctx, U, f)
    st = qn.QnStats()
    assert _call(lib, dim, n, lam, b, U, f, None, st, stream) == qn.QN_OK, qn.qn_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        st = qn.QnStats()
        assert _call(lib, dim, n, lam, b, U, f, None, st, stream) == qn.QN_OK, qn.qn_last_error()
        got = st.as_dict()
        for k in ("res_norm", "f_norm", "fu_min", "fu_max", "beta", "rel"):
            assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-300), k
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_out_of_range(lib):
    from paper_2502_03611_gb300 import qn
    st = qn.QnStats()
    assert lib.qn_residual_noalloc(3, 2048, 0.0, 1.0, None, None, None, ctypes.byref(st), None) == qn.QN_EINVAL
    assert "1024" in qn.qn_last_error()
    assert lib.qn_residual_noalloc(4, 10, 0.0, 1.0, None, None, None, ctypes.byref(st), None) == qn.QN_EINVAL
