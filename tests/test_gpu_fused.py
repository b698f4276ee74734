"""The residual fused into the first forward mode product (k_fused_res_fwd, enabled by
qn_set_fused_residual) against the separate kernels of the same solve and against the FP64
oracle (Sec. 4 eq. F_u and Sec. 4.1 eq. fin_inverse).

The fused kernel evaluates the fixed-point stencil and the float-pair nonlinear term of the
separate residual kernel and hands the same BF16 hi / lo values to the same sequence of
tensor-core products, so its iterates are those of the separate kernels: only the FP32
summation order of ||F||^2 differs, which can move a stop decision only when a relative
residual lies within ~1e-6 of the tolerance. The tests ask for the same iteration count
and max|U_fused - U_separate| <= 1e-13 max|U| (equality in practice), and, where the oracle
solve is affordable, the oracle's solution to 1e-9 max|U| with an FP64 relative residual
<= 1.05e-10 (the solve tolerance 1e-10 plus the FP32 rounding of the stop test's norm).
"""
import numpy as np
import pytest

import oracle as O
from paper_2502_03611_gb300.inputs import manufactured_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch  # noqa: F401
    from paper_2502_03611_gb300 import build as B
    from paper_2502_03611_gb300 import qn as Q
    B.build()
    Q.load_library()
    return Q


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def _solve(qn, n, f, fused, prec="bf16x3", lam=0.0, b=1.0, **opts):
    import torch
    ctx = qn.QnContext(3, n, prec, lam=lam, b=b)
    if fused:
        qn.qn_set_fused_residual(ctx, True)
    qn.qn_profile_enable(ctx, True)
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    o = dict(tol=1e-10, max_it=200)
    o.update(opts)
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), history_len=o["max_it"] + 1, **o)
    prof = qn.qn_profile_read(ctx)
    ctx.close()
    return res, hist, host(U).reshape(f.shape), prof


def _same_iterates(a, b):
    ra, _, Ua, _ = a
    rb, _, Ub, _ = b
    assert ra["iterations"] == rb["iterations"], (ra, rb)
    assert ra["status"] == rb["status"]
    assert np.abs(Ua - Ub).max() <= 1e-13 * np.abs(Ub).max()


@pytest.mark.parametrize("n", [127, 200, 255])
def test_fused_matches_separate_and_oracle(qn, n):
    """P = 128, 256, 256 (split halves of 64 and 128 positions); n = 200 has no middle
    point, the odd sizes have one (its difference slot stays 0)."""
    u, f = manufactured_problem(n, 3, seed=4)
    fz = _solve(qn, n, f, True)
    sp = _solve(qn, n, f, False)
    _same_iterates(fz, sp)
    res, hist, Ug, prof = fz
    assert res["status"] == 0 and res["rel"] <= 1e-10
    its = res["iterations"]
    assert its >= 2
    # iterations 1 .. its evaluate the residual in the fused kernel; their first products
    # (iterations 1 .. its - 1) are not separate launches
    assert prof["fused_launches"] == its, prof
    assert prof["mp_store_launches"] == sp[3]["mp_store_launches"] - (its - 1), (prof, sp[3])
    assert prof["launches"] == sp[3]["launches"] - (its - 1)
    assert prof["split_products"] == 1
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok
    rel = np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()


def test_fused_p384(qn):
    """P = 384: split halves of 192 positions (six pipeline stages per tile, two
    accumulators of 192 columns); against the separate kernels and the FP64 residual."""
    n = 383
    u, f = manufactured_problem(n, 3, seed=1)
    fz = _solve(qn, n, f, True)
    sp = _solve(qn, n, f, False)
    _same_iterates(fz, sp)
    res, _, Ug, prof = fz
    assert res["status"] == 0 and prof["fused_launches"] == res["iterations"]
    rel = np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel


def test_fused_511_identical_to_separate(qn):
    """The benchmark size (P = 512: split halves of 256, two accumulators of 256 columns, all
    of TMEM): with graph replay as the benchmark runs it, the same iterations and the same U
    bit for bit as the separate kernels, and the FP64 relative residual of U below 1.05e-10."""
    n = 511
    u, f = manufactured_problem(n, 3, seed=0)
    fz = _solve(qn, n, f, True, graph=True)
    sp = _solve(qn, n, f, False, graph=True)
    assert fz[0]["status"] == 0 and fz[0]["iterations"] == sp[0]["iterations"]
    assert np.array_equal(fz[2], sp[2])
    assert fz[3]["fused_launches"] == fz[0]["iterations"]
    rel = np.linalg.norm(O.residual(fz[2], f)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel


@pytest.mark.parametrize("lam,b", [(2.5, 0.5), (-3.0, 2.0)])
def test_fused_general_coefficients(qn, lam, b):
    """lam u + b u^3 with lam != 0 and b != 1 (the kernel's general forms)."""
    n = 127
    u, f = manufactured_problem(n, 3, seed=5, lam=lam, b=b)
    fz = _solve(qn, n, f, True, lam=lam, b=b)
    sp = _solve(qn, n, f, False, lam=lam, b=b)
    _same_iterates(fz, sp)
    Uo, ho, ok = O.qn_solve(f, tol=1e-10, lam=lam, b=b)
    assert ok
    Ug = fz[2]
    rel = np.linalg.norm(O.residual(Ug, f, lam=lam, b=b)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("headroom", [0, -6])
def test_fused_exact_path(qn, monkeypatch, headroom):
    """Less exponent headroom puts values above the fixed-point range; the rows whose
    stencil touches one take the exact per-point path (-6: most rows). The solve still
    reaches the oracle's solution."""
    n = 127
    u, f = manufactured_problem(n, 3, seed=2)
    monkeypatch.setenv("QN_RES_FX_HEADROOM", str(headroom))
    res, hist, Ug, prof = _solve(qn, n, f, True)
    assert prof["fused_launches"] >= 1
    Uo, ho, ok = O.qn_solve(f, tol=1e-10)
    assert ok and res["status"] == 0 and res["rel"] <= 1e-10
    rel = np.linalg.norm(O.residual(Ug, f)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert res["iterations"] <= len(ho) - 1 + 2


@pytest.mark.parametrize("max_it", [1, 2, 3])
def test_fused_first_iterations_match_separate(qn, max_it):
    """Stopped after 1, 2 or 3 iterations (iteration 1 takes its fixed-point exponent from
    the max|U_1| scan, later ones from the previous residual; from iteration 2 on the
    iterations replay from a CUDA graph): U equals the separate kernels' iterate."""
    n = 200
    u, f = manufactured_problem(n, 3, seed=8)
    fz = _solve(qn, n, f, True, tol=1e-30, max_it=max_it, graph=True)
    sp = _solve(qn, n, f, False, tol=1e-30, max_it=max_it, graph=True)
    assert fz[0]["status"] == qn.QN_ENOTCONV and fz[0]["iterations"] == max_it
    assert np.array_equal(fz[2], sp[2])


@pytest.mark.parametrize("sync_every,graph", [(1, False), (3, True)])
def test_fused_host_check_forms(qn, sync_every, graph):
    """Plain launches with a host check every iteration, and graph chunks of three."""
    n = 127
    u, f = manufactured_problem(n, 3, seed=3)
    fz = _solve(qn, n, f, True, sync_every=sync_every, graph=graph)
    sp = _solve(qn, n, f, False, sync_every=sync_every, graph=graph)
    _same_iterates(fz, sp)


def test_fused_bf16x6(qn):
    """A BF16X6 context: the fused kernel forms the first product; the backward products
    run at the six-product level as without it."""
    n = 255
    u, f = manufactured_problem(n, 3, seed=6)
    fz = _solve(qn, n, f, True, prec="bf16x6")
    sp = _solve(qn, n, f, False, prec="bf16x6")
    _same_iterates(fz, sp)
    assert fz[3]["x6_from"] == 0 and fz[3]["fused_launches"] == fz[0]["iterations"]


def test_fused_toggle_same_context(qn):
    """On, off and on again in one context with the same buffers (the cached iteration
    graphs are keyed on the form): each solve equals a fresh context's."""
    import torch
    n = 127
    u, f = manufactured_problem(n, 3, seed=7)
    ref = _solve(qn, n, f, False, graph=True)[2]
    ctx = qn.QnContext(3, n, "bf16x3")
    U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    fd = dev(f).reshape(-1)
    for on in (True, False, True):
        qn.qn_set_fused_residual(ctx, on)
        U.zero_()
        res, _ = qn.qn_solve(ctx, U, fd, tol=1e-10, graph=True)
        assert res["status"] == 0
        assert np.abs(host(U).reshape(f.shape) - ref).max() <= 1e-13 * np.abs(ref).max()
    ctx.close()


def test_fused_unsupported_contexts(qn):
    """Contexts the fused kernel does not cover refuse it (QN_EUNSUPPORTED) and solve as
    before; turning it off is always accepted."""
    cases = [dict(dim=3, n=127, precision="fp64"), dict(dim=2, n=255, precision="bf16x3"),
             dict(dim=3, n=127, precision="bf16x3", bc="neumann", length=1.0),
             dict(dim=3, n=600, precision="bf16x3")]
    for kw in cases:
        ctx = qn.QnContext(**kw)
        with pytest.raises(qn.QnError) as e:
            qn.qn_set_fused_residual(ctx, True)
        assert e.value.code == qn.QN_EUNSUPPORTED, kw
        qn.qn_set_fused_residual(ctx, False)
        ctx.close()
