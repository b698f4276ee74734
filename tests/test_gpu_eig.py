"""The nonlinear eigenproblem (Sec. 4.4; Sec. 6.3 Example 2: -Lap u + 1600 u^3 + V u = lambda u
on (-8,8)^3, u = 0 on the boundary) through qn_eig_solve, against the oracle's
qn_eig_solve.

Tolerances: lambda to 1e-9 relative and U to 1e-7 max|U| (the eigen-residual tolerance
1e-10 bounds the eigenvector error by about 1e-10 lambda / gap; run to 1e-13, U agrees to
1e-9 max|U|, test_eig_example2_tight_tolerance_eigenvector); equal iteration counts
within 2 (FP64) or 5 % (BF16X3, whose inverse differs from the oracle's by ~1e-5 per
iteration while the residual, Rayleigh quotient, update and normalisation stay FP64).
"""
import math

import numpy as np
import pytest

from oracle import qn_oracle_bc as ob
from paper_2502_03611_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALPHA = I.EX2_ALPHA


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


def _ex2_ctx(qn, n, prec):
    v, h, x = I.ex2_problem(n)
    ctx = qn.QnContext(3, n, prec, lam=0.0, b=ALPHA, bc="dirichlet", length=I.EX2_LENGTH, potential=v)
    return ctx, v, h


def _gpu_eig(qn, ctx, U0, graph=False, history_len=0, **kw):
    U = dev(U0).reshape(-1).clone()
    res, hist = qn.qn_eig_solve(ctx, U, graph=graph, history_len=history_len, **kw)
    return res, hist, host(U).reshape(U0.shape)


def _check(res, Ug, lam_o, Uo, its_o, prec):
    assert res["status"] == 0 and res["rel"] <= 1e-10, res
    assert res["lambda"] == pytest.approx(lam_o, rel=1e-9)
    assert np.abs(Ug - Uo).max() <= 1e-7 * np.abs(Uo).max()
    if prec == "fp64":
        assert abs(res["iterations"] - its_o) <= 2
    else:
        assert abs(res["iterations"] - its_o) <= max(3, 0.05 * its_o)


@pytest.mark.parametrize("n,prec", [(9, "fp64"), (15, "fp64"), (15, "bf16x3"), (31, "bf16x3")])
def test_eig_example2_matches_oracle(qn, n, prec):
    ctx, v, h = _ex2_ctx(qn, n, prec)
    U0 = I.ex2_start(n, seed=1)
    res, hist, Ug = _gpu_eig(qn, ctx, U0, history_len=5000)
    V = ob.potential(v, 3, n)
    Uo, lam_o, ho, ok = ob.qn_eig_solve(U0, h, "dirichlet", b=ALPHA, V=V)
    assert ok
    _check(res, Ug, lam_o, Uo, len(ho) - 1, prec)
    m = ob.mass_weights(n, 3, h, "dirichlet")
    assert float(np.sum(m * Ug * Ug)) == pytest.approx(1.0, rel=1e-12)
    # the first iterate (same start) matches the oracle's lambda_0 and beta_0 (beta from the
    # FP32 extremes of lam + 3 b U^2 + V: it only chooses the shift)
    assert hist[0]["lambda"] == pytest.approx(ho[0]["lambda"], rel=1e-12)
    assert hist[0]["beta"] == pytest.approx(ho[0]["beta"], rel=1e-6)


@pytest.mark.parametrize("n,prec", [(15, "fp64"), (15, "bf16x3"), (31, "bf16x3")])
def test_eig_example2_tight_tolerance_eigenvector(qn, n, prec):
    """The eigenvector to 1e-9 max|U|. At the stop rule's 1e-10 two converged iterates may
    differ by about 1e-10 lambda / gap (the iteration contracts at ~0.97 per step, so the
    gap is small), which is why the other tests compare U at 1e-7. Run both sides to
    ||F|| / |lambda| <= 1e-13 instead: U then agrees to 1e-9 max|U| and lambda to 1e-12."""
    ctx, v, h = _ex2_ctx(qn, n, prec)
    U0 = I.ex2_start(n, seed=1)
    res, hist, Ug = _gpu_eig(qn, ctx, U0, tol=1e-13, max_it=4096)
    assert res["status"] == 0 and res["rel"] <= 1e-13, res
    Uo, lam_o, ho, ok = ob.qn_eig_solve(U0, h, "dirichlet", b=ALPHA, V=ob.potential(v, 3, n), tol=1e-13,
                                        max_it=5000)
    assert ok
    assert res["lambda"] == pytest.approx(lam_o, rel=1e-12)
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_eig_neumann_matches_oracle(qn, prec):
    """Zero normal derivative (Sec. 4.4's setting): trapezoid-weighted mass, cosine pairs."""
    n, L = 17, 6.0
    h = ob.mesh_width(n, "neumann", L)
    x = -L / 2 + h * np.arange(n)
    tabs = np.stack([3.0 * x * x, 4.0 * (x - 0.5) ** 2, 2.0 * x * x])
    ctx = qn.QnContext(3, n, prec, lam=0.5, b=40.0, bc="neumann", length=L, potential=tabs)
    g = np.cos(0.3 * x)
    U0 = g[None, None, :] * g[None, :, None] * g[:, None, None]
    res, hist, Ug = _gpu_eig(qn, ctx, U0)
    Uo, lam_o, ho, ok = ob.qn_eig_solve(U0, h, "neumann", lam=0.5, b=40.0, V=ob.potential(tabs, 3, n))
    assert ok
    _check(res, Ug, lam_o, Uo, len(ho) - 1, prec)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_eig_2d_matches_oracle(qn, prec):
    n, L = 40, 10.0
    h = ob.mesh_width(n, "dirichlet", L)
    x = -L / 2 + h * np.arange(1, n + 1)
    tabs = np.stack([x * x, 0.5 * (x - 1.0) ** 2])
    ctx = qn.QnContext(2, n, prec, lam=0.0, b=200.0, bc="dirichlet", length=L, potential=tabs)
    g = np.cos(math.pi * x / L)
    U0 = g[:, None] * g[None, :]
    res, hist, Ug = _gpu_eig(qn, ctx, U0)
    Uo, lam_o, ho, ok = ob.qn_eig_solve(U0, h, "dirichlet", b=200.0, V=ob.potential(tabs, 2, n))
    assert ok
    _check(res, Ug, lam_o, Uo, len(ho) - 1, prec)


def test_eig_split_products_match_dense(qn, monkeypatch):
    """n = 65 (P = 128): the residual pass writes the reflection-split order and the split
    products run; against the dense products."""
    n = 65
    U0 = I.ex2_start(n, seed=2)
    outs = []
    for split in ("1", "0"):
        monkeypatch.setenv("QN_SPLIT", split)
        ctx, v, h = _ex2_ctx(qn, n, "bf16x3")
        qn.qn_profile_enable(ctx, True)
        res, _, Ug = _gpu_eig(qn, ctx, U0)
        prof = qn.qn_profile_read(ctx)
        assert prof["split_products"] == (1 if split == "1" else 0)
        assert res["status"] == 0
        outs.append((res, Ug))
    assert outs[0][0]["lambda"] == pytest.approx(outs[1][0]["lambda"], rel=1e-10)
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-7 * np.abs(outs[1][1]).max()
    # the oracle's eigen-residual of the split result
    v, h, x = I.ex2_problem(n)
    F, lam = ob.eig_residual(outs[0][1], h, "dirichlet", 0.0, ALPHA, ob.potential(v, 3, n))
    m = ob.mass_weights(n, 3, h, "dirichlet")
    assert math.sqrt(float(np.sum(m * F * F))) / abs(lam) <= 1.05e-10


def test_eig_graph_replay_bitwise(qn):
    n = 33
    U0 = I.ex2_start(n, seed=3)
    r = []
    for graph in (False, True):
        ctx, v, h = _ex2_ctx(qn, n, "bf16x3")
        res, _, Ug = _gpu_eig(qn, ctx, U0, graph=graph)
        r.append((res, Ug))
    assert r[0][0]["iterations"] == r[1][0]["iterations"]
    assert np.array_equal(r[0][1], r[1][1])


def test_eig_not_converged_status(qn):
    ctx, v, h = _ex2_ctx(qn, 15, "bf16x3")
    res, _, Ug = _gpu_eig(qn, ctx, I.ex2_start(15), max_it=5)
    assert res["status"] == qn.QN_ENOTCONV and res["iterations"] == 5
    m = ob.mass_weights(15, 3, h, "dirichlet")
    assert float(np.sum(m * Ug * Ug)) == pytest.approx(1.0, rel=1e-12)


def test_eig_example2_200_full_size(qn):
    """200^3, the paper's first mesh size (Table results3D_2). The oracle's own solve takes
    thousands of iterations at this size, so the result is judged by the oracle's
    eigen-residual of the GPU eigenfunction and agreement with the FP64-product solve."""
    n = 200
    U0 = I.ex2_start(n, seed=1)
    ctx, v, h = _ex2_ctx(qn, n, "bf16x3")
    res, _, Ug = _gpu_eig(qn, ctx, U0, graph=True)
    assert res["status"] == 0
    F, lam = ob.eig_residual(Ug, h, "dirichlet", 0.0, ALPHA, ob.potential(v, 3, n))
    m = ob.mass_weights(n, 3, h, "dirichlet")
    assert math.sqrt(float(np.sum(m * F * F))) / abs(lam) <= 1.05e-10
    assert lam == pytest.approx(res["lambda"], rel=1e-12)
    ctx64, _, _ = _ex2_ctx(qn, n, "fp64")
    r64, _, U64 = _gpu_eig(qn, ctx64, U0, graph=True)
    assert r64["status"] == 0
    assert r64["lambda"] == pytest.approx(res["lambda"], rel=1e-10)
    assert np.abs(Ug - U64).max() <= 1e-7 * np.abs(U64).max()
