"""Parity of the CUDA path with the oracle for Neumann data (ghost points, Sec. 3.2)
and a separable potential V (Sec. 6.3, Example 1: -Lap u + 10 u + 10 u^3 + V u = f on
(-1,1)^3 with zero normal derivative).

Tolerances as in test_gpu_parity: FP64 operators to ~1e-13 of their scale, one
BF16X3 shifted inverse to 3e-4 of max|V|, solves to the FP64 residual tolerance
1e-10 and the oracle's solution to 1e-9 max|U|.
"""
import math

import numpy as np
import pytest

from oracle import qn_oracle as qo
from oracle import qn_oracle_bc as ob
from paper_2502_03611_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EX1_LAM, EX1_B = I.EX1_A, I.EX1_B


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


def tables(dim, n, seed):
    """Random potential tables (dim, n) in [0, 60)."""
    return I.random_field((dim, n), seed, 0.0, 60.0)


def ex1_ctx(qn, n, prec):
    u, f, v, h = I.ex1_problem(n)
    ctx = qn.QnContext(3, n, prec, lam=EX1_LAM, b=EX1_B, bc="neumann", length=2.0, potential=v)
    return ctx, u, f, v, h


# --------------------------------------------------------------------------------------------
# residual
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 63), (2, 100), (3, 2), (3, 17), (3, 65)])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("with_pot", [False, True])
def test_residual_neumann_matches_oracle(qn, dim, n, prec, with_pot):
    import torch
    U = I.random_field((n,) * dim, seed=n + dim)
    f = I.random_field((n,) * dim, seed=7 * n + dim) * 50.0
    lam, b = 0.3, 1.7
    v = tables(dim, n, 5 * n) if with_pot else None
    ctx = qn.QnContext(dim, n, prec, lam=lam, b=b, bc="neumann", length=2.0, potential=v)
    R = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    st = qn.qn_residual(ctx, dev(U).reshape(-1), dev(f).reshape(-1), R)
    h = ob.mesh_width(n, "neumann", 2.0)
    V = ob.potential(v, dim, n) if with_pot else None
    want = ob.residual(U, f, h, "neumann", lam, b, V)
    got = host(R).reshape(want.shape)
    scale = np.abs(want).max() + 4 * dim / h ** 2 * np.abs(U).max() + (0 if V is None else np.abs(V * U).max())
    assert np.abs(got - want).max() <= 1e-13 * scale
    assert st["res_norm"] == pytest.approx(np.linalg.norm(want), rel=1e-12)
    d = ob.jacobian_diag(U, b, V)
    assert st["fu_min"] == pytest.approx(d.min(), rel=1e-13, abs=1e-300)
    assert st["fu_max"] == pytest.approx(d.max(), rel=1e-13)
    assert st["beta"] == pytest.approx(ob.beta_rule(U, b, V), rel=1e-13)


def test_residual_dirichlet_with_potential_and_length(qn):
    """The potential and the domain size with Dirichlet data (h = L/(n+1))."""
    import torch
    n, dim, L = 40, 3, 2.0
    U = I.random_field((n,) * dim, seed=3)
    f = I.random_field((n,) * dim, seed=4) * 20.0
    v = tables(dim, n, 9)
    ctx = qn.QnContext(dim, n, "fp64", lam=1.5, b=0.7, bc="dirichlet", length=L, potential=v)
    R = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    st = qn.qn_residual(ctx, dev(U).reshape(-1), dev(f).reshape(-1), R)
    h = ob.mesh_width(n, "dirichlet", L)
    V = ob.potential(v, dim, n)
    want = ob.residual(U, f, h, "dirichlet", 1.5, 0.7, V)
    scale = np.abs(want).max() + 4 * dim / h ** 2
    assert np.abs(host(R).reshape(want.shape) - want).max() <= 1e-13 * scale
    assert st["beta"] == pytest.approx(ob.beta_rule(U, 0.7, V), rel=1e-13)


# --------------------------------------------------------------------------------------------
# shifted inverse with the non-orthogonal cosine basis
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 63), (2, 130), (3, 2), (3, 7), (3, 33), (3, 65), (3, 127)])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("shift", [0.5, 12.5])
def test_fast_diag_solve_neumann(qn, dim, n, prec, shift):
    import torch
    r = I.random_field((n,) * dim, seed=31 + n, lo=-10.0, hi=10.0)
    ctx = qn.QnContext(dim, n, prec, bc="neumann", length=2.0)
    V = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    qn.qn_fast_diag_solve(ctx, dev(r).reshape(-1), V, shift)
    torch.cuda.synchronize()
    h = ob.mesh_width(n, "neumann", 2.0)
    S, Si, lam = ob.eig_1d(n, h, "neumann")
    want = qo.fast_diag_solve(r, S, Si, lam, shift)
    got = host(V).reshape(want.shape)
    tol = 1e-11 if prec == "fp64" else 3e-4
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_fast_diag_solve_neumann_rejects_singular_shift(qn):
    import torch
    ctx = qn.QnContext(3, 9, "fp64", bc="neumann", length=2.0)
    r = torch.zeros(9 ** 3, dtype=torch.float64, device="cuda")
    V = torch.empty_like(r)
    with pytest.raises(qn.QnError) as e:
        qn.qn_fast_diag_solve(ctx, r, V, 0.0)     # constants are in the kernel of A_h
    assert e.value.code == qn.QN_EINVAL


# --------------------------------------------------------------------------------------------
# one step and full solves of the Example 1 workload
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [9, 33])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_step_ex1_matches_oracle(qn, n, prec):
    ctx, u, f, v, h = ex1_ctx(qn, n, prec)
    U0 = u + I.ex1_perturbation(n, 5, 0.5)
    Ud = dev(U0).reshape(-1)
    st = qn.qn_step(ctx, Ud, dev(f).reshape(-1), math.nan)
    V = ob.potential(v, 3, n)
    Uo, ho, _ = ob.qn_solve(f, h, "neumann", U0=U0, lam=EX1_LAM, b=EX1_B, V=V, tol=0.0, max_it=1)
    got = host(Ud).reshape(f.shape)
    delta = np.abs(Uo - U0).max()
    if prec == "fp64":
        assert np.abs(got - Uo).max() <= 1e-12 * np.abs(Uo).max()
    else:
        assert np.abs(got - Uo).max() <= 3e-4 * delta
    # the split solve's tiled residual takes the extremes of 3 b U^2 + V in FP32
    assert st["beta"] == pytest.approx(ho[0]["beta"], rel=1e-6 if prec == "bf16x3" else 1e-13)
    assert st["res_norm"] == pytest.approx(ho[0]["res"], rel=1e-6 if prec == "bf16x3" else 1e-12)


def _solve_ex1(qn, n, prec, U0, max_it=300, graph=False):
    import torch
    ctx, u, f, v, h = ex1_ctx(qn, n, prec)
    if not graph:
        qn.qn_profile_enable(ctx, True)
    U = dev(U0).reshape(-1).clone()
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, max_it=max_it, history_len=max_it + 1,
                            graph=graph)
    prof = qn.qn_profile_read(ctx) if not graph else None
    return res, hist, host(U).reshape(f.shape), prof


def _oracle_ex1(n, U0, max_it=300):
    u, f, v, h = I.ex1_problem(n)
    V = ob.potential(v, 3, n)
    return ob.qn_solve(f, h, "neumann", U0=U0, lam=EX1_LAM, b=EX1_B, V=V, tol=1e-10, max_it=max_it)


def _check_ex1(res, Ug, Uo, n):
    u, f, v, h = I.ex1_problem(n)
    V = ob.potential(v, 3, n)
    assert res["status"] == 0 and res["rel"] <= 1e-10, res
    rel = np.linalg.norm(ob.residual(Ug, f, h, "neumann", EX1_LAM, EX1_B, V)) / np.linalg.norm(f)
    assert rel <= 1.05e-10, rel
    if Uo is not None:
        assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()


@pytest.mark.parametrize("n,prec", [(9, "fp64"), (17, "fp64"), (17, "bf16x3"), (33, "fp64"), (33, "bf16x3"),
                                    (65, "bf16x3"), (70, "bf16x3"), (65, "bf16x6"), (128, "bf16x6")])
def test_solve_ex1_perturbed_start_matches_oracle(qn, n, prec):
    """The paper's start: the solution plus 0.1 p, p a normalised random cubic-free
    polynomial of degree 4 per axis. n = 65, 70: P = 128, reflection-split products
    and the mirrored residual; n = 17, 33: dense tensor-core products."""
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 1, 0.1)
    res, hist, Ug, prof = _solve_ex1(qn, n, prec, U0)
    Uo, ho, ok = _oracle_ex1(n, U0)
    assert ok
    _check_ex1(res, Ug, Uo, n)
    its_o = len(ho) - 1
    if prec == "fp64":
        assert abs(res["iterations"] - its_o) <= 1
        for a, b in zip(hist, ho):
            assert a["beta"] == pytest.approx(b["beta"], rel=1e-9)
    else:
        assert abs(res["iterations"] - its_o) <= 2
        if n >= 65:
            assert prof["split_products"] == 1 and prof["residual_tiled_launches"] >= 1


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_solve_ex1_zero_start(qn, prec):
    n = 33
    U0 = np.zeros((n, n, n))
    res, hist, Ug, prof = _solve_ex1(qn, n, prec, U0)
    Uo, ho, ok = _oracle_ex1(n, U0)
    assert ok
    _check_ex1(res, Ug, Uo, n)
    assert abs(res["iterations"] - (len(ho) - 1)) <= (1 if prec == "fp64" else 2)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("n", [50, 129])
def test_solve_2d_neumann_example_matches_oracle(qn, prec, n):
    """Sec. 6.2, Example 1: -Lap u + u^3 + u = f on (-1,1)^2, zero normal derivative."""
    import torch
    u, f, h = I.ex2d1_problem(n)
    ctx = qn.QnContext(2, n, prec, lam=1.0, b=1.0, bc="neumann", length=2.0)
    U0 = u + 0.1 * np.cos(0.5 * np.arange(n))[None, :] * np.ones((n, 1))
    U = dev(U0).reshape(-1).clone()
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, max_it=200, history_len=201)
    Uo, ho, ok = ob.qn_solve(f, h, "neumann", U0=U0, lam=1.0, b=1.0, tol=1e-10, max_it=200)
    assert ok and res["status"] == 0
    Ug = host(U).reshape(f.shape)
    assert np.linalg.norm(ob.residual(Ug, f, h, "neumann", 1.0, 1.0)) / np.linalg.norm(f) <= 1.05e-10
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert abs(res["iterations"] - (len(ho) - 1)) <= (1 if prec == "fp64" else 2)


# --------------------------------------------------------------------------------------------
# kernel-path agreement inside the split solve (Neumann faces, potential)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("max_it", [1, 2, 3, 5])
def test_tiled_neumann_iterates_match_per_point_path(qn, monkeypatch, max_it):
    """Iteration 0 (preparation pass), 1 (max|U| scan), and later ones (max|U| from the
    previous residual's block maxima) of the tiled residual with ghost faces and the
    potential, against the per-point residual (QN_RES_TILED=0); dense products both times."""
    monkeypatch.setenv("QN_SPLIT", "0")
    n = 45
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 2, 0.2)
    outs = []
    for tiled in ("1", "0"):
        monkeypatch.setenv("QN_RES_TILED", tiled)
        import torch
        ctx = qn.QnContext(3, n, "bf16x3", lam=EX1_LAM, b=EX1_B, bc="neumann", length=2.0, potential=v)
        qn.qn_profile_enable(ctx, True)
        U = dev(U0).reshape(-1).clone()
        res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-30, max_it=max_it, history_len=max_it + 1)
        assert res["status"] == qn.QN_ENOTCONV and res["iterations"] == max_it
        prof = qn.qn_profile_read(ctx)
        assert (prof["residual_tiled_launches"] >= 1) == (tiled == "1")
        outs.append((host(U), hist))
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-6 * np.abs(outs[1][0]).max()
    for a, c in zip(outs[0][1], outs[1][1]):
        assert a["beta"] == pytest.approx(c["beta"], rel=1e-6)


@pytest.mark.parametrize("headroom", [0, -6])
def test_tiled_neumann_flagged_planes(qn, monkeypatch, headroom):
    """Flagged planes (exact per-point path) with ghost faces and the potential."""
    monkeypatch.setenv("QN_RES_FX_HEADROOM", str(headroom))
    n = 70
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 3, 0.1)
    res, hist, Ug, prof = _solve_ex1(qn, n, "bf16x3", U0)
    Uo, ho, ok = _oracle_ex1(n, U0)
    assert ok and prof["residual_tiled_launches"] >= 1
    _check_ex1(res, Ug, Uo, n)


@pytest.mark.parametrize("n", [65, 200])
def test_split_products_neumann_match_dense(qn, monkeypatch, n):
    """Reflection-split products with the cosine pairs (forward matrix from S^{-1},
    backward from S) against the dense tensor-core products."""
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 4, 0.1)
    sols = []
    for split in ("1", "0"):
        monkeypatch.setenv("QN_SPLIT", split)
        res, hist, Ug, prof = _solve_ex1(qn, n, "bf16x3", U0)
        assert prof["split_products"] == (1 if split == "1" else 0)
        _check_ex1(res, Ug, None, n)
        sols.append((Ug, res["iterations"]))
    assert abs(sols[0][1] - sols[1][1]) <= 1
    assert np.abs(sols[0][0] - sols[1][0]).max() <= 1e-9 * np.abs(sols[1][0]).max()


def test_graph_replay_neumann_bitwise(qn):
    n = 65
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 6, 0.1)
    r1, _, U1, _ = _solve_ex1(qn, n, "bf16x3", U0, graph=False)
    r2, _, U2, _ = _solve_ex1(qn, n, "bf16x3", U0, graph=True)
    assert r1["iterations"] == r2["iterations"]
    assert np.array_equal(U1, U2)


# --------------------------------------------------------------------------------------------
# the paper's 3-D Example 1 at its first mesh size
# --------------------------------------------------------------------------------------------
def test_ex1_200_full_size(qn):
    """200^3 (Sec. 6.3, Table results3D_mesh, first column), from the perturbed start.
    Judged by properties that hold at any size: the oracle's FP64 residual of the GPU
    solution, agreement with the FP64-product solve, and O(h^2) convergence to u*
    (100 -> 200 nodes: h ratio 199/99)."""
    n = 200
    u, f, v, h = I.ex1_problem(n)
    U0 = u + I.ex1_perturbation(n, 1, 0.1)
    res, hist, Ug, prof = _solve_ex1(qn, n, "bf16x3", U0)
    _check_ex1(res, Ug, None, n)
    assert prof["split_products"] == 1
    r64, _, U64, _ = _solve_ex1(qn, n, "fp64", U0)
    assert r64["status"] == 0 and abs(r64["iterations"] - res["iterations"]) <= 2
    assert np.abs(Ug - U64).max() <= 1e-9 * np.abs(U64).max()
    err200 = np.abs(Ug - u).max()
    u1, f1, v1, h1 = I.ex1_problem(100)
    r1, _, U1, _ = _solve_ex1(qn, 100, "bf16x3", u1 + I.ex1_perturbation(100, 1, 0.1))
    assert r1["status"] == 0
    err100 = np.abs(U1 - u1).max()
    ratio = err100 / err200
    assert 0.9 * (199 / 99) ** 2 < ratio < 1.1 * (199 / 99) ** 2, (err100, err200)


def test_warm_start_rejects_neumann(qn):
    import torch
    ctx = qn.QnContext(3, 33, "bf16x3", bc="neumann", length=2.0)
    net = qn.QnNet(16, modes=4, blocks=1, max_batch=1)
    U = torch.zeros(33 ** 3, dtype=torch.float64, device="cuda")
    f = torch.ones(33 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(qn.QnError) as e:
        qn.qn_solve_warm(ctx, net, U, f)
    assert e.value.code == qn.QN_EUNSUPPORTED


# --------------------------------------------------------------------------------------------
# Robin faces: alpha_1 du/dn + beta_1 u = 0, kappa = beta_1 / alpha_1 (per-node residual path)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 40), (3, 3), (3, 33)])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_robin_residual_and_inverse_match_oracle(qn, dim, n, prec):
    import torch
    kappa, L = 1.7, 2.0
    U = I.random_field((n,) * dim, seed=n + 11)
    f = I.random_field((n,) * dim, seed=n + 12) * 30.0
    ctx = qn.QnContext(dim, n, prec, lam=0.4, b=1.2, bc="robin", length=L, robin_kappa=kappa)
    R = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    st = qn.qn_residual(ctx, dev(U).reshape(-1), dev(f).reshape(-1), R)
    h = ob.mesh_width(n, "robin", L)
    want = ob.residual(U, f, h, "robin", 0.4, 1.2, None, kappa)
    scale = np.abs(want).max() + (4 * dim / h ** 2 + 2 * dim * kappa / h) * np.abs(U).max()
    assert np.abs(host(R).reshape(want.shape) - want).max() <= 1e-13 * scale
    assert st["beta"] == pytest.approx(ob.beta_rule(U, 1.2), rel=1e-13)    # no face term in beta
    V = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    qn.qn_fast_diag_solve(ctx, dev(f).reshape(-1), V, 0.7)
    torch.cuda.synchronize()
    S, Si, lam = ob.eig_1d(n, h, "robin", kappa)
    wantv = qo.fast_diag_solve(f, S, Si, lam, 0.7)
    tol = 1e-11 if prec == "fp64" else 3e-4
    assert np.abs(host(V).reshape(wantv.shape) - wantv).max() <= tol * np.abs(wantv).max()


@pytest.mark.parametrize("dim,n,prec", [(2, 50, "fp64"), (2, 64, "bf16x3"), (3, 17, "fp64"), (3, 33, "bf16x3"),
                                        (3, 65, "bf16x3")])
def test_robin_solve_matches_oracle(qn, dim, n, prec):
    import torch
    kappa, L = 2.5, 2.0
    h = ob.mesh_width(n, "robin", L)
    f = 20.0 + 10.0 * I.random_field((n,) * dim, seed=3 * n)
    ctx = qn.QnContext(dim, n, prec, lam=1.0, b=1.0, bc="robin", length=L, robin_kappa=kappa)
    U = torch.zeros(n ** dim, dtype=torch.float64, device="cuda")
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, max_it=200, history_len=201)
    Uo, ho, ok = ob.qn_solve(f, h, "robin", lam=1.0, b=1.0, kappa=kappa, tol=1e-10)
    assert ok and res["status"] == 0 and res["rel"] <= 1e-10
    Ug = host(U).reshape(f.shape)
    rel = np.linalg.norm(ob.residual(Ug, f, h, "robin", 1.0, 1.0, None, kappa)) / np.linalg.norm(f)
    assert rel <= 1.05e-10
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert abs(res["iterations"] - (len(ho) - 1)) <= (1 if prec == "fp64" else 2)
