"""Q^k spectral elements (Sec. 3.1) through the C-ABI against the oracle
(oracle.qn_oracle_sem). Nodes and sources come from the oracle's assembly and closed
forms, never from the library. Tolerances as in test_gpu_parity."""
import math

import numpy as np
import pytest

from oracle import qn_oracle as qo
from oracle import qn_oracle_sem as so
from paper_2502_03611_gb300 import inputs as I

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


BCS = {"dirichlet": 0, "neumann": 1}


def manufactured(n, k, dim, bc, L=1.0, lam=0.5, b=1.0):
    """u* = prod cos(pi x_a / L) (Neumann) or prod sin(pi x_a / L) (Dirichlet) at the nodes,
    f = -Lap u* + lam u* + b u*^3 in closed form."""
    _, _, x = so.assemble_1d(n, k, L, bc)
    g = np.sin(math.pi * x / L) if bc == "dirichlet" else np.cos(math.pi * x / L)
    u = g[None, :] * g[:, None] if dim == 2 else g[None, None, :] * g[None, :, None] * g[:, None, None]
    f = dim * (math.pi / L) ** 2 * u + lam * u + b * u ** 3
    return u, f


@pytest.mark.parametrize("dim,n,k,bc", [(2, 15, 2, "dirichlet"), (2, 33, 4, "neumann"), (3, 15, 2, "dirichlet"),
                                        (3, 19, 3, "neumann"), (3, 31, 4, "dirichlet"), (3, 9, 1, "neumann")])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("with_pot", [False, True])
def test_sem_residual_matches_oracle(qn, dim, n, k, bc, prec, with_pot):
    import torch
    L = 1.7
    U = I.random_field((n,) * dim, seed=n + k)
    f = 20.0 * I.random_field((n,) * dim, seed=3 * n + k)
    v = I.random_field((dim, n), 9, 0.0, 30.0) if with_pot else None
    ctx = qn.QnContext(dim, n, prec, lam=0.7, b=1.3, bc=bc, length=L, potential=v, sem_k=k)
    R = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    st = qn.qn_residual(ctx, dev(U).reshape(-1), dev(f).reshape(-1), R)
    _, _, _, H = so.eig_1d(n, k, L, bc)
    from oracle import qn_oracle_bc as ob
    V = ob.potential(v, dim, n) if with_pot else None
    want = so.residual(U, f, H, 0.7, 1.3, V)
    scale = np.abs(want).max() + dim * np.abs(H).sum(axis=1).max() * np.abs(U).max()
    assert np.abs(host(R).reshape(want.shape) - want).max() <= 1e-13 * scale
    assert st["res_norm"] == pytest.approx(np.linalg.norm(want), rel=1e-12)
    d = 3 * 1.3 * U * U + (0 if V is None else V)
    assert st["beta"] == pytest.approx(0.5 * (d.max() + d.min()), rel=1e-13)


@pytest.mark.parametrize("dim,n,k,bc", [(2, 31, 4, "dirichlet"), (3, 15, 2, "neumann"), (3, 63, 4, "dirichlet"),
                                        (3, 65, 8, "neumann")])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_sem_fast_diag_matches_oracle(qn, dim, n, k, bc, prec):
    import torch
    r = I.random_field((n,) * dim, seed=5 + n, lo=-10.0, hi=10.0)
    ctx = qn.QnContext(dim, n, prec, bc=bc, length=2.0, sem_k=k)
    V = torch.empty(n ** dim, dtype=torch.float64, device="cuda")
    qn.qn_fast_diag_solve(ctx, dev(r).reshape(-1), V, 3.0)
    torch.cuda.synchronize()
    S_e, Si, lam, _ = so.eig_1d(n, k, 2.0, bc)
    want = qo.fast_diag_solve(r, S_e, Si, lam, 3.0)
    tol = 1e-11 if prec == "fp64" else 3e-4
    assert np.abs(host(V).reshape(want.shape) - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("dim,n,k,bc,prec", [(2, 31, 2, "dirichlet", "fp64"), (2, 65, 4, "neumann", "bf16x3"),
                                             (3, 15, 2, "dirichlet", "fp64"), (3, 23, 3, "dirichlet", "bf16x3"),
                                             (3, 33, 4, "neumann", "fp64"), (3, 33, 4, "neumann", "bf16x3")])
def test_sem_solve_matches_oracle(qn, dim, n, k, bc, prec):
    import torch
    u, f = manufactured(n, k, dim, bc)
    ctx = qn.QnContext(dim, n, prec, lam=0.5, b=1.0, bc=bc, length=1.0, sem_k=k)
    U = torch.zeros(n ** dim, dtype=torch.float64, device="cuda")
    res, hist = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, max_it=200, history_len=201)
    Uo, ho, ok = so.qn_solve(f, k, 1.0, bc, lam=0.5, b=1.0)
    assert ok and res["status"] == 0 and res["rel"] <= 1e-10
    Ug = host(U).reshape(f.shape)
    _, _, _, H = so.eig_1d(n, k, 1.0, bc)
    assert np.linalg.norm(so.residual(Ug, f, H, 0.5, 1.0)) / np.linalg.norm(f) <= 1.05e-10
    assert np.abs(Ug - Uo).max() <= 1e-9 * np.abs(Uo).max()
    assert abs(res["iterations"] - (len(ho) - 1)) <= (1 if prec == "fp64" else 2)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_q1_elements_match_finite_differences(qn, bc):
    """Q^1 with lumped mass is the second-difference scheme: the same solve through both
    discretisations agrees to rounding (different kernels: banded FP64 vs exact stencil)."""
    import torch
    n, L = 33, 2.0
    f = 10.0 * I.random_field((n, n, n), 12)
    outs = []
    for sem_k in (1, 0):
        ctx = qn.QnContext(3, n, "fp64", lam=1.0, b=1.0, bc=bc, length=L, sem_k=sem_k)
        U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        res, _ = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-12, max_it=100)
        assert res["status"] == 0
        outs.append((res["iterations"], host(U)))
    assert outs[0][0] == outs[1][0]
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-11 * np.abs(outs[1][1]).max()


def test_sem_full_size_q4(qn):
    """3-D Q^4 on 64^3 elements (255^3 nodes): the oracle's FP64 residual of the BF16X3
    solution, agreement with the FP64-product solve, and high-order accuracy against u*."""
    import torch
    n, k = 255, 4
    u, f = manufactured(n, k, 3, "dirichlet")
    sols = []
    for prec in ("bf16x3", "fp64"):
        ctx = qn.QnContext(3, n, prec, lam=0.5, b=1.0, bc="dirichlet", length=1.0, sem_k=k)
        U = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        res, _ = qn.qn_solve(ctx, U, dev(f).reshape(-1), tol=1e-10, max_it=100)
        assert res["status"] == 0
        sols.append(host(U).reshape(f.shape))
        del U, ctx
    _, _, _, H = so.eig_1d(n, k, 1.0, "dirichlet")
    assert np.linalg.norm(so.residual(sols[0], f, H, 0.5, 1.0)) / np.linalg.norm(f) <= 1.05e-10
    assert np.abs(sols[0] - sols[1]).max() <= 1e-9 * np.abs(sols[1]).max()
    assert np.abs(sols[0] - u).max() < 1e-7        # Q^4, h = 1/64: far below second order
