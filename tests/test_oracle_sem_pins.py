"""Pins of the spectral element oracle (oracle.qn_oracle_sem, Sec. 3.1) to facts from
outside it: Gauss-Lobatto rules in closed form and their exactness degree, exact
differentiation of polynomials, the identity of the Q^1 element with lumped mass and the
second-difference matrix (both boundary types), spectral accuracy of the 1-D eigenvalues,
dense solves, dense Newton and the high-order convergence of Q^k on a manufactured
solution."""
import math

import numpy as np
import pytest

from oracle import qn_oracle as qo
from oracle import qn_oracle_bc as ob
from oracle import qn_oracle_sem as sem
from paper_2502_03611_gb300 import inputs as I


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_gll_exactness_degree(k):
    """(k+1)-point Gauss-Lobatto integrates x^m exactly for m <= 2k-1, not for m = 2k."""
    x, w = sem.gll(k)
    for m in range(2 * k):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * x ** m) - exact) < 1e-14
    m = 2 * k
    assert abs(np.sum(w * x ** m) - 2.0 / (m + 1)) > 1e-6


def test_gll_closed_forms():
    x, w = sem.gll(2)              # Simpson's rule
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-15)
    x, w = sem.gll(3)
    r = 1 / math.sqrt(5)
    np.testing.assert_allclose(x, [-1, -r, r, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)


@pytest.mark.parametrize("k", [2, 4, 7])
def test_derivative_matrix_exact_on_polynomials(k):
    x, _ = sem.gll(k)
    D = sem.lagrange_derivative(x)
    c = I.random_field((k + 1,), 3)
    p = np.polynomial.Polynomial(c)
    np.testing.assert_allclose(D @ p(x), p.deriv()(x), atol=1e-11)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_q1_lumped_is_second_difference(bc):
    """Linear elements with the Gauss-Lobatto (trapezoid) lumped mass reproduce the
    second-difference matrix exactly, including the Neumann face rows."""
    n, Lx = 9, 2.0
    S_e, Si, lam, H = sem.eig_1d(n, 1, Lx, bc)
    h = ob.mesh_width(n, bc, Lx)
    np.testing.assert_allclose(H, ob.fd_matrix_1d(n, h, bc), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("k", [2, 4])
def test_assembly_structure(bc, k):
    n = 4 * k + (-1 if bc == "dirichlet" else 1)
    S, m, x = sem.assemble_1d(n, k, 3.0, bc)
    assert np.allclose(S, S.T, atol=1e-13)
    ev = np.linalg.eigvalsh(S)
    if bc == "neumann":
        assert np.max(np.abs(S @ np.ones(n))) < 1e-12 and abs(ev[0]) < 1e-12 and ev[1] > 1e-6
        assert abs(np.sum(m) - 3.0) < 1e-14              # the lumped mass integrates 1 exactly
    else:
        assert ev[0] > 1e-6
    assert np.all(np.diff(x) > 0) and np.allclose(x + x[::-1], x[0] + x[-1])   # symmetric nodes


def test_eigenvalues_spectrally_accurate():
    """-u'' on (0, pi) with zero ends has eigenvalues j^2; Q^4 on 8 elements gets the
    lowest ones to ~1e-8."""
    k, E = 4, 8
    n = E * k - 1
    _, _, lam, _ = sem.eig_1d(n, k, math.pi, "dirichlet")
    np.testing.assert_allclose(lam[:3], [1.0, 4.0, 9.0], rtol=1e-7)
    assert abs(lam[3] - 16.0) < 1e-6 * 16.0


@pytest.mark.parametrize("dim", [2, 3])
def test_fast_diag_matches_dense_solve(dim):
    k, n = 3, 10
    S_e, Si, lam, H = sem.eig_1d(n, k, 1.5, "neumann")
    r = I.random_field((n,) * dim, 5)
    v = qo.fast_diag_solve(r, S_e, Si, lam, 2.5)
    ref = np.linalg.solve(sem.dense_operator(H, dim, 2.5), r.ravel())
    np.testing.assert_allclose(v.ravel(), ref, rtol=1e-11, atol=1e-13)


def test_qn_limit_is_newton_solution():
    k, n = 2, 7
    _, _, _, H = sem.eig_1d(n, k, 1.0, "dirichlet")
    f = 30.0 * I.random_field((n, n, n), 2)
    U, hist, ok = sem.qn_solve(f, k, 1.0, "dirichlet", lam=1.0, b=2.0, tol=1e-13)
    assert ok
    A = sem.dense_operator(H, 3, 1.0)
    u = np.zeros(f.size)
    for _ in range(40):
        F = A @ u + 2.0 * u ** 3 - f.ravel()
        u = u - np.linalg.solve(A + np.diag(6.0 * u * u), F)
    np.testing.assert_allclose(U.ravel(), u, atol=1e-11 * np.abs(u).max())


@pytest.mark.parametrize("k", [2, 3])
def test_high_order_convergence(k):
    """-Lap u + u^3 = f on (0,1)^2, u* = sin(pi x) sin(2 pi y): the nodal error of Q^k falls
    at least like h^(k+1) (Gauss-Lobatto SEM superconverges at the nodes)."""
    errs = []
    for E in (4, 8):
        n = E * k - 1
        _, _, x = sem.assemble_1d(n, k, 1.0, "dirichlet")
        u = np.sin(2 * math.pi * x)[:, None] * np.sin(math.pi * x)[None, :]
        f = 5 * math.pi ** 2 * u + u ** 3
        U, _, ok = sem.qn_solve(f, k, 1.0, "dirichlet", tol=1e-13)
        assert ok
        errs.append(np.abs(U - u).max())
    assert errs[0] / errs[1] > 0.8 * 2 ** (k + 1)
