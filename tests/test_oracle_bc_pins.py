"""Pins of the boundary / potential oracle (oracle.qn_oracle_bc) to facts that do not
come from the oracle itself: closed-form eigenvalues, a general eigenvalue
routine on the matrix of Sec. 3.2, Taylor consistency at the faces, the discrete
divergence identity of the ghost-point scheme, dense linear algebra, the
spectral radius that Sec. 5 says governs the linear iteration, and second-order
convergence to the exact solution of the three-dimensional Example 1 (Sec. 6.3).
"""
import math

import numpy as np
import pytest

from oracle import qn_oracle as qo
from oracle import qn_oracle_bc as ob
from paper_2502_03611_gb300 import inputs as I


@pytest.mark.parametrize("n", [2, 3, 8, 33])
def test_neumann_eigenvalues_closed_form(n):
    """DCT-I spectrum of the ghost-point matrix: (4/h^2) sin^2(k pi / (2(n-1))), k = 0..n-1."""
    h = ob.mesh_width(n, "neumann", 2.0)
    _, _, lam = ob.eig_1d(n, h, "neumann")
    k = np.arange(n)
    ref = 4.0 / h ** 2 * np.sin(k * math.pi / (2.0 * (n - 1))) ** 2
    np.testing.assert_allclose(lam, ref, rtol=1e-12, atol=1e-12 / h ** 2)


@pytest.mark.parametrize("n", [6, 21])
def test_neumann_eigenvalues_general_routine(n):
    """The non-symmetric matrix itself through a general (non-symmetric) eigenvalue routine."""
    h = 0.3
    H = ob.fd_matrix_1d(n, h, "neumann")
    ev = np.linalg.eigvals(H)
    assert np.max(np.abs(ev.imag)) < 1e-8 / h ** 2
    _, _, lam = ob.eig_1d(n, h, "neumann")
    np.testing.assert_allclose(np.sort(ev.real), lam, rtol=1e-10, atol=1e-10 / h ** 2)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_eig_factorisation(bc):
    n = 11
    h = ob.mesh_width(n, bc, 2.0)
    H = ob.fd_matrix_1d(n, h, bc)
    S, Si, lam = ob.eig_1d(n, h, bc)
    np.testing.assert_allclose(H @ S, S * lam[None, :], atol=1e-10 / h ** 2)
    np.testing.assert_allclose(Si @ S, np.eye(n), atol=1e-13)
    if bc == "neumann":
        assert np.max(np.abs(S - S.T)) > 1e-3      # not orthogonal: S^{-1} != S^T


def test_neumann_rows_second_order_at_faces():
    """u = cos(pi x) on [-1, 1] has zero slope at both faces and -u'' = pi^2 u. The
    ghost-point matrix reproduces it to O(h^2) at every node, faces included (a
    wrong face row leaves an O(1) error there)."""
    errs = []
    for n in (17, 33):
        x = I.neumann_nodes(n)
        h = ob.mesh_width(n, "neumann", 2.0)
        u = np.cos(math.pi * x)
        e = ob.fd_matrix_1d(n, h, "neumann") @ u - math.pi ** 2 * u
        errs.append(np.max(np.abs(e)))
        assert abs(e[0]) > 0.3 * errs[-1] and abs(e[-1]) > 0.3 * errs[-1]   # faces are not exempt
    assert 3.6 < errs[0] / errs[1] < 4.4


@pytest.mark.parametrize("bc,dim,n", [("neumann", 2, 6), ("neumann", 3, 4), ("dirichlet", 3, 4),
                                      ("dirichlet", 2, 5)])
def test_stencil_matches_kronecker(bc, dim, n):
    """Stencil with ghost reflection (apply_operator) == Kronecker form (dense_operator)."""
    h = ob.mesh_width(n, bc, 2.0)
    U = I.random_field((n,) * dim, 7)
    A = ob.dense_operator(n, dim, h, bc)
    np.testing.assert_allclose(ob.apply_operator(U, h, bc).ravel(), A @ U.ravel(), atol=1e-11 / h ** 2)


def test_neumann_discrete_divergence_and_constants():
    """With zero flux the trapezoid-weighted sum of A_h U vanishes for every U (summation
    by parts of the ghost-point scheme), and constants span the kernel of A_h."""
    n = 7
    h = ob.mesh_width(n, "neumann", 2.0)
    U = I.random_field((n, n, n), 3)
    w = ob.trapezoid_weights(n, "neumann")
    W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    AU = ob.apply_operator(U, h, "neumann")
    assert abs(float(np.sum(W3 * AU))) < 1e-12 * float(np.sum(np.abs(AU)))
    assert np.max(np.abs(ob.apply_operator(np.full((n, n, n), 2.5), h, "neumann"))) < 1e-12


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 5)])
def test_fast_diag_neumann_matches_dense_solve(dim, n):
    h = ob.mesh_width(n, "neumann", 2.0)
    r = I.random_field((n,) * dim, 11)
    S, Si, lam = ob.eig_1d(n, h, "neumann")
    shift = 3.7
    v = qo.fast_diag_solve(r, S, Si, lam, shift)
    ref = np.linalg.solve(ob.dense_operator(n, dim, h, "neumann", shift), r.ravel())
    np.testing.assert_allclose(v.ravel(), ref, rtol=1e-11, atol=1e-13)


def test_potential_axis_order():
    n = 4
    t = np.arange(n, dtype=np.float64)
    V = ob.potential(np.stack([t, 10 * t, 100 * t]), 3, n)
    assert V[3, 2, 1] == 1 + 20 + 300 and V[0, 1, 3] == 3 + 10
    V2 = ob.potential(np.stack([t, 10 * t]), 2, n)
    assert V2[2, 3] == 3 + 20


def test_linear_iteration_rate_is_spectral_radius():
    """b = 0: the iteration is linear, r_{k+1} = (I - (A_h + V)(A_h + (lam + beta) I)^{-1}) r_k
    (Sec. 5, eq. error-update with R_n = 0). Its observed rate must equal the spectral
    radius of that matrix with beta = mid-range of V; this pins V in both the residual
    and the beta rule."""
    n, lam = 5, 1.0
    h = ob.mesh_width(n, "neumann", 2.0)
    x = I.neumann_nodes(n)
    v = np.stack([40 * x * x, 25 * (1 + x), 10 * np.cos(x)])
    V = ob.potential(v, 3, n)
    f = I.random_field((n, n, n), 5)
    U, hist, ok = ob.qn_solve(f, h, "neumann", lam=lam, b=0.0, V=V, tol=1e-13, max_it=400)
    assert ok
    beta = 0.5 * (V.max() + V.min())
    assert abs(hist[0]["beta"] - beta) < 1e-12 * beta
    A = ob.dense_operator(n, 3, h, "neumann", lam)
    M = np.eye(n ** 3) - (A + np.diag(V.ravel())) @ np.linalg.inv(A + beta * np.eye(n ** 3))
    rho = float(np.max(np.abs(np.linalg.eigvals(M))))
    rel = np.array([e["rel"] for e in hist])
    k1 = len(rel) - 3
    k0 = k1 - 15
    rate = (rel[k1] / rel[k0]) ** (1.0 / (k1 - k0))
    assert 0.5 < rho < 1.0
    assert abs(rate - rho) < 0.03 * rho


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_qn_fixed_point_is_newton_solution(bc):
    """The quasi-Newton limit solves F(U) = 0: it agrees with dense Newton (eq. newton)."""
    n = 5
    h = ob.mesh_width(n, bc, 2.0)
    x = I.neumann_nodes(n) if bc == "neumann" else -1.0 + h * np.arange(1, n + 1)
    V = ob.potential(I.ex1_potential_1d(x), 3, n)
    f = 50.0 * I.random_field((n, n, n), 9)
    U, _, ok = ob.qn_solve(f, h, bc, lam=10.0, b=10.0, V=V, tol=1e-13, max_it=2000)
    assert ok
    Un = ob.newton_dense(f, h, bc, lam=10.0, b=10.0, V=V, tol=1e-14)
    np.testing.assert_allclose(U, Un, atol=1e-11 * np.max(np.abs(Un)))


def test_ex1_converges_at_second_order():
    """Example 1 of Sec. 6.3: the discrete solution tends to u* = cos(pi x) + cos(pi y) + cos(pi z)
    as h^2 (error ratio ~4 when h halves)."""
    errs = []
    for n in (9, 17):
        u, f, v, h = I.ex1_problem(n)
        V = ob.potential(v, 3, n)
        U, hist, ok = ob.qn_solve(f, h, "neumann", lam=I.EX1_A, b=I.EX1_B, V=V, tol=1e-12, max_it=1000)
        assert ok
        errs.append(float(np.max(np.abs(U - u))))
    assert 3.3 < errs[0] / errs[1] < 4.7


# ---------------------------------------------------------------------------------------------
# nonlinear eigenproblem (Sec. 4.4)
# ---------------------------------------------------------------------------------------------
def _eig_grid(n, bc, L=16.0):
    h = ob.mesh_width(n, bc, L)
    x = -L / 2 + (h * np.arange(1, n + 1) if bc == "dirichlet" else h * np.arange(n))
    return h, x


def _start(x, L=16.0):
    g = np.cos(math.pi * x / L)
    return g[None, None, :] * g[None, :, None] * g[:, None, None]


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_eig_linear_separable_ground_state(bc):
    """b = 0 with a separable potential: the eigenproblem separates, so the ground state is the
    product of the 1-D ground states of H + diag(v_a) (from a general dense eigensolver) and
    lambda is the sum of their eigenvalues."""
    n = 12
    h, x = _eig_grid(n, bc)
    # harmonic wells: simple, well-separated 1-D ground states (a nearly degenerate pair would
    # leave the eigenvector undetermined)
    tabs = np.stack([0.3 * x * x, 0.5 * x * x, 0.2 * (x - 1.0) ** 2])
    V = ob.potential(tabs, 3, n)
    U, lam, hist, ok = ob.qn_eig_solve(_start(x), h, bc, b=0.0, V=V, tol=1e-11, max_it=20000)
    assert ok
    lam_ref, vecs = 0.0, []
    for a in range(3):
        ev, W = np.linalg.eig(ob.fd_matrix_1d(n, h, bc) + np.diag(tabs[a]))
        k = int(np.argmin(ev.real))
        lam_ref += float(ev[k].real)
        vecs.append(np.real(W[:, k]))
    assert lam == pytest.approx(lam_ref, rel=1e-10)
    Uref = vecs[0][None, None, :] * vecs[1][None, :, None] * vecs[2][:, None, None]
    m = ob.mass_weights(n, 3, h, bc)
    Uref = Uref / math.sqrt(float(np.sum(m * Uref * Uref)))
    Uref = Uref * np.sign(np.sum(Uref * U))
    assert np.abs(U - Uref).max() <= 1e-8 * np.abs(Uref).max()


def test_eig_hellmann_feynman():
    """d lambda / d b at b = 0 equals <U0^3, U0> = sum m U0^4 for the normalised linear ground
    state U0 (first-order perturbation of the Rayleigh quotient)."""
    n, bc = 10, "dirichlet"
    h, x = _eig_grid(n, bc)
    V = ob.potential(np.stack([0.3 * x * x, 0.5 * x * x, 0.2 * (x - 1.0) ** 2]), 3, n)
    U0, lam0, _, ok0 = ob.qn_eig_solve(_start(x), h, bc, b=0.0, V=V, tol=1e-12, max_it=20000)
    db = 1e-3
    _, lam1, _, ok1 = ob.qn_eig_solve(U0, h, bc, b=db, V=V, tol=1e-12, max_it=20000)
    assert ok0 and ok1
    m = ob.mass_weights(n, 3, h, bc)
    slope = float(np.sum(m * U0 ** 4))
    assert (lam1 - lam0) / db == pytest.approx(slope, rel=2e-3)


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_eig_limit_solves_bordered_system(bc):
    """The quasi-Newton limit is a solution of A U + b U^3 + V U = lambda U, <U, U> = 1:
    dense Newton on that bordered system, started off it, converges back to it."""
    n = 5
    h, x = _eig_grid(n, bc)
    V = ob.potential(I.ex1_potential_1d(x), 3, n)
    U, lam, hist, ok = ob.qn_eig_solve(_start(x), h, bc, b=1600.0, V=V, tol=1e-12, max_it=20000)
    assert ok
    Un, lamn = ob.newton_eig_dense(U * (1 + 0.01 * I.random_field(U.shape, 4)), lam * 1.01, h, bc, b=1600.0, V=V)
    assert lamn == pytest.approx(lam, rel=1e-11)
    assert np.abs(Un - U).max() <= 1e-9 * np.abs(U).max()


def test_eig_residual_is_mass_orthogonal():
    """With the Rayleigh quotient in the mass-weighted product, F is M-orthogonal to U for
    every U (<F, U>_M = <A U + f, U>_M - lambda <U, U>_M = 0); with Neumann data the face
    weights matter: the unweighted product would leave a visible <F, U>_M."""
    n, bc = 7, "neumann"
    h, x = _eig_grid(n, bc)
    V = ob.potential(0.4 * x * x, 3, n)
    U = 1.0 + I.random_field((n, n, n), 8)
    F, lam = ob.eig_residual(U, h, bc, 0.3, 50.0, V)
    m = ob.mass_weights(n, 3, h, bc)
    scale = math.sqrt(float(np.sum(m * F * F)) * float(np.sum(m * U * U)))
    assert abs(float(np.sum(m * F * U))) <= 1e-13 * scale
    lam_flat = float(np.sum((F + lam * U) * U)) / float(np.sum(U * U))
    assert abs(lam_flat - lam) > 1e-6 * abs(lam)


def test_eig_linear_rate_is_second_eigenvalue_ratio():
    """b = 0: near the limit, U_{k+1} is proportional to T U_k with
    T = (A_h + c - lambda)^{-1} (c - V), c = (max V + min V)/2 (beta_n + lambda_n = c). U* is
    T's eigenvector with eigenvalue 1, so the observed rate of rel is the largest |mu| of T
    over the other eigenvectors. This pins the sign and size of beta_n."""
    n, bc = 6, "dirichlet"
    h, x = _eig_grid(n, bc, L=6.0)
    V = ob.potential(np.stack([3.0 * x * x, 4.0 * x * x, 2.0 * (x - 0.5) ** 2]), 3, n)
    U, lam, hist, ok = ob.qn_eig_solve(_start(x, L=6.0), h, bc, b=0.0, V=V, tol=1e-13, max_it=20000)
    assert ok
    c = 0.5 * (V.max() + V.min())
    A = ob.dense_operator(n, 3, h, bc)
    T = np.linalg.solve(A + (c - lam) * np.eye(n ** 3), np.diag(c - V.ravel()))
    mu = np.sort(np.abs(np.linalg.eigvals(T)))[::-1]
    assert abs(mu[0] - 1.0) < 1e-8
    rel = np.array([e["rel"] for e in hist])
    k1 = len(rel) - 3
    k0 = max(k1 - 30, 1)
    rate = (rel[k1] / rel[k0]) ** (1.0 / (k1 - k0))
    assert 0.2 < mu[1] < 1.0
    assert rate == pytest.approx(mu[1], rel=0.03)


# ---------------------------------------------------------------------------------------------
# Robin faces (ghost points with alpha_1 du/dn + beta_1 u = 0, kappa = beta_1 / alpha_1)
# ---------------------------------------------------------------------------------------------
def test_robin_rows_taylor_consistency():
    """u = cos(w (x - 1/2)) on [0, 1] satisfies -u'(0) + kappa u(0) = 0 = u'(1) + kappa u(1) for
    kappa = w tan(w/2), and -u'' = w^2 u. Taylor expansion of the ghost-point face row with the
    exact Robin data leaves -u'' - (h/3) u3(0) + O(h^2), u3 the third derivative: the face error
    must match that term (a wrong kappa or face row leaves an O(1) error); the interior rows are
    second order."""
    w = 2.0
    kappa = w * math.tan(w / 2)
    u3_0 = w ** 3 * math.sin(-0.5 * w)                 # third derivative of cos(w (x - 1/2)) at 0
    interior = []
    for n in (33, 65):
        h = ob.mesh_width(n, "robin", 1.0)
        x = h * np.arange(n)
        u = np.cos(w * (x - 0.5))
        e = ob.fd_matrix_1d(n, h, "robin", kappa) @ u - w * w * u
        lead = -(h / 3.0) * u3_0
        assert abs(e[0] - lead) < 0.1 * abs(lead) and abs(e[-1] - lead) < 0.1 * abs(lead)
        interior.append(np.max(np.abs(e[1:-1])))
    assert 3.5 < interior[0] / interior[1] < 4.5


def test_robin_limits_and_spectrum():
    """kappa = 0 is Neumann; the spectrum (general eigensolver on the matrix itself) is real and
    positive for kappa > 0 and increases with kappa towards the Dirichlet spectrum."""
    n, L = 12, 2.0
    h = ob.mesh_width(n, "robin", L)
    np.testing.assert_allclose(ob.fd_matrix_1d(n, h, "robin", 0.0), ob.fd_matrix_1d(n, h, "neumann"))
    prev = None
    for kappa in (0.5, 2.0, 8.0):
        ev = np.sort(np.linalg.eigvals(ob.fd_matrix_1d(n, h, "robin", kappa)).real)
        _, _, lam = ob.eig_1d(n, h, "robin", kappa)
        np.testing.assert_allclose(lam, ev, rtol=1e-10)
        assert lam[0] > 0 and (prev is None or lam[0] > prev)
        prev = lam[0]


@pytest.mark.parametrize("dim,n", [(2, 7), (3, 5)])
def test_robin_stencil_and_inverse_match_dense(dim, n):
    kappa, h = 1.7, ob.mesh_width(n, "robin", 2.0)
    U = I.random_field((n,) * dim, 4)
    A = ob.dense_operator(n, dim, h, "robin", 0.0, kappa)
    np.testing.assert_allclose(ob.apply_operator(U, h, "robin", kappa).ravel(), A @ U.ravel(), atol=1e-11 / h ** 2)
    S, Si, lam = ob.eig_1d(n, h, "robin", kappa)
    v = qo.fast_diag_solve(U, S, Si, lam, 0.3)
    np.testing.assert_allclose(v.ravel(), np.linalg.solve(A + 0.3 * np.eye(n ** dim), U.ravel()), rtol=1e-10,
                               atol=1e-13)


def test_robin_face_term_is_not_in_beta():
    """The Robin face term belongs to A_h: beta_n is the mid-range of 3 b U^2 (+ V) alone, and
    the quasi-Newton limit solves the discrete system (dense Newton)."""
    n, kappa = 5, 2.5
    h = ob.mesh_width(n, "robin", 1.0)
    f = 20.0 * I.random_field((n, n, n), 6)
    U, hist, ok = ob.qn_solve(f, h, "robin", lam=0.5, b=3.0, kappa=kappa, tol=1e-13, max_it=2000)
    assert ok
    d = 3.0 * 3.0 * np.zeros_like(f)
    assert hist[0]["beta"] == 0.0 == 0.5 * (d.max() + d.min())
    A = ob.dense_operator(n, 3, h, "robin", 0.5, kappa)
    u = np.zeros(f.size)
    for _ in range(40):
        F = A @ u + 3.0 * u ** 3 - f.ravel()
        u = u - np.linalg.solve(A + np.diag(9.0 * u * u), F)
    np.testing.assert_allclose(U.ravel(), u, atol=1e-11 * np.abs(u).max())
