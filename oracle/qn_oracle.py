"""Plain FP64 CPU oracle for the quasi-Newton method with tensor-product inverse.

TEST INFRASTRUCTURE. This module is the reference the CUDA library is checked
against. Only tests, the smoke check and the benchmark's CPU-baseline and
reference legs may use it. It shares no code with the CUDA path; the seeded
input generators live in a separate module that holds none of this
arithmetic.

Paper: W. Hao, S. Lee, X. Zhang, "An Efficient Quasi-Newton Method with
Tensor Product Implementation for Solving Quasi-Linear Elliptic Equations and
Systems", arXiv 2502.03611.

What is computed (everything float64, numpy; library calls used as steps:
matmul/tensordot for mode products, eigh for the symmetric 1-D eigenproblem,
solve for dense linear systems):

* Discretisation, Sec. 3.2 (finite differences, Dirichlet): n interior nodes
  per axis on (0,1), h = 1/(n+1); 1-D matrix H = (1/h^2) tridiag(-1, 2, -1)
  (eq. Sy); boundary values are zero so no boundary terms enter F_h.
* Operator, Sec. 4 eqs. A_definition_2D / A_definition_3D:
  A_h = sum_a (I kron .. kron H_a kron .. kron I) + lam I, applied here as the
  5/7-point stencil of eq. fdm-discrete.
* Residual, Sec. 4 eq. F_u: F(U) = A_h vec(U) + N_h(U) with the pointwise
  nonlinearity N_h(U) = b U^3 - f (the model problem's f(x,u), Sec. 2
  eq. main-pde, with lam kept in A_h).
* Quasi-Newton, Sec. 4 eq. identity-method:
  U_{n+1} = U_n - (A_h + beta_n I)^{-1} F(U_n),
  beta_n = (lambda_max + lambda_min)/2 of (N_h)_U(U_n) = diag(3 b U_n^2).
* Inverse by fast diagonalisation, Sec. 4.1 eq. fin_inverse and Sec. 4.2:
  H = S Lambda S^{-1} per axis; apply S^{-1} along every axis, divide
  pointwise by (sum_a lambda_{i_a} + lam + beta_n), apply S along every axis.
* Newton's method, Sec. 4 eq. newton, with the dense Jacobian
  A_h + diag(3 b U^2), for tiny grids only.
* Convergence bound, Sec. 5 (Theorem 1, eq. norm_ratio, Remark "Optimal
  beta"): g(beta) = max_mu |beta - mu| / min_lambda |lambda + beta|.

Readings where the paper is silent or garbled (each also listed in the
design notes):
* Stopping rule: the paper iterates "until the residual is sufficiently
  small" (Sec. 4.4) and states no tolerance. Here: ||F(U_n)||_2 / ||f||_2 <= tol,
  with f the source term (= F(0) for the problems here), default 1e-10.
* The diagonal in the equation before eq. fin_inverse drops beta_n; eq.
  fin_inverse and eq. linear_system keep it. Here: lam + beta_n.
* Interior size: the text says n_x - 2 unknowns but indexes 1..n_x - 1; here
  n interior unknowns with h = 1/(n+1).
* beta_0 at U_0 = 0 is 0 (diag(3 b U^2) = 0); A_h is SPD, so A_h + 0 I is
  invertible (Sec. 5 requires beta_n > -lambda_min(A_h)).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "fd_matrix_1d", "eig_1d", "apply_laplacian", "residual", "jacobian_diag",
    "beta_rule", "mode_product", "fast_diag_solve", "qn_step", "qn_solve",
    "dense_operator", "newton_dense", "contraction_bound", "discrete_source",
    "system_residual", "system_beta", "qn_solve_system",
]


# ----------------------------------------------------------------------------
# 1-D operator and its diagonalisation (Sec. 3.2 eq. Sy; Sec. 4.2)
# ----------------------------------------------------------------------------
def fd_matrix_1d(n: int) -> np.ndarray:
    """H = (1/h^2) tridiag(-1, 2, -1) of size n x n, h = 1/(n+1) (Sec. 3.2, eq. Sy)."""
    h = 1.0 / (n + 1)
    H = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return H / (h * h)


def eig_1d(n: int):
    """Diagonalise H = S Lambda S^{-1} (Sec. 4.2).

    For finite differences the mass matrix is the identity (Sec. 3.2), so
    M^{-1/2} S_x M^{-1/2} = H is symmetric and its eigenvectors are
    orthonormal: S^{-1} = S^T. Eigenvalues ascending.
    Returns (S, S_inv, lam) with S[:, k] the k-th eigenvector.
    """
    lam, S = np.linalg.eigh(fd_matrix_1d(n))
    return S, S.T.copy(), lam


# ----------------------------------------------------------------------------
# Residual (Sec. 3.2 eq. fdm-discrete; Sec. 4 eq. F_u)
# ----------------------------------------------------------------------------
def apply_laplacian(U: np.ndarray) -> np.ndarray:
    """sum over axes of (2 U_i - U_{i-1} - U_{i+1}) / h^2 with zero Dirichlet data.

    U has n points along every axis; h = 1/(n+1).
    """
    n = U.shape[0]
    h2 = (1.0 / (n + 1)) ** 2
    out = np.zeros_like(U)
    for axis in range(U.ndim):
        P = np.pad(U, [(1, 1) if a == axis else (0, 0) for a in range(U.ndim)])
        lo = [slice(None)] * U.ndim
        hi = [slice(None)] * U.ndim
        lo[axis] = slice(0, n)
        hi[axis] = slice(2, n + 2)
        out += (2.0 * U - P[tuple(lo)] - P[tuple(hi)]) / h2
    return out


def residual(U: np.ndarray, f: np.ndarray, lam: float = 0.0, b: float = 1.0) -> np.ndarray:
    """F(U) = A_h vec(U) + N_h(U), A_h = -Lap_h + lam I, N_h(U) = b U^3 - f."""
    return apply_laplacian(U) + lam * U + b * U ** 3 - f


def jacobian_diag(U: np.ndarray, b: float = 1.0) -> np.ndarray:
    """Diagonal of (N_h)_U: d/du (b u^3) = 3 b u^2 (pointwise, Sec. 5 remarks)."""
    return 3.0 * b * U * U


def beta_rule(U: np.ndarray, b: float = 1.0) -> float:
    """beta_n = (lambda_max + lambda_min)/2 of the diagonal (N_h)_U (eq. identity-method)."""
    d = jacobian_diag(U, b)
    return 0.5 * (float(d.max()) + float(d.min()))


# ----------------------------------------------------------------------------
# Tensor-product inverse (Sec. 4.1 eq. fin_inverse)
# ----------------------------------------------------------------------------
def mode_product(X: np.ndarray, M: np.ndarray, axis: int) -> np.ndarray:
    """Y = X x_axis M: Y[.., k, ..] = sum_j M[k, j] X[.., j, ..] (vec(A X B^T) identity)."""
    Y = np.tensordot(M, X, axes=([1], [axis]))   # new axis 0 holds k
    return np.moveaxis(Y, 0, axis)


def fast_diag_solve(r: np.ndarray, S: np.ndarray, S_inv: np.ndarray,
                    lam1d: np.ndarray, shift: float) -> np.ndarray:
    """V with (sum_a I..H_a..I + shift I) vec(V) = vec(r), by eq. fin_inverse.

    R_hat = r x_a S^{-1} for every axis; R_hat /= (sum_a lambda_{i_a} + shift);
    V = R_hat x_a S for every axis.
    """
    d = r.ndim
    X = r
    for axis in range(d):
        X = mode_product(X, S_inv, axis)
    D = np.full(r.shape, shift, dtype=np.float64)
    for axis in range(d):
        shape = [1] * d
        shape[axis] = lam1d.size
        D = D + lam1d.reshape(shape)
    X = X / D
    for axis in range(d):
        X = mode_product(X, S, axis)
    return np.ascontiguousarray(X)


# ----------------------------------------------------------------------------
# Quasi-Newton iteration (Sec. 4 eq. identity-method)
# ----------------------------------------------------------------------------
def qn_step(U: np.ndarray, f: np.ndarray, eig=None, lam: float = 0.0, b: float = 1.0,
            beta: float | None = None, step: float = 1.0):
    """One quasi-Newton update. Returns (U_next, r, beta_used)."""
    n = U.shape[0]
    S, S_inv, lam1d = eig if eig is not None else eig_1d(n)
    r = residual(U, f, lam, b)
    beta_n = _beta_for(U, b, beta)
    delta = fast_diag_solve(r, S, S_inv, lam1d, lam + beta_n)
    return U - step * delta, r, beta_n


def _beta_for(U: np.ndarray, b: float, beta) -> float:
    """beta_n per the paper's rule (beta None), a fixed number, or the
    end points 'min' / 'max' of the spectrum of (N_h)_U (for the optimal-beta
    comparison of Sec. 5, Remark "Optimal beta")."""
    if beta is None:
        return beta_rule(U, b)
    if isinstance(beta, str):
        d = jacobian_diag(U, b)
        return float(d.min()) if beta == "min" else float(d.max())
    return float(beta)


def qn_solve(f: np.ndarray, U0: np.ndarray | None = None, tol: float = 1e-10,
             max_it: int = 200, lam: float = 0.0, b: float = 1.0,
             beta=None, step: float = 1.0):
    """Iterate eq. identity-method until ||F(U)||_2 / ||f||_2 <= tol.

    Returns (U, history, converged). history[i] holds the relative residual,
    residual norm, beta and the extreme values of (N_h)_U at iterate U_i;
    len(history) - 1 updates were made when converged.
    """
    n = f.shape[0]
    eig = eig_1d(n)
    U = np.zeros_like(f) if U0 is None else np.array(U0, dtype=np.float64, copy=True)
    fnorm = float(np.linalg.norm(f.ravel()))
    history = []
    for it in range(max_it + 1):
        r = residual(U, f, lam, b)
        rnorm = float(np.linalg.norm(r.ravel()))
        rel = rnorm / fnorm
        beta_n = _beta_for(U, b, beta)
        d = jacobian_diag(U, b)
        history.append({"rel": rel, "res": rnorm, "beta": beta_n,
                        "fu_min": float(d.min()), "fu_max": float(d.max())})
        if rel <= tol:
            return U, history, True
        if not math.isfinite(rel) or it == max_it:
            break
        S, S_inv, lam1d = eig
        U = U - step * fast_diag_solve(r, S, S_inv, lam1d, lam + beta_n)
    return U, history, False


# ----------------------------------------------------------------------------
# Dense forms for tiny grids (Sec. 4 eqs. A_definition, newton)
# ----------------------------------------------------------------------------
def dense_operator(n: int, dim: int, lam: float = 0.0) -> np.ndarray:
    """A_h as an explicit matrix from Kronecker products of the 1-D H (eq. A_definition).

    Acts on the C-order ravel of U[y, x] (2-D) or U[z, y, x] (3-D), i.e. the
    paper's vec() with x fastest.
    """
    H = fd_matrix_1d(n)
    I = np.eye(n)
    if dim == 2:
        A = np.kron(I, H) + np.kron(H, I)
    elif dim == 3:
        A = np.kron(np.kron(I, I), H) + np.kron(np.kron(I, H), I) + np.kron(np.kron(H, I), I)
    else:
        raise ValueError("dim must be 2 or 3")
    return A + lam * np.eye(n ** dim)


def newton_dense(f: np.ndarray, U0: np.ndarray | None = None, tol: float = 1e-12,
                 max_it: int = 50, lam: float = 0.0, b: float = 1.0):
    """Newton's method with the dense Jacobian A_h + diag(3 b U^2) (eq. newton)."""
    n, dim = f.shape[0], f.ndim
    A = dense_operator(n, dim, lam)
    u = np.zeros(f.size) if U0 is None else np.array(U0, dtype=np.float64).ravel()
    fv = f.ravel()
    fnorm = float(np.linalg.norm(fv))
    for _ in range(max_it):
        F = A @ u + b * u ** 3 - fv
        if np.linalg.norm(F) / fnorm <= tol:
            break
        J = A + np.diag(3.0 * b * u * u)
        u = u - np.linalg.solve(J, F)
    return u.reshape(f.shape)


def contraction_bound(beta: float, fu_min: float, fu_max: float, lam_min_A: float) -> float:
    """g(beta) = max_mu |beta - mu| / min_lambda |lambda + beta| (Sec. 5, eq. norm_ratio).

    mu ranges over the spectrum of the diagonal (N_h)_U (so over [fu_min, fu_max]),
    lambda over the spectrum of the SPD A_h, whose smallest eigenvalue is lam_min_A.
    """
    num = max(abs(beta - fu_min), abs(beta - fu_max))
    return num / abs(lam_min_A + beta)


def discrete_source(u: np.ndarray, lam: float = 0.0, b: float = 1.0) -> np.ndarray:
    """f_disc with F(u) = 0 exactly: f_disc = A_h u + lam u + b u^3 (for exact-recovery tests)."""
    return apply_laplacian(u) + lam * u + b * u ** 3


# ----------------------------------------------------------------------------
# Coupled two-component system (Sec. 4.3 eqs. system, eigen_quad, eigenvalues)
# ----------------------------------------------------------------------------
def system_residual(U, V, f1, f2, alpha: float, D: float, b: float = 1.0):
    """F = [A_h U + b U^3 + alpha V - f1 ; D A_h V + b V^3 - alpha U - f2].

    The second component carries diffusion D (its 1-D matrices are D H, with
    the same eigenvectors S and eigenvalues D lambda).
    """
    Fu = apply_laplacian(U) + b * U ** 3 + alpha * V - f1
    Fv = D * apply_laplacian(V) + b * V ** 3 - alpha * U - f2
    return Fu, Fv


def system_beta(U, V, alpha: float, b: float = 1.0) -> float:
    """beta = (lambda_max + lambda_min)/2 over the eigenvalues of DN_h (Sec. 4.3).

    At every node DN_h is the 2x2 block [[3bU^2, alpha], [-alpha, 3bV^2]]; its
    eigenvalues solve eq. eigen_quad, given by eq. eigenvalues with
    (N_1)_V (N_2)_U = -alpha^2. When the discriminant is negative the pair is
    complex and both share the real part (a + d)/2; the real parts are used.
    """
    a = 3.0 * b * U * U
    d = 3.0 * b * V * V
    disc = (a - d) ** 2 - 4.0 * alpha * alpha
    root = np.sqrt(np.maximum(disc, 0.0))
    hi = 0.5 * (a + d + root)
    lo = 0.5 * (a + d - root)
    return 0.5 * (float(hi.max()) + float(lo.min()))


def qn_solve_system(f1, f2, alpha: float, D: float, tol: float = 1e-10,
                    max_it: int = 200, b: float = 1.0):
    """Quasi-Newton for the coupled pair with the block-diagonal approximation
    diag(A_h + beta I, D A_h + beta I) of the Jacobian (Sec. 4.3)."""
    n = f1.shape[0]
    S, S_inv, lam1d = eig_1d(n)
    U = np.zeros_like(f1)
    V = np.zeros_like(f2)
    fnorm = math.sqrt(float(np.sum(f1 * f1)) + float(np.sum(f2 * f2)))
    history = []
    for it in range(max_it + 1):
        Fu, Fv = system_residual(U, V, f1, f2, alpha, D, b)
        rel = math.sqrt(float(np.sum(Fu * Fu)) + float(np.sum(Fv * Fv))) / fnorm
        beta_n = system_beta(U, V, alpha, b)
        history.append({"rel": rel, "beta": beta_n})
        if rel <= tol:
            return U, V, history, True
        if not math.isfinite(rel) or it == max_it:
            break
        U = U - fast_diag_solve(Fu, S, S_inv, lam1d, beta_n)
        V = V - fast_diag_solve(Fv, S, S_inv, D * lam1d, beta_n)
    return U, V, history, False
