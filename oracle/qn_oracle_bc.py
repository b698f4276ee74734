"""Plain FP64 CPU oracle: boundary conditions, domain size and a separable potential.

TEST INFRASTRUCTURE, like qn_oracle: only tests, the smoke check and the
benchmark's CPU-baseline and reference legs may use it, and the CUDA library
shares no code with it.

It widens the model problem of qn_oracle to

    -Lap u + lam u + b u^3 + V u = f   on a cube of side `length`,

with either homogeneous Dirichlet data (n interior nodes per axis,
h = length/(n+1)) or a zero normal derivative (n nodes per axis including
both faces, h = length/(n-1)), and V a separable potential
V(x, y, z) = v_x(x) + v_y(y) + v_z(z) given by its 1-D tables.

What is computed (float64 numpy; library calls used as steps: eigh for a
symmetric 1-D eigenproblem, tensordot for mode products, solve for dense
systems):

* Neumann rows, Sec. 3.2 (the ghost-point construction): the ghost value
  outside a face equals the first interior neighbour, so the 1-D matrix is
  (1/h^2) tridiag(-1, 2, -1) with its first row (2, -2, 0, ..) and last row
  (.., 0, -2, 2) / h^2. With a zero flux the source term gets no boundary
  correction (the paper's alpha_3 = 0).
* Robin rows (the same ghost construction with alpha_1 du/dn + beta_1 u = 0,
  kappa = beta_1 / alpha_1 >= 0): the ghost value is u_{-1} = u_1 - 2 h kappa u_0,
  so the face rows become ((2 + 2 h kappa), -2) / h^2; the face term belongs to
  A_h (not to N_h, so beta_n does not see it).
* Its diagonalisation, Sec. 4.2: H is not symmetric, but W H is, with
  W = diag(1/2, 1, .., 1, 1/2) (the trapezoid weights). So
  W^{1/2} H W^{-1/2} = Q Lambda Q^T with Q orthogonal, and
  S = W^{-1/2} Q, S^{-1} = Q^T W^{1/2} diagonalise H: H = S Lambda S^{-1}.
* Residual, Sec. 4 eq. F_u: F(U) = A_h vec(U) + N_h(U) with
  N_h(U) = b U^3 + V U - f (the linear coefficient lam stays in A_h, as in
  eq. linear_system).
* Quasi-Newton, Sec. 4 eq. identity-method, beta_n the mid-range of the
  diagonal Jacobian (N_h)_U = diag(3 b U^2 + V).
* Inverse, Sec. 4.1 eq. fin_inverse, with qn_oracle.fast_diag_solve (it takes
  S and S^{-1} separately, so a non-orthogonal S is fine).

* Nonlinear eigenproblem, Sec. 4.4 (eqs. Eigenvalue_p, system_qusi,
  system_normal): with f(U) = lam U + b U^3 + V U, each step takes the
  Rayleigh quotient lambda_n = <A U + f(U), U> / <U, U>, the residual
  F = A U + f(U) - lambda_n U, beta_n = mid-range of diag(3 b U^2 + V) - lambda_n
  (the Jacobian of N_h = f - lambda_n U with lambda_n held fixed), the update
  U~ = U - (A_h + beta_n I)^{-1} F and the normalisation U = U~ / ||U~||.

Readings (also listed in the design notes):
* The three-dimensional Example 1 of Sec. 6.3 has a u as a separate term; it
  is taken as the linear coefficient lam = a. beta_n then only sees
  3 b U^2 + V. Counting a inside N_h instead moves both end points of the
  spectrum by a and gives the same shift lam + beta_n.
* "n^3 degrees of freedom" with Neumann data is read as n nodes per axis,
  boundary nodes included (they are unknowns of the ghost-point scheme).
* Eigenproblem inner product: <U, W> = sum over nodes of m U W with the
  lumped mass m = h^dim times the trapezoid weights (1/2 per face the node
  lies on, Neumann data), the rectangle-rule L2 product the paper's M
  matrices stand for; A_h is self-adjoint in it. The stopping rule is the
  relative eigen-residual ||F|| / |lambda_n| <= tol (||U|| = 1).
"""
from __future__ import annotations

import math

import numpy as np

from .qn_oracle import fast_diag_solve

__all__ = ["mesh_width", "fd_matrix_1d", "eig_1d", "apply_operator", "potential", "residual",
           "jacobian_diag", "beta_rule", "qn_step", "qn_solve", "dense_operator", "newton_dense",
           "trapezoid_weights", "mass_weights", "eig_residual", "qn_eig_solve", "newton_eig_dense"]


def mesh_width(n: int, bc: str, length: float = 1.0) -> float:
    """h for n unknowns per axis: length/(n+1) (Dirichlet, interior nodes) or
    length/(n-1) (Neumann and Robin, both faces included, n >= 2)."""
    if bc == "dirichlet":
        return length / (n + 1)
    if bc in ("neumann", "robin"):
        if n < 2:
            raise ValueError("Neumann data needs n >= 2 nodes per axis")
        return length / (n - 1)
    raise ValueError(bc)


def trapezoid_weights(n: int, bc: str) -> np.ndarray:
    """W: ones, with 1/2 at the two face nodes for Neumann data."""
    w = np.ones(n)
    if bc in ("neumann", "robin"):
        w[0] = w[-1] = 0.5
    return w


def fd_matrix_1d(n: int, h: float, bc: str, kappa: float = 0.0) -> np.ndarray:
    """The 1-D second-difference matrix (Sec. 3.2): Dirichlet tridiag(-1, 2, -1)/h^2
    on the interior nodes; Neumann the same with the ghost rows (2, -2) and (-2, 2);
    Robin with the face diagonals 2 + 2 h kappa."""
    H = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    if bc in ("neumann", "robin"):
        H[0, 1] = -2.0
        H[n - 1, n - 2] = -2.0
    if bc == "robin":
        H[0, 0] += 2.0 * h * kappa
        H[n - 1, n - 1] += 2.0 * h * kappa
    return H / (h * h)


def eig_1d(n: int, h: float, bc: str, kappa: float = 0.0):
    """(S, S_inv, lam) with H = S diag(lam) S^{-1}, lam ascending (Sec. 4.2).

    W^{1/2} H W^{-1/2} is symmetric (W the trapezoid weights; W = I for Dirichlet)."""
    H = fd_matrix_1d(n, h, bc, kappa)
    sw = np.sqrt(trapezoid_weights(n, bc))
    Hs = (sw[:, None] * H) / sw[None, :]
    Hs = 0.5 * (Hs + Hs.T)                   # exact symmetry (the two halves agree to rounding)
    lam, Q = np.linalg.eigh(Hs)
    S = Q / sw[:, None]
    S_inv = Q.T * sw[None, :]
    return S, S_inv, lam


def apply_operator(U: np.ndarray, h: float, bc: str, kappa: float = 0.0) -> np.ndarray:
    """sum over axes of (2 u_i - u_{i-1} - u_{i+1}) / h^2 (eq. fdm-discrete); the
    value past a face is 0 (Dirichlet), the ghost value u_{-1} = u_1,
    u_n = u_{n-2} (Neumann: an even reflection about the face node), or that value
    minus 2 h kappa u_face (Robin)."""
    mode = "reflect" if bc in ("neumann", "robin") else "constant"
    n = U.shape[0]
    out = np.zeros_like(U)
    for axis in range(U.ndim):
        P = np.pad(U, [(1, 1) if a == axis else (0, 0) for a in range(U.ndim)], mode=mode)
        lo = [slice(None)] * U.ndim
        hi = [slice(None)] * U.ndim
        lo[axis] = slice(0, n)
        hi[axis] = slice(2, n + 2)
        out += (2.0 * U - P[tuple(lo)] - P[tuple(hi)]) / (h * h)
        if bc == "robin":   # the ghost's -2 h kappa u_face term, at both faces of this axis
            for face in (0, n - 1):
                sl = [slice(None)] * U.ndim
                sl[axis] = face
                out[tuple(sl)] += (2.0 * kappa / h) * U[tuple(sl)]
    return out


def potential(v, dim: int, n: int) -> np.ndarray:
    """V[.., y, x] = sum_a v_a(x_a) from the 1-D tables v = (v_x, v_y[, v_z]); a single
    table is used on every axis. None gives V = 0."""
    if v is None:
        return np.zeros((n,) * dim)
    v = np.asarray(v, dtype=np.float64)
    tabs = [v] * dim if v.ndim == 1 else [v[a] for a in range(dim)]
    V = np.zeros((n,) * dim)
    for a in range(dim):          # axis a (0 = x) is array axis dim-1-a
        shape = [1] * dim
        shape[dim - 1 - a] = n
        V = V + tabs[a].reshape(shape)
    return V


def residual(U, f, h: float, bc: str, lam: float = 0.0, b: float = 1.0, V=None, kappa: float = 0.0) -> np.ndarray:
    """F(U) = A_h vec(U) + N_h(U): apply_operator + lam U + b U^3 + V U - f."""
    r = apply_operator(U, h, bc, kappa) + lam * U + b * U ** 3 - f
    if V is not None:
        r = r + V * U
    return r


def jacobian_diag(U, b: float = 1.0, V=None) -> np.ndarray:
    """Diagonal of (N_h)_U: 3 b U^2 + V."""
    d = 3.0 * b * U * U
    return d if V is None else d + V


def beta_rule(U, b: float = 1.0, V=None) -> float:
    """beta_n = (lambda_max + lambda_min)/2 of diag(3 b U^2 + V) (eq. identity-method)."""
    d = jacobian_diag(U, b, V)
    return 0.5 * (float(d.max()) + float(d.min()))


def qn_step(U, f, h: float, bc: str, eig=None, lam: float = 0.0, b: float = 1.0, V=None,
            beta=None, step: float = 1.0):
    """One update of eq. identity-method. Returns (U_next, r, beta_used)."""
    S, S_inv, lam1d = eig if eig is not None else eig_1d(f.shape[0], h, bc)
    r = residual(U, f, h, bc, lam, b, V)
    beta_n = beta_rule(U, b, V) if beta is None else float(beta)
    return U - step * fast_diag_solve(r, S, S_inv, lam1d, lam + beta_n), r, beta_n


def qn_solve(f, h: float, bc: str, U0=None, tol: float = 1e-10, max_it: int = 500,
             lam: float = 0.0, b: float = 1.0, V=None, beta=None, step: float = 1.0, kappa: float = 0.0):
    """Iterate eq. identity-method until ||F(U)||_2 / ||f||_2 <= tol.

    Returns (U, history, converged) as qn_oracle.qn_solve; history entries hold
    rel, res, beta, fu_min and fu_max (the extremes of 3 b U^2 + V)."""
    n = f.shape[0]
    S, S_inv, lam1d = eig_1d(n, h, bc, kappa)
    U = np.zeros_like(f) if U0 is None else np.array(U0, dtype=np.float64, copy=True)
    fnorm = float(np.linalg.norm(f.ravel()))
    history = []
    for it in range(max_it + 1):
        r = residual(U, f, h, bc, lam, b, V, kappa)
        rnorm = float(np.linalg.norm(r.ravel()))
        rel = rnorm / fnorm
        d = jacobian_diag(U, b, V)
        beta_n = 0.5 * (float(d.max()) + float(d.min())) if beta is None else float(beta)
        history.append({"rel": rel, "res": rnorm, "beta": beta_n,
                        "fu_min": float(d.min()), "fu_max": float(d.max())})
        if rel <= tol:
            return U, history, True
        if not math.isfinite(rel) or it == max_it:
            break
        U = U - step * fast_diag_solve(r, S, S_inv, lam1d, lam + beta_n)
    return U, history, False


def dense_operator(n: int, dim: int, h: float, bc: str, lam: float = 0.0, kappa: float = 0.0) -> np.ndarray:
    """A_h = sum_a I..H_a..I + lam I as an explicit matrix (Kronecker products of
    fd_matrix_1d, eq. A_definition), acting on the C-order ravel (x fastest)."""
    H = fd_matrix_1d(n, h, bc, kappa)
    I = np.eye(n)
    if dim == 2:
        A = np.kron(I, H) + np.kron(H, I)
    elif dim == 3:
        A = np.kron(np.kron(I, I), H) + np.kron(np.kron(I, H), I) + np.kron(np.kron(H, I), I)
    else:
        raise ValueError("dim must be 2 or 3")
    return A + lam * np.eye(n ** dim)


def newton_dense(f, h: float, bc: str, U0=None, tol: float = 1e-12, max_it: int = 50,
                 lam: float = 0.0, b: float = 1.0, V=None):
    """Newton's method (eq. newton) with the dense Jacobian A_h + diag(3 b U^2 + V)."""
    n, dim = f.shape[0], f.ndim
    A = dense_operator(n, dim, h, bc, lam)
    Vv = np.zeros(f.size) if V is None else V.ravel()
    u = np.zeros(f.size) if U0 is None else np.array(U0, dtype=np.float64).ravel()
    fv = f.ravel()
    fnorm = float(np.linalg.norm(fv))
    for _ in range(max_it):
        F = A @ u + b * u ** 3 + Vv * u - fv
        if np.linalg.norm(F) / fnorm <= tol:
            break
        J = A + np.diag(3.0 * b * u * u + Vv)
        u = u - np.linalg.solve(J, F)
    return u.reshape(f.shape)


# ----------------------------------------------------------------------------
# Nonlinear eigenproblem (Sec. 4.4)
# ----------------------------------------------------------------------------
def mass_weights(n: int, dim: int, h: float, bc: str) -> np.ndarray:
    """Lumped mass per node: h^dim times the product of the 1-D trapezoid weights."""
    w = trapezoid_weights(n, bc)
    m = np.ones((n,) * dim) * h ** dim
    for a in range(dim):
        shape = [1] * dim
        shape[a] = n
        m = m * w.reshape(shape)
    return m


def eig_residual(U, h: float, bc: str, lam: float = 0.0, b: float = 1.0, V=None):
    """(F, lambda_n): lambda_n = <A U + f(U), U> / <U, U> (Sec. 4.4), F = A U + f(U) - lambda_n U
    with f(U) = lam U + b U^3 + V U and the mass-weighted product."""
    m = mass_weights(U.shape[0], U.ndim, h, bc)
    r0 = residual(U, np.zeros_like(U), h, bc, lam, b, V)
    lam_n = float(np.sum(m * r0 * U)) / float(np.sum(m * U * U))
    return r0 - lam_n * U, lam_n


def qn_eig_solve(U0, h: float, bc: str, lam: float = 0.0, b: float = 1.0, V=None, tol: float = 1e-10,
                 max_it: int = 5000):
    """Quasi-Newton for the nonlinear eigenproblem (Sec. 4.4 eqs. system_qusi, system_normal).

    U0 is normalised first (<U0, U0> = 1). Each step: lambda_n and F (eig_residual);
    stop when ||F|| / |lambda_n| <= tol; beta_n = (max + min)/2 of 3 b U^2 + V, minus
    lambda_n (lam counts in f, so A_h here is the difference operator alone and the
    shift is lam + mid-range - lambda_n = beta_n as computed); U~ = U - (A_h + beta_n I)^{-1} F;
    then U = U~ / ||U~||.
    Returns (U, lambda_n, history, converged); history[i] has rel, lambda and beta of U_i."""
    n, dim = U0.shape[0], U0.ndim
    m = mass_weights(n, dim, h, bc)
    S, S_inv, lam1d = eig_1d(n, h, bc)
    U = np.array(U0, dtype=np.float64, copy=True)
    U = U / math.sqrt(float(np.sum(m * U * U)))
    history = []
    for it in range(max_it + 1):
        F, lam_n = eig_residual(U, h, bc, lam, b, V)
        rel = math.sqrt(float(np.sum(m * F * F))) / abs(lam_n)
        d = jacobian_diag(U, b, V) + lam
        beta_n = 0.5 * (float(d.max()) + float(d.min())) - lam_n
        history.append({"rel": rel, "lambda": lam_n, "beta": beta_n})
        if rel <= tol:
            return U, lam_n, history, True
        if not math.isfinite(rel) or it == max_it:
            break
        Ut = U - fast_diag_solve(F, S, S_inv, lam1d, beta_n)
        U = Ut / math.sqrt(float(np.sum(m * Ut * Ut)))
    return U, lam_n, history, False


def newton_eig_dense(U0, lam0: float, h: float, bc: str, lam: float = 0.0, b: float = 1.0, V=None,
                     tol: float = 1e-13, max_it: int = 50):
    """Newton's method on the bordered system A U + f(U) - lambda U = 0, (<U, U> - 1)/2 = 0
    for the unknowns (U, lambda), dense (tiny grids)."""
    n, dim = U0.shape[0], U0.ndim
    A = dense_operator(n, dim, h, bc, lam)
    mv = mass_weights(n, dim, h, bc).ravel()
    Vv = np.zeros(U0.size) if V is None else V.ravel()
    u = np.array(U0, dtype=np.float64).ravel()
    lm = float(lam0)
    N = u.size
    for _ in range(max_it):
        F1 = A @ u + b * u ** 3 + Vv * u - lm * u
        F2 = 0.5 * (float(np.sum(mv * u * u)) - 1.0)
        if math.sqrt(float(np.sum(F1 * F1)) + F2 * F2) <= tol * abs(lm) * math.sqrt(N):
            break
        J = np.zeros((N + 1, N + 1))
        J[:N, :N] = A + np.diag(3.0 * b * u * u + Vv - lm)
        J[:N, N] = -u
        J[N, :N] = mv * u
        step = np.linalg.solve(J, np.concatenate([F1, [F2]]))
        u = u - step[:N]
        lm = lm - step[N]
    return u.reshape(U0.shape), lm
