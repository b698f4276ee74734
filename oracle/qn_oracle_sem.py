"""Plain FP64 CPU oracle for the spectral element discretisation (Sec. 3.1).

TEST INFRASTRUCTURE, like qn_oracle: only tests, the smoke check and the
benchmark's CPU-baseline and reference legs may use it; the CUDA library
shares no code with it.

What is computed (float64 numpy; numpy.polynomial.legendre supplies Legendre
values, derivatives and roots as library steps):

* 1-D Q^k elements with Lagrange bases at the k+1 Gauss-Lobatto points and
  (k+1)-point Gauss-Lobatto quadrature (Sec. 3.1 and its remark on the
  integration): on each element of width h_e the stiffness
  K_ij = int l_i' l_j' and the mass, which the quadrature makes diagonal,
  m_i = (h_e / 2) w_i. Assembled over E equal elements of [0, L]
  (Sec. 3.1 eqs. S_x, M_x).
* Boundary data (Sec. 3.1): Dirichlet keeps the interior nodes (a submatrix
  of S and M), n = E k - 1 unknowns; Neumann keeps all n = E k + 1 nodes
  (zero flux adds no boundary term).
* The system of eq. final-system-3d: A_h = sum_a I..H_a..I + lam I with
  H = M^{-1} S, N_h(U) = b U^3 + V U - f at the nodes (the quadrature
  evaluates the nonlinearity pointwise, Sec. 3.1 remark).
* Diagonalisation (Sec. 4.2): M^{-1/2} S M^{-1/2} = Q Lambda Q^T (eigh),
  S_e = M^{-1/2} Q, S_e^{-1} = Q^T M^{1/2}; the inverse and the quasi-Newton
  loop are qn_oracle's and qn_oracle_bc's.

Readings (also listed in the design notes):
* Degree k and the element count E fix n; the user gives n and k, and n + 1
  (Dirichlet) or n - 1 (Neumann) must be a multiple of k.
* Equal elements on [0, L]; nodes of element e at e h_e + (1 + xi_q) h_e / 2.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as L

from .qn_oracle import fast_diag_solve

__all__ = ["gll", "lagrange_derivative", "element_matrices", "assemble_1d", "eig_1d", "apply_operator",
           "residual", "qn_solve", "dense_operator", "elements_for"]


def gll(k: int):
    """Gauss-Lobatto nodes (ascending, on [-1, 1]) and weights for degree k >= 1:
    the ends and the roots of P_k'; w_i = 2 / (k (k+1) P_k(x_i)^2)."""
    if k < 1:
        raise ValueError("k >= 1")
    ck = np.zeros(k + 1)
    ck[k] = 1.0
    inner = L.legroots(L.legder(ck)) if k >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    w = 2.0 / (k * (k + 1) * L.legval(x, ck) ** 2)
    return x, w


def lagrange_derivative(x: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(x_i) for the Lagrange basis on nodes x (barycentric form)."""
    m = x.size
    b = np.array([1.0 / np.prod([x[j] - x[q] for q in range(m) if q != j]) for j in range(m)])
    D = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def element_matrices(k: int, he: float):
    """(K, m): element stiffness (k+1)^2 and lumped mass diagonal on an element of width he."""
    xi, w = gll(k)
    D = lagrange_derivative(xi)
    K = (2.0 / he) * (D.T * w[None, :]) @ D          # sum_q w_q l_i'(xi_q) l_j'(xi_q) * 2/he
    return K, 0.5 * he * w


def elements_for(n: int, k: int, bc: str) -> int:
    """Element count E for n unknowns per axis."""
    tot = n + 1 if bc == "dirichlet" else n - 1
    if tot < k or tot % k:
        raise ValueError(f"n = {n} does not fit Q^{k} elements with {bc} data")
    return tot // k


def assemble_1d(n: int, k: int, length: float, bc: str):
    """(S, m, x): the assembled stiffness (n x n), lumped mass diagonal (n) and nodes of the
    unknowns on [0, length]."""
    E = elements_for(n, k, bc)
    he = length / E
    K, me = element_matrices(k, he)
    xi, _ = gll(k)
    G = E * k + 1
    S = np.zeros((G, G))
    m = np.zeros(G)
    xs = np.zeros(G)
    for e in range(E):
        idx = e * k + np.arange(k + 1)
        S[np.ix_(idx, idx)] += K
        m[idx] += me
        xs[idx] = e * he + 0.5 * (1.0 + xi) * he
    keep = slice(1, G - 1) if bc == "dirichlet" else slice(0, G)
    return S[keep, keep].copy(), m[keep].copy(), xs[keep].copy()


def eig_1d(n: int, k: int, length: float, bc: str):
    """(S_e, S_e^{-1}, lam, H) with H = M^{-1} S = S_e diag(lam) S_e^{-1}, lam ascending."""
    S, m, _ = assemble_1d(n, k, length, bc)
    r = 1.0 / np.sqrt(m)
    Hs = r[:, None] * S * r[None, :]
    lam, Q = np.linalg.eigh(0.5 * (Hs + Hs.T))
    return r[:, None] * Q, Q.T * np.sqrt(m)[None, :], lam, S / m[:, None]


def apply_operator(U: np.ndarray, H: np.ndarray) -> np.ndarray:
    """sum over axes of H applied along that axis (eq. final-system-3d without lam)."""
    out = np.zeros_like(U)
    for axis in range(U.ndim):
        out += np.moveaxis(np.tensordot(H, U, axes=([1], [axis])), 0, axis)
    return out


def residual(U, f, H, lam: float = 0.0, b: float = 1.0, V=None):
    r = apply_operator(U, H) + lam * U + b * U ** 3 - f
    return r if V is None else r + V * U


def dense_operator(H: np.ndarray, dim: int, lam: float = 0.0) -> np.ndarray:
    n = H.shape[0]
    I = np.eye(n)
    if dim == 2:
        A = np.kron(I, H) + np.kron(H, I)
    else:
        A = np.kron(np.kron(I, I), H) + np.kron(np.kron(I, H), I) + np.kron(np.kron(H, I), I)
    return A + lam * np.eye(n ** dim)


def qn_solve(f, k: int, length: float, bc: str, U0=None, tol: float = 1e-10, max_it: int = 500,
             lam: float = 0.0, b: float = 1.0, V=None, beta=None, step: float = 1.0):
    """Quasi-Newton (Sec. 4 eq. identity-method) on the SEM system; returns (U, history, converged)."""
    n = f.shape[0]
    S_e, S_inv, lam1d, H = eig_1d(n, k, length, bc)
    U = np.zeros_like(f) if U0 is None else np.array(U0, dtype=np.float64, copy=True)
    fnorm = float(np.linalg.norm(f.ravel()))
    history = []
    for it in range(max_it + 1):
        r = residual(U, f, H, lam, b, V)
        rel = float(np.linalg.norm(r.ravel())) / fnorm
        d = 3.0 * b * U * U + (0.0 if V is None else V)
        beta_n = 0.5 * (float(np.max(d)) + float(np.min(d))) if beta is None else float(beta)
        history.append({"rel": rel, "beta": beta_n})
        if rel <= tol:
            return U, history, True
        if not math.isfinite(rel) or it == max_it:
            break
        U = U - step * fast_diag_solve(r, S_e, S_inv, lam1d, lam + beta_n)
    return U, history, False
