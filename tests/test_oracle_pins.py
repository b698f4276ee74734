"""Pins for the FP64 oracle: each check ties the oracle to something other than
itself (a closed form, an independently built dense matrix, a library direct
solve, Newton's method, the convergence theorem), so that a dropped term, a
wrong sign or index, or a transposed operand anywhere in it fails a check.

The `check_*` functions take the oracle module as an argument so that the
mutation tests at the end can plant a mistake in a copy of the oracle (on the
CPU) and confirm that some check catches it.
"""
import copy
import math
import types

import numpy as np
import pytest

import oracle as O
import oracle.qn_oracle as OQ
from paper_2502_03611_gb300.inputs import (SplitMix64, grid_points, manufactured_problem,
                                           random_field)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def closed_form_eigs(n):
    """Textbook (DST-I) eigenpairs of (1/h^2) tridiag(-1,2,-1), h = 1/(n+1):
    lambda_k = (4/h^2) sin^2(k pi h / 2), v_k[j] = sqrt(2h) sin(j k pi h)."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    lam = 4.0 / h ** 2 * np.sin(k * math.pi * h / 2.0) ** 2
    V = math.sqrt(2.0 * h) * np.sin(np.outer(k, k) * math.pi * h)
    return V, lam


def eigenmode(n, ks):
    """prod_a sin(k_a pi x_a) on the grid, C order with x fastest (ks = (k_x, k_y[, k_z]))."""
    x = grid_points(n)
    vecs = [np.sin(k * math.pi * x) for k in ks]
    if len(ks) == 2:
        return np.outer(vecs[1], vecs[0])
    return np.einsum("z,y,x->zyx", vecs[2], vecs[1], vecs[0])


def check_eig(M):
    for n in (1, 2, 7, 63):
        S, S_inv, lam = M.eig_1d(n)
        V, lam_cf = closed_form_eigs(n)
        scale = lam_cf.max()
        assert np.allclose(lam, lam_cf, rtol=0, atol=1e-12 * scale)
        # eigenvectors agree with the closed form up to a sign per column
        for k in range(n):
            s = np.sign(S[:, k] @ V[:, k])
            assert np.abs(S[:, k] - s * V[:, k]).max() < 1e-10
        assert np.abs(S_inv @ S - np.eye(n)).max() < 1e-12
        H = M.fd_matrix_1d(n)
        assert np.abs(H @ S - S * lam[None, :]).max() < 1e-12 * scale


def check_stencil(M):
    # stencil against the Kronecker-sum matrix built from the explicit 1-D matrix
    for n, dim in ((5, 2), (4, 3), (1, 3)):
        U = random_field((n,) * dim, seed=11 + n)
        A = M.dense_operator(n, dim)
        assert np.allclose(M.apply_laplacian(U).ravel(), A @ U.ravel(), rtol=1e-13, atol=1e-10)
    # the same matrix built independently from the paper's eq. Sy entries
    n = 4
    h2 = (1.0 / (n + 1)) ** 2
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] = 2.0 / h2
        if i > 0:
            T[i, i - 1] = -1.0 / h2
        if i + 1 < n:
            T[i, i + 1] = -1.0 / h2
    I = np.eye(n)
    A2 = np.kron(I, T) + np.kron(T, I)
    assert np.allclose(M.dense_operator(n, 2), A2, rtol=1e-14, atol=1e-9)
    # discrete eigenmodes: A_h mode = (sum of closed-form eigenvalues) mode
    n = 9
    _, lam_cf = closed_form_eigs(n)
    for ks in ((1, 1), (2, 5), (9, 3)):
        E = eigenmode(n, ks)
        target = (lam_cf[ks[0] - 1] + lam_cf[ks[1] - 1]) * E
        assert np.abs(M.apply_laplacian(E) - target).max() < 1e-9 * np.abs(target).max()
    for ks in ((1, 2, 3), (7, 1, 4)):
        E = eigenmode(n, ks)
        target = sum(lam_cf[k - 1] for k in ks) * E
        assert np.abs(M.apply_laplacian(E) - target).max() < 1e-9 * np.abs(target).max()


def check_residual(M):
    # F(U) = A_h U + lam U + b U^3 - f, checked pointwise against the stencil
    # written out by hand at one interior and one boundary-adjacent node
    n = 6
    U = random_field((n, n, n), seed=5)
    f = random_field((n, n, n), seed=6)
    lam, b = 0.7, 1.3
    R = M.residual(U, f, lam, b)
    h2 = (1.0 / (n + 1)) ** 2

    def get(z, y, x):
        if 0 <= z < n and 0 <= y < n and 0 <= x < n:
            return U[z, y, x]
        return 0.0

    for (z, y, x) in ((2, 3, 1), (0, 5, 0), (5, 0, 5)):
        lap = (6 * U[z, y, x] - get(z, y, x - 1) - get(z, y, x + 1) - get(z, y - 1, x)
               - get(z, y + 1, x) - get(z - 1, y, x) - get(z + 1, y, x)) / h2
        want = lap + lam * U[z, y, x] + b * U[z, y, x] ** 3 - f[z, y, x]
        assert abs(R[z, y, x] - want) < 1e-12 * max(1.0, abs(lap))


def check_fast_diag(M):
    # against a library dense direct solve of (A_h + shift I) v = r
    for n, dim in ((6, 2), (4, 3), (1, 2)):
        S, S_inv, lam = M.eig_1d(n)
        A = M.dense_operator(n, dim)
        for shift in (0.0, 2.5, 37.0):
            r = random_field((n,) * dim, seed=100 + n)
            v = M.fast_diag_solve(r, S, S_inv, lam, shift)
            want = np.linalg.solve(A + shift * np.eye(n ** dim), r.ravel())
            assert np.abs(v.ravel() - want).max() < 1e-12 * np.abs(want).max()
    # non-cubic-symmetric input (different structure along each axis)
    n = 5
    S, S_inv, lam = M.eig_1d(n)
    r = random_field((n, n, n), seed=9) * np.arange(1, n + 1)[None, None, :]
    A = M.dense_operator(n, 3)
    v = M.fast_diag_solve(r, S, S_inv, lam, 1.0)
    want = np.linalg.solve(A + np.eye(n ** 3), r.ravel())
    assert np.abs(v.ravel() - want).max() < 1e-12 * np.abs(want).max()
    # closed-form special case: an eigenmode right-hand side
    n = 11
    S, S_inv, lam = M.eig_1d(n)
    _, lam_cf = closed_form_eigs(n)
    for ks, shift in (((2, 3, 4), 0.0), ((1, 11, 6), 5.0)):
        E = eigenmode(n, ks)
        v = M.fast_diag_solve(E, S, S_inv, lam, shift)
        want = E / (sum(lam_cf[k - 1] for k in ks) + shift)
        assert np.abs(v - want).max() < 1e-12 * np.abs(want).max()


def check_beta(M):
    U = np.array([[0.5, -2.0], [1.0, 0.0]])
    # (N_h)_U = diag(3 b U^2) -> {0.75, 12, 3, 0}; midpoint of [0, 12] = 6
    assert M.beta_rule(U, 1.0) == pytest.approx(6.0, rel=1e-15)
    assert M.beta_rule(U, 2.0) == pytest.approx(12.0, rel=1e-15)
    assert M.beta_rule(np.zeros((3, 3)), 1.0) == 0.0


def check_linear_one_step(M):
    # b = 0: the problem is linear, (A_h + 0 I)^{-1} is the exact inverse, so
    # one quasi-Newton step from 0 solves it.
    for n, dim in ((17, 2), (9, 3)):
        _, f = manufactured_problem(n, dim, seed=3, b=0.0)
        U, hist, ok = M.qn_solve(f, b=0.0, tol=1e-12, max_it=3)
        assert ok and len(hist) - 1 == 1
        A = M.dense_operator(n, dim)
        assert np.abs(A @ U.ravel() - f.ravel()).max() < 1e-10 * np.abs(f).max()


def check_discrete_recovery(M):
    # f_disc = A_h u* + u*^3 -> the discrete solution is u* itself
    for n, dim in ((63, 2), (15, 3)):
        u, _ = manufactured_problem(n, dim, seed=1)
        f = M.discrete_source(u)
        U, hist, ok = M.qn_solve(f, tol=1e-12)
        assert ok
        assert np.abs(U - u).max() < 1e-10 * np.abs(u).max()


def check_newton(M):
    for n, dim in ((15, 2), (7, 3)):
        _, f = manufactured_problem(n, dim, seed=2)
        Uq, _, ok = M.qn_solve(f, tol=1e-13)
        assert ok
        Un = M.newton_dense(f, tol=1e-14)
        assert np.abs(Uq - Un).max() < 1e-12 * np.abs(Un).max()
        # Newton's own residual, from the explicit dense operator
        A = M.dense_operator(n, dim)
        F = A @ Un.ravel() + Un.ravel() ** 3 - f.ravel()
        assert np.linalg.norm(F) < 1e-12 * np.linalg.norm(f)


def check_second_order(M):
    errs = []
    for n in (15, 31, 63):
        u, f = manufactured_problem(n, 2, seed=0)
        U, _, ok = M.qn_solve(f)
        assert ok
        errs.append(np.abs(U - u).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for q in ratios:
        assert 3.5 < q < 4.5, ratios


def check_contraction(M):
    # Theorem 1: near the solution, ||e_{n+1}|| <= (g(beta_n) + O(||e_n||)) ||e_n||
    n = 31
    _, f = manufactured_problem(n, 2, seed=0)
    f = 20.0 * f
    Uh, _, ok = M.qn_solve(f, tol=1e-13, max_it=400)
    assert ok
    S, S_inv, lam = M.eig_1d(n)
    lam_min_A = 2.0 * lam[0]
    U = np.zeros_like(f)
    checked = 0
    for _ in range(30):
        beta = M.beta_rule(U)
        d = M.jacobian_diag(U)
        g = M.contraction_bound(beta, d.min(), d.max(), lam_min_A)
        e0 = np.linalg.norm(U - Uh)
        U, _, _ = M.qn_step(U, f, (S, S_inv, lam))
        e1 = np.linalg.norm(U - Uh)
        if e0 < 1e-2 * np.linalg.norm(Uh):
            assert e1 <= (g + 0.02) * e0
            checked += 1
    assert checked >= 5
    # Remark "Optimal beta": the midpoint needs fewer iterations than either end point
    its = {}
    for rule in (None, "max"):
        _, hist, ok = M.qn_solve(f, beta=rule, tol=1e-10, max_it=400)
        assert ok
        its[rule] = len(hist) - 1
    _, hist_min, ok_min = M.qn_solve(f, beta="min", tol=1e-10, max_it=400)
    assert its[None] < its["max"]
    assert (not ok_min) or its[None] <= len(hist_min) - 1


def check_system(M):
    # coupled pair (Sec. 4.3): the 2x2 block eigenvalues against numpy's eigvals
    rng = np.random.default_rng(0)
    U = rng.standard_normal((4, 4))
    V = rng.standard_normal((4, 4))
    alpha = 0.6
    lo, hi = np.inf, -np.inf
    for u, v in zip(U.ravel(), V.ravel()):
        ev = np.linalg.eigvals(np.array([[3 * u * u, alpha], [-alpha, 3 * v * v]]))
        lo = min(lo, ev.real.min())
        hi = max(hi, ev.real.max())
    assert M.system_beta(U, V, alpha) == pytest.approx(0.5 * (lo + hi), rel=1e-12)
    # the system solve reaches the dense Newton solution of the coupled problem
    n = 9
    _, f1 = manufactured_problem(n, 2, seed=4)
    _, f2 = manufactured_problem(n, 2, seed=5)
    D = 2.5
    Uq, Vq, hist, ok = M.qn_solve_system(f1, f2, alpha, D, tol=1e-13)
    assert ok
    A = M.dense_operator(n, 2)
    N = n * n
    w = np.zeros(2 * N)
    for _ in range(30):
        u, v = w[:N], w[N:]
        F = np.concatenate([A @ u + u ** 3 + alpha * v - f1.ravel(),
                            D * (A @ v) + v ** 3 - alpha * u - f2.ravel()])
        J = np.block([[A + np.diag(3 * u * u), alpha * np.eye(N)],
                      [-alpha * np.eye(N), D * A + np.diag(3 * v * v)]])
        w = w - np.linalg.solve(J, F)
    assert np.abs(Uq.ravel() - w[:N]).max() < 1e-11 * np.abs(w).max()
    assert np.abs(Vq.ravel() - w[N:]).max() < 1e-11 * np.abs(w).max()


CHECKS = [check_eig, check_stencil, check_residual, check_fast_diag, check_beta,
          check_linear_one_step, check_discrete_recovery, check_newton,
          check_second_order, check_contraction, check_system]


@pytest.mark.parametrize("check", CHECKS, ids=[c.__name__ for c in CHECKS])
def test_oracle_pin(check):
    check(OQ)


# ---------------------------------------------------------------------------
# input generator
# ---------------------------------------------------------------------------
def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 0 (the generator's reference values)
    r = SplitMix64(0)
    got = [r.next_u64() for _ in range(4)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_random_field_matches_stream():
    r = SplitMix64(123)
    want = np.array([r.next_uniform(-1, 1) for _ in range(10)])
    assert np.array_equal(random_field((10,), 123), want)


def test_normals_moments():
    z = SplitMix64(7).normals(20000)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03


def test_manufactured_solution_pointwise():
    n, K = 7, 6
    u, f = manufactured_problem(n, 3, seed=0)
    from paper_2502_03611_gb300.inputs import manufactured_coeffs
    c = 0.1 * manufactured_coeffs(0, 3, K)
    c[0, 0, 0] += 1.0
    x = grid_points(n)
    i, j, k = 1, 4, 6          # x, y, z node indices
    val = lap = 0.0
    for a in range(K):
        for bb in range(K):
            for d in range(K):
                m = (math.sin((d + 1) * math.pi * x[i]) * math.sin((bb + 1) * math.pi * x[j])
                     * math.sin((a + 1) * math.pi * x[k]))
                val += c[a, bb, d] * m
                lap += c[a, bb, d] * math.pi ** 2 * ((a + 1) ** 2 + (bb + 1) ** 2 + (d + 1) ** 2) * m
    assert u[k, j, i] == pytest.approx(val, rel=1e-13, abs=1e-15)
    assert f[k, j, i] == pytest.approx(lap + val ** 3, rel=1e-13)


# ---------------------------------------------------------------------------
# planted mistakes: each mutant of the oracle must fail at least one check
# ---------------------------------------------------------------------------
def _mutant(**overrides):
    m = types.ModuleType("oracle_mutant")
    m.__dict__.update({k: v for k, v in OQ.__dict__.items() if not k.startswith("__")})
    # rebind every function's globals to the mutant namespace so internal
    # calls see the planted mistake
    for name, obj in list(m.__dict__.items()):
        if isinstance(obj, types.FunctionType):
            m.__dict__[name] = types.FunctionType(obj.__code__, m.__dict__, obj.__name__,
                                                  obj.__defaults__, obj.__closure__)
    for name, fn in overrides.items():
        m.__dict__[name] = types.FunctionType(fn.__code__, m.__dict__, name,
                                              fn.__defaults__, fn.__closure__)
    return m


def _lap_one_axis_missing(U):
    n = U.shape[0]
    h2 = (1.0 / (n + 1)) ** 2
    out = np.zeros_like(U)
    for axis in range(U.ndim - 1):
        P = np.pad(U, [(1, 1) if a == axis else (0, 0) for a in range(U.ndim)])
        lo = [slice(None)] * U.ndim
        hi = [slice(None)] * U.ndim
        lo[axis] = slice(0, n)
        hi[axis] = slice(2, n + 2)
        out += (2.0 * U - P[tuple(lo)] - P[tuple(hi)]) / h2
    return out


def _mode_product_transposed(X, M, axis):
    Y = np.tensordot(M.T, X, axes=([1], [axis]))
    return np.moveaxis(Y, 0, axis)


def _h_off_by_one(n):
    h = 1.0 / n
    H = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return H / (h * h)


def _residual_wrong_sign(U, f, lam=0.0, b=1.0):
    return apply_laplacian(U) + lam * U - b * U ** 3 - f  # noqa: F821 (mutant namespace)


def _beta_max_only(U, b=1.0):
    d = jacobian_diag(U, b)  # noqa: F821
    return float(d.max())


def _fast_diag_no_shift(r, S, S_inv, lam1d, shift):
    return _orig_fast_diag(r, S, S_inv, lam1d, 0.0)  # noqa: F821


MUTANTS = {
    "laplacian_drops_axis": dict(apply_laplacian=_lap_one_axis_missing),
    "mode_product_transposed": dict(mode_product=_mode_product_transposed),
    "h_off_by_one": dict(fd_matrix_1d=_h_off_by_one),
    "cube_wrong_sign": dict(residual=_residual_wrong_sign),
    "beta_uses_max": dict(beta_rule=_beta_max_only),
}


@pytest.mark.parametrize("name", sorted(MUTANTS) + ["shift_dropped"])
def test_planted_mistake_is_caught(name):
    if name == "shift_dropped":
        m = _mutant(fast_diag_solve=_fast_diag_no_shift)
        m.__dict__["_orig_fast_diag"] = _mutant().fast_diag_solve
    else:
        m = _mutant(**MUTANTS[name])
    caught = 0
    for check in (check_eig, check_stencil, check_residual, check_fast_diag, check_beta,
                  check_discrete_recovery):
        try:
            check(m)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError):
            caught += 1
    assert caught >= 1, f"planted mistake {name} escaped every pin"
