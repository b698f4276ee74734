"""Seeded synthetic inputs for the quasi-linear elliptic model problem.

This module is shared by the CUDA path's tests and benchmark and by the FP64
oracle's tests. It holds none of the quasi-Newton method's arithmetic
(no residual, no eigen-decomposition, no mode products, no beta rule): it only
draws random coefficients and evaluates the problem data of the model problem
(Sec. 2, eq. main-pde, with lambda u + b u^3 as the nonlinearity) from
closed-form sine series.

Grid (Sec. 3.2, Dirichlet case): n interior points per axis on (0,1),
h = 1/(n+1), x_i = i*h for i = 1..n. Arrays are C-ordered with the x index
fastest: a 2-D field is U[y, x], a 3-D field is U[z, y, x], which is the
column-major vec() ordering the paper uses with vec(A X B^T) = (B kron A) vec(X).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) mapped to (0,1) with 53-bit
resolution and to N(0,1) by the Box-Muller transform (cosine branch).
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 stream: state += golden gamma, then the 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def next_unit(self) -> float:
        """Uniform on the open interval (0, 1): ((u >> 11) + 0.5) * 2^-53."""
        return ((self.next_u64() >> 11) + 0.5) * (1.0 / 9007199254740992.0)

    def next_uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.next_unit()

    def next_normal(self) -> float:
        """Standard normal from two uniforms (Box-Muller, cosine branch only)."""
        u1 = self.next_unit()
        u2 = self.next_unit()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def normals(self, count: int) -> np.ndarray:
        return np.array([self.next_normal() for _ in range(count)], dtype=np.float64)


def grid_h(n: int) -> float:
    """Mesh width for n interior points on (0,1) with Dirichlet ends."""
    return 1.0 / (n + 1)


def grid_points(n: int) -> np.ndarray:
    """Interior nodes x_i = i*h, i = 1..n."""
    return np.arange(1, n + 1, dtype=np.float64) * grid_h(n)


def sine_basis(n: int, kmax: int) -> np.ndarray:
    """B[k-1, i] = sin(k*pi*x_i) for k = 1..kmax, i over interior nodes."""
    k = np.arange(1, kmax + 1, dtype=np.float64)[:, None]
    return np.sin(k * math.pi * grid_points(n)[None, :])


def manufactured_coeffs(seed: int, dim: int, kmax: int) -> np.ndarray:
    """c[k_z, k_y, k_x] ~ N(0,1) (dim=3) or c[k_y, k_x] (dim=2).

    Drawn in C order, i.e. lexicographic with the x mode index fastest.
    """
    rng = SplitMix64(seed)
    return rng.normals(kmax ** dim).reshape((kmax,) * dim)


def sine_series(coef: np.ndarray, n: int) -> np.ndarray:
    """Evaluate sum_k coef[k] * prod_a sin(k_a pi x_a) on the n^dim interior grid.

    The sum is separable, so it is evaluated one axis at a time; the result
    is exact up to rounding (no truncation).
    """
    dim = coef.ndim
    kmax = coef.shape[0]
    B = sine_basis(n, kmax)                      # (kmax, n)
    if dim == 2:
        return B.T @ coef @ B                    # [y, x]
    if dim == 3:
        t = np.tensordot(coef, B, axes=([2], [0]))           # [kz, ky, x]
        t = np.tensordot(t, B, axes=([1], [0]))              # [kz, x, y]
        t = np.ascontiguousarray(t.transpose(0, 2, 1))       # [kz, y, x]
        out = B.T @ t.reshape(kmax, n * n)                   # [z, y*x]
        return out.reshape(n, n, n)
    raise ValueError("dim must be 2 or 3")


def mode_wavenumber_sq(kmax: int, dim: int) -> np.ndarray:
    """|k|^2 = sum_a k_a^2 for the mode index tensor (1-based modes)."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    if dim == 2:
        return k[:, None] ** 2 + k[None, :] ** 2
    return k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2


def manufactured_problem(n: int, dim: int, seed: int, kmax: int | None = None,
                         amp: float = 0.1, lam: float = 0.0, b: float = 1.0):
    """Manufactured solution and source for -Lap u + lam u + b u^3 = f on (0,1)^dim.

    u* = prod_a sin(pi x_a) + amp * sum_{k in {1..kmax}^dim} c_k prod_a sin(k_a pi x_a),
    c_k ~ N(0,1) from SplitMix64(seed). f is the continuous source
    -Lap u* + lam u* + b u*^3 sampled at the interior nodes; -Lap of a sine
    mode is pi^2 |k|^2 times the mode. kmax defaults to 4 in 2-D and 6 in 3-D.

    Returns (u_star, f), float64 arrays of shape (n,)*dim, x fastest.
    """
    if kmax is None:
        kmax = 4 if dim == 2 else 6
    coef = amp * manufactured_coeffs(seed, dim, kmax)
    coef[(0,) * dim] += 1.0
    u = sine_series(coef, n)
    lap = sine_series(coef * (math.pi ** 2) * mode_wavenumber_sq(kmax, dim), n)
    f = lap + lam * u + b * u ** 3
    return u, f


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform random array (for operator tests), drawn in C order.

    Vectorised SplitMix64: element i uses the stream state seed + (i+1)*gamma,
    which is exactly the i-th output of SplitMix64(seed).
    """
    count = int(np.prod(shape))
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    unit = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * unit).reshape(shape)


# ---------------------------------------------------------------------------
# coupled two-component systems (batched workload)
# ---------------------------------------------------------------------------
COUPLED_SIZES = (63, 127, 255, 511)


def coupled_params(seed: int, i: int, sizes=COUPLED_SIZES):
    """(n, alpha, D) of instance i of batch `seed`: SplitMix64(seed*1000 + i)
    draws n uniformly from `sizes`, alpha ~ U[0,1], D ~ U[0.1, 10]."""
    rng = SplitMix64(seed * 1000 + i)
    k = min(int(rng.next_unit() * len(sizes)), len(sizes) - 1)
    alpha = rng.next_uniform(0.0, 1.0)
    D = rng.next_uniform(0.1, 10.0)
    return sizes[k], alpha, D


def coupled_problem(n: int, alpha: float, D: float, seed_i: int, kmax: int = 4, amp: float = 0.1,
                    b: float = 1.0):
    """Manufactured pair for -Lap u + b u^3 + alpha v = f1, -D Lap v + b v^3 - alpha u = f2
    on the n x n interior grid: u*, v* are independent 2-D manufactured solutions
    (coefficient seeds 2*seed_i and 2*seed_i + 1), and f1, f2 are evaluated
    analytically. Returns (u*, v*, f1, f2)."""
    out = []
    laps = []
    for s in (2 * seed_i, 2 * seed_i + 1):
        coef = amp * manufactured_coeffs(s, 2, kmax)
        coef[0, 0] += 1.0
        out.append(sine_series(coef, n))
        laps.append(sine_series(coef * (math.pi ** 2) * mode_wavenumber_sq(kmax, 2), n))
    u, v = out
    f1 = laps[0] + b * u ** 3 + alpha * v
    f2 = D * laps[1] + b * v ** 3 - alpha * u
    return u, v, f1, f2


# ---------------------------------------------------------------------------
# Gaussian random field sources (learned warm-start workload)
# ---------------------------------------------------------------------------
GRF_KMAX = 32


def normals_vec(seed: int, count: int) -> np.ndarray:
    """count standard normals from SplitMix64(seed), vectorised: normal i uses
    the stream outputs 2i and 2i+1 as (u1, u2) of the Box-Muller cosine branch."""
    u = random_field((2 * count,), seed, 0.0, 1.0)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def grf_coeffs(seed: int, kmax: int = GRF_KMAX) -> np.ndarray:
    """Sine-series coefficients xi_k / (1 + |k|^2), k in {1..kmax}^3, xi ~ N(0,1).

    Power spectrum (1 + |k|^2)^-2 (amplitude = its square root); modes above
    kmax per axis are dropped (they carry a small fraction of the variance)."""
    xi = normals_vec(seed, kmax ** 3).reshape(kmax, kmax, kmax)
    return xi / (1.0 + mode_wavenumber_sq(kmax, 3))


def grf_source(n: int, seed: int, kmax: int = GRF_KMAX, scale: float = 1.0) -> np.ndarray:
    """Dirichlet-consistent GRF on the n^3 interior grid, rescaled to RMS `scale`
    (unit empirical variance for scale 1; the field has zero mean in law)."""
    f = sine_series(grf_coeffs(seed, kmax), n)
    return f * (scale / math.sqrt(float(np.mean(f * f))))


def grf_source_torch(n: int, seed: int, device="cuda", kmax: int = GRF_KMAX, scale: float = 1.0):
    """grf_source with the separable synthesis done by torch on `device`
    (FP64; the same coefficients, the same sums, for fast data generation)."""
    import torch
    c = torch.from_numpy(grf_coeffs(seed, kmax)).to(device)
    B = torch.from_numpy(sine_basis(n, kmax)).to(device)            # (kmax, n)
    t = torch.einsum("abk,kx->abx", c, B)                           # [kz, ky, x]
    t = torch.einsum("ky,akx->ayx", B, t)                           # [kz, y, x]
    f = torch.einsum("kz,kyx->zyx", B, t)                           # [z, y, x]
    return f * (scale / torch.sqrt(torch.mean(f * f)))


# ---------------------------------------------------------------------------
# Neumann workload: the three-dimensional Example 1 of Sec. 6.3
# ---------------------------------------------------------------------------
EX1_A = 10.0
EX1_B = 10.0


def neumann_nodes(n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n nodes x_i = lo + i h, i = 0..n-1, both ends included, h = (hi - lo)/(n - 1)
    (the node set of the ghost-point Neumann discretisation, Sec. 3.2)."""
    return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / (n - 1))


def ex1_potential_1d(x: np.ndarray) -> np.ndarray:
    """One axis term of V = v(x) + v(y) + v(z), v(t) = 100 sin^2(pi t / 4) + t^2 (Sec. 6.3, Example 1)."""
    return 100.0 * np.sin(0.25 * math.pi * x) ** 2 + x * x


def ex1_problem(n: int, a: float = EX1_A, b: float = EX1_B):
    """Data of -Lap u + a u + b u^3 + V u = f on (-1,1)^3 with zero normal derivative
    (Sec. 6.3, Example 1), on n nodes per axis.

    u* = cos(pi x) + cos(pi y) + cos(pi z) (zero normal derivative on the faces);
    f is the continuous source -Lap u* + a u* + b u*^3 + V u* at the nodes, with
    -Lap u* = pi^2 u*. Returns (u_star, f, v, h): 3-D arrays [z, y, x], the 1-D
    potential table v (the same on every axis) and the mesh width h = 2/(n-1).
    """
    x = neumann_nodes(n)
    c = np.cos(math.pi * x)
    v = ex1_potential_1d(x)
    u = c[None, None, :] + c[:, None, None] + c[None, :, None]
    V = v[None, None, :] + v[None, :, None] + v[:, None, None]
    f = (math.pi ** 2 + a) * u + b * u ** 3 + V * u
    return u, f, v, 2.0 / (n - 1)


def ex1_perturbation(n: int, seed: int, eps: float, degree: int = 4) -> np.ndarray:
    """eps * p on the n^3 nodes of (-1,1)^3 (Sec. 6.3): p = q / max|q| with
    q = sum_{i,j,k <= degree} c[k, j, i] x^i y^j z^k, c ~ U(-1, 1) drawn from
    SplitMix64(seed) in C order (x power fastest); the maximum is taken over
    the nodes, which include the corners of the cube."""
    m = degree + 1
    c = random_field((m, m, m), seed, -1.0, 1.0)
    x = neumann_nodes(n)
    Vp = np.vander(x, m, increasing=True)                     # Vp[node, power]
    q = np.einsum("kji,zk,yj,xi->zyx", c, Vp, Vp, Vp, optimize=True)
    return eps * q / float(np.max(np.abs(q)))


def ex2d1_problem(n: int):
    """Data of -Lap u + u^3 + u = f on (-1,1)^2 with zero normal derivative (Sec. 6.2,
    Example 1): u* = cos(pi x) cos(2 pi y), -Lap u* = 5 pi^2 u*, on n nodes per axis.
    Returns (u_star [y, x], f, h) with h = 2/(n-1)."""
    x = neumann_nodes(n)
    u = np.cos(2.0 * math.pi * x)[:, None] * np.cos(math.pi * x)[None, :]
    f = (5.0 * math.pi ** 2 + 1.0) * u + u ** 3
    return u, f, 2.0 / (n - 1)


# ---------------------------------------------------------------------------
# Nonlinear eigenproblem: the three-dimensional Example 2 of Sec. 6.3
# ---------------------------------------------------------------------------
EX2_ALPHA = 1600.0
EX2_LENGTH = 16.0


def ex2_problem(n: int):
    """Data of -Lap u + 1600 u^3 + V u = lambda u on (-8,8)^3, u = 0 on the boundary
    (Sec. 6.3, Example 2), V as in Example 1, on n interior nodes per axis.
    Returns (v, h, x): the 1-D potential table, h = 16/(n+1) and the nodes."""
    h = EX2_LENGTH / (n + 1)
    x = -0.5 * EX2_LENGTH + h * np.arange(1, n + 1, dtype=np.float64)
    return ex1_potential_1d(x), h, x


def ex2_start(n: int, seed: int = 0, eps: float = 0.1, degree: int = 4) -> np.ndarray:
    """Start of the eigen iteration: g(x) g(y) g(z) (1 + eps p), g(t) = cos(pi t / 16) (the box's
    ground state, zero on the boundary) and p a random polynomial of degree `degree` per axis
    in (x/8, y/8, z/8) with U(-1,1) coefficients from SplitMix64(seed), normalised by its
    maximum over the nodes (the paper's perturbation, Sec. 6.3). Not normalised."""
    _, _, x = ex2_problem(n)
    m = degree + 1
    c = random_field((m, m, m), seed, -1.0, 1.0)
    Vp = np.vander(x / (0.5 * EX2_LENGTH), m, increasing=True)
    q = np.einsum("kji,zk,yj,xi->zyx", c, Vp, Vp, Vp, optimize=True)
    g = np.cos(math.pi * x / EX2_LENGTH)
    G = g[None, None, :] * g[None, :, None] * g[:, None, None]
    return G * (1.0 + eps * q / float(np.max(np.abs(q))))
