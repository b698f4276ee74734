// Spectral element discretisation (Sec. 3.1): Q^k elements with Lagrange bases at the
// k+1 Gauss-Lobatto points and (k+1)-point Gauss-Lobatto quadrature, so the mass
// matrix is diagonal and the system takes the form of eq. final-system-3d with the
// 1-D matrix H = M^{-1} S.
//
// Host side (qn_setup_1d_sem): the Gauss-Lobatto rule, element stiffness and mass,
// assembly over E equal elements, the boundary rows, and the diagonalisation of the
// symmetric M^{-1/2} S M^{-1/2} (Householder reduction to tridiagonal form, then
// implicit QL iterations with Wilkinson-type shifts; Bowdler, Martin, Reinsch and
// Wilkinson, Numer. Math. 11 (1968)).
//
// Device side (k_residual_sem): the residual A_h U + lam U + b U^3 + V U - f with
// A_h = sum over axes of H applied along that axis. H is banded (a node couples to
// the nodes of its one or two elements): row i holds hlen[i] <= 2k+1 values from
// column hc0[i]. One thread per node, FP64 (the stencil coefficients are not
// integers, so the exact fixed-point form of the difference stencil does not apply).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "qn_internal.h"
#include "qn_numeric.cuh"

namespace qn {

namespace {

// P_k(x) and P_{k-1}(x) by the three-term recurrence.
void legendre_pair(int k, double x, double &pk, double &pkm1) {
    double p0 = 1.0, p1 = x;
    if (k == 0) {
        pk = 1.0;
        pkm1 = 0.0;
        return;
    }
    for (int j = 1; j < k; ++j) {
        const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    pk = p1;
    pkm1 = p0;
}

// Gauss-Lobatto nodes (ascending) and weights of degree k on [-1, 1]: the ends and
// the roots of P_k', found by Newton's method from Chebyshev-Lobatto guesses;
// w_i = 2 / (k (k+1) P_k(x_i)^2).
void gauss_lobatto(int k, std::vector<double> &x, std::vector<double> &w) {
    x.assign(k + 1, 0.0);
    w.assign(k + 1, 0.0);
    const double pi = 3.14159265358979323846;
    x[0] = -1.0;
    x[k] = 1.0;
    for (int i = 1; i < k; ++i) {
        double t = -cos(pi * i / k);
        for (int it = 0; it < 100; ++it) {
            double pk, pkm1;
            legendre_pair(k, t, pk, pkm1);
            // P_k' = k (P_{k-1} - t P_k) / (1 - t^2), P_k'' = (2 t P_k' - k (k+1) P_k) / (1 - t^2)
            const double d1 = k * (pkm1 - t * pk) / (1.0 - t * t);
            const double d2 = (2.0 * t * d1 - k * (k + 1.0) * pk) / (1.0 - t * t);
            const double dt = d1 / d2;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
    }
    std::sort(x.begin(), x.end());
    for (int i = 0; i <= k; ++i) {
        double pk, pkm1;
        legendre_pair(k, x[i], pk, pkm1);
        w[i] = 2.0 / (k * (k + 1.0) * pk * pk);
    }
}

// ---- device: the banded SEM residual ------------------------------------------------------
struct Red4s {
    double r2, f2, mn, mx;
};

__device__ __forceinline__ Red4s warp_red(Red4s v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.r2 += __shfl_xor_sync(0xffffffffu, v.r2, o);
        v.f2 += __shfl_xor_sync(0xffffffffu, v.f2, o);
        v.mn = fmin(v.mn, __shfl_xor_sync(0xffffffffu, v.mn, o));
        v.mx = fmax(v.mx, __shfl_xor_sync(0xffffffffu, v.mx, o));
    }
    return v;
}

__device__ Red4s block_red(Red4s v) {
    __shared__ Red4s sh[32];
    v = warp_red(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : Red4s{0.0, 0.0, INFINITY, -INFINITY};
        v = warp_red(v);
    }
    return v;
}

// One thread per node of a (y, z) row. SPLIT: BF16 hi/lo planes on the padded P grid
// (zeros in the padding); else the FP64 residual (R64 may be null). POT: the partial
// record's slots 2 and 3 hold min / max of 3 b u^2 + V (else of u^2), and max|U| goes
// to *umax_scan.
template <int DIM, bool SPLIT, bool POT>
__global__ void __launch_bounds__(256) k_residual_sem(ResidualArgs a) {
    if (a.done != nullptr && *(volatile const int *)a.done) return;
    const int n = a.n;
    const int P = SPLIT ? a.P : n;
    const long long rows = (DIM == 3) ? (long long)P * P : (long long)P;
    const long long nn = (long long)n * n;
    const double *__restrict__ U = a.U;
    const int *__restrict__ hc0 = a.hc0;
    const int *__restrict__ hlen = a.hlen;
    const double *__restrict__ hval = a.hval;
    const int bw = a.hbw;
    Red4s acc{0.0, 0.0, INFINITY, -INFINITY};
    unsigned long long umax = 0ull;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (DIM == 3) ? (int)(row % P) : (int)row;
        const int z = (DIM == 3) ? (int)(row / P) : 0;
        const bool row_ok = y < n && z < n;
        double vrow = a.lam;
        if (POT && row_ok) {
            vrow += __ldg(a.pot + n + y);
            if (DIM == 3) vrow += __ldg(a.pot + 2 * n + z);
        }
        const long long cbase = ((long long)z * n + y) * n;
        for (int x = threadIdx.x; x < P; x += blockDim.x) {
            double r = 0.0;
            if (row_ok && x < n) {
                const long long c = cbase + x;
                const double u = __ldg(U + c);
                double lap = 0.0;
                {   // along x: row x of H over the same (y, z) row
                    const int j0 = __ldg(hc0 + x), len = __ldg(hlen + x);
                    const double *hv = hval + (long long)x * bw;
                    for (int j = 0; j < len; ++j) lap = fma(__ldg(hv + j), __ldg(U + cbase + j0 + j), lap);
                }
                {   // along y
                    const int j0 = __ldg(hc0 + y), len = __ldg(hlen + y);
                    const double *hv = hval + (long long)y * bw;
                    const long long b0 = (long long)z * nn + x;
                    for (int j = 0; j < len; ++j) lap = fma(__ldg(hv + j), __ldg(U + b0 + (long long)(j0 + j) * n), lap);
                }
                if (DIM == 3) {   // along z
                    const int j0 = __ldg(hc0 + z), len = __ldg(hlen + z);
                    const double *hv = hval + (long long)z * bw;
                    const long long b0 = (long long)y * n + x;
                    for (int j = 0; j < len; ++j) lap = fma(__ldg(hv + j), __ldg(U + b0 + (long long)(j0 + j) * nn), lap);
                }
                const double fv = __ldg(a.f + c);
                const double u2 = u * u;
                double cv = vrow;
                if (POT) cv += __ldg(a.pot + x);
                r = lap + fma(a.b * u2, u, fma(cv, u, -fv));
                acc.r2 = fma(r, r, acc.r2);
                if (a.want_f2) acc.f2 = fma(fv, fv, acc.f2);
                if (POT) {
                    const double d = fma(3.0 * a.b, u2, cv - a.lam);
                    acc.mn = fmin(acc.mn, d);
                    acc.mx = fmax(acc.mx, d);
                    const unsigned long long ab = abs_bits(u);
                    umax = ab > umax ? ab : umax;
                } else {
                    acc.mn = fmin(acc.mn, u2);
                    acc.mx = fmax(acc.mx, u2);
                }
                if (!SPLIT && a.R64 != nullptr) a.R64[c] = r;
            }
            if (SPLIT) {
                const float rf = d2f_rn(r);
                const __nv_bfloat16 hi = __float2bfloat16_rn(rf);
                const long long o = row * P + x;
                a.Rhi[o] = hi;
                a.Rlo[o] = __float2bfloat16_rn(rf - __bfloat162float(hi));
            }
        }
    }
    if (POT) {
        // block max of the |U| bit patterns (for the fixed-point exponent bookkeeping)
        __shared__ unsigned long long shm[32];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, umax, o);
            umax = t > umax ? t : umax;
        }
        if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = umax;
        __syncthreads();
        if (threadIdx.x == 0 && a.umax_scan != nullptr) {
            unsigned long long m = 0ull;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = shm[i] > m ? shm[i] : m;
            atomicMax(a.umax_scan, m);
        }
    }
    acc = block_red(acc);
    if (threadIdx.x == 0) {
        double *p = a.partials + 4ll * blockIdx.x;
        p[0] = acc.r2;
        p[1] = acc.f2;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

template <int DIM, bool SPLIT>
void launch_sem_dim(const ResidualArgs &a, int grid, cudaStream_t s) {
    if (a.pot != nullptr)
        k_residual_sem<DIM, SPLIT, true><<<grid, 256, 0, s>>>(a);
    else
        k_residual_sem<DIM, SPLIT, false><<<grid, 256, 0, s>>>(a);
}

}  // namespace

// Symmetric eigen-decomposition A = Q diag(d) Q^T (A overwritten with Q, row-major n x n),
// eigenvalues ascending. Returns false if the QL iteration does not converge.
bool symmetric_eigen(int n, std::vector<double> &A, std::vector<double> &d) {
    std::vector<double> Q((size_t)n * n, 0.0), e(n, 0.0), v(n), p(n);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    // Householder: for column c, reflect rows c+1.. so that A[c+2.., c] = 0
    for (int c = 0; c + 2 < n; ++c) {
        const int m = n - c - 1;   // length of the reflected part
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += a(c + 1 + i, c) * a(c + 1 + i, c);
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        const double x0 = a(c + 1, c);
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        for (int i = 0; i < m; ++i) v[i] = a(c + 1 + i, c);
        v[0] -= alpha;
        double vn = 0.0;
        for (int i = 0; i < m; ++i) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        const double inv = 1.0 / vn;
        // A <- P A P with P = I - 2 v v^T / (v^T v) on rows/cols c+1..: p = A v, K = v^T p / vn,
        // q = 2 (p - K v) / vn, A <- A - v q^T - q v^T (symmetric rank-2 update)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += a(i, c + 1 + j) * v[j];
            p[i] = s;
        }
        double K = 0.0;
        for (int j = 0; j < m; ++j) K += v[j] * p[c + 1 + j];
        K *= inv;
        std::vector<double> q(n, 0.0);
        for (int i = 0; i < n; ++i) {
            const double vi = (i > c) ? v[i - c - 1] : 0.0;
            q[i] = 2.0 * inv * (p[i] - K * vi);
        }
        for (int i = 0; i < n; ++i) {
            const double vi = (i > c) ? v[i - c - 1] : 0.0;
            for (int j = 0; j < n; ++j) {
                const double vj = (j > c) ? v[j - c - 1] : 0.0;
                a(i, j) -= vi * q[j] + q[i] * vj;
            }
        }
        // Q <- Q P
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += Q[(size_t)i * n + c + 1 + j] * v[j];
            s *= 2.0 * inv;
            for (int j = 0; j < m; ++j) Q[(size_t)i * n + c + 1 + j] -= s * v[j];
        }
    }
    d.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
    e[n - 1] = 0.0;
    // implicit QL on the tridiagonal (d, e), rotations accumulated into Q's columns
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) + dd == dd) break;   // negligible next to its diagonal neighbours
            }
            if (m == l) break;
            if (++iter > 60) return false;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double s = 1.0, c = 1.0, pp = 0.0;
            bool split_early = false;
            for (int i = m - 1; i >= l; --i) {
                double f = s * e[i];
                const double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {   // the rotation decouples: deflate and iterate again
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    split_early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                for (int row = 0; row < n; ++row) {
                    double *qr = &Q[(size_t)row * n];
                    f = qr[i + 1];
                    qr[i + 1] = s * qr[i] + c * f;
                    qr[i] = c * qr[i] - s * f;
                }
            }
            if (split_early) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // ascending order
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] < d[y]; });
    std::vector<double> d2(n);
    for (int j = 0; j < n; ++j) {
        d2[j] = d[ord[j]];
        for (int i = 0; i < n; ++i) A[(size_t)i * n + j] = Q[(size_t)i * n + ord[j]];
    }
    d = d2;
    return true;
}

int launch_residual_sem(const ResidualArgs &a, int grid, cudaStream_t s) {
    const bool split = a.Rhi != nullptr;
    if (a.dim == 3) {
        if (split)
            launch_sem_dim<3, true>(a, grid, s);
        else
            launch_sem_dim<3, false>(a, grid, s);
    } else {
        if (split)
            launch_sem_dim<2, true>(a, grid, s);
        else
            launch_sem_dim<2, false>(a, grid, s);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int sem_setup(int n, int k, double length, int bc, std::vector<double> &H, std::vector<double> &S,
              std::vector<double> &Si, std::vector<double> &lam, std::vector<double> &nodes) {
    if (k < 1 || k > 16 || length <= 0.0 || !isfinite(length) || (bc != QN_BC_DIRICHLET && bc != QN_BC_NEUMANN)) {
        set_error("qn_setup_1d_sem: need 1 <= k <= 16, length > 0 and a known boundary condition");
        return QN_EINVAL;
    }
    const int tot = (bc == QN_BC_DIRICHLET) ? n + 1 : n - 1;
    if (n < 1 || n > 4096 || tot < k || tot % k != 0) {
        set_error("qn_setup_1d_sem: n = %d does not fit Q^%d elements (n %s 1 must be a multiple of k)", n, k,
                  bc == QN_BC_DIRICHLET ? "+" : "-");
        return QN_EINVAL;
    }
    const int E = tot / k, G = E * k + 1;
    const double he = length / E;
    std::vector<double> xi, w;
    gauss_lobatto(k, xi, w);
    // derivative matrix of the Lagrange basis at the Gauss-Lobatto points (Legendre form):
    // D_ij = P_k(x_i) / (P_k(x_j) (x_i - x_j)), D_00 = -k(k+1)/4, D_kk = k(k+1)/4, else D_ii = 0
    std::vector<double> Pk(k + 1);
    for (int i = 0; i <= k; ++i) {
        double pkm1;
        legendre_pair(k, xi[i], Pk[i], pkm1);
    }
    std::vector<double> D((size_t)(k + 1) * (k + 1), 0.0);
    for (int i = 0; i <= k; ++i)
        for (int j = 0; j <= k; ++j)
            if (i != j) D[(size_t)i * (k + 1) + j] = Pk[i] / (Pk[j] * (xi[i] - xi[j]));
    D[0] = -0.25 * k * (k + 1.0);
    D[(size_t)k * (k + 1) + k] = 0.25 * k * (k + 1.0);
    // element stiffness K_ij = (2/he) sum_q w_q D_qi D_qj, lumped mass (he/2) w_i; assembly
    std::vector<double> Sg((size_t)G * G, 0.0), mg(G, 0.0), xg(G, 0.0);
    for (int e = 0; e < E; ++e) {
        for (int i = 0; i <= k; ++i) {
            const int gi = e * k + i;
            mg[gi] += 0.5 * he * w[i];
            xg[gi] = e * he + 0.5 * (1.0 + xi[i]) * he;
            for (int j = 0; j <= k; ++j) {
                double s = 0.0;
                for (int q = 0; q <= k; ++q) s += w[q] * D[(size_t)q * (k + 1) + i] * D[(size_t)q * (k + 1) + j];
                Sg[(size_t)gi * G + e * k + j] += (2.0 / he) * s;
            }
        }
    }
    const int off = (bc == QN_BC_DIRICHLET) ? 1 : 0;
    std::vector<double> Sk((size_t)n * n), m(n);
    nodes.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        m[i] = mg[i + off];
        nodes[i] = xg[i + off];
        for (int j = 0; j < n; ++j) Sk[(size_t)i * n + j] = Sg[(size_t)(i + off) * G + j + off];
    }
    H.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) H[(size_t)i * n + j] = Sk[(size_t)i * n + j] / m[i];
    // M^{-1/2} S M^{-1/2} = Q diag(lam) Q^T; S_e = M^{-1/2} Q, S_e^{-1} = Q^T M^{1/2}
    std::vector<double> A((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = Sk[(size_t)i * n + j] / sqrt(m[i] * m[j]);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double s = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = s;
        }
    if (!symmetric_eigen(n, A, lam)) {
        set_error("qn_setup_1d_sem: the eigenvalue iteration did not converge");
        return QN_ECUDA;
    }
    S.assign((size_t)n * n, 0.0);
    Si.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            S[(size_t)i * n + j] = A[(size_t)i * n + j] / sqrt(m[i]);
            Si[(size_t)j * n + i] = A[(size_t)i * n + j] * sqrt(m[i]);
        }
    return QN_OK;
}

}  // namespace qn

extern "C" int qn_setup_1d_robin(int n, double h, double kappa, double *S, double *S_inv, double *lam) {
    if (n < 2 || n > 65536 || !(h > 0.0) || !isfinite(h) || !(kappa >= 0.0) || !isfinite(kappa)) {
        qn::set_error("qn_setup_1d_robin: need n >= 2, h > 0 and a finite kappa >= 0");
        return QN_EINVAL;
    }
    // W^{1/2} H W^{-1/2}: tridiagonal, symmetric; off-diagonals -1/h^2 inside, -sqrt(2)/h^2 at
    // the faces (W^{1/2} (-2) W^{-1/2} with w = 1/2 on the face and 1 next to it)
    std::vector<double> A((size_t)n * n, 0.0), lamv;
    const double ih2 = 1.0 / (h * h);
    for (int i = 0; i < n; ++i) A[(size_t)i * n + i] = 2.0 * ih2;
    A[0] += 2.0 * kappa / h;
    A[(size_t)(n - 1) * n + n - 1] += 2.0 * kappa / h;
    for (int i = 0; i + 1 < n; ++i) {
        const bool face = (i == 0 || i + 1 == n - 1);
        const double off = face ? -sqrt(2.0) * ih2 : -ih2;
        A[(size_t)i * n + i + 1] = A[(size_t)(i + 1) * n + i] = off;
    }
    if (n == 2) A[1] = A[2] = -2.0 * ih2;   // both nodes are faces: W = I/2, the -2 entries stay
    if (!qn::symmetric_eigen(n, A, lamv)) {
        qn::set_error("qn_setup_1d_robin: the eigenvalue iteration did not converge");
        return QN_ECUDA;
    }
    for (int j = 0; j < n; ++j) {
        const double sw = (j == 0 || j == n - 1) ? sqrt(0.5) : 1.0;   // sqrt(w_j)
        for (int k = 0; k < n; ++k) {
            const double q = A[(size_t)j * n + k];
            if (S) S[(size_t)j * n + k] = q / sw;
            if (S_inv) S_inv[(size_t)k * n + j] = q * sw;
        }
    }
    if (lam) memcpy(lam, lamv.data(), sizeof(double) * n);
    return QN_OK;
}

extern "C" int qn_setup_1d_sem(int n, int k, double length, int bc, double *H, double *S, double *S_inv,
                               double *lam, double *nodes) {
    std::vector<double> h, s, si, l, x;
    const int rc = qn::sem_setup(n, k, length, bc, h, s, si, l, x);
    if (rc != QN_OK) return rc;
    const size_t nn = (size_t)n * n;
    if (H) memcpy(H, h.data(), nn * sizeof(double));
    if (S) memcpy(S, s.data(), nn * sizeof(double));
    if (S_inv) memcpy(S_inv, si.data(), nn * sizeof(double));
    if (lam) memcpy(lam, l.data(), (size_t)n * sizeof(double));
    if (nodes) memcpy(nodes, x.data(), (size_t)n * sizeof(double));
    return QN_OK;
}
