// FP64 mode product on the FP64 pipe (plain-precision path).
//
// One mode product Y = X x_a M of Sec. 4.1 eq. fin_inverse (the paper's
// vec(A X B^T) = (B kron A) vec(X) identity) is written as one GEMM over the
// contiguous axis of X, with the result stored TRANSPOSED:
//
//     out[k][m] = sum_j A[m][j] * M[k][j],   A = X viewed as [Mtot][n].
//
// Storing out[k][m] rotates the tensor's axes by one: a [z][y][x] input
// contracted over x comes out as [k_x][z][y], so the next product again
// contracts the contiguous axis. After dim products the axes are back in
// their original order. Every product is therefore the same K-contiguous
// GEMM, and consecutive threads write consecutive m (coalesced).
//
// Epilogues: EPI_STORE (next product's input), EPI_DIVIDE (pointwise
// division by lambda_k + row eigen-sum + shift, eq. fin_inverse), EPI_UPDATE
// (U -= step * delta; the last backward product's (k, m) is U's own dense
// index k*Mtot + m), EPI_DENSE (plain store to the dense output).
//
// Tiling: 64 (m) x 64 (k) outputs per 256-thread block, 4x4 per thread,
// K staged through shared memory in chunks of 16; small problems use 8 x 8
// output tiles (k_modeprod_f64_small) so that they spread over the SMs.
#include "qn_internal.h"

namespace qn {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <int DIM, int EPI>
__global__ void __launch_bounds__(256) k_modeprod_f64(const double *__restrict__ A,
                                                      const double *__restrict__ B,
                                                      double *__restrict__ out, int Mtot, int n,
                                                      EpiArgs e) {
    if (e.done != nullptr && *(volatile const int *)e.done) return;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long m0 = (long long)blockIdx.x * BM;
    const int k0 = blockIdx.y * BN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    // loader mapping: 256 threads cover a 64 x 16 tile, 4 elements each
    const int lc = threadIdx.x & 15;        // column within the K chunk
    const int lr = threadIdx.x >> 4;        // row 0..15, +16*q
    for (int kk = 0; kk < n; kk += BK) {
        const int col = kk + lc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lr + 16 * q;
            const long long gm = m0 + r;
            As[lc][r] = (gm < Mtot && col < n) ? __ldg(A + gm * n + col) : 0.0;
            const int gk = k0 + r;
            Bs[lc][r] = (gk < n && col < n) ? __ldg(B + (long long)gk * n + col) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < BK; ++c) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[c][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[c][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    double shift = 0.0;
    if (EPI == EPI_DIVIDE) shift = *e.shift;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = m0 + tx + 16 * i;
        if (m >= Mtot) continue;
        double rowlam = 0.0;
        if (EPI == EPI_DIVIDE) {
            if (DIM == 3)
                rowlam = e.lam64[m / n] + e.lam64[m % n];
            else
                rowlam = e.lam64[m];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + ty + 16 * j;
            if (k >= n) continue;
            const long long o = (long long)k * Mtot + m;
            if (EPI == EPI_STORE || EPI == EPI_DENSE) {
                out[o] = acc[i][j];
            } else if (EPI == EPI_DIVIDE) {
                out[o] = acc[i][j] / (e.lam64[k] + rowlam + shift);
            } else {   // EPI_UPDATE
                out[o] = out[o] - e.step * acc[i][j];
            }
        }
    }
}

// Reflection-split products (FD Dirichlet / Neumann eigenpairs, which satisfy
// S[n-1-j][k] = (-1)^k S[j][k] and S^{-1}[k][n-1-j] = (-1)^k S^{-1}[k][j]): half
// the FP64 work, the same natural layout in and out (the butterflies ride in the
// loader and the epilogue).
//   forward: out[k][m] = sum_{j < ceil(n/2)} S^{-1}[k][j] a_j for even k, with
//            a_j = x_j + x_{n-1-j} (the middle x of an odd n alone), and
//            sum_{j < n/2} S^{-1}[k][j] b_j for odd k, b_j = x_j - x_{n-1-j}.
//            A thread's four k = k0 + ty + 16q share the parity of ty, so it reads
//            only the a or only the b tile.
//   backward: out[s][m] = p_s + q_s and out[n-1-s][m] = p_s - q_s for s < ceil(n/2),
//            p_s = sum over even modes q of S[s][q] Y[m][q], q_s over odd modes
//            (the middle row of an odd n: p + q, its own mirror).
template <int DIM, int EPI>
__global__ void __launch_bounds__(256) k_modeprod_f64_fsplit(const double *__restrict__ A,
                                                             const double *__restrict__ B,
                                                             double *__restrict__ out, int Mtot, int n,
                                                             EpiArgs e) {
    if (e.done != nullptr && *(volatile const int *)e.done) return;
    __shared__ double Aa[BK][BM + 1];
    __shared__ double Ab[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long m0 = (long long)blockIdx.x * BM;
    const int k0 = blockIdx.y * BN;
    const int nsym = (n + 1) / 2, nanti = n / 2;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const int lc = threadIdx.x & 15;
    const int lr = threadIdx.x >> 4;
    const double(*As)[BM + 1] = (ty & 1) ? Ab : Aa;   // k0 is a multiple of 64: k's parity is ty's
    for (int kk = 0; kk < nsym; kk += BK) {
        const int col = kk + lc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lr + 16 * q;
            const long long gm = m0 + r;
            double x = 0.0, y = 0.0;
            if (gm < Mtot && col < nsym) {
                x = __ldg(A + gm * n + col);
                if (col < nanti) y = __ldg(A + gm * n + (n - 1 - col));
            }
            Aa[lc][r] = x + y;
            Ab[lc][r] = (col < nanti) ? x - y : 0.0;
            const int gk = k0 + r;
            Bs[lc][r] = (gk < n && col < nsym) ? __ldg(B + (long long)gk * n + col) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < BK; ++c) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[c][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[c][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double shift = 0.0;
    if (EPI == EPI_DIVIDE) shift = *e.shift;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = m0 + tx + 16 * i;
        if (m >= Mtot) continue;
        double rowlam = 0.0;
        if (EPI == EPI_DIVIDE) rowlam = (DIM == 3) ? e.lam64[m / n] + e.lam64[m % n] : e.lam64[m];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + ty + 16 * j;
            if (k >= n) continue;
            const long long o = (long long)k * Mtot + m;
            if (EPI == EPI_DIVIDE)
                out[o] = acc[i][j] / (e.lam64[k] + rowlam + shift);
            else
                out[o] = acc[i][j];   // forward products: EPI_STORE
        }
    }
}

template <int DIM, int EPI>
__global__ void __launch_bounds__(256) k_modeprod_f64_bsplit(const double *__restrict__ A,
                                                             const double *__restrict__ B,
                                                             double *__restrict__ out, int Mtot, int n,
                                                             EpiArgs e) {
    if (e.done != nullptr && *(volatile const int *)e.done) return;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long m0 = (long long)blockIdx.x * BM;
    const int s0 = blockIdx.y * BN;
    const int nsym = (n + 1) / 2, nanti = n / 2;
    double pa[4][4], qa[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) pa[i][j] = qa[i][j] = 0.0;
    const int lc = threadIdx.x & 15;
    const int lr = threadIdx.x >> 4;
    for (int kk = 0; kk < n; kk += BK) {   // BK even: the mode kk + c has the parity of c
        const int col = kk + lc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lr + 16 * q;
            const long long gm = m0 + r;
            As[lc][r] = (gm < Mtot && col < n) ? __ldg(A + gm * n + col) : 0.0;
            const int gs = s0 + r;
            Bs[lc][r] = (gs < nsym && col < n) ? __ldg(B + (long long)gs * n + col) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < BK; c += 2) {
            double a0[4], b0[4], a1[4], b1[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a0[i] = As[c][tx + 16 * i];
                a1[i] = As[c + 1][tx + 16 * i];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                b0[j] = Bs[c][ty + 16 * j];
                b1[j] = Bs[c + 1][ty + 16 * j];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    pa[i][j] = fma(a0[i], b0[j], pa[i][j]);
                    qa[i][j] = fma(a1[i], b1[j], qa[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long m = m0 + tx + 16 * i;
        if (m >= Mtot) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sp = s0 + ty + 16 * j;
            if (sp >= nsym) continue;
            const double vp = pa[i][j] + qa[i][j];
            const double vm = pa[i][j] - qa[i][j];
            const long long o1 = (long long)sp * Mtot + m;
            const long long o2 = (long long)(n - 1 - sp) * Mtot + m;
            if (EPI == EPI_UPDATE) {
                out[o1] = out[o1] - e.step * vp;
                if (sp < nanti) out[o2] = out[o2] - e.step * vm;
            } else {   // EPI_STORE / EPI_DENSE
                out[o1] = vp;
                if (sp < nanti) out[o2] = vm;
            }
        }
    }
}

// Small problems (the 2-D 63^2 solve: one 64 x 64 tile, i.e. one SM bound by its
// FP64 pipe): 8 x 8 outputs per 64-thread block, so the product spreads over many
// SMs. The block stages its 8 rows of A and 8 rows of B (all of K <= kSmallK) in
// shared memory; thread (i, j) forms one dot product. Same epilogues.
constexpr int SB = 8, kSmallK = 256;

template <int DIM, int EPI>
__global__ void __launch_bounds__(64) k_modeprod_f64_small(const double *__restrict__ A,
                                                           const double *__restrict__ B,
                                                           double *__restrict__ out, int Mtot, int n,
                                                           EpiArgs e) {
    if (e.done != nullptr && *(volatile const int *)e.done) return;
    __shared__ double As[SB][kSmallK + 1];
    __shared__ double Bs[SB][kSmallK + 1];
    const long long m0 = (long long)blockIdx.x * SB;
    const int k0 = blockIdx.y * SB;
    for (int t = threadIdx.x; t < SB * n; t += 64) {
        const int r = t / n, c = t - r * n;
        const long long gm = m0 + r;
        const int gk = k0 + r;
        As[r][c] = (gm < Mtot) ? __ldg(A + gm * n + c) : 0.0;
        Bs[r][c] = (gk < n) ? __ldg(B + (long long)gk * n + c) : 0.0;
    }
    __syncthreads();
    const int i = threadIdx.x & 7, j = threadIdx.x >> 3;
    const long long m = m0 + i;
    const int k = k0 + j;
    double acc0 = 0.0, acc1 = 0.0;   // two chains: the FP64 pipe's latency
    int c = 0;
    for (; c + 1 < n; c += 2) {
        acc0 = fma(As[i][c], Bs[j][c], acc0);
        acc1 = fma(As[i][c + 1], Bs[j][c + 1], acc1);
    }
    if (c < n) acc0 = fma(As[i][c], Bs[j][c], acc0);
    const double acc = acc0 + acc1;
    if (m >= Mtot || k >= n) return;
    const long long o = (long long)k * Mtot + m;
    if (EPI == EPI_STORE || EPI == EPI_DENSE) {
        out[o] = acc;
    } else if (EPI == EPI_DIVIDE) {
        const double rowlam = (DIM == 3) ? e.lam64[m / n] + e.lam64[m % n] : e.lam64[m];
        out[o] = acc / (e.lam64[k] + rowlam + *e.shift);
    } else {   // EPI_UPDATE
        out[o] = out[o] - e.step * acc;
    }
}

template <int DIM>
void launch_small(const double *A, const double *B, double *out, const GemmShape &g, Epi epi,
                  const EpiArgs &e, cudaStream_t s) {
    dim3 grid((unsigned)((g.Mtot + SB - 1) / SB), (unsigned)((g.n + SB - 1) / SB));
    switch (epi) {
        case EPI_STORE: k_modeprod_f64_small<DIM, EPI_STORE><<<grid, 64, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_DIVIDE: k_modeprod_f64_small<DIM, EPI_DIVIDE><<<grid, 64, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_UPDATE: k_modeprod_f64_small<DIM, EPI_UPDATE><<<grid, 64, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_DENSE: k_modeprod_f64_small<DIM, EPI_DENSE><<<grid, 64, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
    }
}

template <int DIM>
void launch_dim(const double *A, const double *B, double *out, const GemmShape &g, Epi epi,
                const EpiArgs &e, cudaStream_t s) {
    dim3 grid((unsigned)((g.Mtot + BM - 1) / BM), (unsigned)((g.n + BN - 1) / BN));
    // fewer 64 x 64 tiles than a third of the SMs: the FP64 pipes of the others idle
    if ((long long)grid.x * grid.y < 48 && g.n <= kSmallK) {
        launch_small<DIM>(A, B, out, g, epi, e, s);
        return;
    }
    if (g.split == 1) {   // forward (S^{-1}): EPI_STORE or EPI_DIVIDE
        if (epi == EPI_DIVIDE)
            k_modeprod_f64_fsplit<DIM, EPI_DIVIDE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e);
        else
            k_modeprod_f64_fsplit<DIM, EPI_STORE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e);
        return;
    }
    if (g.split == 2) {   // backward (S): output rows s < ceil(n/2) and their mirrors
        dim3 gb(grid.x, (unsigned)(((g.n + 1) / 2 + BN - 1) / BN));
        if (epi == EPI_UPDATE)
            k_modeprod_f64_bsplit<DIM, EPI_UPDATE><<<gb, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e);
        else
            k_modeprod_f64_bsplit<DIM, EPI_STORE><<<gb, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e);
        return;
    }
    switch (epi) {
        case EPI_STORE: k_modeprod_f64<DIM, EPI_STORE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_DIVIDE: k_modeprod_f64<DIM, EPI_DIVIDE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_UPDATE: k_modeprod_f64<DIM, EPI_UPDATE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
        case EPI_DENSE: k_modeprod_f64<DIM, EPI_DENSE><<<grid, 256, 0, s>>>(A, B, out, g.Mtot, g.n, e); break;
    }
}

}  // namespace

int launch_modeprod_f64(const double *A, const double *B, double *out, const GemmShape &g,
                        Epi epi, const EpiArgs &e, cudaStream_t s) {
    if (g.dim == 3)
        launch_dim<3>(A, B, out, g, epi, e, s);
    else
        launch_dim<2>(A, B, out, g, epi, e, s);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

}  // namespace qn
