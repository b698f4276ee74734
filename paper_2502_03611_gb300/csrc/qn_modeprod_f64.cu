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
// K staged through shared memory in chunks of 16.
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

template <int DIM>
void launch_dim(const double *A, const double *B, double *out, const GemmShape &g, Epi epi,
                const EpiArgs &e, cudaStream_t s) {
    dim3 grid((unsigned)((g.Mtot + BM - 1) / BM), (unsigned)((g.n + BN - 1) / BN));
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
