// Nonlinear eigenproblem (Sec. 4.4 eqs. Eigenvalue_p, system_qusi, system_normal;
// Sec. 6.3 Example 2):
//   -Lap u + f(u) = lambda u,   f(u) = lam u + b u^3 + V u,   ||u|| = 1,
// lambda unknown. One iteration on the device, with no host synchronisation:
//
//   k_eig_rayleigh   r0 = A_h U + f(U) (FP64, kept for the next pass) and the
//                    sums <r0, U>, <U, U>, min/max of lam + 3 b U^2 + V
//   k_eig_finalize1  lambda_n = <r0, U> / <U, U>, beta_n = mid-range - lambda_n,
//                    shift, and the scale |lambda_n| ||U|| of the stop test
//   k_eig_residual2  F = r0 - lambda_n U -> the inverse's input (FP64, or BF16
//                    hi/lo planes in natural or reflection-split order), ||F||^2
//   k_finalize       (qn_residual.cu, eigen mode) stop test
//   mode products    U~ = U - step (A_h + beta_n I)^{-1} F (update epilogue)
//   k_eig_sumsq      <U~, U~>
//   k_eig_scale      U = U~ / ||U~||
//
// <V, W> is the lumped-mass product h^dim sum w V W, with w the product of the
// 1-D trapezoid weights (1/2 at a Neumann face node, else 1): A_h is
// self-adjoint in it, so F is orthogonal to U. All reductions are per-block
// partials summed in a fixed order (deterministic, graph replay is bitwise
// the same as plain launches).
#include <math.h>

#include "qn_internal.h"
#include "qn_numeric.cuh"

namespace qn {

namespace {

struct Sum4 {
    double a, b, mn, mx;
};

__device__ __forceinline__ Sum4 warp_sum4(Sum4 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.a += __shfl_xor_sync(0xffffffffu, v.a, o);
        v.b += __shfl_xor_sync(0xffffffffu, v.b, o);
        v.mn = fmin(v.mn, __shfl_xor_sync(0xffffffffu, v.mn, o));
        v.mx = fmax(v.mx, __shfl_xor_sync(0xffffffffu, v.mx, o));
    }
    return v;
}

// Block reduction (blockDim.x a multiple of 32); the result is valid in thread 0.
__device__ Sum4 block_sum4(Sum4 v) {
    __shared__ Sum4 sh[32];
    v = warp_sum4(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : Sum4{0.0, 0.0, INFINITY, -INFINITY};
        v = warp_sum4(v);
    }
    return v;
}

__device__ __forceinline__ bool state_done(const DevState *st) { return *(volatile const int *)&st->done != 0; }

// 1-D trapezoid weight of node i (the lumped mass without h).
__device__ __forceinline__ double tw(int i, int n, bool neu) { return (neu && (i == 0 || i == n - 1)) ? 0.5 : 1.0; }

// r0 = A_h U + (lam + V) U + b U^3 at every node, with the sums of w u r0 and w u^2
// and the extremes of lam + 3 b u^2 + V per block.
template <int DIM>
__global__ void __launch_bounds__(256) k_eig_rayleigh(const double *__restrict__ U, double *__restrict__ r0, int n,
                                                      int bc, double inv_h2, double lam, double b,
                                                      const double *__restrict__ pot, double *__restrict__ partials,
                                                      const DevState *st) {
    if (state_done(st)) return;
    const bool neu = (bc == QN_BC_NEUMANN);
    const long long rows = (DIM == 3) ? (long long)n * n : (long long)n;
    const long long nn = (long long)n * n;
    Sum4 acc{0.0, 0.0, INFINITY, -INFINITY};
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (DIM == 3) ? (int)(row % n) : (int)row;
        const int z = (DIM == 3) ? (int)(row / n) : 0;
        const double wyz = tw(y, n, neu) * ((DIM == 3) ? tw(z, n, neu) : 1.0);
        double vrow = lam;
        if (pot != nullptr) {
            vrow += __ldg(pot + n + y);
            if (DIM == 3) vrow += __ldg(pot + 2 * n + z);
        }
        const long long cbase = ((long long)z * n + y) * n;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const long long c = cbase + x;
            const double u = __ldg(U + c);
            double nbv[2 * DIM];
            nbv[0] = (x > 0) ? __ldg(U + c - 1) : (neu ? __ldg(U + c + 1) : 0.0);
            nbv[1] = (x < n - 1) ? __ldg(U + c + 1) : (neu ? __ldg(U + c - 1) : 0.0);
            nbv[2] = (y > 0) ? __ldg(U + c - n) : (neu ? __ldg(U + c + n) : 0.0);
            nbv[3] = (y < n - 1) ? __ldg(U + c + n) : (neu ? __ldg(U + c - n) : 0.0);
            if (DIM == 3) {
                nbv[4] = (z > 0) ? __ldg(U + c - nn) : (neu ? __ldg(U + c + nn) : 0.0);
                nbv[5] = (z < n - 1) ? __ldg(U + c + nn) : (neu ? __ldg(U + c - nn) : 0.0);
            }
            const double lap = stencil_fixed<DIM>(u, nbv);          // exact 2 DIM u - sum(nb)
            const double cv = vrow + ((pot != nullptr) ? __ldg(pot + x) : 0.0);
            const double u2 = u * u;
            const double rv = fma(lap, inv_h2, fma(b * u2, u, cv * u));
            r0[c] = rv;
            const double wu = tw(x, n, neu) * wyz * u;
            acc.a = fma(wu, rv, acc.a);
            acc.b = fma(wu, u, acc.b);
            const double d = fma(3.0 * b, u2, cv);                   // lam + 3 b u^2 + V
            acc.mn = fmin(acc.mn, d);
            acc.mx = fmax(acc.mx, d);
        }
    }
    acc = block_sum4(acc);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = acc.b;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

// lambda_n, beta_n, the shift of the divide and the scale of the stop test.
__global__ void __launch_bounds__(256) k_eig_finalize1(const double *partials, int nparts, double hd, DevState *st) {
    if (state_done(st)) return;
    Sum4 acc{0.0, 0.0, INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        acc.a += partials[4 * i + 0];
        acc.b += partials[4 * i + 1];
        acc.mn = fmin(acc.mn, partials[4 * i + 2]);
        acc.mx = fmax(acc.mx, partials[4 * i + 3]);
    }
    acc = block_sum4(acc);
    if (threadIdx.x != 0) return;
    const double lam_n = acc.a / acc.b;
    st->eig_lambda = lam_n;
    st->eig_fu_min = acc.mn;
    st->eig_fu_max = acc.mx;
    // (N_h)_U = diag(lam + 3 b U^2 + V) - lambda_n; A_h here is the difference
    // operator alone (lam belongs to f), so the divide's shift is beta_n itself
    const double beta = (st->beta_mode == QN_BETA_FIXED) ? st->beta_value : 0.5 * (acc.mn + acc.mx) - lam_n;
    st->beta = beta;
    st->shift = beta;
    st->f_norm = fabs(lam_n) * sqrt(hd * acc.b);                   // |lambda_n| ||U||
}

// F = r0 - lambda_n U into the inverse's input, with sum w F^2 (times h^dim).
// OUT 0: FP64 n^DIM array. OUT 1: BF16 hi/lo planes on the padded P^DIM grid in
// natural order. OUT 2 (3-D, P a multiple of 128): the reflection-split order
// of k_residual_mirror (x: sums at i, differences at P/2 + i; y, z folded).
template <int DIM, int OUT>
__global__ void __launch_bounds__(256) k_eig_residual2(const double *__restrict__ U, const double *__restrict__ r0,
                                                       int n, int P, int bc, double hd, double *__restrict__ R64,
                                                       __nv_bfloat16 *__restrict__ Rhi, __nv_bfloat16 *__restrict__ Rlo,
                                                       double *__restrict__ partials, const DevState *st) {
    if (state_done(st)) return;
    const bool neu = (bc == QN_BC_NEUMANN);
    const double lam_n = st->eig_lambda;
    const long long nn = (long long)n * n;
    double sff = 0.0;
    if (OUT == 0) {
        const long long rows = (DIM == 3) ? nn : (long long)n;
        for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
            const int y = (DIM == 3) ? (int)(row % n) : (int)row;
            const int z = (DIM == 3) ? (int)(row / n) : 0;
            const double wyz = tw(y, n, neu) * ((DIM == 3) ? tw(z, n, neu) : 1.0);
            const long long cbase = row * n;
            for (int x = threadIdx.x; x < n; x += blockDim.x) {
                const double F = fma(-lam_n, __ldg(U + cbase + x), __ldg(r0 + cbase + x));
                R64[cbase + x] = F;
                sff = fma(tw(x, n, neu) * wyz * F, F, sff);
            }
        }
    } else if (OUT == 1) {
        const long long rows = (DIM == 3) ? (long long)P * P : (long long)P;
        for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
            const int y = (DIM == 3) ? (int)(row % P) : (int)row;
            const int z = (DIM == 3) ? (int)(row / P) : 0;
            const bool row_ok = y < n && z < n;
            const double wyz = row_ok ? tw(y, n, neu) * ((DIM == 3) ? tw(z, n, neu) : 1.0) : 0.0;
            const long long cbase = ((long long)z * n + y) * n;
            for (int x = threadIdx.x; x < P; x += blockDim.x) {
                float f = 0.0f;
                if (row_ok && x < n) {
                    const double F = fma(-lam_n, __ldg(U + cbase + x), __ldg(r0 + cbase + x));
                    sff = fma(tw(x, n, neu) * wyz * F, F, sff);
                    f = d2f_rn(F);
                }
                const __nv_bfloat16 hi = __float2bfloat16_rn(f);
                const long long o = row * P + x;
                Rhi[o] = hi;
                Rlo[o] = __float2bfloat16_rn(f - __bfloat162float(hi));
            }
        }
    } else {
        const int H = P / 2, nsym = (n + 1) / 2, nanti = n / 2;
        const long long rows = (long long)P * P;
        for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
            // folded row index -> spatial: even r -> r/2, odd r -> n-1-(r-1)/2, r >= n padding
            const int ry = (int)(row % P), rz = (int)(row / P);
            const bool row_ok = ry < n && rz < n;
            const int y = (ry & 1) ? n - 1 - (ry >> 1) : (ry >> 1);
            const int z = (rz & 1) ? n - 1 - (rz >> 1) : (rz >> 1);
            const double wyz = row_ok ? tw(y, n, neu) * tw(z, n, neu) : 0.0;
            const long long cbase = row_ok ? ((long long)z * n + y) * n : 0;
            for (int i = threadIdx.x; i < H; i += blockDim.x) {
                float fa = 0.0f, fb = 0.0f;
                if (row_ok && i < nsym) {
                    const double F1 = fma(-lam_n, __ldg(U + cbase + i), __ldg(r0 + cbase + i));
                    sff = fma(tw(i, n, neu) * wyz * F1, F1, sff);
                    fa = d2f_rn(F1);
                    if (i < nanti) {
                        const int j = n - 1 - i;
                        const double F2 = fma(-lam_n, __ldg(U + cbase + j), __ldg(r0 + cbase + j));
                        sff = fma(tw(j, n, neu) * wyz * F2, F2, sff);
                        const float f2 = d2f_rn(F2);
                        fb = __fsub_rn(fa, f2);
                        fa = __fadd_rn(fa, f2);
                    }
                }
                const long long o = row * P;
                const __nv_bfloat16 ha = __float2bfloat16_rn(fa), hb = __float2bfloat16_rn(fb);
                Rhi[o + i] = ha;
                Rlo[o + i] = __float2bfloat16_rn(fa - __bfloat162float(ha));
                Rhi[o + H + i] = hb;
                Rlo[o + H + i] = __float2bfloat16_rn(fb - __bfloat162float(hb));
            }
        }
    }
    Sum4 acc{hd * sff, 0.0, INFINITY, -INFINITY};
    acc = block_sum4(acc);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = 0.0;
        p[2] = 0.0;
        p[3] = 0.0;
    }
}

// sum w U^2 per block (one double per block).
template <int DIM>
__global__ void __launch_bounds__(256) k_eig_sumsq(const double *__restrict__ U, int n, int bc,
                                                   double *__restrict__ partials, const DevState *st) {
    if (state_done(st)) return;
    const bool neu = (bc == QN_BC_NEUMANN);
    const long long rows = (DIM == 3) ? (long long)n * n : (long long)n;
    double s = 0.0;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (DIM == 3) ? (int)(row % n) : (int)row;
        const int z = (DIM == 3) ? (int)(row / n) : 0;
        const double wyz = tw(y, n, neu) * ((DIM == 3) ? tw(z, n, neu) : 1.0);
        const long long cbase = row * n;
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            const double u = __ldg(U + cbase + x);
            s = fma(tw(x, n, neu) * wyz * u, u, s);
        }
    }
    Sum4 acc{s, 0.0, INFINITY, -INFINITY};
    acc = block_sum4(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc.a;
}

// U *= 1 / sqrt(h^dim sum w U^2); every block sums the partials in the same order.
__global__ void __launch_bounds__(256) k_eig_scale(double *__restrict__ U, long long N, double hd,
                                                   const double *__restrict__ partials, int nparts,
                                                   const DevState *st) {
    if (state_done(st)) return;
    __shared__ double s_scale;
    Sum4 acc{0.0, 0.0, INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc.a += partials[i];
    acc = block_sum4(acc);
    if (threadIdx.x == 0) s_scale = 1.0 / sqrt(hd * acc.a);
    __syncthreads();
    const double sc = s_scale;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) U[i] *= sc;
}

}  // namespace

int launch_eig_rayleigh(const double *U, double *r0, int n, int dim, int bc, double inv_h2, double lam, double b,
                        const double *pot, double *partials, int grid, const DevState *st, cudaStream_t s) {
    if (dim == 3)
        k_eig_rayleigh<3><<<grid, 256, 0, s>>>(U, r0, n, bc, inv_h2, lam, b, pot, partials, st);
    else
        k_eig_rayleigh<2><<<grid, 256, 0, s>>>(U, r0, n, bc, inv_h2, lam, b, pot, partials, st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_eig_finalize1(const double *partials, int nparts, double hd, DevState *st, cudaStream_t s) {
    k_eig_finalize1<<<1, 256, 0, s>>>(partials, nparts, hd, st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_eig_residual2(const double *U, const double *r0, int n, int P, int dim, int bc, double hd, double *R64,
                         __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, bool mirror, double *partials, int grid,
                         const DevState *st, cudaStream_t s) {
    if (R64 != nullptr) {
        if (dim == 3)
            k_eig_residual2<3, 0><<<grid, 256, 0, s>>>(U, r0, n, P, bc, hd, R64, Rhi, Rlo, partials, st);
        else
            k_eig_residual2<2, 0><<<grid, 256, 0, s>>>(U, r0, n, P, bc, hd, R64, Rhi, Rlo, partials, st);
    } else if (mirror) {
        if (dim != 3 || P % 128 != 0) {
            set_error("launch_eig_residual2: the reflection-split layout needs 3-D and P a multiple of 128");
            return QN_EINVAL;
        }
        k_eig_residual2<3, 2><<<grid, 256, 0, s>>>(U, r0, n, P, bc, hd, R64, Rhi, Rlo, partials, st);
    } else if (dim == 3) {
        k_eig_residual2<3, 1><<<grid, 256, 0, s>>>(U, r0, n, P, bc, hd, R64, Rhi, Rlo, partials, st);
    } else {
        k_eig_residual2<2, 1><<<grid, 256, 0, s>>>(U, r0, n, P, bc, hd, R64, Rhi, Rlo, partials, st);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_eig_normalize(double *U, int n, int dim, int bc, double hd, double *partials, int grid,
                         const DevState *st, cudaStream_t s) {
    if (dim == 3)
        k_eig_sumsq<3><<<grid, 256, 0, s>>>(U, n, bc, partials, st);
    else
        k_eig_sumsq<2><<<grid, 256, 0, s>>>(U, n, bc, partials, st);
    QN_CUDA(cudaGetLastError());
    long long N = (long long)n * n;
    if (dim == 3) N *= n;
    k_eig_scale<<<grid, 256, 0, s>>>(U, N, hd, partials, grid, st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

}  // namespace qn
