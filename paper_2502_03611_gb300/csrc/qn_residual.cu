// Residual F(U) = A_h vec(U) + lam U + b U^3 - f (Sec. 4 eq. F_u, with the
// 5/7-point difference operator of Sec. 3.2 eq. fdm-discrete, Dirichlet 0)
// fused with the reductions the iteration needs: sum F^2 and sum f^2 (stop
// test) and min/max U^2 (beta_n = mid-range of diag(3 b U^2), Sec. 4
// eq. identity-method). One pass over U and f; HBM-bound.
//
// Outputs, selected per launch:
//   R64           dense FP64 residual (FP64 path, qn_residual)
//   Rhi/Rlo       residual rounded to FP32 and split into BF16 hi + lo planes
//                 on the zero-padded P^dim grid (input of the tensor-core
//                 mode products; padded entries are written as 0)
// Per-block partials go to a fixed-size array; a one-block finaliser reduces
// them in a fixed order (deterministic) and decides beta_n and convergence on
// the device.
#include <math.h>
#include <string.h>

#include <mutex>

#include "qn_internal.h"
#include "qn_numeric.cuh"

namespace qn {

namespace {

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

struct Red4 {
    double r2, f2, mn, mx;
};

__device__ __forceinline__ Red4 warp_reduce(Red4 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.r2 += __shfl_xor_sync(0xffffffffu, v.r2, o);
        v.f2 += __shfl_xor_sync(0xffffffffu, v.f2, o);
        v.mn = fmin(v.mn, __shfl_xor_sync(0xffffffffu, v.mn, o));
        v.mx = fmax(v.mx, __shfl_xor_sync(0xffffffffu, v.mx, o));
    }
    return v;
}

// Reduce over the block (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
__device__ Red4 block_reduce(Red4 v) {
    __shared__ Red4 sh[32];
    v = warp_reduce(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        v = (l < nw) ? sh[l] : Red4{0.0, 0.0, INFINITY, 0.0};
        v = warp_reduce(v);
    }
    return v;
}

// FP64-pipe budget per interior point (the GPU issues ~2 FP64 ops/clk/SM).
// Two implementations of the stencil 2d*u - sum(neighbours), run by different
// warps of the same block so that the FP64 pipe and the integer pipe work at
// the same time:
//   INT_STENCIL  exact fixed-point sum on the integer pipe (qn_numeric.cuh),
//                ~20x more instructions but no FP64 operation;
//   FP64         five adds and one FMA on the FP64 pipe.
// The rest costs u^2, b u^3 - f and lap/h^2 + (...): 3 FP64 ops (+1 with
// lam != 0, +1 with b != 1, +1 for sum f^2 on the first iteration, +1 for
// sum r^2 outside the split-precision solve, whose stop test sums float(r)^2
// with Kahan in FP32). min/max |U| use the integer bit pattern; the FP32
// rounding of r runs on the integer pipe. Each warp sweeps its own columns
// with one of the two loops (a warp-uniform branch around the whole loop, so
// neither variant is predicated into the other).
// KIND 0: lam u + b u^3 (general); 1: lam = 0; 2: lam = 0 and b = 1.
struct ResAcc {
    double r2, f2;
    float kr2, kc;
    unsigned long long amin, amax;
};

template <int DIM, bool SPLIT, bool FAST, int KIND, bool WANT_F2, bool INT_STENCIL>
__device__ __forceinline__ void residual_sweep(const ResidualArgs &a, ResAcc &s) {
    const int n = a.n;
    const int P = SPLIT ? a.P : n;
    const long long rows = (DIM == 3) ? (long long)P * P : (long long)P;
    const double *__restrict__ U = a.U;
    const double *__restrict__ f = a.f;
    const long long nn = (long long)n * n;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (DIM == 3) ? (int)(row % P) : (int)row;
        const int z = (DIM == 3) ? (int)(row / P) : 0;
        const bool row_ok = (y < n) && (z < n);
        const long long cbase = ((long long)z * n + y) * n;
        for (int x = threadIdx.x; x < P; x += blockDim.x) {
            double r = 0.0;
            if (row_ok && x < n) {
                const long long c = cbase + x;
                const double u = __ldg(U + c);
                double nbv[2 * DIM];
                nbv[0] = (x > 0) ? __ldg(U + c - 1) : 0.0;
                nbv[1] = (x < n - 1) ? __ldg(U + c + 1) : 0.0;
                nbv[2] = (y > 0) ? __ldg(U + c - n) : 0.0;
                nbv[3] = (y < n - 1) ? __ldg(U + c + n) : 0.0;
                if (DIM == 3) {
                    nbv[2 * DIM - 2] = (z > 0) ? __ldg(U + c - nn) : 0.0;
                    nbv[2 * DIM - 1] = (z < n - 1) ? __ldg(U + c + nn) : 0.0;
                }
                const double fv = __ldg(f + c);
                double lap;
                if (INT_STENCIL) {
                    lap = stencil_fixed<DIM>(u, nbv);
                } else {
                    double sum = (nbv[0] + nbv[1]) + (nbv[2] + nbv[3]);
                    if (DIM == 3) sum += nbv[4] + nbv[5];
                    lap = fma(2.0 * DIM, u, -sum);
                }
                const double u2 = u * u;
                double t;
                if (KIND == 2) {
                    t = fma(u2, u, -fv);
                } else {
                    t = fma(a.b, u2 * u, -fv);
                    if (KIND == 0) t = fma(a.lam, u, t);
                }
                r = fma(lap, a.inv_h2, t);
                const unsigned long long ab = abs_bits(u);
                s.amin = ab < s.amin ? ab : s.amin;
                s.amax = ab > s.amax ? ab : s.amax;
                if (WANT_F2) s.f2 = fma(fv, fv, s.f2);
                if (FAST) {
                    const float rf = d2f_rn(r);
                    const float yk = fmaf(rf, rf, -s.kc);
                    const float tk = s.kr2 + yk;
                    s.kc = (tk - s.kr2) - yk;
                    s.kr2 = tk;
                } else {
                    s.r2 = fma(r, r, s.r2);
                }
                if (a.R64 != nullptr) a.R64[c] = r;
            }
            if (SPLIT) {
                const float rf = d2f_rn(r);
                const __nv_bfloat16 hi = __float2bfloat16_rn(rf);
                const __nv_bfloat16 lo = __float2bfloat16_rn(rf - __bfloat162float(hi));
                const long long o = row * P + x;
                a.Rhi[o] = hi;
                a.Rlo[o] = lo;
            }
        }
    }
}

template <int DIM, bool SPLIT, bool FAST, int KIND, bool WANT_F2>
__global__ void __launch_bounds__(256) k_residual(ResidualArgs a) {
    if (a.done != nullptr && *(volatile const int *)a.done) return;
    ResAcc s{0.0, 0.0, 0.0f, 0.0f, 0x7FFFFFFFFFFFFFFFull, 0ull};
    if ((int)(threadIdx.x >> 5) < a.fp64_warps)
        residual_sweep<DIM, SPLIT, FAST, KIND, WANT_F2, false>(a, s);
    else
        residual_sweep<DIM, SPLIT, FAST, KIND, WANT_F2, true>(a, s);
    if (FAST) s.r2 = (double)s.kr2 - (double)s.kc;
    const double umin = __longlong_as_double((long long)s.amin);
    const double umax = __longlong_as_double((long long)s.amax);
    Red4 acc{s.r2, s.f2, (s.amin == 0x7FFFFFFFFFFFFFFFull) ? INFINITY : umin * umin, umax * umax};
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        double *p = a.partials + 4ll * blockIdx.x;
        p[0] = acc.r2;
        p[1] = acc.f2;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

__global__ void __launch_bounds__(256) k_finalize(const double *partials, int nparts, DevState *st,
                                                  qn_stats *hist, int hist_cap, double b,
                                                  double lam, int update_state, int use_saved_fnorm) {
    if (update_state && *(volatile int *)&st->done) return;
    Red4 acc{0.0, 0.0, INFINITY, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        acc.r2 += partials[4 * i + 0];
        acc.f2 += partials[4 * i + 1];
        acc.mn = fmin(acc.mn, partials[4 * i + 2]);
        acc.mx = fmax(acc.mx, partials[4 * i + 3]);
    }
    acc = block_reduce(acc);
    if (threadIdx.x != 0) return;
    const double res = sqrt(acc.r2);
    const double fn = use_saved_fnorm ? st->f_norm : sqrt(acc.f2);
    if (update_state && !use_saved_fnorm) st->f_norm = fn;
    const double fa = 3.0 * b * acc.mn, fb = 3.0 * b * acc.mx;
    const double fu_min = fmin(fa, fb), fu_max = fmax(fa, fb);
    const double beta = (st->beta_mode == QN_BETA_FIXED) ? st->beta_value : 0.5 * (fu_min + fu_max);
    double rel;
    if (fn > 0.0)
        rel = res / fn;
    else
        rel = (res == 0.0) ? 0.0 : INFINITY;
    const int it = st->it;
    if (hist != nullptr && it >= 0 && it < hist_cap) {
        qn_stats s;
        s.res_norm = res;
        s.f_norm = fn;
        s.fu_min = fu_min;
        s.fu_max = fu_max;
        s.beta = beta;
        s.rel = rel;
        hist[it] = s;
    }
    if (!update_state) return;
    st->beta = beta;
    st->shift = lam + beta;
    if (rel <= st->tol) {
        st->status = QN_OK;
        st->done = 1;
    } else if (!isfinite(rel) || rel > 1e8 || !isfinite(beta)) {
        st->status = QN_EDIVERGED;
        st->done = 1;
    } else if (it >= st->max_it) {
        st->status = QN_ENOTCONV;
        st->done = 1;
    } else {
        st->it = it + 1;   // the update about to run produces iterate it+1
    }
}

// Dense FP64 field -> FP32 -> BF16 hi/lo planes on the zero-padded P^dim grid.
template <int DIM>
__global__ void __launch_bounds__(256) k_split_pad(const double *__restrict__ r, int n, int P,
                                                   __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    const long long total = (DIM == 3) ? (long long)P * P * P : (long long)P * P;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % P);
        const long long row = o / P;
        const int y = (int)(row % P);
        const int z = (DIM == 3) ? (int)(row / P) : 0;
        double v = 0.0;
        if (x < n && y < n && z < n) v = r[((long long)z * n + y) * n + x];
        __nv_bfloat16 h, l;
        split_bf16((float)v, h, l);
        hi[o] = h;
        lo[o] = l;
    }
}

}  // namespace

int launch_split_pad(const double *r, int n, int P, int dim, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                     int grid, cudaStream_t s) {
    if (dim == 3)
        k_split_pad<3><<<grid, 256, 0, s>>>(r, n, P, hi, lo);
    else
        k_split_pad<2><<<grid, 256, 0, s>>>(r, n, P, hi, lo);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

template <int DIM, bool SPLIT, bool FAST, bool WF2>
static void launch_res4(const ResidualArgs &a, int grid, cudaStream_t s) {
    if (a.lam != 0.0)
        k_residual<DIM, SPLIT, FAST, 0, WF2><<<grid, 256, 0, s>>>(a);
    else if (a.b != 1.0)
        k_residual<DIM, SPLIT, FAST, 1, WF2><<<grid, 256, 0, s>>>(a);
    else
        k_residual<DIM, SPLIT, FAST, 2, WF2><<<grid, 256, 0, s>>>(a);
}

template <int DIM, bool SPLIT, bool FAST>
static void launch_res3(const ResidualArgs &a, int grid, cudaStream_t s) {
    if (a.want_f2)
        launch_res4<DIM, SPLIT, FAST, true>(a, grid, s);
    else
        launch_res4<DIM, SPLIT, FAST, false>(a, grid, s);
}

template <int DIM, bool SPLIT>
static void launch_res2(const ResidualArgs &a, int grid, cudaStream_t s) {
    if (a.fast)
        launch_res3<DIM, SPLIT, true>(a, grid, s);
    else
        launch_res3<DIM, SPLIT, false>(a, grid, s);
}

int launch_residual(const ResidualArgs &a, int grid, cudaStream_t s) {
    const bool split = a.Rhi != nullptr;
    if (a.dim == 3) {
        if (split)
            launch_res2<3, true>(a, grid, s);
        else
            launch_res2<3, false>(a, grid, s);
    } else {
        if (split)
            launch_res2<2, true>(a, grid, s);
        else
            launch_res2<2, false>(a, grid, s);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_finalize(const double *partials, int nparts, DevState *st, qn_stats *hist,
                        int hist_cap, double b, double lam, int update_state, int use_saved_fnorm,
                        cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nparts, st, hist, hist_cap, b, lam, update_state,
                                 use_saved_fnorm);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free residual (qn_residual_noalloc)
//
// Some callers cannot allocate device memory where they call the residual:
// their device memory is entirely owned by another allocator or a fixed
// budget (a framework's memory pool, a service with a hard memory cap), or
// they run in a section where allocation is not allowed. For them the
// residual kernel's scratch (per-block partial sums and the finalised
// statistics) lives in this fixed device array instead of a context's
// workspace. Every GPU that loads libqn holds it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxBlocks = 1024;               // reduction blocks per call
constexpr int kNoAllocStateDoubles = 16;              // DevState (<= 128 B)
constexpr int kNoAllocStatsDoubles = 8;               // one qn_stats (48 B)
constexpr int kNoAllocDoubles = 4 * kNoAllocMaxBlocks + kNoAllocStateDoubles + kNoAllocStatsDoubles;
static_assert(sizeof(DevState) <= kNoAllocStateDoubles * sizeof(double), "DevState too large");
static_assert(sizeof(qn_stats) <= kNoAllocStatsDoubles * sizeof(double), "qn_stats too large");

// 4096 partial-sum slots + solver state + one statistics record: 33 KB.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[128] = {nullptr};   // device address of the array, per device ordinal

// Device address of g_noalloc_scratch on the current device (looked up once
// per device; in host code the array's name is only a host-side stand-in).
int noalloc_scratch(double **out) {
    int dev = 0;
    QN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) {
        set_error("qn_residual_noalloc: device ordinal %d out of range", dev);
        return QN_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return QN_OK;
}

// Put the solver state in the scratch into "evaluate iterate 0, paper beta".
__global__ void k_noalloc_prepare(DevState *st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->done = 0;
        st->status = QN_OK;
        st->it = 0;
        st->err = 0;
        st->shift = 0.0;
        st->beta = 0.0;
        st->tol = -1.0;
        st->max_it = 0;
        st->beta_mode = QN_BETA_PAPER;
        st->beta_value = 0.0;
        st->f_norm = 0.0;
    }
}

}  // namespace

}  // namespace qn

extern "C" int qn_residual_noalloc(int dim, int n, double lam, double b, const double *U,
                                   const double *f, double *R, qn_stats *st, void *stream) {
    using namespace qn;
    if (dim != 2 && dim != 3) {
        set_error("qn_residual_noalloc: dim must be 2 or 3 (got %d)", dim);
        return QN_EINVAL;
    }
    if (n < 1 || n > 1024) {
        set_error("qn_residual_noalloc: n=%d exceeds the supported range 1..1024", n);
        return QN_EINVAL;
    }
    if (!U || !f || !st) {
        set_error("qn_residual_noalloc: U, f and st must be non-null");
        return QN_EINVAL;
    }
    if (!isfinite(lam) || !isfinite(b)) {
        set_error("qn_residual_noalloc: lam and b must be finite");
        return QN_EINVAL;
    }
    const long long rows = (dim == 3) ? (long long)n * n : (long long)n;
    const int grid = rows < kNoAllocMaxBlocks ? (int)rows : kNoAllocMaxBlocks;
    if (grid > kNoAllocMaxBlocks) {   // cannot happen with n <= 1024; kept as the scratch guard
        set_error("qn_residual_noalloc: %d reduction blocks exceed the scratch maximum %d", grid,
                  kNoAllocMaxBlocks);
        return QN_EINVAL;
    }
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != QN_OK) return rc;
    double *partials = scratch;
    DevState *state = reinterpret_cast<DevState *>(scratch + 4 * kNoAllocMaxBlocks);
    qn_stats *stats = reinterpret_cast<qn_stats *>(scratch + 4 * kNoAllocMaxBlocks + kNoAllocStateDoubles);
    cudaStream_t s = (cudaStream_t)stream;

    // every partial slot read below is written by this call's residual
    // blocks, so only the solver state needs resetting
    k_noalloc_prepare<<<1, 32, 0, s>>>(state);
    QN_CUDA(cudaGetLastError());
    ResidualArgs a;
    a.U = U;
    a.f = f;
    a.n = n;
    a.dim = dim;
    const double h = 1.0 / (n + 1);
    a.inv_h2 = 1.0 / (h * h);
    a.lam = lam;
    a.b = b;
    a.R64 = R;
    a.Rhi = nullptr;
    a.Rlo = nullptr;
    a.P = n;
    a.partials = partials;
    a.done = nullptr;
    a.fast = 0;
    a.want_f2 = 1;
    a.fp64_warps = 0;
    rc = launch_residual(a, grid, s);
    if (rc != QN_OK) return rc;
    rc = launch_finalize(partials, grid, state, stats, 1, b, lam, 0, 0, s);
    if (rc != QN_OK) return rc;
    QN_CUDA(cudaMemcpyAsync(st, stats, sizeof(qn_stats), cudaMemcpyDeviceToHost, s));
    QN_CUDA(cudaStreamSynchronize(s));
    return QN_OK;
}
