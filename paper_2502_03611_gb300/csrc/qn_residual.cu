// Residual F(U) = A_h vec(U) + lam U + b U^3 + V U - f (Sec. 4 eq. F_u, with
// the 5/7-point difference operator of Sec. 3.2 eq. fdm-discrete: Dirichlet 0
// past a face, or the ghost-point reflection of the Neumann rows) fused with
// the reductions the iteration needs: sum F^2 and sum f^2 (stop test) and
// min/max U^2, or min/max of 3 b U^2 + V with a potential (beta_n = mid-range
// of diag(N_h)_U, Sec. 4 eq. identity-method). One pass over U and f.
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
#include "qn_df.cuh"
#include "qn_numeric.cuh"
#include "qn_ptx.cuh"

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

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block-wide max (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
__device__ unsigned long long block_max_u64(unsigned long long v) {
    __shared__ unsigned long long sh[32];
    v = warp_max_u64(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0ull;
        v = warp_max_u64(v);
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
// KIND 0: lam u + b u^3 (general); 1: lam = 0; 2: lam = 0 and b = 1;
// 3: (lam + V) u + b u^3 with the separable potential V. The float-pair copy of f
// that k_residual_tiled reads comes from f_pair (qn_df.cuh).
struct ResAcc {
    double r2, f2;
    float kr2, kc;
    unsigned long long amin, amax;
    float r2s;   // 2^-r2_exp: r is scaled before its FP32 square
    double dmn, dmx;   // KIND 3: extremes of 3 b u^2 + V
};

template <int DIM, bool SPLIT, bool FAST, int KIND, bool WANT_F2, bool INT_STENCIL>
__device__ __forceinline__ void residual_sweep(const ResidualArgs &a, ResAcc &s) {
    const int n = a.n;
    const int P = SPLIT ? a.P : n;
    const long long rows = (DIM == 3) ? (long long)P * P : (long long)P;
    const double *__restrict__ U = a.U;
    const double *__restrict__ f = a.f;
    const long long nn = (long long)n * n;
    // Neumann and Robin faces: the missing neighbour is the ghost value, i.e. the
    // neighbour on the other side (n >= 2 is guaranteed for these data); Robin adds
    // -2 h kappa u to the ghost, i.e. (2 kappa / h) u per face to the residual
    const bool neu = (a.bc == QN_BC_NEUMANN || a.bc == QN_BC_ROBIN);
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int y = (DIM == 3) ? (int)(row % P) : (int)row;
        const int z = (DIM == 3) ? (int)(row / P) : 0;
        const bool row_ok = (y < n) && (z < n);
        const long long cbase = ((long long)z * n + y) * n;
        double vrow = 0.0;   // KIND 3: lam + v_y(y) + v_z(z)
        if (KIND == 3 && row_ok) {
            vrow = a.lam + __ldg(a.pot + n + y);
            if (DIM == 3) vrow += __ldg(a.pot + 2 * n + z);
        }
        for (int x = threadIdx.x; x < P; x += blockDim.x) {
            double r = 0.0;
            if (row_ok && x < n) {
                const long long c = cbase + x;
                const double u = __ldg(U + c);
                double nbv[2 * DIM];
                nbv[0] = (x > 0) ? __ldg(U + c - 1) : (neu ? __ldg(U + c + 1) : 0.0);
                nbv[1] = (x < n - 1) ? __ldg(U + c + 1) : (neu ? __ldg(U + c - 1) : 0.0);
                nbv[2] = (y > 0) ? __ldg(U + c - n) : (neu ? __ldg(U + c + n) : 0.0);
                nbv[3] = (y < n - 1) ? __ldg(U + c + n) : (neu ? __ldg(U + c - n) : 0.0);
                if (DIM == 3) {
                    nbv[2 * DIM - 2] = (z > 0) ? __ldg(U + c - nn) : (neu ? __ldg(U + c + nn) : 0.0);
                    nbv[2 * DIM - 1] = (z < n - 1) ? __ldg(U + c + nn) : (neu ? __ldg(U + c - nn) : 0.0);
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
                if (KIND == 3) {
                    const double cv = vrow + __ldg(a.pot + x);        // lam + V
                    t = fma(cv, u, t);
                    const double d = fma(3.0 * a.b, u2, cv - a.lam);  // 3 b u^2 + V
                    s.dmn = fmin(s.dmn, d);
                    s.dmx = fmax(s.dmx, d);
                }
                r = fma(lap, a.inv_h2, t);
                if (a.robin != 0.0) {
                    int faces = (x == 0) + (x == n - 1) + (y == 0) + (y == n - 1);
                    if (DIM == 3) faces += (z == 0) + (z == n - 1);
                    r = fma(a.robin * faces, u, r);
                }
                const unsigned long long ab = abs_bits(u);
                s.amin = ab < s.amin ? ab : s.amin;
                s.amax = ab > s.amax ? ab : s.amax;
                if (WANT_F2) s.f2 = fma(fv, fv, s.f2);
                if (FAST) {
                    const float rf = __fmul_rn(d2f_rn(r), s.r2s);
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
    const int r2k = FAST ? *a.r2_exp : 0;
    ResAcc s{0.0, 0.0, 0.0f, 0.0f, 0x7FFFFFFFFFFFFFFFull, 0ull, __int_as_float((127 - r2k) << 23),
             INFINITY, -INFINITY};
    if ((int)(threadIdx.x >> 5) < a.fp64_warps)
        residual_sweep<DIM, SPLIT, FAST, KIND, WANT_F2, false>(a, s);
    else
        residual_sweep<DIM, SPLIT, FAST, KIND, WANT_F2, true>(a, s);
    if (FAST) s.r2 = ldexp((double)s.kr2 - (double)s.kc, 2 * r2k);
    const double umin = __longlong_as_double((long long)s.amin);
    const double umax = __longlong_as_double((long long)s.amax);
    Red4 acc{s.r2, s.f2, (s.amin == 0x7FFFFFFFFFFFFFFFull) ? INFINITY : umin * umin, umax * umax};
    if (KIND == 3) {
        acc.mn = s.dmn;
        acc.mx = s.dmx;
        const unsigned long long bm = block_max_u64(s.amax);
        if (threadIdx.x == 0 && a.umax_scan != nullptr) atomicMax(a.umax_scan, bm);
    }
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        double *p = a.partials + 4ll * blockIdx.x;
        p[0] = acc.r2;
        p[1] = acc.f2;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

// Exponent E of the fixed-point stencil of k_residual_tiled for an iterate
// whose max|U| has bit pattern umax: its exponent plus DevState::fx_headroom
// (2: room for U to grow 4x before planes take the exact path). 0 (not
// usable) for a subnormal, non-finite or out-of-range max|U| (outside
// 2^[-60, 36], where the float-pair arithmetic could leave the FP32 range),
// for a source beyond the FP32-pair copy, or for ||f|| < 2^-40.
__device__ __forceinline__ int fx_exponent(unsigned long long umax, const DevState *st) {
    if (st->fx_fbad || !(st->f_norm >= 0x1p-40)) return 0;
    if (umax == 0ull) return 1023;   // U = 0: every fixed-point value is 0, any exponent serves
    const int ex = (int)((umax >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) return 0;
    const int E = ex + st->fx_headroom;
    return (E - 1023 >= -60 && E - 1023 <= 36) ? E : 0;
}

// Iteration 0 of a 3-D split solve, one pass over f and U_0: the padded
// FP32-pair copy of f (zeros in the padding), per-block sums of f^2 (FP64),
// the |f| range check and the max|U_0| bit pattern. MIRROR: the copy is laid
// out for k_residual_mirror, entry (z, y, i < P/2) = (f(i), f(n-1-i)) as two
// FP32 pairs (the second zero where n-1-i <= i); else (z, y, x) = f(x).
// With Rhi != nullptr it also writes the residual of the zero start, r = -f
// rounded to FP32 (what the tiled kernels compute at U = 0, bit for bit), into
// the planes in their layout; the iteration-0 residual then skips its work
// when the pass found U_0 = 0 (DevState::u0_zero), and overwrites the planes
// otherwise.
template <bool MIRROR>
__global__ void __launch_bounds__(256) k_prep_split(const double *__restrict__ U, const double *__restrict__ f,
                                                    int n, int P, float2 *__restrict__ fdf,
                                                    __nv_bfloat16 *__restrict__ Rhi, __nv_bfloat16 *__restrict__ Rlo,
                                                    double *__restrict__ partials, DevState *st) {
    const long long rows = (long long)P * P;
    const int H = P / 2, nsym = (n + 1) / 2, nanti = n / 2;
    double f2 = 0.0;
    unsigned long long umax = 0ull;
    float s2h = 0.0f, s2l = 0.0f;   // sum f^2 as a float pair (MIRROR)
    if (MIRROR) {
        // four rows per step, their loads issued together (the pass is
        // latency-bound with one row per step); rows < P^2 <= 2^22: 32-bit index math
        constexpr int kRows = 4;
        float4 *f4 = reinterpret_cast<float4 *>(fdf);
        const unsigned int urows = (unsigned int)rows, uP = (unsigned int)P;
        for (unsigned int row0 = blockIdx.x; row0 < urows; row0 += (unsigned int)kRows * gridDim.x) {
            int ys[kRows], zs[kRows];
#pragma unroll
            for (int g = 0; g < kRows; ++g) {
                const unsigned int row = row0 + (unsigned int)g * gridDim.x;
                zs[g] = (int)(row / uP);
                ys[g] = (int)(row - (unsigned int)zs[g] * uP);
            }
            for (int i = threadIdx.x; i < H; i += blockDim.x) {
                double fa[kRows], fb[kRows], ua[kRows], ub[kRows];
                bool oka[kRows], okb[kRows];
#pragma unroll
                for (int g = 0; g < kRows; ++g) {
                    const unsigned int row = row0 + (unsigned int)g * gridDim.x;
                    const int y = ys[g], z = zs[g];
                    const bool row_ok = row < urows && (y < n) && (z < n);
                    const long long cbase = ((long long)z * n + y) * n;
                    oka[g] = row_ok && i < nsym;
                    okb[g] = row_ok && i < nanti;
                    fa[g] = oka[g] ? __ldg(f + cbase + i) : 0.0;
                    ua[g] = oka[g] ? __ldg(U + cbase + i) : 0.0;
                    fb[g] = okb[g] ? __ldg(f + cbase + (n - 1 - i)) : 0.0;
                    ub[g] = okb[g] ? __ldg(U + cbase + (n - 1 - i)) : 0.0;
                }
#pragma unroll
                for (int g = 0; g < kRows; ++g) {
                    const unsigned int row = row0 + (unsigned int)g * gridDim.x;
                    if (row >= urows) break;
                    float2 a = make_float2(0.0f, 0.0f), b = a;
                    if (oka[g]) {
                        a = f_pair(fa[g], &st->fx_fbad);
                        const unsigned long long ab = abs_bits(ua[g]);
                        umax = ab > umax ? ab : umax;
                    }
                    if (okb[g]) {
                        b = f_pair(fb[g], &st->fx_fbad);
                        const unsigned long long ab = abs_bits(ub[g]);
                        umax = ab > umax ? ab : umax;
                    }
                    // f^2 = hi^2 + 2 hi lo (+ lo^2, below 2^-46 of it) as a float pair
                    {
                        float p = __fmul_rn(a.x, a.x), e = __fmaf_rn(a.x, a.x, -p);
                        e = __fmaf_rn(__fadd_rn(a.x, a.x), a.y, e);
                        const float q = __fmul_rn(b.x, b.x);
                        float eq = __fmaf_rn(b.x, b.x, -q);
                        eq = __fmaf_rn(__fadd_rn(b.x, b.x), b.y, eq);
                        float t, te;
                        two_sum(p, q, t, te);
                        float s, se;
                        two_sum(s2h, t, s, se);
                        s2l = __fadd_rn(s2l, __fadd_rn(se, __fadd_rn(te, __fadd_rn(e, eq))));
                        s2h = s;
                    }
                    f4[(long long)row * H + i] = make_float4(a.x, a.y, b.x, b.y);
                    if (Rhi != nullptr) {
                        // split order along x, folded rows (rows of the padding stay in place)
                        const int y = ys[g], z = zs[g];
                        const int Fy = (y >= n) ? y : (y < nsym ? 2 * y : 2 * (n - 1 - y) + 1);
                        const int Fz = (z >= n) ? z : (z < nsym ? 2 * z : 2 * (n - 1 - z) + 1);
                        const long long o = ((long long)Fz * P + Fy) * P;
                        // (+ 0.0f: a zero f gives +0, as the residual's arithmetic does)
                        const float ra = oka[g] ? __fadd_rn(-a.x, 0.0f) : 0.0f;
                        const float rb = okb[g] ? __fadd_rn(-b.x, 0.0f) : 0.0f;
                        split_bf16(__fadd_rn(ra, rb), Rhi[o + i], Rlo[o + i]);
                        split_bf16(okb[g] ? __fsub_rn(ra, rb) : 0.0f, Rhi[o + H + i], Rlo[o + H + i]);
                    }
                }
            }
        }
        f2 = (double)s2h + (double)s2l;
    }
    for (long long row = blockIdx.x; !MIRROR && row < rows; row += gridDim.x) {
        const int y = (int)(row % P), z = (int)(row / P);
        const bool row_ok = (y < n) && (z < n);
        const long long cbase = ((long long)z * n + y) * n;
        {
            for (int x = threadIdx.x; x < P; x += blockDim.x) {
                float2 fp = make_float2(0.0f, 0.0f);
                if (row_ok && x < n) {
                    const double fv = __ldg(f + cbase + x);
                    f2 = fma(fv, fv, f2);
                    fp = f_pair(fv, &st->fx_fbad);
                    const unsigned long long ab = abs_bits(__ldg(U + cbase + x));
                    umax = ab > umax ? ab : umax;
                }
                fdf[row * P + x] = fp;
                if (Rhi != nullptr)
                    split_bf16((row_ok && x < n) ? __fadd_rn(-fp.x, 0.0f) : 0.0f, Rhi[row * P + x], Rlo[row * P + x]);
            }
        }
    }
    const unsigned long long bm = block_max_u64(umax);
    Red4 acc{0.0, f2, 0.0, 0.0};
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        partials[4ll * blockIdx.x + 1] = acc.f2;
        atomicMax(&st->umax_scan, bm);
    }
}

// ||f|| (fixed-order sum of the partials), the scale of the FP32 norm sums
// and the fixed-point exponent for the first residual.
__global__ void __launch_bounds__(256) k_prep_split_finish(const double *partials, int nparts, DevState *st) {
    Red4 acc{0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc.f2 += partials[4 * i + 1];
    acc = block_reduce(acc);
    if (threadIdx.x != 0) return;
    const double fn = sqrt(acc.f2);
    st->f_norm = fn;
    const double rms = (st->npts > 0.0) ? fn / sqrt(st->npts) : 0.0;
    const int k = (rms > 0.0 && rms < INFINITY) ? ilogb(rms) : 0;
    st->r2_exp = k < -120 ? -120 : (k > 120 ? 120 : k);
    st->fx_e = fx_exponent(st->umax_scan, st);
    st->u0_zero = (st->umax_scan == 0ull) ? 1 : 0;
    st->umax_scan = 0ull;
}

// The iteration-0 residual of a zero start (the preparation pass wrote r = -f):
// every CTA writes its partial record only, ||r||^2 = ||f||^2 in CTA 0 and
// min / max U^2 = 0. True when it did so.
__device__ __forceinline__ bool zero_start_partials(const ResidualArgs &a) {
    if (a.zero_start == nullptr || !*(volatile const int *)&a.zero_start->u0_zero) return false;
    if (threadIdx.x == 0) {
        double *p = a.partials + 4ll * blockIdx.x;
        const double fn = a.zero_start->f_norm;
        p[0] = (blockIdx.x == 0) ? fn * fn : 0.0;
        p[1] = 0.0;
        p[2] = 0.0;
        p[3] = 0.0;
    }
    return true;
}

// max|U| bit pattern of a dense array (iteration 1: the first update's result).
__global__ void __launch_bounds__(256) k_umax(const double *__restrict__ U, long long N, int vec16, DevState *st) {
    if (*(volatile const int *)&st->done) return;
    const unsigned long long *b = reinterpret_cast<const unsigned long long *>(U);
    unsigned long long m = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long tail = 0;
    if (vec16) {   // U 16-B aligned: two values per load
        const long long N2 = N >> 1;
        const ulonglong2 *b2 = reinterpret_cast<const ulonglong2 *>(b);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N2; i += stride) {
            const ulonglong2 v = __ldg(b2 + i);
            const unsigned long long a0 = v.x & 0x7FFFFFFFFFFFFFFFull, a1 = v.y & 0x7FFFFFFFFFFFFFFFull;
            m = a0 > m ? a0 : m;
            m = a1 > m ? a1 : m;
        }
        tail = 2 * N2;
    }
    for (long long i = tail + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += stride) {
        const unsigned long long a = __ldg(b + i) & 0x7FFFFFFFFFFFFFFFull;
        m = a > m ? a : m;
    }
    const unsigned long long bm = block_max_u64(m);
    if (threadIdx.x == 0) atomicMax(&st->umax_scan, bm);
}

__global__ void k_umax_finish(DevState *st) {
    if (threadIdx.x != 0 || *(volatile const int *)&st->done) return;
    st->fx_e = fx_exponent(st->umax_scan, st);
    st->umax_scan = 0ull;
}

__global__ void __launch_bounds__(256) k_finalize(const double *partials, int nparts, DevState *st,
                                                  qn_stats *hist, int hist_cap, double b,
                                                  double lam, int update_state, int use_saved_fnorm,
                                                  int mode) {
    const bool pot = (mode == 1), eig = (mode == 2);
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
    if (update_state && !use_saved_fnorm) {
        st->f_norm = fn;
        // scale of the FP32 sum of r^2 in the later iterations: 2^k ~ RMS(f)
        const double rms = (st->npts > 0.0) ? fn / sqrt(st->npts) : 0.0;
        int k = (rms > 0.0 && rms < INFINITY) ? ilogb(rms) : 0;
        st->r2_exp = k < -120 ? -120 : (k > 120 ? 120 : k);
    }
    // extremes of diag(N_h)_U: 3 b U^2 from those of U^2, or taken directly with a potential
    const double fa = (pot || eig) ? acc.mn : 3.0 * b * acc.mn, fb = (pot || eig) ? acc.mx : 3.0 * b * acc.mx;
    const double fu_min = fmin(fa, fb), fu_max = fmax(fa, fb);
    // eigen solves: (N_h)_U = diag(lam + 3 b U^2 + V) - lambda_n (extremes from pass 2)
    const double beta = (st->beta_mode == QN_BETA_FIXED) ? st->beta_value
                                                         : 0.5 * (fu_min + fu_max) - (eig ? st->eig_lambda : 0.0);
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
        s.lambda = eig ? st->eig_lambda : 0.0;
        hist[it] = s;
    }
    if (!update_state) return;
    // exponent for the fixed-point stencil of the next residual, from max|U|
    // of this iterate (sqrt of max U^2 has at least max|U|'s exponent: the
    // rounding of u^2 can only carry it up)
    if (pot || eig) {   // max|U| gathered by the residual passes (atomicMax of bit patterns)
        st->fx_e = fx_exponent(st->umax_scan, st);
        st->umax_scan = 0ull;
    } else {
        st->fx_e = (acc.mx < INFINITY) ? fx_exponent((unsigned long long)__double_as_longlong(sqrt(acc.mx)), st) : 0;
    }
    st->beta = beta;
    st->shift = eig ? beta : lam + beta;   // eigen solves: lam is part of f, not of A_h
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

// ---------------------------------------------------------------------------
// k_residual_tiled: the residual of the split-precision 3-D solve with no FP64
// arithmetic per point (used from the third iteration of a solve on).
//
// Every U value is converted once to a signed fixed-point integer in units of
// 2^(E - 1075 - kFxG), E = DevState::fx_e (the biased exponent of max|U| of
// the previous iterate plus 2, i.e. room for U to grow 4x). The 7-point
// stencil 6u - sum(nb) is then an exact int64 sum. The remaining terms,
// lap/h^2 + lam u + b u^3 - f, are evaluated in unevaluated pairs of floats
// (hi + lo, ~48 significant bits) on the FP32 pipe, f being read from its
// FP32-pair copy written by the first residual of the solve.
// Accuracy: each stencil input is truncated toward zero at the unit
// 2^(E-1075-kFxG) (1/8 ulp of max|U|), so 6u - sum(nb) is off by at most 12
// units, 1.5 ulp of max|U| - less than rounding the same sum in FP64; the float-
// pair arithmetic adds ~2^-46 of the largest term (|lap/h^2|, |b u^3|, |f|),
// about 1e-14 ||f||, far below the 1e-10 stop tolerance; the result is
// rounded once to FP32, the precision of the split planes it feeds.
//
// Layout: a block owns a 64 x 16 (x, y) tile of the padded grid and a chunk
// of planes, marching in z. Each thread holds 2 x 2 points (an x pair in two
// consecutive rows) of three consecutive planes in registers; the current
// plane with a one-point halo sits in shared memory (two buffers, one barrier
// per plane) for the x/y neighbours. The loads of plane z+2 and of f on plane
// z+1 are issued before the stencil of plane z.
//
// A plane holding a value whose exponent exceeds E (U grew more than 4x, or a
// non-finite value) is flagged through the barrier's OR; the points whose
// stencil touches it are evaluated by the exact per-point path of k_residual
// instead. E = 0 (not usable) sends every point there.
// ---------------------------------------------------------------------------
constexpr int kTX = 64, kTY = 16, kTThreads = 256;
constexpr int kSRow = 68;                                 // int64 per shared row; x = -1..64 at columns 1..66
constexpr int kSRows = kTY + 2;
constexpr int kHaloPerWarp = (2 * kTX + 2 * kTY) / 8;    // 160 halo points, 20 per warp
static_assert(kTThreads == 8 * 32 && kTY == 2 * 8 && kTX == 2 * 32, "tile / thread mapping");

// r = lap/h^2 + lam u + b u^3 - f in float pairs, rounded to FP32, from u = (uh, ul) and
// lap = (Lh, Ll) as float pairs. KIND 3: (lh, ll) is the point's lam + V, and d receives
// 3 b u^2 + V (FP32, V = vf).
template <int KIND>
__device__ __forceinline__ float residual_core(float uh, float ul, float Lh, float Ll, float fh, float fl,
                                               float ih, float il, float bh, float bl, float lh, float ll,
                                               float vf, float *d) {
    const float p = __fmul_rn(uh, uh);
    float pe = __fmaf_rn(uh, uh, -p);
    pe = __fmaf_rn(__fadd_rn(uh, uh), ul, pe);
    float w = __fmul_rn(p, uh);
    float we = __fmaf_rn(p, uh, -w);
    we = __fmaf_rn(p, ul, we);
    we = __fmaf_rn(pe, uh, we);
    if (KIND != 2) {
        const float w2 = __fmul_rn(bh, w);
        float e2 = __fmaf_rn(bh, w, -w2);
        e2 = __fmaf_rn(bh, we, e2);
        e2 = __fmaf_rn(bl, w, e2);
        w = w2;
        we = e2;
    }
    if (KIND == 3) *d = __fmaf_rn(__fmul_rn(3.0f, bh), p, vf);
    if (KIND == 0 || KIND == 3) {
        const float v = __fmul_rn(lh, uh);
        float ve = __fmaf_rn(lh, uh, -v);
        ve = __fmaf_rn(lh, ul, ve);
        ve = __fmaf_rn(ll, uh, ve);
        float s2, e2;
        two_sum(w, v, s2, e2);
        we = __fadd_rn(__fadd_rn(we, ve), e2);
        w = s2;
    }
    float t, te;
    two_sum(w, -fh, t, te);
    te = __fadd_rn(te, __fsub_rn(we, fl));
    const float L = __fmul_rn(Lh, ih);
    float Le = __fmaf_rn(Lh, ih, -L);
    Le = __fmaf_rn(Ll, ih, Le);
    Le = __fmaf_rn(Lh, il, Le);
    float r, re;
    two_sum(L, t, r, re);
    re = __fadd_rn(re, __fadd_rn(Le, te));
    return __fadd_rn(r, re);
}

// Two points: the fixed-point values of u and of the stencil sum to float pairs with the
// packed FP32x2 instructions (the three chunks of both values in one chain), then the
// float-pair arithmetic per point in scalar FP32. Packing that part as well saves FP32
// instructions but halves the independent chains the schedulers interleave, and this
// kernel is latency-bound at four warps per scheduler: measured 0.869 ms at 511^3 fully
// packed, 0.856 ms this way, 0.887 ms unpacked. The results are the same bit for bit.
template <int KIND>
__device__ __forceinline__ float2 residual_pair2(long long u0, long long u1, long long l0, long long l1, float2 fh,
                                                 float2 fl, float scale, float ih, float il, float bh, float bl,
                                                 float2 lh, float2 ll, float2 vf = make_float2(0.0f, 0.0f),
                                                 float2 *d = nullptr) {
    float2 uh, ul, Lh, Ll;
    fx_to_pair2(u0, u1, scale, uh, ul);
    fx_to_pair2(l0, l1, scale, Lh, Ll);
    float d0 = 0.0f, d1 = 0.0f;
    const float r0 = residual_core<KIND>(uh.x, ul.x, Lh.x, Ll.x, fh.x, fl.x, ih, il, bh, bl, lh.x, ll.x, vf.x, &d0);
    const float r1 = residual_core<KIND>(uh.y, ul.y, Lh.y, Ll.y, fh.y, fl.y, ih, il, bh, bl, lh.y, ll.y, vf.y, &d1);
    if (KIND == 3) *d = make_float2(d0, d1);
    return make_float2(r0, r1);
}

// The exact per-point path (as k_residual), for points next to a flagged plane.
// Returns (r, 3 b u^2 + V); the second entry is 0 without a potential (pot == nullptr).
static __device__ __noinline__ float2 residual_point_exact(const double *U, const double *f, int n, int x, int y,
                                                           int z, double inv_h2, double lam, double b, int bc,
                                                           const double *pot) {
    const long long nn = (long long)n * n;
    const long long c = ((long long)z * n + y) * n + x;
    const bool neu = (bc == QN_BC_NEUMANN);
    const double u = U[c];
    double nb[6];
    nb[0] = (x > 0) ? U[c - 1] : (neu ? U[c + 1] : 0.0);
    nb[1] = (x < n - 1) ? U[c + 1] : (neu ? U[c - 1] : 0.0);
    nb[2] = (y > 0) ? U[c - n] : (neu ? U[c + n] : 0.0);
    nb[3] = (y < n - 1) ? U[c + n] : (neu ? U[c - n] : 0.0);
    nb[4] = (z > 0) ? U[c - nn] : (neu ? U[c + nn] : 0.0);
    nb[5] = (z < n - 1) ? U[c + nn] : (neu ? U[c - nn] : 0.0);
    const double lap = stencil_fixed<3>(u, nb);
    double t = fma(b, (u * u) * u, -f[c]);
    double cv = lam;
    float d = 0.0f;
    if (pot != nullptr) {
        cv += (pot[x] + pot[n + y]) + pot[2 * n + z];
        d = d2f_rn(fma(3.0 * b, u * u, cv - lam));
    }
    t = fma(cv, u, t);
    return make_float2(d2f_rn(fma(lap, inv_h2, t)), d);
}

// Grid index of the value a stencil reads at coordinate i (-1 <= i <= n):
// itself, or for Neumann data the ghost reflection -1 -> 1, n -> n-2.
// Indexes outside [0, n) after the mapping read as 0 (Dirichlet data, padding).
__device__ __forceinline__ int ghost_index(int i, int n, bool neu) {
    return neu ? (i == -1 ? 1 : (i == n ? n - 2 : i)) : i;
}

__device__ __forceinline__ void store_split2(__nv_bfloat162 *hi2, __nv_bfloat162 *lo2, long long i2, float r0,
                                             float r1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
    const float2 hf = __bfloat1622float2(h);
    hi2[i2] = h;
    lo2[i2] = __floats2bfloat162_rn(__fsub_rn(r0, hf.x), __fsub_rn(r1, hf.y));
}

__device__ __forceinline__ void minmax_bits(unsigned long long v, bool valid, unsigned long long &mn,
                                            unsigned long long &mx) {
    const unsigned long long ab = v & 0x7FFFFFFFFFFFFFFFull;
    mn = (valid && ab < mn) ? ab : mn;
    mx = (valid && ab > mx) ? ab : mx;
}

// Block partial record of the tiled residuals: sum r^2 (from the scaled FP32
// Kahan sum) and min / max U^2, or with a potential (KIND 3) min / max of
// 3 b U^2 + V, with max|U| sent to DevState::umax_scan.
template <int KIND>
__device__ __forceinline__ void tile_partials(const ResidualArgs &a, float kr2, float kc, int r2k,
                                              unsigned long long amin, unsigned long long amax, float dmn,
                                              float dmx) {
    const double umin = __longlong_as_double((long long)amin);
    const double umax = __longlong_as_double((long long)amax);
    Red4 acc{ldexp((double)kr2 - (double)kc, 2 * r2k), 0.0,
             (amin == 0x7FFFFFFFFFFFFFFFull) ? INFINITY : umin * umin, umax * umax};
    if (KIND == 3) {
        acc.mn = (double)dmn;
        acc.mx = (double)dmx;
        const unsigned long long bm = block_max_u64(amax);
        if (threadIdx.x == 0) atomicMax(a.umax_scan, bm);
    }
    acc = block_reduce(acc);
    if (threadIdx.x == 0) {
        double *p = a.partials + 4ll * blockIdx.x;
        p[0] = acc.r2;
        p[1] = acc.f2;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kTThreads, 2) k_residual_tiled(ResidualArgs a, int zchunk) {
    if (a.done != nullptr && *(volatile const int *)a.done) return;
    if (KIND != 3 && zero_start_partials(a)) return;
    __shared__ __align__(16) long long spl[2][kSRows * kSRow];
    const int n = a.n, P = a.P;
    const int E = *a.fx_e;
    const bool fx_ok = (E != 0);
    const float scale = __int_as_float(fx_ok ? ((E - 1075 - kFxG + 127) << 23) : 0);
    const float ih = __double2float_rn(a.inv_h2);
    const float il = __double2float_rn(a.inv_h2 - (double)ih);
    float bh = 1.0f, bl = 0.0f, lh = 0.0f, ll = 0.0f;
    if (KIND != 2) {
        bh = __double2float_rn(a.b);
        bl = __double2float_rn(a.b - (double)bh);
    }
    if (KIND == 0 || KIND == 3) {
        lh = __double2float_rn(a.lam);
        ll = __double2float_rn(a.lam - (double)lh);
    }
    const bool neu = (a.bc == QN_BC_NEUMANN);
    float dmn = INFINITY, dmx = -INFINITY;   // KIND 3: extremes of 3 b u^2 + V
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = P / kTX, tiles_y = P / kTY;
    const int nzc = (P + zchunk - 1) / zchunk;
    const long long items = (long long)tiles_x * tiles_y * nzc;
    const long long nn = (long long)n * n;
    const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(a.U);
    const float4 *fdf4 = reinterpret_cast<const float4 *>(a.fdf);
    __nv_bfloat162 *Rhi2 = reinterpret_cast<__nv_bfloat162 *>(a.Rhi);
    __nv_bfloat162 *Rlo2 = reinterpret_cast<__nv_bfloat162 *>(a.Rlo);
    const int s0 = (2 * warp + 1) * kSRow + 2 * lane + 2;   // shared slot of own point (xo, yo)
    const bool hlane = lane < kHaloPerWarp;
    const int hidx = warp * kHaloPerWarp + lane;
    float kr2 = 0.0f, kc = 0.0f;
    unsigned long long amin = 0x7FFFFFFFFFFFFFFFull, amax = 0ull;
    const int r2k = *a.r2_exp;
    const float r2s = __int_as_float((127 - r2k) << 23);   // 2^-r2k

    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int tx = (int)(item % tiles_x);
        const long long q = item / tiles_x;
        const int ty = (int)(q % tiles_y);
        const int z0 = (int)(q / tiles_y) * zchunk;
        const int z1 = min(z0 + zchunk, P);
        const int X0 = tx * kTX, Y0 = ty * kTY;
        const int xo = X0 + 2 * lane, yo = Y0 + 2 * warp;
        // zero planes of the padding (z >= n)
        for (int z = max(z0, n); z < z1; ++z) {
            const long long o = ((long long)z * P + yo) * P + xo;
            const __nv_bfloat162 zz = __floats2bfloat162_rn(0.0f, 0.0f);
            Rhi2[o >> 1] = zz;
            Rlo2[o >> 1] = zz;
            Rhi2[(o + P) >> 1] = zz;
            Rlo2[(o + P) >> 1] = zz;
        }
        const int zl = min(z1, n);
        if (z0 >= zl) continue;   // block-uniform

        const bool v00 = xo < n && yo < n, v10 = xo + 1 < n && yo < n;
        const bool v01 = xo < n && yo + 1 < n, v11 = xo + 1 < n && yo + 1 < n;
        // loaded values: the own points, or at coordinate n the Neumann ghost
        const int gx0 = ghost_index(xo, n, neu), gx1 = ghost_index(xo + 1, n, neu);
        const int gy0 = ghost_index(yo, n, neu), gy1 = ghost_index(yo + 1, n, neu);
        const bool l00 = gx0 < n && gy0 < n, l10 = gx1 < n && gy0 < n;
        const bool l01 = gx0 < n && gy1 < n, l11 = gx1 < n && gy1 < n;
        const int o00 = gy0 * n + gx0, o10 = gy0 * n + gx1, o01 = gy1 * n + gx0, o11 = gy1 * n + gx1;
        float2 cxy[4];   // KIND 3: v_x + v_y of the own points
        if (KIND == 3) {
            const int xa = min(xo, n - 1), xb = min(xo + 1, n - 1);
            const int ya = n + min(yo, n - 1), yb = n + min(yo + 1, n - 1);
            cxy[0] = pair_add(__ldg(a.pot2 + xa), __ldg(a.pot2 + ya));
            cxy[1] = pair_add(__ldg(a.pot2 + xb), __ldg(a.pot2 + ya));
            cxy[2] = pair_add(__ldg(a.pot2 + xa), __ldg(a.pot2 + yb));
            cxy[3] = pair_add(__ldg(a.pot2 + xb), __ldg(a.pot2 + yb));
        }
        int hx, hy, hslot;
        if (hidx < kTX) {
            hx = X0 + hidx;
            hy = Y0 - 1;
            hslot = hidx + 2;
        } else if (hidx < 2 * kTX) {
            hx = X0 + hidx - kTX;
            hy = Y0 + kTY;
            hslot = (kTY + 1) * kSRow + hidx - kTX + 2;
        } else if (hidx < 2 * kTX + kTY) {
            hx = X0 - 1;
            hy = Y0 + hidx - 2 * kTX;
            hslot = (hidx - 2 * kTX + 1) * kSRow + 1;
        } else {
            hx = X0 + kTX;
            hy = Y0 + hidx - 2 * kTX - kTY;
            hslot = (hidx - 2 * kTX - kTY + 1) * kSRow + kTX + 2;
        }
        hx = ghost_index(hx, n, neu);
        hy = ghost_index(hy, n, neu);
        const bool hval = hlane && hx >= 0 && hx < n && hy >= 0 && hy < n;
        const long long hoff = hval ? (long long)hy * n + hx : 0;

        unsigned long long R[4], RH;
        auto load_plane = [&](int z) {
            const int zg = ghost_index(z, n, neu);
            const bool zin = zg >= 0 && zg < n;
            const unsigned long long *p = Ub + (long long)(zin ? zg : 0) * nn;
            R[0] = (zin && l00) ? __ldg(p + o00) : 0ull;
            R[1] = (zin && l10) ? __ldg(p + o10) : 0ull;
            R[2] = (zin && l01) ? __ldg(p + o01) : 0ull;
            R[3] = (zin && l11) ? __ldg(p + o11) : 0ull;
            RH = (zin && hval) ? __ldg(p + hoff) : 0ull;
        };
        auto minmax_own = [&]() {
            minmax_bits(R[0], v00, amin, amax);
            minmax_bits(R[1], v10, amin, amax);
            minmax_bits(R[2], v01, amin, amax);
            minmax_bits(R[3], v11, amin, amax);
        };
        auto f_at = [&](int z, int row) -> float4 {
            return __ldg(fdf4 + ((((long long)z * P + row) * P + xo) >> 1));
        };

        long long Fm[4], Fc[4], Fp[4];
        unsigned bm = 0, bc = 0, bh0 = 0;
        load_plane(z0 - 1);
        for (int i = 0; i < 4; ++i) Fm[i] = fx_of(R[i], E, bm);
        load_plane(z0);
        minmax_own();
        for (int i = 0; i < 4; ++i) Fc[i] = fx_of(R[i], E, bc);
        {
            long long *S = spl[z0 & 1];
            const long long H = fx_of(RH, E, bh0);
            *reinterpret_cast<longlong2 *>(S + s0) = make_longlong2(Fc[0], Fc[1]);
            *reinterpret_cast<longlong2 *>(S + s0 + kSRow) = make_longlong2(Fc[2], Fc[3]);
            if (hlane) S[hslot] = H;
        }
        load_plane(z0 + 1);
        float4 fa = f_at(z0, yo), fb = f_at(z0, yo + 1);
        int blk = __syncthreads_or((int)(bc | bh0));

        for (int z = z0; z < zl; ++z) {
            unsigned bp = 0, bhp = 0;
            for (int i = 0; i < 4; ++i) Fp[i] = fx_of(R[i], E, bp);
            const long long Hp = fx_of(RH, E, bhp);
            if (z + 1 < zl) minmax_own();
            {
                long long *S = spl[(z + 1) & 1];
                *reinterpret_cast<longlong2 *>(S + s0) = make_longlong2(Fp[0], Fp[1]);
                *reinterpret_cast<longlong2 *>(S + s0 + kSRow) = make_longlong2(Fp[2], Fp[3]);
                if (hlane) S[hslot] = Hp;
            }
            load_plane(z + 2);
            float4 fa_n = make_float4(0.f, 0.f, 0.f, 0.f), fb_n = fa_n;
            if (z + 1 < zl) {
                fa_n = f_at(z + 1, yo);
                fb_n = f_at(z + 1, yo + 1);
            }

            float rf[4];
            if (fx_ok && !(blk | bm | bp)) {
                const long long *S = spl[z & 1];
                const longlong2 up = *reinterpret_cast<const longlong2 *>(S + s0 - kSRow);
                const longlong2 dn = *reinterpret_cast<const longlong2 *>(S + s0 + 2 * kSRow);
                const unsigned long long l0 = S[s0 - 1], r0 = S[s0 + 2];
                const unsigned long long l1 = S[s0 + kSRow - 1], r1 = S[s0 + kSRow + 2];
                typedef unsigned long long u64;
                const u64 c0 = Fc[0], c1 = Fc[1], c2 = Fc[2], c3 = Fc[3];
                // 6u - (x- + x+ + y- + y+ + z- + z+), exact (wrap-free: |sum| < 2^62)
                const long long lap0 = (long long)(6ull * c0 - (((l0 + c1) + ((u64)up.x + c2)) + ((u64)Fm[0] + (u64)Fp[0])));
                const long long lap1 = (long long)(6ull * c1 - (((c0 + r0) + ((u64)up.y + c3)) + ((u64)Fm[1] + (u64)Fp[1])));
                const long long lap2 = (long long)(6ull * c2 - (((l1 + c3) + (c0 + (u64)dn.x)) + ((u64)Fm[2] + (u64)Fp[2])));
                const long long lap3 = (long long)(6ull * c3 - (((c2 + r1) + (c1 + (u64)dn.y)) + ((u64)Fm[3] + (u64)Fp[3])));
                if (KIND == 3) {
                    // per point lam + V = (v_x + v_y) + (lam + v_z), V in FP32 for beta
                    const float2 cz = __ldg(a.pot2 + 2 * n + z);
                    float dd[4];
                    float2 cv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cv[i] = pair_add(cxy[i], cz);
                    float2 d01, d23;
                    const float2 r01 = residual_pair2<KIND>(
                        Fc[0], Fc[1], lap0, lap1, make_float2(fa.x, fa.z), make_float2(fa.y, fa.w), scale, ih, il,
                        bh, bl, make_float2(cv[0].x, cv[1].x), make_float2(cv[0].y, cv[1].y),
                        make_float2(__fsub_rn(cv[0].x, lh), __fsub_rn(cv[1].x, lh)), &d01);
                    const float2 r23 = residual_pair2<KIND>(
                        Fc[2], Fc[3], lap2, lap3, make_float2(fb.x, fb.z), make_float2(fb.y, fb.w), scale, ih, il,
                        bh, bl, make_float2(cv[2].x, cv[3].x), make_float2(cv[2].y, cv[3].y),
                        make_float2(__fsub_rn(cv[2].x, lh), __fsub_rn(cv[3].x, lh)), &d23);
                    rf[0] = r01.x;
                    rf[1] = r01.y;
                    rf[2] = r23.x;
                    rf[3] = r23.y;
                    dd[0] = d01.x;
                    dd[1] = d01.y;
                    dd[2] = d23.x;
                    dd[3] = d23.y;
                    if (v00) { dmn = fminf(dmn, dd[0]); dmx = fmaxf(dmx, dd[0]); }
                    if (v10) { dmn = fminf(dmn, dd[1]); dmx = fmaxf(dmx, dd[1]); }
                    if (v01) { dmn = fminf(dmn, dd[2]); dmx = fmaxf(dmx, dd[2]); }
                    if (v11) { dmn = fminf(dmn, dd[3]); dmx = fmaxf(dmx, dd[3]); }
                } else {
                    const float2 r01 = residual_pair2<KIND>(Fc[0], Fc[1], lap0, lap1, make_float2(fa.x, fa.z),
                                                            make_float2(fa.y, fa.w), scale, ih, il, bh, bl,
                                                            f2_splat(lh), f2_splat(ll));
                    const float2 r23 = residual_pair2<KIND>(Fc[2], Fc[3], lap2, lap3, make_float2(fb.x, fb.z),
                                                            make_float2(fb.y, fb.w), scale, ih, il, bh, bl,
                                                            f2_splat(lh), f2_splat(ll));
                    rf[0] = r01.x;
                    rf[1] = r01.y;
                    rf[2] = r23.x;
                    rf[3] = r23.y;
                }
            } else {
                const double *pot = (KIND == 3) ? a.pot : nullptr;
                float dd[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                rf[0] = rf[1] = rf[2] = rf[3] = 0.0f;
                if (v00) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xo, yo, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[0] = e.x;
                    dd[0] = e.y;
                }
                if (v10) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xo + 1, yo, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[1] = e.x;
                    dd[1] = e.y;
                }
                if (v01) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xo, yo + 1, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[2] = e.x;
                    dd[2] = e.y;
                }
                if (v11) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xo + 1, yo + 1, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[3] = e.x;
                    dd[3] = e.y;
                }
                if (KIND == 3) {
                    if (v00) { dmn = fminf(dmn, dd[0]); dmx = fmaxf(dmx, dd[0]); }
                    if (v10) { dmn = fminf(dmn, dd[1]); dmx = fmaxf(dmx, dd[1]); }
                    if (v01) { dmn = fminf(dmn, dd[2]); dmx = fmaxf(dmx, dd[2]); }
                    if (v11) { dmn = fminf(dmn, dd[3]); dmx = fmaxf(dmx, dd[3]); }
                }
            }
            rf[0] = v00 ? rf[0] : 0.0f;
            rf[1] = v10 ? rf[1] : 0.0f;
            rf[2] = v01 ? rf[2] : 0.0f;
            rf[3] = v11 ? rf[3] : 0.0f;
            // sum (r 2^-k)^2 (FP32, Kahan over planes)
            const float q0 = __fmul_rn(rf[0], r2s), q1 = __fmul_rn(rf[1], r2s);
            const float q2 = __fmul_rn(rf[2], r2s), q3 = __fmul_rn(rf[3], r2s);
            const float sq = __fadd_rn(__fmaf_rn(q0, q0, __fmul_rn(q1, q1)), __fmaf_rn(q2, q2, __fmul_rn(q3, q3)));
            const float yk = __fsub_rn(sq, kc);
            const float tk = __fadd_rn(kr2, yk);
            kc = __fsub_rn(__fsub_rn(tk, kr2), yk);
            kr2 = tk;
            const long long o = ((long long)z * P + yo) * P + xo;
            store_split2(Rhi2, Rlo2, o >> 1, rf[0], rf[1]);
            store_split2(Rhi2, Rlo2, (o + P) >> 1, rf[2], rf[3]);

            blk = __syncthreads_or((int)(bp | bhp));
            for (int i = 0; i < 4; ++i) {
                Fm[i] = Fc[i];
                Fc[i] = Fp[i];
            }
            bm = bc;
            bc = bp;
            fa = fa_n;
            fb = fb_n;
        }
    }

    tile_partials<KIND>(a, kr2, kc, r2k, amin, amax, dmn, dmx);
}

// ---------------------------------------------------------------------------
// k_residual_mirror: k_residual_tiled for the reflection-split mode products.
//
// The inverse then contracts every axis through the reflection symmetry of the
// sine basis, S[n-1-j][k] = (-1)^k S[j][k]: the forward products take the
// sums a_j = r_j + r_{n-1-j} and differences b_j = r_j - r_{n-1-j} (j < n/2,
// the middle point of an odd n joining the sums), so this kernel writes the
// residual with
//   x   in split order: a_j at position j, b_j at position P/2 + j (zeros in
//       the padding of either half),
//   y,z in folded order: y < ceil(n/2) at row 2y, y >= ceil(n/2) at row
//       2(n-1-y)+1 (rows >= n are padding), so that the products' epilogues
//       find reflection partners in adjacent TMEM lanes.
// Same arithmetic as k_residual_tiled (fixed-point stencil with exponent E,
// float-pair nonlinear term, exact per-point path for flagged planes); the
// tile is two mirrored strips: lane l of a warp owns x = X0 + l (left strip)
// and its mirror n-1-X0-l (right strip), so both members of each pair are in
// one thread's registers. Shared rows hold the left strip (x = X0-1..X0+32 at
// columns 0..33) and the right strip in lane order (l' = -1..32 at columns
// 34..67, x = n-1-X0-l'). f is read as float pairs of the two strips
// (f_hi(x), f_lo(x), f_hi(x'), f_lo(x')) written by k_prep_split.
// ---------------------------------------------------------------------------
constexpr int kMHaloPerWarp = (4 * 32 + 4 * kTY) / 8;   // 192 halo values, 24 per warp

__device__ __forceinline__ int fold_index(int i, int n, int nsym) {
    return (i >= n) ? i : (i < nsym ? 2 * i : 2 * (n - 1 - i) + 1);
}

template <int KIND>
__global__ void __launch_bounds__(kTThreads, 2) k_residual_mirror(ResidualArgs a, int zchunk) {
    if (a.done != nullptr && *(volatile const int *)a.done) return;
    if (KIND != 3 && zero_start_partials(a)) return;
    __shared__ __align__(16) long long spl[2][kSRows * kSRow];
    const int n = a.n, P = a.P, H = a.P / 2;
    const int nsym = (n + 1) / 2, nanti = n / 2;
    const int E = *a.fx_e;
    const bool fx_ok = (E != 0);
    const float scale = __int_as_float(fx_ok ? ((E - 1075 - kFxG + 127) << 23) : 0);
    const float ih = __double2float_rn(a.inv_h2);
    const float il = __double2float_rn(a.inv_h2 - (double)ih);
    float bh = 1.0f, bl = 0.0f, lh = 0.0f, ll = 0.0f;
    if (KIND != 2) {
        bh = __double2float_rn(a.b);
        bl = __double2float_rn(a.b - (double)bh);
    }
    if (KIND == 0 || KIND == 3) {
        lh = __double2float_rn(a.lam);
        ll = __double2float_rn(a.lam - (double)lh);
    }
    const bool neu = (a.bc == QN_BC_NEUMANN);
    float dmn = INFINITY, dmx = -INFINITY;   // KIND 3: extremes of 3 b u^2 + V
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tiles_x = H / 32, tiles_y = P / kTY;
    const int nzc = (P + zchunk - 1) / zchunk;
    const long long items = (long long)tiles_x * tiles_y * nzc;
    const long long nn = (long long)n * n;
    const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(a.U);
    const float4 *fdf4 = reinterpret_cast<const float4 *>(a.fdf);
    const int r0s = (2 * warp + 1) * kSRow, r1s = r0s + kSRow;   // shared rows of the own points
    const bool hlane = lane < kMHaloPerWarp;
    const int hidx = warp * kMHaloPerWarp + lane;
    float kr2 = 0.0f, kc = 0.0f;
    unsigned long long amin = 0x7FFFFFFFFFFFFFFFull, amax = 0ull;
    const int r2k = *a.r2_exp;
    const float r2s = __int_as_float((127 - r2k) << 23);   // 2^-r2k

    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int tx = (int)(item % tiles_x);
        const long long q = item / tiles_x;
        const int ty = (int)(q % tiles_y);
        const int z0 = (int)(q / tiles_y) * zchunk;
        const int z1 = min(z0 + zchunk, P);
        const int X0 = tx * 32, Y0 = ty * kTY;
        const int xL = X0 + lane, xR = n - 1 - X0 - lane;
        const int y0 = Y0 + 2 * warp, y1 = y0 + 1;
        const int Fy0 = fold_index(y0, n, nsym), Fy1 = fold_index(y1, n, nsym);
        // zero planes of the padding (z >= n), both halves of both rows
        for (int z = max(z0, n); z < z1; ++z) {
            const long long o0 = ((long long)z * P + Fy0) * P, o1 = ((long long)z * P + Fy1) * P;
            const __nv_bfloat16 zb = __float2bfloat16_rn(0.0f);
            a.Rhi[o0 + xL] = zb;
            a.Rlo[o0 + xL] = zb;
            a.Rhi[o0 + H + xL] = zb;
            a.Rlo[o0 + H + xL] = zb;
            a.Rhi[o1 + xL] = zb;
            a.Rlo[o1 + xL] = zb;
            a.Rhi[o1 + H + xL] = zb;
            a.Rlo[o1 + H + xL] = zb;
        }
        const int zl = min(z1, n);
        if (z0 >= zl) continue;   // block-uniform

        // present: the value exists on the grid (else Dirichlet 0); own: this
        // thread evaluates the point (left: x <= middle; right: x > middle)
        const bool pL = xL < n, pR = xR >= 0, py0 = y0 < n, py1 = y1 < n;
        const bool oL = xL < nsym, oR = xL < nanti;
        const bool v0 = oL && py0, v1 = oR && py0, v2 = oL && py1, v3 = oR && py1;   // own points
        // rows read: the own rows, or at y = n the Neumann ghost row n-2
        // (x needs no ghost here: n > 64, so 0 < xR and xL < n)
        const int gy0 = ghost_index(y0, n, neu), gy1 = ghost_index(y1, n, neu);
        const bool ly0 = gy0 < n, ly1 = gy1 < n;
        float2 cxy[4];   // KIND 3: v_x + v_y of the own points
        if (KIND == 3) {
            const int xa = min(max(xL, 0), n - 1), xb = min(max(xR, 0), n - 1);
            const int ya = n + min(y0, n - 1), yb = n + min(y1, n - 1);
            cxy[0] = pair_add(__ldg(a.pot2 + xa), __ldg(a.pot2 + ya));
            cxy[1] = pair_add(__ldg(a.pot2 + xb), __ldg(a.pot2 + ya));
            cxy[2] = pair_add(__ldg(a.pot2 + xa), __ldg(a.pot2 + yb));
            cxy[3] = pair_add(__ldg(a.pot2 + xb), __ldg(a.pot2 + yb));
        }
        int hx, hy, hslot;
        {
            const int h = hidx;
            if (h < 128) {
                const int rr = (h < 64) ? 0 : (kTY + 1);
                const int g = h & 63;
                hy = (h < 64) ? Y0 - 1 : Y0 + kTY;
                if (g < 32) {
                    hx = X0 + g;
                    hslot = rr * kSRow + 1 + g;
                } else {
                    hx = n - 1 - X0 - (g - 32);
                    hslot = rr * kSRow + 35 + (g - 32);
                }
            } else {
                const int g = h - 128;
                const int rr = 1 + (g >> 2);
                hy = Y0 + rr - 1;
                const int w = g & 3;
                hx = (w == 0) ? X0 - 1 : (w == 1) ? X0 + 32 : (w == 2) ? n - X0 : n - 1 - X0 - 32;
                hslot = rr * kSRow + ((w == 0) ? 0 : (w == 1) ? 33 : (w == 2) ? 34 : 67);
            }
        }
        hx = ghost_index(hx, n, neu);
        hy = ghost_index(hy, n, neu);
        const bool hval = hlane && hx >= 0 && hx < n && hy >= 0 && hy < n;
        const long long hoff = hval ? (long long)hy * n + hx : 0;

        unsigned long long R[4], RH;
        auto load_plane = [&](int z) {
            const int zg = ghost_index(z, n, neu);
            const bool zin = zg >= 0 && zg < n;
            const unsigned long long *p = Ub + (long long)(zin ? zg : 0) * nn;
            R[0] = (zin && pL && ly0) ? __ldg(p + (long long)gy0 * n + xL) : 0ull;
            R[1] = (zin && pR && ly0) ? __ldg(p + (long long)gy0 * n + xR) : 0ull;
            R[2] = (zin && pL && ly1) ? __ldg(p + (long long)gy1 * n + xL) : 0ull;
            R[3] = (zin && pR && ly1) ? __ldg(p + (long long)gy1 * n + xR) : 0ull;
            RH = (zin && hval) ? __ldg(p + hoff) : 0ull;
        };
        auto minmax_own = [&]() {
            minmax_bits(R[0], v0, amin, amax);
            minmax_bits(R[1], v1, amin, amax);
            minmax_bits(R[2], v2, amin, amax);
            minmax_bits(R[3], v3, amin, amax);
        };
        auto f_at = [&](int z, int y) -> float4 {
            return __ldg(fdf4 + (((long long)z * P + y) * H + xL));
        };
        auto store_plane = [&](long long *S, const long long (&F)[4], long long Hv) {
            S[r0s + 1 + lane] = F[0];
            S[r0s + 35 + lane] = F[1];
            S[r1s + 1 + lane] = F[2];
            S[r1s + 35 + lane] = F[3];
            if (hlane) S[hslot] = Hv;
        };

        long long Fm[4], Fc[4], Fp[4];
        unsigned bm = 0, bc = 0, bh0 = 0;
        load_plane(z0 - 1);
        for (int i = 0; i < 4; ++i) Fm[i] = fx_of(R[i], E, bm);
        load_plane(z0);
        minmax_own();
        for (int i = 0; i < 4; ++i) Fc[i] = fx_of(R[i], E, bc);
        store_plane(spl[z0 & 1], Fc, fx_of(RH, E, bh0));
        load_plane(z0 + 1);
        float4 fa = f_at(z0, y0), fb = f_at(z0, y1);
        int blk = __syncthreads_or((int)(bc | bh0));

        for (int z = z0; z < zl; ++z) {
            unsigned bp = 0, bhp = 0;
            for (int i = 0; i < 4; ++i) Fp[i] = fx_of(R[i], E, bp);
            const long long Hp = fx_of(RH, E, bhp);
            if (z + 1 < zl) minmax_own();
            store_plane(spl[(z + 1) & 1], Fp, Hp);
            load_plane(z + 2);
            float4 fa_n = make_float4(0.f, 0.f, 0.f, 0.f), fb_n = fa_n;
            if (z + 1 < zl) {
                fa_n = f_at(z + 1, y0);
                fb_n = f_at(z + 1, y1);
            }

            float rf[4];
            if (fx_ok && !(blk | bm | bp)) {
                const long long *S = spl[z & 1];
                typedef unsigned long long u64;
                const u64 c0 = Fc[0], c1 = Fc[1], c2 = Fc[2], c3 = Fc[3];
                // left (x: cols l, l+2) and right (x-1: col 36+l, x+1: col 34+l) neighbours,
                // y-1 / y+1 from the rows above / below (own rows pair up)
                const u64 sl0 = (u64)S[r0s + lane] + (u64)S[r0s + lane + 2];
                const u64 sr0 = (u64)S[r0s + 36 + lane] + (u64)S[r0s + 34 + lane];
                const u64 sl1 = (u64)S[r1s + lane] + (u64)S[r1s + lane + 2];
                const u64 sr1 = (u64)S[r1s + 36 + lane] + (u64)S[r1s + 34 + lane];
                const u64 uL = (u64)S[r0s - kSRow + 1 + lane], uR = (u64)S[r0s - kSRow + 35 + lane];
                const u64 dL = (u64)S[r1s + kSRow + 1 + lane], dR = (u64)S[r1s + kSRow + 35 + lane];
                const long long lap0 = (long long)(6ull * c0 - ((sl0 + (uL + c2)) + ((u64)Fm[0] + (u64)Fp[0])));
                const long long lap1 = (long long)(6ull * c1 - ((sr0 + (uR + c3)) + ((u64)Fm[1] + (u64)Fp[1])));
                const long long lap2 = (long long)(6ull * c2 - ((sl1 + (c0 + dL)) + ((u64)Fm[2] + (u64)Fp[2])));
                const long long lap3 = (long long)(6ull * c3 - ((sr1 + (c1 + dR)) + ((u64)Fm[3] + (u64)Fp[3])));
                if (KIND == 3) {
                    // per point lam + V = (v_x + v_y) + (lam + v_z), V in FP32 for beta
                    const float2 cz = __ldg(a.pot2 + 2 * n + z);
                    float dd[4];
                    float2 cv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cv[i] = pair_add(cxy[i], cz);
                    float2 d01, d23;
                    const float2 r01 = residual_pair2<KIND>(
                        Fc[0], Fc[1], lap0, lap1, make_float2(fa.x, fa.z), make_float2(fa.y, fa.w), scale, ih, il,
                        bh, bl, make_float2(cv[0].x, cv[1].x), make_float2(cv[0].y, cv[1].y),
                        make_float2(__fsub_rn(cv[0].x, lh), __fsub_rn(cv[1].x, lh)), &d01);
                    const float2 r23 = residual_pair2<KIND>(
                        Fc[2], Fc[3], lap2, lap3, make_float2(fb.x, fb.z), make_float2(fb.y, fb.w), scale, ih, il,
                        bh, bl, make_float2(cv[2].x, cv[3].x), make_float2(cv[2].y, cv[3].y),
                        make_float2(__fsub_rn(cv[2].x, lh), __fsub_rn(cv[3].x, lh)), &d23);
                    rf[0] = r01.x;
                    rf[1] = r01.y;
                    rf[2] = r23.x;
                    rf[3] = r23.y;
                    dd[0] = d01.x;
                    dd[1] = d01.y;
                    dd[2] = d23.x;
                    dd[3] = d23.y;
                    if (v0) { dmn = fminf(dmn, dd[0]); dmx = fmaxf(dmx, dd[0]); }
                    if (v1) { dmn = fminf(dmn, dd[1]); dmx = fmaxf(dmx, dd[1]); }
                    if (v2) { dmn = fminf(dmn, dd[2]); dmx = fmaxf(dmx, dd[2]); }
                    if (v3) { dmn = fminf(dmn, dd[3]); dmx = fmaxf(dmx, dd[3]); }
                } else {
                    const float2 r01 = residual_pair2<KIND>(Fc[0], Fc[1], lap0, lap1, make_float2(fa.x, fa.z),
                                                            make_float2(fa.y, fa.w), scale, ih, il, bh, bl,
                                                            f2_splat(lh), f2_splat(ll));
                    const float2 r23 = residual_pair2<KIND>(Fc[2], Fc[3], lap2, lap3, make_float2(fb.x, fb.z),
                                                            make_float2(fb.y, fb.w), scale, ih, il, bh, bl,
                                                            f2_splat(lh), f2_splat(ll));
                    rf[0] = r01.x;
                    rf[1] = r01.y;
                    rf[2] = r23.x;
                    rf[3] = r23.y;
                }
            } else {
                const double *pot = (KIND == 3) ? a.pot : nullptr;
                float dd[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                rf[0] = rf[1] = rf[2] = rf[3] = 0.0f;
                if (v0) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xL, y0, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[0] = e.x;
                    dd[0] = e.y;
                }
                if (v1) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xR, y0, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[1] = e.x;
                    dd[1] = e.y;
                }
                if (v2) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xL, y1, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[2] = e.x;
                    dd[2] = e.y;
                }
                if (v3) {
                    const float2 e = residual_point_exact(a.U, a.f, n, xR, y1, z, a.inv_h2, a.lam, a.b, a.bc, pot);
                    rf[3] = e.x;
                    dd[3] = e.y;
                }
                if (KIND == 3) {
                    if (v0) { dmn = fminf(dmn, dd[0]); dmx = fmaxf(dmx, dd[0]); }
                    if (v1) { dmn = fminf(dmn, dd[1]); dmx = fmaxf(dmx, dd[1]); }
                    if (v2) { dmn = fminf(dmn, dd[2]); dmx = fmaxf(dmx, dd[2]); }
                    if (v3) { dmn = fminf(dmn, dd[3]); dmx = fmaxf(dmx, dd[3]); }
                }
            }
            rf[0] = v0 ? rf[0] : 0.0f;
            rf[1] = v1 ? rf[1] : 0.0f;
            rf[2] = v2 ? rf[2] : 0.0f;
            rf[3] = v3 ? rf[3] : 0.0f;
            // sum (r 2^-k)^2 (FP32, Kahan over planes)
            const float q0 = __fmul_rn(rf[0], r2s), q1 = __fmul_rn(rf[1], r2s);
            const float q2 = __fmul_rn(rf[2], r2s), q3 = __fmul_rn(rf[3], r2s);
            const float sq = __fadd_rn(__fmaf_rn(q0, q0, __fmul_rn(q1, q1)), __fmaf_rn(q2, q2, __fmul_rn(q3, q3)));
            const float yk = __fsub_rn(sq, kc);
            const float tk = __fadd_rn(kr2, yk);
            kc = __fsub_rn(__fsub_rn(tk, kr2), yk);
            kr2 = tk;
            // split-order output: sums at x, differences at P/2 + x, folded rows and plane
            const int Fz = fold_index(z, n, nsym);
            const long long o0 = ((long long)Fz * P + Fy0) * P, o1 = ((long long)Fz * P + Fy1) * P;
            // (rf of a point this thread does not own is 0; the middle point of an
            // odd n has no difference: its slot P/2 + n/2 stays 0)
            split_bf16(__fadd_rn(rf[0], rf[1]), a.Rhi[o0 + xL], a.Rlo[o0 + xL]);
            split_bf16(v1 ? __fsub_rn(rf[0], rf[1]) : 0.0f, a.Rhi[o0 + H + xL], a.Rlo[o0 + H + xL]);
            split_bf16(__fadd_rn(rf[2], rf[3]), a.Rhi[o1 + xL], a.Rlo[o1 + xL]);
            split_bf16(v3 ? __fsub_rn(rf[2], rf[3]) : 0.0f, a.Rhi[o1 + H + xL], a.Rlo[o1 + H + xL]);

            blk = __syncthreads_or((int)(bp | bhp));
            for (int i = 0; i < 4; ++i) {
                Fm[i] = Fc[i];
                Fc[i] = Fp[i];
            }
            bm = bc;
            bc = bp;
            fa = fa_n;
            fb = fb_n;
        }
    }

    tile_partials<KIND>(a, kr2, kc, r2k, amin, amax, dmn, dmx);
}

// ---------------------------------------------------------------------------
// k_fused_res_fwd: the residual of the split solve and the first forward
// reflection-split mode product (the contraction of x, Sec. 4.1 eq.
// fin_inverse, applied to F(U) of Sec. 4 eq. F_u) in one kernel. The residual
// is formed in shared memory as the product's A operand, instead of being
// written to HBM as split planes and read back by the product.
//
// A product tile is 128 rows m = (z_f, y_f) of one folded plane (64 spatial
// rows y and their mirrors n-1-y) times the whole split x axis. One CTA takes
// both halves of a tile (the sums a_j against the even modes, the differences
// b_j against the odd modes: two accumulators of H FP32 columns, all 512 TMEM
// columns), so every point's residual is formed once. Per pipeline stage
// (32 positions j of the split axis):
//   warp 0 lane 0   TMA of the B tiles: the even and odd rows of the forward
//                   matrix [P][H], hi and lo, 32 x H each, 64-byte swizzle
//   warp 1          allocates TMEM; lane 0 issues tcgen05.mma per half:
//                   a_hi b_hi + a_hi b_lo + a_lo b_hi (FP32 accumulators)
//   warps 2..17     the residual: warps 2..9 the even rows (y ascending),
//                   10..17 the odd rows (the mirrors, y descending), eight
//                   consecutive spatial rows per warp; lane l owns the points
//                   x = j0 + l and n-1-j0-l. The fixed-point values march in y
//                   (the rows above and below stay in registers, the loads of
//                   the next row are issued one row ahead); x neighbours come
//                   from the adjacent lanes by shuffles and the four strip ends
//                   from one extra load; the z - 1 and z + 1 values are loaded
//                   and converted per point. The arithmetic is that of
//                   k_residual_mirror (exact int64 stencil, float-pair
//                   nonlinear term, FP32 result; a row that touches a value
//                   above the fixed-point range takes the exact per-point
//                   path). Sums and differences are split into BF16 hi + lo
//                   and stored in the swizzled layout a TMA load would write.
//                   After a tile's last stage the same warps run the first
//                   product's epilogue (the butterflies of y, as the
//                   EPI_STORE_BFLY epilogue of k_modeprod_tc).
// Dirichlet data without a potential (KIND 0-2); per-CTA partial records as
// the other tiled residuals. Every mbarrier wait is bounded (2 s of
// %globaltimer): on expiry the kernel sets the error word and the other roles
// stop; the TMA producer waits (bounded) for its armed stages and the MMA
// issuer for its last commit before TMEM is freed.
// ---------------------------------------------------------------------------
constexpr int kFzThreads = 576;
constexpr int kFzWorkers = 16;
constexpr uint32_t kFzATile = 128u * 64u;   // 128 rows x 32 BF16
constexpr uint32_t kFzBTile = 256u * 64u;   // up to 256 rows x 32 BF16
constexpr uint32_t kFzStage = 4u * kFzATile + 4u * kFzBTile;
constexpr int kFzStages = 2;
constexpr uint32_t kFzSmem = 1024u + kFzStages * kFzStage + 256u;
constexpr unsigned long long kFzTimeoutNs = 2000000000ull;
static_assert(kFzThreads == 64 + 32 * kFzWorkers, "roles");

__device__ __forceinline__ bool fz_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = ptx::globaltimer();
    while (true) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (ptx::globaltimer() - t0 > kFzTimeoutNs) {
            *abort_flag = 1;
            atomicExch(err, QN_ETIMEOUT);
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag (draining after an abort).
__device__ __forceinline__ void fz_drain(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(bar, parity))
        if (ptx::globaltimer() - t0 > kFzTimeoutNs) return;
}

// Byte offset of element (row, col) of a 32-column BF16 tile in the 64-byte
// swizzle (16-byte chunk c of row r at chunk c ^ ((r / 2) mod 4)): the layout
// of a TMA load with CU_TENSOR_MAP_SWIZZLE_64B into a 512-byte aligned tile.
__device__ __forceinline__ uint32_t sw64_off(int row, int col) {
    return (uint32_t)row * 64u + (((((uint32_t)col) >> 3) ^ (((uint32_t)row >> 1) & 3u)) << 4) +
           (((uint32_t)col & 7u) << 1);
}

__device__ __forceinline__ void st_shared_b16(uint32_t addr, __nv_bfloat16 v) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(__bfloat16_as_ushort(v)) : "memory");
}

// Loads of one march row issued a row ahead: planes z - 1 and z + 1 at both
// points, the strip-end value (lanes 0, 1, 30, 31) and the f pairs.
struct FzAhead {
    unsigned long long ml, mr, pl, pr, h;
    float4 f;
};

// 96 registers: the limit for 18 warps per CTA (five of them share one of the SM's four
// 16384-register sub-partitions)
template <int KIND>
__global__ void __maxnreg__(96) k_fused_res_fwd(ResidualArgs a, FusedFwd ff) {
    static_assert(KIND >= 0 && KIND <= 2, "Dirichlet data without a potential");
    if (a.done != nullptr && *(volatile const int *)a.done) return;
    const int n = a.n, P = a.P, H = P / 2;
    const int nsym = (n + 1) / 2, nanti = n / 2;
    const long long Mtot = (long long)P * P;
    const int ntiles = (int)(Mtot / 128);
    const int KB = H / 32;

    extern __shared__ uint8_t fz_raw[];
    const uint32_t raw = ptx::smem_u32(fz_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t ctrl = base + (uint32_t)kFzStages * kFzStage;
    auto full_bar = [&](int s) { return ctrl + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return ctrl + 16u + 8u * (uint32_t)s; };
    const uint32_t tfull_bar = ctrl + 32u, tempty_bar = ctrl + 40u, mma_done_bar = ctrl + 48u;
    const uint32_t tmem_slot = ctrl + 56u;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(fz_raw + (ctrl + 60u - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr unsigned kAll = 0xffffffffu;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFzStages; ++s) {
            ptx::mbar_init(full_bar(s), 1 + kFzWorkers);   // the TMA arrival + one per worker warp
            ptx::mbar_init(empty_bar(s), 1);
        }
        ptx::mbar_init(tfull_bar, 1);
        ptx::mbar_init(tempty_bar, kFzWorkers);
        ptx::mbar_init(mma_done_bar, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
        ptx::prefetch_tensormap(ff.b_hi);
        ptx::prefetch_tensormap(ff.b_lo);
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, 512);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(fz_raw + (tmem_slot - raw));

    // partial sums of the worker threads (the identity elsewhere)
    float kr2 = 0.0f, kc = 0.0f;
    unsigned long long amin = 0x7FFFFFFFFFFFFFFFull, amax = 0ull;
    const int r2k = *a.r2_exp;

    if (warp == 0 && lane == 0) {
        // ------------------------------ TMA of B ----------------------------------
        uint32_t armed_parity[kFzStages];
        uint32_t armed_mask = 0;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        const uint32_t tx = 4u * (uint32_t)H * 64u;
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            for (int kb = 0; kb < KB; ++kb) {
                if (!fz_wait(empty_bar(s), ph ^ 1u, abort_flag, ff.err)) {
                    ok = false;
                    break;
                }
                const uint32_t sb = base + (uint32_t)s * kFzStage + 4u * kFzATile;
                ptx::mbar_arrive_expect_tx(full_bar(s), tx);
                ptx::tma_load_2d(sb, ff.b_hi, full_bar(s), kb * 32, 0);
                ptx::tma_load_2d(sb + kFzBTile, ff.b_lo, full_bar(s), kb * 32, 0);
                ptx::tma_load_2d(sb + 2u * kFzBTile, ff.b_hi, full_bar(s), kb * 32, H);
                ptx::tma_load_2d(sb + 3u * kFzBTile, ff.b_lo, full_bar(s), kb * 32, H);
                armed_parity[s] = ph;
                armed_mask |= 1u << s;
                if (++s == kFzStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        if (!ok) {
            for (int i = 0; i < kFzStages; ++i)
                if (armed_mask & (1u << i)) fz_drain(full_bar(i), armed_parity[i]);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------ MMA issuer --------------------------------
        int s = 0;
        uint32_t ph = 0, aph = 0;
        bool ok = true;
        const uint32_t idesc = ptx::idesc_bf16_f32(128, (uint32_t)H);
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            if (!fz_wait(tempty_bar, aph ^ 1u, abort_flag, ff.err)) break;
            ptx::tc_fence_after();
            for (int kb = 0; kb < KB; ++kb) {
                if (!fz_wait(full_bar(s), ph, abort_flag, ff.err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t st = base + (uint32_t)s * kFzStage;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 32u;
                    const uint64_t sa_hi = ptx::smem_desc_kmajor(st + ko, 64, 4);
                    const uint64_t sa_lo = ptx::smem_desc_kmajor(st + kFzATile + ko, 64, 4);
                    const uint64_t sd_hi = ptx::smem_desc_kmajor(st + 2u * kFzATile + ko, 64, 4);
                    const uint64_t sd_lo = ptx::smem_desc_kmajor(st + 3u * kFzATile + ko, 64, 4);
                    const uint32_t sb = st + 4u * kFzATile + ko;
                    const uint64_t be_hi = ptx::smem_desc_kmajor(sb, 64, 4);
                    const uint64_t be_lo = ptx::smem_desc_kmajor(sb + kFzBTile, 64, 4);
                    const uint64_t bo_hi = ptx::smem_desc_kmajor(sb + 2u * kFzBTile, 64, 4);
                    const uint64_t bo_lo = ptx::smem_desc_kmajor(sb + 3u * kFzBTile, 64, 4);
                    const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                    ptx::mma_bf16(tmem_base, sa_hi, be_hi, idesc, first);
                    ptx::mma_bf16(tmem_base, sa_hi, be_lo, idesc, 1u);
                    ptx::mma_bf16(tmem_base, sa_lo, be_hi, idesc, 1u);
                    ptx::mma_bf16(tmem_base + (uint32_t)H, sd_hi, bo_hi, idesc, first);
                    ptx::mma_bf16(tmem_base + (uint32_t)H, sd_hi, bo_lo, idesc, 1u);
                    ptx::mma_bf16(tmem_base + (uint32_t)H, sd_lo, bo_hi, idesc, 1u);
                }
                ptx::mma_commit(empty_bar(s));
                if (++s == kFzStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            ptx::mma_commit(tfull_bar);
            aph ^= 1u;
        }
        ptx::mma_commit(mma_done_bar);
        fz_drain(mma_done_bar, 0);
    } else if (warp >= 2) {
        // ------------------------- residual workers / epilogue ---------------------
        const int wk = warp - 2;
        const int grp = wk >> 3, wi = wk & 7;   // grp 0: even rows, 1: odd rows (mirrors)
        const int q = warp & 3, part = wk >> 2;  // epilogue: TMEM lane quadrant, column range
        const int E = *a.fx_e;
        const bool fx_ok = (E != 0);
        const float scale = __int_as_float(fx_ok ? ((E - 1075 - kFxG + 127) << 23) : 0);
        const float ih = __double2float_rn(a.inv_h2);
        const float il = __double2float_rn(a.inv_h2 - (double)ih);
        float bh = 1.0f, bl = 0.0f, lh = 0.0f, ll = 0.0f;
        if (KIND != 2) {
            bh = __double2float_rn(a.b);
            bl = __double2float_rn(a.b - (double)bh);
        }
        if (KIND == 0) {
            lh = __double2float_rn(a.lam);
            ll = __double2float_rn(a.lam - (double)lh);
        }
        const float r2s = __int_as_float((127 - r2k) << 23);   // 2^-r2k
        const long long nn = (long long)n * n;
        const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(a.U);
        const float4 *fdf4 = reinterpret_cast<const float4 *>(a.fdf);
        int s = 0;
        uint32_t ph = 0, aph = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            const int m0 = t * 128;
            const int zf = m0 / P, yf0 = m0 % P;
            const int zi = zf >> 1;
            const bool zval = (zf & 1) ? (zi < nanti) : (zi < nsym);
            const int z = (zf & 1) ? n - 1 - zi : zi;
            const int i0 = (yf0 >> 1) + 8 * wi;            // march row k: index i0 + k of its group
            const int ybase = grp ? n - 1 - i0 : i0;       // spatial y of march row k: ybase + ydir k
            const int ydir = grp ? -1 : 1;
            const int own_lim = grp ? nanti : nsym;        // row k is a grid row iff i0 + k < own_lim
            const unsigned long long *pz = Ub + (long long)(zval ? z : 0) * nn;
            const bool zm_in = zval && z > 0, zp_in = zval && z + 1 < n;
            for (int kb = 0; kb < KB; ++kb) {
                const bool ready = fz_wait(empty_bar(s), ph ^ 1u, abort_flag, ff.err);
                if (!__all_sync(kAll, ready)) {
                    ok = false;
                    break;
                }
                const uint32_t st = base + (uint32_t)s * kFzStage;
                const int j0 = kb * 32;
                const int xL = j0 + lane, xR = n - 1 - xL;   // 0 <= xR, xL < n (n > H)
                const bool oL = xL < nsym, oR = xL < nanti;
                // strip ends: lane 0 x = j0 - 1, lane 1 x = n - j0, lane 30 x = j0 + 32, lane 31 x = n - 33 - j0
                const int hx = (lane == 0) ? j0 - 1 : (lane == 1) ? n - j0 : (lane == 30) ? j0 + 32 : (lane == 31) ? n - 33 - j0 : -1;
                const bool hin = hx >= 0 && hx < n;
                if (zval) {
                    auto load_c = [&](int k, unsigned long long &vl, unsigned long long &vr) {
                        const int y = ybase + ydir * k;
                        const bool yin = y >= 0 && y < n;
                        const unsigned long long *p = pz + (long long)(yin ? y : 0) * n;
                        vl = yin ? __ldg(p + xL) : 0ull;
                        vr = yin ? __ldg(p + xR) : 0ull;
                    };
                    auto load_ahead = [&](int k, FzAhead &L) {
                        const int y = ybase + ydir * k;
                        const bool yin = y >= 0 && y < n;
                        const long long yo = (long long)(yin ? y : 0) * n;
                        const unsigned long long *p = pz + yo;
                        L.ml = (yin && zm_in) ? __ldg(p - nn + xL) : 0ull;
                        L.mr = (yin && zm_in) ? __ldg(p - nn + xR) : 0ull;
                        L.pl = (yin && zp_in) ? __ldg(p + nn + xL) : 0ull;
                        L.pr = (yin && zp_in) ? __ldg(p + nn + xR) : 0ull;
                        L.h = (yin && hin) ? __ldg(p + hx) : 0ull;
                        L.f = yin ? __ldg(fdf4 + (((long long)z * P + y) * H + xL)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    };
                    unsigned long long rl, rr, nxl, nxr;
                    unsigned bp = 0, bc = 0;
                    load_c(-1, rl, rr);
                    long long pL = fx_of(rl, E, bp), pR = fx_of(rr, E, bp);
                    load_c(0, rl, rr);
                    long long cL = fx_of(rl, E, bc), cR = fx_of(rr, E, bc);
                    unsigned long long cbl = rl, cbr = rr;   // bit patterns of the current row (min / max)
                    load_c(1, nxl, nxr);
                    FzAhead ah;
                    load_ahead(0, ah);
#pragma unroll 1
                    for (int k = 0; k < 8; ++k) {
                        unsigned bn = 0, bz = 0;
                        const long long nL = fx_of(nxl, E, bn), nR = fx_of(nxr, E, bn);
                        const unsigned long long nbl = nxl, nbr = nxr;
                        const long long zmL = fx_of(ah.ml, E, bz), zmR = fx_of(ah.mr, E, bz);
                        const long long zpL = fx_of(ah.pl, E, bz), zpR = fx_of(ah.pr, E, bz);
                        const long long hv = fx_of(ah.h, E, bz);
                        const float4 fq = ah.f;
                        if (k + 2 <= 8) load_c(k + 2, nxl, nxr);
                        if (k + 1 < 8) load_ahead(k + 1, ah);

                        // x neighbours from the adjacent lanes, the strip ends from lanes 0, 1, 30, 31
                        long long xLm = __shfl_up_sync(kAll, cL, 1), xLp = __shfl_down_sync(kAll, cL, 1);
                        long long xRm = __shfl_down_sync(kAll, cR, 1), xRp = __shfl_up_sync(kAll, cR, 1);
                        const long long hdn = __shfl_down_sync(kAll, hv, 1), hup = __shfl_up_sync(kAll, hv, 1);
                        if (lane == 0) {
                            xLm = hv;
                            xRp = hdn;
                        }
                        if (lane == 31) {
                            xLp = hup;
                            xRm = hv;
                        }
                        const bool row_bad = __any_sync(kAll, (bp | bc | bn | bz) != 0u) || !fx_ok;
                        const int y = ybase + ydir * k;
                        const bool rown = (i0 + k) < own_lim;
                        const bool vL = rown && oL, vR = rown && oR;
                        float rL = 0.0f, rR = 0.0f;
                        if (!row_bad) {
                            typedef unsigned long long u64;
                            // 6u - (x- + x+ + y- + y+ + z- + z+), exact (wrap-free: |sum| < 2^62)
                            const long long lapL = (long long)(6ull * (u64)cL - ((((u64)xLm + (u64)xLp) + ((u64)pL + (u64)nL)) + ((u64)zmL + (u64)zpL)));
                            const long long lapR = (long long)(6ull * (u64)cR - ((((u64)xRm + (u64)xRp) + ((u64)pR + (u64)nR)) + ((u64)zmR + (u64)zpR)));
                            const float2 r01 = residual_pair2<KIND>(cL, cR, lapL, lapR, make_float2(fq.x, fq.z),
                                                                    make_float2(fq.y, fq.w), scale, ih, il, bh, bl,
                                                                    f2_splat(lh), f2_splat(ll));
                            rL = r01.x;
                            rR = r01.y;
                        } else {
                            if (vL) rL = residual_point_exact(a.U, a.f, n, xL, y, z, a.inv_h2, a.lam, a.b, a.bc, nullptr).x;
                            if (vR) rR = residual_point_exact(a.U, a.f, n, xR, y, z, a.inv_h2, a.lam, a.b, a.bc, nullptr).x;
                        }
                        rL = vL ? rL : 0.0f;
                        rR = vR ? rR : 0.0f;
                        minmax_bits(cbl, vL, amin, amax);
                        minmax_bits(cbr, vR, amin, amax);
                        // sum (r 2^-k)^2 (FP32, Kahan)
                        const float q0 = __fmul_rn(rL, r2s), q1 = __fmul_rn(rR, r2s);
                        const float sq = __fmaf_rn(q0, q0, __fmul_rn(q1, q1));
                        const float yk = __fsub_rn(sq, kc);
                        const float tk = __fadd_rn(kr2, yk);
                        kc = __fsub_rn(__fsub_rn(tk, kr2), yk);
                        kr2 = tk;
                        // the sum a_j and the difference b_j (none for the middle point of an odd n)
                        __nv_bfloat16 a_h, a_l, d_h, d_l;
                        split_bf16(__fadd_rn(rL, rR), a_h, a_l);
                        split_bf16(vR ? __fsub_rn(rL, rR) : 0.0f, d_h, d_l);
                        const uint32_t o = st + sw64_off(2 * (8 * wi + k) + grp, lane);
                        st_shared_b16(o, a_h);
                        st_shared_b16(o + kFzATile, a_l);
                        st_shared_b16(o + 2u * kFzATile, d_h);
                        st_shared_b16(o + 3u * kFzATile, d_l);
                        pL = cL;
                        pR = cR;
                        cL = nL;
                        cR = nR;
                        bp = bc;
                        bc = bn;
                        cbl = nbl;
                        cbr = nbr;
                    }
                } else {
                    // a padding plane: zero rows
                    const __nv_bfloat16 zb = __float2bfloat16_rn(0.0f);
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t o = st + sw64_off(2 * (8 * wi + k) + grp, lane);
                        st_shared_b16(o, zb);
                        st_shared_b16(o + kFzATile, zb);
                        st_shared_b16(o + 2u * kFzATile, zb);
                        st_shared_b16(o + 3u * kFzATile, zb);
                    }
                }
                // the generic-proxy stores become visible to the tensor core's async proxy
                ptx::fence_proxy_async();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(full_bar(s));
                if (++s == kFzStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            // ---- epilogue of the tile: butterflies of y into the next product's layout ----
            const bool ready = fz_wait(tfull_bar, aph, abort_flag, ff.err);
            if (!__all_sync(kAll, ready)) break;
            ptx::tc_fence_after();
            {
                const int m = m0 + q * 32 + lane;
                const int F = m % P, slow = m / P, i2 = F >> 1;
                const bool odd = (F & 1) != 0;
                const bool valid = odd ? (i2 < nanti) : (i2 < nsym);
                const long long obase = (long long)slow * P + (odd ? H + i2 : i2);
                const int cols = H / 2;   // 2H accumulator columns over four warps per quadrant
                const int cbeg = part * cols;
                for (int c = cbeg; c < cbeg + cols; c += 16) {
                    uint32_t r[16];
                    ptx::tmem_ld_32x32b_x16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)c, r);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float v = __uint_as_float(r[i]);
                        const float pv = __shfl_xor_sync(kAll, v, 1);
                        const float o = valid ? (odd ? pv - v : v + pv) : 0.0f;
                        __nv_bfloat16 oh, ol;
                        split_bf16(o, oh, ol);
                        const long long idx = (long long)(c + i) * Mtot + obase;
                        ff.out_hi[idx] = oh;
                        ff.out_lo[idx] = ol;
                    }
                }
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(tempty_bar);
            aph ^= 1u;
        }
    }

    tile_partials<KIND>(a, kr2, kc, r2k, amin, amax, INFINITY, -INFINITY);
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, 512);
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
    if (a.pot != nullptr)
        k_residual<DIM, SPLIT, FAST, 3, WF2><<<grid, 256, 0, s>>>(a);
    else if (a.lam != 0.0)
        k_residual<DIM, SPLIT, FAST, 0, WF2><<<grid, 256, 0, s>>>(a);
    else if (a.b != 1.0)
        k_residual<DIM, SPLIT, FAST, 1, WF2><<<grid, 256, 0, s>>>(a);
    else
        k_residual<DIM, SPLIT, FAST, 2, WF2><<<grid, 256, 0, s>>>(a);
}

template <int DIM, bool SPLIT, bool FAST>
static void launch_res3(const ResidualArgs &a, int grid, cudaStream_t s) {
    // the scaled FP32 norm needs RMS(f), known once sum f^2 has been taken:
    // the fast form never sums f^2
    if (!FAST && a.want_f2)
        launch_res4<DIM, SPLIT, false, true>(a, grid, s);
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
    if (a.hval != nullptr) return launch_residual_sem(a, grid, s);
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

template <int KIND>
static int tiled_blocks_per_sm() {
    static int cached = 0;   // per process: every device it runs on is a GB300
    if (cached == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_residual_tiled<KIND>, kTThreads, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        cached = nb;
    }
    return cached;
}

template <int KIND>
static int launch_tiled_kind(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s) {
    int dev = 0, sms = 0;
    QN_CUDA(cudaGetDevice(&dev));
    QN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long items = (long long)(a.P / kTX) * (a.P / kTY) * ((a.P + zchunk - 1) / zchunk);
    long long g = (long long)tiled_blocks_per_sm<KIND>() * sms;
    if (g > max_grid) g = max_grid;
    if (g > items) g = items;
    if (g < 1) g = 1;
    k_residual_tiled<KIND><<<(int)g, kTThreads, 0, s>>>(a, zchunk);
    QN_CUDA(cudaGetLastError());
    *grid_used = (int)g;
    return QN_OK;
}

template <int KIND>
static int mirror_blocks_per_sm() {
    static int cached = 0;
    if (cached == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_residual_mirror<KIND>, kTThreads, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        cached = nb;
    }
    return cached;
}

template <int KIND>
static int launch_mirror_kind(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s) {
    int dev = 0, sms = 0;
    QN_CUDA(cudaGetDevice(&dev));
    QN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long items = (long long)(a.P / 64) * (a.P / kTY) * ((a.P + zchunk - 1) / zchunk);
    long long g = (long long)mirror_blocks_per_sm<KIND>() * sms;
    if (g > max_grid) g = max_grid;
    if (g > items) g = items;
    if (g < 1) g = 1;
    k_residual_mirror<KIND><<<(int)g, kTThreads, 0, s>>>(a, zchunk);
    QN_CUDA(cudaGetLastError());
    *grid_used = (int)g;
    return QN_OK;
}

int launch_residual_mirror(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s) {
    if (a.dim != 3 || a.Rhi == nullptr || a.fdf == nullptr || a.fx_e == nullptr || a.P % 128 != 0 ||
        zchunk < 1) {
        set_error("launch_residual_mirror: needs a 3-D split residual, P a multiple of 128, the f copy");
        return QN_EINVAL;
    }
    if (a.pot != nullptr) {
        if (a.pot2 == nullptr || a.umax_scan == nullptr) {
            set_error("launch_residual_mirror: a potential needs its FP32-pair tables and the max|U| slot");
            return QN_EINVAL;
        }
        return launch_mirror_kind<3>(a, max_grid, zchunk, grid_used, s);
    }
    if (a.lam != 0.0) return launch_mirror_kind<0>(a, max_grid, zchunk, grid_used, s);
    if (a.b != 1.0) return launch_mirror_kind<1>(a, max_grid, zchunk, grid_used, s);
    return launch_mirror_kind<2>(a, max_grid, zchunk, grid_used, s);
}

int fused_set_attributes() {
    QN_CUDA(cudaFuncSetAttribute(k_fused_res_fwd<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFzSmem));
    QN_CUDA(cudaFuncSetAttribute(k_fused_res_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFzSmem));
    QN_CUDA(cudaFuncSetAttribute(k_fused_res_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFzSmem));
    return QN_OK;
}

int launch_fused_residual_fwd(const ResidualArgs &a, const FusedFwd &ff, int *grid_used, cudaStream_t s) {
    const int H = a.P / 2;
    if (a.dim != 3 || a.P % 128 != 0 || H > 256 || a.n <= H || a.fdf == nullptr || a.fx_e == nullptr ||
        a.r2_exp == nullptr || a.pot != nullptr || a.bc != QN_BC_DIRICHLET || ff.b_hi == nullptr ||
        ff.b_lo == nullptr || ff.out_hi == nullptr || ff.out_lo == nullptr || ff.err == nullptr || ff.num_sms < 1) {
        set_error("launch_fused_residual_fwd: needs a 3-D split solve with P a multiple of 128, P <= 512, "
                  "Dirichlet data, no potential, the f copy and the forward matrix maps");
        return QN_EINVAL;
    }
    const int ntiles = (a.P / 128) * a.P;
    const int grid = ntiles < ff.num_sms ? ntiles : ff.num_sms;
    *grid_used = grid;
    if (a.lam != 0.0)
        k_fused_res_fwd<0><<<grid, kFzThreads, kFzSmem, s>>>(a, ff);
    else if (a.b != 1.0)
        k_fused_res_fwd<1><<<grid, kFzThreads, kFzSmem, s>>>(a, ff);
    else
        k_fused_res_fwd<2><<<grid, kFzThreads, kFzSmem, s>>>(a, ff);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_residual_tiled(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s) {
    if (a.dim != 3 || a.Rhi == nullptr || a.fdf == nullptr || a.fx_e == nullptr || a.P % kTX != 0 ||
        zchunk < 1) {
        set_error("launch_residual_tiled: needs a 3-D split residual with the FP32-pair copy of f");
        return QN_EINVAL;
    }
    if (a.pot != nullptr) {
        if (a.pot2 == nullptr || a.umax_scan == nullptr) {
            set_error("launch_residual_tiled: a potential needs its FP32-pair tables and the max|U| slot");
            return QN_EINVAL;
        }
        return launch_tiled_kind<3>(a, max_grid, zchunk, grid_used, s);
    }
    if (a.lam != 0.0) return launch_tiled_kind<0>(a, max_grid, zchunk, grid_used, s);
    if (a.b != 1.0) return launch_tiled_kind<1>(a, max_grid, zchunk, grid_used, s);
    return launch_tiled_kind<2>(a, max_grid, zchunk, grid_used, s);
}

int launch_prep_split(const double *U, const double *f, int n, int P, float2 *fdf, __nv_bfloat16 *Rhi,
                      __nv_bfloat16 *Rlo, double *partials, int nparts, DevState *st, bool mirror, cudaStream_t s) {
    const int g = 2 * nparts;   // (the partials buffer holds 8 records per SM, nparts <= 4 per SM)
    if (mirror)
        k_prep_split<true><<<g, 256, 0, s>>>(U, f, n, P, fdf, Rhi, Rlo, partials, st);
    else
        k_prep_split<false><<<g, 256, 0, s>>>(U, f, n, P, fdf, Rhi, Rlo, partials, st);
    QN_CUDA(cudaGetLastError());
    k_prep_split_finish<<<1, 256, 0, s>>>(partials, g, st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_umax(const double *U, long long N, DevState *st, int grid, cudaStream_t s) {
    const int vec16 = ((reinterpret_cast<uintptr_t>(U) & 15u) == 0) ? 1 : 0;
    k_umax<<<grid, 256, 0, s>>>(U, N, vec16, st);
    QN_CUDA(cudaGetLastError());
    k_umax_finish<<<1, 32, 0, s>>>(st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_finalize(const double *partials, int nparts, DevState *st, qn_stats *hist,
                        int hist_cap, double b, double lam, int update_state, int use_saved_fnorm,
                        int mode, cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nparts, st, hist, hist_cap, b, lam, update_state,
                                 use_saved_fnorm, mode);
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
constexpr int kNoAllocStateDoubles = 20;              // DevState (<= 160 B)
constexpr int kNoAllocStatsDoubles = 8;               // one qn_stats (56 B)
constexpr int kNoAllocDoubles = 4 * kNoAllocMaxBlocks + kNoAllocStateDoubles + kNoAllocStatsDoubles;
static_assert(sizeof(DevState) <= kNoAllocStateDoubles * sizeof(double), "DevState too large");
static_assert(sizeof(qn_stats) <= kNoAllocStatsDoubles * sizeof(double), "qn_stats too large");

// 4096 partial-sum slots + solver state + one statistics record: 33 KB.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
// device address of the array per device ordinal, with the unique ID of the
// context it was looked up in: after a device reset the runtime creates a new
// primary context (a new ID) and reloads the module, so the lookup is redone
struct NoAllocSlot {
    double *ptr;
    unsigned long long ctx_id;
};
NoAllocSlot g_noalloc_slot[128] = {};

typedef int (*PfnCtxGetCurrent)(void **);
typedef int (*PfnCtxGetId)(void *, unsigned long long *);

// Unique ID of the calling thread's current context (driver entry points,
// resolved once; the library links only the runtime).
int current_ctx_id(unsigned long long *id) {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *p1 = nullptr, *p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess || !p1 || !p2) {
            set_error("qn_residual_noalloc: cuCtxGetCurrent / cuCtxGetId unavailable from the driver");
            return QN_ECUDA;
        }
        get_current = reinterpret_cast<PfnCtxGetCurrent>(p1);
        get_id = reinterpret_cast<PfnCtxGetId>(p2);
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, id) != 0) {
        set_error("qn_residual_noalloc: no current CUDA context");
        return QN_ECUDA;
    }
    return QN_OK;
}

// Device address of g_noalloc_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress: once per device, and again whenever that device's
// context has changed since (a cudaDeviceReset in between).
int noalloc_scratch(double **out) {
    int dev = 0;
    QN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) {
        set_error("qn_residual_noalloc: device ordinal %d out of range", dev);
        return QN_EINVAL;
    }
    QN_CUDA(cudaSetDevice(dev));   // makes the device's primary context current (initialising it)
    unsigned long long id = 0;
    int rc = current_ctx_id(&id);
    if (rc != QN_OK) return rc;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot &slot = g_noalloc_slot[dev];
    if (slot.ptr == nullptr || slot.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            slot.ptr = nullptr;
            return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        }
        slot.ptr = static_cast<double *>(p);
        slot.ctx_id = id;
    }
    *out = slot.ptr;
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
    ResidualArgs a{};
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
    rc = launch_finalize(partials, grid, state, stats, 1, b, lam, 0, 0, 0, s);
    if (rc != QN_OK) return rc;
    QN_CUDA(cudaMemcpyAsync(st, stats, sizeof(qn_stats), cudaMemcpyDeviceToHost, s));
    QN_CUDA(cudaStreamSynchronize(s));
    return QN_OK;
}
