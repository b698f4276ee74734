// Nonlinear eigenproblem (Sec. 4.4 eqs. Eigenvalue_p, system_qusi, system_normal;
// Sec. 6.3 Example 2):
//   -Lap u + f(u) = lambda u,   f(u) = lam u + b u^3 + V u,   ||u|| = 1,
// lambda unknown. One iteration on the device, with no host synchronisation.
// The iterate arrives unnormalised (U~ = U - step delta from the previous
// update, or the caller's start); its normalisation U = s U~, s = 1/||U~||,
// is folded into the two residual passes:
//
//   k_eig_pass1      lin = A_h U~ + (lam + V) U~ (FP64, kept for pass 2) and the
//                    sums E1 = <U~, lin>, E4 = b <U~^3, U~>, Q = <U~, U~>
//   k_eig_finalize1  s = 1/sqrt(Q), and the Rayleigh quotient of U = s U~:
//                    lambda_n = <A U + f(U), U> / <U, U> = (E1 + s^2 E4) / Q
//   k_eig_pass2      U = s U~ (written back), F = s lin + b U^3 - lambda_n U into
//                    the inverse's input (FP64, or BF16 hi/lo planes in natural
//                    or reflection-split order), ||F||^2, and the extremes of
//                    lam + 3 b U^2 + V
//   k_finalize       (qn_residual.cu, eigen mode) beta_n = mid-range - lambda_n,
//                    the shift, the stop test ||F|| / |lambda_n|
//   mode products    U~ = U - step (A_h + beta_n I)^{-1} F (update epilogue)
//
// <V, W> is the lumped-mass product h^dim sum w V W, with w the product of the
// 1-D trapezoid weights (1/2 at a Neumann face node, else 1): A_h is
// self-adjoint in it, so F is orthogonal to U. All reductions are per-block
// partials summed in a fixed order (deterministic: graph replay is bitwise
// the same as plain launches).
#include <math.h>

#include "qn_df.cuh"
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

// Block sums of a, b and mn (used as a third sum); result valid in thread 0.
__device__ Sum4 block_sum3(Sum4 v) {
    __shared__ Sum4 sh3[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.a += __shfl_xor_sync(0xffffffffu, v.a, o);
        v.b += __shfl_xor_sync(0xffffffffu, v.b, o);
        v.mn += __shfl_xor_sync(0xffffffffu, v.mn, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh3[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh3[l] : Sum4{0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.a += __shfl_xor_sync(0xffffffffu, v.a, o);
            v.b += __shfl_xor_sync(0xffffffffu, v.b, o);
            v.mn += __shfl_xor_sync(0xffffffffu, v.mn, o);
        }
    }
    return v;
}

// Block reduction of NS float-pair sums (and, with MM, an FP32 min / max) with no FP64 warp
// instruction: GB300 issues those at about 16 cycles per warp, which for a few hundred
// blocks per launch adds up. Thread 0 receives {s0, s1, s2 or min, max} in FP64.
__device__ __forceinline__ float2 shfl_pair(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

template <int NS, bool MM>
__device__ Sum4 block_pair_red(float2 s0, float2 s1, float2 s2, float mn, float mx) {
    __shared__ float2 shs[3][32];
    __shared__ float shm[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 = pair_add(s0, shfl_pair(s0, o));
        if (NS > 1) s1 = pair_add(s1, shfl_pair(s1, o));
        if (NS > 2) s2 = pair_add(s2, shfl_pair(s2, o));
        if (MM) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        shs[0][w] = s0;
        shs[1][w] = s1;
        shs[2][w] = s2;
        shm[0][w] = mn;
        shm[1][w] = mx;
    }
    __syncthreads();
    Sum4 r{0.0, 0.0, 0.0, 0.0};
    if (threadIdx.x == 0) {
        const float2 z = make_float2(0.0f, 0.0f);
        float2 a = z, b = z, c = z;
        float m0 = INFINITY, m1 = -INFINITY;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a = pair_add(a, shs[0][i]);
            if (NS > 1) b = pair_add(b, shs[1][i]);
            if (NS > 2) c = pair_add(c, shs[2][i]);
            if (MM) {
                m0 = fminf(m0, shm[0][i]);
                m1 = fmaxf(m1, shm[1][i]);
            }
        }
        r.a = (double)a.x + (double)a.y;
        r.b = (double)b.x + (double)b.y;
        r.mn = (NS > 2) ? (double)c.x + (double)c.y : (double)m0;
        r.mx = (double)m1;
    }
    return r;
}

__device__ __forceinline__ bool state_done(const DevState *st) { return *(volatile const int *)&st->done != 0; }

// 1-D trapezoid weight of node i (the lumped mass without h).
template <bool NEU>
__device__ __forceinline__ double tw(int i, int n) {
    return (NEU && (i == 0 || i == n - 1)) ? 0.5 : 1.0;
}

// Node coordinates of flat index c (x fastest).
template <int DIM>
__device__ __forceinline__ void node_xyz(long long c, int n, int &x, int &y, int &z) {
    const long long r = c / n;
    x = (int)(c - r * n);
    if (DIM == 3) {
        const long long q = r / n;
        y = (int)(r - q * n);
        z = (int)q;
    } else {
        y = (int)r;
        z = 0;
    }
}

// lin = A_h U + (lam + V) U at every node (U unnormalised), with the per-block
// sums of w U lin, b w U^4 and w U^2.
// vrow: with a potential, lam + v_y(y) (+ v_z(z)) per (y, z) row (n^(DIM-1) entries), so a
// node adds only v_x(x); without one, nullptr (the coefficient is lam).
template <int DIM, bool NEU>
__global__ void __launch_bounds__(256) k_eig_pass1(const double *__restrict__ U, double *__restrict__ lin, int n,
                                                   double inv_h2, double lam, double b,
                                                   const double *__restrict__ pot, const double *__restrict__ vrow,
                                                   double *__restrict__ partials, const DevState *st) {
    if (state_done(st)) return;
    const long long nn = (long long)n * n;
    const long long N = (DIM == 3) ? nn * n : nn;
    Sum4 acc{0.0, 0.0, 0.0, 0.0};   // a: sum w u lin, b: sum w u^4, mn: sum w u^2
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += stride) {
        const long long row = c / n;   // (z, y) row
        const int x = (int)(c - row * n);
        const int y = (DIM == 3) ? (int)(row % n) : (int)row;
        const int z = (DIM == 3) ? (int)(row / n) : 0;
        const double u = __ldg(U + c);
        double nbv[2 * DIM];
        nbv[0] = (x > 0) ? __ldg(U + c - 1) : (NEU ? __ldg(U + c + 1) : 0.0);
        nbv[1] = (x < n - 1) ? __ldg(U + c + 1) : (NEU ? __ldg(U + c - 1) : 0.0);
        nbv[2] = (y > 0) ? __ldg(U + c - n) : (NEU ? __ldg(U + c + n) : 0.0);
        nbv[3] = (y < n - 1) ? __ldg(U + c + n) : (NEU ? __ldg(U + c - n) : 0.0);
        if (DIM == 3) {
            nbv[4] = (z > 0) ? __ldg(U + c - nn) : (NEU ? __ldg(U + c + nn) : 0.0);
            nbv[5] = (z < n - 1) ? __ldg(U + c + nn) : (NEU ? __ldg(U + c - nn) : 0.0);
        }
        const double lap = stencil_fixed<DIM>(u, nbv);          // exact 2 DIM u - sum(nb)
        const double cv = (pot != nullptr) ? __ldg(vrow + row) + __ldg(pot + x) : lam;
        const double lv = fma(lap, inv_h2, cv * u);
        lin[c] = lv;
        const double wu = NEU ? tw<NEU>(x, n) * tw<NEU>(y, n) * ((DIM == 3) ? tw<NEU>(z, n) : 1.0) * u : u;
        const double wu2 = wu * u;
        acc.a = fma(wu, lv, acc.a);
        acc.b = fma(wu2, u * u, acc.b);
        acc.mn += wu2;
    }
    acc = block_sum3(acc);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = b * acc.b;
        p[2] = acc.mn;
        p[3] = 0.0;
    }
}

// s = 1/||U~|| and lambda_n of U = s U~; the scale |lambda_n| of the stop test.
__global__ void __launch_bounds__(256) k_eig_finalize1(const double *partials, int nparts, double hd, DevState *st) {
    if (state_done(st)) return;
    Sum4 acc{0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        acc.a += partials[4 * i + 0];
        acc.b += partials[4 * i + 1];
        acc.mn += partials[4 * i + 2];
    }
    acc = block_sum3(acc);
    if (threadIdx.x != 0) return;
    const double E1 = acc.a, E4 = acc.b, Q = acc.mn;
    const double s2 = 1.0 / (hd * Q);                  // ||s U~||^2 = s^2 h^d Q = 1
    const double sc = sqrt(s2);
    st->eig_scale = sc;
    const double lam_n = (E1 + s2 * E4) / Q;           // <A U + f(U), U> / <U, U> at U = s U~
    st->eig_lambda = lam_n;
    const float sh = __double2float_rn(sc), lh = __double2float_rn(lam_n);
    st->eig_scale2 = make_float2(sh, __double2float_rn(sc - (double)sh));
    st->eig_lambda2 = make_float2(lh, __double2float_rn(lam_n - (double)lh));
    st->f_norm = fabs(lam_n);                          // |lambda_n| ||U||, ||U|| = 1
}

// One node of pass 2: U = s U~ written back; returns F = s lin + b U^3 - lambda_n U;
// accumulates w F^2 and the extremes of lam + 3 b U^2 + V (FP32, from the FP32 potential
// tables pot32: they only set beta_n).
template <int DIM, bool NEU>
__device__ __forceinline__ double eig_point(double *__restrict__ U, const double *__restrict__ lin, long long c,
                                            int x, int y, int z, int n, double sc, double lam_n, float lamf, double b,
                                            const float *__restrict__ pot32, double &sff, float &dmn, float &dmx,
                                            unsigned long long &umax) {
    const double u = sc * U[c];
    U[c] = u;
    const unsigned long long ab = abs_bits(u);
    umax = ab > umax ? ab : umax;
    const double u2 = u * u;
    const double F = fma(sc, __ldg(lin + c), fma(b * u2, u, -lam_n * u));
    const double w = NEU ? tw<NEU>(x, n) * tw<NEU>(y, n) * ((DIM == 3) ? tw<NEU>(z, n) : 1.0) : 1.0;
    sff = fma(w * F, F, sff);
    float cv = lamf;
    if (pot32 != nullptr) {
        cv += __ldg(pot32 + x) + __ldg(pot32 + n + y);
        if (DIM == 3) cv += __ldg(pot32 + 2 * n + z);
    }
    const float d = __fmaf_rn(3.0f * (float)b, d2f_rn(u2), cv);
    dmn = fminf(dmn, d);
    dmx = fmaxf(dmx, d);
    return F;
}

// U = s U~, F into the inverse's input, per-block sum of w F^2 (times h^dim) and the
// extremes of lam + 3 b U^2 + V. OUT 0: FP64 n^DIM array. OUT 1: BF16 hi/lo planes on
// the padded P^DIM grid in natural order. OUT 2 (3-D, P a multiple of 128): the
// reflection-split order of k_residual_mirror (x: sums at i, differences at P/2 + i;
// y, z folded).
template <int DIM, int OUT, bool NEU>
__global__ void __launch_bounds__(256) k_eig_pass2(double *__restrict__ U, const double *__restrict__ lin, int n,
                                                   int P, double hd, float lam, double b,
                                                   const float *__restrict__ pot, double *__restrict__ R64,
                                                   __nv_bfloat16 *__restrict__ Rhi, __nv_bfloat16 *__restrict__ Rlo,
                                                   double *__restrict__ partials, const DevState *st,
                                                   unsigned long long *umax_out) {
    if (state_done(st)) return;
    const double sc = st->eig_scale, lam_n = st->eig_lambda;
    double sff = 0.0;
    float dmn = INFINITY, dmx = -INFINITY;
    unsigned long long umax = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (OUT == 0) {
        const long long N = (DIM == 3) ? (long long)n * n * n : (long long)n * n;
        for (long long c = t0; c < N; c += stride) {
            int x, y, z;
            node_xyz<DIM>(c, n, x, y, z);
            R64[c] = eig_point<DIM, NEU>(U, lin, c, x, y, z, n, sc, lam_n, lam, b, pot, sff, dmn, dmx, umax);
        }
    } else if (OUT == 1) {
        const long long NP = (DIM == 3) ? (long long)P * P * P : (long long)P * P;
        for (long long o = t0; o < NP; o += stride) {
            const long long r = o / P;
            const int x = (int)(o - r * P);
            const int y = (DIM == 3) ? (int)(r % P) : (int)r;
            const int z = (DIM == 3) ? (int)(r / P) : 0;
            float f = 0.0f;
            if (x < n && y < n && z < n) {
                const long long c = ((long long)z * n + y) * n + x;
                f = d2f_rn(eig_point<DIM, NEU>(U, lin, c, x, y, z, n, sc, lam_n, lam, b, pot, sff, dmn, dmx, umax));
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(f);
            Rhi[o] = hi;
            Rlo[o] = __float2bfloat16_rn(f - __bfloat162float(hi));
        }
    } else {
        // folded row (rz, ry), position i < P/2 of the split x axis; folded index
        // r -> spatial: even r -> r/2, odd r -> n-1-(r-1)/2, r >= n padding
        const int H = P / 2, nsym = (n + 1) / 2, nanti = n / 2;
        const long long items = (long long)P * P * H;
        for (long long t = t0; t < items; t += stride) {
            const long long row = t / H;
            const int i = (int)(t - row * H);
            const int ry = (int)(row % P), rz = (int)(row / P);
            float fa = 0.0f, fb = 0.0f;
            if (ry < n && rz < n && i < nsym) {
                const int y = (ry & 1) ? n - 1 - (ry >> 1) : (ry >> 1);
                const int z = (rz & 1) ? n - 1 - (rz >> 1) : (rz >> 1);
                const long long cb = ((long long)z * n + y) * n;
                fa = d2f_rn(eig_point<DIM, NEU>(U, lin, cb + i, i, y, z, n, sc, lam_n, lam, b, pot, sff, dmn, dmx, umax));
                if (i < nanti) {
                    const int j = n - 1 - i;
                    const float f2 =
                        d2f_rn(eig_point<DIM, NEU>(U, lin, cb + j, j, y, z, n, sc, lam_n, lam, b, pot, sff, dmn, dmx, umax));
                    fb = __fsub_rn(fa, f2);
                    fa = __fadd_rn(fa, f2);
                }
            }
            const long long o = row * P + i;
            const __nv_bfloat16 ha = __float2bfloat16_rn(fa), hb = __float2bfloat16_rn(fb);
            Rhi[o] = ha;
            Rlo[o] = __float2bfloat16_rn(fa - __bfloat162float(ha));
            Rhi[o + H] = hb;
            Rlo[o + H] = __float2bfloat16_rn(fb - __bfloat162float(hb));
        }
    }
    Sum4 acc{hd * sff, 0.0, (double)dmn, (double)dmx};
    acc = block_sum4(acc);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = 0.0;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
    if (umax_out != nullptr) {   // max|U| of the normalised iterate (fixed-point exponent of the next pass 1)
        unsigned long long m = umax;
        __shared__ unsigned long long shm2[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
            m = v > m ? v : m;
        }
        if ((threadIdx.x & 31) == 0) shm2[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = shm2[i] > m ? shm2[i] : m;
            atomicMax(umax_out, m);
        }
    }
}

// ---- float-pair forms of the two passes (iterations >= 1) ------------------------------------
// The same arithmetic with no FP64 operation per node in pass 1 and one (U = s U~) in
// pass 2: the stencil 2 DIM u - sum(nb) is an exact int64 sum of fixed-point values in units
// of 2^(E - 1075 - kFxG), E from max|U| of the previous iterate (DevState::fx_e, set by the
// stop-test finaliser from pass 2's block maxima); everything else is in float pairs
// (~48 significant bits). A node whose stencil reads a value beyond E takes the FP64 path.

__device__ __forceinline__ double pair_to_double(float2 a) { return (double)a.x + (double)a.y; }

// FP64 path of one pass-1 node (values beyond the fixed-point range): lin and u as pairs.
template <int DIM, bool NEU>
static __device__ __noinline__ float2 pass1_node_exact(const double *U, long long c, int x, int y, int z, int n,
                                                       double inv_h2, double cv, float2 &up) {
    const long long nn = (long long)n * n;
    const double u = U[c];
    double nbv[2 * DIM];
    nbv[0] = (x > 0) ? U[c - 1] : (NEU ? U[c + 1] : 0.0);
    nbv[1] = (x < n - 1) ? U[c + 1] : (NEU ? U[c - 1] : 0.0);
    nbv[2] = (y > 0) ? U[c - n] : (NEU ? U[c + n] : 0.0);
    nbv[3] = (y < n - 1) ? U[c + n] : (NEU ? U[c - n] : 0.0);
    if (DIM == 3) {
        nbv[4] = (z > 0) ? U[c - nn] : (NEU ? U[c + nn] : 0.0);
        nbv[5] = (z < n - 1) ? U[c + nn] : (NEU ? U[c - nn] : 0.0);
    }
    const double lv = fma(stencil_fixed<DIM>(u, nbv), inv_h2, cv * u);
    up = f_pair_slow(u);
    return f_pair_slow(lv);
}

// vrow2 / pot2: lam + v_y (+ v_z) per row and v_x per column as float pairs (nullptr: no
// potential, the coefficient is lam2).
template <int DIM, bool NEU>
__global__ void __launch_bounds__(256) k_eig_pass1_df(const double *__restrict__ U, float2 *__restrict__ lin, int n,
                                                      double inv_h2, double lam, float2 lam2, double b,
                                                      const double *__restrict__ pot, const double *__restrict__ vrow,
                                                      const float2 *__restrict__ pot2, const float2 *__restrict__ vrow2,
                                                      double *__restrict__ partials, const DevState *st) {
    if (state_done(st)) return;
    const int E = st->fx_e;
    const float scale = __int_as_float(E != 0 ? ((E - 1075 - kFxG + 127) << 23) : 0);
    const float ih = __double2float_rn(inv_h2), il = __double2float_rn(inv_h2 - (double)ih);
    const float2 ih2 = make_float2(ih, il);
    const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(U);
    const long long nn = (long long)n * n;
    const long long N = (DIM == 3) ? nn * n : nn;
    float2 e1 = make_float2(0.f, 0.f), e4 = e1, q = e1;
    // one warp per (y, z) row, lanes along x (one division per row, none per node)
    const int lane = threadIdx.x & 31;
    const int rows = (int)(N / n);
    const int wstride = gridDim.x * (blockDim.x >> 5);
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += wstride) {
      const int y = (DIM == 3) ? row % n : row;
      const int z = (DIM == 3) ? row / n : 0;
      for (int x = lane; x < n; x += 32) {
        const long long c = (long long)row * n + x;
        unsigned long long bn[2 * DIM];
        const unsigned long long bu = __ldg(Ub + c);
        bn[0] = (x > 0) ? __ldg(Ub + c - 1) : (NEU ? __ldg(Ub + c + 1) : 0ull);
        bn[1] = (x < n - 1) ? __ldg(Ub + c + 1) : (NEU ? __ldg(Ub + c - 1) : 0ull);
        bn[2] = (y > 0) ? __ldg(Ub + c - n) : (NEU ? __ldg(Ub + c + n) : 0ull);
        bn[3] = (y < n - 1) ? __ldg(Ub + c + n) : (NEU ? __ldg(Ub + c - n) : 0ull);
        if (DIM == 3) {
            bn[4] = (z > 0) ? __ldg(Ub + c - nn) : (NEU ? __ldg(Ub + c + nn) : 0ull);
            bn[5] = (z < n - 1) ? __ldg(Ub + c + nn) : (NEU ? __ldg(Ub + c - nn) : 0ull);
        }
        unsigned bad = (E == 0) ? 1u : 0u;
        const long long fu = fx_of(bu, E, bad);
        unsigned long long snb = 0ull;
#pragma unroll
        for (int i = 0; i < 2 * DIM; ++i) snb += (unsigned long long)fx_of(bn[i], E, bad);
        float2 lv, up;
        if (!bad) {
            const long long lapfx = (long long)((unsigned long long)(2 * DIM) * (unsigned long long)fu - snb);
            float2 ph, pl;   // the stencil sum and u in one packed FP32x2 chain (the same results)
            fx_to_pair2(lapfx, fu, scale, ph, pl);
            const float lh = ph.x, ll = pl.x, uh = ph.y, ul = pl.y;
            up = make_float2(uh, ul);
            const float2 cv = (pot != nullptr) ? pair_add(__ldg(vrow2 + row), __ldg(pot2 + x)) : lam2;
            lv = pair_add(pair_mul(make_float2(lh, ll), ih2), pair_mul(cv, up));
        } else {
            const double cv = (pot != nullptr) ? __ldg(vrow + row) + __ldg(pot + x) : lam;
            lv = pass1_node_exact<DIM, NEU>(U, c, x, y, z, n, inv_h2, cv, up);
        }
        lin[c] = lv;
        float2 wu = up;
        if (NEU) {   // trapezoid weights are powers of two: exact on both halves
            const float w = (float)(tw<NEU>(x, n) * tw<NEU>(y, n) * ((DIM == 3) ? tw<NEU>(z, n) : 1.0));
            wu = make_float2(wu.x * w, wu.y * w);
        }
        const float2 wu2 = pair_mul(wu, up);
        e1 = pair_add(e1, pair_mul(wu, lv));
        e4 = pair_add(e4, pair_mul(wu2, pair_mul(up, up)));
        q = pair_add(q, wu2);
      }
    }
    Sum4 acc{pair_to_double(e1), pair_to_double(e4), pair_to_double(q), 0.0};
    acc = block_sum3(acc);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = b * acc.b;
        p[2] = acc.mn;
        p[3] = 0.0;
    }
}

// ---- tiled pass 1 (3-D, float pairs) ------------------------------------------------------
// The arithmetic of k_eig_pass1_df with each value converted to fixed point once: a block
// owns a 32 x 8 (x, y) tile of a run of z planes, one warp per y row, and walks z. The
// tile's plane z and its x / y halo sit in shared memory (double-buffered), the z - 1 and
// z + 1 values of the thread's own column in registers; the next plane's loads are in
// flight while the current one is evaluated. A node takes the FP64 path when a value of
// plane z (anywhere in the tile: one block-wide flag) or of its own column at z - 1, z + 1
// lies beyond the fixed-point exponent.
constexpr int kP1W = 32, kP1H = 8;
constexpr int kP1SW = kP1W + 2, kP1SH = kP1H + 2;
constexpr int kP1Halo = 2 * kP1W + 2 * kP1H;   // 80 halo values per plane (no corners)

__device__ __forceinline__ int ghost_of(int i, int n, bool neu) {
    return neu ? (i == -1 ? 1 : (i == n ? n - 2 : i)) : i;
}

// bit pattern of node (z, y, x), the Neumann ghost rule applied, 0 off the grid (Dirichlet)
template <bool NEU>
__device__ __forceinline__ unsigned long long ld_node3(const unsigned long long *__restrict__ Ub, int z, int y,
                                                       int x, int n) {
    z = ghost_of(z, n, NEU);
    y = ghost_of(y, n, NEU);
    x = ghost_of(x, n, NEU);
    const bool in = (unsigned)z < (unsigned)n && (unsigned)y < (unsigned)n && (unsigned)x < (unsigned)n;
    return in ? __ldg(Ub + ((long long)z * n + y) * n + x) : 0ull;
}

template <bool NEU>
__global__ void __launch_bounds__(256, 3) k_eig_pass1_tiled(const double *__restrict__ U, float2 *__restrict__ lin,
                                                            int n, int zchunk, double inv_h2, double lam,
                                                            float2 lam2, double b, const double *__restrict__ pot,
                                                            const double *__restrict__ vrow,
                                                            const float2 *__restrict__ pot2,
                                                            const float2 *__restrict__ vrow2,
                                                            double *__restrict__ partials, const DevState *st) {
    if (state_done(st)) return;
    __shared__ long long sp[2][kP1SH][kP1SW];
    const int E = st->fx_e;
    const float scale = __int_as_float(E != 0 ? ((E - 1075 - kFxG + 127) << 23) : 0);
    const float ih = __double2float_rn(inv_h2), il = __double2float_rn(inv_h2 - (double)ih);
    const float2 ih2 = make_float2(ih, il);
    const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(U);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    // this thread's halo slot: the rows above / below the tile, then the columns left / right
    const bool halo = t < kP1Halo;
    int hr, hc;
    if (t < kP1W) {
        hr = 0;
        hc = t + 1;
    } else if (t < 2 * kP1W) {
        hr = kP1SH - 1;
        hc = t - kP1W + 1;
    } else if (t < 2 * kP1W + kP1H) {
        hr = t - 2 * kP1W + 1;
        hc = 0;
    } else {
        hr = t - 2 * kP1W - kP1H + 1;
        hc = kP1SW - 1;
    }
    if (!halo) hr = hc = 0;
    const int tiles_x = (n + kP1W - 1) / kP1W, tiles_y = (n + kP1H - 1) / kP1H;
    const int nzc = (n + zchunk - 1) / zchunk;
    const long long items = (long long)tiles_x * tiles_y * nzc;
    float2 e1 = make_float2(0.f, 0.f), e4 = e1, q = e1;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int tx = (int)(item % tiles_x);
        const long long rest = item / tiles_x;
        const int ty = (int)(rest % tiles_y);
        const int z0 = (int)(rest / tiles_y) * zchunk;
        const int z1 = min(z0 + zchunk, n);
        const int x = tx * kP1W + lane, y = ty * kP1H + w;
        const int hx = tx * kP1W + hc - 1, hy = ty * kP1H + hr - 1;
        const bool own = x < n && y < n;
        unsigned bm = (E == 0) ? 1u : 0u, bc = bm, bh = bm;   // bad flags: own z-1, own z, plane z (local)
        long long fmv = fx_of(ld_node3<NEU>(Ub, z0 - 1, y, x, n), E, bm);
        long long fc = fx_of(ld_node3<NEU>(Ub, z0, y, x, n), E, bc);
        sp[0][w + 1][lane + 1] = fc;
        if (halo) sp[0][hr][hc] = fx_of(ld_node3<NEU>(Ub, z0, hy, hx, n), E, bh);
        bh |= bc;
        unsigned long long nO = ld_node3<NEU>(Ub, z0 + 1, y, x, n);
        unsigned long long nH = halo ? ld_node3<NEU>(Ub, z0 + 1, hy, hx, n) : 0ull;
        int buf = 0;
        for (int z = z0; z < z1; ++z, buf ^= 1) {
            const bool plane_bad = __syncthreads_or((int)bh) != 0;   // plane z is in sp[buf]
            unsigned bp = (E == 0) ? 1u : 0u;
            const long long fp = fx_of(nO, E, bp);
            bh = bp;
            sp[buf ^ 1][w + 1][lane + 1] = fp;
            if (halo) sp[buf ^ 1][hr][hc] = fx_of(nH, E, bh);
            if (z + 1 < z1) {   // prefetch plane z + 2
                nO = ld_node3<NEU>(Ub, z + 2, y, x, n);
                if (halo) nH = ld_node3<NEU>(Ub, z + 2, hy, hx, n);
            }
            if (own) {
                const long long c = ((long long)z * n + y) * n + x;
                float2 lv, up;
                if (!(plane_bad || bm || bp)) {
                    const long long lapfx = 6 * fc - sp[buf][w + 1][lane] - sp[buf][w + 1][lane + 2] -
                                            sp[buf][w][lane + 1] - sp[buf][w + 2][lane + 1] - fmv - fp;
                    float2 ph, pl;   // the stencil sum and u in one packed FP32x2 chain (the same results)
                    fx_to_pair2(lapfx, fc, scale, ph, pl);
                    const float lh = ph.x, ll = pl.x, uh = ph.y, ul = pl.y;
                    up = make_float2(uh, ul);
                    const float2 cv = (pot != nullptr) ? pair_add(__ldg(vrow2 + (long long)z * n + y), __ldg(pot2 + x))
                                                       : lam2;
                    lv = pair_add(pair_mul(make_float2(lh, ll), ih2), pair_mul(cv, up));
                } else {
                    const double cv = (pot != nullptr) ? __ldg(vrow + (long long)z * n + y) + __ldg(pot + x) : lam;
                    lv = pass1_node_exact<3, NEU>(U, c, x, y, z, n, inv_h2, cv, up);
                }
                lin[c] = lv;
                float2 wu = up;
                if (NEU) {   // trapezoid weights are powers of two: exact on both halves
                    const float wt = ((x == 0 || x == n - 1) ? 0.5f : 1.0f) * ((y == 0 || y == n - 1) ? 0.5f : 1.0f) *
                                     ((z == 0 || z == n - 1) ? 0.5f : 1.0f);
                    wu = make_float2(wu.x * wt, wu.y * wt);
                }
                const float2 wu2 = pair_mul(wu, up);
                e1 = pair_add(e1, pair_mul(wu, lv));
                e4 = pair_add(e4, pair_mul(wu2, pair_mul(up, up)));
                q = pair_add(q, wu2);
            }
            fmv = fc;
            bm = bc;
            fc = fp;
            bc = bp;
        }
        __syncthreads();   // the next item's first plane reuses sp[0]
    }
    const Sum4 acc = block_pair_red<3, false>(e1, e4, q, 0.0f, 0.0f);
    if (threadIdx.x == 0) {
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = b * acc.b;
        p[2] = acc.mn;
        p[3] = 0.0;
    }
}

// One node of pass 2 in float pairs; U = s U~ written back (the one FP64 multiply).
template <int DIM, bool NEU>
__device__ __forceinline__ float eig_point_df(double *__restrict__ U, const float2 *__restrict__ lin, long long c,
                                              int x, int y, int z, int n, double sc, float2 sc2, float2 lamn2,
                                              float2 b2, float lamf, float b3f, const float *__restrict__ pot32,
                                              float &sk, float &kc, float &dmn, float &dmx,
                                              unsigned long long &umax) {
    const double u = sc * U[c];
    U[c] = u;
    const unsigned long long ab = abs_bits(u);
    umax = ab > umax ? ab : umax;
    const float2 up = f_pair(u, nullptr);
    const float2 u2 = pair_mul(up, up);
    const float2 bu3 = pair_mul(b2, pair_mul(u2, up));
    const float2 F = pair_add(pair_add(pair_mul(sc2, __ldg(lin + c)), bu3), pair_neg(pair_mul(lamn2, up)));
    const float Ff = __fadd_rn(F.x, F.y);
    float wF = Ff;
    if (NEU) wF = Ff * (float)(tw<NEU>(x, n) * tw<NEU>(y, n) * ((DIM == 3) ? tw<NEU>(z, n) : 1.0));
    const float yk = __fsub_rn(__fmul_rn(wF, Ff), kc);   // Kahan sum of w F^2
    const float tk = __fadd_rn(sk, yk);
    kc = __fsub_rn(__fsub_rn(tk, sk), yk);
    sk = tk;
    float cv = lamf;
    if (pot32 != nullptr) {
        cv += __ldg(pot32 + x) + __ldg(pot32 + n + y);
        if (DIM == 3) cv += __ldg(pot32 + 2 * n + z);
    }
    const float d = __fmaf_rn(b3f, u2.x, cv);
    dmn = fminf(dmn, d);
    dmx = fmaxf(dmx, d);
    return Ff;
}

template <int DIM, int OUT, bool NEU>
__global__ void __launch_bounds__(256, NEU ? 4 : 5) k_eig_pass2_df(double *__restrict__ U, const float2 *__restrict__ lin, int n,
                                                      int P, double hd, float lamf, float2 b2, float b3f,
                                                      const float *__restrict__ pot32, __nv_bfloat16 *__restrict__ Rhi,
                                                      __nv_bfloat16 *__restrict__ Rlo, double *__restrict__ partials,
                                                      DevState *st) {
    if (state_done(st)) return;
    const double sc = st->eig_scale;
    const float2 sc2 = st->eig_scale2, lamn2 = st->eig_lambda2;   // b2 = b, b3f = 3 b: from the host
    float sk = 0.0f, kc = 0.0f, dmn = INFINITY, dmx = -INFINITY;
    unsigned long long umax = 0ull;
    // one warp per output row of the padded planes, lanes along its x axis
    const int lane = threadIdx.x & 31;
    const int wstride = gridDim.x * (blockDim.x >> 5);
    const int w0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (OUT == 1) {
        const int rows = (DIM == 3) ? P * P : P;
        for (int r = w0; r < rows; r += wstride) {
          const int y = (DIM == 3) ? r % P : r;
          const int z = (DIM == 3) ? r / P : 0;
          for (int x = lane; x < P; x += 32) {
            const long long o = (long long)r * P + x;
            float f = 0.0f;
            if (x < n && y < n && z < n) {
                const long long c = ((long long)z * n + y) * n + x;
                f = eig_point_df<DIM, NEU>(U, lin, c, x, y, z, n, sc, sc2, lamn2, b2, lamf, b3f, pot32, sk, kc, dmn,
                                           dmx, umax);
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(f);
            Rhi[o] = hi;
            Rlo[o] = __float2bfloat16_rn(f - __bfloat162float(hi));
          }
        }
    } else {
        const int H = P / 2, nsym = (n + 1) / 2, nanti = n / 2;
        for (int row = w0; row < P * P; row += wstride) {
          const int ry = row % P, rz = row / P;
          for (int i = lane; i < H; i += 32) {
            float fa = 0.0f, fb = 0.0f;
            if (ry < n && rz < n && i < nsym) {
                const int y = (ry & 1) ? n - 1 - (ry >> 1) : (ry >> 1);
                const int z = (rz & 1) ? n - 1 - (rz >> 1) : (rz >> 1);
                const long long cb = ((long long)z * n + y) * n;
                fa = eig_point_df<DIM, NEU>(U, lin, cb + i, i, y, z, n, sc, sc2, lamn2, b2, lamf, b3f, pot32, sk, kc,
                                            dmn, dmx, umax);
                if (i < nanti) {
                    const int j = n - 1 - i;
                    const float f2 = eig_point_df<DIM, NEU>(U, lin, cb + j, j, y, z, n, sc, sc2, lamn2, b2, lamf, b3f,
                                                            pot32, sk, kc, dmn, dmx, umax);
                    fb = __fsub_rn(fa, f2);
                    fa = __fadd_rn(fa, f2);
                }
            }
            const long long o = (long long)row * P + i;
            const __nv_bfloat16 ha = __float2bfloat16_rn(fa), hb = __float2bfloat16_rn(fb);
            Rhi[o] = ha;
            Rlo[o] = __float2bfloat16_rn(fa - __bfloat162float(ha));
            Rhi[o + H] = hb;
            Rlo[o + H] = __float2bfloat16_rn(fb - __bfloat162float(hb));
          }
        }
    }
    // max|U| of the iterate for the next pass 1's fixed-point exponent
    __shared__ unsigned long long shm[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, umax, o);
        umax = v > umax ? v : umax;
    }
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = umax;
    Sum4 acc = block_pair_red<1, true>(make_float2(sk, -kc), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), dmn,
                                       dmx);   // (its __syncthreads also orders shm)
    acc.a *= hd;
    if (threadIdx.x == 0) {
        unsigned long long m = 0ull;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = shm[i] > m ? shm[i] : m;
        atomicMax(&st->umax_scan, m);
        double *p = partials + 4ll * blockIdx.x;
        p[0] = acc.a;
        p[1] = 0.0;
        p[2] = acc.mn;
        p[3] = acc.mx;
    }
}

}  // namespace

template <int DIM>
static void pass1_dim(const double *U, double *lin, int n, bool neu, double inv_h2, double lam, double b,
                      const double *pot, const double *vrow, double *partials, int grid, const DevState *st,
                      cudaStream_t s) {
    if (neu)
        k_eig_pass1<DIM, true><<<grid, 256, 0, s>>>(U, lin, n, inv_h2, lam, b, pot, vrow, partials, st);
    else
        k_eig_pass1<DIM, false><<<grid, 256, 0, s>>>(U, lin, n, inv_h2, lam, b, pot, vrow, partials, st);
}

int launch_eig_pass1(const double *U, double *lin, int n, int dim, int bc, double inv_h2, double lam, double b,
                     const double *pot, const double *vrow, double *partials, int grid, const DevState *st,
                     cudaStream_t s) {
    const bool neu = (bc == QN_BC_NEUMANN);
    if (pot != nullptr && vrow == nullptr) {
        set_error("launch_eig_pass1: a potential needs its per-row table");
        return QN_EINVAL;
    }
    if (dim == 3)
        pass1_dim<3>(U, lin, n, neu, inv_h2, lam, b, pot, vrow, partials, grid, st, s);
    else
        pass1_dim<2>(U, lin, n, neu, inv_h2, lam, b, pot, vrow, partials, grid, st, s);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

int launch_eig_finalize1(const double *partials, int nparts, double hd, DevState *st, cudaStream_t s) {
    k_eig_finalize1<<<1, 256, 0, s>>>(partials, nparts, hd, st);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

template <int DIM, int OUT>
static void pass2_t(double *U, const double *lin, int n, int P, bool neu, double hd, float lam, double b,
                    const float *pot, double *R64, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, double *partials,
                    int grid, const DevState *st, cudaStream_t s) {
    if (neu)
        k_eig_pass2<DIM, OUT, true><<<grid, 256, 0, s>>>(U, lin, n, P, hd, lam, b, pot, R64, Rhi, Rlo, partials, st,
                                                          &const_cast<DevState *>(st)->umax_scan);
    else
        k_eig_pass2<DIM, OUT, false><<<grid, 256, 0, s>>>(U, lin, n, P, hd, lam, b, pot, R64, Rhi, Rlo, partials, st,
                                                           &const_cast<DevState *>(st)->umax_scan);
}

int launch_eig_pass2(double *U, const double *lin, int n, int P, int dim, int bc, double hd, float lam, double b,
                     const float *pot, double *R64, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, bool mirror,
                     double *partials, int grid, const DevState *st, cudaStream_t s) {
    const bool neu = (bc == QN_BC_NEUMANN);
    if (R64 != nullptr) {
        if (dim == 3)
            pass2_t<3, 0>(U, lin, n, P, neu, hd, lam, b, pot, R64, Rhi, Rlo, partials, grid, st, s);
        else
            pass2_t<2, 0>(U, lin, n, P, neu, hd, lam, b, pot, R64, Rhi, Rlo, partials, grid, st, s);
    } else if (mirror) {
        if (dim != 3 || P % 128 != 0) {
            set_error("launch_eig_pass2: the reflection-split layout needs 3-D and P a multiple of 128");
            return QN_EINVAL;
        }
        pass2_t<3, 2>(U, lin, n, P, neu, hd, lam, b, pot, R64, Rhi, Rlo, partials, grid, st, s);
    } else if (dim == 3) {
        pass2_t<3, 1>(U, lin, n, P, neu, hd, lam, b, pot, R64, Rhi, Rlo, partials, grid, st, s);
    } else {
        pass2_t<2, 1>(U, lin, n, P, neu, hd, lam, b, pot, R64, Rhi, Rlo, partials, grid, st, s);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

template <bool NEU>
static int pass1_tiled(const double *U, float2 *lin, int n, double inv_h2, double lam, float2 lam2, double b,
                       const double *pot, const double *vrow, const float2 *pot2, const float2 *vrow2,
                       double *partials, int grid, int *used, const DevState *st, cudaStream_t s) {
    int dev = 0, sms = 0, nb = 0;
    QN_CUDA(cudaGetDevice(&dev));
    QN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eig_pass1_tiled<NEU>, 256, 0));
    const int zc = n < 400 ? 16 : 32;   // planes per work item (two more are read at its start)
    const long long items = (long long)((n + kP1W - 1) / kP1W) * ((n + kP1H - 1) / kP1H) * ((n + zc - 1) / zc);
    long long g = (long long)(nb > 0 ? nb : 1) * sms;   // one wave of resident blocks
    if (g > grid) g = grid;
    if (g > items) g = items;
    k_eig_pass1_tiled<NEU><<<(int)g, 256, 0, s>>>(U, lin, n, zc, inv_h2, lam, lam2, b, pot, vrow, pot2, vrow2,
                                                  partials, st);
    *used = (int)g;
    return QN_OK;
}

template <int DIM>
static void pass1_df_dim(const double *U, float2 *lin, int n, bool neu, double inv_h2, double lam, double b,
                         const double *pot, const double *vrow, const float2 *pot2, const float2 *vrow2,
                         double *partials, int grid, const DevState *st, cudaStream_t s) {
    const float lh = (float)lam;
    const float2 lam2 = make_float2(lh, (float)(lam - (double)lh));
    if (neu)
        k_eig_pass1_df<DIM, true><<<grid, 256, 0, s>>>(U, lin, n, inv_h2, lam, lam2, b, pot, vrow, pot2, vrow2,
                                                       partials, st);
    else
        k_eig_pass1_df<DIM, false><<<grid, 256, 0, s>>>(U, lin, n, inv_h2, lam, lam2, b, pot, vrow, pot2, vrow2,
                                                        partials, st);
}

int launch_eig_pass1_df(const double *U, float2 *lin, int n, int dim, int bc, double inv_h2, double lam, double b,
                        const double *pot, const double *vrow, const float2 *pot2, const float2 *vrow2,
                        double *partials, int grid, int *used, const DevState *st, cudaStream_t s) {
    if (pot != nullptr && (vrow == nullptr || pot2 == nullptr || vrow2 == nullptr)) {
        set_error("launch_eig_pass1_df: a potential needs its per-row and float-pair tables");
        return QN_EINVAL;
    }
    const bool neu = (bc == QN_BC_NEUMANN);
    *used = grid;
    if (dim == 3) {
        const float lh = (float)lam;
        const float2 lam2 = make_float2(lh, (float)(lam - (double)lh));
        const int rc = neu ? pass1_tiled<true>(U, lin, n, inv_h2, lam, lam2, b, pot, vrow, pot2, vrow2, partials,
                                               grid, used, st, s)
                           : pass1_tiled<false>(U, lin, n, inv_h2, lam, lam2, b, pot, vrow, pot2, vrow2, partials,
                                                grid, used, st, s);
        if (rc) return rc;
    } else {
        pass1_df_dim<2>(U, lin, n, neu, inv_h2, lam, b, pot, vrow, pot2, vrow2, partials, grid, st, s);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

template <int DIM, int OUT>
static int pass2_df_t(double *U, const float2 *lin, int n, int P, bool neu, double hd, float lam, double b,
                      const float *pot32, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, double *partials, int grid,
                      int *used, DevState *st, cudaStream_t s) {
    const float bh = (float)b;
    const float2 b2 = make_float2(bh, (float)(b - (double)bh));
    const float b3f = (float)(3.0 * b);
    // one wave of resident blocks (5 per SM for the Dirichlet forms), at most `grid`
    int dev = 0, sms = 0, nb = 0;
    QN_CUDA(cudaGetDevice(&dev));
    QN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (neu)
        QN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eig_pass2_df<DIM, OUT, true>, 256, 0));
    else
        QN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eig_pass2_df<DIM, OUT, false>, 256, 0));
    const long long rows = (OUT == 2 || DIM == 3) ? (long long)P * P : P;   // one warp per output row
    long long g = (long long)(nb > 0 ? nb : 1) * sms;
    if (g > grid) g = grid;
    if (g > (rows + 7) / 8) g = (rows + 7) / 8;
    if (g < 1) g = 1;
    if (neu)
        k_eig_pass2_df<DIM, OUT, true><<<(int)g, 256, 0, s>>>(U, lin, n, P, hd, lam, b2, b3f, pot32, Rhi, Rlo,
                                                                partials, st);
    else
        k_eig_pass2_df<DIM, OUT, false><<<(int)g, 256, 0, s>>>(U, lin, n, P, hd, lam, b2, b3f, pot32, Rhi, Rlo,
                                                                 partials, st);
    *used = (int)g;
    return QN_OK;
}

int launch_eig_pass2_df(double *U, const float2 *lin, int n, int P, int dim, int bc, double hd, float lam, double b,
                        const float *pot32, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, bool mirror, double *partials,
                        int grid, int *used, DevState *st, cudaStream_t s) {
    const bool neu = (bc == QN_BC_NEUMANN);
    int rc;
    if (mirror) {
        if (dim != 3 || P % 128 != 0) {
            set_error("launch_eig_pass2_df: the reflection-split layout needs 3-D and P a multiple of 128");
            return QN_EINVAL;
        }
        rc = pass2_df_t<3, 2>(U, lin, n, P, neu, hd, lam, b, pot32, Rhi, Rlo, partials, grid, used, st, s);
    } else if (dim == 3) {
        rc = pass2_df_t<3, 1>(U, lin, n, P, neu, hd, lam, b, pot32, Rhi, Rlo, partials, grid, used, st, s);
    } else {
        rc = pass2_df_t<2, 1>(U, lin, n, P, neu, hd, lam, b, pot32, Rhi, Rlo, partials, grid, used, st, s);
    }
    if (rc) return rc;
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

}  // namespace qn
