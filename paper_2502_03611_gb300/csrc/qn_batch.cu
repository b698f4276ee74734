// Batched coupled two-component systems (Sec. 4.3, eq. system; beta from the
// eigenvalues of the 2x2 blocks of DN_h, eqs. eigen_quad and eigenvalues).
//
// Each instance i is a 2-D problem on n_i x n_i interior nodes:
//   F_u = A_h u + u^3 + alpha v - f1,   F_v = D A_h v + v^3 - alpha u - f2,
// solved by the quasi-Newton iteration with the block-diagonal approximate
// Jacobian diag(A_h + beta I, D A_h + beta I); both blocks share the
// eigenvectors of A_h, the second divides by D * (lambda_i + lambda_j) + beta.
// One beta per instance: the midpoint of the extreme (real parts of the)
// eigenvalues of [[3u^2, alpha], [-alpha, 3v^2]] over all nodes.
//
// One iteration of ALL instances is six launches:
//   k_sys_residual   work items (instance, 8 rows) of every active instance:
//                    both residuals (iteration 0 in FP64, later ones on an
//                    exact fixed-point stencil in float pairs), their BF16
//                    hi/lo planes, and partial sums / eigenvalue extremes
//   k_sys_finalize   one block per instance: norms, beta, stop test, and the
//                    device time at which the instance converged
//   4 x k_modeprod_tc one grouped persistent launch per mode product over the
//                    tiles of every instance and component (forward x, forward
//                    y + divide, backward x, backward y + update)
// and is captured once into a CUDA graph that the solve replays; instances
// that have converged make every later launch skip their work.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <mutex>
#include <vector>

#include "qn_df.cuh"
#include "qn_internal.h"
#include "qn_numeric.cuh"
#include "qn_ptx.cuh"

namespace qn {
namespace {

constexpr int kRowsPerItem = 8;

struct SysInst {
    double *U, *V;
    const double *f1, *f2;
    float2 *f1p, *f2p;                               // float-pair copies of f1, f2 (written on iteration 0)
    __nv_bfloat16 *ru_hi, *ru_lo, *rv_hi, *rv_lo;   // buffer 0 planes of both components
    double alpha, D, inv_h2, Dh2;                    // Dh2 = D inv_h2
    float2 ih2, dh2, al2;                            // inv_h2, D inv_h2, alpha as float pairs
    int n, P, item_begin, item_count;
    int df_ok;   // the coefficients are within the float-pair range (|alpha|, D inv_h2 < 2^60)
};

struct SysState {
    int done, status, it;
    int r2_exp;   // k: from the second iteration on, sum r^2 adds (float(r) 2^-k)^2 in FP32 (2^k ~ RMS(f))
    int df;       // iterations >= 1 may take the fixed-point / float-pair residual
    int fbad;     // |f| beyond the float-pair range somewhere
    double beta, f_norm, rel, res;
    unsigned long long t_done;
};

struct SysItem {
    int inst, row0, row1, pad;
};

struct SysCtl {
    double tol;
    int max_it;
    int ndone;
    unsigned long long t0;
};

struct Red4 {
    double r2, f2, mx, mn;
};

__device__ __forceinline__ Red4 warp_red(Red4 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.r2 += __shfl_xor_sync(0xffffffffu, v.r2, o);
        v.f2 += __shfl_xor_sync(0xffffffffu, v.f2, o);
        v.mx = fmax(v.mx, __shfl_xor_sync(0xffffffffu, v.mx, o));
        v.mn = fmin(v.mn, __shfl_xor_sync(0xffffffffu, v.mn, o));
    }
    return v;
}

__device__ Red4 block_red(Red4 v) {
    __shared__ Red4 sh[32];
    v = warp_red(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        v = (l < nw) ? sh[l] : Red4{0.0, 0.0, -INFINITY, INFINITY};
        v = warp_red(v);
    }
    return v;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(v);
    lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__global__ void k_sys_init(SysState *st, int count, SysCtl *ctl, double tol, int max_it) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        SysState s;
        memset(&s, 0, sizeof(s));
        st[i] = s;
    }
    if (i == 0) {
        ctl->tol = tol;
        ctl->max_it = max_it;
        ctl->ndone = 0;
        ctl->t0 = ptx::globaltimer();
    }
}

// Eigenvalues of [[3u^2, alpha], [-alpha, 3v^2]] (real parts), FP32: running extremes. Both
// are >= 0, so they are kept as bit patterns under integer max / min, which the block then
// reduces with one warp instruction each; a rounding below zero is clamped to +0.
__device__ __forceinline__ void sys_extremes(float uf, float vf, float alpha_f, unsigned &mxb, unsigned &mnb) {
    const float a = 3.0f * uf * uf, d = 3.0f * vf * vf;
    const float disc = (a - d) * (a - d) - 4.0f * alpha_f * alpha_f;
    const float sq = disc > 0.0f ? disc * rsqrtf(disc) : 0.0f;   // beta needs no more than FP32 accuracy
    const int hi = __float_as_int(0.5f * (a + d + sq)), lo = __float_as_int(0.5f * (a + d - sq));
    mxb = max(mxb, (unsigned)max(hi, 0));
    mnb = min(mnb, (unsigned)max(lo, 0));
}

// Kahan sum of (F_u 2^-k)^2 + (F_v 2^-k)^2 in FP32.
__device__ __forceinline__ void sys_r2(float Fuf, float Fvf, float r2s, float &kr2, float &kc) {
    const float fu = __fmul_rn(Fuf, r2s), fv = __fmul_rn(Fvf, r2s);
    const float yk = fmaf(fu, fu, fmaf(fv, fv, -kc));
    const float tk = kr2 + yk;
    kc = (tk - kr2) - yk;
    kr2 = tk;
}

// sum f^2 and r^2 in FP64 (first iteration only; out of line so that the FP64
// operations are not predicated into every later iteration's loop)
static __device__ __noinline__ double2 first_iteration_sums(double2 acc, double g1, double g2, double Fu,
                                                          double Fv) {
    return make_double2(fma(g1, g1, fma(g2, g2, acc.x)), fma(Fu, Fu, fma(Fv, Fv, acc.y)));
}

// Both residuals of one node in FP64 (fixed-point stencil, exact up to its final rounding).
__device__ __forceinline__ void sys_node_fp64(const double *__restrict__ U, const double *__restrict__ V,
                                              const double *__restrict__ f1, const double *__restrict__ f2, int c,
                                              int x, int y, int n, double alpha, double inv_h2, double Dh2,
                                              double &u, double &v, double &g1, double &g2, double &Fu, double &Fv) {
    u = __ldg(U + c);
    v = __ldg(V + c);
    double nu[4], nv[4];
    nu[0] = x > 0 ? __ldg(U + c - 1) : 0.0;
    nu[1] = x < n - 1 ? __ldg(U + c + 1) : 0.0;
    nu[2] = y > 0 ? __ldg(U + c - n) : 0.0;
    nu[3] = y < n - 1 ? __ldg(U + c + n) : 0.0;
    nv[0] = x > 0 ? __ldg(V + c - 1) : 0.0;
    nv[1] = x < n - 1 ? __ldg(V + c + 1) : 0.0;
    nv[2] = y > 0 ? __ldg(V + c - n) : 0.0;
    nv[3] = y < n - 1 ? __ldg(V + c + n) : 0.0;
    g1 = __ldg(f1 + c);
    g2 = __ldg(f2 + c);
    const double lu = stencil_fixed<2>(u, nu);
    const double lv = stencil_fixed<2>(v, nv);
    Fu = fma(lu, inv_h2, fma(u * u, u, fma(alpha, v, -g1)));
    Fv = fma(lv, Dh2, fma(v * v, v, fma(-alpha, u, -g2)));
}

// The FP64 node of a float-pair iteration (a value beyond the fixed-point range):
// (F_u, F_v, u, v) rounded to FP32.
static __device__ __noinline__ float4 sys_node_exact(const double *__restrict__ U, const double *__restrict__ V,
                                                     const double *__restrict__ f1, const double *__restrict__ f2,
                                                     int c, int x, int y, int n, double alpha, double inv_h2,
                                                     double Dh2) {
    double u, v, g1, g2, Fu, Fv;
    sys_node_fp64(U, V, f1, f2, c, x, y, n, alpha, inv_h2, Dh2, u, v, g1, g2, Fu, Fv);
    return make_float4(d2f_rn(Fu), d2f_rn(Fv), d2f_rn(u), d2f_rn(v));
}

constexpr int kTW = 32;                  // chunk width (one warp's lanes)
constexpr int kTH = kRowsPerItem;        // chunk height (one row per warp)
constexpr int kHW = kTW + 2, kHH = kTH + 2;

// a * b for a float pair a and a float b (unnormalised pair result)
__device__ __forceinline__ float2 pair_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    return make_float2(p, __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -p)));
}

// a^3 for a float pair a: hi^3 with its exact rounding errors, plus 3 hi^2 lo
__device__ __forceinline__ float2 pair_cube(float2 a) {
    const float s = __fmul_rn(a.x, a.x);
    const float es = __fmaf_rn(a.x, a.x, -s);
    const float c = __fmul_rn(s, a.x);
    const float ec = __fmaf_rn(s, a.x, -c);
    return make_float2(c, __fmaf_rn(3.0f * s, a.y, __fmaf_rn(es, a.x, ec)));
}

// t0 + t1 + t2 + t3 of float pairs, rounded to FP32: the high parts through a chain of
// exact two-sums, every low part and rounding error added once at the end
__device__ __forceinline__ float pair_sum4(float2 t0, float2 t1, float2 t2, float2 t3) {
    float s, e0, e1, e2;
    two_sum(t0.x, t1.x, s, e0);
    two_sum(s, t2.x, s, e1);
    two_sum(s, t3.x, s, e2);
    const float lo = ((t0.y + t1.y) + (t2.y + t3.y)) + ((e0 + e1) + e2);
    return __fadd_rn(s, lo);
}

struct SysTile {   // fixed-point values of one chunk and its halo
    long long u[kHH][kHW], v[kHH][kHW];
};

// bit pattern of node (y, x) of an n x n grid, 0 outside it (the Dirichlet boundary)
__device__ __forceinline__ unsigned long long ld_node(const unsigned long long *__restrict__ B, int y, int x, int n) {
    return (y >= 0 && y < n && x >= 0 && x < n) ? __ldg(B + y * n + x) : 0ull;
}

// high word of |value|: its exponent (bits 20..30) orders magnitudes to within 2x
__device__ __forceinline__ unsigned hi_abs(unsigned long long b) { return (unsigned)(b >> 32) & 0x7FFFFFFFu; }

__device__ __forceinline__ void store_planes(const SysInst &I, int o, float Fuf, float Fvf) {
    __nv_bfloat16 h, l;
    split_bf16(Fuf, h, l);
    I.ru_hi[o] = h;
    I.ru_lo[o] = l;
    split_bf16(Fvf, h, l);
    I.rv_hi[o] = h;
    I.rv_lo[o] = l;
}

// Warp sum of the FP32 Kahan sums (k, -c) as float pairs; lane 0 stores it in out[warp].
__device__ __forceinline__ void warp_pair_sum(float k, float c, float2 *out, int lane) {
    float2 ps = make_float2(k, -c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        ps = pair_add(ps, make_float2(__shfl_xor_sync(0xffffffffu, ps.x, o), __shfl_xor_sync(0xffffffffu, ps.y, o)));
    if (lane == 0) out[threadIdx.x >> 5] = ps;
}

// One block per work item (instance, up to 8 rows of its padded P x P planes), one warp
// per row, lanes along x. Iteration 0, and any iteration without a usable fixed-point
// exponent, runs in FP64 (and writes the float-pair copies of f); later iterations
// evaluate the stencil 4u - sum(nb) as an exact int64 sum of fixed-point values in units
// of 2^(E - 1075 - kFxG), and the rest in float pairs (~48 significant bits). The block
// walks its rows in chunks of 32 columns: it loads the chunk and its halo, takes E from
// the largest |u|, |v| the chunk reads, converts every value to fixed point once into
// shared memory (double-buffered, the next chunk's loads in flight), and forms each
// node's stencil there. A chunk with values of 2^37 or more takes the FP64 path.
__global__ void __launch_bounds__(256, 3) k_sys_residual(const SysInst *__restrict__ inst,
                                                      const SysItem *__restrict__ items, SysState *st,
                                                      double *__restrict__ partials) {
    const SysItem it = items[blockIdx.x];
    const SysState S = st[it.inst];
    if (S.done) return;
    const SysInst I = inst[it.inst];
    const int n = I.n, P = I.P;
    const int lane = threadIdx.x & 31;
    const int y = it.row0 + (threadIdx.x >> 5);
    const double alpha = I.alpha, Dh2 = I.Dh2;
    const float alpha_f = I.al2.x;
    const float r2s = __int_as_float((127 - S.r2_exp) << 23);   // 2^-k
    float kr2 = 0.0f, kc = 0.0f;
    // per-warp partial sums for the block's partials (written at the end of either path)
    __shared__ double sd[2][kTH];
    __shared__ float2 sf[kTH];
    __shared__ unsigned sx[2][kTH];
    unsigned mxb = 0u, mnb = 0x7F800000u;   // +0 and +inf
    if (S.it == 0 || !S.df) {
        const bool first = S.it == 0;   // sum f^2 and r^2 in FP64, copy f as float pairs
        double f2s = 0.0, r2 = 0.0;
        if (y < it.row1) {
            for (int x = lane; x < P; x += 32) {
                float Fuf = 0.0f, Fvf = 0.0f;
                if (y < n && x < n) {
                    const int c = y * n + x;
                    double u, v, g1, g2, Fu, Fv;
                    sys_node_fp64(I.U, I.V, I.f1, I.f2, c, x, y, n, alpha, I.inv_h2, Dh2, u, v, g1, g2, Fu, Fv);
                    Fuf = d2f_rn(Fu);
                    Fvf = d2f_rn(Fv);
                    sys_extremes(d2f_rn(u), d2f_rn(v), alpha_f, mxb, mnb);
                    if (first) {
                        const double2 s2 = first_iteration_sums(make_double2(f2s, r2), g1, g2, Fu, Fv);
                        f2s = s2.x;
                        r2 = s2.y;
                        I.f1p[c] = f_pair(g1, &st[it.inst].fbad);
                        I.f2p[c] = f_pair(g2, &st[it.inst].fbad);
                    } else {
                        sys_r2(Fuf, Fvf, r2s, kr2, kc);
                    }
                }
                store_planes(I, y * P + x, Fuf, Fvf);
            }
        }
        if (first) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                f2s += __shfl_xor_sync(0xffffffffu, f2s, o);
            }
            if (lane == 0) {
                sd[0][threadIdx.x >> 5] = r2;
                sd[1][threadIdx.x >> 5] = f2s;
            }
        } else {
            warp_pair_sum(kr2, kc, sf, lane);
        }
    } else {
        __shared__ SysTile tile[2];
        __shared__ __align__(16) unsigned smax[2][kTH];
        const int t = threadIdx.x, w = t >> 5;
        const unsigned long long *Ub = reinterpret_cast<const unsigned long long *>(I.U);
        const unsigned long long *Vb = reinterpret_cast<const unsigned long long *>(I.V);
        // this thread's halo slot (threads 0 .. 2 kTW + 2 kHH - 1): the rows above and below the
        // chunk, then the columns left and right of it (corners included, unused)
        const bool halo = t < 2 * kTW + 2 * kHH;
        int hr = 0, hc = 0;
        if (t < kTW) {
            hr = 0;
            hc = t + 1;
        } else if (t < 2 * kTW) {
            hr = kHH - 1;
            hc = t - kTW + 1;
        } else if (t < 2 * kTW + kHH) {
            hr = t - 2 * kTW;
            hc = 0;
        } else {
            hr = t - 2 * kTW - kHH;
            hc = kHW - 1;
        }
        const int hy = it.row0 - 1 + hr, hx = hc - 1;   // halo node, x relative to the chunk
        unsigned long long bu = ld_node(Ub, y, lane, n), bv = ld_node(Vb, y, lane, n), hu = 0ull, hv = 0ull;
        if (halo) {
            hu = ld_node(Ub, hy, hx, n);
            hv = ld_node(Vb, hy, hx, n);
        }
        const bool yin = y < n;
        float2 g1 = make_float2(0.0f, 0.0f), g2 = g1;
        if (yin && lane < n) {
            g1 = __ldg(I.f1p + y * n + lane);
            g2 = __ldg(I.f2p + y * n + lane);
        }
        int par = 0;
        for (int x0 = 0; x0 < P; x0 += kTW, par ^= 1) {
            const int x = x0 + lane;
            // the chunk's exponent: the largest |value| it reads (high words carry the exponent)
            unsigned m = max(hi_abs(bu), hi_abs(bv));
            if (halo) m = max(m, max(hi_abs(hu), hi_abs(hv)));
            m = __reduce_max_sync(0xffffffffu, m);
            if (lane == 0) smax[par][w] = m;
            __syncthreads();
            const uint4 m0 = *reinterpret_cast<const uint4 *>(&smax[par][0]);
            const uint4 m1 = *reinterpret_cast<const uint4 *>(&smax[par][4]);
            m = max(max(max(m0.x, m0.y), max(m0.z, m0.w)), max(max(m1.x, m1.y), max(m1.z, m1.w)));
            const int ex = (int)(m >> 20);
            // |values| < 2^37 keep every float-pair product inside the FP32 range; tiny
            // chunks take the exponent 2^-60 (their fixed-point values stay exact to 2^-112)
            const bool ok = ex <= 1023 + 36;
            const int E = ex < 1023 - 60 ? 1023 - 60 : ex;
            SysTile &T = tile[par];
            unsigned nb = 0u;
            const long long fu = fx_of(bu, E, nb), fv = fx_of(bv, E, nb);
            T.u[w + 1][lane + 1] = fu;
            T.v[w + 1][lane + 1] = fv;
            if (halo) {
                T.u[hr][hc] = fx_of(hu, E, nb);
                T.v[hr][hc] = fx_of(hv, E, nb);
            }
            const float2 g1c = g1, g2c = g2;
            if (x0 + kTW < P) {   // prefetch the next chunk
                bu = ld_node(Ub, y, x + kTW, n);
                bv = ld_node(Vb, y, x + kTW, n);
                if (halo) {
                    hu = ld_node(Ub, hy, x0 + kTW + hx, n);
                    hv = ld_node(Vb, hy, x0 + kTW + hx, n);
                }
                if (yin && x + kTW < n) {
                    g1 = __ldg(I.f1p + y * n + x + kTW);
                    g2 = __ldg(I.f2p + y * n + x + kTW);
                }
            }
            __syncthreads();
            float Fuf = 0.0f, Fvf = 0.0f;
            if (yin && x < n) {
                const int c = y * n + x;
                float uf, vf;
                if (ok) {
                    const float scale = __int_as_float((E - 1075 - kFxG + 127) << 23);
                    const long long lu = 4 * fu - T.u[w + 1][lane] - T.u[w + 1][lane + 2] - T.u[w][lane + 1] -
                                         T.u[w + 2][lane + 1];
                    const long long lv = 4 * fv - T.v[w + 1][lane] - T.v[w + 1][lane + 2] - T.v[w][lane + 1] -
                                         T.v[w + 2][lane + 1];
                    // both components' conversions in packed FP32x2 chains (the same results)
                    float2 hi, lo, lu2, lv2, up, vp;
                    fx_to_pair2(lu, lv, scale, hi, lo);
                    lu2 = make_float2(hi.x, lo.x);
                    lv2 = make_float2(hi.y, lo.y);
                    fx_to_pair2(fu, fv, scale, hi, lo);
                    up = make_float2(hi.x, lo.x);
                    vp = make_float2(hi.y, lo.y);
                    // inv_h2 is (n + 1)^2 to FP64 rounding, an FP32 number (n <= 1024): its high part suffices
                    Fuf = pair_sum4(pair_mul_f(lu2, I.ih2.x), pair_cube(up), pair_mul(I.al2, vp), pair_neg(g1c));
                    Fvf = pair_sum4(pair_mul(lv2, I.dh2), pair_cube(vp), pair_neg(pair_mul(I.al2, up)), pair_neg(g2c));
                    uf = up.x;
                    vf = vp.x;
                } else {
                    const float4 r = sys_node_exact(I.U, I.V, I.f1, I.f2, c, x, y, n, alpha, I.inv_h2, Dh2);
                    Fuf = r.x;
                    Fvf = r.y;
                    uf = r.z;
                    vf = r.w;
                }
                sys_extremes(uf, vf, alpha_f, mxb, mnb);
                sys_r2(Fuf, Fvf, r2s, kr2, kc);
            }
            store_planes(I, y * P + x, Fuf, Fvf);
        }
        warp_pair_sum(kr2, kc, sf, lane);
    }
    // Block partials. Iteration 0 sums f^2 and r^2 in FP64; later iterations add the FP32
    // Kahan sums of (r 2^-k)^2 as float pairs and the extremes by integer max / min, so the
    // FP64 pipe (16 cycles per warp instruction) only sees thread 0's last additions.
    const bool first = S.it == 0;
    mxb = __reduce_max_sync(0xffffffffu, mxb);
    mnb = __reduce_min_sync(0xffffffffu, mnb);
    if (lane == 0) {
        sx[0][threadIdx.x >> 5] = mxb;
        sx[1][threadIdx.x >> 5] = mnb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, f = 0.0;
        unsigned mx = 0u, mn = 0x7F800000u;
        float2 ps = make_float2(0.0f, 0.0f);
        for (int i = 0; i < kTH; ++i) {
            if (first) {
                a += sd[0][i];
                f += sd[1][i];
            } else {
                ps = pair_add(ps, sf[i]);
            }
            mx = max(mx, sx[0][i]);
            mn = min(mn, sx[1][i]);
        }
        if (!first)   // (hi + lo) 2^(2k); 2k in [-240, 240], a normal power of two
            a = ((double)ps.x + (double)ps.y) * __longlong_as_double((long long)(1023 + 2 * S.r2_exp) << 52);
        double *p = partials + 4ll * blockIdx.x;
        p[0] = a;
        p[1] = f;
        p[2] = (double)__uint_as_float(mx);
        p[3] = (double)__uint_as_float(mn);
    }
}

__global__ void __launch_bounds__(128) k_sys_finalize(const SysInst *__restrict__ inst, SysState *st,
                                                      const double *__restrict__ partials, SysCtl *ctl) {
    const int i = blockIdx.x;
    if (*(volatile int *)&st[i].done) return;
    const SysInst I = inst[i];
    Red4 acc{0.0, 0.0, -INFINITY, INFINITY};
    for (int k = threadIdx.x; k < I.item_count; k += blockDim.x) {
        const double *p = partials + 4ll * (I.item_begin + k);
        acc.r2 += p[0];
        acc.f2 += p[1];
        acc.mx = fmax(acc.mx, p[2]);
        acc.mn = fmin(acc.mn, p[3]);
    }
    acc = block_red(acc);
    if (threadIdx.x != 0) return;
    SysState s = st[i];
    if (s.it == 0) {
        s.f_norm = sqrt(acc.f2);
        const double rms = s.f_norm / sqrt(2.0 * I.n * I.n);
        int k = (rms > 0.0 && rms < INFINITY) ? ilogb(rms) : 0;
        s.r2_exp = k < -120 ? -120 : (k > 120 ? 120 : k);
    }
    // later iterations in fixed point / float pairs unless a coefficient or |f| is out of
    // the float-pair range, or ||f|| < 2^-40 (relative errors of tiny values would show)
    s.df = (I.df_ok && !s.fbad && s.f_norm >= 0x1p-40) ? 1 : 0;
    const double res = sqrt(acc.r2);
    double rel = s.f_norm > 0.0 ? res / s.f_norm : (res == 0.0 ? 0.0 : INFINITY);
    const double beta = 0.5 * (acc.mx + acc.mn);
    s.rel = rel;
    s.res = res;
    s.beta = beta;
    bool fin = false;
    if (rel <= ctl->tol) {
        s.status = QN_OK;
        fin = true;
    } else if (!isfinite(rel) || rel > 1e8 || !isfinite(beta)) {
        s.status = QN_EDIVERGED;
        fin = true;
    } else if (s.it >= ctl->max_it) {
        s.status = QN_ENOTCONV;
        fin = true;
    } else {
        s.it += 1;
    }
    if (fin) {
        s.done = 1;
        s.t_done = ptx::globaltimer();
        atomicAdd(&ctl->ndone, 1);
    }
    st[i] = s;
}

}  // namespace
}  // namespace qn

using namespace qn;

struct qn_batch {
    int count, device, num_sms, BK;
    std::vector<qn_sys_instance> inst;
    std::vector<int> P, BN;
    // per distinct (P, BN): eigen-data
    struct SizeData {
        int P, n, BN;
        __nv_bfloat16 *S_hi, *S_lo, *Si_hi, *Si_lo;
        float *lam32;
        int map_index;   // 4 maps: s_hi, s_lo, si_hi, si_lo
    };
    std::vector<SizeData> sizes;
    std::vector<int> size_of;          // instance -> sizes index
    __nv_bfloat16 *planes;             // all instance planes
    CUtensorMap *maps;                 // device tensor maps
    TcGroup *groups;                   // [4 steps][2 * count]
    TcTile *tiles;
    int ntiles, grid_mp;
    SysInst *d_inst;
    SysItem *d_items;
    int nitems;
    double *partials;
    float2 *fpairs;                    // float-pair copies of every instance's f1, f2
    SysState *d_state;
    SysCtl *d_ctl;
    int *err;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    int graph_iters;
    cudaStream_t graph_stream;
};

static void batch_free(qn_batch *b) {
    if (!b) return;
    for (auto &z : b->sizes) {
        cudaFree(z.S_hi);
        cudaFree(z.S_lo);
        cudaFree(z.Si_hi);
        cudaFree(z.Si_lo);
        cudaFree(z.lam32);
    }
    cudaFree(b->planes);
    cudaFree(b->maps);
    cudaFree(b->groups);
    cudaFree(b->tiles);
    cudaFree(b->d_inst);
    cudaFree(b->d_items);
    cudaFree(b->partials);
    cudaFree(b->fpairs);
    cudaFree(b->d_state);
    cudaFree(b->d_ctl);
    cudaFree(b->err);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

#define BCK(call)                                  \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) {                   \
            int _r = cuda_fail(_e, #call);         \
            batch_free(b);                         \
            return _r;                             \
        }                                          \
    } while (0)

static void split_host(double v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    const float f = (float)v;
    hi = __float2bfloat16_rn(f);
    lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

extern "C" int qn_batch_create(const qn_sys_instance *inst, int count, int bk, const int *bn,
                               qn_batch **out) {
    if (!inst || !out || count < 1 || count > 65536) {
        set_error("qn_batch_create: need 1..65536 instances and an output pointer");
        return QN_EINVAL;
    }
    *out = nullptr;
    if (bk != 0 && bk != 32 && bk != 64) {
        set_error("qn_batch_create: bk must be 0 (default), 32 or 64");
        return QN_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        const qn_sys_instance &q = inst[i];
        if (q.n < 1 || q.n > 1024 || !q.U || !q.V || !q.f1 || !q.f2 || !isfinite(q.alpha) ||
            !(q.D > 0.0) || !isfinite(q.D)) {
            set_error("qn_batch_create: instance %d invalid (n in 1..1024, D > 0, non-null arrays)", i);
            return QN_EINVAL;
        }
        if (bn && bn[i] != 0 && (bn[i] < 16 || bn[i] > 256 || bn[i] % 16)) {
            set_error("qn_batch_create: bn[%d]=%d must be a multiple of 16 in 16..256", i, bn[i]);
            return QN_EINVAL;
        }
    }
    qn_batch *b = new (std::nothrow) qn_batch();
    if (!b) return QN_ENOMEM;
    b->count = count;
    b->inst.assign(inst, inst + count);
    BCK(cudaGetDevice(&b->device));
    BCK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
    if (!tc_supported(b->device)) {
        set_error("qn_batch_create: needs an sm_103 (tcgen05) device");
        batch_free(b);
        return QN_EUNSUPPORTED;
    }
    if (tc_set_attributes() != QN_OK) {
        batch_free(b);
        return QN_ECUDA;
    }
    b->BK = bk ? bk : 64;
    b->P.resize(count);
    b->BN.resize(count);
    b->size_of.resize(count);
    for (int i = 0; i < count; ++i) {
        b->P[i] = ((inst[i].n + 63) / 64) * 64;
        int want = (bn && bn[i]) ? bn[i] : (b->P[i] <= 256 ? b->P[i] : 256);
        if (want > b->P[i]) want = b->P[i];
        b->BN[i] = want;
    }
    // eigen-data per distinct (n, BN)
    for (int i = 0; i < count; ++i) {
        int found = -1;
        for (size_t z = 0; z < b->sizes.size(); ++z)
            if (b->sizes[z].n == inst[i].n && b->sizes[z].BN == b->BN[i]) found = (int)z;
        if (found < 0) {
            qn_batch::SizeData z;
            memset(&z, 0, sizeof(z));
            z.n = inst[i].n;
            z.P = b->P[i];
            z.BN = b->BN[i];
            b->sizes.push_back(z);
            found = (int)b->sizes.size() - 1;
        }
        b->size_of[i] = found;
    }
    const int nsz = (int)b->sizes.size();
    std::vector<CUtensorMap> hmaps(4 * nsz + 8 * count);
    for (int z = 0; z < nsz; ++z) {
        qn_batch::SizeData &d = b->sizes[z];
        const int n = d.n, P = d.P;
        std::vector<double> S((size_t)n * n), Si((size_t)n * n), lam(n);
        int rc = qn_setup_1d_eig(n, 1.0 / (n + 1), QN_BC_DIRICHLET, S.data(), Si.data(), lam.data());
        if (rc != QN_OK) {
            batch_free(b);
            return rc;
        }
        std::vector<__nv_bfloat16> hS((size_t)P * P), lS((size_t)P * P), hSi((size_t)P * P), lSi((size_t)P * P);
        std::vector<float> l32(P, 1e30f);
        for (int j = 0; j < P; ++j)
            for (int k = 0; k < P; ++k) {
                const double vs = (j < n && k < n) ? S[(size_t)j * n + k] : 0.0;
                const double vi = (j < n && k < n) ? Si[(size_t)j * n + k] : 0.0;
                split_host(vs, hS[(size_t)j * P + k], lS[(size_t)j * P + k]);
                split_host(vi, hSi[(size_t)j * P + k], lSi[(size_t)j * P + k]);
            }
        for (int k = 0; k < n; ++k) l32[k] = (float)lam[k];
        const size_t mb = sizeof(__nv_bfloat16) * P * P;
        BCK(cudaMalloc(&d.S_hi, mb));
        BCK(cudaMalloc(&d.S_lo, mb));
        BCK(cudaMalloc(&d.Si_hi, mb));
        BCK(cudaMalloc(&d.Si_lo, mb));
        BCK(cudaMalloc(&d.lam32, sizeof(float) * P));
        BCK(cudaMemcpy(d.S_hi, hS.data(), mb, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(d.S_lo, lS.data(), mb, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(d.Si_hi, hSi.data(), mb, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(d.Si_lo, lSi.data(), mb, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(d.lam32, l32.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
        d.map_index = 4 * z;
        int rc2 = tc_encode_2d(&hmaps[4 * z + 0], d.S_hi, P, P, b->BK, d.BN, b->BK);
        if (!rc2) rc2 = tc_encode_2d(&hmaps[4 * z + 1], d.S_lo, P, P, b->BK, d.BN, b->BK);
        if (!rc2) rc2 = tc_encode_2d(&hmaps[4 * z + 2], d.Si_hi, P, P, b->BK, d.BN, b->BK);
        if (!rc2) rc2 = tc_encode_2d(&hmaps[4 * z + 3], d.Si_lo, P, P, b->BK, d.BN, b->BK);
        if (rc2) {
            batch_free(b);
            return rc2;
        }
    }
    // planes: per instance, per component, per buffer: hi, lo (P^2 each)
    std::vector<size_t> plane_off(count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        plane_off[i] = total;
        total += (size_t)8 * b->P[i] * b->P[i];
    }
    BCK(cudaMalloc(&b->planes, sizeof(__nv_bfloat16) * total));
    BCK(cudaMemset(b->planes, 0, sizeof(__nv_bfloat16) * total));
    auto plane = [&](int i, int comp, int buf, int lo) {
        const size_t PP = (size_t)b->P[i] * b->P[i];
        return b->planes + plane_off[i] + PP * (size_t)(comp * 4 + buf * 2 + lo);
    };
    const int mapbase = 4 * nsz;
    for (int i = 0; i < count; ++i) {
        const int P = b->P[i];
        for (int comp = 0; comp < 2; ++comp)
            for (int buf = 0; buf < 2; ++buf)
                for (int lo = 0; lo < 2; ++lo) {
                    int rc = tc_encode_2d(&hmaps[mapbase + 8 * i + comp * 4 + buf * 2 + lo], plane(i, comp, buf, lo),
                                          P, P, b->BK, 128, b->BK);
                    if (rc) {
                        batch_free(b);
                        return rc;
                    }
                }
    }
    BCK(cudaMalloc(&b->maps, sizeof(CUtensorMap) * hmaps.size()));
    BCK(cudaMemcpy(b->maps, hmaps.data(), sizeof(CUtensorMap) * hmaps.size(), cudaMemcpyHostToDevice));

    // state, control, items
    BCK(cudaMalloc(&b->d_state, sizeof(SysState) * count));
    BCK(cudaMalloc(&b->d_ctl, sizeof(SysCtl)));
    BCK(cudaMalloc(&b->err, sizeof(int)));
    BCK(cudaMemset(b->err, 0, sizeof(int)));
    size_t npts = 0;
    for (int i = 0; i < count; ++i) npts += (size_t)inst[i].n * inst[i].n;
    BCK(cudaMalloc(&b->fpairs, sizeof(float2) * 2 * npts));
    std::vector<SysInst> hinst(count);
    std::vector<SysItem> hitems;
    size_t poff = 0;
    auto pair_host = [](double v) { const float hi = (float)v; return make_float2(hi, (float)(v - (double)hi)); };
    for (int i = 0; i < count; ++i) {
        SysInst &s = hinst[i];
        s.U = inst[i].U;
        s.V = inst[i].V;
        s.f1 = inst[i].f1;
        s.f2 = inst[i].f2;
        const size_t nn = (size_t)inst[i].n * inst[i].n;
        s.f1p = b->fpairs + poff;
        s.f2p = b->fpairs + poff + nn;
        poff += 2 * nn;
        s.ru_hi = plane(i, 0, 0, 0);
        s.ru_lo = plane(i, 0, 0, 1);
        s.rv_hi = plane(i, 1, 0, 0);
        s.rv_lo = plane(i, 1, 0, 1);
        s.alpha = inst[i].alpha;
        s.D = inst[i].D;
        const double h = 1.0 / (inst[i].n + 1);
        s.inv_h2 = 1.0 / (h * h);
        s.Dh2 = s.D * s.inv_h2;
        s.ih2 = pair_host(s.inv_h2);
        s.dh2 = pair_host(s.D * s.inv_h2);
        s.al2 = pair_host(s.alpha);
        s.df_ok = (fabs(s.alpha) < 0x1p60 && s.D * s.inv_h2 < 0x1p60) ? 1 : 0;
        s.n = inst[i].n;
        s.P = b->P[i];
        s.item_begin = (int)hitems.size();
        for (int r = 0; r < b->P[i]; r += kRowsPerItem) {
            SysItem it;
            it.inst = i;
            it.row0 = r;
            it.row1 = std::min(r + kRowsPerItem, b->P[i]);
            it.pad = 0;
            hitems.push_back(it);
        }
        s.item_count = (int)hitems.size() - s.item_begin;
    }
    b->nitems = (int)hitems.size();
    BCK(cudaMalloc(&b->d_inst, sizeof(SysInst) * count));
    BCK(cudaMemcpy(b->d_inst, hinst.data(), sizeof(SysInst) * count, cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->d_items, sizeof(SysItem) * b->nitems));
    BCK(cudaMemcpy(b->d_items, hitems.data(), sizeof(SysItem) * b->nitems, cudaMemcpyHostToDevice));
    BCK(cudaMalloc(&b->partials, sizeof(double) * 4 * b->nitems));

    // groups: 4 product steps x (instance, component); step s reads buffer (s & 1)
    // and writes buffer 1 - (s & 1); steps 0, 1 forward (S^{-1}), 2, 3 backward (S)
    std::vector<TcGroup> hg((size_t)4 * 2 * count);
    for (int step = 0; step < 4; ++step)
        for (int i = 0; i < count; ++i)
            for (int comp = 0; comp < 2; ++comp) {
                TcGroup &g = hg[(size_t)step * 2 * count + 2 * i + comp];
                const qn_batch::SizeData &z = b->sizes[b->size_of[i]];
                const int src = step & 1, dst = 1 - src;
                const bool fwd = step < 2;
                const CUtensorMap *mb = b->maps;
                g.a_hi = mb + mapbase + 8 * i + comp * 4 + src * 2 + 0;
                g.a_lo = mb + mapbase + 8 * i + comp * 4 + src * 2 + 1;
                g.b_hi = mb + z.map_index + (fwd ? 2 : 0);
                g.b_lo = mb + z.map_index + (fwd ? 3 : 1);
                g.out_hi = step < 3 ? plane(i, comp, dst, 0) : nullptr;
                g.out_lo = step < 3 ? plane(i, comp, dst, 1) : nullptr;
                g.U = comp == 0 ? inst[i].U : inst[i].V;
                g.lam32 = z.lam32;
                g.shift = &b->d_state[i].beta;
                g.done = &b->d_state[i].done;
                g.dscale = comp == 0 ? 1.0f : (float)inst[i].D;
                g.step = 1.0f;
                g.Mtot = b->P[i];
                g.P = b->P[i];
                g.n = inst[i].n;
                g.BN = b->BN[i];
                g.ntile_n = (b->P[i] + b->BN[i] - 1) / b->BN[i];
                g.ntiles = g.ntile_n * ((b->P[i] + 127) / 128);
            }
    BCK(cudaMalloc(&b->groups, sizeof(TcGroup) * hg.size()));
    BCK(cudaMemcpy(b->groups, hg.data(), sizeof(TcGroup) * hg.size(), cudaMemcpyHostToDevice));
    // tiles: largest instances first (longest processing time first)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->P[x] > b->P[y]; });
    std::vector<TcTile> ht;
    for (int i : order)
        for (int comp = 0; comp < 2; ++comp) {
            const TcGroup &g = hg[2 * i + comp];
            for (int mt = 0; mt < (b->P[i] + 127) / 128; ++mt)
                for (int nt = 0; nt < g.ntile_n; ++nt) {
                    TcTile t;
                    t.group = 2 * i + comp;
                    t.m0 = mt * 128;
                    t.n0 = nt * g.BN;
                    t.pad = 0;
                    ht.push_back(t);
                }
        }
    b->ntiles = (int)ht.size();
    b->grid_mp = b->ntiles < b->num_sms ? b->ntiles : b->num_sms;
    BCK(cudaMalloc(&b->tiles, sizeof(TcTile) * b->ntiles));
    BCK(cudaMemcpy(b->tiles, ht.data(), sizeof(TcTile) * b->ntiles, cudaMemcpyHostToDevice));
    *out = b;
    return QN_OK;
}

extern "C" int qn_batch_destroy(qn_batch *b) {
    if (!b) return QN_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return QN_OK;
}

static int enqueue_batch_iteration(qn_batch *b, cudaStream_t s) {
    k_sys_residual<<<b->nitems, 256, 0, s>>>(b->d_inst, b->d_items, b->d_state, b->partials);
    QN_CUDA(cudaGetLastError());
    k_sys_finalize<<<b->count, 128, 0, s>>>(b->d_inst, b->d_state, b->partials, b->d_ctl);
    QN_CUDA(cudaGetLastError());
    const Epi epis[4] = {EPI_STORE, EPI_DIVIDE, EPI_STORE, EPI_UPDATE};
    for (int step = 0; step < 4; ++step) {
        int rc = launch_modeprod_tc_grouped(b->groups + (size_t)step * 2 * b->count, b->tiles, b->ntiles, 2, b->BK,
                                            epis[step], b->err, b->grid_mp, s);
        if (rc) return rc;
    }
    return QN_OK;
}

extern "C" int qn_batch_solve(qn_batch *b, const qn_opts *opts, qn_sys_result *res, void *stream) {
    if (!b) {
        set_error("qn_batch_solve: null batch");
        return QN_EINVAL;
    }
    double tol = 1e-10;
    int max_it = 200;
    int chunk = 4;
    if (opts) {
        tol = opts->tol;
        max_it = opts->max_it;
        if (opts->sync_every >= 1) chunk = opts->sync_every;
        if (opts->beta_mode != QN_BETA_PAPER || opts->step != 1.0) {
            set_error("qn_batch_solve: only the paper's beta rule and step 1 are supported");
            return QN_EUNSUPPORTED;
        }
    }
    if (!(tol >= 0.0) || max_it < 0 || max_it > 4096) {
        set_error("qn_batch_solve: invalid options");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // capture `chunk` iterations once per (batch, stream, chunk)
    if (!b->gexec || b->graph_iters != chunk || b->graph_stream != s) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        if (b->graph) {
            cudaGraphDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cap;
        QN_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_fail(e, "cudaStreamBeginCapture");
        }
        int rc = QN_OK;
        for (int k = 0; k < chunk && rc == QN_OK; ++k) rc = enqueue_batch_iteration(b, cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        b->graph = g;
        QN_CUDA(cudaGraphInstantiate(&b->gexec, g, 0));
        b->graph_iters = chunk;
        b->graph_stream = s;
    }
    k_sys_init<<<(b->count + 255) / 256, 256, 0, s>>>(b->d_state, b->count, b->d_ctl, tol, max_it);
    QN_CUDA(cudaGetLastError());
    int launched = 0;
    SysCtl hctl;
    while (true) {
        QN_CUDA(cudaGraphLaunch(b->gexec, s));
        launched += chunk;
        QN_CUDA(cudaMemcpyAsync(&hctl, b->d_ctl, sizeof(SysCtl), cudaMemcpyDeviceToHost, s));
        QN_CUDA(cudaStreamSynchronize(s));
        if (hctl.ndone >= b->count || launched > max_it + chunk) break;
    }
    int err = 0;
    QN_CUDA(cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        QN_CUDA(cudaMemset(b->err, 0, sizeof(int)));
        set_error("qn_batch_solve: a device-side wait gave up (tensor-core pipeline timeout)");
        return QN_ETIMEOUT;
    }
    std::vector<SysState> hs(b->count);
    QN_CUDA(cudaMemcpy(hs.data(), b->d_state, sizeof(SysState) * b->count, cudaMemcpyDeviceToHost));
    int worst = QN_OK;
    for (int i = 0; i < b->count; ++i) {
        const int st = hs[i].done ? hs[i].status : QN_ENOTCONV;
        if (res) {
            res[i].iterations = hs[i].it;
            res[i].status = st;
            res[i].rel = hs[i].rel;
            res[i].time_ms = hs[i].done ? (double)(hs[i].t_done - hctl.t0) * 1e-6 : -1.0;
        }
        if (st != QN_OK && worst == QN_OK) worst = st;
    }
    return worst;
}

namespace {
// qn_autotune_tile results of this process, per (device, n, copies)
struct TuneKey {
    int dev, n, copies;
    bool operator==(const TuneKey &o) const { return dev == o.dev && n == o.n && copies == o.copies; }
};
struct TuneVal {
    int bk, bn;
    double ms;
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;
}  // namespace

extern "C" int qn_autotune_tile(int n, int copies, int *best_bk, int *best_bn, double *best_ms) {
    if (n < 1 || n > 1024 || copies < 1 || copies > 4096 || !best_bk || !best_bn) {
        set_error("qn_autotune_tile: n in 1..1024, copies in 1..4096, non-null outputs");
        return QN_EINVAL;
    }
    int dev = 0;
    QN_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto &e : g_tune_cache)
            if (e.first == TuneKey{dev, n, copies}) {
                *best_bk = e.second.bk;
                *best_bn = e.second.bn;
                if (best_ms) *best_ms = e.second.ms;
                return QN_OK;
            }
    }
    const int P = ((n + 63) / 64) * 64;
    double *zero = nullptr;
    const size_t nn = (size_t)n * n;
    QN_CUDA(cudaMalloc(&zero, sizeof(double) * nn));
    cudaMemset(zero, 0, sizeof(double) * nn);
    std::vector<qn_sys_instance> inst(copies);
    for (int i = 0; i < copies; ++i) {
        inst[i].n = n;
        inst[i].alpha = 0.5;
        inst[i].D = 1.0;
        inst[i].U = zero;
        inst[i].V = zero;
        inst[i].f1 = zero;
        inst[i].f2 = zero;
    }
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(zero);
        set_error("qn_autotune_tile: stream creation failed");
        return QN_ECUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int bbk = 64, bbn = P < 256 ? P : 256;
    const int bks[2] = {64, 32};
    const int bns[3] = {64, 128, 256};
    int rc = QN_OK;
    for (int a = 0; a < 2 && rc == QN_OK; ++a)
        for (int c = 0; c < 3 && rc == QN_OK; ++c) {
            const int bn = bns[c];
            if (bn > P) continue;
            std::vector<int> bnv(copies, bn);
            qn_batch *b = nullptr;
            rc = qn_batch_create(inst.data(), copies, bks[a], bnv.data(), &b);
            if (rc) break;
            // states all "not done" so that every tile runs
            k_sys_init<<<(copies + 255) / 256, 256, 0, s>>>(b->d_state, copies, b->d_ctl, 0.0, 1);
            const int reps = 10;
            for (int w = 0; w < 2 && rc == QN_OK; ++w)
                rc = launch_modeprod_tc_grouped(b->groups, b->tiles, b->ntiles, 2, b->BK, EPI_STORE, b->err,
                                                b->grid_mp, s);
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == QN_OK; ++r)
                rc = launch_modeprod_tc_grouped(b->groups, b->tiles, b->ntiles, 2, b->BK, EPI_STORE, b->err,
                                                b->grid_mp, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = QN_ECUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            int err = 0;
            cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost);
            if (err) rc = QN_ETIMEOUT;
            qn_batch_destroy(b);
            if (rc == QN_OK && ms / reps < best) {
                best = ms / reps;
                bbk = bks[a];
                bbn = bn;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(zero);
    if (rc) return rc;
    *best_bk = bbk;
    *best_bn = bbn;
    if (best_ms) *best_ms = best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.push_back({TuneKey{dev, n, copies}, TuneVal{bbk, bbn, best}});
    }
    return QN_OK;
}
