// Learned warm start: a small sine-basis neural operator that maps the source
// f (restricted to a coarse G^3 grid) to an initial iterate U_0, trained on
// solutions of the quasi-Newton method itself, plus the trilinear transfers
// between the fine n^3 grid and the coarse grid. The paper has no learned
// component; this is the warm-start extension of the solver.
//
// Network (activations [batch][z][y][x][channel], channel fastest):
//   lift        h0 = f wl + bl                              (1 -> C)
//   block l     hh = analysis_xyz(h_l)                      (G^3 -> M^3 sine modes)
//               g[k][o] = sum_i hh[k][i] R_l[k][i][o]       (per-mode channel mixing)
//               z_l = synthesis_xyz(g) + h_l W_l + b_l
//               h_{l+1} = gelu(z_l) (l < L-1), z_l (last)
//   projection  out = h_L wp + bp                           (C -> 1)
// with the orthonormal sine basis Bm[j][k] = sqrt(2/(G+1)) sin(pi (j+1)(k+1)/(G+1)).
// Storage: activations h_l, z_l in BF16; all arithmetic and accumulation in
// FP32; FP32 master parameters, gradients and AdamW moments.
//
// Kernels: k_lift, k_axis (apply a small matrix along one axis of a
// channel-last tensor: analysis, synthesis and their adjoints), k_modemix
// (+ backward for inputs and weights), k_pointwise (z = s + hW + b, gelu),
// k_pointwise_bwd (gelu', dh = dz W^T, dW, db), k_project (+ backward), k_mse,
// k_adamw, k_interp3d (trilinear transfer).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "qn_internal.h"
#include "qn_numeric.cuh"

namespace qn {
namespace {

constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2/pi)

__device__ __forceinline__ float gelu_f(float x) {
    return 0.5f * x * (1.0f + tanhf(kGeluC * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad_f(float x) {
    const float t = tanhf(kGeluC * (x + 0.044715f * x * x * x));
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * kGeluC * (1.0f + 3.0f * 0.044715f * x * x);
}

template <typename T>
__device__ __forceinline__ float ld(const T *p, long long i);
template <>
__device__ __forceinline__ float ld<float>(const float *p, long long i) {
    return p[i];
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p, long long i) {
    return __bfloat162float(p[i]);
}

// Sum a per-lane value over the warps of the block (same meaning in every
// warp), then one atomicAdd per lane into dst[lane]. All threads must call it.
__device__ __forceinline__ void block_atomic_lanes(float v, float *dst, float *sbuf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    sbuf[warp * 32 + lane] = v;
    __syncthreads();
    if (warp == 0) {
        float t = 0.0f;
        for (int w = 0; w < nw; ++w) t += sbuf[w * 32 + lane];
        atomicAdd(dst + lane, t);
    }
    __syncthreads();
}

// out[o][k][i][c] (+)= sum_j Mt[k][j] in[o][j][i][c]
// The lanes of a warp take the channels c (coalesced loads of the C
// contiguous values at every j); a warp walks a run of `run` consecutive
// (o, k, i) rows, decomposing the first row index once and stepping the
// others (every tensor here has < 2^31 elements); the j loop is unrolled so
// that several loads are in flight. Large tensors take runs of up to 8 rows,
// small ones (latency-bound) one row per warp.
constexpr int kAxisRunMax = 8;
template <typename Tin>
__global__ void __launch_bounds__(256) k_axis(const Tin *__restrict__ in, float *__restrict__ out,
                                              const float *__restrict__ Mt, long long outer, int Kin, int Kout,
                                              int inner, int C, int accumulate, int run) {
    __shared__ float sM[64 * 64];
    for (int t = threadIdx.x; t < Kin * Kout; t += blockDim.x) sM[t] = Mt[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int rows = (int)(outer * Kout * inner);
    const int jstride = inner * C;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int r0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * run; r0 < rows; r0 += nwarps * run) {
        int i = r0 % inner;
        const int rr = r0 / inner;
        int k = rr % Kout;
        int o = rr / Kout;
        const int rend = min(r0 + run, rows);
        for (int row = r0; row < rend; ++row) {
            const Tin *ib = in + ((long long)o * Kin * inner + i) * C;
            const float *mk = sM + k * Kin;
            float *ob = out + (long long)row * C;
            for (int c = lane; c < C; c += 32) {
                float sacc = 0.0f;
#pragma unroll 8
                for (int j = 0; j < Kin; ++j) sacc = fmaf(mk[j], ld(ib, (long long)j * jstride + c), sacc);
                if (accumulate)
                    ob[c] += sacc;
                else
                    ob[c] = sacc;
            }
            if (++i == inner) {
                i = 0;
                if (++k == Kout) {
                    k = 0;
                    ++o;
                }
            }
        }
    }
}

// h0[p][c] = f[p] wl[c] + bl[c]
__global__ void k_lift(const float *__restrict__ f, const float *__restrict__ wl, const float *__restrict__ bl,
                       __nv_bfloat16 *__restrict__ h, long long pts, int C) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < pts * C;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx % C);
        h[idx] = __float2bfloat16_rn(fmaf(f[idx / C], wl[c], bl[c]));
    }
}

// g[b][k][o] = sum_i hh[b][k][i] R[k][i][o]
__global__ void k_modemix(const float *__restrict__ hh, const float *__restrict__ R, float *__restrict__ g, int B,
                          int K, int C) {
    const long long total = (long long)B * K * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(idx % C);
        const long long bk = idx / C;
        const int k = (int)(bk % K);
        const float *x = hh + bk * C;
        const float *w = R + (long long)k * C * C + o;
        float s = 0.0f;
        for (int i = 0; i < C; ++i) s = fmaf(x[i], w[i * C], s);
        g[idx] = s;
    }
}

// dhh[b][k][i] = sum_o dg[b][k][o] R[k][i][o]
__global__ void k_modemix_bwd_in(const float *__restrict__ dg, const float *__restrict__ R, float *__restrict__ dhh,
                                 int B, int K, int C) {
    const long long total = (long long)B * K * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % C);
        const long long bk = idx / C;
        const int k = (int)(bk % K);
        const float *d = dg + bk * C;
        const float *w = R + ((long long)k * C + i) * C;
        float s = 0.0f;
        for (int o = 0; o < C; ++o) s = fmaf(d[o], w[o], s);
        dhh[idx] = s;
    }
}

// dR[k][i][o] = sum_b hh[b][k][i] dg[b][k][o]   (fixed order over b: deterministic)
__global__ void k_modemix_bwd_w(const float *__restrict__ hh, const float *__restrict__ dg, float *__restrict__ dR,
                                int B, int K, int C) {
    const long long total = (long long)K * C * C;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(idx % C);
        const int i = (int)((idx / C) % C);
        const int k = (int)(idx / ((long long)C * C));
        float s = 0.0f;
        for (int b = 0; b < B; ++b)
            s = fmaf(hh[((long long)b * K + k) * C + i], dg[((long long)b * K + k) * C + o], s);
        dR[idx] = s;
    }
}

// z = s + h W + b ; h_next = gelu(z) (or z). One warp per node, lane = output
// channel (C == 32): each lane keeps its column of W in registers; the node's
// 32 input channels are broadcast from shared memory (eight 16-byte reads).
__global__ void __launch_bounds__(256) k_pointwise(const float *__restrict__ sp, const __nv_bfloat16 *__restrict__ h,
                                                   const float *__restrict__ W, const float *__restrict__ bvec,
                                                   __nv_bfloat16 *__restrict__ z, __nv_bfloat16 *__restrict__ hnext,
                                                   long long pts, int act) {
    __shared__ __align__(16) float sh[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float w[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w[i] = __ldg(W + i * 32 + lane);
    const float bo = bvec[lane];
    const float4 *h4 = reinterpret_cast<const float4 *>(sh[warp]);
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        sh[warp][lane] = __bfloat162float(h[p * 32 + lane]);
        __syncwarp();
        float s = sp[p * 32 + lane] + bo;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 v = h4[q];
            s = fmaf(v.x, w[4 * q], s);
            s = fmaf(v.y, w[4 * q + 1], s);
            s = fmaf(v.z, w[4 * q + 2], s);
            s = fmaf(v.w, w[4 * q + 3], s);
        }
        __syncwarp();
        z[p * 32 + lane] = __float2bfloat16_rn(s);
        hnext[p * 32 + lane] = __float2bfloat16_rn(act ? gelu_f(s) : s);
    }
}

// Backward of one block's pointwise path and activation:
//   dz = dh * gelu'(z) (or dh), written to dz;
//   dh_prev = dz W^T (written, the spectral path adds to it later);
//   dW[i][o] += sum_p h[p][i] dz[p][o], db[o] += sum_p dz[p][o] (per-block partials, then atomics).
__global__ void __launch_bounds__(256) k_pointwise_bwd(const float *__restrict__ dh, const __nv_bfloat16 *__restrict__ z,
                                                       const __nv_bfloat16 *__restrict__ h, const float *__restrict__ W,
                                                       float *__restrict__ dz_out, float *__restrict__ dh_prev,
                                                       float *__restrict__ dW, float *__restrict__ db, long long pts,
                                                       int act) {
    __shared__ float sWt[32 * 32];    // transposed: sWt[o][i] = W[i][o]
    __shared__ float sbuf[32 * 32];
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) sWt[(t % 32) * 32 + t / 32] = W[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float gW[32];   // this lane's column o = lane of dW, rows i = 0..31
#pragma unroll
    for (int i = 0; i < 32; ++i) gW[i] = 0.0f;
    float gb = 0.0f;
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        float d = dh[p * 32 + lane];
        if (act) d *= gelu_grad_f(__bfloat162float(z[p * 32 + lane]));
        dz_out[p * 32 + lane] = d;
        const float hin = __bfloat162float(h[p * 32 + lane]);
        // dh_prev[i = lane] = sum_o dz[o] W[lane][o]
        float s = 0.0f;
#pragma unroll
        for (int o = 0; o < 32; ++o) s = fmaf(__shfl_sync(0xffffffffu, d, o), sWt[o * 32 + lane], s);
        dh_prev[p * 32 + lane] = s;
#pragma unroll
        for (int i = 0; i < 32; ++i) gW[i] = fmaf(__shfl_sync(0xffffffffu, hin, i), d, gW[i]);
        gb += d;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) block_atomic_lanes(gW[i], dW + i * 32, sbuf);
    block_atomic_lanes(gb, db, sbuf);
}

// out[p] = sum_c h[p][c] wp[c] + bp
__global__ void k_project(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ wp, const float *__restrict__ bp,
                          float *__restrict__ out, long long pts) {
    const int lane = threadIdx.x & 31;
    const float w = wp[lane];
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        float s = __bfloat162float(h[p * 32 + lane]) * w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[p] = s + bp[0];
    }
}

// dh[p][c] = dout[p] wp[c]; dwp[c] += sum_p dout[p] h[p][c]; dbp += sum_p dout[p]
__global__ void k_project_bwd(const float *__restrict__ dout, const __nv_bfloat16 *__restrict__ h,
                              const float *__restrict__ wp, float *__restrict__ dh, float *__restrict__ dwp,
                              float *__restrict__ dbp, long long pts) {
    const int lane = threadIdx.x & 31;
    const float w = wp[lane];
    float gw = 0.0f, gb = 0.0f;
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        const float d = dout[p];
        dh[p * 32 + lane] = d * w;
        gw = fmaf(d, __bfloat162float(h[p * 32 + lane]), gw);
        gb += d;
    }
    __shared__ float sbuf[32 * 32];
    block_atomic_lanes(gw, dwp, sbuf);
    // every lane of a warp summed the same dout values: take lane 0's sum once per warp
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sbuf[warp] = gb;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < nw; ++w) t += sbuf[w];
        atomicAdd(dbp, t);
    }
}

// dwl[c] += sum_p f[p] dh0[p][c], dbl[c] += sum_p dh0[p][c]
__global__ void k_lift_bwd(const float *__restrict__ f, const float *__restrict__ dh, float *__restrict__ dwl,
                           float *__restrict__ dbl, long long pts) {
    const int lane = threadIdx.x & 31;
    float gw = 0.0f, gb = 0.0f;
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5) {
        const float d = dh[p * 32 + lane];
        gw = fmaf(f[p], d, gw);
        gb += d;
    }
    __shared__ float sbuf[32 * 32];
    block_atomic_lanes(gw, dwl, sbuf);
    block_atomic_lanes(gb, dbl, sbuf);
}

// loss += sum (out - t)^2 / N ; dout = 2 (out - t) / N
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ t, float *__restrict__ dout,
                      double *__restrict__ loss, long long N) {
    double acc = 0.0;
    const float inv = 1.0f / (float)N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - t[i];
        if (dout) dout[i] = 2.0f * d * inv;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)N);
}

__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                        long long n, float lr, float b1, float b2, float eps, float wd, float bc1, float bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / bc1, vh = vi / bc2;
        p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    }
}

// Trilinear transfer: dst (m_to^3) = interpolation of src (m_from^3) at nodes
// i/(m_to+1), with zero values on the boundary of (0,1)^3. Batched over B.
// The 1-D corner indices and weights (the same table for every axis) are
// computed once per block into shared memory; the interpolation runs in FP64
// only when both source and destination are FP64 (the exactly tested
// transfer), else in FP32 - the precision of the FP32 end (the network's
// input or output), without spending the FP64 pipe.
constexpr int kInterpMax = 2048;
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_interp3d(const Tin *__restrict__ src, int m_from, Tout *__restrict__ dst,
                                                  int m_to, int B, double scale) {
    typedef typename std::conditional<(sizeof(Tin) == 8 && sizeof(Tout) == 8), double, float>::type Tc;
    __shared__ int sj[kInterpMax];
    __shared__ Tc sw[kInterpMax];
    for (int i = threadIdx.x; i < m_to; i += blockDim.x) {
        const double t = (double)(i + 1) * (m_from + 1) / (m_to + 1);
        const int j = (int)floor(t);   // 1-based left node; 0 and m_from+1 are the zero boundary
        sj[i] = j;
        sw[i] = (Tc)(t - j);
    }
    __syncthreads();
    const Tc sc = (Tc)scale;
    const long long rows = (long long)B * m_to * m_to;
    const long long sper = (long long)m_from * m_from * m_from;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int iy = (int)(row % m_to);
        const long long r2 = row / m_to;
        const int iz = (int)(r2 % m_to);
        const long long b = r2 / m_to;
        const Tin *sb = src + b * sper;
        const int jz = sj[iz], jy = sj[iy];
        const Tc wz = sw[iz], wy = sw[iy];
        // weights and row offsets of the four (z, y) corner rows (0 outside the grid)
        Tc wr[4];
        long long ro[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int zz = jz + (c >> 1), yy = jy + (c & 1);
            const bool ok = zz >= 1 && zz <= m_from && yy >= 1 && yy <= m_from;
            wr[c] = ok ? ((c >> 1) ? wz : (Tc)1 - wz) * ((c & 1) ? wy : (Tc)1 - wy) : (Tc)0;
            ro[c] = ok ? ((long long)(zz - 1) * m_from + (yy - 1)) * m_from : 0;
        }
        for (int ix = threadIdx.x; ix < m_to; ix += blockDim.x) {
            const int jx = sj[ix];
            const Tc wx = sw[ix];
            const bool okl = jx >= 1, okr = jx + 1 <= m_from;
            Tc acc = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const Tc vl = okl ? (Tc)sb[ro[c] + jx - 1] : (Tc)0;
                const Tc vr = okr ? (Tc)sb[ro[c] + jx] : (Tc)0;
                acc += wr[c] * (((Tc)1 - wx) * vl + wx * vr);
            }
            dst[row * m_to + ix] = (Tout)(acc * sc);
        }
    }
}

// ---------------------------------------------------------------------------
// Inference path (batch 1, qn_net_predict). The training forward keeps one kernel
// per stage because the backward pass reads every intermediate; inference needs
// none of them, so each block runs as three kernels:
//   k_inf_analysis   the x and y analysis: every CTA reduces a chunk of rows of one
//                    z plane to its (ky, kx) sums;
//   k_inf_mix        one CTA per mode k: the z analysis of those sums (fixed order:
//                    deterministic) and the mixing g = hh R_l;
//   k_inf_pointwise  z_l = synthesis_xyz(g) + h_l W_l + b_l, h_{l+1} = gelu(z_l): the
//                    z and y synthesis per CTA and row, the x synthesis per node, so
//                    the FP32 spectral term is never stored; the last block projects
//                    to the output channel directly (z_l itself is not stored).
// The restriction is k_interp3d; the lift and the prolongation have their own
// kernels (one warp per node / per fine row, no 64-bit division per element).
constexpr int kInfRows = 16;   // rows of one z plane per CTA

// h0[p][c] = f[p] wl[c] + bl[c], lane = c
__global__ void __launch_bounds__(256) k_inf_lift(const float *__restrict__ f, const float *__restrict__ wl,
                                                  const float *__restrict__ bl, __nv_bfloat16 *__restrict__ h,
                                                  long long pts) {
    const int lane = threadIdx.x & 31;
    const float w = wl[lane], b = bl[lane];
    for (long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; p < pts;
         p += ((long long)gridDim.x * blockDim.x) >> 5)
        h[p * 32 + lane] = __float2bfloat16_rn(fmaf(f[p], w, b));
}

template <int M>
__global__ void __launch_bounds__(256) k_inf_analysis(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ Ba,
                                                      int G, float *__restrict__ part) {
    __shared__ float sBa[M * 256];        // Ba[k][j] = basis_a[k * G + j], G <= 256
    __shared__ float sQ[M * M * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunks = (G + kInfRows - 1) / kInfRows;
    const int z = blockIdx.x / chunks, y0 = (blockIdx.x % chunks) * kInfRows;
    const int y1 = min(y0 + kInfRows, G);
    for (int t = threadIdx.x; t < M * G; t += blockDim.x) sBa[t] = Ba[t];
    for (int t = threadIdx.x; t < M * M * 32; t += blockDim.x) sQ[t] = 0.0f;
    __syncthreads();
    float Q[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) Q[a][b] = 0.0f;
    for (int y = y0 + warp; y < y1; y += 8) {
        const __nv_bfloat16 *row = h + (((long long)z * G + y) * G) * 32 + lane;
        float t[M];
#pragma unroll
        for (int k = 0; k < M; ++k) t[k] = 0.0f;
#pragma unroll 4
        for (int x = 0; x < G; ++x) {
            const float v = __bfloat162float(row[(long long)x * 32]);
#pragma unroll
            for (int k = 0; k < M; ++k) t[k] = fmaf(sBa[k * G + x], v, t[k]);
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const float b = sBa[a * G + y];
#pragma unroll
            for (int k = 0; k < M; ++k) Q[a][k] = fmaf(b, t[k], Q[a][k]);
        }
    }
    // the CTA's (ky, kx) sums of this z plane's rows (the 8 warps' in a fixed order)
    for (int w = 0; w < 8; ++w) {
        if (warp == w) {
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int k = 0; k < M; ++k) sQ[(a * M + k) * 32 + lane] += Q[a][k];
        }
        __syncthreads();
    }
    float *pb = part + (long long)blockIdx.x * M * M * 32;
    for (int t = threadIdx.x; t < M * M * 32; t += blockDim.x) pb[t] = sQ[t];
}

// hh[k][c] = sum_z Ba[kz][z] sum_chunks part[z][chunk][(ky, kx)][c] for one mode
// k = (kz, ky, kx) per CTA (128 threads: 4 groups of z planes, fixed order), then
// g[k][o] = sum_i hh[k][i] R[k][i][o].
template <int M>
__global__ void __launch_bounds__(128) k_inf_mix(const float *__restrict__ part, const float *__restrict__ Ba, int G,
                                                 const float *__restrict__ R, float *__restrict__ hh,
                                                 float *__restrict__ g) {
    __shared__ float sacc[4][32];
    const int k = blockIdx.x;
    const int kz = k / (M * M), e = k % (M * M);
    const int c = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int chunks = (G + kInfRows - 1) / kInfRows;
    float acc = 0.0f;
#pragma unroll 4
    for (int zz = grp; zz < G; zz += 4) {
        float sz = 0.0f;
        for (int ch = 0; ch < chunks; ++ch) sz += __ldg(part + ((long long)(zz * chunks + ch) * M * M + e) * 32 + c);
        acc = fmaf(__ldg(Ba + kz * G + zz), sz, acc);
    }
    sacc[grp][c] = acc;
    __syncthreads();
    if (grp != 0) return;
    const float v = (sacc[0][c] + sacc[1][c]) + (sacc[2][c] + sacc[3][c]);
    hh[(long long)k * 32 + c] = v;
    sacc[0][c] = v;
    __syncwarp();
    const float *Rk = R + (long long)k * 32 * 32 + c;
    float o = 0.0f;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) o = fmaf(sacc[0][i], __ldg(Rk + i * 32), o);
    g[(long long)k * 32 + c] = o;
}

template <int M, bool LAST>
__global__ void __launch_bounds__(256) k_inf_pointwise(const __nv_bfloat16 *__restrict__ h, const float *__restrict__ Bs,
                                                       int G, const float *__restrict__ g, const float *__restrict__ W,
                                                       const float *__restrict__ bvec, __nv_bfloat16 *__restrict__ hnext,
                                                       const float *__restrict__ wp, const float *__restrict__ bp,
                                                       float *__restrict__ out) {
    __shared__ float sBs[256 * M];        // Bs[j][k] = basis_s[j * M + k]
    __shared__ float sgz[M * M * 32];     // g contracted over kz at this CTA's plane z
    constexpr int U = LAST ? 2 : 4;       // nodes per step (the projection's reductions: two)
    __shared__ __align__(16) float sh[8][U][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunks = (G + kInfRows - 1) / kInfRows;
    const int z = blockIdx.x / chunks, y0 = (blockIdx.x % chunks) * kInfRows;
    const int y1 = min(y0 + kInfRows, G);
    for (int t = threadIdx.x; t < M * G; t += blockDim.x) sBs[t] = Bs[t];
    __syncthreads();
    for (int e = threadIdx.x; e < M * M * 32; e += blockDim.x) {
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < M; ++k) a = fmaf(sBs[z * M + k], g[(long long)k * M * M * 32 + e], a);
        sgz[e] = a;
    }
    float w[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w[i] = __ldg(W + i * 32 + lane);
    const float bo = bvec[lane];
    const float wpl = LAST ? wp[lane] : 0.0f;
    const float bpv = LAST ? bp[0] : 0.0f;
    __syncthreads();
    for (int y = y0 + warp; y < y1; y += 8) {
        float t1r[M];   // z and y synthesis of this row, per kx
#pragma unroll
        for (int kx = 0; kx < M; ++kx) {
            float a = 0.0f;
#pragma unroll
            for (int ky = 0; ky < M; ++ky) a = fmaf(sBs[y * M + ky], sgz[(ky * M + kx) * 32 + lane], a);
            t1r[kx] = a;
        }
        const long long rowbase = ((long long)z * G + y) * G;
        for (int x = 0; x < G; x += U) {   // U nodes per step
            const long long p = rowbase + x;
            float sv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = x + u < G;
                sh[warp][u][lane] = ok ? __bfloat162float(h[(p + u) * 32 + lane]) : 0.0f;
                float a = bo;
#pragma unroll
                for (int kx = 0; kx < M; ++kx) a = fmaf(ok ? sBs[(x + u) * M + kx] : 0.0f, t1r[kx], a);
                sv[u] = a;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float4 v = reinterpret_cast<const float4 *>(sh[warp][u])[q];
                    sv[u] = fmaf(v.x, w[4 * q], sv[u]);
                    sv[u] = fmaf(v.y, w[4 * q + 1], sv[u]);
                    sv[u] = fmaf(v.z, w[4 * q + 2], sv[u]);
                    sv[u] = fmaf(v.w, w[4 * q + 3], sv[u]);
                }
            }
            __syncwarp();
            if (LAST) {
                // the U projections reduced over the channels together (independent shuffle chains)
                float o[U];
#pragma unroll
                for (int u = 0; u < U; ++u) o[u] = sv[u] * wpl;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int u = 0; u < U; ++u) o[u] += __shfl_xor_sync(0xffffffffu, o[u], off);
                if (lane == 0) {
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (x + u < G) out[p + u] = o[u] + bpv;
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (x + u < G) hnext[(p + u) * 32 + lane] = __float2bfloat16_rn(gelu_f(sv[u]));
            }
        }
    }
}

// U0 (mt^3, FP64) = scale * trilinear prolongation of src (mf^3, FP32) at the nodes
// i/(mt+1), zero values on the boundary: one warp per fine row; the 1-D corner
// indices and weights from integer arithmetic (i+1)(mf+1) = j (mt+1) + r, w = r/(mt+1).
// With sq != nullptr it also adds sum U0^2 to *sq (FP32 per warp, one FP64 atomic per CTA).
__global__ void __launch_bounds__(256) k_prolong_f32_f64(const float *__restrict__ src, int mf,
                                                         double *__restrict__ dst, int mt, float scale,
                                                         double *__restrict__ sq) {
    __shared__ int sj[kInterpMax];
    __shared__ float sw[kInterpMax];
    __shared__ float ssq[8];
    for (int i = threadIdx.x; i < mt; i += blockDim.x) {
        const int num = (i + 1) * (mf + 1);
        sj[i] = num / (mt + 1);   // 1-based left node; 0 and mf+1 are the zero boundary
        sw[i] = (float)(num % (mt + 1)) / (float)(mt + 1);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long rows = (long long)mt * mt;
    float wsq = 0.0f;
    for (long long row = (long long)blockIdx.x * 8 + warp; row < rows; row += (long long)gridDim.x * 8) {
        const int iz = (int)(row / mt), iy = (int)(row % mt);
        const int jz = sj[iz], jy = sj[iy];
        const float wz = sw[iz], wy = sw[iy];
        float wr[4];
        const float *ro[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int zz = jz + (c >> 1), yy = jy + (c & 1);
            const bool ok = zz >= 1 && zz <= mf && yy >= 1 && yy <= mf;
            wr[c] = ok ? ((c >> 1) ? wz : 1.0f - wz) * ((c & 1) ? wy : 1.0f - wy) : 0.0f;
            ro[c] = src + (ok ? ((long long)(zz - 1) * mf + (yy - 1)) * mf : 0);
        }
        double *drow = dst + row * mt;
        for (int ix = lane; ix < mt; ix += 32) {
            const int jx = sj[ix];
            const float wx = sw[ix];
            const bool okl = jx >= 1, okr = jx + 1 <= mf;
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float vl = okl ? __ldg(ro[c] + jx - 1) : 0.0f;
                const float vr = okr ? __ldg(ro[c] + jx) : 0.0f;
                acc = fmaf(wr[c], fmaf(wx, vr - vl, vl), acc);
            }
            const float u = acc * scale;
            wsq = fmaf(u, u, wsq);
            drow[ix] = f2d_exact(u);
        }
    }
    if (sq == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsq += __shfl_xor_sync(0xffffffffu, wsq, o);
    if (lane == 0) ssq[warp] = wsq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += (double)ssq[w];
        atomicAdd(sq, t);
    }
}

// Grid for the kernels that end in per-block reductions (few blocks, many nodes each).
inline int grid_reduce(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 2) g = 152 * 2;
    if (g < 1) g = 1;
    return (int)g;
}

inline int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// k_axis: rows of C (= 32) channels per warp so that ~10k warps share the work
inline int axis_run(long long elements) {
    const long long rows = elements / 32;
    long long r = rows / (152 * 64);
    return (int)(r < 1 ? 1 : (r > kAxisRunMax ? kAxisRunMax : r));
}
inline int grid_axis(long long elements) { return grid_for((elements + axis_run(elements) - 1) / axis_run(elements)); }

}  // namespace
}  // namespace qn

using namespace qn;

struct qn_net {
    int G, C, M, L, Bmax;
    long long nparams;
    float *params, *grads, *am, *av;
    float *basis_a;   // M x G (analysis: out[k] = sum_j B[j][k] in[j])
    float *basis_s;   // G x M (synthesis)
    std::vector<__nv_bfloat16 *> h, z;
    std::vector<float *> hh;
    float *t1, *t2, *sp, *g, *dg, *dhh, *out, *dout, *dh, *dz, *dh2, *fin, *tgt;
    float *part;              // inference: per-CTA (ky, kx) sums of k_inf_analysis
    double *wsq;              // warm-started solves: ||U_1 - U_0||^2, ||U_0||^2
    double *loss;
    long long step;
};

static void net_free(qn_net *n) {
    if (!n) return;
    cudaFree(n->params);
    cudaFree(n->grads);
    cudaFree(n->am);
    cudaFree(n->av);
    cudaFree(n->basis_a);
    cudaFree(n->basis_s);
    for (auto p : n->h) cudaFree(p);
    for (auto p : n->z) cudaFree(p);
    for (auto p : n->hh) cudaFree(p);
    cudaFree(n->t1);
    cudaFree(n->t2);
    cudaFree(n->sp);
    cudaFree(n->g);
    cudaFree(n->dg);
    cudaFree(n->dhh);
    cudaFree(n->out);
    cudaFree(n->dout);
    cudaFree(n->dh);
    cudaFree(n->dz);
    cudaFree(n->dh2);
    cudaFree(n->fin);
    cudaFree(n->tgt);
    cudaFree(n->loss);
    cudaFree(n->part);
    cudaFree(n->wsq);
    delete n;
}

#define NCK(call)                             \
    do {                                      \
        cudaError_t _e = (call);              \
        if (_e != cudaSuccess) {              \
            int _r = cuda_fail(_e, #call);    \
            net_free(n);                      \
            return _r;                        \
        }                                     \
    } while (0)

static long long net_param_count(int C, int M, int L) {
    return 2LL * C + (long long)L * ((long long)M * M * M * C * C + (long long)C * C + C) + C + 1;
}

extern "C" long long qn_net_param_count(int channels, int modes, int blocks) {
    return net_param_count(channels, modes, blocks);
}

extern "C" int qn_net_create(int G, int channels, int modes, int blocks, int max_batch, qn_net **out) {
    if (!out || G < 2 || G > 256 || channels != 32 || modes < 1 || modes > G || modes > 16 || blocks < 1 ||
        blocks > 16 || max_batch < 1 || max_batch > 64) {
        set_error("qn_net_create: G in 2..256, channels == 32, 1 <= modes <= min(G, 16), blocks 1..16, batch 1..64");
        return QN_EINVAL;
    }
    *out = nullptr;
    qn_net *n = new (std::nothrow) qn_net();
    if (!n) return QN_ENOMEM;
    n->G = G;
    n->C = channels;
    n->M = modes;
    n->L = blocks;
    n->Bmax = max_batch;
    n->nparams = net_param_count(channels, modes, blocks);
    const long long pts = (long long)max_batch * G * G * G;
    const long long act = pts * channels;
    const long long K = (long long)modes * modes * modes;
    NCK(cudaMalloc(&n->params, sizeof(float) * n->nparams));
    NCK(cudaMalloc(&n->grads, sizeof(float) * n->nparams));
    NCK(cudaMalloc(&n->am, sizeof(float) * n->nparams));
    NCK(cudaMalloc(&n->av, sizeof(float) * n->nparams));
    NCK(cudaMemset(n->params, 0, sizeof(float) * n->nparams));
    NCK(cudaMemset(n->am, 0, sizeof(float) * n->nparams));
    NCK(cudaMemset(n->av, 0, sizeof(float) * n->nparams));
    std::vector<float> ba((size_t)modes * G), bs((size_t)G * modes);
    const double pi = 3.14159265358979323846;
    for (int j = 0; j < G; ++j)
        for (int k = 0; k < modes; ++k) {
            const double v = sqrt(2.0 / (G + 1)) * sin(pi * (double)(j + 1) * (k + 1) / (G + 1));
            ba[(size_t)k * G + j] = (float)v;
            bs[(size_t)j * modes + k] = (float)v;
        }
    NCK(cudaMalloc(&n->basis_a, sizeof(float) * modes * G));
    NCK(cudaMalloc(&n->basis_s, sizeof(float) * modes * G));
    NCK(cudaMemcpy(n->basis_a, ba.data(), sizeof(float) * modes * G, cudaMemcpyHostToDevice));
    NCK(cudaMemcpy(n->basis_s, bs.data(), sizeof(float) * modes * G, cudaMemcpyHostToDevice));
    n->h.assign(blocks + 1, nullptr);
    n->z.assign(blocks, nullptr);
    n->hh.assign(blocks, nullptr);
    for (int l = 0; l <= blocks; ++l) NCK(cudaMalloc(&n->h[l], sizeof(__nv_bfloat16) * act));
    for (int l = 0; l < blocks; ++l) {
        NCK(cudaMalloc(&n->z[l], sizeof(__nv_bfloat16) * act));
        NCK(cudaMalloc(&n->hh[l], sizeof(float) * max_batch * K * channels));
    }
    const long long tsz = (long long)max_batch * G * G * modes * channels;
    NCK(cudaMalloc(&n->t1, sizeof(float) * tsz));
    NCK(cudaMalloc(&n->t2, sizeof(float) * tsz));
    NCK(cudaMalloc(&n->sp, sizeof(float) * act));
    NCK(cudaMalloc(&n->g, sizeof(float) * max_batch * K * channels));
    NCK(cudaMalloc(&n->dg, sizeof(float) * max_batch * K * channels));
    NCK(cudaMalloc(&n->dhh, sizeof(float) * max_batch * K * channels));
    NCK(cudaMalloc(&n->out, sizeof(float) * pts));
    NCK(cudaMalloc(&n->dout, sizeof(float) * pts));
    NCK(cudaMalloc(&n->dh, sizeof(float) * act));
    NCK(cudaMalloc(&n->dz, sizeof(float) * act));
    NCK(cudaMalloc(&n->dh2, sizeof(float) * act));
    NCK(cudaMalloc(&n->fin, sizeof(float) * pts));
    NCK(cudaMalloc(&n->tgt, sizeof(float) * pts));
    NCK(cudaMalloc(&n->loss, sizeof(double)));
    {
        const long long chunks = (G + kInfRows - 1) / kInfRows;
        NCK(cudaMalloc(&n->part, sizeof(float) * (size_t)(G * chunks * modes * modes * channels)));
        NCK(cudaMalloc(&n->wsq, 2 * sizeof(double)));
    }
    n->step = 0;
    *out = n;
    return QN_OK;
}

extern "C" int qn_net_destroy(qn_net *n) {
    if (!n) return QN_OK;
    cudaDeviceSynchronize();
    net_free(n);
    return QN_OK;
}

extern "C" int qn_net_set_params(qn_net *n, const float *host_params, long long count) {
    if (!n || !host_params || count != n->nparams) {
        set_error("qn_net_set_params: expected %lld parameters", n ? n->nparams : 0LL);
        return QN_EINVAL;
    }
    QN_CUDA(cudaMemcpy(n->params, host_params, sizeof(float) * count, cudaMemcpyHostToDevice));
    QN_CUDA(cudaMemset(n->am, 0, sizeof(float) * count));
    QN_CUDA(cudaMemset(n->av, 0, sizeof(float) * count));
    n->step = 0;
    return QN_OK;
}

extern "C" int qn_net_get_params(qn_net *n, float *host_params, long long count) {
    if (!n || !host_params || count != n->nparams) {
        set_error("qn_net_get_params: expected %lld parameters", n ? n->nparams : 0LL);
        return QN_EINVAL;
    }
    QN_CUDA(cudaMemcpy(host_params, n->params, sizeof(float) * count, cudaMemcpyDeviceToHost));
    return QN_OK;
}

// parameter pointers
static float *P_wl(qn_net *n) { return n->params; }
static float *P_bl(qn_net *n) { return n->params + n->C; }
static long long block_base(qn_net *n, int l) {
    const long long K = (long long)n->M * n->M * n->M;
    return 2LL * n->C + (long long)l * (K * n->C * n->C + (long long)n->C * n->C + n->C);
}
static long long off_R(qn_net *n, int l) { return block_base(n, l); }
static long long off_W(qn_net *n, int l) {
    return block_base(n, l) + (long long)n->M * n->M * n->M * n->C * n->C;
}
static long long off_b(qn_net *n, int l) { return off_W(n, l) + (long long)n->C * n->C; }
static long long off_wp(qn_net *n) { return block_base(n, n->L); }

// Forward pass on the coarse input already in n->fin (B samples); out in n->out.
static int net_forward(qn_net *n, int B, cudaStream_t s) {
    const int G = n->G, C = n->C, M = n->M;
    const long long pts = (long long)B * G * G * G;
    const int K = M * M * M;
    k_lift<<<grid_for(pts * C), 256, 0, s>>>(n->fin, P_wl(n), P_bl(n), n->h[0], pts, C);
    for (int l = 0; l < n->L; ++l) {
        // analysis x, y, z
        k_axis<__nv_bfloat16><<<grid_axis((long long)B * G * G * M * C), 256, 0, s>>>(
            n->h[l], n->t1, n->basis_a, (long long)B * G * G, G, M, 1, C, 0, axis_run((long long)B * G * G * M * C));
        k_axis<float><<<grid_axis((long long)B * G * M * M * C), 256, 0, s>>>(n->t1, n->t2, n->basis_a,
                                                                             (long long)B * G, G, M, M, C, 0, axis_run((long long)B * G * M * M * C));
        k_axis<float><<<grid_axis((long long)B * K * C), 256, 0, s>>>(n->t2, n->hh[l], n->basis_a, (long long)B, G, M,
                                                                     M * M, C, 0, axis_run((long long)B * K * C));
        k_modemix<<<grid_for((long long)B * K * C), 256, 0, s>>>(n->hh[l], n->params + off_R(n, l), n->g, B, K, C);
        // synthesis z, y, x
        k_axis<float><<<grid_axis((long long)B * G * M * M * C), 256, 0, s>>>(n->g, n->t2, n->basis_s, (long long)B, M,
                                                                             G, M * M, C, 0, axis_run((long long)B * G * M * M * C));
        k_axis<float><<<grid_axis((long long)B * G * G * M * C), 256, 0, s>>>(n->t2, n->t1, n->basis_s,
                                                                             (long long)B * G, M, G, M, C, 0, axis_run((long long)B * G * G * M * C));
        k_axis<float><<<grid_axis(pts * C), 256, 0, s>>>(n->t1, n->sp, n->basis_s, (long long)B * G * G, M, G, 1, C,
                                                        0, axis_run(pts * C));
        k_pointwise<<<grid_for(pts * 32), 256, 0, s>>>(n->sp, n->h[l], n->params + off_W(n, l),
                                                       n->params + off_b(n, l), n->z[l], n->h[l + 1], pts,
                                                       l < n->L - 1 ? 1 : 0);
    }
    k_project<<<grid_for(pts * 32), 256, 0, s>>>(n->h[n->L], n->params + off_wp(n), n->params + off_wp(n) + C, n->out,
                                                 pts);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

// Inference (batch 1) on n->fin, the result in n->out, through the fused kernels.
template <int M>
static int net_infer_t(qn_net *n, cudaStream_t s) {
    const int G = n->G;
    const long long pts = (long long)G * G * G;
    const int grid = G * ((G + kInfRows - 1) / kInfRows);
    k_inf_lift<<<grid_for(pts * 32), 256, 0, s>>>(n->fin, P_wl(n), P_bl(n), n->h[0], pts);
    for (int l = 0; l < n->L; ++l) {
        k_inf_analysis<M><<<grid, 256, 0, s>>>(n->h[l], n->basis_a, G, n->part);
        k_inf_mix<M><<<M * M * M, 128, 0, s>>>(n->part, n->basis_a, G, n->params + off_R(n, l), n->hh[l], n->g);
        if (l < n->L - 1)
            k_inf_pointwise<M, false><<<grid, 256, 0, s>>>(n->h[l], n->basis_s, G, n->g, n->params + off_W(n, l),
                                                           n->params + off_b(n, l), n->h[l + 1], nullptr, nullptr,
                                                           nullptr);
        else
            k_inf_pointwise<M, true><<<grid, 256, 0, s>>>(n->h[l], n->basis_s, G, n->g, n->params + off_W(n, l),
                                                          n->params + off_b(n, l), nullptr, n->params + off_wp(n),
                                                          n->params + off_wp(n) + n->C, n->out);
    }
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

static int net_infer(qn_net *n, cudaStream_t s) {
    switch (n->M) {
        case 2: return net_infer_t<2>(n, s);
        case 3: return net_infer_t<3>(n, s);
        case 4: return net_infer_t<4>(n, s);
        case 5: return net_infer_t<5>(n, s);
        case 6: return net_infer_t<6>(n, s);
        case 7: return net_infer_t<7>(n, s);
        case 8: return net_infer_t<8>(n, s);
        default: return net_forward(n, 1, s);   // larger mode counts: the unfused kernels
    }
}

// Backward pass after net_forward; gradients (overwritten) in n->grads.
static int net_backward(qn_net *n, int B, cudaStream_t s) {
    const int G = n->G, C = n->C, M = n->M;
    const long long pts = (long long)B * G * G * G;
    const int K = M * M * M;
    QN_CUDA(cudaMemsetAsync(n->grads, 0, sizeof(float) * n->nparams, s));
    k_project_bwd<<<grid_reduce(pts * 32), 256, 0, s>>>(n->dout, n->h[n->L], n->params + off_wp(n), n->dh,
                                                     n->grads + off_wp(n), n->grads + off_wp(n) + C, pts);
    for (int l = n->L - 1; l >= 0; --l) {
        // dz (into n->dz), dh_prev = dz W^T (into n->dh2), dW, db
        k_pointwise_bwd<<<grid_reduce(pts * 32), 256, 0, s>>>(n->dh, n->z[l], n->h[l], n->params + off_W(n, l), n->dz,
                                                           n->dh2, n->grads + off_W(n, l), n->grads + off_b(n, l), pts,
                                                           l < n->L - 1 ? 1 : 0);
        // spectral path: dg = analysis(dz); dR; dhh = dg R^T; dh_prev += synthesis(dhh)
        k_axis<float><<<grid_axis((long long)B * G * G * M * C), 256, 0, s>>>(n->dz, n->t1, n->basis_a,
                                                                             (long long)B * G * G, G, M, 1, C, 0, axis_run((long long)B * G * G * M * C));
        k_axis<float><<<grid_axis((long long)B * G * M * M * C), 256, 0, s>>>(n->t1, n->t2, n->basis_a,
                                                                             (long long)B * G, G, M, M, C, 0, axis_run((long long)B * G * M * M * C));
        k_axis<float><<<grid_axis((long long)B * K * C), 256, 0, s>>>(n->t2, n->dg, n->basis_a, (long long)B, G, M,
                                                                     M * M, C, 0, axis_run((long long)B * K * C));
        k_modemix_bwd_w<<<grid_for((long long)K * C * C), 256, 0, s>>>(n->hh[l], n->dg, n->grads + off_R(n, l), B, K,
                                                                        C);
        k_modemix_bwd_in<<<grid_for((long long)B * K * C), 256, 0, s>>>(n->dg, n->params + off_R(n, l), n->dhh, B, K,
                                                                         C);
        k_axis<float><<<grid_axis((long long)B * G * M * M * C), 256, 0, s>>>(n->dhh, n->t2, n->basis_s, (long long)B,
                                                                             M, G, M * M, C, 0, axis_run((long long)B * G * M * M * C));
        k_axis<float><<<grid_axis((long long)B * G * G * M * C), 256, 0, s>>>(n->t2, n->t1, n->basis_s,
                                                                             (long long)B * G, M, G, M, C, 0, axis_run((long long)B * G * G * M * C));
        k_axis<float><<<grid_axis(pts * C), 256, 0, s>>>(n->t1, n->dh2, n->basis_s, (long long)B * G * G, M, G, 1, C,
                                                        1, axis_run(pts * C));
        float *tmp = n->dh;
        n->dh = n->dh2;
        n->dh2 = tmp;
    }
    k_lift_bwd<<<grid_reduce(pts * 32), 256, 0, s>>>(n->fin, n->dh, n->grads + 0, n->grads + C, pts);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

static int check_batch(qn_net *n, int B) {
    if (!n || B < 1 || B > n->Bmax) {
        set_error("qn_net: batch must be in 1..%d", n ? n->Bmax : 0);
        return QN_EINVAL;
    }
    return QN_OK;
}

extern "C" int qn_net_forward(qn_net *n, const float *f_coarse, float *out, int B, void *stream) {
    int rc = check_batch(n, B);
    if (rc) return rc;
    if (!f_coarse || !out) {
        set_error("qn_net_forward: null array");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long pts = (long long)B * n->G * n->G * n->G;
    QN_CUDA(cudaMemcpyAsync(n->fin, f_coarse, sizeof(float) * pts, cudaMemcpyDeviceToDevice, s));
    rc = net_forward(n, B, s);
    if (rc) return rc;
    QN_CUDA(cudaMemcpyAsync(out, n->out, sizeof(float) * pts, cudaMemcpyDeviceToDevice, s));
    return QN_OK;
}

extern "C" int qn_net_gradients(qn_net *n, const float *f_coarse, const float *target, int B, float *grads_out,
                                double *loss, void *stream) {
    int rc = check_batch(n, B);
    if (rc) return rc;
    if (!f_coarse || !target) {
        set_error("qn_net_gradients: null array");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long pts = (long long)B * n->G * n->G * n->G;
    QN_CUDA(cudaMemcpyAsync(n->fin, f_coarse, sizeof(float) * pts, cudaMemcpyDeviceToDevice, s));
    QN_CUDA(cudaMemcpyAsync(n->tgt, target, sizeof(float) * pts, cudaMemcpyDeviceToDevice, s));
    rc = net_forward(n, B, s);
    if (rc) return rc;
    QN_CUDA(cudaMemsetAsync(n->loss, 0, sizeof(double), s));
    k_mse<<<grid_for(pts), 256, 0, s>>>(n->out, n->tgt, n->dout, n->loss, pts);
    rc = net_backward(n, B, s);
    if (rc) return rc;
    if (grads_out) QN_CUDA(cudaMemcpyAsync(grads_out, n->grads, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, s));
    if (loss) {
        QN_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        QN_CUDA(cudaStreamSynchronize(s));
    }
    return QN_OK;
}

extern "C" int qn_net_train_step(qn_net *n, const float *f_coarse, const float *target, int B, float lr,
                                 float weight_decay, double *loss, void *stream) {
    int rc = qn_net_gradients(n, f_coarse, target, B, nullptr, nullptr, stream);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - powf(b1, (float)n->step), bc2 = 1.0f - powf(b2, (float)n->step);
    k_adamw<<<grid_for(n->nparams), 256, 0, s>>>(n->params, n->grads, n->am, n->av, n->nparams, lr, b1, b2, 1e-8f,
                                                 weight_decay, bc1, bc2);
    QN_CUDA(cudaGetLastError());
    if (loss) {
        QN_CUDA(cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        QN_CUDA(cudaStreamSynchronize(s));
    }
    return QN_OK;
}

extern "C" int qn_interp3d(const double *src, int m_from, double *dst, int m_to, int B, double scale, void *stream) {
    if (!src || !dst || m_from < 1 || m_to < 1 || m_from > kInterpMax || m_to > kInterpMax || B < 1) {
        set_error("qn_interp3d: invalid arguments");
        return QN_EINVAL;
    }
    const long long rows = (long long)m_to * m_to * B;
    k_interp3d<double, double><<<grid_for(rows * 256), 256, 0, (cudaStream_t)stream>>>(src, m_from, dst, m_to, B,
                                                                                      scale);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

extern "C" int qn_interp3d_f32(const double *src, int m_from, float *dst, int m_to, int B, double scale,
                               void *stream) {
    if (!src || !dst || m_from < 1 || m_to < 1 || m_from > kInterpMax || m_to > kInterpMax || B < 1) {
        set_error("qn_interp3d_f32: invalid arguments");
        return QN_EINVAL;
    }
    const long long rows = (long long)m_to * m_to * B;
    k_interp3d<double, float><<<grid_for(rows * 256), 256, 0, (cudaStream_t)stream>>>(src, m_from, dst, m_to, B,
                                                                                     scale);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

// Warm start for one fine n^3 source: restrict f to the G^3 grid, run the
// network, prolong its output to n^3 (times out_scale) into U0.
// U0 = prolong(net(restrict(f))); with u0_sq != nullptr, *u0_sq += ||U0||^2.
static int net_predict(qn_net *n, const double *f_fine, int nf, double in_scale, double out_scale, double *U0,
                       double *u0_sq, cudaStream_t s) {
    const int G = n->G;
    k_interp3d<double, float><<<grid_for((long long)G * G * 256), 256, 0, s>>>(f_fine, nf, n->fin, G, 1, in_scale);
    int rc = net_infer(n, s);
    if (rc) return rc;
    k_prolong_f32_f64<<<grid_for((long long)nf * nf * 32), 256, 0, s>>>(n->out, G, U0, nf, (float)out_scale, u0_sq);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

extern "C" int qn_net_predict(qn_net *n, const double *f_fine, int nf, double in_scale, double out_scale, double *U0,
                              void *stream) {
    if (!n || !f_fine || !U0 || nf < 1 || nf > 2048) {
        set_error("qn_net_predict: invalid arguments");
        return QN_EINVAL;
    }
    return net_predict(n, f_fine, nf, in_scale, out_scale, U0, nullptr, (cudaStream_t)stream);
}

// sums[0] += sum (a - b)^2, sums[1] += sum b^2
__global__ void k_diff_norms(const double *__restrict__ a, const double *__restrict__ b, long long n,
                             double *__restrict__ sums) {
    double d2 = 0.0, b2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = a[i] - b[i];
        d2 = fma(d, d, d2);
        b2 = fma(b[i], b[i], b2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, d2);
        atomicAdd(sums + 1, b2);
    }
}

// Warm-started solve with the zero-start fallback. U0 = prolong(net(restrict(f))).
// The first quasi-Newton correction delta = (A_h + beta I)^{-1} F(U0) estimates
// the error of U0 (the inverse removes the high-frequency error that the
// trilinear prolongation leaves, which inflates ||F(U0)|| without making U0
// a worse start). If ||delta|| < ||U0|| / 2 the solve continues from
// U1 = U0 - delta (that update counts as an iteration); otherwise, or if U0 is
// not finite, it restarts from the standard zero start.
extern "C" int qn_solve_warm(qn_ctx *ctx, qn_net *net, double *U, const double *f, int n, double in_scale,
                             double out_scale, const qn_opts *opts, qn_result *res, int *used_warm, void *stream) {
    if (!ctx || !net || !U || !f || n < 1) {
        set_error("qn_solve_warm: invalid arguments");
        return QN_EINVAL;
    }
    if (!ctx_unit_dirichlet(ctx)) {
        set_error("qn_solve_warm: the network predicts Dirichlet solutions on the unit cube without a potential");
        return QN_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)n * n * n;
    double *sums = net->wsq;
    QN_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(double), s));
    // the prolongation also sums ||U_0||^2 into sums[1]
    int rc = net_predict(net, f, n, in_scale, out_scale, U, sums + 1, s);
    if (rc) return rc;
    if (ctx_split_precision(ctx)) {
        // one solve from U_0; its first iteration measures ||U_1 - U_0|| and
        // falls back to the zero start by itself (solve_internal)
        int used = 0;
        rc = solve_internal(ctx, U, f, opts, res, nullptr, 0, stream, sums + 1, &used);
        if (used_warm) *used_warm = used;
        return rc;
    }
    // FP64 path: a separate first step, then the solve
    double *U0 = nullptr;
    QN_CUDA(cudaMallocAsync(&U0, sizeof(double) * N, s));
    QN_CUDA(cudaMemcpyAsync(U0, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    qn_stats st0;
    rc = qn_step(ctx, U, f, NAN, &st0, stream);          // U1 = U0 - delta
    bool warm = (rc == QN_OK) && isfinite(st0.res_norm);
    if (warm) {
        QN_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(double), s));
        k_diff_norms<<<grid_for(N), 256, 0, s>>>(U, U0, N, sums);
        double h[2] = {0.0, 0.0};
        QN_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
        QN_CUDA(cudaStreamSynchronize(s));
        warm = isfinite(h[0]) && isfinite(h[1]) && h[1] > 0.0 && h[0] < 0.25 * h[1];
    }
    cudaFreeAsync(U0, s);
    if (used_warm) *used_warm = warm ? 1 : 0;
    if (!warm) {
        QN_CUDA(cudaMemsetAsync(U, 0, sizeof(double) * N, s));
        return qn_solve(ctx, U, f, opts, res, nullptr, 0, stream);
    }
    rc = qn_solve(ctx, U, f, opts, res, nullptr, 0, stream);
    if (res && (rc == QN_OK || rc == QN_ENOTCONV || rc == QN_EDIVERGED)) res->iterations += 1;
    return rc;
}
