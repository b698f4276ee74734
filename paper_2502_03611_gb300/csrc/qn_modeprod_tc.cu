// Split-precision mode product on the 5th-generation tensor cores (tcgen05).
//
// Same contraction as the FP64 kernel (Sec. 4.1 eq. fin_inverse, one mode
// product per launch, result stored transposed so the axes rotate and every
// product contracts the contiguous axis):
//
//     out[k][m] = sum_j A[m][j] * B[k][j],   A = [Mtot][P] data, B = S or S^{-1}
//
// with each operand held as an unevaluated sum of two BF16 values
// (x = x_hi + x_lo, x_hi = bf16(x), x_lo = bf16(x - x_hi)) and the product
// formed as A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (TMEM) accumulators.
// The intermediate tensors are stored in the same hi/lo form on a grid padded
// to P = 64*ceil(n/64) points per axis (padded entries are zero, padded
// eigenvalues are 1e30 so the divide keeps them zero).
//
// Kernel organisation (persistent, one CTA of 576 threads per SM, kThreads):
//   warp 0 lane 0  TMA producer: A_hi, A_lo (128 x BK) and B_hi, B_lo (BN x BK)
//                  tiles per pipeline stage, K-major with 128-B or 64-B swizzle
//   warp 1         allocates TMEM (2 accumulators of BN FP32 columns); lane 0
//                  issues tcgen05.mma (M=128, N=BN, K=16) and commits to mbarriers
//   warps 2..17    epilogue (kEpiWarps = 16): tcgen05.ld of the accumulator; four
//                  warps per TMEM lane quadrant (warp w owns lanes 32*(w%4)..+31 =
//                  rows), each taking a quarter of the BN columns in 16-column
//                  loads, then store / divide / update
// Tiles are walked in m-major order (consecutive CTAs share the same A rows;
// S stays resident in L2). The epilogue of tile i overlaps the MMAs of tile
// i+1 through the double-buffered accumulators.
//
// Reflection-split products (MODE 1 and 2; 3-D split solve with P a multiple
// of 128, H = P/2). The sine basis satisfies S[n-1-j][k] = (-1)^k S[j][k], so
// along one axis
//   forward:  Xhat[2i]   = sum_j S[j][2i]   a_j,  a_j = x_j + x_{n-1-j} (+ the middle x of odd n)
//             Xhat[2i+1] = sum_j S[j][2i+1] b_j,  b_j = x_j - x_{n-1-j}
//   backward: x_j = p_j + q_j, x_{n-1-j} = p_j - q_j with p_j = sum_i S[j][2i] Y_{2i},
//             q_j = sum_i S[j][2i+1] Y_{2i+1}
// - two GEMMs of half the contraction length instead of one: half the tensor
// work. Tensors in this form keep the contracted axis in split order (a or
// even modes in [0, H), b or odd modes in [H, P)).
//   MODE 1 (forward): output rows k < H take the A columns [0, H), rows >= H the
//   columns [H, P); B = [P][H] (even-mode rows, then odd-mode rows).
//   MODE 2 (backward): a tile of BN <= 128 output rows j < H accumulates p over
//   the A columns [0, H) and q over [H, P) in two TMEM accumulators; B = [P][H]
//   (rows j of the even-mode half, then of the odd-mode half). The epilogue
//   writes rows j and n-1-j.
// The butterflies that form a and b ride in the epilogues: the axis that the
// next product contracts is the fast part of m, stored in folded order (j at
// 2j, its mirror at 2j+1), so partners sit in adjacent TMEM lanes (one shuffle).
//
// Six-product backward level (template flag L3; the BF16X6 precision). The
// error of a three-product correction is spread evenly over all modes, and A_h
// amplifies it by up to its stiffness ratio lambda_max/lambda_min: the backward
// products set the correction's residual, the forward products' error is
// divided by the eigenvalue sums. With L3 the divide epilogue (MODE 1) writes
// its output as three BF16 levels x = x0 + x1 + x2 (each the rounded remainder
// of the previous), and the backward products (MODE 2) read three levels of A
// and of B and accumulate the six products a0 b0 + a0 b1 + a1 b0 + a1 b1 +
// a0 b2 + a2 b0 (every term down to 2^-16 of the leading one; FP32
// accumulation), writing three levels again. The stages then hold six tiles.
//
// Every mbarrier wait is bounded (2 s of %globaltimer). On expiry the kernel
// sets the device error flag, tells the other roles to stop, waits (bounded)
// for its own outstanding TMA copies and MMAs, frees TMEM and returns.
#include <cudaTypedefs.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "qn_internal.h"
#include "qn_numeric.cuh"
#include "qn_ptx.cuh"

namespace qn {

namespace {

constexpr int BM = 128;
constexpr int BN_MAX = 256;
constexpr int kEpiWarps = 16;                      // four warps per TMEM lane quadrant
constexpr int kEpiParts = kEpiWarps / 4;            // column ranges per quadrant
constexpr int kChunk = 16;                          // accumulator columns per TMEM load
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kMaxStages = 8;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr uint32_t kCtrlBytes = 512;
constexpr uint32_t kTmemCols = 2 * BN_MAX;         // two accumulators of BN_MAX FP32 columns

// B rows per pipeline stage: backward split tiles (MODE 2) are at most 128
// rows wide, so their stages are 64 KB and three fit in shared memory
__host__ __device__ constexpr int bn_slot(int mode) { return mode == 2 ? 128 : BN_MAX; }

// Test-only fault injection (qn_test_withhold_arrival): when set, the TMA producer of
// block 0 of the next launch takes it (atomically, so one launch is affected) and skips
// its first stage, whose full barrier then never completes; the MMA issuer and the
// epilogue give up after kTimeoutNs and report QN_ETIMEOUT. Nothing is left in flight:
// no MMA was issued and the other stages' loads are drained.
__device__ int g_tc_withhold = 0;

// Wait for `parity` on `bar`; false on timeout or when another role aborted.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                         int *err) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer();
    while (true) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (ptx::globaltimer() - t0 > kTimeoutNs) {
            *abort_flag = 1;
            atomicExch(err, QN_ETIMEOUT);
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag (used while draining after an abort).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = ptx::globaltimer();
    while (!ptx::mbar_try_wait(bar, parity)) {
        if (ptx::globaltimer() - t0 > kTimeoutNs) return;
    }
}

__device__ __forceinline__ void split_store(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int o) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Three levels: each the BF16 rounding of what the previous levels leave (the
// remainders are exact in FP32), 8 + 8 + 8 significant bits.
__device__ __forceinline__ void split_store3(float v, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                             __nv_bfloat16 *l2, int o) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    hi[o] = h;
    lo[o] = m;
    l2[o] = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// The third levels of the six-product launches (single-group reflection-split products
// only; a separate kernel argument, so the group records of every launch keep one layout).
struct TcL3 {
    const CUtensorMap *a_l2, *b_l2;   // third operand levels of A and B
    __nv_bfloat16 *out_l2;            // third output level
};

// Store one output value as two or three levels.
template <bool L3>
__device__ __forceinline__ void store_lv(float v, const TcGroup &G, const TcL3 &l3, int o) {
    if (L3)
        split_store3(v, G.out_hi, G.out_lo, l3.out_l2, o);
    else
        split_store(v, G.out_hi, G.out_lo, o);
}

// Group and tile origin of tile t: single-group launches enumerate the tiles
// of `g0` (m-major); grouped launches read the tile table.
__device__ __forceinline__ void tile_info(int t, const TcGroup &g0, const TcGroup *groups,
                                          const TcTile *tiles, TcGroup &G, int &m0, int &n0) {
    if (groups == nullptr) {
        G = g0;
        m0 = (t / g0.ntile_n) * BM;
        n0 = (t % g0.ntile_n) * g0.BN;
    } else {
        const TcTile T = tiles[t];
        G = groups[T.group];
        m0 = T.m0;
        n0 = T.n0;
    }
}

__device__ __forceinline__ bool group_done(const TcGroup &G) {
    return G.done != nullptr && *(volatile const int *)G.done;
}

// 576 threads, one CTA per SM. The register file is split over the SM's four
// sub-partitions of 16384 registers and 18 warps put five on two of them, so a thread may
// hold at most 96 registers (five warps x 32 threads x 96 <= 16384; a 104-register kernel
// of this block size is refused at launch). Every instantiation below compiles to at most
// 96 under the cap of 104 (ptxas -v).
static_assert(5 * 32 * 96 <= 16384 && (kThreads / 32 + 3) / 4 == 5, "register file");

template <int BK, int EPI, int DIM, int MODE, bool L3 = false>
__global__ void __maxnreg__(104)
    k_modeprod_tc(const TcGroup g0, const TcGroup *__restrict__ groups, const TcTile *__restrict__ tiles,
                  const int ntiles, const int stages, int *err, const TcL3 l3) {
    if (groups == nullptr && group_done(g0)) return;

    constexpr uint32_t kRowBytes = BK * 2;                // one swizzle row per tile row
    constexpr uint32_t kLayout = (BK == 64) ? 2u : 4u;    // 128-B : 64-B swizzle
    constexpr int kKSteps = BK / 16;
    constexpr uint32_t a_bytes = BM * kRowBytes;
    constexpr uint32_t b_bytes_max = bn_slot(MODE) * kRowBytes;
    // operand levels in shared memory: three for the six-product backward products
    constexpr bool IN3 = L3 && MODE == 2;
    constexpr uint32_t kLv = IN3 ? 3u : 2u;
    constexpr uint32_t b_off = kLv * a_bytes;   // B levels follow the A levels
    constexpr uint32_t stage_bytes = kLv * a_bytes + kLv * b_bytes_max;
    static_assert(!L3 || (MODE == 1 && EPI == EPI_DIVIDE) || MODE == 2, "three levels: divide or backward");

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = ptx::smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t ctrl = base + (uint32_t)stages * stage_bytes;
    // control block: full[8], empty[8], tfull[2], tempty[2], mma_done, tmem slot, abort
    auto full_bar = [&](int s) { return ctrl + 8u * s; };
    auto empty_bar = [&](int s) { return ctrl + 64u + 8u * s; };
    auto tfull_bar = [&](int b) { return ctrl + 128u + 8u * b; };
    auto tempty_bar = [&](int b) { return ctrl + 144u + 8u * b; };
    const uint32_t mma_done_bar = ctrl + 160u;
    const uint32_t tmem_slot = ctrl + 168u;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem_raw + (ctrl + 172u - raw));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            ptx::mbar_init(full_bar(s), 1);
            ptx::mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(tfull_bar(b), 1);
            ptx::mbar_init(tempty_bar(b), kEpiWarps);
        }
        ptx::mbar_init(mma_done_bar, 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
        ptx::fence_proxy_async();
        if (groups == nullptr) {
            ptx::prefetch_tensormap(g0.a_hi);
            ptx::prefetch_tensormap(g0.a_lo);
            ptx::prefetch_tensormap(g0.b_hi);
            ptx::prefetch_tensormap(g0.b_lo);
        }
    }
    if (warp == 1) {
        ptx::tmem_alloc(tmem_slot, kTmemCols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(smem_raw + (tmem_slot - raw));

    if (warp == 0 && lane == 0) {
        // ------------------------------ TMA producer ------------------------------
        uint32_t armed_parity[kMaxStages];
        uint32_t armed_mask = 0;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        bool withhold = (blockIdx.x == 0) && atomicExch(&g_tc_withhold, 0) != 0;
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            TcGroup G;
            int m0, n0;
            tile_info(t, g0, groups, tiles, G, m0, n0);
            if (group_done(G)) continue;
            const uint32_t tx_bytes = kLv * (a_bytes + (uint32_t)G.BN * kRowBytes);
            const int Hh = G.P >> 1, KBh = Hh / BK;
            const int KB = (MODE == 0) ? G.P / BK : (MODE == 1 ? KBh : 2 * KBh);
            for (int kb = 0; kb < KB; ++kb) {
                if (!wait_bar(empty_bar(s), ph ^ 1u, abort_flag, err)) {
                    ok = false;
                    break;
                }
                // A column (contraction) and B row coordinates of this K step
                int ax = kb * BK, bx = kb * BK, by = n0;
                if (MODE == 1) ax = (n0 >= Hh ? Hh : 0) + kb * BK;
                if (MODE == 2) {
                    const bool second = kb >= KBh;
                    bx = (second ? kb - KBh : kb) * BK;
                    ax = (second ? Hh : 0) + bx;
                    by = (second ? Hh : 0) + n0;
                }
                const uint32_t st = base + (uint32_t)s * stage_bytes;
                if (withhold) {   // test-only: this stage is never armed
                    withhold = false;
                } else {
                    ptx::mbar_arrive_expect_tx(full_bar(s), tx_bytes);
                    ptx::tma_load_2d(st, G.a_hi, full_bar(s), ax, m0);
                    ptx::tma_load_2d(st + a_bytes, G.a_lo, full_bar(s), ax, m0);
                    if (IN3) ptx::tma_load_2d(st + 2 * a_bytes, l3.a_l2, full_bar(s), ax, m0);
                    ptx::tma_load_2d(st + b_off, G.b_hi, full_bar(s), bx, by);
                    ptx::tma_load_2d(st + b_off + b_bytes_max, G.b_lo, full_bar(s), bx, by);
                    if (IN3) ptx::tma_load_2d(st + b_off + 2 * b_bytes_max, l3.b_l2, full_bar(s), bx, by);
                    armed_parity[s] = ph;
                    armed_mask |= 1u << s;
                }
                if (++s == stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        if (!ok) {
            for (int i = 0; i < stages; ++i)
                if (armed_mask & (1u << i)) drain_bar(full_bar(i), armed_parity[i]);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------ MMA issuer --------------------------------
        int s = 0;
        uint32_t ph = 0;
        int acc = 0;
        uint32_t aph = 0;
        bool ok = true;
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            TcGroup G;
            int m0, n0;
            tile_info(t, g0, groups, tiles, G, m0, n0);
            if (group_done(G)) continue;
            const uint32_t idesc = ptx::idesc_bf16_f32(BM, (uint32_t)G.BN);
            const int KBh = (G.P >> 1) / BK;
            const int KB = (MODE == 0) ? G.P / BK : (MODE == 1 ? KBh : 2 * KBh);
            if (!wait_bar(tempty_bar(acc), aph ^ 1u, abort_flag, err)) break;
            ptx::tc_fence_after();
            for (int kb = 0; kb < KB; ++kb) {
                // MODE 2: the second half of the K steps accumulates q, BN columns further on
                const bool second = (MODE == 2) && kb >= KBh;
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN_MAX + (second ? G.BN : 0));
                const int kb0 = second ? kb - KBh : kb;
                if (!wait_bar(full_bar(s), ph, abort_flag, err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t st = base + (uint32_t)s * stage_bytes;
#pragma unroll
                for (int kk = 0; kk < kKSteps; ++kk) {
                    const uint32_t koff = (uint32_t)kk * 32u;
                    const uint64_t a_hi = ptx::smem_desc_kmajor(st + koff, kRowBytes, kLayout);
                    const uint64_t a_lo = ptx::smem_desc_kmajor(st + a_bytes + koff, kRowBytes, kLayout);
                    const uint64_t b_hi = ptx::smem_desc_kmajor(st + b_off + koff, kRowBytes, kLayout);
                    const uint64_t b_lo =
                        ptx::smem_desc_kmajor(st + b_off + b_bytes_max + koff, kRowBytes, kLayout);
                    const uint32_t first = (kb0 == 0 && kk == 0) ? 0u : 1u;
                    ptx::mma_bf16(d_tmem, a_hi, b_hi, idesc, first);
                    ptx::mma_bf16(d_tmem, a_hi, b_lo, idesc, 1u);
                    ptx::mma_bf16(d_tmem, a_lo, b_hi, idesc, 1u);
                    if (IN3) {
                        const uint64_t a_l2 = ptx::smem_desc_kmajor(st + 2 * a_bytes + koff, kRowBytes, kLayout);
                        const uint64_t b_l2 =
                            ptx::smem_desc_kmajor(st + b_off + 2 * b_bytes_max + koff, kRowBytes, kLayout);
                        ptx::mma_bf16(d_tmem, a_lo, b_lo, idesc, 1u);
                        ptx::mma_bf16(d_tmem, a_hi, b_l2, idesc, 1u);
                        ptx::mma_bf16(d_tmem, a_l2, b_hi, idesc, 1u);
                    }
                }
                ptx::mma_commit(empty_bar(s));
                if (++s == stages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            ptx::mma_commit(tfull_bar(acc));
            acc ^= 1;
            if (acc == 0) aph ^= 1u;
        }
        ptx::mma_commit(mma_done_bar);
        drain_bar(mma_done_bar, 0);
    } else if (warp >= 2) {
        // ------------------------------ epilogue ----------------------------------
        const int q = warp & 3;                          // TMEM lanes 32q..32q+31 = tile rows
        const int part = (warp - 2) >> 2;                // which of the kEpiParts column ranges
        const int row = q * 32 + lane;
        int acc = 0;
        uint32_t aph = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            TcGroup G;
            int m0, n0;
            tile_info(t, g0, groups, tiles, G, m0, n0);
            if (group_done(G)) continue;
            // every lane waits; the decision to go on is made warp-uniform so
            // that the .sync.aligned TMEM loads below are never divergent
            const bool ready = wait_bar(tfull_bar(acc), aph, abort_flag, err);
            if (!__all_sync(0xffffffffu, ready)) break;
            ptx::tc_fence_after();
            const int P = G.P, n = G.n, BN = G.BN;
            const int Mtot = G.Mtot;
            const int m = m0 + row;
            const bool m_ok = m < Mtot;
            float rowlam = 0.0f, shift = 0.0f;
            int ubase = -1;   // dense U index without the k term (UPDATE/DENSE)
            if (m_ok) {
                if (EPI == EPI_DIVIDE) {
                    rowlam = (DIM == 3) ? __ldg(G.lam32 + m / P) + __ldg(G.lam32 + m % P) : __ldg(G.lam32 + m);
                    shift = (float)(*G.shift);
                }
                if (EPI == EPI_UPDATE || EPI == EPI_DENSE || EPI == EPI_UPDATE_PQ) {
                    if (DIM == 3) {
                        const int yy = m / P, xx = m % P;
                        if (yy < n && xx < n) ubase = yy * n + xx;
                    } else {
                        if (m < n) ubase = m;
                    }
                }
            }
            const int kstride = (DIM == 3) ? n * n : n;
            const float dscale = G.dscale;
            const float step = G.step;
            const int cols = BN / kEpiParts;   // >= 16: BN is 64, 128 or 256
            const int cbeg = part * cols, cend = cbeg + cols;
            float dsq_acc = 0.0f;   // sum of squared updates (G.dsq)
            const int Hh = P >> 1;
            const int nsym = (n + 1) >> 1, nanti = n >> 1;
            const uint32_t tacc = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN_MAX);
            if (EPI == EPI_STORE_BFLY) {
                // row m = (slow, F): F = 2i holds spatial i, F = 2i+1 its mirror n-1-i
                // (adjacent lanes); the even lane writes a_i at position i, the odd
                // lane b_i at H + i of the next product's split-order axis (zeros in
                // the padding of either half)
                const int F = m % P, slow = m / P, i2 = F >> 1;
                const bool odd = (F & 1) != 0;
                const bool valid = odd ? (i2 < nanti) : (i2 < nsym);
                const int obase = slow * P + (odd ? Hh + i2 : i2);
                for (int c = cbeg; c < cend; c += kChunk) {
                    uint32_t r[kChunk];
                    ptx::tmem_ld_32x32b_x16(tacc + (uint32_t)c, r);
                    ptx::tmem_ld_wait();
                    const int k0 = n0 + c;
#pragma unroll
                    for (int i = 0; i < kChunk; ++i) {
                        const float v = __uint_as_float(r[i]);
                        const float pv = __shfl_xor_sync(0xffffffffu, v, 1);
                        const float o = valid ? (odd ? pv - v : v + pv) : 0.0f;
                        if (k0 + i < P) split_store(o, G.out_hi, G.out_lo, (k0 + i) * Mtot + obase);
                    }
                }
            }
            if (EPI == EPI_STORE_PQ) {
                // p in columns [0, BN), q in [BN, 2 BN) of the accumulator; output
                // rows j (< H) and n-1-j; the middle row of an odd n takes p alone
                for (int c = cbeg; c < cend; c += kChunk) {
                    uint32_t rp[kChunk], rq[kChunk];
                    ptx::tmem_ld_32x32b_x16(tacc + (uint32_t)c, rp);
                    ptx::tmem_ld_32x32b_x16(tacc + (uint32_t)(BN + c), rq);
                    ptx::tmem_ld_wait();
                    if (!m_ok) continue;
                    const int j0 = n0 + c;
#pragma unroll
                    for (int i = 0; i < kChunk; ++i) {
                        if (c + i >= cend) break;   // BN2/kEpiParts may be 24 (P = 384): half a chunk
                        const int j = j0 + i;
                        const float p = __uint_as_float(rp[i]), qv = __uint_as_float(rq[i]);
                        if (j < nanti) {
                            store_lv<L3>(p + qv, G, l3, j * Mtot + m);
                            store_lv<L3>(p - qv, G, l3, (n - 1 - j) * Mtot + m);
                        } else if (j < nsym) {
                            store_lv<L3>(p, G, l3, j * Mtot + m);
                        }
                    }
                }
            }
            if (EPI == EPI_UPDATE_PQ) {
                // as EPI_STORE_PQ, the two rows subtracted from U (8 columns at a
                // time: two FP64 rows of old values per chunk)
                for (int c = cbeg; c < cend; c += 8) {
                    uint32_t rp[8], rq[8];
                    ptx::tmem_ld_32x32b_x8(tacc + (uint32_t)c, rp);
                    ptx::tmem_ld_32x32b_x8(tacc + (uint32_t)(BN + c), rq);
                    ptx::tmem_ld_wait();
                    if (!m_ok) continue;
                    const int j0 = n0 + c;
                    if (ubase >= 0) {
                        double *ub = G.U + ubase;
                        double oa[8], ob[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int j = j0 + i;
                            oa[i] = (j < nsym) ? ub[j * kstride] : 0.0;
                            ob[i] = (j < nanti) ? ub[(n - 1 - j) * kstride] : 0.0;
                        }
                        const double st = (double)step;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int j = j0 + i;
                            const float p = __uint_as_float(rp[i]), qv = __uint_as_float(rq[i]);
                            const float xa = (j < nanti) ? p + qv : p, xb = p - qv;
                            if (j < nsym) dsq_acc = fmaf(xa, xa, dsq_acc);
                            if (j < nanti) dsq_acc = fmaf(xb, xb, dsq_acc);
                            if (j < nsym)
                                ub[j * kstride] = (step == 1.0f) ? oa[i] - f2d_exact(xa) : fma(-st, f2d_exact(xa), oa[i]);
                            if (j < nanti)
                                ub[(n - 1 - j) * kstride] =
                                    (step == 1.0f) ? ob[i] - f2d_exact(xb) : fma(-st, f2d_exact(xb), ob[i]);
                        }
                    }
                }
            }
            for (int c = cbeg; EPI <= EPI_DENSE && c < cend; c += kChunk) {
                uint32_t r[kChunk];
                ptx::tmem_ld_32x32b_x16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN_MAX + c), r);
                ptx::tmem_ld_wait();
                if (!m_ok) continue;
                const int k0 = n0 + c;
                if (EPI == EPI_STORE) {
#pragma unroll
                    for (int i = 0; i < kChunk; ++i)
                        if (k0 + i < P) split_store(__uint_as_float(r[i]), G.out_hi, G.out_lo, (k0 + i) * Mtot + m);
                } else if (EPI == EPI_DIVIDE) {
#pragma unroll
                    for (int i = 0; i < kChunk; ++i) {
                        const int k = k0 + i;
                        if (k < P) {
                            const float den = dscale * (__ldg(G.lam32 + k) + rowlam) + shift;
                            store_lv<L3>(__fdividef(__uint_as_float(r[i]), den), G, l3, k * Mtot + m);
                        }
                    }
                } else if (EPI == EPI_UPDATE) {
                    if (ubase >= 0) {
                        // the chunk's 16 loads of U in flight before its stores,
                        // instead of a serial read-modify-write
                        double *ub = G.U + ubase;
                        // the next chunk's U lines are requested into L2 now
                        // (no registers), its loads then hit L2
                        if (c + kChunk < cend) {
#pragma unroll
                            for (int i = 0; i < kChunk; ++i)
                                if (k0 + kChunk + i < n) ptx::prefetch_l2(ub + (k0 + kChunk + i) * kstride);
                        }
                        double old[kChunk];
#pragma unroll
                        for (int i = 0; i < kChunk; ++i) old[i] = (k0 + i < n) ? ub[(k0 + i) * kstride] : 0.0;
#pragma unroll
                        for (int i = 0; i < kChunk; ++i) {
                            const float x = __uint_as_float(r[i]);
                            if (k0 + i < n) dsq_acc = fmaf(x, x, dsq_acc);
                        }
                        if (step == 1.0f) {
#pragma unroll
                            for (int i = 0; i < kChunk; ++i)
                                if (k0 + i < n) ub[(k0 + i) * kstride] = old[i] - f2d_exact(__uint_as_float(r[i]));
                        } else {
                            const double st = (double)step;
#pragma unroll
                            for (int i = 0; i < kChunk; ++i)
                                if (k0 + i < n)
                                    ub[(k0 + i) * kstride] = fma(-st, f2d_exact(__uint_as_float(r[i])), old[i]);
                        }
                    }
                } else {   // EPI_DENSE
                    if (ubase >= 0) {
                        double *ub = G.U + ubase;
#pragma unroll
                        for (int i = 0; i < kChunk; ++i)
                            if (k0 + i < n) ub[(k0 + i) * kstride] = f2d_exact(__uint_as_float(r[i]));
                    }
                }
            }
            if ((EPI == EPI_UPDATE || EPI == EPI_UPDATE_PQ) && G.dsq != nullptr) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsq_acc += __shfl_xor_sync(0xffffffffu, dsq_acc, o);
                if (lane == 0) atomicAdd(G.dsq, dsq_acc * step * step);
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(tempty_bar(acc));
            acc ^= 1;
            if (acc == 0) aph ^= 1u;
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcPlan {
    int n, P, dim, Mtot, BN, ntile_n, ntiles, grid, stages, BK;
    int split, BN1, BN2, num_sms;   // reflection-split products: forward / backward tile widths
    size_t smem;
    int x6;              // tc_plan_enable_x6 done
    int fused;           // tc_plan_enable_fused done
    const __nv_bfloat16 *bf_hi, *bf_lo;   // the forward split matrix [P][P/2] (tc_plan_enable_split)
    CUtensorMap *maps;   // device: a_hi[2], a_lo[2], s_hi, s_lo, si_hi, si_lo, bf_hi, bf_lo, bb_hi, bb_lo,
                         // a_l2[2], bb_l2, and the fused kernel's bf_hi, bf_lo (kPlanMaps entries)
    __nv_bfloat16 *bufs_hi[2];
    __nv_bfloat16 *bufs_lo[2];
    __nv_bfloat16 *bufs_l2[2];
};

constexpr int kPlanMaps = 18;

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return fn;
}

int tc_encode_2d(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                 uint32_t box_outer, int BK) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled unavailable from the driver");
        return QN_ECUDA;
    }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for %llux%llu box %ux%u", (int)r,
                  (unsigned long long)inner, (unsigned long long)outer, box_inner, box_outer);
        return QN_ECUDA;
    }
    return QN_OK;
}

bool tc_supported(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return false;
    return p.major == 10 && p.minor == 3;
}

// levels: operand levels per stage (3 for the six-product backward products)
static size_t smem_bytes_mode(int BK, int stages, int mode, int levels = 2) {
    const size_t stage = (size_t)levels * (BM + bn_slot(mode)) * BK * 2;
    return 1024 + stage * stages + kCtrlBytes;
}

size_t tc_smem_bytes(int BK, int stages) { return smem_bytes_mode(BK, stages, 0); }

static int stages_mode(int BK, int mode, int levels = 2) {
    const size_t budget = 227 * 1024;
    int stages = kMaxStages;
    while (stages > 2 && smem_bytes_mode(BK, stages, mode, levels) > budget) --stages;
    return stages;
}

int tc_stages(int BK) {
    const size_t budget = 227 * 1024;
    int stages = kMaxStages;
    while (stages > 2 && tc_smem_bytes(BK, stages) > budget) --stages;
    const char *st_env = getenv("QN_TC_STAGES");
    if (st_env && atoi(st_env) >= 2 && atoi(st_env) < stages) stages = atoi(st_env);
    return stages;
}

int tc_plan_create(TcPlan **out, int n, int P, int dim, __nv_bfloat16 *bufs_hi[2],
                   __nv_bfloat16 *bufs_lo[2], const __nv_bfloat16 *S_hi, const __nv_bfloat16 *S_lo,
                   const __nv_bfloat16 *Si_hi, const __nv_bfloat16 *Si_lo, int num_sms) {
    TcPlan *p = (TcPlan *)calloc(1, sizeof(TcPlan));
    if (!p) return QN_ENOMEM;
    p->n = n;
    p->P = P;
    p->dim = dim;
    p->Mtot = (dim == 3) ? P * P : P;
    p->BN = P <= BN_MAX ? P : BN_MAX;
    p->ntile_n = (P + p->BN - 1) / p->BN;
    p->ntiles = p->ntile_n * ((p->Mtot + BM - 1) / BM);
    const char *bk_env = getenv("QN_TC_BK");
    p->BK = (bk_env && atoi(bk_env) == 32) ? 32 : 64;
    p->stages = tc_stages(p->BK);
    p->smem = tc_smem_bytes(p->BK, p->stages);
    p->grid = p->ntiles < num_sms ? p->ntiles : num_sms;
    p->num_sms = num_sms;
    if (tc_set_attributes() != QN_OK) {
        free(p);
        return QN_ECUDA;
    }
    CUtensorMap h[kPlanMaps];
    memset(h, 0, sizeof(h));
    int rc = QN_OK;
    for (int b = 0; b < 2 && rc == QN_OK; ++b) {
        p->bufs_hi[b] = bufs_hi[b];
        p->bufs_lo[b] = bufs_lo[b];
        rc = tc_encode_2d(&h[b], bufs_hi[b], P, p->Mtot, p->BK, BM, p->BK);
        if (rc == QN_OK) rc = tc_encode_2d(&h[2 + b], bufs_lo[b], P, p->Mtot, p->BK, BM, p->BK);
    }
    if (rc == QN_OK) rc = tc_encode_2d(&h[4], S_hi, P, P, p->BK, p->BN, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[5], S_lo, P, P, p->BK, p->BN, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[6], Si_hi, P, P, p->BK, p->BN, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[7], Si_lo, P, P, p->BK, p->BN, p->BK);
    if (rc == QN_OK && cudaMalloc(&p->maps, sizeof(h)) != cudaSuccess) rc = QN_ENOMEM;
    if (rc == QN_OK && cudaMemcpy(p->maps, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) rc = QN_ECUDA;
    if (rc != QN_OK) {
        if (p->maps) cudaFree(p->maps);
        free(p);
        return rc;
    }
    *out = p;
    return QN_OK;
}

int tc_plan_enable_split(TcPlan *p, const __nv_bfloat16 *bf_hi, const __nv_bfloat16 *bf_lo,
                         const __nv_bfloat16 *bb_hi, const __nv_bfloat16 *bb_lo) {
    const int H = p->P / 2;
    if (p->dim != 3 || p->P % 128 != 0) return QN_EUNSUPPORTED;
    // tile widths must divide H (a forward tile stays inside one half; the
    // backward tiles cover the H rows exactly) and give every epilogue warp a
    // whole number of TMEM chunks: BN1/kEpiParts a multiple of kChunk (16),
    // BN2/kEpiParts a multiple of 8; BN2 <= 128 (two accumulators per tile)
    p->BN1 = 0;
    for (int bn = BN_MAX; bn >= 16 * kEpiParts; bn -= 16 * kEpiParts)
        if (H % bn == 0) {
            p->BN1 = bn;
            break;
        }
    p->BN2 = 0;
    for (int bn = 128; bn >= 8 * kEpiParts; bn -= 8 * kEpiParts)
        if (H % bn == 0) {
            p->BN2 = bn;
            break;
        }
    if (p->BN1 == 0 || p->BN2 == 0) return QN_EUNSUPPORTED;
    CUtensorMap h[4];
    int rc = tc_encode_2d(&h[0], bf_hi, H, p->P, p->BK, p->BN1, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[1], bf_lo, H, p->P, p->BK, p->BN1, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[2], bb_hi, H, p->P, p->BK, p->BN2, p->BK);
    if (rc == QN_OK) rc = tc_encode_2d(&h[3], bb_lo, H, p->P, p->BK, p->BN2, p->BK);
    if (rc != QN_OK) return rc;
    QN_CUDA(cudaMemcpy(p->maps + 8, h, sizeof(h), cudaMemcpyHostToDevice));
    p->bf_hi = bf_hi;
    p->bf_lo = bf_lo;
    p->split = 1;
    return QN_OK;
}

int tc_plan_enable_fused(TcPlan *p) {
    if (p == nullptr || !p->split || p->P > 512) return QN_EUNSUPPORTED;
    if (p->fused) return QN_OK;
    const int H = p->P / 2;
    CUtensorMap h[2];
    int rc = tc_encode_2d(&h[0], p->bf_hi, H, p->P, 32, H, 32);
    if (rc == QN_OK) rc = tc_encode_2d(&h[1], p->bf_lo, H, p->P, 32, H, 32);
    if (rc == QN_OK) rc = fused_set_attributes();
    if (rc != QN_OK) return rc;
    QN_CUDA(cudaMemcpy(p->maps + 16, h, sizeof(h), cudaMemcpyHostToDevice));
    p->fused = 1;
    return QN_OK;
}

int tc_plan_fused_args(const TcPlan *p, int dst, int *err, FusedFwd *out) {
    if (p == nullptr || !p->fused || dst < 0 || dst > 1) return QN_EUNSUPPORTED;
    out->b_hi = p->maps + 16;
    out->b_lo = p->maps + 17;
    out->out_hi = p->bufs_hi[dst];
    out->out_lo = p->bufs_lo[dst];
    out->err = err;
    out->num_sms = p->num_sms;
    return QN_OK;
}

bool tc_plan_has_split(const TcPlan *p) { return p != nullptr && p->split; }

int tc_plan_enable_x6(TcPlan *p, __nv_bfloat16 *bufs_l2[2], const __nv_bfloat16 *bb_l2) {
    if (!p->split) return QN_EUNSUPPORTED;
    const int H = p->P / 2;
    CUtensorMap h[3];
    memset(h, 0, sizeof(h));
    int rc = QN_OK;
    for (int b = 0; b < 2 && rc == QN_OK; ++b) {
        p->bufs_l2[b] = bufs_l2[b];
        rc = tc_encode_2d(&h[b], bufs_l2[b], p->P, p->Mtot, p->BK, BM, p->BK);
    }
    if (rc == QN_OK) rc = tc_encode_2d(&h[2], bb_l2, H, p->P, p->BK, p->BN2, p->BK);
    if (rc != QN_OK) return rc;
    QN_CUDA(cudaMemcpy(p->maps + 12, h, sizeof(h), cudaMemcpyHostToDevice));
    p->x6 = 1;
    return QN_OK;
}

void tc_plan_destroy(TcPlan *plan) {
    if (!plan) return;
    cudaFree(plan->maps);
    free(plan);
}

template <int BK, int EPI, int DIM, int MODE = 0, bool L3 = false>
static int launch_t(const TcGroup &g0, const TcGroup *groups, const TcTile *tiles, int ntiles, int stages,
                    int *err, int grid, cudaStream_t s, const TcL3 &l3 = TcL3{nullptr, nullptr, nullptr}) {
    auto kern = k_modeprod_tc<BK, EPI, DIM, MODE, L3>;
    const int levels = (L3 && MODE == 2) ? 3 : 2;
    kern<<<grid, kThreads, smem_bytes_mode(BK, stages, MODE, levels), s>>>(g0, groups, tiles, ntiles, stages, err,
                                                                           l3);
    QN_CUDA(cudaGetLastError());
    return QN_OK;
}

template <int BK, int DIM>
static int launch_epi(Epi epi, const TcGroup &g0, const TcGroup *groups, const TcTile *tiles, int ntiles,
                      int stages, int *err, int grid, cudaStream_t s) {
    switch (epi) {
        case EPI_STORE: return launch_t<BK, EPI_STORE, DIM>(g0, groups, tiles, ntiles, stages, err, grid, s);
        case EPI_DIVIDE: return launch_t<BK, EPI_DIVIDE, DIM>(g0, groups, tiles, ntiles, stages, err, grid, s);
        case EPI_UPDATE: return launch_t<BK, EPI_UPDATE, DIM>(g0, groups, tiles, ntiles, stages, err, grid, s);
        case EPI_DENSE: return launch_t<BK, EPI_DENSE, DIM>(g0, groups, tiles, ntiles, stages, err, grid, s);
    }
    return QN_EINVAL;
}

static int launch_any(int BK, int dim, Epi epi, const TcGroup &g0, const TcGroup *groups, const TcTile *tiles,
                      int ntiles, int stages, int *err, int grid, cudaStream_t s) {
    if (BK == 64)
        return dim == 3 ? launch_epi<64, 3>(epi, g0, groups, tiles, ntiles, stages, err, grid, s)
                        : launch_epi<64, 2>(epi, g0, groups, tiles, ntiles, stages, err, grid, s);
    return dim == 3 ? launch_epi<32, 3>(epi, g0, groups, tiles, ntiles, stages, err, grid, s)
                    : launch_epi<32, 2>(epi, g0, groups, tiles, ntiles, stages, err, grid, s);
}

template <int BK, int EPI, int DIM, int MODE = 0, bool L3 = false>
static int set_attr_one() {
    QN_CUDA(cudaFuncSetAttribute(k_modeprod_tc<BK, EPI, DIM, MODE, L3>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    return QN_OK;
}

template <int BK, int DIM>
static int set_attr_dim() {
    int rc = set_attr_one<BK, EPI_STORE, DIM>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_DIVIDE, DIM>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_UPDATE, DIM>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_DENSE, DIM>();
    return rc;
}

template <int BK>
static int set_attr_split() {
    int rc = set_attr_one<BK, EPI_STORE_BFLY, 3, 1>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_DIVIDE, 3, 1>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_STORE_PQ, 3, 2>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_UPDATE_PQ, 3, 2>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_DIVIDE, 3, 1, true>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_STORE_PQ, 3, 2, true>();
    if (rc == QN_OK) rc = set_attr_one<BK, EPI_UPDATE_PQ, 3, 2, true>();
    return rc;
}

// Opt every instantiation in to the large dynamic shared memory once (before
// any launch, so that launches can be captured into CUDA graphs).
int tc_set_attributes() {
    int rc = set_attr_dim<64, 2>();
    if (rc == QN_OK) rc = set_attr_dim<64, 3>();
    if (rc == QN_OK) rc = set_attr_dim<32, 2>();
    if (rc == QN_OK) rc = set_attr_dim<32, 3>();
    if (rc == QN_OK) rc = set_attr_split<64>();
    if (rc == QN_OK) rc = set_attr_split<32>();
    return rc;
}

template <int BK>
static int split_launch(const TcPlan *p, const TcGroup &g, const TcL3 &l3, Epi epi, bool x6, int *err, int grid,
                        cudaStream_t s) {
    if (x6 && epi != EPI_STORE_BFLY) {
        // the divide writes three levels; the backward products read and write three
        const int st3 = stages_mode(BK, 2, 3);
        switch (epi) {
            case EPI_DIVIDE:
                return launch_t<BK, EPI_DIVIDE, 3, 1, true>(g, nullptr, nullptr, g.ntiles, p->stages, err, grid, s, l3);
            case EPI_STORE_PQ:
                return launch_t<BK, EPI_STORE_PQ, 3, 2, true>(g, nullptr, nullptr, g.ntiles, st3, err, grid, s, l3);
            default:
                return launch_t<BK, EPI_UPDATE_PQ, 3, 2, true>(g, nullptr, nullptr, g.ntiles, st3, err, grid, s, l3);
        }
    }
    const int st2 = stages_mode(BK, 2);
    switch (epi) {
        case EPI_STORE_BFLY:
            return launch_t<BK, EPI_STORE_BFLY, 3, 1>(g, nullptr, nullptr, g.ntiles, p->stages, err, grid, s);
        case EPI_DIVIDE:
            return launch_t<BK, EPI_DIVIDE, 3, 1>(g, nullptr, nullptr, g.ntiles, p->stages, err, grid, s);
        case EPI_STORE_PQ:
            return launch_t<BK, EPI_STORE_PQ, 3, 2>(g, nullptr, nullptr, g.ntiles, st2, err, grid, s);
        default:
            return launch_t<BK, EPI_UPDATE_PQ, 3, 2>(g, nullptr, nullptr, g.ntiles, st2, err, grid, s);
    }
}

int launch_modeprod_tc_split(TcPlan *p, int src, int dst, Epi epi, const EpiArgs &e, cudaStream_t s, bool x6) {
    if (!p->split) {
        set_error("launch_modeprod_tc_split: the plan has no reflection-split matrices");
        return QN_EINVAL;
    }
    if (x6 && !p->x6) {
        set_error("launch_modeprod_tc_split: the plan has no six-product level");
        return QN_EINVAL;
    }
    const bool fwd = (epi == EPI_STORE_BFLY || epi == EPI_DIVIDE);
    if (!fwd && epi != EPI_STORE_PQ && epi != EPI_UPDATE_PQ) {
        set_error("launch_modeprod_tc_split: epilogue %d is not a reflection-split one", (int)epi);
        return QN_EINVAL;
    }
    TcGroup g;
    memset(&g, 0, sizeof(g));
    g.a_hi = p->maps + src;
    g.a_lo = p->maps + 2 + src;
    g.b_hi = p->maps + (fwd ? 8 : 10);
    g.b_lo = p->maps + (fwd ? 9 : 11);
    g.out_hi = (dst >= 0) ? p->bufs_hi[dst] : nullptr;
    g.out_lo = (dst >= 0) ? p->bufs_lo[dst] : nullptr;
    TcL3 l3{nullptr, nullptr, nullptr};
    if (x6) {
        l3.a_l2 = p->maps + 12 + src;
        l3.b_l2 = p->maps + 14;
        l3.out_l2 = (dst >= 0) ? p->bufs_l2[dst] : nullptr;
    }
    g.U = e.U;
    g.dsq = e.dsq;
    g.lam32 = e.lam32;
    g.shift = e.shift;
    g.done = e.done;
    g.dscale = 1.0f;
    g.step = (float)e.step;
    g.Mtot = p->Mtot;
    g.P = p->P;
    g.n = p->n;
    g.BN = fwd ? p->BN1 : p->BN2;
    g.ntile_n = fwd ? p->P / p->BN1 : (p->P / 2) / p->BN2;
    g.ntiles = g.ntile_n * (p->Mtot / BM);
    const int grid = g.ntiles < p->num_sms ? g.ntiles : p->num_sms;
    return p->BK == 64 ? split_launch<64>(p, g, l3, epi, x6, e.err, grid, s)
                       : split_launch<32>(p, g, l3, epi, x6, e.err, grid, s);
}

int launch_modeprod_tc(TcPlan *p, int src, int dst, bool forward, Epi epi, const EpiArgs &e, cudaStream_t s) {
    TcGroup g;
    memset(&g, 0, sizeof(g));
    g.a_hi = p->maps + src;
    g.a_lo = p->maps + 2 + src;
    g.b_hi = p->maps + (forward ? 6 : 4);
    g.b_lo = p->maps + (forward ? 7 : 5);
    g.out_hi = (dst >= 0) ? p->bufs_hi[dst] : nullptr;
    g.out_lo = (dst >= 0) ? p->bufs_lo[dst] : nullptr;
    g.U = e.U;
    g.dsq = e.dsq;
    g.lam32 = e.lam32;
    g.shift = e.shift;
    g.done = e.done;
    g.dscale = 1.0f;
    g.step = (float)e.step;
    g.Mtot = p->Mtot;
    g.P = p->P;
    g.n = p->n;
    g.BN = p->BN;
    g.ntile_n = p->ntile_n;
    g.ntiles = p->ntiles;
    return launch_any(p->BK, p->dim, epi, g, nullptr, nullptr, p->ntiles, p->stages, e.err, p->grid, s);
}

int tc_test_withhold_arrival() {
    const int one = 1;
    QN_CUDA(cudaMemcpyToSymbol(g_tc_withhold, &one, sizeof(int)));
    return QN_OK;
}

int launch_modeprod_tc_grouped(const TcGroup *groups, const TcTile *tiles, int ntiles, int dim, int BK, Epi epi,
                               int *err, int grid, cudaStream_t s) {
    TcGroup dummy;
    memset(&dummy, 0, sizeof(dummy));
    return launch_any(BK, dim, epi, dummy, groups, tiles, ntiles, tc_stages(BK), err, grid, s);
}

}  // namespace qn
