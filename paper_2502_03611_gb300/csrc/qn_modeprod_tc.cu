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
// Kernel organisation (persistent, one CTA of 320 threads per SM):
//   warp 0 lane 0  TMA producer: A_hi, A_lo (128 x BK) and B_hi, B_lo (BN x BK)
//                  tiles per pipeline stage, K-major with 128-B or 64-B swizzle
//   warp 1         allocates TMEM (2 accumulators of BN FP32 columns); lane 0
//                  issues tcgen05.mma (M=128, N=BN, K=16) and commits to mbarriers
//   warps 2..9     epilogue: tcgen05.ld of the accumulator (warp w owns TMEM
//                  lanes 32*(w%4)..+31 = rows and one half of the BN columns),
//                  then store / divide / update
// Tiles are walked in m-major order (consecutive CTAs share the same A rows;
// S stays resident in L2). The epilogue of tile i overlaps the MMAs of tile
// i+1 through the double-buffered accumulators.
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

// 576 threads x 104 registers (one CTA per SM; 112 exceeds the launch limit)
static_assert(kThreads * 104 <= 65536, "register file");

template <int BK, int EPI, int DIM>
__global__ void __maxnreg__(104)
    k_modeprod_tc(const TcGroup g0, const TcGroup *__restrict__ groups, const TcTile *__restrict__ tiles,
                  const int ntiles, const int stages, int *err) {
    if (groups == nullptr && group_done(g0)) return;

    constexpr uint32_t kRowBytes = BK * 2;                // one swizzle row per tile row
    constexpr uint32_t kLayout = (BK == 64) ? 2u : 4u;    // 128-B : 64-B swizzle
    constexpr int kKSteps = BK / 16;
    constexpr uint32_t a_bytes = BM * kRowBytes;
    constexpr uint32_t b_bytes_max = BN_MAX * kRowBytes;
    constexpr uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes_max;

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
        for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
            TcGroup G;
            int m0, n0;
            tile_info(t, g0, groups, tiles, G, m0, n0);
            if (group_done(G)) continue;
            const uint32_t tx_bytes = 2 * a_bytes + 2u * (uint32_t)G.BN * kRowBytes;
            const int KB = G.P / BK;
            for (int kb = 0; kb < KB; ++kb) {
                if (!wait_bar(empty_bar(s), ph ^ 1u, abort_flag, err)) {
                    ok = false;
                    break;
                }
                const uint32_t st = base + (uint32_t)s * stage_bytes;
                ptx::mbar_arrive_expect_tx(full_bar(s), tx_bytes);
                ptx::tma_load_2d(st, G.a_hi, full_bar(s), kb * BK, m0);
                ptx::tma_load_2d(st + a_bytes, G.a_lo, full_bar(s), kb * BK, m0);
                ptx::tma_load_2d(st + 2 * a_bytes, G.b_hi, full_bar(s), kb * BK, n0);
                ptx::tma_load_2d(st + 2 * a_bytes + b_bytes_max, G.b_lo, full_bar(s), kb * BK, n0);
                armed_parity[s] = ph;
                armed_mask |= 1u << s;
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
            const int KB = G.P / BK;
            if (!wait_bar(tempty_bar(acc), aph ^ 1u, abort_flag, err)) break;
            ptx::tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN_MAX);
            for (int kb = 0; kb < KB; ++kb) {
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
                    const uint64_t b_hi = ptx::smem_desc_kmajor(st + 2 * a_bytes + koff, kRowBytes, kLayout);
                    const uint64_t b_lo =
                        ptx::smem_desc_kmajor(st + 2 * a_bytes + b_bytes_max + koff, kRowBytes, kLayout);
                    const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                    ptx::mma_bf16(d_tmem, a_hi, b_hi, idesc, first);
                    ptx::mma_bf16(d_tmem, a_hi, b_lo, idesc, 1u);
                    ptx::mma_bf16(d_tmem, a_lo, b_hi, idesc, 1u);
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
                if (EPI == EPI_UPDATE || EPI == EPI_DENSE) {
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
            for (int c = cbeg; c < cend; c += kChunk) {
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
                            split_store(__fdividef(__uint_as_float(r[i]), den), G.out_hi, G.out_lo, k * Mtot + m);
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
    size_t smem;
    CUtensorMap *maps;   // device: a_hi[2], a_lo[2], s_hi, s_lo, si_hi, si_lo
    __nv_bfloat16 *bufs_hi[2];
    __nv_bfloat16 *bufs_lo[2];
};

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

size_t tc_smem_bytes(int BK, int stages) {
    const size_t stage = (size_t)(2 * BM + 2 * BN_MAX) * BK * 2;
    return 1024 + stage * stages + kCtrlBytes;
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
    if (tc_set_attributes() != QN_OK) {
        free(p);
        return QN_ECUDA;
    }
    CUtensorMap h[8];
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

void tc_plan_destroy(TcPlan *plan) {
    if (!plan) return;
    cudaFree(plan->maps);
    free(plan);
}

template <int BK, int EPI, int DIM>
static int launch_t(const TcGroup &g0, const TcGroup *groups, const TcTile *tiles, int ntiles, int stages,
                    int *err, int grid, cudaStream_t s) {
    auto kern = k_modeprod_tc<BK, EPI, DIM>;
    kern<<<grid, kThreads, tc_smem_bytes(BK, stages), s>>>(g0, groups, tiles, ntiles, stages, err);
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

template <int BK, int DIM>
static int set_attr_dim() {
    QN_CUDA(cudaFuncSetAttribute(k_modeprod_tc<BK, EPI_STORE, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    QN_CUDA(cudaFuncSetAttribute(k_modeprod_tc<BK, EPI_DIVIDE, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    QN_CUDA(cudaFuncSetAttribute(k_modeprod_tc<BK, EPI_UPDATE, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    QN_CUDA(cudaFuncSetAttribute(k_modeprod_tc<BK, EPI_DENSE, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    return QN_OK;
}

// Opt every instantiation in to the large dynamic shared memory once (before
// any launch, so that launches can be captured into CUDA graphs).
int tc_set_attributes() {
    int rc = set_attr_dim<64, 2>();
    if (rc == QN_OK) rc = set_attr_dim<64, 3>();
    if (rc == QN_OK) rc = set_attr_dim<32, 2>();
    if (rc == QN_OK) rc = set_attr_dim<32, 3>();
    return rc;
}

int launch_modeprod_tc(TcPlan *p, int src, int dst, bool forward, Epi epi, const EpiArgs &e, cudaStream_t s) {
    TcGroup g;
    g.a_hi = p->maps + src;
    g.a_lo = p->maps + 2 + src;
    g.b_hi = p->maps + (forward ? 6 : 4);
    g.b_lo = p->maps + (forward ? 7 : 5);
    g.out_hi = (dst >= 0) ? p->bufs_hi[dst] : nullptr;
    g.out_lo = (dst >= 0) ? p->bufs_lo[dst] : nullptr;
    g.U = e.U;
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

int launch_modeprod_tc_grouped(const TcGroup *groups, const TcTile *tiles, int ntiles, int dim, int BK, Epi epi,
                               int *err, int grid, cudaStream_t s) {
    TcGroup dummy;
    memset(&dummy, 0, sizeof(dummy));
    return launch_any(BK, dim, epi, dummy, groups, tiles, ntiles, tc_stages(BK), err, grid, s);
}

}  // namespace qn
