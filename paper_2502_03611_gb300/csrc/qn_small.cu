// Whole-solve persistent kernel for small 2-D FP64 problems (Sec. 4 eq. identity-method
// with the inverse of Sec. 4.1 eq. fin_inverse), n <= kSmallMaxN.
//
// At these sizes every phase of an iteration is a few microseconds of work (the 63^2
// grid has 3969 unknowns; one mode product is 250k FP64 FMAs), so a solve made of
// separate launches is bound by launch and host-check latency. Here one cooperative
// launch runs the whole solve, the phases separated by a grid barrier. Block b owns rows
// b, b + grid, ... of every phase's input: it evaluates the residual on its rows of U, and
// in a product stages its input row in shared memory and forms the n outputs that row
// feeds (the matrix rows come from L1, where S and S^{-1} stay between iterations).
//
//   iteration k:  residual r = A_h U + lam U + b U^3 - f  (+ block partials of ||r||^2,
//                 ||f||^2 at k = 0, min / max U^2), and on the same rows
//                 P1  Y1[kx][y] = sum_x S^{-1}[kx][x] r[y][x]              -> barrier
//                 every block reduces the partial records in the same order, so all
//                 take the same stop decision and the same beta_n = (min + max)/2 of
//                 3 b U^2; block 0 records the iterate's statistics
//                 P2  Y2[ky][kx] = sum_y S^{-1}[ky][y] Y1[kx][y] / (lam_kx + lam_ky + lam + beta_n)
//                                                                           -> barrier
//                 P3  Y3[x][ky] = sum_kx S[x][kx] Y2[ky][kx]               -> barrier
//                 P4  U[y][x] -= step * sum_ky S[y][ky] Y3[x][ky]          -> barrier
//
// Each product stores its output transposed, so every dot product reads two contiguous
// rows. The barrier is a counter and a generation word in global memory; every wait is
// bounded (2 s of %globaltimer), after which the block sets the error word, and all
// blocks leave at their next barrier. The launch is cooperative, so all blocks are
// resident at once.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "qn_internal.h"
#include "qn_numeric.cuh"

namespace qn {

namespace {

constexpr int kSmallThreads = 128;
constexpr int kBarGen = 32;   // the generation word, a 128-byte line away from the counter
constexpr unsigned long long kSmallTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned long long small_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: returns false when a wait gave up (or another block's had), after
// recording QN_ETIMEOUT in *err. Thread 0 arrives with one acquire-release add on the
// counter (after the block's barrier, it releases the block's writes); the last block
// resets the counter and releases the generation word, which the others poll with
// acquire loads.
__device__ bool small_barrier(unsigned *count, unsigned *gen, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = ld_acquire(gen);
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        if (old == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
        } else {
            // the error word and the clock only every 64 polls
            const unsigned long long t0 = small_timer();
            unsigned polls = 0;
            while (ld_acquire(gen) == g) {
                if ((++polls & 63u) == 0 &&
                    (*(volatile int *)err != 0 || small_timer() - t0 > kSmallTimeoutNs)) {
                    atomicExch(err, QN_ETIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

struct SmallArgs {
    double *U;
    const double *f;
    const double *S, *Si, *lam1;   // n x n row-major (S[:, k] eigenvector k), eigenvalues
    double *w0, *w1;               // n^2 work arrays
    double *partials;              // [gridDim][4]
    unsigned *bar;                 // [2] barrier counter, generation
    DevState *st;                  // it / status / done on return
    qn_stats *hist;
    int hist_cap;
    int *err;
    int n, neumann;
    double inv_h2, lam, b, tol, beta_value, step;
    int beta_fixed, max_it;
};

__device__ __forceinline__ double nb_value(const double *U, int x, int y, int n, bool neu) {
    if (neu) {
        x = (x == -1) ? 1 : (x == n ? n - 2 : x);
        y = (y == -1) ? 1 : (y == n ? n - 2 : y);
    }
    return (x < 0 || x >= n || y < 0 || y >= n) ? 0.0 : __ldcg(U + y * n + x);
}

// One product phase: out[a][b] = sum_j M[a][j] X[b][j] (/ (lam_a + lam_b + shift) with a
// divide) for the input rows b this block owns (b = blockIdx.x, + gridDim.x, ...). The
// block stages its row of X (written by other blocks in the previous phase) in shared
// memory, read through L2; M is read-only and stays in L1 from one iteration to the next.
template <bool DIVIDE>
__device__ __forceinline__ void small_product(const double *__restrict__ M, const double *X, double *out, int n,
                                              double *row, const double *lam1, double shift) {
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = __ldcg(X + b * n + j);
        __syncthreads();
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            const double *m = M + a * n;
            double s0 = 0.0, s1 = 0.0;
            int j = 0;
            for (; j + 2 <= n; j += 2) {
                s0 = fma(__ldg(m + j), row[j], s0);
                s1 = fma(__ldg(m + j + 1), row[j + 1], s1);
            }
            if (j < n) s0 = fma(__ldg(m + j), row[j], s0);
            double v = s0 + s1;
            if (DIVIDE) v = v / ((__ldg(lam1 + b) + __ldg(lam1 + a)) + shift);
            out[a * n + b] = v;
        }
    }
}

__global__ void __launch_bounds__(kSmallThreads) k_small2d_fp64(SmallArgs a) {
    extern __shared__ double row[];   // one row of the phase input (n doubles)
    __shared__ double red[4][kSmallThreads / 32];
    __shared__ double sh_beta, sh_fn;
    __shared__ int sh_stop;
    const int n = a.n;
    const bool neu = a.neumann != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double fn = 0.0;
    int it = 0;
    int status = QN_ENOTCONV;
    for (;; ++it) {
        // ---- residual of the rows this block owns, and its partial record
        double r2 = 0.0, f2 = 0.0, mn = INFINITY, mx = 0.0;
        for (int y = blockIdx.x; y < n; y += gridDim.x)
            for (int x = threadIdx.x; x < n; x += blockDim.x) {
                const int p = y * n + x;
                const double u = __ldcg(a.U + p);
                const double lap = ((4.0 * u - nb_value(a.U, x - 1, y, n, neu)) - nb_value(a.U, x + 1, y, n, neu)) -
                                   (nb_value(a.U, x, y - 1, n, neu) + nb_value(a.U, x, y + 1, n, neu));
                const double fv = __ldg(a.f + p);
                double t = fma(a.b, (u * u) * u, -fv);
                t = fma(a.lam, u, t);
                const double r = fma(lap, a.inv_h2, t);
                a.w0[p] = r;
                r2 = fma(r, r, r2);
                if (it == 0) f2 = fma(fv, fv, f2);
                mn = fmin(mn, u * u);
                mx = fmax(mx, u * u);
            }
        for (int o = 16; o > 0; o >>= 1) {
            r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            f2 += __shfl_xor_sync(0xffffffffu, f2, o);
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            red[0][warp] = r2;
            red[1][warp] = f2;
            red[2][warp] = mn;
            red[3][warp] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double q0 = red[0][0], q1 = red[1][0], q2 = red[2][0], q3 = red[3][0];
            for (int w = 1; w < kSmallThreads / 32; ++w) {
                q0 += red[0][w];
                q1 += red[1][w];
                q2 = fmin(q2, red[2][w]);
                q3 = fmax(q3, red[3][w]);
            }
            double *q = a.partials + 4 * blockIdx.x;
            q[0] = q0;
            q[1] = q1;
            q[2] = q2;
            q[3] = q3;
        }
        // P1  Y1[kx][y] = sum_x Si[kx][x] r[y][x] on the rows just evaluated (this block's
        // own), before the barrier: it needs neither the norms nor beta
        small_product<false>(a.Si, a.w0, a.w1, n, row, nullptr, 0.0);
        if (!small_barrier(a.bar, a.bar + kBarGen, a.err)) return;
        // ---- every block: the same reduction, the same decision
        if (warp == 0) {
            double R = 0.0, F = 0.0, MN = INFINITY, MX = 0.0;
            for (int i = lane; i < (int)gridDim.x; i += 32) {
                const double *q = a.partials + 4 * i;
                R += __ldcg(q + 0);
                F += __ldcg(q + 1);
                MN = fmin(MN, __ldcg(q + 2));
                MX = fmax(MX, __ldcg(q + 3));
            }
            for (int o = 16; o > 0; o >>= 1) {
                R += __shfl_xor_sync(0xffffffffu, R, o);
                F += __shfl_xor_sync(0xffffffffu, F, o);
                MN = fmin(MN, __shfl_xor_sync(0xffffffffu, MN, o));
                MX = fmax(MX, __shfl_xor_sync(0xffffffffu, MX, o));
            }
            if (lane == 0) {
                if (it == 0) sh_fn = sqrt(F);
                const double res = sqrt(R);
                const double f_norm = sh_fn;
                const double fa = 3.0 * a.b * MN, fb = 3.0 * a.b * MX;
                const double fu_min = fmin(fa, fb), fu_max = fmax(fa, fb);
                const double beta = a.beta_fixed ? a.beta_value : 0.5 * (fu_min + fu_max);
                const double rel = (f_norm > 0.0) ? res / f_norm : ((res == 0.0) ? 0.0 : INFINITY);
                if (blockIdx.x == 0 && it < a.hist_cap) {
                    qn_stats s;
                    s.res_norm = res;
                    s.f_norm = f_norm;
                    s.fu_min = fu_min;
                    s.fu_max = fu_max;
                    s.beta = beta;
                    s.rel = rel;
                    s.lambda = 0.0;
                    a.hist[it] = s;
                }
                int stop = 0;
                if (rel <= a.tol) {
                    stop = 1;
                    status = QN_OK;
                } else if (!isfinite(rel) || rel > 1e8 || !isfinite(beta)) {
                    stop = 1;
                    status = QN_EDIVERGED;
                } else if (it >= a.max_it) {
                    stop = 1;
                    status = QN_ENOTCONV;
                }
                sh_stop = stop;
                sh_beta = a.lam + beta;
            }
        }
        __syncthreads();
        fn = sh_fn;
        if (sh_stop) break;
        const double shift = sh_beta;
        // P2  Y2[ky][kx] = sum_y Si[ky][y] Y1[kx][y] / (lam_kx + lam_ky + shift)
        small_product<true>(a.Si, a.w1, a.w0, n, row, a.lam1, shift);
        if (!small_barrier(a.bar, a.bar + kBarGen, a.err)) return;
        // P3  Y3[x][ky] = sum_kx S[x][kx] Y2[ky][kx]
        small_product<false>(a.S, a.w0, a.w1, n, row, nullptr, 0.0);
        if (!small_barrier(a.bar, a.bar + kBarGen, a.err)) return;
        // P4  delta[y][x] = sum_ky S[y][ky] Y3[x][ky], U -= step * delta
        for (int b = blockIdx.x; b < n; b += gridDim.x) {   // b = x (the input row)
            __syncthreads();
            for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = __ldcg(a.w1 + b * n + j);
            __syncthreads();
            for (int y = threadIdx.x; y < n; y += blockDim.x) {
                const double *m = a.S + y * n;
                double s0 = 0.0, s1 = 0.0;
                int j = 0;
                for (; j + 2 <= n; j += 2) {
                    s0 = fma(__ldg(m + j), row[j], s0);
                    s1 = fma(__ldg(m + j + 1), row[j + 1], s1);
                }
                if (j < n) s0 = fma(__ldg(m + j), row[j], s0);
                const double d = s0 + s1;
                const int p = y * n + b;
                const double u = __ldcg(a.U + p);
                a.U[p] = (a.step == 1.0) ? u - d : fma(-a.step, d, u);
            }
        }
        if (!small_barrier(a.bar, a.bar + kBarGen, a.err)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->it = it;
        a.st->status = status;
        a.st->done = 1;
        a.st->f_norm = fn;
    }
}

}  // namespace

int small_solve_supported(int dim, int n) { return dim == 2 && n >= 1 && n <= kSmallMaxN; }

int launch_small_solve(const SmallSolve &q, cudaStream_t s) {
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_small2d_fp64, kSmallThreads,
                                                          sizeof(double) * kSmallMaxN) != cudaSuccess)
            nb = 0;
        blocks_per_sm = nb;
    }
    if (blocks_per_sm < 1) {
        set_error("launch_small_solve: the kernel does not fit on an SM");
        return QN_ECUDA;
    }
    // one block per SM (the phases are FP64-FMA bound: about 2 FMAs per clock per SM on
    // this GPU), never more blocks than points
    // one block per row of the phase inputs (each block owns rows b, b + grid, ...)
    const char *eg = getenv("QN_SMALL_GRID");
    int grid = eg ? atoi(eg) : q.n;
    if (grid > q.num_sms) grid = q.num_sms;
    if (grid > q.n) grid = q.n;
    if (grid < 1) grid = 1;
    const int cap = blocks_per_sm * q.num_sms;
    if (grid > cap) grid = cap;
    if (grid > q.partials_cap) grid = q.partials_cap;
    if (grid < 1) grid = 1;
    SmallArgs a;
    a.U = q.U;
    a.f = q.f;
    a.S = q.S;
    a.Si = q.Si;
    a.lam1 = q.lam1;
    a.w0 = q.w0;
    a.w1 = q.w1;
    a.partials = q.partials;
    a.bar = q.bar;
    a.st = q.st;
    a.hist = q.hist;
    a.hist_cap = q.hist_cap;
    a.err = q.err;
    a.n = q.n;
    a.neumann = q.neumann;
    a.inv_h2 = q.inv_h2;
    a.lam = q.lam;
    a.b = q.b;
    a.tol = q.tol;
    a.beta_value = q.beta_value;
    a.step = q.step;
    a.beta_fixed = q.beta_fixed;
    a.max_it = q.max_it;
    QN_CUDA(cudaMemsetAsync(q.bar, 0, kSmallBarWords * sizeof(unsigned), s));
    void *params[] = {&a};
    QN_CUDA(cudaLaunchCooperativeKernel((const void *)k_small2d_fp64, dim3(grid), dim3(kSmallThreads), params,
                                        sizeof(double) * q.n, s));
    return QN_OK;
}

}  // namespace qn
