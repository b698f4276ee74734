// C-ABI entry points of libqn (declared in include/qn.h): context set-up,
// residual, shifted fast-diagonalisation inverse, one quasi-Newton step and
// the solve loop.
//
// One iteration (Sec. 4 eq. identity-method with the inverse of Sec. 4.1
// eq. fin_inverse) is enqueued as
//   residual+reductions -> finalise (beta_n, stop test, on the device)
//   -> dim forward mode products (S^{-1}; the last one divides by the eigen-sums)
//   -> dim backward mode products (S; the last one applies U -= step * delta).
// The finaliser's `done` flag makes every later kernel return at once, so the
// host may queue several iterations before it checks convergence.
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "qn_internal.h"

namespace qn {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return QN_ECUDA;
}

}  // namespace qn

using namespace qn;

static const int kHistCap = 4097;

struct StateMirror;

struct qn_ctx {
    qn_problem prob;
    int device;
    int num_sms;
    int n, P, dim;
    long long N;    // n^dim
    long long NP;   // P^dim (split path)
    double h, inv_h2;
    // eigen-data
    double *S64, *Si64, *lam64;
    __nv_bfloat16 *S_hi, *S_lo, *Si_hi, *Si_lo;
    float *lam32;
    // working buffers
    double *w64[2];
    __nv_bfloat16 *bhi[2], *blo[2];
    double *partials;
    int partials_cap;     // records the partials buffer holds (>= nparts; eigen pass 2 may use more)
    int nparts;
    DevState *st;
    qn_stats *hist;
    int *err;
    TcPlan *plan;
    // host-array staging for qn_solve_host
    double *dU, *df;
    // launch accounting / optional CUDA-event timing of every launch
    struct ProfRec {
        cudaEvent_t a, b;
        int kind;
        int iter;
        int valid;
    };
    std::vector<ProfRec> *prof;
    size_t prof_used;
    int prof_on;
    int cur_iter;
    long long launches;
    int res_fp64_warps;   // residual inside the split solve: FP64-stencil warps per block (of 8)
    float2 *fdf;          // 3-D split solve: padded FP32-pair copy of f (k_residual_tiled)
    int res_tiled;        // 1: iterations >= 2 of a 3-D split solve use k_residual_tiled
    int res_zc;           // planes per work item of k_residual_tiled
    int res_parts;        // partial-sum records written by the last residual launch
    int res_fx_headroom;  // DevState::fx_headroom for the solves of this context
    int res_saved_fnorm;  // 1: the last residual's finaliser takes ||f|| from DevState::f_norm
    // CUDA graph of sync_every steady-state iterations (qn_opts.graph)
    cudaStream_t cap_stream;
    cudaGraphExec_t gexec;
    double *g_U;
    const double *g_f;
    double g_step;
    int g_chunk;
    long long g_launches; // kernels per replay
    // the previously used graph, kept so that two alternating (U, f) pairs (the
    // ping-pong buffers of qn_solve_host_many) do not re-capture on every solve
    struct GraphSlot {
        cudaGraphExec_t exec;
        double *U;
        const double *f;
        double step;
        int chunk, kind, x6, fused;
        long long launches;
    } g_prev;
    // the solver state read by the host: written by a kernel into mapped page-locked host
    // memory, so that the solve loop issues no memory copies (copies would queue behind
    // the large transfers of qn_solve_host_many on the copy engines)
    StateMirror *mir_host, *mir_dev;
    long long aux_launches;   // state-set / state-mirror kernels of the current solve
    // qn_solve_host_many: two device (U, f) buffer pairs and the copy streams / events
    double *hm_U[2], *hm_f[2];
    cudaStream_t hm_h2d, hm_d2h;
    cudaEvent_t hm_in_ready[2], hm_solved[2], hm_out_done[2];
    float *warm_dsq;      // device: ||U_1 - U_0||^2 of a warm-started solve's first iteration
    int warm_dsq_on;      // 1 while that iteration's products are enqueued
    // reflection-split mode products (3-D split solve, P a multiple of 128)
    int split;            // 1: the plan holds the split matrices and the solve loop uses them
    int split_layout;     // 1: the last residual wrote its planes in split / folded order
    int last_split;       // 1: the last shifted inverse used the split products
    int f64_split;        // FP64 path: reflection-split FP64 products (FD Dirichlet / Neumann)
    __nv_bfloat16 *bf_hi, *bf_lo, *bb_hi, *bb_lo;   // [P][P/2] forward / backward matrices
    // six-product backward level (QN_PREC_BF16X6): the third BF16 level of the two working
    // buffers and of the backward matrix; x6 = 1 while the solves use it
    __nv_bfloat16 *bl2[2], *bb_l2;
    int x6;               // the level the products enqueued next use
    int x6_base;          // 1: a QN_PREC_BF16X6 context (every solve starts with the level on)
    // precision escalation of BF16X3 solves (qn_ctx_set_escalation): the observed one-step
    // contraction above esc_rate and above twice the nonlinear bound switches the
    // remaining iterations of the solve to the six-product level
    double esc_rate;      // 0: off
    int esc_at;           // first iteration of the last solve that ran at that level (-1: none)
    int g_x6;             // the captured graph's level
    // the residual fused into the first forward product (qn_set_fused_residual)
    int fused;            // 1: iterations >= 1 of the 3-D split solve use k_fused_res_fwd
    int fused_first;      // 1: the last residual launch also formed the first product
    int fused_used;       // 1: the current solve has used the fused kernel
    int g_fused;          // the captured graph's form
    unsigned *small_bar;  // small 2-D FP64 solves: the persistent kernel's grid barrier words
    int small_solve;      // 1: qn_solve runs the whole-solve persistent kernel (qn_small.cu)
    float *lam32_split;   // eigenvalues in split mode order (even modes, then odd), 1e30 padding
    // separable potential V = v_x + v_y (+ v_z): device tables [dim][n], FP64 and as FP32
    // pairs with lam added to the last axis (k_residual_tiled / mirror); nullptr: V = 0
    double *pot64;
    float2 *pot2;
    double *eig_r0;       // eigen solves, BF16X3: A_h U + f(U) between the two residual passes
    double *eig_vrow;     // eigen solves with a potential: lam + v_y (+ v_z) per (y, z) row
    float *eig_pot32;     //   and the potential tables in FP32
    float2 *eig_vrow2;    //   the per-row table and the x table as FP32 pairs (float-pair passes)
    float2 *eig_potx2;
    int g_kind;           // graph contents: 0 quasi-Newton iterations, 1 eigen iterations
    double lam_min;       // smallest eigenvalue of the 1-D matrix H
    // spectral elements (prob.sem_k > 0): banded H on the device (k_residual_sem)
    int *hc0, *hlen;
    double *hval;
    int hbw;
};

struct StateMirror {
    DevState st;
    int err;        // the device error word (QN_ETIMEOUT), taken and cleared by the mirror kernel
    int pad;
    qn_stats last;  // the statistics of the iterate evaluated last: hist[st.it] once the solve
                    // is done, hist[st.it - 1] before (st.it then names the next iterate)
    qn_stats prev;  // the record before `last` (unchanged when `last` is hist[0])
};

// The solver state from host parameters (one thread; no copy-engine transfer).
__global__ void k_set_state(DevState *st, DevState v) {
    if (threadIdx.x == 0) *st = v;
}

// State, error word and the last statistics record into mapped host memory.
__global__ void k_mirror_state(const DevState *st, int *err, const qn_stats *hist, int hist_cap,
                               StateMirror *out) {
    if (threadIdx.x != 0) return;
    const DevState v = *st;
    out->st = v;
    out->err = atomicExch(err, 0);
    const int li = v.done ? v.it : v.it - 1;
    if (hist != nullptr && li >= 0 && li < hist_cap) out->last = hist[li];
    if (hist != nullptr && li >= 1 && li - 1 < hist_cap) out->prev = hist[li - 1];
    __threadfence_system();
}

enum ProfKind { PK_RESIDUAL = 0, PK_FINALIZE = 1, PK_MP_STORE = 2, PK_MP_DIVIDE = 3, PK_MP_LAST = 4,
                PK_SPLIT = 5, PK_RESIDUAL_TILED = 6, PK_FUSED = 7, PK_COUNT = 8 };

// Begin/end a timed launch. With profiling off these only count launches.
static long prof_begin(qn_ctx *c, int kind, cudaStream_t s) {
    c->launches++;
    if (!c->prof_on) return -1;
    if (c->prof_used == c->prof->size()) {
        qn_ctx::ProfRec r;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
        c->prof->push_back(r);
    }
    qn_ctx::ProfRec &r = (*c->prof)[c->prof_used];
    r.kind = kind;
    r.iter = c->cur_iter;
    r.valid = 1;
    if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
    return (long)c->prof_used++;
}

static void prof_end(qn_ctx *c, long idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord((*c->prof)[idx].b, s);
}

static int check_ctx(qn_ctx *c) {
    if (!c) {
        set_error("null context");
        return QN_EINVAL;
    }
    return QN_OK;
}

static void split_host(double v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    const float f = (float)v;
    hi = __float2bfloat16_rn(f);
    lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

// The third level below split_host's two: what hi + lo leave of v, rounded to BF16.
static __nv_bfloat16 split_host_l2(double v, __nv_bfloat16 hi, __nv_bfloat16 lo) {
    const double r = v - (double)__bfloat162float(hi) - (double)__bfloat162float(lo);
    return __float2bfloat16_rn((float)r);
}

extern "C" int qn_version(void) { return 10400; }

extern "C" const char *qn_last_error(void) { return g_err; }

extern "C" int qn_setup_1d_eig(int n, double h, int bc, double *S, double *S_inv, double *lam) {
    if (n < 1 || n > 65536 || (bc == QN_BC_NEUMANN && n < 2)) {
        set_error("qn_setup_1d_eig: n=%d out of range", n);
        return QN_EINVAL;
    }
    if (!(h > 0.0) || !isfinite(h)) {
        set_error("qn_setup_1d_eig: h=%.17g must be positive and finite", h);
        return QN_EINVAL;
    }
    if (bc != QN_BC_DIRICHLET && bc != QN_BC_NEUMANN) {
        set_error("qn_setup_1d_eig: unknown boundary condition %d", bc);
        return QN_EINVAL;
    }
    const double pi = 3.14159265358979323846;
    if (bc == QN_BC_NEUMANN) {
        // discrete cosine pairs of the ghost-point matrix: H cos(j k pi t) =
        // lam_k cos(j k pi t) in every row (the face rows because the ghost
        // value equals the inner neighbour); the columns are orthogonal in the
        // trapezoid weights w, with squared norms c_k
        const double t = 1.0 / (n - 1);
        for (int k = 0; k < n; ++k) {
            const double sk = sin(0.5 * k * pi * t);
            if (lam) lam[k] = 4.0 / (h * h) * sk * sk;
        }
        for (int j = 0; j < n; ++j) {
            const double w = (j == 0 || j == n - 1) ? 0.5 : 1.0;
            for (int k = 0; k < n; ++k) {
                const double ck = (k == 0 || k == n - 1) ? (double)(n - 1) : 0.5 * (n - 1);
                // cos(j k pi t) with the product reduced mod 2(n-1)
                const long long jk = ((long long)j * k) % (2LL * (n - 1));
                const double v = cos(pi * (double)jk * t) / sqrt(ck);
                if (S) S[(size_t)j * n + k] = v;
                if (S_inv) S_inv[(size_t)k * n + j] = w * v;
            }
        }
        return QN_OK;
    }
    const double hh = 1.0 / (n + 1);
    const double scale = sqrt(2.0 * hh);
    for (int k = 1; k <= n; ++k) {
        const double s = sin(0.5 * k * pi * hh);
        if (lam) lam[k - 1] = 4.0 / (h * h) * s * s;
    }
    for (int j = 1; j <= n; ++j) {
        for (int k = 1; k <= n; ++k) {
            // sin(j k pi h) with the product reduced mod 2(n+1) for accuracy
            const long long jk = ((long long)j * k) % (2LL * (n + 1));
            const double v = scale * sin(pi * (double)jk * hh);
            if (S) S[(size_t)(j - 1) * n + (k - 1)] = v;
            if (S_inv) S_inv[(size_t)(j - 1) * n + (k - 1)] = v;   // symmetric orthogonal
        }
    }
    return QN_OK;
}

static void ctx_free(qn_ctx *c) {
    if (!c) return;
    cudaFree(c->S64);
    cudaFree(c->Si64);
    cudaFree(c->lam64);
    cudaFree(c->S_hi);
    cudaFree(c->S_lo);
    cudaFree(c->Si_hi);
    cudaFree(c->Si_lo);
    cudaFree(c->lam32);
    cudaFree(c->bf_hi);
    cudaFree(c->bf_lo);
    cudaFree(c->bb_hi);
    cudaFree(c->bb_lo);
    cudaFree(c->bb_l2);
    cudaFree(c->small_bar);
    cudaFree(c->bl2[0]);
    cudaFree(c->bl2[1]);
    cudaFree(c->lam32_split);
    cudaFree(c->pot64);
    cudaFree(c->pot2);
    cudaFree(c->eig_r0);
    cudaFree(c->eig_vrow);
    cudaFree(c->eig_pot32);
    cudaFree(c->eig_vrow2);
    cudaFree(c->eig_potx2);
    cudaFree(c->hc0);
    cudaFree(c->hlen);
    cudaFree(c->hval);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->w64[b]);
        cudaFree(c->bhi[b]);
        cudaFree(c->blo[b]);
    }
    cudaFree(c->partials);
    cudaFree(c->warm_dsq);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->g_prev.exec) cudaGraphExecDestroy(c->g_prev.exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->hm_U[b]);
        cudaFree(c->hm_f[b]);
        if (c->hm_in_ready[b]) cudaEventDestroy(c->hm_in_ready[b]);
        if (c->hm_solved[b]) cudaEventDestroy(c->hm_solved[b]);
        if (c->hm_out_done[b]) cudaEventDestroy(c->hm_out_done[b]);
    }
    if (c->hm_h2d) cudaStreamDestroy(c->hm_h2d);
    if (c->hm_d2h) cudaStreamDestroy(c->hm_d2h);
    cudaFree(c->fdf);
    cudaFree(c->st);
    if (c->mir_host) cudaFreeHost(c->mir_host);
    cudaFree(c->hist);
    cudaFree(c->err);
    cudaFree(c->dU);
    cudaFree(c->df);
    if (c->plan) tc_plan_destroy(c->plan);
    if (c->prof) {
        for (auto &r : *c->prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        delete c->prof;
    }
    delete c;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) {                  \
            int _r = cuda_fail(_e, #call);        \
            ctx_free(c);                          \
            return _r;                            \
        }                                         \
    } while (0)

// The working buffers' third level and its tensor maps (once per context).
static int ensure_x6(qn_ctx *c) {
    if (c->bl2[0] != nullptr) return QN_OK;
    if (!c->split || c->bb_l2 == nullptr) return QN_EUNSUPPORTED;
    const size_t pb = sizeof(__nv_bfloat16) * (size_t)c->NP;
    for (int b = 0; b < 2; ++b) {
        if (cudaMalloc(&c->bl2[b], pb) != cudaSuccess) {
            cudaFree(c->bl2[0]);
            c->bl2[0] = nullptr;
            set_error("ensure_x6: out of device memory for the third BF16 level");
            return QN_ENOMEM;
        }
        QN_CUDA(cudaMemset(c->bl2[b], 0, pb));
    }
    return tc_plan_enable_x6(c->plan, c->bl2, c->bb_l2);
}

extern "C" int qn_ctx_create(const qn_problem *p, qn_ctx **out) {
    if (!p || !out) {
        set_error("qn_ctx_create: null argument");
        return QN_EINVAL;
    }
    *out = nullptr;
    if (p->dim != 2 && p->dim != 3) {
        set_error("qn_ctx_create: dim must be 2 or 3 (got %d)", p->dim);
        return QN_EINVAL;
    }
    if (p->bc != QN_BC_DIRICHLET && p->bc != QN_BC_NEUMANN && p->bc != QN_BC_ROBIN) {
        set_error("qn_ctx_create: unknown boundary condition %d", p->bc);
        return QN_EINVAL;
    }
    if (p->bc == QN_BC_ROBIN && (!(p->robin_kappa >= 0.0) || !isfinite(p->robin_kappa) || p->sem_k != 0)) {
        set_error("qn_ctx_create: QN_BC_ROBIN needs a finite robin_kappa >= 0 and finite differences");
        return QN_EINVAL;
    }
    const int nmin = (p->bc == QN_BC_DIRICHLET) ? 1 : 2;
    if (p->n < nmin || p->n > 1024) {
        set_error("qn_ctx_create: n must be in [%d, 1024] (got %d)", nmin, p->n);
        return QN_EINVAL;
    }
    if (p->sem_k < 0 || p->sem_k > 16) {
        set_error("qn_ctx_create: sem_k must be 0 (finite differences) or 1..16 (got %d)", p->sem_k);
        return QN_EINVAL;
    }
    if (!(p->length >= 0.0) || !isfinite(p->length)) {
        set_error("qn_ctx_create: length must be finite and >= 0 (0 = unit cube)");
        return QN_EINVAL;
    }
    if (p->potential_host) {
        for (long long i = 0; i < (long long)p->dim * p->n; ++i)
            if (!isfinite(p->potential_host[i])) {
                set_error("qn_ctx_create: potential table entry %lld is not finite", i);
                return QN_EINVAL;
            }
    }
    if (p->precision != QN_PREC_FP64 && p->precision != QN_PREC_BF16X3 && p->precision != QN_PREC_BF16X6) {
        set_error("qn_ctx_create: unknown precision %d", p->precision);
        return QN_EINVAL;
    }
    if (!isfinite(p->lam) || !isfinite(p->b)) {
        set_error("qn_ctx_create: lam and b must be finite");
        return QN_EINVAL;
    }
    qn_ctx *c = new (std::nothrow) qn_ctx();
    if (!c) return QN_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->prob = *p;
    // BF16X6 is the BF16X3 path with the six-product backward level on: every
    // other part of the context (residual, forward products, state) is the same
    const bool want_x6 = (p->precision == QN_PREC_BF16X6);
    if (want_x6) c->prob.precision = QN_PREC_BF16X3;
    c->prof = new (std::nothrow) std::vector<qn_ctx::ProfRec>();
    if (!c->prof) {
        delete c;
        return QN_ENOMEM;
    }
    CK(cudaGetDevice(&c->device));
    CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    c->n = p->n;
    c->dim = p->dim;
    {
        const char *env = getenv("QN_RES_FP64_WARPS");
        const int w = env ? atoi(env) : 3;
        c->res_fp64_warps = (w >= 0 && w <= 8) ? w : 3;
        const char *et = getenv("QN_RES_TILED");
        c->res_tiled = et ? (atoi(et) != 0) : 1;
        const char *ez = getenv("QN_RES_ZC");
        const int zc = ez ? atoi(ez) : 32;
        c->res_zc = (zc >= 1 && zc <= 4096) ? zc : 32;
        // exponent headroom of the fixed-point stencil (2 = room for 4x growth of
        // max|U|); smaller values route more planes through the exact path
        const char *eh = getenv("QN_RES_FX_HEADROOM");
        const int hr = eh ? atoi(eh) : 2;
        c->res_fx_headroom = (hr >= -16 && hr <= 2) ? hr : 2;
    }
    c->P = ((p->n + 63) / 64) * 64;
    c->N = 1;
    c->NP = 1;
    for (int a = 0; a < c->dim; ++a) {
        c->N *= c->n;
        c->NP *= c->P;
    }
    const double Ldom = (p->length > 0.0) ? p->length : 1.0;
    if (p->sem_k > 0) {   // element width
        c->h = Ldom * p->sem_k / ((p->bc == QN_BC_NEUMANN) ? c->n - 1 : c->n + 1);
    } else {
        c->h = (p->bc == QN_BC_DIRICHLET) ? Ldom / (c->n + 1) : Ldom / (c->n - 1);
    }
    c->prob.potential_host = nullptr;   // not retained
    c->inv_h2 = 1.0 / (c->h * c->h);
    const int n = c->n, P = c->P;

    std::vector<double> S((size_t)n * n), Si((size_t)n * n), lam(n);
    int rc;
    if (p->sem_k > 0) {
        std::vector<double> Hm, nodes;
        rc = sem_setup(n, p->sem_k, Ldom, p->bc, Hm, S, Si, lam, nodes);
        if (rc != QN_OK) {
            ctx_free(c);
            return rc;
        }
        // band of H = M^{-1} S: first and last nonzero column of every row (<= 2k+1 wide)
        const int bw = 2 * p->sem_k + 1;
        std::vector<int> c0(n), len(n);
        std::vector<double> hv((size_t)n * bw, 0.0);
        for (int i = 0; i < n; ++i) {
            int lo = n, hi = -1;
            for (int j = 0; j < n; ++j)
                if (Hm[(size_t)i * n + j] != 0.0) {
                    lo = std::min(lo, j);
                    hi = std::max(hi, j);
                }
            if (hi < lo) lo = hi = i;
            if (hi - lo + 1 > bw) {
                set_error("qn_ctx_create: spectral element matrix wider than its band");
                ctx_free(c);
                return QN_ECUDA;
            }
            c0[i] = lo;
            len[i] = hi - lo + 1;
            for (int j = lo; j <= hi; ++j) hv[(size_t)i * bw + (j - lo)] = Hm[(size_t)i * n + j];
        }
        c->hbw = bw;
        CK(cudaMalloc(&c->hc0, sizeof(int) * n));
        CK(cudaMalloc(&c->hlen, sizeof(int) * n));
        CK(cudaMalloc(&c->hval, sizeof(double) * (size_t)n * bw));
        CK(cudaMemcpy(c->hc0, c0.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->hlen, len.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->hval, hv.data(), sizeof(double) * (size_t)n * bw, cudaMemcpyHostToDevice));
    } else if (p->bc == QN_BC_ROBIN) {
        rc = qn_setup_1d_robin(n, c->h, p->robin_kappa, S.data(), Si.data(), lam.data());
        if (rc != QN_OK) {
            ctx_free(c);
            return rc;
        }
    } else {
        rc = qn_setup_1d_eig(n, c->h, p->bc, S.data(), Si.data(), lam.data());
        if (rc != QN_OK) {
            ctx_free(c);
            return rc;
        }
    }
    c->lam_min = lam[0];
    CK(cudaMalloc(&c->S64, sizeof(double) * n * n));
    CK(cudaMalloc(&c->Si64, sizeof(double) * n * n));
    CK(cudaMalloc(&c->lam64, sizeof(double) * n));
    CK(cudaMemcpy(c->S64, S.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->Si64, Si.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->lam64, lam.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    double vmax = 0.0;   // bound on |lam + V| (range check of the float-pair residual)
    if (p->potential_host) {
        const int dn = c->dim * n;
        std::vector<float2> v2(dn);
        double vsum = fabs(p->lam);
        for (int ax = 0; ax < c->dim; ++ax) {
            double m = 0.0;
            for (int i = 0; i < n; ++i) {
                const double v = p->potential_host[ax * n + i] + ((ax == 2) ? p->lam : 0.0);
                const float hi = (float)v;
                v2[ax * n + i] = make_float2(hi, (float)(v - (double)hi));
                m = fmax(m, fabs(p->potential_host[ax * n + i]));
            }
            vsum += m;
        }
        vmax = vsum;
        CK(cudaMalloc(&c->pot64, sizeof(double) * dn));
        CK(cudaMalloc(&c->pot2, sizeof(float2) * dn));
        CK(cudaMemcpy(c->pot64, p->potential_host, sizeof(double) * dn, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->pot2, v2.data(), sizeof(float2) * dn, cudaMemcpyHostToDevice));
    }

    const int rows = (c->dim == 3) ? P * P : P;
    c->nparts = rows < 4 * c->num_sms ? rows : 4 * c->num_sms;
    c->partials_cap = c->nparts > 8 * c->num_sms ? c->nparts : 8 * c->num_sms;
    CK(cudaMalloc(&c->partials, sizeof(double) * 4 * c->partials_cap));
    CK(cudaMalloc(&c->st, sizeof(DevState)));
    CK(cudaHostAlloc((void **)&c->mir_host, sizeof(StateMirror), cudaHostAllocMapped));
    memset(c->mir_host, 0, sizeof(StateMirror));
    CK(cudaHostGetDevicePointer((void **)&c->mir_dev, c->mir_host, 0));
    CK(cudaMalloc(&c->hist, sizeof(qn_stats) * kHistCap));
    CK(cudaMalloc(&c->err, sizeof(int)));
    CK(cudaMemset(c->err, 0, sizeof(int)));

    if (p->precision == QN_PREC_FP64) {
        for (int b = 0; b < 2; ++b) CK(cudaMalloc(&c->w64[b], sizeof(double) * c->N));
        // small 2-D finite-difference problems without a potential: the whole solve in one
        // persistent launch (launch latency dominates there)
        const char *esm = getenv("QN_SMALL");
        if ((esm ? atoi(esm) != 0 : true) && small_solve_supported(c->dim, c->n) && p->sem_k == 0 &&
            (p->bc == QN_BC_DIRICHLET || p->bc == QN_BC_NEUMANN) && p->potential_host == nullptr) {
            CK(cudaMalloc(&c->small_bar, kSmallBarWords * sizeof(unsigned)));
            CK(cudaMemset(c->small_bar, 0, kSmallBarWords * sizeof(unsigned)));
            c->small_solve = 1;
        }
        // the closed-form sine / cosine pairs have the reflection symmetry the split
        // products use; the numerical (Robin, spectral-element) ones need not
        const char *es = getenv("QN_SPLIT");
        c->f64_split = (es ? (atoi(es) != 0) : true) && p->sem_k == 0 && p->bc != QN_BC_ROBIN;
    } else {
        if (!tc_supported(c->device)) {
            set_error("qn_ctx_create: QN_PREC_BF16X3 needs an sm_103 (tcgen05) device");
            ctx_free(c);
            return QN_EUNSUPPORTED;
        }
        std::vector<__nv_bfloat16> hS((size_t)P * P), lS((size_t)P * P), hSi((size_t)P * P),
            lSi((size_t)P * P);
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
        CK(cudaMalloc(&c->S_hi, mb));
        CK(cudaMalloc(&c->S_lo, mb));
        CK(cudaMalloc(&c->Si_hi, mb));
        CK(cudaMalloc(&c->Si_lo, mb));
        CK(cudaMalloc(&c->lam32, sizeof(float) * P));
        CK(cudaMemcpy(c->S_hi, hS.data(), mb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->S_lo, lS.data(), mb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->Si_hi, hSi.data(), mb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->Si_lo, lSi.data(), mb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->lam32, l32.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
        const size_t pb = sizeof(__nv_bfloat16) * (size_t)c->NP;
        for (int b = 0; b < 2; ++b) {
            CK(cudaMalloc(&c->bhi[b], pb));
            CK(cudaMalloc(&c->blo[b], pb));
            CK(cudaMemset(c->bhi[b], 0, pb));
            CK(cudaMemset(c->blo[b], 0, pb));
        }
        // the float-pair residual needs lam, b and 1/h^2 well inside the FP32 range
        const bool pair_ok = fabs(p->lam) < 0x1p40 && fabs(p->b) < 0x1p20 && c->inv_h2 < 0x1p24 &&
                             vmax < 0x1p40;
        // (the FP64-free residual is the Dirichlet / Neumann FD stencil's)
        if (c->dim == 3 && pair_ok && p->sem_k == 0 && p->bc != QN_BC_ROBIN) {
            CK(cudaMalloc(&c->fdf, sizeof(float2) * (size_t)c->NP));
        } else {
            c->res_tiled = 0;
        }
        rc = tc_plan_create(&c->plan, n, P, c->dim, c->bhi, c->blo, c->S_hi, c->S_lo, c->Si_hi, c->Si_lo,
                            c->num_sms);
        if (rc != QN_OK) {
            ctx_free(c);
            return rc;
        }
        // Reflection-split matrices (qn_modeprod_tc.cu): with H = P/2,
        //   forward  Bf[p][j]: p < H -> S^{-1}[2p][j] for j < ceil(n/2) (the middle
        //            column of an odd n included); p >= H -> S^{-1}[2(p-H)+1][j], j < n/2
        //   backward Bb[r][i]: r < H -> S[r][2i] (r < ceil(n/2));
        //            r >= H -> S[r-H][2i+1] (r-H < n/2)
        // and the eigenvalues in the same mode order. Both the sine (Dirichlet)
        // and the cosine (Neumann) pairs have S[n-1-j][k] = (-1)^k S[j][k] and
        // S^{-1}[k][n-1-j] = (-1)^k S^{-1}[k][j].
        const char *es = getenv("QN_SPLIT");
        const bool want_split = es ? (atoi(es) != 0) : true;
        if (want_split && c->dim == 3 && P % 128 == 0 && c->fdf != nullptr) {
            const int H = P / 2, nsym = (n + 1) / 2, nanti = n / 2;
            std::vector<__nv_bfloat16> fh((size_t)P * H), fl((size_t)P * H), bh((size_t)P * H), blo((size_t)P * H);
            std::vector<float> ls(P, 1e30f);
            for (int p = 0; p < P; ++p) {
                const int k = (p < H) ? 2 * p : 2 * (p - H) + 1;
                const int jmax = (p < H) ? nsym : nanti;
                if (k < n) ls[p] = (float)lam[k];
                for (int j = 0; j < H; ++j) {
                    const double v = (k < n && j < jmax) ? Si[(size_t)k * n + j] : 0.0;
                    split_host(v, fh[(size_t)p * H + j], fl[(size_t)p * H + j]);
                }
            }
            for (int r = 0; r < P; ++r) {
                const int j = (r < H) ? r : r - H;
                const int jmax = (r < H) ? nsym : nanti;
                for (int i = 0; i < H; ++i) {
                    const int k = (r < H) ? 2 * i : 2 * i + 1;
                    const double v = (j < jmax && k < n) ? S[(size_t)j * n + k] : 0.0;
                    split_host(v, bh[(size_t)r * H + i], blo[(size_t)r * H + i]);
                }
            }
            const size_t bb = sizeof(__nv_bfloat16) * (size_t)P * H;
            CK(cudaMalloc(&c->bf_hi, bb));
            CK(cudaMalloc(&c->bf_lo, bb));
            CK(cudaMalloc(&c->bb_hi, bb));
            CK(cudaMalloc(&c->bb_lo, bb));
            CK(cudaMalloc(&c->lam32_split, sizeof(float) * P));
            CK(cudaMemcpy(c->bf_hi, fh.data(), bb, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->bf_lo, fl.data(), bb, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->bb_hi, bh.data(), bb, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->bb_lo, blo.data(), bb, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->lam32_split, ls.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
            rc = tc_plan_enable_split(c->plan, c->bf_hi, c->bf_lo, c->bb_hi, c->bb_lo);
            if (rc == QN_OK) {
                c->split = 1;
            } else if (rc != QN_EUNSUPPORTED) {
                ctx_free(c);
                return rc;
            }
            if (c->split) {
                // third level of the backward matrix (after the hi / lo above; small, kept for
                // qn_ctx_set_escalation too); the working buffers' level only for BF16X6
                std::vector<__nv_bfloat16> bl2v((size_t)P * H);
                for (size_t i = 0; i < bl2v.size(); ++i) {
                    const int r = (int)(i / H), ii = (int)(i % H);
                    const int j = (r < H) ? r : r - H;
                    const int jmax = (r < H) ? nsym : nanti;
                    const int k = (r < H) ? 2 * ii : 2 * ii + 1;
                    const double v = (j < jmax && k < n) ? S[(size_t)j * n + k] : 0.0;
                    bl2v[i] = split_host_l2(v, bh[i], blo[i]);
                }
                CK(cudaMalloc(&c->bb_l2, bb));
                CK(cudaMemcpy(c->bb_l2, bl2v.data(), bb, cudaMemcpyHostToDevice));
            }
            if (c->split && want_x6) {
                rc = ensure_x6(c);
                if (rc != QN_OK) {
                    ctx_free(c);
                    return rc;
                }
                c->x6 = c->x6_base = 1;
            }
        }
        if (want_x6 && !c->x6) {
            set_error("qn_ctx_create: QN_PREC_BF16X6 needs the reflection-split products (3-D finite "
                      "differences, Dirichlet or Neumann, padded size P = 64 ceil(n/64) a multiple of 128)");
            ctx_free(c);
            return QN_EUNSUPPORTED;
        }
    }
    *out = c;
    return QN_OK;
}

extern "C" int qn_ctx_destroy(qn_ctx *c) {
    if (!c) return QN_OK;
    cudaDeviceSynchronize();
    ctx_free(c);
    return QN_OK;
}

// ---- internal enqueue helpers ------------------------------------------------------
static int reset_state(qn_ctx *c, double tol, int max_it, int beta_mode, double beta_value,
                       cudaStream_t s) {
    DevState h;
    memset(&h, 0, sizeof(h));
    h.tol = tol;
    h.max_it = max_it;
    h.beta_mode = beta_mode;
    h.beta_value = beta_value;
    h.fx_headroom = c->res_fx_headroom;
    h.npts = (double)c->N;
    k_set_state<<<1, 32, 0, s>>>(c->st, h);
    QN_CUDA(cudaGetLastError());
    c->aux_launches += 1;
    return QN_OK;
}

static EpiArgs epi_args(qn_ctx *c, double *U, double step) {
    EpiArgs e;
    e.lam64 = c->lam64;
    e.lam32 = c->lam32;
    e.shift = &c->st->shift;
    e.step = step;
    e.U = U;
    e.dsq = c->warm_dsq_on ? c->warm_dsq : nullptr;
    e.done = &c->st->done;
    e.err = c->err;
    return e;
}

// Residual of U into the first working buffer (split planes or FP64), with partials.
static int enqueue_residual(qn_ctx *c, const double *U, const double *f, double *R64_override,
                            bool to_work, const int *done, cudaStream_t s) {
    ResidualArgs a{};
    a.U = U;
    a.f = f;
    a.n = c->n;
    a.dim = c->dim;
    a.inv_h2 = c->inv_h2;
    a.lam = c->prob.lam;
    a.b = c->prob.b;
    a.R64 = R64_override;
    a.Rhi = nullptr;
    a.Rlo = nullptr;
    a.P = c->P;
    if (to_work) {
        if (c->prob.precision == QN_PREC_FP64) {
            a.R64 = c->w64[0];
        } else {
            a.Rhi = c->bhi[0];
            a.Rlo = c->blo[0];
        }
    }
    a.partials = c->partials;
    a.done = done;
    // the split-precision solve only needs ||F|| to ~1e-7 for its stop test:
    // from its second iteration on (RMS(f) known, which scales the sum) its
    // residual sums float(r)^2 (Kahan) instead of an FP64 FMA per point
    const bool split_solve = to_work && c->prob.precision == QN_PREC_BF16X3;
    a.want_f2 = (!to_work || c->cur_iter == 0) ? 1 : 0;
    a.fast = (split_solve && !a.want_f2) ? 1 : 0;
    a.fp64_warps = split_solve ? c->res_fp64_warps : 0;
    a.r2_exp = &c->st->r2_exp;
    // the first residual of a 3-D split solve also writes the FP32-pair copy
    // of f; from the third iteration on (max|U| of the previous iterate known)
    // the residual runs without FP64 arithmetic
    a.fdf = split_solve ? c->fdf : nullptr;
    a.fx_fbad = &c->st->fx_fbad;
    a.fx_e = &c->st->fx_e;
    a.bc = c->prob.bc;
    a.pot = c->pot64;
    a.pot2 = c->pot2;
    a.umax_scan = &c->st->umax_scan;
    a.robin = (c->prob.bc == QN_BC_ROBIN) ? 2.0 * c->prob.robin_kappa / c->h : 0.0;
    a.hc0 = c->hc0;
    a.hlen = c->hlen;
    a.hval = c->hval;
    a.hbw = c->hbw;
    // 3-D split solve: the residual without FP64 arithmetic (k_residual_tiled)
    // in every iteration. It needs the FP32-pair copy of f and a fixed-point
    // exponent from max|U|: iteration 0 prepares both in one pass over f and
    // U_0 (and takes ||f|| there), iteration 1 scans max|U_1|, later ones take
    // max|U| from the previous residual.
    const bool tiled = split_solve && c->fdf != nullptr && c->res_tiled;
    c->res_saved_fnorm = (c->cur_iter > 0 || tiled) ? 1 : 0;
    int rc = QN_OK;
    // reflection-split layout of the planes (read by the split mode products)
    const bool mirror = tiled && c->split;
    c->split_layout = mirror ? 1 : 0;
    if (tiled && c->cur_iter <= 1) {
        const long pp = prof_begin(c, PK_RESIDUAL, s);
        if (c->cur_iter == 0) {
            // without a potential the pass also writes the zero start's residual -f, and the
            // residual below only writes its partial records when U_0 = 0
            const bool zs = (c->pot64 == nullptr);
            rc = launch_prep_split(U, f, c->n, c->P, c->fdf, zs ? a.Rhi : nullptr, zs ? a.Rlo : nullptr, c->partials,
                                   c->nparts, c->st, mirror, s);
            a.zero_start = zs ? c->st : nullptr;
        }
        else
            rc = launch_umax(U, c->N, c->st, 2 * c->num_sms, s);
        prof_end(c, pp, s);
        if (rc) return rc;
        c->launches += 1;   // two kernels per preparation step
    }
    if (tiled) {
        a.fast = 1;
        a.want_f2 = 0;
    }
    // the residual fused into the first forward product: iterations >= 1 (iteration 0
    // keeps the preparation pass and its zero-start shortcut), Dirichlet data, no potential
    c->fused_first = 0;
    const bool fz = mirror && c->fused && c->cur_iter >= 1 && a.pot == nullptr && a.bc == QN_BC_DIRICHLET;
    // the iteration-0 launch after the preparation pass (which skips its work for a zero
    // start) is accounted with the preparation, so that the tiled kind covers full evaluations
    const long pr = prof_begin(c, fz ? PK_FUSED : (tiled && a.zero_start == nullptr) ? PK_RESIDUAL_TILED : PK_RESIDUAL, s);
    if (fz) {
        FusedFwd ff;
        rc = tc_plan_fused_args(c->plan, 1, c->err, &ff);
        if (rc == QN_OK) rc = launch_fused_residual_fwd(a, ff, &c->res_parts, s);
        c->fused_first = 1;
        c->fused_used = 1;
    } else if (mirror) {
        rc = launch_residual_mirror(a, c->nparts, c->res_zc, &c->res_parts, s);
    } else if (tiled) {
        rc = launch_residual_tiled(a, c->nparts, c->res_zc, &c->res_parts, s);
    } else {
        rc = launch_residual(a, c->nparts, s);
        c->res_parts = c->nparts;
    }
    prof_end(c, pr, s);
    return rc;
}

// Shifted inverse of working buffer 0 (or of `r0` for the FP64 path), written
// as U -= step*delta (update=true) or V = delta (update=false).
static int enqueue_inverse(qn_ctx *c, const double *r0, double *target, bool update, double step,
                           cudaStream_t s, bool split = false, bool skip_first = false) {
    const int d = c->dim;
    EpiArgs e = epi_args(c, target, step);
    c->last_split = (split && update) ? 1 : 0;
    if (split && update) {
        // reflection-split products on the split / folded planes of the residual
        e.lam32 = c->lam32_split;
        const Epi seq[6] = {EPI_STORE_BFLY, EPI_STORE_BFLY, EPI_DIVIDE, EPI_STORE_PQ, EPI_STORE_PQ, EPI_UPDATE_PQ};
        // skip_first: the fused residual kernel already wrote the first product to buffer 1
        int cur = skip_first ? 1 : 0;
        for (int i = skip_first ? 1 : 0; i < 6; ++i) {
            const bool last = (i == 5);
            const int next = 1 - cur;
            const long pr = prof_begin(c, last ? PK_MP_LAST : (i == 2 ? PK_MP_DIVIDE : PK_MP_STORE), s);
            const int rc = launch_modeprod_tc_split(c->plan, cur, last ? -1 : next, seq[i], e, s, c->x6 && i >= 2);
            prof_end(c, pr, s);
            if (rc != QN_OK) return rc;
            cur = next;
        }
        return QN_OK;
    }
    int cur = 0;
    for (int i = 0; i < 2 * d; ++i) {
        const bool forward = i < d;
        const bool last = (i == 2 * d - 1);
        Epi epi = EPI_STORE;
        if (i == d - 1) epi = EPI_DIVIDE;
        if (last) epi = update ? EPI_UPDATE : EPI_DENSE;
        const int next = 1 - cur;
        int rc;
        const long pr = prof_begin(c, last ? PK_MP_LAST : (epi == EPI_DIVIDE ? PK_MP_DIVIDE : PK_MP_STORE), s);
        if (c->prob.precision == QN_PREC_FP64) {
            GemmShape g;
            g.n = c->n;
            g.P = c->n;
            g.dim = d;
            g.K = c->n;
            g.N = c->n;
            g.Mtot = (d == 3) ? c->n * c->n : c->n;
            g.split = c->f64_split ? (forward ? 1 : 2) : 0;
            c->last_split = c->f64_split;
            const double *A = (i == 0 && r0 != nullptr) ? r0 : c->w64[cur];
            const double *B = forward ? c->Si64 : c->S64;
            double *o = last ? target : c->w64[next];
            rc = launch_modeprod_f64(A, B, o, g, epi, e, s);
        } else {
            rc = launch_modeprod_tc(c->plan, cur, last ? -1 : next, forward, epi, e, s);
        }
        prof_end(c, pr, s);
        if (rc != QN_OK) return rc;
        cur = next;
    }
    return QN_OK;
}

static int enqueue_iteration(qn_ctx *c, double *U, const double *f, double step, cudaStream_t s) {
    int rc = enqueue_residual(c, U, f, nullptr, true, &c->st->done, s);
    if (rc) return rc;
    const long pr = prof_begin(c, PK_FINALIZE, s);
    rc = launch_finalize(c->partials, c->res_parts, c->st, c->hist, kHistCap, c->prob.b, c->prob.lam, 1,
                         c->res_saved_fnorm, c->pot64 != nullptr, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    return enqueue_inverse(c, nullptr, U, true, step, s, c->split_layout != 0, c->fused_first != 0);
}

// Capture `chunk` steady-state iterations (third iteration on: the residual
// takes its fixed-point exponent from the previous iterate, no preparation
// passes) into a CUDA graph on a private stream, once per (U, f, step, chunk).
static int enqueue_eig_iteration(qn_ctx *c, double *U, double step, cudaStream_t s);

static int ensure_iteration_graph(qn_ctx *c, double *U, const double *f, double step, int chunk, int kind = 0) {
    if (c->gexec && c->g_U == U && c->g_f == f && c->g_step == step && c->g_chunk == chunk && c->g_kind == kind &&
        c->g_x6 == c->x6 && c->g_fused == c->fused)
        return QN_OK;
    qn_ctx::GraphSlot cur{c->gexec, c->g_U, c->g_f, c->g_step, c->g_chunk, c->g_kind, c->g_x6, c->g_fused,
                          c->g_launches};
    const qn_ctx::GraphSlot &pv = c->g_prev;
    if (pv.exec && pv.U == U && pv.f == f && pv.step == step && pv.chunk == chunk && pv.kind == kind &&
        pv.x6 == c->x6 && pv.fused == c->fused) {
        // the previous graph matches: swap it in
        c->gexec = pv.exec;
        c->g_U = pv.U;
        c->g_f = pv.f;
        c->g_step = pv.step;
        c->g_chunk = pv.chunk;
        c->g_kind = pv.kind;
        c->g_x6 = pv.x6;
        c->g_fused = pv.fused;
        c->g_launches = pv.launches;
        c->g_prev = cur;
        return QN_OK;
    }
    // capture a new one; the current one becomes the previous, the older one goes
    if (c->g_prev.exec) cudaGraphExecDestroy(c->g_prev.exec);
    c->g_prev = cur;
    c->gexec = nullptr;
    if (!c->cap_stream) QN_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const long long l0 = c->launches;
    const int it0 = c->cur_iter;
    QN_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = QN_OK;
    for (int k = 0; k < chunk && rc == QN_OK; ++k) {
        c->cur_iter = 2 + k;
        rc = (kind == 1) ? enqueue_eig_iteration(c, U, step, c->cap_stream)
                         : enqueue_iteration(c, U, f, step, c->cap_stream);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->cur_iter = it0;
    c->g_launches = c->launches - l0;
    c->launches = l0;
    if (rc != QN_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture (solve iterations)");
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate (solve iterations)");
    }
    c->g_U = U;
    c->g_f = f;
    c->g_step = step;
    c->g_chunk = chunk;
    c->g_kind = kind;
    c->g_x6 = c->x6;
    c->g_fused = c->fused;
    return QN_OK;
}

// The state after the work queued so far on s: a kernel mirrors it into mapped host
// memory, and the host waits for s alone.
static int read_state(qn_ctx *c, DevState *h, cudaStream_t s) {
    k_mirror_state<<<1, 32, 0, s>>>(c->st, c->err, c->hist, kHistCap, c->mir_dev);
    QN_CUDA(cudaGetLastError());
    c->aux_launches += 1;
    QN_CUDA(cudaStreamSynchronize(s));
    const volatile StateMirror *m = c->mir_host;
    memcpy(h, const_cast<const StateMirror *>(m), sizeof(DevState));
    if (m->err) {
        set_error("a device-side wait gave up (tensor-core pipeline timeout)");
        return QN_ETIMEOUT;
    }
    return QN_OK;
}

static bool bad_ptr(const void *p) { return p == nullptr; }

// ---- public entry points -----------------------------------------------------------------
extern "C" int qn_residual(qn_ctx *c, const double *U, const double *f, double *R, qn_stats *st,
                           void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(U) || bad_ptr(f)) {
        set_error("qn_residual: null U or f");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = reset_state(c, -1.0, 0, QN_BETA_PAPER, 0.0, s);
    if (rc) return rc;
    rc = enqueue_residual(c, U, f, R, false, nullptr, s);
    if (rc) return rc;
    const long pr = prof_begin(c, PK_FINALIZE, s);
    rc = launch_finalize(c->partials, c->res_parts, c->st, c->hist, kHistCap, c->prob.b, c->prob.lam, 0, 0,
                         c->pot64 != nullptr, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    if (st) {
        QN_CUDA(cudaMemcpyAsync(st, c->hist, sizeof(qn_stats), cudaMemcpyDeviceToHost, s));
        QN_CUDA(cudaStreamSynchronize(s));
    }
    return QN_OK;
}

extern "C" int qn_fast_diag_solve(qn_ctx *c, const double *r, double *V, double shift, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(r) || bad_ptr(V) || r == V) {
        set_error("qn_fast_diag_solve: r and V must be distinct non-null device arrays");
        return QN_EINVAL;
    }
    if (!isfinite(shift)) {
        set_error("qn_fast_diag_solve: shift must be finite");
        return QN_EINVAL;
    }
    // smallest eigenvalue of sum_a H_a is dim * lambda_1 (0 for Neumann data: constants)
    const double l1 = (c->prob.bc == QN_BC_NEUMANN) ? 0.0 : fmax(c->lam_min, 0.0);
    if (!(shift > -c->dim * l1)) {
        set_error("qn_fast_diag_solve: shift %.6g makes the operator singular or indefinite", shift);
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = reset_state(c, -1.0, 0, QN_BETA_FIXED, 0.0, s);
    if (rc) return rc;
    QN_CUDA(cudaMemcpyAsync(&c->st->shift, &shift, sizeof(double), cudaMemcpyHostToDevice, s));
    if (c->prob.precision == QN_PREC_FP64) {
        return enqueue_inverse(c, r, V, false, 1.0, s);
    }
    const long pr = prof_begin(c, PK_SPLIT, s);
    rc = launch_split_pad(r, c->n, c->P, c->dim, c->bhi[0], c->blo[0], 4 * c->num_sms, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    return enqueue_inverse(c, nullptr, V, false, 1.0, s);
}

extern "C" int qn_step(qn_ctx *c, double *U, const double *f, double beta, qn_stats *st, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(U) || bad_ptr(f)) {
        set_error("qn_step: null U or f");
        return QN_EINVAL;
    }
    if (isinf(beta)) {
        set_error("qn_step: beta must be finite or NaN (paper rule)");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool paper = isnan(beta);
    c->x6 = c->x6_base;
    rc = reset_state(c, -1.0, 1, paper ? QN_BETA_PAPER : QN_BETA_FIXED, paper ? 0.0 : beta, s);
    if (rc) return rc;
    c->cur_iter = 0;
    rc = enqueue_iteration(c, U, f, 1.0, s);
    if (rc) return rc;
    DevState h;
    rc = read_state(c, &h, s);
    if (rc) return rc;
    if (st) QN_CUDA(cudaMemcpy(st, c->hist, sizeof(qn_stats), cudaMemcpyDeviceToHost));
    if (h.done && h.status == QN_EDIVERGED) {
        set_error("qn_step: non-finite residual or beta");
        return QN_EDIVERGED;
    }
    return QN_OK;
}

bool qn::ctx_split_precision(const qn_ctx *c) { return c != nullptr && c->prob.precision == QN_PREC_BF16X3; }

bool qn::ctx_unit_dirichlet(const qn_ctx *c) {
    return c != nullptr && c->prob.bc == QN_BC_DIRICHLET && c->pot64 == nullptr && c->prob.sem_k == 0 &&
           fabs(c->h * (c->n + 1) - 1.0) < 1e-12;
}

// Precision escalation: the one-step contraction rel_it / rel_{it-1} of the residual
// against the quasi-Newton bound max|(N_h)_U - beta| / (lambda_min(A_h) + beta) at U_it
// (Sec. 5: the error of the simplified Jacobian). A contraction above esc_rate and above
// twice that bound comes from the split products' precision, not from the nonlinearity.
static bool escalation_due(const qn_ctx *c, int it) {
    if (it < 1) return false;   // `it`: the iterate evaluated last (the mirror's `last`)
    const volatile StateMirror *m = c->mir_host;
    const double rel = m->last.rel, rel0 = m->prev.rel, beta = m->last.beta;
    if (!(rel0 > 0.0) || !std::isfinite(rel)) return false;
    const double rho = rel / rel0;
    const double l1 = (c->prob.bc == QN_BC_NEUMANN) ? 0.0 : fmax(c->lam_min, 0.0);
    const double den = c->dim * l1 + c->prob.lam + beta;
    if (!(den > 0.0)) return false;
    const double bound = fmax(fabs(m->last.fu_max - beta), fabs(m->last.fu_min - beta)) / den;
    return rho > c->esc_rate && rho > 2.0 * bound;
}

extern "C" int qn_set_escalation(qn_ctx *c, double rate) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!(rate >= 0.0) || !std::isfinite(rate)) {
        set_error("qn_set_escalation: rate must be finite and >= 0");
        return QN_EINVAL;
    }
    if (rate > 0.0 && c->x6_base == 0) {
        if (c->prob.precision != QN_PREC_BF16X3 || !c->split) {
            set_error("qn_set_escalation: needs a BF16X3 context with the reflection-split products");
            return QN_EUNSUPPORTED;
        }
        rc = ensure_x6(c);
        if (rc) return rc;
    }
    c->esc_rate = rate;
    return QN_OK;
}

extern "C" int qn_set_fused_residual(qn_ctx *c, int on) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (on) {
        if (c->dim != 3 || c->prob.precision != QN_PREC_BF16X3 || !c->split || c->fdf == nullptr || !c->res_tiled ||
            c->prob.bc != QN_BC_DIRICHLET || c->pot64 != nullptr || c->prob.sem_k > 0) {
            set_error("qn_set_fused_residual: needs a 3-D BF16X3 / BF16X6 finite-difference context with the "
                      "reflection-split products, Dirichlet data and no potential");
            return QN_EUNSUPPORTED;
        }
        rc = tc_plan_enable_fused(c->plan);
        if (rc == QN_EUNSUPPORTED) set_error("qn_set_fused_residual: the fused kernel takes P <= 512");
        if (rc) return rc;
    }
    c->fused = on ? 1 : 0;
    return QN_OK;
}

extern "C" int qn_solve(qn_ctx *c, double *U, const double *f, const qn_opts *opts, qn_result *res,
                        qn_stats *history, int history_len, void *stream) {
    return solve_internal(c, U, f, opts, res, history, history_len, stream, nullptr, nullptr);
}

int qn::solve_internal(qn_ctx *c, double *U, const double *f, const qn_opts *opts, qn_result *res,
                       qn_stats *history, int history_len, void *stream, const double *u0_sq, int *used_warm) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(U) || bad_ptr(f)) {
        set_error("qn_solve: null U or f");
        return QN_EINVAL;
    }
    qn_opts o;
    if (opts) {
        o = *opts;
    } else {
        o.tol = 1e-10;
        o.max_it = 200;
        o.beta_mode = QN_BETA_PAPER;
        o.beta_value = 0.0;
        o.step = 1.0;
        o.sync_every = 2;
        o.graph = 0;
    }
    if (!(o.tol >= 0.0) || o.max_it < 0 || o.max_it > kHistCap - 1 || !isfinite(o.step) ||
        (o.beta_mode != QN_BETA_PAPER && o.beta_mode != QN_BETA_FIXED) ||
        (o.beta_mode == QN_BETA_FIXED && !isfinite(o.beta_value))) {
        set_error("qn_solve: invalid options");
        return QN_EINVAL;
    }
    if (o.sync_every < 1) o.sync_every = 1;
    if (history_len < 0 || (history_len > 0 && history == nullptr)) {
        set_error("qn_solve: invalid history buffer");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->aux_launches = 0;
    c->x6 = c->x6_base;
    c->esc_at = c->x6_base ? 0 : -1;
    c->fused_used = 0;
    rc = reset_state(c, o.tol, o.max_it, o.beta_mode, o.beta_value, s);
    if (rc) return rc;
    DevState h;
    memset(&h, 0, sizeof(h));
    int enqueued = 0;
    size_t first_rec = c->prof_used;
    long long launches0 = c->launches;
    if (u0_sq != nullptr && c->prob.precision == QN_PREC_BF16X3) {
        // warm start: the first iteration from U_0 also sums ||U_1 - U_0||^2 =
        // ||step * delta||^2 in its last mode product. delta estimates the
        // error of U_0: keep going from U_1 if it is below ||U_0|| / 2, else
        // restart from the zero start
        if (!c->warm_dsq) QN_CUDA(cudaMalloc(&c->warm_dsq, sizeof(float)));
        QN_CUDA(cudaMemsetAsync(c->warm_dsq, 0, sizeof(float), s));
        c->cur_iter = 0;
        c->warm_dsq_on = 1;
        rc = enqueue_iteration(c, U, f, o.step, s);
        c->warm_dsq_on = 0;
        if (rc) return rc;
        enqueued = 1;
        rc = read_state(c, &h, s);
        if (rc) return rc;
        float dsq = 0.0f;
        double u2 = 0.0;
        QN_CUDA(cudaMemcpy(&dsq, c->warm_dsq, sizeof(float), cudaMemcpyDeviceToHost));
        QN_CUDA(cudaMemcpy(&u2, u0_sq, sizeof(double), cudaMemcpyDeviceToHost));
        const bool converged0 = h.done && h.status == QN_OK && h.it == 0;
        const bool keep = converged0 || (std::isfinite(dsq) && std::isfinite(u2) && u2 > 0.0 &&
                                         (double)dsq < 0.25 * u2 && !(h.done && h.status != QN_OK));
        if (used_warm) *used_warm = keep ? 1 : 0;
        if (!keep) {
            // restart from U = 0: the launches so far stay in the accounting
            QN_CUDA(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)c->N, s));
            rc = reset_state(c, o.tol, o.max_it, o.beta_mode, o.beta_value, s);
            if (rc) return rc;
            memset(&h, 0, sizeof(h));
            enqueued = 0;
            first_rec = c->prof_used;
            launches0 = c->launches;
        }
    } else if (used_warm) {
        *used_warm = 0;
    }
    const bool use_graph = o.graph != 0 && !c->prof_on;
    const bool small = c->small_solve && u0_sq == nullptr && !c->prof_on;
    if (small) {
        SmallSolve q;
        q.U = U;
        q.f = f;
        q.S = c->S64;
        q.Si = c->Si64;
        q.lam1 = c->lam64;
        q.w0 = c->w64[0];
        q.w1 = c->w64[1];
        q.partials = c->partials;
        q.partials_cap = c->partials_cap;
        q.bar = c->small_bar;
        q.st = c->st;
        q.hist = c->hist;
        q.hist_cap = kHistCap;
        q.err = c->err;
        q.n = c->n;
        q.neumann = (c->prob.bc == QN_BC_NEUMANN) ? 1 : 0;
        q.num_sms = c->num_sms;
        q.inv_h2 = c->inv_h2;
        q.lam = c->prob.lam;
        q.b = c->prob.b;
        q.tol = o.tol;
        q.beta_value = o.beta_value;
        q.step = o.step;
        q.beta_fixed = (o.beta_mode == QN_BETA_FIXED) ? 1 : 0;
        q.max_it = o.max_it;
        rc = launch_small_solve(q, s);
        if (rc) return rc;
        rc = read_state(c, &h, s);
        if (rc) return rc;
    }
    while (!small && !h.done && enqueued <= o.max_it) {
        if (use_graph && enqueued >= 2 && enqueued + o.sync_every <= o.max_it + 1) {
            // steady-state iterations (the same launches every time): replay
            rc = ensure_iteration_graph(c, U, f, o.step, o.sync_every);
            if (rc) return rc;
            QN_CUDA(cudaGraphLaunch(c->gexec, s));
            c->launches += c->g_launches;
            enqueued += o.sync_every;
        } else {
            for (int k = 0; k < o.sync_every && enqueued <= o.max_it; ++k, ++enqueued) {
                c->cur_iter = enqueued;
                rc = enqueue_iteration(c, U, f, o.step, s);
                if (rc) return rc;
            }
        }
        rc = read_state(c, &h, s);
        if (rc) return rc;
        if (h.done) break;
        if (c->esc_rate > 0.0 && !c->x6 && escalation_due(c, h.it - 1)) {
            c->x6 = 1;
            c->esc_at = enqueued;
        }
    }
    if (!h.done) {   // cannot happen: the finaliser stops at max_it
        set_error("qn_solve: internal iteration accounting error");
        return QN_ECUDA;
    }
    const int its = h.it;
    int status = h.status;
    // launches queued past convergence returned at once: drop them from the accounting
    for (size_t i = first_rec; i < c->prof_used; ++i) {
        qn_ctx::ProfRec &r = (*c->prof)[i];
        const bool mp = r.kind >= PK_MP_STORE && r.kind <= PK_MP_LAST;
        if ((mp && r.iter >= its) || (!mp && r.iter > its)) r.valid = 0;
    }
    c->launches = small ? launches0 + 1 + c->aux_launches
                        : launches0 + 2LL * (its + 1) + 2LL * c->dim * its + c->aux_launches;
    if (c->prob.precision == QN_PREC_BF16X3 && c->fdf != nullptr && c->res_tiled)
        c->launches += 2 + (its >= 1 ? 2 : 0);   // preparation kernels of iterations 0 and 1
    // the fused residual of iterations 1 .. its - 1 also formed their first product
    if (!small && c->fused_used && its >= 2) c->launches -= its - 1;
    // the statistics of the final iterate came with the last state mirror
    qn_stats last;
    memcpy(&last, const_cast<const qn_stats *>(&((const volatile StateMirror *)c->mir_host)->last), sizeof(last));
    if (history && history_len > 0) {
        const int cnt = (its + 1) < history_len ? (its + 1) : history_len;
        QN_CUDA(cudaMemcpy(history, c->hist, sizeof(qn_stats) * cnt, cudaMemcpyDeviceToHost));
    }
    if (res) {
        res->iterations = its;
        res->status = status;
        res->rel = last.rel;
    }
    if (status == QN_ENOTCONV) set_error("qn_solve: max_it reached (rel %.3e)", last.rel);
    if (status == QN_EDIVERGED) set_error("qn_solve: diverged (rel %.3e)", last.rel);
    return status;
}

// Host-array solve: f_host (and, unless zero_start, the start U_host) to context-owned
// device buffers, the solve, the result back into U_host.
static int solve_host(qn_ctx *c, double *U_host, const double *f_host, bool zero_start, const qn_opts *opts,
                      qn_result *res, qn_stats *history, int history_len, void *stream, const char *who) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(U_host) || bad_ptr(f_host)) {
        set_error("%s: null U_host or f_host", who);
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)c->N;
    if (!c->dU) {
        QN_CUDA(cudaMalloc(&c->dU, bytes));
        QN_CUDA(cudaMalloc(&c->df, bytes));
    }
    QN_CUDA(cudaMemcpyAsync(c->df, f_host, bytes, cudaMemcpyHostToDevice, s));
    if (zero_start)
        QN_CUDA(cudaMemsetAsync(c->dU, 0, bytes, s));   // +0.0 is all-zero bits
    else
        QN_CUDA(cudaMemcpyAsync(c->dU, U_host, bytes, cudaMemcpyHostToDevice, s));
    rc = qn_solve(c, c->dU, c->df, opts, res, history, history_len, stream);
    if (rc != QN_OK && rc != QN_ENOTCONV && rc != QN_EDIVERGED) return rc;
    QN_CUDA(cudaMemcpyAsync(U_host, c->dU, bytes, cudaMemcpyDeviceToHost, s));
    QN_CUDA(cudaStreamSynchronize(s));
    return rc;
}

extern "C" int qn_solve_host(qn_ctx *c, double *U_host, const double *f_host, const qn_opts *opts,
                             qn_result *res, qn_stats *history, int history_len, void *stream) {
    return solve_host(c, U_host, f_host, false, opts, res, history, history_len, stream, "qn_solve_host");
}

extern "C" int qn_solve_host_zero_start(qn_ctx *c, double *U_host, const double *f_host, const qn_opts *opts,
                                        qn_result *res, qn_stats *history, int history_len, void *stream) {
    return solve_host(c, U_host, f_host, true, opts, res, history, history_len, stream,
                      "qn_solve_host_zero_start");
}

// A sequence of host-array solves with one context: problem i+1 is copied in and
// problem i-1 copied out on two copy streams while problem i is solved on `stream`,
// through two pairs of context-owned device buffers.
extern "C" int qn_solve_host_many(qn_ctx *c, int count, double *const *U_host, const double *const *f_host,
                                  int zero_start, const qn_opts *opts, qn_result *results, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!U_host || !f_host || !results))) {
        set_error("qn_solve_host_many: count < 0 or null arrays");
        return QN_EINVAL;
    }
    for (int i = 0; i < count; ++i)
        if (bad_ptr(U_host[i]) || bad_ptr(f_host[i])) {
            set_error("qn_solve_host_many: null U_host[%d] or f_host[%d]", i, i);
            return QN_EINVAL;
        }
    if (count == 0) return QN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)c->N;
    for (int b = 0; b < 2; ++b) {
        if (!c->hm_U[b]) {
            QN_CUDA(cudaMalloc(&c->hm_U[b], bytes));
            QN_CUDA(cudaMalloc(&c->hm_f[b], bytes));
            QN_CUDA(cudaEventCreateWithFlags(&c->hm_in_ready[b], cudaEventDisableTiming));
            QN_CUDA(cudaEventCreateWithFlags(&c->hm_solved[b], cudaEventDisableTiming));
            QN_CUDA(cudaEventCreateWithFlags(&c->hm_out_done[b], cudaEventDisableTiming));
        }
    }
    if (!c->hm_h2d) QN_CUDA(cudaStreamCreateWithFlags(&c->hm_h2d, cudaStreamNonBlocking));
    if (!c->hm_d2h) QN_CUDA(cudaStreamCreateWithFlags(&c->hm_d2h, cudaStreamNonBlocking));
    // inputs of problem i into buffer pair i & 1, once problem i - 2 has left it
    auto enqueue_in = [&](int i) -> int {
        const int b = i & 1;
        if (i >= 2) QN_CUDA(cudaStreamWaitEvent(c->hm_h2d, c->hm_out_done[b], 0));
        QN_CUDA(cudaMemcpyAsync(c->hm_f[b], f_host[i], bytes, cudaMemcpyHostToDevice, c->hm_h2d));
        if (zero_start)
            QN_CUDA(cudaMemsetAsync(c->hm_U[b], 0, bytes, c->hm_h2d));   // +0.0 is all-zero bits
        else
            QN_CUDA(cudaMemcpyAsync(c->hm_U[b], U_host[i], bytes, cudaMemcpyHostToDevice, c->hm_h2d));
        QN_CUDA(cudaEventRecord(c->hm_in_ready[b], c->hm_h2d));
        return QN_OK;
    };
    int err = enqueue_in(0);
    for (int i = 0; i < count && err == QN_OK; ++i) {
        const int b = i & 1;
        if (i + 1 < count) {
            err = enqueue_in(i + 1);
            if (err != QN_OK) break;
        }
        cudaError_t ce = cudaStreamWaitEvent(s, c->hm_in_ready[b], 0);
        if (ce != cudaSuccess) {
            err = cuda_fail(ce, "cudaStreamWaitEvent (qn_solve_host_many)");
            break;
        }
        rc = qn_solve(c, c->hm_U[b], c->hm_f[b], opts, &results[i], nullptr, 0, stream);
        if (rc != QN_OK && rc != QN_ENOTCONV && rc != QN_EDIVERGED) {
            err = rc;
            break;
        }
        if ((ce = cudaEventRecord(c->hm_solved[b], s)) != cudaSuccess ||
            (ce = cudaStreamWaitEvent(c->hm_d2h, c->hm_solved[b], 0)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(U_host[i], c->hm_U[b], bytes, cudaMemcpyDeviceToHost, c->hm_d2h)) != cudaSuccess ||
            (ce = cudaEventRecord(c->hm_out_done[b], c->hm_d2h)) != cudaSuccess) {
            err = cuda_fail(ce, "copy-out (qn_solve_host_many)");
            break;
        }
    }
    // every copy has landed (or been abandoned after an error) before the call returns
    const cudaError_t e1 = cudaStreamSynchronize(c->hm_h2d);
    const cudaError_t e2 = cudaStreamSynchronize(c->hm_d2h);
    const cudaError_t e3 = cudaStreamSynchronize(s);
    if (err != QN_OK) return err;
    if (e1 != cudaSuccess) return cuda_fail(e1, "cudaStreamSynchronize (copy-in)");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize (copy-out)");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize (solve stream)");
    return QN_OK;
}

extern "C" int qn_test_withhold_arrival(void) { return tc_test_withhold_arrival(); }

extern "C" int qn_profile_enable(qn_ctx *c, int on) {
    int rc = check_ctx(c);
    if (rc) return rc;
    c->prof_on = on ? 1 : 0;
    c->prof_used = 0;
    c->launches = 0;
    return QN_OK;
}

extern "C" int qn_profile_read(qn_ctx *c, qn_profile *out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!out) {
        set_error("qn_profile_read: null output");
        return QN_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    out->launches = c->launches;
    double ms[PK_COUNT] = {0};
    int cnt[PK_COUNT] = {0};
    for (size_t i = 0; i < c->prof_used; ++i) {
        qn_ctx::ProfRec &r = (*c->prof)[i];
        if (!r.valid) continue;
        QN_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        QN_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.kind] += t;
        cnt[r.kind] += 1;
    }
    out->residual_launches = cnt[PK_RESIDUAL] + cnt[PK_RESIDUAL_TILED];
    out->residual_ms = ms[PK_RESIDUAL] + ms[PK_RESIDUAL_TILED];
    out->residual_tiled_launches = cnt[PK_RESIDUAL_TILED];
    out->residual_tiled_ms = ms[PK_RESIDUAL_TILED];
    out->split_products = c->last_split;
    out->x6_from = c->esc_at;
    out->finalize_launches = cnt[PK_FINALIZE];
    out->finalize_ms = ms[PK_FINALIZE];
    out->modeprod_launches = cnt[PK_MP_STORE] + cnt[PK_MP_DIVIDE] + cnt[PK_MP_LAST];
    out->modeprod_ms = ms[PK_MP_STORE] + ms[PK_MP_DIVIDE] + ms[PK_MP_LAST];
    out->mp_store_launches = cnt[PK_MP_STORE];
    out->mp_store_ms = ms[PK_MP_STORE];
    out->mp_divide_launches = cnt[PK_MP_DIVIDE];
    out->mp_divide_ms = ms[PK_MP_DIVIDE];
    out->mp_last_launches = cnt[PK_MP_LAST];
    out->mp_last_ms = ms[PK_MP_LAST];
    out->fused_launches = cnt[PK_FUSED];
    out->fused_ms = ms[PK_FUSED];
    return QN_OK;
}

// ---- nonlinear eigenproblem (Sec. 4.4) ----------------------------------------------------------
// One iteration (qn_eig.cu): pass 1 (A U~ + (lam + V) U~ and the Rayleigh sums), lambda_n and
// the normalisation factor, pass 2 (U = s U~, F into the inverse's input, beta's extremes), stop
// test and beta_n, the shifted inverse with the update. In split precision the passes run in
// float pairs from iteration 1 on (their fixed-point exponent comes from the previous iterate).
static int enqueue_eig_iteration(qn_ctx *c, double *U, double step, cudaStream_t s) {
    const double hd = pow(c->h, c->dim);
    const int grid = c->nparts;
    const bool fp64 = (c->prob.precision == QN_PREC_FP64);
    const bool df = !fp64 && c->cur_iter >= 1;
    double *lin = fp64 ? c->w64[1] : c->eig_r0;   // w64[1] is free until the first mode product
    float2 *lin2 = reinterpret_cast<float2 *>(c->eig_r0);   // the same 8 bytes per node, as a pair
    const bool mirror = !fp64 && c->split;
    long pr = prof_begin(c, PK_RESIDUAL, s);
    int grid1 = grid;   // blocks (partial sums) of pass 1
    int rc = df ? launch_eig_pass1_df(U, lin2, c->n, c->dim, c->prob.bc, c->inv_h2, c->prob.lam, c->prob.b, c->pot64,
                                      c->eig_vrow, c->eig_potx2, c->eig_vrow2, c->partials, grid, &grid1, c->st, s)
                : launch_eig_pass1(U, lin, c->n, c->dim, c->prob.bc, c->inv_h2, c->prob.lam, c->prob.b, c->pot64,
                                   c->eig_vrow, c->partials, grid, c->st, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    pr = prof_begin(c, PK_FINALIZE, s);
    rc = launch_eig_finalize1(c->partials, grid1, hd, c->st, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    pr = prof_begin(c, PK_RESIDUAL, s);
    int grid2 = grid;   // blocks (partial sums) of pass 2
    if (df)
        rc = launch_eig_pass2_df(U, lin2, c->n, c->P, c->dim, c->prob.bc, hd, (float)c->prob.lam, c->prob.b,
                                 c->eig_pot32, c->bhi[0], c->blo[0], mirror, c->partials, c->partials_cap, &grid2,
                                 c->st, s);
    else
        rc = launch_eig_pass2(U, lin, c->n, c->P, c->dim, c->prob.bc, hd, (float)c->prob.lam, c->prob.b,
                              c->eig_pot32, fp64 ? c->w64[0] : nullptr, fp64 ? nullptr : c->bhi[0],
                              fp64 ? nullptr : c->blo[0], mirror, c->partials, grid, c->st, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    pr = prof_begin(c, PK_FINALIZE, s);
    rc = launch_finalize(c->partials, grid2, c->st, c->hist, kHistCap, c->prob.b, c->prob.lam, 1, 1, 2, s);
    prof_end(c, pr, s);
    if (rc) return rc;
    return enqueue_inverse(c, nullptr, U, true, step, s, mirror);
}

extern "C" int qn_eig_solve(qn_ctx *c, double *U, const qn_opts *opts, qn_result *res, double *lambda,
                            qn_stats *history, int history_len, void *stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (bad_ptr(U)) {
        set_error("qn_eig_solve: null U");
        return QN_EINVAL;
    }
    if (c->prob.sem_k > 0 || c->prob.bc == QN_BC_ROBIN) {
        set_error("qn_eig_solve: finite differences with Dirichlet or Neumann data only");
        return QN_EUNSUPPORTED;
    }
    qn_opts o;
    if (opts) {
        o = *opts;
    } else {
        o.tol = 1e-10;
        o.max_it = kHistCap - 1;
        o.beta_mode = QN_BETA_PAPER;
        o.beta_value = 0.0;
        o.step = 1.0;
        o.sync_every = 8;
        o.graph = 0;
    }
    if (!(o.tol >= 0.0) || o.max_it < 0 || o.max_it > kHistCap - 1 || !isfinite(o.step) ||
        (o.beta_mode != QN_BETA_PAPER && o.beta_mode != QN_BETA_FIXED) ||
        (o.beta_mode == QN_BETA_FIXED && !isfinite(o.beta_value))) {
        set_error("qn_eig_solve: invalid options");
        return QN_EINVAL;
    }
    if (o.sync_every < 1) o.sync_every = 1;
    if (history_len < 0 || (history_len > 0 && history == nullptr)) {
        set_error("qn_eig_solve: invalid history buffer");
        return QN_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->x6 = c->x6_base;
    if (c->prob.precision == QN_PREC_BF16X3 && !c->eig_r0)
        QN_CUDA(cudaMalloc(&c->eig_r0, sizeof(double) * (size_t)c->N));
    if (c->pot64 != nullptr && !c->eig_vrow) {
        // per (y, z) row: lam + v_y + v_z; and FP32 copies of the tables (beta's extremes)
        const int n = c->n, dn = c->dim * n;
        std::vector<double> pt(dn);
        QN_CUDA(cudaMemcpy(pt.data(), c->pot64, sizeof(double) * dn, cudaMemcpyDeviceToHost));
        const size_t rows = (c->dim == 3) ? (size_t)n * n : (size_t)n;
        std::vector<double> vr(rows);
        for (size_t r = 0; r < rows; ++r) {
            const int y = (int)(r % n), z = (int)(r / n);
            vr[r] = c->prob.lam + pt[n + y] + ((c->dim == 3) ? pt[2 * n + z] : 0.0);
        }
        std::vector<float> p32(dn);
        for (int i = 0; i < dn; ++i) p32[i] = (float)pt[i];
        std::vector<float2> vr2(rows), px2(n);
        for (size_t r = 0; r < rows; ++r) {
            const float hi = (float)vr[r];
            vr2[r] = make_float2(hi, (float)(vr[r] - (double)hi));
        }
        for (int i = 0; i < n; ++i) {
            const float hi = (float)pt[i];
            px2[i] = make_float2(hi, (float)(pt[i] - (double)hi));
        }
        QN_CUDA(cudaMalloc(&c->eig_vrow2, sizeof(float2) * rows));
        QN_CUDA(cudaMalloc(&c->eig_potx2, sizeof(float2) * n));
        QN_CUDA(cudaMemcpy(c->eig_vrow2, vr2.data(), sizeof(float2) * rows, cudaMemcpyHostToDevice));
        QN_CUDA(cudaMemcpy(c->eig_potx2, px2.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
        QN_CUDA(cudaMalloc(&c->eig_vrow, sizeof(double) * rows));
        QN_CUDA(cudaMalloc(&c->eig_pot32, sizeof(float) * dn));
        QN_CUDA(cudaMemcpy(c->eig_vrow, vr.data(), sizeof(double) * rows, cudaMemcpyHostToDevice));
        QN_CUDA(cudaMemcpy(c->eig_pot32, p32.data(), sizeof(float) * dn, cudaMemcpyHostToDevice));
    }
    c->aux_launches = 0;
    rc = reset_state(c, o.tol, o.max_it, o.beta_mode, o.beta_value, s);
    if (rc) return rc;
    const size_t first_rec = c->prof_used;
    const long long launches0 = c->launches;
    DevState h;
    memset(&h, 0, sizeof(h));
    int enqueued = 0;
    const bool use_graph = o.graph != 0 && !c->prof_on;
    while (!h.done && enqueued <= o.max_it) {
        if (use_graph && enqueued >= 1 && enqueued + o.sync_every <= o.max_it + 1) {
            rc = ensure_iteration_graph(c, U, nullptr, o.step, o.sync_every, 1);
            if (rc) return rc;
            QN_CUDA(cudaGraphLaunch(c->gexec, s));
            enqueued += o.sync_every;
        } else {
            for (int k = 0; k < o.sync_every && enqueued <= o.max_it; ++k, ++enqueued) {
                c->cur_iter = enqueued;
                rc = enqueue_eig_iteration(c, U, o.step, s);
                if (rc) return rc;
            }
        }
        rc = read_state(c, &h, s);
        if (rc) return rc;
    }
    if (!h.done) {
        set_error("qn_eig_solve: internal iteration accounting error");
        return QN_ECUDA;
    }
    const int its = h.it;
    const int status = h.status;
    for (size_t i = first_rec; i < c->prof_used; ++i) {
        qn_ctx::ProfRec &r = (*c->prof)[i];
        const bool mp = r.kind >= PK_MP_STORE && r.kind <= PK_MP_LAST;
        if ((mp && r.iter >= its) || (!mp && r.iter > its)) r.valid = 0;
    }
    // per evaluated iterate 2 residual passes + 2 finalisers; per update 2 dim products
    c->launches = launches0 + 4LL * (its + 1) + 2LL * c->dim * its + c->aux_launches;
    qn_stats last;
    memcpy(&last, const_cast<const qn_stats *>(&((const volatile StateMirror *)c->mir_host)->last), sizeof(last));
    if (history && history_len > 0) {
        const int cnt = (its + 1) < history_len ? (its + 1) : history_len;
        QN_CUDA(cudaMemcpy(history, c->hist, sizeof(qn_stats) * cnt, cudaMemcpyDeviceToHost));
    }
    if (res) {
        res->iterations = its;
        res->status = status;
        res->rel = last.rel;
    }
    if (lambda) *lambda = last.lambda;
    if (status == QN_ENOTCONV) set_error("qn_eig_solve: max_it reached (rel %.3e)", last.rel);
    if (status == QN_EDIVERGED) set_error("qn_eig_solve: diverged (rel %.3e)", last.rel);
    return status;
}
