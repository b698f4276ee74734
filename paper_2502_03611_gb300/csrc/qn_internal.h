// Internal declarations shared by the libqn translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/qn.h"

namespace qn {

// Device-resident solver state: written by the reduction finaliser, read by
// every later kernel of the iteration (so the host need not synchronise
// between the residual and the inverse).
struct DevState {
    int done;        // 1 once converged / diverged / out of iterations: later kernels return at once
    int status;      // QN_OK, QN_ENOTCONV, QN_EDIVERGED
    int it;          // index of the iterate whose residual was evaluated last
    int err;         // nonzero if a device-side wait gave up (QN_ETIMEOUT)
    double shift;    // lam + beta_n used by the pointwise divide
    double beta;     // beta_n
    double tol;
    int max_it;
    int beta_mode;
    double beta_value;
    double f_norm;   // ||f||_2, computed on the first iteration of a solve
    int fx_e;        // fixed-point exponent for the next residual of the split solve
                     // (biased exponent of max|U| + 2; 0: not usable, see k_residual_tiled)
    int fx_fbad;     // 1: some |f| is too large for the FP32-pair copy of f
    int fx_headroom; // fx_e = biased exponent of max|U| + fx_headroom (2: U may grow 4x
                     // before a plane takes the exact path; smaller values send more there)
    int r2_exp;      // k: the FP32 sum of r^2 inside the split solve adds (r 2^-k)^2,
                     // 2^k ~ RMS(f) (set on the first iteration), so it neither
                     // overflows nor underflows for any scale of f
    double npts;     // number of unknowns (for RMS(f))
    unsigned long long umax_scan;   // max|U| bit pattern from a scan pass (k_prep_split, k_umax)
    double eig_lambda;   // eigen solves: Rayleigh quotient lambda_n of the current iterate
    double eig_scale;    //   and the normalisation factor 1/||U~|| applied to it
    float2 eig_lambda2, eig_scale2;   // the same two as FP32 pairs (hi, lo)
    int u0_zero;     // 1: the preparation pass found U_0 = 0 (and wrote the residual -f)
};

// Residual kernel outputs.
struct ResidualArgs {
    const double *U;
    const double *f;
    int n, dim;
    double inv_h2, lam, b;
    double *R64;               // dense FP64 residual or nullptr
    __nv_bfloat16 *Rhi;        // padded split planes (P per axis) or nullptr
    __nv_bfloat16 *Rlo;
    int P;
    double *partials;          // [grid][4] : sum r^2, sum f^2, min U^2, max U^2
    const int *done;           // skip when *done != 0 (nullptr: never skip)
    int fast;                  // 1: sum r^2 from float(r) (Kahan, FP32) -- inside the solve loop
    int want_f2;               // 1: also sum f^2 (first iteration / standalone residual)
    int fp64_warps;            // warps (of 8) per block that sum the stencil on the FP64 pipe;
                               // the others use the exact fixed-point sum on the integer pipe
    float2 *fdf;               // padded P^3 copy of f as FP32 pairs (hi, lo): written by the
                               // first residual of a split 3-D solve, read by k_residual_tiled
    int *fx_fbad;              // set when some |f| does not fit the FP32-pair copy
    const int *fx_e;           // DevState::fx_e (k_residual_tiled)
    const int *r2_exp;         // DevState::r2_exp (fast == 1)
    int bc;                    // QN_BC_DIRICHLET (0 past a face) or QN_BC_NEUMANN (the ghost
                               // value past face node 0 is node 1, past node n-1 node n-2)
    const double *pot;         // separable potential: 1-D tables [dim][n], x first (nullptr: V = 0).
                               // With it the partial records hold min / max of 3 b U^2 + V in
                               // their slots 2 and 3, and max|U| goes to *umax_scan
    const float2 *pot2;        // the same tables as FP32 pairs (hi, lo), lam added to the last
                               // axis' table: [dim][n] (k_residual_tiled / k_residual_mirror)
    unsigned long long *umax_scan;   // DevState::umax_scan (atomicMax of |U| bit patterns)
    // spectral elements (k_residual_sem): banded H = M^{-1} S, row i = hlen[i] values from
    // column hc0[i], stored with row stride hbw; hval == nullptr: finite differences
    const int *hc0;
    const int *hlen;
    const double *hval;
    int hbw;
    double robin;              // QN_BC_ROBIN: 2 kappa / h, added times u once per face a node lies on
    const DevState *zero_start;  // iteration 0 of a split solve (KIND 0-2): when the preparation pass
                                 // found U_0 = 0 it already wrote the residual -f, so the tiled kernels
                                 // only write their partial records (nullptr: always evaluate)
};

// Epilogue selector shared by both mode-product kernels.
enum Epi : int {
    EPI_STORE = 0,    // out[k][m] = acc (next product's input)
    EPI_DIVIDE = 1,   // out[k][m] = acc / (lambda_k + row eigen-sum + shift)
    EPI_UPDATE = 2,   // U[dense(k, m)] -= step * acc
    EPI_DENSE = 3,    // V[dense(k, m)] = acc  (FP64 dense output)
    // reflection-split products (3-D split solve, see k_modeprod_tc):
    EPI_STORE_BFLY = 4,   // forward: sums / differences of reflection partners along the next axis
    EPI_STORE_PQ = 5,     // backward: rows j and n-1-j from the even- and odd-mode partial sums
    EPI_UPDATE_PQ = 6,    // backward, last product: U -= step * (the same two rows)
};

struct EpiArgs {
    const double *lam64;      // eigenvalues (n), FP64
    const float *lam32;       // eigenvalues padded to P with 1e30 (split path)
    const double *shift;      // device pointer to lam + beta_n
    double step;
    double *U;                // EPI_UPDATE / EPI_DENSE target (dense n^dim)
    float *dsq;               // update epilogues: += sum (step * delta)^2 (nullptr: off)
    const int *done;          // skip when *done != 0
    int *err;                 // device error flag
};

// Per-launch geometry of one mode product: out = (A * B^T)^T with
// A: [Mtot][K] (K = contraction axis, contiguous), B: [N][K].
struct GemmShape {
    int Mtot;   // rows of A (= n^(dim-1), or P^(dim-1) padded)
    int K;      // contraction length (n, or P padded)
    int N;      // output modes (n, or P padded)
    int n;      // logical extent per axis
    int P;      // padded extent per axis (split path), = n for FP64
    int dim;
    int split = 0;   // FP64 products: 0 dense, 1 forward / 2 backward reflection split
};

// ---- launchers (implemented in the .cu files) ---------------------------------
int launch_residual(const ResidualArgs &a, int grid, cudaStream_t s);
// spectral elements (qn_sem.cu): the per-node residual with the banded H
int launch_residual_sem(const ResidualArgs &a, int grid, cudaStream_t s);
// 3-D split solve, iterations >= 2: no FP64 arithmetic per point (k_residual_tiled).
// Uses at most max_grid blocks; the number of partial records written goes to *grid_used.
int launch_residual_tiled(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s);
// Before the first two tiled residuals of a solve (no previous iterate to take
// the fixed-point exponent from): iteration 0 -> the FP32-pair copy of f, sum
// f^2 (DevState::f_norm, r2_exp) and max|U_0|; iteration 1 -> max|U_1|. Both
// end by setting DevState::fx_e from the scanned max|U|.
int launch_prep_split(const double *U, const double *f, int n, int P, float2 *fdf, __nv_bfloat16 *Rhi,
                      __nv_bfloat16 *Rlo, double *partials,
                      int nparts, DevState *st, bool mirror, cudaStream_t s);
// The same residual written in split order along x and folded order along y
// and z, the input layout of the reflection-split mode products.
int launch_residual_mirror(const ResidualArgs &a, int max_grid, int zchunk, int *grid_used, cudaStream_t s);
// The residual fused into the first forward reflection-split mode product
// (k_fused_res_fwd): what k_residual_mirror and the EPI_STORE_BFLY product that reads
// its planes compute, in one launch. FusedFwd carries the product's side: the
// forward matrix [P][H] as hi / lo tensor maps with 32 x H boxes and the 64-byte
// swizzle, the output planes of the product and the device error word.
struct FusedFwd {
    const CUtensorMap *b_hi, *b_lo;
    __nv_bfloat16 *out_hi, *out_lo;
    int *err;
    int num_sms;
};
struct TcPlan;
int fused_set_attributes();
int launch_fused_residual_fwd(const ResidualArgs &a, const FusedFwd &ff, int *grid_used, cudaStream_t s);
// Encodes the fused kernel's maps of the plan's forward matrix (once; not during a
// stream capture) and opts the kernel in to its shared memory. QN_EUNSUPPORTED
// without reflection-split products or for P > 512.
int tc_plan_enable_fused(TcPlan *p);
// The FusedFwd of a plan prepared by tc_plan_enable_fused, writing working buffer dst.
int tc_plan_fused_args(const TcPlan *p, int dst, int *err, FusedFwd *out);
int launch_umax(const double *U, long long N, DevState *st, int grid, cudaStream_t s);
// mode 0: the partial records hold min / max U^2. 1 (a potential is present): min / max of
// 3 b U^2 + V, and the fixed-point exponent comes from DevState::umax_scan. 2 (eigen solve):
// min / max of lam + 3 b U^2 + V; beta_n = mid-range - lambda_n is the whole shift.
int launch_finalize(const double *partials, int nparts, DevState *st, qn_stats *hist,
                    int hist_cap, double b, double lam, int update_state, int use_saved_fnorm,
                    int mode, cudaStream_t s);

// ---- nonlinear eigenproblem (qn_eig.cu) ------------------------------------------------
// hd = h^dim (the lumped mass without the trapezoid weights); partials: 4 doubles per block.
// U arrives unnormalised; pass 2 writes it back normalised (DevState::eig_scale).
// vrow: lam + v_y (+ v_z) per (y, z) row when a potential is present (else nullptr)
int launch_eig_pass1(const double *U, double *lin, int n, int dim, int bc, double inv_h2, double lam, double b,
                     const double *pot, const double *vrow, double *partials, int grid, const DevState *st,
                     cudaStream_t s);
int launch_eig_finalize1(const double *partials, int nparts, double hd, DevState *st, cudaStream_t s);
// Float-pair forms (split precision, iterations >= 1): lin as FP32 pairs; pot2 / vrow2 the
// potential's per-column and per-row tables as pairs; the fixed-point exponent comes from
// DevState::fx_e. Pass 2 writes planes only (natural or reflection-split order). Pass 1
// launches at most `grid` blocks and returns in `used` how many (the partial sums to add).
int launch_eig_pass1_df(const double *U, float2 *lin, int n, int dim, int bc, double inv_h2, double lam, double b,
                        const double *pot, const double *vrow, const float2 *pot2, const float2 *vrow2,
                        double *partials, int grid, int *used, const DevState *st, cudaStream_t s);
int launch_eig_pass2_df(double *U, const float2 *lin, int n, int P, int dim, int bc, double hd, float lam, double b,
                        const float *pot32, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, bool mirror, double *partials,
                        int grid, int *used, DevState *st, cudaStream_t s);   // grid: at most; used: launched
// exactly one of R64 (FP64 output) or Rhi/Rlo (split planes; mirror: reflection-split order)
// pot32: the potential tables in FP32 (for beta's extremes only), or nullptr
int launch_eig_pass2(double *U, const double *lin, int n, int P, int dim, int bc, double hd, float lam, double b,
                     const float *pot32, double *R64, __nv_bfloat16 *Rhi, __nv_bfloat16 *Rlo, bool mirror,
                     double *partials, int grid, const DevState *st, cudaStream_t s);

int launch_split_pad(const double *r, int n, int P, int dim, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                     int grid, cudaStream_t s);
int launch_modeprod_f64(const double *A, const double *B, double *out, const GemmShape &g,
                        Epi epi, const EpiArgs &e, cudaStream_t s);

// ---- tcgen05 split-precision mode products ------------------------------------------
// One group = one GEMM out[k][m] = sum_j A[m][j] B[k][j] (one mode product of
// one tensor). A launch processes the tiles of one group (single-instance
// solve) or of many groups (batched solve: every instance and component).
struct TcGroup {
    const CUtensorMap *a_hi, *a_lo, *b_hi, *b_lo;   // tensor maps in global memory (64-B aligned)
    __nv_bfloat16 *out_hi, *out_lo;                   // EPI_STORE / EPI_DIVIDE destination planes
    double *U;                                        // EPI_UPDATE / EPI_DENSE target (dense n^dim)
    float *dsq;                                       // update epilogues: += sum (step * delta)^2 (nullptr: off)
    const float *lam32;                               // padded eigenvalues (P entries, 1e30 past n)
    const double *shift;                              // lam + beta_n of the group's instance
    const int *done;                                  // the instance's stop flag (nullptr: never)
    float dscale;                                     // divisor = dscale * eigen-sum + shift
    float step;                                       // update scale
    int Mtot, P, n, BN, ntile_n, ntiles;
};

struct TcTile {
    int group, m0, n0, pad;
};

struct TcPlan;   // tensor maps + tile config of the single-instance tcgen05 path
int tc_plan_create(TcPlan **plan, int n, int P, int dim, __nv_bfloat16 *bufs_hi[2],
                   __nv_bfloat16 *bufs_lo[2], const __nv_bfloat16 *S_hi,
                   const __nv_bfloat16 *S_lo, const __nv_bfloat16 *Si_hi,
                   const __nv_bfloat16 *Si_lo, int num_sms);
void tc_plan_destroy(TcPlan *plan);
// One split-precision mode product: src buffer index -> dst buffer index (or
// the FP64 dense target for EPI_UPDATE / EPI_DENSE). forward selects S^{-1}.
int launch_modeprod_tc(TcPlan *plan, int src, int dst, bool forward, Epi epi,
                       const EpiArgs &e, cudaStream_t s);
// Reflection-split products (3-D, P a multiple of 128): B_fwd, B_bwd are the
// [P][P/2] split-precision matrices described in qn_modeprod_tc.cu. Returns
// QN_EUNSUPPORTED when the sizes do not allow it (the plan keeps the dense path).
int tc_plan_enable_split(TcPlan *plan, const __nv_bfloat16 *bf_hi, const __nv_bfloat16 *bf_lo,
                         const __nv_bfloat16 *bb_hi, const __nv_bfloat16 *bb_lo);
bool tc_plan_has_split(const TcPlan *plan);
// Six-product backward level of the reflection-split products: the third BF16
// level of the two working buffers (P^3 each) and of the backward matrix
// ([P][P/2]). Needs tc_plan_enable_split first.
int tc_plan_enable_x6(TcPlan *plan, __nv_bfloat16 *bufs_l2[2], const __nv_bfloat16 *bb_l2);
// One reflection-split product: EPI_STORE_BFLY / EPI_DIVIDE (forward) or
// EPI_STORE_PQ / EPI_UPDATE_PQ (backward). x6: the divide writes three BF16
// levels and the backward products read three levels and form six products
// (and write three levels); needs tc_plan_enable_x6.
int launch_modeprod_tc_split(TcPlan *plan, int src, int dst, Epi epi, const EpiArgs &e, cudaStream_t s,
                             bool x6 = false);
// ---- whole-solve persistent kernel for small 2-D FP64 problems (qn_small.cu) ----------
constexpr int kSmallMaxN = 128;
constexpr int kSmallBarWords = 64;   // the grid barrier's counter and generation words, apart
struct SmallSolve {
    double *U;
    const double *f;
    const double *S, *Si, *lam1;   // n x n eigenvector matrices and the eigenvalues (device, FP64)
    double *w0, *w1;               // two n^2 work arrays
    double *partials;              // partials_cap records of 4 doubles
    int partials_cap;
    unsigned *bar;                 // kSmallBarWords words (barrier counter, generation)
    DevState *st;
    qn_stats *hist;
    int hist_cap;
    int *err;
    int n, neumann, num_sms;
    double inv_h2, lam, b, tol, beta_value, step;
    int beta_fixed, max_it;
};
int small_solve_supported(int dim, int n);
// One cooperative launch that runs the whole solve; on return (asynchronous) st holds
// it / status / done as the finaliser leaves them, hist the per-iterate statistics.
int launch_small_solve(const SmallSolve &q, cudaStream_t s);

// Grouped launch over a device tile table (batched solves).
// Test-only: the next k_modeprod_tc launch has block 0's producer withhold its first stage.
int tc_test_withhold_arrival();
int launch_modeprod_tc_grouped(const TcGroup *groups, const TcTile *tiles, int ntiles, int dim, int BK,
                               Epi epi, int *err, int grid, cudaStream_t s);
// Encode a 2-D BF16 tensor map [outer][inner] with a (box_inner x box_outer) box.
int tc_encode_2d(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                 uint32_t box_outer, int BK);
size_t tc_smem_bytes(int BK, int stages);
int tc_set_attributes();
int tc_stages(int BK);
bool tc_supported(int device);

// qn_solve with an optional check of the first correction (warm-started
// solves, split precision): with u0_sq (device, ||U_0||^2) non-null, the
// first iteration also sums ||U_1 - U_0||^2 in its last mode product; if it
// is not below ||U_0||^2 / 4 (or anything is not finite), U restarts from 0.
// *used_warm tells which happened. Other arguments as qn_solve.
int solve_internal(::qn_ctx *c, double *U, const double *f, const qn_opts *opts, qn_result *res,
                   qn_stats *history, int history_len, void *stream, const double *u0_sq, int *used_warm);
bool ctx_split_precision(const ::qn_ctx *c);
// Symmetric eigen-decomposition on the host (qn_sem.cu): A (row-major n x n) is replaced by
// Q with A = Q diag(d) Q^T, d ascending; false if the QL iteration does not converge.
bool symmetric_eigen(int n, std::vector<double> &A, std::vector<double> &d);
// host setup of the Q^k spectral element matrices (qn_sem.cu); see qn_setup_1d_sem
int sem_setup(int n, int k, double length, int bc, std::vector<double> &H, std::vector<double> &S,
              std::vector<double> &Si, std::vector<double> &lam, std::vector<double> &nodes);
// Dirichlet data on the unit cube and no potential (the learned warm start's setting)
bool ctx_unit_dirichlet(const ::qn_ctx *c);

// error reporting
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

}  // namespace qn

#define QN_CUDA(call)                                         \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return qn::cuda_fail(_e, #call); \
    } while (0)
