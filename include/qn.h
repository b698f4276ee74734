/*
 * qn.h - C ABI of libqn: GPU quasi-Newton solver for discretised quasi-linear
 * elliptic equations A_h U + N_h(U) = 0 with a fast-diagonalisation inverse.
 *
 * Method: W. Hao, S. Lee, X. Zhang, "An Efficient Quasi-Newton Method with
 * Tensor Product Implementation for Solving Quasi-Linear Elliptic Equations
 * and Systems" (arXiv 2502.03611).
 *
 * Problem solved (Sec. 2 eq. main-pde, Sec. 3.2, Sec. 4 eq. F_u):
 *   -Lap u + lam u + b u^3 + V u = f   on a cube of side L (default (0,1)^dim),
 * with u = 0 on the boundary (QN_BC_DIRICHLET) or a zero normal derivative
 * (QN_BC_NEUMANN), and V an optional separable potential
 * V(x, y, z) = v_x(x) + v_y(y) + v_z(z). Discretised by second-order central
 * differences (5-point in 2-D, 7-point in 3-D, eq. fdm-discrete) on n nodes
 * per axis: Dirichlet n interior nodes, h = L/(n+1); Neumann n nodes with
 * both faces included, h = L/(n-1), the value past a face taken from the
 * ghost point u_{-1} = u_1 (Sec. 3.2, Neumann rows):
 *   F(U) = A_h vec(U) + N_h(U),  A_h = sum_a I..H_a..I + lam I,
 *   H_a = (1/h^2) tridiag(-1, 2, -1) (Neumann: first row (2, -2), last
 *   row (-2, 2)),  N_h(U) = b U^3 + V U - f.
 * Quasi-Newton update (Sec. 4 eq. identity-method):
 *   U <- U - step * (A_h + beta_n I)^{-1} F(U),
 *   beta_n = (lambda_max + lambda_min)/2 of (N_h)_U = diag(3 b U^2 + V),
 * with the inverse applied by fast diagonalisation (Sec. 4.1 eq. fin_inverse):
 * mode products with S^{-1} along every axis, pointwise division by
 * (sum_a lambda_{i_a} + lam + beta_n), mode products with S along every axis.
 * Stopping rule: ||F(U)||_2 / ||f||_2 <= tol (the paper leaves the tolerance
 * open; this library takes the relative l2 residual against the source).
 *
 * Conventions for every entry point:
 *  - Arrays are float64, C order with the x index fastest: U[y][x] in 2-D and
 *    U[z][y][x] in 3-D, interior nodes only (n^dim values). This is the
 *    paper's vec() ordering.
 *  - Array pointers are DEVICE pointers unless the name ends in _host. The
 *    caller owns them; the library never frees or retains them past the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it. Entry points that return statistics to
 *    host structs synchronise that stream before returning.
 *  - Every call returns QN_OK (0) or a negative QN_E* code. Arguments are
 *    validated on the host before anything is launched. No call exits the
 *    process or throws across the ABI. qn_last_error() returns a message for
 *    the last failure on the calling thread.
 */
#ifndef QN_H
#define QN_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QN_OK            0
#define QN_EINVAL       -1  /* bad argument (null pointer, size, non-finite parameter) */
#define QN_ENOMEM       -2  /* device or host allocation failed */
#define QN_ECUDA        -3  /* a CUDA runtime/driver call failed (see qn_last_error) */
#define QN_ENOTCONV     -4  /* max_it reached before the tolerance; U holds the last iterate */
#define QN_EDIVERGED    -5  /* residual became non-finite or grew past 1e8 x ||f|| */
#define QN_ETIMEOUT     -6  /* a device-side wait gave up (kernel returned early, no hang) */
#define QN_EUNSUPPORTED -7  /* valid request the library does not implement */

/* ---- enumerations -------------------------------------------------------- */
#define QN_BC_DIRICHLET 0   /* homogeneous Dirichlet, interior unknowns only (Sec. 3.2) */
#define QN_BC_NEUMANN   1   /* zero normal derivative by ghost points, face nodes are unknowns
                               (Sec. 3.2, Neumann rows with alpha_3 = 0; a nonzero flux only
                               adds a constant to f at the face nodes, so pass it in f) */
#define QN_BC_ROBIN     2   /* alpha_1 du/dn + beta_1 u = 0 by the same ghost points:
                               u_{-1} = u_1 - 2 h kappa u_0, kappa = beta_1/alpha_1 =
                               qn_problem.robin_kappa >= 0 (the face term belongs to A_h);
                               finite differences, per-node residual kernel */

#define QN_PREC_FP64   0    /* mode products in FP64 on the FP64 pipe */
#define QN_PREC_BF16X3 1    /* mode products on tcgen05 tensor cores as
                               hi*hi + hi*lo + lo*hi BF16 products, FP32
                               accumulation; residual, beta, update and stop
                               test stay FP64 (outer loop = iterative refinement) */
#define QN_PREC_BF16X6 2    /* QN_PREC_BF16X3 with the backward mode products as six
                               BF16 products of three-level operands (x = x0 + x1 + x2,
                               each level the BF16 rounding of what the previous ones
                               leave): a0 b0 + a0 b1 + a1 b0 + a1 b1 + a0 b2 + a2 b0, FP32
                               accumulation; the spectral coefficients and the backward
                               intermediates are stored as three levels. The forward
                               products stay three-term: their error is divided by the
                               eigenvalue sums, while the backward products' error is
                               spread over all modes and A_h amplifies it by up to its
                               stiffness ratio, so it sets a BF16X3 correction's residual
                               (about 2e-2 of ||F|| at 255^3, growing as n^2) and
                               BF16X6 cuts it about 20-fold. 3-D finite differences with
                               the reflection-split products only (Dirichlet or Neumann,
                               P = 64 ceil(n/64) a multiple of 128); QN_EUNSUPPORTED
                               otherwise. Two more padded n^3 x 2-byte buffers. */

#define QN_BETA_PAPER 0     /* beta_n = (max + min)/2 of diag(3 b U^2 + V) (eq. identity-method) */
#define QN_BETA_FIXED 1     /* beta_n = qn_opts.beta_value every iteration */

/* ---- structures ------------------------------------------------------------ */
typedef struct qn_problem {
    int dim;          /* 2 or 3 */
    int n;            /* unknowns per axis (same on every axis): Dirichlet 1..1024 interior
                         nodes, Neumann 2..1024 nodes with both faces */
    int bc;           /* QN_BC_DIRICHLET or QN_BC_NEUMANN */
    int precision;    /* QN_PREC_FP64, QN_PREC_BF16X3 or QN_PREC_BF16X6 */
    double lam;       /* linear coefficient lam of -Lap u + lam u + b u^3 + V u = f */
    double b;         /* cubic coefficient b */
    double length;    /* side L of the cubic domain; 0 selects 1 (the unit cube) */
    const double *potential_host;   /* NULL (V = 0) or host array of dim*n doubles: the
                         1-D tables v_x[n], v_y[n](, v_z[n]) of V = v_x + v_y (+ v_z) at the
                         nodes, x first. Copied by qn_ctx_create; the caller keeps it. */
    int sem_k;        /* 0: finite differences. 1..16: Q^k spectral elements (Sec. 3.1) on E
                         equal elements, n = E k - 1 (Dirichlet) or E k + 1 (Neumann) nodes per
                         axis at the Gauss-Lobatto points (qn_setup_1d_sem gives them); the
                         residual applies H = M^{-1} S along every axis (FP64), the inverse uses
                         its numerical eigenpairs. f and the potential are nodal values. */
    double robin_kappa;   /* QN_BC_ROBIN: kappa = beta_1 / alpha_1 >= 0 (ignored otherwise) */
} qn_problem;

typedef struct qn_stats {
    double res_norm;  /* ||F(U)||_2 at the evaluated iterate */
    double f_norm;    /* ||f||_2 */
    double fu_min;    /* smallest entry of diag(N_h)_U = 3 b U^2 + V */
    double fu_max;    /* largest entry */
    double beta;      /* beta_n applied to this iterate (paper rule or fixed) */
    double rel;       /* res_norm / f_norm */
    double lambda;    /* qn_eig_solve: the Rayleigh quotient lambda_n of this iterate; else 0 */
} qn_stats;

typedef struct qn_opts {
    double tol;        /* stop when rel <= tol (1e-10 in the benchmarks) */
    int max_it;        /* at most this many updates (>= 0, <= 4096) */
    int beta_mode;     /* QN_BETA_PAPER or QN_BETA_FIXED */
    double beta_value; /* used with QN_BETA_FIXED */
    double step;       /* update scale; 1.0 is the paper's plain update */
    int sync_every;    /* host checks convergence every this many iterations
                          (>= 1); kernels queued past convergence exit at once */
    int graph;         /* 1: from the third iteration on, each group of sync_every
                          iterations is replayed from a CUDA graph captured once per
                          context (re-captured when U, f, step or sync_every change);
                          ignored while launch profiling is on. 0: plain launches */
} qn_opts;

typedef struct qn_result {
    int iterations;    /* updates applied */
    int status;        /* QN_OK, QN_ENOTCONV, QN_EDIVERGED or QN_ETIMEOUT */
    double rel;        /* final ||F(U)||_2 / ||f||_2 */
} qn_result;

typedef struct qn_ctx qn_ctx;  /* opaque; owns device workspace for one problem shape */

/* ---- entry points ------------------------------------------------------------ */

/* Version of this ABI (major*10000 + minor*100 + patch). */
int qn_version(void);

/* Message for the last failing call on this thread ("" if none). Owned by the library. */
const char *qn_last_error(void);

/* 1-D diagonalisation H = S diag(lam) S^{-1} (Sec. 4.2; H from Sec. 3.2 eq. Sy
 * and the Neumann rows). Host-only, FP64. h > 0 is the mesh width (it scales
 * lam only); n >= 1 (Dirichlet) or n >= 2 (Neumann). Closed forms, ascending
 * in k:
 *  QN_BC_DIRICHLET (discrete sine pairs, 1-based j, k, t = 1/(n+1)):
 *    lam_k = (4/h^2) sin^2(k pi t/2), S[j][k] = sqrt(2t) sin(j k pi t);
 *    S is symmetric orthogonal, S_inv = S.
 *  QN_BC_NEUMANN (discrete cosine pairs, 0-based j, k, t = 1/(n-1)):
 *    lam_k = (4/h^2) sin^2(k pi t/2), S[j][k] = cos(j k pi t) / sqrt(c_k),
 *    S_inv[k][j] = w_j cos(j k pi t) / sqrt(c_k), with w_j = 1/2 at the two
 *    faces and 1 elsewhere, c_k = (n-1)/2, or n-1 for k = 0 and k = n-1.
 *    S is not orthogonal (W^{1/2} S is), lam_0 = 0 (constants).
 * S, S_inv: caller-owned host buffers of n*n doubles, row-major (S[j*n+k]).
 * lam: caller-owned host buffer of n doubles. Any output may be NULL. */
int qn_setup_1d_eig(int n, double h, int bc, double *S, double *S_inv, double *lam);

/* 1-D Robin matrix (Sec. 3.2 ghost points with alpha_1 du/dn + beta_1 u = 0): the Neumann
 * matrix with face diagonals (2 + 2 h kappa)/h^2, n >= 2 nodes including both faces,
 * kappa >= 0. H = S diag(lam) S^{-1} from the symmetric W^{1/2} H W^{-1/2} = Q diag(lam) Q^T
 * (W = diag(1/2, 1, .., 1, 1/2)): S = W^{-1/2} Q, S_inv = Q^T W^{1/2}, lam ascending.
 * Host-only, FP64, outputs as qn_setup_1d_eig (any may be NULL). */
int qn_setup_1d_robin(int n, double h, double kappa, double *S, double *S_inv, double *lam);

/* 1-D Q^k spectral element matrices (Sec. 3.1 eqs. S_x, M_x, final-system-3d; Sec. 4.2).
 * Host-only, FP64. E = (n+1)/k (Dirichlet) or (n-1)/k (Neumann) equal elements of
 * [0, length]; Lagrange bases at the k+1 Gauss-Lobatto points, Gauss-Lobatto quadrature
 * (diagonal mass M), assembled stiffness S, Dirichlet keeping the interior nodes.
 *   H = M^{-1} S (n x n), and H = S diag(lam) S^{-1} from the symmetric
 *   M^{-1/2} S M^{-1/2} = Q diag(lam) Q^T: S = M^{-1/2} Q, S_inv = Q^T M^{1/2};
 *   nodes: the node coordinates on [0, length].
 * 1 <= k <= 16, length > 0, n + 1 (Dirichlet) or n - 1 (Neumann) a positive multiple of k
 * (QN_EINVAL otherwise). Outputs are caller-owned host buffers (n*n or n doubles,
 * row-major), any of which may be NULL. */
int qn_setup_1d_sem(int n, int k, double length, int bc, double *H, double *S, double *S_inv,
                    double *lam, double *nodes);

/* Create a context for one problem shape on the current CUDA device: uploads
 * S, S^{-1} and the eigenvalues (and their BF16 hi/lo splits for
 * QN_PREC_BF16X3 / BF16X6), allocates the working buffers (about 2 n^dim doubles for
 * FP64, 2 padded n^dim x 4 bytes for BF16X3) and, for BF16X3, builds the TMA
 * tensor maps. QN_EUNSUPPORTED for BF16X3 on a device without sm_103a
 * tcgen05 support. *out is owned by the library until qn_ctx_destroy. */
int qn_ctx_create(const qn_problem *p, qn_ctx **out);

/* Free everything the context owns. NULL is accepted. Synchronises the device. */
int qn_ctx_destroy(qn_ctx *ctx);

/* Residual F(U) = A_h vec(U) + lam U + b U^3 + V U - f (Sec. 4 eq. F_u) in FP64.
 * U, f: device, n^dim doubles. R: device, n^dim doubles, or NULL to compute
 * only the statistics. st (host, may be NULL): norms and extreme entries of
 * diag(3 b U^2 + V); beta is the paper's beta_n for U. Synchronises `stream`
 * when st != NULL. */
int qn_residual(qn_ctx *ctx, const double *U, const double *f, double *R,
                qn_stats *st, void *stream);

/* Shifted inverse by fast diagonalisation (Sec. 4.1 eq. fin_inverse):
 * V = (sum_a I..H_a..I + shift I)^{-1} r, i.e. A_h without lam, plus shift.
 * r, V: device, n^dim doubles, distinct. Runs in the context's precision
 * (FP64 or BF16X3 mode products). shift must be finite and
 * > -dim * lambda_min(H) (> 0 for Neumann data, where lambda_min = 0).
 * Does not synchronise. */
int qn_fast_diag_solve(qn_ctx *ctx, const double *r, double *V, double shift, void *stream);

/* One quasi-Newton update in place (Sec. 4 eq. identity-method):
 * U <- U - step (A_h + beta I)^{-1} F(U) with step = 1 and beta = the paper's
 * beta_n when `beta` is NaN, else the given beta. U, f: device, n^dim doubles.
 * st (host, may be NULL): statistics of the iterate BEFORE the update.
 * Synchronises `stream` when st != NULL. */
int qn_step(qn_ctx *ctx, double *U, const double *f, double beta, qn_stats *st, void *stream);

/* Iterate qn_step until ||F(U)||/||f|| <= opts->tol or opts->max_it updates.
 * U: device, n^dim doubles: in = initial iterate U_0 (zeros for the standard
 * start, or a warm start), out = last iterate. f: device, n^dim doubles.
 * opts: host (NULL = tol 1e-10, max_it 200, paper beta, step 1, sync_every 2).
 * res (host, may be NULL): iteration count, status, final relative residual.
 * history (host, may be NULL): receives the statistics of iterates
 * U_0 .. U_iterations (history_len entries at most). Synchronises `stream`.
 * 2-D FP64 finite-difference contexts with n <= 128 and no potential (Dirichlet or
 * Neumann data) run the whole solve as one cooperative kernel that takes the stop
 * decision on the device (opts->sync_every and opts->graph do not apply; the environment
 * variable QN_SMALL=0 at context creation, or launch profiling, selects the per-phase
 * launches). Returns res->status (QN_OK when converged). */
int qn_solve(qn_ctx *ctx, double *U, const double *f, const qn_opts *opts,
             qn_result *res, qn_stats *history, int history_len, void *stream);

/* Precision escalation for the solves of a BF16X3 context. rate > 0: at every host
 * check of qn_solve (every opts->sync_every iterations) the one-step contraction
 * rho = rel_it / rel_{it-1} is compared with the quasi-Newton bound
 * b = max|diag(N_h)_U - beta| / (lambda_min(A_h) + beta) at U_it (Sec. 5: the error of the
 * simplified Jacobian); when rho > rate and rho > 2 b, the precision of the split products,
 * not the nonlinearity, sets the rate, and the remaining iterations of that solve run the
 * backward products at the six-product level of QN_PREC_BF16X6. rate = 0 (the default)
 * turns it off. The first call with rate > 0 allocates the third BF16 level of the working
 * buffers (two padded n^3 x 2-byte buffers); QN_ENOMEM if that fails. QN_EUNSUPPORTED
 * unless the context is BF16X3 with the reflection-split products (the shapes
 * QN_PREC_BF16X6 accepts); a BF16X6 context runs every iteration at that level and only
 * records the rate. QN_EINVAL for a negative or non-finite rate. Does not synchronise.
 * qn_profile.x6_from reports where the last solve switched. */
int qn_set_escalation(qn_ctx *ctx, double rate);

/* The residual fused into the first mode product (the one-kernel form of the residual
 * F(U) of Sec. 4 eq. F_u and the first forward mode product of the inverse, Sec. 4.1
 * eq. fin_inverse). on != 0: from the second iteration of each qn_solve on, one kernel
 * evaluates the residual inside the producer of the first forward reflection-split
 * product, writing the product's shared-memory operand instead of the residual planes
 * (no HBM round trip of the planes); on = 0 (the default) restores the separate residual
 * kernel and product. The iterates are those of the separate kernels: the same fixed-point
 * stencil, float-pair nonlinear term and products; only the FP32 summation order of
 * ||F||^2 differs. QN_EUNSUPPORTED (on != 0) unless the context is a 3-D BF16X3 or
 * BF16X6 finite-difference context with the reflection-split products, n <= 512,
 * Dirichlet data and no potential. The first call with on != 0 encodes two tensor maps
 * (a blocking copy to the device): call it outside a stream capture. Does not
 * synchronise otherwise. qn_profile.fused_launches / fused_ms time the fused kernel.
 * Off by default: its producer re-reads and re-converts the z-neighbours of every point,
 * which makes it slower than the separate kernels from n = 255 on (1.70 against
 * 0.86 + 0.20 ms per iteration at 511^3); at n <= 128 (P = 128) it saves a launch and the
 * residual planes' round trip and is about 3 % faster per solve. */
int qn_set_fused_residual(qn_ctx *ctx, int on);

/* qn_solve with HOST arrays: copies f_host and U_host (initial iterate) to
 * context-owned device buffers, solves, copies the result back into U_host.
 * U_host, f_host: host, n^dim doubles (pinned memory gives full copy speed).
 * Synchronises `stream`. */
int qn_solve_host(qn_ctx *ctx, double *U_host, const double *f_host, const qn_opts *opts,
                  qn_result *res, qn_stats *history, int history_len, void *stream);

/* qn_solve_host from the zero start U_0 = 0 (the start of the paper's FD and SEM
 * runs): only f_host is copied to the device; U_host is output only (its
 * contents on entry are ignored) and receives the result. Same arguments, errors
 * and synchronisation as qn_solve_host; the iterates and the result are those
 * of qn_solve_host with U_host = 0. */
int qn_solve_host_zero_start(qn_ctx *ctx, double *U_host, const double *f_host, const qn_opts *opts,
                             qn_result *res, qn_stats *history, int history_len, void *stream);

/* A sequence of independent host-array solves with one context, pipelined: the
 * inputs of problem i+1 are copied in and the result of problem i-1 copied out on
 * two copy streams of the context while problem i is solved on `stream`, so that
 * the host link works alongside the GPU (a serving loop). No counterpart in the
 * paper (its solves start from device-resident data).
 *   count >= 0 problems. U_host[i], f_host[i]: host arrays of n^dim doubles in the
 *   context's layout; U_host[i] holds the start unless zero_start != 0 (then it is
 *   output only), and receives the result. Distinct problems may share an f array,
 *   and may share a U array when the later one is at least two positions on (the
 *   copies out run in order). Page-locked arrays (cudaHostAlloc / cudaHostRegister)
 *   let the copies overlap the solves; pageable ones work, with less overlap.
 *   opts: as qn_solve (NULL for the defaults). results: count records, written for
 *   every problem solved.
 * Allocates two pairs of device buffers (4 n^dim doubles), two streams and six
 * events on the first call; the context frees them. Synchronises `stream` and the
 * copy streams before it returns. Returns QN_OK when every problem ran (each
 * record's status says whether it converged: QN_OK, QN_ENOTCONV, QN_EDIVERGED),
 * QN_EINVAL for bad arguments (before any copy), or the first hard error
 * (QN_ECUDA, QN_ETIMEOUT, ...), after which the later problems are not solved. */
int qn_solve_host_many(qn_ctx *ctx, int count, double *const *U_host, const double *const *f_host,
                       int zero_start, const qn_opts *opts, qn_result *results, void *stream);

/* Allocation-free variant of qn_residual, for callers that cannot allocate
 * device memory where they need a residual: their device memory is owned in
 * full by another allocator or a fixed budget, or they run in a section that
 * must not allocate. No context is needed and nothing is allocated; the
 * paper has no counterpart to this entry point (it is a deployment aid).
 * Computes the same F(U) = A_h vec(U) + lam U + b U^3 - f and statistics as
 * qn_residual for a dim-D grid with n interior nodes per axis.
 *   dim: 2 or 3. n: 1..1024 (larger n is rejected with QN_EINVAL).
 *   U, f: device, n^dim doubles. R: device, n^dim doubles, or NULL.
 *   st: host struct, required. Synchronises `stream`.
 * Scratch: a fixed 33 KB device array inside libqn (4096 partial sums plus
 * the solver state and one statistics record), present on every GPU that
 * loads the library until the process exits. The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and keeps it;
 * make that first call before any stream capture. The lookup is redone when
 * the device's context has changed since (after a cudaDeviceReset, which
 * reloads the library's module). Every call reads the statistics back to the
 * host and synchronises `stream` before it returns. All calls share the one
 * array, so calls that overlap on the GPU (other streams, other host threads)
 * race; serialise them. Each call rewrites every scratch entry it reads. */
int qn_residual_noalloc(int dim, int n, double lam, double b, const double *U, const double *f,
                        double *R, qn_stats *st, void *stream);

/* Test-only fault injection for the bounded device waits (no GPU fault, no hang):
 * the next tensor-core mode-product launch in this process has the TMA producer
 * of its block 0 skip its first stage, so that stage's barrier never completes.
 * The MMA issuer and the epilogue give up after 2 s of %globaltimer, set
 * QN_ETIMEOUT in the launch's error word and return; nothing is left in flight
 * (no MMA was issued, the other stages' loads are drained), and the device and
 * the context stay usable. The solve or product call that contains the launch
 * returns QN_ETIMEOUT when it reads that word (qn_solve at its next convergence
 * check). Only the one launch is affected (the request is taken atomically).
 * Returns QN_OK, or QN_ECUDA without a device. */
int qn_test_withhold_arrival(void);

/* ---- batched coupled two-component systems (Sec. 4.3) ---------------------------
 * Many independent 2-D instances of
 *   -Lap u + u^3 + alpha v = f1,   -D Lap v + v^3 - alpha u = f2   (Dirichlet 0)
 * with uneven grid sizes, solved together. Each iteration evaluates both
 * residuals (iteration 0 in FP64; later ones on an exact fixed-point stencil
 * with float-pair arithmetic, ~48 significant bits, FP64 for any value of 2^37
 * or more), takes one beta per instance as the midpoint of the extreme
 * eigenvalues of the 2x2 blocks [[3u^2, alpha], [-alpha, 3v^2]] over all nodes
 * (Sec. 4.3 eqs. eigen_quad, eigenvalues; real parts when the pair is complex),
 * and updates u -= (A_h + beta I)^{-1} F_u, v -= (D A_h + beta I)^{-1} F_v by
 * fast diagonalisation with BF16x3 tensor-core mode products. Each of the four
 * mode-product phases is one grouped persistent launch over every instance
 * and component; an iteration (six launches) is captured into a CUDA graph. */
typedef struct qn_sys_instance {
    int n;                  /* interior nodes per axis (n x n grid), 1..1024 */
    double alpha;           /* coupling coefficient (finite) */
    double D;               /* diffusion of the second component, > 0 */
    double *U, *V;          /* device, n*n doubles each: initial iterates in, solutions out */
    const double *f1, *f2;  /* device, n*n doubles each */
} qn_sys_instance;

typedef struct qn_sys_result {
    int iterations;         /* updates applied to this instance */
    int status;             /* QN_OK, QN_ENOTCONV or QN_EDIVERGED */
    double rel;             /* final sqrt(|F_u|^2 + |F_v|^2) / sqrt(|f1|^2 + |f2|^2) */
    double time_ms;         /* device time from the start of the batch solve to this
                               instance's convergence (-1 if it never stopped) */
} qn_sys_result;

typedef struct qn_batch qn_batch;   /* opaque; owns workspace, tensor maps, tile tables, graph */

/* Create a batch over `count` instances (host array; the device arrays it
 * points to must stay valid until qn_batch_destroy). bk: K-tile of the mode
 * products, 0 (= 64), 32 or 64. bn: NULL, or one N-tile width per instance
 * (multiple of 16 in 16..256, 0 = default min(P, 256)), e.g. from
 * qn_autotune_tile. */
int qn_batch_create(const qn_sys_instance *inst, int count, int bk, const int *bn, qn_batch **out);

/* Solve every instance from its current U, V. opts: tol, max_it and
 * sync_every (iterations per captured graph launch, the host checks between
 * launches); beta_mode must be QN_BETA_PAPER and step 1. res: host array of
 * `count` results (may be NULL). Returns QN_OK if every instance converged,
 * else the first non-OK instance status. Synchronises `stream`. */
int qn_batch_solve(qn_batch *b, const qn_opts *opts, qn_sys_result *res, void *stream);

int qn_batch_destroy(qn_batch *b);

/* Project autotuner for the batched mode products: times the grouped
 * split-precision product over `copies` synthetic instances of size n for
 * each candidate (bk in {32, 64}) x (bn in {64, 128, 256}, bn <= P) and
 * returns the fastest. best_ms: mean time of one grouped launch (host). The
 * result is kept for the process, per (device, n, copies): later calls with
 * the same arguments return it without timing again. */
int qn_autotune_tile(int n, int copies, int *best_bk, int *best_bn, double *best_ms);

/* ---- learned warm start ---------------------------------------------------------
 * A small neural operator maps the source f, restricted to a coarse G^3 grid,
 * to a coarse initial iterate, which is prolonged to the fine grid as U_0.
 * Network: lift 1 -> 32 channels; `blocks` blocks of
 *   z = synthesis(R_k . analysis(h)) + h W + b,  h <- gelu(z) (not after the last),
 * with analysis / synthesis in the first `modes` sine modes per axis
 * (orthonormal Dirichlet sine basis) and per-mode 32x32 mixing R_k; then a
 * projection 32 -> 1. Activations are stored in BF16; arithmetic,
 * accumulation, master weights, gradients and AdamW moments are FP32.
 * Flat parameter order: wl(32), bl(32), per block R(modes^3*32*32, index
 * [kz][ky][kx][i][o]), W(32*32, [i][o]), b(32); then wp(32), bp(1).
 * The paper has no learned component (this extends the solver's start). */
typedef struct qn_net qn_net;

/* Number of parameters for channels (must be 32), modes, blocks. */
long long qn_net_param_count(int channels, int modes, int blocks);

/* Create a network on the current device. G: coarse grid nodes per axis
 * (2..256), channels == 32, modes in 1..min(G, 16), blocks 1..16,
 * max_batch 1..64 (activation buffers are sized for it). Parameters start at
 * zero: set them with qn_net_set_params. */
int qn_net_create(int G, int channels, int modes, int blocks, int max_batch, qn_net **out);
int qn_net_destroy(qn_net *net);

/* Copy all parameters from / to a host float array of qn_net_param_count
 * entries. Setting parameters resets the AdamW moments and step count. */
int qn_net_set_params(qn_net *net, const float *host_params, long long count);
int qn_net_get_params(qn_net *net, float *host_params, long long count);

/* Inference on B coarse inputs: f_coarse, out: device float arrays [B][G^3]. */
int qn_net_forward(qn_net *net, const float *f_coarse, float *out, int B, void *stream);

/* Mean-squared loss against target [B][G^3] and its gradient (forward +
 * backward). grads_out: device float array of qn_net_param_count entries, or
 * NULL. loss: host, or NULL (then the call does not synchronise). */
int qn_net_gradients(qn_net *net, const float *f_coarse, const float *target, int B, float *grads_out,
                     double *loss, void *stream);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight decay)
 * on the loss of qn_net_gradients. loss: host, or NULL. */
int qn_net_train_step(qn_net *net, const float *f_coarse, const float *target, int B, float lr,
                      float weight_decay, double *loss, void *stream);

/* U0 (device, n^3 doubles) = out_scale * prolong(net(in_scale * restrict(f))),
 * f: device, n^3 doubles. */
int qn_net_predict(qn_net *net, const double *f_fine, int n, double in_scale, double out_scale,
                   double *U0, void *stream);

/* Trilinear transfer of B fields from the m_from^3 to the m_to^3 interior grid
 * of (0,1)^3 (nodes j/(m+1), zero boundary), times scale. src, dst: device. */
int qn_interp3d(const double *src, int m_from, double *dst, int m_to, int B, double scale, void *stream);
int qn_interp3d_f32(const double *src, int m_from, float *dst, int m_to, int B, double scale, void *stream);

/* Warm-started solve. U0 from qn_net_predict, then one quasi-Newton step
 * U1 = U0 - delta. The correction delta estimates the error of U0, so if
 * ||delta|| < ||U0|| / 2 the solve continues from U1 (the step counts as an
 * iteration, *used_warm = 1); otherwise, or if U0 is not finite, it restarts
 * from the zero start (*used_warm = 0). ||F(U0)|| is not the criterion: the
 * trilinear prolongation leaves high-frequency error that A_h amplifies in
 * the residual while the first correction removes it. ctx: 3-D context with
 * the same n, Dirichlet data on the unit cube and no potential (the network's
 * basis; QN_EUNSUPPORTED otherwise). U, f: device, n^3. Uses stream-ordered
 * temporary memory. */
int qn_solve_warm(qn_ctx *ctx, qn_net *net, double *U, const double *f, int n, double in_scale,
                  double out_scale, const qn_opts *opts, qn_result *res, int *used_warm, void *stream);

/* ---- nonlinear eigenproblem (Sec. 4.4; Sec. 6.3 Example 2) ------------------------------
 * Finds u and lambda with -Lap u + f(u) = lambda u, ||u|| = 1, f(u) = lam u + b u^3 + V u
 * (the context's boundary data, lam, b and potential). Iteration (eqs. system_qusi,
 * system_normal):
 *   lambda_n = <A_h U + f(U), U> / <U, U>,   F = A_h U + f(U) - lambda_n U,
 *   beta_n = (max + min)/2 of diag(lam + 3 b U^2 + V) - lambda_n (or opts->beta_value),
 *   U~ = U - step (A_h + beta_n I)^{-1} F  (A_h the difference operator alone),
 *   U = U~ / ||U~||,
 * stopping when ||F|| / |lambda_n| <= opts->tol. <V, W> = h^dim sum w V W, w the product
 * of the 1-D trapezoid weights (1/2 at Neumann face nodes, else 1).
 * U: device, n^dim doubles: in = start (any nonzero scale; each iteration normalises the
 * iterate it evaluates), out = the last evaluated iterate, with ||U|| = 1. opts: host, NULL = tol 1e-10, max_it 4096, paper beta, step 1, sync_every 8.
 * lambda: host, may be NULL: lambda_n of the returned iterate. history (host, may be NULL):
 * per iterate res_norm = ||F||, f_norm = |lambda_n| ||U||, fu_min / fu_max = extremes of
 * lam + 3 b U^2 + V, beta = beta_n, rel, lambda = lambda_n. With opts->graph every group of
 * sync_every iterations is replayed from a CUDA graph. BF16X3 contexts allocate n^dim
 * doubles on the first call. Synchronises `stream`. Returns res->status. */
int qn_eig_solve(qn_ctx *ctx, double *U, const qn_opts *opts, qn_result *res, double *lambda,
                 qn_stats *history, int history_len, void *stream);

/* ---- measurement ------------------------------------------------------------- */
typedef struct qn_profile {
    long long launches;       /* kernels launched that did work since qn_profile_enable
                                 (launches queued past convergence are not counted) */
    int residual_launches;    /* residual + reduction kernel (and, in a 3-D split solve, the
                                 preparation passes of its first two iterations) */
    double residual_ms;       /* summed CUDA-event time on the launching stream */
    int finalize_launches;    /* one-block reduction finaliser (beta_n, stop test) */
    double finalize_ms;
    int modeprod_launches;    /* all mode-product launches (sum of the three below) */
    double modeprod_ms;
    int mp_store_launches;    /* products that store the next product's input */
    double mp_store_ms;
    int mp_divide_launches;   /* last forward product, with the eigen-sum divide */
    double mp_divide_ms;
    int mp_last_launches;     /* last backward product, with the update (or dense store) */
    double mp_last_ms;
    int residual_tiled_launches;   /* of residual_launches: the residuals of a 3-D split solve
                                      from its third iteration on (no FP64 arithmetic) */
    double residual_tiled_ms;
    int split_products;       /* 1: the last shifted inverse used the reflection-split mode
                                 products (3-D split solve, n+ padding a multiple of 128):
                                 half the tensor work of the dense products */
    int x6_from;              /* the last qn_solve: the first iteration whose backward products
                                 ran at the six-product level (0 in a QN_PREC_BF16X6 context,
                                 the escalation point after qn_set_escalation), -1: none */
    int fused_launches;       /* qn_set_fused_residual: the fused residual + first product
                                 kernels (counted in neither residual_ nor modeprod_) */
    double fused_ms;
} qn_profile;

/* on != 0: from now on record a pair of CUDA events around every kernel
 * launch of this context (on the launching stream); on == 0: stop recording.
 * Either way the counters are reset. */
int qn_profile_enable(qn_ctx *ctx, int on);

/* Sum the recorded launch times per kernel class (waits for the events).
 * out: host struct. */
int qn_profile_read(qn_ctx *ctx, qn_profile *out);

#ifdef __cplusplus
}
#endif
#endif /* QN_H */
