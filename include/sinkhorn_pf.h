/*
 * sinkhorn_pf.h -- C ABI of libsinkhorn_pf.so, a GB300 (sm_103a) implementation of
 * linear-time Sinkhorn divergences with positive features (Scetbon & Cuturi,
 * arXiv 2006.07057).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All functions return an int status (lsf_status). They never abort or throw.
 *    On failure lsf_last_error() returns a message for the calling thread.
 *  - "device" pointers are CUDA global-memory pointers owned by the caller; the
 *    library never allocates, frees or keeps them. "host" pointers are plain
 *    host memory. Every device call is asynchronous on the given CUDA stream
 *    (a cudaStream_t passed as void*; NULL is the legacy default stream).
 *  - Floating point data is FP32, row-major, contiguous. Points are n x d.
 *  - Features are stored point-major: F is n x ldr with F[i*ldr + k] the k-th
 *    shifted feature of point i (the transpose of the paper's r x n xi).
 *    ldr >= r, ldr % 4 == 0, ldr <= 1024; columns r..ldr-1 hold zeros.
 *  - Row shifts: shift[i] = max_k log phi_theta(x_i)_k, and F holds
 *    phi_theta(x_i)_k * exp(-shift[i]), so every stored row has maximum 1.
 *  - Scalings are stored shifted: u~_i = u_i exp(shift_x[i]) * exp(M) and
 *    v~_j = v_j exp(shift_y[j]) * exp(-M), where M = max_j shift_y[j] is the
 *    global factor fixed at start (lsf_result.log_scale). Hence
 *      log u_i = log u~_i - shift_x[i] - M,   log v_j = log v~_j - shift_y[j] + M.
 *  - Device-side failures (a non-finite scaling, a bounded wait that ran out)
 *    are reported in lsf_result.status on the device; host-side checks
 *    (arguments, launch errors) in the return value.
 *  - Sizes: a measure has at least one point (n >= 1); empty measures are an
 *    argument error (LSF_ERR_ARG).
 */
#ifndef SINKHORN_PF_H
#define SINKHORN_PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSF_OK = 0,
  LSF_ERR_ARG = 1,         /* invalid argument: NULL pointer, bad size, misalignment  */
  LSF_ERR_NONFINITE = 2,   /* a scaling became 0, inf or NaN (device status bit)       */
  LSF_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out (device status bit)   */
  LSF_ERR_WORKSPACE = 8,   /* workspace smaller than lsf_workspace_bytes() asks for    */
  LSF_ERR_CUDA = 16,       /* a CUDA runtime call or launch failed                     */
  LSF_ERR_UNSUPPORTED = 32 /* a size outside what the kernels handle                   */
} lsf_status;

/* Solver variants for the fused passes of Alg. 1 (Sec. 2) on K = xi zeta^T (Sec. 3.1). */
typedef enum {
  LSF_MODE_STORED = 0,     /* stream stored shifted features F (HBM-bound)            */
  LSF_MODE_RECOMPUTE = 1,  /* recompute features from X, U in registers (ALU-bound)   */
  LSF_MODE_LOG = 2,        /* stored LOG features, log-domain iterates (stabilised):
                              F holds log features (lsf_log_features), the scalings
                              u, v hold log u~, log v~, t_u, t_v hold log t, and the
                              global factor M is 0                                    */
  LSF_MODE_HYBRID = 3,     /* the first c0 feature columns recomputed in registers (as
                              RECOMPUTE), the other ldr - c0 streamed from a stored
                              block (as STORED), in the same pass, so HBM and the
                              FP32 pipe work at once. F holds the stored block
                              (lsf_hybrid_features, n x (ldr - c0)); X is needed too.
                              c0 = lsf_hybrid_columns(ldr). Scalings as STORED.       */
  LSF_MODE_AUTO = 4        /* lsf_solve / lsf_debiased pick the domain: F and shift of
                              both clouds are OUTPUT buffers here (F: n x ldr floats,
                              16-byte aligned); the library builds the features
                              itself from X and theta, with the within-row
                              log-feature spread. Spread above LSF_AUTO_SPREAD nats:
                              log features and LSF_MODE_LOG. Otherwise shifted
                              features and LSF_MODE_STORED, and if that run reports
                              LSF_ERR_NONFINITE, F is rebuilt as log features and the
                              solve repeated in LSF_MODE_LOG. lsf_result.mode records
                              the mode whose features, scalings and W are returned.
                              Synchronises the stream (the spread and the status are
                              read on the host).                                      */
} lsf_mode;

/* AUTO's spread threshold (nats): the shifted features of rows whose log-features
   spread more than this underflow so far that a scaling-domain run is pointless. */
#define LSF_AUTO_SPREAD 4000.0

/* Feature parameters theta = (U, c), shared by every term of Eq. (2). Device pointers. */
typedef struct {
  const float* U;   /* r x d anchors u_k (Lemma 1: u_k ~ N(0, sigma^2 I))                */
  const float* c;   /* r per-anchor log-constants
                       c_k = (d/4) log(2q) - (1/2) log r + ||u_k||^2 / (eps q)            */
  int r;            /* number of features, 1 <= r <= ldr                                  */
  int ldr;          /* row stride of stored features (multiple of 4, <= 1024)             */
  int d;            /* dimension of the points, 1 <= d                                    */
  double eps;       /* entropic regularisation eps > 0                                    */
} lsf_theta;

/* One weighted point cloud with its features. Device pointers. */
typedef struct {
  const float* X;      /* n x d points (needed by RECOMPUTE and by the gradient)         */
  const float* F;      /* n x ldr shifted features (needed by STORED; may be NULL else)  */
  const float* shift;  /* n row log-shifts                                               */
  const float* w;      /* n positive weights (a or b)                                    */
  int64_t n;           /* number of points, >= 1                                         */
} lsf_cloud;

/* Outputs of one solve: shifted scalings and the two r-vectors of the last state. */
typedef struct {
  float* u;     /* n   u~ (see conventions)                                               */
  float* v;     /* m   v~                                                                 */
  float* t_u;   /* ldr xi~^T u~   (zero beyond r)                                         */
  float* t_v;   /* ldr zeta~^T v~ (zero beyond r)                                         */
} lsf_scalings;

/* Device-resident result record of one solve (caller allocates sizeof(lsf_result)). */
typedef struct {
  double W;          /* Eq. (6) estimate eps (a^T log u + b^T log v); set by lsf_divergence  */
  double residual;   /* ||u o (K v) - a||_1 after the last v-half (Alg. 1 stopping quantity)  */
  double log_scale;  /* M, the global factor of the scalings (see conventions)                */
  int32_t status;    /* OR of device-side status bits (LSF_ERR_NONFINITE, LSF_ERR_TIMEOUT).
                        Once a scaling-domain run (stored or recompute) has set
                        LSF_ERR_NONFINITE, its remaining passes stream nothing: the
                        run is void and W, the scalings and the r-vectors are not
                        meaningful (repeat it with LSF_MODE_LOG).                    */
  int32_t iters;     /* iterations run                                                         */
  int32_t mode;      /* the lsf_mode the scalings and W are in (LSF_MODE_LOG: logs); with
                        LSF_MODE_AUTO the mode it picked                                     */
  int32_t reserved;  /* zero                                                                  */
} lsf_result;

/* ---------------------------------------------------------------- library */

/* ABI version of this header (increments on any incompatible change): 2. */
int lsf_version(void);

/* Last error message of the calling host thread ("" if none). Never NULL. */
const char* lsf_last_error(void);

/* ---------------------------------------------------------------- host math */

/*
 * Lemma 1 (Sec. 3.2): q = R^2 / (2 eps d W0(R^2/(eps d))) with W0 the principal
 * Lambert branch, sigma = sqrt(q eps / 4). R = 0 gives the limit q = 1/2.
 * Host only. Errors: LSF_ERR_ARG if eps <= 0, d < 1, R < 0 or R not finite,
 * or q/sigma NULL.
 */
int lsf_gaussian_params(double R, double eps, int d, double* q, double* sigma);

/* ---------------------------------------------------------------- features */

/*
 * R for Lemma 1: the largest Euclidean norm over the rows of X (n x d) and
 * Y (m x d), written as one float to device R_out. Lemma 1 needs x, y in
 * B(0, R); this is the smallest such ball centred at 0.
 */
int lsf_radius(const float* X, int64_t n, const float* Y, int64_t m, int d,
               float* R_out, void* stream);

/*
 * Anchors and their log-constants (Lemma 1 and the definition of phi_theta,
 * Sec. 3.2): U = sigma * Z for standard normal draws Z (r x d, device), and
 * c_k = (d/4) log(2q) - (1/2) log r + ||u_k||^2 / (eps q) (computed in FP64,
 * stored FP32). Outputs U (r x d) and c (r), device.
 */
int lsf_anchors(const float* Z, int r, int d, double q, double sigma, double eps,
                float* U, float* c, void* stream);

/*
 * Stored shifted features (Lemma 1 map, phi_theta of Sec. 3.2):
 *   L_ik = c_k - (2/eps) ||x_i - u_k||^2,   shift[i] = max_{k<r} L_ik,
 *   F[i*ldr + k] = exp(L_ik - shift[i]) for k < r, 0 for r <= k < ldr.
 * X: n x d device; F: n x ldr device (16-byte aligned); shift: n device.
 * spread (device float, may be NULL) receives max_i (max_k L_ik - min_k L_ik)
 * via an atomic maximum; zero it before the first call.
 */
int lsf_features(const float* X, int64_t n, const lsf_theta* theta,
                 float* F, float* shift, float* spread, void* stream);

/*
 * Log form of the stored features, for LSF_MODE_LOG: L[i*ldr + k] = L_ik - shift[i]
 * (<= 0) for k < r and -inf for r <= k < ldr. Same arguments as lsf_features.
 * Used when the within-row spread max_k L_ik - min_k L_ik leaves the FP32 range
 * of exp (the shifted features would underflow to 0 and a scaling could divide
 * by zero).
 */
int lsf_log_features(const float* X, int64_t n, const lsf_theta* theta,
                     float* L, float* shift, float* spread, void* stream);

/* As lsf_features but writes only shift (and spread): the RECOMPUTE prologue. */
int lsf_row_shift(const float* X, int64_t n, const lsf_theta* theta,
                  float* shift, float* spread, void* stream);

/*
 * Column split of LSF_MODE_HYBRID for row stride ldr (multiple of 4 in
 * [8, 1024]): *c0 receives the first stored column. Columns [0, c0) are rebuilt
 * in the pass, columns [c0, ldr) are read from the stored block (half of the
 * float4 column groups, rounded down, are stored). Host only.
 * Errors: LSF_ERR_ARG (NULL), LSF_ERR_UNSUPPORTED (ldr).
 */
int lsf_hybrid_columns(int ldr, int* c0);

/*
 * Features of LSF_MODE_HYBRID (Lemma 1 map, as lsf_features): the row shifts
 * over all r features, shift[i] = max_{k<r} L_ik, and the stored block
 *   Fs[i*(ldr - c0) + (k - c0)] = exp(L_ik - shift[i]) for c0 <= k < r, 0 for k >= r,
 * with c0 = lsf_hybrid_columns(theta->ldr). X: n x d device; Fs: n x (ldr - c0)
 * device (16-byte aligned); shift: n device; spread as lsf_features.
 */
int lsf_hybrid_features(const float* X, int64_t n, const lsf_theta* theta,
                        float* Fs, float* shift, float* spread, void* stream);

/*
 * Arc-cosine positive features (Sec. 3.2, "Arc-cosine kernels", and the lemma
 * in the appendix): the perturbed kernel k_s(x,y) + kappa, where
 *   k_s(x,y) = int Theta_s(u.x) Theta_s(u.y) dN(0,I)(u),  Theta_s(w) = sqrt(2) max(0,w)^s,
 * has the features phi(x,u) = (sigma^{d/2} sqrt(2) max(0,u.x)^s
 * exp(-||u||^2 (1 - 1/sigma^2)/4), sqrt(kappa)) for u ~ N(0, sigma^2 I),
 * sigma > 1. With r anchors the r constant entries only enter K through their
 * sum, so they are merged into one last feature: r + 1 features per point,
 *   L_ik = c_k + s log(u_k.x_i)  (u_k.x_i > 0; -inf, i.e. an exact zero, else),
 *   L_ir = log sqrt(kappa),
 * c_k = (d/2) log sigma + (1/2) log 2 - (1/2) log r - ||u_k||^2 (1 - 1/sigma^2)/4.
 * The kernel has no bandwidth: Sinkhorn runs on K = xi zeta^T as it is, and eps
 * (lsf_theta.eps of the solve) only scales the divergence, W = eps (a.log u + b.log v).
 * The stored solve, the log-domain solve and the batched solver take these
 * features unchanged (an lsf_theta with r + 1 features and the solve's eps).
 * The recompute mode and lsf_gradient / lsf_anchor_gradient evaluate the
 * Gaussian map and its derivatives; they must not be given arc-cosine
 * features (the library cannot tell the maps apart from F).
 */
typedef struct {
  const float* U;   /* r x d anchors (lsf_arccos_anchors)                          */
  const float* c;   /* r log-constants c_k                                          */
  int r;            /* anchors, >= 1                                                */
  int ldr;          /* row stride: multiple of 4, >= r + 1, <= 1024                */
  int d;            /* dimension, >= 1                                              */
  int s;            /* exponent 0, 1 or 2 (max(0,w)^0 is taken as 0 for w <= 0)     */
  double kappa;     /* perturbation > 0 (k >= kappa keeps every entry of K positive) */
} lsf_arccos;

/* U = sigma * Z (Z: r x d standard normal draws, device) and the constants c_k
 * above. sigma > 1. Outputs U (r x d) and c (r), device. */
int lsf_arccos_anchors(const float* Z, int r, int d, double sigma, float* U, float* c,
                       void* stream);

/* Stored shifted arc-cosine features: shift[i] = max_{k<=r} L_ik,
 * F[i*ldr + k] = exp(L_ik - shift[i]) for k <= r, 0 beyond. Arguments, layout
 * and the spread output as lsf_features (the spread ignores exact zeros). */
int lsf_arccos_features(const float* X, int64_t n, const lsf_arccos* params,
                        float* F, float* shift, float* spread, void* stream);

/* Log form for LSF_MODE_LOG: L[i*ldr + k] = L_ik - shift[i], -inf beyond r. */
int lsf_arccos_log_features(const float* X, int64_t n, const lsf_arccos* params,
                            float* L, float* shift, float* spread, void* stream);

/* ---------------------------------------------------------------- solver */

/*
 * Bytes of scratch workspace one solve or one debiased solve needs for a given
 * ldr on the current device. The same workspace must not be used by two calls
 * that can overlap on the GPU.
 */
int lsf_workspace_bytes(int ldr, size_t* bytes);

/*
 * Alg. 1 (Sec. 2) on the factored kernel K_theta = xi^T zeta (Sec. 3.1),
 * in this order: from v = 1, `iters` times u <- a/(K v), v <- b/(K^T u).
 * Each half is one fused pass over a feature matrix that forms s = F t,
 * divides the weights by s and accumulates the transposed product in the same
 * read. After the loop one more read of F gives the residual
 * ||u o (K v) - a||_1. x->w = a, y->w = b.
 * Writes out (u~, v~, t_u, t_v) and result->{residual, log_scale, status, iters}.
 * workspace: >= lsf_workspace_bytes(theta->ldr) bytes, device, 256-byte aligned.
 */
int lsf_solve(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
              int mode, const lsf_scalings* out, lsf_result* result,
              void* workspace, size_t ws_bytes, void* stream);

/*
 * Eq. (6) for up to three solved pairs and their weighted sum:
 *   result[t].W = eps (sum_i a_i log u_i + sum_j b_j log v_j)   (FP64 compensated sum)
 *   *combined   = sum_t coef[t] * result[t].W    (combined may be NULL)
 * With coef = {1, -1/2, -1/2} over (xy, xx, yy) this is Eq. (2).
 * mode: the lsf_mode the scalings were produced in (LSF_MODE_LOG scalings are logs);
 * LSF_MODE_AUTO takes each term's mode from its result record (lsf_result.mode).
 */
int lsf_divergence(const lsf_theta* theta, int nterms, const lsf_cloud* const* xs,
                   const lsf_cloud* const* ys, const lsf_scalings* const* s,
                   lsf_result* const* result, const double* coef, double* combined, int mode,
                   void* workspace, size_t ws_bytes, void* stream);

/*
 * Debiased Sinkhorn divergence, Eq. (2): W(a,b) - (W(a,a) + W(b,b))/2 with one
 * shared theta. The three solves run in lock-step so that per iteration xi is
 * read twice ({XY-u, XX-u}, {XX-v}) and zeta twice ({XY-v, YY-u}, {YY-v}).
 * result: device array of 3 lsf_result (xy, xx, yy), each with W filled in.
 * wbar: device double receiving W_bar (may be NULL).
 */
int lsf_debiased(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
                 int mode, const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                 const lsf_scalings* s_yy, lsf_result* result, double* wbar,
                 void* workspace, size_t ws_bytes, void* stream);

/*
 * Alg. 1 (Sec. 2) with its stopping rule: as lsf_solve, but the loop ends at the
 * first check where the residual ||u o (K v) - a||_1 (after the v-half) is at
 * most tol. The residual is evaluated every check_every iterations (1: after
 * every iteration, as Alg. 1 states it; a larger interval trades up to
 * check_every - 1 extra iterations for fewer residual reads of F), and after
 * max_iters iterations at the latest. result->iters receives the iterations run
 * and result->residual the last residual evaluated (above tol if max_iters was
 * reached first). Every check synchronises the stream (the residual is read on
 * the host), so this call blocks and is not for stream capture; the passes are
 * those of lsf_solve (the single-launch small-problem solver is not used).
 * Errors: LSF_ERR_ARG for max_iters < 1, tol < 0 or NaN, check_every < 1; then as
 * lsf_solve. A run that reports LSF_ERR_NONFINITE stops at that check.
 */
int lsf_solve_tol(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int max_iters,
                  double tol, int check_every, int mode, const lsf_scalings* out,
                  lsf_result* result, void* workspace, size_t ws_bytes, void* stream);

/*
 * Eq. (2) with Alg. 1's stopping rule on each of its three terms: as
 * lsf_debiased, but each term (xy, xx, yy) stops at the first check (every
 * check_every iterations, and at max_iters) where its own residual is at most
 * tol; the lock-step passes then carry only the terms still running. Each
 * result record gets its own iteration count and last residual; W and W_bar are
 * formed from every term's final scalings. Synchronises the stream at every
 * check, as lsf_solve_tol. Errors as lsf_solve_tol.
 */
int lsf_debiased_tol(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int max_iters,
                     double tol, int check_every, int mode, const lsf_scalings* s_xy,
                     const lsf_scalings* s_xx, const lsf_scalings* s_yy, lsf_result* result,
                     double* wbar, void* workspace, size_t ws_bytes, void* stream);

/*
 * lsf_solve for callers that cannot allocate device memory. The paper has no
 * counterpart; this exists for the library's users.
 *
 * Who needs it: code that runs inside a framework whose memory pool owns all of
 * the device memory (an outside cudaMalloc breaks the pool's accounting and
 * synchronises the whole device), or a latency-bound serving loop that must not
 * block on the allocator. Such a caller still passes its inputs and outputs
 * exactly as for lsf_solve, but no workspace.
 *
 * Scratch: a fixed 12 MiB array in the library's device image (kept by every GPU
 * that loads the library until the process exits). Problems whose
 * lsf_workspace_bytes(theta->ldr) exceeds 12 MiB are rejected with
 * LSF_ERR_UNSUPPORTED and a message; nothing is allocated, ever. (The scratch
 * grows with the SM count: at ldr = 1024 it is about 8.0 MB on 152 SMs, so the
 * rejection is only reached on parts with about 240 SMs or more.)
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture. The address is kept for the life of the process:
 * after cudaDeviceReset on a device, do not call this entry point on that device
 * again in the same process. Every call shares the one array: the solve clears
 * the parts that must start at zero, and two calls that can overlap on the GPU
 * (different streams, or different host threads) race on it and give wrong
 * results. Results, errors and device status are those of lsf_solve.
 */
int lsf_solve_noalloc(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
                      int mode, const lsf_scalings* out, lsf_result* result, void* stream);

/* ---------------------------------------------------------------- whole path */

/*
 * One divergence problem from host inputs to host results, for callers that
 * hold their data in host memory (a request in a serving loop, an end-to-end
 * measurement): Lemma 1 (R from both clouds, then q and sigma from the Lambert
 * W0 of Sec. 3.2 evaluated on the device, anchors U = sigma Z and constants
 * c_k), the features of the chosen mode, Alg. 1 (Sec. 2) on K = xi zeta^T
 * (Sec. 3.1) for each term, Eq. (6) and, when debiased, Eq. (2) with one shared
 * theta. Every device buffer lives in one caller-owned arena.
 */
typedef struct {
  int64_t n, m;    /* points of X and Y, >= 1                                       */
  int d;           /* dimension, >= 1                                               */
  int r;           /* features (anchors), >= 1                                      */
  int ldr;         /* feature row stride (0: r rounded up to a multiple of 4)       */
  double eps;      /* entropic regularisation, > 0                                  */
  int iters;       /* Alg. 1 iterations per solve, >= 1                             */
  int debiased;    /* 1: Eq. (2) (three solves); 0: Eq. (6) of W(a, b) alone        */
  int mode;        /* LSF_MODE_STORED, _RECOMPUTE, _HYBRID, _LOG or _AUTO          */
} lsf_pipeline;

/* Host results of lsf_pipeline_run. */
typedef struct {
  double W;                 /* Eq. (2) when debiased, else Eq. (6) of W(a, b)       */
  double W_xy, W_xx, W_yy;  /* Eq. (6) per term (W_xx, W_yy zero when not debiased) */
  double residual_xy, residual_xx, residual_yy;  /* ||u o (K v) - a||_1 per term    */
  double R, q, sigma;       /* the Lemma 1 parameters used                          */
  int32_t status;           /* OR of the device status bits of every solve          */
  int32_t mode;             /* the lsf_mode that produced the result                */
  int32_t iters;            /* iterations run                                       */
  int32_t reserved;
} lsf_pipeline_out;

/* Arena bytes lsf_pipeline_run needs for a problem description. Host only.
 * Errors: LSF_ERR_ARG / LSF_ERR_UNSUPPORTED for an invalid description. */
int lsf_pipeline_bytes(const lsf_pipeline* p, size_t* bytes);

/*
 * Run the whole path. X (n x d), Y (m x d), a (n), b (m): host points and
 * weights (a, b positive, each summing to 1); Z (r x d): host standard normal
 * draws of the anchors. arena: device, 256-byte aligned, >= lsf_pipeline_bytes;
 * it holds copies of the inputs, theta, features, scalings, results and the
 * solver workspace, and no two calls that can overlap on the GPU may share it.
 * out: host record, written by a copy at the end of the call's work on the
 * stream.
 * Nothing is allocated. Except in LSF_MODE_AUTO, the call never waits on the
 * device: the host-to-device copies of the inputs, every kernel and the copy of
 * *out are queued on the stream, and *out is valid once the stream has
 * reached it (cudaStreamSynchronize, or an event recorded after the call). Host
 * inputs in pinned memory must stay unchanged until then; pageable ones are
 * staged by the copy. LSF_MODE_AUTO synchronises the stream inside (see
 * lsf_mode). Errors: those of the steps, with device status bits in out->status.
 *
 * With p->iters == 0 the call only prepares the problem (inputs in, Lemma 1,
 * anchors and the features of p->mode, which must then be LSF_MODE_STORED or
 * LSF_MODE_LOG); out may be NULL. A batched solve (lsf_batch_plan and
 * lsf_solve_batched on the buffers lsf_pipeline_layout names) then solves the
 * terms, and lsf_pipeline_finish writes the record.
 */
int lsf_pipeline_run(const lsf_pipeline* p, const float* X, const float* Y, const float* a,
                     const float* b, const float* Z, void* arena, size_t arena_bytes,
                     lsf_pipeline_out* out, void* stream);

/* Device views into a pipeline arena: theta, both clouds (X, features, shifts,
 * weights), the scalings of the terms (xy, xx, yy) and their 3 result records. */
typedef struct {
  lsf_theta theta;
  lsf_cloud x, y;
  lsf_scalings s[3];
  lsf_result* result;
} lsf_pipeline_views;

/* Fill *v for a description and an arena (host only; nothing is launched). */
int lsf_pipeline_layout(const lsf_pipeline* p, void* arena, lsf_pipeline_views* v);

/* The host record of a problem whose terms were solved on the arena's buffers
 * by another call (a batched solve): Eq. (2) (when debiased) from the three
 * result records' Eq. (6) values, R, q, sigma, status, mode; copied to the host
 * record *out on the stream (valid once the stream has reached it). */
int lsf_pipeline_finish(const lsf_pipeline* p, void* arena, lsf_pipeline_out* out, void* stream);

/* ---------------------------------------------------------------- batched */

/*
 * Many independent problems W(a_p, b_p) (Eq. 6 after Alg. 1 on each problem's
 * K_p = xi_p zeta_p^T) solved together by one persistent, cooperative kernel:
 * every half iteration streams the rows of all problems' features through the
 * same shared-memory ring, so small problems do not leave SMs idle and no
 * kernel is launched per problem and per half iteration. All problems of one
 * batch share ldr (group problems by feature width); n, m, d, r <= ldr and eps
 * may differ. Features are stored (lsf_features) and stay resident.
 * Device pointers in each record; result: one lsf_result per problem (W,
 * residual, log_scale, status filled in).
 */
typedef struct {
  const float* Fx;       /* n x ldr shifted features of X   */
  const float* Fy;       /* m x ldr shifted features of Y   */
  const float* shift_x;  /* n                              */
  const float* shift_y;  /* m                              */
  const float* a;        /* n weights                      */
  const float* b;        /* m weights                      */
  int64_t n, m;
  double eps;
  float* u;              /* n   u~ (output)                */
  float* v;              /* m   v~ (output)                */
  float* t_u;            /* ldr (output)                   */
  float* t_v;            /* ldr (output)                   */
  lsf_result* result;    /* 1 record (output)              */
} lsf_batch_problem;

/* Host description of a batch plan (filled by lsf_batch_plan). */
typedef struct {
  int count;          /* problems                                  */
  int ldr;            /* common row stride                         */
  int mode;           /* LSF_MODE_STORED or LSF_MODE_LOG            */
  int tile_rows;      /* rows per shared-memory tile               */
  int stages;         /* copy-ring depth                           */
  int grid;           /* CTAs of the persistent kernel (co-resident) */
  int64_t tiles_x;    /* tiles over all X-side rows                */
  int64_t tiles_y;    /* tiles over all Y-side rows                */
  int64_t rows_x;     /* sum of n over the batch                   */
  int64_t rows_y;     /* sum of m over the batch                   */
  size_t plan_bytes;  /* device plan size                          */
  size_t smem_bytes;  /* dynamic shared memory of the kernel       */
  int strategy;       /* 0 persistent kernel, 1 one cluster per problem */
} lsf_batch_info;

/*
 * Plan a batch: mode LSF_MODE_STORED (Fx, Fy shifted features; u, v, t hold
 * scalings) or LSF_MODE_LOG (Fx, Fy log features from lsf_log_features; u, v, t
 * hold logs; for problems outside the FP32 range of the scaling domain). Choose
 * the tiling (tile_bytes = 0 picks the default; the
 * autotuner passes candidates), partition the concatenated tiles of all problems
 * over the CTAs, and lay out the device plan (problem table, tile tables,
 * partial buffers, arrival counters, round flags). With plan == NULL only
 * *info is filled (to size the buffer); otherwise the plan (info->plan_bytes,
 * device, 256-byte aligned) is written with a copy that completes before
 * return. probs: host array of `count` records.
 */
int lsf_batch_plan(const lsf_batch_problem* probs, int count, int ldr, int mode, int tile_bytes,
                   lsf_batch_info* info, void* plan, size_t plan_bytes, void* stream);

/*
 * Run `iters` iterations of Alg. 1 on every problem of a planned batch, then the
 * residual pass and Eq. (6): a start kernel (v = 1 per problem), one persistent
 * cooperative kernel for all half iterations (problems advance independently,
 * ordered by per-problem round flags with bounded waits), and a reduction
 * kernel. Only kernel launches: capturable in a CUDA graph.
 */
int lsf_solve_batched(const lsf_batch_info* info, void* plan, int iters, void* stream);

/*
 * How lsf_batch_plan lays out a stored batch (the iterates are the same): 0 one
 * persistent kernel streaming all problems' tiles every round (problems of any
 * size); 1 one 8-CTA thread-block cluster per problem, all problems in one
 * launch, each cluster running its problem's iterations with its features read
 * from L2; 2 the cluster layout when the batch has at least 2 * SMs / 8
 * problems and each has (n + m) * ldr <= 2^18. The default is 0 (on the batched
 * workload of n, m up to 2^16 the persistent kernel is 1.4x faster). Log-domain
 * batches always use the persistent kernel. Recorded in
 * lsf_batch_info.strategy; process-wide.
 * Errors: LSF_ERR_ARG for a value outside 0..2.
 */
int lsf_set_batch_strategy(int strategy);

/*
 * Failure-detection hook of the batched solver, for tests (not a paper
 * quantity). Every wait of the persistent kernel is bounded; this makes one run
 * out on purpose, without a GPU fault.
 * wait_limit_ns: the limit of the kernel's waits on round flags and on its
 * shared-memory ring (default 4e9 ns; range [1e4, 6e10]). The drain of the
 * copies still in flight at exit keeps the default limit.
 * stall_rounds: 0 (default) or 1. With 1, each consumer waits for a problem's
 * round flag to pass one round beyond the round the kernel will ever publish (a
 * flag nothing sets): from the second round on every such wait runs out, the
 * kernel stops streaming, drains its copies and returns, and every problem's
 * lsf_result.status gets LSF_ERR_TIMEOUT. The device stays usable.
 * Process-wide; reset with lsf_set_batch_fault(4000000000, 0).
 * Errors: LSF_ERR_ARG for values outside those ranges.
 */
int lsf_set_batch_fault(unsigned long long wait_limit_ns, int stall_rounds);

/* ---------------------------------------------------------------- adjoint */

/*
 * Envelope gradient (Prop. 3.3 and the formula after it, Sec. 3.3) with theta
 * held fixed. For W(a,b): dW/dK = -eps u v^T, chained through the features:
 *   grad x_i = 4 u~_i sum_k t_v[k] F_ik (x_i - u_k)   (t_v = zeta~^T v~)
 *   grad y_j = 4 v~_j sum_k t_u[k] G_jk (y_j - u_k)   (t_u = xi~^T u~)
 *   grad a_i = eps log u_i,  grad b_j = eps log v_j.
 * With debiased != 0 the gradient is that of Eq. (2): the self terms W(a,a),
 * W(b,b) (kernel xi xi^T, X on both sides) enter with weight -1/2, using
 * s_xx, s_yy and result[1], result[2].
 * mode: LSF_MODE_STORED (F = xi~) or LSF_MODE_LOG (F, scalings and r-vectors
 * in log form); the recompute mode keeps no features and is not supported.
 * gX (n x d), gY (m x d), ga (n), gb (m): device outputs (any may be NULL).
 * result: device array of 1 (or 3 when debiased) lsf_result from the solve.
 */
int lsf_gradient(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y,
                 const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                 const lsf_scalings* s_yy, const lsf_result* result, int debiased, int mode,
                 float* gX, float* gY, float* ga, float* gb, void* stream);

/*
 * Envelope gradient w.r.t. the anchors U (r x d), with q held fixed: the
 * gradient a learned feature map needs (Sec. 3.3 learns the features through
 * the same envelope gradient, Prop. 3.3). Every feature of both clouds depends
 * on u_k through ||p - u_k||^2 and the weight ||u_k||^2/(eps q) of Lemma 1:
 *   grad u_k = -sum_i A_ik (4 (x_i - u_k) + 2 u_k/q) - sum_j B_jk (4 (y_j - u_k) + 2 u_k/q),
 *   A_ik = u~_i t_v[k] F_ik (the mass of gradient x_i), B_jk = v~_j t_u[k] G_jk,
 * with the self terms of Eq. (2) at weight -1/2 when debiased != 0 (s_xx,
 * s_yy). q is the Lemma 1 parameter the features were built with. mode:
 * LSF_MODE_STORED or LSF_MODE_LOG, as in lsf_gradient. The device output gU
 * (r x d) is overwritten with scale * grad U (scale = sigma gives the gradient
 * w.r.t. the normal draws Z of U = sigma Z). x->X, x->F, y->X, y->F and the
 * r-vectors of the scalings are required (the r-vectors 16-byte aligned).
 * workspace: the solve's workspace (lsf_workspace_bytes(ldr) bytes); its
 * partial region is overwritten, so no solve may use it concurrently.
 * Summation order is fixed: the result is deterministic.
 * Errors: LSF_ERR_ARG (NULL or misaligned pointers, bad sizes),
 * LSF_ERR_UNSUPPORTED (recompute mode, or d so large that the partials do
 * not fit the workspace: d above 8 * floor(8 * SMs / 9), 1080 on 152 SMs),
 * LSF_ERR_WORKSPACE.
 */
int lsf_anchor_gradient(const lsf_theta* theta, double q, const lsf_cloud* x, const lsf_cloud* y,
                        const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                        const lsf_scalings* s_yy, int debiased, int mode, double scale, float* gU,
                        void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- tuning */

/*
 * Tiling of the stored-feature pass: target bytes per shared-memory tile
 * (rounded to whole rows for every consumer warp, and shrunk for small inputs so
 * that every SM gets work) and the maximum depth of the copy ring (limited by
 * shared memory). Not a paper quantity: a launch parameter picked by the
 * autotuner. Process-wide; set it before launching. Errors: LSF_ERR_ARG if
 * tile_bytes is outside [512, 131072] or max_stages outside [2, 16].
 */
int lsf_set_pass_tiling(int tile_bytes, int max_stages);
int lsf_get_pass_tiling(int* tile_bytes, int* max_stages);

/*
 * Solver choice for stored-feature problems whose features stay in L2 (not a
 * paper quantity; the iterates are the same). Small problems spend most of a
 * multi-launch solve in launch and grid-reduction latency, so lsf_solve and
 * lsf_debiased run them instead in one launch of a cluster-persistent kernel
 * (one thread-block cluster per solve, the r-vector reduced across the cluster
 * in distributed shared memory every half iteration). policy: 0 never, 1 when
 * (n + m) * ldr <= max_entries for every solve of the call (default, with
 * max_entries = 2^24), 2 always. Process-wide; set it before launching.
 * Errors: LSF_ERR_ARG for a policy outside 0..2 or max_entries < 0.
 */
int lsf_set_small_solver(int policy, int64_t max_entries);

/* ---------------------------------------------------------------- measurement */

/* ---------------------------------------------------------------- accelerated */

/* Statistics of an accelerated solve (host memory, filled on return). */
typedef struct {
  int32_t iters;     /* accepted iterations                                   */
  int32_t attempts;  /* line-search attempts (three log-domain passes each)   */
  double A;          /* A_k after the last iteration (the estimate sequence)  */
  double L;          /* Lipschitz estimate of the last accepted attempt       */
} lsf_accel_info;

/*
 * Bytes of workspace lsf_solve_accelerated needs for n points in x, m in y and
 * row stride ldr: the pass workspace of lsf_workspace_bytes(ldr) followed by
 * six n-vectors, six m-vectors, two r-vectors and the reduction partials.
 */
int lsf_accel_workspace_bytes(int64_t n, int64_t m, int ldr, size_t* bytes);

/*
 * Accelerated Sinkhorn (App. A.2) on the factored kernel, log domain only. The
 * appendix's listing is garbled; this follows the accelerated alternating
 * minimisation it cites: minimise phi(eta) = log <e^eta1, K e^eta2> -
 * <eta1, a> - <eta2, b> (W = -eps min phi) from eta = zeta = 0 with an estimate
 * sequence and an adaptive Lipschitz estimate L (starting at L0 > 0, halved at
 * every iteration, doubled after every rejected attempt). An attempt
 * interpolates lam = tau zeta + (1 - tau) eta, takes the gradient
 * (P 1 - a, P^T 1 - b) at lam, refits the block with the larger gradient norm by
 * a Sinkhorn half-step and accepts when phi drops by ||g||^2/(2L); then
 * zeta -= a_k g. Each attempt is three log-domain passes (x->F, y->F hold log
 * features from lsf_log_features) and four small kernels.
 *
 * Writes out->u = log u~ = eta1 + x->shift and out->v = log v~ = eta2 + y->shift
 * (the LSF_MODE_LOG conventions, so lsf_divergence(..., LSF_MODE_LOG) gives
 * Eq. (6) at the final point), out->t_u, out->t_v (log r-vectors at that point),
 * result->residual = ||P 1 - a||_1 + ||P^T 1 - b||_1 there, result->iters, and
 * *info (may be NULL). An iteration with more than 30 attempts ends the solve
 * early (the required decrease is below the rounding of phi: the point is
 * stationary to working precision); result->iters and info->iters then count
 * the iterations done. Synchronises `stream` once per attempt (the host reads
 * the acceptance decision). Errors: LSF_ERR_ARG for iters < 1 or L0 not
 * positive, LSF_ERR_WORKSPACE below lsf_accel_workspace_bytes,
 * LSF_ERR_NONFINITE when a dual value is not finite.
 */
int lsf_solve_accelerated(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
                          double L0, const lsf_scalings* out, lsf_result* result,
                          lsf_accel_info* info, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------ many weight vectors on one support */

/*
 * Features in the form the tensor-core pass reads (lsf_solve_multi): two bf16
 * planes of n x ldr2 in one buffer, plane 0 (F2[0 .. n*ldr2)) hi = RN_bf16(F) and
 * plane 1 (F2[n*ldr2 .. 2*n*ldr2)) lo = RN_bf16(F - hi), so that hi + lo equals
 * the shifted features F of lsf_features to 2^-16 relative, in the same 4 bytes
 * per entry. Columns r..ldr2-1 are zero. Row shifts are those of lsf_features.
 * F: n x ldr FP32 (device); F2: 2 x n x ldr2 uint16 bf16 bit patterns (device,
 * 256-byte aligned for lsf_solve_multi). ldr2 is a multiple of 128, <= 1024, >= r.
 * Errors: LSF_ERR_ARG (NULL, n < 1, r outside [1, min(ldr, ldr2)]),
 * LSF_ERR_UNSUPPORTED (ldr2).
 */
int lsf_split_features(const float* F, int64_t n, int ldr, int r, uint16_t* F2, int ldr2,
                       void* stream);

/* One cloud with k weight vectors (device pointers). */
typedef struct {
  const uint16_t* F2;   /* bf16 pair planes, 2 x n x ldr2 (lsf_split_features)       */
  const float* shift;   /* n row log-shifts                                           */
  const float* W;       /* k x n weights: row p is the p-th measure's weights         */
  int64_t n;            /* number of points, >= 1                                     */
} lsf_multi_cloud;

/* Scalings of k solves on one support (device pointers, caller-owned). */
typedef struct {
  float* U;    /* k x n   u~ of each solve (the lsf_scalings conventions)             */
  float* V;    /* k x m   v~                                                          */
  float* Tu;   /* kp x ldr2 xi~^T u~ per solve, kp = 16 if k <= 16 else 32; rows k..kp-1 zero */
  float* Tv;   /* kp x ldr2 zeta~^T v~                                                */
} lsf_multi_scalings;

/* Workspace bytes of lsf_solve_multi for row stride ldr2 and k solves. */
int lsf_multi_workspace_bytes(int ldr2, int k, size_t* bytes);

/*
 * Alg. 1 (Sec. 2) on the factored kernel K = xi zeta^T (Sec. 3.1) for k pairs of
 * weights (a_p, b_p) on the same two point clouds and features, then Eq. (6) for
 * each: results[p] gets W, the residual ||u_p o (K v_p) - a_p||_1 after the last
 * v-half, log_scale, status and iters, exactly as lsf_solve + lsf_divergence
 * give them for the p-th pair alone. With many potentials on one support, each
 * half iteration becomes two n x r x k contractions, which run on the tensor
 * cores (tcgen05, bf16 pair features and bf16 pair splits of the scalings and
 * r-vectors, FP32 accumulation): one read of the features serves all k solves.
 * k in [1, 32]; ldr2 a multiple of 128 with r <= ldr2 <= 1024 (the accumulators,
 * 4 kp + 2 kp ldr2/128 columns for k <= 16 and 4 kp + kp ldr2/128 for k <= 32,
 * fit TMEM's 512 columns at every ldr2). theta supplies r and eps (its ldr is not used). Iterates start
 * from v = 1 as in lsf_solve. Errors: LSF_ERR_ARG, LSF_ERR_UNSUPPORTED (shapes
 * above), LSF_ERR_WORKSPACE (below lsf_multi_workspace_bytes), LSF_ERR_CUDA;
 * device status bits per solve in results[p].status.
 */
int lsf_solve_multi(const lsf_theta* theta, int ldr2, const lsf_multi_cloud* x,
                    const lsf_multi_cloud* y, int k, int iters, const lsf_multi_scalings* out,
                    lsf_result* results, void* workspace, size_t ws_bytes, void* stream);

/*
 * Eq. (2) for each of the k weight pairs (a_p, b_p) on the same two clouds and
 * features: W_bar_p = W(a_p, b_p) - (W(a_p, a_p) + W(b_p, b_p)) / 2 with one
 * shared theta. Three lsf_solve_multi calls (on (x, y), (x, x) and (y, y), with
 * the scalings s_xy, s_xx, s_yy) and a device combination: results is a device
 * array of 3k records, [0, k) for the (x, y) terms, [k, 2k) for (x, x) and
 * [2k, 3k) for (y, y), each with W, residual, log_scale, iters; the three
 * records of a pair carry the OR of their status bits. wbar: device array of k
 * doubles receiving W_bar_p (may be NULL). Other arguments, shapes and errors as
 * lsf_solve_multi; one workspace serves the three solves in turn.
 */
int lsf_multi_debiased(const lsf_theta* theta, int ldr2, const lsf_multi_cloud* x,
                       const lsf_multi_cloud* y, int k, int iters, const lsf_multi_scalings* s_xy,
                       const lsf_multi_scalings* s_xx, const lsf_multi_scalings* s_yy,
                       lsf_result* results, double* wbar, void* workspace, size_t ws_bytes,
                       void* stream);

/*
 * Tuning of lsf_solve_multi (process-wide, not thread-safe against concurrent
 * solves). The pass reads each 64-point x 128-feature chunk twice: from HBM for
 * the row products and again, a tile later, for the transposed products, which
 * must find it in L2. prefetch_chunks: how many row chunks ahead of its
 * shared-memory ring the pass requests into L2 (0 to 16; default 0).
 * l2_hints: the L2 eviction priority of the chunk reads: 0 default for both, 1
 * (default) evict first on the second read (the chunk's last use), 2
 * additionally evict last on the first read. r_vectors_resident: 1 keeps the
 * split r-vectors of the row products in shared memory for the whole launch
 * when that leaves room for at least four ring stages, 0 (default) loads their
 * 128-feature block with every row chunk (one more ring stage; faster at
 * r = 1024). Errors: LSF_ERR_ARG outside those ranges.
 */
int lsf_set_multi_tuning(int prefetch_chunks, int l2_hints, int r_vectors_resident);

/* Kernel classes timed by the optional event recorder. */
typedef enum {
  LSF_KERNEL_PASS = 0,       /* fused Sinkhorn passes (stored features)   */
  LSF_KERNEL_PASS_RECOMPUTE, /* fused Sinkhorn passes (recompute)         */
  LSF_KERNEL_FEATURES,       /* feature build and row shifts              */
  LSF_KERNEL_OTHER,          /* small kernels: init, reductions           */
  LSF_KERNEL_PASS_LOG,       /* fused Sinkhorn passes (log domain)        */
  LSF_KERNEL_BATCHED,        /* batched persistent solver                 */
  LSF_KERNEL_ADJOINT,        /* gradient kernels (points, weights, anchors) */
  LSF_KERNEL_SMALL,          /* cluster-persistent small-problem solver   */
  LSF_KERNEL_PASS_MULTI,     /* tensor-core passes, many right-hand sides */
  LSF_KERNEL_PASS_HYBRID,    /* fused passes, stored and recomputed columns */
  LSF_KERNEL_NCLASSES
} lsf_kernel_class;

/*
 * Optional CUDA-event timing of every launch the library makes, on the stream
 * it is launched on. lsf_profile_enable(1) starts recording (and clears past
 * records); lsf_profile_read synchronises the recorded events and returns, per
 * class, the summed device time in milliseconds, the number of launches and the
 * algorithmic bytes those launches move (as the library counts them).
 * Not thread-safe; meant for a benchmark driving one stream.
 */
int lsf_profile_enable(int on);
int lsf_profile_read(int kernel_class, double* total_ms, int64_t* launches, double* bytes);

/*
 * NVTX ranges on the host timeline, for a profiler that records them (ncu
 * --nvtx, Nsight Systems). level 0: none. Level 1 (the default): one range per
 * call of the main entry points, named after the call (the features, solve,
 * divergence and gradient calls, the whole-path, batched, multi-pair and
 * accelerated solves). Level 2: also one range around every kernel launch, named
 * after its lsf_kernel_class ("pass", "pass_hybrid", "features", ...). Without a
 * profiler attached a range costs a few nanoseconds of host time. previous
 * (host, may be NULL) receives the level in force before the call. Errors:
 * LSF_ERR_ARG for a level outside 0..2 (the level is then unchanged).
 * Process-wide; set it once, before the work, not concurrently with it.
 * (Measurement plumbing; the paper has no counterpart.)
 */
int lsf_set_tracing(int level, int* previous);

/*
 * Measured issue rates of the pipes the recompute and hybrid passes are bound by,
 * per SM clock per SM (not a paper quantity: the denominators of their ALU
 * roofline). One CTA of 1024 threads per SM runs independent chains of one
 * instruction kind; the SM cycle counter around the loop gives, per clock and
 * SM, the FP32 lane operations of the packed two-lane FMA (*ffma2_lane_ops) and
 * of the scalar FMA (*ffma_lane_ops), and the ex2 results of the special-function
 * unit (*ex2_ops). Host outputs; synchronises the stream.
 */
int lsf_probe_pipe_rates(double* ffma2_lane_ops, double* ffma_lane_ops, double* ex2_ops, void* stream);

/* Number of kernel launches the library issued since the last lsf_launch_count_reset(). */
int64_t lsf_launch_count(void);
void lsf_launch_count_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* SINKHORN_PF_H */
