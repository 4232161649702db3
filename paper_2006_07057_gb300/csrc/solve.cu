// Alg. 1 on the factored kernel (Sec. 3.1), Eq. (6) and Eq. (2): host orchestration
// of the fused passes plus the small kernels around them (start vector, the
// divergence reduction).
#include <cuda_runtime.h>

#include <algorithm>

#include "pass.cuh"
#include "recompute.cuh"
#include "small.cuh"
#include "solve.cuh"

namespace lsf {
namespace {

// Running maximum of a float array as an order-preserving key (key 0 = -inf).
__global__ void max_key_kernel(const float* __restrict__ x, int64_t n, unsigned* __restrict__ key) {
  float best = -INFINITY;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    best = fmaxf(best, x[i]);
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) atomicMax(key, float_key(best));
}

// v = 1 in shifted form: v~_j = exp(shift_j - M) with M = max shift (the global
// factor exp(-M) cancels in P and W and is recorded in log_scale).
// In the log domain v~ = e^shift needs no factor: log v~ = shift, and M = 0.
__global__ void init_scaling_kernel(const float* __restrict__ shift, int64_t n,
                                    const unsigned* __restrict__ key, float* __restrict__ v,
                                    double* log_scale_a, double* log_scale_b, int log_domain) {
  const float M = log_domain ? 0.f : key_float(*key);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[i] = log_domain ? shift[i] : expf(shift[i] - M);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (log_scale_a) *log_scale_a = static_cast<double>(M);
    if (log_scale_b) *log_scale_b = static_cast<double>(M);
  }
}

__global__ void set_iters_kernel(lsf_result* r0, lsf_result* r1, lsf_result* r2, int iters, int mode) {
  if (threadIdx.x == 0) {
    lsf_result* rs[3] = {r0, r1, r2};
    for (lsf_result* r : rs)
      if (r) {
        r->iters = iters;
        r->mode = mode;
      }
  }
}

// The three solves of Eq. (2) report their status bits jointly (as the lock-step
// schedule does, where they share passes): OR them and mirror.
__global__ void merge_status_kernel(lsf_result* r0, lsf_result* r1, lsf_result* r2) {
  if (threadIdx.x == 0) {
    const int32_t s = r0->status | r1->status | r2->status;
    r0->status = s;
    r1->status = s;
    r2->status = s;
  }
}

SProb small_problem(const lsf_cloud* x, const lsf_cloud* y, const lsf_scalings* s, lsf_result* r) {
  SProb p{};
  p.F[0] = x->F; p.F[1] = y->F;
  p.w[0] = x->w; p.w[1] = y->w;
  p.shift[0] = x->shift; p.shift[1] = y->shift;
  p.s[0] = s->u; p.s[1] = s->v;
  p.t[0] = s->t_u; p.t[1] = s->t_v;
  p.result = r;
  p.n[0] = x->n; p.n[1] = y->n;
  return p;
}

// ---------------------------------------------------------------- Eq. (6) reduction

struct DivSeg {
  const float* s;      // shifted scaling u~ or v~
  const float* shift;  // row shifts
  const float* w;      // weights
  int64_t n;
  int term;            // which result record
  double sign;         // +1: log u = log u~ - shift - M ; -1: log v = log v~ - shift + M
  int is_log;          // 1: the scaling array holds log u~ (log-domain mode); 0: u~;
                       // -1: as the term's result record says (its mode field)
};

struct DivArgs {
  DivSeg seg[6];
  int nseg;
  int nterms;
  double eps;
  double coef[3];
  lsf_result* res[3];
  double* combined;
  double* dpart;       // [gridDim][3]
  unsigned* counter;
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Eq. (6) for up to three solves, W_t = eps sum over the segments of term t of
// w_i (log s_i - shift_i -+ M_t). Each thread sums its elements in FP64 (a few
// dozen terms); the cross-thread and cross-block folds are fixed-order, and the
// final fold over the blocks is compensated (Neumaier, FP64).
__global__ void __launch_bounds__(256) divergence_kernel(const DivArgs a) {
  __shared__ double s_w[8][3];
  __shared__ double s_lane[32][3];
  __shared__ int s_last;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int sgi = 0; sgi < a.nseg; ++sgi) {
    const DivSeg sg = a.seg[sgi];
    const double off = static_cast<double>(sg.sign) * a.res[sg.term]->log_scale;
    const bool lg = sg.is_log < 0 ? a.res[sg.term]->mode == LSF_MODE_LOG : sg.is_log != 0;
    const int64_t chunk = (sg.n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = chunk * blockIdx.x;
    const int64_t hi = min(sg.n, lo + chunk);
    double part = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double ls = lg ? static_cast<double>(sg.s[i]) : static_cast<double>(logf(sg.s[i]));
      part = fma(static_cast<double>(sg.w[i]), ls - static_cast<double>(sg.shift[i]) - off, part);
    }
    if (sg.term == 0) acc[0] += part;
    else if (sg.term == 1) acc[1] += part;
    else acc[2] += part;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const double v = warp_sum_d(acc[t]);
    if (lane == 0) s_w[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 0; t < 3; ++t) {
      double b = 0.0;
      for (int w = 0; w < 8; ++w) b += s_w[w][t];
      a.dpart[blockIdx.x * 3 + t] = b;
    }
    __threadfence();
    s_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last || warp != 0) return;
  __threadfence();
  // lane l folds blocks l, l + 32, ... (compensated), then lane 0 folds the lanes in order
  for (int t = 0; t < a.nterms; ++t) {
    KahanSum k;
    for (unsigned g = lane; g < gridDim.x; g += 32) k.add(__ldcg(a.dpart + g * 3 + t));
    s_lane[lane][t] = k.value();
  }
  __syncwarp();
  if (lane != 0) return;
  double comb = 0.0;
  for (int t = 0; t < a.nterms; ++t) {
    KahanSum tot;
    for (int l = 0; l < 32; ++l) tot.add(s_lane[l][t]);
    const double W = a.eps * tot.value();
    a.res[t]->W = W;
    comb += a.coef[t] * W;
  }
  if (a.combined) *a.combined = comb;
  *a.counter = 0u;
}

}  // namespace

// ---------------------------------------------------------------- validation

int check_theta(const lsf_theta* th) {
  if (!th) return fail(LSF_ERR_ARG, "theta is NULL");
  if (th->r < 1 || th->d < 1 || th->r > th->ldr)
    return fail(LSF_ERR_ARG, "theta: need r >= 1, d >= 1, r <= ldr");
  if (th->ldr % 4 != 0 || th->ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "theta: ldr must be a multiple of 4, <= 1024");
  if (!(th->eps > 0.0)) return fail(LSF_ERR_ARG, "theta: eps must be > 0");
  return LSF_OK;
}

int check_cloud(const lsf_cloud* c, int mode, const char* name) {
  if (!c) return fail(LSF_ERR_ARG, "%s cloud is NULL", name);
  if (c->n < 1) return fail(LSF_ERR_ARG, "%s: a measure needs n >= 1 points", name);
  if (!c->shift || !c->w) return fail(LSF_ERR_ARG, "%s: shift and w are required", name);
  if (mode == LSF_MODE_STORED) {
    if (!c->F) return fail(LSF_ERR_ARG, "%s: stored mode needs F", name);
    if (reinterpret_cast<uintptr_t>(c->F) % 16 != 0)
      return fail(LSF_ERR_ARG, "%s: F must be 16-byte aligned", name);
  } else if (mode == LSF_MODE_RECOMPUTE) {
    if (!c->X) return fail(LSF_ERR_ARG, "%s: recompute mode needs X", name);
  } else if (mode == LSF_MODE_HYBRID) {
    if (!c->X || !c->F) return fail(LSF_ERR_ARG, "%s: hybrid mode needs X and the stored block in F", name);
    if (reinterpret_cast<uintptr_t>(c->F) % 16 != 0)
      return fail(LSF_ERR_ARG, "%s: F must be 16-byte aligned", name);
  } else if (mode == LSF_MODE_LOG) {
    if (!c->F) return fail(LSF_ERR_ARG, "%s: log mode needs the log features in F", name);
    if (reinterpret_cast<uintptr_t>(c->F) % 16 != 0)
      return fail(LSF_ERR_ARG, "%s: F must be 16-byte aligned", name);
  } else {
    return fail(LSF_ERR_ARG, "unknown mode %d", mode);
  }
  return LSF_OK;
}

int check_scalings(const lsf_scalings* s, const char* name) {
  if (!s || !s->u || !s->v || !s->t_u || !s->t_v)
    return fail(LSF_ERR_ARG, "%s scalings: u, v, t_u, t_v are required", name);
  if (reinterpret_cast<uintptr_t>(s->t_u) % 16 || reinterpret_cast<uintptr_t>(s->t_v) % 16)
    return fail(LSF_ERR_ARG, "%s scalings: t_u, t_v must be 16-byte aligned", name);
  return LSF_OK;
}

// One fused pass on one cloud in the chosen mode.
int run_pass(int mode, const lsf_theta* th, const lsf_cloud* cl, int pmode, int nrhs,
             const PassRhs* rhs, const Workspace& ws, int* status, cudaStream_t st) {
  if (mode == LSF_MODE_STORED || mode == LSF_MODE_LOG) {
    PassArgs a{};
    a.F = cl->F;
    a.n = cl->n;
    a.ldr = th->ldr;
    for (int k = 0; k < nrhs; ++k) a.rhs[k] = rhs[k];
    a.part = ws.part;
    a.gpart = ws.gpart;
    a.rpart = ws.rpart;
    a.counter = ws.counters + kPassCounter;
    a.status = status;
    return mode == LSF_MODE_LOG ? launch_logpass(pmode, nrhs, a, st) : launch_pass(pmode, nrhs, a, st);
  }
  RecomputeArgs a{};
  a.X = cl->X;
  a.shift = cl->shift;
  a.n = cl->n;
  a.U = th->U;
  a.c = th->c;
  a.r = th->r;
  a.ldr = th->ldr;
  a.d = th->d;
  a.two_over_eps = static_cast<float>(2.0 / th->eps);
  for (int k = 0; k < nrhs; ++k) a.rhs[k] = rhs[k];
  a.part = ws.part;
  a.gpart = ws.gpart;
  a.rpart = ws.rpart;
  a.counter = ws.counters + kPassCounter;
  a.status = status;
  if (mode == LSF_MODE_HYBRID) {
    HybridArgs h{};
    h.rc = a;
    h.Fs = cl->F;
    h.c0 = hybrid_first_stored(th->ldr);
    return launch_hybrid_pass(pmode, nrhs, h, st);
  }
  return launch_recompute_pass(pmode, nrhs, a, st);
}

int start_solve(void* workspace, size_t ws_bytes, int ldr, lsf_result* result, int nres,
                Workspace* ws, cudaStream_t st) {
  LSF_TRY(carve_workspace(workspace, ws_bytes, ldr, ws));
  if (!result) return fail(LSF_ERR_ARG, "result is NULL");
  if (cudaMemsetAsync(result, 0, sizeof(lsf_result) * nres, st) != cudaSuccess ||
      cudaMemsetAsync(ws->counters, 0, sizeof(unsigned) * workspace_counters(), st) != cudaSuccess ||
      cudaMemsetAsync(ws->keys, 0, sizeof(unsigned) * 8, st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "solve: memset failed");
  return LSF_OK;
}

namespace {

// LSF_MODE_AUTO: build the features of both clouds into their (output) F and
// shift buffers with the spread, pick the domain, run, and repeat in the log
// domain after a range failure. run(mode) launches the solve in one mode;
// status0 is the record that collects the device status bits.
template <class Run>
int solve_auto(const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y, lsf_result* status0,
               void* workspace, size_t ws_bytes, cudaStream_t st, Run run) {
  for (const lsf_cloud* c : {x, y}) {
    if (!c || c->n < 1 || !c->X || !c->F || !c->shift || !c->w)
      return fail(LSF_ERR_ARG, "auto mode: each cloud needs n >= 1, X, w and F, shift buffers");
    if (reinterpret_cast<uintptr_t>(c->F) % 16 != 0)
      return fail(LSF_ERR_ARG, "auto mode: F must be 16-byte aligned");
  }
  if (!th->U || !th->c) return fail(LSF_ERR_ARG, "auto mode: theta needs U and c");
  if (!status0) return fail(LSF_ERR_ARG, "result is NULL");
  Workspace ws{};
  LSF_TRY(carve_workspace(workspace, ws_bytes, th->ldr, &ws));
  float* spread = reinterpret_cast<float*>(ws.keys + 4);
  auto build = [&](bool logd, float* spr) -> int {
    for (const lsf_cloud* c : {x, y}) {
      if (c == y && y->F == x->F) break;  // one cloud on both sides
      float* F = const_cast<float*>(c->F);
      float* sh = const_cast<float*>(c->shift);
      LSF_TRY(logd ? lsf_log_features(c->X, c->n, th, F, sh, spr, st)
                   : lsf_features(c->X, c->n, th, F, sh, spr, st));
    }
    return LSF_OK;
  };
  if (cudaMemsetAsync(spread, 0, sizeof(float), st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "auto mode: memset failed");
  LSF_TRY(build(false, spread));
  float h_spread = 0.f;
  if (cudaMemcpyAsync(&h_spread, spread, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "auto mode: spread read-back failed");
  if (static_cast<double>(h_spread) > LSF_AUTO_SPREAD) {
    LSF_TRY(build(true, nullptr));
    return run(LSF_MODE_LOG);
  }
  LSF_TRY(run(LSF_MODE_STORED));
  int32_t status = 0;
  if (cudaMemcpyAsync(&status, &status0->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "auto mode: status read-back failed");
  if (!(status & LSF_ERR_NONFINITE)) return LSF_OK;
  LSF_TRY(build(true, nullptr));
  return run(LSF_MODE_LOG);
}

int init_side(const lsf_cloud* cl, unsigned* key, float* v, double* ls_a, double* ls_b, int mode,
              cudaStream_t st) {
  const int grid = device_info().sms * 2;
  LaunchScope ls(st, LSF_KERNEL_OTHER, 8.0 * cl->n);
  max_key_kernel<<<grid, 256, 0, st>>>(cl->shift, cl->n, key);
  init_scaling_kernel<<<grid, 256, 0, st>>>(cl->shift, cl->n, key, v, ls_a, ls_b,
                                            mode == LSF_MODE_LOG ? 1 : 0);
  return check_launch("init_scaling_kernel");
}

}  // namespace

int launch_divergence(const lsf_theta* th, int nterms, const lsf_cloud* const* xs,
                      const lsf_cloud* const* ys, const lsf_scalings* const* s,
                      lsf_result* const* res, const double* coef, double* combined,
                      const Workspace& ws, cudaStream_t st, int is_log) {
  DivArgs a{};
  a.nterms = nterms;
  a.eps = th->eps;
  a.combined = combined;
  a.dpart = ws.dpart;
  a.counter = ws.counters + 1;
  double bytes = 0.0;
  for (int t = 0; t < nterms; ++t) {
    a.coef[t] = coef ? coef[t] : 1.0;
    a.res[t] = res[t];
    a.seg[a.nseg++] = DivSeg{s[t]->u, xs[t]->shift, xs[t]->w, xs[t]->n, t, +1.0, is_log};
    a.seg[a.nseg++] = DivSeg{s[t]->v, ys[t]->shift, ys[t]->w, ys[t]->n, t, -1.0, is_log};
    bytes += 12.0 * (xs[t]->n + ys[t]->n);
  }
  for (int t = nterms; t < 3; ++t) a.res[t] = res[0];
  LaunchScope ls(st, LSF_KERNEL_OTHER, bytes);
  int64_t most = 1;
  for (int t = 0; t < a.nseg; ++t) most = std::max<int64_t>(most, a.seg[t].n);
  const int grid = static_cast<int>(std::min<int64_t>(max_pass_ctas(), (most + 255) / 256));
  divergence_kernel<<<grid, 256, 0, st>>>(a);
  return check_launch("divergence_kernel");
}

// `count` iterations of Alg. 1 on one pair: u <- a/(K v) then v <- b/(K^T u).
int single_iterations(int mode, const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y,
                      const lsf_scalings* out, int count, const Workspace& ws, int* status,
                      cudaStream_t st) {
  for (int it = 0; it < count; ++it) {
    PassRhs ru{};
    ru.t_in = out->t_v; ru.w = x->w; ru.out = out->u; ru.t_out = out->t_u;
    LSF_TRY(run_pass(mode, th, x, kPassUpdate, 1, &ru, ws, status, st));
    PassRhs rv{};
    rv.t_in = out->t_u; rv.w = y->w; rv.out = out->v; rv.t_out = out->t_v;
    LSF_TRY(run_pass(mode, th, y, kPassUpdate, 1, &rv, ws, status, st));
  }
  return LSF_OK;
}

// The residual ||u o (K v) - a||_1 of one pair after its last v-half.
int single_residual(int mode, const lsf_theta* th, const lsf_cloud* x, const lsf_scalings* out,
                    lsf_result* result, const Workspace& ws, int* status, cudaStream_t st) {
  PassRhs rd{};
  rd.t_in = out->t_v; rd.w = x->w; rd.old = out->u; rd.res_out = &result->residual;
  return run_pass(mode, th, x, kPassDot, 1, &rd, ws, status, st);
}

// Passes over one feature matrix with the right-hand sides of the active terms
// (none: no pass).
int run_active(int mode, const lsf_theta* th, const lsf_cloud* cl, int pmode, const PassRhs* r0,
               bool a0, const PassRhs* r1, bool a1, const Workspace& ws, int* status, cudaStream_t st) {
  PassRhs r[2];
  int k = 0;
  if (a0) r[k++] = *r0;
  if (a1) r[k++] = *r1;
  if (k == 0) return LSF_OK;
  return run_pass(mode, th, cl, pmode, k, r, ws, status, st);
}

// `count` lock-step iterations of the debiased solves (Eq. (2)) whose flags act[]
// (xy, xx, yy) are set: xi pass {XY u-half, XX u-half}, zeta pass {XY v-half,
// YY u-half}, xi pass {XX v-half}, zeta pass {YY v-half}; a pass carries only the
// active terms' right-hand sides.
int debiased_iterations(int mode, const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y,
                        const lsf_scalings* s_xy, const lsf_scalings* s_xx, const lsf_scalings* s_yy,
                        const bool act[3], int count, const Workspace& ws, int* status,
                        cudaStream_t st) {
  for (int it = 0; it < count; ++it) {
    PassRhs p1a{}, p1b{};
    p1a.t_in = s_xy->t_v; p1a.w = x->w; p1a.out = s_xy->u; p1a.t_out = s_xy->t_u;
    p1b.t_in = s_xx->t_v; p1b.w = x->w; p1b.out = s_xx->u; p1b.t_out = s_xx->t_u;
    LSF_TRY(run_active(mode, th, x, kPassUpdate, &p1a, act[0], &p1b, act[1], ws, status, st));
    PassRhs p2a{}, p2b{};
    p2a.t_in = s_xy->t_u; p2a.w = y->w; p2a.out = s_xy->v; p2a.t_out = s_xy->t_v;
    p2b.t_in = s_yy->t_v; p2b.w = y->w; p2b.out = s_yy->u; p2b.t_out = s_yy->t_u;
    LSF_TRY(run_active(mode, th, y, kPassUpdate, &p2a, act[0], &p2b, act[2], ws, status, st));
    PassRhs p3{};
    p3.t_in = s_xx->t_u; p3.w = x->w; p3.out = s_xx->v; p3.t_out = s_xx->t_v;
    LSF_TRY(run_active(mode, th, x, kPassUpdate, &p3, act[1], nullptr, false, ws, status, st));
    PassRhs p4{};
    p4.t_in = s_yy->t_u; p4.w = y->w; p4.out = s_yy->v; p4.t_out = s_yy->t_v;
    LSF_TRY(run_active(mode, th, y, kPassUpdate, &p4, act[2], nullptr, false, ws, status, st));
  }
  return LSF_OK;
}

// The residuals of the active debiased terms after their last v-half.
int debiased_residuals(int mode, const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y,
                       const lsf_scalings* s_xy, const lsf_scalings* s_xx, const lsf_scalings* s_yy,
                       lsf_result* rxy, lsf_result* rxx, lsf_result* ryy, const bool act[3],
                       const Workspace& ws, int* status, cudaStream_t st) {
  PassRhs d1a{}, d1b{};
  d1a.t_in = s_xy->t_v; d1a.w = x->w; d1a.old = s_xy->u; d1a.res_out = &rxy->residual;
  d1b.t_in = s_xx->t_v; d1b.w = x->w; d1b.old = s_xx->u; d1b.res_out = &rxx->residual;
  LSF_TRY(run_active(mode, th, x, kPassDot, &d1a, act[0], &d1b, act[1], ws, status, st));
  PassRhs d2{};
  d2.t_in = s_yy->t_v; d2.w = y->w; d2.old = s_yy->u; d2.res_out = &ryy->residual;
  return run_active(mode, th, y, kPassDot, &d2, act[2], nullptr, false, ws, status, st);
}

// Host copies of `count` device result records (synchronises the stream).
int read_results(const lsf_result* dev, lsf_result* host, int count, cudaStream_t st) {
  if (cudaMemcpyAsync(host, dev, sizeof(lsf_result) * count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "reading the result records failed");
  return LSF_OK;
}

int check_stop(int max_iters, double tol, int check_every) {
  if (max_iters < 1) return fail(LSF_ERR_ARG, "max_iters must be >= 1");
  if (!(tol >= 0.0)) return fail(LSF_ERR_ARG, "tol must be >= 0");
  if (check_every < 1) return fail(LSF_ERR_ARG, "check_every must be >= 1");
  return LSF_OK;
}

}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_solve(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters, int mode,
              const lsf_scalings* out, lsf_result* result, void* workspace, size_t ws_bytes,
              void* stream) {
  lsf::TraceRange trace_range("lsf_solve");
  LSF_TRY(check_theta(theta));
  if (mode == LSF_MODE_AUTO) {
    if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
    return solve_auto(theta, x, y, result, workspace, ws_bytes, as_stream(stream), [&](int m) {
      return lsf_solve(theta, x, y, iters, m, out, result, workspace, ws_bytes, stream);
    });
  }
  LSF_TRY(check_cloud(x, mode, "x"));
  LSF_TRY(check_cloud(y, mode, "y"));
  LSF_TRY(check_scalings(out, "out"));
  if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
  cudaStream_t st = as_stream(stream);
  Workspace ws{};
  LSF_TRY(start_solve(workspace, ws_bytes, theta->ldr, result, 1, &ws, st));
  int* status = &result->status;
  if (mode == LSF_MODE_STORED && small_solver_takes(x->n, y->n, theta->ldr)) {
    const SProb p = small_problem(x, y, out, result);
    return small_solve(&p, 1, theta->ldr, iters, st);
  }

  LSF_TRY(init_side(y, ws.keys + 0, out->v, &result->log_scale, nullptr, mode, st));
  {
    PassRhs r{};
    r.old = out->v;
    r.t_out = out->t_v;
    LSF_TRY(run_pass(mode, theta, y, kPassAxpy, 1, &r, ws, status, st));
  }
  LSF_TRY(single_iterations(mode, theta, x, y, out, iters, ws, status, st));
  LSF_TRY(single_residual(mode, theta, x, out, result, ws, status, st));
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    set_iters_kernel<<<1, 32, 0, st>>>(result, nullptr, nullptr, iters, mode);
  }
  return check_launch("set_iters_kernel");
}

int lsf_solve_tol(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int max_iters,
                  double tol, int check_every, int mode, const lsf_scalings* out, lsf_result* result,
                  void* workspace, size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_solve_tol");
  LSF_TRY(check_theta(theta));
  LSF_TRY(check_stop(max_iters, tol, check_every));
  if (mode == LSF_MODE_AUTO)
    return solve_auto(theta, x, y, result, workspace, ws_bytes, as_stream(stream), [&](int m) {
      return lsf_solve_tol(theta, x, y, max_iters, tol, check_every, m, out, result, workspace,
                           ws_bytes, stream);
    });
  LSF_TRY(check_cloud(x, mode, "x"));
  LSF_TRY(check_cloud(y, mode, "y"));
  LSF_TRY(check_scalings(out, "out"));
  cudaStream_t st = as_stream(stream);
  Workspace ws{};
  LSF_TRY(start_solve(workspace, ws_bytes, theta->ldr, result, 1, &ws, st));
  int* status = &result->status;
  LSF_TRY(init_side(y, ws.keys + 0, out->v, &result->log_scale, nullptr, mode, st));
  {
    PassRhs r{};
    r.old = out->v;
    r.t_out = out->t_v;
    LSF_TRY(run_pass(mode, theta, y, kPassAxpy, 1, &r, ws, status, st));
  }
  int done = 0;
  while (done < max_iters) {
    const int chunk = std::min(check_every, max_iters - done);
    LSF_TRY(single_iterations(mode, theta, x, y, out, chunk, ws, status, st));
    done += chunk;
    LSF_TRY(single_residual(mode, theta, x, out, result, ws, status, st));
    lsf_result h{};
    LSF_TRY(read_results(result, &h, 1, st));
    if ((h.status & LSF_ERR_NONFINITE) || h.residual <= tol) break;
  }
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    set_iters_kernel<<<1, 32, 0, st>>>(result, nullptr, nullptr, done, mode);
  }
  return check_launch("set_iters_kernel");
}

int lsf_divergence(const lsf_theta* theta, int nterms, const lsf_cloud* const* xs,
                   const lsf_cloud* const* ys, const lsf_scalings* const* s,
                   lsf_result* const* result, const double* coef, double* combined, int mode,
                   void* workspace, size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_divergence");
  LSF_TRY(check_theta(theta));
  if (nterms < 1 || nterms > 3) return fail(LSF_ERR_ARG, "nterms must be 1..3");
  if (!xs || !ys || !s || !result) return fail(LSF_ERR_ARG, "lsf_divergence: NULL array");
  for (int t = 0; t < nterms; ++t) {
    if (!xs[t] || !ys[t] || !s[t] || !result[t]) return fail(LSF_ERR_ARG, "NULL term %d", t);
    if (!xs[t]->shift || !xs[t]->w || !ys[t]->shift || !ys[t]->w || !s[t]->u || !s[t]->v)
      return fail(LSF_ERR_ARG, "term %d: missing arrays", t);
    if (xs[t]->n < 1 || ys[t]->n < 1) return fail(LSF_ERR_ARG, "term %d: empty measure", t);
  }
  cudaStream_t st = as_stream(stream);
  Workspace ws{};
  LSF_TRY(carve_workspace(workspace, ws_bytes, theta->ldr, &ws));
  if (cudaMemsetAsync(ws.counters + 1, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_divergence: memset failed");
  return launch_divergence(theta, nterms, xs, ys, s, result, coef, combined, ws, st,
                           mode == LSF_MODE_LOG ? 1 : mode == LSF_MODE_AUTO ? -1 : 0);
}

int lsf_debiased(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
                 int mode, const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                 const lsf_scalings* s_yy, lsf_result* result, double* wbar, void* workspace,
                 size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_debiased");
  LSF_TRY(check_theta(theta));
  if (mode == LSF_MODE_AUTO) {
    if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
    return solve_auto(theta, x, y, result, workspace, ws_bytes, as_stream(stream), [&](int m) {
      return lsf_debiased(theta, x, y, iters, m, s_xy, s_xx, s_yy, result, wbar, workspace,
                          ws_bytes, stream);
    });
  }
  LSF_TRY(check_cloud(x, mode, "x"));
  LSF_TRY(check_cloud(y, mode, "y"));
  LSF_TRY(check_scalings(s_xy, "xy"));
  LSF_TRY(check_scalings(s_xx, "xx"));
  LSF_TRY(check_scalings(s_yy, "yy"));
  if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
  cudaStream_t st = as_stream(stream);
  Workspace ws{};
  LSF_TRY(start_solve(workspace, ws_bytes, theta->ldr, result, 3, &ws, st));
  lsf_result* rxy = result + 0;
  lsf_result* rxx = result + 1;
  lsf_result* ryy = result + 2;
  int* status = &rxy->status;
  if (mode == LSF_MODE_STORED && small_solver_takes(x->n, y->n, theta->ldr) &&
      small_solver_takes(x->n, x->n, theta->ldr) && small_solver_takes(y->n, y->n, theta->ldr)) {
    // one cluster per solve of Eq. (2), all in one launch
    const SProb p[3] = {small_problem(x, y, s_xy, rxy), small_problem(x, x, s_xx, rxx),
                        small_problem(y, y, s_yy, ryy)};
    LSF_TRY(small_solve(p, 3, theta->ldr, iters, st));
    {
      LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
      merge_status_kernel<<<1, 32, 0, st>>>(rxy, rxx, ryy);
      LSF_TRY(check_launch("merge_status_kernel"));
    }
    const lsf_cloud* xs[3] = {x, x, y};
    const lsf_cloud* ys[3] = {y, x, y};
    const lsf_scalings* ss[3] = {s_xy, s_xx, s_yy};
    lsf_result* rs[3] = {rxy, rxx, ryy};
    const double coef[3] = {1.0, -0.5, -0.5};
    return launch_divergence(theta, 3, xs, ys, ss, rs, coef, wbar, ws, st, 0);
  }

  // v = 1 for all three solves: v~ = exp(shift - max shift) on the side each v lives on.
  LSF_TRY(init_side(y, ws.keys + 0, s_xy->v, &rxy->log_scale, &ryy->log_scale, mode, st));
  if (cudaMemcpyAsync(s_yy->v, s_xy->v, sizeof(float) * y->n, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return fail(LSF_ERR_CUDA, "debiased: copy of the start vector failed");
  LSF_TRY(init_side(x, ws.keys + 1, s_xx->v, &rxx->log_scale, nullptr, mode, st));
  {
    PassRhs r[2] = {};
    r[0].old = s_xy->v; r[0].t_out = s_xy->t_v;
    r[1].old = s_yy->v; r[1].t_out = s_yy->t_v;
    LSF_TRY(run_pass(mode, theta, y, kPassAxpy, 2, r, ws, status, st));
    PassRhs q{};
    q.old = s_xx->v; q.t_out = s_xx->t_v;
    LSF_TRY(run_pass(mode, theta, x, kPassAxpy, 1, &q, ws, status, st));
  }
  const bool all[3] = {true, true, true};
  LSF_TRY(debiased_iterations(mode, theta, x, y, s_xy, s_xx, s_yy, all, iters, ws, status, st));
  LSF_TRY(debiased_residuals(mode, theta, x, y, s_xy, s_xx, s_yy, rxy, rxx, ryy, all, ws, status, st));
  {
    const lsf_cloud* xs[3] = {x, x, y};
    const lsf_cloud* ys[3] = {y, x, y};
    const lsf_scalings* ss[3] = {s_xy, s_xx, s_yy};
    lsf_result* rs[3] = {rxy, rxx, ryy};
    const double coef[3] = {1.0, -0.5, -0.5};
    LSF_TRY(launch_divergence(theta, 3, xs, ys, ss, rs, coef, wbar, ws, st,
                              mode == LSF_MODE_LOG ? 1 : 0));
  }
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    set_iters_kernel<<<1, 32, 0, st>>>(rxy, rxx, ryy, iters, mode);
  }
  // Status bits of all passes were collected in the first record; mirror them.
  if (cudaMemcpyAsync(&rxx->status, &rxy->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&ryy->status, &rxy->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return fail(LSF_ERR_CUDA, "debiased: status copy failed");
  return check_launch("set_iters_kernel");
}

int lsf_debiased_tol(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int max_iters,
                     double tol, int check_every, int mode, const lsf_scalings* s_xy,
                     const lsf_scalings* s_xx, const lsf_scalings* s_yy, lsf_result* result,
                     double* wbar, void* workspace, size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_debiased_tol");
  LSF_TRY(check_theta(theta));
  LSF_TRY(check_stop(max_iters, tol, check_every));
  if (mode == LSF_MODE_AUTO)
    return solve_auto(theta, x, y, result, workspace, ws_bytes, as_stream(stream), [&](int m) {
      return lsf_debiased_tol(theta, x, y, max_iters, tol, check_every, m, s_xy, s_xx, s_yy, result,
                              wbar, workspace, ws_bytes, stream);
    });
  LSF_TRY(check_cloud(x, mode, "x"));
  LSF_TRY(check_cloud(y, mode, "y"));
  LSF_TRY(check_scalings(s_xy, "xy"));
  LSF_TRY(check_scalings(s_xx, "xx"));
  LSF_TRY(check_scalings(s_yy, "yy"));
  cudaStream_t st = as_stream(stream);
  Workspace ws{};
  LSF_TRY(start_solve(workspace, ws_bytes, theta->ldr, result, 3, &ws, st));
  lsf_result* rxy = result + 0;
  lsf_result* rxx = result + 1;
  lsf_result* ryy = result + 2;
  int* status = &rxy->status;
  LSF_TRY(init_side(y, ws.keys + 0, s_xy->v, &rxy->log_scale, &ryy->log_scale, mode, st));
  if (cudaMemcpyAsync(s_yy->v, s_xy->v, sizeof(float) * y->n, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return fail(LSF_ERR_CUDA, "debiased: copy of the start vector failed");
  LSF_TRY(init_side(x, ws.keys + 1, s_xx->v, &rxx->log_scale, nullptr, mode, st));
  {
    PassRhs r[2] = {};
    r[0].old = s_xy->v; r[0].t_out = s_xy->t_v;
    r[1].old = s_yy->v; r[1].t_out = s_yy->t_v;
    LSF_TRY(run_pass(mode, theta, y, kPassAxpy, 2, r, ws, status, st));
    PassRhs q{};
    q.old = s_xx->v; q.t_out = s_xx->t_v;
    LSF_TRY(run_pass(mode, theta, x, kPassAxpy, 1, &q, ws, status, st));
  }
  // each term of Eq. (2) stops on its own test; the others keep their lock-step
  // passes
  bool act[3] = {true, true, true};
  int done[3] = {0, 0, 0};
  int it = 0;
  while (it < max_iters && (act[0] || act[1] || act[2])) {
    const int chunk = std::min(check_every, max_iters - it);
    LSF_TRY(debiased_iterations(mode, theta, x, y, s_xy, s_xx, s_yy, act, chunk, ws, status, st));
    it += chunk;
    LSF_TRY(debiased_residuals(mode, theta, x, y, s_xy, s_xx, s_yy, rxy, rxx, ryy, act, ws, status, st));
    lsf_result h[3];
    LSF_TRY(read_results(result, h, 3, st));
    const bool void_run = (h[0].status & LSF_ERR_NONFINITE) != 0;
    for (int t = 0; t < 3; ++t)
      if (act[t]) {
        done[t] = it;
        if (void_run || h[t].residual <= tol) act[t] = false;
      }
  }
  {
    const lsf_cloud* xs[3] = {x, x, y};
    const lsf_cloud* ys[3] = {y, x, y};
    const lsf_scalings* ss[3] = {s_xy, s_xx, s_yy};
    lsf_result* rs[3] = {rxy, rxx, ryy};
    const double coef[3] = {1.0, -0.5, -0.5};
    LSF_TRY(launch_divergence(theta, 3, xs, ys, ss, rs, coef, wbar, ws, st,
                              mode == LSF_MODE_LOG ? 1 : 0));
  }
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    set_iters_kernel<<<1, 32, 0, st>>>(rxy, nullptr, nullptr, done[0], mode);
    set_iters_kernel<<<1, 32, 0, st>>>(rxx, nullptr, nullptr, done[1], mode);
    set_iters_kernel<<<1, 32, 0, st>>>(ryy, nullptr, nullptr, done[2], mode);
  }
  if (cudaMemcpyAsync(&rxx->status, &rxy->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&ryy->status, &rxy->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return fail(LSF_ERR_CUDA, "debiased: status copy failed");
  return check_launch("set_iters_kernel");
}

}  // extern "C"
