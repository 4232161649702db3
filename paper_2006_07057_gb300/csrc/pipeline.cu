// The whole hot path in one call, from host inputs to host results:
// radius and Lemma 1 parameters on the device (no host round trip), anchors,
// features of the chosen mode, Alg. 1 on K = xi zeta^T (Sec. 3.1) for each term,
// Eq. (6) and Eq. (2). Every device buffer is carved from one caller arena, so a
// call allocates nothing and, except in the automatic mode, never waits on the
// device: the host inputs are copied in and the results copied out on the
// stream, and the caller synchronises when it wants the numbers.
#include <cuda_runtime.h>

#include <algorithm>

#include "recompute.cuh"
#include "solve.cuh"

namespace lsf {
namespace {

size_t al256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// The device record a run fills and copies to the host.
__global__ void pipeline_out_kernel(const lsf_result* res, int nres, const double* wbar,
                                    const float* R, const double* qs, lsf_pipeline_out* out) {
  if (threadIdx.x != 0) return;
  lsf_pipeline_out o{};
  o.W = nres == 3 ? *wbar : res[0].W;
  o.W_xy = res[0].W;
  o.residual_xy = res[0].residual;
  o.status = res[0].status;
  o.mode = res[0].mode;
  if (nres == 3) {
    o.W_xx = res[1].W;
    o.W_yy = res[2].W;
    o.residual_xx = res[1].residual;
    o.residual_yy = res[2].residual;
    o.status |= res[1].status | res[2].status;
  }
  o.R = static_cast<double>(R[0]);
  o.q = qs[0];
  o.sigma = qs[1];
  o.iters = res[0].iters;
  *out = o;
}

// The record of a problem whose three terms were solved elsewhere (a batched
// solve on the arena's buffers): Eq. (2) from the three Eq. (6) values.
__global__ void finish_out_kernel(const lsf_result* res, int nres, const float* R, const double* qs,
                                  lsf_pipeline_out* out) {
  if (threadIdx.x != 0) return;
  lsf_pipeline_out o{};
  o.W_xy = res[0].W;
  o.residual_xy = res[0].residual;
  o.status = res[0].status;
  o.mode = res[0].mode;
  o.W = res[0].W;
  if (nres == 3) {
    o.W_xx = res[1].W;
    o.W_yy = res[2].W;
    o.residual_xx = res[1].residual;
    o.residual_yy = res[2].residual;
    o.status |= res[1].status | res[2].status;
    o.W = res[0].W - 0.5 * (res[1].W + res[2].W);
  }
  o.R = static_cast<double>(R[0]);
  o.q = qs[0];
  o.sigma = qs[1];
  o.iters = res[0].iters;
  *out = o;
}

// Offsets of every buffer in the arena (bytes, each 256-aligned).
struct Layout {
  size_t X, Y, a, b, Z, U, c, R, qs, Fx, Fy, sx, sy, s[3][4], res, wbar, out, ws, total;
  int ldr, ldf;
};

int layout(const lsf_pipeline* p, Layout* L) {
  if (!p) return fail(LSF_ERR_ARG, "pipeline: NULL description");
  if (p->n < 1 || p->m < 1) return fail(LSF_ERR_ARG, "pipeline: need n, m >= 1");
  if (p->d < 1 || p->r < 1) return fail(LSF_ERR_ARG, "pipeline: need d, r >= 1");
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(LSF_ERR_ARG, "pipeline: eps must be > 0");
  if (p->iters < 0) return fail(LSF_ERR_ARG, "pipeline: iters must be >= 0");
  if (p->iters == 0 && p->mode != LSF_MODE_STORED && p->mode != LSF_MODE_LOG)
    return fail(LSF_ERR_ARG, "pipeline: preparing (iters = 0) takes the stored or log mode");
  const int ldr = p->ldr ? p->ldr : (p->r + 3) / 4 * 4;
  if (ldr < p->r || ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "pipeline: ldr must be a multiple of 4 in [r, 1024]");
  int ldf = 0;
  switch (p->mode) {
    case LSF_MODE_STORED:
    case LSF_MODE_LOG:
    case LSF_MODE_AUTO: ldf = ldr; break;
    case LSF_MODE_RECOMPUTE: ldf = 0; break;
    case LSF_MODE_HYBRID:
      if (ldr < 8) return fail(LSF_ERR_UNSUPPORTED, "pipeline: the hybrid mode needs ldr >= 8");
      ldf = ldr - hybrid_first_stored(ldr);
      break;
    default: return fail(LSF_ERR_ARG, "pipeline: unknown mode %d", p->mode);
  }
  size_t ws = 0;
  LSF_TRY(lsf_workspace_bytes(ldr, &ws));
  const size_t n = static_cast<size_t>(p->n), m = static_cast<size_t>(p->m);
  const size_t d = static_cast<size_t>(p->d), r = static_cast<size_t>(p->r);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += al256(std::max<size_t>(bytes, 1));
    return o;
  };
  L->X = take(4 * n * d);
  L->Y = take(4 * m * d);
  L->a = take(4 * n);
  L->b = take(4 * m);
  L->Z = take(4 * r * d);
  L->U = take(4 * r * d);
  L->c = take(4 * static_cast<size_t>(ldr));
  L->R = take(4);
  L->qs = take(16);
  L->Fx = take(4 * n * ldf);
  L->Fy = take(4 * m * ldf);
  L->sx = take(4 * n);
  L->sy = take(4 * m);
  const size_t rows[3][2] = {{n, m}, {n, n}, {m, m}};
  const int nterms = p->debiased ? 3 : 1;
  for (int t = 0; t < 3; ++t) {
    const bool used = t < nterms;
    L->s[t][0] = used ? take(4 * rows[t][0]) : 0;
    L->s[t][1] = used ? take(4 * rows[t][1]) : 0;
    L->s[t][2] = used ? take(4 * static_cast<size_t>(ldr)) : 0;
    L->s[t][3] = used ? take(4 * static_cast<size_t>(ldr)) : 0;
  }
  L->res = take(sizeof(lsf_result) * 3);
  L->wbar = take(sizeof(double));
  L->out = take(sizeof(lsf_pipeline_out));
  L->ws = take(ws);
  L->total = off;
  L->ldr = ldr;
  L->ldf = ldf;
  return LSF_OK;
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_pipeline_bytes(const lsf_pipeline* p, size_t* bytes) {
  if (!bytes) return fail(LSF_ERR_ARG, "lsf_pipeline_bytes: NULL output");
  Layout L{};
  LSF_TRY(layout(p, &L));
  *bytes = L.total;
  return LSF_OK;
}

int lsf_pipeline_run(const lsf_pipeline* p, const float* X, const float* Y, const float* a,
                     const float* b, const float* Z, void* arena, size_t arena_bytes,
                     lsf_pipeline_out* out, void* stream) {
  lsf::TraceRange trace_range("lsf_pipeline_run");
  Layout L{};
  LSF_TRY(layout(p, &L));
  if (!X || !Y || !a || !b || !Z || (!out && p->iters > 0))
    return fail(LSF_ERR_ARG, "lsf_pipeline_run: NULL argument");
  if (!arena || reinterpret_cast<uintptr_t>(arena) % 256 != 0)
    return fail(LSF_ERR_ARG, "lsf_pipeline_run: the arena must be 256-byte aligned");
  if (arena_bytes < L.total)
    return fail(LSF_ERR_WORKSPACE, "lsf_pipeline_run: arena has %zu bytes, needs %zu", arena_bytes, L.total);
  cudaStream_t st = as_stream(stream);
  char* base = static_cast<char*>(arena);
  auto F = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
  const size_t n = static_cast<size_t>(p->n), m = static_cast<size_t>(p->m);
  const size_t d = static_cast<size_t>(p->d), r = static_cast<size_t>(p->r);
  // inputs in
  const struct { size_t off; const float* src; size_t bytes; } in[5] = {
      {L.X, X, 4 * n * d}, {L.Y, Y, 4 * m * d}, {L.a, a, 4 * n}, {L.b, b, 4 * m}, {L.Z, Z, 4 * r * d}};
  for (const auto& c : in)
    if (cudaMemcpyAsync(base + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "lsf_pipeline_run: input copy failed");
  // Lemma 1 on the device: R, then q and sigma, then the anchors
  float* dR = F(L.R);
  double* qs = reinterpret_cast<double*>(base + L.qs);
  LSF_TRY(lsf_radius(F(L.X), p->n, F(L.Y), p->m, p->d, dR, stream));
  LSF_TRY(launch_params_device(dR, p->eps, p->d, qs, st));
  if (cudaMemsetAsync(F(L.c), 0, 4 * static_cast<size_t>(L.ldr), st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_pipeline_run: memset failed");
  LSF_TRY(launch_anchors_device(F(L.Z), p->r, p->d, qs, p->eps, F(L.U), F(L.c), st));
  lsf_theta th{F(L.U), F(L.c), p->r, L.ldr, p->d, p->eps};
  // features of the mode (the automatic mode builds its own inside the solve)
  lsf_cloud cx{F(L.X), L.ldf ? F(L.Fx) : nullptr, F(L.sx), F(L.a), p->n};
  lsf_cloud cy{F(L.Y), L.ldf ? F(L.Fy) : nullptr, F(L.sy), F(L.b), p->m};
  for (lsf_cloud* c : {&cx, &cy}) {
    float* Fc = const_cast<float*>(c->F);
    float* sh = const_cast<float*>(c->shift);
    switch (p->mode) {
      case LSF_MODE_STORED: LSF_TRY(lsf_features(c->X, c->n, &th, Fc, sh, nullptr, stream)); break;
      case LSF_MODE_LOG: LSF_TRY(lsf_log_features(c->X, c->n, &th, Fc, sh, nullptr, stream)); break;
      case LSF_MODE_RECOMPUTE: LSF_TRY(lsf_row_shift(c->X, c->n, &th, sh, nullptr, stream)); break;
      case LSF_MODE_HYBRID: LSF_TRY(lsf_hybrid_features(c->X, c->n, &th, Fc, sh, nullptr, stream)); break;
      default: break;
    }
  }
  if (p->iters == 0) return LSF_OK;  // prepared: a batched solve takes it from here
  lsf_scalings s[3];
  for (int t = 0; t < 3; ++t)
    s[t] = lsf_scalings{F(L.s[t][0]), F(L.s[t][1]), F(L.s[t][2]), F(L.s[t][3])};
  lsf_result* res = reinterpret_cast<lsf_result*>(base + L.res);
  double* wbar = reinterpret_cast<double*>(base + L.wbar);
  void* ws = base + L.ws;
  const size_t ws_bytes = L.total - L.ws;
  if (p->debiased) {
    LSF_TRY(lsf_debiased(&th, &cx, &cy, p->iters, p->mode, &s[0], &s[1], &s[2], res, wbar, ws,
                         ws_bytes, stream));
  } else {
    LSF_TRY(lsf_solve(&th, &cx, &cy, p->iters, p->mode, &s[0], res, ws, ws_bytes, stream));
    const lsf_cloud* xs[1] = {&cx};
    const lsf_cloud* ys[1] = {&cy};
    const lsf_scalings* ss[1] = {&s[0]};
    lsf_result* rs[1] = {res};
    const double one = 1.0;
    LSF_TRY(lsf_divergence(&th, 1, xs, ys, ss, rs, &one, wbar, LSF_MODE_AUTO, ws, ws_bytes, stream));
  }
  lsf_pipeline_out* dout = reinterpret_cast<lsf_pipeline_out*>(base + L.out);
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    pipeline_out_kernel<<<1, 32, 0, st>>>(res, p->debiased ? 3 : 1, wbar, dR, qs, dout);
    LSF_TRY(check_launch("pipeline_out_kernel"));
  }
  if (cudaMemcpyAsync(out, dout, sizeof(lsf_pipeline_out), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_pipeline_run: result copy failed");
  return LSF_OK;
}

int lsf_pipeline_layout(const lsf_pipeline* p, void* arena, lsf_pipeline_views* v) {
  Layout L{};
  LSF_TRY(layout(p, &L));
  if (!arena || !v) return fail(LSF_ERR_ARG, "lsf_pipeline_layout: NULL argument");
  char* base = static_cast<char*>(arena);
  auto F = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
  v->theta = lsf_theta{F(L.U), F(L.c), p->r, L.ldr, p->d, p->eps};
  v->x = lsf_cloud{F(L.X), L.ldf ? F(L.Fx) : nullptr, F(L.sx), F(L.a), p->n};
  v->y = lsf_cloud{F(L.Y), L.ldf ? F(L.Fy) : nullptr, F(L.sy), F(L.b), p->m};
  for (int t = 0; t < 3; ++t)
    v->s[t] = lsf_scalings{F(L.s[t][0]), F(L.s[t][1]), F(L.s[t][2]), F(L.s[t][3])};
  v->result = reinterpret_cast<lsf_result*>(base + L.res);
  return LSF_OK;
}

int lsf_pipeline_finish(const lsf_pipeline* p, void* arena, lsf_pipeline_out* out, void* stream) {
  lsf::TraceRange trace_range("lsf_pipeline_finish");
  Layout L{};
  LSF_TRY(layout(p, &L));
  if (!arena || !out) return fail(LSF_ERR_ARG, "lsf_pipeline_finish: NULL argument");
  cudaStream_t st = as_stream(stream);
  char* base = static_cast<char*>(arena);
  lsf_pipeline_out* dout = reinterpret_cast<lsf_pipeline_out*>(base + L.out);
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    finish_out_kernel<<<1, 32, 0, st>>>(reinterpret_cast<const lsf_result*>(base + L.res),
                                        p->debiased ? 3 : 1, reinterpret_cast<const float*>(base + L.R),
                                        reinterpret_cast<const double*>(base + L.qs), dout);
    LSF_TRY(check_launch("finish_out_kernel"));
  }
  if (cudaMemcpyAsync(out, dout, sizeof(lsf_pipeline_out), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_pipeline_finish: result copy failed");
  return LSF_OK;
}

}  // extern "C"
