// Accelerated Sinkhorn (App. A.2) on the factored kernel K = xi zeta^T, log domain.
//
// The appendix cites the accelerated alternating minimisation of Guminov et al.;
// its printed listing is garbled, and this follows the cited method: minimise
//   phi(eta) = log <e^eta1, K e^eta2> - <eta1, a> - <eta2, b>
// (W = -eps min phi) with an estimate sequence. One attempt at iteration k, with
// Lipschitz estimate L:
//   a_+ = 1/(2L) + sqrt(1/(4L^2) + A/L),  tau = a_+/(A + a_+),
//   lam = tau zeta + (1 - tau) eta,  g = grad phi(lam) = (P 1 - a, P^T 1 - b),
//   eta' = lam with the block of larger ||g_i|| replaced by its exact minimiser
//          (a Sinkhorn half-step),
//   accepted when phi(eta') <= phi(lam) - ||g||^2/(2L); else L doubles.
// Accepted: zeta -= a_+ g, eta = eta', A += a_+; L halves at the next iteration.
// An iteration that needs more than kMaxAttempts attempts ends the solve: the
// required decrease ||g||^2/(2L) has fallen below the rounding of phi, so eta is
// stationary to working precision (result->iters then counts the iterations
// done).
//
// The gradient needs both products K e^lam2 and K^T e^lam1. In factored log form
// (L~ = log features minus the row shift s):
//   log (xi^T e^lam1)_k   = LSE_i(L~x_ik + lam1_i + sx_i)       X pass, column side
//   log (K^T e^lam1)_j    = sy_j + LSE_k(L~y_jk + that)         Y pass, row side
//   log (zeta^T e^lam2)_k = LSE_j(L~y_jk + lam2_j + sy_j)       same Y pass, column side
//   log (K e^lam2)_i      = sx_i + LSE_k(L~x_ik + that)         X pass, row side
// so an attempt is three log-domain passes (X column, Y rows and column, X rows)
// and three small kernels: the interpolation, the log-sum-exp of the plan's mass
// c, and the gradient with the six sums the two decisions need (||g_1||^2,
// ||g_2||^2, <lam, w> and <eta', w> per block), reduced in a fixed order. At a
// point with one block exactly minimised c = 1, so phi(eta') = -<eta'1, a> -
// <eta'2, b> needs no further product. The host reads the decision once per
// attempt (the only synchronisation).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "pass.cuh"
#include "reduce.cuh"
#include "solve.cuh"

namespace lsf {
namespace {

constexpr int kAccThreads = 256;
constexpr int kAccSums = 8;  // n1, n2, l1, l2, <lam1, a>, <lam2, b>, <eta'1, a>, <eta'2, b>
constexpr int kMaxAttempts = 30;  // per iteration, before the solve stops

// One side's vectors (n entries each) in the workspace.
struct AccSide {
  int64_t n;
  const float* shift;  // row log-shifts
  const float* w;      // weights
  float* zeta;         // gradient-step sequence
  float* eta;          // block-minimised sequence
  float* lam;          // interpolated point of the current attempt
  float* f;            // lam + shift: the column input of the passes
  float* ls;           // log of the row products (the pass's row output)
  float* g;            // gradient block at lam
};

struct AccDecision {
  int accept;
  int block;      // 1 or 2
  double logc;    // log of the plan's mass at lam
  double sums[kAccSums];
  double phi_lam, phi_new;
};

__device__ __forceinline__ int64_t side_index(int64_t i, int64_t n1, bool& second) {
  second = i >= n1;
  return second ? i - n1 : i;
}

// lam = tau zeta + (1 - tau) eta and f = lam + shift, both sides in one launch.
__global__ void accel_mix_kernel(AccSide s1, AccSide s2, float tau, float omt) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < s1.n + s2.n;
       i += stride) {
    bool second;
    const int64_t j = side_index(i, s1.n, second);
    const AccSide& s = second ? s2 : s1;
    const float l = tau * s.zeta[j] + omt * s.eta[j];
    s.lam[j] = l;
    s.f[j] = l + s.shift[j];
  }
}

// Online log-sum-exp (m, s) update and merge, accurate exponentials.
__device__ __forceinline__ void lse_add(float& m, float& s, float y) {
  if (y == -INFINITY) return;
  if (y > m) {
    s = s * expf(m - y) + 1.f;
    m = y;
  } else {
    s += expf(y - m);
  }
}
__device__ __forceinline__ void lse_join(float& m, float& s, float m2, float s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) {
    m = m2;
    s = s2;
    return;
  }
  if (m2 > m) {
    s = s * expf(m - m2) + s2;
    m = m2;
  } else {
    s += s2 * expf(m2 - m);
  }
}

// Per-block (max, sum) of log c = LSE_i(lam1_i + sx_i + ls1_i): the mass of the
// plan at lam, taken on the row side.
__global__ void accel_mass_kernel(AccSide s1, float2* part) {
  __shared__ float2 s_w[kAccThreads / 32];
  float m = -INFINITY, s = 0.f;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < s1.n; i += stride)
    lse_add(m, s, s1.f[i] + s1.ls[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float m2 = __shfl_down_sync(0xffffffffu, m, o), s2 = __shfl_down_sync(0xffffffffu, s, o);
    lse_join(m, s, m2, s2);
  }
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = make_float2(m, s);
  __syncthreads();
  if (threadIdx.x == 0) {
    float M = -INFINITY, S = 0.f;
    for (int w = 0; w < kAccThreads / 32; ++w) lse_join(M, S, s_w[w].x, s_w[w].y);
    part[blockIdx.x] = make_float2(M, S);
  }
}

// log c from the per-block partials, in block order.
__device__ double merge_mass(const float2* part, int nparts) {
  float M = -INFINITY, S = 0.f;
  for (int b = 0; b < nparts; ++b) lse_join(M, S, part[b].x, part[b].y);
  return static_cast<double>(M) + log(static_cast<double>(S));
}

// g = exp(lam + shift + ls - log c) - w per side and the block's eight sums.
__global__ void accel_grad_kernel(AccSide s1, AccSide s2, const float2* mass, int nmass,
                                  double* part, AccDecision* dec) {
  __shared__ double s_logc;
  __shared__ double s_w[kAccThreads / 32][kAccSums];
  if (threadIdx.x == 0) {
    s_logc = merge_mass(mass, nmass);
    if (blockIdx.x == 0) dec->logc = s_logc;
  }
  __syncthreads();
  const float logc = static_cast<float>(s_logc);
  double acc[kAccSums];
#pragma unroll
  for (int q = 0; q < kAccSums; ++q) acc[q] = 0.0;
  // each side over its own index range with the same partition, so that two
  // sides holding the same data (the self terms of Eq. (2)) give bit-equal sums
  // and an exact tie of the block norms is decided as the oracle decides it
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const AccSide& s = o ? s2 : s1;
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < s.n; j += stride) {
      const float lk = s.shift[j] + s.ls[j];  // log of (K e^lam2)_i, or of (K^T e^lam1)_j
      const float wj = s.w[j];
      const float g = expf(s.lam[j] + lk - logc) - wj;
      s.g[j] = g;
      const double gd = g, wd = wj;
      acc[0 + o] += gd * gd;
      acc[2 + o] += fabs(gd);
      acc[4 + o] += static_cast<double>(s.lam[j]) * wd;
      acc[6 + o] += (static_cast<double>(logf(wj)) - static_cast<double>(lk)) * wd;
    }
  }
#pragma unroll
  for (int q = 0; q < kAccSums; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < kAccSums) {
    double v = 0.0;
    for (int w = 0; w < kAccThreads / 32; ++w) v += s_w[w][threadIdx.x];
    part[static_cast<size_t>(blockIdx.x) * kAccSums + threadIdx.x] = v;
  }
}

// The two decisions of an attempt (block, acceptance) from the sums, in block
// order; with `final` set, the residual ||P 1 - a||_1 + ||P^T 1 - b||_1 instead.
__global__ void accel_decide_kernel(const double* part, int nparts, double L, AccDecision* dec,
                                    lsf_result* result, int final_iters) {
  if (threadIdx.x != 0) return;
  double S[kAccSums];
  for (int q = 0; q < kAccSums; ++q) S[q] = 0.0;
  for (int b = 0; b < nparts; ++b)
    for (int q = 0; q < kAccSums; ++q) S[q] += part[static_cast<size_t>(b) * kAccSums + q];
  for (int q = 0; q < kAccSums; ++q) dec->sums[q] = S[q];
  const double phi_lam = dec->logc - S[4] - S[5];
  const int block = S[0] >= S[1] ? 1 : 2;
  // the fitted block's plan marginal is its weight vector, so the mass is 1
  const double phi_new = block == 1 ? -S[6] - S[5] : -S[4] - S[7];
  dec->phi_lam = phi_lam;
  dec->phi_new = phi_new;
  dec->block = block;
  dec->accept = phi_new <= phi_lam - (S[0] + S[1]) / (2.0 * L) ? 1 : 0;
  if (!isfinite(phi_lam) || !isfinite(phi_new)) atomicOr(&result->status, LSF_ERR_NONFINITE);
  if (final_iters > 0) {
    result->residual = S[2] + S[3];
    result->iters = final_iters;
    result->mode = LSF_MODE_LOG;
  }
}

// An accepted attempt: zeta -= a_+ g; eta = lam with the chosen block refitted.
__global__ void accel_step_kernel(AccSide s1, AccSide s2, float an, const AccDecision* dec) {
  const int block = dec->block;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < s1.n + s2.n;
       i += stride) {
    bool second;
    const int64_t j = side_index(i, s1.n, second);
    const AccSide& s = second ? s2 : s1;
    s.zeta[j] -= an * s.g[j];
    const bool fit = block == (second ? 2 : 1);
    s.eta[j] = fit ? logf(s.w[j]) - (s.shift[j] + s.ls[j]) : s.lam[j];
  }
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

int vec_grid(int64_t n) {
  return static_cast<int>(std::max<int64_t>(
      1, std::min<int64_t>(2LL * device_info().sms, (n + kAccThreads - 1) / kAccThreads)));
}

size_t accel_extra_bytes(int64_t n, int64_t m, int ldr) {
  size_t b = 0;
  b += 6 * align256(sizeof(float) * static_cast<size_t>(n));
  b += 6 * align256(sizeof(float) * static_cast<size_t>(m));
  b += 2 * align256(sizeof(float) * static_cast<size_t>(ldr));  // log r-vectors of an attempt
  const int grid = 2 * device_info().sms;
  b += align256(sizeof(float2) * grid);
  b += align256(sizeof(double) * grid * kAccSums);
  b += align256(sizeof(AccDecision));
  return b;
}

// The gradient machinery at lam = tau zeta + (1 - tau) eta (tau = 0: at eta):
// interpolation, three passes, mass, gradient and decision.
int accel_evaluate(const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y, AccSide s1, AccSide s2,
                   float tau, float* lt_x, float* lt_y, float2* mpart, double* spart, AccDecision* dec,
                   double L, lsf_result* result, int final_iters, const Workspace& ws,
                   cudaStream_t st) {
  const int gv = vec_grid(s1.n + s2.n);
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 16.0 * (s1.n + s2.n));
    accel_mix_kernel<<<gv, kAccThreads, 0, st>>>(s1, s2, tau, 1.f - tau);
  }
  LSF_TRY(check_launch("accel_mix_kernel"));
  int* status = &result->status;
  PassRhs p1{};  // X: log (xi^T e^lam1)
  p1.old = s1.f;
  p1.t_out = lt_x;
  LSF_TRY(run_pass(LSF_MODE_LOG, th, x, kPassAxpy, 1, &p1, ws, status, st));
  PassRhs p2{};  // Y: log (K^T e^lam1) rows and log (zeta^T e^lam2) columns
  p2.t_in = lt_x;
  p2.old = s2.f;
  p2.out = s2.ls;
  p2.t_out = lt_y;
  LSF_TRY(run_pass(LSF_MODE_LOG, th, y, kPassRowsAxpy, 1, &p2, ws, status, st));
  PassRhs p3{};  // X: log (K e^lam2) rows
  p3.t_in = lt_y;
  p3.out = s1.ls;
  LSF_TRY(run_pass(LSF_MODE_LOG, th, x, kPassRows, 1, &p3, ws, status, st));
  const int gm = vec_grid(s1.n);
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 20.0 * (s1.n + s2.n) + 8.0 * s1.n);
    accel_mass_kernel<<<gm, kAccThreads, 0, st>>>(s1, mpart);
    accel_grad_kernel<<<gv, kAccThreads, 0, st>>>(s1, s2, mpart, gm, spart, dec);
    accel_decide_kernel<<<1, 32, 0, st>>>(spart, gv, L, dec, result, final_iters);
  }
  return check_launch("accel_decide_kernel");
}

}  // namespace

size_t accel_workspace_bytes(int64_t n, int64_t m, int ldr) {
  return align256(workspace_bytes(ldr)) + accel_extra_bytes(n, m, ldr);
}

int accel_solve(const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y, int iters, double L0,
                const lsf_scalings* out, lsf_result* result, lsf_accel_info* info, void* workspace,
                size_t ws_bytes, cudaStream_t st) {
  LSF_TRY(check_theta(th));
  LSF_TRY(check_cloud(x, LSF_MODE_LOG, "x"));
  LSF_TRY(check_cloud(y, LSF_MODE_LOG, "y"));
  LSF_TRY(check_scalings(out, "out"));
  if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
  if (!(L0 > 0.0) || !std::isfinite(L0)) return fail(LSF_ERR_ARG, "L0 must be positive and finite");
  const size_t need = accel_workspace_bytes(x->n, y->n, th->ldr);
  if (ws_bytes < need)
    return fail(LSF_ERR_WORKSPACE, "accelerated solve: workspace has %zu bytes, needs %zu", ws_bytes, need);
  Workspace ws{};
  LSF_TRY(start_solve(workspace, ws_bytes, th->ldr, result, 1, &ws, st));
  // the vectors follow the pass workspace
  char* p = static_cast<char*>(workspace) + align256(workspace_bytes(th->ldr));
  auto take = [&](size_t bytes) {
    char* q = p;
    p += align256(bytes);
    return q;
  };
  AccSide s1{}, s2{};
  for (int side = 0; side < 2; ++side) {
    AccSide& s = side ? s2 : s1;
    const lsf_cloud* c = side ? y : x;
    s.n = c->n;
    s.shift = c->shift;
    s.w = c->w;
    float** v[6] = {&s.zeta, &s.eta, &s.lam, &s.f, &s.ls, &s.g};
    for (float** q : v) *q = reinterpret_cast<float*>(take(sizeof(float) * static_cast<size_t>(c->n)));
  }
  float* lt_x = reinterpret_cast<float*>(take(sizeof(float) * th->ldr));
  float* lt_y = reinterpret_cast<float*>(take(sizeof(float) * th->ldr));
  const int grid = 2 * device_info().sms;
  float2* mpart = reinterpret_cast<float2*>(take(sizeof(float2) * grid));
  double* spart = reinterpret_cast<double*>(take(sizeof(double) * grid * kAccSums));
  AccDecision* dec = reinterpret_cast<AccDecision*>(take(sizeof(AccDecision)));
  // eta = zeta = 0
  for (const AccSide* s : {&s1, &s2}) {
    if (cudaMemsetAsync(s->zeta, 0, sizeof(float) * s->n, st) != cudaSuccess ||
        cudaMemsetAsync(s->eta, 0, sizeof(float) * s->n, st) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "accelerated solve: memset failed");
  }

  double A = 0.0, L = L0;
  int attempts = 0, done = 0;
  for (int k = 0; k < iters; ++k) {
    const double L_prev = L;
    L /= 2.0;
    double an = 0.0;
    bool accepted = false;
    for (int tries = 0; tries < kMaxAttempts; ++tries) {
      ++attempts;
      an = 1.0 / (2.0 * L) + std::sqrt(1.0 / (4.0 * L * L) + A / L);
      const float tau = static_cast<float>(an / (A + an));
      LSF_TRY(accel_evaluate(th, x, y, s1, s2, tau, lt_x, lt_y, mpart, spart, dec, L, result, 0, ws, st));
      AccDecision h{};
      if (cudaMemcpyAsync(&h, dec, sizeof(AccDecision), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail(LSF_ERR_CUDA, "accelerated solve: reading the decision failed");
      if (!std::isfinite(h.phi_lam) || !std::isfinite(h.phi_new))
        return fail(LSF_ERR_NONFINITE, "accelerated solve: non-finite dual value at iteration %d", k);
      if (h.accept) {
        accepted = true;
        break;
      }
      L *= 2.0;
    }
    if (!accepted) {  // stationary to working precision
      L = L_prev;
      break;
    }
    {
      LaunchScope ls(st, LSF_KERNEL_OTHER, 24.0 * (s1.n + s2.n));
      accel_step_kernel<<<vec_grid(s1.n + s2.n), kAccThreads, 0, st>>>(s1, s2, static_cast<float>(an), dec);
    }
    LSF_TRY(check_launch("accel_step_kernel"));
    A += an;
    done = k + 1;
  }
  // the final point: log u~ = eta1 + shift and log v~ = eta2 + shift (the log-mode
  // scalings), its r-vectors and its residual
  AccSide f1 = s1, f2 = s2;
  f1.f = out->u;
  f2.f = out->v;
  LSF_TRY(accel_evaluate(th, x, y, f1, f2, 0.f, out->t_u, out->t_v, mpart, spart, dec, L, result,
                         std::max(done, 1), ws, st));
  if (done == 0) {  // no iteration accepted: report 0 iterations
    if (cudaMemsetAsync(&result->iters, 0, sizeof(int32_t), st) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "accelerated solve: memset failed");
  }
  if (info) {
    info->iters = done;
    info->attempts = attempts;
    info->A = A;
    info->L = L;
  }
  return LSF_OK;
}

}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_accel_workspace_bytes(int64_t n, int64_t m, int ldr, size_t* bytes) {
  if (!bytes) return fail(LSF_ERR_ARG, "bytes is NULL");
  if (n < 1 || m < 1) return fail(LSF_ERR_ARG, "n and m must be >= 1");
  if (ldr < 4 || ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "ldr must be a multiple of 4 in [4, 1024]");
  *bytes = accel_workspace_bytes(n, m, ldr);
  return LSF_OK;
}

int lsf_solve_accelerated(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y, int iters,
                          double L0, const lsf_scalings* out, lsf_result* result, lsf_accel_info* info,
                          void* workspace, size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_solve_accelerated");
  return accel_solve(theta, x, y, iters, L0, out, result, info, workspace, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"
