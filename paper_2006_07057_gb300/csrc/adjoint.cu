// Envelope gradient of W and of the debiased W_bar (Prop. 3.3 and the
// formula after it, Sec. 3.3) with theta held fixed.
//
// dW/dK = -eps u v^T at the optimum. Through K = xi zeta^T and
// d xi_ik / d x_i = xi_ik (-4/eps)(x_i - u_k), for one cloud:
//   grad x_i = 4 sum_k A_ik (x_i - u_k) = 4 (x_i rs_i - (A U)_i),
//   A_ik = F_ik sum_p coef_p alpha^p_i T^p_k,   rs_i = sum_k A_ik,
// in the shifted variables (F = xi~, alpha = u~ or v~, T = t_u or t_v; the
// row shifts and the global factor M cancel in every product alpha_i F_ik T_k).
// Terms p for the X cloud: W(a,b): (u~_xy, t_v_xy) with coef 1; debiased adds
// W(a,a) (kernel xi xi^T): (u~_xx, t_v_xx) and (v~_xx, t_u_xx) with coef -1/2.
// The Y cloud is symmetric. Weights: grad a = eps log u (Eq. 5, alpha* = eps log u*).
// In the log domain (LOGD) F, alpha and T hold logs and each term is formed as
// exp(L~_ik + f_i + lt_k), a coupling mass that stays in range.
#include <cuda_runtime.h>

#include "common.cuh"

namespace lsf {
namespace {

constexpr int kMaxTerms = 3;
constexpr int kRowsDMax = 32;  // warp-per-row kernel handles d <= 32

struct AdjArgs {
  const float* X;      // n x d
  const float* F;      // n x ldr
  const float* U;      // r x d
  int64_t n;
  int r, ldr, d;
  int nterms;
  const float* alpha[kMaxTerms];  // n
  const float* T[kMaxTerms];      // ldr
  float coef[kMaxTerms];
  float* gX;                      // n x d
};

// Warp-per-row: lane l owns columns 4l + 128j; U^T (d x ldr) and the T vectors
// sit in shared memory; the d + 1 row sums are butterfly reductions.
template <int C, bool LOGD>
__global__ void __launch_bounds__(256) adjoint_rows_kernel(const AdjArgs a) {
  extern __shared__ __align__(16) float sm[];
  float* sUT = sm;                                        // [d][ldr]
  float* sT = sm + static_cast<size_t>(a.d) * a.ldr;      // [nterms][ldr]
  const int ldr = a.ldr, d = a.d;
  for (int idx = threadIdx.x; idx < d * ldr; idx += blockDim.x) {
    const int dd = idx / ldr, k = idx - dd * ldr;
    sUT[idx] = (k < a.r) ? a.U[static_cast<int64_t>(k) * d + dd] : 0.f;
  }
  for (int idx = threadIdx.x; idx < a.nterms * ldr; idx += blockDim.x) {
    const int p = idx / ldr, k = idx - p * ldr;
    sT[idx] = a.T[p][k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < a.n;
       i += warps) {
    float al[kMaxTerms];
#pragma unroll
    for (int p = 0; p < kMaxTerms; ++p)
      al[p] = (p < a.nterms) ? (LOGD ? a.alpha[p][i] : a.coef[p] * a.alpha[p][i]) : 0.f;
    float rs = 0.f;
    float g[kRowsDMax];
#pragma unroll
    for (int dd = 0; dd < kRowsDMax; ++dd) g[dd] = 0.f;
    const float* Fi = a.F + i * ldr;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int col = 4 * lane + 128 * j;
      if (col >= ldr) continue;
      const float4 f = *reinterpret_cast<const float4*>(Fi + col);
      float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
      if (LOGD) {
#pragma unroll
        for (int p = 0; p < kMaxTerms; ++p) {
          if (p < a.nterms) {
            const float4 t = *reinterpret_cast<const float4*>(sT + static_cast<size_t>(p) * ldr + col);
            const float c = a.coef[p];
            A.x = fmaf(c, ex2_approx((f.x + al[p] + t.x) * kLog2e), A.x);
            A.y = fmaf(c, ex2_approx((f.y + al[p] + t.y) * kLog2e), A.y);
            A.z = fmaf(c, ex2_approx((f.z + al[p] + t.z) * kLog2e), A.z);
            A.w = fmaf(c, ex2_approx((f.w + al[p] + t.w) * kLog2e), A.w);
          }
        }
      } else {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < kMaxTerms; ++p) {
          if (p < a.nterms) {
            const float4 t = *reinterpret_cast<const float4*>(sT + static_cast<size_t>(p) * ldr + col);
            w.x = fmaf(al[p], t.x, w.x); w.y = fmaf(al[p], t.y, w.y);
            w.z = fmaf(al[p], t.z, w.z); w.w = fmaf(al[p], t.w, w.w);
          }
        }
        A = make_float4(f.x * w.x, f.y * w.y, f.z * w.z, f.w * w.w);
      }
      rs += (A.x + A.y) + (A.z + A.w);
#pragma unroll
      for (int dd = 0; dd < kRowsDMax; ++dd) {
        if (dd < d) {
          const float4 u = *reinterpret_cast<const float4*>(sUT + static_cast<size_t>(dd) * ldr + col);
          g[dd] = fmaf(A.x, u.x, fmaf(A.y, u.y, fmaf(A.z, u.z, fmaf(A.w, u.w, g[dd]))));
        }
      }
    }
    rs = warp_sum(rs);
    const float* xi = a.X + i * d;
#pragma unroll
    for (int dd = 0; dd < kRowsDMax; ++dd) {
      if (dd < d) {
        const float gs = warp_sum(g[dd]);
        if (lane == dd) a.gX[i * d + dd] = 4.f * (xi[dd] * rs - gs);
      }
    }
  }
}

// Register-tiled FP32 contraction for larger d: block 64 rows x 128 columns of
// the n x d result, k-tiles of 32 features. A_ik is formed while staging F.
constexpr int kBM = 64, kBN = 128, kBK = 32;

template <bool LOGD>
__global__ void __launch_bounds__(256) adjoint_gemm_kernel(const AdjArgs a) {
  __shared__ __align__(16) float As[kBK][kBM + 4];
  __shared__ __align__(16) float Bs[kBK][kBN];
  __shared__ float sAl[kMaxTerms][kBM];
  __shared__ float sRs[kBM];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
  const int n0 = blockIdx.y * kBN;
  const int ldr = a.ldr, d = a.d;
  for (int idx = tid; idx < kMaxTerms * kBM; idx += blockDim.x) {
    const int p = idx / kBM, rr = idx - p * kBM;
    const int64_t i = m0 + rr;
    sAl[p][rr] = (p < a.nterms && i < a.n) ? (LOGD ? a.alpha[p][i] : a.coef[p] * a.alpha[p][i]) : 0.f;
  }
  __syncthreads();
  // loader roles: A tile: row lr = tid / 4, k-offset lk = (tid % 4) * 8 (8 values)
  const int lr = tid >> 2, lk = (tid & 3) * 8;
  const int64_t arow = m0 + lr;
  float rs_part = 0.f;
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < ldr; k0 += kBK) {
    // stage A = F * (sum_p al_p T_p), transposed into As[k][row]
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + lk + q;
      float v = 0.f;
      if (arow < a.n && k < ldr) {
        const float fv = __ldg(a.F + arow * ldr + k);
        if (LOGD) {
#pragma unroll
          for (int p = 0; p < kMaxTerms; ++p)
            if (p < a.nterms)
              v = fmaf(a.coef[p], ex2_approx((fv + sAl[p][lr] + __ldg(a.T[p] + k)) * kLog2e), v);
        } else {
          float w = 0.f;
#pragma unroll
          for (int p = 0; p < kMaxTerms; ++p)
            if (p < a.nterms) w = fmaf(sAl[p][lr], __ldg(a.T[p] + k), w);
          v = fv * w;
        }
      }
      As[lk + q][lr] = v;
      rs_part += v;
    }
    // stage B = U[k0:k0+32, n0:n0+128]
    for (int idx = tid; idx < kBK * kBN; idx += blockDim.x) {
      const int kk = idx / kBN, c = idx - kk * kBN;
      const int k = k0 + kk, col = n0 + c;
      Bs[kk][c] = (k < a.r && col < d) ? __ldg(a.U + static_cast<int64_t>(k) * d + col) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
      const float am[4] = {av.x, av.y, av.z, av.w};
      const float bm[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(am[i], bm[j], acc[i][j]);
    }
    __syncthreads();
  }
  // row sums: the 4 loader threads of a row are adjacent lanes
  rs_part += __shfl_xor_sync(0xffffffffu, rs_part, 1);
  rs_part += __shfl_xor_sync(0xffffffffu, rs_part, 2);
  if ((tid & 3) == 0) sRs[lr] = rs_part;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = ty * 4 + i;
    const int64_t row = m0 + rr;
    if (row >= a.n) continue;
    const float rs = sRs[rr];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + tx * 8 + j;
      if (col < d) a.gX[row * d + col] = 4.f * (a.X[row * d + col] * rs - acc[i][j]);
    }
  }
}

// grad w_i = eps * sum_p coef_p (log s^p_i - shift_i - sign_p M_p)
struct WeightArgs {
  const float* s[kMaxTerms];
  const lsf_result* res[kMaxTerms];
  double sign[kMaxTerms];
  double coef[kMaxTerms];
  int nterms;
  const float* shift;
  int64_t n;
  double eps;
  float* g;
  int is_log;  // the scalings hold logs
};

__global__ void weight_grad_kernel(const WeightArgs a) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < a.n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double v = 0.0;
    for (int p = 0; p < a.nterms; ++p) {
      const double M = a.res[p]->log_scale;
      const double ls = a.is_log ? static_cast<double>(a.s[p][i]) : static_cast<double>(logf(a.s[p][i]));
      v += a.coef[p] * (ls - a.shift[i] - a.sign[p] * M);
    }
    a.g[i] = static_cast<float>(a.eps * v);
  }
}

template <bool LOGD>
int launch_points(const AdjArgs& a, cudaStream_t st) {
  if (a.d <= kRowsDMax) {
    const int C = (a.ldr + 127) / 128;
    const size_t smem = sizeof(float) * (static_cast<size_t>(a.d) + a.nterms) * a.ldr;
    int64_t grid = (a.n + 7) / 8;
    const int64_t cap = static_cast<int64_t>(device_info().sms) * 8;
    if (grid > cap) grid = cap;
    LaunchScope ls(st, LSF_KERNEL_OTHER, 4.0 * a.n * (a.ldr + 2 * a.d + a.nterms));
#define LSF_ADJ_CASE(CC)                                                                    \
  case CC: {                                                                                \
    cudaFuncSetAttribute(adjoint_rows_kernel<CC, LOGD>,                                     \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    adjoint_rows_kernel<CC, LOGD><<<(unsigned)grid, 256, smem, st>>>(a);                    \
  } break;
    switch (C <= 1 ? 1 : C <= 2 ? 2 : C <= 4 ? 4 : 8) {
      LSF_ADJ_CASE(1)
      LSF_ADJ_CASE(2)
      LSF_ADJ_CASE(4)
      LSF_ADJ_CASE(8)
    }
#undef LSF_ADJ_CASE
    return check_launch("adjoint_rows_kernel");
  }
  dim3 grid(static_cast<unsigned>((a.n + kBM - 1) / kBM), static_cast<unsigned>((a.d + kBN - 1) / kBN));
  LaunchScope ls(st, LSF_KERNEL_OTHER, 4.0 * a.n * (a.ldr + 2 * a.d + a.nterms));
  adjoint_gemm_kernel<LOGD><<<grid, 256, 0, st>>>(a);
  return check_launch("adjoint_gemm_kernel");
}

int launch_weights(const WeightArgs& a, cudaStream_t st) {
  const int grid = device_info().sms * 2;
  LaunchScope ls(st, LSF_KERNEL_OTHER, 4.0 * a.n * (a.nterms + 2));
  weight_grad_kernel<<<grid, 256, 0, st>>>(a);
  return check_launch("weight_grad_kernel");
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" int lsf_gradient(const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y,
                            const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                            const lsf_scalings* s_yy, const lsf_result* result, int debiased,
                            int mode, float* gX, float* gY, float* ga, float* gb, void* stream) {
  if (!th || !x || !y || !s_xy || !result) return fail(LSF_ERR_ARG, "lsf_gradient: NULL argument");
  if (debiased && (!s_xx || !s_yy))
    return fail(LSF_ERR_ARG, "lsf_gradient: the debiased gradient needs s_xx and s_yy");
  if (th->r < 1 || th->d < 1 || th->r > th->ldr || th->ldr % 4 != 0 || th->ldr > 1024 || !th->U)
    return fail(LSF_ERR_ARG, "lsf_gradient: bad theta");
  if (x->n < 1 || y->n < 1) return fail(LSF_ERR_ARG, "lsf_gradient: empty measure");
  if (mode != LSF_MODE_STORED && mode != LSF_MODE_LOG)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_gradient: needs stored (or stored log) features");
  const bool logd = mode == LSF_MODE_LOG;
  if ((gX && (!x->F || !x->X)) || (gY && (!y->F || !y->X)))
    return fail(LSF_ERR_ARG, "lsf_gradient: point gradients need X and stored features F");
  if ((x->F && reinterpret_cast<uintptr_t>(x->F) % 16) || (y->F && reinterpret_cast<uintptr_t>(y->F) % 16))
    return fail(LSF_ERR_ARG, "lsf_gradient: F must be 16-byte aligned");
  cudaStream_t st = as_stream(stream);
  const lsf_result* rxy = result;
  const lsf_result* rxx = result + 1;
  const lsf_result* ryy = result + 2;
  for (int side = 0; side < 2; ++side) {
    const lsf_cloud* cl = side == 0 ? x : y;
    float* gP = side == 0 ? gX : gY;
    float* gw = side == 0 ? ga : gb;
    const lsf_scalings* self = side == 0 ? s_xx : s_yy;
    const lsf_result* rself = side == 0 ? rxx : ryy;
    if (gP) {
      AdjArgs a{};
      a.X = cl->X; a.F = cl->F; a.U = th->U; a.n = cl->n;
      a.r = th->r; a.ldr = th->ldr; a.d = th->d;
      a.gX = gP;
      a.alpha[0] = side == 0 ? s_xy->u : s_xy->v;
      a.T[0] = side == 0 ? s_xy->t_v : s_xy->t_u;
      a.coef[0] = 1.f;
      a.nterms = 1;
      if (debiased) {
        a.alpha[1] = self->u; a.T[1] = self->t_v; a.coef[1] = -0.5f;
        a.alpha[2] = self->v; a.T[2] = self->t_u; a.coef[2] = -0.5f;
        a.nterms = 3;
      }
      int rc = logd ? launch_points<true>(a, st) : launch_points<false>(a, st);
      if (rc != LSF_OK) return rc;
    }
    if (gw) {
      WeightArgs w{};
      w.shift = cl->shift; w.n = cl->n; w.eps = th->eps; w.g = gw; w.is_log = logd ? 1 : 0;
      w.s[0] = side == 0 ? s_xy->u : s_xy->v;
      w.res[0] = rxy;
      w.sign[0] = side == 0 ? 1.0 : -1.0;
      w.coef[0] = 1.0;
      w.nterms = 1;
      if (debiased) {
        w.s[1] = self->u; w.res[1] = rself; w.sign[1] = 1.0; w.coef[1] = -0.5;
        w.s[2] = self->v; w.res[2] = rself; w.sign[2] = -1.0; w.coef[2] = -0.5;
        w.nterms = 3;
      }
      int rc = launch_weights(w, st);
      if (rc != LSF_OK) return rc;
    }
  }
  return LSF_OK;
}
