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

#include <algorithm>

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
    LaunchScope ls(st, LSF_KERNEL_ADJOINT, 4.0 * a.n * (a.ldr + 2 * a.d + a.nterms));
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
  LaunchScope ls(st, LSF_KERNEL_ADJOINT, 4.0 * a.n * (a.ldr + 2 * a.d + a.nterms));
  adjoint_gemm_kernel<LOGD><<<grid, 256, 0, st>>>(a);
  return check_launch("adjoint_gemm_kernel");
}

int launch_weights(const WeightArgs& a, cudaStream_t st) {
  const int grid = device_info().sms * 2;
  LaunchScope ls(st, LSF_KERNEL_ADJOINT, 4.0 * a.n * (a.nterms + 2));
  weight_grad_kernel<<<grid, 256, 0, st>>>(a);
  return check_launch("weight_grad_kernel");
}


// ---------------------------------------------------------------- anchors
//
// Gradient w.r.t. the anchors u_k (q held fixed). With the same A as above and
// d xi_ik / d u_k = xi_ik ((4/eps)(x_i - u_k) + 2 u_k/(eps q)):
//   grad u_k = - sum_i A_ik (4 (x_i - u_k) + 2 u_k / q)
//            = -4 sum_i A_ik (x_i - u_k) - (2/q) cs_k u_k,   cs_k = sum_i A_ik,
// summed over both clouds. Accumulating A_ik (x_i - u_k) rather than A^T X and
// cs u separately avoids their cancellation.
//
// Kernel: a CTA takes a contiguous chunk of rows and DC of the d coordinates;
// thread (g, c4) owns the four feature columns 4 c4 .. 4 c4 + 3 and walks rows
// g, g + G, ... of the chunk, reading each row's float4 directly (coalesced
// across the warp); x_i and the row scalings are warp-broadcast loads. The G row
// groups are folded in shared memory in a fixed order and the CTA writes its
// partial [DC + 1][ldr] (the last row is cs) to the workspace; a second kernel
// sums the chunks in a fixed order in FP64.
constexpr int kAnchorThreads = 512;

struct AnchorArgs {
  const float* X;  // n x d
  const float* F;  // n x ldr
  const float* U;  // r x d
  int64_t n;
  int r, ldr, d;
  int nterms;
  const float* alpha[kMaxTerms];
  const float* T[kMaxTerms];
  float coef[kMaxTerms];
  int dchunks;
  int64_t rows_per_chunk;
  float* part;  // [chunks * dchunks][DC + 1][ldr]
};

template <int DC, bool LOGD>
__global__ void __launch_bounds__(kAnchorThreads) anchor_grad_kernel(const AnchorArgs a) {
  extern __shared__ __align__(16) float red[];  // [G][DC + 1][ldr]
  constexpr int kUnroll = DC <= 4 ? 4 : 2;  // rows in flight per thread
  const int ldr = a.ldr, d = a.d;
  const int tcols = ldr >> 2;
  const int CT = (tcols + 31) & ~31;
  const int G = blockDim.x / CT;
  const int g = threadIdx.x / CT;
  const int c4 = threadIdx.x - g * CT;
  const bool active = g < G && c4 < tcols;
  const int col = 4 * c4;
  const int d0 = blockIdx.y * DC;
  const int64_t i0 = blockIdx.x * a.rows_per_chunk;
  const int64_t i1 = min(a.n, i0 + a.rows_per_chunk);

  float acc[DC][4], cs[4] = {0.f, 0.f, 0.f, 0.f};
  float uk[DC][4];
  float4 t[kMaxTerms];
#pragma unroll
  for (int c = 0; c < DC; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      acc[c][e] = 0.f;
      const int k = col + e;
      uk[c][e] = (active && k < a.r && d0 + c < d) ? a.U[static_cast<int64_t>(k) * d + d0 + c] : 0.f;
    }
#pragma unroll
  for (int p = 0; p < kMaxTerms; ++p)
    t[p] = (active && p < a.nterms) ? *reinterpret_cast<const float4*>(a.T[p] + col)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) {
#pragma unroll kUnroll
    for (int64_t i = i0 + g; i < i1; i += G) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(a.F + i * ldr + col));
      float A[4];
      if (LOGD) {
        A[0] = A[1] = A[2] = A[3] = 0.f;
#pragma unroll
        for (int p = 0; p < kMaxTerms; ++p) {
          if (p < a.nterms) {
            const float al = __ldg(a.alpha[p] + i), c = a.coef[p];
            A[0] = fmaf(c, ex2_approx((f.x + al + t[p].x) * kLog2e), A[0]);
            A[1] = fmaf(c, ex2_approx((f.y + al + t[p].y) * kLog2e), A[1]);
            A[2] = fmaf(c, ex2_approx((f.z + al + t[p].z) * kLog2e), A[2]);
            A[3] = fmaf(c, ex2_approx((f.w + al + t[p].w) * kLog2e), A[3]);
          }
        }
      } else {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < kMaxTerms; ++p) {
          if (p < a.nterms) {
            const float al = a.coef[p] * __ldg(a.alpha[p] + i);
            w.x = fmaf(al, t[p].x, w.x); w.y = fmaf(al, t[p].y, w.y);
            w.z = fmaf(al, t[p].z, w.z); w.w = fmaf(al, t[p].w, w.w);
          }
        }
        A[0] = f.x * w.x; A[1] = f.y * w.y; A[2] = f.z * w.z; A[3] = f.w * w.w;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) cs[e] += A[e];
      const float* xi = a.X + i * d + d0;
#pragma unroll
      for (int c = 0; c < DC; ++c) {
        if (d0 + c < d) {
          const float x = __ldg(xi + c);
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[c][e] = fmaf(A[e], x - uk[c][e], acc[c][e]);
        }
      }
    }
  }
  // fold the G row groups in a fixed order
  if (active) {
#pragma unroll
    for (int c = 0; c <= DC; ++c) {
      float* dst = red + (static_cast<size_t>(g) * (DC + 1) + c) * ldr + col;
      const float4 v = c < DC ? make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3])
                              : make_float4(cs[0], cs[1], cs[2], cs[3]);
      *reinterpret_cast<float4*>(dst) = v;
    }
  }
  __syncthreads();
  float* out = a.part + (static_cast<size_t>(blockIdx.x) * a.dchunks + blockIdx.y) * (DC + 1) * ldr;
  for (int idx = threadIdx.x; idx < (DC + 1) * ldr; idx += blockDim.x) {
    float s = 0.f;
    for (int gg = 0; gg < G; ++gg) s += red[static_cast<size_t>(gg) * (DC + 1) * ldr + idx];
    out[idx] = s;
  }
}

// gU[k][c] (=|+=) scale * (-4 sum_chunks S[c][k] - (2/q) cs_k u_kc)
template <int DC>
__global__ void anchor_finish_kernel(const float* part, int chunks, int dchunks, int ldr, int r, int d,
                                     const float* U, double q, double scale, int accumulate, float* gU) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= r * d) return;
  const int k = idx / d, c = idx - k * d;
  const int dc = c / DC, cc = c - dc * DC;
  double s = 0.0, cs = 0.0;
  for (int ch = 0; ch < chunks; ++ch) {
    const float* pp = part + (static_cast<size_t>(ch) * dchunks + dc) * (DC + 1) * ldr;
    s += pp[static_cast<size_t>(cc) * ldr + k];
    cs += pp[static_cast<size_t>(DC) * ldr + k];
  }
  const double v = scale * (-4.0 * s - (2.0 / q) * cs * static_cast<double>(U[idx]));
  gU[idx] = static_cast<float>(accumulate ? static_cast<double>(gU[idx]) + v : v);
}

template <int DC>
int launch_anchor_side(const AnchorArgs& in, bool logd, double q, double scale, int accumulate,
                       float* gU, const Workspace& ws, cudaStream_t st) {
  AnchorArgs a = in;
  const int sms = device_info().sms;
  a.dchunks = (a.d + DC - 1) / DC;
  // the chunk partials live in the workspace's partial region: slots * ldr * 4 floats
  const int64_t cap_slots = static_cast<int64_t>(max_pass_ctas()) * 4 / (DC + 1);
  // one CTA of 512 threads per SM (the kernel's register use allows one): a single wave
  int64_t chunks = std::min<int64_t>(cap_slots / a.dchunks, std::max(1, sms / a.dchunks));
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (a.n + 63) / 64));
  if (chunks * a.dchunks > cap_slots)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_anchor_gradient: d = %d needs more workspace than the solve's", a.d);
  a.rows_per_chunk = (a.n + chunks - 1) / chunks;
  chunks = (a.n + a.rows_per_chunk - 1) / a.rows_per_chunk;
  a.part = ws.part;
  const int tcols = a.ldr / 4;
  const int CT = (tcols + 31) & ~31;
  const int G = std::max(1, kAnchorThreads / CT);
  const int threads = G * CT;
  const size_t smem = sizeof(float) * static_cast<size_t>(G) * (DC + 1) * a.ldr;
  {
    LaunchScope ls(st, LSF_KERNEL_ADJOINT, 4.0 * a.n * (a.ldr + a.dchunks * (DC + a.nterms)));
    void (*kern)(AnchorArgs) = logd ? anchor_grad_kernel<DC, true> : anchor_grad_kernel<DC, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
      return fail(LSF_ERR_CUDA, "anchor_grad_kernel: smem attribute: %s", cudaGetErrorString(e));
    kern<<<dim3(static_cast<unsigned>(chunks), static_cast<unsigned>(a.dchunks)), threads, smem, st>>>(a);
    int rc = check_launch("anchor_grad_kernel");
    if (rc != LSF_OK) return rc;
  }
  LaunchScope ls(st, LSF_KERNEL_ADJOINT, 4.0 * chunks * a.dchunks * (DC + 1) * a.ldr);
  const int total = a.r * a.d;
  anchor_finish_kernel<DC><<<(total + 255) / 256, 256, 0, st>>>(
      ws.part, static_cast<int>(chunks), a.dchunks, a.ldr, a.r, a.d, a.U, q, scale, accumulate, gU);
  return check_launch("anchor_finish_kernel");
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" int lsf_gradient(const lsf_theta* th, const lsf_cloud* x, const lsf_cloud* y,
                            const lsf_scalings* s_xy, const lsf_scalings* s_xx,
                            const lsf_scalings* s_yy, const lsf_result* result, int debiased,
                            int mode, float* gX, float* gY, float* ga, float* gb, void* stream) {
  lsf::TraceRange trace_range("lsf_gradient");
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

extern "C" int lsf_anchor_gradient(const lsf_theta* th, double q, const lsf_cloud* x,
                                   const lsf_cloud* y, const lsf_scalings* s_xy,
                                   const lsf_scalings* s_xx, const lsf_scalings* s_yy, int debiased,
                                   int mode, double scale, float* gU, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_anchor_gradient");
  if (!th || !x || !y || !s_xy || !gU) return fail(LSF_ERR_ARG, "lsf_anchor_gradient: NULL argument");
  if (debiased && (!s_xx || !s_yy))
    return fail(LSF_ERR_ARG, "lsf_anchor_gradient: the debiased gradient needs s_xx and s_yy");
  if (th->r < 1 || th->d < 1 || th->r > th->ldr || th->ldr % 4 != 0 || th->ldr > 1024 || !th->U)
    return fail(LSF_ERR_ARG, "lsf_anchor_gradient: bad theta");
  if (!(q > 0.5) || !std::isfinite(q)) return fail(LSF_ERR_ARG, "lsf_anchor_gradient: q must exceed 1/2");
  if (x->n < 1 || y->n < 1) return fail(LSF_ERR_ARG, "lsf_anchor_gradient: empty measure");
  if (mode != LSF_MODE_STORED && mode != LSF_MODE_LOG)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_anchor_gradient: needs stored (or stored log) features");
  if (!x->F || !x->X || !y->F || !y->X)
    return fail(LSF_ERR_ARG, "lsf_anchor_gradient: needs X, Y and their stored features");
  const lsf_scalings* all[3] = {s_xy, debiased ? s_xx : nullptr, debiased ? s_yy : nullptr};
  for (const lsf_scalings* s : all) {
    if (!s) continue;
    if (!s->u || !s->v || !s->t_u || !s->t_v)
      return fail(LSF_ERR_ARG, "lsf_anchor_gradient: scalings need u, v, t_u, t_v");
    if (reinterpret_cast<uintptr_t>(s->t_u) % 16 || reinterpret_cast<uintptr_t>(s->t_v) % 16)
      return fail(LSF_ERR_ARG, "lsf_anchor_gradient: r-vectors must be 16-byte aligned");
  }
  if (reinterpret_cast<uintptr_t>(x->F) % 16 || reinterpret_cast<uintptr_t>(y->F) % 16)
    return fail(LSF_ERR_ARG, "lsf_anchor_gradient: F must be 16-byte aligned");
  Workspace ws{};
  int rc = carve_workspace(workspace, workspace_bytes, th->ldr, &ws);
  if (rc != LSF_OK) return rc;
  const bool logd = mode == LSF_MODE_LOG;
  cudaStream_t st = as_stream(stream);
  for (int side = 0; side < 2; ++side) {
    const lsf_cloud* cl = side == 0 ? x : y;
    const lsf_scalings* self = side == 0 ? s_xx : s_yy;
    AnchorArgs a{};
    a.X = cl->X; a.F = cl->F; a.U = th->U; a.n = cl->n;
    a.r = th->r; a.ldr = th->ldr; a.d = th->d;
    a.alpha[0] = side == 0 ? s_xy->u : s_xy->v;
    a.T[0] = side == 0 ? s_xy->t_v : s_xy->t_u;
    a.coef[0] = 1.f;
    a.nterms = 1;
    if (debiased) {
      a.alpha[1] = self->u; a.T[1] = self->t_v; a.coef[1] = -0.5f;
      a.alpha[2] = self->v; a.T[2] = self->t_u; a.coef[2] = -0.5f;
      a.nterms = 3;
    }
    rc = th->d <= 4 ? launch_anchor_side<4>(a, logd, q, scale, side, gU, ws, st)
                    : launch_anchor_side<8>(a, logd, q, scale, side, gU, ws, st);
    if (rc != LSF_OK) return rc;
  }
  return LSF_OK;
}
