// Lemma 1 feature map on the device: radius R, anchors u_k and their
// log-constants, and the stored shifted features F = exp(L - shift) with
//   L_ik = c_k - (2/eps) ||x_i - u_k||^2.
#include <cuda_runtime.h>

#include "common.cuh"

namespace lsf {
namespace {

constexpr int kFeatWarps = 8;
constexpr int kFeatRowsPerWarp = 2;
constexpr int kFeatDChunk = 32;

__global__ void radius_kernel(const float* __restrict__ P, int64_t n, int d,
                              unsigned* __restrict__ key) {
  float best = 0.f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float* p = P + i * d;
    float s = 0.f;
    for (int k = 0; k < d; ++k) s = fmaf(p[k], p[k], s);
    best = fmaxf(best, s);
  }
  best = warp_max(best);
  // Non-negative floats order like their bit patterns, so an unsigned maximum works.
  if ((threadIdx.x & 31) == 0) atomicMax(key, __float_as_uint(best));
}

__global__ void radius_finish_kernel(const unsigned* __restrict__ key, float* __restrict__ R) {
  if (threadIdx.x == 0) R[0] = sqrtf(__uint_as_float(key[0]));
}

__global__ void anchors_kernel(const float* __restrict__ Z, int r, int d, double q, double sigma,
                               double eps, float* __restrict__ U, float* __restrict__ c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r) return;
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) {
    const float u = static_cast<float>(sigma * static_cast<double>(Z[static_cast<int64_t>(k) * d + j]));
    U[static_cast<int64_t>(k) * d + j] = u;
    nrm += static_cast<double>(u) * u;
  }
  c[k] = static_cast<float>(0.25 * d * log(2.0 * q) - 0.5 * log(static_cast<double>(r)) +
                            nrm / (eps * q));
}

// Warp-per-row feature kernel. Lane l owns columns 4l + 128j + e (j < C, e < 4).
// U is staged transposed in shared memory (d-chunk x ldr) so that lanes read
// consecutive columns. KIND 0 computes only the row shifts, KIND 1 stores
// F = exp(L - shift) (padding 0), KIND 2 stores the log form L - shift
// (padding -inf) for the log-domain passes.
template <int C, int KIND>
__global__ void __launch_bounds__(kFeatWarps * 32)
    features_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ U,
                    const float* __restrict__ c, int r, int ldr, float two_over_eps,
                    float* __restrict__ F, float* __restrict__ shift, unsigned* spread_key) {
  extern __shared__ __align__(16) float sU[];  // [min(d, kFeatDChunk)][ldr] then c[ldr]
  float* sc = sU + static_cast<size_t>(min(d, kFeatDChunk)) * ldr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (d + kFeatDChunk - 1) / kFeatDChunk;

  for (int k = threadIdx.x; k < ldr; k += blockDim.x) sc[k] = (k < r) ? c[k] : 0.f;
  auto load_chunk = [&](int ch) {
    const int d0 = ch * kFeatDChunk;
    const int dc = min(kFeatDChunk, d - d0);
    for (int idx = threadIdx.x; idx < dc * ldr; idx += blockDim.x) {
      const int dd = idx / ldr, k = idx - dd * ldr;
      sU[idx] = (k < r) ? U[static_cast<int64_t>(k) * d + d0 + dd] : 0.f;
    }
  };
  if (nchunks == 1) load_chunk(0);
  __syncthreads();

  float local_spread = 0.f;
  const int64_t rows_per_cta = kFeatWarps * kFeatRowsPerWarp;
  for (int64_t base = blockIdx.x * rows_per_cta; base < n; base += gridDim.x * rows_per_cta) {
    float acc[kFeatRowsPerWarp][C][4];
#pragma unroll
    for (int q = 0; q < kFeatRowsPerWarp; ++q)
#pragma unroll
      for (int j = 0; j < C; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][j][e] = 0.f;

    for (int ch = 0; ch < nchunks; ++ch) {
      if (nchunks > 1) {
        __syncthreads();
        load_chunk(ch);
        __syncthreads();
      }
      const int d0 = ch * kFeatDChunk;
      const int dc = min(kFeatDChunk, d - d0);
#pragma unroll
      for (int q = 0; q < kFeatRowsPerWarp; ++q) {
        const int64_t i = base + warp * kFeatRowsPerWarp + q;
        if (i >= n) continue;
        const float* xi = X + i * d + d0;
        for (int dd = 0; dd < dc; ++dd) {
          const float xv = __ldg(xi + dd);
          const float* urow = sU + static_cast<size_t>(dd) * ldr;
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            if (col < ldr) {
              const float4 u4 = *reinterpret_cast<const float4*>(urow + col);
              float t;
              t = xv - u4.x; acc[q][j][0] = fmaf(t, t, acc[q][j][0]);
              t = xv - u4.y; acc[q][j][1] = fmaf(t, t, acc[q][j][1]);
              t = xv - u4.z; acc[q][j][2] = fmaf(t, t, acc[q][j][2]);
              t = xv - u4.w; acc[q][j][3] = fmaf(t, t, acc[q][j][3]);
            }
          }
        }
      }
    }

#pragma unroll
    for (int q = 0; q < kFeatRowsPerWarp; ++q) {
      const int64_t i = base + warp * kFeatRowsPerWarp + q;
      if (i >= n) continue;
      float mx = -INFINITY, mn = INFINITY;
#pragma unroll
      for (int j = 0; j < C; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * lane + 128 * j + e;
          if (k < r) {
            const float L = sc[k] - two_over_eps * acc[q][j][e];
            acc[q][j][e] = L;
            mx = fmaxf(mx, L);
            mn = fminf(mn, L);
          }
        }
      }
      mx = warp_max(mx);
      mn = warp_min(mn);
      if (lane == 0) shift[i] = mx;
      local_spread = fmaxf(local_spread, mx - mn);
      if (KIND == 1) {
        float* Fi = F + i * ldr;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (col < ldr) {
            float4 o;
            o.x = (col + 0 < r) ? expf(acc[q][j][0] - mx) : 0.f;
            o.y = (col + 1 < r) ? expf(acc[q][j][1] - mx) : 0.f;
            o.z = (col + 2 < r) ? expf(acc[q][j][2] - mx) : 0.f;
            o.w = (col + 3 < r) ? expf(acc[q][j][3] - mx) : 0.f;
            *reinterpret_cast<float4*>(Fi + col) = o;
          }
        }
      } else if (KIND == 2) {
        float* Fi = F + i * ldr;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (col < ldr) {
            float4 o;
            o.x = (col + 0 < r) ? acc[q][j][0] - mx : -INFINITY;
            o.y = (col + 1 < r) ? acc[q][j][1] - mx : -INFINITY;
            o.z = (col + 2 < r) ? acc[q][j][2] - mx : -INFINITY;
            o.w = (col + 3 < r) ? acc[q][j][3] - mx : -INFINITY;
            *reinterpret_cast<float4*>(Fi + col) = o;
          }
        }
      }
    }
  }
  // Non-negative floats order like their bit patterns, so an unsigned maximum works.
  if (spread_key && lane == 0 && local_spread > 0.f)
    atomicMax(spread_key, __float_as_uint(local_spread));
}

template <int KIND>
int launch_features(const float* X, int64_t n, const lsf_theta* th, float* F, float* shift,
                    float* spread, cudaStream_t st) {
  constexpr bool STORE = KIND != 0;
  if (!X || !th || !shift || (STORE && !F)) return fail(LSF_ERR_ARG, "features: NULL argument");
  if (!th->U || !th->c) return fail(LSF_ERR_ARG, "features: theta has NULL U or c");
  if (n < 1) return fail(LSF_ERR_ARG, "features: n must be >= 1");
  if (th->d < 1 || th->r < 1 || th->r > th->ldr)
    return fail(LSF_ERR_ARG, "features: need d >= 1 and 1 <= r <= ldr");
  if (th->ldr % 4 != 0 || th->ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "features: ldr must be a multiple of 4, <= 1024");
  if (!(th->eps > 0.0)) return fail(LSF_ERR_ARG, "features: eps must be > 0");
  if (STORE && reinterpret_cast<uintptr_t>(F) % 16 != 0)
    return fail(LSF_ERR_ARG, "features: F must be 16-byte aligned");
  const int ldr = th->ldr;
  const int C = (ldr + 127) / 128;
  const int dchunk = th->d < kFeatDChunk ? th->d : kFeatDChunk;
  const size_t smem = sizeof(float) * (static_cast<size_t>(dchunk) * ldr + ldr);
  const int64_t rows_per_cta = kFeatWarps * kFeatRowsPerWarp;
  int64_t grid = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = static_cast<int64_t>(device_info().sms) * 8;
  if (grid > cap) grid = cap;
  const float toe = static_cast<float>(2.0 / th->eps);
  unsigned* skey = reinterpret_cast<unsigned*>(spread);
  double bytes = 4.0 * n * th->d + 4.0 * n + (STORE ? 4.0 * n * ldr : 0.0);
  LaunchScope ls(st, LSF_KERNEL_FEATURES, bytes);
#define LSF_FEAT_CASE(CC)                                                                  \
  case CC: {                                                                               \
    auto kern = features_kernel<CC, KIND>;                                                \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
    kern<<<(unsigned)grid, kFeatWarps * 32, smem, st>>>(X, n, th->d, th->U, th->c, th->r,  \
                                                        ldr, toe, F, shift, skey);         \
  } break;
  switch (C <= 1 ? 1 : C <= 2 ? 2 : C <= 4 ? 4 : 8) {
    LSF_FEAT_CASE(1)
    LSF_FEAT_CASE(2)
    LSF_FEAT_CASE(4)
    LSF_FEAT_CASE(8)
  }
#undef LSF_FEAT_CASE
  return check_launch("features_kernel");
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_radius(const float* X, int64_t n, const float* Y, int64_t m, int d, float* R_out,
               void* stream) {
  if (!X || !Y || !R_out) return fail(LSF_ERR_ARG, "lsf_radius: NULL argument");
  if (n < 1 || m < 1 || d < 1) return fail(LSF_ERR_ARG, "lsf_radius: need n, m, d >= 1");
  cudaStream_t st = as_stream(stream);
  // The maximum squared norm is accumulated in the output word, then rooted.
  unsigned* key = reinterpret_cast<unsigned*>(R_out);
  if (cudaMemsetAsync(key, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_radius: memset failed");
  const int grid = device_info().sms * 2;
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 4.0 * (n + m) * d);
    radius_kernel<<<grid, 256, 0, st>>>(X, n, d, key);
    radius_kernel<<<grid, 256, 0, st>>>(Y, m, d, key);
    radius_finish_kernel<<<1, 32, 0, st>>>(key, R_out);
  }
  return check_launch("radius_kernel");
}

int lsf_anchors(const float* Z, int r, int d, double q, double sigma, double eps, float* U,
                float* c, void* stream) {
  if (!Z || !U || !c) return fail(LSF_ERR_ARG, "lsf_anchors: NULL argument");
  if (r < 1 || d < 1) return fail(LSF_ERR_ARG, "lsf_anchors: need r, d >= 1");
  if (!(q > 0.0) || !(sigma >= 0.0) || !(eps > 0.0))
    return fail(LSF_ERR_ARG, "lsf_anchors: need q > 0, sigma >= 0, eps > 0");
  cudaStream_t st = as_stream(stream);
  LaunchScope ls(st, LSF_KERNEL_OTHER, 8.0 * r * d + 4.0 * r);
  anchors_kernel<<<(r + 127) / 128, 128, 0, st>>>(Z, r, d, q, sigma, eps, U, c);
  return check_launch("anchors_kernel");
}

int lsf_features(const float* X, int64_t n, const lsf_theta* theta, float* F, float* shift,
                 float* spread, void* stream) {
  return launch_features<1>(X, n, theta, F, shift, spread, as_stream(stream));
}

int lsf_log_features(const float* X, int64_t n, const lsf_theta* theta, float* L, float* shift,
                     float* spread, void* stream) {
  return launch_features<2>(X, n, theta, L, shift, spread, as_stream(stream));
}

int lsf_row_shift(const float* X, int64_t n, const lsf_theta* theta, float* shift,
                  float* spread, void* stream) {
  return launch_features<0>(X, n, theta, nullptr, shift, spread, as_stream(stream));
}

}  // extern "C"
