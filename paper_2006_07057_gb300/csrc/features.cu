// Lemma 1 feature map on the device: radius R, anchors u_k and their
// log-constants, and the stored shifted features F = exp(L - shift) with
//   L_ik = c_k - (2/eps) ||x_i - u_k||^2.
#include <cuda_runtime.h>

#include "common.cuh"
#include "recompute.cuh"

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

// Principal Lambert branch W0(z), z >= 0, in FP64 on the device: Newton's
// iteration on w e^w - z from log(1 + z), as on the host (the iterates decrease
// monotonically to the root).
__device__ double lambert_w0_device(double z) {
  if (z == 0.0) return 0.0;
  double w = log1p(z);
  for (int i = 0; i < 200; ++i) {
    const double ew = exp(w);
    const double next = w - (w * ew - z) / (ew * (w + 1.0));
    if (fabs(next - w) <= 1e-16 * fabs(next)) return next;
    w = next;
  }
  return w;
}

// Lemma 1 parameters from the device radius: q = z / (2 W0(z)) with
// z = R^2 / (eps d) (q = 1/2 at R = 0), sigma = sqrt(q eps / 4); qs = {q, sigma}.
// A non-finite R gives NaN parameters (and, downstream, a non-finite status).
__global__ void params_kernel(const float* __restrict__ R, double eps, int d, double* __restrict__ qs) {
  if (threadIdx.x != 0) return;
  const double Rd = static_cast<double>(R[0]);
  const double z = Rd * Rd / (eps * d);
  double q = 0.5;
  if (!isfinite(z)) q = NAN;
  else if (z > 0.0) q = z / (2.0 * lambert_w0_device(z));
  qs[0] = q;
  qs[1] = sqrt(q * eps / 4.0);
}

// Anchors u_k = sigma z_k and log-constants c_k; q and sigma come from the host
// arguments, or from the device pair qs = {q, sigma} when qs is not NULL.
__global__ void anchors_kernel(const float* __restrict__ Z, int r, int d, double q, double sigma,
                               const double* __restrict__ qs, double eps, float* __restrict__ U,
                               float* __restrict__ c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r) return;
  if (qs) {
    q = qs[0];
    sigma = qs[1];
  }
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) {
    const float u = static_cast<float>(sigma * static_cast<double>(Z[static_cast<int64_t>(k) * d + j]));
    U[static_cast<int64_t>(k) * d + j] = u;
    nrm += static_cast<double>(u) * u;
  }
  c[k] = static_cast<float>(0.25 * d * log(2.0 * q) - 0.5 * log(static_cast<double>(r)) +
                            nrm / (eps * q));
}

// Which feature map a kernel evaluates, with its constants. Gaussian (Lemma 1):
// L_ik = c_k - (2/eps) ||x_i - u_k||^2 for k < r. Arc-cosine (Sec. 3.2 lemma):
// L_ik = c_k + s log(u_k . x_i) for u_k . x_i > 0 (else -inf, an exact zero
// feature) and k < r, and L_ir = log sqrt(kappa) (the merged constant feature).
// rf is the number of feature columns: r, or r + 1 for the arc-cosine map.
struct MapArgs {
  int r;
  int rf;
  float two_over_eps;  // Gaussian
  float s;             // arc-cosine exponent
  float lk;            // arc-cosine log sqrt(kappa)
};
enum FeatureMap : int { kMapGauss = 0, kMapArccos = 1 };

// accumulate one coordinate of the distance (Gaussian) or projection (arc-cosine)
template <int MAP>
__device__ __forceinline__ float map_acc(float x, float u, float acc) {
  if (MAP == kMapGauss) {
    const float t = x - u;
    return fmaf(t, t, acc);
  }
  return fmaf(x, u, acc);
}

// the log-feature of column k from its accumulated distance / projection
template <int MAP>
__device__ __forceinline__ float map_log(float acc, float ck, int k, const MapArgs& m) {
  if (MAP == kMapGauss) return ck - m.two_over_eps * acc;
  if (k == m.r) return m.lk;
  if (!(acc > 0.f)) return -INFINITY;
  return m.s == 0.f ? ck : ck + m.s * logf(acc);
}

// Warp-per-row feature kernel. Lane l owns columns 4l + 128j + e (j < C, e < 4).
// U is staged transposed in shared memory (d-chunk x ldr) so that lanes read
// consecutive columns. KIND 0 computes only the row shifts, KIND 1 stores
// F = exp(L - shift) (padding 0), KIND 2 stores the log form L - shift
// (padding -inf) for the log-domain passes. The spread is max - min over the
// finite log-features of a row (an exact zero feature has no range to lose).
// The stored kinds write columns [c0, ldr) of every row (c0 a multiple of 4) to
// F + i * ldf + (k - c0): the whole row for c0 = 0, ldf = ldr, or the stored
// block of a hybrid pass.
template <int C, int KIND, int MAP>
__global__ void __launch_bounds__(kFeatWarps * 32)
    features_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ U,
                    const float* __restrict__ c, int ldr, const MapArgs m,
                    float* __restrict__ F, float* __restrict__ shift, unsigned* spread_key,
                    int c0, int ldf) {
  extern __shared__ __align__(16) float sU[];  // [min(d, kFeatDChunk)][ldr] then c[ldr]
  float* sc = sU + static_cast<size_t>(min(d, kFeatDChunk)) * ldr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (d + kFeatDChunk - 1) / kFeatDChunk;
  const int r = m.r;

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
              acc[q][j][0] = map_acc<MAP>(xv, u4.x, acc[q][j][0]);
              acc[q][j][1] = map_acc<MAP>(xv, u4.y, acc[q][j][1]);
              acc[q][j][2] = map_acc<MAP>(xv, u4.z, acc[q][j][2]);
              acc[q][j][3] = map_acc<MAP>(xv, u4.w, acc[q][j][3]);
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
          if (k < m.rf) {
            const float L = map_log<MAP>(acc[q][j][e], sc[k < r ? k : 0], k, m);
            acc[q][j][e] = L;
            mx = fmaxf(mx, L);
            if (L != -INFINITY) mn = fminf(mn, L);
          }
        }
      }
      mx = warp_max(mx);
      mn = warp_min(mn);
      if (lane == 0) shift[i] = mx;
      local_spread = fmaxf(local_spread, mx - mn);
      if (KIND == 1) {
        float* Fi = F + i * ldf - c0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (col < ldr && col >= c0) {
            float4 o;
            o.x = (col + 0 < m.rf) ? expf(acc[q][j][0] - mx) : 0.f;
            o.y = (col + 1 < m.rf) ? expf(acc[q][j][1] - mx) : 0.f;
            o.z = (col + 2 < m.rf) ? expf(acc[q][j][2] - mx) : 0.f;
            o.w = (col + 3 < m.rf) ? expf(acc[q][j][3] - mx) : 0.f;
            *reinterpret_cast<float4*>(Fi + col) = o;
          }
        }
      } else if (KIND == 2) {
        float* Fi = F + i * ldf - c0;
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (col < ldr && col >= c0) {
            float4 o;
            o.x = (col + 0 < m.rf) ? acc[q][j][0] - mx : -INFINITY;
            o.y = (col + 1 < m.rf) ? acc[q][j][1] - mx : -INFINITY;
            o.z = (col + 2 < m.rf) ? acc[q][j][2] - mx : -INFINITY;
            o.w = (col + 3 < m.rf) ? acc[q][j][3] - mx : -INFINITY;
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

// ---------------------------------------------------------------- large d
//
// For d > kFeatDChunk the warp-per-row kernel would restage U for every block
// of rows. There the distances are a register-tiled contraction instead: a CTA
// computes a 128-row x 128-anchor tile of D_ik = sum_d (x_id - u_kd)^2 (the same
// direct differences, accumulated over d in the same order), stages 16 dims of
// X and U at a time in shared memory, writes L_ik = c_k - (2/eps) D_ik to the
// output and folds the row maxima into order-preserving keys (a maximum does
// not depend on the order of the atomics). A warp-per-row pass then turns each
// row into its shifted form (exp or log) and records the spread.
constexpr int kTM = 128, kTN = 128, kTK = 16;

template <int MAP>
__global__ void __launch_bounds__(256)
    features_tile_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ U,
                         const float* __restrict__ c, int ldr, const MapArgs m,
                         float* __restrict__ L, unsigned* __restrict__ row_key) {
  const int r = m.r;
  // rows padded by 4 floats: the transposing stores hit 2 banks at most
  __shared__ __align__(16) float sX[kTK][kTM + 4];
  __shared__ __align__(16) float sU[kTK][kTN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kTM;
  const int k0 = blockIdx.y * kTN;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  // loader roles: dim kk = tid % 16, rows/anchors tid / 16 + 16 s
  const int lk = tid & 15, lr = tid >> 4;
  for (int d0 = 0; d0 < d; d0 += kTK) {
    const int dd = d0 + lk;
#pragma unroll
    for (int s8 = 0; s8 < 8; ++s8) {
      const int rr = lr + 16 * s8;
      const int64_t i = i0 + rr;
      sX[lk][rr] = (i < n && dd < d) ? __ldg(X + i * d + dd) : 0.f;
      const int k = k0 + rr;
      sU[lk][rr] = (k < r && dd < d) ? __ldg(U + static_cast<int64_t>(k) * d + dd) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      const float4 xa = *reinterpret_cast<const float4*>(&sX[kk][4 * ty]);
      const float4 xb = *reinterpret_cast<const float4*>(&sX[kk][64 + 4 * ty]);
      const float4 ua = *reinterpret_cast<const float4*>(&sU[kk][4 * tx]);
      const float4 ub = *reinterpret_cast<const float4*>(&sU[kk][64 + 4 * tx]);
      const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
      const float uv[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          acc[a][b] = map_acc<MAP>(xv[a], uv[b], acc[a][b]);
        }
    }
    __syncthreads();
  }
  // epilogue: rows 4ty + a (a < 4) and 64 + 4ty + a - 4 (a >= 4); anchors likewise
  float cv[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int k = k0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + b - 4);
    cv[b] = (k < r) ? __ldg(c + k) : 0.f;
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t i = i0 + (a < 4 ? 4 * ty + a : 64 + 4 * ty + a - 4);
    float mx = -INFINITY;
    float Lv[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int k = k0 + (b < 4 ? 4 * tx + b : 64 + 4 * tx + b - 4);
      Lv[b] = map_log<MAP>(acc[a][b], cv[b], k, m);
      if (k < m.rf) mx = fmaxf(mx, Lv[b]);
    }
    // the 16 threads of a half-warp hold the same rows
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (i < n) {
      float* Li = L + i * ldr;
      const int ka = k0 + 4 * tx, kb = k0 + 64 + 4 * tx;
      if (ka < ldr) *reinterpret_cast<float4*>(Li + ka) = make_float4(Lv[0], Lv[1], Lv[2], Lv[3]);
      if (kb < ldr) *reinterpret_cast<float4*>(Li + kb) = make_float4(Lv[4], Lv[5], Lv[6], Lv[7]);
      if (tx == 0 && mx != -INFINITY) atomicMax(row_key + i, float_key(mx));
    }
  }
}

// Warp per row: shift = the row's maximum (decoded from its key, in place),
// F_ik = exp(L_ik - shift) (KIND 1, padding 0) or L_ik - shift (KIND 2,
// padding -inf), and the row's spread max - min.
template <int KIND>
__global__ void __launch_bounds__(256)
    features_shift_kernel(int64_t n, int rf, int ldr, float* __restrict__ F, float* shift,
                          unsigned* spread_key) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  float local_spread = 0.f;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    const float mx = key_float(reinterpret_cast<const unsigned*>(shift)[i]);
    __syncwarp();
    float* Fi = F + i * ldr;
    float mn = INFINITY;
    for (int col = 4 * lane; col < ldr; col += 128) {
      float4 v = *reinterpret_cast<float4*>(Fi + col);
      float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (col + q < rf) {
          if (e[q] != -INFINITY) mn = fminf(mn, e[q]);
          e[q] = KIND == 1 ? expf(e[q] - mx) : e[q] - mx;
        } else {
          e[q] = KIND == 1 ? 0.f : -INFINITY;
        }
      }
      *reinterpret_cast<float4*>(Fi + col) = make_float4(e[0], e[1], e[2], e[3]);
    }
    mn = warp_min(mn);
    if (lane == 0) shift[i] = mx;
    local_spread = fmaxf(local_spread, mx - mn);
  }
  if (spread_key && lane == 0 && local_spread > 0.f)
    atomicMax(spread_key, __float_as_uint(local_spread));
}

template <int KIND, int MAP>
int launch_features_tiled(const float* X, int64_t n, int d, const float* U, const float* c, int ldr,
                          const MapArgs& m, float* F, float* shift, unsigned* skey, cudaStream_t st) {
  if (cudaMemsetAsync(shift, 0, sizeof(float) * static_cast<size_t>(n), st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "features: memset failed");
  {
    LaunchScope ls(st, LSF_KERNEL_FEATURES, 4.0 * n * d + 4.0 * n * ldr);
    dim3 grid(static_cast<unsigned>((n + kTM - 1) / kTM), static_cast<unsigned>((ldr + kTN - 1) / kTN));
    features_tile_kernel<MAP><<<grid, 256, 0, st>>>(X, n, d, U, c, ldr, m, F,
                                                    reinterpret_cast<unsigned*>(shift));
    int rc = check_launch("features_tile_kernel");
    if (rc != LSF_OK) return rc;
  }
  LaunchScope ls(st, LSF_KERNEL_FEATURES, 8.0 * n * ldr + 4.0 * n);
  int64_t grid = (n + 7) / 8;
  const int64_t cap = static_cast<int64_t>(device_info().sms) * 8;
  if (grid > cap) grid = cap;
  features_shift_kernel<KIND><<<static_cast<unsigned>(grid), 256, 0, st>>>(n, m.rf, ldr, F, shift, skey);
  return check_launch("features_shift_kernel");
}

// Shared front end of the feature entry points (both maps, all three kinds).
template <int KIND, int MAP>
int launch_map(const float* X, int64_t n, int d, const float* U, const float* c, int ldr,
               const MapArgs& m, float* F, float* shift, float* spread, cudaStream_t st,
               int c0 = 0) {
  constexpr bool STORE = KIND != 0;
  const int ldf = ldr - c0;
  if (!X || !shift || (STORE && !F)) return fail(LSF_ERR_ARG, "features: NULL argument");
  if (!U || !c) return fail(LSF_ERR_ARG, "features: NULL anchors or constants");
  if (n < 1) return fail(LSF_ERR_ARG, "features: n must be >= 1");
  if (d < 1 || m.r < 1 || m.rf > ldr) return fail(LSF_ERR_ARG, "features: need d >= 1, r >= 1 and room in ldr");
  if (ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "features: ldr must be a multiple of 4, <= 1024");
  if (STORE && reinterpret_cast<uintptr_t>(F) % 16 != 0)
    return fail(LSF_ERR_ARG, "features: F must be 16-byte aligned");
  unsigned* skey = reinterpret_cast<unsigned*>(spread);
  if (c0 < 0 || c0 % 4 != 0 || c0 >= ldr) return fail(LSF_ERR_ARG, "features: bad column window");
  if (STORE && d > kFeatDChunk) {
    if (c0 != 0) return fail(LSF_ERR_UNSUPPORTED, "features: a column window needs d <= 32");
    return launch_features_tiled<KIND, MAP>(X, n, d, U, c, ldr, m, F, shift, skey, st);
  }
  const int C = (ldr + 127) / 128;
  const int dchunk = d < kFeatDChunk ? d : kFeatDChunk;
  const size_t smem = sizeof(float) * (static_cast<size_t>(dchunk) * ldr + ldr);
  const int64_t rows_per_cta = kFeatWarps * kFeatRowsPerWarp;
  int64_t grid = (n + rows_per_cta - 1) / rows_per_cta;
  const int64_t cap = static_cast<int64_t>(device_info().sms) * 8;
  if (grid > cap) grid = cap;
  double bytes = 4.0 * n * d + 4.0 * n + (STORE ? 4.0 * n * ldf : 0.0);
  LaunchScope ls(st, LSF_KERNEL_FEATURES, bytes);
#define LSF_FEAT_CASE(CC)                                                                   \
  case CC: {                                                                                \
    auto kern = features_kernel<CC, KIND, MAP>;                                            \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    kern<<<(unsigned)grid, kFeatWarps * 32, smem, st>>>(X, n, d, U, c, ldr, m, F, shift, skey, c0, ldf); \
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

template <int KIND>
int launch_features(const float* X, int64_t n, const lsf_theta* th, float* F, float* shift,
                    float* spread, cudaStream_t st, int c0 = 0) {
  if (!th) return fail(LSF_ERR_ARG, "features: NULL theta");
  if (th->r > th->ldr) return fail(LSF_ERR_ARG, "features: need r <= ldr");
  if (!(th->eps > 0.0)) return fail(LSF_ERR_ARG, "features: eps must be > 0");
  MapArgs m{};
  m.r = th->r;
  m.rf = th->r;
  m.two_over_eps = static_cast<float>(2.0 / th->eps);
  return launch_map<KIND, kMapGauss>(X, n, th->d, th->U, th->c, th->ldr, m, F, shift, spread, st, c0);
}

template <int KIND>
int launch_arccos(const float* X, int64_t n, const lsf_arccos* th, float* F, float* shift,
                  float* spread, cudaStream_t st) {
  if (!th) return fail(LSF_ERR_ARG, "arc-cosine features: NULL parameters");
  if (th->s < 0 || th->s > 2) return fail(LSF_ERR_UNSUPPORTED, "arc-cosine features: s must be 0, 1 or 2");
  if (!(th->kappa > 0.0)) return fail(LSF_ERR_ARG, "arc-cosine features: kappa must be > 0");
  if (th->r + 1 > th->ldr) return fail(LSF_ERR_ARG, "arc-cosine features: need r + 1 <= ldr");
  MapArgs m{};
  m.r = th->r;
  m.rf = th->r + 1;
  m.s = static_cast<float>(th->s);
  m.lk = static_cast<float>(0.5 * log(th->kappa));
  return launch_map<KIND, kMapArccos>(X, n, th->d, th->U, th->c, th->ldr, m, F, shift, spread, st);
}

__global__ void arccos_anchors_kernel(const float* __restrict__ Z, int r, int d, double sigma,
                                      float* __restrict__ U, float* __restrict__ c) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= r) return;
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) {
    const float u = static_cast<float>(sigma * static_cast<double>(Z[static_cast<int64_t>(k) * d + j]));
    U[static_cast<int64_t>(k) * d + j] = u;
    nrm += static_cast<double>(u) * u;
  }
  c[k] = static_cast<float>(0.5 * d * log(sigma) + 0.5 * log(2.0) - 0.5 * log(static_cast<double>(r)) -
                            0.25 * nrm * (1.0 - 1.0 / (sigma * sigma)));
}

}  // namespace

int launch_params_device(const float* R, double eps, int d, double* qs, cudaStream_t st) {
  LaunchScope ls(st, LSF_KERNEL_OTHER, 20.0);
  params_kernel<<<1, 32, 0, st>>>(R, eps, d, qs);
  return check_launch("params_kernel");
}

int launch_anchors_device(const float* Z, int r, int d, const double* qs, double eps, float* U,
                          float* c, cudaStream_t st) {
  LaunchScope ls(st, LSF_KERNEL_OTHER, 8.0 * r * d + 4.0 * r);
  anchors_kernel<<<(r + 127) / 128, 128, 0, st>>>(Z, r, d, 0.0, 0.0, qs, eps, U, c);
  return check_launch("anchors_kernel");
}

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
  anchors_kernel<<<(r + 127) / 128, 128, 0, st>>>(Z, r, d, q, sigma, nullptr, eps, U, c);
  return check_launch("anchors_kernel");
}

int lsf_features(const float* X, int64_t n, const lsf_theta* theta, float* F, float* shift,
                 float* spread, void* stream) {
  lsf::TraceRange trace_range("lsf_features");
  return launch_features<1>(X, n, theta, F, shift, spread, as_stream(stream));
}

int lsf_log_features(const float* X, int64_t n, const lsf_theta* theta, float* L, float* shift,
                     float* spread, void* stream) {
  lsf::TraceRange trace_range("lsf_log_features");
  return launch_features<2>(X, n, theta, L, shift, spread, as_stream(stream));
}

int lsf_row_shift(const float* X, int64_t n, const lsf_theta* theta, float* shift,
                  float* spread, void* stream) {
  return launch_features<0>(X, n, theta, nullptr, shift, spread, as_stream(stream));
}

int lsf_hybrid_columns(int ldr, int* c0) {
  if (!c0) return fail(LSF_ERR_ARG, "lsf_hybrid_columns: NULL output");
  if (ldr < 8 || ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_hybrid_columns: ldr must be a multiple of 4 in [8, 1024]");
  *c0 = hybrid_first_stored(ldr);
  return LSF_OK;
}

int lsf_hybrid_features(const float* X, int64_t n, const lsf_theta* theta, float* Fs, float* shift,
                        float* spread, void* stream) {
  lsf::TraceRange trace_range("lsf_hybrid_features");
  if (!theta) return fail(LSF_ERR_ARG, "lsf_hybrid_features: NULL theta");
  int c0 = 0;
  const int rc = lsf_hybrid_columns(theta->ldr, &c0);
  if (rc != LSF_OK) return rc;
  return launch_features<1>(X, n, theta, Fs, shift, spread, as_stream(stream), c0);
}

int lsf_arccos_anchors(const float* Z, int r, int d, double sigma, float* U, float* c, void* stream) {
  if (!Z || !U || !c) return fail(LSF_ERR_ARG, "lsf_arccos_anchors: NULL argument");
  if (r < 1 || d < 1) return fail(LSF_ERR_ARG, "lsf_arccos_anchors: need r, d >= 1");
  if (!(sigma > 1.0)) return fail(LSF_ERR_ARG, "lsf_arccos_anchors: sigma must be > 1");
  cudaStream_t st = as_stream(stream);
  LaunchScope ls(st, LSF_KERNEL_OTHER, 8.0 * r * d + 4.0 * r);
  arccos_anchors_kernel<<<(r + 127) / 128, 128, 0, st>>>(Z, r, d, sigma, U, c);
  return check_launch("arccos_anchors_kernel");
}

int lsf_arccos_features(const float* X, int64_t n, const lsf_arccos* th, float* F, float* shift,
                        float* spread, void* stream) {
  lsf::TraceRange trace_range("lsf_arccos_features");
  return launch_arccos<1>(X, n, th, F, shift, spread, as_stream(stream));
}

int lsf_arccos_log_features(const float* X, int64_t n, const lsf_arccos* th, float* L, float* shift,
                            float* spread, void* stream) {
  lsf::TraceRange trace_range("lsf_arccos_log_features");
  return launch_arccos<2>(X, n, th, L, shift, spread, as_stream(stream));
}

}  // extern "C"
