// Fused Sinkhorn pass over stored shifted features (stored-feature variant).
//
// One half of Alg. 1 on K = xi~ zeta~^T reads each row F_i once and uses it twice:
// for the row product s_i = F_i . t (the plain product K v), and, after the
// division new_i = w_i / s_i, for the transposed accumulation t' += new_i F_i.
//
// Layout: a persistent grid of one CTA per SM. Warp 7 is a producer that streams
// tiles of consecutive rows (one contiguous span of F) into a ring of shared
// memory stages with bulk TMA copies (cp.async.bulk), plus the per-row weights
// and previous scalings with 4-byte cp.async, all completing on one mbarrier
// per stage. Warps 0-6 consume rows warp-per-row: lane l holds columns
// 4l + 128j (+0..3) in registers, the row product is a butterfly shuffle sum,
// and the transposed accumulation stays in registers for the whole launch.
// At the end each CTA writes its partial r-vector; the last CTA to arrive sums
// the partials in CTA order (FP64), so results do not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>

#include "reduce.cuh"

namespace lsf {
namespace {

template <int C, int NRHS, int MODE>
__global__ void __launch_bounds__(kPassThreads, 1) pass_kernel(const PassArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = a.nstages;
  const int ldr = a.ldr;
  const int TR = a.tile_rows;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + S;
  float* sF = reinterpret_cast<float*>(smem + 128 * ((16 * S + 127) / 128));
  float* sV = sF + static_cast<size_t>(S) * TR * ldr;  // [S][NRHS][2][TR]: w, old

  __shared__ double s_res[kConsumerWarps][2];
  __shared__ int s_flag;
  __shared__ int s_last;

  constexpr bool kNeedT = MODE != kPassAxpy;
  constexpr bool kAcc = MODE != kPassDot;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1 + 32);  // producer expect_tx arrival + 32 cp.async arrivals
      mbar_init(&empty[s], kConsumerWarps);
    }
    fence_mbarrier_init();
    s_flag = 0;
  }
  __syncthreads();

  int flag = 0;
  float acc[NRHS][C][4];
  double res[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    res[k] = 0.0;
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[k][j][e] = 0.f;
  }
  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
      const int s = it % S;
      const uint32_t ph = static_cast<uint32_t>(it / S) & 1u;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_bounded(&empty[s], ph ^ 1u) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        flag |= LSF_ERR_TIMEOUT;
        break;
      }
      const int64_t row0 = tile * TR;
      const int rows = static_cast<int>(min(static_cast<int64_t>(TR), a.n - row0));
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(rows) * static_cast<uint32_t>(ldr) * 4u;
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_copy_g2s(sF + static_cast<size_t>(s) * TR * ldr, a.F + row0 * ldr, bytes, &full[s]);
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        float* dw = sV + static_cast<size_t>((s * NRHS + k) * 2) * TR;
        float* dold = dw + TR;
        const float* w = a.rhs[k].w;
        const float* old = a.rhs[k].old;
        for (int i = lane; i < rows; i += 32) {
          if (MODE != kPassAxpy) cp_async_4(dw + i, w + row0 + i);
          if (old) cp_async_4(dold + i, old + row0 + i);
        }
      }
      cp_async_mbar_arrive(&full[s]);
    }
    // Drain: every copy this CTA issued has landed before shared memory is reused.
    const int used = min(it, S);
    for (int j = 0; j < used; ++j) {
      const int itj = it - 1 - j;
      const int s = itj % S;
      const uint32_t ph = static_cast<uint32_t>(itj / S) & 1u;
      if (lane == 0 && !mbar_wait_bounded(&full[s], ph)) flag |= LSF_ERR_TIMEOUT;
    }
  } else {
    // ------------------------------------------------------------ consumers
    float t[NRHS][C][4];
    bool has_old[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      has_old[k] = a.rhs[k].old != nullptr;
#pragma unroll
      for (int j = 0; j < C; ++j) {
        const int col = 4 * lane + 128 * j;
        float4 tv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kNeedT && col < ldr) tv = *reinterpret_cast<const float4*>(a.rhs[k].t_in + col);
        t[k][j][0] = tv.x; t[k][j][1] = tv.y; t[k][j][2] = tv.z; t[k][j][3] = tv.w;
      }
    }

    // Each warp takes RW rows of a tile at once (rows rr and rr + kConsumerWarps):
    // their chains of shared loads, FMAs and shuffles are independent, which hides
    // latency with only two warps per SMSP. With two right-hand sides the two dot
    // products of one row already give that independence.
    constexpr int RW = (NRHS == 1) ? 2 : 1;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
      const int s = it % S;
      const uint32_t ph = static_cast<uint32_t>(it / S) & 1u;
      int ok = 1;
      if (lane == 0) ok = mbar_wait_bounded(&full[s], ph) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        flag |= LSF_ERR_TIMEOUT;
        break;
      }
      const int64_t row0 = tile * TR;
      const int rows = static_cast<int>(min(static_cast<int64_t>(TR), a.n - row0));
      const float* tF = sF + static_cast<size_t>(s) * TR * ldr;
      for (int rr = warp; rr < rows; rr += RW * kConsumerWarps) {
        float4 f[RW][C];
        bool valid[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          const int row = rr + q * kConsumerWarps;
          valid[q] = row < rows;
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            f[q][j] = (valid[q] && col < ldr)
                          ? *reinterpret_cast<const float4*>(tF + static_cast<size_t>(row) * ldr + col)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          const float* vw = sV + static_cast<size_t>((s * NRHS + k) * 2) * TR;
          const float* vold = vw + TR;
          float scale[RW];
          if (MODE == kPassAxpy) {
#pragma unroll
            for (int q = 0; q < RW; ++q) scale[q] = valid[q] ? vold[rr + q * kConsumerWarps] : 0.f;
          } else {
            float dot[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
              for (int j = 0; j < C; ++j) {
                d0 = fmaf(f[q][j].x, t[k][j][0], d0);
                d1 = fmaf(f[q][j].y, t[k][j][1], d1);
                d2 = fmaf(f[q][j].z, t[k][j][2], d2);
                d3 = fmaf(f[q][j].w, t[k][j][3], d3);
              }
              dot[q] = (d0 + d1) + (d2 + d3);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
              for (int q = 0; q < RW; ++q) dot[q] += __shfl_xor_sync(0xffffffffu, dot[q], o);
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              const int row = rr + q * kConsumerWarps;
              scale[q] = 0.f;
              if (!valid[q]) continue;
              const float wi = vw[row];
              if (has_old[k] && lane == 0)
                res[k] += fabs(static_cast<double>(vold[row]) * static_cast<double>(dot[q]) -
                               static_cast<double>(wi));
              if (MODE == kPassUpdate) {
                scale[q] = wi * __frcp_rn(dot[q]);
                if (lane == 0) {
                  a.rhs[k].out[row0 + row] = scale[q];
                  if (!(dot[q] > 0.f) || !isfinite(scale[q])) flag |= LSF_ERR_NONFINITE;
                }
              }
            }
          }
          if (kAcc) {
#pragma unroll
            for (int q = 0; q < RW; ++q)
#pragma unroll
              for (int j = 0; j < C; ++j) {
                acc[k][j][0] = fmaf(scale[q], f[q][j].x, acc[k][j][0]);
                acc[k][j][1] = fmaf(scale[q], f[q][j].y, acc[k][j][1]);
                acc[k][j][2] = fmaf(scale[q], f[q][j].z, acc[k][j][2]);
                acc[k][j][3] = fmaf(scale[q], f[q][j].w, acc[k][j][3]);
              }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  // All tiles are consumed and every copy has landed: shared memory is free.
  __syncthreads();
  if (warp < kConsumerWarps) {
    // Park the register partials in shared memory.
    float* red = sF;  // [kConsumerWarps][NRHS][ldr]
    if (kAcc) {
#pragma unroll
      for (int k = 0; k < NRHS; ++k)
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (col < ldr)
            *reinterpret_cast<float4*>(red + static_cast<size_t>(warp * NRHS + k) * ldr + col) =
                make_float4(acc[k][j][0], acc[k][j][1], acc[k][j][2], acc[k][j][3]);
        }
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) s_res[warp][k] = res[k];
  }
  if (flag) atomicOr(&s_flag, flag);
  __syncthreads();

  finish_pass<NRHS, kAcc>(sF, kConsumerWarps, &s_res[0][0], ldr, a.rhs, a.part, a.rpart, a.counter,
                         a.status, s_flag, &s_last);
}

}  // namespace

namespace {

template <int C, int NRHS>
int launch_c_nrhs(int mode, const PassArgs& a, unsigned grid, size_t smem, cudaStream_t st) {
  void (*kern)(PassArgs) = nullptr;
  if (mode == kPassUpdate) kern = pass_kernel<C, NRHS, kPassUpdate>;
  else if (mode == kPassAxpy) kern = pass_kernel<C, NRHS, kPassAxpy>;
  else kern = pass_kernel<C, NRHS, kPassDot>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "pass: smem attribute: %s", cudaGetErrorString(e));
  kern<<<grid, kPassThreads, smem, st>>>(a);
  return check_launch("pass_kernel");
}

int g_tile_bytes = 56 * 1024;
int g_max_stages = 8;

}  // namespace

int set_pass_tiling(int tile_bytes, int max_stages) {
  if (tile_bytes < 512 || tile_bytes > 128 * 1024 || max_stages < 2 || max_stages > 16)
    return fail(LSF_ERR_ARG, "pass tiling: tile_bytes in [512, 131072], stages in [2, 16]");
  g_tile_bytes = tile_bytes;
  g_max_stages = max_stages;
  return LSF_OK;
}

void get_pass_tiling(int* tile_bytes, int* max_stages) {
  *tile_bytes = g_tile_bytes;
  *max_stages = g_max_stages;
}

double pass_bytes(int mode, int nrhs, int64_t n, int ldr, bool with_old) {
  double per_row = 4.0 * ldr;
  if (mode == kPassUpdate) per_row += nrhs * 4.0 * (2 + (with_old ? 1 : 0));  // w, out, old
  if (mode == kPassAxpy) per_row += nrhs * 4.0;                                // given scaling
  if (mode == kPassDot) per_row += nrhs * 8.0;                                 // w, old
  return per_row * static_cast<double>(n);
}

int launch_pass(int mode, int nrhs, PassArgs a, cudaStream_t st) {
  const DeviceInfo& dev = device_info();
  if (a.n < 1) return fail(LSF_ERR_ARG, "pass: n must be >= 1");
  if (a.ldr < 4 || a.ldr % 4 != 0 || a.ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "pass: ldr must be a multiple of 4 in [4, 1024]");
  if (reinterpret_cast<uintptr_t>(a.F) % 16 != 0)
    return fail(LSF_ERR_ARG, "pass: features must be 16-byte aligned");
  const int64_t row_bytes = 4LL * a.ldr;
  // Tile of consecutive rows: about g_tile_bytes, a whole number of rows for
  // every consumer warp, but small enough to give every SM work.
  const int64_t unit = (nrhs == 1 ? 2 : 1) * kConsumerWarps;
  int64_t tr = std::max<int64_t>(1, g_tile_bytes / row_bytes);
  if (tr >= unit) tr -= tr % unit;
  const int64_t want_tiles = 2LL * dev.sms;
  if ((a.n + tr - 1) / tr < want_tiles) tr = std::max<int64_t>(1, (a.n + want_tiles - 1) / want_tiles);
  tr = std::min<int64_t>(tr, 256);
  a.tile_rows = static_cast<int>(tr);
  a.ntiles = (a.n + tr - 1) / tr;
  const size_t stage_bytes = static_cast<size_t>(tr * row_bytes) + static_cast<size_t>(nrhs) * 2 * tr * 4;
  const size_t static_smem = 1024;  // s_res and flags, with margin
  const size_t budget = static_cast<size_t>(dev.smem_optin) - static_smem;
  int S = static_cast<int>(std::min<size_t>(static_cast<size_t>(g_max_stages), (budget - 256) / stage_bytes));
  if (S < 2) return fail(LSF_ERR_UNSUPPORTED, "pass: tile does not fit in shared memory");
  a.nstages = S;
  size_t smem = 128 * ((16 * S + 127) / 128) + S * stage_bytes;
  const size_t red_bytes = 128 * ((16 * S + 127) / 128) +
                           static_cast<size_t>(kConsumerWarps) * nrhs * a.ldr * 4;
  smem = std::max(smem, red_bytes);
  if (smem > budget) return fail(LSF_ERR_UNSUPPORTED, "pass: shared memory over budget");
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(dev.sms, a.ntiles));
  const int C = (a.ldr + 127) / 128;
  const int Cp = C <= 1 ? 1 : C <= 2 ? 2 : C <= 4 ? 4 : 8;
  bool with_old = false;
  for (int k = 0; k < nrhs; ++k) with_old |= a.rhs[k].old != nullptr;
  LaunchScope ls(st, LSF_KERNEL_PASS, pass_bytes(mode, nrhs, a.n, a.ldr, with_old));
  if (nrhs == 1) {
    switch (Cp) {
      case 1: return launch_c_nrhs<1, 1>(mode, a, grid, smem, st);
      case 2: return launch_c_nrhs<2, 1>(mode, a, grid, smem, st);
      case 4: return launch_c_nrhs<4, 1>(mode, a, grid, smem, st);
      default: return launch_c_nrhs<8, 1>(mode, a, grid, smem, st);
    }
  }
  switch (Cp) {
    case 1: return launch_c_nrhs<1, 2>(mode, a, grid, smem, st);
    case 2: return launch_c_nrhs<2, 2>(mode, a, grid, smem, st);
    case 4: return launch_c_nrhs<4, 2>(mode, a, grid, smem, st);
    default: return launch_c_nrhs<8, 2>(mode, a, grid, smem, st);
  }
}

}  // namespace lsf
