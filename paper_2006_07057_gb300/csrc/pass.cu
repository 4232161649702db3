// Fused Sinkhorn pass over stored shifted features (stored-feature variant).
//
// One half of Alg. 1 on K = xi~ zeta~^T reads each row F_i once and uses it twice:
// for the row product s_i = F_i . t (the plain product K v), and, after the
// division new_i = w_i / s_i, for the transposed accumulation t' += new_i F_i.
//
// Layout. A persistent grid of one CTA per SM. Warp 11 is a producer that streams
// tiles of consecutive rows (one contiguous span of F) into a ring of shared
// memory stages with bulk TMA copies (cp.async.bulk), plus the per-row weights
// and previous scalings with 4-byte cp.async, all completing on one mbarrier
// per stage. Warps 0-10 consume, independently of each other: a warp takes
// RW = 8/C consecutive rows of a tile at full width (lane l holds columns
// 4l + 128j, j < C, of each), so that every lane has 8 float4 of features in
// flight whatever r is. The RW row products are folded across the warp by a
// multi-row butterfly (RW - 1 + 5 - log2 RW shuffles instead of 5 RW), which
// also gives RW independent dependency chains. The transposed accumulation
// stays in registers for the whole launch (the right-hand sides t too, unless
// two of them at r = 1024 would not fit: then t is read from shared memory).
// For r > 512 a warp takes one row from each of two consecutive ring stages, so
// it still has two independent rows in flight with tiles of modest size.
// Every wait is bounded and reports LSF_ERR_TIMEOUT. At the end each CTA writes
// its partial r-vector; the partials are summed in two fixed-order levels
// (groups of CTAs, then groups; compensated FP32), so results do not depend on
// timing.
#include <cuda_runtime.h>

#include <algorithm>

#include "reduce.cuh"
#include "ring.cuh"

namespace lsf {
namespace {

template <int C, int NRHS, int MODE>
__global__ void __launch_bounds__(kPassThreads, 1) pass_kernel(const PassArgs a) {
  constexpr int RW = 8 / C;                      // rows per warp in one tile
  constexpr int TP = PassShape<C>::kTilesPerStep;  // tiles a warp works on at once
  constexpr int RT = RW * TP;                    // rows per warp at once
  constexpr int SH = RowFold<RT>::kShift;        // owner lane of row q is q << SH
  constexpr bool kTsmem = NRHS * C > 8;          // t read from shared memory
  constexpr bool kNeedT = MODE != kPassAxpy;
  constexpr bool kAcc = MODE != kPassDot;
  extern __shared__ __align__(128) unsigned char smem[];
  const int ldr = a.ldr;
  const Ring ring = ring_layout(smem, a.nstages, a.tile_rows, ldr);
  const int S = ring.S;
  const int TR = ring.TR;

  __shared__ __align__(16) float s_t[kTsmem ? NRHS : 1][kTsmem ? 128 * C : 4];
  __shared__ double s_res[kConsumerWarps][2];
  __shared__ int s_flag;
  __shared__ int s_last;
  __shared__ int s_skip;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    ring_init(ring, kConsumerWarps);
    fence_mbarrier_init();
    s_flag = 0;
    // a scaling-domain run that already produced a non-finite scaling is void
    // (it is repeated in the log domain): stream no tiles, but take part in the
    // cross-CTA reduction so that its counters stay consistent. Read once per
    // CTA, so the producer and the consumers agree.
    s_skip = (*reinterpret_cast<volatile int*>(a.status) & LSF_ERR_NONFINITE) != 0;
  }
  if (kTsmem && kNeedT) {
    for (int idx = threadIdx.x; idx < NRHS * 128 * C; idx += blockDim.x) {
      const int k = idx / (128 * C), c = idx - k * 128 * C;
      s_t[k][c] = (c < ldr) ? a.rhs[k].t_in[c] : 0.f;
    }
  }
  __syncthreads();

  int flag = 0;
  float acc[NRHS][C][4];
  // residual terms |old s - w| of the rows this lane owns: each in one rounding
  // (a fused multiply-add), summed with compensation in FP32 and widened once at
  // the end (no FP64 arithmetic per row)
  CompSum racc[NRHS];
  double res[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    res[k] = 0.0;
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[k][j][e] = 0.f;
  }
  const int64_t ntiles = s_skip ? 0 : a.ntiles;
  if (warp == kConsumerWarps) {
    ring_produce<NRHS>(ring, a.F, a.n, ntiles, a.rhs, MODE != kPassAxpy, lane, flag);
  } else {
    float t[kTsmem ? 1 : NRHS][C][4];
    bool has_old[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) has_old[k] = a.rhs[k].old != nullptr;
    if (!kTsmem) {
#pragma unroll
      for (int k = 0; k < (kTsmem ? 1 : NRHS); ++k)
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          float4 tv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (kNeedT && col < ldr) tv = *reinterpret_cast<const float4*>(a.rhs[k].t_in + col);
          t[k][j][0] = tv.x; t[k][j][1] = tv.y; t[k][j][2] = tv.z; t[k][j][3] = tv.w;
        }
    }
    const int myq = (lane >> SH) & (RT - 1);           // row (of the RT) this lane owns
    const bool owner = (lane & ((1 << SH) - 1)) == 0;  // exactly one owner lane per row

    int it = 0;
    bool dead = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !dead; tile += static_cast<int64_t>(TP) * gridDim.x) {
      // the TP tiles this step works on: tile, tile + grid, ... (consecutive ring stages)
      int rows_u[TP];
      int64_t row0_u[TP];
      const float* tF_u[TP];
      const float* vbase_u[TP];
      int nt = 0;
#pragma unroll
      for (int u = 0; u < TP; ++u) {
        const int64_t tu = tile + static_cast<int64_t>(u) * gridDim.x;
        rows_u[u] = 0;
        row0_u[u] = 0;
        tF_u[u] = ring.sF;
        vbase_u[u] = ring.sV;
        if (tu < ntiles) {
          const int s = (it + u) % S;
          if (!ring_wait_full(ring, it + u, lane)) {
            flag |= LSF_ERR_TIMEOUT;
            dead = true;
            break;
          }
          row0_u[u] = tu * TR;
          rows_u[u] = static_cast<int>(min(static_cast<int64_t>(TR), a.n - row0_u[u]));
          tF_u[u] = ring.sF + static_cast<size_t>(s) * TR * ldr;
          vbase_u[u] = ring.sV + static_cast<size_t>(s * NRHS * 2) * TR;
          ++nt;
        }
      }
      if (dead) break;
      for (int rr = warp * RW; rr < TR; rr += RW * kConsumerWarps) {
        float4 f[RT][C];
#pragma unroll
        for (int u = 0; u < TP; ++u)
#pragma unroll
          for (int q = 0; q < RW; ++q)
#pragma unroll
            for (int j = 0; j < C; ++j) {
              const int col = 4 * lane + 128 * j;
              f[u * RW + q][j] =
                  (rr + q < rows_u[u] && col < ldr)
                      ? *reinterpret_cast<const float4*>(tF_u[u] + static_cast<size_t>(rr + q) * ldr + col)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        // this lane's owned row: tile mu, row rr + mq. The per-tile values are
        // picked by compile-time indices (a runtime index would put the arrays in
        // local memory).
        const int mu = myq / RW, mq = myq - (myq / RW) * RW;
        const int mrow = rr + mq;
        int rows_m = rows_u[0];
        int64_t row0_m = row0_u[0];
        const float* vbase_m = vbase_u[0];
#pragma unroll
        for (int u = 1; u < TP; ++u)
          if (mu == u) {
            rows_m = rows_u[u];
            row0_m = row0_u[u];
            vbase_m = vbase_u[u];
          }
        const bool mvalid = mrow < rows_m;
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          float scale[RT];
          if (MODE == kPassAxpy) {
#pragma unroll
            for (int u = 0; u < TP; ++u) {
              const float* vold = vbase_u[u] + static_cast<size_t>(k * 2 + 1) * TR;
#pragma unroll
              for (int q = 0; q < RW; ++q) scale[u * RW + q] = (rr + q < rows_u[u]) ? vold[rr + q] : 0.f;
            }
          } else {
            float p[RT];
#pragma unroll
            for (int x = 0; x < RT; ++x) {
              float d0 = 0.f, d1 = 0.f;
#pragma unroll
              for (int j = 0; j < C; ++j) {
                float4 tv;
                if (kTsmem) {
                  tv = *reinterpret_cast<const float4*>(&s_t[kTsmem ? k : 0][4 * lane + 128 * j]);
                } else {
                  tv = make_float4(t[kTsmem ? 0 : k][j][0], t[kTsmem ? 0 : k][j][1],
                                   t[kTsmem ? 0 : k][j][2], t[kTsmem ? 0 : k][j][3]);
                }
                d0 = fmaf(f[x][j].x, tv.x, d0);
                d1 = fmaf(f[x][j].y, tv.y, d1);
                d0 = fmaf(f[x][j].z, tv.z, d0);
                d1 = fmaf(f[x][j].w, tv.w, d1);
              }
              p[x] = d0 + d1;
            }
            const float dot = fold_rows<RT>(p, lane, OpAdd());
            float sc = 0.f;
            if (mvalid) {
              const float* vw = vbase_m + static_cast<size_t>(k * 2) * TR;
              const float* vold = vw + TR;
              const float wi = vw[mrow];
              if (has_old[k] && owner)
                racc[k].add(fabsf(fmaf(vold[mrow], dot, -wi)));
              if (MODE == kPassUpdate) {
                sc = wi * __frcp_rn(dot);
                if (owner) {
                  a.rhs[k].out[row0_m + mrow] = sc;
                  if (!(dot > 0.f) || !isfinite(sc)) flag |= LSF_ERR_NONFINITE;
                }
              }
            }
#pragma unroll
            for (int x = 0; x < RT; ++x) scale[x] = __shfl_sync(0xffffffffu, sc, x << SH);
          }
          if (kAcc) {
#pragma unroll
            for (int x = 0; x < RT; ++x)
#pragma unroll
              for (int j = 0; j < C; ++j) {
                acc[k][j][0] = fmaf(scale[x], f[x][j].x, acc[k][j][0]);
                acc[k][j][1] = fmaf(scale[x], f[x][j].y, acc[k][j][1]);
                acc[k][j][2] = fmaf(scale[x], f[x][j].z, acc[k][j][2]);
                acc[k][j][3] = fmaf(scale[x], f[x][j].w, acc[k][j][3]);
              }
          }
        }
      }
      __syncwarp();
      if (lane == 0)
        for (int u = 0; u < nt; ++u) mbar_arrive(&ring.empty[(it + u) % S]);
      it += nt;
    }
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      double r = static_cast<double>(racc[k].s) + static_cast<double>(racc[k].c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      res[k] = r;
    }
  }
  // All tiles are consumed and every copy has landed: shared memory is free.
  __syncthreads();
  float* red = ring.sF;  // [kConsumerWarps][NRHS][ldr]
  if (warp < kConsumerWarps) {
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
  finish_pass<NRHS, kAcc>(red, kConsumerWarps, &s_res[0][0], ldr, a.rhs, a.part, a.gpart, a.rpart,
                          a.counter, a.status, s_flag, &s_last);
}

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

template <int NRHS>
int launch_nrhs(int mode, const PassArgs& a, unsigned grid, size_t smem, cudaStream_t st) {
  switch (pass_columns(a.ldr)) {
    case 1: return launch_c_nrhs<1, NRHS>(mode, a, grid, smem, st);
    case 2: return launch_c_nrhs<2, NRHS>(mode, a, grid, smem, st);
    case 4: return launch_c_nrhs<4, NRHS>(mode, a, grid, smem, st);
    default: return launch_c_nrhs<8, NRHS>(mode, a, grid, smem, st);
  }
}

int g_tile_bytes = 44 * 1024;
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
  if (mode == kPassRows) per_row += nrhs * 4.0;                                // out
  if (mode == kPassRowsAxpy) per_row += nrhs * 8.0;                            // out, given scaling
  return per_row * static_cast<double>(n);
}

int pass_columns(int ldr) {
  const int c = (ldr + 127) / 128;
  return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : 8;
}

int plan_pass(PassArgs& a, int nrhs, int red_floats_per_warp_rhs, size_t* smem_out,
              unsigned* grid_out) {
  const DeviceInfo& dev = device_info();
  if (a.n < 1) return fail(LSF_ERR_ARG, "pass: n must be >= 1");
  if (a.ldr < 4 || a.ldr % 4 != 0 || a.ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "pass: ldr must be a multiple of 4 in [4, 1024]");
  if (reinterpret_cast<uintptr_t>(a.F) % 16 != 0)
    return fail(LSF_ERR_ARG, "pass: features must be 16-byte aligned");
  const int64_t row_bytes = 4LL * a.ldr;
  const int RW = 8 / pass_columns(a.ldr);
  // Tile: whole row groups (RW rows) for every consumer warp, about g_tile_bytes,
  // but small enough to give every SM work.
  const int64_t unit = static_cast<int64_t>(RW) * kConsumerWarps;
  int64_t tr = std::max<int64_t>(unit, (g_tile_bytes / row_bytes) / unit * unit);
  const int64_t want_tiles = 2LL * dev.sms;
  if ((a.n + tr - 1) / tr < want_tiles) {
    tr = std::max<int64_t>(1, (a.n + want_tiles - 1) / want_tiles);
    if (tr > RW) tr = (tr + RW - 1) / RW * RW;
  }
  tr = std::min<int64_t>(tr, 1024);
  a.tile_rows = static_cast<int>(tr);
  a.ntiles = (a.n + tr - 1) / tr;
  const size_t stage_bytes = static_cast<size_t>(tr * row_bytes) + static_cast<size_t>(nrhs) * 2 * tr * 4;
  const size_t static_smem = 12 * 1024;  // t copies, residuals, flags, with margin
  const size_t budget = static_cast<size_t>(dev.smem_optin) - static_smem;
  const size_t bars = 128 * ((16 * static_cast<size_t>(g_max_stages) + 127) / 128);
  int S = static_cast<int>(std::min<size_t>(static_cast<size_t>(g_max_stages), (budget - bars) / stage_bytes));
  if (S < 2) return fail(LSF_ERR_UNSUPPORTED, "pass: tile does not fit in shared memory");
  a.nstages = S;
  size_t smem = ring_bytes(S, tr, a.ldr, nrhs);
  const size_t red_bytes = 128 * ((16 * S + 127) / 128) +
                           static_cast<size_t>(kConsumerWarps) * nrhs * red_floats_per_warp_rhs * 4;
  smem = std::max(smem, red_bytes);
  if (smem > budget) return fail(LSF_ERR_UNSUPPORTED, "pass: shared memory over budget");
  *smem_out = smem;
  *grid_out = static_cast<unsigned>(std::min<int64_t>(std::min(dev.sms, max_pass_ctas()), a.ntiles));
  return LSF_OK;
}

int launch_pass(int mode, int nrhs, PassArgs a, cudaStream_t st) {
  size_t smem = 0;
  unsigned grid = 0;
  int rc = plan_pass(a, nrhs, a.ldr, &smem, &grid);
  if (rc != LSF_OK) return rc;
  bool with_old = false;
  for (int k = 0; k < nrhs; ++k) with_old |= a.rhs[k].old != nullptr;
  LaunchScope ls(st, LSF_KERNEL_PASS, pass_bytes(mode, nrhs, a.n, a.ldr, with_old));
  if (nrhs == 1) return launch_nrhs<1>(mode, a, grid, smem, st);
  return launch_nrhs<2>(mode, a, grid, smem, st);
}

}  // namespace lsf
