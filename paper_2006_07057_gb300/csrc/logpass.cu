// Log-domain fused Sinkhorn pass (stabilised variant).
//
// The same half iteration of Alg. 1 as the stored-feature pass, on the log form
// of everything, for problems whose features or scalings leave the FP32 range:
//   stored rows  L~_ik = log phi_theta(x_i)_k - shift_i   (<= 0, padding -inf)
//   r-vector     lt_k  = log t_k                          (padding -inf)
//   scaling      f_i   = log u~_i
// The row product becomes log s_i = LSE_k(L~_ik + lt_k), the division
// f_i = log w_i - log s_i, and the transposed product
// lt'_k = LSE_i(L~_ik + f_i). Every log-sum-exp is shifted by its maximum, so no
// term under- or overflows.
//
// Layout is that of the stored pass (same copy ring; a warp takes RW = 8/C rows at
// full width): the RW row maxima and then the shifted row sums are folded across
// the warp by the multi-row butterfly; the column side keeps a running (max, sum)
// pair per column, updated online as m' = max(m, y), s' = s e^(m - m') +
// e^(y - m') (two exponentials and no branch: one of the two is exactly 1, so
// this equals the one-exponential update with a branch on the sign of y - m, in
// fewer instructions), and warps then CTAs are merged in a fixed order at the
// end. Every exponent is a difference taken in natural units before the scaling
// by log2(e) (exact near the maximum), so no rounding is shared by all the terms
// of a sum. The FP32 arithmetic runs on column pairs with the packed two-lane
// instructions (add/mul/fma .f32x2). A two right-hand-side pass at C >= 4 runs as
// two one-RHS launches: two (max, sum) states per column would not fit in
// registers, and the pass is bound by ex2, not by the second read of F.
#include <cuda_runtime.h>

#include "reduce.cuh"
#include "ring.cuh"

namespace lsf {
namespace {

// EXACT: ldr = 128 C (no padded columns), so no column needs a bounds test.
// NOOLD: no right-hand side carries previous scalings (no residual terms).
template <int C, int NRHS, int MODE, bool EXACT = false, bool NOOLD = false>
__global__ void __launch_bounds__(kPassThreads, 1) logpass_kernel(const PassArgs a) {
  constexpr int RW = 8 / C;
  constexpr int SH = RowFold<RW>::kShift;
  constexpr bool kNeedT = MODE != kPassAxpy;
  constexpr bool kAcc = MODE != kPassDot && MODE != kPassRows;
  constexpr bool kRowsOut = MODE == kPassRows || MODE == kPassRowsAxpy;  // log s to `out`
  constexpr bool kGivenF = MODE == kPassAxpy || MODE == kPassRowsAxpy;   // column side from `old`
  extern __shared__ __align__(128) unsigned char smem[];
  const int ldr = a.ldr;
  const Ring ring = ring_layout(smem, a.nstages, a.tile_rows, ldr);
  const int S = ring.S;
  const int TR = ring.TR;

  __shared__ __align__(16) float s_lt[NRHS][128 * C];  // log t (padding -inf)
  __shared__ double s_res[kConsumerWarps][2];
  __shared__ int s_flag;
  __shared__ int s_last;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    ring_init(ring, kConsumerWarps);
    fence_mbarrier_init();
    s_flag = 0;
  }
  for (int idx = threadIdx.x; idx < NRHS * 128 * C; idx += blockDim.x) {
    const int k = idx / (128 * C), c = idx - k * 128 * C;
    s_lt[k][c] = (kNeedT && c < ldr) ? a.rhs[k].t_in[c] : -INFINITY;
  }
  __syncthreads();

  int flag = 0;
  // running column (max, sum), as column pairs
  float2 lm[NRHS][C][2], ls[NRHS][C][2];
  double res[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    res[k] = 0.0;
#pragma unroll
    for (int j = 0; j < C; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        lm[k][j][h] = make_float2(kLogFloor, kLogFloor);
        ls[k][j][h] = make_float2(0.f, 0.f);
      }
  }
  const float2 kL2 = make_float2(kLog2e, kLog2e);
  const float2 kNeg1 = make_float2(-1.f, -1.f);
  if (warp == kConsumerWarps) {
    ring_produce<NRHS>(ring, a.F, a.n, a.ntiles, a.rhs, MODE == kPassUpdate || MODE == kPassDot, lane, flag);
  } else {
    bool has_old[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) has_old[k] = !NOOLD && a.rhs[k].old != nullptr;
    const int myq = (lane >> SH) & (RW - 1);
    const bool owner = (lane & ((1 << SH) - 1)) == 0;

    int it = 0;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
      const int s = it % S;
      if (!ring_wait_full(ring, it, lane)) {
        flag |= LSF_ERR_TIMEOUT;
        break;
      }
      const int64_t row0 = tile * TR;
      const int rows = static_cast<int>(min(static_cast<int64_t>(TR), a.n - row0));
      const float* tF = ring.sF + static_cast<size_t>(s) * TR * ldr;
      for (int rr = warp * RW; rr < rows; rr += RW * kConsumerWarps) {
        float4 f[RW][C];
#pragma unroll
        for (int q = 0; q < RW; ++q)
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            f[q][j] = ((RW == 1 || rr + q < rows) && (EXACT || col < ldr))
                          ? *reinterpret_cast<const float4*>(tF + static_cast<size_t>(rr + q) * ldr + col)
                          : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
          }
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          const float* vw = ring.sV + static_cast<size_t>((s * NRHS + k) * 2) * TR;
          const float* vold = vw + TR;
          float fq[RW];  // the RW rows' log scalings
          if (MODE == kPassAxpy) {
#pragma unroll
            for (int q = 0; q < RW; ++q) fq[q] = (rr + q < rows) ? vold[rr + q] : -INFINITY;
          } else {
            float p[RW];
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              float m = -INFINITY;
#pragma unroll
              for (int j = 0; j < C; ++j) {
                const float4 lt = *reinterpret_cast<const float4*>(&s_lt[k][4 * lane + 128 * j]);
                const float2 y0 = __fadd2_rn(make_float2(f[q][j].x, f[q][j].y), make_float2(lt.x, lt.y));
                const float2 y1 = __fadd2_rn(make_float2(f[q][j].z, f[q][j].w), make_float2(lt.z, lt.w));
                m = fmaxf(m, fmaxf(fmaxf(y0.x, y0.y), fmaxf(y1.x, y1.y)));
              }
              p[q] = m;
            }
            const float mrow = fold_rows<RW>(p, lane, OpMax());
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              const float mq = __shfl_sync(0xffffffffu, mrow, q << SH);
              const float2 nm = make_float2(-mq, -mq);
              float2 sum = make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < C; ++j) {
                const float4 lt = *reinterpret_cast<const float4*>(&s_lt[k][4 * lane + 128 * j]);
                const float2 y0 = __fadd2_rn(make_float2(f[q][j].x, f[q][j].y), make_float2(lt.x, lt.y));
                const float2 y1 = __fadd2_rn(make_float2(f[q][j].z, f[q][j].w), make_float2(lt.z, lt.w));
                const float2 e0 = __fmul2_rn(__fadd2_rn(y0, nm), kL2);
                const float2 e1 = __fmul2_rn(__fadd2_rn(y1, nm), kL2);
                sum = __fadd2_rn(sum, make_float2(ex2_approx(e0.x), ex2_approx(e0.y)));
                sum = __fadd2_rn(sum, make_float2(ex2_approx(e1.x), ex2_approx(e1.y)));
              }
              p[q] = sum.x + sum.y;
            }
            const float srow = fold_rows<RW>(p, lane, OpAdd());
            const int row = rr + myq;
            float fi = -INFINITY;
            if (kRowsOut) {
              if (row < rows && owner) a.rhs[k].out[row0 + row] = mrow + logf(srow);
            } else if (row < rows) {
              const float logs = mrow + logf(srow);
              const float wi = vw[row];
              if (has_old[k] && owner)
                res[k] += fabs(exp(static_cast<double>(vold[row]) + static_cast<double>(logs)) -
                               static_cast<double>(wi));
              if (MODE == kPassUpdate) {
                fi = logf(wi) - logs;
                if (owner) {
                  a.rhs[k].out[row0 + row] = fi;
                  if (!isfinite(fi)) flag |= LSF_ERR_NONFINITE;
                }
                if (!isfinite(fi)) fi = -INFINITY;
              }
            }
            if (kGivenF) {
#pragma unroll
              for (int q = 0; q < RW; ++q) fq[q] = (rr + q < rows) ? vold[rr + q] : -INFINITY;
            } else {
#pragma unroll
              for (int q = 0; q < RW; ++q) fq[q] = __shfl_sync(0xffffffffu, fi, q << SH);
            }
          }
          if (kAcc) {
            // column side: online (max, sum) per column
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              const float2 fq2 = make_float2(fq[q], fq[q]);
#pragma unroll
              for (int j = 0; j < C; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const float2 fp = h ? make_float2(f[q][j].z, f[q][j].w) : make_float2(f[q][j].x, f[q][j].y);
                  const float2 y = __fadd2_rn(fp, fq2);
                  float2& m = lm[k][j][h];
                  const float2 mn = make_float2(fmaxf(m.x, y.x), fmaxf(m.y, y.y));
                  // m - m' and y - m' (one of them is 0), in log2 units
                  const float2 a1 = __fmul2_rn(__ffma2_rn(mn, kNeg1, m), kL2);
                  const float2 a2 = __fmul2_rn(__ffma2_rn(mn, kNeg1, y), kL2);
                  ls[k][j][h] = __ffma2_rn(ls[k][j][h], make_float2(ex2_approx(a1.x), ex2_approx(a1.y)),
                                           make_float2(ex2_approx(a2.x), ex2_approx(a2.y)));
                  m = mn;
                }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ring.empty[s]);
    }
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      double r = res[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      res[k] = r;
    }
  }
  __syncthreads();
  float* red = ring.sF;  // [kConsumerWarps][NRHS][2][ldr]
  if (warp < kConsumerWarps) {
    if (kAcc) {
#pragma unroll
      for (int k = 0; k < NRHS; ++k)
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = 4 * lane + 128 * j;
          if (EXACT || col < ldr) {
            float* rg = red + (static_cast<size_t>(warp) * NRHS + k) * 2 * ldr;
            *reinterpret_cast<float4*>(rg + col) =
                make_float4(lm[k][j][0].x, lm[k][j][0].y, lm[k][j][1].x, lm[k][j][1].y);
            *reinterpret_cast<float4*>(rg + ldr + col) =
                make_float4(ls[k][j][0].x, ls[k][j][0].y, ls[k][j][1].x, ls[k][j][1].y);
          }
        }
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) s_res[warp][k] = res[k];
  }
  if (flag) atomicOr(&s_flag, flag);
  __syncthreads();
  finish_pass_log<NRHS, kAcc>(red, kConsumerWarps, &s_res[0][0], ldr, a.rhs, a.part, a.gpart, a.rpart,
                              a.counter, a.status, s_flag, &s_last);
}

template <int C, int NRHS>
int launch_log_c_nrhs(int mode, const PassArgs& a, unsigned grid, size_t smem, cudaStream_t st) {
  void (*kern)(PassArgs) = nullptr;
  // (at C = 8 the unpredicated loads raise the register need past the file: spills)
  bool noold = true;
  for (int k = 0; k < NRHS; ++k) noold = noold && a.rhs[k].old == nullptr;
  const bool exact = C <= 4 && a.ldr == 128 * C;
  // (NOOLD pays at C <= 4; at C = 8 it measured about 1 % slower)
  if (mode == kPassUpdate && noold && C <= 4)
    kern = exact ? logpass_kernel<C, NRHS, kPassUpdate, C <= 4, C <= 4>
                 : logpass_kernel<C, NRHS, kPassUpdate, false, C <= 4>;
  else if (mode == kPassUpdate && exact) kern = logpass_kernel<C, NRHS, kPassUpdate, C <= 4>;
  else if (mode == kPassUpdate) kern = logpass_kernel<C, NRHS, kPassUpdate>;
  else if (mode == kPassAxpy) kern = logpass_kernel<C, NRHS, kPassAxpy>;
  else if (mode == kPassDot) kern = logpass_kernel<C, NRHS, kPassDot>;
  else if constexpr (NRHS == 1) {
    if (mode == kPassRows) kern = logpass_kernel<C, 1, kPassRows>;
    else kern = logpass_kernel<C, 1, kPassRowsAxpy>;
  } else {
    return fail(LSF_ERR_UNSUPPORTED, "logpass: row-product modes take one right-hand side");
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "logpass: smem attribute: %s", cudaGetErrorString(e));
  kern<<<grid, kPassThreads, smem, st>>>(a);
  return check_launch("logpass_kernel");
}

template <int NRHS>
int launch_log_nrhs(int mode, const PassArgs& a, unsigned grid, size_t smem, cudaStream_t st) {
  const int c = pass_columns(a.ldr);
  if (c == 1) return launch_log_c_nrhs<1, NRHS>(mode, a, grid, smem, st);
  if (c == 2) return launch_log_c_nrhs<2, NRHS>(mode, a, grid, smem, st);
  if constexpr (NRHS == 1) {
    if (c == 4) return launch_log_c_nrhs<4, 1>(mode, a, grid, smem, st);
    return launch_log_c_nrhs<8, 1>(mode, a, grid, smem, st);
  } else {
    return fail(LSF_ERR_UNSUPPORTED, "logpass: two right-hand sides need ldr <= 256");
  }
}

}  // namespace

int launch_logpass(int mode, int nrhs, PassArgs a, cudaStream_t st) {
  size_t smem = 0;
  unsigned grid = 0;
  int rc = plan_pass(a, nrhs, 2 * a.ldr, &smem, &grid);
  if (rc != LSF_OK) return rc;
  bool with_old = false;
  for (int k = 0; k < nrhs; ++k) with_old |= a.rhs[k].old != nullptr;
  LaunchScope ls(st, LSF_KERNEL_PASS_LOG, pass_bytes(mode, nrhs, a.n, a.ldr, with_old));
  if (nrhs == 1) return launch_log_nrhs<1>(mode, a, grid, smem, st);
  if (pass_columns(a.ldr) >= 4) {
    for (int k = 0; k < 2; ++k) {
      PassArgs one = a;
      one.rhs[0] = a.rhs[k];
      one.rhs[1] = PassRhs{};
      size_t smem1 = 0;
      unsigned grid1 = 0;
      int rc1 = plan_pass(one, 1, 2 * a.ldr, &smem1, &grid1);
      if (rc1 != LSF_OK) return rc1;
      rc1 = launch_log_nrhs<1>(mode, one, grid1, smem1, st);
      if (rc1 != LSF_OK) return rc1;
    }
    return LSF_OK;
  }
  return launch_log_nrhs<2>(mode, a, grid, smem, st);
}

}  // namespace lsf
