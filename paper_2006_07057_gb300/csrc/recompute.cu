// Fused Sinkhorn pass that recomputes the shifted features in registers.
//
// Instead of streaming a stored n x r feature matrix, each entry is rebuilt
// from the points and the anchors in the log2 domain:
//   log2 F_ik = A_k + B_i + sum_d x_id W_kd,
//   A_k = log2(e) (c_k - (2/eps)||u_k||^2),  W_kd = log2(e) (4/eps) u_kd,
//   B_i = -log2(e) ((2/eps)||x_i||^2 + shift_i),
// (the expansion of c_k - (2/eps)||x_i - u_k||^2 - shift_i, Lemma 1), then one
// hardware ex2 per entry, shared by the row product and the transposed
// accumulation of the same pass. HBM traffic drops to the points and vectors;
// the bound becomes instruction issue. The FP32 arithmetic runs on column pairs
// with the packed two-lane instructions (fma/add/mul .f32x2): a thread's four
// columns are two pairs, so the exponent's affine form, the row products and the
// transposed accumulation take half the instructions of scalar code.
//
// Layout: 8 compute warps and one service warp. A row group of GW compute warps
// covers a row, each thread holding four consecutive feature columns (their
// A_k and W_kd stay in registers for the whole launch). A batch gives every
// group 8 rows. A warp folds its 8 row products with the multi-row butterfly (9
// shuffles) and writes them to shared memory; after one barrier every compute
// warp of the group sums the group's partials for the 8 rows in the same fixed
// order and forms the new scalings itself, so no warp waits for another to
// finish a row. The side work of a batch (loading the rows' records three
// batches ahead and packing them two ahead, writing the new scalings, the
// residual terms and the status)
// belongs to the service warp, so the compute warps carry identical
// instruction streams and meet at the barrier together (done by one of them,
// that work made the other seven wait at every barrier). One barrier per batch
// suffices: the partials are double-buffered, and the rows' records (x, B,
// weights, previous scalings; float4-packed) go through a three-deep ring.
#include <cuda_runtime.h>

#include <algorithm>

#include "recompute.cuh"
#include "reduce.cuh"
#include "ring.cuh"

namespace lsf {
namespace {

constexpr int kRcWarps = 8;                      // compute warps
constexpr int kRcThreads = (kRcWarps + 1) * 32;  // + the service warp
constexpr int kRcRB = 8;  // rows per group per batch

// FIXED: the update pass without previous scalings at ldr = 1024 (every pass of
// the solvers' loops on the large workload), compiled with the mode and the
// row stride fixed.
template <int GW, int D, int NRHS, bool FIXED = false>
__global__ void __launch_bounds__(kRcThreads, D <= 4 ? 2 : 1)
    recompute_kernel(const RecomputeArgs a, const int mode_in) {
  const int mode = FIXED ? static_cast<int>(kPassUpdate) : mode_in;
  constexpr int NG = kRcWarps / GW;         // row groups per CTA
  constexpr int RPB = NG * kRcRB;           // rows per batch
  constexpr int TPG = GW * 32;              // threads per group
  constexpr int XV = RowPack<D>::kXV;
  constexpr int SV = RowPack<D>::kSV;
  constexpr int kItems = NG * NRHS * kRcRB;  // (group, rhs, row) records per batch
  __shared__ __align__(16) float4 s_rows[3][RPB * SV];
  __shared__ __align__(16) float s_red[2][NRHS][kRcRB][kRcWarps];  // per-warp partial row products
  __shared__ double s_res[kRcWarps + 1][2];
  __shared__ int s_flag, s_last, s_skip;
  extern __shared__ __align__(16) float s_part[];  // [NG][NRHS * ldr] at the end

  const bool kUpd = mode == kPassUpdate, kAx = mode == kPassAxpy, kDt = mode == kPassDot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool service = warp == kRcWarps;
  const int g = service ? 0 : warp / GW;    // my group
  const int tg = tid - g * TPG;             // my thread index inside the group
  const int ldr = FIXED ? 1024 : a.ldr, d = a.d;
  const int col0 = 4 * tg;                  // my four columns

  if (tid == 0) {
    s_flag = 0;
    // a run that already produced a non-finite scaling is void (repeated in the
    // log domain): process no rows, but take part in the cross-CTA reduction
    s_skip = (*reinterpret_cast<volatile int*>(a.status) & LSF_ERR_NONFINITE) != 0;
  }
  __syncthreads();
  const int64_t nbatch = s_skip ? 0 : (a.n + RPB - 1) / RPB;
  double res[NRHS];
  float2 acc2[NRHS][2];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    res[k] = 0.0;
    acc2[k][0] = acc2[k][1] = make_float2(0.f, 0.f);
  }
  int flag = 0;

  if (service) {
    // ---- service warp: row records in, scalings out ----
    bool has_old[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) has_old[k] = !FIXED && a.rhs[k].old != nullptr;
    // Each lane serves one right-hand side (items in steps of 32 with kRcRB = 8)
    // and sums the residual terms |old s - w| of its rows: each term in one
    // rounding (a fused multiply-add), the sum compensated in FP32, widened once
    // at the end (no FP64 arithmetic per batch).
    const int kq_lane = (lane / kRcRB) % NRHS;
    const bool lane_old = kq_lane == 0 ? has_old[0] : has_old[NRHS - 1];
    CompSum racc;
    constexpr int kPer = (RPB + 31) / 32;  // rows per lane
    // A row's raw record (x, shift, weights, previous scalings) is loaded two
    // batches before its batch and only turned into the packed record (x
    // doubled, B = -log2(e) ((2/eps)||x||^2 + shift)) when it is parked in shared
    // memory, so the service warp does not wait for the loads before a barrier.
    struct Raw {
      float x[D];
      float sh;
      float w[NRHS];
      float o[NRHS];
    };
    Raw ra[kPer], rb[kPer];
    auto load_raw = [&](int64_t b, Raw (&r)[kPer]) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int64_t i = b * RPB + lane + 32 * u;
        const bool ok = b < nbatch && i < a.n;
#pragma unroll
        for (int dd = 0; dd < D; ++dd) r[u].x[dd] = (ok && dd < d) ? a.X[i * d + dd] : 0.f;
        r[u].sh = ok ? a.shift[i] : INFINITY;  // rows past the end: B = -inf, no mass
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          r[u].w[k] = (ok && !kAx) ? a.rhs[k].w[i] : 0.f;
          r[u].o[k] = (ok && has_old[k]) ? a.rhs[k].old[i] : 0.f;
        }
      }
    };
    auto park_raw = [&](const Raw (&r)[kPer], int bf) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int rr = lane + 32 * u;
        float rec[4 * SV];
#pragma unroll
        for (int q = 0; q < 4 * SV; ++q) rec[q] = 0.f;
        float nrm = 0.f;
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
          rec[2 * dd] = rec[2 * dd + 1] = r[u].x[dd];
          nrm = fmaf(r[u].x[dd], r[u].x[dd], nrm);
        }
        rec[2 * D] = rec[2 * D + 1] = -kLog2e * (a.two_over_eps * nrm + r[u].sh);
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          rec[4 * XV + 2 * k] = r[u].w[k];
          rec[4 * XV + 2 * k + 1] = r[u].o[k];
        }
        if (rr < RPB)
#pragma unroll
          for (int v = 0; v < SV; ++v)
            s_rows[bf][rr * SV + v] = make_float4(rec[4 * v], rec[4 * v + 1], rec[4 * v + 2], rec[4 * v + 3]);
      }
    };
    // prime the ring with the first two batches; the third batch's raw records
    // are parked after the first barrier
    const int64_t G = gridDim.x;
    load_raw(blockIdx.x, ra);
    park_raw(ra, 0);
    load_raw(blockIdx.x + G, ra);
    park_raw(ra, 1);
    load_raw(blockIdx.x + 2 * G, ra);
    __syncthreads();
    // one batch: the raw records of batch b + 3G load into `ld` (waited for two
    // batches later), the records of batch b + 2G (in `pk`) are parked
    auto step = [&](int64_t b, int it, Raw (&ld)[kPer], const Raw (&pk)[kPer]) {
      load_raw(b + 3 * G, ld);
      __syncthreads();
      if (!kAx) {
        // the batch's records: row sums from the group partials (the same fixed
        // order the compute warps use), new scalings, residual terms, status
        const float4* rows = s_rows[it % 3];
        const int64_t row0 = b * RPB;
#pragma unroll
        for (int item0 = 0; item0 < kItems; item0 += 32) {
          const int item = item0 + lane;
          if (item < kItems) {
            const int gg = item / (NRHS * kRcRB), kq = (item / kRcRB) % NRHS, qq = item % kRcRB;
            const int64_t i = row0 + gg * kRcRB + qq;
            if (i < a.n) {
              const float s = sum_partials<GW>(&s_red[it & 1][kq][qq][gg * GW]);
              const float4 wo = rows[(gg * kRcRB + qq) * SV + XV];
              const bool k0 = NRHS == 1 || kq == 0;
              const float w = k0 ? wo.x : wo.z, o = k0 ? wo.y : wo.w;
              if (lane_old) racc.add(fabsf(fmaf(o, s, -w)));
              if (kUpd) {
                const float sc = w * __frcp_rn(s);
                (k0 ? a.rhs[0].out : a.rhs[NRHS - 1].out)[i] = sc;
                if (!(s > 0.f) || !isfinite(sc)) flag |= LSF_ERR_NONFINITE;
              }
            }
          }
        }
      }
      // the batch two ahead goes to the slot the compute warps last read in the
      // previous batch (before this barrier)
      park_raw(pk, (it + 2) % 3);
    };
    int it = 0;
    for (int64_t b = blockIdx.x; b < nbatch;) {
      step(b, it, rb, ra);
      b += G;
      ++it;
      if (b >= nbatch) break;
      step(b, it, ra, rb);
      b += G;
      ++it;
    }
#pragma unroll
    for (int k = 0; k < NRHS; ++k)
      res[k] = kq_lane == k ? static_cast<double>(racc.s) + static_cast<double>(racc.c) : 0.0;
  } else {
    // ---- compute warps ----
    // per-column constants, as column pairs (col0, col0 + 1), (col0 + 2, col0 + 3)
    float2 A2[2], W2[2][D];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float Ap[2], Wp[2][D];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = col0 + 2 * p + h;
        if (k < a.r) {
          float nrm = 0.f;
#pragma unroll
          for (int dd = 0; dd < D; ++dd) {
            const float u = (dd < d) ? a.U[static_cast<int64_t>(k) * d + dd] : 0.f;
            nrm = fmaf(u, u, nrm);
            Wp[h][dd] = kLog2e * (2.f * a.two_over_eps) * u;
          }
          Ap[h] = kLog2e * (a.c[k] - a.two_over_eps * nrm);
        } else {
#pragma unroll
          for (int dd = 0; dd < D; ++dd) Wp[h][dd] = 0.f;
          Ap[h] = -INFINITY;  // ex2(-inf) = 0: padded columns carry no mass
        }
      }
      A2[p] = make_float2(Ap[0], Ap[1]);
#pragma unroll
      for (int dd = 0; dd < D; ++dd) W2[p][dd] = make_float2(Wp[0][dd], Wp[1][dd]);
    }
    float2 t2[NRHS][2];
#pragma unroll
    for (int k = 0; k < NRHS; ++k)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int c = col0 + 2 * p;
        t2[k][p] = make_float2((!kAx && c < ldr) ? a.rhs[k].t_in[c] : 0.f,
                               (!kAx && c + 1 < ldr) ? a.rhs[k].t_in[c + 1] : 0.f);
      }
    __syncthreads();  // the ring is primed
    int it = 0;
    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x, ++it) {
      const float4* rows = s_rows[it % 3];
      float2 F[kRcRB][2];  // the row's four entries as two column pairs
      float dots[NRHS][kRcRB];
#pragma unroll
      for (int q = 0; q < kRcRB; ++q) {
        const float4* rw = rows + (g * kRcRB + q) * SV;
        float2 xb[2 * XV];  // (x_dd, x_dd) for dd < D, then (B, B)
#pragma unroll
        for (int v = 0; v < XV; ++v) {
          const float4 f4 = rw[v];
          xb[2 * v] = make_float2(f4.x, f4.y);
          xb[2 * v + 1] = make_float2(f4.z, f4.w);
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          float2 E = __fadd2_rn(A2[p], xb[D]);
#pragma unroll
          for (int dd = 0; dd < D; ++dd) E = __ffma2_rn(xb[dd], W2[p][dd], E);
          F[q][p] = make_float2(ex2_approx(E.x), ex2_approx(E.y));
        }
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          const float2 P = __ffma2_rn(F[q][0], t2[k][0], __fmul2_rn(F[q][1], t2[k][1]));
          dots[k][q] = P.x + P.y;
        }
      }
      if (!kAx) {
        // warp partials of the 8 rows: lanes 4q .. 4q + 3 hold row q after the fold
        float v[NRHS];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) v[k] = fold_rows<kRcRB>(dots[k], lane, OpAdd());
        if ((lane & 3) == 0)
#pragma unroll
          for (int k = 0; k < NRHS; ++k) s_red[it & 1][k][lane >> 2][warp] = v[k];
      }
      __syncthreads();
      if (kDt) continue;
      float sc[NRHS][kRcRB];
      if (kAx) {
#pragma unroll
        for (int qq = 0; qq < kRcRB; ++qq) {
          const float4 wo = rows[(g * kRcRB + qq) * SV + XV];
          sc[0][qq] = wo.y;
          if (NRHS > 1) sc[NRHS - 1][qq] = wo.w;
        }
      } else {
        // lane (kq, qq) forms the scaling of row qq of rhs kq from the group's
        // partials, in the order the service warp uses
        const int kq = lane >> 3, qq = lane & 7;
        float scl = 0.f;  // rows past the end: 0 (their weight over their zero sum is NaN)
        if (kq < NRHS && b * RPB + g * kRcRB + qq < a.n) {
          const float s = sum_partials<GW>(&s_red[it & 1][kq][qq][g * GW]);
          const float4 wo = rows[(g * kRcRB + qq) * SV + XV];
          scl = ((NRHS == 1 || kq == 0) ? wo.x : wo.z) * __frcp_rn(s);
        }
#pragma unroll
        for (int k = 0; k < NRHS; ++k)
#pragma unroll
          for (int r8 = 0; r8 < kRcRB; ++r8) sc[k][r8] = __shfl_sync(0xffffffffu, scl, k * 8 + r8);
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k)
#pragma unroll
        for (int qq = 0; qq < kRcRB; ++qq) {
          const float2 s2 = make_float2(sc[k][qq], sc[k][qq]);
#pragma unroll
          for (int p = 0; p < 2; ++p) acc2[k][p] = __ffma2_rn(s2, F[qq][p], acc2[k][p]);
        }
    }
  }

  // partials: group g writes its columns into s_part[g][k][col]
  if (!kDt && !service) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = col0 + e;
        const float v = (e & 1) ? acc2[k][e >> 1].y : acc2[k][e >> 1].x;
        if (col < ldr) s_part[static_cast<size_t>(g) * NRHS * ldr + k * ldr + col] = v;
      }
  }
  // residual terms live in the service warp: per-warp sums, then all warps into
  // slot 0 in order (the other slots zero)
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    double r = res[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s_res[warp][k] = r;
  }
  if (flag) atomicOr(&s_flag, flag);
  __syncthreads();
  if (tid == 0) {
    for (int k = 0; k < NRHS; ++k) {
      double r = 0.0;
      for (int w = 0; w <= kRcWarps; ++w) r += s_res[w][k];
      s_res[0][k] = r;
      for (int w = 1; w <= kRcWarps; ++w) s_res[w][k] = 0.0;
    }
  }
  __syncthreads();
  if (kDt)
    finish_pass<NRHS, false>(s_part, NG, &s_res[0][0], ldr, a.rhs, a.part, a.gpart, a.rpart, a.counter,
                             a.status, s_flag, &s_last);
  else
    finish_pass<NRHS, true>(s_part, NG, &s_res[0][0], ldr, a.rhs, a.part, a.gpart, a.rpart, a.counter,
                            a.status, s_flag, &s_last);
}

template <int GW, int D, int NRHS>
int launch_gdn(int mode, const RecomputeArgs& a, cudaStream_t st) {
  constexpr int NG = kRcWarps / GW;
  const size_t smem = sizeof(float) * static_cast<size_t>(NG) * NRHS * a.ldr;
  auto kern = recompute_kernel<GW, D, NRHS>;
  if constexpr (GW == 8 && D <= 4) {
    bool old = false;
    for (int k = 0; k < NRHS; ++k) old = old || a.rhs[k].old != nullptr;
    if (mode == kPassUpdate && !old && a.ldr == 1024) kern = recompute_kernel<GW, D, NRHS, true>;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "recompute: smem attribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRcThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t rpb = NG * kRcRB;
  const int64_t nbatch = (a.n + rpb - 1) / rpb;
  // one workspace partial slot per CTA: never more CTAs than the workspace holds
  const int64_t cap = std::min<int64_t>(static_cast<int64_t>(device_info().sms) * per_sm, max_pass_ctas());
  const int64_t grid = std::min<int64_t>(cap, nbatch);
  kern<<<static_cast<unsigned>(grid), kRcThreads, smem, st>>>(a, mode);
  return check_launch("recompute_kernel");
}

template <int GW, int NRHS>
int launch_gn(int mode, const RecomputeArgs& a, int Dp, cudaStream_t st) {
  switch (Dp) {
    case 2: return launch_gdn<GW, 2, NRHS>(mode, a, st);
    case 3: return launch_gdn<GW, 3, NRHS>(mode, a, st);
    case 4: return launch_gdn<GW, 4, NRHS>(mode, a, st);
    case 8: return launch_gdn<GW, 8, NRHS>(mode, a, st);
    default: return launch_gdn<GW, 16, NRHS>(mode, a, st);
  }
}

template <int NRHS>
int launch_n(int mode, const RecomputeArgs& a, int GW, int Dp, cudaStream_t st) {
  switch (GW) {
    case 1: return launch_gn<1, NRHS>(mode, a, Dp, st);
    case 2: return launch_gn<2, NRHS>(mode, a, Dp, st);
    case 4: return launch_gn<4, NRHS>(mode, a, Dp, st);
    default: return launch_gn<8, NRHS>(mode, a, Dp, st);
  }
}

}  // namespace

int launch_recompute_pass(int mode, int nrhs, RecomputeArgs a, cudaStream_t st) {
  if (a.n < 1) return fail(LSF_ERR_ARG, "recompute: n must be >= 1");
  if (a.d < 1 || a.d > 16)
    return fail(LSF_ERR_UNSUPPORTED, "recompute mode handles 1 <= d <= 16 (stored mode otherwise)");
  if (a.ldr < 4 || a.ldr % 4 != 0 || a.ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "recompute: ldr must be a multiple of 4 in [4, 1024]");
  if (!a.X || !a.U || !a.c || !a.shift) return fail(LSF_ERR_ARG, "recompute: NULL argument");
  int quads = (a.ldr + 3) / 4;
  int qpr = 32;
  while (qpr < quads) qpr *= 2;
  const int GW = qpr / 32;  // 1, 2, 4 or 8 warps per row
  const int Dp = a.d <= 2 ? 2 : a.d <= 3 ? 3 : a.d <= 4 ? 4 : a.d <= 8 ? 8 : 16;
  double bytes = 4.0 * a.n * (a.d + 1) + 4.0 * a.n * nrhs * 3.0;
  LaunchScope ls(st, LSF_KERNEL_PASS_RECOMPUTE, bytes);
  if (nrhs == 1) return launch_n<1>(mode, a, GW, Dp, st);
  return launch_n<2>(mode, a, GW, Dp, st);
}

}  // namespace lsf
