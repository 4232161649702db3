// Fused Sinkhorn pass with the feature columns split between HBM and the ALUs.
//
// One half of Alg. 1 on K = xi zeta^T (Sec. 3.1) reads every shifted feature
// entry of one cloud once. The stored pass streams all of them from HBM
// (bandwidth-bound, the FP32 pipe mostly idle); the recompute pass rebuilds all
// of them in registers from the points and anchors (issue-bound, HBM idle). This
// pass does both at once: the first c0 columns of every row are rebuilt in
// registers exactly as the recompute pass does (one ex2 of the log2-domain
// exponent A_k + B_i + x_i . W_k, Lemma 1), and the remaining ldr - c0 columns
// are read from a stored block Fs (n x (ldr - c0), the same shifted features
// F = exp(L - shift) with the row shift taken over all ldr columns). Both halves
// feed the same row products, divisions and transposed products, so the
// iterates are those of Alg. 1; only the source of each entry differs.
//
// Layout: 4 compute warps and one service warp per CTA, three CTAs per SM (128
// registers a thread: 15 warps leave at most 4 on each of an SM's four
// sub-partitions, whose register files hold 4 x 32 x 128 each; a 9-warp CTA at
// more than 96 registers fits only once per SM). A row group of GW warps covers a
// row: thread tg of the group owns the recomputed columns 4tg..4tg+3 (when below
// c0) and the stored columns c0+4tg..c0+4tg+3 (when below ldr). A batch gives
// each group 8 rows. The service warp copies a
// batch's stored rows (one contiguous block of the stored matrix) into a
// three-slot shared-memory ring with one bulk copy, two batches ahead, on an
// mbarrier; the compute warps read their stored entries from shared memory twice
// (for the row products before the batch's barrier and for the transposed
// products after it) instead of holding them in registers across the barrier.
// The rest (row records, partial row products, one barrier per batch, scalings,
// residual terms, cross-CTA reduction) is the recompute pass's.
#include <cuda_runtime.h>

#include <algorithm>

#include "recompute.cuh"
#include "reduce.cuh"
#include "ring.cuh"

namespace lsf {
namespace {

constexpr int kHyWarps = 4;                      // compute warps
constexpr int kHyThreads = (kHyWarps + 1) * 32;  // + the service warp
constexpr int kHyRB = 8;                         // rows per group per batch
constexpr int kHySlots = 3;                      // stored-row ring depth
constexpr int kAhead = 6;                        // row records copied this many batches ahead

// FLDR = 0: any row stride and pass mode. FLDR > 0: the update pass over rows of
// exactly FLDR columns, compiled with the row stride, the column split and the
// mode fixed, and with every compute thread owning both a recomputed and a
// stored column quad (the configuration of the large workload, r = 1024).
template <int GW, int D, int NRHS, int FLDR>
__device__ __forceinline__ void hybrid_body(const HybridArgs& h, const int mode_in) {
  constexpr int NG = kHyWarps / GW;   // row groups per CTA
  constexpr int RPB = NG * kHyRB;     // rows per batch
  constexpr int TPG = GW * 32;        // threads per group
  static_assert(FLDR == 0 || (4 * TPG == hybrid_first_stored(FLDR) && 4 * TPG == FLDR - hybrid_first_stored(FLDR)),
                "the fixed-stride variant needs one column quad of each kind per thread");
  const int mode = FLDR > 0 ? static_cast<int>(kPassUpdate) : mode_in;
  constexpr int XV = RowPack<D>::kXV;
  constexpr int SV = RowPack<D>::kSV;
  constexpr int kItems = NG * NRHS * kHyRB;
  __shared__ __align__(16) float4 s_rows[3][RPB * SV];
  __shared__ __align__(16) float s_red[2][NRHS][kHyRB][kHyWarps];
  __shared__ double s_res[kHyWarps + 1][2];
  __shared__ __align__(8) uint64_t s_full[kHySlots];
  // row records in flight: [stage][row][x (D), shift, (w, old) per rhs]
  __shared__ float s_stage[kAhead][RPB][D + 1 + 2 * NRHS];
  __shared__ int s_flag, s_last, s_skip;
  // [kHySlots][RPB][lds] stored rows; after the last batch, the per-group
  // partial r-vectors [NG][NRHS * ldr]
  extern __shared__ __align__(128) float s_ring[];

  const RecomputeArgs& a = h.rc;
  const bool kUpd = mode == kPassUpdate, kAx = mode == kPassAxpy, kDt = mode == kPassDot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool service = warp == kHyWarps;
  const int g = (NG == 1 || service) ? 0 : warp / GW;
  const int tg = tid - g * TPG;
  const int ldr = FLDR > 0 ? FLDR : a.ldr, d = a.d;
  const int c0 = FLDR > 0 ? hybrid_first_stored(FLDR) : h.c0;
  const int lds = ldr - c0;       // stored columns per row
  const int col0 = 4 * tg;        // my recomputed columns (valid below c0)
  const bool has_rc = FLDR > 0 ? !service : col0 < c0;
  const bool has_st = FLDR > 0 ? !service : col0 < lds; // my stored columns c0 + col0 .. + 3

  if (tid == 0) {
    s_flag = 0;
    s_skip = (*reinterpret_cast<volatile int*>(a.status) & LSF_ERR_NONFINITE) != 0;
    for (int s = 0; s < kHySlots; ++s) mbar_init(&s_full[s], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  const int64_t nbatch = s_skip ? 0 : (a.n + RPB - 1) / RPB;
  double res[NRHS];
  float2 acc2[NRHS][2];
  float4 accs[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) {
    res[k] = 0.0;
    acc2[k][0] = acc2[k][1] = make_float2(0.f, 0.f);
    accs[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int flag = 0;

  if (service) {
    // ---- service warp: row records and stored rows in, scalings out ----
    // (the fixed-stride variant runs only without previous scalings)
    bool has_old[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) has_old[k] = FLDR == 0 && a.rhs[k].old != nullptr;
    // Each lane serves one right-hand side (kItems <= 64 items in steps of
    // 32 with kHyRB = 8) and sums the residual terms |old s - w| of its rows:
    // each term in one rounding (a fused multiply-add), the sum compensated in
    // FP32, widened once at the end (no FP64 arithmetic per batch).
    const int kq_lane = (lane / kHyRB) % NRHS;
    const bool lane_old = kq_lane == 0 ? has_old[0] : has_old[NRHS - 1];
    CompSum racc;
    constexpr int kPer = (RPB + 31) / 32;  // rows per lane
    // A row's raw record (x, shift, weights, previous scalings) is copied
    // into a shared-memory stage by 4-byte asynchronous copies kAhead batches
    // before its batch, and turned into the packed record (x doubled, B =
    // -log2(e) ((2/eps)||x||^2 + shift)) when it is parked two batches ahead:
    // nothing waits for the copies until then, kAhead - 2 batches after their
    // issue, so their latency (from HBM under the stored stream, which also
    // evicts the points from L2) stays off the barrier. Each lane copies and
    // later reads only its own rows' entries. Batch j uses stage j % kAhead,
    // last read when batch j - kAhead was parked, kAhead - 2 batches earlier.
    auto load_raw = [&](int64_t b, int stage) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int rr = lane + 32 * u;
        if (rr < RPB) {
          const int64_t i = b * RPB + rr;
          const bool ok = b < nbatch && i < a.n;
          float* st = s_stage[stage][rr];
#pragma unroll
          for (int dd = 0; dd < D; ++dd) {
            if (ok && dd < d) cp_async_4(st + dd, a.X + i * d + dd);
            else st[dd] = 0.f;
          }
          if (ok) cp_async_4(st + D, a.shift + i);
          else st[D] = INFINITY;  // rows past the end: B = -inf, no mass
#pragma unroll
          for (int k = 0; k < NRHS; ++k) {
            if (ok && !kAx) cp_async_4(st + D + 1 + 2 * k, a.rhs[k].w + i);
            else st[D + 1 + 2 * k] = 0.f;
            if (ok && has_old[k]) cp_async_4(st + D + 2 + 2 * k, a.rhs[k].old + i);
            else st[D + 2 + 2 * k] = 0.f;
          }
        }
      }
      cp_async_commit();
    };
    auto park_raw = [&](int stage, int bf) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int rr = lane + 32 * u;
        if (rr < RPB) {
          const float* st = s_stage[stage][rr];
          float rec[4 * SV];
#pragma unroll
          for (int q = 0; q < 4 * SV; ++q) rec[q] = 0.f;
          float nrm = 0.f;
#pragma unroll
          for (int dd = 0; dd < D; ++dd) {
            const float x = st[dd];
            rec[2 * dd] = rec[2 * dd + 1] = x;
            nrm = fmaf(x, x, nrm);
          }
          rec[2 * D] = rec[2 * D + 1] = -kLog2e * (a.two_over_eps * nrm + st[D]);
#pragma unroll
          for (int k = 0; k < NRHS; ++k) {
            rec[4 * XV + 2 * k] = st[D + 1 + 2 * k];
            rec[4 * XV + 2 * k + 1] = st[D + 2 + 2 * k];
          }
#pragma unroll
          for (int v = 0; v < SV; ++v)
            s_rows[bf][rr * SV + v] = make_float4(rec[4 * v], rec[4 * v + 1], rec[4 * v + 2], rec[4 * v + 3]);
        }
      }
    };
    // the stored rows of batch b into ring slot s (one bulk copy; lane 0)
    int issued = 0;
    auto copy_stored = [&](int64_t b, int s) {
      if (b >= nbatch) return;
      ++issued;
      const int64_t row0 = b * RPB;
      const int rows = static_cast<int>(min(static_cast<int64_t>(RPB), a.n - row0));
      float* dst = s_ring + static_cast<size_t>(s) * RPB * lds;
      if (rows < RPB) {
        // the last batch: its rows past the end read as zeros, so that the
        // compute warps take every row of a batch unpredicated (the slot may
        // hold stale rows or nothing yet); these stores reach them through the
        // arrive below, as the copy's bytes do through its completion
        float4* z = reinterpret_cast<float4*>(dst + static_cast<size_t>(rows) * lds);
        const int nz = (RPB - rows) * (lds >> 2);
        for (int j = lane; j < nz; j += 32) z[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        __threadfence_block();
        __syncwarp();
      }
      if (lane == 0) {
        const uint32_t bytes = static_cast<uint32_t>(rows) * static_cast<uint32_t>(lds) * 4u;
        mbar_arrive_expect_tx(&s_full[s], bytes);
        bulk_copy_g2s(dst, h.Fs + row0 * lds, bytes, &s_full[s]);
      }
    };
    // prime both rings with the first two batches
    for (int j = 0; j < kHySlots - 1; ++j) copy_stored(static_cast<int64_t>(blockIdx.x) + j * gridDim.x, j);
    const int64_t G = gridDim.x;
    // one commit group per batch, in batch order: batches 0 .. kAhead - 1 here
#pragma unroll
    for (int j = 0; j < kAhead; ++j) load_raw(blockIdx.x + j * G, j);
    cp_async_wait<kAhead - 1>();
    park_raw(0, 0);
    cp_async_wait<kAhead - 2>();
    park_raw(1, 1);
    __syncthreads();
    // one batch (the it-th of this CTA): the records of batch it + kAhead start
    // to load, those of batch it + 2 (the group kAhead - 2 groups back) are parked
    auto step = [&](int64_t b, int it) {
      load_raw(b + kAhead * G, it % kAhead);
      __syncthreads();
      // slot (it + 2) % 3 was last read in the previous batch, before this barrier
      copy_stored(b + (kHySlots - 1) * G, (it + kHySlots - 1) % kHySlots);
      if (!kAx) {
        const float4* rows = s_rows[it % 3];
        const int64_t row0 = b * RPB;
#pragma unroll
        for (int item0 = 0; item0 < kItems; item0 += 32) {
          const int item = item0 + lane;
          if (item < kItems) {
            const int gg = item / (NRHS * kHyRB), kq = (item / kHyRB) % NRHS, qq = item % kHyRB;
            const int64_t i = row0 + gg * kHyRB + qq;
            if (i < a.n) {
              const float s = sum_partials<GW>(&s_red[it & 1][kq][qq][gg * GW]);
              const float4 wo = rows[(gg * kHyRB + qq) * SV + XV];
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
      cp_async_wait<kAhead - 2>();
      park_raw((it + 2) % kAhead, (it + 2) % 3);
    };
    int it = 0;
    for (int64_t b = blockIdx.x; b < nbatch; b += G, ++it) step(b, it);
    cp_async_wait<0>();  // copies for batches past the end (none issued) and stores settle
#pragma unroll
    for (int k = 0; k < NRHS; ++k)
      res[k] = kq_lane == k ? static_cast<double>(racc.s) + static_cast<double>(racc.c) : 0.0;
    // drain: every issued copy must have landed before the shared memory is
    // reused for the partials and before the CTA exits (the compute warps have
    // waited on each of them unless a wait ran out)
    for (int j = 0; j < min(issued, kHySlots); ++j) {
      const int itj = issued - 1 - j;
      if (lane == 0 && !mbar_wait_bounded(&s_full[itj % kHySlots], static_cast<uint32_t>(itj / kHySlots) & 1u))
        flag |= LSF_ERR_TIMEOUT;
    }
  } else {
    // ---- compute warps ----
    float2 A2[2], W2[2][D];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float Ap[2], Wp[2][D];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int k = col0 + 2 * p + hh;
        if (has_rc && k < a.r) {
          float nrm = 0.f;
#pragma unroll
          for (int dd = 0; dd < D; ++dd) {
            const float u = (dd < d) ? a.U[static_cast<int64_t>(k) * d + dd] : 0.f;
            nrm = fmaf(u, u, nrm);
            Wp[hh][dd] = kLog2e * (2.f * a.two_over_eps) * u;
          }
          Ap[hh] = kLog2e * (a.c[k] - a.two_over_eps * nrm);
        } else {
#pragma unroll
          for (int dd = 0; dd < D; ++dd) Wp[hh][dd] = 0.f;
          Ap[hh] = -INFINITY;  // ex2(-inf) = 0: padded or stored columns carry no mass here
        }
      }
      A2[p] = make_float2(Ap[0], Ap[1]);
#pragma unroll
      for (int dd = 0; dd < D; ++dd) W2[p][dd] = make_float2(Wp[0][dd], Wp[1][dd]);
    }
    float2 t2[NRHS][2];
    float4 ts[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int c = col0 + 2 * p;
        t2[k][p] = make_float2((!kAx && has_rc) ? a.rhs[k].t_in[c] : 0.f,
                               (!kAx && has_rc) ? a.rhs[k].t_in[c + 1] : 0.f);
      }
      ts[k] = (!kAx && has_st) ? *reinterpret_cast<const float4*>(a.rhs[k].t_in + c0 + col0)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();  // the rings are primed
    // batch it uses record buffer it % 3, ring slot it % kHySlots and that
    // slot's mbarrier phase (it / kHySlots) & 1, kept as running counters
    int it = 0, slot = 0, rbuf = 0;
    uint32_t phase = 0;
    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x, ++it) {
      const float4* rows = s_rows[rbuf];
      const float4* srow = reinterpret_cast<const float4*>(s_ring + (static_cast<size_t>(slot) * RPB + g * kHyRB) * lds) + tg;
      const int ldq = lds >> 2;  // float4s per stored row
      // the recomputed entries first: they need only the row records, so the
      // stored rows' copy lands meanwhile
      float2 F[kHyRB][2];
#pragma unroll
      for (int q = 0; q < kHyRB; ++q) {
        const float4* rw = rows + (g * kHyRB + q) * SV;
        float2 xb[2 * XV];
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
      }
      if (!mbar_wait_bounded(&s_full[slot], phase)) flag |= LSF_ERR_TIMEOUT;
      if (++slot == kHySlots) {
        slot = 0;
        phase ^= 1u;
      }
      if (++rbuf == 3) rbuf = 0;
      float dots[NRHS][kHyRB];
#pragma unroll
      for (int q = 0; q < kHyRB; ++q) {
        const float4 fs = has_st ? srow[q * ldq] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 fs0 = make_float2(fs.x, fs.y), fs1 = make_float2(fs.z, fs.w);
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          float2 S = __fmul2_rn(F[q][0], t2[k][0]);
          S = __ffma2_rn(F[q][1], t2[k][1], S);
          S = __ffma2_rn(fs0, make_float2(ts[k].x, ts[k].y), S);
          S = __ffma2_rn(fs1, make_float2(ts[k].z, ts[k].w), S);
          dots[k][q] = S.x + S.y;
        }
      }
      if (!kAx) {
        float v[NRHS];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) v[k] = fold_rows<kHyRB>(dots[k], lane, OpAdd());
        if ((lane & 3) == 0)
#pragma unroll
          for (int k = 0; k < NRHS; ++k) s_red[it & 1][k][lane >> 2][warp] = v[k];
      }
      __syncthreads();
      if (kDt) continue;
      // lane (kq, qq) forms the scaling of row qq of rhs kq from the group's
      // partials (the service warp's order); each row's scalings are then
      // broadcast right where the row is used
      float scl = 0.f;
      if (!kAx) {
        const int kq = lane >> 3, qq = lane & 7;
        // rows past the end have no mass (s = 0): their scaling stays 0
        if (kq < NRHS && b * RPB + g * kHyRB + qq < a.n) {
          const float s = sum_partials<GW>(&s_red[it & 1][kq][qq][g * GW]);
          const float4 wo = rows[(g * kHyRB + qq) * SV + XV];
          scl = ((NRHS == 1 || kq == 0) ? wo.x : wo.z) * __frcp_rn(s);
        }
      }
#pragma unroll
      for (int qq = 0; qq < kHyRB; ++qq) {
        const float4 fs = has_st ? srow[qq * ldq] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 fs0 = make_float2(fs.x, fs.y), fs1 = make_float2(fs.z, fs.w);
        float4 wo;
        if (kAx) wo = rows[(g * kHyRB + qq) * SV + XV];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          const float sk = kAx ? ((NRHS == 1 || k == 0) ? wo.y : wo.w)
                               : __shfl_sync(0xffffffffu, scl, k * 8 + qq);
          const float2 s2 = make_float2(sk, sk);
#pragma unroll
          for (int p = 0; p < 2; ++p) acc2[k][p] = __ffma2_rn(s2, F[qq][p], acc2[k][p]);
          const float2 lo = __ffma2_rn(s2, fs0, make_float2(accs[k].x, accs[k].y));
          const float2 hi = __ffma2_rn(s2, fs1, make_float2(accs[k].z, accs[k].w));
          accs[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
  }

  // every compute warp has passed its last batch and the service warp has
  // drained the ring: the ring's shared memory now takes the partials
  __syncthreads();
  float* s_part = s_ring;
  if (!kDt && !service) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      float* dst = s_part + static_cast<size_t>(g) * NRHS * ldr + k * ldr;
      if (has_rc) {
        dst[col0 + 0] = acc2[k][0].x;
        dst[col0 + 1] = acc2[k][0].y;
        dst[col0 + 2] = acc2[k][1].x;
        dst[col0 + 3] = acc2[k][1].y;
      }
      if (has_st) *reinterpret_cast<float4*>(dst + c0 + col0) = accs[k];
    }
  }
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
      for (int w = 0; w <= kHyWarps; ++w) r += s_res[w][k];
      s_res[0][k] = r;
      for (int w = 1; w <= kHyWarps; ++w) s_res[w][k] = 0.0;
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

// Three CTAs of 160 threads per SM for d <= 4 (128 registers a thread); for
// larger d each thread takes its full register need.
template <int GW, int D, int NRHS, int FLDR>
__global__ void __maxnreg__(128) hybrid_kernel(const HybridArgs h, const int mode) {
  hybrid_body<GW, D, NRHS, FLDR>(h, mode);
}
template <int GW, int D, int NRHS>
__global__ void __launch_bounds__(kHyThreads, 1) hybrid_kernel_wide(const HybridArgs h, const int mode) {
  hybrid_body<GW, D, NRHS, 0>(h, mode);
}

template <int GW, int D, int NRHS, int FLDR = 0>
int launch_gdn(int mode, const HybridArgs& h, cudaStream_t st) {
  constexpr int NG = kHyWarps / GW;
  constexpr int RPB = NG * kHyRB;
  const int lds = h.rc.ldr - h.c0;
  const size_t ring = sizeof(float) * static_cast<size_t>(kHySlots) * RPB * lds;
  const size_t parts = sizeof(float) * static_cast<size_t>(NG) * NRHS * h.rc.ldr;
  const size_t smem = std::max(ring, parts);
  void (*kern)(HybridArgs, int);
  if constexpr (D <= 4)
    kern = hybrid_kernel<GW, D, NRHS, FLDR>;
  else
    kern = hybrid_kernel_wide<GW, D, NRHS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  // the whole unified L1 as shared memory, so that the CTAs the registers allow
  // are not cut by a smaller carveout
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             static_cast<int>(cudaSharedmemCarveoutMaxShared));
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "hybrid: smem attribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHyThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t nbatch = (h.rc.n + RPB - 1) / RPB;
  const int64_t cap = std::min<int64_t>(static_cast<int64_t>(device_info().sms) * per_sm, max_pass_ctas());
  const int64_t grid = std::min<int64_t>(cap, nbatch);
  kern<<<static_cast<unsigned>(grid), kHyThreads, smem, st>>>(h, mode);
  return check_launch("hybrid_kernel");
}

template <int GW, int NRHS>
int launch_gn(int mode, const HybridArgs& h, int Dp, cudaStream_t st) {
  if constexpr (GW == 4) {
    // the update pass at r = 1024 without residual terms (the solvers' loop
    // passes), compiled for that stride
    bool old = false;
    for (int k = 0; k < NRHS; ++k) old = old || h.rc.rhs[k].old != nullptr;
    if (mode == kPassUpdate && !old && h.rc.ldr == 1024 && Dp <= 4) {
      switch (Dp) {
        case 2: return launch_gdn<GW, 2, NRHS, 1024>(mode, h, st);
        case 3: return launch_gdn<GW, 3, NRHS, 1024>(mode, h, st);
        default: return launch_gdn<GW, 4, NRHS, 1024>(mode, h, st);
      }
    }
  }
  switch (Dp) {
    case 2: return launch_gdn<GW, 2, NRHS>(mode, h, st);
    case 3: return launch_gdn<GW, 3, NRHS>(mode, h, st);
    case 4: return launch_gdn<GW, 4, NRHS>(mode, h, st);
    case 8: return launch_gdn<GW, 8, NRHS>(mode, h, st);
    default: return launch_gdn<GW, 16, NRHS>(mode, h, st);
  }
}

template <int NRHS>
int launch_n(int mode, const HybridArgs& h, int GW, int Dp, cudaStream_t st) {
  switch (GW) {
    case 1: return launch_gn<1, NRHS>(mode, h, Dp, st);
    case 2: return launch_gn<2, NRHS>(mode, h, Dp, st);
    default: return launch_gn<4, NRHS>(mode, h, Dp, st);
  }
}

}  // namespace

int launch_hybrid_pass(int mode, int nrhs, HybridArgs h, cudaStream_t st) {
  const RecomputeArgs& a = h.rc;
  if (a.n < 1) return fail(LSF_ERR_ARG, "hybrid: n must be >= 1");
  if (a.d < 1 || a.d > 16)
    return fail(LSF_ERR_UNSUPPORTED, "hybrid mode handles 1 <= d <= 16 (stored mode otherwise)");
  if (a.ldr < 8 || a.ldr % 4 != 0 || a.ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "hybrid: ldr must be a multiple of 4 in [8, 1024]");
  if (h.c0 != hybrid_first_stored(a.ldr)) return fail(LSF_ERR_ARG, "hybrid: column split mismatch");
  if (!a.X || !a.U || !a.c || !a.shift || !h.Fs) return fail(LSF_ERR_ARG, "hybrid: NULL argument");
  if (reinterpret_cast<uintptr_t>(h.Fs) % 16 != 0) return fail(LSF_ERR_ARG, "hybrid: Fs must be 16-byte aligned");
  for (int k = 0; k < nrhs; ++k)
    if (a.rhs[k].t_in && reinterpret_cast<uintptr_t>(a.rhs[k].t_in) % 16 != 0)
      return fail(LSF_ERR_ARG, "hybrid: r-vectors must be 16-byte aligned");
  const int qr = h.c0 / 4;
  int tpg = 32;
  while (tpg < qr) tpg *= 2;
  const int GW = tpg / 32;  // 1, 2 or 4 warps per row (qr <= 128)
  const int Dp = a.d <= 2 ? 2 : a.d <= 3 ? 3 : a.d <= 4 ? 4 : a.d <= 8 ? 8 : 16;
  const double bytes = 4.0 * a.n * (a.d + 1) + 4.0 * a.n * nrhs * 3.0 + 4.0 * a.n * (a.ldr - h.c0);
  LaunchScope ls(st, LSF_KERNEL_PASS_HYBRID, bytes);
  if (nrhs == 1) return launch_n<1>(mode, h, GW, Dp, st);
  return launch_n<2>(mode, h, GW, Dp, st);
}

}  // namespace lsf
