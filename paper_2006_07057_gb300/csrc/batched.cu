// Batched solver: many independent problems, Alg. 1 on each, one persistent
// cooperative kernel for all half iterations.
//
// Rows of all problems' features on one side are cut into tiles that never
// straddle two problems; the tile list of a side is split into contiguous ranges,
// one per CTA, identical in every round on that side. A round is one half
// iteration of every problem (round 0: t_v = zeta~^T v~ from the start vector;
// odd rounds: u-halves on the X side; even rounds: v-halves on the Y side; the
// last round: the residual pass on the X side). The copy ring streams the tiles
// of all rounds back to back, so the next round's features are in flight while
// the current one finishes. Consumers work as in the single-problem stored pass;
// when their tile moves to another problem they flush their partial r-vector for
// the old one and take the new one's right-hand side once that problem has
// finished the previous round (per-problem round flag, bounded wait). The last
// warp to flush a problem sums its partials in a fixed order, writes the new
// r-vector and raises the flag: problems advance independently, and results do
// not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "reduce.cuh"
#include "ring.cuh"
#include "small.cuh"

namespace lsf {
namespace {

struct BProb {
  const float* F[2];      // side 0: X (xi~), side 1: Y (zeta~)
  const float* w[2];      // a, b
  const float* shift[2];
  float* s[2];            // u~, v~
  float* t[2];            // t_u = xi~^T u~ (written by X rounds), t_v = zeta~^T v~
  lsf_result* result;
  int64_t n[2];
  double eps;
  float* part[2];         // [nslots][kConsumerWarps][ldr] partial r-vectors
  double* rpart;          // [nslots_x][kConsumerWarps] residual partials
  int first_cta[2];
  int nslots[2];          // slots first_cta .. last owner (empty CTAs in between stay zero)
  int nown[2];            // CTAs that own tiles of this problem: each flushes once per round
};

struct BTile {
  int p;
  int rows;
  int64_t row0;
};

struct BatchArgs {
  BProb* probs;
  const BTile* tiles[2];
  int64_t ntiles[2];
  unsigned* counter;  // [count] warp arrivals of the current round
  unsigned* flag;     // [count] rounds completed
  int count;
  int ldr;
  int tile_rows;
  int nstages;
  int rounds;
  unsigned long long wait_ns;  // limit of the bounded waits on flags and ring slots
  unsigned stall;              // failure-detection hook: rounds added to every flag target
};

__device__ __forceinline__ int round_side(int r, int rounds) {
  if (r == 0) return 1;               // start: t_v from v~
  if (r == rounds - 1) return 0;      // residual on X
  return (r & 1) ? 0 : 1;             // u-halves on X, v-halves on Y
}
__device__ __forceinline__ int round_mode(int r, int rounds) {
  if (r == 0) return kPassAxpy;
  if (r == rounds - 1) return kPassDot;
  return kPassUpdate;
}
__device__ __forceinline__ void tile_range(int64_t ntiles, int64_t* lo, int64_t* hi) {
  *lo = ntiles * blockIdx.x / gridDim.x;
  *hi = ntiles * (blockIdx.x + 1) / gridDim.x;
}

// The current value of a status word that other CTAs OR bits into (no caching).
__device__ __forceinline__ int ld_status(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int C, bool LOGD>
__global__ void __launch_bounds__(kPassThreads, 1) batched_kernel(const BatchArgs A) {
  constexpr int RW = 8 / C;
  constexpr int SH = RowFold<RW>::kShift;
  extern __shared__ __align__(128) unsigned char smem[];
  const int ldr = A.ldr;
  const Ring ring = ring_layout(smem, A.nstages, A.tile_rows, ldr);
  const int S = ring.S;
  const int TR = ring.TR;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  __shared__ int s_flag;
  if (threadIdx.x == 0) {
    ring_init(ring, kConsumerWarps);
    fence_mbarrier_init();
    s_flag = 0;
  }
  __syncthreads();
  int flag = 0;

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------ producer
    int it = 0;
    bool dead = false;
    int prod_p = -1, prod_void = 0;
    for (int r = 0; r < A.rounds && !dead; ++r) {
      const int side = round_side(r, A.rounds);
      const bool copy_w = round_mode(r, A.rounds) != kPassAxpy;
      prod_p = -1;
      int64_t lo, hi;
      tile_range(side ? A.ntiles[1] : A.ntiles[0], &lo, &hi);
      for (int64_t ti = lo; ti < hi; ++ti, ++it) {
        const int s = it % S;
        const uint32_t ph = static_cast<uint32_t>(it / S) & 1u;
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&ring.empty[s], ph ^ 1u, A.wait_ns) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          flag |= LSF_ERR_TIMEOUT;
          dead = true;
          break;
        }
        const BTile tl = (side ? A.tiles[1] : A.tiles[0])[ti];
        const BProb& pb = A.probs[tl.p];
        // a problem that has produced a non-finite scaling is void (it is solved
        // again in the log domain): its tiles are not streamed; the stage still
        // completes (one plain arrival instead of the copy's). The status is read
        // once per run of tiles of one problem.
        if (tl.p != prod_p) {
          prod_p = tl.p;
          int v = 0;
          if (lane == 0) v = (ld_status(&pb.result->status) & LSF_ERR_NONFINITE) ? 1 : 0;
          prod_void = __shfl_sync(0xffffffffu, v, 0);
        }
        const int void_p = prod_void;
        if (lane == 0) {
          if (void_p) {
            mbar_arrive(&ring.full[s]);
          } else {
            const uint32_t bytes = static_cast<uint32_t>(tl.rows) * static_cast<uint32_t>(ldr) * 4u;
            mbar_arrive_expect_tx(&ring.full[s], bytes);
            bulk_copy_g2s(ring.sF + static_cast<size_t>(s) * TR * ldr, pb.F[side] + tl.row0 * ldr, bytes,
                          &ring.full[s]);
          }
        }
        if (copy_w && !void_p) {
          float* dw = ring.sV + static_cast<size_t>(s * 2) * TR;
          const float* w = pb.w[side];
          for (int i = lane; i < tl.rows; i += 32) cp_async_4(dw + i, w + tl.row0 + i);
        }
        cp_async_mbar_arrive(&ring.full[s]);
      }
    }
    // drain: the copies still in flight land in this CTA's shared memory, so wait
    // for each of them (with the full default limit) before the CTA may exit
    const int used = min(it, S);
    for (int j = 0; j < used; ++j) {
      const int itj = it - 1 - j;
      if (lane == 0 && !mbar_wait_bounded(&ring.full[itj % S], static_cast<uint32_t>(itj / S) & 1u))
        flag |= LSF_ERR_TIMEOUT;
    }
  } else {
    // ------------------------------------------------------------ consumers
    const int myq = (lane >> SH) & (RW - 1);
    const bool owner = (lane & ((1 << SH) - 1)) == 0;
    int it = 0;
    bool dead = false;
    for (int r = 0; r < A.rounds && !dead; ++r) {
      const int side = round_side(r, A.rounds);
      const int mode = round_mode(r, A.rounds);
      int64_t lo, hi;
      tile_range(side ? A.ntiles[1] : A.ntiles[0], &lo, &hi);
      int cur = -1;
      // whether problem cur is void (read at each switch of problem, after the
      // producer read it for the same tiles: the bit only gets set, so a tile the
      // producer did not copy is always skipped here)
      int cur_void = 0;
      // scaling domain: t = r-vector, acc = transposed product;
      // log domain: t = log r-vector, acc = running column max, lsum = column sums
      float t[C][4], acc[C][4], lsum[LOGD ? C : 1][4];
      double res = 0.0;
      auto flush = [&](int p) {
        // this warp's partial r-vector (and residual) for problem p, this round
        const BProb& pb = A.probs[p];
        const int slot = static_cast<int>(blockIdx.x) - pb.first_cta[side];
        constexpr int kVec = LOGD ? 2 : 1;  // floats per column in a partial
        float* dst = pb.part[side] + (static_cast<size_t>(slot) * kConsumerWarps + warp) * kVec * ldr;
        if (mode != kPassDot) {
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            if (col < ldr) {
              *reinterpret_cast<float4*>(dst + col) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
              if (LOGD)
                *reinterpret_cast<float4*>(dst + ldr + col) =
                    make_float4(lsum[LOGD ? j : 0][0], lsum[LOGD ? j : 0][1], lsum[LOGD ? j : 0][2],
                                lsum[LOGD ? j : 0][3]);
            }
          }
        } else {
          double rr = res;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
          if (lane == 0) pb.rpart[static_cast<size_t>(slot) * kConsumerWarps + warp] = rr;
        }
        __threadfence();
        __syncwarp();
        unsigned last = 0;
        if (lane == 0) {
          const unsigned need = static_cast<unsigned>(pb.nown[side]) * kConsumerWarps;
          last = (atomicAdd(&A.counter[p], 1u) == need - 1u) ? 1u : 0u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return;
        __threadfence();
        const int nparts = pb.nslots[side] * kConsumerWarps;
        if (mode != kPassDot) {
          float* tout = pb.t[side];
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            if (col >= ldr) continue;
            if (LOGD) {
              float m[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY}, sm[4] = {0.f, 0.f, 0.f, 0.f};
              for (int q = 0; q < nparts; ++q) {
                const float* base = pb.part[side] + static_cast<size_t>(q) * 2 * ldr;
                const float4 vm = __ldcg(reinterpret_cast<const float4*>(base + col));
                const float4 vs = __ldcg(reinterpret_cast<const float4*>(base + ldr + col));
                lse_merge(m[0], sm[0], vm.x, vs.x);
                lse_merge(m[1], sm[1], vm.y, vs.y);
                lse_merge(m[2], sm[2], vm.z, vs.z);
                lse_merge(m[3], sm[3], vm.w, vs.w);
              }
              float o[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) o[e] = sm[e] > 0.f ? m[e] + logf(sm[e]) : -INFINITY;
              *reinterpret_cast<float4*>(tout + col) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
              double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
              for (int q = 0; q < nparts; ++q) {
                const float4 v = __ldcg(reinterpret_cast<const float4*>(pb.part[side] + static_cast<size_t>(q) * ldr + col));
                s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
              }
              *reinterpret_cast<float4*>(tout + col) =
                  make_float4(static_cast<float>(s0), static_cast<float>(s1), static_cast<float>(s2),
                              static_cast<float>(s3));
            }
          }
        } else if (lane == 0) {
          double tot = 0.0;
          for (int q = 0; q < nparts; ++q) tot += __ldcg(pb.rpart + q);
          pb.result->residual = tot;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          A.counter[p] = 0u;
          __threadfence();
          st_release(&A.flag[p], static_cast<unsigned>(r + 1));
        }
      };

      for (int64_t ti = lo; ti < hi && !dead; ++ti, ++it) {
        const int s = it % S;
        if (!ring_wait_full(ring, it, lane, A.wait_ns)) {
          flag |= LSF_ERR_TIMEOUT;
          dead = true;
          break;
        }
        const BTile tl = (side ? A.tiles[1] : A.tiles[0])[ti];
        if (tl.p != cur) {
          if (cur >= 0) flush(cur);
          cur = tl.p;
          // wait until problem cur has finished the previous round
          int ok = 1;
          if (lane == 0 && r > 0) {
            const unsigned* fp = A.flag + cur;
            const unsigned target = static_cast<unsigned>(r) + A.stall;
            if (ld_acquire(fp) < target) {
              const uint64_t t0 = globaltimer_ns();
              while (ld_acquire(fp) < target) {
                if (globaltimer_ns() - t0 > A.wait_ns) {
                  ok = 0;
                  break;
                }
              }
            }
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) {
            flag |= LSF_ERR_TIMEOUT;
            dead = true;
          }
          int v = 0;
          if (lane == 0) v = (ld_status(&A.probs[cur].result->status) & LSF_ERR_NONFINITE) ? 1 : 0;
          cur_void = __shfl_sync(0xffffffffu, v, 0);
          const BProb& pb = A.probs[cur];
          const float* tin = pb.t[1 - side];
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = 4 * lane + 128 * j;
            const float z = LOGD ? -INFINITY : 0.f;
            float4 tv = make_float4(z, z, z, z);
            if (mode != kPassAxpy && col < ldr) tv = __ldcg(reinterpret_cast<const float4*>(tin + col));
            t[j][0] = tv.x; t[j][1] = tv.y; t[j][2] = tv.z; t[j][3] = tv.w;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              acc[j][e] = LOGD ? kLogFloor : 0.f;  // empty online log-sum-exp, or 0
              if (LOGD) lsum[LOGD ? j : 0][e] = 0.f;
            }
          }
          res = 0.0;
        }
        if (!dead && !cur_void) {
          const BProb& pb = A.probs[cur];
          const int rows = tl.rows;
          const float* tF = ring.sF + static_cast<size_t>(s) * TR * ldr;
          const float* vw = ring.sV + static_cast<size_t>(s * 2) * TR;
          float* sc_out = pb.s[side];
          for (int rr = warp * RW; rr < rows; rr += RW * kConsumerWarps) {
            const float pad = LOGD ? -INFINITY : 0.f;
            float4 f[RW][C];
#pragma unroll
            for (int q = 0; q < RW; ++q)
#pragma unroll
              for (int j = 0; j < C; ++j) {
                const int col = 4 * lane + 128 * j;
                f[q][j] = (rr + q < rows && col < ldr)
                              ? *reinterpret_cast<const float4*>(tF + static_cast<size_t>(rr + q) * ldr + col)
                              : make_float4(pad, pad, pad, pad);
              }
            const int row = rr + myq;
            float scale[RW];  // scaling domain: the rows' scalings; log domain: their logs
            if (mode == kPassAxpy) {
              // the given start vector, written before this kernel
              float g = pad;
              if (owner && row < rows) g = sc_out[tl.row0 + row];
#pragma unroll
              for (int q = 0; q < RW; ++q) scale[q] = __shfl_sync(0xffffffffu, g, q << SH);
            } else {
              float p[RW];
              float rowlog = 0.f;  // log of the row product (log domain)
              float dot = 0.f;     // row product (scaling domain)
              if (LOGD) {
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                  float m = -INFINITY;
#pragma unroll
                  for (int j = 0; j < C; ++j)
                    m = fmaxf(m, fmaxf(fmaxf(f[q][j].x + t[j][0], f[q][j].y + t[j][1]),
                                       fmaxf(f[q][j].z + t[j][2], f[q][j].w + t[j][3])));
                  p[q] = m;
                }
                const float mrow = fold_rows<RW>(p, lane, OpMax());
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                  const float mq = __shfl_sync(0xffffffffu, mrow, q << SH);
                  float sum = 0.f;
#pragma unroll
                  for (int j = 0; j < C; ++j)
                    sum += ex2_approx((f[q][j].x + t[j][0] - mq) * kLog2e) +
                           ex2_approx((f[q][j].y + t[j][1] - mq) * kLog2e) +
                           ex2_approx((f[q][j].z + t[j][2] - mq) * kLog2e) +
                           ex2_approx((f[q][j].w + t[j][3] - mq) * kLog2e);
                  p[q] = sum;
                }
                const float srow = fold_rows<RW>(p, lane, OpAdd());
                rowlog = mrow + logf(srow);
              } else {
#pragma unroll
                for (int q = 0; q < RW; ++q) {
                  float d0 = 0.f, d1 = 0.f;
#pragma unroll
                  for (int j = 0; j < C; ++j) {
                    d0 = fmaf(f[q][j].x, t[j][0], d0);
                    d1 = fmaf(f[q][j].y, t[j][1], d1);
                    d0 = fmaf(f[q][j].z, t[j][2], d0);
                    d1 = fmaf(f[q][j].w, t[j][3], d1);
                  }
                  p[q] = d0 + d1;
                }
                dot = fold_rows<RW>(p, lane, OpAdd());
              }
              float sc = pad;
              if (row < rows) {
                const float wi = vw[row];
                if (mode == kPassDot) {
                  // residual: the previous scaling was written by this same lane in
                  // the last u-half (the X-side partition is the same every round)
                  if (owner) {
                    const double prev = static_cast<double>(sc_out[tl.row0 + row]);
                    const double us = LOGD ? exp(prev + static_cast<double>(rowlog))
                                           : prev * static_cast<double>(dot);
                    res += fabs(us - static_cast<double>(wi));
                  }
                } else {
                  sc = LOGD ? logf(wi) - rowlog : wi * __frcp_rn(dot);
                  if (owner) {
                    sc_out[tl.row0 + row] = sc;
                    const bool bad = LOGD ? !isfinite(sc) : (!(dot > 0.f) || !isfinite(sc));
                    if (bad) {
                      flag |= LSF_ERR_NONFINITE;
                      atomicOr(&pb.result->status, LSF_ERR_NONFINITE);
                    }
                  }
                  if (LOGD && !isfinite(sc)) sc = -INFINITY;
                }
              }
#pragma unroll
              for (int q = 0; q < RW; ++q) scale[q] = __shfl_sync(0xffffffffu, sc, q << SH);
            }
            if (mode != kPassDot) {
              if (LOGD) {
                // online (max, sum) per column, one ex2 per entry
#pragma unroll
                for (int j = 0; j < C; ++j)
#pragma unroll
                  for (int q = 0; q < RW; ++q) {
                    lse_push(acc[j][0], lsum[LOGD ? j : 0][0], f[q][j].x + scale[q]);
                    lse_push(acc[j][1], lsum[LOGD ? j : 0][1], f[q][j].y + scale[q]);
                    lse_push(acc[j][2], lsum[LOGD ? j : 0][2], f[q][j].z + scale[q]);
                    lse_push(acc[j][3], lsum[LOGD ? j : 0][3], f[q][j].w + scale[q]);
                  }
              } else {
#pragma unroll
                for (int q = 0; q < RW; ++q)
#pragma unroll
                  for (int j = 0; j < C; ++j) {
                    acc[j][0] = fmaf(scale[q], f[q][j].x, acc[j][0]);
                    acc[j][1] = fmaf(scale[q], f[q][j].y, acc[j][1]);
                    acc[j][2] = fmaf(scale[q], f[q][j].z, acc[j][2]);
                    acc[j][3] = fmaf(scale[q], f[q][j].w, acc[j][3]);
                  }
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring.empty[s]);
      }
      if (cur >= 0 && !dead) flush(cur);
    }
  }
  if (flag) atomicOr(&s_flag, flag);
  __syncthreads();
  // timeouts are reported on every problem's record (which problem stalled is not known)
  if ((s_flag & LSF_ERR_TIMEOUT) && threadIdx.x == 0)
    for (int p = 0; p < A.count; ++p) atomicOr(&A.probs[p].result->status, LSF_ERR_TIMEOUT);
}

// v = 1 per problem: v~ = exp(shift_y - M_p); also resets the round state.
__global__ void __launch_bounds__(256) batched_start_kernel(BProb* probs, unsigned* counter,
                                                            unsigned* flag, int iters, int log_domain) {
  const BProb pb = probs[blockIdx.x];
  __shared__ float s_m[8];
  float m = -INFINITY;
  for (int64_t j = threadIdx.x; j < pb.n[1]; j += blockDim.x) m = fmaxf(m, pb.shift[1][j]);
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  float M = s_m[0];
  for (int w = 1; w < 8; ++w) M = fmaxf(M, s_m[w]);
  if (log_domain) M = 0.f;  // log v~ = shift exactly, no global factor needed
  for (int64_t j = threadIdx.x; j < pb.n[1]; j += blockDim.x)
    pb.s[1][j] = log_domain ? pb.shift[1][j] : expf(pb.shift[1][j] - M);
  if (threadIdx.x == 0) {
    pb.result->W = 0.0;
    pb.result->residual = 0.0;
    pb.result->log_scale = static_cast<double>(M);
    pb.result->status = 0;
    pb.result->iters = iters;
    pb.result->mode = log_domain ? LSF_MODE_LOG : LSF_MODE_STORED;
    pb.result->reserved = 0;
    counter[blockIdx.x] = 0u;
    flag[blockIdx.x] = 0u;
  }
}

// Eq. (6) per problem with an FP64 compensated sum (one block per problem).
__global__ void __launch_bounds__(256) batched_divergence_kernel(const BProb* probs, int log_domain) {
  const BProb pb = probs[blockIdx.x];
  const double M = pb.result->log_scale;
  KahanSum acc;
  for (int side = 0; side < 2; ++side) {
    const double sign = side == 0 ? 1.0 : -1.0;
    for (int64_t i = threadIdx.x; i < pb.n[side]; i += blockDim.x)
      acc.add(static_cast<double>(pb.w[side][i]) *
              ((log_domain ? static_cast<double>(pb.s[side][i]) : static_cast<double>(logf(pb.s[side][i]))) -
               pb.shift[side][i] - sign * M));
  }
  __shared__ double s_w[8];
  double v = acc.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    KahanSum tot;
    for (int w = 0; w < 8; ++w) tot.add(s_w[w]);
    pb.result->W = pb.eps * tot.value();
  }
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

using BatchKernel = void (*)(BatchArgs);
BatchKernel batched_kernel_for(int C, bool logd) {
  if (logd)
    return C == 1 ? batched_kernel<1, true> : C == 2 ? batched_kernel<2, true>
         : C == 4 ? batched_kernel<4, true> : batched_kernel<8, true>;
  return C == 1 ? batched_kernel<1, false> : C == 2 ? batched_kernel<2, false>
       : C == 4 ? batched_kernel<4, false> : batched_kernel<8, false>;
}

struct PlanLayout {
  size_t probs, sprobs, tiles_x, tiles_y, counter, flag, part_x, part_y, rpart, total;
};

// How a stored batch is solved: 0 one persistent kernel over all problems'
// tiles (default: on the batched workload, n and m up to 2^16, it is 1.4x faster
// than one cluster per problem), 1 one thread-block cluster per problem (all in
// one launch), 2 by rule (clusters when there are enough problems to occupy
// every SM with clusters and every problem is small: (n + m) ldr <= 2^18).
int g_batch_strategy = 0;
unsigned long long g_batch_wait_ns = kWaitLimitNs;  // lsf_set_batch_fault
int g_batch_stall = 0;

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" int lsf_batch_plan(const lsf_batch_problem* probs, int count, int ldr, int mode,
                              int tile_bytes, lsf_batch_info* info, void* plan, size_t plan_bytes,
                              void* stream) {
  if (!probs || !info) return fail(LSF_ERR_ARG, "lsf_batch_plan: NULL argument");
  if (count < 1) return fail(LSF_ERR_ARG, "lsf_batch_plan: count must be >= 1");
  if (mode != LSF_MODE_STORED && mode != LSF_MODE_LOG)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_batch_plan: mode must be stored or log");
  const bool logd = mode == LSF_MODE_LOG;
  if (ldr < 4 || ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_batch_plan: ldr must be a multiple of 4 in [4, 1024]");
  for (int p = 0; p < count; ++p) {
    const lsf_batch_problem& q = probs[p];
    if (q.n < 1 || q.m < 1) return fail(LSF_ERR_ARG, "problem %d: empty measure", p);
    if (!q.Fx || !q.Fy || !q.shift_x || !q.shift_y || !q.a || !q.b || !q.u || !q.v || !q.t_u ||
        !q.t_v || !q.result)
      return fail(LSF_ERR_ARG, "problem %d: NULL pointer", p);
    if (reinterpret_cast<uintptr_t>(q.Fx) % 16 || reinterpret_cast<uintptr_t>(q.Fy) % 16 ||
        reinterpret_cast<uintptr_t>(q.t_u) % 16 || reinterpret_cast<uintptr_t>(q.t_v) % 16)
      return fail(LSF_ERR_ARG, "problem %d: F and t vectors must be 16-byte aligned", p);
    if (!(q.eps > 0.0)) return fail(LSF_ERR_ARG, "problem %d: eps must be > 0", p);
  }
  const DeviceInfo& dev = device_info();
  const int C = pass_columns(ldr);
  const int RW = 8 / C;
  const int64_t row_bytes = 4LL * ldr;
  const int64_t unit = static_cast<int64_t>(RW) * kConsumerWarps;
  int tb = tile_bytes > 0 ? tile_bytes : 44 * 1024;
  int64_t tr = std::max<int64_t>(unit, (tb / row_bytes) / unit * unit);
  tr = std::min<int64_t>(tr, 1024);
  const size_t stage_bytes = static_cast<size_t>(tr * row_bytes) + 2 * tr * 4;
  const size_t budget = static_cast<size_t>(dev.smem_optin) - 4096;
  int S = static_cast<int>(std::min<size_t>(8, (budget - 256) / stage_bytes));
  if (S < 2) return fail(LSF_ERR_UNSUPPORTED, "lsf_batch_plan: tile does not fit in shared memory");
  const size_t smem = ring_bytes(S, tr, ldr, 1);

  // co-resident grid (the kernel's CTAs wait on one another)
  int per_sm = 0;
  void (*kern)(BatchArgs) = batched_kernel_for(C, logd);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPassThreads, smem) != cudaSuccess ||
      per_sm < 1)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_batch_plan: kernel cannot be resident");
  const int grid = dev.sms * std::min(per_sm, 1);

  // tiles and CTA partition per side
  std::vector<BTile> tiles[2];
  for (int side = 0; side < 2; ++side)
    for (int p = 0; p < count; ++p) {
      const int64_t n = side == 0 ? probs[p].n : probs[p].m;
      for (int64_t r0 = 0; r0 < n; r0 += tr)
        tiles[side].push_back(BTile{p, static_cast<int>(std::min<int64_t>(tr, n - r0)), r0});
    }
  std::vector<int> first[2], last[2], nown[2];
  for (int side = 0; side < 2; ++side) {
    first[side].assign(count, -1);
    last[side].assign(count, -1);
    nown[side].assign(count, 0);
    const int64_t T = static_cast<int64_t>(tiles[side].size());
    for (int c = 0; c < grid; ++c) {
      const int64_t lo = T * c / grid, hi = T * (c + 1) / grid;
      int prev = -1;
      for (int64_t ti = lo; ti < hi; ++ti) {
        const int p = tiles[side][ti].p;
        if (first[side][p] < 0) first[side][p] = c;
        last[side][p] = c;
        if (p != prev) ++nown[side][p];
        prev = p;
      }
    }
  }
  size_t nslot_total[2] = {0, 0};
  for (int side = 0; side < 2; ++side)
    for (int p = 0; p < count; ++p) nslot_total[side] += last[side][p] - first[side][p] + 1;

  PlanLayout L{};
  size_t off = 0;
  L.probs = off; off += align256(sizeof(BProb) * count);
  L.sprobs = off; off += align256(sizeof(SProb) * count);
  L.tiles_x = off; off += align256(sizeof(BTile) * tiles[0].size());
  L.tiles_y = off; off += align256(sizeof(BTile) * tiles[1].size());
  L.counter = off; off += align256(sizeof(unsigned) * count);
  L.flag = off; off += align256(sizeof(unsigned) * count);
  const size_t vec = logd ? 2 : 1;  // (max, sum) pairs in the log domain
  L.part_x = off; off += align256(sizeof(float) * nslot_total[0] * kConsumerWarps * ldr * vec);
  L.part_y = off; off += align256(sizeof(float) * nslot_total[1] * kConsumerWarps * ldr * vec);
  L.rpart = off; off += align256(sizeof(double) * nslot_total[0] * kConsumerWarps);
  L.total = off;

  info->count = count;
  info->ldr = ldr;
  info->mode = mode;
  info->tile_rows = static_cast<int>(tr);
  info->stages = S;
  info->grid = grid;
  info->tiles_x = static_cast<int64_t>(tiles[0].size());
  info->tiles_y = static_cast<int64_t>(tiles[1].size());
  info->rows_x = 0;
  info->rows_y = 0;
  for (int p = 0; p < count; ++p) {
    info->rows_x += probs[p].n;
    info->rows_y += probs[p].m;
  }
  info->plan_bytes = L.total;
  info->smem_bytes = smem;
  // clusters of 8 CTAs: enough problems to occupy every SM, each of them small
  bool small = true;
  for (int p = 0; p < count; ++p) small &= (probs[p].n + probs[p].m) * static_cast<int64_t>(ldr) <= (1 << 18);
  const bool many = count >= 2 * (dev.sms / 8);
  info->strategy = (!logd && (g_batch_strategy == 1 || (g_batch_strategy == 2 && many && small))) ? 1 : 0;
  if (!plan) return LSF_OK;
  if (plan_bytes < L.total) return fail(LSF_ERR_WORKSPACE, "batch plan needs %zu bytes", L.total);
  if (reinterpret_cast<uintptr_t>(plan) % 256) return fail(LSF_ERR_ARG, "batch plan must be 256-byte aligned");

  char* base = static_cast<char*>(plan);
  std::vector<char> host(L.tiles_y + sizeof(BTile) * tiles[1].size(), 0);
  BProb* hp = reinterpret_cast<BProb*>(host.data() + L.probs);
  SProb* hs = reinterpret_cast<SProb*>(host.data() + L.sprobs);
  size_t px = 0, py = 0, pr = 0;
  for (int p = 0; p < count; ++p) {
    const lsf_batch_problem& q = probs[p];
    BProb b{};
    b.F[0] = q.Fx; b.F[1] = q.Fy;
    b.w[0] = q.a; b.w[1] = q.b;
    b.shift[0] = q.shift_x; b.shift[1] = q.shift_y;
    b.s[0] = q.u; b.s[1] = q.v;
    b.t[0] = q.t_u; b.t[1] = q.t_v;
    b.result = q.result;
    b.n[0] = q.n; b.n[1] = q.m;
    b.eps = q.eps;
    for (int side = 0; side < 2; ++side) {
      b.first_cta[side] = first[side][p];
      b.nslots[side] = last[side][p] - first[side][p] + 1;
      b.nown[side] = nown[side][p];
    }
    b.part[0] = reinterpret_cast<float*>(base + L.part_x) + px * kConsumerWarps * ldr * vec;
    b.part[1] = reinterpret_cast<float*>(base + L.part_y) + py * kConsumerWarps * ldr * vec;
    b.rpart = reinterpret_cast<double*>(base + L.rpart) + pr * kConsumerWarps;
    px += b.nslots[0];
    py += b.nslots[1];
    pr += b.nslots[0];
    hp[p] = b;
    SProb sp{};
    sp.F[0] = q.Fx; sp.F[1] = q.Fy;
    sp.w[0] = q.a; sp.w[1] = q.b;
    sp.shift[0] = q.shift_x; sp.shift[1] = q.shift_y;
    sp.s[0] = q.u; sp.s[1] = q.v;
    sp.t[0] = q.t_u; sp.t[1] = q.t_v;
    sp.result = q.result;
    sp.n[0] = q.n; sp.n[1] = q.m;
    hs[p] = sp;
  }
  std::copy(tiles[0].begin(), tiles[0].end(), reinterpret_cast<BTile*>(host.data() + L.tiles_x));
  std::copy(tiles[1].begin(), tiles[1].end(), reinterpret_cast<BTile*>(host.data() + L.tiles_y));
  cudaStream_t st = as_stream(stream);
  if (cudaMemcpyAsync(plan, host.data(), host.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(base + L.counter, 0, L.total - L.counter, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_batch_plan: copy of the plan failed");
  return LSF_OK;
}

extern "C" int lsf_solve_batched(const lsf_batch_info* info, void* plan, int iters, void* stream) {
  lsf::TraceRange trace_range("lsf_solve_batched");
  if (!info || !plan) return fail(LSF_ERR_ARG, "lsf_solve_batched: NULL argument");
  if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
  cudaStream_t st = as_stream(stream);
  char* base = static_cast<char*>(plan);
  // rebuild the layout offsets exactly as lsf_batch_plan did
  const int count = info->count;
  size_t off = 0;
  const size_t o_probs = off; off += align256(sizeof(BProb) * count);
  const size_t o_sprobs = off; off += align256(sizeof(SProb) * count);
  const size_t o_tx = off; off += align256(sizeof(BTile) * info->tiles_x);
  const size_t o_ty = off; off += align256(sizeof(BTile) * info->tiles_y);
  const size_t o_counter = off; off += align256(sizeof(unsigned) * count);
  const size_t o_flag = off;
  BatchArgs A{};
  A.probs = reinterpret_cast<BProb*>(base + o_probs);
  A.tiles[0] = reinterpret_cast<const BTile*>(base + o_tx);
  A.tiles[1] = reinterpret_cast<const BTile*>(base + o_ty);
  A.ntiles[0] = info->tiles_x;
  A.ntiles[1] = info->tiles_y;
  A.counter = reinterpret_cast<unsigned*>(base + o_counter);
  A.flag = reinterpret_cast<unsigned*>(base + o_flag);
  A.count = count;
  A.ldr = info->ldr;
  A.tile_rows = info->tile_rows;
  A.nstages = info->stages;
  A.rounds = 2 * iters + 2;
  A.wait_ns = g_batch_wait_ns;
  A.stall = static_cast<unsigned>(g_batch_stall);
  if (info->strategy == 1) {
    // one cluster per problem, then the Eq. (6) reduction of every problem
    int rc = small_solve_table(reinterpret_cast<const SProb*>(base + o_sprobs), count, info->ldr, iters, st);
    if (rc != LSF_OK) return rc;
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    batched_divergence_kernel<<<count, 256, 0, st>>>(A.probs, 0);
    return check_launch("batched_divergence_kernel");
  }
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    batched_start_kernel<<<count, 256, 0, st>>>(A.probs, A.counter, A.flag, iters,
                                                 info->mode == LSF_MODE_LOG ? 1 : 0);
  }
  int rc = check_launch("batched_start_kernel");
  if (rc != LSF_OK) return rc;
  void (*kern)(BatchArgs) = batched_kernel_for(pass_columns(info->ldr), info->mode == LSF_MODE_LOG);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)info->smem_bytes);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(info->grid);
  cfg.blockDim = dim3(kPassThreads);
  cfg.dynamicSmemBytes = info->smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  {
    // algorithmic bytes: every feature row once per round (X side in iters + 1
    // rounds, Y side in iters + 1), plus weights and scalings (12 B per row)
    const double bytes = static_cast<double>(iters + 1) *
                         (static_cast<double>(info->rows_x) + static_cast<double>(info->rows_y)) *
                         (4.0 * info->ldr + 12.0);
    LaunchScope ls(st, LSF_KERNEL_BATCHED, bytes);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, A);
    if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "batched kernel launch: %s", cudaGetErrorString(e));
  }
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    batched_divergence_kernel<<<count, 256, 0, st>>>(A.probs, info->mode == LSF_MODE_LOG ? 1 : 0);
  }
  return check_launch("batched_divergence_kernel");
}

extern "C" int lsf_set_batch_fault(unsigned long long wait_limit_ns, int stall_rounds) {
  if (wait_limit_ns < 10000ull || wait_limit_ns > 60000000000ull)
    return fail(LSF_ERR_ARG, "lsf_set_batch_fault: wait_limit_ns outside [1e4, 6e10]");
  if (stall_rounds != 0 && stall_rounds != 1)
    return fail(LSF_ERR_ARG, "lsf_set_batch_fault: stall_rounds must be 0 or 1");
  g_batch_wait_ns = wait_limit_ns;
  g_batch_stall = stall_rounds;
  return LSF_OK;
}

extern "C" int lsf_set_batch_strategy(int strategy) {
  if (strategy < 0 || strategy > 2) return fail(LSF_ERR_ARG, "lsf_set_batch_strategy: 0, 1 or 2");
  g_batch_strategy = strategy;
  return LSF_OK;
}
