// Cluster-persistent Sinkhorn solve (Alg. 1 on K = xi~ zeta~^T) for problems
// whose stored features fit in L2.
//
// The multi-launch path pays a launch and a grid-wide reduction for every half
// iteration, about 15-35 us, which is most of the time of a problem of a few
// thousand points. Here one thread-block cluster (16 CTAs, or 8 where 16 cannot
// be scheduled) runs the whole solve in one launch: the start v~ = exp(shift_y -
// M), every half iteration, and the residual pass. Each CTA owns a contiguous
// slice of the rows of both clouds (kept in shared memory with their weights and
// scalings when they fit, read from L2 otherwise); a half iteration is
//   row products s_i = F_i . t, new_i = w_i / s_i, t'_k += new_i F_ik
// with warp-per-row dot products (two rows in flight per warp) and the
// transposed product in registers. The warps' partials are folded in shared
// memory and each CTA pushes its partial r-vector into every CTA of the cluster
// (asynchronous distributed-shared-memory stores that complete transaction
// bytes on the receiver's mbarrier); a CTA then waits on its own barrier only,
// and sums the CTAs' partials in rank order, so all CTAs hold the same t'. Two
// gather buffers alternate: a CTA pushes into buffer b for half h + 2 only after
// every peer has pushed half h + 1, which each peer does after it consumed
// buffer b of half h.
//
// Waits are bounded (status LSF_ERR_TIMEOUT). Sums are in a fixed order (rows
// within a warp, warps, then ranks), so results are deterministic.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "reduce.cuh"
#include "small.cuh"

namespace lsf {
namespace cg = cooperative_groups;
namespace {

constexpr int kSmallWarps = 8;
constexpr int kSmallThreads = kSmallWarps * 32;

enum SmallHalf : int { kHalfInit = 0, kHalfUpdate = 1, kHalfDot = 2 };

struct SmallArgs {
  SProb probs[kSmallMaxProblems];
  const SProb* table;  // device problem table (batches), or NULL: probs[] above
  int ldr;
  int iters;
};

template <int C, bool RES>
__device__ __forceinline__ void small_load(float4 (&f)[C], const float* F, const float* rows,
                                           int64_t i, int64_t lo, int ldr, int lane) {
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int col = 4 * lane + 128 * j;
    if (col < ldr) {
      f[j] = RES ? *reinterpret_cast<const float4*>(rows + (i - lo) * ldr + col)
                 : __ldcg(reinterpret_cast<const float4*>(F + i * ldr + col));
    } else {
      f[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

template <int C>
__device__ __forceinline__ float small_dot(const float4 (&f)[C], const float4 (&t)[C]) {
  float d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    d0 = fmaf(f[j].x, t[j].x, d0);
    d1 = fmaf(f[j].y, t[j].y, d1);
    d0 = fmaf(f[j].z, t[j].z, d0);
    d1 = fmaf(f[j].w, t[j].w, d1);
  }
  return d0 + d1;
}

template <int C>
__device__ __forceinline__ void small_axpy(float (&acc)[C][4], float sc, const float4 (&f)[C]) {
#pragma unroll
  for (int j = 0; j < C; ++j) {
    acc[j][0] = fmaf(sc, f[j].x, acc[j][0]);
    acc[j][1] = fmaf(sc, f[j].y, acc[j][1]);
    acc[j][2] = fmaf(sc, f[j].z, acc[j][2]);
    acc[j][3] = fmaf(sc, f[j].w, acc[j][3]);
  }
}

// One half iteration on one side. KIND: kHalfInit (scale = exp(shift - M),
// written as the start scaling), kHalfUpdate (scale = w / (F t), written), or
// kHalfDot (residual |old (F t) - w| only). For Init and Update the cluster's
// transposed product ends up in tb (every CTA) and, from rank 0, in t_out.
// Returns this thread's residual sum (Dot).
// Exchange state of one cluster: gather buffers [2][kMaxCluster][ldr], their
// mbarriers, and which buffer / phase the next half uses.
constexpr int kMaxCluster = 16;
struct Exchange {
  float* gbuf;
  uint64_t* gbar;
  unsigned rank, CL;
  int h;  // halves exchanged so far
};

// w and s are indexed by i - off (off = lo for rows held in shared memory)
template <int C, bool RES, int KIND>
__device__ __forceinline__ double small_half(const float* F, const float* w, const float* shift,
                                             float* s, int64_t off, float* t_out, const float* rows,
                                             int64_t lo, int64_t hi, float M, float* tb,
                                             float* red, int ldr, Exchange& ex, int& flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[C][4];
#pragma unroll
  for (int j = 0; j < C; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
  float4 tv[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int col = 4 * lane + 128 * j;
    tv[j] = (KIND != kHalfInit && col < ldr) ? *reinterpret_cast<const float4*>(tb + col)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  double res = 0.0;
  // rows read from L2 are prefetched one step ahead (shared-memory rows need not)
  float4 na[C], nb[C];
  auto fetch = [&](int64_t i) {
    if (i < hi) small_load<C, RES>(na, F, rows, i, lo, ldr, lane);
    if (i + kSmallWarps < hi) {
      small_load<C, RES>(nb, F, rows, i + kSmallWarps, lo, ldr, lane);
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) nb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (!RES) fetch(lo + warp);
  for (int64_t i = lo + warp; i < hi; i += 2 * kSmallWarps) {
    const int64_t i2 = i + kSmallWarps;
    const bool has2 = i2 < hi;
    float4 fa[C], fb[C];
    if (RES) {
      small_load<C, RES>(fa, F, rows, i, lo, ldr, lane);
      if (has2) {
        small_load<C, RES>(fb, F, rows, i2, lo, ldr, lane);
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j) fb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int j = 0; j < C; ++j) {
        fa[j] = na[j];
        fb[j] = nb[j];
      }
      fetch(i + 2 * kSmallWarps);
    }
    float sa, sb = 0.f;
    if (KIND == kHalfInit) {
      sa = expf(shift[i] - M);
      if (has2) sb = expf(shift[i2] - M);
      if (lane == 0) {
        s[i - off] = sa;
        if (has2) s[i2 - off] = sb;
      }
    } else {
      float da = small_dot<C>(fa, tv), db = small_dot<C>(fb, tv);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        da += __shfl_xor_sync(0xffffffffu, da, o);
        db += __shfl_xor_sync(0xffffffffu, db, o);
      }
      const float wa = w[i - off], wb = has2 ? w[i2 - off] : 0.f;
      if (KIND == kHalfDot) {
        // the previous scalings were written by this same lane in the last update
        if (lane == 0) {
          res += fabs(static_cast<double>(s[i - off]) * static_cast<double>(da) - static_cast<double>(wa));
          if (has2)
            res += fabs(static_cast<double>(s[i2 - off]) * static_cast<double>(db) - static_cast<double>(wb));
        }
        continue;
      }
      sa = wa * __frcp_rn(da);
      sb = has2 ? wb * __frcp_rn(db) : 0.f;
      if (lane == 0) {
        s[i - off] = sa;
        if (!(da > 0.f) || !isfinite(sa)) flag |= LSF_ERR_NONFINITE;
        if (has2) {
          s[i2 - off] = sb;
          if (!(db > 0.f) || !isfinite(sb)) flag |= LSF_ERR_NONFINITE;
        }
      }
    }
    small_axpy<C>(acc, sa, fa);
    small_axpy<C>(acc, sb, fb);
  }
  if constexpr (KIND == kHalfDot) {
    return res;
  } else {
    // warps -> CTA partial (fixed order) -> cluster barrier -> ranks (fixed order)
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int col = 4 * lane + 128 * j;
      if (col < ldr)
        *reinterpret_cast<float4*>(red + static_cast<size_t>(warp) * ldr + col) =
            make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
    }
    __syncthreads();
    const int nv4 = ldr >> 2;
    const int b = ex.h & 1;
    const uint32_t parity = static_cast<uint32_t>(ex.h >> 1) & 1u;
    // fold the warps and push this CTA's partial into slot `rank` of every CTA's buffer b
    const uint32_t slot = smem_u32(ex.gbuf + (static_cast<size_t>(b) * kMaxCluster + ex.rank) * ldr);
    const uint32_t bar = smem_u32(ex.gbar + b);
    for (int i4 = threadIdx.x; i4 < nv4; i4 += blockDim.x) {
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int wq = 0; wq < kSmallWarps; ++wq) {
        const float4 v = *reinterpret_cast<const float4*>(red + static_cast<size_t>(wq) * ldr + 4 * i4);
        sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
      }
      for (unsigned rk = 0; rk < ex.CL; ++rk) {
        uint32_t rdst, rbar;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rdst) : "r"(slot + 16u * i4), "r"(rk));
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(bar), "r"(rk));
        asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
                     :: "r"(rdst), "f"(sum.x), "f"(sum.y), "f"(sum.z), "f"(sum.w), "r"(rbar) : "memory");
      }
    }
    // every CTA's partial of this half has landed in buffer b
    if (!mbar_wait_bounded(ex.gbar + b, parity)) flag |= LSF_ERR_TIMEOUT;
    const float* g = ex.gbuf + static_cast<size_t>(b) * kMaxCluster * ldr;
    for (int i4 = threadIdx.x; i4 < nv4; i4 += blockDim.x) {
      CompSum a0, a1, a2, a3;
      for (unsigned rk = 0; rk < ex.CL; ++rk) {
        const float4 v = *reinterpret_cast<const float4*>(g + static_cast<size_t>(rk) * ldr + 4 * i4);
        a0.add(v.x); a1.add(v.y); a2.add(v.z); a3.add(v.w);
      }
      const float4 tot = make_float4(a0.value(), a1.value(), a2.value(), a3.value());
      *reinterpret_cast<float4*>(tb + 4 * i4) = tot;
      if (ex.rank == 0) *reinterpret_cast<float4*>(t_out + 4 * i4) = tot;
    }
    __syncthreads();
    // buffer b is consumed: arm its barrier for its next use (half h + 2)
    if (threadIdx.x == 0) mbar_arrive_expect_tx(ex.gbar + b, ex.CL * ldr * 4u);
    ++ex.h;
    return 0.0;
  }
}

template <int C, bool RES>
__global__ void __launch_bounds__(kSmallThreads) small_solve_kernel(const SmallArgs A) {
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned CL = cluster.num_blocks();
  const unsigned rank = cluster.block_rank();
  const unsigned pid = blockIdx.x / CL;
  // the problem record: from the device table, or picked by compile-time indices
  SProb P = A.probs[0];
  if (A.table) {
    P = A.table[pid];
  } else {
#pragma unroll
    for (int q = 1; q < kSmallMaxProblems; ++q)
      if (pid == static_cast<unsigned>(q)) P = A.probs[q];
  }
  const int ldr = A.ldr;
  extern __shared__ __align__(16) float sm[];
  float* tb = sm;                                   // [ldr] current r-vector
  float* red = tb + ldr;                            // [kSmallWarps][ldr]
  float* gbuf = red + kSmallWarps * ldr;            // [2][kMaxCluster][ldr] gathered partials
  float* rows = gbuf + 2 * kMaxCluster * ldr;       // resident rows (RES), then w and s
  __shared__ __align__(8) uint64_t s_gbar[2];
  __shared__ double s_dred[kSmallWarps];
  __shared__ double s_dpart;
  __shared__ float s_fred[kSmallWarps];
  __shared__ float s_fpart;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const int64_t lo0 = P.n[0] * rank / CL, hi0 = P.n[0] * (rank + 1) / CL;
  const int64_t lo1 = P.n[1] * rank / CL, hi1 = P.n[1] * (rank + 1) / CL;
  const int64_t nr0 = hi0 - lo0, nr1 = hi1 - lo1;
  float* rows0 = rows;
  float* rows1 = rows + nr0 * ldr;
  // resident weights and scalings (RES): w0, w1, s0, s1 after the rows
  float* rw0 = rows1 + nr1 * ldr;
  float* rw1 = rw0 + nr0;
  float* rs0 = rw1 + nr1;
  float* rs1 = rs0 + nr0;
  if (RES) {
    const int64_t c0 = nr0 * ldr / 4, c1 = nr1 * ldr / 4;
    const float4* g0 = reinterpret_cast<const float4*>(P.F[0] + lo0 * ldr);
    const float4* g1 = reinterpret_cast<const float4*>(P.F[1] + lo1 * ldr);
    for (int64_t q = threadIdx.x; q < c0; q += blockDim.x) reinterpret_cast<float4*>(rows0)[q] = __ldg(g0 + q);
    for (int64_t q = threadIdx.x; q < c1; q += blockDim.x) reinterpret_cast<float4*>(rows1)[q] = __ldg(g1 + q);
    for (int64_t q = threadIdx.x; q < nr0; q += blockDim.x) rw0[q] = __ldg(P.w[0] + lo0 + q);
    for (int64_t q = threadIdx.x; q < nr1; q += blockDim.x) rw1[q] = __ldg(P.w[1] + lo1 + q);
  }
  if (threadIdx.x == 0) {
    mbar_init(s_gbar + 0, 1);
    mbar_init(s_gbar + 1, 1);
    fence_mbarrier_init();
    // first use of each gather buffer: every CTA of the cluster pushes ldr floats
    mbar_arrive_expect_tx(s_gbar + 0, CL * ldr * 4u);
    mbar_arrive_expect_tx(s_gbar + 1, CL * ldr * 4u);
  }
  if (A.table && rank == 0 && threadIdx.x == 0) {
    // batches: the record is cleared before the cluster barrier below, so before
    // any CTA can OR its status bits into it
    P.result->W = 0.0;
    P.result->residual = 0.0;
    P.result->status = 0;
    P.result->mode = LSF_MODE_STORED;
    P.result->reserved = 0;
  }
  // M = max_j shift_y(j) over the whole cloud (the start v = 1 as v~ = exp(shift - M))
  float m = -INFINITY;
  for (int64_t j = lo1 + threadIdx.x; j < hi1; j += blockDim.x) m = fmaxf(m, P.shift[1][j]);
  m = warp_max(m);
  if (lane == 0) s_fred[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = s_fred[0];
    for (int wq = 1; wq < kSmallWarps; ++wq) mm = fmaxf(mm, s_fred[wq]);
    s_fpart = mm;
  }
  // also orders every CTA's barrier setup before any push
  cluster.sync();
  float M = -INFINITY;
  for (unsigned rk = 0; rk < CL; ++rk) M = fmaxf(M, *cluster.map_shared_rank(&s_fpart, rk));
  if (rank == 0 && threadIdx.x == 0) {
    P.result->log_scale = static_cast<double>(M);
    P.result->iters = A.iters;
  }


  Exchange ex{gbuf, s_gbar, rank, CL, 0};
  const float* w0 = RES ? rw0 : P.w[0];
  const float* w1 = RES ? rw1 : P.w[1];
  float* s0 = RES ? rs0 : P.s[0];
  float* s1 = RES ? rs1 : P.s[1];
  const int64_t off0 = RES ? lo0 : 0, off1 = RES ? lo1 : 0;
  int flag = 0;
  small_half<C, RES, kHalfInit>(P.F[1], w1, P.shift[1], s1, off1, P.t[1], rows1, lo1, hi1, M, tb,
                                red, ldr, ex, flag);
  for (int it = 0; it < A.iters; ++it) {
    small_half<C, RES, kHalfUpdate>(P.F[0], w0, P.shift[0], s0, off0, P.t[0], rows0, lo0, hi0, M,
                                    tb, red, ldr, ex, flag);
    small_half<C, RES, kHalfUpdate>(P.F[1], w1, P.shift[1], s1, off1, P.t[1], rows1, lo1, hi1, M,
                                    tb, red, ldr, ex, flag);
  }
  const double res = small_half<C, RES, kHalfDot>(P.F[0], w0, P.shift[0], s0, off0, P.t[0], rows0,
                                                  lo0, hi0, M, tb, red, ldr, ex, flag);
  if (RES) {
    // the scalings go out once, at the end
    for (int64_t q = threadIdx.x; q < nr0; q += blockDim.x) P.s[0][lo0 + q] = rs0[q];
    for (int64_t q = threadIdx.x; q < nr1; q += blockDim.x) P.s[1][lo1 + q] = rs1[q];
  }
  if (lane == 0) s_dred[warp] = res;
  if (flag) atomicOr(&P.result->status, flag);
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int wq = 0; wq < kSmallWarps; ++wq) r += s_dred[wq];
    s_dpart = r;
  }
  cluster.sync();
  if (rank == 0 && threadIdx.x == 0) {
    double r = 0.0;
    for (unsigned rk = 0; rk < CL; ++rk) r += *cluster.map_shared_rank(&s_dpart, rk);
    P.result->residual = r;
  }
  // no CTA leaves while rank 0 may still read its shared memory
  cluster.sync();
}

int g_small_policy = 1;                  // 0 never, 1 by size, 2 whenever possible
int64_t g_small_max_entries = 1LL << 24;  // (n + m) * ldr limit of the size rule

size_t small_smem(int ldr, int64_t rows, bool res) {
  return sizeof(float) * (static_cast<size_t>(1 + kSmallWarps + 2 * kMaxCluster) * ldr +
                          (res ? static_cast<size_t>(rows) * (ldr + 2) : 0));
}

template <int C, bool RES>
int launch_small_c(const SmallArgs& a, int count, size_t smem, cudaStream_t st) {
  const int prefs[2] = {a.table ? 8 : 16, 8};
  void (*kern)(SmallArgs) = small_solve_kernel<C, RES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "small solve: smem attribute: %s", cudaGetErrorString(e));
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) (void)cudaGetLastError();
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kSmallThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int cl = 0;
  for (int want : prefs) {
    attr[0].val.clusterDim.x = want;
    cfg.gridDim = dim3(static_cast<unsigned>(want), 1, 1);
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e == cudaSuccess && nclusters > 0) {
      cl = want;
      break;
    }
    (void)cudaGetLastError();
  }
  if (cl == 0) return fail(LSF_ERR_UNSUPPORTED, "small solve: no cluster size can be scheduled");
  attr[0].val.clusterDim.x = cl;
  cfg.gridDim = dim3(static_cast<unsigned>(cl * count), 1, 1);
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "small solve: launch: %s", cudaGetErrorString(e));
  return check_launch("small_solve_kernel");
}

template <bool RES>
int launch_small(const SmallArgs& a, int count, size_t smem, cudaStream_t st) {
  switch (pass_columns(a.ldr)) {
    case 1: return launch_small_c<1, RES>(a, count, smem, st);
    case 2: return launch_small_c<2, RES>(a, count, smem, st);
    case 4: return launch_small_c<4, RES>(a, count, smem, st);
    default: return launch_small_c<8, RES>(a, count, smem, st);
  }
}

}  // namespace

bool small_solver_takes(int64_t n, int64_t m, int ldr) {
  if (g_small_policy == 0) return false;
  if (g_small_policy == 2) return true;
  return (n + m) * static_cast<int64_t>(ldr) <= g_small_max_entries;
}

int small_solve_table(const SProb* table, int count, int ldr, int iters, cudaStream_t st) {
  if (!table || count < 1) return fail(LSF_ERR_ARG, "small solve: empty problem table");
  SmallArgs a{};
  a.table = table;
  a.ldr = ldr;
  a.iters = iters;
  LaunchScope ls(st, LSF_KERNEL_SMALL, 0.0);
  return launch_small<false>(a, count, small_smem(ldr, 0, false), st);
}

int small_solve(const SProb* probs, int count, int ldr, int iters, cudaStream_t st) {
  if (count < 1 || count > kSmallMaxProblems) return fail(LSF_ERR_ARG, "small solve: 1..3 problems");
  SmallArgs a{};
  a.ldr = ldr;
  a.iters = iters;
  int64_t rows = 0;
  double bytes = 0.0;
  for (int p = 0; p < count; ++p) {
    a.probs[p] = probs[p];
    // rows of both sides held by one CTA of a 16-CTA cluster (8-CTA clusters need twice as many)
    const int64_t r8 = (probs[p].n[0] + 7) / 8 + (probs[p].n[1] + 7) / 8;
    rows = std::max(rows, r8);
    bytes += 4.0 * ldr * (probs[p].n[0] + probs[p].n[1]) * (2.0 * iters + 2.0);
  }
  const DeviceInfo& dev = device_info();
  const bool res = small_smem(ldr, rows, true) + 1024 <= static_cast<size_t>(dev.smem_optin);
  LaunchScope ls(st, LSF_KERNEL_SMALL, bytes);
  return res ? launch_small<true>(a, count, small_smem(ldr, rows, true), st)
             : launch_small<false>(a, count, small_smem(ldr, 0, false), st);
}

}  // namespace lsf

using namespace lsf;

extern "C" int lsf_set_small_solver(int policy, int64_t max_entries) {
  if (policy < 0 || policy > 2 || max_entries < 0)
    return fail(LSF_ERR_ARG, "lsf_set_small_solver: policy 0, 1 or 2 and max_entries >= 0");
  g_small_policy = policy;
  g_small_max_entries = max_entries;
  return LSF_OK;
}
