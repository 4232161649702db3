// Many weight vectors on one support: Alg. 1 for k right-hand sides at once, the
// fused pass written as a tensor-core contraction (tcgen05, TMEM accumulators,
// TMA-staged bf16 pair features).
//
// k pairs of weights (a_p, b_p), p < k, on the same points share the features of
// Sec. 3.1, so one half iteration of Alg. 1 for all of them is
//   S  = F T^T        n x kp   row products s_p = xi~ t_p         (T: kp x ldr2)
//   u_p = a_p / s_p             elementwise, per right-hand side
//   T' = U F          kp x ldr2 transposed products t'_p = xi~^T u_p
// two n x r x kp contractions that read F once. kp is k rounded up to 16 (the
// MMA's N granularity); the padding sides carry u = 0 and t = 0.
//
// Precision. F is stored as a pair of bf16 planes, hi = RN(F) and lo = RN(F - hi),
// so hi + lo equals F to 2^-16 relative (4 bytes per entry, as FP32). The small
// operands are split the same way each pass (T and U into hi, lo). The row
// products take all four terms (the stacked hi/lo operand makes lo*lo free), the
// transposed products hi*hi + hi*lo + lo*hi, accumulated in FP32 in TMEM; the
// dropped term is below 2^-16 relative.
//
// Kernel. One CTA per SM, persistent over tiles of 64 points. Per tile the
// producer warp streams the tile's feature chunks (64 points x 128 features,
// both planes, 32 KB, plus the chunk's block of [T_hi; T_lo]) into a shared-memory
// ring with TMA (128-byte swizzle), twice: first for the row products, then again
// (from L2, a tile later, evict-first) for the transposed products. One elected
// thread issues the MMAs:
//   row sweep:  D_S (128 x 2kp)   += [A_hi; A_lo] . [T_hi; T_lo]^T   A = F chunk, K-major,
//               the hi and lo boxes of a 64-feature half stacked as 128 rows
//   col sweep:  D_T[c] (128 x 2kp) += A_hi^T . [U_hi; U_lo],  (128 x kp) += A_lo^T . U_hi
//               A^T = the same smem chunk read MN-major (M = features, K = points),
//               no transposed copy (with 32 right-hand sides: three MMAs into kp columns)
// Four epilogue warps read D_S from TMEM (lanes 0-63: the hi plane's sums of the
// tile's points, lanes 64-127: the lo plane's); each warp pair hands the other its
// partial sums for the other half of the right-hand sides through shared memory,
// forms u = a / s for its half, writes it, splits it into bf16 hi/lo and stores it
// as the B operand of the col sweep. D_T holds this CTA's partial T' for the whole
// launch; at the end it is read out to a per-CTA slot and summed over the CTAs in
// a fixed order by a second kernel. 64-point tiles keep the data between a chunk's
// two reads at 256 KB per SM, which L2 holds for all SMs at once.
// Every wait is bounded; a wait that runs out sets LSF_ERR_TIMEOUT and the CTA
// still drains its copies and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "solve.cuh"

namespace lsf {
namespace {

constexpr int kTileRows = 64;                  // points per tile (M of the row product)
constexpr int kChunkCols = 128;                // features per chunk (M of the col product)
constexpr int kBoxCols = 64;                   // features per TMA box: 128 B of bf16
constexpr int kBoxBytes = kTileRows * kBoxCols * 2;   // 8 KB
constexpr int kStageBytes = 4 * kBoxBytes;     // two boxes of each plane: 32 KB
constexpr int kMultiThreads = 192;             // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kMaxStages = 6;
// Columns of the transposed-product accumulator of one feature chunk: with 16
// right-hand sides the hi and lo parts of the scalings are separate columns (two
// MMAs per K step, N = 2 kp and kp); with 32 they share kp columns (three MMAs of
// N = kp: F_hi U_hi, F_hi U_lo, F_lo U_hi), so that r = 1024 fits in TMEM.
__host__ __device__ constexpr int dt_cols(int kp) { return kp == 32 ? kp : 2 * kp; }

// Row chunks of a phase issued before its first transposed chunk: the slack the
// epilogue has to form the previous tile's scalings (measured best of 1..8: 2
// with 16 right-hand sides, 4 with 32, whose epilogue does twice the work).
__host__ __device__ constexpr int skew_chunks(int kp) { return kp == 32 ? 4 : 2; }

enum MultiMode : int { kMultiUpdate = 0, kMultiAxpy = 1, kMultiDot = 2 };

struct MultiArgs {
  int64_t n;
  int64_t ntiles;
  int ldr2;
  int k;             // real right-hand sides (<= kp)
  int mode;
  int nstages;
  int prefetch;        // row chunks requested into L2 ahead of the ring
  int l2_hints;        // 0 none, 1 evict-first on the re-read, 2 also evict-last on the first read
  int t_resident;      // the split r-vectors stay in shared memory for the launch (else a box per row chunk)
  uint32_t tmem_cols;
  const float* w;      // k x n weights (Update, Dot)
  const float* old;    // k x n previous scalings (Dot) or the given scalings (Axpy)
  float* out;          // k x n new scalings (Update)
  float* part;         // [grid][kp][ldr2] per-CTA partial T' (Update, Axpy)
  double* rpart;       // [grid][kp] per-CTA residual partials (Dot)
  lsf_result* res;     // k result records (status bits)
};

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of the sm_100 family
  d |= static_cast<uint64_t>(2) << 61;  // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(a_mn_major) << 15) |
         (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive TMEM columns of this warp's 32 lanes (lane i of the warp reads
// TMEM lane base + i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// TMA: one 64-feature x 128-point box of plane z at feature x, point y (the 3-D
// map of the feature planes), with an L2 eviction policy for the lines read.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int x, int y, int z,
                                        uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 policies: keep (a row chunk will be read again), drop first (its last read),
// or the default priority.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// L2 prefetch of one box of the 3-D feature map (no shared memory is written).
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(map),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}

// TMA: the r-vector map viewed as (64 features, 2 kp rows, ldr2 / 64 halves):
// two consecutive halves starting at half h.
__device__ __forceinline__ void tma_box3d_t(void* dst, const CUtensorMap* map, int h, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(0), "r"(0), "r"(h), "r"(smem_u32(bar))
      : "memory");
}

// Element (row, col) of a thread-written K-major operand region with the 128-byte
// swizzle: rows of 64 bf16 (128 B), 16-byte chunk c stored at c ^ (row % 8).
__device__ __forceinline__ int sw128(int row, int col) {
  return row * 64 + ((((col >> 3) ^ row) & 7) << 3) + (col & 7);
}

__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

// Shared memory of the pass. A ring stage holds one feature chunk (64 points x
// 128 features, both planes, 32 KB) as four 8 KB boxes [hi h=0 | lo h=0 | hi h=1 |
// lo h=1] (h: the 64-feature half), so that the hi and lo boxes of a half form
// one 128-row K-major operand, and, for a row-product item, the matching
// 128-feature block of the split r-vectors [T_hi; T_lo] (2 kp rows x 128
// features, loaded by TMA from the pair buffer the previous pass's reduction
// wrote).
struct MultiSmem {
  unsigned char* stages;  // [S][32 KB features | 2 x (2 kp x 128 B) r-vector boxes]
  uint16_t* sT;           // [ldr2 / 64][2 kp][64]: resident split r-vectors (t_resident)
  uint16_t* sU;           // [2][2 kp][64]: the split scalings of a tile, double-buffered
  float* xbuf;            // [2][64][kp]: lo-plane row products handed between epilogue warps
  uint64_t* full;         // [S]
  uint64_t* empty;        // [S]
  uint64_t* s_full;       // [2] row products of a tile in D_S[b]
  uint64_t* s_empty;      // [2] D_S[b] read out
  uint64_t* u_full;       // [2] sU[b] written
  uint64_t* u_empty;      // [2] sU[b] read by the transposed products
  uint64_t* t_done;       // every MMA of the launch completed
  uint64_t* t_full;       // resident r-vectors loaded
  uint32_t* tmem_slot;
  double* red;            // [4][kp]
};

__host__ __device__ inline int multi_tbox_bytes(int kp) { return 2 * kp * 128; }
__host__ __device__ inline int multi_stage_bytes(int kp, bool tres) {
  return kStageBytes + (tres ? 0 : 2 * multi_tbox_bytes(kp));
}
__host__ __device__ inline size_t multi_t_bytes(int kp, int ldr2, bool tres) {
  return tres ? static_cast<size_t>(ldr2 / kBoxCols) * multi_tbox_bytes(kp) : 0;
}

__host__ __device__ inline size_t multi_u_bytes(int kp) { return static_cast<size_t>(2 * kp) * kTileRows * 2; }

__host__ __device__ inline size_t multi_x_bytes(int kp) { return static_cast<size_t>(kTileRows) * kp * 4; }

__host__ __device__ inline size_t multi_smem_bytes(int kp, int stages, int ldr2, bool tres) {
  return 1024 + static_cast<size_t>(stages) * multi_stage_bytes(kp, tres) +
         multi_t_bytes(kp, ldr2, tres) + 2 * multi_u_bytes(kp) +
         2 * multi_x_bytes(kp) + 256 + static_cast<size_t>(4) * kp * 8;
}

__device__ __forceinline__ MultiSmem multi_layout(unsigned char* raw, int kp, int stages, int ldr2,
                                                  bool tres) {
  MultiSmem s;
  unsigned char* p = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                                      ~static_cast<uintptr_t>(1023));
  s.stages = p;
  p += static_cast<size_t>(stages) * multi_stage_bytes(kp, tres);
  s.sT = reinterpret_cast<uint16_t*>(p);
  p += multi_t_bytes(kp, ldr2, tres);
  s.sU = reinterpret_cast<uint16_t*>(p);
  p += 2 * multi_u_bytes(kp);
  s.xbuf = reinterpret_cast<float*>(p);
  p += 2 * multi_x_bytes(kp);
  uint64_t* b = reinterpret_cast<uint64_t*>(p);
  s.full = b;
  s.empty = b + kMaxStages;
  s.s_full = b + 2 * kMaxStages;
  s.s_empty = s.s_full + 2;
  s.u_full = s.s_full + 4;
  s.u_empty = s.s_full + 6;
  s.t_done = s.s_full + 8;
  s.t_full = s.s_full + 9;
  s.tmem_slot = reinterpret_cast<uint32_t*>(s.s_full + 10);
  p += 256;
  s.red = reinterpret_cast<double*>(p);
  return s;
}

// Bounded wait that suspends the thread in hardware (try_wait with a suspend-time
// hint) instead of spinning, so that waiting warps leave the issue slots to the
// MMA and TMA warps; false if kWaitLimitNs ran out.
__device__ __forceinline__ bool mbar_wait_suspend(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(200000u)
        : "memory");
    if (ok) return true;
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// Bounded wait by one lane, result broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait_suspend(bar, parity) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void flag_all(lsf_result* res, int k, int bits) {
  for (int p = 0; p < k; ++p) atomicOr(&res[p].status, bits);
}

// Order of the work of one CTA. Its tiles are j = 0 .. nt-1 (tile blockIdx.x +
// j gridDim.x). With both products (Update), phase ph interleaves the
// row-product chunks of tile ph (from HBM) with the transposed-product chunks
// of tile ph - 1 (re-read from L2): R(ph, 0), C(ph-1, 0), R(ph, 1), C(ph-1, 1),
// ...; so HBM loads stay in flight while tile ph - 1 finishes, and the
// scalings of tile ph - 1 are formed while R(ph, 0) runs. Dot runs R items
// only, Axpy C items only. The producer and the MMA issuer walk the same
// sequence.
struct Schedule {
  int nt, nchunks, lag;
  int skew;  // row chunks issued in a phase before its first transposed chunk
  bool rows, cols;
  __device__ int phases() const { return nt + lag; }
  __device__ bool c_on(int ph) const { return cols && ph - lag >= 0 && ph - lag < nt; }
  __device__ bool r_on(int ph) const { return rows && ph < nt; }
};

// ---------------------------------------------------------------- the pass kernel

template <int KP>
__global__ void __launch_bounds__(kMultiThreads, 1)
    multi_pass_kernel(const __grid_constant__ CUtensorMap fmap, const __grid_constant__ CUtensorMap tmap,
                      const MultiArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const bool rows = a.mode != kMultiAxpy;
  const bool cols = a.mode != kMultiDot;
  const bool tres = a.t_resident && rows;
  const MultiSmem sm = multi_layout(smem_raw, KP, a.nstages, a.ldr2, tres);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = a.ldr2 / kChunkCols;
  const int64_t n = a.n;
  const int stage_bytes = multi_stage_bytes(KP, tres);
  const int tbox = multi_tbox_bytes(KP);
  Schedule sch;
  sch.nt = static_cast<int>((a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  sch.nchunks = nchunks;
  sch.rows = rows;
  sch.cols = cols;
  sch.lag = (rows && cols) ? 1 : 0;
  sch.skew = (rows && cols) ? min(skew_chunks(KP), nchunks) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.nstages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.s_full[b], 1);
      mbar_init(&sm.s_empty[b], 128);
      mbar_init(&sm.u_full[b], 128);
      mbar_init(&sm.u_empty[b], 1);
    }
    mbar_init(sm.t_done, 1);
    mbar_init(sm.t_full, 1);
    fence_mbarrier_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(sm.tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sm.tmem_slot;
  const uint32_t tmem_S = tmem;             // D_S[b] at b * 2 kp
  const uint32_t tmem_T = tmem + 4 * KP;    // D_T[c] at c * dt_cols(kp)
  constexpr int kDT = dt_cols(KP);
  int err = 0;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    // L2 policy of the first (row) and the last (transposed) read of a chunk
    const uint64_t pol_r = a.l2_hints == 2 ? policy_evict_last() : policy_evict_normal();
    const uint64_t pol_c = a.l2_hints >= 1 ? policy_evict_first() : policy_evict_normal();
    auto issue = [&](int64_t tile, int c, bool with_t) -> bool {
      const uint64_t pol = with_t ? pol_r : pol_c;
      const int s = it % a.nstages;
      const uint32_t ph = static_cast<uint32_t>(it / a.nstages) & 1u;
      ++it;
      if (!warp_wait(&sm.empty[s], ph ^ 1u, lane)) return false;
      if (lane == 0) {
        unsigned char* dst = sm.stages + static_cast<size_t>(s) * stage_bytes;
        mbar_arrive_expect_tx(&sm.full[s], kStageBytes + (with_t ? 2 * tbox : 0));
        const int y = static_cast<int>(tile * kTileRows);
        const int x = c * kChunkCols;
        // a box spans both planes of a 64-feature half: [hi | lo], 16 KB
        tma_box(dst, &fmap, x, y, 0, &sm.full[s], pol);
        tma_box(dst + 2 * kBoxBytes, &fmap, x + kBoxCols, y, 0, &sm.full[s], pol);
        // the chunk's two 64-feature blocks of [T_hi; T_lo] in one box
        if (with_t) tma_box3d_t(dst + kStageBytes, &tmap, x / kBoxCols, &sm.full[s]);
      }
      __syncwarp();
      return true;
    };
    // Row chunks come from HBM: a.prefetch of them ahead are requested into L2
    // (no shared memory held), so more HBM requests are in flight than the ring
    // holds; the distance stays small because L2 must also keep each tile until
    // its transposed-product re-read.
    const int rtotal = rows ? sch.nt * nchunks : 0;
    auto prefetch = [&](int q) {
      if (lane != 0 || q >= rtotal) return;
      const int y = static_cast<int>((blockIdx.x + static_cast<int64_t>(q / nchunks) * gridDim.x) * kTileRows);
      const int x = (q % nchunks) * kChunkCols;
      tma_prefetch(&fmap, x, y, 0);
      tma_prefetch(&fmap, x + kBoxCols, y, 0);
      tma_prefetch(&fmap, x, y, 1);
      tma_prefetch(&fmap, x + kBoxCols, y, 1);
    };
    if (tres && lane == 0) {
      // the launch's r-vectors, once: one box per 64 features
      const int nb = a.ldr2 / kBoxCols;
      mbar_arrive_expect_tx(sm.t_full, static_cast<uint32_t>(nb * tbox));
      for (int b = 0; b < nb; b += 2)
        tma_box3d_t(reinterpret_cast<unsigned char*>(sm.sT) + b * tbox, &tmap, b, sm.t_full);
    }
    __syncwarp();
    for (int q = 0; q < a.prefetch; ++q) prefetch(q);
    int rq = 0;
    for (int ph = 0; ph < sch.phases() && !err; ++ph) {
      const int64_t tc = blockIdx.x + static_cast<int64_t>(ph - sch.lag) * gridDim.x;
      const int64_t tr = blockIdx.x + static_cast<int64_t>(ph) * gridDim.x;
      for (int i = 0; i < nchunks + sch.skew && !err; ++i) {
        if (sch.r_on(ph) && i < nchunks) {
          prefetch(rq + a.prefetch);
          ++rq;
          if (!issue(tr, i, !tres)) err = LSF_ERR_TIMEOUT;
        }
        if (!err && sch.c_on(ph) && i >= sch.skew && !issue(tc, i - sch.skew, false)) err = LSF_ERR_TIMEOUT;
      }
    }
    // drain: every issued copy has landed before the CTA may exit
    if (tres && !warp_wait(sm.t_full, 0u, lane)) err = LSF_ERR_TIMEOUT;
    const int used = min(it, a.nstages);
    for (int j = 0; j < used; ++j) {
      const int itj = it - 1 - j;
      if (!warp_wait(&sm.full[itj % a.nstages], static_cast<uint32_t>(itj / a.nstages) & 1u, lane))
        err = LSF_ERR_TIMEOUT;
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer (one thread)
    // row products: M = 128 = the 64 points of the hi plane stacked on those of
    // the lo plane; transposed products: M = 128 features
    constexpr uint32_t kRow = idesc_bf16(2 * kTileRows, 2 * KP, 0);
    constexpr uint32_t kColHi = idesc_bf16(kChunkCols, 2 * KP, 1);
    constexpr uint32_t kColLo = idesc_bf16(kChunkCols, KP, 1);
    constexpr bool kSplit3 = kDT == KP;
    // descriptors are built once; an operand at a byte offset o adds o >> 4 to
    // the start-address field (addresses stay below 256 KB: no carry)
    const uint32_t st_base = smem_u32(sm.stages);
    const uint32_t sU_base = smem_u32(sm.sU);
    const uint64_t dK0 = smem_desc(st_base, 16, 1024);         // K-major, 128-byte swizzle
    const uint64_t dM0 = smem_desc(st_base, 2 * kBoxBytes, 1024);  // MN-major A^T: halves 16 KB apart
    const uint32_t sT_off = smem_u32(sm.sT) - st_base;
    if (tres && !warp_wait(sm.t_full, 0u, lane)) err = LSF_ERR_TIMEOUT;
    int it = 0;
    auto take = [&](uint32_t& st) -> bool {
      const int s = it % a.nstages;
      const uint32_t ph = static_cast<uint32_t>(it / a.nstages) & 1u;
      ++it;
      // the TMA copy completed on this mbarrier: its bytes are visible to the
      // tensor core (both async proxy) without a tcgen05 fence
      if (!warp_wait(&sm.full[s], ph, lane)) return false;
      st = st_base + s * stage_bytes;
      return true;
    };
    auto release = [&]() {
      if (lane == 0) mma_commit(&sm.empty[(it - 1) % a.nstages]);
      __syncwarp();
    };
    for (int ph = 0; ph < sch.phases() && !err; ++ph) {
      const int jc = ph - sch.lag, jr = ph;
      const bool con = sch.c_on(ph), ron = sch.r_on(ph);
      if (ron && jr >= 2) {
        if (!warp_wait(&sm.s_empty[jr & 1], static_cast<uint32_t>((jr - 2) >> 1) & 1u, lane)) {
          err = LSF_ERR_TIMEOUT;
          break;
        }
        tc_fence_after();
      }
      const uint32_t dS = tmem_S + (jr & 1) * 2 * KP;
      const uint32_t sU_b = sU_base + (jc & 1) * static_cast<uint32_t>(multi_u_bytes(KP));
      for (int i = 0; i < nchunks + sch.skew && !err; ++i) {
        uint32_t st;
        if (ron && i < nchunks) {
          const int c = i;
          if (!take(st)) { err = LSF_ERR_TIMEOUT; break; }
          if (lane == 0) {
            const uint64_t ds = dK0 + ((st - st_base) >> 4);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                // A: the hi and lo boxes of half h (128 rows), B: [T_hi; T_lo] of half h
                const uint64_t ad = ds + ((h * 2 * kBoxBytes + ks * 32) >> 4);
                const uint64_t bd = tres ? dK0 + ((sT_off + (2 * c + h) * tbox + ks * 32) >> 4)
                                         : ds + ((kStageBytes + h * tbox + ks * 32) >> 4);
                mma_bf16(dS, ad, bd, kRow, (c | h | ks) != 0);
              }
            }
            // the tile's row products are complete once these MMAs are
            if (c == nchunks - 1) mma_commit(&sm.s_full[jr & 1]);
          }
          release();
        }
        if (con && i >= sch.skew) {
          const int c = i - sch.skew;
          if (c == 0) {
            // the scalings of tile jc, formed while this phase's first row chunks ran
            if (!warp_wait(&sm.u_full[jc & 1], static_cast<uint32_t>(jc >> 1) & 1u, lane)) {
              err = LSF_ERR_TIMEOUT;
              break;
            }
            tc_fence_after();
          }
          if (!take(st)) { err = LSF_ERR_TIMEOUT; break; }
          if (lane == 0) {
            const uint32_t dT = tmem_T + c * kDT;
            const uint64_t dm = dM0 + ((st - st_base) >> 4);
            const uint64_t du = dK0 + ((sU_b - st_base) >> 4);
#pragma unroll
            for (int ks = 0; ks < kTileRows / 16; ++ks) {
              // A^T: M = the chunk's 128 features (the two halves' boxes of a plane,
              // 16 KB apart), K = 16 points (two 8-point groups of 1024 B)
              const uint64_t bd = du + ((ks * 32) >> 4);
              if (kSplit3) {
                // U_lo: rows kp .. 2kp - 1 of the B operand, kp x 128 B further
                const uint64_t bd_lo = bd + ((KP * 128) >> 4);
                mma_bf16(dT, dm + ((ks * 2048) >> 4), bd, kColLo, (jc > 0 || ks > 0) ? 1 : 0);
                mma_bf16(dT, dm + ((ks * 2048) >> 4), bd_lo, kColLo, 1);
                mma_bf16(dT, dm + ((kBoxBytes + ks * 2048) >> 4), bd, kColLo, 1);
              } else {
                mma_bf16(dT, dm + ((ks * 2048) >> 4), bd, kColHi, (jc > 0 || ks > 0) ? 1 : 0);
                mma_bf16(dT, dm + ((kBoxBytes + ks * 2048) >> 4), bd, kColLo, 1);
              }
            }
            if (c == nchunks - 1) mma_commit(&sm.u_empty[jc & 1]);
          }
          release();
        }
      }
      if (err) break;
      __syncwarp();
    }
    if (lane == 0) mma_commit(sm.t_done);
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue warps 2..5
    // D_S has one TMEM lane per row of the stacked operand: lanes 0-63 hold the hi
    // plane's row products of the tile's 64 points, lanes 64-127 the lo plane's.
    // Warps on lanes 0-63 finish the first half of the right-hand sides of their
    // points and warps on lanes 64-127 the second half: each hands the other its
    // partial sums for the other half through shared memory. Waits that run out
    // are agreed on by all four warps at the per-tile named barrier, so they
    // leave together.
    const int quarter = warp & 3;               // TMEM lanes this warp may access
    const int half = quarter >> 1;              // 0: hi-plane lanes, 1: lo-plane lanes
    const int rloc = (quarter & 1) * 32 + lane;  // point within the tile
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    constexpr int kHalf = KP / 2;
    auto mine = [&](int p) { return (p >= kHalf) == (half == 1); };  // warp-uniform
    double resid[KP];
#pragma unroll
    for (int p = 0; p < KP; ++p) resid[p] = 0.0;
    uint32_t bad = 0u;
    bool fail = false;
    // with row products every exit goes through the per-tile named barrier, so the
    // loop itself must not stop a warp on its own; without them (Axpy) there is no
    // collective and a failed warp leaves at once
    for (int j = 0; j < sch.nt && !(fail && !rows); ++j) {
      const int64_t row = (blockIdx.x + static_cast<int64_t>(j) * gridDim.x) * kTileRows + rloc;
      const bool valid = row < n && !fail;
      // this tile's weights (and previous scalings) of my half, fetched before the wait
      float w[KP], o[KP];
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        const bool on = p < a.k && valid && mine(p);
        w[p] = (on && rows) ? __ldg(a.w + p * n + row) : 0.f;
        o[p] = (on && a.mode != kMultiUpdate) ? __ldg(a.old + p * n + row) : 0.f;
      }
      float u[KP];
      if (rows) {
        if (!fail && !warp_wait(&sm.s_full[j & 1], static_cast<uint32_t>(j >> 1) & 1u, lane)) {
          fail = true;
          err = LSF_ERR_TIMEOUT;
        }
        tc_fence_after();
        float d[2 * KP];
#pragma unroll
        for (int h = 0; h < 2 * KP / 32; ++h) {
          float v[32];
          tmem_ld32(tmem_S + (j & 1) * 2 * KP + lane_base + 32 * h, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) d[32 * h + i] = v[i];
        }
        tc_fence_before();
        mbar_arrive(&sm.s_empty[j & 1]);
        float* xb = sm.xbuf + (j & 1) * (KP * kTileRows);
#pragma unroll
        for (int p = 0; p < KP; ++p)
          if (!mine(p)) xb[p * kTileRows + rloc] = d[p] + d[KP + p];
        // all four warps: the hand-over is visible, and nobody has failed
        int all_ok;
        asm volatile(
            "{\n\t.reg .pred q, r;\n\tsetp.ne.b32 q, %1, 0;\n\t"
            "bar.red.and.pred r, 1, 128, q;\n\tselp.u32 %0, 1, 0, r;\n\t}"
            : "=r"(all_ok)
            : "r"(fail ? 0 : 1)
            : "memory");
        if (!all_ok) {
          err |= LSF_ERR_TIMEOUT;
          break;
        }
        // (the mode is tested once, outside the unrolled loops, so that an update
        // launch issues none of the residual's FP64 instructions)
        if (a.mode == kMultiUpdate) {
#pragma unroll
          for (int p = 0; p < KP; ++p) {
            u[p] = 0.f;
            if (mine(p) && p < a.k && valid) {
              // hi-plane part + lo-plane part (the same sum on either side)
              const float sp = (d[p] + d[KP + p]) + xb[p * kTileRows + rloc];
              const float v = w[p] * __frcp_rn(sp);
              if (!(v > 0.f && v < INFINITY)) bad |= 1u << p;
              u[p] = v;
            }
          }
        } else {
#pragma unroll
          for (int p = 0; p < KP; ++p) {
            u[p] = 0.f;
            if (mine(p) && p < a.k && valid) {
              const float sp = (d[p] + d[KP + p]) + xb[p * kTileRows + rloc];
              resid[p] += fabs(static_cast<double>(o[p]) * static_cast<double>(sp) - static_cast<double>(w[p]));
            }
          }
        }
      } else {
#pragma unroll
        for (int p = 0; p < KP; ++p) u[p] = o[p];
      }
      if (cols) {
        if (!fail && j >= 2 &&
            !warp_wait(&sm.u_empty[j & 1], static_cast<uint32_t>((j - 2) >> 1) & 1u, lane)) {
          fail = true;
          err = LSF_ERR_TIMEOUT;
        }
        uint16_t* sUb = sm.sU + (j & 1) * (2 * KP * kTileRows);
        if (!fail) {
#pragma unroll
          for (int p = 0; p < KP; ++p) {
            if (!mine(p)) continue;
            uint16_t hi, lo;
            split_bf16(u[p], hi, lo);
            sUb[sw128(p, rloc)] = hi;
            sUb[sw128(KP + p, rloc)] = lo;
          }
          fence_async_smem();
          mbar_arrive(&sm.u_full[j & 1]);
        }
      }
      // the new scalings to global memory, off the MMA issuer's critical path
      if (a.mode == kMultiUpdate) {
#pragma unroll
        for (int p = 0; p < KP; ++p)
          if (mine(p) && p < a.k && valid) a.out[p * n + row] = u[p];
      }
    }
    // the launch's partial T' (this CTA's points) out of TMEM
    if (cols && !err) {
      if (!warp_wait(sm.t_done, 0u, lane)) {
        err = LSF_ERR_TIMEOUT;
      } else {
        tc_fence_after();
        float* dst = a.part + static_cast<size_t>(blockIdx.x) * KP * a.ldr2;
        for (int c = 0; c < nchunks; ++c) {
          float d[kDT];
#pragma unroll
          for (int h = 0; h < kDT / 32; ++h) {
            float v[32];
            tmem_ld32(tmem_T + c * kDT + lane_base + 32 * h, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) d[32 * h + i] = v[i];
          }
          const int f = c * kChunkCols + quarter * 32 + lane;  // M = 128: lane = feature
#pragma unroll
          for (int p = 0; p < KP; ++p)
            dst[static_cast<size_t>(p) * a.ldr2 + f] = kDT == KP ? d[p] : d[p] + d[(KP + p) % kDT];
        }
      }
    }
    if (a.mode == kMultiDot) {
      // fixed-order fold of the residual terms: lanes, then the four warps
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        double v = resid[p];
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
        if (lane == 0) sm.red[quarter * KP + p] = v;
      }
    }
#pragma unroll
    for (int p = 0; p < KP; ++p) {
      const unsigned any = __ballot_sync(0xffffffffu, (bad >> p) & 1u);
      if (any && lane == 0) atomicOr(&a.res[p].status, LSF_ERR_NONFINITE);
    }
  }
  if (err && lane == 0) flag_all(a.res, a.k, err);
  tc_fence_before();
  __syncthreads();
  if (a.mode == kMultiDot && threadIdx.x < KP) {
    const int p = threadIdx.x;
    a.rpart[static_cast<size_t>(blockIdx.x) * KP + p] =
        sm.red[0 * KP + p] + sm.red[1 * KP + p] + sm.red[2 * KP + p] + sm.red[3 * KP + p];
  }
  if (warp == 1) {
    // every MMA has completed: the issuer's last commit (t_done) tracks all of them
    if (!warp_wait(sm.t_done, 0u, lane) && lane == 0) flag_all(a.res, a.k, LSF_ERR_TIMEOUT);
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols)
                 : "memory");
  }
}

// Sum of the per-CTA partials in CTA order: a block covers 32 outputs with 8
// warps, warp w summing CTAs w, w + 8, ...; the 8 warp sums are folded in order.
// Also writes the bf16 split of the result, [T_hi; T_lo] (2 kp x ldr2), which
// the next pass's row products load with TMA.
__global__ void __launch_bounds__(256) multi_reduce_kernel(const float* __restrict__ part, int G,
                                                           int kp, int ldr2, float* __restrict__ t_out,
                                                           uint16_t* __restrict__ t_pair) {
  __shared__ double s[8][33];
  const int total = kp * ldr2;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (idx < total)
    for (int g = w; g < G; g += 8) acc += static_cast<double>(__ldcg(part + static_cast<size_t>(g) * total + idx));
  s[w][lane] = acc;
  __syncthreads();
  if (w == 0 && idx < total) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += s[i][lane];
    const float tf = static_cast<float>(t);
    t_out[idx] = tf;
    uint16_t hi, lo;
    split_bf16(tf, hi, lo);
    t_pair[idx] = hi;           // row p of the hi block
    t_pair[total + idx] = lo;   // row kp + p: the lo block
  }
}

__global__ void multi_residual_kernel(const double* __restrict__ rpart, int G, int kp, int k,
                                      lsf_result* res) {
  const int p = threadIdx.x;
  if (p >= k) return;
  KahanSum s;
  for (int g = 0; g < G; ++g) s.add(rpart[static_cast<size_t>(g) * kp + p]);
  res[p].residual = s.value();
}

__global__ void multi_max_kernel(const float* __restrict__ x, int64_t n, unsigned* __restrict__ key) {
  float best = -INFINITY;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    best = fmaxf(best, x[i]);
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) atomicMax(key, float_key(best));
}

// v = 1 for every right-hand side in shifted form: v~_j = exp(shift_j - M).
__global__ void multi_init_kernel(const float* __restrict__ shift, int64_t n, int k,
                                  const unsigned* __restrict__ key, float* __restrict__ V,
                                  lsf_result* res) {
  const float M = key_float(*key);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float v = expf(shift[i] - M);
    for (int p = 0; p < k; ++p) V[p * n + i] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x < k) res[threadIdx.x].log_scale = static_cast<double>(M);
}

// Eq. (2) per weight pair from the three terms' Eq. (6) values:
// wbar[p] = W(a_p, b_p) - (W(a_p, a_p) + W(b_p, b_p)) / 2. The three records of a
// pair report their status bits jointly, as the single-pair debiased solve does.
__global__ void multi_debias_kernel(lsf_result* rxy, lsf_result* rxx, lsf_result* ryy, int k,
                                    double* wbar) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= k) return;
  if (wbar) wbar[p] = rxy[p].W - 0.5 * (rxx[p].W + ryy[p].W);
  const int32_t s = rxy[p].status | rxx[p].status | ryy[p].status;
  rxy[p].status = s;
  rxx[p].status = s;
  ryy[p].status = s;
}

__global__ void multi_iters_kernel(lsf_result* res, int k, int iters) {
  if (static_cast<int>(threadIdx.x) < k) {
    res[threadIdx.x].iters = iters;
    res[threadIdx.x].mode = LSF_MODE_STORED;
    res[threadIdx.x].reserved = 0;
  }
}

// bf16 pair planes from stored FP32 features (zero beyond r).
__global__ void split_features_kernel(const float* __restrict__ F, int64_t n, int ldr, int r,
                                      uint16_t* __restrict__ F2, int ldr2) {
  const int64_t total = n * ldr2;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / ldr2;
    const int k = static_cast<int>(idx - i * ldr2);
    const float f = k < r ? F[i * ldr + k] : 0.f;
    uint16_t hi, lo;
    split_bf16(f, hi, lo);
    F2[idx] = hi;
    F2[total + idx] = lo;
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q{};
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of the two bf16 planes: dims (ldr2, n, 2), boxes of 64 features x
// 64 points x both planes ([hi | lo], 16 KB), 128-byte swizzle; rows past n read
// as zeros.
int make_pair_map(const uint16_t* F2, int64_t n, int ldr2, CUtensorMap* map) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(LSF_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  if (reinterpret_cast<uintptr_t>(F2) % 256 != 0)
    return fail(LSF_ERR_ARG, "F2 must be 256-byte aligned");
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(ldr2), static_cast<cuuint64_t>(n), 2};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ldr2) * 2, static_cast<cuuint64_t>(n) * ldr2 * 2};
  cuuint32_t box[3] = {kBoxCols, kTileRows, 2};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(F2), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(LSF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return LSF_OK;
}

// Tensor map of a split r-vector block [T_hi; T_lo] (2 kp rows x ldr2 bf16),
// viewed as (64 features, 2 kp rows, ldr2 / 64 halves): a box of two halves
// lands as two K-major B operands of 2 kp rows x 128 B (128-byte swizzle).
int make_t_map(const uint16_t* t_pair, int kp, int ldr2, CUtensorMap* map) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(LSF_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(kBoxCols), static_cast<cuuint64_t>(2 * kp),
                        static_cast<cuuint64_t>(ldr2 / kBoxCols)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ldr2) * 2, static_cast<cuuint64_t>(kBoxCols) * 2};
  cuuint32_t box[3] = {kBoxCols, static_cast<cuuint32_t>(2 * kp), 2};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(t_pair), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(LSF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return LSF_OK;
}

int multi_kp(int k) { return k <= 16 ? 16 : 32; }

int g_multi_prefetch = 0;  // row chunks prefetched into L2 (lsf_set_multi_tuning)
int g_multi_l2_hints = 1;  // L2 eviction hints of the chunk reads (lsf_set_multi_tuning)
int g_multi_t_resident = 0;  // split r-vectors resident in shared memory (lsf_set_multi_tuning)

// TMEM columns: D_S double-buffered (2 x 2 kp) and one 2 kp block per feature chunk.
int tmem_need(int kp, int ldr2) { return 4 * kp + dt_cols(kp) * (ldr2 / kChunkCols); }

uint32_t tmem_columns(int kp, int ldr2) {
  uint32_t c = 32;
  while (static_cast<int>(c) < tmem_need(kp, ldr2)) c <<= 1;
  return c;
}

// The shapes this kernel takes: ldr2 a multiple of 128 up to 1024, k <= 32, the
// accumulators within TMEM's 512 columns and two ring stages in shared memory.
int check_multi_shape(int ldr2, int k) {
  if (k < 1 || k > 32) return fail(LSF_ERR_UNSUPPORTED, "multi solve: k must be in [1, 32]");
  if (ldr2 < 128 || ldr2 % 128 != 0 || ldr2 > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "multi solve: ldr2 must be a multiple of 128 in [128, 1024]");
  const int kp = multi_kp(k);
  if (tmem_need(kp, ldr2) > 512)
    return fail(LSF_ERR_UNSUPPORTED, "multi solve: %d right-hand sides at ldr2 = %d exceed TMEM", k, ldr2);
  if (multi_smem_bytes(kp, 2, ldr2, false) > static_cast<size_t>(device_info().smem_optin))
    return fail(LSF_ERR_UNSUPPORTED, "multi solve: shared memory too small");
  return LSF_OK;
}

int multi_grid_max() { return device_info().sms; }

size_t align256m(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

size_t multi_extra_bytes(int ldr2, int kp) {
  const size_t G = static_cast<size_t>(multi_grid_max());
  return align256m(G * kp * ldr2 * sizeof(float)) + align256m(G * kp * sizeof(double)) +
         2 * align256m(static_cast<size_t>(kp) * ldr2 * 4);
}

struct MultiWs {
  Workspace ws;
  float* part;
  double* rpart;
  uint16_t* t_pair[2];  // bf16 splits of Tu (0) and Tv (1)
};

template <int KP>
int launch_multi_kp(const MultiArgs& a0, const CUtensorMap& fmap, const CUtensorMap& tmap,
                    cudaStream_t st, int* grid_out) {
  MultiArgs a = a0;
  const size_t optin = static_cast<size_t>(device_info().smem_optin);
  // resident r-vectors when they leave room for at least 4 ring stages
  const bool tres = g_multi_t_resident && a.mode != kMultiAxpy &&
                    multi_smem_bytes(KP, 4, a.ldr2, true) <= optin;
  int stages = kMaxStages;
  while (stages > 2 && multi_smem_bytes(KP, stages, a.ldr2, tres) > optin) --stages;
  const size_t smem = multi_smem_bytes(KP, stages, a.ldr2, tres);
  a.t_resident = tres ? 1 : 0;
  if (smem > optin) return fail(LSF_ERR_UNSUPPORTED, "multi pass: %zu bytes of shared memory", smem);
  a.nstages = stages;
  a.prefetch = g_multi_prefetch;
  a.l2_hints = g_multi_l2_hints;
  a.tmem_cols = tmem_columns(KP, a.ldr2);
  static int configured[2] = {0, 0};
  const int dev = device_info().device;
  if (configured[KP == 32] != dev + 1) {
    if (cudaFuncSetAttribute(multi_pass_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(optin)) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "multi pass: cannot raise the shared-memory limit");
    configured[KP == 32] = dev + 1;
  }
  const int grid = static_cast<int>(std::min<int64_t>(multi_grid_max(), a.ntiles));
  const double bytes = static_cast<double>(a.n) * a.ldr2 * 4.0 +
                       static_cast<double>(a.n) * a.k * 4.0 * (a.mode == kMultiAxpy ? 1 : 2);
  {
    LaunchScope ls(st, LSF_KERNEL_PASS_MULTI, bytes);
    multi_pass_kernel<KP><<<grid, kMultiThreads, smem, st>>>(fmap, tmap, a);
    LSF_TRY(check_launch("multi_pass_kernel"));
  }
  *grid_out = grid;
  return LSF_OK;
}

// One pass and its reduction. tmap: the split r-vectors the row products read
// (Update, Dot); t_out, t_pair_out: the reduced transposed products and their
// split (Update, Axpy). Returns LSF_OK or an error status.
int multi_pass(int mode, int k, int64_t n, int ldr2, const CUtensorMap& fmap, const CUtensorMap& tmap,
               const float* w, const float* old, float* out, float* t_out, uint16_t* t_pair_out,
               lsf_result* res, const MultiWs& mw, cudaStream_t st) {
  const int kp = multi_kp(k);
  MultiArgs a{};
  a.n = n;
  a.ntiles = (n + kTileRows - 1) / kTileRows;
  a.ldr2 = ldr2;
  a.k = k;
  a.mode = mode;
  a.w = w;
  a.old = old;
  a.out = out;
  a.part = mw.part;
  a.rpart = mw.rpart;
  a.res = res;
  int grid = 0;
  LSF_TRY(kp == 16 ? launch_multi_kp<16>(a, fmap, tmap, st, &grid)
                   : launch_multi_kp<32>(a, fmap, tmap, st, &grid));
  LaunchScope ls(st, LSF_KERNEL_OTHER, 4.0 * grid * kp * ldr2);
  if (mode == kMultiDot) {
    multi_residual_kernel<<<1, 32, 0, st>>>(mw.rpart, grid, kp, k, res);
    return check_launch("multi_residual_kernel");
  }
  const int total = kp * ldr2;
  multi_reduce_kernel<<<(total + 31) / 32, 256, 0, st>>>(mw.part, grid, kp, ldr2, t_out, t_pair_out);
  return check_launch("multi_reduce_kernel");
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_split_features(const float* F, int64_t n, int ldr, int r, uint16_t* F2, int ldr2,
                       void* stream) {
  if (!F || !F2) return fail(LSF_ERR_ARG, "lsf_split_features: NULL pointer");
  if (n < 1 || r < 1 || r > ldr || r > ldr2) return fail(LSF_ERR_ARG, "lsf_split_features: bad sizes");
  if (ldr2 % 128 != 0 || ldr2 > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "lsf_split_features: ldr2 must be a multiple of 128, <= 1024");
  cudaStream_t st = as_stream(stream);
  const int grid = device_info().sms * 4;
  LaunchScope ls(st, LSF_KERNEL_FEATURES, static_cast<double>(n) * (4.0 * ldr + 4.0 * ldr2));
  split_features_kernel<<<grid, 256, 0, st>>>(F, n, ldr, r, F2, ldr2);
  return check_launch("split_features_kernel");
}

int lsf_set_multi_tuning(int prefetch_chunks, int l2_hints, int r_vectors_resident) {
  if (prefetch_chunks < 0 || prefetch_chunks > 16)
    return fail(LSF_ERR_ARG, "lsf_set_multi_tuning: prefetch_chunks must be in [0, 16]");
  if (l2_hints < 0 || l2_hints > 2) return fail(LSF_ERR_ARG, "lsf_set_multi_tuning: l2_hints must be 0, 1 or 2");
  if (r_vectors_resident < 0 || r_vectors_resident > 1)
    return fail(LSF_ERR_ARG, "lsf_set_multi_tuning: r_vectors_resident must be 0 or 1");
  g_multi_prefetch = prefetch_chunks;
  g_multi_l2_hints = l2_hints;
  g_multi_t_resident = r_vectors_resident;
  return LSF_OK;
}

int lsf_multi_workspace_bytes(int ldr2, int k, size_t* bytes) {
  if (!bytes) return fail(LSF_ERR_ARG, "lsf_multi_workspace_bytes: NULL output");
  LSF_TRY(check_multi_shape(ldr2, k));
  *bytes = align256m(workspace_bytes(ldr2)) + multi_extra_bytes(ldr2, multi_kp(k));
  return LSF_OK;
}

int lsf_solve_multi(const lsf_theta* theta, int ldr2, const lsf_multi_cloud* x,
                    const lsf_multi_cloud* y, int k, int iters, const lsf_multi_scalings* out,
                    lsf_result* results, void* workspace, size_t ws_bytes, void* stream) {
  lsf::TraceRange trace_range("lsf_solve_multi");
  LSF_TRY(check_theta(theta));
  LSF_TRY(check_multi_shape(ldr2, k));
  if (theta->r > ldr2) return fail(LSF_ERR_ARG, "multi solve: r exceeds ldr2");
  if (!x || !y || !out || !results) return fail(LSF_ERR_ARG, "multi solve: NULL argument");
  if (x->n < 1 || y->n < 1) return fail(LSF_ERR_ARG, "multi solve: a measure needs n >= 1 points");
  if (!x->F2 || !y->F2 || !x->shift || !y->shift || !x->W || !y->W)
    return fail(LSF_ERR_ARG, "multi solve: F2, shift and W are required on both sides");
  if (!out->U || !out->V || !out->Tu || !out->Tv)
    return fail(LSF_ERR_ARG, "multi solve: U, V, Tu, Tv are required");
  if (iters < 1) return fail(LSF_ERR_ARG, "iters must be >= 1");
  if (x->n > (int64_t(1) << 31) - kTileRows || y->n > (int64_t(1) << 31) - kTileRows)
    return fail(LSF_ERR_UNSUPPORTED, "multi solve: too many points for 32-bit TMA coordinates");
  const int kp = multi_kp(k);
  size_t need = 0;
  LSF_TRY(lsf_multi_workspace_bytes(ldr2, k, &need));
  if (ws_bytes < need)
    return fail(LSF_ERR_WORKSPACE, "multi solve: workspace has %zu bytes, needs %zu", ws_bytes, need);
  cudaStream_t st = as_stream(stream);
  MultiWs mw{};
  LSF_TRY(start_solve(workspace, ws_bytes, ldr2, results, k, &mw.ws, st));
  char* p = static_cast<char*>(workspace) + align256m(workspace_bytes(ldr2));
  mw.part = reinterpret_cast<float*>(p);
  p += align256m(static_cast<size_t>(multi_grid_max()) * kp * ldr2 * sizeof(float));
  mw.rpart = reinterpret_cast<double*>(p);
  p += align256m(static_cast<size_t>(multi_grid_max()) * kp * sizeof(double));
  mw.t_pair[0] = reinterpret_cast<uint16_t*>(p);
  p += align256m(static_cast<size_t>(kp) * ldr2 * 4);
  mw.t_pair[1] = reinterpret_cast<uint16_t*>(p);
  CUtensorMap mx, my, mtu, mtv;
  LSF_TRY(make_pair_map(x->F2, x->n, ldr2, &mx));
  LSF_TRY(make_pair_map(y->F2, y->n, ldr2, &my));
  LSF_TRY(make_t_map(mw.t_pair[0], kp, ldr2, &mtu));
  LSF_TRY(make_t_map(mw.t_pair[1], kp, ldr2, &mtv));
  if (cudaMemsetAsync(out->Tu, 0, sizeof(float) * kp * ldr2, st) != cudaSuccess ||
      cudaMemsetAsync(out->Tv, 0, sizeof(float) * kp * ldr2, st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "multi solve: memset failed");
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 8.0 * y->n * (1 + k));
    const int grid = device_info().sms * 2;
    multi_max_kernel<<<grid, 256, 0, st>>>(y->shift, y->n, mw.ws.keys);
    multi_init_kernel<<<grid, 256, 0, st>>>(y->shift, y->n, k, mw.ws.keys, out->V, results);
    LSF_TRY(check_launch("multi_init_kernel"));
  }
  // t_v = zeta~^T v~ from v = 1; then u-halves (row products with t_v) and v-halves
  LSF_TRY(multi_pass(kMultiAxpy, k, y->n, ldr2, my, mtv, nullptr, out->V, nullptr, out->Tv,
                     mw.t_pair[1], results, mw, st));
  for (int it = 0; it < iters; ++it) {
    LSF_TRY(multi_pass(kMultiUpdate, k, x->n, ldr2, mx, mtv, x->W, nullptr, out->U, out->Tu,
                       mw.t_pair[0], results, mw, st));
    LSF_TRY(multi_pass(kMultiUpdate, k, y->n, ldr2, my, mtu, y->W, nullptr, out->V, out->Tv,
                       mw.t_pair[1], results, mw, st));
  }
  LSF_TRY(multi_pass(kMultiDot, k, x->n, ldr2, mx, mtv, x->W, out->U, nullptr, nullptr, nullptr,
                     results, mw, st));
  {
    LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
    multi_iters_kernel<<<1, 32, 0, st>>>(results, k, iters);
    LSF_TRY(check_launch("multi_iters_kernel"));
  }
  // Eq. (6) for every right-hand side, three per reduction launch
  for (int p0 = 0; p0 < k; p0 += 3) {
    const int nt = std::min(3, k - p0);
    lsf_cloud cx[3], cy[3];
    lsf_scalings ss[3];
    const lsf_cloud* xs[3];
    const lsf_cloud* ys[3];
    const lsf_scalings* sp[3];
    lsf_result* rs[3];
    for (int t = 0; t < nt; ++t) {
      const int q = p0 + t;
      cx[t] = lsf_cloud{nullptr, nullptr, x->shift, x->W + static_cast<int64_t>(q) * x->n, x->n};
      cy[t] = lsf_cloud{nullptr, nullptr, y->shift, y->W + static_cast<int64_t>(q) * y->n, y->n};
      ss[t] = lsf_scalings{out->U + static_cast<int64_t>(q) * x->n, out->V + static_cast<int64_t>(q) * y->n,
                           nullptr, nullptr};
      xs[t] = &cx[t];
      ys[t] = &cy[t];
      sp[t] = &ss[t];
      rs[t] = results + q;
    }
    LSF_TRY(launch_divergence(theta, nt, xs, ys, sp, rs, nullptr, nullptr, mw.ws, st, 0));
  }
  return LSF_OK;
}

int lsf_multi_debiased(const lsf_theta* theta, int ldr2, const lsf_multi_cloud* x,
                       const lsf_multi_cloud* y, int k, int iters, const lsf_multi_scalings* s_xy,
                       const lsf_multi_scalings* s_xx, const lsf_multi_scalings* s_yy,
                       lsf_result* results, double* wbar, void* workspace, size_t ws_bytes,
                       void* stream) {
  lsf::TraceRange trace_range("lsf_multi_debiased");
  if (!x || !y || !results) return fail(LSF_ERR_ARG, "lsf_multi_debiased: NULL argument");
  if (k < 1 || k > 32) return fail(LSF_ERR_UNSUPPORTED, "lsf_multi_debiased: k must be 1..32");
  LSF_TRY(lsf_solve_multi(theta, ldr2, x, y, k, iters, s_xy, results, workspace, ws_bytes, stream));
  LSF_TRY(lsf_solve_multi(theta, ldr2, x, x, k, iters, s_xx, results + k, workspace, ws_bytes, stream));
  LSF_TRY(lsf_solve_multi(theta, ldr2, y, y, k, iters, s_yy, results + 2 * k, workspace, ws_bytes, stream));
  cudaStream_t st = as_stream(stream);
  LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
  multi_debias_kernel<<<1, 32, 0, st>>>(results, results + k, results + 2 * k, k, wbar);
  return check_launch("multi_debias_kernel");
}

}  // extern "C"
