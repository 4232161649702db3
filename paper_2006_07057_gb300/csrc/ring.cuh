// Shared-memory copy ring used by the stored-feature passes: a producer warp
// streams tiles of consecutive feature rows into S stages with one bulk TMA copy
// each (cp.async.bulk), plus the per-row vectors (weights, previous scalings)
// with 4-byte cp.async, all completing on the stage's "full" mbarrier; the
// consumer warps release a stage on its "empty" mbarrier.
#pragma once

#include "pass.cuh"

namespace lsf {

struct Ring {
  uint64_t* full;   // [S]
  uint64_t* empty;  // [S]
  float* sF;        // [S][TR][ldr]
  float* sV;        // [S][NRHS][2][TR]: weights, previous scalings
  int S, TR, ldr;
};

__device__ __forceinline__ Ring ring_layout(unsigned char* smem, int S, int TR, int ldr) {
  Ring r;
  r.full = reinterpret_cast<uint64_t*>(smem);
  r.empty = r.full + S;
  r.sF = reinterpret_cast<float*>(smem + 128 * ((16 * S + 127) / 128));
  r.sV = r.sF + static_cast<size_t>(S) * TR * ldr;
  r.S = S;
  r.TR = TR;
  r.ldr = ldr;
  return r;
}

// Host side: bytes of dynamic shared memory for S stages of TR rows.
inline size_t ring_bytes(int S, int64_t TR, int ldr, int nrhs) {
  return 128 * ((16 * static_cast<size_t>(S) + 127) / 128) +
         static_cast<size_t>(S) * (static_cast<size_t>(TR) * ldr * 4 + static_cast<size_t>(nrhs) * 2 * TR * 4);
}

// Thread 0: initialise the stage barriers (expect_tx arrival + 32 cp.async
// arrivals per fill; one arrival per consumer warp per release).
__device__ __forceinline__ void ring_init(const Ring& r, int consumer_warps) {
  for (int s = 0; s < r.S; ++s) {
    mbar_init(&r.full[s], 1 + 32);
    mbar_init(&r.empty[s], consumer_warps);
  }
}

// The producer warp's whole job: fill stages for tiles blockIdx.x, +gridDim.x, ...
// then wait (bounded) until every issued copy has landed. copy_w: also copy the
// weights; old vectors are copied where non-NULL.
template <int NRHS>
__device__ __forceinline__ void ring_produce(const Ring& r, const float* F, int64_t n, int64_t ntiles,
                                             const PassRhs* rhs, bool copy_w, int lane, int& flag) {
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it % r.S;
    const uint32_t ph = static_cast<uint32_t>(it / r.S) & 1u;
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(&r.empty[s], ph ^ 1u) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      flag |= LSF_ERR_TIMEOUT;
      break;
    }
    const int64_t row0 = tile * r.TR;
    const int rows = static_cast<int>(min(static_cast<int64_t>(r.TR), n - row0));
    if (lane == 0) {
      const uint32_t bytes = static_cast<uint32_t>(rows) * static_cast<uint32_t>(r.ldr) * 4u;
      mbar_arrive_expect_tx(&r.full[s], bytes);
      bulk_copy_g2s(r.sF + static_cast<size_t>(s) * r.TR * r.ldr, F + row0 * r.ldr, bytes, &r.full[s]);
    }
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      float* dw = r.sV + static_cast<size_t>((s * NRHS + k) * 2) * r.TR;
      float* dold = dw + r.TR;
      const float* w = rhs[k].w;
      const float* old = rhs[k].old;
      for (int i = lane; i < rows; i += 32) {
        if (copy_w) cp_async_4(dw + i, w + row0 + i);
        if (old) cp_async_4(dold + i, old + row0 + i);
      }
    }
    cp_async_mbar_arrive(&r.full[s]);
  }
  const int used = min(it, r.S);
  for (int j = 0; j < used; ++j) {
    const int itj = it - 1 - j;
    const int s = itj % r.S;
    const uint32_t ph = static_cast<uint32_t>(itj / r.S) & 1u;
    if (lane == 0 && !mbar_wait_bounded(&r.full[s], ph)) flag |= LSF_ERR_TIMEOUT;
  }
}

// Consumer side: wait (bounded) until the stage of the it-th tile is full.
__device__ __forceinline__ bool ring_wait_full(const Ring& r, int it, int lane,
                                               unsigned long long limit_ns = kWaitLimitNs) {
  const int s = it % r.S;
  const uint32_t ph = static_cast<uint32_t>(it / r.S) & 1u;
  int ok = 1;
  if (lane == 0) ok = mbar_wait_bounded(&r.full[s], ph, limit_ns) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Fold RW per-lane partial values p[0..RW-1] (one per row; RW = 1, 2, 4 or 8)
// across the warp with an associative op: log2(RW) exchange steps halve the
// values per lane, the remaining steps combine within lane groups. Afterwards
// every lane holds the op over all 32 lanes of row (lane >> (5 - log2 RW)) &
// (RW - 1); the owner lane of row q is q << (5 - log2 RW). The order of the
// combines depends only on the lane, so the result is reproducible. RW - 1 +
// 5 - log2(RW) shuffles (9 for 8 rows instead of 40).
template <int RW, typename Op>
__device__ __forceinline__ float fold_rows(float (&p)[RW], int lane, Op op) {
  int off = 16;
#pragma unroll
  for (int half = RW / 2; half >= 1; half /= 2) {
    const bool h = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = h ? p[i] : p[i + half];
      const float keep = h ? p[i + half] : p[i];
      p[i] = op(keep, __shfl_xor_sync(0xffffffffu, send, off));
    }
    off >>= 1;
  }
  float v = p[0];
#pragma unroll
  for (; off >= 1; off >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

template <int RW>
struct RowFold {
  static constexpr int kShift = RW == 8 ? 2 : RW == 4 ? 3 : RW == 2 ? 4 : 5;
};

struct OpAdd {
  __device__ __forceinline__ float operator()(float a, float b) const { return a + b; }
};
struct OpMax {
  __device__ __forceinline__ float operator()(float a, float b) const { return fmaxf(a, b); }
};

}  // namespace lsf
