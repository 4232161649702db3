// Fused Sinkhorn pass that recomputes the features in registers (recompute variant).
#pragma once

#include "pass.cuh"

namespace lsf {

struct RecomputeArgs {
  const float* X;      // n x d points
  const float* shift;  // n row log-shifts
  int64_t n;
  const float* U;      // r x d anchors
  const float* c;      // r anchor log-constants
  int r, ldr, d;
  float two_over_eps;
  PassRhs rhs[2];
  float* part;
  float* gpart;
  double* rpart;
  unsigned* counter;
  int* status;
};

int launch_recompute_pass(int mode, int nrhs, RecomputeArgs a, cudaStream_t st);

// Row record of the recompute and hybrid passes in shared memory, in float4s:
// (x_0, x_0, x_1, x_1), ..., (B, B) (each value twice, so one load gives the
// broadcast pair a packed instruction takes; padded to a float4 boundary), then
// (w, old) of each right-hand side.
template <int D>
struct RowPack {
  static constexpr int kXV = (2 * (D + 1) + 3) / 4;  // float4s of x and B, doubled
  static constexpr int kSV = kXV + 1;                // + (w0, old0, w1, old1)
};

// The GW warp partials of one row, summed in a fixed tree order (vector loads;
// the partials of a row are contiguous and GW-aligned).
template <int GW>
__device__ __forceinline__ float sum_partials(const float* p) {
  if constexpr (GW == 8) {
    const float4 lo = reinterpret_cast<const float4*>(p)[0], hi = reinterpret_cast<const float4*>(p)[1];
    return ((lo.x + lo.y) + (lo.z + lo.w)) + ((hi.x + hi.y) + (hi.z + hi.w));
  } else if constexpr (GW == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return (v.x + v.y) + (v.z + v.w);
  } else if constexpr (GW == 2) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return v.x + v.y;
  } else {
    return p[0];
  }
}

// Stored / recomputed column split of a hybrid pass for row stride ldr: the
// first c0 columns are rebuilt in registers, the last ldr - c0 are streamed from
// a stored block (half of the float4 columns, rounded down, are stored).
constexpr int hybrid_first_stored(int ldr) {
  const int q = ldr / 4;
  return 4 * (q - q / 2);
}

// Arguments of the hybrid pass: the recompute arguments (columns [0, c0)) plus
// the stored block Fs (n x (ldr - c0), row stride ldr - c0) of columns [c0, ldr).
struct HybridArgs {
  RecomputeArgs rc;
  const float* Fs;
  int c0;
};

int launch_hybrid_pass(int mode, int nrhs, HybridArgs a, cudaStream_t st);

}  // namespace lsf
