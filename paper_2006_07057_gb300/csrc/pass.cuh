// Fused Sinkhorn pass over a stored feature matrix (one half of Alg. 1).
#pragma once

#include "common.cuh"

namespace lsf {

enum PassMode : int {
  kPassUpdate = 0,  // s = F t; res += |old s - w|; new = w / s; t' += new F
  kPassAxpy = 1,    // t' += given F            (given scaling in `old`)
  kPassDot = 2,     // s = F t; res += |old s - w|  (no update)
  // log-domain pass only (the products of the accelerated solver):
  kPassRows = 3,     // out = log s, s = F t
  kPassRowsAxpy = 4  // out = log s, s = F t; and t' = the transposed product with `old`
};

// One right-hand side of a pass: the r-vector it multiplies and what it updates.
struct PassRhs {
  const float* t_in;  // ldr   (Update, Dot, Rows, RowsAxpy)
  const float* w;     // n     weights (Update, Dot)
  const float* old;   // n     previous scaling (residual) or the given scaling (Axpy, RowsAxpy); may be NULL in Update
  float* out;         // n     new scaling (Update) or log of the row product (Rows, RowsAxpy)
  float* t_out;       // ldr   reduced F^T new (Update, Axpy, RowsAxpy)
  double* res_out;    // 1     residual sum |old s - w| (Update with old, Dot)
};

struct PassArgs {
  const float* F;   // n x ldr
  int64_t n;
  int ldr;
  int tile_rows;
  int64_t ntiles;
  int nstages;
  PassRhs rhs[2];
  float* part;        // workspace partial r-vectors
  float* gpart;       // workspace per-group partials of the two-level reduction
  double* rpart;      // workspace partial residuals
  unsigned* counter;  // workspace arrival counters [1 + groups] (zero between launches)
  int* status;        // device status word (lsf_result.status)
};

// Launch one fused pass (nrhs = 1 or 2) with tiling chosen for F's shape.
// bytes_moved is the algorithmic traffic of the launch, recorded for profiling.
int launch_pass(int mode, int nrhs, PassArgs args, cudaStream_t st);

// Shape of a stored-pass consumer step for C float4 columns per lane: it works
// on kTilesPerStep consecutive ring stages at once (8 / C rows of each).
template <int C>
struct PassShape {
  static constexpr int kTilesPerStep = C == 8 ? 2 : 1;
};

// float4 columns per lane of a stored pass (1, 2, 4 or 8) for a row stride ldr;
// a consumer warp takes 8 / that many rows at once.
int pass_columns(int ldr);

// Choose tile rows, ring depth, dynamic shared memory and grid for a pass over F.
// red_floats_per_warp_rhs: floats per consumer warp and right-hand side of the
// end-of-launch reduction buffer (ldr, or 2 ldr for the log-domain pass).
int plan_pass(PassArgs& a, int nrhs, int red_floats_per_warp_rhs, size_t* smem, unsigned* grid);

// Log-domain pass (same ring, log-sum-exp arithmetic); see logpass.cu.
int launch_logpass(int mode, int nrhs, PassArgs args, cudaStream_t st);

// Target tile size and maximum ring depth of the stored-feature pass (tuning).
int set_pass_tiling(int tile_bytes, int max_stages);
void get_pass_tiling(int* tile_bytes, int* max_stages);

// Algorithmic bytes of one pass launch.
double pass_bytes(int mode, int nrhs, int64_t n, int ldr, bool with_old);

}  // namespace lsf
