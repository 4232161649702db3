// Host runtime of libsinkhorn_pf: errors, device queries, launch accounting,
// optional event timing, workspace layout, and the Lemma 1 host math.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "pass.cuh"

namespace lsf {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

struct ProfileRecord {
  int cls;
  double bytes;
  cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfileRecord> g_prof;      // recorded launches
std::vector<cudaEvent_t> g_event_pool;  // reusable events

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

DeviceInfo g_info[64];
}  // namespace

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return status;
}

const DeviceInfo& device_info() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  DeviceInfo& info = g_info[dev];
  if (info.device != dev) {
    int sms = 0, smem = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    info.sms = sms > 0 ? sms : 1;
    info.smem_optin = smem;
    info.device = dev;
  }
  return info;
}

namespace {
std::atomic<int> g_trace_level{1};
const char* const kClassNames[LSF_KERNEL_NCLASSES] = {
    "pass", "pass_recompute", "features", "other", "pass_log", "batched",
    "adjoint", "small", "pass_multi", "pass_hybrid"};
}  // namespace

TraceRange::TraceRange(const char* name) : on(g_trace_level.load(std::memory_order_relaxed) >= 1) {
  if (on) nvtxRangePushA(name);
}

TraceRange::~TraceRange() {
  if (on) nvtxRangePop();
}

LaunchScope::LaunchScope(cudaStream_t s, int kernel_class, double nbytes)
    : stream(s), cls(kernel_class), bytes(nbytes), slot(-1),
      traced(g_trace_level.load(std::memory_order_relaxed) >= 2 && kernel_class >= 0 &&
             kernel_class < LSF_KERNEL_NCLASSES) {
  if (traced) nvtxRangePushA(kClassNames[kernel_class]);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfileRecord rec{cls, bytes, take_event(), take_event()};
  if (!rec.start || !rec.stop) return;
  cudaEventRecord(rec.start, stream);
  g_prof.push_back(rec);
  slot = static_cast<int>(g_prof.size()) - 1;
}

LaunchScope::~LaunchScope() {
  if (traced) nvtxRangePop();
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot < static_cast<int>(g_prof.size())) cudaEventRecord(g_prof[slot].stop, stream);
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LSF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return LSF_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int max_pass_ctas() { return device_info().sms * kMaxPassCtasPerSm; }

int workspace_counters() { return kPassCounter + 1 + reduce_groups(max_pass_ctas()); }

size_t workspace_bytes(int ldr) {
  const int grid = max_pass_ctas();
  size_t b = 0;
  b += align256(sizeof(float) * static_cast<size_t>(grid) * 4 * ldr);
  b += align256(sizeof(float) * static_cast<size_t>(reduce_groups(grid)) * 4 * ldr);
  b += align256(sizeof(double) * static_cast<size_t>(grid) * 2);
  b += align256(sizeof(double) * static_cast<size_t>(grid) * 3);
  b += align256(sizeof(unsigned) * workspace_counters());
  b += align256(sizeof(unsigned) * 8);
  return b;
}

int carve_workspace(void* base, size_t bytes, int ldr, Workspace* ws) {
  const size_t need = workspace_bytes(ldr);
  if (!base) return fail(LSF_ERR_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(base) % 256 != 0)
    return fail(LSF_ERR_ARG, "workspace must be 256-byte aligned");
  if (bytes < need)
    return fail(LSF_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", bytes, need);
  const int grid = max_pass_ctas();
  char* p = static_cast<char*>(base);
  ws->part = reinterpret_cast<float*>(p);
  p += align256(sizeof(float) * static_cast<size_t>(grid) * 4 * ldr);
  ws->gpart = reinterpret_cast<float*>(p);
  p += align256(sizeof(float) * static_cast<size_t>(reduce_groups(grid)) * 4 * ldr);
  ws->rpart = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * static_cast<size_t>(grid) * 2);
  ws->dpart = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * static_cast<size_t>(grid) * 3);
  ws->counters = reinterpret_cast<unsigned*>(p);
  p += align256(sizeof(unsigned) * workspace_counters());
  ws->keys = reinterpret_cast<unsigned*>(p);
  p += align256(sizeof(unsigned) * 8);
  ws->bytes = need;
  return LSF_OK;
}

// Principal Lambert branch for z >= 0: Newton's iteration on f(w) = w e^w - z,
// started at log(1 + z) (above the root for z > 0, and f is convex there, so
// the iterates decrease monotonically to the root).
static double lambert_w0_host(double z) {
  if (z == 0.0) return 0.0;
  double w = std::log1p(z);
  for (int i = 0; i < 200; ++i) {
    const double ew = std::exp(w);
    const double f = w * ew - z;
    const double step = f / (ew * (w + 1.0));
    const double next = w - step;
    if (std::fabs(next - w) <= 1e-16 * std::fabs(next)) {
      w = next;
      break;
    }
    w = next;
  }
  return w;
}

}  // namespace lsf

using namespace lsf;

extern "C" {

int lsf_version(void) { return 2; }

const char* lsf_last_error(void) { return g_last_error.c_str(); }

int lsf_gaussian_params(double R, double eps, int d, double* q, double* sigma) {
  if (!q || !sigma) return fail(LSF_ERR_ARG, "lsf_gaussian_params: NULL output");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(LSF_ERR_ARG, "eps must be > 0");
  if (d < 1) return fail(LSF_ERR_ARG, "d must be >= 1");
  if (!(R >= 0.0) || !std::isfinite(R)) return fail(LSF_ERR_ARG, "R must be finite and >= 0");
  const double z = R * R / (eps * d);
  double qq = 0.5;
  if (z > 0.0) qq = R * R / (2.0 * eps * d * lambert_w0_host(z));
  *q = qq;
  *sigma = std::sqrt(qq * eps / 4.0);
  return LSF_OK;
}

int lsf_workspace_bytes(int ldr, size_t* bytes) {
  if (!bytes) return fail(LSF_ERR_ARG, "lsf_workspace_bytes: NULL output");
  if (ldr < 4 || ldr % 4 != 0 || ldr > 1024)
    return fail(LSF_ERR_UNSUPPORTED, "ldr must be a multiple of 4 in [4, 1024]");
  *bytes = workspace_bytes(ldr);
  return LSF_OK;
}

int lsf_set_tracing(int level, int* previous) {
  if (level < 0 || level > 2) return lsf::fail(LSF_ERR_ARG, "tracing level must be 0, 1 or 2");
  const int prev = lsf::g_trace_level.exchange(level);
  if (previous) *previous = prev;
  return LSF_OK;
}

int lsf_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    g_event_pool.push_back(r.start);
    g_event_pool.push_back(r.stop);
  }
  g_prof.clear();
  g_prof_on = on != 0;
  return LSF_OK;
}

int lsf_profile_read(int kernel_class, double* total_ms, int64_t* launches, double* bytes) {
  if (!total_ms || !launches || !bytes) return fail(LSF_ERR_ARG, "lsf_profile_read: NULL output");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  double ms = 0.0, by = 0.0;
  int64_t cnt = 0;
  for (auto& r : g_prof) {
    if (r.cls != kernel_class) continue;
    if (cudaEventSynchronize(r.stop) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "event synchronize failed");
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.start, r.stop) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "event elapsed time failed");
    ms += t;
    by += r.bytes;
    ++cnt;
  }
  *total_ms = ms;
  *launches = cnt;
  *bytes = by;
  return LSF_OK;
}

int lsf_set_pass_tiling(int tile_bytes, int max_stages) {
  return set_pass_tiling(tile_bytes, max_stages);
}

int lsf_get_pass_tiling(int* tile_bytes, int* max_stages) {
  if (!tile_bytes || !max_stages) return fail(LSF_ERR_ARG, "lsf_get_pass_tiling: NULL output");
  get_pass_tiling(tile_bytes, max_stages);
  return LSF_OK;
}

int64_t lsf_launch_count(void) { return g_launches.load(); }
void lsf_launch_count_reset(void) { g_launches.store(0); }

}  // extern "C"
