// Runtime services of libhnv.so: error strings, the device allocator hook,
// the kernel launch counter and per-phase CUDA-event timing.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "hnv_internal.cuh"

namespace hnv {

NvtxRange::NvtxRange(const char* fmt, ...) {
  char name[96];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(name, sizeof(name), fmt, ap);
  va_end(ap);
  nvtxRangePushA(name);
}

NvtxRange::~NvtxRange() { nvtxRangePop(); }

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

static thread_local char g_detail[512] = {0};

void set_error_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

void clear_error_detail() { g_detail[0] = 0; }

int cuda_status(cudaError_t e, const char* what) {
  set_error_detail("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return HNV_ERR_OOM;
  }
  return HNV_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Launch bookkeeping
// ---------------------------------------------------------------------------

static std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    cached = v;
  }
  return cached;
}

unsigned grid_for(int64_t items, int64_t per_block, int waves) {
  if (items <= 0) return 0;
  int64_t blocks = (items + per_block - 1) / per_block;
  int64_t cap = (int64_t)num_sms() * waves;
  if (blocks > cap) blocks = cap;
  return (unsigned)blocks;
}

// ---------------------------------------------------------------------------
// Allocator
// ---------------------------------------------------------------------------

static hnv_alloc_fn g_alloc = nullptr;
static hnv_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

// The library's own stream-ordered memory pool per device. Its release
// threshold is unlimited: memory freed by one call stays mapped for the
// next (the default pool returns it to the system at every synchronisation,
// and a V-cycle step allocates and frees about 1.5 GB at the 1M-node size).
// hnv_release_cached_memory() gives the unused part back.
constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[kMaxPoolDevices] = {nullptr};

static int device_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxPoolDevices) HNV_FAIL(HNV_ERR_INVALID_ARG, "device %d", dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return cuda_status(e, "cudaMemPoolCreate");
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return cuda_status(e, "cudaMemPoolSetAttribute");
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return HNV_OK;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (g_alloc) {
    *p = g_alloc(bytes, reinterpret_cast<hnv_stream_t>(s), g_alloc_ctx);
    if (!*p) HNV_FAIL(HNV_ERR_OOM, "allocator hook returned NULL for %zu bytes", bytes);
    return HNV_OK;
  }
  cudaMemPool_t pool = nullptr;
  HNV_CHECK(device_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    HNV_FAIL(e == cudaErrorMemoryAllocation ? HNV_ERR_OOM : HNV_ERR_CUDA,
             "cudaMallocFromPoolAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  return HNV_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (g_free) {
    g_free(p, reinterpret_cast<hnv_stream_t>(s), g_alloc_ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------
// Timing
// ---------------------------------------------------------------------------

struct TimedRegion {
  int phase;
  cudaEvent_t start, stop;
  double bytes;
};

static std::mutex g_tmu;
static bool g_timing = false;
static std::vector<TimedRegion> g_regions;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

bool timing_on() { return g_timing; }

int timing_begin(int phase, cudaStream_t s, double alg_bytes) {
  std::lock_guard<std::mutex> lk(g_tmu);
  TimedRegion r{phase, take_event(), take_event(), alg_bytes};
  if (!r.start || !r.stop) return -1;
  cudaEventRecord(r.start, s);
  g_regions.push_back(r);
  return (int)g_regions.size() - 1;
}

void timing_end(int slot, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (slot < 0 || slot >= (int)g_regions.size()) return;
  cudaEventRecord(g_regions[slot].stop, s);
}

}  // namespace hnv

using namespace hnv;

extern "C" {

const char* hnv_error_string(int code) {
  switch (code) {
    case HNV_OK: return "HNV_OK";
    case HNV_ERR_INVALID_ARG: return "HNV_ERR_INVALID_ARG";
    case HNV_ERR_OUT_OF_RANGE: return "HNV_ERR_OUT_OF_RANGE";
    case HNV_ERR_TOO_LARGE: return "HNV_ERR_TOO_LARGE";
    case HNV_ERR_OOM: return "HNV_ERR_OOM";
    case HNV_ERR_CUDA: return "HNV_ERR_CUDA";
    case HNV_ERR_TIMEOUT: return "HNV_ERR_TIMEOUT";
    case HNV_ERR_UNSUPPORTED_D: return "HNV_ERR_UNSUPPORTED_D";
    case HNV_ERR_STATE: return "HNV_ERR_STATE";
    default: return "HNV_ERR_UNKNOWN";
  }
}

const char* hnv_last_error_detail(void) { return g_detail; }

int hnv_set_allocator(hnv_alloc_fn alloc_fn, hnv_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr))
    HNV_FAIL(HNV_ERR_INVALID_ARG, "allocator and free function must both be set or both be NULL");
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return HNV_OK;
}

int hnv_release_cached_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < kMaxPoolDevices; ++d) {
    if (!g_pools[d]) continue;
    const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
    if (e != cudaSuccess) return cuda_status(e, "cudaMemPoolTrimTo");
  }
  return HNV_OK;
}

int64_t hnv_kernel_launch_count(void) { return g_launches.load(); }

int hnv_timing_enable(int enable) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_timing = enable != 0;
  return HNV_OK;
}

int hnv_timing_reset(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& r : g_regions) {
    g_event_pool.push_back(r.start);
    g_event_pool.push_back(r.stop);
  }
  g_regions.clear();
  return HNV_OK;
}

int hnv_timing_read(int phase, double* total_ms, int64_t* launches, double* alg_bytes) {
  if (phase < 0 || phase >= HNV_PHASE_COUNT) HNV_FAIL(HNV_ERR_INVALID_ARG, "bad phase %d", phase);
  std::lock_guard<std::mutex> lk(g_tmu);
  double ms = 0.0, bytes = 0.0;
  int64_t cnt = 0;
  for (auto& r : g_regions) {
    if (r.phase != phase) continue;
    cudaError_t e = cudaEventSynchronize(r.stop);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventSynchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, r.start, r.stop);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventElapsedTime");
    ms += t;
    bytes += r.bytes;
    ++cnt;
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = cnt;
  if (alg_bytes) *alg_bytes = bytes;
  return HNV_OK;
}

}  // extern "C"
