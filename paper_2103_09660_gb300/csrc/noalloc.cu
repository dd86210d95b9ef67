// hnv_refine_noalloc: the two-phase refinement of hnv_refine for callers that
// may not allocate device memory while the call runs.
//
// Why such callers exist: some host programs reserve their whole device
// memory budget up front (a serving process with a fixed pool, an embedded
// deployment with a hard memory cap) and treat any later cudaMalloc as a
// failure, since it can run out of memory at a bad moment and may stall the
// device while it synchronises. hnv_refine allocates its split-row scratch
// lazily on first use; this entry point instead keeps that scratch in a
// fixed device array that lives in the library image, so the call itself
// never asks the allocator for anything.
//
// The array is a file-scope __device__ object of kNoAllocScratchBytes. Every
// GPU that loads the library holds it until the process exits. In host code
// its name is only a host-side stand-in, not a device address, so the host
// asks the runtime for the real address once per device (with that device
// current) and passes that pointer to the kernels.
#include <mutex>

#include "hnv_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)HNV_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Split-row partial sums of the refinement half-sweeps. Shared by every call
// on a device; contents persist between calls.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float)];

std::mutex g_mu;
float* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on `device` (which must be current).
// The first call on a device looks it up; later calls reuse it. A
// cudaDeviceReset unloads the module and makes the cached address stale,
// which is why the header rules out calls on a device that has been reset.
int scratch_address(int device, float** out) {
  if (device < 0 || device >= kMaxDevices)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "device %d out of range for the static scratch table", device);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hnv::cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_dev[device] = static_cast<float*>(p);
  }
  *out = g_scratch_dev[device];
  return HNV_OK;
}

}  // namespace

extern "C" int hnv_refine_noalloc(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt,
                                  int d, float omega, int sweeps, hnv_stream_t stream) {
  using namespace hnv;
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  if (dt != HNV_F32) HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "hnv_refine_noalloc supports HNV_F32 only");
  if (d < 4 || d > 1024 || d % 4 != 0)
    HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d: need 4 <= d <= 1024 and d %% 4 == 0", d);
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps < 0");
  const Level& lv = g->levels[level];
  if ((lv.n > 0 && !z_v) || (lv.m > 0 && !z_e)) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL embedding");
  if ((reinterpret_cast<uintptr_t>(z_v) | reinterpret_cast<uintptr_t>(z_e)) & 15u)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "embeddings must be 16-byte aligned");
  const int64_t chunks = lv.planE.n_chunks > lv.planV.n_chunks ? lv.planE.n_chunks : lv.planV.n_chunks;
  const size_t need = sizeof(float) * (size_t)chunks * (size_t)d;
  if (need > kNoAllocScratchBytes)
    HNV_FAIL(HNV_ERR_TOO_LARGE,
             "level %d needs %zu bytes of split-row scratch at d = %d; the static scratch holds %zu",
             level, need, d, kNoAllocScratchBytes);

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) HNV_CUDA(cudaSetDevice(g->device));
  float* scratch = nullptr;
  int rc = scratch_address(g->device, &scratch);
  if (rc == HNV_OK)
    rc = refine_two_phase_with_partials(g, level, static_cast<float*>(z_v), static_cast<float*>(z_e),
                                        d, omega, sweeps, scratch,
                                        reinterpret_cast<cudaStream_t>(stream));
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  return rc;
}
