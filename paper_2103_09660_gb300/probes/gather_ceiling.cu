// Gather ceilings of this GPU: how fast random 512-byte rows (one row of
// 128 float32, the refinement's row size) can be read, by table size, and
// by which route. It measures the ceilings the refinement kernels are held
// against: random row gathers from a table that fits in L2 against one that
// does not, and a plain copy for the DRAM peak. It computes nothing of the
// method.
//
//   regs     ld.global.nc into registers: each warp sums the 128 rows of an
//            item, each lane one 16-byte column, U rows in flight per lane
//   cp.async 16-byte cp.async per lane into a shared-memory ring of S
//            stages of 32 rows, consumed from shared memory
//   bulk     one cp.async.bulk (TMA, 512 bytes) per row into the ring, one
//            mbarrier per stage
//
// Every index is drawn on the host in [0, rows) and every mbarrier wait is
// bounded by %globaltimer (0.2 s): a wait that gives up sets an error flag,
// which main() reports, and the kernel returns. Prints one JSON line.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e_ = (x);                                                       \
    if (e_ != cudaSuccess) {                                                    \
      fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
      exit(1);                                                                  \
    }                                                                           \
  } while (0)

namespace {

constexpr int K = 128;      // rows per item
constexpr int CH = 32;      // rows per shared-memory stage
constexpr int WARPS = 4;    // warps per CTA of the shared-memory variants

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > 200000000ull) return false;
  }
}

template <int U>
__global__ void __launch_bounds__(256) gather_regs(const int* __restrict__ idx, long n_items,
                                                   const uint4* __restrict__ tab,
                                                   float4* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long w0 = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long it = w0; it < n_items; it += nw) {
    const int* ix = idx + it * K;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < K; k += U) {
      uint4 x[U];
#pragma unroll
      for (int u = 0; u < U; ++u) x[u] = __ldg(tab + (size_t)__ldg(ix + k + u) * 32 + lane);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        acc.x += __uint_as_float(x[u].x);
        acc.y += __uint_as_float(x[u].y);
        acc.z += __uint_as_float(x[u].z);
        acc.w += __uint_as_float(x[u].w);
      }
    }
    out[it * 32 + lane] = acc;
  }
}

// MODE 1: cp.async; MODE 2: cp.async.bulk
template <int MODE, int S>
__global__ void __launch_bounds__(WARPS * 32) gather_smem(const int* __restrict__ idx, long n_items,
                                                          const uint4* __restrict__ tab,
                                                          float4* __restrict__ out, int* err) {
  extern __shared__ __align__(128) uint4 sm[];
  __shared__ __align__(8) uint64_t bars[WARPS][S];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint4* ring = sm + (size_t)wid * S * CH * 32;
  if (MODE == 2 && lane == 0)
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[wid][s])) : "memory");
  if (MODE == 2) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  const long w = (long)blockIdx.x * WARPS + wid, nw = (long)gridDim.x * WARPS;
  const int cpi = K / CH;
  const long my_items = w < n_items ? (n_items - w + nw - 1) / nw : 0;
  const long total = my_items * cpi;
  auto rows_of = [&](long c) -> const int* {
    return idx + (w + (c / cpi) * nw) * K + (c % cpi) * CH;
  };
  auto issue = [&](long c) {
    const int st = (int)(c % S);
    const int* ix = rows_of(c);
    uint4* dst = ring + (size_t)st * CH * 32;
    if (MODE == 1) {
      for (int r = 0; r < CH; ++r) {
        const uint4* src = tab + (size_t)__ldg(ix + r) * 32 + lane;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst + r * 32 + lane)),
                     "l"(src)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
      const uint32_t bar = smem_addr(&bars[wid][st]);
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(CH * 512)
                     : "memory");
      __syncwarp();
      const uint4* src = tab + (size_t)__ldg(ix + lane) * 32;
      asm volatile(
          "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], 512, [%2];" ::"r"(
              smem_addr(dst + lane * 32)),
          "l"(src), "r"(bar)
          : "memory");
    }
  };
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  bool bad = false;
  for (long c = 0; c < total && c < S; ++c) issue(c);
  for (long c = 0; c < total; ++c) {
    const int st = (int)(c % S);
    if (MODE == 1) {
      long after = total - 1 - c;
      if (after > S - 1) after = S - 1;
      if (after >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
      else if (after == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
      else asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (!wait_parity(smem_addr(&bars[wid][st]), (uint32_t)((c / S) & 1))) {
      bad = true;
      break;
    }
    __syncwarp();
    const uint4* src = ring + (size_t)st * CH * 32;
#pragma unroll 8
    for (int r = 0; r < CH; ++r) {
      const uint4 x = src[r * 32 + lane];
      acc.x += __uint_as_float(x.x);
      acc.y += __uint_as_float(x.y);
      acc.z += __uint_as_float(x.z);
      acc.w += __uint_as_float(x.w);
    }
    if ((c % cpi) == cpi - 1) {
      out[(w + (c / cpi) * nw) * 32 + lane] = acc;
      acc = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    if (MODE == 2) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (c + S < total) issue(c + S);
  }
  if (bad) {
    if (lane == 0) atomicOr(err, 1);
    for (int s = 0; s < S; ++s) {      // let the copies this warp issued land (bounded)
      wait_parity(smem_addr(&bars[wid][s]), 0);
      wait_parity(smem_addr(&bars[wid][s]), 1);
    }
  }
}

__global__ void copy_kernel(const uint4* __restrict__ a, uint4* __restrict__ b, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const long n_items = 1 << 16;                 // 8.4M row gathers (4.3 GB) per launch
  const long max_rows = 1L << 22;               // a 2 GB table
  uint4* tab = nullptr;
  float4* out = nullptr;
  int* d_idx = nullptr;
  int* err = nullptr;
  CK(cudaMalloc(&tab, (size_t)max_rows * 512));
  CK(cudaMemset(tab, 0, (size_t)max_rows * 512));
  CK(cudaMalloc(&out, (size_t)n_items * 512));
  CK(cudaMalloc(&d_idx, (size_t)n_items * K * 4));
  CK(cudaMalloc(&err, 4));
  CK(cudaMemset(err, 0, 4));
  std::vector<int> h((size_t)n_items * K);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  printf("{\"probe\": \"gather ceiling, random 512-byte rows\", \"sms\": %d, \"results\": [", sms);
  bool first = true;
  auto timeit = [&](long rows, const char* route, auto run) {
    run();
    run();
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0));
    for (int r = 0; r < 5; ++r) run();
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 5;
    printf("%s{\"table_MB\": %.1f, \"route\": \"%s\", \"ms\": %.4f, \"TBps\": %.2f}", first ? "" : ", ",
           rows * 512.0 / 1e6, route, ms, (double)n_items * K * 512 / ms / 1e9);
    first = false;
  };
  for (long rows : {4096L, 32768L, 131072L, 262144L, 1L << 20, 1L << 22}) {
    uint64_t s = 88172645463325252ull;            // xorshift64
    for (auto& v : h) {
      s ^= s << 13;
      s ^= s >> 7;
      s ^= s << 17;
      v = (int)(s % (uint64_t)rows);
    }
    CK(cudaMemcpy(d_idx, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
    timeit(rows, "regs U=4", [&] { gather_regs<4><<<sms * 8, 256>>>(d_idx, n_items, tab, out); });
    timeit(rows, "regs U=8", [&] { gather_regs<8><<<sms * 8, 256>>>(d_idx, n_items, tab, out); });
    if (rows == 32768L || rows == (1L << 20)) {
      {
        auto k = gather_smem<1, 2>;
        const int bytes = WARPS * 2 * CH * 512;
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        timeit(rows, "cp.async S=2", [&] { k<<<sms, WARPS * 32, bytes>>>(d_idx, n_items, tab, out, err); });
      }
      {
        auto k = gather_smem<2, 1>;
        const int bytes = WARPS * 1 * CH * 512;
        CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        timeit(rows, "bulk S=1 3 CTA/SM",
               [&] { k<<<sms * 3, WARPS * 32, bytes>>>(d_idx, n_items, tab, out, err); });
      }
    }
  }
  const long n4 = max_rows * 32 / 2;
  CK(cudaEventRecord(e0));
  for (int r = 0; r < 5; ++r) copy_kernel<<<sms * 8, 256>>>(tab, tab + n4, n4);
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  ms /= 5;
  int herr = 0;
  CK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
  CK(cudaGetLastError());
  printf("], \"copy_1GB_TBps_read_plus_write\": %.2f, \"wait_timeouts\": %d}\n",
         2.0 * n4 * 16 / ms / 1e9, herr);
  return herr ? 2 : 0;
}
