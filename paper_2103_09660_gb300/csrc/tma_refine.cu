// TMA-gather refinement half-sweep (sm_103a), for d in {32, 64, 128, 256}.
//
// Same arithmetic as gather_kernel (refine.cu): for every work item of the
// plan, sum its neighbour rows in incidence order, then relax its own row
// (rows) or write the un-normalised partial (chunks). What differs is how
// rows reach the SM: instead of per-lane 16-byte loads, the Tensor Memory
// Accelerator copies them into shared memory.
//
//  * A unit is up to 4 consecutive incidences of one item. Lane 0 of a warp
//    issues one cp.async.bulk.tensor ... tile::gather4 per unit (4 rows of the
//    neighbour table into one shared-memory slot) and, for the first unit of
//    a row item, a 1-row tile load of the item's own row into the same slot.
//    The slot's mbarrier counts the bytes (complete_tx).
//  * Every warp runs its own ring of S slots: it consumes unit v while units
//    v+1 .. v+S-1 are in flight, then reissues the freed slot for unit v+S.
//    No register holds an in-flight row, so occupancy does not limit the
//    number of rows in flight (4*S per warp).
//  * Units are laid out in windows of 32, one per lane: an item class with
//    at most 4*UPI incidences gives each item UPI consecutive lanes (UPI = 1,
//    4, 16, 32 for items of <= 4, 16, 64, 128 incidences). A lane loads its
//    unit's descriptor, 4 indices and 4 weights; the window after the current
//    one is loaded ahead, so issuing never waits on an index load.
//  * Consumption: lane groups of min(32, d/4) lanes each hold a float4 column
//    set of one row; P = 32/group rows of a unit are read in parallel and the
//    group sums are combined by a fixed xor tree. Order is fixed: results are
//    deterministic and need no atomics.
//  * Every mbarrier wait is bounded by %globaltimer (kWaitLimitNs); on expiry
//    the warp records HNV_ERR_TIMEOUT in the error word, drains its slots
//    (bounded too) and stops.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTmaWarps = 8;                          // warps per CTA
constexpr uint64_t kWaitLimitNs = 2000000000ull;      // 2 s per wait
constexpr uint64_t kDrainLimitNs = 20000000ull;       // 20 ms per slot when draining

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int32_t r0,
                                            int32_t r1, int32_t r2, int32_t r3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_row(uint32_t dst, const CUtensorMap* map, int32_t row,
                                        uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void f4_add(float4& a, const float4& b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

__device__ __forceinline__ void f4_fma(float4& a, float s, const float4& b) {
  a.x = fmaf(s, b.x, a.x);
  a.y = fmaf(s, b.y, a.y);
  a.z = fmaf(s, b.z, a.z);
  a.w = fmaf(s, b.w, a.w);
}

__device__ __forceinline__ float4 f4_xor(const float4& a, int o) {
  return make_float4(__shfl_xor_sync(FULL, a.x, o), __shfl_xor_sync(FULL, a.y, o),
                     __shfl_xor_sync(FULL, a.z, o), __shfl_xor_sync(FULL, a.w, o));
}

__device__ __forceinline__ float4 relax4(float keep, float sc, const float4& self, const float4& acc) {
  return make_float4(fmaf(keep, self.x, sc * acc.x), fmaf(keep, self.y, sc * acc.y),
                     fmaf(keep, self.z, sc * acc.z), fmaf(keep, self.w, sc * acc.w));
}

// One lane's unit of a window.
struct Unit {
  int4 d;        // item descriptor {row, beg, len, slot}
  int32_t r[4];  // neighbour rows (padded with r[0])
  float w[4];    // their weights (0 past the end)
  int32_t nv;    // valid rows in the unit (0: nothing to do)
};

template <int D4>
struct TmaShape {
  static constexpr int ROW_B = D4 * 16;
  static constexpr int SLOT_B = 5 * ROW_B;               // 4 gathered rows + own row
  static constexpr int S_RAW = 8192 / (4 * ROW_B);
  static constexpr int S = S_RAW < 2 ? 2 : (S_RAW > 16 ? 16 : S_RAW);   // slots per warp
  static constexpr int VPL = D4 > 32 ? D4 / 32 : 1;      // float4 columns per lane
  static constexpr int GW = D4 >= 32 ? 32 : D4;          // lanes per row group
  static constexpr int P = 32 / GW;                      // rows read in parallel
  static constexpr size_t SMEM = (size_t)kTmaWarps * S * SLOT_B + (size_t)kTmaWarps * S * 8;
};

template <int D4, int UPI, bool WEIGHTED>
__global__ void __launch_bounds__(kTmaWarps * 32, 1)
tma_gather_kernel(const __grid_constant__ CUtensorMap map_src,
                  const __grid_constant__ CUtensorMap map_self, const int4* __restrict__ items,
                  int32_t n_items, const int32_t* __restrict__ idx,
                  const float* __restrict__ inc_w, const float* __restrict__ inv_norm,
                  float4* __restrict__ out, float omega, float4* __restrict__ partials,
                  int32_t* __restrict__ err) {
  using Sh = TmaShape<D4>;
  constexpr int S = Sh::S;
  constexpr int IPW = 32 / UPI;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint8_t* ring = smem + (size_t)wid * S * Sh::SLOT_B;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)kTmaWarps * S * Sh::SLOT_B) + wid * S;
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  const int64_t total_warps = (int64_t)gridDim.x * kTmaWarps;
  const int64_t n_windows = ((int64_t)n_items + IPW - 1) / IPW;
  const int grp = lane / Sh::GW;
  const int gl = lane % Sh::GW;
  const float keep = 1.0f - omega;

  auto load_unit = [&](int64_t win) {
    Unit x;
    x.d = make_int4(-1, 0, 0, -1);
    x.nv = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      x.r[t] = 0;
      x.w[t] = 0.f;
    }
    if (win < n_windows) {
      const int64_t it = win * IPW + lane / UPI;
      const int q = lane % UPI;
      if (it < n_items) {
        x.d = __ldg(items + it);
        const int32_t rem = x.d.z - 4 * q;
        x.nv = rem <= 0 ? 0 : (rem >= 4 ? 4 : rem);
        const int32_t base = x.d.y + 4 * q;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (t < x.nv) {
            x.r[t] = __ldg(idx + base + t);
            if (WEIGHTED) x.w[t] = __ldg(inc_w + base + t);
          }
        }
#pragma unroll
        for (int t = 1; t < 4; ++t)
          if (t >= x.nv) x.r[t] = x.r[0];
      }
    }
    return x;
  };

  // issue unit `u` (a lane index of window `x`) into slot `slot`
  auto issue = [&](const Unit& x, int u, int slot) {
    const int nv = __shfl_sync(FULL, x.nv, u);
    if (nv == 0) return;
    const int32_t r0 = __shfl_sync(FULL, x.r[0], u);
    const int32_t r1 = __shfl_sync(FULL, x.r[1], u);
    const int32_t r2 = __shfl_sync(FULL, x.r[2], u);
    const int32_t r3 = __shfl_sync(FULL, x.r[3], u);
    const int32_t row = __shfl_sync(FULL, x.d.x, u);
    const int32_t pslot = __shfl_sync(FULL, x.d.w, u);
    const bool self_load = (u % UPI == 0) && pslot < 0;
    if (lane == 0) {
      const uint32_t bar = smem_u32(&bars[slot]);
      const uint32_t dst = smem_u32(ring + (size_t)slot * Sh::SLOT_B);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, 4 * Sh::ROW_B + (self_load ? Sh::ROW_B : 0));
      tma_gather4(dst, &map_src, r0, r1, r2, r3, bar);
      if (self_load) tma_row(dst + 4 * Sh::ROW_B, &map_self, row, bar);
    }
  };

  int64_t win = (int64_t)blockIdx.x * kTmaWarps + wid;
  if (win >= n_windows) return;
  Unit cur = load_unit(win);
  Unit nxt = load_unit(win + total_warps);
  uint32_t phase = 0;      // parity bit per slot
  uint32_t pending = 0;    // slots with an issued, unconsumed unit
  int64_t v = 0;           // units visited by this warp
  bool failed = false;

  // prologue: the first S units of the first window
#pragma unroll 1
  for (int u = 0; u < S; ++u) {
    issue(cur, u, u);
    if (__shfl_sync(FULL, cur.nv, u) > 0) pending |= 1u << u;
  }

  float4 acc[Sh::VPL];
  float4 sv[Sh::VPL];
#pragma unroll
  for (int j = 0; j < Sh::VPL; ++j) {
    acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    sv[j] = acc[j];
  }

  while (win < n_windows && !failed) {
#pragma unroll 1
    for (int u = 0; u < 32; ++u, ++v) {
      const int slot = (int)(v % S);
      const int q = u % UPI;
      const int nv = __shfl_sync(FULL, cur.nv, u);
      if (nv > 0) {
        int ok = 0;
        if (lane == 0) ok = mbar_wait_bounded(smem_u32(&bars[slot]), (phase >> slot) & 1u, kWaitLimitNs);
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) {
          failed = true;
          break;
        }
        // lane 0 saw the phase complete; the other lanes now observe it too
        // (returns at once; bounded all the same)
        int seen = mbar_wait_bounded(smem_u32(&bars[slot]), (phase >> slot) & 1u, kDrainLimitNs);
        if (!__all_sync(FULL, seen)) {
          failed = true;
          break;
        }
        phase ^= 1u << slot;
        pending &= ~(1u << slot);
        const float4* sl = reinterpret_cast<const float4*>(ring + (size_t)slot * Sh::SLOT_B);
        if (q == 0 && __shfl_sync(FULL, cur.d.w, u) < 0) {
#pragma unroll
          for (int j = 0; j < Sh::VPL; ++j) sv[j] = sl[4 * (Sh::ROW_B / 16) + gl + j * 32];
        }
        float wt[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) wt[t] = WEIGHTED ? __shfl_sync(FULL, cur.w[t], u) : 1.f;
#pragma unroll
        for (int t0 = 0; t0 < 4; t0 += Sh::P) {
          const int t = t0 + grp;
          if (t < nv) {
#pragma unroll
            for (int j = 0; j < Sh::VPL; ++j) {
              const float4 x = sl[t * (Sh::ROW_B / 16) + gl + j * 32];
              if (WEIGHTED)
                f4_fma(acc[j], wt[t], x);
              else
                f4_add(acc[j], x);
            }
          }
        }
      }
      __syncwarp();
      // reuse the slot for unit v + S
      {
        const int un = u + S;
        if (un < 32) {
          issue(cur, un, slot);
          if (__shfl_sync(FULL, cur.nv, un) > 0) pending |= 1u << slot;
        } else {
          issue(nxt, un - 32, slot);
          if (__shfl_sync(FULL, nxt.nv, un - 32) > 0) pending |= 1u << slot;
        }
      }
      if (q == UPI - 1) {
        const int4 d = make_int4(__shfl_sync(FULL, cur.d.x, u - q), 0, 0,
                                 __shfl_sync(FULL, cur.d.w, u - q));
        // combine the row groups (fixed xor tree)
#pragma unroll
        for (int o = Sh::GW; o < 32; o <<= 1) {
#pragma unroll
          for (int j = 0; j < Sh::VPL; ++j) {
            const float4 y = f4_xor(acc[j], o);
            f4_add(acc[j], y);
          }
        }
        if (d.x >= 0 && grp == 0) {
          if (d.w < 0) {
            const float sc = omega * inv_norm[d.x];
#pragma unroll
            for (int j = 0; j < Sh::VPL; ++j)
              out[(size_t)d.x * D4 + gl + j * 32] = relax4(keep, sc, sv[j], acc[j]);
          } else {
#pragma unroll
            for (int j = 0; j < Sh::VPL; ++j) partials[(size_t)d.w * D4 + gl + j * 32] = acc[j];
          }
        }
#pragma unroll
        for (int j = 0; j < Sh::VPL; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (failed) break;
    win += total_warps;
    cur = nxt;
    nxt = load_unit(win + total_warps);
  }

  if (failed) {
    if (lane == 0) {
      atomicOr(err, ERRBIT_TIMEOUT);
      // let the copies already issued into this warp's slots land (bounded)
      for (int s = 0; s < S; ++s)
        if (pending & (1u << s))
          mbar_wait_bounded(smem_u32(&bars[s]), (phase >> s) & 1u, kDrainLimitNs);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
bool g_encode_ok = false;

int encode_rows_map(CUtensorMap* map, const float* base, int64_t rows, int d) {
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn) {
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
      g_encode_ok = true;
    }
  });
  if (!g_encode_ok) HNV_FAIL(HNV_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t gdim[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)d * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)d, 1u};
  const cuuint32_t estride[2] = {1u, 1u};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim,
                        gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) HNV_FAIL(HNV_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return HNV_OK;
}

template <int D4, int UPI, bool W>
int launch_tma_class(const CUtensorMap& msrc, const CUtensorMap& mself, const int4* items,
                     int32_t n_items, const int32_t* idx, const float* inc_w, const float* inv_norm,
                     float* out, float omega, float* partials, int32_t* err, cudaStream_t s) {
  if (n_items <= 0) return HNV_OK;
  using Sh = TmaShape<D4>;
  auto kern = tma_gather_kernel<D4, UPI, W>;
  HNV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
  int per_sm = 0;
  HNV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaWarps * 32, Sh::SMEM));
  if (per_sm < 1) per_sm = 1;
  const int64_t windows = ((int64_t)n_items + (32 / UPI) - 1) / (32 / UPI);
  int64_t blocks = (windows + kTmaWarps - 1) / kTmaWarps;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (blocks > cap) blocks = cap;
  return launch("tma_gather", kern, (unsigned)blocks, kTmaWarps * 32, Sh::SMEM, s, msrc, mself,
                items, n_items, idx, inc_w, inv_norm, (float4*)out, omega, (float4*)partials, err);
}

template <int D4, bool W>
int run_tma_classes(const CUtensorMap& msrc, const CUtensorMap& mself, const SplitPlan& p,
                    const int32_t* idx, const float* inc_w, const float* inv_norm, float* out,
                    float omega, float* partials, int32_t* err, cudaStream_t s) {
  const int4* it = p.items;
  HNV_CHECK((launch_tma_class<D4, 1, W>(msrc, mself, it, p.n_a, idx, inc_w, inv_norm, out, omega,
                                        partials, err, s)));
  it += p.n_a;
  HNV_CHECK((launch_tma_class<D4, 4, W>(msrc, mself, it, p.n_b, idx, inc_w, inv_norm, out, omega,
                                        partials, err, s)));
  it += p.n_b;
  HNV_CHECK((launch_tma_class<D4, 16, W>(msrc, mself, it, p.n_c, idx, inc_w, inv_norm, out, omega,
                                         partials, err, s)));
  it += p.n_c;
  return launch_tma_class<D4, 32, W>(msrc, mself, it, p.n_d + p.n_chunks, idx, inc_w, inv_norm,
                                     out, omega, partials, err, s);
}

// Self-test of the bounded waits: one warp initialises an mbarrier that
// nothing arrives at (no copy is issued, nothing is expected) and waits on
// its first phase with mbar_wait_bounded, the helper the TMA gather uses.
// The wait must give up after limit_ns; the kernel then records the timeout
// in the error word exactly as the gather does.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int32_t* err) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  const bool done = mbar_wait_bounded(b, 0, limit_ns);
  if (!done && threadIdx.x == 0) atomicOr(err, (int32_t)ERRBIT_TIMEOUT);
}

}  // namespace

int wait_selftest(int32_t* err, uint64_t limit_ns, cudaStream_t s) {
  return launch("wait_selftest", wait_selftest_kernel, 1, 32, 0, s, limit_ns, err);
}

bool tma_supported(int d) { return d == 32 || d == 64 || d == 128 || d == 256; }

int tma_half_sweep(const SplitPlan& plan, const int32_t* idx, const float* inc_w,
                   const float* inv_norm, const float* src, int64_t src_rows, const float* self_in,
                   float* out, int64_t self_rows, int d, float omega, float* partials,
                   int32_t* err, cudaStream_t s) {
  if (plan.n_a + plan.n_b + plan.n_c + plan.n_d + plan.n_chunks == 0) return HNV_OK;
  CUtensorMap msrc, mself;
  HNV_CHECK(encode_rows_map(&msrc, src, src_rows, d));
  HNV_CHECK(encode_rows_map(&mself, self_in, self_rows, d));
  const bool w = inc_w != nullptr;
  switch (d) {
    case 32:
      return w ? run_tma_classes<8, true>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s)
               : run_tma_classes<8, false>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s);
    case 64:
      return w ? run_tma_classes<16, true>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s)
               : run_tma_classes<16, false>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s);
    case 128:
      return w ? run_tma_classes<32, true>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s)
               : run_tma_classes<32, false>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s);
    case 256:
      return w ? run_tma_classes<64, true>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s)
               : run_tma_classes<64, false>(msrc, mself, plan, idx, inc_w, inv_norm, out, omega, partials, err, s);
    default:
      HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "TMA path has no variant for d = %d", d);
  }
}

}  // namespace hnv
