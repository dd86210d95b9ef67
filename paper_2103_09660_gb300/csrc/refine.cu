// Refinement (Algorithm 2, Section 3.3) and projection on one level.
//
// A half-sweep updates every row of one side of the star expansion from its
// neighbours on the other side:
//   hyperedge rows: out_e = (1-w) z_e + w * (1/|e|)          * sum_{v in e} z_v
//   node rows:      out_v = (1-w) z_v + w * (1/sum_e w_e)    * sum_{e ∋ v} w_e z_e
// It is a sparse-rows-times-dense-rows gather, HBM-bound (about 0.5 flop per
// gathered byte): no tensor-core work exists here.
//
// Work decomposition. Each half-sweep has a plan of work items (SplitPlan):
// rows of 1..4, 5..16 and 17..T incidences (classes A, B, C) and chunks of
// at most T incidences cut from longer rows. gather_kernel<G, VPL, W> gives
// each item a group of G lanes (R = 32/G items per warp at once); each lane
// holds VPL float4 columns (G * VPL * 4 >= d). Classes A and B run with
// G = 16, C and chunks with 32 (for d = 128), so a warp works on two short
// rows at once. A group loads its item descriptor (16 bytes) and
// its own row early, loads G neighbour indices with one coalesced access,
// broadcasts them by shuffle and issues U independent 16-byte row loads per
// lane before accumulating them in incidence order (fixed order: results are
// deterministic, no atomics). A chunk writes its un-normalised partial sum;
// finalize_kernel reduces a split row's partials in chunk order and applies
// the relaxation.
#include <cuda_bf16.h>

#include <cstdlib>

#include "refine_device.cuh"

namespace hnv {

namespace {

using dev::VecT;

// Threads per block of the gather kernels. A block's slot on the SM frees
// only when all its warps are done, and the warps of a block wait on
// different DRAM and L2 latencies; two-warp blocks let the scheduler refill
// an SM warp pair by warp pair. Measured on the 1M-node workload (d = 128,
// FP32): the V-cycle took 97.1 ms with 256-thread blocks, 92.5 ms with 128
// and 91.0 ms with 64, every level and both sides faster.
constexpr int kGatherThreads = 64;

// Passes per warp of the packed short-row kernel (see gather_packed_kernel).
constexpr int kPackedPasses = 4;

template <typename T, int G, int VPL, bool WEIGHTED, bool WIDE_U = false>
__global__ void __launch_bounds__(256)
gather_kernel(const int4* __restrict__ items, int32_t n_items, const int32_t* __restrict__ idx,
              const float* __restrict__ inc_w, const float* __restrict__ inv_norm,
              const uint4* __restrict__ src, const uint4* self_in, uint4* out, int32_t dv,
              float keep, float scale, float* __restrict__ partials) {
  constexpr int R = 32 / G;                                    // items per warp pass
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * R;
       wbase < n_items; wbase += warps_total * R) {
    const int64_t item = wbase + grp;
    int4 it = make_int4(-1, 0, 0, -1);
    if (item < n_items) it = __ldg(items + item);
    dev::gather_item<T, G, VPL, WEIGHTED, false, WIDE_U>(it, lg, idx, inc_w, inv_norm, src,
                                                         self_in, out, dv, keep, scale, partials);
  }
}

// The short rows of an unweighted side whose plan packs their neighbours
// next to their items (SplitPlan::a_members: rows of 1-4 members, PK = 1;
// b_members: rows of 5-16, PK = 2). A group reads a row's descriptor and its
// neighbour indices side by side, not one after the other. Each warp takes
// PASSES consecutive passes (R rows each) and loads the descriptors and
// neighbours of the pass after next while it gathers the current one, so a
// row's gathers never wait for its descriptor; it also prefetches the next
// pass's own rows into L2, so their DRAM latency is spent during the
// current pass. The register budget is capped so that 32 warps stay
// resident per SM. Measured in one process on the 1M-node workload: against
// one pass per warp (64-thread blocks both) the hyperedge half-sweeps were
// 6-15% faster on levels 1-4 and even on level 0, the V-cycle 89.4 against
// 92.5 ms; the own-row prefetch took the V-cycle from 89.1 to 86.8 ms
// (hyperedge half-sweeps of levels 1-4 5-8% faster).
template <typename T, int G, int VPL, int PK, int PASSES>
__global__ void __launch_bounds__(256, 4)
gather_packed_kernel(const int4* __restrict__ items, const void* __restrict__ members,
                     int32_t n_items, const int32_t* __restrict__ idx,
                     const float* __restrict__ inc_w, const float* __restrict__ inv_norm,
                     const uint4* __restrict__ src, const uint4* self_in, uint4* out, int32_t dv,
                     float keep, float scale, float* __restrict__ partials) {
  static_assert(PK == 1 || PK == 2, "packed class A or B");
  static_assert(PK == 1 || G >= 16, "a group holds the 16 packed neighbours one per lane");
  constexpr int R = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
  // 32-bit item arithmetic: the grid covers n_items < 2^31
  const int32_t warp = (int32_t)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  const int32_t first = warp * (PASSES * R);
  if (first >= n_items) return;                    // warp-uniform
  auto item_of = [&](int k) { return first + k * R + grp; };
  auto load_it = [&](int k) -> int4 {
    const int32_t item = item_of(k);
    return (k < PASSES && item < n_items) ? __ldg(items + item) : make_int4(-1, 0, 0, -1);
  };
  // this lane's first neighbour of the row its group takes in pass k
  auto load_head = [&](int k, int32_t& i0, float& w0) {
    const int32_t item = item_of(k);
    const bool valid = k < PASSES && item < n_items;
    i0 = 0;
    w0 = 0.f;
    if (PK == 1) {
      if (valid) {
        const int4 mem = __ldg(reinterpret_cast<const int4*>(members) + item);
        i0 = lg == 0 ? mem.x : lg == 1 ? mem.y : lg == 2 ? mem.z : mem.w;
      }
    } else if (valid && lg < 16) {
      i0 = __ldg(reinterpret_cast<const int32_t*>(members) + (size_t)item * 16 + lg);
    }
  };
  int4 cur = load_it(0);
  int32_t ci;
  float cw;
  load_head(0, ci, cw);
  int4 nxt = load_it(1);
  int32_t xi;
  float xw;
  load_head(1, xi, xw);
#pragma unroll 1
  for (int k = 0; k < PASSES; ++k) {
    if (first + k * R >= n_items) break;           // warp-uniform
    // the next pass's own row (its descriptor arrived during the previous
    // pass) is brought into L2 while this pass gathers
    if (nxt.x >= 0 && nxt.w < 0 && keep != 0.f) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < dv)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(self_in + (size_t)nxt.x * dv + col));
      }
    }
    int32_t ni;
    float nw;
    const int4 nn = load_it(k + 2);
    load_head(k + 2, ni, nw);
    dev::gather_item<T, G, VPL, false, true>(cur, lg, idx, inc_w, inv_norm, src, self_in, out,
                                             dv, keep, scale, partials, ci, cw);
    cur = nxt;
    ci = xi;
    cw = xw;
    nxt = nn;
    xi = ni;
    xw = nw;
  }
}

// Reduces the chunk partials of split rows. Blocks [0, mid_blocks) give one
// warp to each of the first n_mid rows (at most kMidChunks chunks); each
// later block takes one of the n_huge rows (slices of the block sum
// contiguous runs of chunks, slice 0 adds the slices in order).
constexpr int kFinThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(const int4* __restrict__ long_desc, int32_t n_mid, int32_t n_huge,
                int32_t mid_blocks, const float* __restrict__ partials,
                const float* __restrict__ inv_norm, const uint4* self_in, uint4* out,
                int32_t dv, float keep, float scale) {
  extern __shared__ float4 sm4[];
  if ((int32_t)blockIdx.x < mid_blocks) {
    const int32_t k = blockIdx.x * (kFinThreads / 32) + (threadIdx.x >> 5);
    if (k >= n_mid) return;
    dev::finalize_mid<T>(long_desc[k], threadIdx.x & 31, partials, inv_norm, self_in, out, dv, keep,
                         scale);
    return;
  }
  const int32_t k = n_mid + (int32_t)blockIdx.x - mid_blocks;
  if (k >= n_mid + n_huge) return;
  dev::finalize_huge<T>(long_desc[k], reinterpret_cast<float*>(sm4), partials, inv_norm, self_in,
                        out, dv, keep, scale);
}

// Out-of-place sweeps (Jacobi): rows without neighbours carry over.
__global__ void copy_rows_kernel(const int32_t* __restrict__ rows, int32_t n_rows,
                                 const uint4* __restrict__ src, uint4* __restrict__ dst,
                                 int32_t dv) {
  const int64_t total = (int64_t)n_rows * dv;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / dv;
    const int32_t col = (int32_t)(i - k * dv);
    const size_t o = (size_t)rows[k] * dv + col;
    dst[o] = src[o];
  }
}

// Projection: bitwise row copies through rep_v / rep_e (any element type).
__global__ void project_kernel(int32_t n, int32_t m, const int32_t* __restrict__ rep_v,
                               const int32_t* __restrict__ rep_e, const uint4* __restrict__ zc_v,
                               const uint4* __restrict__ zc_e, uint4* __restrict__ zf_v,
                               uint4* __restrict__ zf_e, int32_t dv) {
  const int64_t total = ((int64_t)n + m) * dv;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / dv;
    const int32_t col = (int32_t)(i - row * dv);
    if (row < n) {
      zf_v[i] = zc_v[(size_t)rep_v[row] * dv + col];
    } else {
      const int64_t e = row - n;
      const int32_t r = rep_e[e];
      const uint4* s = (r >= 0) ? zc_e + (size_t)r * dv : zc_v + (size_t)(-1 - r) * dv;
      zf_e[e * dv + col] = s[col];
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct HalfSweep {
  const int32_t* idx;
  const float* inc_w;      // null: unweighted (hyperedge side)
  const float* inv_norm;
  const SplitPlan* plan;
  int64_t src_rows;        // rows of the neighbour table
  int64_t self_rows;       // rows of this side's table
  int32_t* err;            // device error word (bounded waits)
  bool allow_tma = true;   // forward relaxations only
  // optional: run the row classes concurrently on these side streams
  const hnv_graph* conc = nullptr;
};

// Which gather path the half-sweeps use. The default is the per-lane load
// path (gather_kernel). HNV_GATHER=tma selects the TMA-gather path
// (tma_refine.cu) for float32 rows where it has a variant for d; both
// compute the same sums. Measured on the 1M-node workload the TMA path is
// slower (per-row tensor copies of 512-byte rows cap its throughput), so it
// is opt-in.
bool use_tma(int d) {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("HNV_GATHER");
    mode = (e && e[0] == 't') ? 1 : 0;
  }
  return mode == 1 && tma_supported(d);
}

template <typename T, int G, int VPL>
int launch_items(const HalfSweep& h, const int4* items, int32_t n_items, const void* src,
                 const void* self_in, void* out, int dv, float keep, float scale,
                 float* partials, cudaStream_t s) {
  if (n_items <= 0) return HNV_OK;
  constexpr int R = 32 / G;
  constexpr int WPB = kGatherThreads / 32;
  const int64_t warps = ((int64_t)n_items + R - 1) / R;
  const int64_t blocks64 = (warps + WPB - 1) / WPB;
  const unsigned blocks = (unsigned)(blocks64 > 0x7fffffff ? 0x7fffffff : blocks64);
  // the weighted long-row kernel keeps 8 row loads in flight per lane (not
  // the weighted default of 4): the coarse levels' node half-sweeps, bound
  // by L2 latency, got 1-2% faster; level 0 is unchanged
  if (h.inc_w && G == 32 && VPL == 1)
    return launch("gather_w", gather_kernel<T, G, VPL, true, true>, blocks, kGatherThreads, 0, s,
                  items, n_items, h.idx, h.inc_w, h.inv_norm, (const uint4*)src,
                  (const uint4*)self_in, (uint4*)out, dv, keep, scale, partials);
  if (h.inc_w)
    return launch("gather_w", gather_kernel<T, G, VPL, true>, blocks, kGatherThreads, 0, s,
                  items, n_items, h.idx, h.inc_w, h.inv_norm, (const uint4*)src,
                  (const uint4*)self_in, (uint4*)out, dv, keep, scale, partials);
  return launch("gather", gather_kernel<T, G, VPL, false>, blocks, kGatherThreads, 0, s, items,
                n_items, h.idx, h.inc_w, h.inv_norm, (const uint4*)src, (const uint4*)self_in,
                (uint4*)out, dv, keep, scale, partials);
}

template <typename T, int G, int VPL, int PK>
int launch_packed(const HalfSweep& h, const int4* items, const void* members, int32_t n_items,
                  const void* src, const void* self_in, void* out, int dv, float keep,
                  float scale, float* partials, cudaStream_t s) {
  if (n_items <= 0) return HNV_OK;
  constexpr int R = 32 / G;
  constexpr int WPB = kGatherThreads / 32;
  const int64_t warps = ((int64_t)n_items + R * kPackedPasses - 1) / (R * kPackedPasses);
  const unsigned blocks = (unsigned)((warps + WPB - 1) / WPB);
  return launch("gather_packed", gather_packed_kernel<T, G, VPL, PK, kPackedPasses>, blocks,
                kGatherThreads, 0, s, items, members, n_items, h.idx, (const float*)nullptr,
                h.inv_norm, (const uint4*)src, (const uint4*)self_in, (uint4*)out, dv, keep,
                scale, partials);
}

// 1: no packed variant for (G, VPL) (not an error code); the caller takes
// the regular kernel. Class-A rows have at most 4 members, so G >= 4.
template <typename T>
int launch_packed_dispatch(int G, int VPL, const HalfSweep& h, const int4* items,
                           const int4* members, int32_t n_items, const void* src,
                           const void* self_in, void* out, int dv, float keep, float scale,
                           float* partials, cudaStream_t s) {
#define HNV_PCASE(g, v)                                                                      \
  if (G == g && VPL == v)                                                                    \
    return launch_packed<T, g, v, 1>(h, items, members, n_items, src, self_in, out, dv,     \
                                     keep, scale, partials, s);
  HNV_PCASE(4, 1) HNV_PCASE(8, 1) HNV_PCASE(8, 2) HNV_PCASE(8, 4)
  HNV_PCASE(16, 1) HNV_PCASE(16, 2) HNV_PCASE(16, 4) HNV_PCASE(32, 1) HNV_PCASE(32, 2)
#undef HNV_PCASE
  return 1;
}

// As launch_packed_dispatch for the class-B rows (16 packed slots, G >= 16).
template <typename T>
int launch_packed16_dispatch(int G, int VPL, const HalfSweep& h, const int4* items,
                             const int32_t* members, int32_t n_items, const void* src,
                             const void* self_in, void* out, int dv, float keep, float scale,
                             float* partials, cudaStream_t s) {
#define HNV_PCASE(g, v)                                                                      \
  if (G == g && VPL == v)                                                                    \
    return launch_packed<T, g, v, 2>(h, items, members, n_items, src, self_in, out, dv,     \
                                     keep, scale, partials, s);
  HNV_PCASE(16, 1) HNV_PCASE(16, 2) HNV_PCASE(16, 4) HNV_PCASE(32, 1) HNV_PCASE(32, 2)
#undef HNV_PCASE
  return 1;
}

template <typename T>
int launch_items_dispatch(int G, int VPL, const HalfSweep& h, const int4* items, int32_t n_items,
                          const void* src, const void* self_in, void* out, int dv, float keep,
                          float scale, float* partials, cudaStream_t s) {
#define HNV_CASE(g, v)                                                                       \
  if (G == g && VPL == v)                                                                    \
    return launch_items<T, g, v>(h, items, n_items, src, self_in, out, dv, keep, scale,     \
                                 partials, s);
  HNV_CASE(1, 1) HNV_CASE(2, 1) HNV_CASE(4, 1)
  HNV_CASE(8, 1) HNV_CASE(8, 2) HNV_CASE(8, 4) HNV_CASE(8, 8)
  HNV_CASE(16, 1) HNV_CASE(16, 2) HNV_CASE(16, 4) HNV_CASE(16, 8)
  HNV_CASE(32, 1) HNV_CASE(32, 2) HNV_CASE(32, 4) HNV_CASE(32, 8)
#undef HNV_CASE
  HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "no gather variant for G=%d VPL=%d", G, VPL);
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Lanes per item for a class whose natural width is `cls` lanes: at most the
// row width in vectors (rounded up to a power of two), at least enough that
// a lane holds no more than 8 vectors.
int group_lanes(int cls, int dv) {
  int g = cls < next_pow2(dv) ? cls : next_pow2(dv);
  const int gmin = next_pow2((dv + 7) / 8);
  if (g < gmin) g = gmin;
  return g > 32 ? 32 : g;
}

// The split-row reduction of a plan (nothing if it has no split rows).
template <typename T>
int launch_finalize(const HalfSweep& h, const SplitPlan& p, float* partials, const void* self_in,
                    void* out, int dv, float keep, float scale, cudaStream_t s) {
  if (p.n_mid + p.n_huge == 0) return HNV_OK;
  constexpr int N = VecT<T>::N;
  const int32_t mid_blocks = (p.n_mid + kFinThreads / 32 - 1) / (kFinThreads / 32);
  const int S = kFinThreads / dv;
  const size_t smem = sizeof(float) * (size_t)S * dv * N;
  return launch("finalize", finalize_kernel<T>, (unsigned)(mid_blocks + p.n_huge), kFinThreads,
                smem, s, (const int4*)p.long_desc, p.n_mid, p.n_huge, mid_blocks,
                (const float*)partials, h.inv_norm, (const uint4*)self_in, (uint4*)out, dv, keep,
                scale);
}

template <typename T>
int run_half(const HalfSweep& h, const void* src, const void* self_in, void* out, int d,
             float keep, float scale, float* partials, cudaStream_t s) {
  constexpr int N = VecT<T>::N;
  const int dv = d / N;
  if (dv < 1 || dv > 256) HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d out of range", d);
  const SplitPlan& p = *h.plan;
  if (sizeof(T) == 4 && h.allow_tma && keep == 1.0f - scale && h.inv_norm && use_tma(d)) {
    HNV_CHECK(tma_half_sweep(p, h.idx, h.inc_w, h.inv_norm, (const float*)src, h.src_rows,
                             (const float*)self_in, (float*)out, h.self_rows, d, scale, partials,
                             h.err, s));
    HNV_CHECK(launch_finalize<T>(h, p, partials, self_in, out, dv, keep, scale, s));
  } else {
    const int4* items = p.items;
    // lanes per item of classes A, B and the rest. With 16 lanes on rows of
    // 1-4 incidences each lane holds fewer columns and keeps all of a short
    // row's neighbour loads in flight at once (measured on the 1M workload at
    // d = 128: hyperedge half-sweeps 4-7% faster than with 8 lanes).
    const int cls_lanes[3] = {16, 16, 32};
    const int32_t counts[3] = {p.n_a, p.n_b, p.n_c + p.n_d + p.n_chunks};
    // The classes touch disjoint rows of `out` (chunks only write partials),
    // so they may run at once: classes B and the rest go to side streams
    // forked from s and joined back before the split-row reduction.
    const bool conc = h.conc && counts[1] > 0 && counts[2] > 0;
    cudaStream_t cs[3] = {s, s, s};
    if (conc) {
      HNV_CUDA(cudaEventRecord(h.conc->fork_ev, s));
      for (int i = 0; i < 2; ++i) {
        HNV_CUDA(cudaStreamWaitEvent(h.conc->aux[i], h.conc->fork_ev, 0));
        cs[i + 1] = h.conc->aux[i];
      }
    }
    int32_t off = 0;
    for (int c = 0; c < 3; ++c) {
      const int G = group_lanes(cls_lanes[c], dv);
      const int VPL = next_pow2((dv + G - 1) / G);
      int rc = 1;
      if (c == 0 && p.a_members && !h.inc_w)
        rc = launch_packed_dispatch<T>(G, VPL, h, items, p.a_members, counts[0], src, self_in, out,
                                       dv, keep, scale, partials, cs[c]);
      if (c == 1 && p.b_members && !h.inc_w)
        rc = launch_packed16_dispatch<T>(G, VPL, h, items + off, p.b_members, counts[1], src,
                                         self_in, out, dv, keep, scale, partials, cs[c]);
      if (rc == 1)
        rc = launch_items_dispatch<T>(G, VPL, h, items + off, counts[c], src, self_in, out, dv,
                                      keep, scale, partials, cs[c]);
      HNV_CHECK(rc);
      off += counts[c];
    }
    // the split rows' reduction needs only the chunks (the last class), and
    // writes only split rows: it follows that class on its stream
    HNV_CHECK(launch_finalize<T>(h, p, partials, self_in, out, dv, keep, scale, cs[2]));
    if (conc) {
      for (int i = 0; i < 2; ++i) {
        HNV_CUDA(cudaEventRecord(h.conc->join_ev[i], h.conc->aux[i]));
        HNV_CUDA(cudaStreamWaitEvent(s, h.conc->join_ev[i], 0));
      }
    }
  }
  if (self_in != out && p.n_zero > 0)
    HNV_CHECK(launch("copy_rows", copy_rows_kernel, grid_for((int64_t)p.n_zero * dv, 256), 256, 0,
                     s, (const int32_t*)p.zero_rows, p.n_zero, (const uint4*)self_in,
                     (uint4*)out, dv));
  return HNV_OK;
}

int run_half_dispatch(const HalfSweep& h, const void* src, const void* self_in, void* out,
                      int dtype, int d, float omega, float* partials, cudaStream_t s) {
  const float keep = 1.0f - omega;
  if (dtype == HNV_BF16)
    return run_half<__nv_bfloat16>(h, src, self_in, out, d, keep, omega, partials, s);
  return run_half<float>(h, src, self_in, out, d, keep, omega, partials, s);
}

size_t elem_size(int dtype) { return dtype == HNV_BF16 ? 2 : 4; }

}  // namespace

// out[row] = keep * self[row] + scale * norm[row] * sum over the plan's row of
// wgt[k] * src[idx[k]] (float32 rows; see gather_kernel). norm and wgt may be
// null (1). The load path only; with conc (a graph that has side streams) the
// row classes run concurrently, as in a refinement half-sweep.
int gather_rows_f32(const SplitPlan& plan, const int32_t* idx, const float* wgt,
                    const float* norm, const float* src, const float* self_in, float* out, int d,
                    float keep, float scale, float* partials, cudaStream_t s,
                    const hnv_graph* conc) {
  HalfSweep h{idx, wgt, norm, &plan, 0, 0, nullptr, false};
  if (conc && conc->aux[0] && conc->aux[1]) h.conc = conc;
  return run_half<float>(h, src, self_in, out, d, keep, scale, partials, s);
}

namespace {

int ensure_scratch(float** p, size_t* have, size_t need, cudaStream_t s) {
  if (need <= *have && *p) return HNV_OK;
  if (*p) dev_free(*p, s);
  *p = nullptr;
  *have = 0;
  void* q = nullptr;
  HNV_CHECK(dev_alloc(&q, need, s));
  *p = static_cast<float*>(q);
  *have = need;
  return HNV_OK;
}

}  // namespace

int refine_level(hnv_graph* g, int level, void* z_v, void* z_e, int dtype, int d, float omega,
                 int sweeps, int mode, cudaStream_t s) {
  NvtxRange nvtx("hnv refine level %d (%d sweeps)", level, sweeps);
  Level& lv = g->levels[level];
  const size_t es = elem_size(dtype);
  const SplitPlan* planE = &lv.planE;
  const SplitPlan* planV = &lv.planV;
  if (!use_tma(d)) {
    HNV_CHECK(side_plan(g, &lv, 0, es * (size_t)d, &planE, s));
    HNV_CHECK(side_plan(g, &lv, 1, es * (size_t)d, &planV, s));
  }
  const int64_t chunks = planE->n_chunks > planV->n_chunks ? planE->n_chunks : planV->n_chunks;
  HNV_CHECK(ensure_scratch(&g->partials, &g->partials_bytes,
                           sizeof(float) * (size_t)(chunks > 0 ? chunks : 1) * d, s));
  if (mode == HNV_SWEEP_JACOBI)
    HNV_CHECK(ensure_scratch(&g->jacobi_tmp, &g->jacobi_bytes,
                             es * ((size_t)lv.m > 0 ? lv.m : 1) * d, s));
  HalfSweep E{lv.e_nodes, nullptr, lv.inv_size_e, planE, lv.n, lv.m, g->d_err};
  HalfSweep V{lv.v_edges, lv.v_w, lv.inv_deg_v, planV, lv.m, lv.n, g->d_err};
  if (g->aux[0] && g->aux[1]) E.conc = V.conc = g;
  const double n = lv.n, m = lv.m, nnz = (double)lv.nnz;
  const double bytesE = (double)es * (n * d + 2.0 * m * d) + 4.0 * (nnz + 2.0 * m + 1.0);
  const double bytesV = (double)es * (m * d + 2.0 * n * d) + 4.0 * (2.0 * nnz + 2.0 * n + 1.0);
  for (int it = 0; it < sweeps; ++it) {
    if (mode == HNV_SWEEP_TWO_PHASE) {
      {
        PhaseScope ps(HNV_PHASE_REFINE_E, s, bytesE);
        HNV_CHECK(run_half_dispatch(E, z_v, z_e, z_e, dtype, d, omega, g->partials, s));
      }
      {
        PhaseScope ps(HNV_PHASE_REFINE_V, s, bytesV);
        HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, dtype, d, omega, g->partials, s));
      }
    } else {
      {
        PhaseScope ps(HNV_PHASE_REFINE_E, s, bytesE);
        HNV_CHECK(run_half_dispatch(E, z_v, z_e, g->jacobi_tmp, dtype, d, omega, g->partials, s));
      }
      {
        PhaseScope ps(HNV_PHASE_REFINE_V, s, bytesV);
        HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, dtype, d, omega, g->partials, s));
      }
      if (lv.m > 0)
        HNV_CUDA(cudaMemcpyAsync(z_e, g->jacobi_tmp, es * (size_t)lv.m * d,
                                 cudaMemcpyDeviceToDevice, s));
    }
  }
  return HNV_OK;
}

int refine_two_phase_with_partials(const hnv_graph* g, int level, float* z_v, float* z_e, int d,
                                   float omega, int sweeps, float* partials, cudaStream_t s) {
  const Level& lv = g->levels[level];
  const HalfSweep E{lv.e_nodes, nullptr, lv.inv_size_e, &lv.planE, lv.n, lv.m, g->d_err};
  const HalfSweep V{lv.v_edges, lv.v_w, lv.inv_deg_v, &lv.planV, lv.m, lv.n, g->d_err};
  for (int it = 0; it < sweeps; ++it) {
    HNV_CHECK(run_half_dispatch(E, z_v, z_e, z_e, HNV_F32, d, omega, partials, s));
    HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, HNV_F32, d, omega, partials, s));
  }
  return HNV_OK;
}

int project_level(const hnv_graph* g, int fine_level, const void* zc_v, const void* zc_e,
                  void* zf_v, void* zf_e, int dtype, int d, cudaStream_t s) {
  NvtxRange nvtx("hnv project onto level %d", fine_level);
  const Level& f = g->levels[fine_level];
  const Level& c = g->levels[fine_level + 1];
  const size_t es = elem_size(dtype);
  const int dv = (int)(d * es / 16);
  const double bytes = (double)es * (((double)f.n + f.m) * d + ((double)c.n + c.m) * d) +
                       4.0 * ((double)f.n + f.m);
  PhaseScope ps(HNV_PHASE_PROJECT, s, bytes);
  const int64_t total = ((int64_t)f.n + f.m) * dv;
  return launch("project", project_kernel, grid_for(total, 256, 16), 256, 0, s, f.n, f.m,
                (const int32_t*)f.rep_v, (const int32_t*)f.rep_e, (const uint4*)zc_v,
                (const uint4*)zc_e, (uint4*)zf_v, (uint4*)zf_e, dv);
}

}  // namespace hnv
