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
// holds VPL float4 columns (G * VPL * 4 >= d). Class A runs with G = 8,
// B with 16, C and chunks with 32 (for d = 128), so a warp works on up to
// four short rows at once. A group loads its item descriptor (16 bytes) and
// its own row early, loads G neighbour indices with one coalesced access,
// broadcasts them by shuffle and issues U independent 16-byte row loads per
// lane before accumulating them in incidence order (fixed order: results are
// deterministic, no atomics). A chunk writes its un-normalised partial sum;
// finalize_kernel reduces a split row's partials in chunk order and applies
// the relaxation.
#include <cstdlib>

#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

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

// (1 - w) * self + (w * inv) * acc
__device__ __forceinline__ float4 relax4(float keep, float sc, const float4& self, const float4& acc) {
  return make_float4(fmaf(keep, self.x, sc * acc.x), fmaf(keep, self.y, sc * acc.y),
                     fmaf(keep, self.z, sc * acc.z), fmaf(keep, self.w, sc * acc.w));
}

template <int G, int VPL, bool WEIGHTED>
__global__ void __launch_bounds__(256)
gather_kernel(const int4* __restrict__ items, int32_t n_items, const int32_t* __restrict__ idx,
              const float* __restrict__ inc_w, const float* __restrict__ inv_norm,
              const float4* __restrict__ src, const float4* self_in, float4* out, int32_t d4,
              float omega, float4* __restrict__ partials) {
  constexpr int R = 32 / G;                                    // items per warp pass
  // row loads in flight per lane (the weighted variant also holds a weight
  // per load, so it takes half as many to keep its register count down)
  constexpr int UB0 = (VPL == 1) ? 8 : (VPL == 2 ? 4 : (VPL == 4 ? 2 : 1));
  constexpr int UB = (WEIGHTED && UB0 > 1) ? UB0 / 2 : UB0;
  constexpr int U = UB < G ? UB : G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float keep = 1.0f - omega;

  for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * R;
       wbase < n_items; wbase += warps_total * R) {
    const int64_t item = wbase + grp;
    int4 it = make_int4(-1, 0, 0, -1);
    if (item < n_items) it = __ldg(items + item);
    const int32_t row = it.x, beg = it.y, len = it.z, slot = it.w;
    const bool is_row = (row >= 0) && (slot < 0);

    float4 sv[VPL];
    if (is_row) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        sv[j] = (col < d4) ? self_in[(size_t)row * d4 + col] : f4_zero();
      }
    }
    float4 acc[VPL];
#pragma unroll
    for (int j = 0; j < VPL; ++j) acc[j] = f4_zero();

    const int32_t maxlen = __reduce_max_sync(FULL, len);
    for (int32_t off = 0; off < maxlen; off += G) {
      const int32_t mine = len - off;
      const bool have = lg < mine;
      const int32_t my_idx = have ? __ldg(idx + beg + off + lg) : 0;
      float my_w = 0.f;
      if (WEIGHTED) my_w = have ? __ldg(inc_w + beg + off + lg) : 0.f;
      const int32_t cnt = min(G, maxlen - off);
      for (int32_t t = 0; t < cnt; t += U) {
        float4 x[U][VPL];
        float wt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int sl = (t + u) & (G - 1);
          const int32_t nb = __shfl_sync(FULL, my_idx, sl, G);
          const bool ok = (t + u) < mine;
          wt[u] = WEIGHTED ? (ok ? __shfl_sync(FULL, my_w, sl, G) : 0.f) : 1.f;
          const float4* rowp = src + (size_t)nb * d4;
#pragma unroll
          for (int j = 0; j < VPL; ++j) {
            const int col = lg + j * G;
            x[u][j] = (ok && col < d4) ? __ldg(rowp + col) : f4_zero();
          }
        }
        // invalid slots loaded zeros (and weight 0): adding them is exact
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
          for (int j = 0; j < VPL; ++j) {
            if (WEIGHTED)
              f4_fma(acc[j], wt[u], x[u][j]);
            else
              f4_add(acc[j], x[u][j]);
          }
        }
      }
    }

    if (is_row) {
      const float sc = omega * inv_norm[row];
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < d4) out[(size_t)row * d4 + col] = relax4(keep, sc, sv[j], acc[j]);
      }
    } else if (slot >= 0) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < d4) partials[(size_t)slot * d4 + col] = acc[j];
      }
    }
  }
}

// Reduces the chunk partials of split rows in chunk order and relaxes.
// Blocks [0, mid_blocks) give one warp to each of the first n_mid rows (at
// most kMidChunks chunks: lanes over columns, four interleaved
// accumulators); each later block takes one of the n_huge rows: S =
// blockDim / d4 slices sum contiguous runs of chunks (four interleaved
// accumulators each) and slice 0 adds the slices in order.
constexpr int kFinThreads = 1024;

__device__ __forceinline__ float4 sum_strided4(const float4* __restrict__ p, int32_t count,
                                               int32_t stride) {
  float4 a0 = f4_zero(), a1 = f4_zero(), a2 = f4_zero(), a3 = f4_zero();
  int32_t c = 0;
  for (; c + 4 <= count; c += 4) {
    const float4 p0 = p[(size_t)c * stride];
    const float4 p1 = p[(size_t)(c + 1) * stride];
    const float4 p2 = p[(size_t)(c + 2) * stride];
    const float4 p3 = p[(size_t)(c + 3) * stride];
    f4_add(a0, p0);
    f4_add(a1, p1);
    f4_add(a2, p2);
    f4_add(a3, p3);
  }
  for (; c < count; ++c) f4_add(a0, p[(size_t)c * stride]);
  f4_add(a0, a1);
  f4_add(a2, a3);
  f4_add(a0, a2);
  return a0;
}

__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(const int4* __restrict__ long_desc, int32_t n_mid, int32_t n_huge,
                int32_t mid_blocks, const float4* __restrict__ partials,
                const float* __restrict__ inv_norm, const float4* self_in, float4* out,
                int32_t d4, float omega) {
  extern __shared__ float4 sm[];
  const float keep = 1.0f - omega;
  if ((int32_t)blockIdx.x < mid_blocks) {
    const int32_t k = blockIdx.x * (kFinThreads / 32) + (threadIdx.x >> 5);
    if (k >= n_mid) return;
    const int4 ds = long_desc[k];
    const int lane = threadIdx.x & 31;
    const float sc = omega * inv_norm[ds.x];
    for (int col = lane; col < d4; col += 32) {
      const float4 tot = sum_strided4(partials + (size_t)ds.y * d4 + col, ds.z, d4);
      const size_t o = (size_t)ds.x * d4 + col;
      out[o] = relax4(keep, sc, self_in[o], tot);
    }
    return;
  }
  const int32_t k = n_mid + (int32_t)blockIdx.x - mid_blocks;
  if (k >= n_mid + n_huge) return;
  const int4 ds = long_desc[k];
  const int S = (int)blockDim.x / d4;
  const int t = threadIdx.x;
  const int slice = t / d4;
  const int col = t - slice * d4;
  if (slice < S) {
    const int32_t a = (int32_t)((int64_t)ds.z * slice / S);
    const int32_t b = (int32_t)((int64_t)ds.z * (slice + 1) / S);
    sm[slice * d4 + col] = sum_strided4(partials + (size_t)(ds.y + a) * d4 + col, b - a, d4);
  }
  __syncthreads();
  if (slice == 0) {
    float4 tot = sm[col];
    for (int q = 1; q < S; ++q) f4_add(tot, sm[q * d4 + col]);
    const size_t o = (size_t)ds.x * d4 + col;
    out[o] = relax4(keep, omega * inv_norm[ds.x], self_in[o], tot);
  }
}

// Out-of-place sweeps (Jacobi): rows without neighbours carry over.
__global__ void copy_rows_kernel(const int32_t* __restrict__ rows, int32_t n_rows,
                                 const float4* __restrict__ src, float4* __restrict__ dst,
                                 int32_t d4) {
  const int64_t total = (int64_t)n_rows * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / d4;
    const int32_t col = (int32_t)(i - k * d4);
    const size_t o = (size_t)rows[k] * d4 + col;
    dst[o] = src[o];
  }
}

__global__ void project_kernel(int32_t n, int32_t m, const int32_t* __restrict__ rep_v,
                               const int32_t* __restrict__ rep_e, const float4* __restrict__ zc_v,
                               const float4* __restrict__ zc_e, float4* __restrict__ zf_v,
                               float4* __restrict__ zf_e, int32_t d4) {
  const int64_t total = ((int64_t)n + m) * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / d4;
    const int32_t col = (int32_t)(i - row * d4);
    if (row < n) {
      zf_v[i] = zc_v[(size_t)rep_v[row] * d4 + col];
    } else {
      const int64_t e = row - n;
      const int32_t r = rep_e[e];
      const float4* s = (r >= 0) ? zc_e + (size_t)r * d4 : zc_v + (size_t)(-1 - r) * d4;
      zf_e[e * d4 + col] = s[col];
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
};

// Which gather path the half-sweeps use. The default is the per-lane load
// path (gather_kernel). HNV_GATHER=tma selects the TMA-gather path
// (tma_refine.cu) where it has a variant for d; both compute the same sums.
// Measured on the 1M-node workload the TMA path is slower (per-row tensor
// copies of 512-byte rows cap its throughput), so it is opt-in.
bool use_tma(int d) {
  static int mode = -1;
  if (mode < 0) {
    const char* e = getenv("HNV_GATHER");
    mode = (e && e[0] == 't') ? 1 : 0;
  }
  return mode == 1 && tma_supported(d);
}

template <int G, int VPL>
int launch_items(const HalfSweep& h, const int4* items, int32_t n_items, const float* src,
                 const float* self_in, float* out, int d4, float omega, float* partials,
                 cudaStream_t s) {
  if (n_items <= 0) return HNV_OK;
  constexpr int R = 32 / G;
  const int64_t warps = ((int64_t)n_items + R - 1) / R;
  const int64_t blocks64 = (warps + 7) / 8;
  const unsigned blocks = (unsigned)(blocks64 > 0x7fffffff ? 0x7fffffff : blocks64);
  if (h.inc_w)
    return launch("gather_w", gather_kernel<G, VPL, true>, blocks, 256, 0, s, items, n_items,
                  h.idx, h.inc_w, h.inv_norm, (const float4*)src, (const float4*)self_in,
                  (float4*)out, d4, omega, (float4*)partials);
  return launch("gather", gather_kernel<G, VPL, false>, blocks, 256, 0, s, items, n_items, h.idx,
                h.inc_w, h.inv_norm, (const float4*)src, (const float4*)self_in, (float4*)out,
                d4, omega, (float4*)partials);
}

int launch_items_dispatch(int G, int VPL, const HalfSweep& h, const int4* items, int32_t n_items,
                          const float* src, const float* self_in, float* out, int d4,
                          float omega, float* partials, cudaStream_t s) {
#define HNV_CASE(g, v)                                                                 \
  if (G == g && VPL == v)                                                              \
    return launch_items<g, v>(h, items, n_items, src, self_in, out, d4, omega, partials, s);
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
// row width in float4s (rounded up to a power of two), at least enough that
// a lane holds no more than 8 float4s.
int group_lanes(int cls, int d4) {
  int g = cls < next_pow2(d4) ? cls : next_pow2(d4);
  const int gmin = next_pow2((d4 + 7) / 8);
  if (g < gmin) g = gmin;
  return g > 32 ? 32 : g;
}

int run_half_dispatch(const HalfSweep& h, const float* src, const float* self_in, float* out,
                      int d, float omega, float* partials, cudaStream_t s) {
  const int d4 = d / 4;
  if (d4 < 1 || d4 > 256) HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d not in [4, 1024]", d);
  const SplitPlan& p = *h.plan;
  if (use_tma(d)) {
    HNV_CHECK(tma_half_sweep(p, h.idx, h.inc_w, h.inv_norm, src, h.src_rows, self_in, out,
                             h.self_rows, d, omega, partials, h.err, s));
  } else {
    const int4* items = p.items;
    const int cls_lanes[3] = {8, 16, 32};
    const int32_t counts[3] = {p.n_a, p.n_b, p.n_c + p.n_d + p.n_chunks};
    int32_t off = 0;
    for (int c = 0; c < 3; ++c) {
      const int G = group_lanes(cls_lanes[c], d4);
      const int VPL = next_pow2((d4 + G - 1) / G);
      HNV_CHECK(launch_items_dispatch(G, VPL, h, items + off, counts[c], src, self_in, out, d4,
                                      omega, partials, s));
      off += counts[c];
    }
  }
  if (p.n_mid + p.n_huge > 0) {
    const int32_t mid_blocks = (p.n_mid + kFinThreads / 32 - 1) / (kFinThreads / 32);
    const int S = kFinThreads / d4;
    const size_t smem = sizeof(float4) * (size_t)S * d4;
    HNV_CHECK(launch("finalize", finalize_kernel, (unsigned)(mid_blocks + p.n_huge), kFinThreads,
                     smem, s, (const int4*)p.long_desc, p.n_mid, p.n_huge, mid_blocks,
                     (const float4*)partials, h.inv_norm, (const float4*)self_in, (float4*)out,
                     d4, omega));
  }
  if (self_in != out && p.n_zero > 0)
    HNV_CHECK(launch("copy_rows", copy_rows_kernel, grid_for((int64_t)p.n_zero * d4, 256), 256, 0,
                     s, (const int32_t*)p.zero_rows, p.n_zero, (const float4*)self_in,
                     (float4*)out, d4));
  return HNV_OK;
}

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

int refine_level(hnv_graph* g, int level, float* z_v, float* z_e, int d, float omega, int sweeps,
                 int mode, cudaStream_t s) {
  Level& lv = g->levels[level];
  const int64_t chunks = lv.planE.n_chunks > lv.planV.n_chunks ? lv.planE.n_chunks : lv.planV.n_chunks;
  HNV_CHECK(ensure_scratch(&g->partials, &g->partials_bytes,
                           sizeof(float) * (size_t)(chunks > 0 ? chunks : 1) * d, s));
  if (mode == HNV_SWEEP_JACOBI)
    HNV_CHECK(ensure_scratch(&g->jacobi_tmp, &g->jacobi_bytes,
                             sizeof(float) * ((size_t)lv.m > 0 ? lv.m : 1) * d, s));
  const HalfSweep E{lv.e_nodes, nullptr, lv.inv_size_e, &lv.planE, lv.n, lv.m, g->d_err};
  const HalfSweep V{lv.v_edges, lv.v_w, lv.inv_deg_v, &lv.planV, lv.m, lv.n, g->d_err};
  const double n = lv.n, m = lv.m, nnz = (double)lv.nnz;
  const double bytesE = 4.0 * (n * d + 2.0 * m * d + nnz + 2.0 * m + 1.0);
  const double bytesV = 4.0 * (m * d + 2.0 * n * d + 2.0 * nnz + 2.0 * n + 1.0);
  for (int it = 0; it < sweeps; ++it) {
    if (mode == HNV_SWEEP_TWO_PHASE) {
      {
        PhaseScope ps(HNV_PHASE_REFINE_E, s, bytesE);
        HNV_CHECK(run_half_dispatch(E, z_v, z_e, z_e, d, omega, g->partials, s));
      }
      {
        PhaseScope ps(HNV_PHASE_REFINE_V, s, bytesV);
        HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, d, omega, g->partials, s));
      }
    } else {
      {
        PhaseScope ps(HNV_PHASE_REFINE_E, s, bytesE);
        HNV_CHECK(run_half_dispatch(E, z_v, z_e, g->jacobi_tmp, d, omega, g->partials, s));
      }
      {
        PhaseScope ps(HNV_PHASE_REFINE_V, s, bytesV);
        HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, d, omega, g->partials, s));
      }
      if (lv.m > 0)
        HNV_CUDA(cudaMemcpyAsync(z_e, g->jacobi_tmp, sizeof(float) * (size_t)lv.m * d,
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
    HNV_CHECK(run_half_dispatch(E, z_v, z_e, z_e, d, omega, partials, s));
    HNV_CHECK(run_half_dispatch(V, z_e, z_v, z_v, d, omega, partials, s));
  }
  return HNV_OK;
}

int project_level(const hnv_graph* g, int fine_level, const float* zc_v, const float* zc_e,
                  float* zf_v, float* zf_e, int d, cudaStream_t s) {
  const Level& f = g->levels[fine_level];
  const Level& c = g->levels[fine_level + 1];
  const int d4 = d / 4;
  const double bytes = 4.0 * (((double)f.n + f.m) * d * 1.0 + ((double)c.n + c.m) * d +
                              (double)f.n + f.m);
  PhaseScope ps(HNV_PHASE_PROJECT, s, bytes);
  const int64_t total = ((int64_t)f.n + f.m) * d4;
  return launch("project", project_kernel, grid_for(total, 256, 16), 256, 0, s, f.n, f.m,
                (const int32_t*)f.rep_v, (const int32_t*)f.rep_e, (const float4*)zc_v,
                (const float4*)zc_e, (float4*)zf_v, (float4*)zf_e, d4);
}

}  // namespace hnv
