// Refinement (Algorithm 2, Section 3.3) and projection on one level.
//
// A half-sweep updates every row of one side of the star expansion from its
// neighbours on the other side:
//   hyperedge rows: out_e = (1-w) z_e + w * (1/|e|)          * sum_{v in e} z_v
//   node rows:      out_v = (1-w) z_v + w * (1/sum_e w_e)    * sum_{e ∋ v} w_e z_e
// It is a sparse-rows-times-dense-rows gather, HBM-bound (about 0.5 flop per
// gathered byte): no tensor-core work exists here.
//
// Work decomposition (gather_kernel): a group of G lanes owns one row; each
// lane holds VPL float4 columns (G * VPL * 4 >= d). The group loads G
// neighbour indices with one coalesced access, broadcasts them by shuffle,
// and issues U independent 16-byte row loads per lane before accumulating
// them in incidence order (fixed order: results are deterministic). Rows
// longer than T incidences are cut into chunks of T; each chunk is one work
// item writing an un-normalised partial sum, and finalize_kernel reduces a
// row's partials in chunk order and applies the relaxation.
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
gather_kernel(int32_t n_rows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
              const float* __restrict__ inc_w, const float* __restrict__ inv_norm,
              const float4* __restrict__ src, const float4* self_in, float4* out, int32_t d4,
              float omega, int32_t T, int32_t n_chunks, const int2* __restrict__ chunk_range,
              float4* __restrict__ partials) {
  constexpr int R = 32 / G;                                   // rows per warp pass
  constexpr int UB = (VPL == 1) ? 8 : (VPL == 2 ? 4 : 2);     // row loads in flight
  constexpr int U = UB < G ? UB : G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t n_items = (int64_t)n_rows + n_chunks;
  const float keep = 1.0f - omega;

  for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * R;
       wbase < n_items; wbase += warps_total * R) {
    const int64_t item = wbase + grp;
    int32_t beg = 0, len = 0, row = -1, chunk = -1;
    bool copy_only = false;
    if (item < n_rows) {
      const int32_t r = (int32_t)item;
      const int32_t b = ptr[r], e = ptr[r + 1];
      const int32_t dg = e - b;
      if (dg == 0) {
        if (self_in != out) {   // out-of-place (Jacobi): carry the row over
          copy_only = true;
          row = r;
        }
      } else if (dg <= T) {
        row = r;
        beg = b;
        len = dg;
      }
    } else if (item < n_items) {
      chunk = (int32_t)(item - n_rows);
      const int2 cr = chunk_range[chunk];
      beg = cr.x;
      len = cr.y - cr.x;
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

    if (row >= 0) {
      const float sc = copy_only ? 0.f : omega * inv_norm[row];
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < d4) {
          const size_t o = (size_t)row * d4 + col;
          const float4 sv = self_in[o];
          out[o] = copy_only ? sv : relax4(keep, sc, sv, acc[j]);
        }
      }
    } else if (chunk >= 0) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < d4) partials[(size_t)chunk * d4 + col] = acc[j];
      }
    }
  }
}

// One block per long row: S = blockDim / d4 slices each sum a contiguous
// run of the row's chunk partials (four interleaved accumulators), then
// slice 0 adds the slices in order and applies the relaxation.
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(int32_t n_long, const int32_t* __restrict__ long_rows,
                const int32_t* __restrict__ chunk_ptr, const float4* __restrict__ partials,
                const float* __restrict__ inv_norm, const float4* self_in, float4* out,
                int32_t d4, float omega) {
  extern __shared__ float4 sm[];
  const int S = (int)blockDim.x / d4;
  const int t = threadIdx.x;
  const int slice = t / d4;
  const int col = t - slice * d4;
  const float keep = 1.0f - omega;
  for (int64_t k = blockIdx.x; k < n_long; k += gridDim.x) {
    const int32_t row = long_rows[k];
    const int32_t c0 = chunk_ptr[k], c1 = chunk_ptr[k + 1];
    const int64_t nc = c1 - c0;
    if (slice < S) {
      const int32_t a = c0 + (int32_t)(nc * slice / S);
      const int32_t b = c0 + (int32_t)(nc * (slice + 1) / S);
      float4 a0 = f4_zero(), a1 = f4_zero(), a2 = f4_zero(), a3 = f4_zero();
      int32_t c = a;
      for (; c + 4 <= b; c += 4) {
        const float4 p0 = partials[(size_t)c * d4 + col];
        const float4 p1 = partials[(size_t)(c + 1) * d4 + col];
        const float4 p2 = partials[(size_t)(c + 2) * d4 + col];
        const float4 p3 = partials[(size_t)(c + 3) * d4 + col];
        f4_add(a0, p0);
        f4_add(a1, p1);
        f4_add(a2, p2);
        f4_add(a3, p3);
      }
      for (; c < b; ++c) f4_add(a0, partials[(size_t)c * d4 + col]);
      f4_add(a0, a1);
      f4_add(a2, a3);
      f4_add(a0, a2);
      sm[slice * d4 + col] = a0;
    }
    __syncthreads();
    if (slice == 0) {
      float4 tot = sm[col];
      for (int q = 1; q < S; ++q) f4_add(tot, sm[q * d4 + col]);
      const size_t o = (size_t)row * d4 + col;
      out[o] = relax4(keep, omega * inv_norm[row], self_in[o], tot);
    }
    __syncthreads();
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
  int32_t rows;
  const int32_t* ptr;
  const int32_t* idx;
  const float* inc_w;      // null: unweighted (hyperedge side)
  const float* inv_norm;
  const SplitPlan* plan;
};

template <int G, int VPL>
int run_half(const HalfSweep& h, const float* src, const float* self_in, float* out, int d4,
             float omega, float* partials, cudaStream_t s) {
  constexpr int R = 32 / G;
  const int64_t items = (int64_t)h.rows + h.plan->n_chunks;
  const int64_t warps = (items + R - 1) / R;
  const int64_t blocks64 = (warps + 7) / 8;
  const unsigned blocks = (unsigned)(blocks64 > 0x7fffffff ? 0x7fffffff : blocks64);
  if (h.inc_w) {
    HNV_CHECK(launch("gather_w", gather_kernel<G, VPL, true>, blocks, 256, 0, s, h.rows, h.ptr,
                     h.idx, h.inc_w, h.inv_norm, (const float4*)src, (const float4*)self_in,
                     (float4*)out, d4, omega, h.plan->T, h.plan->n_chunks,
                     (const int2*)h.plan->chunk_range, (float4*)partials));
  } else {
    HNV_CHECK(launch("gather", gather_kernel<G, VPL, false>, blocks, 256, 0, s, h.rows, h.ptr,
                     h.idx, h.inc_w, h.inv_norm, (const float4*)src, (const float4*)self_in,
                     (float4*)out, d4, omega, h.plan->T, h.plan->n_chunks,
                     (const int2*)h.plan->chunk_range, (float4*)partials));
  }
  if (h.plan->n_long > 0) {
    const int S = kFinThreads / d4;
    const size_t smem = sizeof(float4) * (size_t)S * d4;
    const unsigned fb = (unsigned)(h.plan->n_long < 65535 * 16 ? h.plan->n_long : 65535 * 16);
    HNV_CHECK(launch("finalize", finalize_kernel, fb, kFinThreads, smem, s, h.plan->n_long,
                     (const int32_t*)h.plan->long_rows, (const int32_t*)h.plan->chunk_ptr,
                     (const float4*)partials, h.inv_norm, (const float4*)self_in, (float4*)out,
                     d4, omega));
  }
  return HNV_OK;
}

int run_half_dispatch(const HalfSweep& h, const float* src, const float* self_in, float* out,
                      int d, float omega, float* partials, cudaStream_t s) {
  const int d4 = d / 4;
  if (d4 <= 1) return run_half<1, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 2) return run_half<2, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 4) return run_half<4, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 8) return run_half<8, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 16) return run_half<16, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 32) return run_half<32, 1>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 64) return run_half<32, 2>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 128) return run_half<32, 4>(h, src, self_in, out, d4, omega, partials, s);
  if (d4 <= 256) return run_half<32, 8>(h, src, self_in, out, d4, omega, partials, s);
  HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d is larger than 1024", d);
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
  const HalfSweep E{lv.m, lv.e_ptr, lv.e_nodes, nullptr, lv.inv_size_e, &lv.planE};
  const HalfSweep V{lv.n, lv.v_ptr, lv.v_edges, lv.v_w, lv.inv_deg_v, &lv.planV};
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
  const HalfSweep E{lv.m, lv.e_ptr, lv.e_nodes, nullptr, lv.inv_size_e, &lv.planE};
  const HalfSweep V{lv.n, lv.v_ptr, lv.v_edges, lv.v_w, lv.inv_deg_v, &lv.planV};
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
