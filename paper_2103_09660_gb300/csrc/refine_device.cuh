// Device code shared by the single-graph (refine.cu) and batched (batch.cu)
// refinement kernels: row vectors, the per-item gather, and the split-row
// reductions. See refine.cu for the work decomposition.
#pragma once

#include <cuda_bf16.h>

#include "hnv_internal.cuh"

namespace hnv {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// A row is a sequence of 16-byte vectors: 4 float32 or 8 bfloat16 values.
// Arithmetic is float32 either way; VecT converts a vector to and from its
// float values (bfloat16 to float is exact; float to bfloat16 rounds to
// nearest even on store).
template <typename T>
struct VecT;

template <>
struct VecT<float> {
  static constexpr int N = 4;
  __device__ __forceinline__ static void unpack(const uint4& v, float* f) {
    f[0] = __uint_as_float(v.x);
    f[1] = __uint_as_float(v.y);
    f[2] = __uint_as_float(v.z);
    f[3] = __uint_as_float(v.w);
  }
  __device__ __forceinline__ static uint4 pack(const float* f) {
    return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]),
                      __float_as_uint(f[3]));
  }
};

template <>
struct VecT<__nv_bfloat16> {
  static constexpr int N = 8;
  // each 32-bit word holds two values, the lower-indexed one in the low half
  __device__ __forceinline__ static void unpack(const uint4& v, float* f) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f[2 * k] = __uint_as_float(w[k] << 16);
      f[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
  __device__ __forceinline__ static uint32_t pair(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ __forceinline__ static uint4 pack(const float* f) {
    return make_uint4(pair(f[0], f[1]), pair(f[2], f[3]), pair(f[4], f[5]), pair(f[6], f[7]));
  }
};

// One work item of a half-sweep, processed by a group of G lanes (all 32
// lanes of the warp call this together; R = 32/G groups hold R items).
//   item {row, first incidence, length, partial slot or -1}
//   row item:  out[row] = keep * self[row] + scale * norm[row] * sum_k wgt_k src[idx_k]
//   chunk:     partials[slot] = sum_k wgt_k src[idx_k]   (float32)
// norm (inv_norm) may be null (1); with keep == 0 the own row is not read.
// PRE: the caller supplies this lane's first neighbour index (incidence
// beg + lg, any value where lg >= len) in idx0 instead of it being loaded,
// and for a weighted side that incidence's weight in w0.
template <typename T, int G, int VPL, bool WEIGHTED, bool PRE = false, bool WIDE_U = false>
__device__ __forceinline__ void gather_item(int4 it, int lg, const int32_t* __restrict__ idx,
                                            const float* __restrict__ inc_w,
                                            const float* __restrict__ inv_norm,
                                            const uint4* __restrict__ src, const uint4* self_in,
                                            uint4* out, int32_t dv, float keep, float scale,
                                            float* __restrict__ partials, int32_t idx0 = 0,
                                            float w0 = 0.f) {
  using V = VecT<T>;
  constexpr int N = V::N;
  // row loads in flight per lane (the weighted variant also holds a weight
  // per load, so it takes half as many to keep its register count down,
  // unless WIDE_U)
  constexpr int UB0 = (VPL == 1) ? 8 : (VPL == 2 ? 4 : (VPL == 4 ? 2 : 1));
  constexpr int UB = (WEIGHTED && UB0 > 1 && !WIDE_U) ? UB0 / 2 : UB0;
  constexpr int U = UB < G ? UB : G;
  const bool read_self = keep != 0.f;
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    const int32_t row = it.x, beg = it.y, len = it.z, slot = it.w;
    const bool is_row = (row >= 0) && (slot < 0);

    uint4 sv[VPL];
#pragma unroll
    for (int j = 0; j < VPL; ++j) sv[j] = zero4;
    if (is_row && read_self) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < dv) sv[j] = self_in[(size_t)row * dv + col];
      }
    }
    float acc[VPL][N];
#pragma unroll
    for (int j = 0; j < VPL; ++j)
#pragma unroll
      for (int e = 0; e < N; ++e) acc[j][e] = 0.f;

    const int32_t maxlen = __reduce_max_sync(kFull, len);
    for (int32_t off = 0; off < maxlen; off += G) {
      const int32_t mine = len - off;
      const bool have = lg < mine;
      const int32_t my_idx =
          have ? ((PRE && off == 0) ? idx0 : __ldg(idx + beg + off + lg)) : 0;
      float my_w = 0.f;
      if (WEIGHTED) my_w = have ? ((PRE && off == 0) ? w0 : __ldg(inc_w + beg + off + lg)) : 0.f;
      const int32_t cnt = min(G, maxlen - off);
      for (int32_t t = 0; t < cnt; t += U) {
        uint4 x[U][VPL];
        float wt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int sl = (t + u) & (G - 1);
          // every lane takes part in both shuffles (a shuffle skipped by some
          // lanes of its mask is undefined and can hang the warp)
          const int32_t nb = __shfl_sync(kFull, my_idx, sl, G);
          const bool ok = (t + u) < mine;
          if (WEIGHTED) {
            const float w_sl = __shfl_sync(kFull, my_w, sl, G);
            wt[u] = ok ? w_sl : 0.f;
          } else {
            wt[u] = 1.f;
          }
          const uint4* rowp = src + (size_t)nb * dv;
#pragma unroll
          for (int j = 0; j < VPL; ++j) {
            const int col = lg + j * G;
            x[u][j] = (ok && col < dv) ? __ldg(rowp + col) : zero4;
          }
        }
        // invalid slots loaded zeros (and weight 0): adding them is exact
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
          for (int j = 0; j < VPL; ++j) {
            float xf[N];
            V::unpack(x[u][j], xf);
#pragma unroll
            for (int e = 0; e < N; ++e) {
              if (WEIGHTED)
                acc[j][e] = fmaf(wt[u], xf[e], acc[j][e]);
              else
                acc[j][e] += xf[e];
            }
          }
        }
      }
    }

    if (is_row) {
      const float sc = inv_norm ? scale * inv_norm[row] : scale;
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < dv) {
          float sf[N], r[N];
          V::unpack(sv[j], sf);
#pragma unroll
          for (int e = 0; e < N; ++e) r[e] = fmaf(keep, sf[e], sc * acc[j][e]);
          out[(size_t)row * dv + col] = V::pack(r);
        }
      }
    } else if (slot >= 0) {
#pragma unroll
      for (int j = 0; j < VPL; ++j) {
        const int col = lg + j * G;
        if (col < dv) {
          float4* pp = reinterpret_cast<float4*>(partials + ((size_t)slot * dv + col) * N);
#pragma unroll
          for (int q = 0; q < N / 4; ++q)
            pp[q] = make_float4(acc[j][4 * q], acc[j][4 * q + 1], acc[j][4 * q + 2],
                                acc[j][4 * q + 3]);
        }
      }
    }
}

// Split-row reduction: a row's chunk partials are summed in chunk order
// (four interleaved accumulators), then relaxed like a row item
// (out = keep * own row + scale * normaliser * sum).

__device__ __forceinline__ void f4_add(float4& a, const float4& b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

// Sum of count float4 values p[0], p[stride], p[2*stride], ... in a fixed
// order: ACC interleaved accumulators (value c goes to accumulator c mod ACC
// while ACC remain), the tail into the first, then a fixed tree.
template <int ACC = 4>
__device__ __forceinline__ float4 sum_strided4(const float4* __restrict__ p, int32_t count,
                                               int32_t stride) {
  float4 a[ACC];
#pragma unroll
  for (int q = 0; q < ACC; ++q) a[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  int32_t c = 0;
  for (; c + ACC <= count; c += ACC) {
    float4 v[ACC];
#pragma unroll
    for (int q = 0; q < ACC; ++q) v[q] = p[(size_t)(c + q) * stride];
#pragma unroll
    for (int q = 0; q < ACC; ++q) f4_add(a[q], v[q]);
  }
  for (; c < count; ++c) f4_add(a[0], p[(size_t)c * stride]);
#pragma unroll
  for (int w = 1; w < ACC; w *= 2)
#pragma unroll
    for (int q = 0; q + w < ACC; q += 2 * w) f4_add(a[q], a[q + w]);
  return a[0];
}

// Sum over `count` chunks of one row vector's N partial floats.
template <int N, int ACC = 4>
__device__ __forceinline__ void sum_chunks(const float* __restrict__ partials, int32_t first,
                                           int32_t count, int32_t dv, int32_t col, float* out) {
  const float4* base = reinterpret_cast<const float4*>(partials) + ((size_t)first * dv + col) * (N / 4);
#pragma unroll
  for (int q = 0; q < N / 4; ++q) {
    const float4 t = sum_strided4<ACC>(base + q, count, dv * (N / 4));
    out[4 * q] = t.x;
    out[4 * q + 1] = t.y;
    out[4 * q + 2] = t.z;
    out[4 * q + 3] = t.w;
  }
}


// Split row with at most kMidChunks chunks: one warp, lanes over row vectors.
template <typename T>
__device__ __forceinline__ void finalize_mid(int4 ds, int lane, const float* __restrict__ partials,
                                             const float* __restrict__ inv_norm,
                                             const uint4* self_in, uint4* out, int32_t dv,
                                             float keep, float scale) {
  using V = VecT<T>;
  constexpr int N = V::N;
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const float sc = inv_norm ? scale * inv_norm[ds.x] : scale;
  for (int col = lane; col < dv; col += 32) {
    float tot[N], sf[N], r[N];
    sum_chunks<N>(partials, ds.y, ds.z, dv, col, tot);
    const size_t o = (size_t)ds.x * dv + col;
    V::unpack(keep != 0.f ? self_in[o] : zero4, sf);
#pragma unroll
    for (int e = 0; e < N; ++e) r[e] = fmaf(keep, sf[e], sc * tot[e]);
    out[o] = V::pack(r);
  }
}

// Split row with more chunks: the whole block; S = blockDim / dv slices sum
// contiguous runs of chunks, slice 0 adds the slices in order. `sm` holds
// S * dv * N floats. One block reduces such a row alone (a hub node at the
// 1M-node workload's level 4 has 6,300 chunks), so each thread keeps eight
// loads in flight (ACC = 8): the coarse levels' node half-sweeps got 3-17 us
// faster than with four, the V-cycle 86.9 -> 86.2 ms.
template <typename T, int ACC = 8>
__device__ __forceinline__ void finalize_huge(int4 ds, float* sm, const float* __restrict__ partials,
                                              const float* __restrict__ inv_norm,
                                              const uint4* self_in, uint4* out, int32_t dv,
                                              float keep, float scale) {
  using V = VecT<T>;
  constexpr int N = V::N;
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const int S = (int)blockDim.x / dv;
  const int t = threadIdx.x;
  const int slice = t / dv;
  const int col = t - slice * dv;
  if (slice < S) {
    const int32_t a = (int32_t)((int64_t)ds.z * slice / S);
    const int32_t b = (int32_t)((int64_t)ds.z * (slice + 1) / S);
    float part[N];
    sum_chunks<N, ACC>(partials, ds.y + a, b - a, dv, col, part);
#pragma unroll
    for (int e = 0; e < N; ++e) sm[((size_t)slice * dv + col) * N + e] = part[e];
  }
  __syncthreads();
  if (slice == 0) {
    float tot[N], sf[N], r[N];
#pragma unroll
    for (int e = 0; e < N; ++e) tot[e] = sm[(size_t)col * N + e];
    for (int q = 1; q < S; ++q)
#pragma unroll
      for (int e = 0; e < N; ++e) tot[e] += sm[((size_t)q * dv + col) * N + e];
    const size_t o = (size_t)ds.x * dv + col;
    V::unpack(keep != 0.f ? self_in[o] : zero4, sf);
    const float sc = inv_norm ? scale * inv_norm[ds.x] : scale;
#pragma unroll
    for (int e = 0; e < N; ++e) r[e] = fmaf(keep, sf[e], sc * tot[e]);
    out[o] = V::pack(r);
  }
}

}  // namespace dev
}  // namespace hnv
