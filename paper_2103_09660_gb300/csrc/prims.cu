// Integer primitives for the coarsening path: exclusive scan, a stable LSD
// radix sort of 64-bit keys and the CSR transpose built on it. All integer,
// all deterministic (atomics only count into integer histograms).
#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (three kernels per level of recursion)
// ---------------------------------------------------------------------------

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Exclusive scan of one value per thread over a 256-thread block. Returns the
// exclusive prefix; *block_total receives the block's sum.
__device__ int32_t block_exclusive_scan(int32_t v, int32_t* block_total) {
  __shared__ int32_t warp_part[SCAN_THREADS / 32];
  __shared__ int32_t total_s;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_part[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < SCAN_THREADS / 32 ? warp_part[lane] : 0;
    int32_t t = s;
#pragma unroll
    for (int o = 1; o < SCAN_THREADS / 32; o <<= 1) {
      int32_t y = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t += y;
    }
    if (lane < SCAN_THREADS / 32) warp_part[lane] = t - s;
    if (lane == SCAN_THREADS / 32 - 1) total_s = t;
  }
  __syncthreads();
  int32_t r = x - v + warp_part[w];
  *block_total = total_s;
  __syncthreads();  // warp_part / total_s may be reused by the next call
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_tiles(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j)
    if (base + j < n) s += in[base + j];
  int32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// in == out allowed: each thread reads its items before writing them.
__global__ void __launch_bounds__(SCAN_THREADS)
scan_tiles(const int32_t* in, int32_t* out, int64_t n, const int32_t* __restrict__ tile_off,
           int32_t* __restrict__ total) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int32_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    v[j] = (base + j < n) ? in[base + j] : 0;
    s += v[j];
  }
  int32_t tot;
  int32_t run = block_exclusive_scan(s, &tot);
  if (tile_off) run += tile_off[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (total && threadIdx.x == 0) *total = tot;
}

// ---------------------------------------------------------------------------
// Radix sort (stable LSD, 8-bit digits, 4096-key tiles)
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;                     // keys per thread
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // 4096

__global__ void __launch_bounds__(RS_THREADS)
rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
        int32_t ntiles) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int j = 0; j < RS_ITEMS; ++j) {
    int64_t k = base + j * RS_THREADS + threadIdx.x;
    if (k < n) atomicAdd(&cnt[(unsigned)(keys[k] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Each warp ranks a contiguous run of 512 keys in order, so the tile's order
// (warp, round, lane) is the input order and the scatter is stable. The tile
// is first reordered by digit in shared memory, so that the global writes go
// out as runs of consecutive addresses (one run per digit) instead of one
// scattered 8-byte store per key.
__global__ void __launch_bounds__(RS_THREADS)
rs_scatter(const uint64_t* __restrict__ keys, uint64_t* __restrict__ out, int64_t n, int shift,
           const int32_t* __restrict__ hist_scanned, int32_t ntiles) {
  __shared__ int32_t wcnt[RS_WARPS][256];
  __shared__ int32_t toff[256];    // first output position of digit d for this tile
  __shared__ int32_t tstart[256];  // first tile position of digit d
  __shared__ int32_t wsum[RS_WARPS];
  __shared__ uint64_t stage[RS_TILE];
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  toff[threadIdx.x] = hist_scanned[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t base = tile0 + (int64_t)w * (32 * RS_ITEMS);
  uint64_t kv[RS_ITEMS];
  int32_t loc[RS_ITEMS];
  int32_t dg[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t k = base + j * 32 + lane;
    const bool valid = k < n;
    const uint64_t key = valid ? keys[k] : 0ull;
    const int d = valid ? (int)((unsigned)(key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(FULL, d);
    const int rank = __popc(peers & lt);
    const int32_t b = valid ? wcnt[w][d] : 0;
    __syncwarp();
    if (valid && rank == 0) wcnt[w][d] = b + __popc(peers);
    __syncwarp();
    kv[j] = key;
    loc[j] = b + rank;
    dg[j] = d;
  }
  __syncthreads();
  // per digit (thread t = digit): warps' exclusive offsets, then the digit's
  // tile start as an exclusive scan over digits (warp scans, then warp sums)
  int32_t run = 0;
#pragma unroll
  for (int q = 0; q < RS_WARPS; ++q) {
    const int32_t c = wcnt[q][threadIdx.x];
    wcnt[q][threadIdx.x] = run;
    run += c;
  }
  int32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int32_t before = 0;
  for (int q = 0; q < w; ++q) before += wsum[q];
  tstart[threadIdx.x] = before + inc - run;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j)
    if (dg[j] < 256) stage[tstart[dg[j]] + wcnt[w][dg[j]] + loc[j]] = kv[j];
  __syncthreads();
  const int32_t count = (int32_t)(n - tile0 < RS_TILE ? n - tile0 : RS_TILE);
  for (int32_t i = threadIdx.x; i < count; i += RS_THREADS) {
    const uint64_t key = stage[i];
    const int d = (int)((unsigned)(key >> shift) & 255u);
    out[toff[d] + (i - tstart[d])] = key;
  }
}

// ---------------------------------------------------------------------------
// Misc
// ---------------------------------------------------------------------------

__global__ void fill_i32_kernel(int32_t* p, int32_t v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// key = (col << 32) | row for every CSR entry.
__global__ void pack_col_row(int32_t n_rows, const int32_t* __restrict__ row_ptr,
                             const int32_t* __restrict__ cols, uint64_t* __restrict__ keys) {
  csr_rows_warp_visit(n_rows, row_ptr, [&](int64_t r, int64_t k) {
    keys[k] = ((uint64_t)(uint32_t)cols[k] << 32) | (uint32_t)r;
  });
}

// col_ptr of keys sorted by their high word (the column): position i starts
// every column in (col(i-1), col(i)], with col(-1) = -1 and col(n) = n_cols,
// so col_ptr[c] = first position whose column is >= c. No atomics: each
// entry of col_ptr[0..n_cols] is written by exactly one position.
__global__ void col_starts(const uint64_t* __restrict__ keys, int64_t n, int32_t n_cols,
                           int32_t* __restrict__ col_ptr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t prev = i > 0 ? (int64_t)(uint32_t)(keys[i - 1] >> 32) : -1;
    const int64_t cur = i < n ? (int64_t)(uint32_t)(keys[i] >> 32) : (int64_t)n_cols;
    for (int64_t c = prev + 1; c <= cur; ++c) col_ptr[c] = (int32_t)i;
  }
}

__global__ void low_words(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)(uint32_t)keys[i];
}

// Segmented sort by the low 32 bits of 64-bit keys whose high words are the
// segment index. Segments of at most 256 keys: a warp each, a bitonic
// network over 32 lanes x K registers (element i = register i / 32, lane
// i % 32). Up to kSegSortMax: a block each, a bitonic network in shared
// memory.
constexpr int kSegThreads = 512;

template <int K>
__device__ __forceinline__ void warp_bitonic(uint32_t (&x)[K], int lane) {
  constexpr int N = 32 * K;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const int rr = r ^ (j >> 5);
          if (rr > r) {
            const bool ascending = ((r * 32 + lane) & k) == 0;
            const uint32_t a = x[r], b = x[rr];
            const bool swap = (a > b) == ascending;
            x[r] = swap ? b : a;
            x[rr] = swap ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < K; ++r) {
          const uint32_t o = __shfl_xor_sync(FULL, x[r], j);
          const bool ascending = ((r * 32 + lane) & k) == 0;
          const bool lower = (lane & j) == 0;
          x[r] = (lower == ascending) ? min(x[r], o) : max(x[r], o);
        }
      }
    }
  }
}

template <int K>
__device__ __forceinline__ void warp_sort_segment(uint64_t* keys, int64_t b, int32_t len,
                                                  uint32_t e, int lane) {
  uint32_t x[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const int i = r * 32 + lane;
    x[r] = i < len ? (uint32_t)keys[b + i] : 0xffffffffu;
  }
  warp_bitonic<K>(x, lane);
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const int i = r * 32 + lane;
    if (i < len) keys[b + i] = ((uint64_t)e << 32) | x[r];
  }
}

// A lane sorts a segment of 2..8 keys by itself: Knuth's 19-comparator
// network for 8 inputs over the low words, padded with 0xffffffff.
__device__ __forceinline__ void lane_sort8(uint64_t* keys, int64_t b, int32_t len, uint32_t e) {
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = i < len ? (uint32_t)keys[b + i] : 0xffffffffu;
#define HNV_CE(i, j)                       \
  {                                        \
    const uint32_t lo = min(x[i], x[j]);   \
    x[j] = max(x[i], x[j]);                \
    x[i] = lo;                             \
  }
  HNV_CE(0, 2) HNV_CE(1, 3) HNV_CE(4, 6) HNV_CE(5, 7)
  HNV_CE(0, 4) HNV_CE(1, 5) HNV_CE(2, 6) HNV_CE(3, 7)
  HNV_CE(0, 1) HNV_CE(2, 3) HNV_CE(4, 5) HNV_CE(6, 7)
  HNV_CE(2, 4) HNV_CE(3, 5)
  HNV_CE(1, 4) HNV_CE(3, 6)
  HNV_CE(1, 2) HNV_CE(3, 4) HNV_CE(5, 6)
#undef HNV_CE
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (i < len) keys[b + i] = ((uint64_t)e << 32) | x[i];
}

// A warp takes 32 consecutive segments: each lane sorts its own if it has
// 2..8 keys; the warp then sorts the ones of 9..256 keys together, one after
// another; longer ones are appended to `long_segs` for the block kernels.
template <typename P>
__global__ void seg_sort_warp(int32_t m, const P* __restrict__ e_ptr,
                              uint64_t* __restrict__ keys, int32_t* __restrict__ long_segs,
                              int32_t* __restrict__ n_long) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; e0 < m;
       e0 += warps * 32) {
    const int64_t e = e0 + lane;
    int64_t b = 0;
    int32_t len = 0;
    if (e < m) {
      b = e_ptr[e];
      len = (int32_t)(e_ptr[e + 1] - b);
    }
    if (len >= 2 && len <= 8) lane_sort8(keys, b, len, (uint32_t)e);
    if (len > 256) long_segs[atomicAdd(n_long, 1)] = (int32_t)e;
    unsigned mid = __ballot_sync(FULL, len > 8 && len <= 256);
    while (mid) {
      const int src = __ffs(mid) - 1;
      mid &= mid - 1u;
      const int64_t sb = __shfl_sync(FULL, b, src);
      const int32_t sl = __shfl_sync(FULL, len, src);
      const uint32_t se = (uint32_t)(e0 + src);
      if (sl <= 32) warp_sort_segment<1>(keys, sb, sl, se, lane);
      else if (sl <= 64) warp_sort_segment<2>(keys, sb, sl, se, lane);
      else if (sl <= 128) warp_sort_segment<4>(keys, sb, sl, se, lane);
      else warp_sort_segment<8>(keys, sb, sl, se, lane);
    }
  }
}

// The listed segments (257 .. kSegSortMax keys), one block each.
template <typename P>
__global__ void __launch_bounds__(kSegThreads)
seg_sort_block(const int32_t* __restrict__ long_segs, const int32_t* __restrict__ n_long,
               const P* __restrict__ e_ptr, uint64_t* __restrict__ keys) {
  __shared__ uint32_t sk[kSegSortMax];
  const int32_t count = *n_long;
  for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int32_t e = long_segs[q];
    const int64_t b = e_ptr[e];
    const int32_t len = (int32_t)(e_ptr[e + 1] - b);
    if (len > kSegSortMax) continue;         // block-uniform (the caller rules it out)
    int32_t n2 = 512;
    while (n2 < len) n2 <<= 1;
    for (int32_t i = threadIdx.x; i < n2; i += kSegThreads)
      sk[i] = i < len ? (uint32_t)keys[b + i] : 0xffffffffu;
    __syncthreads();
    for (int32_t k = 2; k <= n2; k <<= 1) {
      for (int32_t j = k >> 1; j > 0; j >>= 1) {
        // pair t: positions i = (t / j) * 2j + t % j and i + j
        for (int32_t t = threadIdx.x; t < (n2 >> 1); t += kSegThreads) {
          const int32_t i = (t / j) * (2 * j) + (t % j);
          const int32_t p = i + j;
          const uint32_t a = sk[i], c = sk[p];
          const bool ascending = (i & k) == 0;
          if ((a > c) == ascending) {
            sk[i] = c;
            sk[p] = a;
          }
        }
        __syncthreads();
      }
    }
    for (int32_t i = threadIdx.x; i < len; i += kSegThreads)
      keys[b + i] = ((uint64_t)(uint32_t)e << 32) | sk[i];
    __syncthreads();
  }
}

// The listed segments (more than 256 keys) when only their sorted distinct
// low words matter and those lie in [0, range): one block each marks the
// values in a shared-memory bitmap (bm, one bit per value), then writes the
// set bits in ascending order and fills the rest of the segment with copies
// of its largest value: linear in the segment and the bitmap, where the
// bitonic network of seg_sort_block is O(len log^2 len) with a barrier a
// step. TWO_LEVEL (large ranges): a summary bitmap (sm, one bit per word of
// bm) lets the scan skip empty words, and only the words a segment touched
// are cleared after it, so the work per segment is linear in its length plus
// range / 1024; otherwise every thread scans and clears its share of bm.
template <typename P, bool TWO_LEVEL>
__global__ void __launch_bounds__(kSegThreads)
seg_dedup_bitmap(const int32_t* __restrict__ long_segs, const int32_t* __restrict__ n_long,
                 const P* __restrict__ e_ptr, uint64_t* __restrict__ keys, int32_t words) {
  extern __shared__ uint32_t bm[];
  __shared__ int32_t wsum[kSegThreads / 32];
  __shared__ uint32_t vmax;
  const int32_t swords = TWO_LEVEL ? (words + 31) / 32 : 0;
  uint32_t* sm = bm + words;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  // thread t owns scan words [t * per, min(nscan, (t + 1) * per)) of sm
  // (TWO_LEVEL) or of bm
  const int32_t nscan = TWO_LEVEL ? swords : words;
  const int32_t per = (nscan + kSegThreads - 1) / kSegThreads;
  const int32_t s0 = min(nscan, (int32_t)threadIdx.x * per);
  const int32_t s1 = min(nscan, s0 + per);
  for (int32_t i = threadIdx.x; i < words + swords; i += kSegThreads) bm[i] = 0u;
  const int32_t count = *n_long;
  for (int32_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int32_t e = long_segs[q];
    const int64_t b = e_ptr[e];
    const int32_t len = (int32_t)(e_ptr[e + 1] - b);
    if (threadIdx.x == 0) vmax = 0u;
    __syncthreads();
    for (int32_t i = threadIdx.x; i < len; i += kSegThreads) {
      const uint32_t v = (uint32_t)keys[b + i];
      atomicOr(&bm[v >> 5], 1u << (v & 31));
      if (TWO_LEVEL) atomicOr(&sm[v >> 10], 1u << ((v >> 5) & 31));
      atomicMax(&vmax, v);
    }
    __syncthreads();
    int32_t c = 0;
    for (int32_t i = s0; i < s1; ++i) {
      if (TWO_LEVEL) {
        uint32_t sbits = sm[i];
        while (sbits) {
          const int t = __ffs(sbits) - 1;
          sbits &= sbits - 1u;
          c += __popc(bm[i * 32 + t]);
        }
      } else {
        c += __popc(bm[i]);
      }
    }
    int32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int32_t off = inc - c;
    for (int q2 = 0; q2 < w; ++q2) off += wsum[q2];
    int32_t distinct = 0;
    for (int q2 = 0; q2 < kSegThreads / 32; ++q2) distinct += wsum[q2];
    const uint64_t hi = (uint64_t)(uint32_t)e << 32;
    for (int32_t i = s0; i < s1; ++i) {
      uint32_t sbits = TWO_LEVEL ? sm[i] : 1u;
      while (sbits) {
        const int t = __ffs(sbits) - 1;
        sbits &= sbits - 1u;
        const int32_t wi = TWO_LEVEL ? i * 32 + t : i;
        uint32_t bits = bm[wi];
        while (bits) {
          const int u = __ffs(bits) - 1;
          bits &= bits - 1u;
          keys[b + off++] = hi | ((uint32_t)wi * 32u + (uint32_t)u);
        }
      }
    }
    for (int32_t i = distinct + threadIdx.x; i < len; i += kSegThreads) keys[b + i] = hi | vmax;
    __syncthreads();
    if (TWO_LEVEL) {
      // clear what this segment set (values are re-read from the first
      // `distinct` keys just written, all of them < range)
      for (int32_t i = threadIdx.x; i < distinct; i += kSegThreads) {
        const uint32_t v = (uint32_t)keys[b + i];
        bm[v >> 5] = 0u;
        sm[v >> 10] = 0u;
      }
    } else {
      for (int32_t i = s0; i < s1; ++i) bm[i] = 0u;
    }
    __syncthreads();
  }
}

template <typename P, bool TWO>
int launch_dedup(unsigned grid, size_t smem, cudaStream_t s, const int32_t* long_segs,
                 const int32_t* n_long, const P* ptr, uint64_t* keys, int32_t words) {
  HNV_CUDA(cudaFuncSetAttribute(seg_dedup_bitmap<P, TWO>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return launch("seg_dedup_bitmap", seg_dedup_bitmap<P, TWO>, grid, kSegThreads, smem, s,
                long_segs, n_long, ptr, keys, words);
}

}  // namespace

int segmented_sort_low32(int32_t segs, const int32_t* ptr32, const int64_t* ptr64,
                         int32_t max_len, int64_t total_keys, uint64_t* keys, cudaStream_t s,
                         uint32_t distinct_range) {
  if (max_len > kSegSortMax) HNV_FAIL(HNV_ERR_INVALID_ARG, "segment of %d keys", max_len);
  if (segs <= 0 || max_len < 2) return HNV_OK;
  TempPool pool(s);
  int32_t *long_segs = nullptr, *n_long = nullptr;
  HNV_CHECK(pool.get(&long_segs, (size_t)(total_keys / 257 + 1)));
  HNV_CHECK(pool.get(&n_long, 1));
  HNV_CUDA(cudaMemsetAsync(n_long, 0, sizeof(int32_t), s));
  const unsigned gw = grid_for((int64_t)segs, 256);  // a warp per 32 segments
  const unsigned gb = (unsigned)(4 * num_sms());
  const int32_t words = (int32_t)(((uint64_t)distinct_range + 31) / 32);
  const int32_t swords = (words + 31) / 32;
  const bool bitmap = distinct_range > 0 && (size_t)(words + swords) * 4 <= kSegBitmapBytes;
  if (ptr32)
    HNV_CHECK(launch("seg_sort_warp", seg_sort_warp<int32_t>, gw, 256, 0, s, segs, ptr32, keys,
                     long_segs, n_long));
  else
    HNV_CHECK(launch("seg_sort_warp", seg_sort_warp<int64_t>, gw, 256, 0, s, segs, ptr64, keys,
                     long_segs, n_long));
  if (max_len <= 256) return HNV_OK;
  if (bitmap) {
    // the summary pays off once a thread would scan more than 8 words
    const bool two = words > 8 * kSegThreads;
    const size_t smem = (size_t)(words + (two ? swords : 0)) * 4;
    const unsigned gd = (unsigned)(num_sms() * (smem <= 48 * 1024 ? 4 : 1));
    if (ptr32)
      return two ? launch_dedup<int32_t, true>(gd, smem, s, long_segs, n_long, ptr32, keys, words)
                 : launch_dedup<int32_t, false>(gd, smem, s, long_segs, n_long, ptr32, keys, words);
    return two ? launch_dedup<int64_t, true>(gd, smem, s, long_segs, n_long, ptr64, keys, words)
               : launch_dedup<int64_t, false>(gd, smem, s, long_segs, n_long, ptr64, keys, words);
  }
  if (ptr32)
    return launch("seg_sort_block", seg_sort_block<int32_t>, gb, kSegThreads, 0, s,
                  (const int32_t*)long_segs, (const int32_t*)n_long, ptr32, keys);
  return launch("seg_sort_block", seg_sort_block<int64_t>, gb, kSegThreads, 0, s,
                (const int32_t*)long_segs, (const int32_t*)n_long, ptr64, keys);
}

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                       cudaStream_t s) {
  if (n <= 0) {
    if (total) HNV_CUDA(cudaMemsetAsync(total, 0, sizeof(int32_t), s));
    return HNV_OK;
  }
  const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt == 1)
    return launch("scan_tiles", scan_tiles, 1, SCAN_THREADS, 0, s, in, out, n,
                  (const int32_t*)nullptr, total);
  TempPool pool(s);
  int32_t* sums = nullptr;
  HNV_CHECK(pool.get(&sums, (size_t)nt));
  HNV_CHECK(launch("scan_reduce_tiles", scan_reduce_tiles, (unsigned)nt, SCAN_THREADS, 0, s,
                   in, n, sums));
  HNV_CHECK(exclusive_scan_i32(sums, sums, nt, total, s));
  return launch("scan_tiles", scan_tiles, (unsigned)nt, SCAN_THREADS, 0, s, in, out, n,
                (const int32_t*)sums, (int32_t*)nullptr);
}

int bits_for_count(int64_t count) {
  int b = 0;
  while (b < 63 && (int64_t(1) << b) < count) ++b;
  return b;
}

int radix_shifts(int low_bits, int high_bits, int* shifts) {
  int k = 0;
  for (int b = 0; b < low_bits; b += 8) shifts[k++] = b;
  for (int b = 0; b < high_bits; b += 8) shifts[k++] = 32 + b;
  return k;
}

int radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, const int* shifts, int npasses,
                   cudaStream_t s, uint64_t** result) {
  *result = keys;
  if (n <= 1 || npasses == 0) return HNV_OK;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  if (ntiles * 256 >= (int64_t(1) << 31)) HNV_FAIL(HNV_ERR_TOO_LARGE, "radix sort too large");
  TempPool pool(s);
  int32_t* hist = nullptr;
  HNV_CHECK(pool.get(&hist, (size_t)(ntiles * 256)));
  uint64_t* src = keys;
  uint64_t* dst = alt;
  for (int p = 0; p < npasses; ++p) {
    HNV_CHECK(launch("rs_hist", rs_hist, (unsigned)ntiles, RS_THREADS, 0, s,
                     (const uint64_t*)src, n, shifts[p], hist, (int32_t)ntiles));
    HNV_CHECK(exclusive_scan_i32(hist, hist, ntiles * 256, nullptr, s));
    HNV_CHECK(launch("rs_scatter", rs_scatter, (unsigned)ntiles, RS_THREADS, 0, s,
                     (const uint64_t*)src, dst, n, shifts[p], (const int32_t*)hist,
                     (int32_t)ntiles));
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  *result = src;
  return HNV_OK;
}

int fill_i32(int32_t* p, int32_t value, int64_t n, cudaStream_t s) {
  if (n <= 0) return HNV_OK;
  return launch("fill_i32", fill_i32_kernel, grid_for(n, 256), 256, 0, s, p, value, n);
}

int transpose_csr(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* row_ptr,
                  const int32_t* cols, int32_t* col_ptr, int32_t* col_rows, cudaStream_t s) {
  if (nnz == 0) {
    HNV_CUDA(cudaMemsetAsync(col_ptr, 0, ((size_t)n_cols + 1) * sizeof(int32_t), s));
    return HNV_OK;
  }
  TempPool pool(s);
  uint64_t *k0 = nullptr, *k1 = nullptr, *sorted = nullptr;
  HNV_CHECK(pool.get(&k0, (size_t)nnz));
  HNV_CHECK(pool.get(&k1, (size_t)nnz));
  HNV_CHECK(launch("pack_col_row", pack_col_row, grid_for((int64_t)n_rows, 256), 256, 0, s,
                   n_rows, row_ptr, cols, k0));
  int shifts[16];
  int np = radix_shifts(0, bits_for_count(n_cols), shifts);
  HNV_CHECK(radix_sort_u64(k0, k1, nnz, shifts, np, s, &sorted));
  HNV_CHECK(launch("col_starts", col_starts, grid_for(nnz + 1, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz, n_cols, col_ptr));
  return launch("low_words", low_words, grid_for(nnz, 256), 256, 0, s, (const uint64_t*)sorted,
                nnz, col_rows);
}

}  // namespace hnv
