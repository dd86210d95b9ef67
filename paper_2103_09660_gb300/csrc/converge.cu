// The stopping rule of Section 4's experiments (stop once two consecutive
// iterates differ by at most eps): refinement one sweep at a time, with the
// largest change of any coordinate read back after each sweep.
#include <cuda_bf16.h>

#include <cstring>

#include "refine_device.cuh"

namespace hnv {

using dev::VecT;

namespace {

// out = max(out, max_i |a_i - b_i|) over `count` 16-byte vectors of T rows.
// The bit patterns of non-negative floats order like the floats, so the
// running maximum is an unsigned atomicMax (exact and order-independent).
template <typename T>
__global__ void max_abs_diff_kernel(int64_t count, const uint4* __restrict__ a,
                                    const uint4* __restrict__ b, unsigned* __restrict__ out) {
  using V = VecT<T>;
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float fa[V::N], fb[V::N];
    V::unpack(a[i], fa);
    V::unpack(b[i], fb);
#pragma unroll
    for (int e = 0; e < V::N; ++e) mx = fmaxf(mx, fabsf(fa[e] - fb[e]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(out, __float_as_uint(mx));
}

}  // namespace

int refine_level_until(hnv_graph* g, int level, void* z_v, void* z_e, int dtype, int d,
                       float omega, int max_sweeps, float eps, int mode, int32_t* sweeps_done,
                       float* last_delta, cudaStream_t s) {
  const Level& lv = g->levels[level];
  const size_t rb = (dtype == HNV_BF16 ? 2 : 4) * (size_t)d;
  const int64_t vec_v = (int64_t)lv.n * (int64_t)(rb / 16), vec_e = (int64_t)lv.m * (int64_t)(rb / 16);
  TempPool pool(s);
  uint8_t *pv = nullptr, *pe = nullptr;
  HNV_CHECK(pool.get(&pv, (size_t)lv.n * rb));
  HNV_CHECK(pool.get(&pe, (size_t)lv.m * rb));
  unsigned* dmax = reinterpret_cast<unsigned*>(g->d_buf + 32);
  int32_t done = 0;
  float delta = 0.f;
  for (int it = 0; it < max_sweeps; ++it) {
    if (lv.n) HNV_CUDA(cudaMemcpyAsync(pv, z_v, (size_t)lv.n * rb, cudaMemcpyDeviceToDevice, s));
    if (lv.m) HNV_CUDA(cudaMemcpyAsync(pe, z_e, (size_t)lv.m * rb, cudaMemcpyDeviceToDevice, s));
    HNV_CHECK(refine_level(g, level, z_v, z_e, dtype, d, omega, 1, mode, s));
    HNV_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned), s));
    auto kern = dtype == HNV_BF16 ? max_abs_diff_kernel<__nv_bfloat16> : max_abs_diff_kernel<float>;
    HNV_CHECK(launch("max_abs_diff", kern, grid_for(vec_v, 256), 256, 0, s, vec_v,
                     (const uint4*)z_v, (const uint4*)pv, dmax));
    HNV_CHECK(launch("max_abs_diff", kern, grid_for(vec_e, 256), 256, 0, s, vec_e,
                     (const uint4*)z_e, (const uint4*)pe, dmax));
    int32_t bits = 0;
    HNV_CHECK(read_ints(g, reinterpret_cast<const int32_t*>(dmax), 1, &bits, s));
    std::memcpy(&delta, &bits, sizeof(float));
    done = it + 1;
    if (delta <= eps) break;
  }
  *sweeps_done = done;
  *last_delta = delta;
  return HNV_OK;
}

}  // namespace hnv
