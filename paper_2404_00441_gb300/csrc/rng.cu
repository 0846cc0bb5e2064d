// rng.cu -- the library's random-number generator exposed on its own:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
// generator behind every draw of the method (the random first pattern and the
// draw among the K best of Algorithm 1, the path mirroring of line 3). The
// host and device forms below compile the same function the kernels call
// (philox4x32_10 in ccw_internal.cuh).
#include <cstring>

#include "ccw_internal.cuh"

namespace ccw {

__global__ void k_philox(int64_t n, const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 c = reinterpret_cast<const uint4*>(ctr)[i];
    const U32x4 r = philox4x32_10(c.x, c.y, c.z, c.w, k0, k1);
    reinterpret_cast<uint4*>(out)[i] = make_uint4(r.v[0], r.v[1], r.v[2], r.v[3]);
  }
}

}  // namespace ccw

extern "C" {

int ccw_philox_host(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return CCW_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    const ccw::U32x4 r = ccw::philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2],
                                            ctr[4 * i + 3], key[0], key[1]);
    std::memcpy(out + 4 * i, r.v, sizeof(r.v));
  }
  return CCW_OK;
}

int ccw_philox_dev(int64_t n, const uint32_t* ctr_dev, const uint32_t key[2], uint32_t* out_dev,
                   void* stream) {
  if (n < 0 || (n > 0 && (!ctr_dev || !key || !out_dev))) return CCW_EINVAL;
  if (n == 0) return CCW_OK;
  if ((reinterpret_cast<uintptr_t>(ctr_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15)
    return CCW_EINVAL;   // read and written as 16-byte words
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  const int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
  ccw::k_philox<<<grid, threads, 0, (cudaStream_t)stream>>>(n, ctr_dev, key[0], key[1], out_dev);
  return cudaGetLastError() == cudaSuccess ? CCW_OK : CCW_ECUDA;
}

}  // extern "C"
