// alto_fill_uniform: seeded uniform [0, 1) floats on the device, for initial
// CP-ALS factors drawn where the run executes (the paper leaves the
// initialisation to the caller). Counter-based: element i of a fill with
// seed s is the top 24 bits of SplitMix64 (Steele, Lea and Flood, 2014)
// applied to s * 2^32 + i, times 2^-24, so any element can be recomputed on
// its own, on the host or the device.
#include "handle.cuh"

namespace alto {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) fill_uniform_kernel(float *__restrict__ dst, uint64_t n,
                                                           uint64_t base) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    dst[i] = (float)(splitmix64(base + i) >> 40) * (1.0f / 16777216.0f);
}

}  // namespace alto

using namespace alto;

extern "C" alto_status alto_fill_uniform(float *dst, uint64_t n, uint64_t seed, void *stream) {
  if (n == 0) return ALTO_OK;
  if (!dst) return fail(ALTO_ERR_INVALID_ARG, "dst is NULL");
  if (seed >= (1ull << 32)) return fail(ALTO_ERR_INVALID_ARG, "seed must be < 2^32");
  if (n > (1ull << 32)) return fail(ALTO_ERR_INVALID_ARG, "n must be <= 2^32");
  int dev = 0, sms = 1;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  uint64_t grid = (n + 255) / 256;
  if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
  fill_uniform_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(dst, n, seed << 32);
  note_launches(1);
  CUDA_TRY(cudaGetLastError());
  return ALTO_OK;
}
