// gen.cu -- device twin of the seeded input generators of
// paper_2602_05179_gb300/workloads/__init__.py (SplitMix64 in counter mode).
// Inputs only: none of the Split / reinsertion arithmetic is here.  Every
// value is an integer function of (seed, stream, index), so the device arrays
// equal the numpy ones bit for bit (checked by the GPU tests).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

uint64_t stream_base(uint64_t seed, uint64_t stream) {
  return mix64(mix64(seed + kG) + stream * kG);
}

__global__ void uniform_int_kernel(uint64_t base, int64_t k0, int64_t count, int32_t lo,
                                   uint64_t span, int32_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = mix64(base + (uint64_t)(k0 + k + 1) * kG);
    out[k] = lo + (int32_t)(u % span);
  }
}

__global__ void poisson_clip_kernel(uint64_t base, int64_t k0, int64_t count,
                                    const double* __restrict__ cdf, int ncdf, int32_t lo,
                                    int32_t hi, int32_t* out) {
  __shared__ double tab[256];
  for (int j = threadIdx.x; j < ncdf; j += blockDim.x) tab[j] = cdf[j];
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = mix64(base + (uint64_t)(k0 + k + 1) * kG);
    const double x = (double)(u >> 11) * 0x1.0p-53;
    int a = 0, b = ncdf;  // number of table entries <= x
    while (a < b) {
      const int m = (a + b) >> 1;
      if (tab[m] <= x) a = m + 1; else b = m;
    }
    out[k] = a < lo ? lo : (a > hi ? hi : a);
  }
}

int grid_for(int64_t count) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (count + 255) / 256;
  int64_t cap = (int64_t)sms * 8;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

extern "C" {

// out[k] = lo + u(seed, stream, k0+k) mod (hi-lo+1), k < count (device out)
int sdpgen_uniform_int(uint64_t seed, uint64_t stream, int64_t k0, int64_t count, int32_t lo,
                       int32_t hi, int32_t* out, void* cuda_stream) {
  if (count <= 0) return 0;
  if (hi < lo || !out) return -1;
  uniform_int_kernel<<<grid_for(count), 256, 0, (cudaStream_t)cuda_stream>>>(
      stream_base(seed, stream), k0, count, lo, (uint64_t)((int64_t)hi - lo + 1), out);
  return (int)cudaGetLastError();
}

// Poisson inversion with the FP64 CDF table cdf[0..ncdf) (device), clipped
int sdpgen_poisson_clip(uint64_t seed, uint64_t stream, int64_t k0, int64_t count,
                        const double* cdf, int ncdf, int32_t lo, int32_t hi, int32_t* out,
                        void* cuda_stream) {
  if (count <= 0) return 0;
  if (!cdf || ncdf < 1 || ncdf > 256 || !out) return -1;
  poisson_clip_kernel<<<grid_for(count), 256, 0, (cudaStream_t)cuda_stream>>>(
      stream_base(seed, stream), k0, count, cdf, ncdf, lo, hi, out);
  return (int)cudaGetLastError();
}

}  // extern "C"
