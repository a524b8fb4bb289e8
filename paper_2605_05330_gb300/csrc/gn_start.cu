// gn_start.cu -- the random simplex start of the appendix module (gn_random_start):
//   p = -log u (exponential draws), p <- p / max(p) over every start, x0 = clamp(p, 1e-3, 1).
// The uniform numbers u are an input (the caller's generator), so the CPU reference and this
// kernel see the same draws.
#include <cmath>

#include "gn_internal.cuh"

namespace gn {

__global__ void k_neglog_max(int64_t m, const float* __restrict__ u, float* __restrict__ p,
                             unsigned* __restrict__ maxbits, int* __restrict__ bad) {
  float best = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float ui = u[i];
    if (!(ui > 0.0f && ui <= 1.0f)) atomicOr(bad, 1);
    const float pi = -logf(ui);
    p[i] = pi;
    best = fmaxf(best, pi);
  }
  best = dev::warp_max(best);
  // non-negative floats order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(best));
}

__global__ void k_scale_clamp(int64_t m, float* __restrict__ p, const unsigned* __restrict__ maxbits) {
  const float mx = __uint_as_float(*maxbits);
  const float inv = mx > 0.0f ? 1.0f / mx : 1.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fminf(fmaxf(p[i] * inv, 1e-3f), 1.0f);
}

}  // namespace gn

extern "C" gn_status gn_random_start(int64_t m, const float* u, float* x0, void* stream_v) {
  using namespace gn;
  if (m < 0 || (m > 0 && (!u || !x0))) return fail(GN_ERR_ARG, "gn_random_start: bad argument");
  if (m == 0) return GN_OK;
  cudaStream_t stream = (cudaStream_t)stream_v;
  unsigned* scratch = nullptr;  // [0] max bits, [1] bad flag
  GN_CUDA(cudaMallocAsync((void**)&scratch, 2 * sizeof(unsigned), stream));
  GN_CUDA(cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned), stream));
  const unsigned grid = (unsigned)std::min<int64_t>(4096, (m + 255) / 256);
  k_neglog_max<<<grid, 256, 0, stream>>>(m, u, x0, scratch, (int*)(scratch + 1));
  GN_LAUNCHED();
  k_scale_clamp<<<grid, 256, 0, stream>>>(m, x0, scratch);
  GN_LAUNCHED();
  unsigned bad = 0;
  GN_CUDA(cudaMemcpyAsync(&bad, scratch + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
  GN_CUDA(cudaFreeAsync(scratch, stream));
  GN_CUDA(cudaStreamSynchronize(stream));
  if (bad) return fail(GN_ERR_ARG, "gn_random_start: a uniform draw is outside (0, 1]");
  return GN_OK;
}
