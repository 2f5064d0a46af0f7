// FP64 throughput probe (mgcccs_fp64_probe): a measurement utility, with no counterpart in
// the paper.  The complex128 kernels of the solve are bound by the FP64 pipe, whose rate on
// this part (2 lanes per clock per SM) is far below its memory bandwidth; this kernel runs
// nothing but independent FP64 fused multiply-adds, so the caller can time the pipe's
// attainable rate beside its nominal one and compare the solve's kernels with both.
#include "common.cuh"

namespace {

constexpr int kProbeThreads = 256;

// Each thread advances MGCCCS_PROBE_CHAINS independent recurrences a <- a m + b for
// `iters` rounds (m, b are arguments, so the compiler cannot fold them), then the block
// sums its threads' values into out[blockIdx.x], which keeps every operation live.
__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int iters, double m, double b,
                                                              double* __restrict__ out) {
  __shared__ double sh[kProbeThreads / 32];
  double a[MGCCCS_PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < MGCCCS_PROBE_CHAINS; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + 7 * c);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < MGCCCS_PROBE_CHAINS; ++c) a[c] = fma(a[c], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < MGCCCS_PROBE_CHAINS; ++c) s += a[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kProbeThreads / 32; ++w) tot += sh[w];
    out[blockIdx.x] = tot;
  }
}

}  // namespace

extern "C" int mgcccs_fp64_probe(int blocks, int iters, double m, double b, double* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out) return MGCCCS_EINVAL;
  k_fp64_probe<<<blocks, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(iters, m, b, out);
  return cudaGetLastError() == cudaSuccess ? MGCCCS_OK : MGCCCS_ECUDA;
}
