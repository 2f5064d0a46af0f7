// Allocation-free squared 2-norm of a device complex128 vector (mgcccs_norm2_noalloc).
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA graph is
// being captured in the global capture mode (where allocation calls are illegal),
// code inside a framework whose caching allocator owns all device memory under a hard
// cap, and latency-critical loops that must not hit the implicit device
// synchronisation an allocation can cause.  For them this file offers one entry point
// that needs no workspace: its scratch is a file-scope __device__ array that every GPU
// which loads the library keeps until the process exits.
//
// The paper has no counterpart; this is a service for monitoring convergence (||r||^2
// of a residual produced elsewhere).
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNaBlock = 256;                       // threads per block
constexpr int kNaPerThread = 8;                     // elements per thread
constexpr int kNaMaxBlocks = MGCCCS_NOALLOC_MAX_N / (kNaBlock * kNaPerThread);

// One partial sum per block; the last call's values stay here (fully overwritten by
// the next call, so nothing needs clearing).
static __device__ __align__(256) double g_noalloc_partials[kNaMaxBlocks];

__global__ void __launch_bounds__(kNaBlock) k_norm2_partials_static(const cplx* __restrict__ v, long long n,
                                                                    double* __restrict__ part) {
  __shared__ double sh[kNaBlock / 32];
  double acc = 0.0;
  const long long base = (long long)blockIdx.x * kNaBlock * kNaPerThread + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kNaPerThread; ++k) {
    const long long p = base + (long long)k * kNaBlock;
    if (p < n) acc += cabs2(__ldg(v + p));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kNaBlock / 32; ++w) tot += sh[w];
    part[blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(kNaBlock) k_norm2_finish_static(const double* __restrict__ part, int nblk,
                                                                  double* __restrict__ out) {
  __shared__ double sh[kNaBlock / 32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kNaBlock) acc += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kNaBlock / 32; ++w) tot += sh[w];
    *out = tot;
  }
}

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_lookup_mutex;
double* g_partials_addr[kMaxDevices] = {};

int partials_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MGCCCS_ECUDA;
  std::lock_guard<std::mutex> lock(g_lookup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return MGCCCS_ECUDA;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return MGCCCS_OK;
}

}  // namespace

extern "C" int mgcccs_norm2_noalloc(const mgcccs_c128* v, size_t n, double* norm2, void* stream) {
  if (!norm2 || (!v && n)) return MGCCCS_EINVAL;   // an empty vector may come as NULL
  if (n > (size_t)MGCCCS_NOALLOC_MAX_N) return MGCCCS_EINVAL;
  double* part = nullptr;
  int rc = partials_address(&part);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nblk = n == 0 ? 1 : (int)((n + (size_t)kNaBlock * kNaPerThread - 1) / ((size_t)kNaBlock * kNaPerThread));
  k_norm2_partials_static<<<nblk, kNaBlock, 0, st>>>(reinterpret_cast<const cplx*>(v), (long long)n, part);
  if (cudaGetLastError() != cudaSuccess) return MGCCCS_ECUDA;
  k_norm2_finish_static<<<1, kNaBlock, 0, st>>>(part, nblk, norm2);
  if (cudaGetLastError() != cudaSuccess) return MGCCCS_ECUDA;
  return MGCCCS_OK;
}
