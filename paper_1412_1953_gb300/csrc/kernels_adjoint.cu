// Kernels of the amplitude functional J = <g|u> = sum_k w_k g_k u_k and of its adjoint
// gradients.  W (H - E) is complex symmetric (Sec. 2.5), so the adjoint solve is a
// forward solve (H - E) mu = g and, for a parameter p, dJ/dp = -sum_k w_k mu_k
// ((d(H-E)/dp) u)_k; these kernels form the weighted sums and products on the fine
// grid, with w_k = w_x(i) w_y(j) the quadrature weights of the ECS contour.
#include "common.cuh"

namespace {

constexpr int NT = 256;

// partial[b] = sum over block b of w_x(i) w_y(j) a_k b_k (d_k), grid-stride, fixed order.
__global__ void __launch_bounds__(NT) k_wdot_partials(int mx, int my, const cplx* __restrict__ wx,
                                                      const cplx* __restrict__ wy, const cplx* __restrict__ a,
                                                      const cplx* __restrict__ b, const cplx* __restrict__ d,
                                                      cplx* __restrict__ part) {
  __shared__ double sh[2][NT / 32];
  const long long n = (long long)mx * my;
  cplx acc = cmk(0.0, 0.0);
  for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < n; p += (long long)gridDim.x * NT) {
    const int i = (int)(p % mx), j = (int)(p / mx);
    cplx t = cmul(cmul(__ldg(wx + i), __ldg(wy + j)), cmul(__ldg(a + p), __ldg(b + p)));
    if (d) t = cmul(t, __ldg(d + p));
    acc = cadd(acc, t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc.x; sh[1][threadIdx.x >> 5] = acc.y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx tot = cmk(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) tot = cadd(tot, cmk(sh[0][w], sh[1][w]));
    part[blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(NT) k_wdot_finish(int nblk, const cplx* __restrict__ part, cplx scale,
                                                    cplx* __restrict__ out) {
  __shared__ double sh[2][NT / 32];
  cplx acc = cmk(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += NT) acc = cadd(acc, part[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc.x; sh[1][threadIdx.x >> 5] = acc.y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx tot = cmk(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) tot = cadd(tot, cmk(sh[0][w], sh[1][w]));
    *out = cmul(scale, tot);
  }
}

// out_k = scale * w_x(i) w_y(j) a_k b_k
__global__ void __launch_bounds__(NT) k_wproduct(int mx, int my, const cplx* __restrict__ wx,
                                                 const cplx* __restrict__ wy, const cplx* __restrict__ a,
                                                 const cplx* __restrict__ b, cplx scale, cplx* __restrict__ out) {
  const long long n = (long long)mx * my;
  for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < n; p += (long long)gridDim.x * NT) {
    const int i = (int)(p % mx), j = (int)(p / mx);
    out[p] = cmul(scale, cmul(cmul(__ldg(wx + i), __ldg(wy + j)), cmul(__ldg(a + p), __ldg(b + p))));
  }
}

}  // namespace

int wdot_blocks(long long n) {
  const long long b = (n + NT - 1) / NT, cap = 4LL * mgc_sm_count();
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

cudaError_t launch_weighted_dot(int mx, int my, const cplx* wx, const cplx* wy, const cplx* a, const cplx* b,
                                const cplx* d, cplx scale, cplx* part, cplx* out, cudaStream_t st) {
  const int nblk = wdot_blocks((long long)mx * my);
  k_wdot_partials<<<nblk, NT, 0, st>>>(mx, my, wx, wy, a, b, d, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_wdot_finish<<<1, NT, 0, st>>>(nblk, part, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_weighted_product(int mx, int my, const cplx* wx, const cplx* wy, const cplx* a, const cplx* b,
                                    cplx scale, cplx* out, cudaStream_t st) {
  k_wproduct<<<wdot_blocks((long long)mx * my), NT, 0, st>>>(mx, my, wx, wy, a, b, scale, out);
  return cudaGetLastError();
}
