// Multigrid kernels of MG-CCCS: omega-Jacobi smoothing, residual, full-weighting
// restriction, bilinear interpolation and the coarsest-level direct solve
// (Sec. 3.2 of Cools & Vanroose; the operator is Eq. (11) on the ECS grid of Sec. 2.5).
//
// All arrays are interior-only, row-major [j][i] with pitch mx; values outside the
// interior are the homogeneous Dirichlet boundary (zero).  The complex128 path is
// bound by the FP64 pipe on this GPU, so every kernel computes each output exactly
// once (no overlapped halo recomputation) and the uniform-spacing box uses a single
// neighbour coefficient.
#include "common.cuh"

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ cplx ldz(const cplx* __restrict__ a, int p, bool ok) {
  return ok ? __ldg(a + p) : cmk(0.0, 0.0);
}

// (H - E) u at interior node (i, j), given the centre value uc.
__device__ __forceinline__ cplx apply_op(const StencilView& s, const cplx* __restrict__ u, int i, int j, cplx uc) {
  const int p = j * s.mx + i;
  cplx uw = ldz(u, p - 1, i > 0);
  cplx ue = ldz(u, p + 1, i + 1 < s.mx);
  cplx us = ldz(u, p - s.mx, j > 0);
  cplx un = ldz(u, p + s.mx, j + 1 < s.my);
  cplx a = cmul(__ldg(s.D + p), uc);
  if (i < s.ux && j < s.uy) {
    cplx sum = cadd(cadd(uw, ue), cadd(us, un));
    a = cfma(s.cu, sum, a);
  } else {
    a = cfma(__ldg(s.west_x + i), uw, a);
    a = cfma(__ldg(s.east_x + i), ue, a);
    a = cfma(__ldg(s.west_y + j), us, a);
    a = cfma(__ldg(s.east_y + j), un, a);
  }
  return a;
}

// Real part of a complex array element (only 8 bytes are loaded).
__device__ __forceinline__ double ldre(const cplx* __restrict__ a, int p) {
  return __ldg(reinterpret_cast<const double*>(a) + 2 * p);
}

// (H - E) u in the real box: real coefficient cu.x and real diagonal.
__device__ __forceinline__ cplx apply_op_rbox(const StencilView& s, const cplx* __restrict__ u, int i, int j,
                                              cplx uc) {
  const int p = j * s.mx + i;
  cplx sum = cadd(cadd(ldz(u, p - 1, i > 0), ldz(u, p + 1, i + 1 < s.mx)),
                  cadd(ldz(u, p - s.mx, j > 0), ldz(u, p + s.mx, j + 1 < s.my)));
  const double d = ldre(s.D, p);
  return cmk(fma(s.cu.x, sum.x, d * uc.x), fma(s.cu.x, sum.y, d * uc.y));
}

__global__ void __launch_bounds__(BX * BY) k_jacobi(StencilView s, const cplx* __restrict__ u_in,
                                                    cplx* __restrict__ u_out, const cplx* __restrict__ f) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= s.mx || j >= s.my) return;
  const int p = j * s.mx + i;
  cplx uc = __ldg(u_in + p);
  if (s.rbox && i < s.ux && j < s.uy) {
    cplx r = csub(__ldg(f + p), apply_op_rbox(s, u_in, i, j, uc));
    const double di = ldre(s.Dinv, p);
    u_out[p] = cmk(fma(di, r.x, uc.x), fma(di, r.y, uc.y));
  } else {
    cplx r = csub(__ldg(f + p), apply_op(s, u_in, i, j, uc));
    u_out[p] = cfma(__ldg(s.Dinv + p), r, uc);
  }
}

// First sweep from a zero initial guess: u = omega D^{-1} f.
__global__ void __launch_bounds__(256) k_jacobi_zero(long long n, const cplx* __restrict__ Dinv,
                                                    cplx* __restrict__ u_out, const cplx* __restrict__ f) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < n) u_out[p] = cmul(__ldg(Dinv + p), __ldg(f + p));
}

// Deterministic block reduction of one double (fixed tree order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  double tot = 0.0;
  if (t == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) tot += sh[w];
  }
  return tot;
}

__global__ void __launch_bounds__(BX * BY) k_residual(StencilView s, const cplx* __restrict__ u,
                                                      const cplx* __restrict__ f, cplx* __restrict__ r,
                                                      double* __restrict__ norm_part) {
  __shared__ double sh[BX * BY / 32];
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double n2 = 0.0;
  if (i < s.mx && j < s.my) {
    const int p = j * s.mx + i;
    const cplx uc = __ldg(u + p);
    cplx rv = csub(__ldg(f + p), (s.rbox && i < s.ux && j < s.uy) ? apply_op_rbox(s, u, i, j, uc)
                                                                    : apply_op(s, u, i, j, uc));
    if (r) r[p] = rv;
    n2 = cabs2(rv);
  }
  if (norm_part) {
    double tot = block_sum<BX * BY>(n2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) norm_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

// Full weighting 1/16 [1 2 1; 2 4 2; 1 2 1] onto the coincident nodes: coarse interior
// (I, J) sits on fine interior (2I+1, 2J+1); all nine taps are interior nodes.
__global__ void __launch_bounds__(256) k_restrict(int mx, int mcx, int mcy, const cplx* __restrict__ r,
                                                  cplx* __restrict__ rc) {
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 8 + threadIdx.y;
  if (I >= mcx || J >= mcy) return;
  const int c = (2 * J + 1) * mx + (2 * I + 1);
  cplx corners = cadd(cadd(__ldg(r + c - mx - 1), __ldg(r + c - mx + 1)),
                      cadd(__ldg(r + c + mx - 1), __ldg(r + c + mx + 1)));
  cplx edges = cadd(cadd(__ldg(r + c - 1), __ldg(r + c + 1)), cadd(__ldg(r + c - mx), __ldg(r + c + mx)));
  cplx centre = __ldg(r + c);
  cplx acc = cmk(fma(2.0, edges.x, fma(4.0, centre.x, corners.x)),
                 fma(2.0, edges.y, fma(4.0, centre.y, corners.y)));
  rc[J * mcx + I] = cscal(0.0625, acc);
}

__device__ __forceinline__ cplx coarse_at(const cplx* __restrict__ ec, int mcx, int mcy, int K, int Kp) {
  // coarse node (K, Kp), 0..mc+1; boundary nodes carry zero
  return (K >= 1 && K <= mcx && Kp >= 1 && Kp <= mcy) ? __ldg(ec + (Kp - 1) * mcx + (K - 1)) : cmk(0.0, 0.0);
}

// u += bilinear interpolation of the coarse correction (fine node k = i+1).
__global__ void __launch_bounds__(BX * BY) k_prolong_add(int mx, int my, int mcx, int mcy,
                                                         const cplx* __restrict__ ec, cplx* __restrict__ u) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= mx || j >= my) return;
  const int kx = i + 1, ky = j + 1;
  const int Kx = kx >> 1, Ky = ky >> 1;
  cplx v;
  if (!(kx & 1) && !(ky & 1)) {
    v = coarse_at(ec, mcx, mcy, Kx, Ky);
  } else if (!(ky & 1)) {
    v = cscal(0.5, cadd(coarse_at(ec, mcx, mcy, Kx, Ky), coarse_at(ec, mcx, mcy, Kx + 1, Ky)));
  } else if (!(kx & 1)) {
    v = cscal(0.5, cadd(coarse_at(ec, mcx, mcy, Kx, Ky), coarse_at(ec, mcx, mcy, Kx, Ky + 1)));
  } else {
    v = cscal(0.25, cadd(cadd(coarse_at(ec, mcx, mcy, Kx, Ky), coarse_at(ec, mcx, mcy, Kx + 1, Ky)),
                         cadd(coarse_at(ec, mcx, mcy, Kx, Ky + 1), coarse_at(ec, mcx, mcy, Kx + 1, Ky + 1))));
  }
  const int p = j * mx + i;
  u[p] = cadd(u[p], v);
}

// Coarsest level: u = A_c^{-1} f with the dense inverse built at setup; one warp per row.
__global__ void __launch_bounds__(256) k_coarse_solve(int nc, const cplx* __restrict__ Ainv,
                                                      const cplx* __restrict__ f, cplx* __restrict__ u) {
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nc) return;
  cplx acc = cmk(0.0, 0.0);
  const cplx* a = Ainv + (size_t)row * nc;
  for (int c = lane; c < nc; c += 32) acc = cfma(__ldg(a + c), __ldg(f + c), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) u[row] = acc;
}

// Sum of n partials in a fixed order (one block), result to out[0]; skipped when
// `gate` is given and *gate == 0.
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ part, int n,
                                                      double* __restrict__ out, const int* __restrict__ gate) {
  __shared__ double sh[8];
  if (gate && *gate == 0) return;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) v += part[k];
  double tot = block_sum<256>(v, sh);
  if (threadIdx.x == 0) out[0] = tot;
}

__global__ void __launch_bounds__(256) k_norm2(const cplx* __restrict__ v, long long n, double* __restrict__ part) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256)
    acc += cabs2(__ldg(v + p));
  double tot = block_sum<256>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(BX * BY) k_apply(StencilView s, const cplx* __restrict__ x, cplx* __restrict__ y,
                                                   double* __restrict__ norm_part) {
  __shared__ double sh[BX * BY / 32];
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  double n2 = 0.0;
  if (i < s.mx && j < s.my) {
    const int p = j * s.mx + i;
    const cplx xc = __ldg(x + p);
    cplx v = (s.rbox && i < s.ux && j < s.uy) ? apply_op_rbox(s, x, i, j, xc) : apply_op(s, x, i, j, xc);
    y[p] = v;
    n2 = cabs2(v);
  }
  if (norm_part) {
    double tot = block_sum<BX * BY>(n2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) norm_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

inline dim3 grid2(int mx, int my) { return dim3((mx + BX - 1) / BX, (my + BY - 1) / BY); }

}  // namespace

cudaError_t launch_jacobi(const StencilView& s, const cplx* u_in, cplx* u_out, const cplx* f, cudaStream_t st) {
  k_jacobi<<<grid2(s.mx, s.my), dim3(BX, BY), 0, st>>>(s, u_in, u_out, f);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_zero(const StencilView& s, cplx* u_out, const cplx* f, cudaStream_t st) {
  long long n = (long long)s.mx * s.my;
  k_jacobi_zero<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s.Dinv, u_out, f);
  return cudaGetLastError();
}

int residual_norm_blocks(const StencilView& s) {
  dim3 g = grid2(s.mx, s.my);
  return (int)(g.x * g.y);
}

cudaError_t launch_residual(const StencilView& s, const cplx* u, const cplx* f, cplx* r, double* norm_part,
                            cudaStream_t st) {
  k_residual<<<grid2(s.mx, s.my), dim3(BX, BY), 0, st>>>(s, u, f, r, norm_part);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int mx, int my, const cplx* r, cplx* rc, cudaStream_t st) {
  int mcx = (mx - 1) / 2, mcy = (my - 1) / 2;
  k_restrict<<<dim3((mcx + 31) / 32, (mcy + 7) / 8), dim3(32, 8), 0, st>>>(mx, mcx, mcy, r, rc);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(int mx, int my, const cplx* ec, cplx* u, cudaStream_t st) {
  int mcx = (mx - 1) / 2, mcy = (my - 1) / 2;
  k_prolong_add<<<grid2(mx, my), dim3(BX, BY), 0, st>>>(mx, my, mcx, mcy, ec, u);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(int nc, const cplx* Ainv, const cplx* f, cplx* u, cudaStream_t st) {
  k_coarse_solve<<<(nc + 7) / 8, 256, 0, st>>>(nc, Ainv, f, u);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t st, const int* gate) {
  k_sum_partials<<<1, 256, 0, st>>>(part, n, out, gate);
  return cudaGetLastError();
}

int norm2_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

cudaError_t launch_norm2(const cplx* v, long long n, double* part, int nblocks, cudaStream_t st) {
  k_norm2<<<nblocks, 256, 0, st>>>(v, n, part);
  return cudaGetLastError();
}

cudaError_t launch_apply(const StencilView& s, const cplx* x, cplx* y, cudaStream_t st, double* norm_part) {
  k_apply<<<grid2(s.mx, s.my), dim3(BX, BY), 0, st>>>(s, x, y, norm_part);
  return cudaGetLastError();
}
