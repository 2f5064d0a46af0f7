// Eigenvalues of the complex-symmetric tridiagonal of a 1D bound-state problem (Eq. (9)
// on the ECS grid) by the Ehrlich-Aberth simultaneous iteration with divide-and-conquer
// starting values, after D. A. Bini, L. Gemignani and F. Tisseur, "The Ehrlich-Aberth
// method for the nonsymmetric tridiagonal eigenvalue problem", SIAM J. Matrix Anal.
// Appl. 27 (2005).
//
// Level by level the matrix is cut into blocks of bs = 2, 4, 8, ... rows; the
// eigenvalues of the two halves of a block (the previous level's converged values) are
// the starting values for the block.  One thread owns one approximation z_i and per
// iteration evaluates
//   the Newton correction N_i = p(z_i)/p'(z_i) of the block's characteristic polynomial
//     by the three-term recurrence p_k = (d_k - z) p_{k-1} - e2_{k-1} p_{k-2} and its
//     derivative p'_k = (d_k - z) p'_{k-1} - p_{k-1} - e2_{k-1} p'_{k-2}, rescaled by
//     powers of two (the starting values are exact eigenvalues of the two half blocks,
//     where a leading minor vanishes, so a ratio form p_k/p_{k-1} would divide by zero);
//   the Aberth step z_i <- z_i - N_i / (1 - N_i sum_{j != i} 1/(z_i - z_j)).
// An approximation whose step falls below the tolerance is frozen.  The squared
// off-diagonals e2_k = east_k west_{k+1} are all the recurrence needs, so no square
// root is taken and the complex-symmetric form is never built.
#include "common.cuh"

namespace {

constexpr int EIG_THREADS = 32;    // one warp per block: the approximations spread over many SMs

__device__ __forceinline__ cplx recip(cplx z) { return cdiv(cmk(1.0, 0.0), z); }

__global__ void k_eig_init(int m, const cplx* __restrict__ west, const cplx* __restrict__ east,
                           const cplx* __restrict__ diag, const cplx* __restrict__ v, cplx* __restrict__ d,
                           cplx* __restrict__ e2, cplx* __restrict__ z, unsigned long long* __restrict__ scale_bits) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const cplx dk = cadd(diag[k], v[k]);
  const cplx ek = (k + 1 < m) ? cmul(east[k], west[k + 1]) : cmk(0.0, 0.0);
  d[k] = dk;
  e2[k] = ek;
  z[k] = dk;                                     // 1 x 1 blocks: their eigenvalues
  // a bound on the spectral radius (Gershgorin with |e_k| = sqrt|e2_k|) sets the absolute
  // tolerance; nonnegative doubles order like their bit patterns
  const double bound = cabs1(dk) + 2.0 * sqrt(cabs1(ek));
  atomicMax(scale_bits, (unsigned long long)__double_as_longlong(bound));
}

__global__ void __launch_bounds__(EIG_THREADS) k_eig_aberth(int m, int bs, const cplx* __restrict__ d,
                                                            const cplx* __restrict__ e2,
                                                            const cplx* __restrict__ zin, cplx* __restrict__ zout,
                                                            int* __restrict__ done, int* __restrict__ active,
                                                            const unsigned long long* __restrict__ scale_bits) {
  const int i = blockIdx.x * EIG_THREADS + threadIdx.x;
  if (i >= m) return;
  const int s0 = (i / bs) * bs;
  const int s1 = min(s0 + bs, m);
  const cplx zi = zin[i];
  // a block without its second half is the previous level's block: already converged
  if (s1 - s0 <= bs / 2 || done[i]) {
    zout[i] = zi;
    return;
  }
  const double scale = __longlong_as_double((long long)*scale_bits);
  // p and p' of the block's leading principal minors by the three-term recurrence,
  // rescaled by exact powers of two when they leave [2^-400, 2^400] (only p/p' is used,
  // so a common factor drops out; no division, so a vanishing minor is harmless)
  cplx pm1 = cmk(1.0, 0.0), pm2 = cmk(0.0, 0.0);
  cplx qm1 = cmk(0.0, 0.0), qm2 = cmk(0.0, 0.0);
  for (int k = s0; k < s1; ++k) {
    const cplx dz = csub(d[k], zi);
    const cplx ek = k > s0 ? e2[k - 1] : cmk(0.0, 0.0);
    const cplx pk = cfms(ek, pm2, cmul(dz, pm1));
    const cplx qk = csub(cfms(ek, qm2, cmul(dz, qm1)), pm1);
    pm2 = pm1; pm1 = pk;
    qm2 = qm1; qm1 = qk;
    const double mx = fmax(cabs1(pm1), cabs1(qm1));
    if (mx > 0x1p400 || (mx < 0x1p-400 && mx > 0.0)) {
      const double f = ldexp(1.0, -ilogb(mx));
      pm1 = cscal(f, pm1); pm2 = cscal(f, pm2);
      qm1 = cscal(f, qm1); qm2 = cscal(f, qm2);
    }
  }
  // Aberth's implicit deflation by the other approximations of the block
  cplx A = cmk(0.0, 0.0);
  for (int j = s0; j < s1; ++j) {
    if (j == i) continue;
    const cplx dz = csub(zi, zin[j]);
    if (cabs1(dz) > 0.0) A = cadd(A, recip(dz));
  }
  cplx step;
  if (cabs1(qm1) == 0.0) {
    step = cmk(1e-8 * scale, 1e-8 * scale);                  // critical point of p: move off it
  } else {
    const cplx N = cdiv(pm1, qm1);                           // Newton correction p/p'
    step = cdiv(N, csub(cmk(1.0, 0.0), cmul(N, A)));
  }
  const cplx zn = csub(zi, step);
  const bool fin = isfinite(zn.x) && isfinite(zn.y);
  zout[i] = fin ? zn : zi;
  if (fin && cabs1(step) <= 4e-15 * cabs1(zi) + 1e-14 * scale) {
    done[i] = 1;
  } else {
    atomicAdd(active, fin ? 1 : (1 << 20));                  // non-finite steps count as failure
  }
}

// Trace check: sum z_i must equal sum d_k (the trace) to rounding, else flag.
__global__ void __launch_bounds__(256) k_eig_check(int m, const cplx* __restrict__ d, const cplx* __restrict__ z,
                                                   const unsigned long long* __restrict__ scale_bits,
                                                   int* __restrict__ bad) {
  __shared__ double sh[4][256];
  double a = 0, b = 0, c = 0, e = 0;
  for (int k = threadIdx.x; k < m; k += 256) {
    a += d[k].x; b += d[k].y; c += z[k].x; e += z[k].y;
  }
  sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c; sh[3][threadIdx.x] = e;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double scale = __longlong_as_double((long long)*scale_bits);
    const double err = fabs(sh[0][0] - sh[2][0]) + fabs(sh[1][0] - sh[3][0]);
    *bad = !(err <= 1e-10 * scale * sqrt((double)m) + 1e-300);
  }
}

}  // namespace

size_t eig_scratch_entries(int m) {
  // d, e2, two approximation buffers, then done flags, counters and the scale (as ints)
  const size_t ints = (size_t)m + 8;
  return (size_t)4 * m + (ints * sizeof(int) + sizeof(cplx) - 1) / sizeof(cplx) + 1;
}

cudaError_t eig_aberth(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v, cplx* scratch,
                       cplx* out, bool* ok, cudaStream_t st) {
  *ok = false;
  cplx* d = scratch;
  cplx* e2 = scratch + m;
  cplx* za = scratch + 2 * m;
  cplx* zb = scratch + 3 * m;
  int* done = reinterpret_cast<int*>(scratch + 4 * m);
  int* active = done + m;
  int* bad = done + m + 1;
  unsigned long long* scale_bits = reinterpret_cast<unsigned long long*>(
      scratch + 4 * m + ((size_t)(m + 8) * sizeof(int) + sizeof(cplx) - 1) / sizeof(cplx));
  cudaError_t e = cudaMemsetAsync(scale_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int grid = (m + EIG_THREADS - 1) / EIG_THREADS;
  k_eig_init<<<(m + 255) / 256, 256, 0, st>>>(m, west, east, diag, v, d, e2, za, scale_bits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cplx* cur = za;
  cplx* nxt = zb;
  constexpr int kChunk = 4, kMaxIter = 240;
  for (int bs = 2; bs / 2 < m; bs *= 2) {
    if ((e = cudaMemsetAsync(done, 0, sizeof(int) * (size_t)m, st)) != cudaSuccess) return e;
    bool converged = false;
    for (int it = 0; it < kMaxIter && !converged; it += kChunk) {
      for (int c = 0; c < kChunk; ++c) {
        if ((e = cudaMemsetAsync(active, 0, sizeof(int), st)) != cudaSuccess) return e;
        k_eig_aberth<<<grid, EIG_THREADS, 0, st>>>(m, bs, d, e2, cur, nxt, done, active, scale_bits);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cplx* x = cur; cur = nxt; nxt = x;
      }
      int act = 0;
      if ((e = cudaMemcpyAsync(&act, active, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      if (act >= (1 << 20)) return cudaSuccess;                // non-finite: *ok stays false
      converged = act == 0;
    }
    if (!converged) return cudaSuccess;
  }
  k_eig_check<<<1, 256, 0, st>>>(m, d, cur, scale_bits, bad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int b = 1;
  if ((e = cudaMemcpyAsync(&b, bad, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if (b) return cudaSuccess;
  if ((e = cudaMemcpyAsync(out, cur, sizeof(cplx) * (size_t)m, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return e;
  *ok = true;
  return cudaSuccess;
}
