// Kernels of the restarted GMRES(m) outer solver, right-preconditioned by one MG-CCCS
// iteration (Sec. 6: MG-CCCS as a Krylov preconditioner).  Arnoldi uses classical
// Gram-Schmidt (each pass: one fused multi-dot, one fused multi-axpy) with a second pass
// when a cancellation test asks for it (decided on the device);
// the Hessenberg least-squares problem is reduced by complex Givens rotations on the
// device, so the host only reads one residual estimate per step.
//
// Basis vectors are stored contiguously: V_i = V + i * ld.
#include "common.cuh"

namespace {

constexpr int NT = 256;

// Block sum of a complex value: warp sums in the element precision, the per-warp totals
// in FP64 by thread 0 (fixed order).  Complex64 data keeps the FP64 pipe out of the
// per-thread work.
template <int NTH, class C>
__device__ __forceinline__ cplx block_sum_c(C v, double (*sh)[NTH / 32]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  if ((t & 31) == 0) { sh[0][t >> 5] = (double)v.x; sh[1][t >> 5] = (double)v.y; }
  __syncthreads();
  cplx tot = cmk(0.0, 0.0);
  if (t == 0)
    for (int w = 0; w < NTH / 32; ++w) tot = cadd(tot, cmk(sh[0][w], sh[1][w]));
  return tot;
}

// partial[i][b] = sum over block b's points of conj(V_i) w   (grid: nblk x k).
// When `gate` is given and *gate == 0 the pass is skipped (partials set to zero).
// A vector V_i that is w itself gives |w|^2 (two FMAs per point; the block's branch).
// (Each thread accumulates in the element precision; the block sum is FP64.)
template <class C>
__global__ void __launch_bounds__(NT) k_multidot(long long n, const C* __restrict__ V, long long ld,
                                                 const C* __restrict__ w, cplx* __restrict__ partial,
                                                 const int* __restrict__ gate) {
  mgc_pdl_enter();
  __shared__ double sh[2][NT / 32];
  const int i = blockIdx.y;
  if (gate && *gate == 0) {
    if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = cmk(0.0, 0.0);
    return;
  }
  const C* v = V + (size_t)i * ld;
  C acc = CT<C>::make(0.0, 0.0);
  if (v == w) {
    for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < n; p += (long long)gridDim.x * NT) {
      C b = __ldg(w + p);
      acc.x = fma(b.x, b.x, fma(b.y, b.y, acc.x));
    }
  } else {
    for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < n; p += (long long)gridDim.x * NT) {
      C a = __ldg(v + p), b = __ldg(w + p);
      acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
      acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    }
  }
  cplx tot = block_sum_c<NT>(acc, sh);
  if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = tot;
}

// out[i] = sum_b partial[i][b] (fixed order); acc_into[i] += out[i] when given.
__global__ void __launch_bounds__(NT) k_reduce_dots(int nblk, const cplx* __restrict__ partial,
                                                    cplx* __restrict__ out, cplx* __restrict__ acc_into) {
  mgc_pdl_enter();
  __shared__ double sh[2][NT / 32];
  const int i = blockIdx.x;
  cplx acc = cmk(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += NT) acc = cadd(acc, partial[(size_t)i * nblk + b]);
  cplx tot = block_sum_c<NT>(acc, sh);
  if (threadIdx.x == 0) {
    out[i] = tot;
    if (acc_into) acc_into[i] = cadd(acc_into[i], tot);
  }
}

// w += sgn * sum_{i<k} coef[i] V_i ; optional per-block partials of |w|^2.
template <class C>
__global__ void __launch_bounds__(NT) k_multiaxpy(long long n, int k, const C* __restrict__ V, long long ld,
                                                  const cplx* __restrict__ coef, double sgn, C* __restrict__ w,
                                                  double* __restrict__ norm_part, const int* __restrict__ gate,
                                                  const int* __restrict__ dk) {
  mgc_pdl_enter();
  __shared__ C sc[64];
  __shared__ double sh[NT / 32];
  if (gate && *gate == 0) return;
  if (dk) k = min(k, *dk);
  for (int i = threadIdx.x; i < k; i += NT) {
    const cplx q = cscal(sgn, coef[i]);
    sc[i] = CT<C>::make(q.x, q.y);
  }
  __syncthreads();
  typename CT<C>::R n2 = 0;
  for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < n; p += (long long)gridDim.x * NT) {
    C acc = w[p];
    for (int i = 0; i < k; ++i) acc = cfma(sc[i], __ldg(V + (size_t)i * ld + p), acc);
    w[p] = acc;
    n2 += cabs2(acc);
  }
  if (norm_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)n2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int q = 0; q < NT / 32; ++q) tot += sh[q];
      norm_part[blockIdx.x] = tot;
    }
  }
}

// ---- complex64 update on element pairs.  With an even basis pitch every V_i + 2q and w + 2q
// is 16-byte aligned, so a thread moves two complex64 values per load; the loads of four
// basis vectors are issued before their FMAs, so each thread keeps four 16-byte loads in
// flight.  An odd last element is handled by one thread at the end.  (The same pair form
// of the multi-dot measured slower than the element form, 22.7 against 21.0 us a step,
// so the multi-dot keeps one element per thread.)

// acc += c * (a.x + i a.y) and c * (a.z + i a.w): two complex FMAs on a pair.
__device__ __forceinline__ float4 cfma2(float2 c, float4 a, float4 acc) {
  acc.x = fmaf(c.x, a.x, fmaf(-c.y, a.y, acc.x));
  acc.y = fmaf(c.x, a.y, fmaf(c.y, a.x, acc.y));
  acc.z = fmaf(c.x, a.z, fmaf(-c.y, a.w, acc.z));
  acc.w = fmaf(c.x, a.w, fmaf(c.y, a.z, acc.w));
  return acc;
}

// w += sgn * sum_{i<k} coef[i] V_i (complex64, pitch even, V and w 16-byte aligned);
// optional per-block partials of |w|^2.  Same operation as k_multiaxpy<float2>.
__global__ void __launch_bounds__(NT, 6) k_multiaxpy_c64(long long n, int k, const float2* __restrict__ V, long long ld,
                                                      const cplx* __restrict__ coef, double sgn,
                                                      float2* __restrict__ w, double* __restrict__ norm_part,
                                                      const int* __restrict__ gate, const int* __restrict__ dk) {
  mgc_pdl_enter();
  __shared__ float2 sc[64];
  __shared__ double sh[NT / 32];
  if (gate && *gate == 0) return;
  if (dk) k = min(k, *dk);
  for (int i = threadIdx.x; i < k; i += NT) {
    const cplx q = cscal(sgn, coef[i]);
    sc[i] = make_float2((float)q.x, (float)q.y);
  }
  __syncthreads();
  const float4* __restrict__ V4 = reinterpret_cast<const float4*>(V);
  float4* __restrict__ w4 = reinterpret_cast<float4*>(w);
  const long long ld4 = ld >> 1, np = n >> 1;
  float n2 = 0.f;
  for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < np; q += (long long)gridDim.x * NT) {
    float4 acc = w4[q];
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      const float4 a0 = __ldg(V4 + (size_t)i * ld4 + q), a1 = __ldg(V4 + (size_t)(i + 1) * ld4 + q);
      const float4 a2 = __ldg(V4 + (size_t)(i + 2) * ld4 + q), a3 = __ldg(V4 + (size_t)(i + 3) * ld4 + q);
      acc = cfma2(sc[i], a0, acc);
      acc = cfma2(sc[i + 1], a1, acc);
      acc = cfma2(sc[i + 2], a2, acc);
      acc = cfma2(sc[i + 3], a3, acc);
    }
    for (; i < k; ++i) acc = cfma2(sc[i], __ldg(V4 + (size_t)i * ld4 + q), acc);
    w4[q] = acc;
    n2 += acc.x * acc.x + acc.y * acc.y + acc.z * acc.z + acc.w * acc.w;
  }
  if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == NT - 1) {
    const long long p = n - 1;
    float2 acc = w[p];
    for (int i = 0; i < k; ++i) acc = cfma(sc[i], __ldg(V + (size_t)i * ld + p), acc);
    w[p] = acc;
    n2 += cabs2(acc);
  }
  if (norm_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)n2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int q = 0; q < NT / 32; ++q) tot += sh[q];
      norm_part[blockIdx.x] = tot;
    }
  }
}

// Whether the pair kernels apply: 16-byte aligned bases and an even pitch.
__host__ __forceinline__ bool pairs_ok(const void* a, const void* b, long long ld) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0 && (ld & 1) == 0;
}

// out = w / sqrt(*norm2) (zeros if the norm vanishes); *store = sqrt(*norm2) + 0i.
template <class C>
__global__ void __launch_bounds__(NT) k_scale_by_norm(long long n, const C* __restrict__ w, C* __restrict__ out,
                                                      const double* __restrict__ norm2, cplx* __restrict__ store) {
  mgc_pdl_enter();
  __shared__ double sb[2];
  if (threadIdx.x == 0) {
    const double b = sqrt(*norm2);
    sb[0] = b;
    sb[1] = b > 0.0 ? 1.0 / b : 0.0;
  }
  __syncthreads();
  const double beta = sb[0], s = sb[1];
  const long long p0 = blockIdx.x * (long long)NT + threadIdx.x;
  if (p0 == 0 && store) *store = cmk(beta, 0.0);
  for (long long p = p0; p < n; p += (long long)gridDim.x * NT) out[p] = cscal((typename CT<C>::R)s, w[p]);
}

// Apply rotations 0..j-1 to column j of H (h_{j+1,j} = sqrt(hn2)), build rotation j,
// update g; est = |g[j+1]|.  Called by every thread of one block.
// H is column-major with leading dimension m+1.  Rotation j maps rows (j, j+1) by
// [conj(c) conj(s); -s c] with c = a/rho, s = b/rho, rho = sqrt(|a|^2 + |b|^2).
__device__ __forceinline__ void givens_step(int j, int m, cplx* __restrict__ H, cplx* __restrict__ cs,
                                            cplx* __restrict__ sn, cplx* __restrict__ g, double* __restrict__ est,
                                            double hn2) {
  // the column and the earlier rotations are staged in shared memory by the block, so the
  // sequential chain of thread 0 waits on no global load
  __shared__ cplx col[MGC_MAX_RESTART + 1], rc[MGC_MAX_RESTART], rs[MGC_MAX_RESTART];
  cplx* colg = H + (size_t)j * (m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = colg[i];
  // h_{j+1,j} = |w| from its square (the value the normalisation of v_{j+1} uses), so the
  // rotation need not wait for that kernel
  if (threadIdx.x == 0) col[j + 1] = cmk(sqrt(hn2), 0.0);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    rc[i] = cs[i];
    rs[i] = sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // x carries entry i of the column through the chain in a register (rotation i - 1
    // wrote it), so each step waits on arithmetic only, not on a shared-memory round trip
    cplx x = col[0];
    for (int i = 0; i < j; ++i) {
      const cplx y = col[i + 1], c = rc[i], s = rs[i];
      col[i] = cadd(cmul(cmk(c.x, -c.y), x), cmul(cmk(s.x, -s.y), y));
      x = csub(cmul(c, y), cmul(s, x));
    }
    cplx a = x, b = col[j + 1];
    double rho = sqrt(cabs2(a) + cabs2(b));
    cplx c, s;
    if (rho == 0.0) {
      c = cmk(1.0, 0.0);
      s = cmk(0.0, 0.0);
    } else {
      c = cscal(1.0 / rho, a);
      s = cscal(1.0 / rho, b);
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = cmk(rho, 0.0);
    col[j + 1] = cmk(0.0, 0.0);
    cplx gj = g[j];
    g[j + 1] = cneg(cmul(s, gj));
    g[j] = cmul(cmk(c.x, -c.y), gj);
    *est = cmod(g[j + 1]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) colg[i] = col[i];
}

// The Givens update of step j on its own (after a second Gram-Schmidt pass); skipped when
// `gate` is given and *gate == 0 (the update then ran inside k_sum_dgks).
__global__ void k_givens(int j, int m, cplx* __restrict__ H, cplx* __restrict__ cs, cplx* __restrict__ sn,
                         cplx* __restrict__ g, double* __restrict__ est, const double* __restrict__ hnorm2,
                         const int* __restrict__ gate) {
  mgc_pdl_enter();
  if (gate && *gate == 0) return;
  givens_step(j, m, H, cs, sn, g, est, *hnorm2);
}

// Back substitution R y = g[0..k-1] with the rotated (upper-triangular) H.
__global__ void k_hess_solve(int k, int m, const cplx* __restrict__ H, const cplx* __restrict__ g,
                             cplx* __restrict__ y, const int* __restrict__ dk) {
  mgc_pdl_enter();
  if (threadIdx.x != 0) return;
  if (dk) k = min(k, *dk);
  for (int i = k - 1; i >= 0; --i) {
    cplx t = g[i];
    for (int q = i + 1; q < k; ++q) t = cfms(H[(size_t)q * (m + 1) + i], y[q], t);
    y[i] = cdiv(t, H[(size_t)i * (m + 1) + i]);
  }
}

// ---- device-driven GMRES: stop tests that steer the conditional nodes of a solve graph.
// One thread each; every value a test needs lives in the SolveCtl record.

// After the true residual |r|^2 of a restart: stop (converged, out of steps, non-finite,
// or a zero right-hand side) or open the next cycle with its estimate scale and target.
__global__ void k_outer_control(SolveCtl* __restrict__ c, const double* __restrict__ rn2p,
                                cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_cycle,
                                cudaGraphConditionalHandle h_inner, cudaGraphConditionalHandle h_switch) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  c->outer += 1;
  const double fn = sqrt(c->fn2);
  const double rn2 = *rn2p;
  bool stop = true;
  if (fn == 0.0) {
    c->rr = 0.0;
    c->status = SOLVECTL_ZERO_RHS;
  } else {
    const double rr = sqrt(rn2) / fn;
    c->rr = rr;
    if (rr < c->rr_min) c->rr_min = rr;
    if (!isfinite(rr)) {
      c->status = SOLVECTL_NONFINITE;
    } else if (rr > MGC_DIVERGENCE_FACTOR * c->rr_min) {
      c->status = SOLVECTL_DIVERGED;
    } else if (rr <= c->rtol) {
      c->status = SOLVECTL_CONVERGED;
    } else if (c->steps >= c->max_iter) {
      c->status = SOLVECTL_MAXITER;
    } else {
      const double beta = sqrt(rn2);
      if (c->mixed) {
        c->scale = beta / fn;
        c->target = fmax(c->inner_rtol, 0.5 * c->rtol * fn / beta) * beta / fn;
      } else {
        c->scale = 1.0 / fn;
        c->target = c->rtol;
      }
      c->j = 0;
      c->k = 0;
      c->cycles += 1;
      stop = false;
    }
  }
  cudaGraphSetConditional(h_outer, stop ? 0u : 1u);
  cudaGraphSetConditional(h_cycle, stop ? 0u : 1u);
  cudaGraphSetConditional(h_inner, stop ? 0u : 1u);
  cudaGraphSetConditional(h_switch, 0u);
}

// After Arnoldi step j: count it, and run step j+1 unless its residual estimate met the
// target, the step budget is spent, the cycle is full, or the estimate is not finite.
__global__ void k_step_control(SolveCtl* __restrict__ c, const double* __restrict__ est_raw,
                               cudaGraphConditionalHandle h_inner, cudaGraphConditionalHandle h_switch) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double est = *est_raw * c->scale;
  c->steps += 1;
  c->j += 1;
  c->k = c->j;
  const bool cont = isfinite(est) && est > c->target && c->steps < c->max_iter && c->j < c->m;
  cudaGraphSetConditional(h_switch, (unsigned)c->j);
  cudaGraphSetConditional(h_inner, cont ? 1u : 0u);
}

// Reorthogonalisation test: a second Gram-Schmidt pass runs only when the first pass
// cancelled |w| by more than a factor 1e3 (|w_after|^2 < 1e-6 |w_before|^2), so one
// pass never loses more than about 1e3 ulps of orthogonality.  (The classic threshold
// 1/sqrt(2) fires on almost every step here: with a good preconditioner A M^{-1} v_j is
// close to v_j and a first pass routinely removes half of |w|^2, harmlessly.)
// |w|^2 after the first pass comes from the block partials in the fixed summation order
// of k_sum_partials, and the decision is taken in the same kernel; in a device-driven
// solve graph it also sets the conditional node that holds the second pass (use_cond)
// and counts the passes that run.  When H is given and no second pass is needed (nearly
// every step), the Givens update of step j runs here as well, with the |w|^2 just
// summed, so it costs no launch of its own; after a second pass k_givens does it.
__global__ void __launch_bounds__(256) k_sum_dgks(const double* __restrict__ part, int n, double* __restrict__ out,
                                                  const double* __restrict__ before, int* __restrict__ gate,
                                                  cudaGraphConditionalHandle hd, int use_cond,
                                                  int* __restrict__ fired, int j, int m, cplx* __restrict__ H,
                                                  cplx* __restrict__ cs, cplx* __restrict__ sn,
                                                  cplx* __restrict__ g, double* __restrict__ est) {
  __shared__ double sh[8];
  __shared__ double s_tot;
  __shared__ int s_second;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) v += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) tot += sh[w];
    *out = tot;
    const int second = (tot < 1e-6 * *before) ? 1 : 0;
    *gate = second;
    if (use_cond) {
      cudaGraphSetConditional(hd, (unsigned)second);
      if (second) *fired += 1;
    }
    s_tot = tot;
    s_second = second;
  }
  __syncthreads();
  if (H && !s_second) givens_step(j, m, H, cs, sn, g, est, s_tot);
}

__global__ void k_zero_c(int n, cplx* __restrict__ a) {
  mgc_pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = cmk(0.0, 0.0);
}

}  // namespace

int krylov_blocks(long long n, int per_sm) {
  const long long b = (n + NT - 1) / NT, cap = (long long)per_sm * mgc_sm_count();
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// Blocks per vector of a k-vector multi-dot: about one full wave (8 blocks per SM) over
// all k vectors, so that each thread folds many elements before its share of the block
// reduction; never more than krylov_blocks(n), never fewer than 64.
int multidot_blocks(long long n, int k) {
  const int cap = krylov_blocks(n, 4);
  int b = 8 * mgc_sm_count() / (k < 1 ? 1 : k);
  if (b < 64) b = 64;
  return b < cap ? b : cap;
}

template <class C>
cudaError_t launch_multidot(long long n, int k, const C* V, long long ld, const C* w, cplx* partial,
                            int nblk, const int* gate, cudaStream_t st) {
  return mgc_launch(k_multidot<C>, dim3(nblk, k), dim3(NT), 0, st, n, V, ld, w, partial, gate);
}

cudaError_t launch_reduce_dots(int nblk, int k, const cplx* partial, cplx* out, cplx* acc_into, cudaStream_t st) {
  return mgc_launch(k_reduce_dots, dim3(k), dim3(NT), 0, st, nblk, partial, out, acc_into);
}

template <class C>
cudaError_t launch_multiaxpy(long long n, int k, const C* V, long long ld, const cplx* coef, double sgn,
                             C* w, double* norm_part, int nblk, const int* gate, cudaStream_t st, const int* dk) {
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (pairs_ok(V, w, ld)) {
      return mgc_launch(k_multiaxpy_c64, dim3(nblk), dim3(NT), 0, st, n, k, V, ld, coef, sgn, w, norm_part, gate, dk);
    }
  }
  return mgc_launch(k_multiaxpy<C>, dim3(nblk), dim3(NT), 0, st, n, k, V, ld, coef, sgn, w, norm_part, gate, dk);
}

template <class C>
cudaError_t launch_scale_by_norm(long long n, const C* w, C* out, const double* norm2, cplx* store,
                                 int nblk, cudaStream_t st) {
  return mgc_launch(k_scale_by_norm<C>, dim3(nblk), dim3(NT), 0, st, n, w, out, norm2, store);
}

#define MGC_INSTANTIATE(C)                                                                                  \
  template cudaError_t launch_multidot<C>(long long, int, const C*, long long, const C*, cplx*, int,        \
                                         const int*, cudaStream_t);                                       \
  template cudaError_t launch_multiaxpy<C>(long long, int, const C*, long long, const cplx*, double, C*,   \
                                          double*, int, const int*, cudaStream_t, const int*);            \
  template cudaError_t launch_scale_by_norm<C>(long long, const C*, C*, const double*, cplx*, int,         \
                                              cudaStream_t);
MGC_INSTANTIATE(double2)
MGC_INSTANTIATE(float2)
#undef MGC_INSTANTIATE

cudaError_t launch_givens(int j, int m, cplx* H, cplx* cs, cplx* sn, cplx* g, double* est, const double* hnorm2,
                          cudaStream_t st, const int* gate) {
  return mgc_launch(k_givens, dim3(1), dim3(32), 0, st, j, m, H, cs, sn, g, est, hnorm2, gate);
}

cudaError_t launch_hess_solve(int k, int m, const cplx* H, const cplx* g, cplx* y, cudaStream_t st,
                              const int* dk) {
  return mgc_launch(k_hess_solve, dim3(1), dim3(32), 0, st, k, m, H, g, y, dk);
}


cudaError_t launch_outer_control(SolveCtl* c, const double* rn2, cudaGraphConditionalHandle h_outer,
                                 cudaGraphConditionalHandle h_cycle, cudaGraphConditionalHandle h_inner,
                                 cudaGraphConditionalHandle h_switch, cudaStream_t st) {
  k_outer_control<<<1, 32, 0, st>>>(c, rn2, h_outer, h_cycle, h_inner, h_switch);
  return cudaGetLastError();
}

cudaError_t launch_step_control(SolveCtl* c, const double* est, cudaGraphConditionalHandle h_inner,
                                cudaGraphConditionalHandle h_switch, cudaStream_t st) {
  k_step_control<<<1, 32, 0, st>>>(c, est, h_inner, h_switch);
  return cudaGetLastError();
}

cudaError_t launch_sum_dgks(const double* part, int n, double* out, const double* before, int* gate,
                           cudaStream_t st, cudaGraphConditionalHandle hd, int* fired, const GivensArgs* gv) {
  if (gv)
    k_sum_dgks<<<1, 256, 0, st>>>(part, n, out, before, gate, hd, fired ? 1 : 0, fired, gv->j, gv->m, gv->H, gv->cs,
                                  gv->sn, gv->g, gv->est);
  else
    k_sum_dgks<<<1, 256, 0, st>>>(part, n, out, before, gate, hd, fired ? 1 : 0, fired, 0, 0, nullptr, nullptr,
                                  nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_zero_c(int n, cplx* a, cudaStream_t st) {
  return mgc_launch(k_zero_c, dim3((n + 255) / 256), dim3(256), 0, st, n, a);
}
