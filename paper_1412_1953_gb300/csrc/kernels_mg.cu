// Multigrid kernels of MG-CCCS: omega-Jacobi smoothing, residual, full-weighting
// restriction, bilinear interpolation and the coarsest-level direct solve
// (Sec. 3.2 of Cools & Vanroose; the operator is Eq. (11) on the ECS grid of Sec. 2.5).
//
// All arrays are interior-only, row-major [j][i] with pitch mx; values outside the
// interior are the homogeneous Dirichlet boundary (zero).  Every kernel is a template
// over the element type C: double2 (complex128, the plain path, bound by the FP64
// pipe on this GPU) or float2 (complex64, the mixed-precision smoother and transfers,
// bound by HBM).  The one-step kernels compute each output once; the fused level passes
// further down recompute a one-node halo of their tiles instead of a launch.  The uniform
// parts of each axis use a single neighbour coefficient.
#include <atomic>

#include "common.cuh"

thread_local cudaStream_t g_mgc_last_kernel_stream = nullptr;
thread_local bool g_mgc_last_was_kernel = false;

const char* mgc_level_range_name(int level) {
  static const char* names[MGC_MAX_LEVELS] = {
      "mgcccs level 0",  "mgcccs level 1",  "mgcccs level 2",  "mgcccs level 3",
      "mgcccs level 4",  "mgcccs level 5",  "mgcccs level 6",  "mgcccs level 7",
      "mgcccs level 8",  "mgcccs level 9",  "mgcccs level 10", "mgcccs level 11",
      "mgcccs level 12", "mgcccs level 13", "mgcccs level 14", "mgcccs level 15"};
  return level >= 0 && level < MGC_MAX_LEVELS ? names[level] : "mgcccs level";
}

int mgc_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 152;
  }
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

namespace {

constexpr int BX = 32, BY = 8;

// u_p, or zero outside the interior (the homogeneous Dirichlet boundary).
template <class C>
__device__ __forceinline__ C ldz(const C* __restrict__ a, int p, bool ok) {
  return ok ? __ldg(a + p) : CT<C>::make(0.0, 0.0);
}

// The four neighbour values of interior node p = (i, j) (zero outside the interior).
#define MGC_NEIGHBOURS(s, u, p, i, j)                                                          \
  ldz(u, (p) - 1, (i) > 0), ldz(u, (p) + 1, (i) + 1 < (s).mx), ldz(u, (p) - (s).mx, (j) > 0), \
      ldz(u, (p) + (s).mx, (j) + 1 < (s).my)

// Template arguments of the per-node helpers from the IntC arguments of dispatch_kinds.
#define MGC_KINDS(kx, ky, ir, dg) decltype(kx)::value, decltype(ky)::value, decltype(ir)::value, decltype(dg)::value

// (H - E) u at interior node (i, j), given the centre value uc.
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C apply_pt(const StencilViewT<C>& s, const C* __restrict__ u, int i, int j, C uc) {
  const int p = j * s.mx + i;
  return apply_vals<KX, KY, IR, DG>(s, i, j, p, uc, MGC_NEIGHBOURS(s, u, p, i, j));
}

// ---- per-node arithmetic

// One omega-Jacobi update at (i, j): u + (omega/D)(f - (H-E)u).
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C jacobi_pt(const StencilViewT<C>& s, const C* __restrict__ u_in,
                                       const C* __restrict__ f, int i, int j) {
  const int p = j * s.mx + i;
  return jacobi_vals<KX, KY, IR, DG>(s, i, j, p, __ldg(u_in + p), MGC_NEIGHBOURS(s, u_in, p, i, j),
                                     __ldg(f + p));
}

template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C residual_pt(const StencilViewT<C>& s, const C* __restrict__ u, const C* __restrict__ f,
                                         int i, int j) {
  const int p = j * s.mx + i;
  return residual_vals<KX, KY, IR, DG>(s, i, j, p, __ldg(u + p), MGC_NEIGHBOURS(s, u, p, i, j),
                                       __ldg(f + p));
}

// dispatch_kinds for the block of this thread.
template <class C, class F>
__device__ __forceinline__ void block_kinds(const StencilViewT<C>& s, F&& f) {
  const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
  dispatch_kinds(s, i0, min(i0 + (int)blockDim.x, s.mx), j0, min(j0 + (int)blockDim.y, s.my), f);
}


// Full weighting 1/16 [1 2 1; 2 4 2; 1 2 1] from the residuals r(dx, dy) at offsets
// dx, dy in {-1, 0, 1} around the coincident fine node.
template <class C, class G>
__device__ __forceinline__ C restrict_at(G&& r) {
  typedef typename CT<C>::R R;
  C corners = cadd(cadd(r(-1, -1), r(1, -1)), cadd(r(-1, 1), r(1, 1)));
  C edges = cadd(cadd(r(-1, 0), r(1, 0)), cadd(r(0, -1), r(0, 1)));
  C centre = r(0, 0);
  C acc;
  acc.x = fma(R(2), edges.x, fma(R(4), centre.x, corners.x));
  acc.y = fma(R(2), edges.y, fma(R(4), centre.y, corners.y));
  return cscal(R(0.0625), acc);
}

// Full weighting onto coarse interior node (I, J), which sits on fine interior node
// (2I+1, 2J+1); all nine taps are interior nodes.
template <class C>
__device__ __forceinline__ C restrict_pt(int mx, const C* __restrict__ r, int I, int J) {
  const int c = (2 * J + 1) * mx + (2 * I + 1);
  return restrict_at<C>([&](int dx, int dy) { return __ldg(r + c + dy * mx + dx); });
}

// v + w s (w a power of two, so w s is exact and the update rounds once).
template <class C>
__device__ __forceinline__ C add_scaled(typename CT<C>::R w, C s, C v) {
  v.x = fma(w, s.x, v.x);
  v.y = fma(w, s.y, v.y);
  return v;
}

template <class C>
__device__ __forceinline__ C coarse_at(const C* __restrict__ ec, int mcx, int mcy, int K, int Kp) {
  // coarse node (K, Kp), 0..mc+1; boundary nodes carry zero
  return (K >= 1 && K <= mcx && Kp >= 1 && Kp <= mcy) ? __ldg(ec + (Kp - 1) * mcx + (K - 1))
                                                       : CT<C>::make(0.0, 0.0);
}

template <class C>
__global__ void __launch_bounds__(BX * BY) k_jacobi(StencilViewT<C> s, const C* __restrict__ u_in,
                                                    C* __restrict__ u_out, const C* __restrict__ f) {
  mgc_pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= s.mx || j >= s.my) return;
  block_kinds(s, [&](auto kx, auto ky, auto ir, auto dg) {
    u_out[j * s.mx + i] = jacobi_pt<MGC_KINDS(kx, ky, ir, dg)>(s, u_in, f, i, j);
  });
}

// First sweep from a zero initial guess: u = omega D^{-1} f.
template <class C>
__global__ void __launch_bounds__(256) k_jacobi_zero(long long n, const C* __restrict__ Dinv, C* __restrict__ u_out,
                                                    const C* __restrict__ f) {
  mgc_pdl_enter();
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < n) u_out[p] = cmul(__ldg(Dinv + p), __ldg(f + p));
}

// First sweep from a zero initial guess on the Krylov vector w, fused with its
// normalisation: v = w / sqrt(*norm2) (zeros if the norm vanishes) is written back in
// place and u = omega D^{-1} v; the same arithmetic as k_scale_by_norm then k_jacobi_zero.
// Two consecutive nodes per thread, their loads issued before the barrier (so they
// overlap thread 0's square root); for complex64 the pair is one 16-byte access per
// array when all three arrays are 16-byte aligned (the Krylov vectors and level buffers
// are), else two 8-byte ones.
template <class C>
__global__ void __launch_bounds__(256) k_scale_jacobi_zero(long long n, C* w, const double* __restrict__ norm2,
                                                          const C* __restrict__ Dinv, C* __restrict__ u_out) {
  mgc_pdl_enter();
  __shared__ double sb;
  const long long p = 2 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  C wv[2], dv[2];
  const bool vec = sizeof(C) == sizeof(float2) && p + 1 < n &&
                   ((reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(Dinv) |
                     reinterpret_cast<uintptr_t>(u_out)) & 15) == 0;
  if (vec) {
    const float4 a = *reinterpret_cast<const float4*>(w + p);
    const float4 d = __ldg(reinterpret_cast<const float4*>(Dinv + p));
    wv[0] = CT<C>::make(a.x, a.y); wv[1] = CT<C>::make(a.z, a.w);
    dv[0] = CT<C>::make(d.x, d.y); dv[1] = CT<C>::make(d.z, d.w);
  } else {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      wv[e] = p + e < n ? w[p + e] : CT<C>::make(0.0, 0.0);
      dv[e] = p + e < n ? __ldg(Dinv + p + e) : CT<C>::make(0.0, 0.0);
    }
  }
  if (threadIdx.x == 0) {
    const double b = sqrt(*norm2);
    sb = b > 0.0 ? 1.0 / b : 0.0;
  }
  __syncthreads();
  const typename CT<C>::R sc = (typename CT<C>::R)sb;
  C v[2], o[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    v[e] = cscal(sc, wv[e]);
    o[e] = cmul(dv[e], v[e]);
  }
  if (vec) {
    *reinterpret_cast<float4*>(w + p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    *reinterpret_cast<float4*>(u_out + p) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
  } else {
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (p + e < n) {
        w[p + e] = v[e];
        u_out[p + e] = o[e];
      }
  }
}

// Deterministic block reduction (fixed tree order): warp sums in the value's own
// precision R, the per-warp totals summed in FP64 by thread 0.  For complex64 data this
// keeps the FP64 pipe (1/64 of the FP32 rate here) out of the per-element work.
template <int NT, class R>
__device__ __forceinline__ double block_sum_r(R v, double* sh) {
  const int t = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((t & 31) == 0) sh[t >> 5] = (double)v;
  __syncthreads();
  double tot = 0.0;
  if (t == 0) {
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) tot += sh[w];
  }
  return tot;
}

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

template <class C>
__global__ void __launch_bounds__(BX * BY) k_residual(StencilViewT<C> s, const C* __restrict__ u,
                                                      const C* __restrict__ f, C* __restrict__ r,
                                                      double* __restrict__ norm_part) {
  mgc_pdl_enter();
  __shared__ double sh[BX * BY / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  typename CT<C>::R n2 = 0;
  if (i < s.mx && j < s.my) {
    const int p = j * s.mx + i;
    block_kinds(s, [&](auto kx, auto ky, auto ir, auto dg) {
      C rv = residual_pt<MGC_KINDS(kx, ky, ir, dg)>(s, u, f, i, j);
      if (r) r[p] = rv;
      if (norm_part) n2 = cabs2(rv);
    });
  }
  if (norm_part) {
    double tot = block_sum_r<BX * BY>(n2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) norm_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

template <class C>
__global__ void __launch_bounds__(256) k_restrict(int mx, int mcx, int mcy, const C* __restrict__ r,
                                                  C* __restrict__ rc) {
  mgc_pdl_enter();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= mcx || J >= mcy) return;
  rc[J * mcx + I] = restrict_pt(mx, r, I, J);
}

// u += bilinear interpolation of the coarse correction on the fine nodes of coarse cell
// [K, K+1] x [L, L+1] (coarse nodes; 0 and mc+1 are the boundary): the fine nodes
// k = 2K+1, 2K+2 by l = 2L+1, 2L+2 inside it share the cell's corner values and pair
// sums, so the four updates take 16 FP64 operations and need no parity branch.  The
// interpolated value at a fine node is d, (b + d)/2, (c + d)/2 or ((a + b) + (c + d))/4.
template <class C>
__device__ __forceinline__ void prolong_cell(int mx, int my, int mcx, int mcy, const C* __restrict__ ec,
                                             C* __restrict__ u, int K, int L) {
  typedef typename CT<C>::R R;
  const C a = coarse_at(ec, mcx, mcy, K, L), b = coarse_at(ec, mcx, mcy, K + 1, L);
  const C c = coarse_at(ec, mcx, mcy, K, L + 1), d = coarse_at(ec, mcx, mcy, K + 1, L + 1);
  const int i = 2 * K, j = 2 * L;             // fine interior indices of the nodes k = 2K+1, l = 2L+1
  const bool xe = i + 1 < mx, ye = j + 1 < my;  // whether k = 2K+2 (l = 2L+2) is interior
  const C cd = cadd(c, d);
  u[j * mx + i] = add_scaled(R(0.25), cadd(cadd(a, b), cd), u[j * mx + i]);
  if (xe) u[j * mx + i + 1] = add_scaled(R(0.5), cadd(b, d), u[j * mx + i + 1]);
  if (ye) {
    u[(j + 1) * mx + i] = add_scaled(R(0.5), cd, u[(j + 1) * mx + i]);
    if (xe) u[(j + 1) * mx + i + 1] = cadd(u[(j + 1) * mx + i + 1], d);
  }
}

// One thread per coarse cell (no warp diverges on the parity of a fine node).
template <class C>
__global__ void __launch_bounds__(BX * BY) k_prolong_add(int mx, int my, int mcx, int mcy, const C* __restrict__ ec,
                                                         C* __restrict__ u) {
  mgc_pdl_enter();
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = blockIdx.y * blockDim.y + threadIdx.y;
  if (K > mcx || L > mcy) return;
  prolong_cell(mx, my, mcx, mcy, ec, u, K, L);
}

// ---- fused level passes: the small levels are bound by launch latency, not by their work

// Prolongation and the first post-smoothing sweep of a level in one pass.  A block forms
// u + P e on its BX x by fine nodes and a one-node halo in shared memory (one thread per
// coarse cell, the arithmetic of prolong_cell; zero outside the interior), then applies
// the omega-Jacobi update from there.  u + P e is not stored: only the smoothed values
// are, so the results are those of k_prolong_add followed by k_jacobi.
template <class C>
__global__ void __launch_bounds__(BX * BY) k_prolong_jacobi(StencilViewT<C> s, int mcx, int mcy,
                                                            const C* __restrict__ ec, const C* __restrict__ u,
                                                            C* __restrict__ o, const C* __restrict__ f) {
  mgc_pdl_enter();
  typedef typename CT<C>::R R;
  constexpr int TW = BX + 2;
  __shared__ C T[BY + 2][TW];
  const int by = blockDim.y;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * by;
  const int tid = threadIdx.y * BX + threadIdx.x, nth = BX * by;
  for (int q = tid; q < TW * (by + 2); q += nth) T[q / TW][q % TW] = CT<C>::make(0.0, 0.0);
  __syncthreads();
  // coarse cells K (fine i = 2K, 2K+1) meeting the tile's fine range [i0 - 1, i0 + BX]
  const int K0 = (i0 - 1) >> 1, K1 = (i0 + BX) >> 1;
  const int L0 = (j0 - 1) >> 1, L1 = (j0 + by) >> 1;
  const int nkx = K1 - K0 + 1, ncell = nkx * (L1 - L0 + 1);
  for (int q = tid; q < ncell; q += nth) {
    const int K = K0 + q % nkx, L = L0 + q / nkx;
    if (K < 0 || L < 0 || K > mcx || L > mcy) continue;   // no interior fine node in the cell
    const C a = coarse_at(ec, mcx, mcy, K, L), b = coarse_at(ec, mcx, mcy, K + 1, L);
    const C c = coarse_at(ec, mcx, mcy, K, L + 1), d = coarse_at(ec, mcx, mcy, K + 1, L + 1);
    const C cd = cadd(c, d);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const int i = 2 * K + (n & 1), j = 2 * L + (n >> 1);
      if (i >= s.mx || j >= s.my || i < i0 - 1 || i > i0 + BX || j < j0 - 1 || j > j0 + by) continue;
      const C v = __ldg(u + j * s.mx + i);
      T[j - j0 + 1][i - i0 + 1] = n == 0   ? add_scaled(R(0.25), cadd(cadd(a, b), cd), v)
                                  : n == 1 ? add_scaled(R(0.5), cadd(b, d), v)
                                  : n == 2 ? add_scaled(R(0.5), cd, v)
                                           : cadd(v, d);
    }
  }
  __syncthreads();
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  if (i >= s.mx || j >= s.my) return;
  const int p = j * s.mx + i, tx = threadIdx.x + 1, ty = threadIdx.y + 1;
  block_kinds(s, [&](auto kx, auto ky, auto ir, auto dg) {
    o[p] = jacobi_vals<MGC_KINDS(kx, ky, ir, dg)>(s, i, j, p, T[ty][tx], T[ty][tx - 1], T[ty][tx + 1], T[ty - 1][tx],
                                                  T[ty + 1][tx], __ldg(f + p));
  });
}

// The residual and the full-weighting restriction of a level in one pass, from a given
// iterate u (ZERO false) or after the zero-start sweep u0 = (omega/D) f (ZERO true).  A
// block takes DBX x cby coarse nodes and runs one thread per entry of each stage, so every
// stage costs one round of memory latency: u on the fine nodes
// [2 I0 - 1, 2 I0 + 2 DBX + 1] x [2 J0 - 1, 2 J0 + 2 cby + 1] (zero outside the interior)
// into shared memory, the residuals on [2 I0, 2 I0 + 2 DBX] x [2 J0, 2 J0 + 2 cby], then the
// restriction.  With ZERO, u0 is written for the fine nodes the block owns (i >> 1 and
// j >> 1, clamped to the last coarse index, inside the block's coarse range); r is not
// stored.  The results are those of (k_jacobi_zero,) k_residual and k_restrict.
constexpr int DBX = 16, DBY = 8;
constexpr int DUW = 2 * DBX + 3, DRW = 2 * DBX + 1;

template <bool ZERO, class C>
__global__ void __launch_bounds__(DUW * (2 * DBY + 3)) k_zero_residual_restrict(StencilViewT<C> s, int mcx, int mcy,
                                                                                const C* __restrict__ f,
                                                                                C* __restrict__ u,
                                                                                C* __restrict__ fc) {
  mgc_pdl_enter();
  __shared__ C U[2 * DBY + 3][DUW];
  __shared__ C Rt[2 * DBY + 1][DRW];
  const int cby = (blockDim.x / DUW - 3) / 2;   // coarse rows of the block
  const int I0 = blockIdx.x * DBX, J0 = blockIdx.y * cby;
  const int t = threadIdx.x;
  const int rh = 2 * cby + 1;
  // f and D of this thread's residual node, loaded with the tile so that the pass waits
  // on memory once
  const int ra = t % DRW, rb = t / DRW, ri = 2 * I0 + ra, rj = 2 * J0 + rb;
  const bool rown = t < DRW * rh && ri < s.mx && rj < s.my;
  const int rp = rj * s.mx + ri;
  C rf = CT<C>::make(0.0, 0.0), rd = rf;
  if (rown) {
    rf = __ldg(f + rp);
    rd = __ldg(s.D + rp);
  }
  {
    const int a = t % DUW, b = t / DUW;
    const int i = 2 * I0 - 1 + a, j = 2 * J0 - 1 + b;
    C v = CT<C>::make(0.0, 0.0);
    if (i >= 0 && j >= 0 && i < s.mx && j < s.my) {
      const int p = j * s.mx + i;
      if constexpr (ZERO) {
        v = cmul(__ldg(s.Dinv + p), __ldg(f + p));
        const int oi = min(i >> 1, mcx - 1), oj = min(j >> 1, mcy - 1);
        if (oi >= I0 && oi < I0 + DBX && oj >= J0 && oj < J0 + cby) u[p] = v;
      } else {
        v = __ldg(u + p);
      }
    }
    U[b][a] = v;
  }
  __syncthreads();
  if (rown) {
    const int a = ra, b = rb;
    dispatch_kinds(s, 2 * I0, min(2 * I0 + DRW, s.mx), 2 * J0, min(2 * J0 + rh, s.my),
                   [&](auto kx, auto ky, auto ir, auto dg) {
                     Rt[b][a] = residual_vals_d<MGC_KINDS(kx, ky, ir, dg)>(
                         s, ri, rj, rd, U[b + 1][a + 1], U[b + 1][a], U[b + 1][a + 2], U[b][a + 1], U[b + 2][a + 1],
                         rf);
                   });
  }
  __syncthreads();
  if (t < DBX * cby) {
    const int I = I0 + t % DBX, J = J0 + t / DBX;
    if (I < mcx && J < mcy) {
      const int a = 2 * (t % DBX) + 1, b = 2 * (t / DBX) + 1;   // (2I+1, 2J+1) in Rt
      fc[J * mcx + I] = restrict_at<C>([&](int dx, int dy) { return Rt[b + dy][a + dx]; });
    }
  }
}

// ---- complex64 residual + restriction from a given iterate, as a gather.  On the FP32
// pipe recomputing neighbour values costs little, so one thread per coarse node (I, J) on
// the fine node (2I+1, 2J+1) loads u on the 21 fine nodes its nine residuals read
// (|dx|, |dy| <= 2 without the corners), f and D at the nine nodes -- all loads
// independent and issued before any arithmetic -- and forms the nine residuals and their
// weighted sum without shared memory or a barrier.  Same per-node arithmetic as the tiled
// pass, so the same results.  Measured against the tiled pass: equal at 1024^2 (13.3
// against 13.7 us), faster at 2048^2 (33.9 against 40 us); the same gather for the
// zero-start form, and a gather form of the prolongation pass, were slower (the small
// levels have too few coarse nodes per SM, the prolongation reloads its coarse values per
// node), so those keep their tiles.
constexpr int RG_BY = 4;

template <class C>
__global__ void __launch_bounds__(BX * RG_BY) k_residual_restrict_gather(StencilViewT<C> s, int mcx, int mcy,
                                                                         const C* __restrict__ f,
                                                                         const C* __restrict__ u, C* __restrict__ fc) {
  mgc_pdl_enter();
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * RG_BY + threadIdx.y;
  if (I >= mcx || J >= mcy) return;
  const int ic = 2 * I + 1, jc = 2 * J + 1;
  C U[5][5], F[3][3], Dd[3][3];
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      if ((dx == -2 || dx == 2) && (dy == -2 || dy == 2)) continue;
      const int fi = ic + dx, fj = jc + dy;
      const bool in = fi >= 0 && fj >= 0 && fi < s.mx && fj < s.my;
      const int q = fj * s.mx + fi;
      U[dy + 2][dx + 2] = ldz(u, q, in);
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
        F[dy + 1][dx + 1] = ldz(f, q, in);
        Dd[dy + 1][dx + 1] = ldz(s.D, q, in);
      }
    }
  C R[3][3];
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * RG_BY;
  dispatch_kinds(s, 2 * I0, min(2 * I0 + 2 * BX + 1, s.mx), 2 * J0, min(2 * J0 + 2 * RG_BY + 1, s.my),
                 [&](auto kx, auto ky, auto ir, auto dg) {
#pragma unroll
                   for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                     for (int dx = -1; dx <= 1; ++dx) {
                       const int a = dx + 2, b = dy + 2;
                       R[dy + 1][dx + 1] = residual_vals_d<MGC_KINDS(kx, ky, ir, dg)>(
                           s, ic + dx, jc + dy, Dd[dy + 1][dx + 1], U[b][a], U[b][a - 1], U[b][a + 1], U[b - 1][a],
                           U[b + 1][a], F[dy + 1][dx + 1]);
                     }
                 });
  fc[J * mcx + I] = restrict_at<C>([&](int dx, int dy) { return R[dy + 1][dx + 1]; });
}

// Coarsest level: u = A_c^{-1} f with the FP64 dense inverse built at setup, accumulated
// in FP64 for either element type; the FP64 pipe (2 DFMA per clock per SM) bounds the
// 4 nc^2 operations.  One block of CS_THREADS threads per row, so the block scheduler
// spreads the rows evenly over the SMs; thread t takes columns t, t + CS_THREADS, ... (f
// read through L1, complex64 f widened as it is used), and the warps of the ~6 rows each
// SM holds hide the load latency.  Two warps per row keep the shuffle reduction (10 FP64
// adds a thread) small
// beside the 4 x 16 FMAs of each thread; with four warps per row it cost a third of the
// FMA work, and one warp per row of four per block left SMs idle.
constexpr int CS_THREADS = 64, CS_UNROLL = (MGC_MAX_COARSE + CS_THREADS - 1) / CS_THREADS;

template <class C>
__global__ void __launch_bounds__(CS_THREADS) k_coarse_solve(int nc, const cplx* __restrict__ Ainv,
                                                              const C* __restrict__ f, C* __restrict__ u) {
  mgc_pdl_enter();
  __shared__ double sh[2][CS_THREADS / 32];
  const int row = blockIdx.x, t = threadIdx.x;
  const cplx* __restrict__ a = Ainv + (size_t)row * nc;
  cplx av[CS_UNROLL];
  C fv[CS_UNROLL];
#pragma unroll
  for (int q = 0; q < CS_UNROLL; ++q) {
    const int c = t + q * CS_THREADS;
    const bool ok = c < nc;
    av[q] = ok ? __ldg(a + c) : cmk(0.0, 0.0);
    fv[q] = ok ? __ldg(f + c) : CT<C>::make(0.0, 0.0);
  }
  cplx acc0 = cmk(0.0, 0.0), acc1 = cmk(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < CS_UNROLL; q += 2) {
    acc0 = cfma(av[q], to_c128(fv[q]), acc0);
    acc1 = cfma(av[q + 1], to_c128(fv[q + 1]), acc1);
  }
  acc0 = cadd(acc0, acc1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc0.x += __shfl_down_sync(0xffffffffu, acc0.x, o);
    acc0.y += __shfl_down_sync(0xffffffffu, acc0.y, o);
  }
  if ((t & 31) == 0) {
    sh[0][t >> 5] = acc0.x;
    sh[1][t >> 5] = acc0.y;
  }
  __syncthreads();
  if (t == 0) {
    cplx tot = cmk(0.0, 0.0);
#pragma unroll
    for (int w = 0; w < CS_THREADS / 32; ++w) tot = cadd(tot, cmk(sh[0][w], sh[1][w]));
    u[row] = CT<C>::make(tot.x, tot.y);
  }
}


// Sum of n partials in a fixed order (one block), result to out[0]; skipped when
// `gate` is given and *gate == 0.
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ part, int n,
                                                      double* __restrict__ out, const int* __restrict__ gate) {
  mgc_pdl_enter();
  __shared__ double sh[8];
  if (gate && *gate == 0) return;
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) v += part[k];
  double tot = block_sum<256>(v, sh);
  if (threadIdx.x == 0) out[0] = tot;
}

template <class C>
__global__ void __launch_bounds__(256) k_norm2(const C* __restrict__ v, long long n, double* __restrict__ part) {
  mgc_pdl_enter();
  __shared__ double sh[8];
  typename CT<C>::R acc = 0;
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256)
    acc += cabs2(__ldg(v + p));
  double tot = block_sum_r<256>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class C>
__global__ void __launch_bounds__(BX * BY) k_apply(StencilViewT<C> s, const C* __restrict__ x, C* __restrict__ y,
                                                   double* __restrict__ norm_part) {
  mgc_pdl_enter();
  __shared__ double sh[BX * BY / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  typename CT<C>::R n2 = 0;
  if (i < s.mx && j < s.my) {
    const int p = j * s.mx + i;
    block_kinds(s, [&](auto kx, auto ky, auto ir, auto dg) {
      C v = apply_pt<MGC_KINDS(kx, ky, ir, dg)>(s, x, i, j, __ldg(x + p));
      y[p] = v;
      if (norm_part) n2 = cabs2(v);
    });
  }
  if (norm_part) {
    double tot = block_sum_r<BX * BY>(n2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) norm_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

// y32 = (x64 * scale) rounded to complex64, scale = 1/sqrt(*norm2) (1 when norm2 is null).
__global__ void __launch_bounds__(256) k_demote(long long n, const cplx* __restrict__ x, const double* __restrict__ norm2,
                                                float2* __restrict__ y) {
  mgc_pdl_enter();
  __shared__ double s_sh;
  if (threadIdx.x == 0) s_sh = norm2 ? (*norm2 > 0.0 ? 1.0 / sqrt(*norm2) : 0.0) : 1.0;
  __syncthreads();
  const double s = s_sh;
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256) {
    cplx v = __ldg(x + p);
    y[p] = make_float2((float)(s * v.x), (float)(s * v.y));
  }
}

// u64 += sqrt(*norm2) * e32 (the iterative-refinement update in FP64).
__global__ void __launch_bounds__(256) k_promote_add(long long n, const float2* __restrict__ e,
                                                     const double* __restrict__ norm2, cplx* __restrict__ u) {
  mgc_pdl_enter();
  __shared__ double s_sh;
  if (threadIdx.x == 0) s_sh = sqrt(*norm2);
  __syncthreads();
  const double s = s_sh;
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256) {
    float2 v = __ldg(e + p);
    cplx a = u[p];
    u[p] = cmk(fma(s, (double)v.x, a.x), fma(s, (double)v.y, a.y));
  }
}

// y64 = x32 (exact widening).
__global__ void __launch_bounds__(256) k_promote(long long n, const float2* __restrict__ x, cplx* __restrict__ y) {
  mgc_pdl_enter();
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256)
    y[p] = to_c128(__ldg(x + p));
}

// b32 = a64 rounded (setup: single-precision copies of coefficients and states).
__global__ void __launch_bounds__(256) k_round_copy(long long n, const cplx* __restrict__ a, float2* __restrict__ b) {
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < n; p += (long long)gridDim.x * 256)
    b[p] = make_float2((float)a[p].x, (float)a[p].y);
}

inline dim3 grid2(int mx, int my) { return dim3((mx + BX - 1) / BX, (my + BY - 1) / BY); }

// Block height for a level of mx x my nodes: 64-thread blocks below two full 256-thread
// blocks per SM, so the work of a small level spreads over more SMs' FP64 pipes.
// small_rows: the handle's tile-rows setting (0 = 2)
inline bool small_level(int mx, int my) { return (long long)mx * my < 2LL * mgc_sm_count() * BX * BY; }
inline int level_by(int mx, int my, int small_rows = 0) {
  return small_level(mx, my) ? (small_rows > 0 ? small_rows : 2) : BY;
}
inline dim3 level_grid(int mx, int my, int by) { return dim3((mx + BX - 1) / BX, (my + by - 1) / by); }

inline unsigned stride_blocks(long long n) {
  const long long b = (n + 255) / 256, cap = 8LL * mgc_sm_count();
  return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

template <class C>
cudaError_t launch_jacobi(const StencilViewT<C>& s, const C* u_in, C* u_out, const C* f, cudaStream_t st) {
  const int by = level_by(s.mx, s.my, s.tile_rows);
  return mgc_launch(k_jacobi<C>, level_grid(s.mx, s.my, by), dim3(BX, by), 0, st, s, u_in, u_out, f);
}

template <class C>
cudaError_t launch_jacobi_zero(const StencilViewT<C>& s, C* u_out, const C* f, cudaStream_t st) {
  long long n = (long long)s.mx * s.my;
  return mgc_launch(k_jacobi_zero<C>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, n, s.Dinv, u_out, f);
}

template <class C>
cudaError_t launch_scale_jacobi_zero(const StencilViewT<C>& s, C* w, const double* norm2, C* u_out,
                                     cudaStream_t st) {
  long long n = (long long)s.mx * s.my;
  return mgc_launch(k_scale_jacobi_zero<C>, dim3((unsigned)((n + 511) / 512)), dim3(256), 0, st, n, w, norm2, s.Dinv,
                    u_out);
}

template <class C>
int residual_norm_blocks(const StencilViewT<C>& s) {
  dim3 g = grid2(s.mx, s.my);
  return (int)(g.x * g.y);
}

template <class C>
cudaError_t launch_residual(const StencilViewT<C>& s, const C* u, const C* f, C* r, double* norm_part,
                            cudaStream_t st) {
  const int by = norm_part ? BY : level_by(s.mx, s.my, s.tile_rows);   // norm partials: one per full block
  return mgc_launch(k_residual<C>, level_grid(s.mx, s.my, by), dim3(BX, by), 0, st, s, u, f, r, norm_part);
}

template <class C>
cudaError_t launch_restrict(int mx, int my, const C* r, C* rc, cudaStream_t st) {
  int mcx = (mx - 1) / 2, mcy = (my - 1) / 2;
  const int by = level_by(mcx, mcy);
  return mgc_launch(k_restrict<C>, level_grid(mcx, mcy, by), dim3(BX, by), 0, st, mx, mcx, mcy, r, rc);
}

template <class C>
cudaError_t launch_prolong_jacobi(const StencilViewT<C>& s, const C* ec, const C* u, C* o, const C* f,
                                  cudaStream_t st) {
  const int mcx = (s.mx - 1) / 2, mcy = (s.my - 1) / 2;
  if (s.mx != 2 * mcx + 1 || s.my != 2 * mcy + 1) return cudaErrorInvalidValue;
  const int by = level_by(s.mx, s.my, s.tile_rows);
  return mgc_launch(k_prolong_jacobi<C>, level_grid(s.mx, s.my, by), dim3(BX, by), 0, st, s, mcx, mcy, ec, u, o, f);
}

template <class C>
cudaError_t launch_zero_residual_restrict(const StencilViewT<C>& s, const C* f, C* u, C* fc, bool zero,
                                          cudaStream_t st) {
  const int mcx = (s.mx - 1) / 2, mcy = (s.my - 1) / 2;
  if (s.mx != 2 * mcx + 1 || s.my != 2 * mcy + 1) return cudaErrorInvalidValue;
  if constexpr (sizeof(C) == sizeof(float2)) {
    if (!zero) {
      const dim3 g((mcx + BX - 1) / BX, (mcy + RG_BY - 1) / RG_BY), b(BX, RG_BY);
      return mgc_launch(k_residual_restrict_gather<C>, g, b, 0, st, s, mcx, mcy, f, (const C*)u, fc);
    }
  }
  const int cby = (long long)mcx * mcy < 2LL * mgc_sm_count() * DBX * DBY ? (s.tile_rows > 0 ? s.tile_rows : 2) : DBY;
  const dim3 grid((mcx + DBX - 1) / DBX, (mcy + cby - 1) / cby);
  const dim3 block(DUW * (2 * cby + 3));
  if (zero) return mgc_launch(k_zero_residual_restrict<true, C>, grid, block, 0, st, s, mcx, mcy, f, u, fc);
  return mgc_launch(k_zero_residual_restrict<false, C>, grid, block, 0, st, s, mcx, mcy, f, u, fc);
}

template <class C>
cudaError_t launch_prolong_add(int mx, int my, const C* ec, C* u, cudaStream_t st) {
  int mcx = (mx - 1) / 2, mcy = (my - 1) / 2;
  if (mx != 2 * mcx + 1 || my != 2 * mcy + 1) return cudaErrorInvalidValue;   // coarse = every other fine node
  const int by = level_by(mcx + 1, mcy + 1);
  return mgc_launch(k_prolong_add<C>, dim3((mcx + BX) / BX, (mcy + by) / by), dim3(BX, by), 0, st, mx, my, mcx, mcy,
                    ec, u);
}

template <class C>
cudaError_t launch_coarse_solve(int nc, const cplx* Ainv, const C* f, C* u, cudaStream_t st) {
  if (nc < 1 || nc > MGC_MAX_COARSE) return cudaErrorInvalidValue;
  return mgc_launch(k_coarse_solve<C>, dim3(nc), dim3(CS_THREADS), 0, st, nc, Ainv, f, u);
}


template <class C>
cudaError_t launch_apply(const StencilViewT<C>& s, const C* x, C* y, cudaStream_t st, double* norm_part) {
  const int by = norm_part ? BY : level_by(s.mx, s.my, s.tile_rows);
  return mgc_launch(k_apply<C>, level_grid(s.mx, s.my, by), dim3(BX, by), 0, st, s, x, y, norm_part);
}

template <class C>
cudaError_t launch_norm2(const C* v, long long n, double* part, int nblocks, cudaStream_t st) {
  return mgc_launch(k_norm2<C>, dim3(nblocks), dim3(256), 0, st, v, n, part);
}

#define MGC_INSTANTIATE(C)                                                                                  \
  template cudaError_t launch_jacobi<C>(const StencilViewT<C>&, const C*, C*, const C*, cudaStream_t);     \
  template cudaError_t launch_jacobi_zero<C>(const StencilViewT<C>&, C*, const C*, cudaStream_t);          \
  template cudaError_t launch_scale_jacobi_zero<C>(const StencilViewT<C>&, C*, const double*, C*,          \
                                                   cudaStream_t);                                         \
  template int residual_norm_blocks<C>(const StencilViewT<C>&);                                           \
  template cudaError_t launch_residual<C>(const StencilViewT<C>&, const C*, const C*, C*, double*,        \
                                          cudaStream_t);                                                  \
  template cudaError_t launch_restrict<C>(int, int, const C*, C*, cudaStream_t);                          \
  template cudaError_t launch_prolong_add<C>(int, int, const C*, C*, cudaStream_t);                       \
  template cudaError_t launch_prolong_jacobi<C>(const StencilViewT<C>&, const C*, const C*, C*, const C*,   \
                                               cudaStream_t);                                            \
  template cudaError_t launch_zero_residual_restrict<C>(const StencilViewT<C>&, const C*, C*, C*, bool,      \
                                                        cudaStream_t);                                   \
  template cudaError_t launch_coarse_solve<C>(int, const cplx*, const C*, C*, cudaStream_t);              \
  template cudaError_t launch_apply<C>(const StencilViewT<C>&, const C*, C*, cudaStream_t, double*);      \
  template cudaError_t launch_norm2<C>(const C*, long long, double*, int, cudaStream_t);
MGC_INSTANTIATE(double2)
MGC_INSTANTIATE(float2)
#undef MGC_INSTANTIATE

cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t st, const int* gate) {
  return mgc_launch(k_sum_partials, dim3(1), dim3(256), 0, st, part, n, out, gate);
}

int norm2_blocks(long long n) {
  const long long b = (n + 255) / 256, cap = 8LL * mgc_sm_count();
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

cudaError_t launch_demote(long long n, const cplx* x, const double* norm2, float2* y, cudaStream_t st) {
  return mgc_launch(k_demote, dim3(stride_blocks(n)), dim3(256), 0, st, n, x, norm2, y);
}

cudaError_t launch_promote_add(long long n, const float2* e, const double* norm2, cplx* u, cudaStream_t st) {
  return mgc_launch(k_promote_add, dim3(stride_blocks(n)), dim3(256), 0, st, n, e, norm2, u);
}

cudaError_t launch_promote(long long n, const float2* x, cplx* y, cudaStream_t st) {
  return mgc_launch(k_promote, dim3(stride_blocks(n)), dim3(256), 0, st, n, x, y);
}

cudaError_t launch_round_copy(long long n, const cplx* a, float2* b, cudaStream_t st) {
  k_round_copy<<<stride_blocks(n), 256, 0, st>>>(n, a, b);
  return cudaGetLastError();
}
