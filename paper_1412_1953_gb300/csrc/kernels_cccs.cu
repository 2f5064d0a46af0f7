// Coupled Channel Correction Step kernels (Sec. 4 of Cools & Vanroose).
//
//   residual r = f - (H - E) u                                   (Sec. 4.3)
//   P^x_i(y) = sum_x w phi_i r,  P^y_j(x) = sum_y w vphi_j r      (projections, Sec. 4.1)
//   c_ij = sum_y w vphi_j P^x_i = a_ji + b_ij                     (Eq. (27))
//   a_ji = c_ij (j <= i), b_ij = c_ij (j > i)                     (Eqs. (25)-(26))
//   r^A_i = P^x_i - sum_{l>i} c_il vphi_l,  r^B_j = P^y_j - sum_{m>=j} c_mj phi_m
//   coupled-channel solves for e^A, e^B                           (Eqs. (28)-(29))
//   u += sum_m phi_m(x) e^A_m(y) + sum_l e^B_l(x) vphi_l(y)       (Eq. (30))
//
// The projections are fused into the residual pass and reduced deterministically:
// per 32 x 32 tile, sums along x and along y through a shared-memory tile give
// per-tile partials, which a second kernel sums in a fixed order.
#include <cooperative_groups.h>

#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TX = 32;        // tile width (one warp per row)
constexpr int WY = 8;         // warps per block
constexpr int SY = 4;         // rows per warp
constexpr int TY = WY * SY;   // tile height

template <class C>
__device__ __forceinline__ C ldz(const C* __restrict__ a, int p, bool ok) {
  return ok ? __ldg(a + p) : CT<C>::make(0.0, 0.0);
}

template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C residual_at(const StencilViewT<C>& s, const C* __restrict__ u, const C* __restrict__ f,
                                         int i, int j) {
  const int p = j * s.mx + i;
  return residual_vals<KX, KY, IR, DG>(s, i, j, p, __ldg(u + p), ldz(u, p - 1, i > 0), ldz(u, p + 1, i + 1 < s.mx),
                                       ldz(u, p - s.mx, j > 0), ldz(u, p + s.mx, j + 1 < s.my), __ldg(f + p));
}

// One 32 x 32 tile per block: each thread computes the residual at four nodes into a
// padded shared tile; then, with the tile transposed through shared memory, one thread
// per (row, state) sums P^x over the tile's 32 columns and one thread per (column,
// state) sums P^y over its 32 rows.  Each residual costs 4 n_b FP64 FMAs of projection
// work and no shuffle reductions.
template <int NB, class C>
__global__ void __launch_bounds__(TX * WY) k_residual_project(StencilViewT<C> s, CCViewT<C> c, const C* __restrict__ u,
                                                              const C* __restrict__ f) {
  mgc_pdl_enter();
  __shared__ C R[TY][TX + 1];
  const int lane = threadIdx.x;
  const int wy = threadIdx.y;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int i = i0 + lane;
  dispatch_kinds(s, i0, min(i0 + TX, s.mx), j0, min(j0 + TY, s.my), [&](auto kx, auto ky, auto ir, auto dg) {
    for (int q = 0; q < SY; ++q) {
      const int row = q * WY + wy;
      const int j = j0 + row;
      R[row][lane] = (i < s.mx && j < s.my)
                         ? residual_at<decltype(kx)::value, decltype(ky)::value, decltype(ir)::value,
                                       decltype(dg)::value>(s, u, f, i, j)
                         : CT<C>::make(0.0, 0.0);
    }
  });
  __syncthreads();
  const int t = wy * TX + lane;
  for (int w = t; w < 2 * TX * NB; w += TX * WY) {
    if (w < TX * NB) {
      // P^x partial: row `row`, state m, over the tile's columns
      const int m = w / TX, row = w % TX;
      const int ncol = min(TX, s.mx - i0);
      const C* wp = c.wphi + (size_t)m * s.mx + i0;
      C acc = CT<C>::make(0.0, 0.0);
      for (int cc = 0; cc < ncol; ++cc) acc = cfma(__ldg(wp + cc), R[row][cc], acc);
      if (j0 + row < s.my) c.Px_part[((size_t)blockIdx.x * NB + m) * s.my + j0 + row] = acc;
    } else {
      // P^y partial: column `col`, state l, over the tile's rows
      const int w2 = w - TX * NB;
      const int l = w2 / TX, col = w2 % TX;
      const int nrow = min(TY, s.my - j0);
      const C* wv = c.wvphi + (size_t)l * s.my + j0;
      C acc = CT<C>::make(0.0, 0.0);
      for (int rr = 0; rr < nrow; ++rr) acc = cfma(__ldg(wv + rr), R[rr][col], acc);
      if (i0 + col < s.mx) c.Py_part[((size_t)blockIdx.y * NB + l) * s.mx + i0 + col] = acc;
    }
  }
}

// Sum the per-tile partials (in FP64 for either partial type): eight lanes per output
// each sum a strided subset of tiles, then a fixed shuffle tree adds the eight.
template <class C>
__global__ void __launch_bounds__(256) k_reduce_partials(int nb, int mx, int my, int ntx, int nty,
                                                         const C* __restrict__ Px_part,
                                                         const C* __restrict__ Py_part,
                                                         cplx* __restrict__ Px, cplx* __restrict__ Py) {
  mgc_pdl_enter();
  const int g = blockIdx.x * 256 + threadIdx.x;
  const int t = g >> 3, sub = g & 7;
  const int nx_tot = nb * my, ny_tot = nb * mx;
  cplx acc = cmk(0.0, 0.0);
  if (t < nx_tot) {
    for (int k = sub; k < ntx; k += 8) acc = cadd(acc, to_c128(Px_part[(size_t)k * nx_tot + t]));
  } else if (t < nx_tot + ny_tot) {
    const int q = t - nx_tot;
    for (int k = sub; k < nty; k += 8) acc = cadd(acc, to_c128(Py_part[(size_t)k * ny_tot + q]));
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, 8);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, 8);
  }
  if (sub == 0) {
    if (t < nx_tot) Px[t] = acc;
    else if (t < nx_tot + ny_tot) Py[t - nx_tot] = acc;
  }
}

// c[a][b] = sum_j w_y(j) vphi_b(j) P^x_a(j): one block per (a, b).
__global__ void __launch_bounds__(256) k_cc_coef(int nb, int my, const cplx* __restrict__ wvphi,
                                                 const cplx* __restrict__ Px, cplx* __restrict__ cmat) {
  mgc_pdl_enter();
  __shared__ double sh[2][8];
  const int a = blockIdx.x / nb, b = blockIdx.x % nb;
  cplx acc = cmk(0.0, 0.0);
  for (int j = threadIdx.x; j < my; j += 256) acc = cfma(__ldg(wvphi + b * my + j), __ldg(Px + a * my + j), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc.x; sh[1][threadIdx.x >> 5] = acc.y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx tot = cmk(0.0, 0.0);
    for (int w = 0; w < 8; ++w) tot = cadd(tot, cmk(sh[0][w], sh[1][w]));
    cmat[a * nb + b] = tot;
  }
}

// Coupled-channel solves (Eqs. (28)-(29)) by parallel cyclic reduction with setup-time
// factors: each system is solved by one thread-block cluster of CR_CLUSTER CTAs (cluster
// 0: channel A along y, cluster 1: channel B along x); every level is one pass over the
// (row, component) pairs split across the cluster.  Levels are separated by split
// cluster barriers: every thread arrives (release) after its stores, loads the read-only
// factor rows of its first item of the next level, and only then waits (acquire), so
// the factor loads overlap the barrier.  Arrive and wait sit outside all data-dependent
// branches, so each warp executes them convergently.  Sums are formed as independent
// length-nb dot products, which keeps the dependent FP64 chain short.
constexpr int CR_CLUSTER = 16;           // non-portable size: allowed per kernel at setup
constexpr int CR_THREADS = 256;

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <int NB>
__device__ __forceinline__ void load_row(cplx (&d)[NB], const cplx* __restrict__ src) {
#pragma unroll
  for (int p = 0; p < NB; ++p) d[p] = __ldg(src + p);
}

template <int NB>
__device__ __forceinline__ cplx dot_row(const cplx (&a)[NB], const cplx* x) {
  cplx s = cmul(a[0], x[0]);
#pragma unroll
  for (int p = 1; p < NB; ++p) s = cfma(a[p], x[p], s);
  return s;
}

// Level l (stride s = 2^l) updates every row, x_k <- x_k - pa_k x_{k-s} - pg_k x_{k+s}
// (X and Y alternate); after ceil(log2 m) levels x_k = pbinv_k x_k.  Against block cyclic
// reduction (2 log2 m dependent levels on half the rows) this halves the dependent levels
// for log2(m)/2 times the arithmetic, which 16-CTA clusters absorb: 37 us against 57 us
// per CCCS at 1023 rows, n_b = 3.
// Rows per CTA when one 16-CTA cluster holds the m block rows of a system.
__host__ __device__ __forceinline__ int cr_rows(int m) { return (m + CR_CLUSTER - 1) / CR_CLUSTER; }

// One system per 16-CTA cluster.  CTA `rank` owns block rows [rank R, rank R + R) and keeps
// their current right-hand sides in its shared memory (two buffers, one per parity of the
// level); a level reads rows k - s and k + s from the shared memory of the CTAs that own
// them (distributed shared memory), and the split cluster barrier between levels orders
// those reads against the next level's writes.  The factor rows of the next level are
// fetched between the barrier's arrive and wait.
template <int NB>
__global__ void __cluster_dims__(CR_CLUSTER, 1, 1) __launch_bounds__(CR_THREADS)
k_channel_solve_pcr(CRSystem SA, CRSystem SB) {
  mgc_pdl_enter();
  extern __shared__ cplx cr_x[];   // [2][R * NB]
  cg::cluster_group cl = cg::this_cluster();
  const int sys = blockIdx.x / CR_CLUSTER;
  const int rank = (int)cl.block_rank();
  const CRSystem S = sys == 0 ? SA : SB;
  constexpr int nb2 = NB * NB;
  const int m = S.m, pq = S.pq;
  const int R = cr_rows(m), nloc = R * NB, k0 = rank * R;
  cplx* X = cr_x;
  cplx* Y = cr_x + nloc;
  // the channel right-hand sides with the uniqueness conventions (Eqs. (25)-(26))
  for (int e = threadIdx.x; e < nloc; e += CR_THREADS) {
    const int k = k0 + e / NB, comp = e % NB;
    cplx v = cmk(0.0, 0.0);
    if (k < m) {
      v = S.P[comp * m + k];
      if (S.chan == 0) {
        for (int l = comp + 1; l < NB; ++l) v = cfms(S.cmat[comp * NB + l], __ldg(S.basis + l * m + k), v);   // b_al
      } else {
        for (int l = comp; l < NB; ++l) v = cfms(S.cmat[l * NB + comp], __ldg(S.basis + l * m + k), v);       // a_bl
      }
    }
    X[e] = v;
  }
  cluster_arrive();
  const int e0 = threadIdx.x, kf = k0 + e0 / NB;
  const bool first_ok = e0 < nloc && kf < m;
  cplx fa[NB], fb[NB];
  for (int l = 0; l < pq; ++l) {
    const int s = 1 << l;
    const cplx* pa = S.pa + (size_t)l * m * nb2;
    const cplx* pg = S.pg + (size_t)l * m * nb2;
    if (first_ok) {
      const size_t fo = (size_t)kf * nb2 + (e0 % NB) * NB;
      load_row<NB>(fa, pa + fo);
      load_row<NB>(fb, pg + fo);
    }
    cluster_wait();
    for (int e = e0; e < nloc; e += CR_THREADS) {
      const int k = k0 + e / NB, comp = e % NB;
      if (k >= m) break;
      if (e != e0) {
        const size_t fo = (size_t)k * nb2 + comp * NB;
        load_row<NB>(fa, pa + fo);
        load_row<NB>(fb, pg + fo);
      }
      cplx acc = X[e];
      if (k - s >= 0) {
        const int q = (k - s) / R;
        acc = csub(acc, dot_row<NB>(fa, cl.map_shared_rank(X + (k - s - q * R) * NB, q)));
      }
      if (k + s < m) {
        const int q = (k + s) / R;
        acc = csub(acc, dot_row<NB>(fb, cl.map_shared_rank(X + (k + s - q * R) * NB, q)));
      }
      Y[e] = acc;
    }
    cluster_arrive();
    cplx* t = X; X = Y; Y = t;
  }
  if (first_ok) load_row<NB>(fa, S.pbinv + (size_t)kf * nb2 + (e0 % NB) * NB);
  cluster_wait();   // every CTA is past its last remote read: each now reads only its own rows
  for (int e = e0; e < nloc; e += CR_THREADS) {
    const int k = k0 + e / NB, comp = e % NB;
    if (k >= m) break;
    if (e != e0) load_row<NB>(fa, S.pbinv + (size_t)k * nb2 + comp * NB);
    const cplx v = dot_row<NB>(fa, X + (e / NB) * NB);
    S.e[comp * m + k] = v;
    if (S.e32) S.e32[comp * m + k] = make_float2((float)v.x, (float)v.y);
  }
}

// u += sum_m phi_m(x) e^A_m(y) + sum_l e^B_l(x) vphi_l(y) (Eq. (30)).  A thread takes one
// column i and cc_rows<C>() consecutive rows: phi_m(i) and e^B_l(i) stay in registers
// across its rows (per node only the warp-uniform e^A_m(j), vphi_l(j) are loaded), and the
// loads of its values of u are issued together, so a complex64 warp has 8 x 256 bytes of u
// in flight (the complex64 pass is bound by how much of u is in flight).  Same sums in the
// same order per node.  Rows per thread: 8 for complex64 (memory-bound), 4 for complex128
// (FP64-bound, where the register cost of more rows would only lower occupancy).
template <class C>
__host__ __device__ constexpr int cc_rows() { return sizeof(C) == sizeof(float2) ? 8 : 4; }

template <int NB, class C>
__global__ void __launch_bounds__(256) k_cccs_correct(int mx, int my, const C* __restrict__ phi,
                                                      const C* __restrict__ vphi, const C* __restrict__ eA,
                                                      const C* __restrict__ eB, C* __restrict__ u) {
  mgc_pdl_enter();
  const int i = blockIdx.x * 32 + threadIdx.x;
  constexpr int CC_ROWS = cc_rows<C>();
  const int j0 = (blockIdx.y * 8 + threadIdx.y) * CC_ROWS;
  if (i >= mx || j0 >= my) return;
  C a[NB], b[NB];
#pragma unroll
  for (int m = 0; m < NB; ++m) {
    a[m] = __ldg(phi + m * mx + i);
    b[m] = __ldg(eB + m * mx + i);
  }
  C v[CC_ROWS];
#pragma unroll
  for (int r = 0; r < CC_ROWS; ++r)
    if (j0 + r < my) v[r] = u[(j0 + r) * mx + i];
#pragma unroll
  for (int r = 0; r < CC_ROWS; ++r) {
    const int j = j0 + r;
    if (j >= my) break;
    C w = v[r];
#pragma unroll
    for (int m = 0; m < NB; ++m) w = cfma(a[m], __ldg(eA + m * my + j), w);
#pragma unroll
    for (int l = 0; l < NB; ++l) w = cfma(b[l], __ldg(vphi + l * my + j), w);
    u[j * mx + i] = w;
  }
}

template <int NB, class C>
cudaError_t rp_launch(const StencilViewT<C>& s, const CCViewT<C>& c, const C* u, const C* f, cudaStream_t st) {
  dim3 g(cc_tiles_x(s.mx), cc_tiles_y(s.my));
  return mgc_launch(k_residual_project<NB, C>, g, dim3(TX, WY), 0, st, s, c, u, f);
}

template <int NB, class C>
cudaError_t corr_launch(const CCViewT<C>& c, C* u, cudaStream_t st) {
  dim3 g((c.mx + 31) / 32, (c.my + 8 * cc_rows<C>() - 1) / (8 * cc_rows<C>()));
  return mgc_launch(k_cccs_correct<NB, C>, g, dim3(32, 8), 0, st, c.mx, c.my, c.phi, c.vphi, c.eAc, c.eBc, u);
}

}  // namespace

int cc_tiles_x(int mx) { return (mx + TX - 1) / TX; }
int cc_tiles_y(int my) { return (my + TY - 1) / TY; }

template <class C>
cudaError_t launch_residual_project(const StencilViewT<C>& s, const CCViewT<C>& c, const C* u, const C* f,
                                    cudaStream_t st) {
  switch (c.nb) {
    case 1: return rp_launch<1, C>(s, c, u, f, st);
    case 2: return rp_launch<2, C>(s, c, u, f, st);
    case 3: return rp_launch<3, C>(s, c, u, f, st);
    case 4: return rp_launch<4, C>(s, c, u, f, st);
    case 5: return rp_launch<5, C>(s, c, u, f, st);
    case 6: return rp_launch<6, C>(s, c, u, f, st);
    case 7: return rp_launch<7, C>(s, c, u, f, st);
    case 8: return rp_launch<8, C>(s, c, u, f, st);
  }
  return cudaErrorInvalidValue;
}

template <class C>
cudaError_t launch_cc_rhs(const CCViewT<C>& c, cudaStream_t st) {
  int tot = c.nb * (c.mx + c.my);
  cudaError_t e = mgc_launch(k_reduce_partials<C>, dim3((8 * tot + 255) / 256), dim3(256), 0, st, c.nb, c.mx, c.my,
                             cc_tiles_x(c.mx), cc_tiles_y(c.my), c.Px_part, c.Py_part, c.Px, c.Py);
  if (e != cudaSuccess) return e;
  return mgc_launch(k_cc_coef, dim3(c.nb * c.nb), dim3(256), 0, st, c.nb, c.my, c.wvphi64, c.Px, c.c);
}

// Clusters of more than 8 CTAs must be allowed per kernel (once, before any launch or
// capture); called by setup.
// Raises (never lowers) the kernel's dynamic shared-memory limit to what m_max rows need,
// so every handle set up so far can still launch.
cudaError_t channel_solve_prepare(int nb, int m_max) {
  static std::mutex mu;
  static int granted[MGC_MAX_NB + 1] = {0};
  if (nb < 1 || nb > MGC_MAX_NB) return cudaErrorInvalidValue;
  const int smem = 2 * cr_rows(m_max) * nb * (int)sizeof(cplx);
  std::lock_guard<std::mutex> lock(mu);
  if (granted[nb] > 0 && smem <= granted[nb]) return cudaSuccess;
  const int want = smem > 48 * 1024 ? smem : 48 * 1024;
  cudaError_t e = cudaErrorInvalidValue;
  switch (nb) {
#define MGC_PREP(K)                                                                                        \
  case K:                                                                                                  \
    e = cudaFuncSetAttribute(k_channel_solve_pcr<K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); \
    if (e == cudaSuccess)                                                                                \
      e = cudaFuncSetAttribute(k_channel_solve_pcr<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, want); \
    break;
    MGC_PREP(1) MGC_PREP(2) MGC_PREP(3) MGC_PREP(4) MGC_PREP(5) MGC_PREP(6) MGC_PREP(7) MGC_PREP(8)
#undef MGC_PREP
  }
  if (e == cudaSuccess) granted[nb] = want;
  return e;
}

cudaError_t launch_channel_solve(const CRSystem& A, const CRSystem& B, cudaStream_t st) {
  const int mm = A.m > B.m ? A.m : B.m;
  const size_t smem = 2 * (size_t)cr_rows(mm) * A.nb * sizeof(cplx);
  switch (A.nb) {
    case 1: return mgc_launch(k_channel_solve_pcr<1>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 2: return mgc_launch(k_channel_solve_pcr<2>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 3: return mgc_launch(k_channel_solve_pcr<3>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 4: return mgc_launch(k_channel_solve_pcr<4>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 5: return mgc_launch(k_channel_solve_pcr<5>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 6: return mgc_launch(k_channel_solve_pcr<6>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 7: return mgc_launch(k_channel_solve_pcr<7>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    case 8: return mgc_launch(k_channel_solve_pcr<8>, dim3(2 * CR_CLUSTER), dim3(CR_THREADS), smem, st, A, B);
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_cccs_correct(const CCViewT<C>& c, C* u, cudaStream_t st) {
  switch (c.nb) {
    case 1: return corr_launch<1, C>(c, u, st);
    case 2: return corr_launch<2, C>(c, u, st);
    case 3: return corr_launch<3, C>(c, u, st);
    case 4: return corr_launch<4, C>(c, u, st);
    case 5: return corr_launch<5, C>(c, u, st);
    case 6: return corr_launch<6, C>(c, u, st);
    case 7: return corr_launch<7, C>(c, u, st);
    case 8: return corr_launch<8, C>(c, u, st);
  }
  return cudaErrorInvalidValue;
}

#define MGC_INSTANTIATE(C)                                                                                  \
  template cudaError_t launch_residual_project<C>(const StencilViewT<C>&, const CCViewT<C>&, const C*,     \
                                                  const C*, cudaStream_t);                                \
  template cudaError_t launch_cc_rhs<C>(const CCViewT<C>&, cudaStream_t);                                 \
  template cudaError_t launch_cccs_correct<C>(const CCViewT<C>&, C*, cudaStream_t);
MGC_INSTANTIATE(double2)
MGC_INSTANTIATE(float2)
#undef MGC_INSTANTIATE
