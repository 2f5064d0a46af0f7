// Coarsest-level direct solve by block parallel cyclic reduction, for coarsest grids with
// more unknowns than the dense inverse holds (Sec. 3.2 solves the coarsest level exactly;
// how is left open).
//
// Ordered by grid rows j, the coarsest operator is block tridiagonal with nr = my block
// rows of size m = mx:  L_j u_{j-1} + D_j u_j + U_j u_{j+1} = f_j, where D_j is the
// tridiagonal x-part plus the diagonal of row j, and L_j = west_y[j] I, U_j = east_y[j] I.
// Level l of the reduction (stride s = 2^l) eliminates every row's couplings to the rows
// j -+ s with the rows j -+ s themselves:
//     alpha_j = L_j D_{j-s}^{-1},  gamma_j = U_j D_{j+s}^{-1},
//     D_j' = D_j - alpha_j U_{j-s} - gamma_j L_{j+s},  L_j' = -alpha_j L_{j-s},
//     U_j' = -gamma_j U_{j+s},     f_j' = f_j - alpha_j f_{j-s} - gamma_j f_{j+s},
// with the terms of rows outside 0..nr-1 dropped.  After ceil(log2 nr) levels no row is
// coupled, and u_j = D_j^{-1} f_j.  Setup forms alpha, gamma and the last D^{-1} once
// (dense m x m blocks, complex128, Gauss-Jordan with partial pivoting for the block
// inverses); a solve is then ceil(log2 nr) launches of block matrix-vector products,
// the final D^{-1} folded into the last level's products (u_j = D_j^{-1} f_j -
// (D_j^{-1} alpha_j) f_{j-s} - (D_j^{-1} gamma_j) f_{j+s}).  A solve costs
// (2 ceil(log2 nr) + 1) nr m^2 complex multiply-adds, 13 M FP64 FMAs for the 63 x 63
// coarsest grid of a 1024^2 problem on 5 levels, against 63 M for the dense inverse of
// the same grid.  Everything stays FP64 in both precisions.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int BP_THREADS = 256;
constexpr int BP_KQ = 8;            // warps of a solve block: parts of the k range
constexpr int BP_KC = 8;            // k per warp (BP_KQ * BP_KC >= MGC_BP_MAX_M)
static_assert(BP_KQ * BP_KC >= MGC_BP_MAX_M, "the warps of a solve block must cover every k");
static_assert(32 * BP_KQ >= 3 * MGC_BP_MAX_M, "a solve block stages its three rows of b with one thread each");
constexpr int BP_GEMM_SPLIT = 4;    // blocks per batched product (row slices)

int bp_levels(int nr) {
  int n = 0;
  for (int s = 1; s < nr; s *= 2) ++n;
  return n;
}

// Dense blocks of the coarsest operator: D_j (tridiagonal), L_j = west_y[j] I (0 for
// j = 0), U_j = east_y[j] I (0 for j = nr - 1); each block m x m row-major.
__global__ void k_bp_assemble(StencilView s, cplx* __restrict__ Dm, cplx* __restrict__ Lm, cplx* __restrict__ Um) {
  const int m = s.mx, nr = s.my;
  const long long mm = (long long)m * m, tot = mm * nr;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(q / mm), e = (int)(q % mm), r = e / m, c = e % m;
    cplx d = cmk(0.0, 0.0), l = cmk(0.0, 0.0), u = cmk(0.0, 0.0);
    if (c == r) {
      d = s.D[(size_t)j * m + r];
      if (j > 0) l = s.west_y[j];
      if (j + 1 < nr) u = s.east_y[j];
    } else if (c == r - 1) {
      d = s.west_x[r];
    } else if (c == r + 1) {
      d = s.east_x[r];
    }
    Dm[q] = d;
    Lm[q] = l;
    Um[q] = u;
  }
}

// The first reduction level needs no products: L_j = west_y[j] I and U_j = east_y[j] I are
// scalar multiples of the identity, so with Di_j = D_j^{-1}
//   alpha_j = wy_j Di_{j-1},  gamma_j = ey_j Di_{j+1},
//   D_j' = D_j - wy_j ey_{j-1} Di_{j-1} - ey_j wy_{j+1} Di_{j+1},
//   L_j' = -wy_j wy_{j-1} Di_{j-1} (j >= 2),  U_j' = -ey_j ey_{j+1} Di_{j+1} (j <= nr - 3),
// one elementwise pass (alpha^T, gamma^T stored transposed; L', U' skipped on the last level).
__global__ void k_bp_setup0(int nr, int m, const cplx* __restrict__ wy, const cplx* __restrict__ ey,
                            const cplx* __restrict__ Di, cplx* __restrict__ AT, cplx* __restrict__ GT,
                            cplx* __restrict__ Dm, cplx* __restrict__ Ln, cplx* __restrict__ Un, int last) {
  const long long mm = (long long)m * m, tot = mm * nr;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(q / mm), e = (int)(q % mm), r = e / m, c = e % m;
    const long long tq = (long long)j * mm + (long long)c * m + r;
    const cplx z = cmk(0.0, 0.0);
    const cplx a = j >= 1 ? cmul(wy[j], Di[q - mm]) : z;
    const cplx g = j + 1 < nr ? cmul(ey[j], Di[q + mm]) : z;
    AT[tq] = a;
    GT[tq] = g;
    cplx d = Dm[q];
    if (j >= 1) d = cfms(a, ey[j - 1], d);
    if (j + 1 < nr) d = cfms(g, wy[j + 1], d);
    Dm[q] = d;
    if (!last) {
      Ln[q] = j >= 2 ? cneg(cmul(a, wy[j - 1])) : z;
      Un[q] = j + 2 < nr ? cneg(cmul(g, ey[j + 1])) : z;
    }
  }
}

// dst_j = src_j^{-1} (or its transpose when trans) for each block j: Gauss-Jordan with
// partial pivoting (largest |re| + |im| in the column, lowest row on ties), a zero pivot
// setting MGC_ST_PIVOT and leaving dst unwritten, with each block's elimination split over
// a cluster of two CTAs: CTA r keeps columns [32 r, 32 r + 32) in its shared memory, so
// two SMs share the O(m^3) FP64 work of a block (one CTA per block took 502 against 408 us
// a launch of 63 blocks of 63 x 63, most of either being the per-pivot barriers).
// Per pivot k: the owner of column k finds the pivot row and publishes it (cluster barrier);
// both swap their rows k and p; the owner publishes 1/pivot and column k (barrier); both
// scale row k and update their columns (barrier).  The row interchanges are undone at the
// write-out: output column c is column sigma(c) of the reduced matrix, sigma the composition
// of the interchanges in pivot order, read from whichever CTA holds it.
constexpr int BP_HALF = 32;                      // columns per CTA (MGC_BP_MAX_M / 2)
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(BP_THREADS)
    k_bp_invert2(int m, const cplx* __restrict__ src, cplx* __restrict__ dst, int trans, int* __restrict__ status) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ cplx A[MGC_BP_MAX_M][BP_HALF];
  __shared__ cplx fcol[MGC_BP_MAX_M];
  __shared__ cplx s_d;
  __shared__ int perm[MGC_BP_MAX_M];
  __shared__ int s_piv, s_fail;
  const int rank = (int)cl.block_rank(), t = threadIdx.x;
  const int blk = blockIdx.x / 2;
  const int c0 = rank * BP_HALF, nc = max(0, min(BP_HALF, m - c0));
  const int mm = m * m;
  const cplx* __restrict__ a = src + (size_t)blk * mm;
  for (int q = t; q < m * BP_HALF; q += blockDim.x) {
    const int r = q / BP_HALF, c = q - r * BP_HALF;
    A[r][c] = c < nc ? a[r * m + c0 + c] : cmk(0.0, 0.0);
  }
  if (t == 0) s_fail = 0;
  cl.sync();
  int* piv_peer = cl.map_shared_rank(&s_piv, rank ^ 1);
  int* fail_peer = cl.map_shared_rank(&s_fail, rank ^ 1);
  cplx* fcol_peer = cl.map_shared_rank(fcol, rank ^ 1);
  cplx* d_peer = cl.map_shared_rank(&s_d, rank ^ 1);
  for (int k = 0; k < m; ++k) {
    const int own = k / BP_HALF, kc = k - own * BP_HALF;
    if (rank == own && t < 32) {
      double best = -1.0;
      int bi = m;
      for (int r = k + t; r < m; r += 32) {
        const double v = cabs1(A[r][kc]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
      }
      if (t == 0) {
        const int f = (!(best > 0.0) || bi >= m) ? 1 : 0;
        s_piv = bi;
        *piv_peer = bi;
        s_fail = f;
        *fail_peer = f;
      }
    }
    cl.sync();
    if (s_fail) break;
    const int p = s_piv;
    if (p != k) {
      for (int c = t; c < BP_HALF; c += blockDim.x) {
        const cplx x = A[k][c];
        A[k][c] = A[p][c];
        A[p][c] = x;
      }
    }
    if (t == 0) perm[k] = p;
    __syncthreads();
    if (rank == own) {
      const cplx d = cdiv(cmk(1.0, 0.0), A[k][kc]);
      if (t == 0) {
        s_d = d;
        *d_peer = d;
      }
      for (int r = t; r < m; r += blockDim.x) {
        const cplx v = A[r][kc];
        fcol[r] = v;
        fcol_peer[r] = v;
      }
    }
    cl.sync();
    const cplx d = s_d;
    for (int c = t; c < BP_HALF; c += blockDim.x)
      A[k][c] = (rank == own && c == kc) ? d : cmul(A[k][c], d);
    __syncthreads();
    for (int q = t; q < m * BP_HALF; q += blockDim.x) {
      const int r = q / BP_HALF, c = q - r * BP_HALF;
      if (r == k) continue;
      const cplx old = (rank == own && c == kc) ? cmk(0.0, 0.0) : A[r][c];
      A[r][c] = cfms(fcol[r], A[k][c], old);
    }
    cl.sync();
  }
  if (s_fail) {
    if (rank == 0 && t == 0) atomicOr(status, MGC_ST_PIVOT);
    cl.sync();
    return;
  }
  // write-out: column c of the inverse is column sigma(c) of A, held by CTA sigma(c) / 32
  cplx* __restrict__ o = dst + (size_t)blk * mm;
  for (int q = t; q < m * nc; q += blockDim.x) {
    const int r = q / nc, cl_ = q - r * nc, c = c0 + cl_;
    int idx = c;
    for (int k = 0; k < m; ++k) {
      const int pk = perm[k];
      if (idx == k) idx = pk;
      else if (idx == pk) idx = k;
    }
    const int src_rank = idx / BP_HALF;
    const cplx* col = src_rank == rank ? &A[0][0] : cl.map_shared_rank(&A[0][0], src_rank);
    const cplx v = col[r * BP_HALF + (idx - src_rank * BP_HALF)];
    o[trans ? c * m + r : r * m + c] = v;
  }
  cl.sync();                        // the partner's shared memory stays live until both have read
}

// One batched product of the reduction's setup:
//   out_j = beta out_j + sigma X_{j+dx} Y_{j+dy}     (j = 0..nr-1, blockIdx.x)
// where a block stored transposed (tx, ty) is read as its transpose, out is written
// transposed when to, and the product term is dropped when j + dx or j + dy lies outside
// 0..nr-1.  blockIdx.y selects a slice of output rows; Y is staged in shared memory.
__global__ void __launch_bounds__(BP_THREADS) k_bp_gemm(int nr, int m, cplx* __restrict__ out, int to, double beta,
                                                        double sigma, const cplx* __restrict__ X, int dx, int tx,
                                                        const cplx* __restrict__ Y, int dy, int ty) {
  extern __shared__ cplx ys[];        // m * m, row-major Y_{j+dy}
  const int j = blockIdx.x, t = threadIdx.x, mm = m * m;
  const int jx = j + dx, jy = j + dy;
  const bool term = jx >= 0 && jx < nr && jy >= 0 && jy < nr;
  if (term) {
    const cplx* __restrict__ y = Y + (size_t)jy * mm;
    for (int q = t; q < mm; q += blockDim.x) {
      const int r = q / m, c = q - r * m;
      ys[q] = ty ? y[c * m + r] : y[q];
    }
  }
  __syncthreads();
  const int rows = (m + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows, r1 = min(m, r0 + rows);
  const cplx* __restrict__ x = X + (size_t)(term ? jx : 0) * mm;
  cplx* __restrict__ o = out + (size_t)j * mm;
  for (int q = r0 * m + t; q < r1 * m; q += blockDim.x) {
    const int r = q / m, c = q - r * m;
    cplx acc = cmk(0.0, 0.0);
    if (term) {
      for (int k = 0; k < m; ++k) acc = cfma(tx ? x[k * m + r] : x[r * m + k], ys[k * m + c], acc);
    }
    const int oi = to ? c * m + r : q;
    cplx v = cscal(sigma, acc);
    if (beta != 0.0) v = cadd(v, cscal(beta, o[oi]));
    o[oi] = v;
  }
}

// One level of a solve: for block row j = blockIdx.x and outputs i = 32 blockIdx.y + lane,
//   out_j[i] = (DT ? sum_k DT_j[k][i] b_j[k] : b_j[i])
//              - sum_k AT_j[k][i] b_{j-s}[k] - sum_k GT_j[k][i] b_{j+s}[k]
// with the factors stored transposed, so a warp's 32 lanes read 32 consecutive entries of
// one factor row.  The three rows of b are staged in shared memory (read there as
// broadcasts); warp w takes k = BP_KC w .. BP_KC w + BP_KC - 1 and issues all of its factor
// loads before anything else (the factors come from DRAM: the Krylov vectors stream
// through L2 between two coarsest solves); the warps' sums meet in shared memory and are
// added in a fixed order.
template <class CI, class CO>
__global__ void __launch_bounds__(32 * BP_KQ) k_bp_level(int nr, int m, int s, const cplx* __restrict__ AT,
                                                         const cplx* __restrict__ GT, const cplx* __restrict__ DT,
                                                         const CI* __restrict__ b, CO* __restrict__ out) {
  __shared__ cplx part[BP_KQ][32];
  __shared__ cplx bs[3][BP_KQ * BP_KC];
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int i = blockIdx.y * 32 + lane;
  const bool has_a = j - s >= 0, has_g = j + s < nr;
  const size_t mm = (size_t)m * m;
  const int ii = i < m ? i : 0, k0 = w * BP_KC;
  // the factors were written at setup, before the solve began: they are read while the
  // preceding kernel of the solve drains, ahead of the wait for its results
  cplx fa[BP_KC], fg[BP_KC], fd[BP_KC];
#pragma unroll
  for (int q = 0; q < BP_KC; ++q) {
    const int k = k0 + q;
    const bool ok = k < m;
    fa[q] = ok && has_a ? __ldg(AT + j * mm + (size_t)k * m + ii) : cmk(0.0, 0.0);
    fg[q] = ok && has_g ? __ldg(GT + j * mm + (size_t)k * m + ii) : cmk(0.0, 0.0);
    fd[q] = ok && DT ? __ldg(DT + j * mm + (size_t)k * m + ii) : cmk(0.0, 0.0);
  }
  mgc_pdl_enter();
  if (t < 3 * m) {
    const int r = t / m, k = t - r * m;
    const int jr = j + (r - 1) * s;
    if (jr >= 0 && jr < nr) bs[r][k] = to_c128(b[(size_t)jr * m + k]);
  }
  __syncthreads();
  cplx acc0 = cmk(0.0, 0.0), acc1 = cmk(0.0, 0.0);
  if (!DT && w == 0 && i < m) acc0 = bs[1][i];
#pragma unroll
  for (int q = 0; q < BP_KC; ++q) {
    const int k = k0 + q < m ? k0 + q : 0;
    if (has_a) acc1 = cfms(fa[q], bs[0][k], acc1);
    if (has_g) acc0 = cfms(fg[q], bs[2][k], acc0);
    if (DT) acc0 = cfma(fd[q], bs[1][k], acc0);
  }
  part[w][lane] = cadd(acc0, acc1);
  __syncthreads();
  if (w == 0 && i < m) {
    cplx tot = part[0][lane];
#pragma unroll
    for (int q = 1; q < BP_KQ; ++q) tot = cadd(tot, part[q][lane]);
    out[(size_t)j * m + i] = CT<CO>::make(tot.x, tot.y);
  }
}

template <class CI, class CO>
cudaError_t launch_level(int nr, int m, int s, const cplx* AT, const cplx* GT, const cplx* DT, const CI* b, CO* out,
                         cudaStream_t st) {
  return mgc_launch(k_bp_level<CI, CO>, dim3(nr, (m + 31) / 32), dim3(32 * BP_KQ), 0, st, nr, m, s, AT, GT, DT, b,
                    out);
}

}  // namespace

bool bpcr_fits(int mx, int my) { return mx >= 1 && mx <= MGC_BP_MAX_M && my >= 1 && my <= MGC_BP_MAX_ROWS; }

size_t bpcr_factor_entries(int mx, int my) {
  return (size_t)(2 * bp_levels(my) + 1) * my * mx * mx;
}

size_t bpcr_scratch_entries(int mx, int my) { return (size_t)6 * my * mx * mx; }

cudaError_t launch_bpcr_setup(const StencilView& s, cplx* fac, cplx* scratch, int* status, cudaStream_t st) {
  const int m = s.mx, nr = s.my;
  if (!bpcr_fits(m, nr)) return cudaErrorInvalidValue;
  const size_t B = (size_t)nr * m * m;
  cplx* Dm = scratch;
  cplx* Di = scratch + B;
  cplx* Lm[2] = {scratch + 2 * B, scratch + 3 * B};
  cplx* Um[2] = {scratch + 4 * B, scratch + 5 * B};
  const int Lp = bp_levels(nr);
  cplx* DfT = fac + (size_t)2 * Lp * B;
  const size_t mm_smem = sizeof(cplx) * (size_t)m * m;
  {
    // the limit for the largest block size, set once: handles set up from several host
    // threads must not lower it under another thread's launch
    static std::mutex mu;
    static bool granted = false;
    std::lock_guard<std::mutex> lock(mu);
    if (!granted) {
      const int M = MGC_BP_MAX_M;
      cudaError_t e =
          cudaFuncSetAttribute(k_bp_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(cplx) * M * M));
      if (e != cudaSuccess) return e;
      granted = true;
    }
  }
  const int grid = (int)std::min<long long>(((long long)B + 255) / 256, 8LL * mgc_sm_count());
  k_bp_assemble<<<grid, 256, 0, st>>>(s, Dm, Lm[0], Um[0]);
  const dim3 gg(nr, BP_GEMM_SPLIT);
  auto gemm = [&](cplx* out, int to, double beta, double sigma, const cplx* X, int dx, int tx, const cplx* Y, int dy,
                  int ty) {
    k_bp_gemm<<<gg, BP_THREADS, mm_smem, st>>>(nr, m, out, to, beta, sigma, X, dx, tx, Y, dy, ty);
  };
  int cur = 0;
  for (int l = 0, s2 = 1; l < Lp; ++l, s2 *= 2) {
    const bool last = l == Lp - 1;
    // the last level keeps alpha^T, gamma^T in the free L/U buffers until D^{-1} is known
    cplx* AT = last ? Lm[cur ^ 1] : fac + (size_t)(2 * l) * B;
    cplx* GT = last ? Um[cur ^ 1] : fac + (size_t)(2 * l + 1) * B;
    k_bp_invert2<<<2 * nr, BP_THREADS, 0, st>>>(m, Dm, Di, 0, status);
    if (l == 0) {
      // scalar off-diagonal blocks: alpha, gamma, D', L', U' elementwise
      k_bp_setup0<<<grid, 256, 0, st>>>(nr, m, s.west_y, s.east_y, Di, AT, GT, Dm, Lm[cur ^ 1], Um[cur ^ 1],
                                        last ? 1 : 0);
      if (!last) cur ^= 1;
      continue;
    }
    gemm(AT, 1, 0.0, 1.0, Lm[cur], 0, 0, Di, -s2, 0);           // alpha_j = L_j D_{j-s}^{-1}
    gemm(GT, 1, 0.0, 1.0, Um[cur], 0, 0, Di, s2, 0);            // gamma_j = U_j D_{j+s}^{-1}
    gemm(Dm, 0, 1.0, -1.0, AT, 0, 1, Um[cur], -s2, 0);          // D_j -= alpha_j U_{j-s}
    gemm(Dm, 0, 1.0, -1.0, GT, 0, 1, Lm[cur], s2, 0);           // D_j -= gamma_j L_{j+s}
    if (!last) {
      gemm(Lm[cur ^ 1], 0, 0.0, -1.0, AT, 0, 1, Lm[cur], -s2, 0);   // L_j' = -alpha_j L_{j-s}
      gemm(Um[cur ^ 1], 0, 0.0, -1.0, GT, 0, 1, Um[cur], s2, 0);    // U_j' = -gamma_j U_{j+s}
      cur ^= 1;
    }
  }
  k_bp_invert2<<<2 * nr, BP_THREADS, 0, st>>>(m, Dm, DfT, 1, status);
  if (Lp > 0) {
    // fold D^{-1} into the last level: (D^{-1} alpha)^T and (D^{-1} gamma)^T
    gemm(fac + (size_t)(2 * (Lp - 1)) * B, 1, 0.0, 1.0, DfT, 0, 1, Lm[cur ^ 1], 0, 1);
    gemm(fac + (size_t)(2 * (Lp - 1) + 1) * B, 1, 0.0, 1.0, DfT, 0, 1, Um[cur ^ 1], 0, 1);
  }
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_bpcr_solve(int mx, int my, const cplx* fac, const C* f, C* u, cplx* buf, cudaStream_t st) {
  const int m = mx, nr = my;
  if (!bpcr_fits(m, nr)) return cudaErrorInvalidValue;
  const size_t B = (size_t)nr * m * m;
  const int Lp = bp_levels(nr);
  const cplx* DfT = fac + (size_t)2 * Lp * B;
  if (Lp == 0) return launch_level<C, C>(nr, m, 1, nullptr, nullptr, DfT, f, u, st);
  cplx* pb[2] = {buf, buf + (size_t)nr * m};
  cudaError_t e = cudaSuccess;
  for (int l = 0, s = 1; l < Lp && e == cudaSuccess; ++l, s *= 2) {
    const cplx* AT = fac + (size_t)(2 * l) * B;
    const cplx* GT = fac + (size_t)(2 * l + 1) * B;
    const bool first = l == 0, last = l == Lp - 1;
    if (first && last) e = launch_level<C, C>(nr, m, s, AT, GT, DfT, f, u, st);
    else if (first) e = launch_level<C, cplx>(nr, m, s, AT, GT, nullptr, f, pb[0], st);
    else if (last) e = launch_level<cplx, C>(nr, m, s, AT, GT, DfT, pb[(l - 1) & 1], u, st);
    else e = launch_level<cplx, cplx>(nr, m, s, AT, GT, nullptr, pb[(l - 1) & 1], pb[l & 1], st);
  }
  return e;
}

template cudaError_t launch_bpcr_solve<double2>(int, int, const cplx*, const double2*, double2*, cplx*,
                                                cudaStream_t);
template cudaError_t launch_bpcr_solve<float2>(int, int, const cplx*, const float2*, float2*, cplx*, cudaStream_t);
