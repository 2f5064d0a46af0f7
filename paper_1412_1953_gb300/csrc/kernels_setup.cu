// Setup kernels of MG-CCCS (run once per grid / potential / energy).
//
//  * ECS node coordinates and the 3-point nonuniform second-difference coefficients
//    per axis and level (Sec. 2.5, Eq. (11)); coarse levels optionally on a rotated
//    contour.
//  * Diagonal D of H - E and omega/D per node, potentials injected at coincident nodes.
//  * Dense inverse of the coarsest-level operator (Gauss-Jordan, partial pivoting).
//  * Bound states of H1, H2 (Eq. (9)): eigenvalues by implicit QL with a Wilkinson
//    shift applied without conjugation to the complex-symmetric tridiagonal
//    (Bowdler, Martin, Reinsch & Wilkinson, Numer. Math. 11, 1968; the
//    complex-symmetric use follows Cullum & Willoughby), the n_b with smallest real
//    part, eigenvectors by inverse iteration with a pivoted tridiagonal LU, bilinear
//    normalisation int phi^2 dz = 1 (Sec. 3.1, Remark 3), then two shift-and-invert
//    steps and a bilinear Rayleigh quotient (Sec. 5.1.2, Sec. 5.2).
//  * Channel potentials V^A, V^B (Sec. 4.2) and the block-Thomas factors of the
//    coupled-channel systems (Eqs. (28)-(29)).
#include "common.cuh"

namespace {

__device__ __forceinline__ cplx node_z(int k, int n, double L, double R0, double ct, double st,
                                       double cg, double sg) {
  double x = (double)k * L / (double)n;
  cplx z = (x <= R0) ? cmk(x, 0.0) : cmk(R0 + (x - R0) * ct, (x - R0) * st);
  if (cg != 1.0 || sg != 0.0) z = cmul(z, cmk(cg, sg));
  return z;
}

__global__ void k_setup_axis(AxisSetup a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // interior index, node k = i + 1
  if (i >= a.n - 1) return;
  double ct, st, cg = 1.0, sg = 0.0;
  sincos(a.theta, &st, &ct);
  if (a.gamma != 0.0) sincos(a.gamma, &sg, &cg);
  const int k = i + 1;
  cplx zm = node_z(k - 1, a.n, a.L, a.R0, ct, st, cg, sg);
  cplx z0 = node_z(k, a.n, a.L, a.R0, ct, st, cg, sg);
  cplx zp = node_z(k + 1, a.n, a.L, a.R0, ct, st, cg, sg);
  cplx hm = csub(z0, zm), hp = csub(zp, z0);
  cplx s = cadd(hm, hp);
  cplx west = cneg(cdiv(cmk(1.0, 0.0), cmul(s, hm)));
  cplx east = cneg(cdiv(cmk(1.0, 0.0), cmul(s, hp)));
  a.west[i] = west;
  a.east[i] = east;
  a.diag[i] = cneg(cadd(west, east));
  a.w[i] = cscal(0.5, s);
}

__global__ void k_setup_diag(int mx, int my, int stride, int fine_mx, const cplx* __restrict__ dx,
                             const cplx* __restrict__ dy, const cplx* __restrict__ v1, const cplx* __restrict__ v2,
                             const cplx* __restrict__ v12, double E, double omega, cplx* __restrict__ D,
                             cplx* __restrict__ Dinv, int* status) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  if (i >= mx || j >= my) return;
  const int fi = stride * (i + 1) - 1, fj = stride * (j + 1) - 1;   // injection at coincident nodes
  cplx d = cadd(cadd(cadd(cadd(dx[i], dy[j]), v1[fi]), v2[fj]), v12[(size_t)fj * fine_mx + fi]);
  d.x -= E;
  const size_t p = (size_t)j * mx + i;
  D[p] = d;
  if (d.x == 0.0 && d.y == 0.0) {
    atomicOr(status, MGC_ST_PIVOT);
    Dinv[p] = cmk(0.0, 0.0);
  } else {
    Dinv[p] = cdiv(cmk(omega, 0.0), d);
  }
}

// Dense inverse of the coarsest operator by Gauss-Jordan elimination with partial
// pivoting on the augmented matrix [A | I] (nc x 2nc, in global memory), one block.
__global__ void __launch_bounds__(1024) k_coarse_inverse(StencilView s, cplx* __restrict__ aug,
                                                         cplx* __restrict__ Ainv, int* status) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  __shared__ cplx fac[MGC_MAX_COARSE];
  const int nc = s.mx * s.my;
  const int w2 = 2 * nc;
  const int t = threadIdx.x;
  // assemble [A | I]
  for (long long q = t; q < (long long)nc * w2; q += blockDim.x) aug[q] = cmk(0.0, 0.0);
  __syncthreads();
  for (int p = t; p < nc; p += blockDim.x) {
    const int i = p % s.mx, j = p / s.mx;
    cplx* row = aug + (size_t)p * w2;
    row[p] = s.D[p];
    if (i > 0) row[p - 1] = s.west_x[i];
    if (i + 1 < s.mx) row[p + 1] = s.east_x[i];
    if (j > 0) row[p - s.mx] = s.west_y[j];
    if (j + 1 < s.my) row[p + s.mx] = s.east_y[j];
    row[nc + p] = cmk(1.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    // pivot search over rows k..nc-1 (largest modulus, lowest index on ties)
    double best = -1.0;
    int bi = k;
    for (int r = k + t; r < nc; r += blockDim.x) {
      double v = cmod(aug[(size_t)r * w2 + k]);
      if (v > best) { best = v; bi = r; }
    }
    sval[t] = best;
    sidx[t] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (t < o) {
        double v2 = sval[t + o];
        int i2 = sidx[t + o];
        if (v2 > sval[t] || (v2 == sval[t] && i2 < sidx[t])) { sval[t] = v2; sidx[t] = i2; }
      }
      __syncthreads();
    }
    const int piv = sidx[0];
    const double pmod = sval[0];
    __syncthreads();
    if (pmod == 0.0) {
      if (t == 0) atomicOr(status, MGC_ST_PIVOT);
      return;
    }
    if (piv != k) {
      for (int c = t; c < w2; c += blockDim.x) {
        cplx a = aug[(size_t)k * w2 + c];
        aug[(size_t)k * w2 + c] = aug[(size_t)piv * w2 + c];
        aug[(size_t)piv * w2 + c] = a;
      }
    }
    __syncthreads();
    const cplx pv = aug[(size_t)k * w2 + k];
    __syncthreads();
    for (int c = t; c < w2; c += blockDim.x) aug[(size_t)k * w2 + c] = cdiv(aug[(size_t)k * w2 + c], pv);
    for (int r = t; r < nc; r += blockDim.x) fac[r] = aug[(size_t)r * w2 + k];
    __syncthreads();
    for (long long q = t; q < (long long)nc * w2; q += blockDim.x) {
      const int r = (int)(q / w2), c = (int)(q % w2);
      if (r == k) continue;
      aug[q] = cfms(fac[r], aug[(size_t)k * w2 + c], aug[q]);
    }
    __syncthreads();
  }
  for (long long q = t; q < (long long)nc * nc; q += blockDim.x) {
    const int r = (int)(q / nc), c = (int)(q % nc);
    Ainv[q] = aug[(size_t)r * w2 + nc + c];
  }
}

// ---- bound states ---------------------------------------------------------------

// Eigenvalues of the complex-symmetric tridiagonal (d, e) by implicit QL; d is
// overwritten with the eigenvalues.  Returns false if an eigenvalue needs more than
// 60 sweeps or a rotation breaks down.
__device__ bool ql_eigenvalues(int m, cplx* d, cplx* e) {
  e[m - 1] = cmk(0.0, 0.0);
  for (int l = 0; l < m; ++l) {
    int sweeps = 0;
    for (;;) {
      int mm = l;
      for (; mm < m - 1; ++mm) {
        double dd = cabs1(d[mm]) + cabs1(d[mm + 1]);
        if (cabs1(e[mm]) + dd == dd) break;
      }
      if (mm == l) break;
      if (++sweeps > 60) return false;
      // shift from the leading 2x2 block
      cplx g = cdiv(csub(d[l + 1], d[l]), cscal(2.0, e[l]));
      cplx r = csqrt_p(cadd(cmul(g, g), cmk(1.0, 0.0)));
      cplx gp = cadd(g, r), gm = csub(g, r);
      cplx den = (cabs2(gp) >= cabs2(gm)) ? gp : gm;
      g = cadd(csub(d[mm], d[l]), cdiv(e[l], den));
      cplx s = cmk(1.0, 0.0), c = cmk(1.0, 0.0), p = cmk(0.0, 0.0);
      bool restart = false;
      for (int i = mm - 1; i >= l; --i) {
        cplx f = cmul(s, e[i]);
        cplx b = cmul(c, e[i]);
        r = csqrt_p(cadd(cmul(f, f), cmul(g, g)));
        e[i + 1] = r;
        if (r.x == 0.0 && r.y == 0.0) {
          if (f.x != 0.0 || f.y != 0.0) return false;       // isotropic breakdown
          d[i + 1] = csub(d[i + 1], p);
          e[mm] = cmk(0.0, 0.0);
          restart = true;
          break;
        }
        s = cdiv(f, r);
        c = cdiv(g, r);
        g = csub(d[i + 1], p);
        r = cadd(cmul(csub(d[i], g), s), cscal(2.0, cmul(c, b)));
        p = cmul(s, r);
        d[i + 1] = cadd(g, p);
        g = csub(cmul(c, r), b);
      }
      if (restart) continue;
      d[l] = csub(d[l], p);
      e[l] = g;
      e[mm] = cmk(0.0, 0.0);
    }
  }
  for (int k = 0; k < m; ++k)
    if (!isfinite(d[k].x) || !isfinite(d[k].y)) return false;
  return true;
}

// Pivoted LU of the tridiagonal T - sigma I (T: sub `west` (row k couples to k-1),
// diagonal `diag + v`, super `east`).  Row k of U holds u0 (col k), u1 (col k+1),
// u2 (col k+2); mu[k] is the multiplier of step k and sw[k] says whether rows k, k+1
// were exchanged.
struct TriLU {
  cplx *u0, *u1, *u2, *mu;
  int* sw;
};

__device__ void tri_lu(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v, cplx sigma,
                       TriLU lu) {
  cplx Dk = csub(cadd(diag[0], v[0]), sigma);
  cplx U1 = (m > 1) ? east[0] : cmk(0.0, 0.0);
  for (int k = 0; k < m - 1; ++k) {
    cplx L = west[k + 1];
    cplx dn = csub(cadd(diag[k + 1], v[k + 1]), sigma);
    cplx cn = (k + 2 < m) ? east[k + 1] : cmk(0.0, 0.0);
    if (cabs2(L) > cabs2(Dk)) {
      // exchange: pivot row is row k+1
      cplx mu = cdiv(Dk, L);
      lu.u0[k] = L; lu.u1[k] = dn; lu.u2[k] = cn; lu.mu[k] = mu; lu.sw[k] = 1;
      Dk = cfms(mu, dn, U1);
      U1 = cneg(cmul(mu, cn));
    } else {
      cplx mu = (Dk.x == 0.0 && Dk.y == 0.0) ? cmk(0.0, 0.0) : cdiv(L, Dk);
      lu.u0[k] = Dk; lu.u1[k] = U1; lu.u2[k] = cmk(0.0, 0.0); lu.mu[k] = mu; lu.sw[k] = 0;
      Dk = cfms(mu, U1, dn);
      U1 = cn;
    }
  }
  lu.u0[m - 1] = Dk;
  lu.u1[m - 1] = cmk(0.0, 0.0);
  lu.u2[m - 1] = cmk(0.0, 0.0);
}

// Solve with the factors in place on b; an exactly zero pivot (the shift equals an
// eigenvalue to the last bit) is replaced by a tiny one, the usual inverse-iteration device.
__device__ void tri_solve(int m, TriLU lu, cplx* b, double tiny) {
  for (int k = 0; k < m - 1; ++k) {
    if (lu.sw[k]) { cplx t = b[k]; b[k] = b[k + 1]; b[k + 1] = t; }
    b[k + 1] = cfms(lu.mu[k], b[k], b[k + 1]);
  }
  for (int k = m - 1; k >= 0; --k) {
    cplx t = b[k];
    if (k + 1 < m) t = cfms(lu.u1[k], b[k + 1], t);
    if (k + 2 < m) t = cfms(lu.u2[k], b[k + 2], t);
    cplx piv = lu.u0[k];
    if (piv.x == 0.0 && piv.y == 0.0) piv = cmk(tiny, 0.0);
    b[k] = cdiv(t, piv);
  }
}

// Bilinear normalisation sum w x^2 = 1, then Re x > 0 at the entry of largest modulus.
__device__ void bilinear_normalise(int m, const cplx* w, cplx* x) {
  cplx s = cmk(0.0, 0.0);
  for (int k = 0; k < m; ++k) s = cfma(w[k], cmul(x[k], x[k]), s);
  cplx inv = cdiv(cmk(1.0, 0.0), csqrt_p(s));
  double best = -1.0;
  int kb = 0;
  for (int k = 0; k < m; ++k) {
    x[k] = cmul(x[k], inv);
    double a = cabs2(x[k]);
    if (a > best) { best = a; kb = k; }
  }
  if (x[kb].x < 0.0)
    for (int k = 0; k < m; ++k) x[k] = cneg(x[k]);
}

__device__ void max_normalise(int m, cplx* x) {
  double best = 0.0;
  for (int k = 0; k < m; ++k) best = fmax(best, cabs1(x[k]));
  if (best > 0.0) {
    double s = 1.0 / best;
    for (int k = 0; k < m; ++k) x[k] = cscal(s, x[k]);
  }
}

__device__ cplx rayleigh(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                         const cplx* w, const cplx* x) {
  cplx acc = cmk(0.0, 0.0);
  for (int k = 0; k < m; ++k) {
    cplx hx = cmul(cadd(diag[k], v[k]), x[k]);
    if (k > 0) hx = cfma(west[k], x[k - 1], hx);
    if (k + 1 < m) hx = cfma(east[k], x[k + 1], hx);
    acc = cfma(cmul(x[k], w[k]), hx, acc);
  }
  return acc;
}

__global__ void __launch_bounds__(32) k_bound_states(int m, const cplx* __restrict__ west,
                                                     const cplx* __restrict__ east, const cplx* __restrict__ diag,
                                                     const cplx* __restrict__ v, const cplx* __restrict__ w, int nb,
                                                     cplx* __restrict__ lam, cplx* __restrict__ phi,
                                                     cplx* __restrict__ scratch, int* status) {
  __shared__ cplx sel[MGC_MAX_NB];
  __shared__ int ok;
  const int q = threadIdx.x;
  cplx* d = scratch;            // m
  cplx* e = scratch + m;        // m
  if (q == 0) {
    // symmetric form: e_k^2 = east_k * west_{k+1}
    for (int k = 0; k < m; ++k) {
      d[k] = cadd(diag[k], v[k]);
      e[k] = (k + 1 < m) ? csqrt_p(cmul(east[k], west[k + 1])) : cmk(0.0, 0.0);
    }
    ok = ql_eigenvalues(m, d, e) ? 1 : 0;
    if (ok) {
      // the nb eigenvalues with the smallest real part, ascending (ties: lower index)
      for (int s = 0; s < nb; ++s) {
        int kb = -1;
        for (int k = 0; k < m; ++k) {
          if (e[k].x == 1.0e300) continue;           // already taken
          if (kb < 0 || d[k].x < d[kb].x) kb = k;
        }
        sel[s] = d[kb];
        e[kb] = cmk(1.0e300, 0.0);
      }
    } else {
      atomicOr(status, MGC_ST_EIG);
    }
  }
  __syncthreads();
  if (!ok || q >= nb) return;
  // per-state scratch
  cplx* base = scratch + 2 * m + (size_t)q * 5 * m;
  TriLU lu{base, base + m, base + 2 * m, base + 3 * m,
           reinterpret_cast<int*>(scratch + 2 * m + (size_t)nb * 5 * m) + (size_t)q * m};
  cplx* x = base + 4 * m;
  double scale = 0.0;
  for (int k = 0; k < m; ++k) scale = fmax(scale, cabs1(cadd(diag[k], v[k])));
  const double tiny = 1e-300 + 1e-16 * scale;
  cplx lmb = sel[q];
  // eigenvector by inverse iteration at the QL eigenvalue
  tri_lu(m, west, east, diag, v, lmb, lu);
  for (int k = 0; k < m; ++k) x[k] = cmk(1.0, 0.0);
  for (int it = 0; it < 3; ++it) {
    tri_solve(m, lu, x, tiny);
    max_normalise(m, x);
  }
  bilinear_normalise(m, w, x);
  // two shift-and-invert refinement steps with a Rayleigh-quotient update
  for (int it = 0; it < 2; ++it) {
    tri_lu(m, west, east, diag, v, lmb, lu);
    tri_solve(m, lu, x, tiny);
    max_normalise(m, x);
    bilinear_normalise(m, w, x);
    lmb = rayleigh(m, west, east, diag, v, w, x);
  }
  bool fin = isfinite(lmb.x) && isfinite(lmb.y);
  for (int k = 0; k < m; ++k) {
    phi[(size_t)q * m + k] = x[k];
    fin = fin && isfinite(x[k].x) && isfinite(x[k].y);
  }
  lam[q] = lmb;
  if (!fin) atomicOr(status, MGC_ST_EIG);
}

__global__ void k_weight_states(int m, int nb, const cplx* __restrict__ w, const cplx* __restrict__ phi,
                                cplx* __restrict__ wphi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * nb) return;
  wphi[t] = cmul(w[t % m], phi[t]);
}

// out[row][a][b] = out[row][b][a] = sum_k wst_a(k) st_b(k) v12(row, k);
// v12(row, k) = v12[row * rs + k * ks].  One block per (row, pair a <= b).
__global__ void __launch_bounds__(256) k_channel_potentials(int rows, int len, int nb, long long rs, long long ks,
                                                            const cplx* __restrict__ wst,
                                                            const cplx* __restrict__ st,
                                                            const cplx* __restrict__ v12, cplx* __restrict__ out) {
  __shared__ double sh[2][8];
  const int row = blockIdx.x;
  int pair = blockIdx.y, a = 0;
  while (pair >= nb - a) { pair -= nb - a; ++a; }
  const int b = a + pair;
  cplx acc = cmk(0.0, 0.0);
  for (int k = threadIdx.x; k < len; k += 256)
    acc = cfma(cmul(wst[(size_t)a * len + k], st[(size_t)b * len + k]), v12[row * rs + k * ks], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = acc.x; sh[1][threadIdx.x >> 5] = acc.y; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx tot = cmk(0.0, 0.0);
    for (int k = 0; k < 8; ++k) tot = cadd(tot, cmk(sh[0][k], sh[1][k]));
    out[((size_t)row * nb + a) * nb + b] = tot;
    out[((size_t)row * nb + b) * nb + a] = tot;
  }
}

// In-place inverse of an n x n matrix (n <= MGC_MAX_NB) by Gauss-Jordan with partial pivoting.
__device__ bool small_inverse(int n, cplx* A /* n*n row-major, replaced by inverse */) {
  cplx aug[MGC_MAX_NB][2 * MGC_MAX_NB];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) aug[r][c] = (c < n) ? A[r * n + c] : cmk(c - n == r ? 1.0 : 0.0, 0.0);
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = cabs2(aug[k][k]);
    for (int r = k + 1; r < n; ++r)
      if (cabs2(aug[r][k]) > best) { best = cabs2(aug[r][k]); piv = r; }
    if (best == 0.0) return false;
    if (piv != k)
      for (int c = 0; c < 2 * n; ++c) { cplx t = aug[k][c]; aug[k][c] = aug[piv][c]; aug[piv][c] = t; }
    cplx inv = cdiv(cmk(1.0, 0.0), aug[k][k]);
    for (int c = 0; c < 2 * n; ++c) aug[k][c] = cmul(aug[k][c], inv);
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      cplx fct = aug[r][k];
      for (int c = 0; c < 2 * n; ++c) aug[r][c] = cfms(fct, aug[k][c], aug[r][c]);
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) A[r * n + c] = aug[r][n + c];
  return true;
}

// Block-Thomas factors of the coupled-channel system along one axis:
// B_k = (diag_k + v_k - E) I + diag(lam) + Vc_k,  G_0 = B_0^{-1},
// G_k = (B_k - a_k c_{k-1} G_{k-1})^{-1}.
__global__ void k_channel_factor(int m, int nb, const cplx* __restrict__ diag, const cplx* __restrict__ v,
                                 double E, const cplx* __restrict__ lam, const cplx* __restrict__ Vc,
                                 const cplx* __restrict__ a, const cplx* __restrict__ c, cplx* __restrict__ G,
                                 int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cplx M[MGC_MAX_NB * MGC_MAX_NB];
  for (int k = 0; k < m; ++k) {
    cplx base = cadd(diag[k], v[k]);
    base.x -= E;
    for (int r = 0; r < nb; ++r)
      for (int q = 0; q < nb; ++q) {
        cplx val = Vc[((size_t)k * nb + r) * nb + q];
        if (r == q) val = cadd(val, cadd(base, lam[r]));
        if (k > 0) val = cfms(cmul(a[k], c[k - 1]), G[((size_t)(k - 1) * nb + r) * nb + q], val);
        M[r * nb + q] = val;
      }
    if (!small_inverse(nb, M)) {
      atomicOr(status, MGC_ST_PIVOT);
      return;
    }
    for (int r = 0; r < nb * nb; ++r) G[(size_t)k * nb * nb + r] = M[r];
  }
}

}  // namespace

cudaError_t launch_setup_axis(const AxisSetup& a, cudaStream_t st) {
  int m = a.n - 1;
  k_setup_axis<<<(m + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_setup_diag(int mx, int my, int stride, int fine_mx, const cplx* dx, const cplx* dy,
                              const cplx* v1, const cplx* v2, const cplx* v12, double E, double omega,
                              cplx* D, cplx* Dinv, int* status, cudaStream_t st) {
  k_setup_diag<<<dim3((mx + 31) / 32, (my + 7) / 8), dim3(32, 8), 0, st>>>(mx, my, stride, fine_mx, dx, dy, v1, v2,
                                                                           v12, E, omega, D, Dinv, status);
  return cudaGetLastError();
}

cudaError_t launch_coarse_inverse(const StencilView& s, cplx* aug, cplx* Ainv, int* status, cudaStream_t st) {
  k_coarse_inverse<<<1, 1024, 0, st>>>(s, aug, Ainv, status);
  return cudaGetLastError();
}

size_t bound_states_scratch(int m, int nb) {
  // d, e + per state (u0, u1, u2, mu, x) + per state int pivots
  return sizeof(cplx) * ((size_t)2 * m + (size_t)nb * 5 * m) + sizeof(int) * (size_t)nb * m;
}

cudaError_t launch_bound_states(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                                const cplx* w, int nb, cplx* lam, cplx* phi, cplx* scratch, int* status,
                                cudaStream_t st) {
  k_bound_states<<<1, 32, 0, st>>>(m, west, east, diag, v, w, nb, lam, phi, scratch, status);
  return cudaGetLastError();
}

cudaError_t launch_weight_states(int m, int nb, const cplx* w, const cplx* phi, cplx* wphi, cudaStream_t st) {
  k_weight_states<<<(m * nb + 255) / 256, 256, 0, st>>>(m, nb, w, phi, wphi);
  return cudaGetLastError();
}

cudaError_t launch_channel_potentials(int mx, int my, int nb, const cplx* wphi, const cplx* phi,
                                      const cplx* wvphi, const cplx* vphi, const cplx* v12,
                                      cplx* VA, cplx* VB, cudaStream_t st) {
  const int npairs = nb * (nb + 1) / 2;
  // V^A_ab(y_j) = sum_i w_i phi_a(i) phi_b(i) V12(j, i)
  k_channel_potentials<<<dim3(my, npairs), 256, 0, st>>>(my, mx, nb, mx, 1, wphi, phi, v12, VA);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // V^B_ab(x_i) = sum_j w_j vphi_a(j) vphi_b(j) V12(j, i)
  k_channel_potentials<<<dim3(mx, npairs), 256, 0, st>>>(mx, my, nb, 1, mx, wvphi, vphi, v12, VB);
  return cudaGetLastError();
}

cudaError_t launch_channel_factor(int m, int nb, const cplx* diag, const cplx* v, double E, const cplx* lam,
                                  const cplx* Vc, const cplx* a, const cplx* c, cplx* G, int* status,
                                  cudaStream_t st) {
  k_channel_factor<<<1, 1, 0, st>>>(m, nb, diag, v, E, lam, Vc, a, c, G, status);
  return cudaGetLastError();
}
