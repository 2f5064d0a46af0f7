// Setup kernels of MG-CCCS (run once per grid / potential / energy).
//
//  * ECS node coordinates and the 3-point nonuniform second-difference coefficients
//    per axis and level (Sec. 2.5, Eq. (11)); coarse levels optionally on a rotated
//    contour.
//  * Diagonal D of H - E and omega/D per node, potentials injected at coincident nodes.
//  * Dense inverse of the coarsest-level operator (Gauss-Jordan, partial pivoting).
//  * Bound states of H1, H2 (Eq. (9)): all eigenvalues by root-free implicit QR on the
//    squared off-diagonals (Pal-Walker-Kahan form) applied without conjugation to the
//    complex-symmetric tridiagonal; the n_b with smallest real part are refined by
//    inverse and Rayleigh-quotient iteration with a pivoted tridiagonal LU, normalised
//    bilinearly, int phi^2 dz = 1 (Sec. 3.1, Remark 3), then two shift-and-invert steps
//    and a bilinear Rayleigh quotient (Sec. 5.1.2, Sec. 5.2).
//  * Channel potentials V^A, V^B (Sec. 4.2) and the cyclic-reduction factors of the
//    coupled-channel systems (Eqs. (28)-(29)).
#include <algorithm>

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

// flag := 1 if a[k] != b[k] for some k (bitwise comparison of the values).
__global__ void k_compare(int n, const cplx* __restrict__ a, const cplx* __restrict__ b, int* flag) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && (a[k].x != b[k].x || a[k].y != b[k].y)) atomicOr(flag, 1);
}

// flag := 1 if some node of the uniform box has a complex diagonal.
__global__ void k_box_real_check(int mx, int ux, int uy, const cplx* __restrict__ D, int* flag) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  if (i >= ux || j >= uy) return;
  if (D[(size_t)j * mx + i].y != 0.0) atomicOr(flag, 1);
}

// Dense inverse of the coarsest operator by Gauss-Jordan elimination with partial
// pivoting on the augmented matrix [A | I] (nc x 2nc, row-major, in global memory),
// one pivot per pair of launches: k_gj_pivot (one block: pivot search, row swap, row
// scaling, multiplier column) and k_gj_eliminate (all SMs: rank-1 update of the
// columns right of the pivot).  A zero pivot sets MGC_ST_PIVOT and every later launch
// of the elimination returns at once.

__global__ void k_gj_assemble(StencilView s, cplx* __restrict__ aug) {
  const int nc = s.mx * s.my;
  const long long w2 = 2LL * nc;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nc * w2;
       q += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(q / w2), c = (int)(q % w2);
    const int i = p % s.mx, j = p / s.mx;
    cplx v = cmk(0.0, 0.0);
    if (c == p) v = s.D[p];
    else if (i > 0 && c == p - 1) v = s.west_x[i];
    else if (i + 1 < s.mx && c == p + 1) v = s.east_x[i];
    else if (j > 0 && c == p - s.mx) v = s.west_y[j];
    else if (j + 1 < s.my && c == p + s.mx) v = s.east_y[j];
    else if (c == nc + p) v = cmk(1.0, 0.0);
    aug[q] = v;
  }
}

__global__ void __launch_bounds__(1024) k_gj_pivot(int nc, cplx* __restrict__ aug, cplx* __restrict__ fac, int k,
                                                   int* __restrict__ status) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  const int t = threadIdx.x;
  const long long w2 = 2LL * nc;
  if (*status & MGC_ST_PIVOT) return;
  // pivot search over rows k..nc-1 (largest modulus, lowest index on ties)
  double best = -1.0;
  int bi = k;
  for (int r = k + t; r < nc; r += blockDim.x) {
    const double v = cmod(aug[r * w2 + k]);
    if (v > best) { best = v; bi = r; }
  }
  sval[t] = best;
  sidx[t] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) {
      const double v2 = sval[t + o];
      const int i2 = sidx[t + o];
      if (v2 > sval[t] || (v2 == sval[t] && i2 < sidx[t])) { sval[t] = v2; sidx[t] = i2; }
    }
    __syncthreads();
  }
  const int piv = sidx[0];
  if (sval[0] == 0.0) {
    if (t == 0) atomicOr(status, MGC_ST_PIVOT);
    return;
  }
  if (piv != k)
    for (int c = k + t; c < w2; c += blockDim.x) {
      const cplx a = aug[k * w2 + c];
      aug[k * w2 + c] = aug[piv * w2 + c];
      aug[piv * w2 + c] = a;
    }
  __syncthreads();
  const cplx pv = aug[k * w2 + k];
  __syncthreads();
  for (int c = k + t; c < w2; c += blockDim.x) aug[k * w2 + c] = cdiv(aug[k * w2 + c], pv);
  for (int r = t; r < nc; r += blockDim.x) fac[r] = r == k ? cmk(0.0, 0.0) : aug[r * w2 + k];
}

__global__ void k_gj_eliminate(int nc, cplx* __restrict__ aug, const cplx* __restrict__ fac, int k,
                               const int* __restrict__ status) {
  if (*status & MGC_ST_PIVOT) return;
  const long long w2 = 2LL * nc;
  const long long w = w2 - k - 1;                    // columns right of the pivot
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nc * w;
       q += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(q / w);
    if (r == k) continue;
    const long long c = k + 1 + q % w;
    aug[r * w2 + c] = cfms(fac[r], aug[k * w2 + c], aug[r * w2 + c]);
  }
}

__global__ void k_gj_extract(int nc, const cplx* __restrict__ aug, cplx* __restrict__ Ainv) {
  const long long w2 = 2LL * nc;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)nc * nc;
       q += (long long)gridDim.x * blockDim.x) {
    const long long r = q / nc, c = q % nc;
    Ainv[q] = aug[r * w2 + nc + c];
  }
}

// ---- bound states ---------------------------------------------------------------

// 1/z = conj(z)/|z|^2 (magnitudes here stay far from under/overflow).
__device__ __forceinline__ cplx crecip(cplx z) {
  const double q = 1.0 / (z.x * z.x + z.y * z.y);
  return cmk(z.x * q, -z.y * q);
}

// Eigenvalues of the complex-symmetric tridiagonal with diagonal a[0..m) and squared
// off-diagonals b2[k] (coupling k and k+1; the squares are the products east_k west_{k+1},
// so no square root is taken) by implicit QR sweeps in the root-free form of Pal,
// Walker and Kahan (B. N. Parlett, The Symmetric Eigenvalue Problem, Sec. 8-15), applied
// without conjugation, with a Wilkinson shift from the trailing 2x2 block and deflation
// at the bottom of the unreduced block.  a is overwritten with the eigenvalues.
// Returns false on a zero pivot or when the sweep budget is exhausted.
__device__ bool qr_rootfree_eigenvalues(int m, cplx* a, cplx* b2) {
  const double eps2 = 4.93038065763132e-32;          // (2^-52)^2
  long long budget = 40LL * m + 100;
  int hi = m - 1;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0 && cabs1(b2[lo - 1]) > eps2 * cabs1(a[lo - 1]) * cabs1(a[lo])) --lo;
    if (lo == hi) {
      --hi;
      continue;
    }
    if (--budget < 0) return false;
    // shift: eigenvalue of the trailing 2x2 block nearest a[hi]
    const cplx dlt = cscal(0.5, csub(a[hi - 1], a[hi]));
    const cplx rt = csqrt_p(cadd(cmul(dlt, dlt), b2[hi - 1]));
    const cplx dp = cadd(dlt, rt), dm = csub(dlt, rt);
    const cplx den = (cabs2(dp) >= cabs2(dm)) ? dp : dm;
    const cplx sigma = (den.x == 0.0 && den.y == 0.0) ? a[hi] : csub(a[hi], cmul(b2[hi - 1], crecip(den)));
    // one root-free QR sweep over lo..hi
    cplx c2 = cmk(1.0, 0.0), s2 = cmk(0.0, 0.0);
    cplx gam = csub(a[lo], sigma);
    cplx p = cmul(gam, gam);
    for (int k = lo; k < hi; ++k) {
      const cplx r = cadd(p, b2[k]);
      if (r.x == 0.0 && r.y == 0.0) return false;
      if (k > lo) b2[k - 1] = cmul(s2, r);
      const cplx c2old = c2;
      const cplx rinv = crecip(r);
      c2 = cmul(p, rinv);
      s2 = cmul(b2[k], rinv);
      const cplx gold = gam;
      const cplx alpha = csub(a[k + 1], sigma);
      gam = csub(cmul(c2, alpha), cmul(s2, gold));
      a[k] = cadd(csub(cadd(gold, alpha), gam), sigma);
      p = (c2.x == 0.0 && c2.y == 0.0) ? cmul(c2old, b2[k]) : cmul(cmul(gam, gam), crecip(c2));
    }
    b2[hi - 1] = cmul(s2, p);
    a[hi] = cadd(gam, sigma);
  }
  for (int k = 0; k < m; ++k)
    if (!isfinite(a[k].x) || !isfinite(a[k].y)) return false;
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

// bilinear Rayleigh quotient x^T W H x / x^T W x (x not normalised)
__device__ cplx rayleigh_ratio(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                               const cplx* w, const cplx* x) {
  cplx num = cmk(0.0, 0.0), den = cmk(0.0, 0.0);
  for (int k = 0; k < m; ++k) {
    cplx hx = cmul(cadd(diag[k], v[k]), x[k]);
    if (k > 0) hx = cfma(west[k], x[k - 1], hx);
    if (k + 1 < m) hx = cfma(east[k], x[k + 1], hx);
    cplx xw = cmul(x[k], w[k]);
    num = cfma(xw, hx, num);
    den = cfma(xw, x[k], den);
  }
  return cdiv(num, den);
}

// Eigenvalues by root-free QR (thread 0), the n_b with the smallest real part; then per
// state (thread q): inverse iteration at the eigenvalue, Rayleigh-quotient iteration,
// bilinear normalisation, and the paper's two shift-and-invert steps.  Coinciding refined
// eigenvalues flag a failure.
__global__ void __launch_bounds__(32) k_bound_states(int m, const cplx* __restrict__ west,
                                                     const cplx* __restrict__ east, const cplx* __restrict__ diag,
                                                     const cplx* __restrict__ v, const cplx* __restrict__ w, int nb,
                                                     cplx* __restrict__ lam, cplx* __restrict__ phi,
                                                     cplx* __restrict__ scratch, int* status,
                                                     const cplx* __restrict__ eig) {
  __shared__ cplx sel[MGC_MAX_NB];
  __shared__ cplx fin_l[MGC_MAX_NB];
  __shared__ int ok;
  const int q = threadIdx.x;
  cplx* d = scratch;            // m
  cplx* e2 = scratch + m;       // m
  if (q == 0) {
    if (eig) {
      // all eigenvalues given (the Ehrlich-Aberth iteration of kernels_eig.cu)
      for (int k = 0; k < m; ++k) {
        d[k] = eig[k];
        e2[k] = cmk(0.0, 0.0);
      }
      ok = 1;
    } else {
      // squared off-diagonals of the symmetric form: e_k^2 = east_k * west_{k+1}
      for (int k = 0; k < m; ++k) {
        d[k] = cadd(diag[k], v[k]);
        e2[k] = (k + 1 < m) ? cmul(east[k], west[k + 1]) : cmk(0.0, 0.0);
      }
      ok = qr_rootfree_eigenvalues(m, d, e2) ? 1 : 0;
    }
    if (ok) {
      // the nb eigenvalues with the smallest real part, ascending (ties: lower index)
      for (int s = 0; s < nb; ++s) {
        int kb = -1;
        for (int k = 0; k < m; ++k) {
          if (e2[k].x == 1.0e300) continue;            // already taken
          if (kb < 0 || d[k].x < d[kb].x) kb = k;
        }
        sel[s] = d[kb];
        e2[kb] = cmk(1.0e300, 0.0);
      }
    } else {
      atomicOr(status, MGC_ST_EIG);
    }
  }
  __syncthreads();
  if (ok && q < nb) {
    cplx* base = scratch + 2 * m + (size_t)q * 5 * m;
    TriLU lu{base, base + m, base + 2 * m, base + 3 * m,
             reinterpret_cast<int*>(scratch + 2 * m + (size_t)nb * 5 * m) + (size_t)q * m};
    cplx* x = base + 4 * m;
    double scale = 0.0;
    for (int k = 0; k < m; ++k) scale = fmax(scale, cabs1(cadd(diag[k], v[k])));
    const double tiny = 1e-300 + 1e-16 * scale;
    cplx lmb = sel[q];
    for (int k = 0; k < m; ++k) x[k] = cmk(1.0, 0.0);
    // two inverse-iteration steps at the QR eigenvalue
    tri_lu(m, west, east, diag, v, lmb, lu);
    for (int it = 0; it < 2; ++it) {
      tri_solve(m, lu, x, tiny);
      max_normalise(m, x);
    }
    // Rayleigh-quotient iteration to the double-precision eigenvalue
    for (int it = 0; it < 6; ++it) {
      cplx ln = rayleigh_ratio(m, west, east, diag, v, w, x);
      const bool conv = cabs1(csub(ln, lmb)) <= 1e-14 * fmax(1.0, cabs1(ln));
      lmb = ln;
      tri_lu(m, west, east, diag, v, lmb, lu);
      tri_solve(m, lu, x, tiny);
      max_normalise(m, x);
      if (conv) break;
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
    fin_l[q] = lmb;
    if (!fin) atomicOr(status, MGC_ST_EIG);
  }
  __syncthreads();
  if (ok && q == 0) {
    // two states that refined onto the same eigenvalue mean the estimates were too poor
    for (int a = 0; a < nb; ++a)
      for (int b = a + 1; b < nb; ++b)
        if (cabs1(csub(fin_l[a], fin_l[b])) <= 1e-10 * fmax(1.0, cabs1(fin_l[a]))) atomicOr(status, MGC_ST_EIG);
  }
}

// All eigenvalues by the FP64 root-free QR (one thread), for the spectrum entry point.
__global__ void k_qr_spectrum(int m, const cplx* __restrict__ west, const cplx* __restrict__ east,
                              const cplx* __restrict__ diag, const cplx* __restrict__ v, cplx* __restrict__ scratch,
                              cplx* __restrict__ out, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cplx* d = scratch;
  cplx* e2 = scratch + m;
  for (int k = 0; k < m; ++k) {
    d[k] = cadd(diag[k], v[k]);
    e2[k] = (k + 1 < m) ? cmul(east[k], west[k + 1]) : cmk(0.0, 0.0);
  }
  if (!qr_rootfree_eigenvalues(m, d, e2)) {
    atomicOr(status, MGC_ST_EIG);
    return;
  }
  for (int k = 0; k < m; ++k) out[k] = d[k];
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

// C = A B for n x n row-major blocks.
__device__ void small_matmul(int n, const cplx* A, const cplx* B, cplx* C) {
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      cplx acc = cmk(0.0, 0.0);
      for (int k = 0; k < n; ++k) acc = cfma(A[r * n + k], B[k * n + c], acc);
      C[r * n + c] = acc;
    }
}

// Cyclic-reduction factors of the coupled-channel system along one axis (one block):
// B_k = (diag_k + v_k - E) I + diag(lam) + Vc_k, A_k = a_k I, C_k = c_k I, rows padded
// with identity to M = 2^q - 1.  `scratch` holds the current A, B, C of rows 0..M.
// Parallel cyclic reduction factors of one coupled-channel system (Eqs. (28)-(29)):
// rows k = 0..m-1 of A_k x_{k-1} + B_k x_k + C_k x_{k+1} = r_k with n_b x n_b blocks
// (A_k, C_k the 1D Laplacian couplings times the identity, B_k the channel block).
// Level l (stride s = 2^l) eliminates every row's couplings to k +- s with the rows
// k +- s themselves: alpha = A_k B_{k-s}^{-1}, gamma = C_k B_{k+s}^{-1},
//   A_k <- -alpha A_{k-s},  B_k <- B_k - alpha C_{k-s} - gamma A_{k+s},  C_k <- -gamma C_{k+s};
// after ceil(log2 m) levels no coupling is left and x_k = B_k^{-1} r_k.  One block, the
// rows of a level in parallel, double-buffered blocks.
__global__ void __launch_bounds__(256) k_channel_factor_pcr(CRSystem S, const cplx* __restrict__ diag,
                                                            const cplx* __restrict__ v, double E,
                                                            const cplx* __restrict__ lam, const cplx* __restrict__ Vc,
                                                            const cplx* __restrict__ sub, const cplx* __restrict__ sup,
                                                            cplx* __restrict__ scratch, int* status) {
  const int nb = S.nb, nb2 = nb * nb, m = S.m;
  const size_t blk = (size_t)m * nb2;
  cplx* Ab[2] = {scratch, scratch + 3 * blk};
  cplx* Bb[2] = {scratch + blk, scratch + 4 * blk};
  cplx* Cb[2] = {scratch + 2 * blk, scratch + 5 * blk};
  cplx* Binv = scratch + 6 * blk;
  const int t0 = threadIdx.x, nt = blockDim.x;
  for (int k = t0; k < m; k += nt) {
    cplx* A = Ab[0] + (size_t)k * nb2;
    cplx* B = Bb[0] + (size_t)k * nb2;
    cplx* C = Cb[0] + (size_t)k * nb2;
    cplx base = cadd(diag[k], v[k]);
    base.x -= E;
    for (int r = 0; r < nb; ++r)
      for (int c = 0; c < nb; ++c) {
        cplx val = Vc[((size_t)k * nb + r) * nb + c];
        if (r == c) val = cadd(val, cadd(base, lam[r]));
        B[r * nb + c] = val;
        A[r * nb + c] = (r == c && k > 0) ? sub[k] : cmk(0.0, 0.0);
        C[r * nb + c] = (r == c && k < m - 1) ? sup[k] : cmk(0.0, 0.0);
      }
  }
  __syncthreads();
  cplx T1[MGC_MAX_NB * MGC_MAX_NB], T2[MGC_MAX_NB * MGC_MAX_NB], al[MGC_MAX_NB * MGC_MAX_NB],
      ga[MGC_MAX_NB * MGC_MAX_NB];
  int cur = 0;
  for (int l = 0; l < S.pq; ++l) {
    const int s = 1 << l;
    const cplx* A = Ab[cur];
    const cplx* B = Bb[cur];
    const cplx* C = Cb[cur];
    for (int k = t0; k < m; k += nt) {
      for (int r = 0; r < nb2; ++r) T1[r] = B[(size_t)k * nb2 + r];
      if (!small_inverse(nb, T1)) {
        atomicOr(status, MGC_ST_PIVOT);
        for (int r = 0; r < nb2; ++r) T1[r] = cmk(0.0, 0.0);
      }
      for (int r = 0; r < nb2; ++r) Binv[(size_t)k * nb2 + r] = T1[r];
    }
    __syncthreads();
    cplx* A2 = Ab[cur ^ 1];
    cplx* B2 = Bb[cur ^ 1];
    cplx* C2 = Cb[cur ^ 1];
    for (int k = t0; k < m; k += nt) {
      const bool lo = k - s >= 0, hi = k + s < m;
      if (lo) small_matmul(nb, A + (size_t)k * nb2, Binv + (size_t)(k - s) * nb2, al);
      else for (int r = 0; r < nb2; ++r) al[r] = cmk(0.0, 0.0);
      if (hi) small_matmul(nb, C + (size_t)k * nb2, Binv + (size_t)(k + s) * nb2, ga);
      else for (int r = 0; r < nb2; ++r) ga[r] = cmk(0.0, 0.0);
      cplx* pa = S.pa + ((size_t)l * m + k) * nb2;
      cplx* pg = S.pg + ((size_t)l * m + k) * nb2;
      for (int r = 0; r < nb2; ++r) {
        pa[r] = al[r];
        pg[r] = ga[r];
        B2[(size_t)k * nb2 + r] = B[(size_t)k * nb2 + r];
        A2[(size_t)k * nb2 + r] = cmk(0.0, 0.0);
        C2[(size_t)k * nb2 + r] = cmk(0.0, 0.0);
      }
      if (lo) {
        small_matmul(nb, al, C + (size_t)(k - s) * nb2, T1);
        small_matmul(nb, al, A + (size_t)(k - s) * nb2, T2);
        for (int r = 0; r < nb2; ++r) {
          B2[(size_t)k * nb2 + r] = csub(B2[(size_t)k * nb2 + r], T1[r]);
          A2[(size_t)k * nb2 + r] = cneg(T2[r]);
        }
      }
      if (hi) {
        small_matmul(nb, ga, A + (size_t)(k + s) * nb2, T1);
        small_matmul(nb, ga, C + (size_t)(k + s) * nb2, T2);
        for (int r = 0; r < nb2; ++r) {
          B2[(size_t)k * nb2 + r] = csub(B2[(size_t)k * nb2 + r], T1[r]);
          C2[(size_t)k * nb2 + r] = cneg(T2[r]);
        }
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int k = t0; k < m; k += nt) {
    for (int r = 0; r < nb2; ++r) T1[r] = Bb[cur][(size_t)k * nb2 + r];
    if (!small_inverse(nb, T1)) {
      atomicOr(status, MGC_ST_PIVOT);
      for (int r = 0; r < nb2; ++r) T1[r] = cmk(0.0, 0.0);
    }
    for (int r = 0; r < nb2; ++r) S.pbinv[(size_t)k * nb2 + r] = T1[r];
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

cudaError_t launch_compare(int n, const cplx* a, const cplx* b, int* flag, cudaStream_t st) {
  k_compare<<<(n + 255) / 256, 256, 0, st>>>(n, a, b, flag);
  return cudaGetLastError();
}

cudaError_t launch_box_real_check(const StencilView& s, int* flag, cudaStream_t st) {
  if (s.cx.u <= 0 || s.cy.u <= 0) return cudaSuccess;
  k_box_real_check<<<dim3((s.cx.u + 31) / 32, (s.cy.u + 7) / 8), dim3(32, 8), 0, st>>>(s.mx, s.cx.u, s.cy.u, s.D,
                                                                                        flag);
  return cudaGetLastError();
}

size_t coarse_inverse_scratch(int nc) { return (size_t)nc * 2 * nc + nc; }

cudaError_t launch_coarse_inverse(const StencilView& s, cplx* aug, cplx* Ainv, int* status, cudaStream_t st) {
  const int nc = s.mx * s.my;
  cplx* fac = aug + (size_t)nc * 2 * nc;
  const long long total = 2LL * nc * nc;
  const int grid = (int)std::min<long long>((total + 255) / 256, 8LL * mgc_sm_count());
  k_gj_assemble<<<grid, 256, 0, st>>>(s, aug);
  cudaError_t e = cudaGetLastError();
  for (int k = 0; k < nc && e == cudaSuccess; ++k) {
    k_gj_pivot<<<1, 1024, 0, st>>>(nc, aug, fac, k, status);
    const long long work = (long long)nc * (2LL * nc - k - 1);
    const int g = (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 8LL * mgc_sm_count()));
    k_gj_eliminate<<<g, 256, 0, st>>>(nc, aug, fac, k, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  k_gj_extract<<<grid, 256, 0, st>>>(nc, aug, Ainv);
  return cudaGetLastError();
}

size_t bound_states_scratch(int m, int nb) {
  // d, e^2 + per state (u0, u1, u2, mu, x) + per state int pivots
  return sizeof(cplx) * ((size_t)2 * m + (size_t)nb * 5 * m) + sizeof(int) * (size_t)nb * m;
}

cudaError_t launch_bound_states(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                                const cplx* w, int nb, cplx* lam, cplx* phi, cplx* scratch, int* status,
                                cudaStream_t st, const cplx* eig) {
  k_bound_states<<<1, 32, 0, st>>>(m, west, east, diag, v, w, nb, lam, phi, scratch, status, eig);
  return cudaGetLastError();
}

cudaError_t launch_qr_spectrum(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                               cplx* scratch, cplx* out, int* status, cudaStream_t st) {
  k_qr_spectrum<<<1, 32, 0, st>>>(m, west, east, diag, v, scratch, out, status);
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

int pcr_levels(int m) {
  int q = 0;
  while ((1 << q) < m) ++q;
  return q;
}

size_t channel_factor_pcr_scratch(int m, int nb) { return (size_t)7 * m * nb * nb; }

cudaError_t launch_channel_factor_pcr(const CRSystem& S, const cplx* diag, const cplx* v, double E, const cplx* lam,
                                      const cplx* Vc, const cplx* a, const cplx* c, cplx* scratch, int* status,
                                      cudaStream_t st) {
  k_channel_factor_pcr<<<1, 256, 0, st>>>(S, diag, v, E, lam, Vc, a, c, scratch, status);
  return cudaGetLastError();
}

