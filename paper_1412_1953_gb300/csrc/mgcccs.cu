// Host side of the MG-CCCS library: workspace layout, setup sequence, V-cycle
// recursion, CCCS sequence, solve loop and the C ABI declared in include/mgcccs.h.
// Every numerical step runs in the kernels of kernels_*.cu; this file only orders
// launches on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace {

struct LevelBufs {
  int nxc, nyc;            // cells
  int mx, my;              // interior nodes
  double gamma;            // contour rotation of this level
  cplx *west_x, *east_x, *diag_x, *w_x;
  cplx *west_y, *east_y, *diag_y, *w_y;
  cplx *D, *Dinv;
  cplx *u, *f, *t, *r;     // level 0: only t, r (u and f belong to the caller)
  StencilView sv;
  // complex64 copies for the mixed-precision preconditioner (precision == 1)
  float2 *west_x32, *east_x32, *west_y32, *east_y32, *D32, *Dinv32;
  float2 *u32, *f32, *t32, *r32;
  StencilView32 sv32;
};

}  // namespace

struct mgcccs_handle {
  mgcccs_params p;
  cudaStream_t st;
  int L;
  LevelBufs lv[MGC_MAX_LEVELS];
  int nc;
  cplx* Ainv;              // dense inverse of the coarsest operator (nc <= MGC_MAX_COARSE)
  cplx* aug;
  int coarse_bp;           // 1: larger coarsest grid, solved by block cyclic reduction
  cplx *bp_fac, *bp_scr, *bp_buf;
  int nb;
  cplx *lam, *mu, *phi, *vphi, *wphi, *wvphi, *VA, *VB;
  CRSystem crA, crB;       // channel A (along y, x bound states), channel B (along x)
  cplx* cr_scratch;
  cplx* eig_scratch;
  cplx *eig_ab, *eig_vals;  // Ehrlich-Aberth scratch and its eigenvalues (one axis at a time)
  cplx *v1c, *v2c;          // copies of V1, V2 (the spectrum entry point reads them)
  int eig_fallbacks;        // axes whose eigenvalues needed the QR fallback
  CCView cc;
  double* norm_part;
  int norm_nparts;
  double* norm_out;
  int* status;
  cplx *hu, *hf;
  cplx* wdot_part;         // partials of the weighted dot products
  // mixed precision: complex64 states, projections and GMRES basis; FP64 outer residual
  int mixed;
  double inner_rtol;
  float2 *phi32, *vphi32, *wphi32, *wvphi32;
  CCView32 cc32;
  float2 *V32, *Z32, *e32;
  cplx* r64;
  cudaGraphExec_t step_exec32[MGC_MAX_RESTART];
  long long step_launches32[MGC_MAX_RESTART];
  // GMRES(m) outer solver
  int km;
  int kr_nblk;
  long long kld;            // pitch of the Krylov basis vectors: N rounded up to 32 entries, so
                            // every vector starts 256-byte aligned and complex64 pairs load as 16 bytes
  cplx *V, *Z, *Hh, *cs, *sn, *g, *y, *hc, *dotpart;
  int* gate;
  cudaStream_t cap_st;                       // capture stream for the step graphs
  cudaGraphExec_t step_exec[MGC_MAX_RESTART];
  long long step_launches[MGC_MAX_RESTART];
  cudaEvent_t ev[2];
  double* est_host;                          // pinned, one residual estimate per step + |r|^2
  // device-driven solves: control record, its pinned staging copy, capture streams, and
  // the kernel counts of the solve graph's parts (prologue, restart, cycle, step)
  SolveCtl* ctl;
  SolveCtl* ctl_host;
  cudaStream_t gst[2];
  bool device_loop;
  const double* pend_norm2;                  // set: the next fine zero-start sweep first normalises f
  int driver;                                // MGCCCS_DRIVER_GRAPH or MGCCCS_DRIVER_HOST
  cudaGraphExec_t solve_exec[4];             // device-driven solve graphs by (u, f) pointers
  const void *solve_u[4], *solve_f[4];
  int solve_next;
  long long sg_pro, sg_outer, sg_cycle, sg_step, sg_dgks;
  cudaGraphConditionalHandle dgks_cond[MGC_MAX_RESTART];
  long long launches;
};

namespace {

constexpr size_t kAlign = 256;

// Two-pass workspace carving: with base == nullptr only the size is accumulated.
struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* ptr = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return ptr;
  }
};

bool valid_params(const mgcccs_params* p) {
  if (!p) return false;
  if (p->levels < 1 || p->levels > MGC_MAX_LEVELS) return false;
  if (p->nx < 2 || p->ny < 2) return false;
  const int s = 1 << (p->levels - 1);
  if (p->nx % s || p->ny % s) return false;
  const int cx = p->nx / s, cy = p->ny / s;
  if (cx < 2 || cy < 2) return false;
  if ((long long)(cx - 1) * (cy - 1) > MGC_MAX_COARSE && !bpcr_fits(cx - 1, cy - 1)) return false;
  if (p->n_b < 0 || p->n_b > MGC_MAX_NB || p->n_b > p->nx - 1 || p->n_b > p->ny - 1) return false;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 > 64) return false;
  if (!(p->Lx > 0) || !(p->Ly > 0) || !std::isfinite(p->E) || !std::isfinite(p->omega)) return false;
  if (!std::isfinite(p->theta) || !std::isfinite(p->coarse_gamma)) return false;
  if (p->krylov_restart < 0 || p->krylov_restart > MGC_MAX_RESTART) return false;
  if (p->precision < 0 || p->precision > 1) return false;
  if (p->precision == 1 && p->krylov_restart < 1) return false;
  if (!(p->inner_rtol >= 0.0) || !(p->inner_rtol < 1.0)) return false;
  return true;
}

void layout(mgcccs_handle* h, Carver& cv) {
  const mgcccs_params& p = h->p;
  const int L = p.levels;
  for (int l = 0; l < L; ++l) {
    LevelBufs& b = h->lv[l];
    b.nxc = p.nx >> l;
    b.nyc = p.ny >> l;
    b.mx = b.nxc - 1;
    b.my = b.nyc - 1;
    const size_t n2 = (size_t)b.mx * b.my;
    b.west_x = cv.take<cplx>(b.mx); b.east_x = cv.take<cplx>(b.mx);
    b.diag_x = cv.take<cplx>(b.mx); b.w_x = cv.take<cplx>(b.mx);
    b.west_y = cv.take<cplx>(b.my); b.east_y = cv.take<cplx>(b.my);
    b.diag_y = cv.take<cplx>(b.my); b.w_y = cv.take<cplx>(b.my);
    b.D = cv.take<cplx>(n2);
    b.Dinv = cv.take<cplx>(n2);
    b.t = cv.take<cplx>(n2);
    b.r = cv.take<cplx>(n2);
    if (l > 0) {
      b.u = cv.take<cplx>(n2);
      b.f = cv.take<cplx>(n2);
    } else {
      b.u = b.f = nullptr;
    }
    if (p.precision == 1) {
      b.west_x32 = cv.take<float2>(b.mx); b.east_x32 = cv.take<float2>(b.mx);
      b.west_y32 = cv.take<float2>(b.my); b.east_y32 = cv.take<float2>(b.my);
      b.D32 = cv.take<float2>(n2);
      b.Dinv32 = cv.take<float2>(n2);
      b.t32 = cv.take<float2>(n2);
      b.r32 = cv.take<float2>(n2);
      b.u32 = l > 0 ? cv.take<float2>(n2) : nullptr;
      b.f32 = l > 0 ? cv.take<float2>(n2) : nullptr;
    }
  }
  h->mixed = p.precision == 1;
  h->inner_rtol = p.inner_rtol > 0.0 ? p.inner_rtol : 1e-5;
  const LevelBufs& c = h->lv[L - 1];
  h->nc = c.mx * c.my;
  h->coarse_bp = h->nc > MGC_MAX_COARSE;
  if (h->coarse_bp) {
    h->Ainv = h->aug = nullptr;
    h->bp_fac = cv.take<cplx>(bpcr_factor_entries(c.mx, c.my));
    h->bp_scr = cv.take<cplx>(bpcr_scratch_entries(c.mx, c.my));
    h->bp_buf = cv.take<cplx>((size_t)2 * h->nc);
  } else {
    h->Ainv = cv.take<cplx>((size_t)h->nc * h->nc);
    h->aug = cv.take<cplx>(coarse_inverse_scratch(h->nc));
    h->bp_fac = h->bp_scr = h->bp_buf = nullptr;
  }
  {
    const int mm = h->lv[0].mx > h->lv[0].my ? h->lv[0].mx : h->lv[0].my;
    h->v1c = cv.take<cplx>(h->lv[0].mx);
    h->v2c = cv.take<cplx>(h->lv[0].my);
    h->eig_ab = cv.take<cplx>(eig_scratch_entries(mm));
    h->eig_vals = cv.take<cplx>(mm);
  }
  const int nb = p.n_b, mx = h->lv[0].mx, my = h->lv[0].my;
  h->nb = nb;
  if (nb > 0) {
    h->lam = cv.take<cplx>(nb);
    h->mu = cv.take<cplx>(nb);
    h->phi = cv.take<cplx>((size_t)nb * mx);
    h->vphi = cv.take<cplx>((size_t)nb * my);
    h->wphi = cv.take<cplx>((size_t)nb * mx);
    h->wvphi = cv.take<cplx>((size_t)nb * my);
    h->VA = cv.take<cplx>((size_t)my * nb * nb);
    h->VB = cv.take<cplx>((size_t)mx * nb * nb);
    for (int c = 0; c < 2; ++c) {
      CRSystem& S = c == 0 ? h->crA : h->crB;
      S.m = c == 0 ? my : mx;
      S.nb = nb;
      const size_t nb2 = (size_t)nb * nb;
      S.pq = pcr_levels(S.m);
      S.pa = cv.take<cplx>((size_t)S.pq * S.m * nb2);
      S.pg = cv.take<cplx>((size_t)S.pq * S.m * nb2);
      S.pbinv = cv.take<cplx>((size_t)S.m * nb2);
    }
    {
      const int mmax = h->crA.m > h->crB.m ? h->crA.m : h->crB.m;
      h->cr_scratch = cv.take<cplx>(channel_factor_pcr_scratch(mmax, nb));
    }
    size_t es = bound_states_scratch(mx > my ? mx : my, nb);
    h->eig_scratch = cv.take<cplx>((es + sizeof(cplx) - 1) / sizeof(cplx));
    CCView& cc = h->cc;
    cc.mx = mx; cc.my = my; cc.nb = nb;
    cc.wphi = h->wphi; cc.wvphi = h->wvphi; cc.phi = h->phi; cc.vphi = h->vphi;
    cc.wvphi64 = h->wvphi;
    cc.Px_part = cv.take<cplx>((size_t)cc_tiles_x(mx) * nb * my);
    cc.Py_part = cv.take<cplx>((size_t)cc_tiles_y(my) * nb * mx);
    cc.Px = cv.take<cplx>((size_t)nb * my);
    cc.Py = cv.take<cplx>((size_t)nb * mx);
    cc.c = cv.take<cplx>((size_t)nb * nb);
    cc.eA = cv.take<cplx>((size_t)nb * my);
    cc.eB = cv.take<cplx>((size_t)nb * mx);
    cc.eAc = cc.eA; cc.eBc = cc.eB;
    h->crA.chan = 0; h->crA.P = cc.Px; h->crA.cmat = cc.c; h->crA.basis = h->vphi;
    h->crB.chan = 1; h->crB.P = cc.Py; h->crB.cmat = cc.c; h->crB.basis = h->phi;
    h->crA.e = cc.eA; h->crA.e32 = nullptr;
    h->crB.e = cc.eB; h->crB.e32 = nullptr;
    if (p.precision == 1) {
      h->phi32 = cv.take<float2>((size_t)nb * mx);
      h->vphi32 = cv.take<float2>((size_t)nb * my);
      h->wphi32 = cv.take<float2>((size_t)nb * mx);
      h->wvphi32 = cv.take<float2>((size_t)nb * my);
      CCView32& c3 = h->cc32;
      c3.mx = mx; c3.my = my; c3.nb = nb;
      c3.wphi = h->wphi32; c3.wvphi = h->wvphi32; c3.phi = h->phi32; c3.vphi = h->vphi32;
      c3.Px_part = cv.take<float2>((size_t)cc_tiles_x(mx) * nb * my);
      c3.Py_part = cv.take<float2>((size_t)cc_tiles_y(my) * nb * mx);
      c3.Px = cc.Px; c3.Py = cc.Py; c3.c = cc.c; c3.eA = cc.eA; c3.eB = cc.eB;
      float2* eA32 = cv.take<float2>((size_t)nb * my);
      float2* eB32 = cv.take<float2>((size_t)nb * mx);
      c3.eAc = eA32; c3.eBc = eB32;
      h->crA.e32 = eA32;
      h->crB.e32 = eB32;
      c3.wvphi64 = h->wvphi;
    }
  }
  StencilView s0{};
  s0.mx = mx; s0.my = my;
  int nparts = residual_norm_blocks(s0);
  int n2b = norm2_blocks((long long)mx * my);
  h->norm_nparts = nparts > n2b ? nparts : n2b;
  const long long N = (long long)mx * my;
  h->km = p.krylov_restart;
  // complex128 Krylov kernels are FP64-bound at 4 blocks per SM; the complex64 update is
  // bound by memory latency and gets 6, which its register count allows
  h->kr_nblk = krylov_blocks(N, p.precision == 1 ? 6 : 4);
  h->kld = (N + 31) / 32 * 32;
  if (h->km > 0) {
    const int m = h->km;
    if (p.precision == 1) {
      h->V32 = cv.take<float2>((size_t)(m + 1) * h->kld);
      h->Z32 = cv.take<float2>((size_t)m * h->kld);
      h->e32 = cv.take<float2>((size_t)N);
      h->r64 = cv.take<cplx>((size_t)N);
    } else {
      h->V = cv.take<cplx>((size_t)(m + 1) * h->kld);
      h->Z = cv.take<cplx>((size_t)m * h->kld);
    }
    h->Hh = cv.take<cplx>((size_t)(m + 1) * m);
    h->cs = cv.take<cplx>(m);
    h->sn = cv.take<cplx>(m);
    h->g = cv.take<cplx>(m + 1);
    h->y = cv.take<cplx>(m);
    h->hc = cv.take<cplx>(m + 1);
    h->dotpart = cv.take<cplx>((size_t)(m + 1) * h->kr_nblk);
    h->gate = cv.take<int>(4);
    h->ctl = cv.take<SolveCtl>(1);
    if (h->kr_nblk > h->norm_nparts) h->norm_nparts = h->kr_nblk;
  }
  h->norm_part = cv.take<double>(h->norm_nparts);
  h->norm_out = cv.take<double>(4);
  h->status = cv.take<int>(4);
  h->hu = cv.take<cplx>((size_t)mx * my);
  h->hf = cv.take<cplx>((size_t)mx * my);
  h->wdot_part = cv.take<cplx>(wdot_blocks((long long)mx * my));
}

// Number of leading interior nodes whose 3-point stencil lies on the unbent part of
// the contour (both adjacent cells real before the level rotation).
int uniform_count(int n, double L, double R0) {
  int m = n - 1, cnt = 0;
  for (int i = 0; i < m; ++i) {
    double x = (double)(i + 2) * L / (double)n;
    if (x <= R0) cnt = i + 1; else break;
  }
  return cnt;
}

// Inner uniform region of one axis and its coefficient (Eq. (11) with equal adjacent
// cells h e^{i gamma}: west = east = -1/(2 h^2) e^{-2 i gamma}).
AxisCoefT<cplx> axis_coef(int n, double L, double R0, double gamma) {
  AxisCoefT<cplx> a;
  const double h = L / n, c = -0.5 / (h * h);
  a.u = uniform_count(n, L, R0);
  a.cin = cmk(c * std::cos(2.0 * gamma), -c * std::sin(2.0 * gamma));
  a.in_real = a.cin.y == 0.0;
  return a;
}

AxisCoefT<float2> axis_coef32(const AxisCoefT<cplx>& a) {
  AxisCoefT<float2> b;
  b.u = a.u; b.in_real = a.in_real;
  b.cin = make_float2((float)a.cin.x, (float)a.cin.y);
  return b;
}

#define MGC_LAUNCH(expr)                         \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    h->launches++;                               \
    if (e_ != cudaSuccess) return MGCCCS_ECUDA;  \
  } while (0)

// every runtime call other than a kernel launch ends a chain of programmatic launches
#define MGC_CUDA(expr)                           \
  do {                                           \
    mgc_not_a_kernel();                          \
    if ((expr) != cudaSuccess) return MGCCCS_ECUDA; \
  } while (0)

int read_status(mgcccs_handle* h) {
  int st = 0;
  MGC_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  MGC_CUDA(cudaStreamSynchronize(h->st));
  if (st & (MGC_ST_PIVOT | MGC_ST_EIG)) return MGCCCS_EBREAKDOWN;
  if (st & MGC_ST_NONFINITE) return MGCCCS_ENONFINITE;
  return MGCCCS_OK;
}

// Bound states of one axis (Eq. (9)): all eigenvalues by the Ehrlich-Aberth iteration
// (parallel; the one-thread FP64 QR when it does not converge), then selection and
// refinement in k_bound_states.
int axis_states(mgcccs_handle* h, int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                const cplx* w, cplx* lam, cplx* phi) {
  bool ok = false;
  MGC_CUDA(eig_aberth(m, west, east, diag, v, h->eig_ab, h->eig_vals, &ok, h->st));
  h->launches += 4;
  if (!ok) h->eig_fallbacks += 1;
  MGC_LAUNCH(launch_bound_states(m, west, east, diag, v, w, h->nb, lam, phi, h->eig_scratch, h->status, h->st,
                                 ok ? h->eig_vals : nullptr));
  return MGCCCS_OK;
}

int do_setup(mgcccs_handle* h, const cplx* v1, const cplx* v2, const cplx* v12, const cplx* lam_in = nullptr,
             const cplx* phi_in = nullptr, const cplx* mu_in = nullptr, const cplx* vphi_in = nullptr) {
  const mgcccs_params& p = h->p;
  cudaStream_t st = h->st;
  MGC_CUDA(cudaMemsetAsync(h->status, 0, 4 * sizeof(int), st));
  MGC_CUDA(cudaMemcpyAsync(h->v1c, v1, sizeof(cplx) * h->lv[0].mx, cudaMemcpyDeviceToDevice, st));
  MGC_CUDA(cudaMemcpyAsync(h->v2c, v2, sizeof(cplx) * h->lv[0].my, cudaMemcpyDeviceToDevice, st));
  h->eig_fallbacks = 0;
  const int fine_mx = h->lv[0].mx;
  for (int l = 0; l < h->L; ++l) {
    LevelBufs& b = h->lv[l];
    b.gamma = (l > 0) ? p.coarse_gamma : 0.0;
    AxisSetup ax{b.nxc, p.Lx, p.R0x, p.theta, b.gamma, b.west_x, b.east_x, b.diag_x, b.w_x};
    AxisSetup ay{b.nyc, p.Ly, p.R0y, p.theta, b.gamma, b.west_y, b.east_y, b.diag_y, b.w_y};
    MGC_LAUNCH(launch_setup_axis(ax, st));
    MGC_LAUNCH(launch_setup_axis(ay, st));
    MGC_LAUNCH(launch_setup_diag(b.mx, b.my, 1 << l, fine_mx, b.diag_x, b.diag_y, v1, v2, v12, p.E, p.omega,
                                 b.D, b.Dinv, h->status, st));
    StencilView& s = b.sv;
    s.mx = b.mx; s.my = b.my;
    s.west_x = b.west_x; s.east_x = b.east_x; s.west_y = b.west_y; s.east_y = b.east_y;
    s.D = b.D; s.Dinv = b.Dinv;
    s.cx = axis_coef(b.nxc, p.Lx, p.R0x, b.gamma);
    s.cy = axis_coef(b.nyc, p.Ly, p.R0y, b.gamma);
    s.keep = 1.0 - p.omega;
    s.rbox = 0;
  }
  // a level whose inner coefficients are real and whose diagonal is real on the inner
  // box uses real arithmetic for D and omega/D there (scan on the device, flag read back)
  for (int l = 0; l < h->L; ++l) {
    StencilView& s = h->lv[l].sv;
    if (s.cx.u > 0 && s.cy.u > 0 && s.cx.in_real && s.cy.in_real) {
      int complex_seen = 0;
      MGC_CUDA(cudaMemsetAsync(h->status + 3, 0, sizeof(int), st));
      MGC_LAUNCH(launch_box_real_check(s, h->status + 3, st));
      MGC_CUDA(cudaMemcpyAsync(&complex_seen, h->status + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
      MGC_CUDA(cudaStreamSynchronize(st));
      s.rbox = complex_seen ? 0 : 1;
    }
  }
  if (h->coarse_bp) {
    MGC_LAUNCH(launch_bpcr_setup(h->lv[h->L - 1].sv, h->bp_fac, h->bp_scr, h->status, st));
  } else {
    MGC_LAUNCH(launch_coarse_inverse(h->lv[h->L - 1].sv, h->aug, h->Ainv, h->status, st));
  }
  if (h->nb > 0) {
    const LevelBufs& b = h->lv[0];
    const int nb = h->nb;
    MGC_CUDA(channel_solve_prepare(nb, h->crA.m > h->crB.m ? h->crA.m : h->crB.m));
    if (lam_in) {
      // states supplied by the caller (a previous setup on the same grid and V1, V2)
      MGC_CUDA(cudaMemcpyAsync(h->lam, lam_in, sizeof(cplx) * nb, cudaMemcpyHostToDevice, st));
      MGC_CUDA(cudaMemcpyAsync(h->mu, mu_in, sizeof(cplx) * nb, cudaMemcpyHostToDevice, st));
      MGC_CUDA(cudaMemcpyAsync(h->phi, phi_in, sizeof(cplx) * nb * b.mx, cudaMemcpyDeviceToDevice, st));
      MGC_CUDA(cudaMemcpyAsync(h->vphi, vphi_in, sizeof(cplx) * nb * b.my, cudaMemcpyDeviceToDevice, st));
    } else {
      int rc = axis_states(h, b.mx, b.west_x, b.east_x, b.diag_x, v1, b.w_x, h->lam, h->phi);
      if (rc) return rc;
      // the y eigenproblem is the x one when both axes and potentials coincide (square TP grids)
      bool same = p.nx == p.ny && p.Lx == p.Ly && p.R0x == p.R0y;
      if (same) {
        int differs = 0;
        MGC_CUDA(cudaMemsetAsync(h->status + 3, 0, sizeof(int), st));
        MGC_LAUNCH(launch_compare(b.mx, v1, v2, h->status + 3, st));
        MGC_CUDA(cudaMemcpyAsync(&differs, h->status + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
        MGC_CUDA(cudaStreamSynchronize(st));
        same = differs == 0;
      }
      if (same) {
        MGC_CUDA(cudaMemcpyAsync(h->mu, h->lam, sizeof(cplx) * nb, cudaMemcpyDeviceToDevice, st));
        MGC_CUDA(cudaMemcpyAsync(h->vphi, h->phi, sizeof(cplx) * nb * b.mx, cudaMemcpyDeviceToDevice, st));
      } else {
        rc = axis_states(h, b.my, b.west_y, b.east_y, b.diag_y, v2, b.w_y, h->mu, h->vphi);
        if (rc) return rc;
      }
    }
    MGC_LAUNCH(launch_weight_states(b.mx, nb, b.w_x, h->phi, h->wphi, st));
    MGC_LAUNCH(launch_weight_states(b.my, nb, b.w_y, h->vphi, h->wvphi, st));
    MGC_LAUNCH(launch_channel_potentials(b.mx, b.my, nb, h->wphi, h->phi, h->wvphi, h->vphi, v12, h->VA, h->VB,
                                         st));
    // channel A runs along y with the x bound states; channel B along x with the y ones
    MGC_LAUNCH(launch_channel_factor_pcr(h->crA, b.diag_y, v2, p.E, h->lam, h->VA, b.west_y, b.east_y,
                                         h->cr_scratch, h->status, st));
    MGC_LAUNCH(launch_channel_factor_pcr(h->crB, b.diag_x, v1, p.E, h->mu, h->VB, b.west_x, b.east_x,
                                         h->cr_scratch, h->status, st));
  }
  int rc0 = read_status(h);
  if (rc0 || !h->mixed) return rc0;
  // complex64 copies of every level's operator and of the bound states
  for (int l = 0; l < h->L; ++l) {
    LevelBufs& b = h->lv[l];
    const long long n2 = (long long)b.mx * b.my;
    MGC_LAUNCH(launch_round_copy(b.mx, b.west_x, b.west_x32, st));
    MGC_LAUNCH(launch_round_copy(b.mx, b.east_x, b.east_x32, st));
    MGC_LAUNCH(launch_round_copy(b.my, b.west_y, b.west_y32, st));
    MGC_LAUNCH(launch_round_copy(b.my, b.east_y, b.east_y32, st));
    MGC_LAUNCH(launch_round_copy(n2, b.D, b.D32, st));
    MGC_LAUNCH(launch_round_copy(n2, b.Dinv, b.Dinv32, st));
    StencilView32& s3 = b.sv32;
    s3.mx = b.mx; s3.my = b.my; s3.rbox = b.sv.rbox;
    s3.cx = axis_coef32(b.sv.cx); s3.cy = axis_coef32(b.sv.cy);
    s3.keep = (float)b.sv.keep;
    s3.west_x = b.west_x32; s3.east_x = b.east_x32; s3.west_y = b.west_y32; s3.east_y = b.east_y32;
    s3.D = b.D32; s3.Dinv = b.Dinv32;
  }
  if (h->nb > 0) {
    const int nb = h->nb;
    MGC_LAUNCH(launch_round_copy((long long)nb * h->lv[0].mx, h->phi, h->phi32, st));
    MGC_LAUNCH(launch_round_copy((long long)nb * h->lv[0].my, h->vphi, h->vphi32, st));
    MGC_LAUNCH(launch_round_copy((long long)nb * h->lv[0].mx, h->wphi, h->wphi32, st));
    MGC_LAUNCH(launch_round_copy((long long)nb * h->lv[0].my, h->wvphi, h->wvphi32, st));
  }
  return read_status(h);
}

// Typed views of a level's operator and buffers: complex128 for the plain path,
// complex64 for the mixed-precision preconditioner.
template <class C>
struct LevelIO {
  const StencilViewT<C>* sv;
  C *u, *f, *t, *r;
  int mx, my;
};
template <class C>
LevelIO<C> level_io(mgcccs_handle* h, int l);
template <>
LevelIO<cplx> level_io<cplx>(mgcccs_handle* h, int l) {
  LevelBufs& b = h->lv[l];
  return LevelIO<cplx>{&b.sv, b.u, b.f, b.t, b.r, b.mx, b.my};
}
template <>
LevelIO<float2> level_io<float2>(mgcccs_handle* h, int l) {
  LevelBufs& b = h->lv[l];
  return LevelIO<float2>{&b.sv32, b.u32, b.f32, b.t32, b.r32, b.mx, b.my};
}
template <class C>
const CCViewT<C>& cc_view(mgcccs_handle* h);
template <>
const CCViewT<cplx>& cc_view<cplx>(mgcccs_handle* h) { return h->cc; }
template <>
const CCViewT<float2>& cc_view<float2>(mgcccs_handle* h) { return h->cc32; }

// One V-cycle on level l.  `u` holds the initial guess unless zero_init; the result is
// returned in *out (either u or the level's t buffer).
// Whether level passes are fused (zero-start sweep + residual + restriction; prolongation +
// first post-smoothing sweep): always for complex64, whose FP32 work is cheap; for
// complex128 below 512^2 nodes, where launch latency outweighs the halo recomputation.
// The coarsest-level solve u = A_c^{-1} f: the dense inverse, or block cyclic reduction
// for coarsest grids beyond MGC_MAX_COARSE unknowns.
template <class C>
cudaError_t coarse_solve(mgcccs_handle* h, const C* f, C* u, cudaStream_t st) {
  const LevelBufs& c = h->lv[h->L - 1];
  if (h->coarse_bp) return launch_bpcr_solve<C>(c.mx, c.my, h->bp_fac, f, u, h->bp_buf, st);
  return launch_coarse_solve(h->nc, h->Ainv, f, u, st);
}

template <class C>
bool fuse_level(const LevelIO<C>& b) {
  return sizeof(C) == sizeof(float2) || (long long)b.mx * b.my < 512LL * 512;
}

template <class C>
int vcycle_rec(mgcccs_handle* h, int l, C* u, const C* f, bool zero_init, C** out) {
  MgcRange nvtx_range(mgc_level_range_name(l));
  cudaStream_t st = h->st;
  LevelIO<C> b = level_io<C>(h, l);
  if (l == h->L - 1) {
    MGC_LAUNCH(coarse_solve<C>(h, f, u, st));
    *out = u;
    return MGCCCS_OK;
  }
  C* cur = u;
  C* oth = b.t;
  bool zero = zero_init;
  LevelIO<C> c = level_io<C>(h, l + 1);
  const bool fuse = fuse_level(b);
  if (fuse && zero && h->p.nu1 == 1 && !(l == 0 && h->pend_norm2)) {
    // the zero-start sweep, residual and restriction in one pass
    MGC_LAUNCH(launch_zero_residual_restrict(*b.sv, f, oth, c.f, true, st));
    cur = oth;
    oth = u;
  } else {
    for (int s = 0; s < h->p.nu1; ++s) {
      if (zero && l == 0 && h->pend_norm2) {
        // the Krylov vector f = w is normalised by the same pass (see issue_arnoldi_step)
        MGC_LAUNCH(launch_scale_jacobi_zero(*b.sv, const_cast<C*>(f), h->pend_norm2, oth, st));
        h->pend_norm2 = nullptr;
      } else if (zero) {
        MGC_LAUNCH(launch_jacobi_zero(*b.sv, oth, f, st));
      } else {
        MGC_LAUNCH(launch_jacobi(*b.sv, (const C*)cur, oth, f, st));
      }
      zero = false;
      C* tmp = cur; cur = oth; oth = tmp;
    }
    if (zero) {
      // no pre-smoothing and a zero guess: the residual is f itself
      MGC_CUDA(cudaMemsetAsync(cur, 0, sizeof(C) * (size_t)b.mx * b.my, st));
    }
    // the residual and the restriction in one pass
    MGC_LAUNCH(launch_zero_residual_restrict(*b.sv, f, cur, c.f, false, st));
  }
  C* ec = nullptr;
  int rc = vcycle_rec<C>(h, l + 1, c.u, c.f, true, &ec);
  if (rc) return rc;
  if (h->p.nu2 == 0 || !fuse) {
    MGC_LAUNCH(launch_prolong_add(b.mx, b.my, (const C*)ec, cur, st));
    if (h->p.nu2 > 0) {
      MGC_LAUNCH(launch_jacobi(*b.sv, (const C*)cur, oth, f, st));
      C* tmp = cur; cur = oth; oth = tmp;
    }
  } else {
    // the prolongation and the first post-smoothing sweep in one pass
    MGC_LAUNCH(launch_prolong_jacobi(*b.sv, (const C*)ec, (const C*)cur, oth, f, st));
    C* tmp = cur; cur = oth; oth = tmp;
  }
  for (int s = 1; s < h->p.nu2; ++s) {
    MGC_LAUNCH(launch_jacobi(*b.sv, (const C*)cur, oth, f, st));
    C* tmp = cur; cur = oth; oth = tmp;
  }
  *out = cur;
  return MGCCCS_OK;
}

template <class C>
int vcycle_fine(mgcccs_handle* h, C* u, const C* f, bool zero_init) {
  C* res = nullptr;
  int rc = vcycle_rec<C>(h, 0, u, f, zero_init, &res);
  if (rc) return rc;
  if (res != u) {
    const LevelBufs& b = h->lv[0];
    MGC_CUDA(cudaMemcpyAsync(u, res, sizeof(C) * (size_t)b.mx * b.my, cudaMemcpyDeviceToDevice, h->st));
  }
  return MGCCCS_OK;
}

template <class C>
int cccs_fine(mgcccs_handle* h, C* u, const C* f) {
  cudaStream_t st = h->st;
  const CCViewT<C>& cc = cc_view<C>(h);
  MGC_LAUNCH(launch_residual_project(*level_io<C>(h, 0).sv, cc, (const C*)u, f, st));
  MGC_LAUNCH(launch_cc_rhs(cc, st));
  h->launches += 1;   // launch_cc_rhs issues two kernels
  MGC_LAUNCH(launch_channel_solve(h->crA, h->crB, st));
  MGC_LAUNCH(launch_cccs_correct(cc, u, st));
  return MGCCCS_OK;
}

int residual_norm2(mgcccs_handle* h, const cplx* u, const cplx* f, cplx* r, double* norm2) {
  cudaStream_t st = h->st;
  const StencilView& s = h->lv[0].sv;
  MGC_LAUNCH(launch_residual(s, u, f, r, norm2 ? h->norm_part : nullptr, st));
  if (norm2) {
    MGC_LAUNCH(launch_sum_partials(h->norm_part, residual_norm_blocks(s), h->norm_out, st));
    MGC_CUDA(cudaMemcpyAsync(norm2, h->norm_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGC_CUDA(cudaStreamSynchronize(st));
  }
  return MGCCCS_OK;
}

int vec_norm2(mgcccs_handle* h, const cplx* v, double* out) {
  cudaStream_t st = h->st;
  long long n = (long long)h->lv[0].mx * h->lv[0].my;
  int nbk = norm2_blocks(n);
  MGC_LAUNCH(launch_norm2(v, n, h->norm_part, nbk, st));
  MGC_LAUNCH(launch_sum_partials(h->norm_part, nbk, h->norm_out, st));
  MGC_CUDA(cudaMemcpyAsync(out, h->norm_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  MGC_CUDA(cudaStreamSynchronize(st));
  return MGCCCS_OK;
}

int read_double(mgcccs_handle* h, const double* dev, double* out) {
  MGC_CUDA(cudaMemcpyAsync(out, dev, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  MGC_CUDA(cudaStreamSynchronize(h->st));
  return MGCCCS_OK;
}

// ---- stream-capture helpers for graphs with conditional nodes

struct CaptureGuard {          // ends a capture on error so that the stream stays usable
  cudaStream_t s;
  bool open;
  ~CaptureGuard() {
    if (open) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      mgc_not_a_kernel();
    }
  }
};

int capture_into(CaptureGuard& cg, cudaGraph_t g) {
  MGC_CUDA(cudaStreamBeginCaptureToGraph(cg.s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cg.open = true;
  return MGCCCS_OK;
}

int capture_end(CaptureGuard& cg) {
  cudaGraph_t g = nullptr;
  cg.open = false;
  MGC_CUDA(cudaStreamEndCapture(cg.s, &g));
  return MGCCCS_OK;
}

// Appends a conditional node after the capture's current tail; returns its body graphs.
int add_conditional(cudaStream_t s, cudaGraphConditionalHandle hd, cudaGraphConditionalNodeType type,
                    unsigned size, cudaGraph_t** bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  MGC_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return MGCCCS_ECUDA;
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = hd;
  prm.conditional.type = type;
  prm.conditional.size = size;
  cudaGraphNode_t node;
  MGC_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
  *bodies = prm.conditional.phGraph_out;
  MGC_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return MGCCCS_OK;
}

// z = M^{-1} r: one V-cycle from zero, then the CCCS.
template <class C>
int precond(mgcccs_handle* h, C* z, const C* r) {
  int rc = vcycle_fine<C>(h, z, r, true);
  if (rc) return rc;
  if (h->nb > 0) rc = cccs_fine<C>(h, z, r);
  return rc;
}

// Krylov basis and graph cache of the two precisions.
template <class C> C* kv_V(mgcccs_handle* h);
template <class C> C* kv_Z(mgcccs_handle* h);
template <> cplx* kv_V<cplx>(mgcccs_handle* h) { return h->V; }
template <> cplx* kv_Z<cplx>(mgcccs_handle* h) { return h->Z; }
template <> float2* kv_V<float2>(mgcccs_handle* h) { return h->V32; }
template <> float2* kv_Z<float2>(mgcccs_handle* h) { return h->Z32; }
template <class C> cudaGraphExec_t* step_cache(mgcccs_handle* h);
template <> cudaGraphExec_t* step_cache<cplx>(mgcccs_handle* h) { return h->step_exec; }
template <> cudaGraphExec_t* step_cache<float2>(mgcccs_handle* h) { return h->step_exec32; }
template <class C> long long* step_count(mgcccs_handle* h);
template <> long long* step_count<cplx>(mgcccs_handle* h) { return h->step_launches; }
template <> long long* step_count<float2>(mgcccs_handle* h) { return h->step_launches32; }

// Arnoldi step j of GMRES(m) with a basis of element type C: z_j = M^{-1} v_j,
// w = A z_j, classical Gram-Schmidt with a cancellation-gated second pass,
// h_{j+1,j} = |w|, v_{j+1} = w / h_{j+1,j}, Givens rotation j, and the residual estimate
// |g_{j+1}| copied to est_host[j].  Touches only buffers of the handle, so the launch
// sequence of each j is fixed and can be replayed as a graph.  The Hessenberg matrix,
// rotations and inner products are FP64 in both precisions.
template <class C>
int issue_arnoldi_step(mgcccs_handle* h, int j) {
  cudaStream_t st = h->st;
  const int m = h->km;
  const StencilViewT<C>& s0 = *level_io<C>(h, 0).sv;
  const long long N = (long long)s0.mx * s0.my;
  const int nb = h->kr_nblk;
  const long long ld = h->kld;
  C* V = kv_V<C>(h);
  C* vj = V + (size_t)j * ld;
  C* w = V + (size_t)(j + 1) * ld;
  C* zj = kv_Z<C>(h) + (size_t)j * ld;
  cplx* col = h->Hh + (size_t)j * (m + 1);
  // v_j = w_j / |w_j| (|w_j|^2 left in norm_out[1] by step j-1; v_0 is normalised by the
  // cycle start): fused into the first pre-smoothing sweep of the preconditioner when
  // the fine level starts one, else a launch of its own
  if (j > 0) {
    if (h->p.nu1 >= 1 && h->L > 1) {
      h->pend_norm2 = h->norm_out + 1;
    } else {
      MGC_LAUNCH(launch_scale_by_norm(N, (const C*)vj, vj, h->norm_out + 1, (cplx*)nullptr, nb, st));
    }
  }
  int rc = precond<C>(h, zj, vj);
  h->pend_norm2 = nullptr;
  if (rc) return rc;
  // w = A z_j
  MGC_LAUNCH(launch_apply(s0, (const C*)zj, w, st, (double*)nullptr));
  // Gram-Schmidt, first pass: H(0:j, j) = V^H w ; w -= V H(0:j, j).  w is column j+1 of V,
  // so the multi-dot over columns 0..j+1 also yields |w|^2 (for the reorthogonalisation
  // test), left in H(j+1, j) until the Givens rotation writes that entry.
  const int nbd = multidot_blocks(N, j + 2);
  MGC_LAUNCH(launch_multidot(N, j + 2, (const C*)V, ld, (const C*)w, h->dotpart, nbd, (const int*)nullptr, st));
  MGC_LAUNCH(launch_reduce_dots(nbd, j + 2, h->dotpart, col, nullptr, st));
  const double* w_norm2 = reinterpret_cast<const double*>(col + j + 1);
  MGC_LAUNCH(launch_multiaxpy(N, j + 1, (const C*)V, ld, col, -1.0, w, h->norm_part, nb, (const int*)nullptr, st));
  // second pass only when the first one cancelled |w| by more than 1e3;
  // the corrections are added into H(0:j, j).  The Givens rotation j takes h_{j+1,j} = |w|
  // from its square; without a second pass (nearly every step) k_sum_dgks applies it, after
  // one the pass ends with it.  w is normalised at the start of step j+1 (a cycle that
  // stops here never uses it).
  const GivensArgs gv{j, m, h->Hh, h->cs, h->sn, h->g, h->norm_out + 2};
  if (h->device_loop) {
    // device-driven graph: the pass is the body of a conditional node, so it costs no
    // launch when it does not run
    MGC_LAUNCH(launch_sum_dgks(h->norm_part, nb, h->norm_out + 1, w_norm2, h->gate, st, h->dgks_cond[j],
                               &h->ctl->dgks, &gv));
    cudaGraph_t* body = nullptr;
    int rc2 = add_conditional(st, h->dgks_cond[j], cudaGraphCondTypeIf, 1, &body);
    if (rc2) return rc2;
    CaptureGuard cg{h->gst[0], false};
    rc2 = capture_into(cg, body[0]);
    if (rc2) return rc2;
    cudaStream_t bs = h->gst[0];
    const long long b0 = h->launches;
    MGC_LAUNCH(launch_multidot(N, j + 1, (const C*)V, ld, (const C*)w, h->dotpart, nbd, (const int*)nullptr, bs));
    MGC_LAUNCH(launch_reduce_dots(nbd, j + 1, h->dotpart, h->hc, col, bs));
    MGC_LAUNCH(launch_multiaxpy(N, j + 1, (const C*)V, ld, h->hc, -1.0, w, h->norm_part, nb, (const int*)nullptr, bs));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, nb, h->norm_out + 1, bs));
    MGC_LAUNCH(launch_givens(j, m, h->Hh, h->cs, h->sn, h->g, h->norm_out + 2, h->norm_out + 1, bs));
    h->sg_dgks = h->launches - b0;
    h->launches = b0;
    rc2 = capture_end(cg);
    if (rc2) return rc2;
  } else {
    MGC_LAUNCH(launch_sum_dgks(h->norm_part, nb, h->norm_out + 1, w_norm2, h->gate, st, 0, nullptr, &gv));
    MGC_LAUNCH(launch_multidot(N, j + 1, (const C*)V, ld, (const C*)w, h->dotpart, nbd, (const int*)h->gate, st));
    MGC_LAUNCH(launch_reduce_dots(nbd, j + 1, h->dotpart, h->hc, col, st));
    MGC_LAUNCH(launch_multiaxpy(N, j + 1, (const C*)V, ld, h->hc, -1.0, w, h->norm_part, nb, (const int*)h->gate,
                                st));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, nb, h->norm_out + 1, st, h->gate));
    MGC_LAUNCH(launch_givens(j, m, h->Hh, h->cs, h->sn, h->g, h->norm_out + 2, h->norm_out + 1, st, h->gate));
  }
  if (!h->device_loop)
    MGC_CUDA(cudaMemcpyAsync(h->est_host + j, h->norm_out + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
  return MGCCCS_OK;
}

// Launch Arnoldi step j: replay its graph, capturing it on first use.
template <class C>
int launch_arnoldi_step(mgcccs_handle* h, int j) {
  cudaGraphExec_t* cache = step_cache<C>(h);
  long long* count = step_count<C>(h);
  if (!cache[j]) {
    cudaStream_t orig = h->st;
    const long long before = h->launches;
    h->st = h->cap_st;
    MGC_CUDA(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal));
    int rc = issue_arnoldi_step<C>(h, j);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
    mgc_not_a_kernel();
    h->st = orig;
    count[j] = h->launches - before;
    h->launches = before;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return MGCCCS_ECUDA;
    e = cudaGraphInstantiate(&cache[j], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cache[j] = nullptr;
      return MGCCCS_ECUDA;
    }
  }
  MGC_CUDA(cudaGraphLaunch(cache[j], h->st));
  h->launches += count[j];
  return MGCCCS_OK;
}

// One GMRES(m) cycle on the basis of type C whose v_0 is already in place and whose
// g = (beta, 0, ...): launches Arnoldi steps (the host checks step j-1 while step j
// runs) until est/scale <= target or m steps or the step budget; returns the number k
// of steps to use.  est/scale is recorded in history.
template <class C>
int arnoldi_cycle(mgcccs_handle* h, double scale, double target, int* steps, int max_iter, double* history,
                  int* k_out, bool* nonfinite) {
  cudaStream_t st = h->st;
  const int m = h->km;
  int k = 0;
  *nonfinite = false;
  for (int j = 0; j <= m; ++j) {
    if (j < m) {
      int rc = launch_arnoldi_step<C>(h, j);
      if (rc) return rc;
      MGC_CUDA(cudaEventRecord(h->ev[j & 1], st));
    }
    if (j == 0) continue;
    // residual estimate of step j-1 (step j, if launched, runs meanwhile)
    MGC_CUDA(cudaEventSynchronize(h->ev[(j - 1) & 1]));
    const double est = h->est_host[j - 1] * scale;
    if (history) history[*steps] = est;
    ++*steps;
    k = j;
    if (!std::isfinite(est)) { *nonfinite = true; break; }
    if (est <= target || *steps >= max_iter) break;
  }
  *k_out = k;
  return MGCCCS_OK;
}

// Restarted GMRES(m), right-preconditioned by one MG-CCCS iteration (graph-replayed
// Arnoldi steps).  The host checks the residual estimate of step j-1 while step j
// runs, so the device never waits for the host inside a cycle; a step launched after
// convergence is simply not used (the solution only needs columns and g entries
// below it).  Counts Arnoldi steps as iterations.
int gmres_impl(mgcccs_handle* h, cplx* u, const cplx* f, double fn, double rtol, int max_iter, int* iters,
               double* relres, double* history) {
  cudaStream_t st = h->st;
  const int m = h->km;
  const StencilView& s0 = h->lv[0].sv;
  const long long N = (long long)s0.mx * s0.my;
  const int nb = h->kr_nblk;
  int steps = 0;
  double rr = INFINITY, rr_min = INFINITY;
  for (;;) {
    // true residual r = f - A u into V_0
    MGC_LAUNCH(launch_residual(s0, (const cplx*)u, f, h->V, h->norm_part, st));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, residual_norm_blocks(s0), h->norm_out, st));
    double rn2 = 0.0;
    int rc = read_double(h, h->norm_out, &rn2);
    if (rc) return rc;
    rr = std::sqrt(rn2) / fn;
    if (!std::isfinite(rr)) {
      if (iters) *iters = steps;
      if (relres) *relres = rr;
      return MGCCCS_ENONFINITE;
    }
    if (rr > MGC_DIVERGENCE_FACTOR * rr_min) {
      if (iters) *iters = steps;
      if (relres) *relres = rr;
      return MGCCCS_EDIVERGED;
    }
    rr_min = std::min(rr_min, rr);
    if (rr <= rtol || steps >= max_iter) break;
    MGC_LAUNCH(launch_zero_c(m + 1, h->g, st));
    MGC_LAUNCH(launch_scale_by_norm(N, (const cplx*)h->V, h->V, h->norm_out, h->g, nb, st));
    int k = 0;
    bool nonfinite = false;
    rc = arnoldi_cycle<cplx>(h, 1.0 / fn, rtol, &steps, max_iter, history, &k, &nonfinite);
    if (rc) return rc;
    if (nonfinite) {
      MGC_CUDA(cudaStreamSynchronize(st));
      if (iters) *iters = steps;
      if (relres) *relres = NAN;
      return MGCCCS_ENONFINITE;
    }
    MGC_LAUNCH(launch_hess_solve(k, m, h->Hh, h->g, h->y, st));
    MGC_LAUNCH(launch_multiaxpy(N, k, (const cplx*)h->Z, h->kld, h->y, 1.0, u, (double*)nullptr, nb, (const int*)nullptr, st));
  }
  if (iters) *iters = steps;
  if (relres) *relres = rr;
  return rr <= rtol ? MGCCCS_OK : MGCCCS_ENOTCONV;
}

// Mixed precision: iterative refinement in FP64 around one complex64 GMRES(m) cycle per
// refinement step (GMRES-IR).  Each step forms the true residual r = f - A u in FP64,
// rounds r/|r| to complex64 as v_0, runs one preconditioned GMRES cycle in complex64
// (V-cycle, projections, corrections and the Krylov basis in complex64; coarsest solve,
// channel solves, Hessenberg and rotations in FP64) until the cycle's estimate reaches
// the inner tolerance, and adds |r| e to u in FP64.  Counts Arnoldi steps as iterations.
int gmres_ir_impl(mgcccs_handle* h, cplx* u, const cplx* f, double fn, double rtol, int max_iter, int* iters,
                  double* relres, double* history) {
  cudaStream_t st = h->st;
  const int m = h->km;
  const StencilView& s0 = h->lv[0].sv;
  const long long N = (long long)s0.mx * s0.my;
  const int nb = h->kr_nblk;
  int steps = 0;
  double rr = INFINITY, rr_min = INFINITY;
  for (;;) {
    MGC_LAUNCH(launch_residual(s0, (const cplx*)u, f, h->r64, h->norm_part, st));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, residual_norm_blocks(s0), h->norm_out, st));
    double rn2 = 0.0;
    int rc = read_double(h, h->norm_out, &rn2);
    if (rc) return rc;
    rr = std::sqrt(rn2) / fn;
    if (!std::isfinite(rr)) {
      if (iters) *iters = steps;
      if (relres) *relres = rr;
      return MGCCCS_ENONFINITE;
    }
    if (rr > MGC_DIVERGENCE_FACTOR * rr_min) {
      if (iters) *iters = steps;
      if (relres) *relres = rr;
      return MGCCCS_EDIVERGED;
    }
    rr_min = std::min(rr_min, rr);
    if (rr <= rtol || steps >= max_iter) break;
    // v_0 = r/|r| in complex64, renormalised in the rounded precision; g = (|v_0|, 0, ...)
    MGC_LAUNCH(launch_demote(N, h->r64, h->norm_out, h->V32, st));
    MGC_LAUNCH(launch_norm2(h->V32, N, h->norm_part, norm2_blocks(N), st));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, norm2_blocks(N), h->norm_out + 1, st));
    MGC_LAUNCH(launch_zero_c(m + 1, h->g, st));
    MGC_LAUNCH(launch_scale_by_norm(N, (const float2*)h->V32, h->V32, h->norm_out + 1, h->g, nb, st));
    // inner target: the cycle's own tolerance, and no deeper than the outer goal needs
    const double beta = std::sqrt(rn2);
    const double target = std::max(h->inner_rtol, 0.5 * rtol * fn / beta);
    int k = 0;
    bool nonfinite = false;
    rc = arnoldi_cycle<float2>(h, beta / fn, target * beta / fn, &steps, max_iter, history, &k, &nonfinite);
    if (rc) return rc;
    if (nonfinite) {
      MGC_CUDA(cudaStreamSynchronize(st));
      if (iters) *iters = steps;
      if (relres) *relres = NAN;
      return MGCCCS_ENONFINITE;
    }
    MGC_LAUNCH(launch_hess_solve(k, m, h->Hh, h->g, h->y, st));
    MGC_CUDA(cudaMemsetAsync(h->e32, 0, sizeof(float2) * (size_t)N, st));
    MGC_LAUNCH(launch_multiaxpy(N, k, (const float2*)h->Z32, h->kld, h->y, 1.0, h->e32, (double*)nullptr, nb,
                                (const int*)nullptr, st));
    MGC_LAUNCH(launch_promote_add(N, h->e32, h->norm_out, u, st));
  }
  if (iters) *iters = steps;
  if (relres) *relres = rr;
  return rr <= rtol ? MGCCCS_OK : MGCCCS_ENOTCONV;
}

// ---- batched solves: per-problem GMRES cycles advanced in lock-step ---------------
// The cycle of gmres_impl / gmres_ir_impl split into phases so that the host can
// interleave many handles, each on its own stream: (1) every unfinished problem
// enqueues its true residual and norm read-back, then the host reads them all;
// (2) Arnoldi step j is launched for every problem still in its cycle, and the
// estimate of step j-1 of each is checked while step j runs; (3) every problem
// solves its Hessenberg system and updates u.

struct BatchItem {
  mgcccs_handle* h;
  cplx* u;
  const cplx* f;
  double fn, rr, scale, target, rr_min;
  int steps, k;
  bool active, in_cycle;
  int status;
};

int batch_residual_enqueue(BatchItem& it) {
  mgcccs_handle* h = it.h;
  const StencilView& s0 = h->lv[0].sv;
  cplx* rbuf = h->mixed ? h->r64 : h->V;
  MGC_LAUNCH(launch_residual(s0, (const cplx*)it.u, it.f, rbuf, h->norm_part, h->st));
  MGC_LAUNCH(launch_sum_partials(h->norm_part, residual_norm_blocks(s0), h->norm_out, h->st));
  MGC_CUDA(cudaMemcpyAsync(h->est_host + MGC_MAX_RESTART, h->norm_out, sizeof(double), cudaMemcpyDeviceToHost,
                           h->st));
  return MGCCCS_OK;
}

// Stop test on the residual read back by batch_residual_enqueue; if the problem goes
// on, v_0 and g of its next cycle are enqueued.
int batch_cycle_begin(BatchItem& it, double rtol, int max_iter) {
  mgcccs_handle* h = it.h;
  cudaStream_t st = h->st;
  MGC_CUDA(cudaStreamSynchronize(st));
  const double rn2 = h->est_host[MGC_MAX_RESTART];
  it.rr = std::sqrt(rn2) / it.fn;
  it.in_cycle = false;
  if (!std::isfinite(it.rr)) {
    it.active = false;
    it.status = MGCCCS_ENONFINITE;
    return MGCCCS_OK;
  }
  if (it.rr > MGC_DIVERGENCE_FACTOR * it.rr_min) {
    it.active = false;
    it.status = MGCCCS_EDIVERGED;
    return MGCCCS_OK;
  }
  it.rr_min = std::min(it.rr_min, it.rr);
  if (it.rr <= rtol || it.steps >= max_iter) {
    it.active = false;
    it.status = it.rr <= rtol ? MGCCCS_OK : MGCCCS_ENOTCONV;
    return MGCCCS_OK;
  }
  const StencilView& s0 = h->lv[0].sv;
  const long long N = (long long)s0.mx * s0.my;
  const int nb = h->kr_nblk;
  const double beta = std::sqrt(rn2);
  MGC_LAUNCH(launch_zero_c(h->km + 1, h->g, st));
  if (h->mixed) {
    MGC_LAUNCH(launch_demote(N, h->r64, h->norm_out, h->V32, st));
    MGC_LAUNCH(launch_norm2(h->V32, N, h->norm_part, norm2_blocks(N), st));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, norm2_blocks(N), h->norm_out + 1, st));
    MGC_LAUNCH(launch_scale_by_norm(N, (const float2*)h->V32, h->V32, h->norm_out + 1, h->g, nb, st));
    it.scale = beta / it.fn;
    it.target = std::max(h->inner_rtol, 0.5 * rtol * it.fn / beta) * beta / it.fn;
  } else {
    MGC_LAUNCH(launch_scale_by_norm(N, (const cplx*)h->V, h->V, h->norm_out, h->g, nb, st));
    it.scale = 1.0 / it.fn;
    it.target = rtol;
  }
  it.in_cycle = true;
  it.k = 0;
  return MGCCCS_OK;
}

int batch_cycle_end(BatchItem& it) {
  mgcccs_handle* h = it.h;
  cudaStream_t st = h->st;
  const StencilView& s0 = h->lv[0].sv;
  const long long N = (long long)s0.mx * s0.my;
  const int nb = h->kr_nblk;
  MGC_LAUNCH(launch_hess_solve(it.k, h->km, h->Hh, h->g, h->y, st));
  if (h->mixed) {
    MGC_CUDA(cudaMemsetAsync(h->e32, 0, sizeof(float2) * (size_t)N, st));
    MGC_LAUNCH(launch_multiaxpy(N, it.k, (const float2*)h->Z32, h->kld, h->y, 1.0, h->e32, (double*)nullptr, nb,
                                (const int*)nullptr, st));
    MGC_LAUNCH(launch_promote_add(N, h->e32, h->norm_out, it.u, st));
  } else {
    MGC_LAUNCH(launch_multiaxpy(N, it.k, (const cplx*)h->Z, h->kld, h->y, 1.0, it.u, (double*)nullptr, nb,
                                (const int*)nullptr, st));
  }
  return MGCCCS_OK;
}

int batch_solve_impl(std::vector<BatchItem>& items, double rtol, int max_iter) {
  for (;;) {
    for (auto& it : items)
      if (it.active) {
        int rc = batch_residual_enqueue(it);
        if (rc) return rc;
      }
    bool any = false;
    int mmax = 0;
    for (auto& it : items)
      if (it.active) {
        int rc = batch_cycle_begin(it, rtol, max_iter);
        if (rc) return rc;
        if (it.in_cycle) {
          any = true;
          mmax = std::max(mmax, it.h->km);
        }
      }
    if (!any) return MGCCCS_OK;
    for (int j = 0; j <= mmax; ++j) {
      for (auto& it : items) {
        if (!it.in_cycle || j >= it.h->km) continue;
        mgcccs_handle* h = it.h;
        int rc = h->mixed ? launch_arnoldi_step<float2>(h, j) : launch_arnoldi_step<cplx>(h, j);
        if (rc) return rc;
        MGC_CUDA(cudaEventRecord(h->ev[j & 1], h->st));
      }
      if (j == 0) continue;
      for (auto& it : items) {
        if (!it.in_cycle || it.k != j - 1) continue;
        mgcccs_handle* h = it.h;
        MGC_CUDA(cudaEventSynchronize(h->ev[(j - 1) & 1]));
        const double est = h->est_host[j - 1] * it.scale;
        ++it.steps;
        it.k = j;
        if (!std::isfinite(est)) {
          MGC_CUDA(cudaStreamSynchronize(h->st));
          it.in_cycle = it.active = false;
          it.status = MGCCCS_ENONFINITE;
          it.rr = NAN;
          continue;
        }
        if (est <= it.target || it.steps >= max_iter || j == h->km) {
          int rc = batch_cycle_end(it);
          if (rc) return rc;
          it.in_cycle = false;
        }
      }
    }
  }
}


// ---- device-driven solves: a whole GMRES(m) solve as one CUDA graph ------------------
// Conditional graph nodes carry the solver's control flow, so a solve is one graph
// launch and the host neither waits nor decides between steps:
//
//   |f|^2 -> ctl.fn2
//   WHILE (outer):                          one restart
//     r = f - A u, |r|^2; k_outer_control   (stop test; opens the next cycle)
//     IF (cycle):
//       v_0 = r/|r| (complex64 in the mixed form), g = (|v_0|, 0, ...)
//       WHILE (inner):
//         SWITCH (j): Arnoldi step j        (the same launches as the host-driven step j)
//         k_step_control                    (count the step; continue unless done)
//       y = R^{-1} g (k = ctl.k columns); u += Z y   (mixed: u += promote(Z32 y))
//
// Several problems are independent root branches of one graph (batched solves).

template <class C>
int append_steps(mgcccs_handle* h, cudaGraph_t* bodies, cudaStream_t s) {
  cudaStream_t orig = h->st;
  h->st = s;
  h->device_loop = true;
  int rc = MGCCCS_OK;
  for (int j = 0; j < h->km && rc == MGCCCS_OK; ++j) {
    CaptureGuard cg{s, false};
    rc = capture_into(cg, bodies[j]);
    const long long before = h->launches;
    if (rc == MGCCCS_OK) rc = issue_arnoldi_step<C>(h, j);
    if (j == 0) h->sg_step = h->launches - before;
    if (rc == MGCCCS_OK) rc = capture_end(cg);
  }
  h->st = orig;
  h->device_loop = false;
  return rc;
}

// Adds one problem's solve (u, f on handle h) to graph G as an independent branch.
int append_solve(mgcccs_handle* h, cplx* u, const cplx* f, cudaGraph_t G) {
  const StencilView& s0 = h->lv[0].sv;
  const long long N = (long long)s0.mx * s0.my;
  const int m = h->km, nb = h->kr_nblk;
  cudaStream_t S = h->gst[0];
  cudaGraphConditionalHandle h_outer, h_cycle, h_inner, h_switch;
  MGC_CUDA(cudaGraphConditionalHandleCreate(&h_outer, G, 1, cudaGraphCondAssignDefault));
  MGC_CUDA(cudaGraphConditionalHandleCreate(&h_cycle, G, 0, 0));
  MGC_CUDA(cudaGraphConditionalHandleCreate(&h_inner, G, 0, 0));
  MGC_CUDA(cudaGraphConditionalHandleCreate(&h_switch, G, 0, 0));
  const long long base = h->launches;
  cudaGraph_t* b1 = nullptr;
  {
    CaptureGuard cg{S, false};
    int rc = capture_into(cg, G);
    if (rc) return rc;
    const int nbk = norm2_blocks(N);
    MGC_LAUNCH(launch_norm2(f, N, h->norm_part, nbk, S));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, nbk, &h->ctl->fn2, S));
    rc = add_conditional(S, h_outer, cudaGraphCondTypeWhile, 1, &b1);
    if (rc) return rc;
    rc = capture_end(cg);
    if (rc) return rc;
  }
  h->sg_pro = h->launches - base;
  cudaGraph_t* b2 = nullptr;
  {
    const long long b0 = h->launches;
    CaptureGuard cg{S, false};
    int rc = capture_into(cg, b1[0]);
    if (rc) return rc;
    cplx* rbuf = h->mixed ? h->r64 : h->V;
    MGC_LAUNCH(launch_residual(s0, (const cplx*)u, f, rbuf, h->norm_part, S));
    MGC_LAUNCH(launch_sum_partials(h->norm_part, residual_norm_blocks(s0), h->norm_out, S));
    MGC_LAUNCH(launch_outer_control(h->ctl, h->norm_out, h_outer, h_cycle, h_inner, h_switch, S));
    rc = add_conditional(S, h_cycle, cudaGraphCondTypeIf, 1, &b2);
    if (rc) return rc;
    rc = capture_end(cg);
    if (rc) return rc;
    h->sg_outer = h->launches - b0;
  }
  cudaGraph_t* b3 = nullptr;
  {
    const long long b0 = h->launches;
    CaptureGuard cg{S, false};
    int rc = capture_into(cg, b2[0]);
    if (rc) return rc;
    MGC_LAUNCH(launch_zero_c(m + 1, h->g, S));
    if (h->mixed) {
      MGC_LAUNCH(launch_demote(N, h->r64, h->norm_out, h->V32, S));
      MGC_LAUNCH(launch_norm2(h->V32, N, h->norm_part, norm2_blocks(N), S));
      MGC_LAUNCH(launch_sum_partials(h->norm_part, norm2_blocks(N), h->norm_out + 1, S));
      MGC_LAUNCH(launch_scale_by_norm(N, (const float2*)h->V32, h->V32, h->norm_out + 1, h->g, nb, S));
    } else {
      MGC_LAUNCH(launch_scale_by_norm(N, (const cplx*)h->V, h->V, h->norm_out, h->g, nb, S));
    }
    rc = add_conditional(S, h_inner, cudaGraphCondTypeWhile, 1, &b3);
    if (rc) return rc;
    MGC_LAUNCH(launch_hess_solve(m, m, h->Hh, h->g, h->y, S, &h->ctl->k));
    if (h->mixed) {
      MGC_CUDA(cudaMemsetAsync(h->e32, 0, sizeof(float2) * (size_t)N, S));
      MGC_LAUNCH(launch_multiaxpy(N, m, (const float2*)h->Z32, h->kld, h->y, 1.0, h->e32, (double*)nullptr, nb,
                                  (const int*)nullptr, S, &h->ctl->k));
      MGC_LAUNCH(launch_promote_add(N, h->e32, h->norm_out, u, S));
    } else {
      MGC_LAUNCH(launch_multiaxpy(N, m, (const cplx*)h->Z, h->kld, h->y, 1.0, u, (double*)nullptr, nb,
                                  (const int*)nullptr, S, &h->ctl->k));
    }
    rc = capture_end(cg);
    if (rc) return rc;
    h->sg_cycle = h->launches - b0;
  }
  cudaGraph_t* b4 = nullptr;
  {
    CaptureGuard cg{S, false};
    int rc = capture_into(cg, b3[0]);
    if (rc) return rc;
    rc = add_conditional(S, h_switch, cudaGraphCondTypeSwitch, (unsigned)m, &b4);
    if (rc) return rc;
    MGC_LAUNCH(launch_step_control(h->ctl, h->norm_out + 2, h_inner, h_switch, S));
    rc = capture_end(cg);
    if (rc) return rc;
  }
  for (int j = 0; j < m; ++j) MGC_CUDA(cudaGraphConditionalHandleCreate(&h->dgks_cond[j], G, 0, 0));
  int rc = h->mixed ? append_steps<float2>(h, b4, h->gst[1]) : append_steps<cplx>(h, b4, h->gst[1]);
  if (rc) return rc;
  h->sg_step += 1;                     // + k_step_control
  h->launches = base;                  // capture is not execution
  return MGCCCS_OK;
}

int instantiate_solves(mgcccs_handle* const* hs, cplx* const* u, const cplx* const* f, int count,
                       cudaGraphExec_t* exec) {
  cudaGraph_t G = nullptr;
  if (cudaGraphCreate(&G, 0) != cudaSuccess) return MGCCCS_ECUDA;
  int rc = MGCCCS_OK;
  for (int k = 0; k < count && rc == MGCCCS_OK; ++k) rc = append_solve(hs[k], u[k], f[k], G);
  if (rc == MGCCCS_OK && cudaGraphInstantiate(exec, G, 0) != cudaSuccess) {
    *exec = nullptr;
    rc = MGCCCS_ECUDA;
  }
  cudaGraphDestroy(G);
  return rc;
}

// Inputs of the control record, staged through pinned memory on stream st.
int stage_ctl(mgcccs_handle* h, double rtol, int max_iter, cudaStream_t st) {
  SolveCtl c{};
  c.rtol = rtol;
  c.inner_rtol = h->inner_rtol;
  c.max_iter = max_iter;
  c.mixed = h->mixed;
  c.m = h->km;
  c.rr_min = INFINITY;
  *h->ctl_host = c;
  MGC_CUDA(cudaMemcpyAsync(h->ctl, h->ctl_host, sizeof(SolveCtl), cudaMemcpyHostToDevice, st));
  return MGCCCS_OK;
}

int fetch_ctl(mgcccs_handle* h, cudaStream_t st) {
  MGC_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, st));
  return MGCCCS_OK;
}

// Outcome of a finished device-driven solve (ctl_host already fetched and synchronised).
int finish_ctl(mgcccs_handle* h, cplx* u, int* iters, double* relres) {
  const SolveCtl& c = *h->ctl_host;
  h->launches += h->sg_pro + (long long)c.outer * h->sg_outer + (long long)c.cycles * h->sg_cycle +
                 (long long)c.steps * h->sg_step + (long long)c.dgks * h->sg_dgks;
  if (iters) *iters = c.steps;
  if (relres) *relres = c.rr;
  switch (c.status) {
    case SOLVECTL_CONVERGED: return MGCCCS_OK;
    case SOLVECTL_ZERO_RHS:
      MGC_CUDA(cudaMemsetAsync(u, 0, sizeof(cplx) * (size_t)h->lv[0].mx * h->lv[0].my, h->st));
      MGC_CUDA(cudaStreamSynchronize(h->st));
      return MGCCCS_OK;
    case SOLVECTL_MAXITER: return MGCCCS_ENOTCONV;
    case SOLVECTL_NONFINITE: return MGCCCS_ENONFINITE;
    case SOLVECTL_DIVERGED: return MGCCCS_EDIVERGED;
    default: return MGCCCS_ECUDA;
  }
}

int graph_solve(mgcccs_handle* h, cplx* u, const cplx* f, double rtol, int max_iter, int* iters, double* relres) {
  int slot = -1;
  for (int q = 0; q < 4; ++q)
    if (h->solve_exec[q] && h->solve_u[q] == u && h->solve_f[q] == f) slot = q;
  if (slot < 0) {
    slot = h->solve_next;
    h->solve_next = (h->solve_next + 1) % 4;
    if (h->solve_exec[slot]) cudaGraphExecDestroy(h->solve_exec[slot]);
    h->solve_exec[slot] = nullptr;
    mgcccs_handle* hs[1] = {h};
    cplx* us[1] = {u};
    const cplx* fs[1] = {f};
    int rc = instantiate_solves(hs, us, fs, 1, &h->solve_exec[slot]);
    if (rc) return rc;
    h->solve_u[slot] = u;
    h->solve_f[slot] = f;
  }
  int rc = stage_ctl(h, rtol, max_iter, h->st);
  if (rc) return rc;
  MGC_CUDA(cudaGraphLaunch(h->solve_exec[slot], h->st));
  rc = fetch_ctl(h, h->st);
  if (rc) return rc;
  MGC_CUDA(cudaStreamSynchronize(h->st));
  return finish_ctl(h, u, iters, relres);
}

int create_krylov_objects(mgcccs_handle* h) {
  MGC_CUDA(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  for (int q = 0; q < 2; ++q) MGC_CUDA(cudaEventCreateWithFlags(&h->ev[q], cudaEventDisableTiming));
  MGC_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h->est_host), sizeof(double) * (MGC_MAX_RESTART + 1)));
  MGC_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h->ctl_host), sizeof(SolveCtl)));
  for (int q = 0; q < 2; ++q) MGC_CUDA(cudaStreamCreateWithFlags(&h->gst[q], cudaStreamNonBlocking));
  return MGCCCS_OK;
}

int solve_impl(mgcccs_handle* h, cplx* u, const cplx* f, double rtol, int max_iter, int* iters, double* relres,
               double* history) {
  if (max_iter < 1) return MGCCCS_EINVAL;
  if (h->km > 0 && !history && h->driver == MGCCCS_DRIVER_GRAPH)
    return graph_solve(h, u, f, rtol, max_iter, iters, relres);
  double fn2 = 0.0;
  int rc = vec_norm2(h, f, &fn2);
  if (rc) return rc;
  if (fn2 == 0.0) {
    MGC_CUDA(cudaMemsetAsync(u, 0, sizeof(cplx) * (size_t)h->lv[0].mx * h->lv[0].my, h->st));
    MGC_CUDA(cudaStreamSynchronize(h->st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return MGCCCS_OK;
  }
  if (h->km > 0 && h->mixed) return gmres_ir_impl(h, u, f, std::sqrt(fn2), rtol, max_iter, iters, relres, history);
  if (h->km > 0) return gmres_impl(h, u, f, std::sqrt(fn2), rtol, max_iter, iters, relres, history);
  double rr = INFINITY, rr_min = INFINITY;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    rc = vcycle_fine(h, u, f, false);
    if (rc) return rc;
    if (h->nb > 0) {
      rc = cccs_fine(h, u, f);
      if (rc) return rc;
    }
    double rn2 = 0.0;
    rc = residual_norm2(h, u, f, nullptr, &rn2);
    if (rc) return rc;
    rr = std::sqrt(rn2 / fn2);
    if (history) history[it - 1] = rr;
    if (!std::isfinite(rr)) {
      if (iters) *iters = it;
      if (relres) *relres = rr;
      return MGCCCS_ENONFINITE;
    }
    if (rr > MGC_DIVERGENCE_FACTOR * rr_min) {
      if (iters) *iters = it;
      if (relres) *relres = rr;
      return MGCCCS_EDIVERGED;
    }
    rr_min = std::min(rr_min, rr);
    if (rr <= rtol) break;
  }
  if (it > max_iter) it = max_iter;
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return rr <= rtol ? MGCCCS_OK : MGCCCS_ENOTCONV;
}

}  // namespace

extern "C" {

size_t mgcccs_workspace_size(const mgcccs_params* p) {
  if (!valid_params(p)) return 0;
  mgcccs_handle* h = new (std::nothrow) mgcccs_handle();
  if (!h) return 0;
  h->p = *p;
  h->L = p->levels;
  Carver cv{nullptr};
  layout(h, cv);
  delete h;
  return cv.off + kAlign;
}

int mgcccs_setup(mgcccs_t* out, const mgcccs_params* p, const mgcccs_c128* v1, const mgcccs_c128* v2,
                 const mgcccs_c128* v12, void* workspace, size_t workspace_bytes, void* stream) {
  MgcRange nvtx_range("mgcccs_setup");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!out || !valid_params(p) || !v1 || !v2 || !v12 || !workspace) return MGCCCS_EINVAL;
  *out = nullptr;
  size_t need = mgcccs_workspace_size(p);
  if (workspace_bytes < need) return MGCCCS_ENOSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return MGCCCS_EINVAL;
  mgcccs_handle* h = new (std::nothrow) mgcccs_handle();
  if (!h) return MGCCCS_EINVAL;
  h->p = *p;
  h->L = p->levels;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  Carver cv{reinterpret_cast<char*>(workspace)};
  layout(h, cv);
  int rc = do_setup(h, reinterpret_cast<const cplx*>(v1), reinterpret_cast<const cplx*>(v2),
                    reinterpret_cast<const cplx*>(v12));
  if (!rc && h->km > 0) rc = create_krylov_objects(h);
  if (rc) {
    mgcccs_destroy(h);
    return rc;
  }
  *out = h;
  return MGCCCS_OK;
}

int mgcccs_setup_with_states(mgcccs_t* out, const mgcccs_params* p, const mgcccs_c128* v1, const mgcccs_c128* v2,
                             const mgcccs_c128* v12, const mgcccs_c128* lambda, const mgcccs_c128* phi,
                             const mgcccs_c128* mu, const mgcccs_c128* vphi, void* workspace, size_t workspace_bytes,
                             void* stream) {
  MgcRange nvtx_range("mgcccs_setup_with_states");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!out || !valid_params(p) || !v1 || !v2 || !v12 || !workspace) return MGCCCS_EINVAL;
  if (p->n_b > 0 && (!lambda || !phi || !mu || !vphi)) return MGCCCS_EINVAL;
  *out = nullptr;
  size_t need = mgcccs_workspace_size(p);
  if (workspace_bytes < need) return MGCCCS_ENOSPACE;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return MGCCCS_EINVAL;
  mgcccs_handle* h = new (std::nothrow) mgcccs_handle();
  if (!h) return MGCCCS_EINVAL;
  h->p = *p;
  h->L = p->levels;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  Carver cv{reinterpret_cast<char*>(workspace)};
  layout(h, cv);
  int rc = do_setup(h, reinterpret_cast<const cplx*>(v1), reinterpret_cast<const cplx*>(v2),
                    reinterpret_cast<const cplx*>(v12), reinterpret_cast<const cplx*>(lambda),
                    reinterpret_cast<const cplx*>(phi), reinterpret_cast<const cplx*>(mu),
                    reinterpret_cast<const cplx*>(vphi));
  if (!rc && h->km > 0) rc = create_krylov_objects(h);
  if (rc) {
    mgcccs_destroy(h);
    return rc;
  }
  *out = h;
  return MGCCCS_OK;
}

int mgcccs_vcycle(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f) {
  MgcRange nvtx_range("mgcccs_vcycle");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f) return MGCCCS_EINVAL;
  return vcycle_fine(h, reinterpret_cast<cplx*>(u), reinterpret_cast<const cplx*>(f), false);
}

int mgcccs_cccs(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f) {
  MgcRange nvtx_range("mgcccs_cccs");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f || h->nb <= 0) return MGCCCS_EINVAL;
  return cccs_fine(h, reinterpret_cast<cplx*>(u), reinterpret_cast<const cplx*>(f));
}

int mgcccs_solve(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f, double rtol, int max_iter, int* iters,
                 double* relres, double* history) {
  MgcRange nvtx_range("mgcccs_solve");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f) return MGCCCS_EINVAL;
  return solve_impl(h, reinterpret_cast<cplx*>(u), reinterpret_cast<const cplx*>(f), rtol, max_iter, iters, relres,
                    history);
}

int mgcccs_solve_host(mgcccs_t h, mgcccs_c128* u_host, const mgcccs_c128* f_host, double rtol, int max_iter,
                      int* iters, double* relres) {
  MgcRange nvtx_range("mgcccs_solve_host");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u_host || !f_host) return MGCCCS_EINVAL;
  const size_t bytes = sizeof(cplx) * (size_t)h->lv[0].mx * h->lv[0].my;
  MGC_CUDA(cudaMemcpyAsync(h->hf, f_host, bytes, cudaMemcpyHostToDevice, h->st));
  MGC_CUDA(cudaMemcpyAsync(h->hu, u_host, bytes, cudaMemcpyHostToDevice, h->st));
  int rc = solve_impl(h, h->hu, h->hf, rtol, max_iter, iters, relres, nullptr);
  if (rc && rc != MGCCCS_ENOTCONV) return rc;
  MGC_CUDA(cudaMemcpyAsync(u_host, h->hu, bytes, cudaMemcpyDeviceToHost, h->st));
  MGC_CUDA(cudaStreamSynchronize(h->st));
  return rc;
}

int mgcccs_precond_apply(mgcccs_t h, mgcccs_c128* z, const mgcccs_c128* r) {
  MgcRange nvtx_range("mgcccs_precond_apply");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !z || !r || (const void*)z == (const void*)r) return MGCCCS_EINVAL;
  if (!h->mixed) return precond(h, reinterpret_cast<cplx*>(z), reinterpret_cast<const cplx*>(r));
  // mixed handle: the complex64 preconditioner between a rounding and a widening
  const long long N = (long long)h->lv[0].mx * h->lv[0].my;
  MGC_LAUNCH(launch_demote(N, reinterpret_cast<const cplx*>(r), nullptr, h->V32, h->st));
  int rc = precond<float2>(h, h->Z32, h->V32);
  if (rc) return rc;
  MGC_LAUNCH(launch_promote(N, h->Z32, reinterpret_cast<cplx*>(z), h->st));
  return MGCCCS_OK;
}

int mgcccs_matvec(mgcccs_t h, const mgcccs_c128* x, mgcccs_c128* y) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !x || !y || (const void*)x == (const void*)y) return MGCCCS_EINVAL;
  MGC_LAUNCH(launch_apply(h->lv[0].sv, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y), h->st));
  return MGCCCS_OK;
}

int mgcccs_residual(mgcccs_t h, const mgcccs_c128* u, const mgcccs_c128* f, mgcccs_c128* r, double* norm2) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f || !r || (const void*)r == (const void*)u) return MGCCCS_EINVAL;
  return residual_norm2(h, reinterpret_cast<const cplx*>(u), reinterpret_cast<const cplx*>(f),
                        reinterpret_cast<cplx*>(r), norm2);
}

int mgcccs_smooth(mgcccs_t h, int level, mgcccs_c128* u, const mgcccs_c128* f, int sweeps) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f || level < 0 || level >= h->L || sweeps < 0) return MGCCCS_EINVAL;
  LevelBufs& b = h->lv[level];
  cplx* uu = reinterpret_cast<cplx*>(u);
  cplx* cur = uu;
  cplx* oth = b.t;
  for (int s = 0; s < sweeps; ++s) {
    MGC_LAUNCH(launch_jacobi(b.sv, cur, oth, reinterpret_cast<const cplx*>(f), h->st));
    cplx* tmp = cur; cur = oth; oth = tmp;
  }
  if (cur != uu)
    MGC_CUDA(cudaMemcpyAsync(uu, cur, sizeof(cplx) * (size_t)b.mx * b.my, cudaMemcpyDeviceToDevice, h->st));
  return MGCCCS_OK;
}

int mgcccs_level_residual(mgcccs_t h, int level, const mgcccs_c128* u, const mgcccs_c128* f, mgcccs_c128* r) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !u || !f || !r || level < 0 || level >= h->L) return MGCCCS_EINVAL;
  MGC_LAUNCH(launch_residual(h->lv[level].sv, reinterpret_cast<const cplx*>(u), reinterpret_cast<const cplx*>(f),
                             reinterpret_cast<cplx*>(r), nullptr, h->st));
  return MGCCCS_OK;
}

int mgcccs_restrict(mgcccs_t h, int level, const mgcccs_c128* r, mgcccs_c128* rc) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !r || !rc || level < 0 || level + 1 >= h->L) return MGCCCS_EINVAL;
  MGC_LAUNCH(launch_restrict(h->lv[level].mx, h->lv[level].my, reinterpret_cast<const cplx*>(r),
                             reinterpret_cast<cplx*>(rc), h->st));
  return MGCCCS_OK;
}

int mgcccs_prolong_add(mgcccs_t h, int level, const mgcccs_c128* ec, mgcccs_c128* u) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !ec || !u || level < 0 || level + 1 >= h->L) return MGCCCS_EINVAL;
  MGC_LAUNCH(launch_prolong_add(h->lv[level].mx, h->lv[level].my, reinterpret_cast<const cplx*>(ec),
                                reinterpret_cast<cplx*>(u), h->st));
  return MGCCCS_OK;
}

int mgcccs_coarse_solve(mgcccs_t h, const mgcccs_c128* f, mgcccs_c128* u) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !f || !u) return MGCCCS_EINVAL;
  MGC_LAUNCH(coarse_solve<cplx>(h, reinterpret_cast<const cplx*>(f), reinterpret_cast<cplx*>(u), h->st));
  return MGCCCS_OK;
}

int mgcccs_gs_dots(mgcccs_t h, const mgcccs_c128* V, long long ld, int k, const mgcccs_c128* w,
                   mgcccs_c128* out) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !V || !w || !out || h->km < 1 || k < 1 || k > h->km + 1) return MGCCCS_EINVAL;
  const long long N = (long long)h->lv[0].mx * h->lv[0].my;
  if (ld < N) return MGCCCS_EINVAL;
  const int nbd = multidot_blocks(N, k);
  MGC_LAUNCH(launch_multidot(N, k, reinterpret_cast<const cplx*>(V), ld, reinterpret_cast<const cplx*>(w),
                             h->dotpart, nbd, (const int*)nullptr, h->st));
  MGC_LAUNCH(launch_reduce_dots(nbd, k, h->dotpart, reinterpret_cast<cplx*>(out), nullptr, h->st));
  return MGCCCS_OK;
}

int mgcccs_gs_update(mgcccs_t h, const mgcccs_c128* V, long long ld, int k, const mgcccs_c128* coef,
                     mgcccs_c128* w) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !V || !coef || !w || k < 1 || k > MGC_MAX_RESTART + 1) return MGCCCS_EINVAL;
  const long long N = (long long)h->lv[0].mx * h->lv[0].my;
  if (ld < N) return MGCCCS_EINVAL;
  MGC_LAUNCH(launch_multiaxpy(N, k, reinterpret_cast<const cplx*>(V), ld, reinterpret_cast<const cplx*>(coef),
                              -1.0, reinterpret_cast<cplx*>(w), (double*)nullptr, h->kr_nblk, (const int*)nullptr,
                              h->st));
  return MGCCCS_OK;
}

int mgcccs_gs_dots_c64(mgcccs_t h, const mgcccs_c64* V, long long ld, int k, const mgcccs_c64* w,
                       mgcccs_c128* out) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !V || !w || !out || h->km < 1 || k < 1 || k > h->km + 1) return MGCCCS_EINVAL;
  const long long N = (long long)h->lv[0].mx * h->lv[0].my;
  if (ld < N) return MGCCCS_EINVAL;
  const int nbd = multidot_blocks(N, k);
  MGC_LAUNCH(launch_multidot(N, k, reinterpret_cast<const float2*>(V), ld, reinterpret_cast<const float2*>(w),
                             h->dotpart, nbd, (const int*)nullptr, h->st));
  MGC_LAUNCH(launch_reduce_dots(nbd, k, h->dotpart, reinterpret_cast<cplx*>(out), nullptr, h->st));
  return MGCCCS_OK;
}

int mgcccs_gs_update_c64(mgcccs_t h, const mgcccs_c64* V, long long ld, int k, const mgcccs_c128* coef,
                         mgcccs_c64* w) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !V || !coef || !w || k < 1 || k > MGC_MAX_RESTART + 1) return MGCCCS_EINVAL;
  const long long N = (long long)h->lv[0].mx * h->lv[0].my;
  if (ld < N) return MGCCCS_EINVAL;
  // the launch shape the mixed solve uses for its complex64 update
  MGC_LAUNCH(launch_multiaxpy(N, k, reinterpret_cast<const float2*>(V), ld, reinterpret_cast<const cplx*>(coef),
                              -1.0, reinterpret_cast<float2*>(w), (double*)nullptr, krylov_blocks(N, 6),
                              (const int*)nullptr, h->st));
  return MGCCCS_OK;
}

int mgcccs_get_bound_states(mgcccs_t h, mgcccs_c128* lambda, mgcccs_c128* phi, mgcccs_c128* mu,
                            mgcccs_c128* vphi) {
  if (!h || h->nb <= 0) return MGCCCS_EINVAL;
  const int nb = h->nb;
  cudaStream_t st = h->st;
  if (lambda) MGC_CUDA(cudaMemcpyAsync(lambda, h->lam, sizeof(cplx) * nb, cudaMemcpyDeviceToHost, st));
  if (mu) MGC_CUDA(cudaMemcpyAsync(mu, h->mu, sizeof(cplx) * nb, cudaMemcpyDeviceToHost, st));
  if (phi)
    MGC_CUDA(cudaMemcpyAsync(phi, h->phi, sizeof(cplx) * nb * h->lv[0].mx, cudaMemcpyDeviceToDevice, st));
  if (vphi)
    MGC_CUDA(cudaMemcpyAsync(vphi, h->vphi, sizeof(cplx) * nb * h->lv[0].my, cudaMemcpyDeviceToDevice, st));
  MGC_CUDA(cudaStreamSynchronize(st));
  return MGCCCS_OK;
}

int mgcccs_weighted_dot(mgcccs_t h, const mgcccs_c128* a, const mgcccs_c128* b, const mgcccs_c128* d,
                        mgcccs_c128 scale, mgcccs_c128* out) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !a || !b || !out) return MGCCCS_EINVAL;
  const LevelBufs& l0 = h->lv[0];
  MGC_LAUNCH(launch_weighted_dot(l0.mx, l0.my, l0.w_x, l0.w_y, reinterpret_cast<const cplx*>(a),
                                 reinterpret_cast<const cplx*>(b), reinterpret_cast<const cplx*>(d),
                                 cmk(scale.re, scale.im), h->wdot_part, reinterpret_cast<cplx*>(out), h->st));
  h->launches++;   // two kernels
  return MGCCCS_OK;
}

int mgcccs_weighted_product(mgcccs_t h, const mgcccs_c128* a, const mgcccs_c128* b, mgcccs_c128 scale,
                            mgcccs_c128* out) {
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!h || !a || !b || !out) return MGCCCS_EINVAL;
  const LevelBufs& l0 = h->lv[0];
  MGC_LAUNCH(launch_weighted_product(l0.mx, l0.my, l0.w_x, l0.w_y, reinterpret_cast<const cplx*>(a),
                                     reinterpret_cast<const cplx*>(b), cmk(scale.re, scale.im),
                                     reinterpret_cast<cplx*>(out), h->st));
  return MGCCCS_OK;
}

int mgcccs_batch_solve(mgcccs_t* handles, int count, mgcccs_c128* const* u, const mgcccs_c128* const* f,
                       double rtol, int max_iter, int* iters, double* relres, int* status) {
  MgcRange nvtx_range("mgcccs_batch_solve");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!handles || count < 1 || !u || !f || max_iter < 1 || !(rtol >= 0.0)) return MGCCCS_EINVAL;
  std::vector<BatchItem> items(count);
  for (int k = 0; k < count; ++k) {
    mgcccs_handle* h = handles[k];
    if (!h || h->km < 1 || !u[k] || !f[k]) return MGCCCS_EINVAL;
    for (int q = 0; q < k; ++q)
      if (handles[q] == h) return MGCCCS_EINVAL;   // a handle's buffers serve one problem
    items[k] = BatchItem{h, reinterpret_cast<cplx*>(u[k]), reinterpret_cast<const cplx*>(f[k]), 0.0, INFINITY,
                         1.0, rtol, INFINITY, 0, 0, true, false, MGCCCS_OK};
  }
  for (auto& it : items) {
    double fn2 = 0.0;
    int rc = vec_norm2(it.h, it.f, &fn2);
    if (rc) return rc;
    it.fn = std::sqrt(fn2);
    if (fn2 == 0.0) {
      const LevelBufs& b = it.h->lv[0];
      MGC_CUDA(cudaMemsetAsync(it.u, 0, sizeof(cplx) * (size_t)b.mx * b.my, it.h->st));
      it.active = false;
      it.rr = 0.0;
    } else if (!std::isfinite(it.fn)) {
      it.active = false;
      it.rr = NAN;
      it.status = MGCCCS_ENONFINITE;
    }
  }
  int rc = batch_solve_impl(items, rtol, max_iter);
  if (rc) return rc;
  int worst = MGCCCS_OK;
  for (int k = 0; k < count; ++k) {
    MGC_CUDA(cudaStreamSynchronize(items[k].h->st));
    if (iters) iters[k] = items[k].steps;
    if (relres) relres[k] = items[k].rr;
    if (status) status[k] = items[k].status;
    if (items[k].status == MGCCCS_ENONFINITE || items[k].status == MGCCCS_EDIVERGED) worst = items[k].status;
    else if (items[k].status == MGCCCS_ENOTCONV && worst == MGCCCS_OK) worst = MGCCCS_ENOTCONV;
  }
  return worst;
}

int mgcccs_axis_spectrum(mgcccs_t h, int axis, int method, mgcccs_c128* lam_host) {
  if (!h || !lam_host || (axis != 0 && axis != 1) || (method != 0 && method != 1)) return MGCCCS_EINVAL;
  const LevelBufs& b = h->lv[0];
  const int m = axis == 0 ? b.mx : b.my;
  const cplx* west = axis == 0 ? b.west_x : b.west_y;
  const cplx* east = axis == 0 ? b.east_x : b.east_y;
  const cplx* diag = axis == 0 ? b.diag_x : b.diag_y;
  const cplx* v = axis == 0 ? h->v1c : h->v2c;
  if (method == 0) {
    bool ok = false;
    MGC_CUDA(eig_aberth(m, west, east, diag, v, h->eig_ab, h->eig_vals, &ok, h->st));
    if (!ok) return MGCCCS_EBREAKDOWN;
  } else {
    MGC_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), h->st));
    MGC_LAUNCH(launch_qr_spectrum(m, west, east, diag, v, h->eig_ab, h->eig_vals, h->status, h->st));
    int st = 0;
    MGC_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    MGC_CUDA(cudaStreamSynchronize(h->st));
    if (st) return MGCCCS_EBREAKDOWN;
  }
  MGC_CUDA(cudaMemcpyAsync(lam_host, h->eig_vals, sizeof(cplx) * m, cudaMemcpyDeviceToHost, h->st));
  MGC_CUDA(cudaStreamSynchronize(h->st));
  return MGCCCS_OK;
}

int mgcccs_eig_fallbacks(mgcccs_t h) { return h ? h->eig_fallbacks : -1; }

int mgcccs_set_solve_driver(mgcccs_t h, int driver) {
  if (!h || (driver != MGCCCS_DRIVER_GRAPH && driver != MGCCCS_DRIVER_HOST)) return MGCCCS_EINVAL;
  h->driver = driver;
  return MGCCCS_OK;
}

int mgcccs_set_tile_rows(mgcccs_t h, int rows) {
  if (!h || (rows != 0 && rows != 2 && rows != 4 && rows != 8)) return MGCCCS_EINVAL;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return MGCCCS_ECUDA;
  for (int l = 0; l < h->L; ++l) {
    h->lv[l].sv.tile_rows = rows;
    h->lv[l].sv32.tile_rows = rows;
  }
  // the cached graphs hold the old launch shapes
  for (int j = 0; j < MGC_MAX_RESTART; ++j) {
    if (h->step_exec[j]) cudaGraphExecDestroy(h->step_exec[j]);
    if (h->step_exec32[j]) cudaGraphExecDestroy(h->step_exec32[j]);
    h->step_exec[j] = h->step_exec32[j] = nullptr;
  }
  for (int q = 0; q < 4; ++q) {
    if (h->solve_exec[q]) cudaGraphExecDestroy(h->solve_exec[q]);
    h->solve_exec[q] = nullptr;
    h->solve_u[q] = h->solve_f[q] = nullptr;
  }
  return MGCCCS_OK;
}

struct mgcccs_batch {
  std::vector<mgcccs_handle*> hs;
  std::vector<cplx*> u;
  cudaStream_t st;
  cudaGraphExec_t exec;
};

int mgcccs_batch_create(mgcccs_batch_t* out, mgcccs_t* handles, int count, mgcccs_c128* const* u,
                        const mgcccs_c128* const* f, void* stream) {
  MgcRange nvtx_range("mgcccs_batch_create");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!out || !handles || count < 1 || !u || !f) return MGCCCS_EINVAL;
  *out = nullptr;
  std::vector<mgcccs_handle*> hs(count);
  std::vector<cplx*> us(count);
  std::vector<const cplx*> fs(count);
  for (int k = 0; k < count; ++k) {
    hs[k] = handles[k];
    us[k] = reinterpret_cast<cplx*>(u[k]);
    fs[k] = reinterpret_cast<const cplx*>(f[k]);
    if (!hs[k] || hs[k]->km < 1 || !us[k] || !fs[k]) return MGCCCS_EINVAL;
    for (int q = 0; q < k; ++q)
      if (hs[q] == hs[k]) return MGCCCS_EINVAL;
  }
  mgcccs_batch* b = new (std::nothrow) mgcccs_batch();
  if (!b) return MGCCCS_EINVAL;
  b->hs = hs;
  b->u = us;
  b->st = reinterpret_cast<cudaStream_t>(stream);
  b->exec = nullptr;
  int rc = instantiate_solves(hs.data(), us.data(), fs.data(), count, &b->exec);
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return MGCCCS_OK;
}

int mgcccs_batch_run(mgcccs_batch_t b, double rtol, int max_iter, int* iters, double* relres, int* status) {
  MgcRange nvtx_range("mgcccs_batch_run");
  mgc_not_a_kernel();   // the caller's stream: start a new chain of programmatic launches
  if (!b || max_iter < 1 || !(rtol >= 0.0)) return MGCCCS_EINVAL;
  for (mgcccs_handle* h : b->hs) {
    int rc = stage_ctl(h, rtol, max_iter, b->st);
    if (rc) return rc;
  }
  mgc_not_a_kernel();
  if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return MGCCCS_ECUDA;
  for (mgcccs_handle* h : b->hs) {
    int rc = fetch_ctl(h, b->st);
    if (rc) return rc;
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return MGCCCS_ECUDA;
  int worst = MGCCCS_OK;
  for (size_t k = 0; k < b->hs.size(); ++k) {
    int s = finish_ctl(b->hs[k], b->u[k], iters ? iters + k : nullptr, relres ? relres + k : nullptr);
    if (s == MGCCCS_ECUDA) return s;
    if (status) status[k] = s;
    if (s == MGCCCS_ENONFINITE || s == MGCCCS_EDIVERGED) worst = s;
    else if (s == MGCCCS_ENOTCONV && worst == MGCCCS_OK) worst = MGCCCS_ENOTCONV;
  }
  return worst;
}

void mgcccs_batch_destroy(mgcccs_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
}

long long mgcccs_launch_count(mgcccs_t h) { return h ? h->launches : -1; }

const char* mgcccs_strerror(int code) {
  switch (code) {
    case MGCCCS_OK: return "ok";
    case MGCCCS_EINVAL: return "invalid argument (sizes, levels, n_b, null or misaligned pointer)";
    case MGCCCS_ECUDA: return "CUDA runtime error or kernel launch failure";
    case MGCCCS_ENOSPACE: return "workspace smaller than mgcccs_workspace_size()";
    case MGCCCS_EBREAKDOWN: return "zero pivot or eigen-solve breakdown during setup";
    case MGCCCS_ENONFINITE: return "residual is not finite";
    case MGCCCS_ENOTCONV: return "max_iter reached before rtol";
    case MGCCCS_EDIVERGED: return "the residual grew above 1e6 times its minimum: the iteration diverges";
  }
  return "unknown error code";
}

void mgcccs_destroy(mgcccs_t h) {
  if (!h) return;
  for (int j = 0; j < MGC_MAX_RESTART; ++j) {
    if (h->step_exec[j]) cudaGraphExecDestroy(h->step_exec[j]);
    if (h->step_exec32[j]) cudaGraphExecDestroy(h->step_exec32[j]);
  }
  for (int q = 0; q < 2; ++q)
    if (h->ev[q]) cudaEventDestroy(h->ev[q]);
  for (int q = 0; q < 4; ++q)
    if (h->solve_exec[q]) cudaGraphExecDestroy(h->solve_exec[q]);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  for (int q = 0; q < 2; ++q)
    if (h->gst[q]) cudaStreamDestroy(h->gst[q]);
  if (h->est_host) cudaFreeHost(h->est_host);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  delete h;
}

}  // extern "C"
