// Internal types and device helpers of the MG-CCCS library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "mgcccs.h"

typedef double2 cplx;

#define MGC_MAX_LEVELS 16
#define MGC_MAX_NB 8
#define MGC_MAX_COARSE 1024    // unknowns of a coarsest grid solved by its dense inverse
#define MGC_BP_MAX_M 64        // larger coarsest grids: block cyclic reduction, rows of at most
#define MGC_BP_MAX_ROWS 4096   //   64 nodes and at most 4096 rows
#define MGC_MAX_RESTART 60

// ---------------------------------------------------------------- complex arithmetic
__host__ __device__ __forceinline__ cplx cmk(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cneg(cplx a) { return cmk(-a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscal(double s, cplx a) { return cmk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
__host__ __device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx acc) {
  return cmk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc - a*b
__host__ __device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx acc) {
  return cmk(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs1(cplx a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ __forceinline__ double cmod(cplx a) { return hypot(a.x, a.y); }

// a / b by Smith's algorithm (R. L. Smith, "Algorithm 116: Complex division",
// CACM 5(8), 1962): scale by the larger component of b to avoid overflow.
__host__ __device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  if (fabs(b.y) <= fabs(b.x)) {
    double r = b.y / b.x;
    double den = b.x + b.y * r;
    return cmk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    double r = b.x / b.y;
    double den = b.x * r + b.y;
    return cmk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}

// Principal square root: sqrt(z) = sqrt((|z|+Re z)/2) + i sgn(Im z) sqrt((|z|-Re z)/2),
// evaluated from the larger of the two to avoid cancellation.
__host__ __device__ __forceinline__ cplx csqrt_p(cplx z) {
  double m = hypot(z.x, z.y);
  if (m == 0.0) return cmk(0.0, 0.0);
  if (z.x >= 0.0) {
    double t = sqrt(0.5 * (m + z.x));
    return cmk(t, z.y / (2.0 * t));
  } else {
    double t = sqrt(0.5 * (m - z.x));
    double s = (z.y < 0.0) ? -t : t;
    return cmk(z.y / (2.0 * s), s);
  }
}

// single-precision complex (complex64) counterparts, used by the mixed-precision
// smoother, transfers and inner Krylov solve
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscal(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 acc) {
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// Complex element type traits: C = double2 (complex128) or float2 (complex64).
template <class C> struct CT;
template <> struct CT<double2> {
  typedef double R;
  static __host__ __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct CT<float2> {
  typedef float R;
  static __host__ __device__ __forceinline__ float2 make(double a, double b) {
    return make_float2((float)a, (float)b);
  }
};
// binary32 -> binary64 by integer operations (exact, IEEE 754 layouts: 8/23-bit and
// 11/52-bit exponent/fraction fields, biases 127 and 1023).  On this part a conversion
// instruction issues on the FP64 pipe, 1/64 of the FP32 rate and the unit the
// mixed-precision path's FP64 kernels are bound by; the integer form issues on the ALU.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu;
  unsigned m = b & 0x7fffffu;
  int ed;
  if (e == 0u) {
    if (m == 0u) return __hiloint2double((int)sign, 0);          // +-0
    const int s = __clz((int)m) - 8;                              // subnormal: normalise
    m = (m << s) & 0x7fffffu;
    ed = 897 - s;
  } else {
    ed = e == 0xffu ? 0x7ff : (int)e + 896;                       // inf / nan keep their fraction
  }
  return __hiloint2double((int)(sign | ((unsigned)ed << 20) | (m >> 3)), (int)(m << 29));
}
__host__ __device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_c128(float2 a) {
#ifdef __CUDA_ARCH__
  return make_double2(f2d_exact(a.x), f2d_exact(a.y));
#else
  return make_double2(a.x, a.y);
#endif
}

// ---------------------------------------------------------------- level descriptors

// Neighbour coefficients of one axis of one level (Eq. (11)).  Interior indices i < u have
// both neighbours at the inner grid spacing h e^{i gamma}, so west = east = cin, the closed
// form -1/(2 h^2) e^{-2 i gamma}.  Indices i >= u (the kink at R0 and the complex-scaled
// part) read west/east from the per-node arrays, which the setup forms from the node
// coordinates as Eq. (11) does; u = 0 sends every index there.
template <class C>
struct AxisCoefT {
  int u;
  int in_real;             // 1: cin has zero imaginary part (a level on the unrotated contour)
  C cin;
};

// 5-point operator of one level, (H - E)u = D u + west_x u_W + east_x u_E + west_y u_S + east_y u_N.
template <class C>
struct StencilViewT {
  int mx, my;              // interior nodes per axis (row pitch = mx)
  AxisCoefT<C> cx, cy;     // per-axis uniform regions and their coefficients
  int rbox;                // 1: both cin real and D real for i < cx.u, j < cy.u (real potential)
  typename CT<C>::R keep;  // 1 - omega: the share of u an omega-Jacobi update keeps
  const C* west_x;         // [mx]
  const C* east_x;         // [mx]
  const C* west_y;         // [my]
  const C* east_y;         // [my]
  const C* D;              // [my*mx] full diagonal of H - E
  const C* Dinv;           // [my*mx] omega / D
  int tile_rows;           // block height of the stencil passes on levels too small to fill the
                           // GPU with 32 x 8 blocks (2, 4 or 8; 0 = 2); a tuning knob only
};
typedef StencilViewT<cplx> StencilView;
typedef StencilViewT<float2> StencilView32;

// How the nodes of one block take the neighbour coefficients of an axis: all inside the
// inner region (AX_IN, the closed-form coefficient), all beyond it (AX_ARR, per-node
// arrays) or straddling it (AX_GEN, a test per node); and how they take D and omega/D:
// complex (DG_CPLX), real (DG_REAL, the block lies in the real box) or by a test per node
// (DG_GEN).  The stencil kernels select one instantiation per block, so the per-node code
// of nearly every block is free of data-dependent branches: the compiler turns such short
// branches into predicated code, and a warp then issues the FP64 instructions of both
// sides.  Every instantiation gives the same result at a node: the real forms are the
// complex ones with zero imaginary parts dropped.
enum { AX_GEN = 0, AX_IN = 1, AX_ARR = 2 };
enum { DG_CPLX = 0, DG_REAL = 1, DG_GEN = 2 };
template <int V>
struct IntC {
  static constexpr int value = V;
};

// acc - (west_i u_m + east_i u_p) along one axis (SUB) or acc + (...) (!SUB), where u_m, u_p
// are the neighbour values (zero outside the interior).  In the inner region one
// coefficient multiplies u_m + u_p: 4 FP64 operations per complex value with a real
// coefficient (IR = 1), 6 with a complex one, against 8 with two per-node coefficients.
template <int K, int IR, bool SUB, class C>
__device__ __forceinline__ C axis_acc(const AxisCoefT<C>& a, const C* __restrict__ west, const C* __restrict__ east,
                                      int i, C um, C up, C acc) {
  typedef typename CT<C>::R R;
  if constexpr (K == AX_GEN) {
    if (i < a.u) return axis_acc<AX_IN, IR, SUB>(a, west, east, i, um, up, acc);
    return axis_acc<AX_ARR, IR, SUB>(a, west, east, i, um, up, acc);
  } else if constexpr (K == AX_IN) {
    const C sm = cadd(um, up);
    if constexpr (IR) {
      const R c = SUB ? -a.cin.x : a.cin.x;
      acc.x = fma(c, sm.x, acc.x);
      acc.y = fma(c, sm.y, acc.y);
      return acc;
    } else {
      return SUB ? cfms(a.cin, sm, acc) : cfma(a.cin, sm, acc);
    }
  } else {
    const C w = __ldg(west + i), e = __ldg(east + i);
    return SUB ? cfms(e, up, cfms(w, um, acc)) : cfma(e, up, cfma(w, um, acc));
  }
}

// Whether node (i, j) lies in the region where D and omega/D are real.
template <class C>
__device__ __forceinline__ bool in_rbox(const StencilViewT<C>& s, int i, int j) {
  return s.rbox && i < s.cx.u && j < s.cy.u;
}

template <int DG, class C>
__device__ __forceinline__ bool diag_real(const StencilViewT<C>& s, int i, int j) {
  if constexpr (DG == DG_GEN) return in_rbox(s, i, j);
  else return DG == DG_REAL;
}

// Real part of a complex array element (only the real word is loaded).
template <class C>
__device__ __forceinline__ typename CT<C>::R ldre(const C* __restrict__ a, int p) {
  return __ldg(reinterpret_cast<const typename CT<C>::R*>(a) + 2 * p);
}

// f - (H - E)u at node p = (i, j) from the centre value uc, the neighbour values (west,
// east, south, north) and f_p.
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C residual_vals(const StencilViewT<C>& s, int i, int j, int p, C uc, C uw, C ue, C us,
                                           C un, C fp) {
  typedef typename CT<C>::R R;
  C t = axis_acc<KX, IR, true>(s.cx, s.west_x, s.east_x, i, uw, ue, fp);
  t = axis_acc<KY, IR, true>(s.cy, s.west_y, s.east_y, j, us, un, t);
  if (diag_real<DG>(s, i, j)) {
    const R d = ldre(s.D, p);
    t.x = fma(-d, uc.x, t.x);
    t.y = fma(-d, uc.y, t.y);
    return t;
  }
  return cfms(__ldg(s.D + p), uc, t);
}

// (H - E)u at node p = (i, j) from the centre and neighbour values.
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C apply_vals(const StencilViewT<C>& s, int i, int j, int p, C uc, C uw, C ue, C us,
                                        C un) {
  typedef typename CT<C>::R R;
  C a;
  if (diag_real<DG>(s, i, j)) {
    const R d = ldre(s.D, p);
    a.x = d * uc.x;
    a.y = d * uc.y;
  } else {
    a = cmul(__ldg(s.D + p), uc);
  }
  a = axis_acc<KX, IR, false>(s.cx, s.west_x, s.east_x, i, uw, ue, a);
  return axis_acc<KY, IR, false>(s.cy, s.west_y, s.east_y, j, us, un, a);
}

// One omega-Jacobi update u + (omega/D)(f - (H - E)u) at node p = (i, j), evaluated as
// (1 - omega) u + (omega/D)(f - N u) with N the off-diagonal part of H - E: the diagonal
// term (omega/D) D u is omega u, so D is not read.  FP64 operations per node: 12 where
// the coefficients and omega/D are real, 18 with one complex-scaled axis, 22 with two.
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C jacobi_vals(const StencilViewT<C>& s, int i, int j, int p, C uc, C uw, C ue, C us,
                                         C un, C fp) {
  typedef typename CT<C>::R R;
  C t = axis_acc<KX, IR, true>(s.cx, s.west_x, s.east_x, i, uw, ue, fp);
  t = axis_acc<KY, IR, true>(s.cy, s.west_y, s.east_y, j, us, un, t);
  C o = cscal(s.keep, uc);
  if (diag_real<DG>(s, i, j)) {
    const R di = ldre(s.Dinv, p);
    o.x = fma(di, t.x, o.x);
    o.y = fma(di, t.y, o.y);
    return o;
  }
  return cfma(__ldg(s.Dinv + p), t, o);
}

// Kind of an axis for the index range [lo, hi) of a block.
template <class C>
__device__ __forceinline__ int axis_kind(const AxisCoefT<C>& a, int lo, int hi) {
  return hi <= a.u ? AX_IN : (lo >= a.u ? AX_ARR : AX_GEN);
}

template <int KX, int KY, class F>
__device__ __forceinline__ void dispatch_ir_dg(bool ir, bool rb, F& f) {
  if constexpr (KX == AX_ARR || KY == AX_ARR) {
    if (ir) f(IntC<KX>(), IntC<KY>(), IntC<1>(), IntC<DG_CPLX>());
    else f(IntC<KX>(), IntC<KY>(), IntC<0>(), IntC<DG_CPLX>());
  } else {
    constexpr int DGR = (KX == AX_IN && KY == AX_IN) ? DG_REAL : DG_GEN;
    if (rb) f(IntC<KX>(), IntC<KY>(), IntC<1>(), IntC<DGR>());   // a real box needs real inner coefficients
    else if (ir) f(IntC<KX>(), IntC<KY>(), IntC<1>(), IntC<DG_CPLX>());
    else f(IntC<KX>(), IntC<KY>(), IntC<0>(), IntC<DG_CPLX>());
  }
}

// Calls f(IntC<KX>, IntC<KY>, IntC<IR>, IntC<DG>) with the kinds of the block covering
// interior indices [i0, i1) x [j0, j1) (clipped to the interior by the caller).
template <class C, class F>
__device__ __forceinline__ void dispatch_kinds(const StencilViewT<C>& s, int i0, int i1, int j0, int j1, F&& f) {
  const int kx = axis_kind(s.cx, i0, i1), ky = axis_kind(s.cy, j0, j1);
  const bool ir = s.cx.in_real && s.cy.in_real;
  const bool rb = s.rbox && ir;
  switch (kx * 3 + ky) {
    case AX_GEN * 3 + AX_GEN: dispatch_ir_dg<AX_GEN, AX_GEN>(ir, rb, f); break;
    case AX_GEN * 3 + AX_IN: dispatch_ir_dg<AX_GEN, AX_IN>(ir, rb, f); break;
    case AX_GEN * 3 + AX_ARR: dispatch_ir_dg<AX_GEN, AX_ARR>(ir, rb, f); break;
    case AX_IN * 3 + AX_GEN: dispatch_ir_dg<AX_IN, AX_GEN>(ir, rb, f); break;
    case AX_IN * 3 + AX_IN: dispatch_ir_dg<AX_IN, AX_IN>(ir, rb, f); break;
    case AX_IN * 3 + AX_ARR: dispatch_ir_dg<AX_IN, AX_ARR>(ir, rb, f); break;
    case AX_ARR * 3 + AX_GEN: dispatch_ir_dg<AX_ARR, AX_GEN>(ir, rb, f); break;
    case AX_ARR * 3 + AX_IN: dispatch_ir_dg<AX_ARR, AX_IN>(ir, rb, f); break;
    default: dispatch_ir_dg<AX_ARR, AX_ARR>(ir, rb, f); break;
  }
}

// residual_vals and jacobi_vals with D (respectively omega/D) at the node already loaded
// by the caller (dv; only its real part is used where the diagonal is real): a fused pass
// issues that load together with its other loads, before its block barrier.  Same
// arithmetic, so the same results.
template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C residual_vals_d(const StencilViewT<C>& s, int i, int j, C dv, C uc, C uw, C ue, C us,
                                             C un, C fp) {
  C t = axis_acc<KX, IR, true>(s.cx, s.west_x, s.east_x, i, uw, ue, fp);
  t = axis_acc<KY, IR, true>(s.cy, s.west_y, s.east_y, j, us, un, t);
  if (diag_real<DG>(s, i, j)) {
    t.x = fma(-dv.x, uc.x, t.x);
    t.y = fma(-dv.x, uc.y, t.y);
    return t;
  }
  return cfms(dv, uc, t);
}

template <int KX, int KY, int IR, int DG, class C>
__device__ __forceinline__ C jacobi_vals_d(const StencilViewT<C>& s, int i, int j, C dinv, C uc, C uw, C ue, C us,
                                           C un, C fp) {
  C t = axis_acc<KX, IR, true>(s.cx, s.west_x, s.east_x, i, uw, ue, fp);
  t = axis_acc<KY, IR, true>(s.cy, s.west_y, s.east_y, j, us, un, t);
  C o = cscal(s.keep, uc);
  if (diag_real<DG>(s, i, j)) {
    o.x = fma(dinv.x, t.x, o.x);
    o.y = fma(dinv.x, t.y, o.y);
    return o;
  }
  return cfma(dinv, t, o);
}


// Error bits written by kernels into the handle's device status word.
enum {
  MGC_ST_PIVOT = 1,        // zero pivot in a dense or block factorisation
  MGC_ST_EIG = 2,          // eigen-solve failed to converge
  MGC_ST_NONFINITE = 4
};

// ---------------------------------------------------------------- programmatic dependent launch
// The kernels of the solve path are launched with the programmatic-stream-serialization
// attribute (PDL, sm_90 and later) whenever the previous operation the library enqueued on
// the same stream was one of its kernels: the next kernel is then launched, and its blocks
// dispatched, as the blocks of the current one exit, instead of after the whole grid and
// its launch bookkeeping have retired.  Correctness does not depend on it: every kernel
// launched this way calls mgc_pdl_enter() before it touches anything an earlier kernel of
// the solve writes (the block-reduction levels first load their setup-time factors, which
// no solve kernel writes), and griddepcontrol.wait returns only once the preceding kernel
// has completed and its writes are visible.  No kernel triggers its successor early (griddepcontrol.launch_dependents):
// measured on the 1024^2 solve, an early trigger made the FP64 solve slower (34.8 against
// 33.0 ms; the FP64-bound kernels then share their SMs with resident, waiting blocks),
// while the trigger at block exit gives 33.0 ms FP64 and 12.9 ms mixed against 33.2 and
// 13.2 ms with plain stream-ordered launches (-DMGC_NO_PDL builds those).
__device__ __forceinline__ void mgc_pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Host side: the stream of the last kernel the library enqueued on this thread, or null
// after any other operation (copy, memset, event, capture boundary, conditional node).
extern thread_local cudaStream_t g_mgc_last_kernel_stream;
extern thread_local bool g_mgc_last_was_kernel;
inline void mgc_not_a_kernel() { g_mgc_last_was_kernel = false; }

template <typename... KArgs, typename... Args>
inline cudaError_t mgc_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
#ifndef MGC_NO_PDL   // -DMGC_NO_PDL builds the library with plain stream-ordered launches
  if (g_mgc_last_was_kernel && g_mgc_last_kernel_stream == st) {
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
#endif
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
  g_mgc_last_was_kernel = e == cudaSuccess;
  g_mgc_last_kernel_stream = st;
  return e;
}

// ---------------------------------------------------------------- tracing
// Host-side NVTX range for the lifetime of the object: every C-ABI entry point and every
// V-cycle level opens one, so a timeline tool shows which call and level enqueued each
// kernel (inside a captured graph the ranges mark the capture, not the replays).  Without
// a tool attached the calls return at once.
struct MgcRange {
  explicit MgcRange(const char* name) { nvtxRangePushA(name); }
  ~MgcRange() { nvtxRangePop(); }
  MgcRange(const MgcRange&) = delete;
  MgcRange& operator=(const MgcRange&) = delete;
};
const char* mgc_level_range_name(int level);   // "mgcccs level <l>"

// ---------------------------------------------------------------- launchers (defined in the .cu files)
// Streaming multiprocessors of the current device, queried once per device; grid sizes
// of the grid-stride kernels and the block-height switch of the stencil kernels scale
// with it.  Without a usable device (a size query on a host with no GPU) it returns 152,
// the count of the part this library is tuned on, which only shapes the workspace.
int mgc_sm_count();
// All return cudaGetLastError() of their launch.

// kernels_mg.cu (templates instantiated for C = double2 and C = float2)
template <class C>
cudaError_t launch_jacobi(const StencilViewT<C>& s, const C* u_in, C* u_out, const C* f, cudaStream_t st);
template <class C>
cudaError_t launch_jacobi_zero(const StencilViewT<C>& s, C* u_out, const C* f, cudaStream_t st);
// w <- w / sqrt(*norm2) in place, and u_out = omega D^{-1} w (zero-start sweep)
template <class C>
cudaError_t launch_scale_jacobi_zero(const StencilViewT<C>& s, C* w, const double* norm2, C* u_out,
                                     cudaStream_t st);
template <class C>
cudaError_t launch_residual(const StencilViewT<C>& s, const C* u, const C* f, C* r, double* norm_part,
                            cudaStream_t st);
template <class C>
int residual_norm_blocks(const StencilViewT<C>& s);
template <class C>
cudaError_t launch_restrict(int mx, int my, const C* r, C* rc, cudaStream_t st);
template <class C>
cudaError_t launch_prolong_add(int mx, int my, const C* ec, C* u, cudaStream_t st);
// o = one omega-Jacobi sweep from u + P ec (the level's prolongation and first
// post-smoothing sweep in one pass; u itself is left unchanged)
template <class C>
cudaError_t launch_prolong_jacobi(const StencilViewT<C>& s, const C* ec, const C* u, C* o, const C* f,
                                  cudaStream_t st);
// fc = restriction of f - (H - E) u: a level's residual and restriction in one pass, from the
// given u, or (zero) after the zero-start sweep u = omega D^{-1} f, which is then stored
template <class C>
cudaError_t launch_zero_residual_restrict(const StencilViewT<C>& s, const C* f, C* u, C* fc, bool zero,
                                          cudaStream_t st);
template <class C>
cudaError_t launch_coarse_solve(int nc, const cplx* Ainv, const C* f, C* u, cudaStream_t st);
template <class C>
cudaError_t launch_apply(const StencilViewT<C>& s, const C* x, C* y, cudaStream_t st, double* norm_part = nullptr);
template <class C>
cudaError_t launch_norm2(const C* v, long long n, double* part, int nblocks, cudaStream_t st);
cudaError_t launch_sum_partials(const double* part, int n, double* out, cudaStream_t st,
                                const int* gate = nullptr);
int norm2_blocks(long long n);
cudaError_t launch_demote(long long n, const cplx* x, const double* norm2, float2* y, cudaStream_t st);
cudaError_t launch_promote_add(long long n, const float2* e, const double* norm2, cplx* u, cudaStream_t st);
cudaError_t launch_round_copy(long long n, const cplx* a, float2* b, cudaStream_t st);
cudaError_t launch_promote(long long n, const float2* x, cplx* y, cudaStream_t st);

// kernels_krylov.cu
// grid of the grid-stride Krylov kernels: per_sm blocks of 256 threads per SM at most
int krylov_blocks(long long n, int per_sm);
int multidot_blocks(long long n, int k);
template <class C>
cudaError_t launch_multidot(long long n, int k, const C* V, long long ld, const C* w, cplx* partial,
                            int nblk, const int* gate, cudaStream_t st);
cudaError_t launch_reduce_dots(int nblk, int k, const cplx* partial, cplx* out, cplx* acc_into, cudaStream_t st);
template <class C>
cudaError_t launch_multiaxpy(long long n, int k, const C* V, long long ld, const cplx* coef, double sgn,
                             C* w, double* norm_part, int nblk, const int* gate, cudaStream_t st,
                             const int* dk = nullptr);
template <class C>
cudaError_t launch_scale_by_norm(long long n, const C* w, C* out, const double* norm2, cplx* store,
                                 int nblk, cudaStream_t st);
// the Givens update of Arnoldi step j (skipped when gate is given and *gate == 0)
cudaError_t launch_givens(int j, int m, cplx* H, cplx* cs, cplx* sn, cplx* g, double* est, const double* hnorm2,
                          cudaStream_t st, const int* gate = nullptr);
// Arguments of the Givens update of step j when k_sum_dgks performs it.
struct GivensArgs {
  int j, m;
  cplx *H, *cs, *sn, *g;
  double* est;
};
// |w|^2 from partials into *out plus the second-pass decision (*gate; in a device-driven
// graph also the conditional node hd and the counter *fired); with gv, the Givens update
// of step j whenever no second pass follows
cudaError_t launch_sum_dgks(const double* part, int n, double* out, const double* before, int* gate,
                           cudaStream_t st, cudaGraphConditionalHandle hd = 0, int* fired = nullptr,
                           const GivensArgs* gv = nullptr);
cudaError_t launch_hess_solve(int k, int m, const cplx* H, const cplx* g, cplx* y, cudaStream_t st,
                              const int* dk = nullptr);

// Control record of a device-driven GMRES solve (one per handle, in its workspace).
// The host writes the inputs before each launch of the solve graph; the control kernels
// keep the counters and the outcome.
enum { SOLVECTL_RUNNING = 0, SOLVECTL_CONVERGED = 1, SOLVECTL_MAXITER = 2, SOLVECTL_NONFINITE = 3,
       SOLVECTL_ZERO_RHS = 4, SOLVECTL_DIVERGED = 5 };
// divergence test on the true relative residual: rr above 1e6 times its minimum so far
constexpr double MGC_DIVERGENCE_FACTOR = 1e6;
struct SolveCtl {
  double fn2;          // |f|^2, written inside the graph
  double rtol, inner_rtol;
  int max_iter, mixed, m, pad0;
  int steps, k, j, cycles, outer, status;
  double rr, scale, target;
  int dgks, pad1;      // second Gram-Schmidt passes run
  double rr_min;       // smallest true relative residual so far (host sets +inf)
};
cudaError_t launch_outer_control(SolveCtl* c, const double* rn2, cudaGraphConditionalHandle h_outer,
                                 cudaGraphConditionalHandle h_cycle, cudaGraphConditionalHandle h_inner,
                                 cudaGraphConditionalHandle h_switch, cudaStream_t st);
cudaError_t launch_step_control(SolveCtl* c, const double* est, cudaGraphConditionalHandle h_inner,
                                cudaGraphConditionalHandle h_switch, cudaStream_t st);
cudaError_t launch_zero_c(int n, cplx* a, cudaStream_t st);

// kernels_cccs.cu
// Bound-state data of the CCCS for grid element type C: the states and weighted states
// and the per-tile projection partials are of type C; reduced projections, channel
// right-hand sides and channel solutions are always FP64 (the channel solves stay FP64).
template <class C>
struct CCViewT {
  int mx, my, nb;
  const C* wphi;           // [nb][mx]  w_x(i) phi_m(i)
  const C* wvphi;          // [nb][my]  w_y(j) vphi_l(j)
  const C* phi;            // [nb][mx]
  const C* vphi;           // [nb][my]
  C* Px_part;              // [ntx][nb][my]
  C* Py_part;              // [nty][nb][mx]
  cplx* Px;                // [nb][my]
  cplx* Py;                // [nb][mx]
  cplx* c;                 // [nb][nb]  c[a][b] = int int phi_a vphi_b r
  cplx* eA;                // [nb][my]
  cplx* eB;                // [nb][mx]
  const C* eAc;            // eA, eB in the element precision (the same arrays for complex128)
  const C* eBc;
  const cplx* wvphi64;     // [nb][my] FP64 weighted states for the coupling coefficients
};
typedef CCViewT<cplx> CCView;
typedef CCViewT<float2> CCView32;

// One coupled-channel system (Eqs. (28)-(29)) with its parallel-cyclic-reduction factors.
struct CRSystem {
  int m, nb;
  // right-hand side r[a][k] = P[a][k] - sum_l coef(a, l) basis[l][k] with the conventions of
  // Eqs. (25)-(26): channel A (chan 0) l > a, coef = c[a][l], basis = vphi (along y);
  // channel B (chan 1) l >= a, coef = c[l][a], basis = phi (along x)
  int chan;
  const cplx* P;           // [nb][m] projections P^x (channel A) or P^y (channel B)
  const cplx* cmat;        // [nb][nb] c
  const cplx* basis;       // [nb][m]
  cplx* e;                 // [nb][m] solution
  float2* e32;             // [nb][m] solution rounded to complex64 (mixed precision), or null
  // parallel cyclic reduction: pq = ceil(log2 m) levels; level l with stride s = 2^l
  // updates every row k by x_k -= pa_k x_{k-s} + pg_k x_{k+s}; then x_k = pbinv_k x_k.
  // Rows are 0..m-1; terms outside them are absent.
  int pq;
  cplx* pa;                // [pq][m][nb*nb]
  cplx* pg;                // [pq][m][nb*nb]
  cplx* pbinv;             // [m][nb*nb]
};
int pcr_levels(int m);
int cc_tiles_x(int mx);
int cc_tiles_y(int my);
template <class C>
cudaError_t launch_residual_project(const StencilViewT<C>& s, const CCViewT<C>& c, const C* u, const C* f,
                                    cudaStream_t st);
template <class C>
cudaError_t launch_cc_rhs(const CCViewT<C>& c, cudaStream_t st);
cudaError_t channel_solve_prepare(int nb, int m_max);
cudaError_t launch_channel_solve(const CRSystem& A, const CRSystem& B, cudaStream_t st);
template <class C>
cudaError_t launch_cccs_correct(const CCViewT<C>& c, C* u, cudaStream_t st);

// kernels_setup.cu
struct AxisSetup {
  int n;                   // cells
  double L, R0, theta, gamma;
  cplx* west; cplx* east; cplx* diag; cplx* w;   // [n-1] each
};
cudaError_t launch_setup_axis(const AxisSetup& a, cudaStream_t st);
cudaError_t launch_box_real_check(const StencilView& s, int* flag, cudaStream_t st);
cudaError_t launch_compare(int n, const cplx* a, const cplx* b, int* flag, cudaStream_t st);
cudaError_t launch_setup_diag(int mx, int my, int stride, int fine_mx, const cplx* dx, const cplx* dy,
                              const cplx* v1, const cplx* v2, const cplx* v12, double E, double omega,
                              cplx* D, cplx* Dinv, int* status, cudaStream_t st);
size_t coarse_inverse_scratch(int nc);                       // complex entries of aug
cudaError_t launch_coarse_inverse(const StencilView& s, cplx* aug, cplx* Ainv, int* status, cudaStream_t st);
// kernels_coarse.cu: coarsest grids beyond MGC_MAX_COARSE unknowns, block parallel cyclic
// reduction over the grid rows (mx <= MGC_BP_MAX_M, my <= MGC_BP_MAX_ROWS)
bool bpcr_fits(int mx, int my);
size_t bpcr_factor_entries(int mx, int my);                  // complex entries of the factors
size_t bpcr_scratch_entries(int mx, int my);                 // complex entries of setup scratch
cudaError_t launch_bpcr_setup(const StencilView& s, cplx* fac, cplx* scratch, int* status, cudaStream_t st);
// u = A_c^{-1} f through the factors; buf holds 2 mx my complex entries
template <class C>
cudaError_t launch_bpcr_solve(int mx, int my, const cplx* fac, const C* f, C* u, cplx* buf, cudaStream_t st);
// eig: all m eigenvalues when already computed (eig_aberth), else null (FP64 QR inside)
cudaError_t launch_bound_states(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                                const cplx* w, int nb, cplx* lam, cplx* phi, cplx* scratch, int* status,
                                cudaStream_t st, const cplx* eig = nullptr);
size_t bound_states_scratch(int m, int nb);
// kernels_eig.cu: all eigenvalues of diag + v with squared off-diagonals east_k west_{k+1}
// into out[m]; *ok false when the iteration did not converge (the caller falls back to QR).
size_t eig_scratch_entries(int m);
cudaError_t eig_aberth(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v, cplx* scratch,
                       cplx* out, bool* ok, cudaStream_t st);
cudaError_t launch_qr_spectrum(int m, const cplx* west, const cplx* east, const cplx* diag, const cplx* v,
                               cplx* scratch, cplx* out, int* status, cudaStream_t st);
cudaError_t launch_weight_states(int m, int nb, const cplx* w, const cplx* phi, cplx* wphi, cudaStream_t st);
cudaError_t launch_channel_potentials(int mx, int my, int nb, const cplx* wphi, const cplx* phi,
                                      const cplx* wvphi, const cplx* vphi, const cplx* v12,
                                      cplx* VA, cplx* VB, cudaStream_t st);
cudaError_t launch_channel_factor_pcr(const CRSystem& S, const cplx* diag, const cplx* v, double E, const cplx* lam,
                                      const cplx* Vc, const cplx* a, const cplx* c, cplx* scratch, int* status,
                                      cudaStream_t st);
size_t channel_factor_pcr_scratch(int m, int nb);
// kernels_adjoint.cu
int wdot_blocks(long long n);
cudaError_t launch_weighted_dot(int mx, int my, const cplx* wx, const cplx* wy, const cplx* a, const cplx* b,
                                const cplx* d, cplx scale, cplx* part, cplx* out, cudaStream_t st);
cudaError_t launch_weighted_product(int mx, int my, const cplx* wx, const cplx* wy, const cplx* a, const cplx* b,
                                    cplx scale, cplx* out, cudaStream_t st);
