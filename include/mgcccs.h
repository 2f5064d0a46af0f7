/*
 * mgcccs.h -- C ABI of the GB300 (sm_103a) MG-CCCS library.
 *
 * MG-CCCS (Cools & Vanroose, arXiv:1412.1953) solves the 2D driven Schrodinger
 * equation of Eq. (7),
 *
 *     (-1/2 Laplacian + V1(x) + V2(y) + V12(x,y) - E) u = f ,
 *
 * discretised by second-order finite differences (Eq. (11)) on a uniform grid
 * whose nodes are bent into the complex plane beyond R0 (exterior complex
 * scaling, Sec. 2.5).  One MG-CCCS iteration is one multigrid V(nu1,nu2)-cycle
 * with omega-Jacobi smoothing, full-weighting restriction and bilinear
 * interpolation (Sec. 3.2), followed by one Coupled Channel Correction Step
 * (Sec. 4.3, Eq. (30)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex values are mgcccs_c128 = {re, im} doubles, bit-compatible with
 *    cuDoubleComplex and torch.complex128.
 *  - A grid has nx x ny cells on [0,Lx] x [0,Ly]; the unknowns are the
 *    (nx-1)*(ny-1) interior nodes, stored row-major [j][i] with x (i) fastest,
 *    no padding.  Dirichlet zero is implied on the boundary ring.
 *  - "device" pointers are CUDA global-memory pointers of the current device,
 *    16-byte aligned; "host" pointers are ordinary host memory.  The caller
 *    owns every pointer it passes; the library never frees them.
 *  - All device work is issued on the stream given to mgcccs_setup (NULL =
 *    legacy default stream).  Entry points marked "async" return once the
 *    work is queued; the others synchronise that stream before returning.
 *  - Every entry point returns 0 on success or a negative MGCCCS_E* code;
 *    mgcccs_strerror() turns a code into text.  On error no output is
 *    guaranteed unless stated.
 */
#ifndef MGCCCS_H
#define MGCCCS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } mgcccs_c128;
typedef struct { float re, im; } mgcccs_c64;     /* the mixed form's Krylov vectors (torch.complex64) */
typedef struct mgcccs_handle* mgcccs_t;
typedef struct mgcccs_batch* mgcccs_batch_t;

enum {
  MGCCCS_OK = 0,
  MGCCCS_EINVAL = -1,      /* bad size, level count, null pointer, n_b, ... */
  MGCCCS_ECUDA = -2,       /* a CUDA runtime call or kernel launch failed */
  MGCCCS_ENOSPACE = -3,    /* workspace smaller than mgcccs_workspace_size() */
  MGCCCS_EBREAKDOWN = -4,  /* zero pivot in the coarsest or channel factorisation,
                              or the bound-state eigen-solve did not converge */
  MGCCCS_ENONFINITE = -5,  /* residual became NaN/Inf during a solve */
  MGCCCS_ENOTCONV = -6,    /* max_iter reached without meeting rtol (u, relres valid) */
  MGCCCS_EDIVERGED = -7    /* the relative residual rose above 1e6 times its smallest value
                              so far: the iteration diverges (u, relres valid) */
};

/* Problem and solver parameters (Sec. 2.5, Sec. 3.2, Sec. 4, Sec. 6). */
typedef struct {
  int nx, ny;            /* cells per axis; both divisible by 2^(levels-1) */
  double Lx, Ly;         /* box [0,Lx] x [0,Ly] */
  double R0x, R0y;       /* ECS start per axis; R0 >= L means no complex scaling */
  double theta;          /* ECS angle (radians), z = R0 + (x - R0) e^{i theta} */
  double E;              /* total energy (real) */
  int levels;            /* multigrid levels including the fine one (>= 1);
                            the coarsest, with (nx>>(levels-1))-1 by
                            (ny>>(levels-1))-1 interior nodes, is solved by a
                            direct method: its dense inverse up to 1024 nodes,
                            else block cyclic reduction over its rows, which
                            needs at most 64 nodes per row and 4096 rows */
  int nu1, nu2;          /* pre/post omega-Jacobi sweeps per level */
  double omega;          /* Jacobi weight (2/3 in Sec. 3.2) */
  int n_b;               /* bound states per axis used by the CCCS, 0..8;
                            0 disables the CCCS (plain multigrid) */
  double coarse_gamma;   /* the coarse levels (>= 1) use the fine ECS contour
                            rotated as a whole by e^{i coarse_gamma} */
  int krylov_restart;    /* outer solver of mgcccs_solve: 0 = stand-alone MG-CCCS
                            iteration; m in 1..60 = GMRES(m) right-preconditioned by
                            one MG-CCCS iteration per Arnoldi step (Sec. 6) */
  int precision;         /* 0: complex128 throughout.  1 (needs krylov_restart >= 1):
                            iterative refinement with the residual and solution in
                            FP64 around complex64 GMRES(m) cycles whose MG-CCCS
                            preconditioner smooths, restricts, interpolates and
                            projects in complex64; the bound states, channel solves,
                            coarsest solve and Hessenberg stay FP64 */
  double inner_rtol;     /* precision 1: relative residual reduction asked of each
                            complex64 cycle (0 selects 1e-5) */
} mgcccs_params;

/* Bytes of device workspace needed for `p` (0 when p is invalid). */
size_t mgcccs_workspace_size(const mgcccs_params* p);

/*
 * Build the solver: ECS node coordinates and 5-point coefficients on every
 * level (Eq. (11)), the diagonal and omega/diagonal arrays, the dense inverse
 * of the coarsest operator (or, for a coarsest grid of more than 1024 nodes, the
 * factors of its block cyclic reduction), the n_b bound states of H1 and H2 (Eq. (9)) with
 * bilinear normalisation int phi^2 dz = 1 (Sec. 3.1, Remark 3) and two
 * shift-and-invert refinement steps (Sec. 5.1.2), the channel potentials
 * V^A, V^B (Sec. 4.2) and the factorised coupled-channel systems
 * (Eqs. (28)-(29)).  All of it runs in device kernels.
 *
 *   out        receives the handle (host memory owned by the library until
 *              mgcccs_destroy)
 *   v1, v2     device, nx-1 and ny-1 values of V1, V2 at the interior nodes of
 *              the ECS contour
 *   v12        device, (ny-1)*(nx-1) values of V12 at the interior nodes, [j][i]
 *   workspace  device, >= mgcccs_workspace_size(p) bytes, 256-byte aligned,
 *              caller-owned, must stay allocated and untouched until destroy
 *   stream     cudaStream_t (as void*) for all work of this handle
 * The potentials are copied; they may be freed after this call returns.
 * Synchronous.  Errors: EINVAL, ENOSPACE, ECUDA, EBREAKDOWN.
 */
int mgcccs_setup(mgcccs_t* out, const mgcccs_params* p,
                 const mgcccs_c128* v1, const mgcccs_c128* v2, const mgcccs_c128* v12,
                 void* workspace, size_t workspace_bytes, void* stream);

/* mgcccs_setup with the bound states supplied instead of computed: lambda, mu are
 * host arrays of n_b eigenvalues, phi, vphi device arrays [n_b][nx-1], [n_b][ny-1]
 * as returned by mgcccs_get_bound_states of a handle with the same grid, ECS
 * contour, V1 and V2 (the states do not depend on E or V12).  Lets energy sweeps and
 * batches skip the eigen-solve.  Same conventions and errors as mgcccs_setup. */
int mgcccs_setup_with_states(mgcccs_t* out, const mgcccs_params* p,
                             const mgcccs_c128* v1, const mgcccs_c128* v2, const mgcccs_c128* v12,
                             const mgcccs_c128* lambda, const mgcccs_c128* phi,
                             const mgcccs_c128* mu, const mgcccs_c128* vphi,
                             void* workspace, size_t workspace_bytes, void* stream);

/* One V(nu1,nu2)-cycle on the fine level, u updated in place (Sec. 3.2).
 * u, f: device, (nx-1)*(ny-1).  Async. */
int mgcccs_vcycle(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f);

/* One Coupled Channel Correction Step, u updated in place (Sec. 4.3, Eq. (30)):
 * residual r = f - (H-E)u, projections onto the bound states with the
 * conventions of Eqs. (25)-(27), the coupled-channel solves of Eqs. (28)-(29)
 * for the error, and u += sum_m e^A_m(y) phi_m(x) + sum_l e^B_l(x) vphi_l(y).
 * Requires n_b > 0.  Async. */
int mgcccs_cccs(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f);

/* Solve (H-E)u = f from the given u until ||f - (H-E)u||_2 / ||f||_2 <= rtol
 * (Table 1 uses a relative-residual stop) or max_iter iterations.  With
 * krylov_restart = 0 an iteration is one MG-CCCS iteration (V-cycle then CCCS,
 * Sec. 6); with krylov_restart = m > 0 it is one Arnoldi step of restarted
 * GMRES(m) whose right preconditioner is one MG-CCCS iteration from zero (the
 * paper's MG-CCCS-preconditioned Krylov solver, Sec. 6); the true residual is
 * recomputed at every restart and at exit.  u: device in/out (start from zeros
 * for a cold solve); f: device.  iters, relres: host, may be NULL (relres is
 * the true relative residual at exit); history: host array of max_iter
 * doubles receiving the relative residual (GMRES: its least-squares estimate)
 * after each iteration, may be NULL.  Synchronous.  Returns ENOTCONV when
 * max_iter is reached (u, relres valid), ENONFINITE if the residual is not
 * finite, EDIVERGED when the true relative residual (after each stand-alone
 * iteration, at each GMRES restart) exceeds 1e6 times its smallest value so far.
 * GMRES solves without history run device-driven by default: the whole solve is
 * one CUDA graph whose conditional nodes (while / if / switch) carry the restart
 * loop, the Arnoldi loop and the stop tests, so the host launches it once and
 * waits once.  The graph is built on the first call for a given (u, f) pair of
 * pointers and replayed while they stay the same.  With history, or after
 * mgcccs_set_solve_driver(h, MGCCCS_DRIVER_HOST), the host drives the cycles
 * (one replayed graph per Arnoldi step; the same arithmetic in the same order). */
int mgcccs_solve(mgcccs_t h, mgcccs_c128* u, const mgcccs_c128* f, double rtol,
                 int max_iter, int* iters, double* relres, double* history);

/* Same as mgcccs_solve with HOST u and f: copies f (and the initial u) to the
 * device, solves, copies u back.  Uses device buffers inside the workspace.
 * Synchronous. */
int mgcccs_solve_host(mgcccs_t h, mgcccs_c128* u_host, const mgcccs_c128* f_host,
                      double rtol, int max_iter, int* iters, double* relres);

/* All eigenvalues of the fine-grid 1D Hamiltonian H1 = -1/2 d^2/dz^2 + V of one axis
 * (axis 0: x with V1, axis 1: y with V2) on the ECS grid, the matrix whose n_b
 * smallest-real-part eigenpairs are the bound states (Eq. (9), Sec. 4.1).
 * method 0: Ehrlich-Aberth simultaneous iteration with divide-and-conquer starting
 * values (what setup uses); method 1: the one-thread FP64 root-free QR (setup's
 * fallback; its rotations are complex-orthogonal, not unitary, and on this
 * non-Hermitian matrix part of its large-modulus spectrum is inaccurate, while the
 * smallest-real-part eigenvalues that setup takes from it are right).  lam_host: host
 * array of (n-1) entries, unordered.  Synchronous.
 * EBREAKDOWN if the chosen method did not converge. */
int mgcccs_axis_spectrum(mgcccs_t h, int axis, int method, mgcccs_c128* lam_host);
/* Number of axes whose bound-state eigenvalues needed the QR fallback in the last
 * setup of h (0 normally), or -1 for a NULL handle. */
int mgcccs_eig_fallbacks(mgcccs_t h);

/* Solve drivers for mgcccs_set_solve_driver. */
enum { MGCCCS_DRIVER_GRAPH = 0, MGCCCS_DRIVER_HOST = 1 };
int mgcccs_set_solve_driver(mgcccs_t h, int driver);

/* Block height (2, 4 or 8 rows; 0 = the default 2) of the smoothing, residual, transfer
 * and operator passes on the levels of h that are too small to fill the GPU with 32 x 8
 * blocks; a tuning knob for the batch autotuner (the results do not depend on it).
 * Waits for h's stream, then drops h's cached solve graphs (they hold the old launch
 * shapes); batch graphs built earlier keep the shapes they were built with.  EINVAL for
 * another value. */
int mgcccs_set_tile_rows(mgcccs_t h, int rows);

/* Batched device-driven solves: one CUDA graph holding the device-driven solves of
 * `count` problems (one handle each, krylov_restart >= 1, any mix of grids, energies
 * and precisions) as independent branches, so that one launch runs them all
 * concurrently.  u[k], f[k]: device arrays of problem k, fixed for the life of the
 * batch (the graph holds the pointers).  stream: the stream that run() launches on.
 * The batch uses the handles' buffers: run no other call on its handles while a
 * batch runs, and destroy the batch before its handles.  EINVAL for a handle listed
 * twice, a handle without GMRES, or NULL pointers; ECUDA if the graph cannot be
 * built. */
int mgcccs_batch_create(mgcccs_batch_t* out, mgcccs_t* handles, int count, mgcccs_c128* const* u,
                        const mgcccs_c128* const* f, void* stream);
/* One launch of the batch graph: every problem from its current u until
 * ||f - (H-E)u|| / ||f|| <= rtol or max_iter Arnoldi steps.  iters, relres, status:
 * host arrays of count entries, may be NULL (status[k]: OK, ENOTCONV, ENONFINITE or EDIVERGED).
 * Synchronous.  Returns the worst status. */
int mgcccs_batch_run(mgcccs_batch_t b, double rtol, int max_iter, int* iters, double* relres, int* status);
void mgcccs_batch_destroy(mgcccs_batch_t b);

/* Batched solve of `count` independent problems, one handle each (handles with
 * krylov_restart >= 1, any mix of grids, energies and precisions; give every handle
 * its own stream at setup so that their work overlaps).  GMRES cycles of all unfinished
 * problems advance in lock-step: each cycle starts from the true residual, then the
 * Arnoldi steps of all problems are launched round-robin (each a replayed CUDA graph on
 * its handle's stream), and each problem keeps the first step whose residual estimate
 * met its target.  A problem leaves the batch when ||f - (H-E)u|| / ||f|| <= rtol or
 * after max_iter used steps.  u[k], f[k]: device arrays of problem k (u in/out).
 * iters, relres, status: host arrays of count entries, may be NULL (status[k] is
 * MGCCCS_OK, ENOTCONV, ENONFINITE or EDIVERGED).  Synchronous.  Returns the worst status, or
 * EINVAL (a handle listed twice, a handle without GMRES, NULL pointers). */
int mgcccs_batch_solve(mgcccs_t* handles, int count, mgcccs_c128* const* u, const mgcccs_c128* const* f,
                       double rtol, int max_iter, int* iters, double* relres, int* status);

/* Preconditioner application z = M^{-1} r (Sec. 6: one V-cycle, then the
 * CCCS when n_b > 0, from a zero initial guess).  z, r: device, distinct.
 * With precision 1 the complex64 preconditioner is applied to r rounded to
 * complex64 and z is its exact widening.  Async. */
int mgcccs_precond_apply(mgcccs_t h, mgcccs_c128* z, const mgcccs_c128* r);

/* y = (H-E)x on the fine level (Eq. (11)); x, y: device, distinct.  Async. */
int mgcccs_matvec(mgcccs_t h, const mgcccs_c128* x, mgcccs_c128* y);

/* r = f - (H-E)u on the fine level (Eq. (11)); if norm2 is not NULL the
 * host receives ||r||_2^2 (then synchronous, else async).  u, f, r: device;
 * r may not alias u. */
int mgcccs_residual(mgcccs_t h, const mgcccs_c128* u, const mgcccs_c128* f,
                    mgcccs_c128* r, double* norm2);

/* ---- amplitude functional and adjoint gradients ----------------------------
 * With w_k = w_x(i) w_y(j) the fine-level quadrature weights (h_{i-1}+h_i)/2 of the
 * ECS contour (the weights of the bilinear normalisation, Sec. 3.1), the amplitude
 * J = <g|u> = sum_k w_k g_k u_k is bilinear (no conjugation).  W(H-E) is complex
 * symmetric (Sec. 2.5), so the adjoint of (H-E)u = f for J is the forward problem
 * (H-E) mu = g (solve it with mgcccs_solve), and for any parameter p of H - E,
 * dJ/dp = -sum_k w_k mu_k ((d(H-E)/dp) u)_k.  The two entry points below form these
 * sums and products; a, b, d, out are device arrays of (nx-1)*(ny-1) values (out of
 * mgcccs_weighted_dot is one device value).  Async. */

/* *out = scale * sum_k w_k a_k b_k d_k  (d may be NULL: d_k = 1).  Deterministic order. */
int mgcccs_weighted_dot(mgcccs_t h, const mgcccs_c128* a, const mgcccs_c128* b, const mgcccs_c128* d,
                        mgcccs_c128 scale, mgcccs_c128* out);
/* out_k = scale * w_k a_k b_k  (e.g. dJ/d(dV_k) = -w_k mu_k u_k with scale = -1). */
int mgcccs_weighted_product(mgcccs_t h, const mgcccs_c128* a, const mgcccs_c128* b, mgcccs_c128 scale,
                            mgcccs_c128* out);

/* ---- single steps of the V-cycle, for component checks (Sec. 3.2) ---------
 * `level` counts from 0 (fine).  Arrays are device, interior-sized for the
 * level they live on.  All async. */

/* `sweeps` omega-Jacobi sweeps u <- u + omega D^{-1}(f - (H-E)u) on `level`. */
int mgcccs_smooth(mgcccs_t h, int level, mgcccs_c128* u, const mgcccs_c128* f, int sweeps);
/* r = f - (H-E)u on `level`. */
int mgcccs_level_residual(mgcccs_t h, int level, const mgcccs_c128* u,
                          const mgcccs_c128* f, mgcccs_c128* r);
/* Full weighting of r (on `level`) onto rc (on level+1). */
int mgcccs_restrict(mgcccs_t h, int level, const mgcccs_c128* r, mgcccs_c128* rc);
/* u (on `level`) += bilinear interpolation of ec (on level+1). */
int mgcccs_prolong_add(mgcccs_t h, int level, const mgcccs_c128* ec, mgcccs_c128* u);
/* Direct solve of the coarsest-level system: u = A_c^{-1} f. */
int mgcccs_coarse_solve(mgcccs_t h, const mgcccs_c128* f, mgcccs_c128* u);

/* Bound states found by setup (Eq. (9)).  lambda, mu: host arrays of n_b;
 * phi: device (nx-1)*n_b, vphi: device (ny-1)*n_b, column-major per state
 * (phi[k*(nx-1) + i]).  Any pointer may be NULL.  Synchronous. */
int mgcccs_get_bound_states(mgcccs_t h, mgcccs_c128* lambda, mgcccs_c128* phi,
                            mgcccs_c128* mu, mgcccs_c128* vphi);

/* ---- allocation-free helper (the paper has no counterpart) -----------------
 * Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being
 * captured in the global capture mode (allocation calls are illegal there), code
 * inside a framework whose caching allocator owns all device memory under a hard
 * cap, and latency-critical loops that must avoid the device synchronisation an
 * allocation can trigger.  mgcccs_norm2_noalloc needs neither a handle nor a
 * workspace: it writes sum_k |v_k|^2 (the squared 2-norm used for relative
 * residuals) of the device complex128 vector v[0..n) to the device double
 * *norm2, on `stream` (cudaStream_t as void*; NULL = legacy default stream),
 * asynchronously.  Its scratch is a file-scope device array of
 * MGCCCS_NOALLOC_MAX_N / 2048 doubles (32 KiB) that every GPU which loads the
 * library keeps until the process exits.  The first call on a device looks up
 * that array's device address (with that device current); make that first call
 * before any stream capture.  All calls share the one array and each call
 * overwrites the slots it uses, so calls that overlap on the GPU (on different
 * streams, or from several host threads) race and give wrong sums.
 * n = 0 writes 0 (v may then be NULL).  Returns MGCCCS_EINVAL for a NULL norm2, a
 * NULL v with n > 0, or n > MGCCCS_NOALLOC_MAX_N (nothing is launched), MGCCCS_ECUDA
 * if the address lookup or a launch fails. */
#define MGCCCS_NOALLOC_MAX_N 8388608
int mgcccs_norm2_noalloc(const mgcccs_c128* v, size_t n, double* norm2, void* stream);

/* ---- FP64 throughput probe (a measurement utility; the paper has no counterpart) ----
 * The complex128 kernels are bound by the FP64 pipe.  mgcccs_fp64_probe launches
 * `blocks` blocks of 256 threads on `stream` (cudaStream_t as void*; NULL = legacy
 * default stream), each thread running MGCCCS_PROBE_CHAINS independent recurrences
 * a <- fma(a, m, b) for `iters` rounds, and writes one sum per block to the device
 * array out[0..blocks).  FP64 lane operations executed:
 * blocks * 256 * iters * MGCCCS_PROBE_CHAINS (2 flops each); the caller times the
 * launch (asynchronous) with events on `stream`.  Returns MGCCCS_EINVAL for
 * blocks < 1, iters < 1 or a NULL out (nothing is launched), MGCCCS_ECUDA if the
 * launch fails. */
#define MGCCCS_PROBE_CHAINS 8
int mgcccs_fp64_probe(int blocks, int iters, double m, double b, double* out, void* stream);

/*
 * The two halves of one classical Gram-Schmidt pass of the Arnoldi process of the
 * GMRES(m) solver that MG-CCCS preconditions (Sec. 6), exposed for component tests and
 * for timing the kernels the solve spends most of its time in:
 *
 *   mgcccs_gs_dots:   out[i] = sum_p conj(V_i[p]) w[p]            for i < k
 *   mgcccs_gs_update: w[p]  -= sum_{i<k} coef[i] V_i[p]          (every p)
 *
 * V: device, k vectors of (nx-1)*(ny-1) values, vector i at V + i*ld (ld >= (nx-1)*(ny-1));
 * w: device, (nx-1)*(ny-1) values (gs_update overwrites it); out, coef: device, k values.
 * A vector V_i that is w itself (same address) gives out[i] = |w|^2.  The sums are FP64
 * in a fixed order (per-block partials, then one block), so repeated calls give identical
 * results.  mgcccs_gs_dots needs a handle set up with krylov_restart >= 1 and
 * k <= krylov_restart + 1 (it uses the handle's partial-sum buffer); mgcccs_gs_update
 * takes 1 <= k <= 61.  Async.  Errors: EINVAL (null pointer, k or ld out of range), ECUDA.
 */
int mgcccs_gs_dots(mgcccs_t h, const mgcccs_c128* V, long long ld, int k, const mgcccs_c128* w,
                   mgcccs_c128* out);
int mgcccs_gs_update(mgcccs_t h, const mgcccs_c128* V, long long ld, int k, const mgcccs_c128* coef,
                     mgcccs_c128* w);
/* The same two halves on complex64 vectors, the kernels the mixed form (precision 1) runs
 * in its complex64 GMRES cycles: V and w complex64 (mgcccs_c64), out and coef complex128;
 * products accumulate in FP32 within a warp and in FP64 beyond.  With a 16-byte aligned V
 * and w and an even ld, gs_update reads and writes entry pairs as 16-byte accesses.  Same
 * contract and errors as above; mgcccs_gs_dots_c64 needs krylov_restart >= 1. */
int mgcccs_gs_dots_c64(mgcccs_t h, const mgcccs_c64* V, long long ld, int k, const mgcccs_c64* w,
                       mgcccs_c128* out);
int mgcccs_gs_update_c64(mgcccs_t h, const mgcccs_c64* V, long long ld, int k, const mgcccs_c128* coef,
                         mgcccs_c64* w);

/* Number of kernel launches issued since setup (for launch accounting). */
long long mgcccs_launch_count(mgcccs_t h);

const char* mgcccs_strerror(int code);

/* Release the handle (host memory and CUDA objects; not the workspace). */
void mgcccs_destroy(mgcccs_t h);

#ifdef __cplusplus
}
#endif

#endif /* MGCCCS_H */
