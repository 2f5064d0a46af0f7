"""CPU oracle for MG-CCCS (Cools & Vanroose, arXiv:1412.1953) -- TEST INFRASTRUCTURE ONLY.

Only tests, the package's smoke check and the benchmark's CPU-baseline leg may
import this module.  The product (the CUDA library and its Python binding)
never calls it; it shares no code, constants or helpers with the CUDA path.

Plain, slow, obviously-correct complex128 NumPy/SciPy restatement of the
method, in the paper's order:

* Discretisation (Sec. 2.5, Eq. (11)): second-order finite differences of
  -1/2 Laplacian + V - E on a uniform grid whose nodes are bent into the
  complex plane beyond R0 (exterior complex scaling), Dirichlet zero on the
  boundary ring.  Nonuniform complex spacings h_i = z_{i+1} - z_i.
* Multigrid V(nu1, nu2)-cycle with omega-Jacobi smoothing, full-weighting
  restriction and bilinear interpolation (Sec. 3.2); coarse levels are the same
  discretisation on the coarser grid of the same box and contour; the coarsest
  level is solved directly.
* 1D bound states of Eq. (9) with the bilinear normalisation int phi^2 dz = 1
  (Sec. 3.1 Remark 3, footnote of Sec. 4.2) and two shift-and-invert refinement
  steps (Sec. 5.1.2, Sec. 5.2).
* Coupled Channel Correction Step (Sec. 4.1-4.3): projections Eq. (27) with the
  uniqueness conventions Eqs. (25)-(26), channel equations Eqs. (28)-(29) for
  the error, correction Eq. (30).
* MG-CCCS iteration: one V-cycle then one CCCS (Sec. 6.1), relative residual
  stop (Table 1).

Readings of points where the paper is silent (each one is listed in the design
notes of the repository):
  R1  n = number of cells per axis, interior (n-1)^2, h = L/n.
  R2  the ECS start R0 need not be a node; the straddling cell simply gets
      h = z_{i+1} - z_i.
  R3  V is evaluated at complex nodes; V12 = 1/z(max(x, y)).
  R4  the V-cycle works on the unweighted residual; FW and bilinear are the
      index-space stencils, also inside the ECS layer; the coarse initial guess is 0.
  R5  coarse operators re-discretise on n/2^l cells of the same box; the coarse
      levels (l >= 1) lie on a complex contour: the fine ECS contour rotated as a
      whole by gamma (default 14.6 degrees, the rotation of Sec. 3.2), the
      fine level keeps the ECS contour itself.  Potentials are injected at the
      coincident (even) nodes; the coarsest level is solved by dense LU.
  R6  the n_b bound states are the eigenpairs of H1 with smallest Re(lambda);
      sign fixed so that Re(phi) > 0 at argmax |phi|; lambda is updated by the
      bilinear Rayleigh quotient after the shift-and-invert steps.
  R7  all quadratures use the complex trapezoid weights w_i = (h_{i-1} + h_i)/2.
  R8  the channel equations include V^A_ii inside the coupling sum; the typos
      "V^B_jl(y)", "f^B_j(y)" in Eq. (29) are read as functions of x.
  R9  relres = ||f - (H-E)u||_2 / ||f||_2 over the interior, after the CCCS, u_0 = 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg


# --------------------------------------------------------------------------------------
# Grid and operator (Sec. 2.5, Eq. (7), Eq. (11))
# --------------------------------------------------------------------------------------

def ecs_nodes(n: int, L: float, R0: float, theta: float) -> np.ndarray:
    """Complex node coordinates z_0..z_n of an n-cell grid on [0, L] with ECS beyond R0."""
    z = np.empty(n + 1, dtype=np.complex128)
    for i in range(n + 1):
        x = i * L / n
        z[i] = x if x <= R0 else R0 + (x - R0) * np.exp(1j * theta)
    return z


@dataclasses.dataclass
class Axis:
    """Second-difference coefficients along one axis, interior nodes 1..n-1.

    -1/2 d^2u/dz^2 at node i is  west*u_{i-1} + diag*u_i + east*u_{i+1}  with
    west = -1/((h_{i-1}+h_i) h_{i-1}),  east = -1/((h_{i-1}+h_i) h_i),
    diag = -(west + east)  (the 3-point nonuniform formula, exact for quadratics).
    """
    n: int
    z: np.ndarray
    h: np.ndarray        # n cell widths (complex)
    w: np.ndarray        # n-1 quadrature weights (h_{i-1} + h_i)/2
    west: np.ndarray
    east: np.ndarray
    diag: np.ndarray


def make_axis(n: int, L: float, R0: float, theta: float, gamma: float = 0.0) -> Axis:
    z = ecs_nodes(n, L, R0, theta)
    if gamma:
        z = z * np.exp(1j * gamma)          # full complex contour (coarse-level option)
    h = z[1:] - z[:-1]
    hm, hp = h[:-1], h[1:]                  # h_{i-1}, h_i for i = 1..n-1
    west = -1.0 / ((hm + hp) * hm)
    east = -1.0 / ((hm + hp) * hp)
    diag = -(west + east)
    return Axis(n, z, h, 0.5 * (hm + hp), west, east, diag)


@dataclasses.dataclass
class Level:
    ax: Axis             # x axis
    ay: Axis             # y axis
    v1: np.ndarray
    v2: np.ndarray
    v12: np.ndarray      # [j][i]
    E: float

    @property
    def shape(self):
        return (self.ay.n - 1, self.ax.n - 1)

    def diagonal(self) -> np.ndarray:
        """Full diagonal D_ij of (H - E), including potential and energy."""
        return (self.ax.diag[None, :] + self.ay.diag[:, None] + self.v1[None, :]
                + self.v2[:, None] + self.v12 - self.E)


def apply_operator(lev: Level, u: np.ndarray) -> np.ndarray:
    """(H - E) u for the unweighted 5-point operator, u = 0 on the boundary ring."""
    up = np.zeros((u.shape[0] + 2, u.shape[1] + 2), dtype=np.complex128)
    up[1:-1, 1:-1] = u
    out = lev.diagonal() * u
    out += lev.ax.west[None, :] * up[1:-1, :-2] + lev.ax.east[None, :] * up[1:-1, 2:]
    out += lev.ay.west[:, None] * up[:-2, 1:-1] + lev.ay.east[:, None] * up[2:, 1:-1]
    return out


def residual(lev: Level, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    return f - apply_operator(lev, u)


def tridiag_1d(ax: Axis, v: np.ndarray) -> scipy.sparse.csr_matrix:
    """Unweighted 1D Hamiltonian -1/2 d^2/dz^2 + V on the interior nodes."""
    return scipy.sparse.diags([ax.west[1:], ax.diag + v, ax.east[:-1]], [-1, 0, 1], format="csr")


def assemble_unweighted(lev: Level) -> scipy.sparse.csr_matrix:
    """Sparse (H - E) in the [j][i] (x fastest) ordering; unknown index j*(nx-1)+i."""
    Hx = tridiag_1d(lev.ax, np.zeros_like(lev.v1))
    Hy = tridiag_1d(lev.ay, np.zeros_like(lev.v2))
    Ix = scipy.sparse.identity(lev.ax.n - 1, format="csr")
    Iy = scipy.sparse.identity(lev.ay.n - 1, format="csr")
    V = (lev.v1[None, :] + lev.v2[:, None] + lev.v12 - lev.E).ravel()
    return (scipy.sparse.kron(Iy, Hx) + scipy.sparse.kron(Hy, Ix) + scipy.sparse.diags(V)).tocsr()


def weights_2d(lev: Level) -> np.ndarray:
    return (lev.ay.w[:, None] * lev.ax.w[None, :]).ravel()


def assemble_weighted(lev: Level) -> scipy.sparse.csr_matrix:
    """Complex-symmetric form A = W (H - E), W = diag(w_i w_j) (Sec. 2.5: A = A^T)."""
    return (scipy.sparse.diags(weights_2d(lev)) @ assemble_unweighted(lev)).tocsr()


# --------------------------------------------------------------------------------------
# Multigrid components (Sec. 3.2: V(1,1)-cycles, omega-Jacobi, FW, bilinear)
# --------------------------------------------------------------------------------------

def jacobi(lev: Level, u: np.ndarray, f: np.ndarray, omega: float, sweeps: int) -> np.ndarray:
    """omega-Jacobi: u <- u + omega D^{-1} (f - (H-E)u), simultaneous update."""
    D = lev.diagonal()
    for _ in range(sweeps):
        u = u + omega * residual(lev, u, f) / D
    return u


def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full weighting 1/16 [1 2 1; 2 4 2; 1 2 1] onto the coincident (even) fine nodes.

    Fine interior (2m-1)^2 -> coarse interior (m-1)^2; coarse node I sits on fine node 2I.
    The padded array index equals the node index, with zeros on the boundary ring.
    """
    ny, nx = r.shape
    rp = np.zeros((ny + 2, nx + 2), dtype=np.complex128)
    rp[1:-1, 1:-1] = r
    my, mx = (ny + 1) // 2, (nx + 1) // 2          # coarse cell counts
    J = slice(2, 2 * my - 1, 2)                     # fine rows 2J,   J = 1..my-1
    Jm = slice(1, 2 * my - 2, 2)                    # fine rows 2J-1
    Jp = slice(3, 2 * my, 2)                        # fine rows 2J+1
    I = slice(2, 2 * mx - 1, 2)
    Im = slice(1, 2 * mx - 2, 2)
    Ip = slice(3, 2 * mx, 2)
    return (4 * rp[J, I]
            + 2 * (rp[J, Im] + rp[J, Ip] + rp[Jm, I] + rp[Jp, I])
            + rp[Jm, Im] + rp[Jm, Ip] + rp[Jp, Im] + rp[Jp, Ip]) / 16.0


def prolong_bilinear(e: np.ndarray, fine_shape) -> np.ndarray:
    """Bilinear interpolation from coarse interior to fine interior, zero boundary values.

    Coincident nodes copy, edge midpoints average two coarse neighbours, cell
    centres average four.
    """
    ny, nx = fine_shape
    my, mx = (ny + 1) // 2, (nx + 1) // 2
    ep = np.zeros((my + 1, mx + 1), dtype=np.complex128)    # coarse nodes 0..m
    ep[1:-1, 1:-1] = e
    out = np.zeros((ny + 2, nx + 2), dtype=np.complex128)  # fine nodes 0..n
    out[0::2, 0::2] = ep
    out[0::2, 1::2] = 0.5 * (ep[:, :-1] + ep[:, 1:])
    out[1::2, 0::2] = 0.5 * (ep[:-1, :] + ep[1:, :])
    out[1::2, 1::2] = 0.25 * (ep[:-1, :-1] + ep[:-1, 1:] + ep[1:, :-1] + ep[1:, 1:])
    return out[1:-1, 1:-1]


COARSE_GAMMA_DEFAULT = 14.6 * math.pi / 180.0


@dataclasses.dataclass
class Params:
    nx: int
    ny: int
    Lx: float
    Ly: float
    R0x: float
    R0y: float
    theta: float
    E: float
    levels: int = 5
    nu1: int = 1
    nu2: int = 1
    omega: float = 2.0 / 3.0
    n_b: int = 3
    coarse_gamma: float = COARSE_GAMMA_DEFAULT   # rotation of the coarse-level contour (R5)


def build_levels(p: Params, v1, v2, v12) -> list[Level]:
    """Level 0 is the fine grid; level l has n/2^l cells; potentials injected at even nodes."""
    levels = []
    for l in range(p.levels):
        mx, my = p.nx >> l, p.ny >> l
        if (mx << l) != p.nx or (my << l) != p.ny or mx < 2 or my < 2:
            raise ValueError("grid not coarsenable to the requested depth")
        s = 1 << l
        g = p.coarse_gamma if l > 0 else 0.0
        ax = make_axis(mx, p.Lx, p.R0x, p.theta, g)
        ay = make_axis(my, p.Ly, p.R0y, p.theta, g)
        levels.append(Level(ax, ay, v1[s - 1::s].copy(), v2[s - 1::s].copy(),
                            v12[s - 1::s, s - 1::s].copy(), p.E))
    return levels


def coarsest_solve(lev: Level, f: np.ndarray) -> np.ndarray:
    """The exact coarsest-level solve of the V-cycle (Sec. 3.2): dense LU with partial
    pivoting of the coarsest operator, factorised on first use and kept on the level (a
    level's operator never changes), then a forward and a back substitution per call."""
    lu = lev.__dict__.get("_dense_lu")
    if lu is None:
        lu = scipy.linalg.lu_factor(assemble_unweighted(lev).toarray())
        lev.__dict__["_dense_lu"] = lu
    return scipy.linalg.lu_solve(lu, f.ravel()).reshape(f.shape)


def vcycle(levels: list[Level], p: Params, u: np.ndarray, f: np.ndarray, l: int = 0) -> np.ndarray:
    """One V(nu1, nu2)-cycle on level l: pre-smooth, residual, restrict, recurse,
    interpolate and add, post-smooth.  The coarsest level is solved exactly."""
    lev = levels[l]
    if l == len(levels) - 1:
        return coarsest_solve(lev, f)
    u = jacobi(lev, u, f, p.omega, p.nu1)
    rc = restrict_fw(residual(lev, u, f))
    ec = vcycle(levels, p, np.zeros_like(rc), rc, l + 1)
    u = u + prolong_bilinear(ec, u.shape)
    u = jacobi(lev, u, f, p.omega, p.nu2)
    return u


# --------------------------------------------------------------------------------------
# Bound states (Eq. (9); normalisation Sec. 3.1; shift-and-invert Sec. 5.1.2)
# --------------------------------------------------------------------------------------

def bound_states(ax: Axis, v: np.ndarray, n_b: int, refine_steps: int = 2):
    """n_b eigenpairs of H1 = -1/2 d^2/dz^2 + V with the smallest real part.

    Dense eigen-solve, bilinear normalisation phi^T W phi = 1 (no conjugation),
    then `refine_steps` shift-and-invert steps phi <- (H1 - lambda)^{-1} phi,
    renormalised, and the bilinear Rayleigh quotient for lambda.
    """
    H = tridiag_1d(ax, v).toarray()
    evals, evecs = np.linalg.eig(H)
    order = np.argsort(evals.real, kind="stable")[:n_b]
    lam = evals[order].astype(np.complex128)
    phi = evecs[:, order].astype(np.complex128)
    w = ax.w
    m = H.shape[0]
    # banded storage of H for the shift-and-invert solves
    for k in range(n_b):
        v_k = _normalise(phi[:, k], w)
        for _ in range(refine_steps):
            ab = np.zeros((3, m), dtype=np.complex128)
            ab[0, 1:] = ax.east[:-1]
            ab[1, :] = ax.diag + v - lam[k]
            ab[2, :-1] = ax.west[1:]
            v_k = _normalise(scipy.linalg.solve_banded((1, 1), ab, v_k), w)
            lam[k] = v_k @ (w * (H @ v_k))
        phi[:, k] = v_k
    return lam, phi


def _normalise(v: np.ndarray, w: np.ndarray) -> np.ndarray:
    v = v / np.sqrt(np.sum(w * v * v))
    k = int(np.argmax(np.abs(v)))
    return -v if v[k].real < 0 else v


# --------------------------------------------------------------------------------------
# Coupled Channel Correction Step (Sec. 4)
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Channels:
    lam: np.ndarray      # (n_b,) eigenvalues of H1 (x)
    phi: np.ndarray      # (nx-1, n_b)
    mu: np.ndarray       # (n_b,) eigenvalues of H2 (y)
    vphi: np.ndarray     # (ny-1, n_b)
    VA: np.ndarray       # (ny-1, n_b, n_b):  V^A_im(y_j) = sum_x w phi_i phi_m V12
    VB: np.ndarray       # (nx-1, n_b, n_b):  V^B_jl(x_i) = sum_y w vphi_j vphi_l V12


def setup_channels(lev: Level, n_b: int) -> Channels:
    lam, phi = bound_states(lev.ax, lev.v1, n_b)
    mu, vphi = bound_states(lev.ay, lev.v2, n_b)
    wx, wy = lev.ax.w, lev.ay.w
    VA = np.einsum("i,ia,ib,ji->jab", wx, phi, phi, lev.v12)
    VB = np.einsum("j,ja,jb,ji->iab", wy, vphi, vphi, lev.v12)
    return Channels(lam, phi, mu, vphi, VA, VB)


def channel_matrix_banded(axis: Axis, v: np.ndarray, eig: np.ndarray, Vc: np.ndarray, E: float):
    """Banded storage (l = u = n_b) of the coupled-channel system Eq. (28)/(29) in the
    interleaved ordering k = node*n_b + channel:
      west e(node-1) + [(diag + v - E) I + diag(eig) + Vc(node)] e(node) + east e(node+1)."""
    m, nb = axis.n - 1, len(eig)
    N = m * nb
    full_band = 2 * nb + 1
    ab = np.zeros((full_band, N), dtype=np.complex128)
    # ab[nb + r - c, c] = M[r, c]
    for node in range(m):
        for a in range(nb):
            r = node * nb + a
            for b in range(nb):
                c = node * nb + b
                val = Vc[node, a, b]
                if a == b:
                    val = val + axis.diag[node] + v[node] - E + eig[a]
                ab[nb + r - c, c] += val
            if node > 0:
                c = (node - 1) * nb + a
                ab[nb + r - c, c] += axis.west[node]
            if node < m - 1:
                c = (node + 1) * nb + a
                ab[nb + r - c, c] += axis.east[node]
    return ab


def cccs_rhs(lev: Level, ch: Channels, r: np.ndarray):
    """Split the residual into channel right-hand sides r^A_i(y), r^B_j(x).

    P^x_i(y) = int r phi_i dx,  P^y_j(x) = int r vphi_j dy,  c_ij = a_ji + b_ij (Eq. (27));
    conventions Eq. (25)-(26): a_ji = c_ij for j <= i, b_ij = c_ij for j > i;
    r^A_i = P^x_i - sum_l b_il vphi_l,  r^B_j = P^y_j - sum_m a_jm phi_m  (Sec. 4.1).
    """
    wx, wy = lev.ax.w, lev.ay.w
    nb = ch.phi.shape[1]
    Px = np.einsum("i,ia,ji->aj", wx, ch.phi, r)          # (n_b, ny-1)
    Py = np.einsum("j,jb,ji->bi", wy, ch.vphi, r)         # (n_b, nx-1)
    c = np.einsum("j,jb,aj->ab", wy, ch.vphi, Px)         # c[i, j] = int int phi_i vphi_j r
    rA = Px.copy()
    rB = Py.copy()
    for i in range(nb):
        for l in range(nb):
            if l > i:                                     # b_il = c_il
                rA[i] -= c[i, l] * ch.vphi[:, l]
    for j in range(nb):
        for m in range(nb):
            if m >= j:                                    # a_jm = c_mj
                rB[j] -= c[m, j] * ch.phi[:, m]
    return Px, Py, c, rA, rB


def solve_channels(lev: Level, ch: Channels, rA: np.ndarray, rB: np.ndarray):
    nb = ch.phi.shape[1]
    abA = channel_matrix_banded(lev.ay, lev.v2, ch.lam, ch.VA, lev.E)
    abB = channel_matrix_banded(lev.ax, lev.v1, ch.mu, ch.VB, lev.E)
    eA = scipy.linalg.solve_banded((nb, nb), abA, rA.T.ravel()).reshape(-1, nb).T   # (n_b, ny-1)
    eB = scipy.linalg.solve_banded((nb, nb), abB, rB.T.ravel()).reshape(-1, nb).T   # (n_b, nx-1)
    return eA, eB


def cccs(lev: Level, ch: Channels, u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """One Coupled Channel Correction Step, Eq. (30):
    u* = u + sum_m e^A_m(y) phi_m(x) + sum_l e^B_l(x) vphi_l(y)."""
    r = residual(lev, u, f)
    _, _, _, rA, rB = cccs_rhs(lev, ch, r)
    eA, eB = solve_channels(lev, ch, rA, rB)
    return u + np.einsum("mj,im->ji", eA, ch.phi) + np.einsum("li,jl->ji", eB, ch.vphi)


# --------------------------------------------------------------------------------------
# MG-CCCS solver (Sec. 6)
# --------------------------------------------------------------------------------------

class Solver:
    def __init__(self, p: Params, v1, v2, v12):
        self.p = p
        self.levels = build_levels(p, np.asarray(v1), np.asarray(v2), np.asarray(v12))
        self.ch = setup_channels(self.levels[0], p.n_b) if p.n_b > 0 else None

    def vcycle(self, u, f):
        return vcycle(self.levels, self.p, u, f)

    def cccs(self, u, f):
        return cccs(self.levels[0], self.ch, u, f)

    def iterate(self, u, f):
        u = self.vcycle(u, f)
        if self.ch is not None:
            u = self.cccs(u, f)
        return u

    def precond_apply(self, r):
        """z = M^{-1} r: one V-cycle from zero then one CCCS (Sec. 6)."""
        return self.iterate(np.zeros_like(r), r)

    def relres(self, u, f):
        return np.linalg.norm(residual(self.levels[0], u, f)) / np.linalg.norm(f)

    def solve(self, f, rtol=1e-10, max_iter=100, u0=None):
        u = np.zeros_like(f) if u0 is None else u0.copy()
        hist = []
        for _ in range(max_iter):
            u = self.iterate(u, f)
            hist.append(self.relres(u, f))
            if not np.isfinite(hist[-1]) or hist[-1] <= rtol:
                break
        return u, hist


def params_from_problem(prob, levels=5, n_b=3, nu1=1, nu2=1, omega=2.0 / 3.0,
                        coarse_gamma=COARSE_GAMMA_DEFAULT) -> Params:
    return Params(prob.nx, prob.ny, prob.Lx, prob.Ly, prob.R0x, prob.R0y, prob.theta, prob.E,
                  levels, nu1, nu2, omega, n_b, coarse_gamma)


def direct_solve(lev: Level, f: np.ndarray) -> np.ndarray:
    """Reference direct solution of the fine system by sparse LU of the weighted
    (complex-symmetric) form A = W (H - E): A u = W f (the paper's LU reference, Sec. 3.2)."""
    A = assemble_weighted(lev).tocsc()
    rhs = weights_2d(lev) * f.ravel()
    return scipy.sparse.linalg.splu(A).solve(rhs).reshape(f.shape)


# --------------------------------------------------------------------------------------
# Krylov acceleration: restarted GMRES(m), right-preconditioned by one MG-CCCS iteration
# (Sec. 6: MG-CCCS as a Krylov preconditioner, one V-cycle per application)
# --------------------------------------------------------------------------------------

def gmres(solver: Solver, f: np.ndarray, m: int = 20, rtol: float = 1e-10, max_iter: int = 1000,
          u0: np.ndarray | None = None, precondition: bool = True):
    """Restarted GMRES(m) for (H - E)u = f with right preconditioning z = M^{-1} v.

    Textbook form (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Alg. 9.5):
    Arnoldi with modified Gram-Schmidt on the Hermitian inner product, the small
    least-squares problem min || beta e_1 - H y || solved directly, u += Z y at the end of
    each cycle, true residual recomputed at every restart.  Returns (u, history of the
    estimated relative residual per Arnoldi step, true relative residual at exit).
    """
    lev = solver.levels[0]
    A = lambda v: apply_operator(lev, v)
    Minv = (lambda v: solver.precond_apply(v)) if precondition else (lambda v: v.copy())
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    hist = []
    steps = 0
    while steps < max_iter:
        r = f - A(u)
        beta = np.linalg.norm(r)
        if beta <= rtol * fn or beta == 0.0:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        y = np.zeros(0, dtype=np.complex128)
        for j in range(m):
            Z.append(Minv(V[j]))
            w = A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            steps += 1
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
            est = np.linalg.norm(H[: j + 2, : j + 1] @ y - e1) / fn
            hist.append(est)
            if est <= rtol or H[j + 1, j] == 0.0 or steps >= max_iter:
                break
            V.append(w / H[j + 1, j])
        for k in range(len(y)):
            u = u + y[k] * Z[k]
        if hist and hist[-1] <= rtol:
            if np.linalg.norm(f - A(u)) <= rtol * fn:
                break
    return u, hist, np.linalg.norm(f - A(u)) / fn


# --------------------------------------------------------------------------------------
# Amplitude functional and its adjoint gradients (differentiation form)
# --------------------------------------------------------------------------------------
# J = <g|u> = sum_k w_k g_k u_k (bilinear, quadrature weights of Sec. 3.1's
# normalisation, no conjugation), u solving (H - E)u = f with f held fixed.
# Because W (H - E) is complex symmetric (Sec. 2.5), the adjoint equation
# (H - E)^T lambda = W g is (H - E) mu = g with lambda = W mu, and for a parameter p
#     dJ/dp = - sum_k w_k mu_k ((d(H - E)/dp) u)_k .
# For E: d(H-E)/dE = -I.  For the charge Z in V1 + V2 = -Z/x - Z/y:
# d(H-E)/dZ = diag(-1/x - 1/y).  For a per-node perturbation dV_k of V: e_k e_k^T.

def amplitude(lev: Level, g: np.ndarray, u: np.ndarray) -> complex:
    return complex(np.sum(weights_2d(lev) * g.ravel() * u.ravel()))


def adjoint_gradients(lev: Level, u: np.ndarray, mu: np.ndarray, dAdZ: np.ndarray):
    """(dJ/dE, dJ/dZ, dJ/ddV) from the forward solution u and the adjoint solution mu
    of (H - E) mu = g; dAdZ is the diagonal of d(H - E)/dZ on the interior nodes."""
    wmu_u = weights_2d(lev).reshape(u.shape) * mu * u
    dE = complex(np.sum(wmu_u))
    dZ = complex(-np.sum(wmu_u * dAdZ))
    ddV = -wmu_u
    return dE, dZ, ddV
