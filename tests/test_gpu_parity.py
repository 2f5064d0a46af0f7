"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle, step by step
and end to end, on seeded TP/ECS problems.  Tolerances: 1e-13 relative for single
linear steps, 1e-12 for a V-cycle / CCCS / the first iterates (accumulated rounding of
two different operation orders), relres <= 1e-10 for solves with the GPU solution
re-checked by the oracle's operator."""
import math

import numpy as np
import pytest

from oracle import mgcccs_oracle as O
from paper_1412_1953_gb300 import build, inputs
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def tp_small(n, E=0.5, seed=0, ny=None):
    L = 30.0 * n / 128
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, seed=seed, ny=ny)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def pair(prob, levels, n_b, **kw):
    okw = {k: v for k, v in kw.items() if k != "krylov_restart"}
    po = O.params_from_problem(prob, levels=levels, n_b=n_b, **okw)
    so = O.Solver(po, prob.v1, prob.v2, prob.v12)
    pg = M.params_for(prob, levels=levels, n_b=n_b, **kw)
    sg = M.Solver(pg, prob.v1, prob.v2, prob.v12)
    return so, sg


def rand_c(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ------------------------------------------------------------------ single steps

@pytest.mark.parametrize("level", [0, 1, 2])
def test_level_steps_match_oracle(level):
    prob = tp_small(64)
    so, sg = pair(prob, 4, 3)
    lev = so.levels[level]
    shape = lev.shape
    u, f = rand_c(shape, 1 + level), rand_c(shape, 11 + level)
    # omega-Jacobi, one and two sweeps
    for sweeps in (1, 2):
        ud = dev(u)
        sg.smooth(level, ud, dev(f), sweeps)
        assert rel(host(ud), O.jacobi(lev, u, f, 2.0 / 3.0, sweeps)) <= 1e-13
    # residual
    rd = torch.empty_like(dev(u))
    sg.level_residual(level, dev(u), dev(f), rd)
    assert rel(host(rd), O.residual(lev, u, f)) <= 1e-13
    # full weighting and bilinear interpolation + add
    cshape = so.levels[level + 1].shape
    rc = torch.empty(cshape, dtype=torch.complex128, device="cuda")
    sg.restrict(level, dev(u), rc)
    assert rel(host(rc), O.restrict_fw(u)) <= 1e-14
    ec = rand_c(cshape, 21 + level)
    ud = dev(u)
    sg.prolong_add(level, dev(ec), ud)
    assert rel(host(ud), u + O.prolong_bilinear(ec, shape)) <= 1e-14


def test_coarse_solve_matches_dense_solve():
    prob = tp_small(64)
    so, sg = pair(prob, 4, 0)
    lev = so.levels[-1]
    f = rand_c(lev.shape, 5)
    ud = torch.empty_like(dev(f))
    sg.coarse_solve(dev(f), ud)
    ref = np.linalg.solve(O.assemble_unweighted(lev).toarray(), f.ravel()).reshape(f.shape)
    assert rel(host(ud), ref) <= 1e-12


@pytest.mark.parametrize("n,nb", [(64, 3), (128, 3), (128, 6), (512, 6)])
def test_bound_states_match_oracle(n, nb):
    prob = tp_small(n) if n == 64 else inputs.temkin_poet(n)
    so, sg = pair(prob, 3 if n <= 128 else n.bit_length() - 4, nb)
    lam, phi, mu, vphi = sg.bound_states()
    np.testing.assert_allclose(lam, so.ch.lam, rtol=0, atol=1e-12 * np.abs(so.ch.lam).max())
    np.testing.assert_allclose(mu, so.ch.mu, rtol=0, atol=1e-12 * np.abs(so.ch.mu).max())
    assert rel(host(phi).T, so.ch.phi) <= 1e-10
    assert rel(host(vphi).T, so.ch.vphi) <= 1e-10


# ------------------------------------------------------------------ cycle, correction, iterates

def test_vcycle_matches_oracle():
    prob = tp_small(64, seed=3)
    so, sg = pair(prob, 4, 3)
    u = rand_c(so.levels[0].shape, 7)
    ud = dev(u)
    sg.vcycle(ud, dev(prob.f))
    assert rel(host(ud), so.vcycle(u, prob.f)) <= 1e-12


@pytest.mark.parametrize("nb", [1, 3, 6])
def test_cccs_matches_oracle(nb):
    prob = tp_small(64, seed=4)
    so, sg = pair(prob, 4, nb)
    u = rand_c(so.levels[0].shape, 8)
    ud = dev(u)
    sg.cccs(ud, dev(prob.f))
    assert rel(host(ud), so.cccs(u, prob.f)) <= 1e-11


def test_precond_apply_matches_oracle():
    prob = tp_small(64, seed=5)
    so, sg = pair(prob, 4, 3)
    r = rand_c(so.levels[0].shape, 9)
    zd = torch.zeros_like(dev(r))
    sg.precond_apply(zd, dev(r))
    assert rel(host(zd), so.precond_apply(r)) <= 1e-12


def test_first_iterates_match_oracle():
    prob = inputs.temkin_poet(128)
    so, sg = pair(prob, 5, 3)
    u = np.zeros_like(prob.f)
    ud = torch.zeros_like(dev(u))
    fd = dev(prob.f)
    for k in range(3):
        u = so.iterate(u, prob.f)
        sg.vcycle(ud, fd)
        sg.cccs(ud, fd)
        assert rel(host(ud), u) <= 1e-12, k


# ------------------------------------------------------------------ solves

def test_solve_128_to_1e10_matches_oracle():
    """The 128^2 TP/ECS workload (E = 0.5, n_b = 3, V(1,1), omega = 2/3, 5 levels)."""
    prob = inputs.temkin_poet(128)
    so, sg = pair(prob, 5, 3)
    uo, hist = so.solve(prob.f, rtol=1e-10, max_iter=1200)
    ud = torch.zeros_like(dev(prob.f))
    its, rr, gh = sg.solve(ud, dev(prob.f), rtol=1e-10, max_iter=1200, history=True)
    u = host(ud)
    assert rr <= 1e-10
    assert abs(its - len(hist)) <= 1
    assert so.relres(u, prob.f) <= 1.001e-10                # re-checked with the oracle operator
    # relres near 1e-10 carries ~eps/1e-10 relative rounding noise from the cancellation in f - Au
    k = min(len(hist), its) - 1
    assert abs(gh[k] - hist[k]) <= 1e-5 * hist[k]
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)


def test_setup_with_cached_states_reproduces_solve():
    """A second handle on the same grid and V1, V2 at another energy reuses the bound
    states (mgcccs_setup_with_states); its solve is bit-identical to a fresh setup's."""
    p1 = tp_small(64, E=0.5, seed=3)
    p2 = tp_small(64, E=0.9, seed=3)
    M._STATE_CACHE.clear()
    s1 = M.Solver(M.params_for(p1, levels=4, n_b=3, krylov_restart=20), p1.v1, p1.v2, p1.v12, reuse_states=True)
    assert len(M._STATE_CACHE) == 1
    s2 = M.Solver(M.params_for(p2, levels=4, n_b=3, krylov_restart=20), p2.v1, p2.v2, p2.v12, reuse_states=True)
    s3 = M.Solver(M.params_for(p2, levels=4, n_b=3, krylov_restart=20), p2.v1, p2.v2, p2.v12)
    f = dev(p2.f)
    u2, u3 = torch.zeros_like(f), torch.zeros_like(f)
    its2, _ = s2.solve(u2, f, rtol=1e-10, max_iter=400)
    its3, _ = s3.solve(u3, f, rtol=1e-10, max_iter=400)
    assert its2 == its3
    assert torch.equal(u2, u3)
    M._STATE_CACHE.clear()


def test_solve_host_matches_device_solve():
    prob = tp_small(64, seed=6)
    _, sg = pair(prob, 4, 3)
    ud = torch.zeros_like(dev(prob.f))
    its, rr = sg.solve(ud, dev(prob.f), rtol=1e-10, max_iter=500)
    uh = np.zeros_like(prob.f)
    its2, rr2 = sg.solve_host(uh, np.ascontiguousarray(prob.f), rtol=1e-10, max_iter=500)
    assert its2 == its
    assert rel(uh, host(ud)) <= 1e-15


@pytest.mark.parametrize("case", ["plain_mg", "nb1", "nb6", "nonsquare", "nu21", "single_level", "deep"])
def test_variants_match_oracle(case):
    kw = dict(levels=4, n_b=3)
    prob = tp_small(64, seed=2)
    if case == "plain_mg":
        kw["n_b"] = 0
    elif case == "nb1":
        kw["n_b"] = 1
    elif case == "nb6":
        kw["n_b"] = 6
    elif case == "nonsquare":
        L = 30.0 * 64 / 128
        prob = inputs.temkin_poet(64, L=L, R0=2 * L / 3, theta=math.pi / 6, E=0.7, seed=2, ny=32)
        prob.Ly = L / 2
        prob.R0y = 2 * prob.Ly / 3
        # regenerate y-dependent inputs on the shorter y box
        x, zx = inputs.node_coordinates(64, L, 2 * L / 3, math.pi / 6)
        y, zy = inputs.node_coordinates(32, L / 2, L / 3, math.pi / 6)
        prob.v2 = (-1.0 / zy[1:-1]).astype(np.complex128)
        X, Y = np.meshgrid(x[1:-1], y[1:-1])
        ZX, ZY = np.meshgrid(zx[1:-1], zy[1:-1])
        prob.v12 = np.ascontiguousarray(1.0 / np.where(X >= Y, ZX, ZY))
        prob.f = np.ascontiguousarray(rand_c((31, 63), 12) * 1e-3)
    elif case == "nu21":
        kw.update(nu1=2, nu2=1)
    elif case == "single_level":
        prob = tp_small(32, seed=2)
        kw["levels"] = 1
    elif case == "deep":
        kw["levels"] = 6          # coarsest 2 cells: one unknown
    so, sg = pair(prob, **kw)
    u = rand_c(so.levels[0].shape, 13)
    ud = dev(u)
    fd = dev(prob.f)
    for _ in range(2):
        u = so.iterate(u, prob.f)
        sg.vcycle(ud, fd)
        if kw["n_b"] > 0:
            sg.cccs(ud, fd)
    assert rel(host(ud), u) <= 1e-11


def test_error_codes_leave_gpu_usable():
    prob = tp_small(32)
    _, sg = pair(prob, 3, 2)
    f = dev(prob.f)
    f[3, 4] = complex(float("nan"), 0.0)
    ud = torch.zeros_like(f)
    with pytest.raises(M.MGCCCSError) as ei:
        sg.solve(ud, f, rtol=1e-10, max_iter=5)
    assert ei.value.code == M.ENONFINITE
    # too small a workspace and a bad pointer are rejected before any launch
    p = M.params_for(prob, levels=3, n_b=2)
    h = M.ctypes.c_void_p()
    z = dev(np.zeros(31, dtype=np.complex128))
    z2 = dev(np.zeros((31, 31), dtype=np.complex128))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    assert M.lib().mgcccs_setup(M.ctypes.byref(h), M.ctypes.byref(p), z.data_ptr(), z.data_ptr(),
                                z2.data_ptr(), ws.data_ptr(), 1024, None) == M.ENOSPACE
    # the context still works
    ud = torch.zeros_like(dev(prob.f))
    its, rr = sg.solve(ud, dev(prob.f), rtol=1e-8, max_iter=300)
    assert rr <= 1e-8


def test_matvec_matches_oracle():
    prob = tp_small(64, seed=7)
    so, sg = pair(prob, 4, 3)
    x = rand_c(so.levels[0].shape, 14)
    yd = torch.empty_like(dev(x))
    sg.matvec(dev(x), yd)
    assert rel(host(yd), O.apply_operator(so.levels[0], x)) <= 1e-13


@pytest.mark.parametrize("k", [1, 11, 21])
def test_gram_schmidt_halves_match_definition(k):
    """mgcccs_gs_dots and mgcccs_gs_update (the two halves of a classical Gram-Schmidt pass
    of the Arnoldi process, Sec. 6) against their plain definitions: out_i = V_i^H w and
    w - sum_i coef_i V_i, on a basis with a padded leading dimension; a vector that is w
    itself gives |w|^2."""
    prob = tp_small(64, seed=9)
    _, sg = pair(prob, 4, 0, krylov_restart=21)
    N = 63 * 63
    ld = N + 5
    V = rand_c((k + 1, ld), 30 + k)
    w = rand_c(N, 40 + k)
    V[k, :N] = w
    Vd, wd = dev(V), dev(w)
    out = torch.empty(k + 1, dtype=torch.complex128, device="cuda")
    sg.gs_dots(Vd, k + 1, Vd[k, :N], out)
    ref = V[:, :N].conj() @ w
    got = host(out)
    assert rel(got, ref) <= 1e-13
    n2 = np.vdot(w, w).real
    assert got[k].imag == 0.0 and abs(got[k].real - n2) <= 1e-13 * n2
    coef = rand_c(k, 50 + k)
    sg.gs_update(Vd, k, dev(coef), wd)
    assert rel(host(wd), w - coef @ V[:k, :N]) <= 1e-13
    # repeated calls give identical results (fixed summation order)
    out2 = torch.empty_like(out)
    sg.gs_dots(Vd, k + 1, Vd[k, :N], out2)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("ld_pad", [0, 1, 64])
def test_complex64_gram_schmidt_halves_match_definition(ld_pad):
    """mgcccs_gs_dots_c64 and mgcccs_gs_update_c64 (the kernels of the mixed form's
    complex64 GMRES cycles) against their definitions evaluated in FP64 from the same
    complex64 values: the products accumulate in FP32 within a warp, so the bound is
    single-precision rounding of the sums.  Even and odd leading dimensions take the
    paired and the per-entry update."""
    prob = tp_small(128, seed=9)
    _, sg = pair(prob, 3, 0, krylov_restart=20)
    N = 127 * 127
    ld = N + ld_pad
    k = 11
    V = rand_c((k + 1, ld), 60).astype(np.complex64)
    w = rand_c(N, 61).astype(np.complex64)
    V[k, :N] = w
    Vd, wd = dev(V), dev(w)
    out = torch.empty(k + 1, dtype=torch.complex128, device="cuda")
    sg.gs_dots_c64(Vd, k + 1, Vd[k, :N], out)
    V64, w64 = V[:, :N].astype(np.complex128), w.astype(np.complex128)
    ref = V64.conj() @ w64
    got = host(out)
    scale = np.sqrt((np.abs(V64) ** 2).sum(axis=1) * (np.abs(w64) ** 2).sum())
    assert np.all(np.abs(got - ref) <= 1e-5 * scale)
    coef = rand_c(k, 62)
    sg.gs_update_c64(Vd, k, dev(coef), wd)
    want = w64 - coef @ V64[:k]
    got_w = host(wd).astype(np.complex128)
    assert np.abs(got_w - want).max() <= 1e-5 * np.abs(want).max()


def test_gmres_partial_cycle_matches_oracle():
    """Ten Arnoldi steps of right-preconditioned GMRES(20) (one partial cycle): the GPU
    iterate (CGS2 Arnoldi, Givens least squares) equals the oracle's (MGS, dense
    least squares): both are the residual minimiser over the same Krylov space."""
    prob = tp_small(64, seed=8)
    so, sg = pair(prob, 4, 3, krylov_restart=20)
    uo, hist, rr_o = O.gmres(so, prob.f, m=20, rtol=1e-14, max_iter=10)
    ud = torch.zeros_like(dev(prob.f))
    its, rr, gh = sg.solve(ud, dev(prob.f), rtol=1e-14, max_iter=10, history=True, raise_on_notconv=False)
    assert its == 10
    assert rel(host(ud), uo) <= 1e-9
    np.testing.assert_allclose(gh, hist, rtol=1e-7)
    assert abs(rr - rr_o) <= 1e-6 * rr_o


def test_gmres_solve_128_matches_oracle():
    """GMRES(20) + MG-CCCS on the 128^2 TP/ECS workload to 1e-10."""
    prob = inputs.temkin_poet(128)
    so, sg = pair(prob, 5, 3, krylov_restart=20)
    uo, hist, rr_o = O.gmres(so, prob.f, m=20, rtol=1e-10, max_iter=400)
    ud = torch.zeros_like(dev(prob.f))
    its, rr = sg.solve(ud, dev(prob.f), rtol=1e-10, max_iter=400)
    assert rr <= 1e-10 and abs(its - len(hist)) <= 2
    u = host(ud)
    assert so.relres(u, prob.f) <= 1.001e-10
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)


def test_coarse_solve_961_unknowns_matches_dense_solve():
    """The largest coarsest grid the benchmark uses: 32 cells per axis on [0,30]^2, i.e. a
    31^2 = 961-unknown dense system (128^2 with 3 levels has the same coarsest grid as
    1024^2 with 6), inverted at setup by the multi-SM Gauss-Jordan kernels (Sec. 3.2, the
    direct coarsest solve), against numpy's dense solve of the oracle's coarsest operator."""
    prob = inputs.temkin_poet(128)
    so, sg = pair(prob, 3, 0)
    lev = so.levels[-1]
    assert lev.shape == (31, 31)
    A = O.assemble_unweighted(lev).toarray()
    for seed in (5, 6):
        f = rand_c(lev.shape, seed)
        ud = torch.empty_like(dev(f))
        sg.coarse_solve(dev(f), ud)
        ref = np.linalg.solve(A, f.ravel()).reshape(f.shape)
        assert rel(host(ud), ref) <= 1e-12


@pytest.mark.parametrize("n,ny,levels,tol,back_tol", [(128, None, 2, 1e-12, 1e-14), (64, 40, 1, 1e-12, 1e-14),
                                                      (40, 64, 1, 1e-12, 1e-14), (64, 34, 1, 1e-12, 1e-14),
                                                      (65, None, 1, 1e-12, 1e-14), (2, 1026, 1, 1e-10, 1e-12)])
def test_coarse_solve_block_reduction_matches_dense_solve(n, ny, levels, tol, back_tol):
    """Coarsest grids beyond 1024 nodes are solved by block cyclic reduction over their rows
    (setup-time block factors, one launch per reduction level).  Against numpy's dense solve
    of the oracle's coarsest operator: 63 x 63 (the coarsest grid of 1024^2 on 5 levels),
    39 rows of 63, 63 rows of 39 and 33 rows of 63 (row counts that are not one less than
    a power of two), the largest block size (64 x 64 nodes) and the smallest (1025 rows of
    one node, 11 reduction levels).  Both are direct solves, so they agree to the
    condition number times the rounding unit: 1e-12 where kappa is about 60, and 1e-10 for
    the one-node chain (y spacing 4.6e-4, kappa 2.8e5, measured by numpy here; the bound is
    checked to exceed kappa times the unit roundoff).  The normwise backward error of the
    solutions is at most 1e-14, and 1e-12 for the chain, whose eleven levels of reduction
    without pivoting combine coefficients from 37 (x) to 4.7e6 (y) (measured 1.7e-13)."""
    prob = tp_small(n, ny=ny)
    so, sg = pair(prob, levels, 0)
    lev = so.levels[-1]
    assert lev.shape[0] * lev.shape[1] > 1024
    A = O.assemble_unweighted(lev).toarray()
    if tol > 1e-12:
        assert tol >= 0.5 * np.finfo(float).eps * np.linalg.cond(A)
    for seed in (5, 6):
        f = rand_c(lev.shape, seed)
        ud = torch.empty_like(dev(f))
        sg.coarse_solve(dev(f), ud)
        x = host(ud)
        ref = np.linalg.solve(A, f.ravel()).reshape(f.shape)
        assert rel(x, ref) <= tol
        back = np.abs(A @ x.ravel() - f.ravel()).max() / (np.abs(A).sum(axis=1).max() * np.abs(x).max())
        assert back <= back_tol


def test_solve_with_block_reduction_on_a_non_square_grid_matches_oracle():
    """GMRES(20) + MG-CCCS on 128 x 80 cells with 2 levels: a 63 x 39 coarsest grid (2457
    nodes) solved by block cyclic reduction in every V-cycle.  The solve meets 1e-10 under
    the oracle's operator, takes the oracle's step count within 2 and lies within 1e-8 of
    the oracle's GMRES(20) solution."""
    prob = tp_small(128, ny=80)
    so, sg = pair(prob, 2, 3, krylov_restart=20)
    assert so.levels[-1].shape == (39, 63)
    fd = dev(prob.f)
    ud = torch.zeros_like(fd)
    its, rr = sg.solve(ud, fd, rtol=1e-10, max_iter=400)
    u = host(ud)
    assert rr <= 1e-10 and so.relres(u, prob.f) <= 1.001e-10
    uo, hist, rr_o = O.gmres(so, prob.f, m=20, rtol=1e-10, max_iter=400)
    assert rr_o <= 1e-10 and abs(its - len(hist)) <= 2
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)


BENCH_LEVELS = 5


@pytest.fixture(scope="module")
def bench_pair():
    """The benchmark workload: 1024^2 TP/ECS on [0,30]^2, E = 0.5, n_b = 3, V(1,1), 5 levels
    (63^2 coarsest grid, block cyclic reduction), GMRES(20); the oracle on the same problem."""
    prob = inputs.temkin_poet(1024)
    so = O.Solver(O.params_from_problem(prob, levels=BENCH_LEVELS, n_b=3), prob.v1, prob.v2, prob.v12)
    sg = M.Solver(M.params_for(prob, levels=BENCH_LEVELS, n_b=3, krylov_restart=20), prob.v1, prob.v2, prob.v12)
    yield prob, so, sg
    sg.close()


def test_benchmark_configuration_steps_match_oracle(bench_pair):
    """At the benchmarked size and depth: the 3969-unknown coarsest solve (<= 1e-12 against a
    dense solve), one V-cycle from zero (<= 1e-12), the bound states, and one CCCS after it
    (<= 1e-9: the correction is built from the third, nearly continuum-embedded eigenvector,
    whose last digits depend on how it was refined)."""
    prob, so, sg = bench_pair
    lev = so.levels[-1]
    assert lev.shape == (63, 63)
    fc = rand_c(lev.shape, 17)
    uc = torch.empty_like(dev(fc))
    sg.coarse_solve(dev(fc), uc)
    ref = np.linalg.solve(O.assemble_unweighted(lev).toarray(), fc.ravel()).reshape(fc.shape)
    assert rel(host(uc), ref) <= 1e-12
    fd = dev(prob.f)
    uv = so.vcycle(np.zeros_like(prob.f), prob.f)
    ud = torch.zeros_like(fd)
    sg.vcycle(ud, fd)
    assert rel(host(ud), uv) <= 1e-12
    lam, phi, mu, vphi = sg.bound_states()
    assert np.abs(lam - so.ch.lam).max() <= 1e-12
    assert rel(host(phi).T, so.ch.phi) <= 1e-8
    u1 = so.cccs(uv, prob.f)
    sg.cccs(ud, fd)
    assert rel(host(ud), u1) <= 1e-9


def test_benchmark_solve_matches_oracle_gmres(bench_pair):
    """The solve the benchmark times (device-driven GMRES(20) + MG-CCCS to 1e-10): its
    solution meets 1e-10 under the oracle's own operator, takes the oracle's step count
    within 2, and is within 1e-8 of the oracle's GMRES(20) solution of the same problem."""
    prob, so, sg = bench_pair
    fd = dev(prob.f)
    ud = torch.zeros_like(fd)
    its, rr = sg.solve(ud, fd, rtol=1e-10, max_iter=400)
    u = host(ud)
    assert rr <= 1e-10
    assert so.relres(u, prob.f) <= 1.001e-10
    uo, hist, rr_o = O.gmres(so, prob.f, m=20, rtol=1e-10, max_iter=400)
    assert rr_o <= 1e-10 and abs(its - len(hist)) <= 2
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)
