"""Pins for the CPU oracle: each test checks the oracle against something other than
itself -- a closed form, a value the paper prints, an exact invariant, a textbook
special case or an independent direct solve.  The last group plants plausible
mistakes in the oracle and checks that a pin catches each one."""
import math
import os

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

from oracle import mgcccs_oracle as O
from paper_1412_1953_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden(key):
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v, *_ = line.split()
            if k == key:
                return float(v)
    raise KeyError(key)


def free_level(n, L, R0, theta, E=0.0, gamma=0.0):
    ax = O.make_axis(n, L, R0, theta, gamma)
    z = np.zeros(n - 1, dtype=np.complex128)
    return O.Level(ax, O.make_axis(n, L, R0, theta, gamma), z, z.copy(),
                   np.zeros((n - 1, n - 1), dtype=np.complex128), E)


def tp_level(n, E=0.5, L=30.0, R0=20.0, theta=math.pi / 6):
    prob = inputs.temkin_poet(n, L=L, R0=R0, theta=theta, E=E)
    p = O.params_from_problem(prob, levels=1, n_b=0)
    return O.build_levels(p, prob.v1, prob.v2, prob.v12)[0], prob


def tp_small(n, E=0.5, seed=0):
    """TP problem with the 128^2 workload's spacing h = 30/128 on a box scaled with n
    (L = 30 n/128, ECS from 2L/3), so that small grids still resolve the waves."""
    L = 30.0 * n / 128
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, seed=seed)


def sine_mode(n, k, l):
    i = np.arange(1, n)
    return np.outer(np.sin(l * math.pi * i / n), np.sin(k * math.pi * i / n)).astype(np.complex128)


# ------------------------------------------------------------------ operator (Eq. (11))

def test_weighted_operator_is_complex_symmetric():
    """Sec. 2.5: with ECS the discrete operator is complex symmetric, A = A^T for
    A = W (H - E) (R0 = 20 falls inside a cell here, so the kink cell is covered)."""
    lev, _ = tp_level(32)
    A = O.assemble_weighted(lev)
    asym = abs(A - A.T).max()
    assert asym <= 4e-16 * abs(A).max()
    # and it is not Hermitian: the ECS layer makes it genuinely complex
    assert abs(A - A.conj().T).max() > 1e-3 * abs(A).max()


def test_poisson_stencil_on_sine_modes():
    """theta = 0, V = 0, E = 0: -1/2 Laplacian on sin modes has eigenvalue
    (2/h^2)(sin^2(k pi/2n) + sin^2(l pi/2n))."""
    n, L = 16, 3.0
    lev = free_level(n, L, 10.0, 0.0)
    h = L / n
    for k, l in [(1, 1), (3, 7), (15, 2), (8, 8)]:
        u = sine_mode(n, k, l)
        lam = 2.0 / h ** 2 * (math.sin(k * math.pi / (2 * n)) ** 2 + math.sin(l * math.pi / (2 * n)) ** 2)
        np.testing.assert_allclose(O.apply_operator(lev, u), lam * u, atol=1e-12 * lam)


def test_stencil_exact_for_quadratics_on_ecs_contour():
    """The 3-point nonuniform second difference is exact for quadratics in z, also with
    complex, kinked spacings: -1/2 Lap(q(x) q(y)) = q(x) + q(y) for q(z) = z (z_n - z)."""
    n = 24
    lev = free_level(n, 30.0, 20.0, math.pi / 6)
    z = lev.ax.z
    q = z * (z[-1] - z)
    u = np.outer(q[1:-1], q[1:-1])
    expect = q[1:-1][None, :] + q[1:-1][:, None]
    got = O.apply_operator(lev, u)
    assert abs(got - expect).max() <= 1e-11 * abs(expect).max()


def test_full_rotation_scales_operator():
    """On a fully rotated contour z = x e^{i g} (R0 = 0) the kinetic operator is
    e^{-2 i g} times the real one; the same holds for the coarse-level rotation."""
    n, g = 20, 0.3
    rng = np.random.default_rng(3)
    u = rng.standard_normal((n - 1, n - 1)) + 1j * rng.standard_normal((n - 1, n - 1))
    real = O.apply_operator(free_level(n, 5.0, 99.0, 0.0), u)
    rot = O.apply_operator(free_level(n, 5.0, 0.0, g), u)
    np.testing.assert_allclose(rot, np.exp(-2j * g) * real, atol=1e-12 * abs(real).max())
    rot2 = O.apply_operator(free_level(n, 5.0, 99.0, 0.0, gamma=g), u)
    np.testing.assert_allclose(rot2, np.exp(-2j * g) * real, atol=1e-12 * abs(real).max())


def test_stencil_and_sparse_assembly_agree():
    lev, prob = tp_level(20)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((19, 19)) + 1j * rng.standard_normal((19, 19))
    A = O.assemble_unweighted(lev)
    np.testing.assert_allclose((A @ u.ravel()).reshape(u.shape), O.apply_operator(lev, u), rtol=0, atol=1e-12)


# ------------------------------------------------------------------ transfers and smoother

def test_full_weighting_is_quarter_bilinear_transpose():
    """In 2D, full weighting equals 1/4 times the transpose of bilinear interpolation."""
    nf, nc = 15, 7
    P = np.zeros((nf * nf, nc * nc), dtype=np.complex128)
    for k in range(nc * nc):
        e = np.zeros(nc * nc, dtype=np.complex128)
        e[k] = 1
        P[:, k] = O.prolong_bilinear(e.reshape(nc, nc), (nf, nf)).ravel()
    R = np.zeros((nc * nc, nf * nf), dtype=np.complex128)
    for k in range(nf * nf):
        e = np.zeros(nf * nf, dtype=np.complex128)
        e[k] = 1
        R[:, k] = O.restrict_fw(e.reshape(nf, nf)).ravel()
    assert abs(R - P.T / 4).max() == 0.0


def test_full_weighting_on_quadratic():
    """1D weights [1 2 1]/4 map x^2 to x^2 + 1/2 (index units); tensor product in 2D."""
    n = 16
    i = np.arange(1, n, dtype=np.float64)
    r = np.outer(np.ones(n - 1), i ** 2).astype(np.complex128)
    I = np.arange(1, n // 2, dtype=np.float64)
    expect = np.outer(np.ones(n // 2 - 1), (2 * I) ** 2 + 0.5)
    np.testing.assert_allclose(O.restrict_fw(r), expect, rtol=0, atol=1e-13)


def test_bilinear_reproduces_bilinear_functions():
    """Away from the boundary ring, bilinear interpolation is exact for a + bx + cy + dxy."""
    nc, nf = 8, 16
    I = np.arange(1, nc, dtype=np.float64)
    g = lambda x, y: 1.5 - 0.25 * x + 0.75 * y + 0.125 * x * y
    ec = g(I[None, :] * 2, I[:, None] * 2).astype(np.complex128)
    ef = O.prolong_bilinear(ec, (nf - 1, nf - 1))
    i = np.arange(1, nf, dtype=np.float64)
    expect = g(i[None, :], i[:, None])
    np.testing.assert_allclose(ef[1:-1, 1:-1], expect[1:-1, 1:-1], rtol=0, atol=1e-13)


def test_jacobi_symbol():
    """One omega-Jacobi sweep on the Poisson error mode multiplies it by 1 - omega lambda/D."""
    n, L, om = 16, 2.0, 2.0 / 3.0
    lev = free_level(n, L, 99.0, 0.0)
    h = L / n
    for k, l in [(1, 2), (9, 13), (15, 15)]:
        u = sine_mode(n, k, l)
        lam = 2.0 / h ** 2 * (math.sin(k * math.pi / (2 * n)) ** 2 + math.sin(l * math.pi / (2 * n)) ** 2)
        out = O.jacobi(lev, u, np.zeros_like(u), om, 1)
        np.testing.assert_allclose(out, (1 - om * lam / (2.0 / h ** 2)) * u, atol=1e-13)


def _lfa_two_grid(n, h, om, nu1, nu2):
    """Two-grid error propagation of the V(nu1, nu2) cycle for -1/2 Laplacian with
    Dirichlet conditions, in the sine basis (k, l), from the textbook Fourier symbols:
    FW maps mode k to cos^2(k pi/2n) and mode n-k to -sin^2(k pi/2n) times coarse mode k;
    bilinear interpolation is the transpose relation; coarse operator re-discretised."""
    m = n // 2
    N = (n - 1) ** 2
    idx = lambda k, l: (l - 1) * (n - 1) + (k - 1)
    lam = lambda k, l: 2.0 / h ** 2 * (math.sin(k * math.pi / (2 * n)) ** 2 + math.sin(l * math.pi / (2 * n)) ** 2)
    D = 2.0 / h ** 2
    S = np.zeros((N, N))
    for k in range(1, n):
        for l in range(1, n):
            S[idx(k, l), idx(k, l)] = 1 - om * lam(k, l) / D
    CGC = np.eye(N)
    c2 = lambda k: math.cos(k * math.pi / (2 * n)) ** 2
    s2 = lambda k: math.sin(k * math.pi / (2 * n)) ** 2
    hc = 2 * h
    for k in range(1, m):
        for l in range(1, m):
            harm = [(k, l, c2(k) * c2(l)), (n - k, l, -s2(k) * c2(l)),
                    (k, n - l, -c2(k) * s2(l)), (n - k, n - l, s2(k) * s2(l))]
            lc = 2.0 / hc ** 2 * (math.sin(k * math.pi / (2 * m)) ** 2 + math.sin(l * math.pi / (2 * m)) ** 2)
            for (a, b, pa) in harm:          # interpolation weight
                for (c, d, rc) in harm:      # restriction weight
                    CGC[idx(a, b), idx(c, d)] -= pa * rc * lam(c, d) / lc
    return np.linalg.matrix_power(S, nu2) @ CGC @ np.linalg.matrix_power(S, nu1)


def test_two_grid_cycle_matches_fourier_analysis():
    """The oracle's 2-level V(1,1) cycle, written in the sine basis, equals the exact
    two-grid Fourier (LFA) operator entry by entry (Poisson, Dirichlet, uniform grid)."""
    n, L = 16, 4.0
    h = L / n
    p = O.Params(n, n, L, L, 99.0, 99.0, 0.0, 0.0, levels=2, n_b=0, coarse_gamma=0.0)
    z = np.zeros(n - 1, dtype=np.complex128)
    levels = O.build_levels(p, z, z, np.zeros((n - 1, n - 1), dtype=np.complex128))
    N = (n - 1) ** 2
    M = np.zeros((N, N), dtype=np.complex128)
    f0 = np.zeros((n - 1, n - 1), dtype=np.complex128)
    for q in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[q] = 1
        M[:, q] = O.vcycle(levels, p, e.reshape(n - 1, n - 1), f0).ravel()
    i = np.arange(1, n)
    Q1 = np.sin(np.outer(i, i) * math.pi / n)           # DST-I, Q1 @ Q1 = n/2 I
    Q = np.kron(Q1, Q1)                                  # column (l, k) -> mode, row (j, i)
    Mhat = (Q @ M @ Q) / (n / 2) ** 2
    expect = _lfa_two_grid(n, h, 2.0 / 3.0, 1, 1)
    assert abs(Mhat - expect).max() <= 1e-12


@pytest.mark.parametrize("n,levels,L,R0", [(64, 4, 15.0, 10.0), (128, 5, 30.0, 20.0), (96, 3, 22.5, 15.0)])
def test_coarse_level_potentials_are_the_potentials_at_the_coarse_nodes(n, levels, L, R0):
    """Sec. 3.2 re-discretises the operator on the coarser grid of the same box, so level l
    needs V1, V2, V12 at its own n/2^l-cell nodes.  The oracle injects them from the fine
    arrays; the values must equal, bit for bit, the potentials evaluated independently on an
    (n >> l)-cell grid of the same box and ECS contour (the coarse node I is the fine node
    I 2^l, and x = I L/(n/2^l) is the same double as (I 2^l) L/n)."""
    prob = inputs.temkin_poet(n, L=L, R0=R0, theta=math.pi / 6, E=0.5)
    lv = O.build_levels(O.params_from_problem(prob, levels=levels, n_b=0), prob.v1, prob.v2, prob.v12)
    for l in range(levels):
        ref = inputs.temkin_poet(n >> l, L=L, R0=R0, theta=math.pi / 6, E=0.5)
        assert lv[l].v1.shape == ref.v1.shape and lv[l].v12.shape == ref.v12.shape
        assert np.array_equal(lv[l].v1, ref.v1), l
        assert np.array_equal(lv[l].v2, ref.v2), l
        assert np.array_equal(lv[l].v12, ref.v12), l
        # the operator of level l lives on the (n >> l)-cell contour, rotated by gamma for l >= 1
        _, z = inputs.node_coordinates(n >> l, L, R0, math.pi / 6)
        np.testing.assert_allclose(lv[l].ax.z, z * np.exp(1j * (O.COARSE_GAMMA_DEFAULT if l else 0.0)),
                                   rtol=0, atol=1e-13 * L)


def _lfa_symbols(n, h, rho, c, om):
    """Fourier symbols on an n-cell Dirichlet grid of spacing h whose kinetic part is scaled
    by rho (rho = e^{-2 i gamma} on a contour rotated by gamma) and whose potential minus
    energy is the constant c: operator, omega-Jacobi smoother."""
    ks = np.arange(1, n)
    s2 = np.sin(ks * math.pi / (2 * n)) ** 2
    lam = rho * 2.0 / h ** 2 * (s2[None, :] + s2[:, None]) + c        # [l][k]
    D = rho * 2.0 / h ** 2 + c
    return np.diag(lam.ravel()), np.diag((1 - om * lam / D).ravel())


def _lfa_restriction(n):
    """Full weighting in the sine bases: fine mode (a, b) -> coarse mode (k, l) with weight
    w(a) w(b), w(k) = cos^2(k pi/2n), w(n-k) = -sin^2(k pi/2n); bilinear interpolation is the
    transpose in these (DST-I) bases."""
    m = n // 2
    R = np.zeros(((m - 1) ** 2, (n - 1) ** 2))
    c2 = lambda k: math.cos(k * math.pi / (2 * n)) ** 2
    s2 = lambda k: math.sin(k * math.pi / (2 * n)) ** 2
    for k in range(1, m):
        for l in range(1, m):
            for a, wa in ((k, c2(k)), (n - k, -s2(k))):
                for b, wb in ((l, c2(l)), (n - l, -s2(l))):
                    R[(l - 1) * (m - 1) + (k - 1), (b - 1) * (n - 1) + (a - 1)] = wa * wb
    return R


def _lfa_three_grid(n, h, gamma, c, om, nu1, nu2):
    """Three-level V(nu1, nu2) error propagation for -1/2 Laplacian + c (c constant, complex)
    with Dirichlet conditions: fine level on the real axis, levels 1 and 2 on the contour
    rotated by gamma (kinetic symbol times e^{-2 i gamma}, potential unchanged), the coarsest
    solved exactly, the coarse-grid correction on level 1 approximated by a two-grid cycle
    from zero: B_1 = (I - M_1) A_1^{-1}."""
    rho = np.exp(-2j * gamma)
    A0, S0 = _lfa_symbols(n, h, 1.0, c, om)
    A1, S1 = _lfa_symbols(n // 2, 2 * h, rho, c, om)
    A2, _ = _lfa_symbols(n // 4, 4 * h, rho, c, om)
    R0, R1 = _lfa_restriction(n), _lfa_restriction(n // 2)
    mp = np.linalg.matrix_power
    M1 = mp(S1, nu2) @ (np.eye(len(A1)) - R1.T @ np.linalg.solve(A2, R1) @ A1) @ mp(S1, nu1)
    B1 = (np.eye(len(A1)) - M1) @ np.linalg.inv(A1)
    return mp(S0, nu2) @ (np.eye(len(A0)) - R0.T @ B1 @ R0 @ A0) @ mp(S0, nu1)


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 1)])
def test_three_level_cycle_with_potential_matches_fourier_analysis(nu1, nu2):
    """With constant potentials V1, V2, V12 (not zero) and E, the oracle's 3-level V-cycle,
    with the coarse levels on the rotated contour of reading R5, written in the sine basis,
    equals the three-level Fourier operator entry by entry.  This pins the recursion (the
    coarse cycle from zero, the exact coarsest solve), the potential and energy on every
    coarse level, and that the rotation scales the kinetic part only."""
    n, L, gamma = 16, 4.0, math.radians(14.6)
    h = L / n
    v1c, v2c, v12c, E = -0.8 + 0.1j, -0.6, 0.3 - 0.05j, 0.4
    p = O.Params(n, n, L, L, 99.0, 99.0, 0.0, E, levels=3, n_b=0, nu1=nu1, nu2=nu2, coarse_gamma=gamma)
    v1 = np.full(n - 1, v1c, dtype=np.complex128)
    v2 = np.full(n - 1, v2c, dtype=np.complex128)
    v12 = np.full((n - 1, n - 1), v12c, dtype=np.complex128)
    levels = O.build_levels(p, v1, v2, v12)
    N = (n - 1) ** 2
    M = np.zeros((N, N), dtype=np.complex128)
    f0 = np.zeros((n - 1, n - 1), dtype=np.complex128)
    for q in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[q] = 1
        M[:, q] = O.vcycle(levels, p, e.reshape(n - 1, n - 1), f0).ravel()
    i = np.arange(1, n)
    Q1 = np.sin(np.outer(i, i) * math.pi / n)
    Q = np.kron(Q1, Q1)
    Mhat = (Q @ M @ Q) / (n / 2) ** 2
    expect = _lfa_three_grid(n, h, gamma, v1c + v2c + v12c - E, 2.0 / 3.0, nu1, nu2)
    assert abs(expect).max() > 0.05
    assert abs(Mhat - expect).max() <= 1e-12


def test_direct_solve_parity():
    """MG-CCCS iterated to 1e-13 agrees with sparse LU of the weighted system (the
    paper's direct reference method, Sec. 3.2), TP potentials, ECS grid."""
    for n, lv in [(16, 2), (32, 3)]:
        prob = tp_small(n)
        s = O.Solver(O.params_from_problem(prob, levels=lv, n_b=3), prob.v1, prob.v2, prob.v12)
        u, hist = s.solve(prob.f, rtol=1e-13, max_iter=400)
        assert hist[-1] <= 1e-13
        ud = O.direct_solve(s.levels[0], prob.f)
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
        assert s.relres(ud, prob.f) <= 1e-13


# ------------------------------------------------------------------ bound states (Eq. (9))

def test_threshold_eigenvalue_matches_paper():
    """Exponential model, 300 + 150 ECS cells of h = 0.05, theta = pi/7 (Sec. 3.3):
    the lowest eigenvalue is the single-ionisation threshold printed in Fig. 4."""
    ax = O.make_axis(450, 22.5, 15.0, math.pi / 7)
    v = -4.5 * np.exp(-ax.z[1:-1] ** 2)
    lam, _ = O.bound_states(ax, v, 1)
    assert abs(lam[0] - golden("exp_model_threshold")) <= 1e-8


def test_hydrogen_bound_states_converge_at_second_order():
    """-1/2 d^2/dx^2 - 1/x has lambda_n = -1/(2 n^2); FD error is O(h^2)."""
    lam = {}
    for n in (128, 256, 512):
        ax = O.make_axis(n, 30.0, 20.0, math.pi / 6)
        lam[n], _ = O.bound_states(ax, -1.0 / ax.z[1:-1], 2)
    assert abs(lam[128][0] + 0.5) <= 7e-3
    ratio = (lam[256][0] + 0.5) / (lam[512][0] + 0.5)
    assert 3.8 < ratio.real < 4.2
    rich1 = (4 * lam[512][0] - lam[256][0]) / 3
    rich2 = (4 * lam[512][1] - lam[256][1]) / 3
    assert abs(rich1 + 0.5) <= 1e-5
    assert abs(rich2 + 0.125) <= 1e-5


def test_bound_states_bilinear_orthonormal_and_refined():
    """phi^T W phi = I without conjugation (Sec. 3.1); after shift-and-invert the
    eigen-residual is at round-off level (Sec. 5.1.2)."""
    ax = O.make_axis(128, 30.0, 20.0, math.pi / 6)
    v = -1.0 / ax.z[1:-1]
    lam, phi = O.bound_states(ax, v, 4)
    G = phi.T @ (ax.w[:, None] * phi)
    assert abs(G - np.eye(4)).max() <= 1e-12
    H = O.tridiag_1d(ax, v)
    for k in range(4):
        assert np.linalg.norm(H @ phi[:, k] - lam[k] * phi[:, k]) <= 1e-12 * abs(lam[k]) * np.linalg.norm(phi[:, k])


# ------------------------------------------------------------------ CCCS (Sec. 4)

def _free_solver(n, E, n_b):
    prob = inputs.temkin_poet(n, E=E)
    prob.v12 = np.zeros_like(prob.v12)
    s = O.Solver(O.params_from_problem(prob, levels=2, n_b=n_b), prob.v1, prob.v2, prob.v12)
    return s, prob


@pytest.mark.parametrize("which", [0, 1, 2])
def test_cccs_exact_for_separable_residual(which):
    """Without V12, (H-E)(phi_i x e) = phi_i x (H2 + lambda_i - E) e, so one CCCS from
    u = 0 solves f = phi_i(x) g(y) exactly, for any g (not orthogonal to the bound
    states, so the conventions Eqs. (25)-(26) are exercised); mirrored for
    f = g(x) vphi_j(y)."""
    s, prob = _free_solver(32, 0.5, 3)
    rng = np.random.default_rng(which)
    g = rng.standard_normal(31) + 1j * rng.standard_normal(31)
    f = np.outer(g, s.ch.phi[:, which])                   # [j][i] = g(y_j) phi(x_i)
    u = s.cccs(np.zeros_like(f), f)
    assert s.relres(u, f) <= 1e-12
    f2 = np.outer(s.ch.vphi[:, which], g)
    u2 = s.cccs(np.zeros_like(f2), f2)
    assert s.relres(u2, f2) <= 1e-12


def test_cccs_clears_bound_state_projections():
    """Without V12, after one CCCS the new residual has zero projection onto every
    phi_i along x and every vphi_j along y, for an arbitrary right-hand side."""
    s, prob = _free_solver(32, 0.7, 3)
    lev = s.levels[0]
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((31, 31)) + 1j * rng.standard_normal((31, 31))
    r0 = O.residual(lev, u0, prob.f)
    Px0, Py0, *_ = O.cccs_rhs(lev, s.ch, r0)
    u1 = s.cccs(u0, prob.f)
    Px1, Py1, *_ = O.cccs_rhs(lev, s.ch, O.residual(lev, u1, prob.f))
    assert abs(Px1).max() <= 1e-11 * abs(Px0).max()
    assert abs(Py1).max() <= 1e-11 * abs(Py0).max()


def _banded_to_dense(ab, nb):
    N = ab.shape[1]
    M = np.zeros((N, N), dtype=np.complex128)
    for r in range(N):
        for c in range(max(0, r - nb), min(N, r + nb + 1)):
            M[r, c] = ab[nb + r - c, c]
    return M


def test_channel_systems_are_projected_2d_operator():
    """Eqs. (28)-(29) are the 2D operator projected on the bound states:
    (I x Phi^T W_x)(H - E)(I x Phi) equals the channel-A matrix, and the same along y
    for channel B (TP potentials, V12 included).  Also V^A_im = V^A_mi."""
    n, nb = 24, 3
    prob = inputs.temkin_poet(n, E=0.5)
    s = O.Solver(O.params_from_problem(prob, levels=2, n_b=nb), prob.v1, prob.v2, prob.v12)
    lev, ch = s.levels[0], s.ch
    assert abs(ch.VA - ch.VA.transpose(0, 2, 1)).max() <= 1e-15 * abs(ch.VA).max()
    assert abs(ch.VB - ch.VB.transpose(0, 2, 1)).max() <= 1e-15 * abs(ch.VB).max()
    A = O.assemble_unweighted(lev).toarray()
    m = n - 1
    Iy = np.eye(m)
    proj = np.kron(Iy, (ch.phi * lev.ax.w[:, None]).T)
    lift = np.kron(Iy, ch.phi)
    CA = proj @ A @ lift
    MA = _banded_to_dense(O.channel_matrix_banded(lev.ay, lev.v2, ch.lam, ch.VA, lev.E), nb)
    assert abs(CA - MA).max() <= 1e-10 * abs(MA).max()
    # along y: reorder unknowns to [i][j] so the y operator acts within blocks
    perm = np.arange(m * m).reshape(m, m).T.ravel()
    At = A[np.ix_(perm, perm)]
    projB = np.kron(np.eye(m), (ch.vphi * lev.ay.w[:, None]).T)
    liftB = np.kron(np.eye(m), ch.vphi)
    CB = projB @ At @ liftB
    MB = _banded_to_dense(O.channel_matrix_banded(lev.ax, lev.v1, ch.mu, ch.VB, lev.E), nb)
    assert abs(CB - MB).max() <= 1e-10 * abs(MB).max()


def test_mgcccs_converges_on_tp_ecs_problem():
    """Stand-alone MG-CCCS with complex-contour coarse levels converges on the
    128^2 TP/ECS workload (5 levels, V(1,1), omega = 2/3, n_b = 3)."""
    prob = inputs.temkin_poet(128, E=0.5)
    s = O.Solver(O.params_from_problem(prob, levels=5, n_b=3), prob.v1, prob.v2, prob.v12)
    u, hist = s.solve(prob.f, rtol=1e-3, max_iter=120)
    assert hist[-1] <= 1e-3
    rate = (hist[-1] / hist[5]) ** (1.0 / (len(hist) - 6))
    assert rate < 0.95


# ------------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible bug, planted in the oracle, makes at least one pin fail."""
    # 1. full weighting with 1D weights [1 2 1]/2 instead of /4 (scaling slip)
    orig = O.restrict_fw
    monkeypatch.setattr(O, "restrict_fw", lambda r: 2 * orig(r))
    with pytest.raises(AssertionError):
        test_two_grid_cycle_matches_fourier_analysis()
    monkeypatch.setattr(O, "restrict_fw", orig)
    # 2. convention slip: b_il taken for l >= i instead of l > i
    orig_rhs = O.cccs_rhs

    def bad_rhs(lev, ch, r):
        Px, Py, c, rA, rB = orig_rhs(lev, ch, r)
        for i in range(c.shape[0]):
            rA[i] -= c[i, i] * ch.vphi[:, i]
        return Px, Py, c, rA, rB
    monkeypatch.setattr(O, "cccs_rhs", bad_rhs)
    with pytest.raises(AssertionError):
        test_cccs_exact_for_separable_residual(0)
    monkeypatch.setattr(O, "cccs_rhs", orig_rhs)
    # 3. conjugated ECS rotation
    orig_nodes = O.ecs_nodes
    monkeypatch.setattr(O, "ecs_nodes", lambda n, L, R0, th: orig_nodes(n, L, R0, -th))
    with pytest.raises(AssertionError):
        test_full_rotation_scales_operator()
    monkeypatch.setattr(O, "ecs_nodes", orig_nodes)
    # 4. dropped channel coupling V^A
    orig_setup = O.setup_channels

    def bad_setup(lev, n_b):
        ch = orig_setup(lev, n_b)
        ch.VA = np.zeros_like(ch.VA)
        return ch
    monkeypatch.setattr(O, "setup_channels", bad_setup)
    with pytest.raises(AssertionError):
        test_channel_systems_are_projected_2d_operator()
    monkeypatch.setattr(O, "setup_channels", orig_setup)
    # 5. conjugating normalisation (Hermitian instead of bilinear)
    orig_norm = O._normalise
    monkeypatch.setattr(O, "_normalise", lambda v, w: v / np.sqrt(np.sum(w * v * np.conj(v))))
    with pytest.raises(AssertionError):
        test_bound_states_bilinear_orthonormal_and_refined()
    monkeypatch.setattr(O, "_normalise", orig_norm)


def _planted_build_levels(offset=0, coarse_potential=1.0, rotate_potential=False, rotate=True):
    """build_levels with one plausible mistake: the injection stride shifted by `offset`,
    the coarse potentials scaled by `coarse_potential`, the contour rotation applied to the
    potentials as well, or the coarse levels left unrotated."""
    def bad(p, v1, v2, v12):
        out = []
        for l in range(p.levels):
            s = 1 << l
            g = p.coarse_gamma if (l > 0 and rotate) else 0.0
            o = s - 1 + (offset if l > 0 else 0)
            sc = (coarse_potential if l > 0 else 1.0) * (np.exp(-2j * p.coarse_gamma) if rotate_potential and l else 1.0)
            out.append(O.Level(O.make_axis(p.nx >> l, p.Lx, p.R0x, p.theta, g),
                               O.make_axis(p.ny >> l, p.Ly, p.R0y, p.theta, g),
                               sc * v1[o::s][: (p.nx >> l) - 1].copy(), sc * v2[o::s][: (p.ny >> l) - 1].copy(),
                               sc * v12[o::s, o::s][: (p.ny >> l) - 1, : (p.nx >> l) - 1].copy(), p.E))
        return out
    return bad


@pytest.mark.parametrize("mistake", [dict(offset=1), dict(offset=-1), dict(coarse_potential=0.0),
                                     dict(rotate_potential=True), dict(rotate=False)])
def test_planted_coarse_level_mistakes_are_caught(monkeypatch, mistake):
    """A mistake planted in the oracle's coarse levels (an injection offset off by one
    either way, no potential on the coarse levels, the rotation applied to the potential,
    unrotated coarse levels) fails the coarse-level pins; the unplanted oracle passes both."""
    test_coarse_level_potentials_are_the_potentials_at_the_coarse_nodes(64, 4, 15.0, 10.0)
    test_three_level_cycle_with_potential_matches_fourier_analysis(1, 1)
    monkeypatch.setattr(O, "build_levels", _planted_build_levels(**mistake))
    with pytest.raises(AssertionError):
        test_coarse_level_potentials_are_the_potentials_at_the_coarse_nodes(64, 4, 15.0, 10.0)
        test_three_level_cycle_with_potential_matches_fourier_analysis(1, 1)


# ------------------------------------------------------------------ GMRES acceleration (Sec. 6)

def test_gmres_with_exact_preconditioner_takes_one_step():
    """levels = 1 and n_b = 0 make one 'V-cycle' the exact solve, so right-preconditioned
    GMRES converges in exactly one Arnoldi step."""
    prob = tp_small(16)
    s = O.Solver(O.params_from_problem(prob, levels=1, n_b=0), prob.v1, prob.v2, prob.v12)
    u, hist, rr = O.gmres(s, prob.f, m=5, rtol=1e-12)
    assert len(hist) == 1 and rr <= 1e-12


def test_gmres_finite_termination_without_preconditioner():
    """Unpreconditioned full GMRES on N = 9 unknowns terminates in at most 9 steps."""
    prob = tp_small(4)
    s = O.Solver(O.params_from_problem(prob, levels=1, n_b=0), prob.v1, prob.v2, prob.v12)
    u, hist, rr = O.gmres(s, prob.f, m=9, rtol=1e-12, precondition=False)
    assert len(hist) <= 9 and rr <= 1e-11


def test_gmres_estimate_matches_true_residual_and_direct_solve():
    """The least-squares residual estimate equals the true residual at exit, the residual
    estimates never increase within a cycle, and the converged u is the LU solution."""
    prob = tp_small(32)
    s = O.Solver(O.params_from_problem(prob, levels=3, n_b=3), prob.v1, prob.v2, prob.v12)
    u, hist, rr = O.gmres(s, prob.f, m=20, rtol=1e-11)
    assert rr <= 1e-11
    assert abs(rr - hist[-1]) <= 1e-3 * rr + 1e-14
    for c in range(0, len(hist), 20):
        seg = hist[c:c + 20]
        assert all(b <= a * (1 + 1e-12) for a, b in zip(seg, seg[1:]))
    ud = O.direct_solve(s.levels[0], prob.f)
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)


def test_gmres_accelerates_mgcccs_on_tp_workload():
    """On the 128^2 TP/ECS workload GMRES(20) right-preconditioned by MG-CCCS reaches
    1e-10 in about a hundred Arnoldi steps, where the stand-alone iteration needs
    several hundred."""
    prob = inputs.temkin_poet(128)
    s = O.Solver(O.params_from_problem(prob, levels=5, n_b=3), prob.v1, prob.v2, prob.v12)
    u, hist, rr = O.gmres(s, prob.f, m=20, rtol=1e-10, max_iter=300)
    assert rr <= 1e-10 and len(hist) <= 150


# ------------------------------------------------------------------ adjoint gradients

def _tp_direct(n, E, Z, dV):
    L = 30.0 * n / 128
    prob = inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, Z=Z, seed=4)
    prob.v12 = prob.v12 + dV
    lev = O.build_levels(O.params_from_problem(prob, levels=1, n_b=0), prob.v1, prob.v2, prob.v12)[0]
    return prob, lev


def test_adjoint_gradients_match_central_differences():
    """dJ/dE, dJ/dZ and dJ/ddV_k from one adjoint solve equal central differences
    (step 1e-6) of J computed with exact (LU) forward solves; f held fixed."""
    n, E, Z = 24, 0.5, 1.0
    dV = np.zeros((n - 1, n - 1), dtype=np.complex128)
    prob, lev = _tp_direct(n, E, Z, dV)
    f = prob.f
    x = np.arange(1, n) * prob.Lx / n
    g = np.exp(-((x[None, :] - 3.0) ** 2 + (x[:, None] - 3.0) ** 2) / 8.0).astype(np.complex128)
    u = O.direct_solve(lev, f)
    mu = O.direct_solve(lev, g)
    zx = lev.ax.z[1:-1]
    dAdZ = -(1.0 / zx[None, :] + 1.0 / zx[:, None])
    dE, dZ, ddV = O.adjoint_gradients(lev, u, mu, dAdZ)

    def J(E_, Z_, dV_):
        p_, l_ = _tp_direct(n, E_, Z_, dV_)
        return O.amplitude(l_, g, O.direct_solve(l_, f))
    h = 1e-6
    fdE = (J(E + h, Z, dV) - J(E - h, Z, dV)) / (2 * h)
    fdZ = (J(E, Z + h, dV) - J(E, Z - h, dV)) / (2 * h)
    assert abs(dE - fdE) <= 1e-6 * abs(fdE)
    assert abs(dZ - fdZ) <= 1e-6 * abs(fdZ)
    # a single-node derivative is ~1e-4 of J, so the difference quotient carries the
    # relative rounding of J (about cond * eps) amplified by |J| / (2 h |dJ|): 1e-4 bound
    for (j, i) in [(3, 4), (10, 2), (20, 21)]:
        e = np.zeros_like(dV)
        e[j, i] = h
        fd = (J(E, Z, dV + e) - J(E, Z, dV - e)) / (2 * h)
        assert abs(ddV[j, i] - fd) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("n,L,R0,gamma", [(128, 30.0, 20.0, 0.0), (1024, 30.0, 20.0, 0.0),
                                          (64, 15.0, 10.0, math.radians(14.6)), (96, 30.0, 20.0, 0.3)])
def test_inner_uniform_coefficients_have_the_closed_form(n, L, R0, gamma):
    """Where both cells of a node lie inside R0, Eq. (11) with equal cells h e^{i gamma}
    gives west = east = -1/(2 h^2) e^{-2 i gamma}: the single coefficient the GPU stencil
    uses on that region.  The oracle's coefficients, formed from node differences, agree
    to rounding, and the node just before R0 (one cell scaled) does not."""
    ax = O.make_axis(n, L, R0, math.pi / 6, gamma)
    h = L / n
    c = -0.5 / h ** 2 * np.exp(-2j * gamma)
    inner = [i for i in range(n - 1) if (i + 2) * L / n <= R0]       # interior index i = node i+1
    assert inner == list(range(len(inner))) and len(inner) > 0
    np.testing.assert_allclose(ax.west[inner], c, rtol=1e-12)
    np.testing.assert_allclose(ax.east[inner], c, rtol=1e-12)
    kink = len(inner)
    assert abs(ax.east[kink] - c) > 1e-3 * abs(c)


def test_coarsest_solve_is_the_exact_solve_on_every_call():
    """The V-cycle's coarsest solve (Sec. 3.2: exact) factorises the level once and reuses the
    factors: on two right-hand sides in a row, and on two levels of different size, it
    solves the assembled operator to a residual of rounding size, and equals a sparse LU
    solve of the same operator."""
    lev_a, _ = tp_level(16)
    lev_b, _ = tp_level(32, E=1.1)
    rng = np.random.default_rng(4)
    for lev in (lev_a, lev_b, lev_a):
        A = O.assemble_unweighted(lev).tocsc()
        for _ in range(2):
            f = rng.standard_normal(lev.shape) + 1j * rng.standard_normal(lev.shape)
            x = O.coarsest_solve(lev, f)
            back = np.linalg.norm(A @ x.ravel() - f.ravel()) / (
                scipy.sparse.linalg.norm(A) * np.linalg.norm(x) + np.linalg.norm(f))
            assert back <= 1e-15
            ref = scipy.sparse.linalg.splu(A).solve(f.ravel()).reshape(f.shape)
            assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()
