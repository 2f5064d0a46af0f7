"""Eigenvalues of the 1D bound-state Hamiltonians (Eq. (9) on the ECS grid) by the
Ehrlich-Aberth iteration that setup uses: the whole spectrum matches a dense eigen-solve
of the oracle's tridiagonal (one-to-one), the QR fallback agrees on the bound part, and
setup on the benchmark grids never needs the fallback."""
import math

import numpy as np
import pytest

from oracle import mgcccs_oracle as O
from paper_1412_1953_gb300 import build, inputs
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
scipy_opt = pytest.importorskip("scipy.optimize")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _match(a, b):
    """Largest distance of an optimal one-to-one pairing of two eigenvalue sets."""
    D = np.abs(a[:, None] - b[None, :])
    r, c = scipy_opt.linear_sum_assignment(D)
    return float(D[r, c].max())


@pytest.mark.parametrize("n,levels", [(128, 5), (256, 6), (512, 7)])
def test_spectrum_matches_dense_eigensolve(n, levels):
    prob = inputs.temkin_poet(n)
    sv = M.Solver(M.params_for(prob, levels=levels, n_b=3), prob.v1, prob.v2, prob.v12)
    assert sv.eig_fallbacks() == 0
    ax = O.make_axis(n, prob.Lx, prob.R0x, prob.theta)
    H = O.tridiag_1d(ax, prob.v1).toarray()
    ev = np.linalg.eigvals(H)
    scale = float(np.abs(ev).max())
    lam = sv.axis_spectrum(0, method=0)
    assert lam.shape == ev.shape and np.all(np.isfinite(lam))
    assert _match(lam, ev) <= 1e-11 * scale
    # the n_b smallest real parts, which setup selects, agree to far better than their gaps
    a = np.sort(lam.real)[:3]
    b = np.sort(ev.real)[:3]
    assert np.max(np.abs(a - b)) <= 1e-11 * scale


def test_spectrum_1024_matches_dense_and_qr_on_the_bound_part():
    """At 1023 unknowns the whole Ehrlich-Aberth spectrum matches the dense eigen-solve.
    The one-thread QR fallback is compared on the smallest real parts only: its rotations
    are complex-orthogonal, not unitary, and part of its upper spectrum is inaccurate on
    this non-Hermitian matrix (eigenvalues that the dense solve does not have)."""
    prob = inputs.temkin_poet(1024)
    sv = M.Solver(M.params_for(prob, levels=8, n_b=3), prob.v1, prob.v2, prob.v12)
    assert sv.eig_fallbacks() == 0
    ab = sv.axis_spectrum(1, method=0)
    qr = sv.axis_spectrum(1, method=1)
    ax = O.make_axis(1024, prob.Ly, prob.R0y, prob.theta)
    ev = np.linalg.eigvals(O.tridiag_1d(ax, prob.v2).toarray())
    scale = float(np.abs(ev).max())
    assert _match(ab, ev) <= 1e-11 * scale
    low = lambda x: x[np.argsort(x.real, kind="stable")[:3]]
    assert np.max(np.abs(low(qr) - low(ev))) <= 1e-11 * scale
    assert np.max(np.abs(low(ab) - low(ev))) <= 1e-11 * scale


def test_precision_form_grid_needs_no_fallback():
    """2048^2 on [0,60]^2 with ECS beyond 40 and n_b = 6 (the precision form's grid)."""
    prob = inputs.temkin_poet(2048, L=60.0, R0=40.0, theta=math.pi / 6)
    sv = M.Solver(M.params_for(prob, levels=9, n_b=6, krylov_restart=20, precision=1), prob.v1, prob.v2,
                  prob.v12)
    assert sv.eig_fallbacks() == 0
    lam, _, mu, _ = sv.bound_states()
    assert np.all(np.diff(lam.real) >= 0) and np.all(lam.real < 0)
