"""The mixed-precision form keeps the bound states FP64 where they are computed, refined and
stored, and uses complex64 copies of them inside the complex64 preconditioner (its
projections and corrections).  This checks, on the oracle alone, what that rounding does:
it perturbs one preconditioner application by the same order as rounding the residual the
complex64 preconditioner acts on anyway, and it leaves the GMRES(20) step count and the
converged solution unchanged.  The outer residual and the refinement stay FP64, so the
stopping test is unaffected."""
import numpy as np
import pytest

from oracle import mgcccs_oracle as O
from paper_1412_1953_gb300 import inputs


def _round32(a):
    return a.astype(np.complex64).astype(np.complex128)


@pytest.fixture(scope="module")
def solvers():
    prob = inputs.temkin_poet(128)
    p = O.params_from_problem(prob, levels=3, n_b=3)
    s64 = O.Solver(p, prob.v1, prob.v2, prob.v12)
    s32 = O.Solver(p, prob.v1, prob.v2, prob.v12)
    s32.ch.phi = _round32(s32.ch.phi)
    s32.ch.vphi = _round32(s32.ch.vphi)
    return prob, s64, s32


def test_rounded_states_perturb_the_preconditioner_like_a_rounded_residual(solvers):
    prob, s64, s32 = solvers
    rng = np.random.default_rng(3)
    r = rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)
    z = s64.precond_apply(r)
    d_states = np.abs(s32.precond_apply(r) - z).max() / np.abs(z).max()
    d_input = np.abs(s64.precond_apply(_round32(r)) - z).max() / np.abs(z).max()
    assert 0 < d_states <= 1e-7
    assert d_states <= 10 * d_input


def test_rounded_states_leave_the_gmres_solve_unchanged(solvers):
    prob, s64, s32 = solvers
    u64, h64, rr64 = O.gmres(s64, prob.f, m=20, rtol=1e-10, max_iter=400)
    u32, h32, rr32 = O.gmres(s32, prob.f, m=20, rtol=1e-10, max_iter=400)
    assert rr64 <= 1e-10 and rr32 <= 1e-10
    assert abs(len(h32) - len(h64)) <= 1
    assert np.linalg.norm(u32 - u64) <= 1e-9 * np.linalg.norm(u64)
