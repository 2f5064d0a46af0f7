"""Mixed-precision form on the GPU: complex64 smoothing, transfers, projections and inner
GMRES cycles inside FP64 iterative refinement.  The complex64 preconditioner matches the
oracle's (FP64) preconditioner to single-precision rounding; the refined solution meets
1e-10 under the oracle's FP64 operator and matches the oracle solution."""
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


def _pair(prob, levels, nb, **kw):
    so = O.Solver(O.params_from_problem(prob, levels=levels, n_b=nb), prob.v1, prob.v2, prob.v12)
    sg = M.Solver(M.params_for(prob, levels=levels, n_b=nb, krylov_restart=20, precision=1, **kw),
                  prob.v1, prob.v2, prob.v12)
    return so, sg


@pytest.mark.parametrize("n,levels", [(64, 4), (128, 2)])
def test_complex64_preconditioner_matches_oracle_to_single_precision(n, levels):
    """(128, 2): a 63 x 63 coarsest grid, solved by block cyclic reduction in FP64 from the
    complex64 restricted residual."""
    L = 30.0 * n / 128
    prob = inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=0.5, seed=5)
    so, sg = _pair(prob, levels, 3)
    rng = np.random.default_rng(9)
    r = rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)
    z = torch.zeros(prob.f.shape, dtype=torch.complex128, device="cuda")
    sg.precond_apply(z, torch.as_tensor(r).to("cuda"))
    zo = so.precond_apply(r)
    err = np.abs(z.cpu().numpy() - zo).max() / np.abs(zo).max()
    assert 1e-10 < err <= 2e-5          # single-precision, and genuinely not FP64


@pytest.mark.parametrize("n,levels,nb", [(128, 5, 3), (256, 6, 6)])
def test_mixed_solve_meets_1e10_and_matches_oracle(n, levels, nb):
    prob = inputs.temkin_poet(n, E=0.5)
    so, sg = _pair(prob, levels, nb)
    f = torch.as_tensor(prob.f).to("cuda")
    u = torch.zeros_like(f)
    its, rr = sg.solve(u, f, rtol=1e-10, max_iter=600)
    uh = u.cpu().numpy()
    assert rr <= 1e-10
    assert so.relres(uh, prob.f) <= 1.001e-10
    uo, hist, rro = O.gmres(so, prob.f, m=20, rtol=1e-12, max_iter=600)
    assert np.linalg.norm(uh - uo) <= 1e-8 * np.linalg.norm(uo)
    assert its <= 2 * len(hist) + 40
