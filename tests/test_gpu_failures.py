"""Failure detection without a GPU fault: a diverging iteration, a one-iteration budget and
bad arguments each end with their error code, and the context keeps working.  The
divergence case is the stand-alone MG-CCCS iteration with the coarse levels left on the
unrotated ECS contour, which the oracle shows growing by about 1e3 per iteration."""
import dataclasses

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


def test_divergence_is_detected_like_the_oracle_sees_it():
    prob = inputs.temkin_poet(128)
    po = dataclasses.replace(O.params_from_problem(prob, levels=5, n_b=3), coarse_gamma=0.0)
    so = O.Solver(po, prob.v1, prob.v2, prob.v12)
    u = np.zeros_like(prob.f)
    hist = []
    while True:
        u = so.iterate(u, prob.f)
        hist.append(so.relres(u, prob.f))
        if hist[-1] > 1e6 * min(hist):
            break
    sv = M.Solver(M.params_for(prob, levels=5, n_b=3, coarse_gamma=0.0), prob.v1, prob.v2, prob.v12)
    f = torch.as_tensor(prob.f).to("cuda")
    ud = torch.zeros_like(f)
    it_c = M.ctypes.c_int(0)
    rr_c = M.ctypes.c_double(0.0)
    code = M.lib().mgcccs_solve(sv.h, ud.data_ptr(), f.data_ptr(), 1e-10, 50, M.ctypes.byref(it_c),
                                M.ctypes.byref(rr_c), None)
    assert code == M.EDIVERGED
    assert it_c.value == len(hist)
    assert abs(rr_c.value - hist[-1]) <= 1e-6 * hist[-1]
    # the GPU context is healthy: a well-posed solve on a fresh handle converges
    good = M.Solver(M.params_for(prob, levels=5, n_b=3, krylov_restart=20), prob.v1, prob.v2, prob.v12)
    u2 = torch.zeros_like(f)
    its, rr = good.solve(u2, f, rtol=1e-10, max_iter=400)
    assert rr <= 1e-10


def test_one_iteration_budget_and_bad_arguments():
    L = 30.0 * 64 / 128
    prob = inputs.temkin_poet(64, L=L, R0=2 * L / 3)
    sv = M.Solver(M.params_for(prob, levels=4, n_b=3), prob.v1, prob.v2, prob.v12)
    f = torch.as_tensor(prob.f).to("cuda")
    u = torch.zeros_like(f)
    its, rr = sv.solve(u, f, rtol=1e-10, max_iter=1, raise_on_notconv=False)
    assert its == 1 and 1e-10 < rr < 1.0
    lib = M.lib()
    assert lib.mgcccs_solve(sv.h, None, f.data_ptr(), 1e-10, 10, None, None, None) == M.EINVAL
    assert lib.mgcccs_solve(sv.h, u.data_ptr(), f.data_ptr(), 1e-10, 0, None, None, None) == M.EINVAL
    assert lib.mgcccs_vcycle(None, u.data_ptr(), f.data_ptr()) == M.EINVAL
    # and the handle still solves
    u.zero_()
    its, rr = sv.solve(u, f, rtol=1e-6, max_iter=400)
    assert rr <= 1e-6
