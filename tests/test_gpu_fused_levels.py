"""The fused level passes (zero-start sweep + residual + restriction in one kernel,
prolongation + first post-smoothing sweep in another) against the one-step kernels: a
V(1,1) cycle through mgcccs_vcycle / mgcccs_precond_apply equals the same cycle composed
level by level from the C-ABI step calls (mgcccs_smooth, mgcccs_level_residual,
mgcccs_restrict, mgcccs_coarse_solve, mgcccs_prolong_add), which launch only the one-step
kernels.  The passes repeat the one-step kernels' per-node arithmetic; the only freedom
left is how the compiler contracts the complex product of a zero-start sweep, hence a
tolerance of a few units in the last place rather than bit equality."""
import math

import numpy as np
import pytest

from paper_1412_1953_gb300 import build, inputs
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _problem(nx, ny):
    L = 30.0 * nx / 128
    return inputs.temkin_poet(nx, L=L, R0=2 * L / 3, theta=math.pi / 6, E=0.5, seed=3, ny=ny)


def _composed_vcycle(sv, levels, f, u_fine=None):
    """V(1,1) from the one-step C-ABI calls; u_fine is the finest initial guess (zero when
    None, in which case the finest pre-smoothing sweep starts from zero as well)."""
    zeros = lambda l: torch.zeros(sv.level_size(l), dtype=torch.complex128, device="cuda")
    fs, us = [f], []
    for l in range(levels - 1):
        u = zeros(l) if (l > 0 or u_fine is None) else u_fine.clone()
        sv.smooth(l, u, fs[l], 1)
        r = zeros(l)
        sv.level_residual(l, u, fs[l], r)
        fc = zeros(l + 1)
        sv.restrict(l, r, fc)
        us.append(u)
        fs.append(fc)
    e = zeros(levels - 1)
    sv.coarse_solve(fs[-1], e)
    for l in reversed(range(levels - 1)):
        u = us[l]
        sv.prolong_add(l, e, u)
        sv.smooth(l, u, fs[l], 1)
        e = u
    return e


def _rel(a, b):
    torch.cuda.synchronize()
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("nx,ny,levels", [(128, 128, 5), (256, 128, 5), (128, 64, 4)])
def test_vcycle_equals_composed_one_step_kernels(nx, ny, levels):
    prob = _problem(nx, ny)
    sv = M.Solver(M.params_for(prob, levels=levels, n_b=0), prob.v1, prob.v2, prob.v12)
    f = torch.as_tensor(prob.f.reshape(-1)).to("cuda")
    u = torch.zeros_like(f)
    sv.vcycle(u, f)
    ref = _composed_vcycle(sv, levels, f, u_fine=torch.zeros_like(f))
    assert _rel(u, ref) <= 1e-14
    # the preconditioner starts every level from zero, the finest one included
    z = torch.zeros_like(f)
    sv.precond_apply(z, f)
    ref0 = _composed_vcycle(sv, levels, f)
    assert _rel(z, ref0) <= 1e-14
    sv.close()
