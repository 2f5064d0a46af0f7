"""The allocation-free norm entry point, for callers that cannot call cudaMalloc: code
running while a CUDA graph is captured in the global mode (allocation is illegal there),
code under a framework allocator that owns all device memory with a hard cap, and loops
that must not take the implicit synchronisation an allocation can cause.  Its result is
checked against the residual norm the solver's own entry point computes and against a
host sum of the same vector, on two calls in a row, plus the empty vector.

Kept in a file that pytest collects last, so a failure here stops a first-failure run
only after every other test has run."""
import math

import numpy as np
import pytest

from paper_1412_1953_gb300 import build, inputs
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _problem(n):
    L = 30.0 * n / 128
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=0.5, seed=3)


def _residual_and_norm(n, seed):
    """r = f - (H-E)u and ||r||^2 from mgcccs_residual (the existing entry point)."""
    prob = _problem(n)
    levels = int(round(math.log2(n))) - 2          # coarsest grid of 8 cells
    sg = M.Solver(M.params_for(prob, levels=levels, n_b=0), prob.v1, prob.v2, prob.v12)
    rng = np.random.default_rng(seed)
    u = torch.as_tensor(rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)).to("cuda")
    f = torch.as_tensor(prob.f).to("cuda")
    r = torch.empty_like(f)
    n2 = sg.residual(u, f, r, norm=True)
    return sg, r, n2


def _host_norm2(r):
    a = r.cpu().numpy().ravel()
    return float(np.sum(a.real * a.real + a.imag * a.imag))


def test_norm2_noalloc_matches_residual_norm_on_two_calls():
    build.build()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    # first call on this device (looks up the scratch array's address), small vector
    sg1, r1, ref1 = _residual_and_norm(64, 1)
    M.mgcccs_norm2_noalloc(r1, out)
    torch.cuda.synchronize()
    assert abs(out.item() - ref1) <= 1e-13 * ref1
    assert abs(out.item() - _host_norm2(r1)) <= 1e-13 * ref1
    # second call in a row, a vector that spans many scratch slots
    sg2, r2, ref2 = _residual_and_norm(512, 2)
    out.fill_(-1.0)
    M.mgcccs_norm2_noalloc(r2, out)
    torch.cuda.synchronize()
    assert abs(out.item() - ref2) <= 1e-13 * ref2
    assert abs(out.item() - _host_norm2(r2)) <= 1e-13 * ref2
    # sizes beyond the stated maximum are refused before any launch
    code = M.lib().mgcccs_norm2_noalloc(r2.data_ptr(), M.NOALLOC_MAX_N + 1, out.data_ptr(), None)
    assert code == M.EINVAL
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(ref2, rel=1e-13)
    # the empty vector: 0, whether it comes as a real pointer or as NULL
    out.fill_(-1.0)
    assert M.lib().mgcccs_norm2_noalloc(r2.data_ptr(), 0, out.data_ptr(), None) == M.OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
    out.fill_(-1.0)
    M.mgcccs_norm2_noalloc(torch.empty(0, dtype=torch.complex128, device="cuda"), out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
