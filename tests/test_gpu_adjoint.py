"""Differentiation form on the GPU: amplitude J = <g|u> and its gradients with respect to
E, Z and a per-node potential perturbation from one adjoint MG-CCCS solve, against the
oracle's exact (LU) adjoint gradients and against central differences (step 1e-6)."""
import math

import numpy as np
import pytest

from oracle import mgcccs_oracle as O
from paper_1412_1953_gb300 import build, inputs
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

N = 64
L = 30.0 * N / 128
GEOM = dict(n=N, L=L, R0=2 * L / 3, theta=math.pi / 6)
KW = dict(levels=4, n_b=3, krylov_restart=20)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _fg(E=0.5):
    prob = inputs.temkin_poet(N, L=L, R0=GEOM["R0"], theta=GEOM["theta"], E=E, seed=4)
    g = inputs.gaussian_window(N, L, L / 2, L / 2, 2.0)
    return prob, torch.as_tensor(prob.f).to("cuda"), torch.as_tensor(g).to("cuda"), g


def _oracle_gradients(prob, g, E, Z, dV):
    p = inputs.temkin_poet(N, L=L, R0=GEOM["R0"], theta=GEOM["theta"], E=E, Z=Z, noise_amplitude=0.0)
    lev = O.build_levels(O.params_from_problem(p, levels=1, n_b=0), p.v1, p.v2, p.v12 + dV)[0]
    u = O.direct_solve(lev, prob.f)
    mu = O.direct_solve(lev, g)
    dAdZ = inputs.tp_charge_derivative(N, L, GEOM["R0"], GEOM["theta"])
    return O.amplitude(lev, g, u), O.adjoint_gradients(lev, u, mu, dAdZ), lev


def test_weighted_dot_and_product_match_oracle():
    from paper_1412_1953_gb300 import adjoint as A
    prob, f, gd, g = _fg()
    solver = A.setup_tp(0.5, 1.0, None, GEOM, KW)
    lev = O.build_levels(O.params_from_problem(prob, levels=1, n_b=0), prob.v1, prob.v2, prob.v12)[0]
    rng = np.random.default_rng(2)
    a = rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)
    b = rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)
    d = rng.standard_normal(prob.f.shape) + 1j * rng.standard_normal(prob.f.shape)
    w = O.weights_2d(lev).reshape(a.shape)
    out = torch.zeros(1, dtype=torch.complex128, device="cuda")
    ta, tb, td = (torch.as_tensor(x).to("cuda") for x in (a, b, d))
    solver.weighted_dot(ta, tb, out, d=td, scale=-2.0)
    ref = -2.0 * np.sum(w * a * b * d)
    assert abs(out.item() - ref) <= 1e-13 * abs(ref)
    pr = torch.empty_like(ta)
    solver.weighted_product(ta, tb, pr, scale=-1.0)
    np.testing.assert_allclose(pr.cpu().numpy(), -w * a * b, rtol=1e-14, atol=0)


def test_adjoint_gradients_match_oracle_lu_gradients():
    from paper_1412_1953_gb300 import adjoint as A
    E, Z = 0.5, 1.0
    prob, f, gd, g = _fg(E)
    dV = np.zeros(prob.f.shape)
    res = A.amplitude_and_gradients(E, Z, torch.as_tensor(dV).to("cuda"), f, gd, GEOM, KW, rtol=1e-13)
    J, (dE, dZ, ddV), _ = _oracle_gradients(prob, g, E, Z, dV)
    assert abs(res["J"] - J) <= 1e-9 * abs(J)
    assert abs(res["dE"] - dE) <= 1e-8 * abs(dE)
    assert abs(res["dZ"] - dZ) <= 1e-8 * abs(dZ)
    gv = res["ddV"].cpu().numpy()
    assert np.abs(gv - ddV).max() <= 1e-8 * np.abs(ddV).max()


def test_adjoint_gradients_match_central_differences_on_gpu():
    from paper_1412_1953_gb300 import adjoint as A
    E, Z, h = 0.5, 1.0, 1e-6
    prob, f, gd, g = _fg(E)
    dV0 = torch.zeros(prob.f.shape, dtype=torch.float64, device="cuda")
    res = A.amplitude_and_gradients(E, Z, dV0, f, gd, GEOM, KW, rtol=1e-13)

    def J(E_, Z_, dV_):
        return A.amplitude_and_gradients(E_, Z_, dV_, f, gd, GEOM, KW, rtol=1e-13)["J"]
    fdE = (J(E + h, Z, dV0) - J(E - h, Z, dV0)) / (2 * h)
    fdZ = (J(E, Z + h, dV0) - J(E, Z - h, dV0)) / (2 * h)
    assert abs(res["dE"] - fdE) <= 1e-5 * abs(fdE)
    assert abs(res["dZ"] - fdZ) <= 1e-5 * abs(fdZ)
    for (j, i) in [(20, 20), (31, 12)]:
        e = torch.zeros_like(dV0)
        e[j, i] = h
        fd = (J(E, Z, dV0 + e) - J(E, Z, dV0 - e)) / (2 * h)
        assert abs(res["ddV"][j, i].item() - fd) <= 1e-3 * abs(fd)


def test_autograd_function_matches_adjoint_gradients():
    from paper_1412_1953_gb300 import adjoint as A
    E0, Z0 = 0.5, 1.0
    prob, f, gd, g = _fg(E0)
    E = torch.tensor(E0, dtype=torch.float64, device="cuda", requires_grad=True)
    Z = torch.tensor(Z0, dtype=torch.float64, device="cuda", requires_grad=True)
    dV = torch.zeros(prob.f.shape, dtype=torch.float64, device="cuda", requires_grad=True)
    Jr, Ji = A.TPAmplitude.apply(E, Z, dV, f, gd, GEOM, KW, 1e-13)
    loss = 3.0 * Jr - 2.0 * Ji
    gE, gZ, gdV = torch.autograd.grad(loss, (E, Z, dV))
    ref = A.amplitude_and_gradients(E0, Z0, dV.detach(), f, gd, GEOM, KW, rtol=1e-13)
    assert abs(gE.item() - (3 * ref["dE"].real - 2 * ref["dE"].imag)) <= 1e-9 * abs(ref["dE"])
    assert abs(gZ.item() - (3 * ref["dZ"].real - 2 * ref["dZ"].imag)) <= 1e-9 * abs(ref["dZ"])
    want = 3 * ref["ddV"].real - 2 * ref["ddV"].imag
    assert torch.abs(gdV - want).max().item() <= 1e-9 * torch.abs(ref["ddV"]).max().item()


def test_adjoint_gradients_through_block_reduction_match_oracle():
    """The same gradients on 128^2 cells with 2 levels: the 63 x 63 coarsest grid is solved
    by block cyclic reduction in every V-cycle of the forward and the adjoint solve."""
    from paper_1412_1953_gb300 import adjoint as A
    n, Lb = 128, 30.0
    geom = dict(n=n, L=Lb, R0=2 * Lb / 3, theta=math.pi / 6)
    kw = dict(levels=2, n_b=3, krylov_restart=20)
    E, Z = 0.5, 1.0
    prob = inputs.temkin_poet(n, L=Lb, R0=geom["R0"], theta=geom["theta"], E=E, seed=4)
    g = inputs.gaussian_window(n, Lb, Lb / 2, Lb / 2, 2.0)
    f, gd = torch.as_tensor(prob.f).to("cuda"), torch.as_tensor(g).to("cuda")
    dV = np.zeros(prob.f.shape)
    res = A.amplitude_and_gradients(E, Z, torch.as_tensor(dV).to("cuda"), f, gd, geom, kw, rtol=1e-13)
    p = inputs.temkin_poet(n, L=Lb, R0=geom["R0"], theta=geom["theta"], E=E, Z=Z, noise_amplitude=0.0)
    lev = O.build_levels(O.params_from_problem(p, levels=1, n_b=0), p.v1, p.v2, p.v12 + dV)[0]
    u = O.direct_solve(lev, prob.f)
    mu = O.direct_solve(lev, g)
    dAdZ = inputs.tp_charge_derivative(n, Lb, geom["R0"], geom["theta"])
    J = O.amplitude(lev, g, u)
    dE, dZ, ddV = O.adjoint_gradients(lev, u, mu, dAdZ)
    assert abs(res["J"] - J) <= 1e-9 * abs(J)
    assert abs(res["dE"] - dE) <= 1e-8 * abs(dE)
    assert abs(res["dZ"] - dZ) <= 1e-8 * abs(dZ)
    assert np.abs(res["ddV"].cpu().numpy() - ddV).max() <= 1e-8 * np.abs(ddV).max()
