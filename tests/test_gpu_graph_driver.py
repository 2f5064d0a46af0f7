"""Device-driven GMRES solves: the whole solve as one CUDA graph with conditional nodes
(restart loop, Arnoldi loop, stop tests on the device).  It runs the same arithmetic
in the same order as the host-driven cycles, so iterations, relres and u are identical
to the host driver's, in both precisions; edge cases (zero source, step budget,
non-finite source) end with the same codes; batched graphs equal one-at-a-time solves."""
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


def _small(n, E=0.5, seed=0):
    L = 30.0 * n / 128
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, seed=seed)


def _solver(prob, levels, precision=0, nb=3):
    return M.Solver(M.params_for(prob, levels=levels, n_b=nb, krylov_restart=20, precision=precision),
                    prob.v1, prob.v2, prob.v12)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_driver_equals_host_driver(precision):
    prob = _small(64, seed=4)
    sv = _solver(prob, 4, precision)
    f = torch.as_tensor(prob.f).to("cuda")
    ug, uh = torch.zeros_like(f), torch.zeros_like(f)
    its_g, rr_g = sv.solve(ug, f, rtol=1e-10, max_iter=400)
    M.mgcccs_set_solve_driver(sv, M.DRIVER_HOST)
    its_h, rr_h = sv.solve(uh, f, rtol=1e-10, max_iter=400)
    torch.cuda.synchronize()
    assert its_g == its_h and rr_g == rr_h
    assert torch.equal(ug, uh)
    so = O.Solver(O.params_from_problem(prob, levels=4, n_b=3), prob.v1, prob.v2, prob.v12)
    assert so.relres(ug.cpu().numpy(), prob.f) <= 1.001e-10


def test_graph_driver_128_matches_oracle_gmres():
    prob = inputs.temkin_poet(128)
    so = O.Solver(O.params_from_problem(prob, levels=5, n_b=3), prob.v1, prob.v2, prob.v12)
    sv = _solver(prob, 5)
    uo, hist, _ = O.gmres(so, prob.f, m=20, rtol=1e-10, max_iter=400)
    f = torch.as_tensor(prob.f).to("cuda")
    u = torch.zeros_like(f)
    its, rr = sv.solve(u, f, rtol=1e-10, max_iter=400)
    uh = u.cpu().numpy()
    assert rr <= 1e-10 and abs(its - len(hist)) <= 2
    assert so.relres(uh, prob.f) <= 1.001e-10
    assert np.linalg.norm(uh - uo) <= 1e-8 * np.linalg.norm(uo)


def test_graph_driver_rebuilds_for_new_buffers_and_resumes():
    prob = _small(64, seed=1)
    sv = _solver(prob, 4)
    f1 = torch.as_tensor(prob.f).to("cuda")
    f2 = 2.0 * f1
    u1, u2 = torch.zeros_like(f1), torch.zeros_like(f1)
    its1, _ = sv.solve(u1, f1, rtol=1e-10, max_iter=400)
    its2, _ = sv.solve(u2, f2, rtol=1e-10, max_iter=400)
    assert its1 == its2
    assert torch.allclose(u2, 2.0 * u1, rtol=0, atol=1e-9 * float(u1.abs().max()))
    # a converged u resumes with no step
    its3, rr3 = sv.solve(u1, f1, rtol=1e-10, max_iter=400)
    assert its3 == 0 and rr3 <= 1e-10


def test_graph_driver_edge_cases():
    prob = _small(64, seed=2)
    sv = _solver(prob, 4)
    f = torch.as_tensor(prob.f).to("cuda")
    # zero source: u = 0 with no step
    z = torch.zeros_like(f)
    u = torch.full_like(f, 1.0 - 2.0j)
    its, rr = sv.solve(u, z, rtol=1e-10, max_iter=50)
    assert its == 0 and rr == 0.0 and bool((u == 0).all())
    # step budget: ENOTCONV after exactly max_iter steps, u and relres valid
    u = torch.zeros_like(f)
    its, rr = sv.solve(u, f, rtol=1e-10, max_iter=7, raise_on_notconv=False)
    assert its == 7 and 1e-10 < rr < 1.0
    with pytest.raises(M.MGCCCSError) as e:
        sv.solve(torch.zeros_like(f), f, rtol=1e-10, max_iter=7)
    assert e.value.code == M.ENOTCONV
    # non-finite source
    fb = f.clone()
    fb[3, 5] = complex("nan")
    with pytest.raises(M.MGCCCSError) as e:
        sv.solve(torch.zeros_like(f), fb, rtol=1e-10, max_iter=50)
    assert e.value.code == M.ENONFINITE
    # the handle still solves afterwards
    u = torch.zeros_like(f)
    its, rr = sv.solve(u, f, rtol=1e-10, max_iter=400)
    assert rr <= 1e-10


def _batch_problem(n, E, seed):
    L = 30.0 * n / 512
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, seed=seed)


def test_batch_graph_equals_single_solves_and_replays():
    cases = [(64, 0.3, 4, 0), (96, 0.8, 4, 1), (128, 1.2, 5, 1), (64, 1.9, 4, 0)]
    probs = [_batch_problem(n, E, k) for k, (n, E, _, _) in enumerate(cases)]
    svs = [M.Solver(M.params_for(p, levels=lv, n_b=3, krylov_restart=20, precision=pr), p.v1, p.v2, p.v12)
           for p, (_, _, lv, pr) in zip(probs, cases)]
    fs = [torch.as_tensor(p.f).to("cuda") for p in probs]
    us = [torch.zeros_like(f) for f in fs]
    b = M.Batch(svs, us, fs)
    its, rr, st = b.run(rtol=1e-10, max_iter=800)
    torch.cuda.synchronize()
    assert st == [M.OK] * len(cases)
    first = [u.clone() for u in us]
    for u in us:
        u.zero_()
    its2, rr2, _ = b.run(rtol=1e-10, max_iter=800)
    torch.cuda.synchronize()
    assert its2 == its and rr2 == rr
    for p, sv, f, u, u0, k in zip(probs, svs, fs, us, first, its):
        assert torch.equal(u, u0)
        u1 = torch.zeros_like(f)
        k1, _ = sv.solve(u1, f, rtol=1e-10, max_iter=800)
        torch.cuda.synchronize()
        assert k1 == k and torch.equal(u1, u)
        so = O.Solver(O.params_from_problem(p, levels=sv.p.levels, n_b=3), p.v1, p.v2, p.v12)
        assert so.relres(u.cpu().numpy(), p.f) <= 1.001e-10
    b.close()
