"""Batched solves through mgcccs_batch_solve: several problems on uneven grids, at
different energies and in both precisions, each on its own stream, advance their GMRES
cycles in lock-step.  Each problem follows exactly the cycle sequence of its own
mgcccs_solve, so iterations and solutions equal the one-at-a-time solves, and every
solution meets the tolerance under the oracle's operator."""
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


def _problem(n, E, seed):
    """Batching workload shape: L = 30 n / 512 (constant spacing), ECS beyond 2L/3."""
    L = 30.0 * n / 512
    return inputs.temkin_poet(n, L=L, R0=2 * L / 3, theta=math.pi / 6, E=E, seed=seed)


CASES = [(64, 0.3, 4, 0), (96, 0.8, 4, 1), (128, 1.2, 5, 0), (128, 0.5, 5, 1), (64, 1.9, 4, 1)]


def _solvers(cases, **kw):
    out = []
    for k, (n, E, levels, prec) in enumerate(cases):
        prob = _problem(n, E, seed=k)
        sv = M.Solver(M.params_for(prob, levels=levels, n_b=3, krylov_restart=20, precision=prec, **kw),
                      prob.v1, prob.v2, prob.v12, stream=torch.cuda.Stream())
        out.append((prob, sv))
    return out


def test_batch_equals_individual_solves_and_meets_tolerance():
    pairs = _solvers(CASES)
    fs = [torch.as_tensor(p.f).to("cuda") for p, _ in pairs]
    us = [torch.zeros_like(f) for f in fs]
    its, rr, st = M.mgcccs_batch_solve([s for _, s in pairs], us, fs, rtol=1e-10, max_iter=800)
    torch.cuda.synchronize()
    assert st == [M.OK] * len(CASES)
    for (prob, sv), u, f, k, r in zip(pairs, us, fs, its, rr):
        assert r <= 1e-10
        u1 = torch.zeros_like(f)
        k1, r1 = sv.solve(u1, f, rtol=1e-10, max_iter=800)
        torch.cuda.synchronize()
        assert k == k1
        assert r == r1
        assert torch.equal(u, u1)
        so = O.Solver(O.params_from_problem(prob, levels=sv.p.levels, n_b=3), prob.v1, prob.v2, prob.v12)
        assert so.relres(u.cpu().numpy(), prob.f) <= 1.001e-10


def test_batch_per_problem_status_and_zero_rhs():
    pairs = _solvers(CASES[:3])
    fs = [torch.as_tensor(p.f).to("cuda") for p, _ in pairs]
    fs[1] = torch.zeros_like(fs[1])
    us = [torch.full_like(f, 1.0 + 1.0j) for f in fs]
    # 5 steps: the problems with a source stop unconverged, the zero source gives u = 0
    its, rr, st = M.mgcccs_batch_solve([s for _, s in pairs], us, fs, rtol=1e-10, max_iter=5)
    torch.cuda.synchronize()
    assert st == [M.ENOTCONV, M.OK, M.ENOTCONV]
    assert its[0] == 5 and its[1] == 0 and its[2] == 5
    assert rr[1] == 0.0 and bool((us[1] == 0).all())
    assert rr[0] > 1e-10 and np.isfinite(rr[0])


def test_batch_rejects_bad_arguments():
    pairs = _solvers(CASES[:2])
    fs = [torch.as_tensor(p.f).to("cuda") for p, _ in pairs]
    us = [torch.zeros_like(f) for f in fs]
    s0 = pairs[0][1]
    with pytest.raises(M.MGCCCSError) as e:
        M.mgcccs_batch_solve([s0, s0], [us[0], us[0]], [fs[0], fs[0]])   # one handle twice
    assert e.value.code == M.EINVAL
    prob = pairs[0][0]
    plain = M.Solver(M.params_for(prob, levels=4, n_b=3), prob.v1, prob.v2, prob.v12)
    with pytest.raises(M.MGCCCSError) as e:
        M.mgcccs_batch_solve([plain], us[:1], fs[:1])    # handle without GMRES
    assert e.value.code == M.EINVAL
    with pytest.raises(M.MGCCCSError) as e:
        M.mgcccs_batch_solve([s0], us[:1], fs[:1], max_iter=0)
    assert e.value.code == M.EINVAL


def test_autotune_picks_a_converging_schedule_per_grid(tmp_path):
    """The batch autotuner runs its candidate schedules on the batch itself: it returns one
    schedule per grid size, drawn from its candidates, that converges every problem, and
    reads it back from the cache file the second time."""
    from paper_1412_1953_gb300 import batch as BT
    problems = [_problem(n, E, seed=k) for k, (n, E) in enumerate([(64, 0.4), (128, 1.1), (64, 1.7), (128, 0.2)])]
    cache = str(tmp_path / "tune.json")
    sched = BT.autotune(problems, precision=1, cache_path=cache, repeats=1)
    assert sorted(sched) == [64, 128]
    for n, s in sched.items():
        assert (s["nu1"], s["nu2"]) in BT.SWEEPS
        assert s["levels"] in BT.level_candidates(n)
        assert s["tile_rows"] in BT.TILE_ROWS
    bs = BT.BatchSolver(problems, sched, n_b=3, precision=1)
    g = bs.graph()
    its, rr, st = g.run(rtol=1e-10, max_iter=2000)
    assert st == [M.OK] * len(problems) and max(rr) <= 1e-10
    g.close()
    bs.close()
    assert BT.autotune(problems, precision=1, cache_path=cache) == sched


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_rows_do_not_change_the_solve(precision):
    """The small levels' tile height (the autotuner's tile knob) changes launch shapes only:
    every tile kind evaluates the same per-node arithmetic, so the solves are bit-identical."""
    prob = _problem(128, 0.6, seed=5)
    sv = M.Solver(M.params_for(prob, levels=5, n_b=3, krylov_restart=20, precision=precision),
                  prob.v1, prob.v2, prob.v12)
    f = torch.as_tensor(prob.f).to("cuda")
    out = {}
    for rows in (0, 4, 8, 2):
        sv.set_tile_rows(rows)
        u = torch.zeros_like(f)
        its, rr = sv.solve(u, f, rtol=1e-10, max_iter=600)
        out[rows] = (its, u)
    for rows in (4, 8, 2):
        assert out[rows][0] == out[0][0]
        assert torch.equal(out[rows][1], out[0][1])
    with pytest.raises(M.MGCCCSError):
        sv.set_tile_rows(3)


def test_concurrent_setups_with_block_reduction_match_sequential_setups():
    """Problems of a batch are set up from several host threads at once.  Here the coarsest
    grids take block cyclic reduction with two block sizes (63 rows of 63 at 256^2 on 3
    levels, 47 of 47 at 384^2 on 4 levels), whose setup kernels share launch limits: the
    concurrent setups give the same solves, bit for bit, as setups made one at a time."""
    from paper_1412_1953_gb300 import batch as BT
    problems = [_problem(n, E, seed=k) for k, (n, E) in enumerate([(256, 0.4), (384, 1.1), (256, 1.7),
                                                                     (384, 0.2), (256, 0.9), (384, 1.4)])]
    sched = {256: {"levels": 3, "nu1": 1, "nu2": 1}, 384: {"levels": 4, "nu1": 1, "nu2": 1}}
    out = {}
    for threads in (1, 4):
        bs = BT.BatchSolver(problems, sched, n_b=3, precision=1, setup_threads=threads)
        g = bs.graph()
        for u in bs.u:
            u.zero_()
        its, rr, st = g.run(rtol=1e-10, max_iter=2000)
        torch.cuda.synchronize()
        assert st == [M.OK] * len(problems) and max(rr) <= 1e-10
        out[threads] = (its, [u.clone() for u in bs.u])
        g.close()
        bs.close()
    assert out[1][0] == out[4][0]
    for a, b in zip(out[1][1], out[4][1]):
        assert torch.equal(a, b)
