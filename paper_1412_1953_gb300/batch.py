"""Batched MG-CCCS solves of many (grid, energy) problems on one GPU, with an autotuned
multigrid schedule per grid size.

Every problem gets its own setup handle and CUDA stream.  Two drivers run them together:
a batch graph (mgcccs_batch_create / _run: every problem's device-driven solve as an
independent branch of one CUDA graph, launched once) and the host lock-step driver
(mgcccs_batch_solve: GMRES cycles of all problems advanced together, each Arnoldi step
a replayed graph on the problem's stream).  Either way small grids overlap on the GPU
instead of running one by one.

The autotuner picks, for each grid size and precision, the number of levels and the
pre/post smoothing sweep counts (nu1, nu2) with the shortest measured setup + solve time
to the tolerance on a probe problem of that size (each energy of a batch needs its own
setup), and caches the choice in a JSON file keyed by (n, precision, GPU name).  Tile shapes of the kernels are fixed (chosen for the
FP64 pipe and HBM), so the schedule is what varies with the grid.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import inputs
from . import mgcccs as M

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
SWEEPS = ((1, 1), (2, 1), (1, 2), (2, 2))


def level_candidates(n: int, coarsest_min: int = 8, coarsest_max: int = 32) -> list[int]:
    """Level counts whose coarsest grid has n / 2^(levels-1) cells per side in
    [coarsest_min, coarsest_max] (the dense coarsest solve holds at most 31^2 unknowns)."""
    out = []
    for lv in range(2, 16):
        step = 1 << (lv - 1)
        if n % step:
            break
        if coarsest_min <= n // step <= coarsest_max:
            out.append(lv)
    return out


def default_schedule(n: int) -> dict:
    lv = level_candidates(n)
    return {"levels": lv[-1] if lv else 1, "nu1": 1, "nu2": 1}


def _cache_key(n: int, precision: int, gpu: str) -> str:
    return f"{n}|{'mixed' if precision else 'fp64'}|{gpu}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def autotune(n: int, precision: int = 1, E: float = 1.0, n_b: int = 3, krylov_restart: int = 20,
             rtol: float = 1e-10, max_iter: int = 2000, cache_path: str | None = DEFAULT_CACHE,
             repeats: int = 2, force: bool = False) -> dict:
    """Schedule {levels, nu1, nu2, seconds, iterations} for n x n grids of the batching
    workload shape, measured on the problem at energy E (cached unless force)."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _cache_key(n, precision, gpu)
    cache = _load(cache_path) if cache_path else {}
    if key in cache and not force:
        return cache[key]
    L = 30.0 * n / 512
    prob = inputs.temkin_poet(n, L=L, R0=2.0 * L / 3.0, theta=math.pi / 6, E=E, seed=0)
    f = torch.as_tensor(prob.f).to("cuda")
    u = torch.zeros_like(f)
    best = None
    trials = []
    for lv in level_candidates(n):
        for nu1, nu2 in SWEEPS:
            torch.cuda.synchronize()
            t = time.perf_counter()
            sv = M.Solver(M.params_for(prob, levels=lv, nu1=nu1, nu2=nu2, n_b=n_b, krylov_restart=krylov_restart,
                                       precision=precision), prob.v1, prob.v2, prob.v12, reuse_states=True)
            torch.cuda.synchronize()
            setup = time.perf_counter() - t
            sv.solve(u, f, rtol=rtol, max_iter=5, raise_on_notconv=False)        # build the solve graph
            times, its, rr = [], 0, math.inf
            for _ in range(repeats):
                u.zero_()
                torch.cuda.synchronize()
                t = time.perf_counter()
                its, rr = sv.solve(u, f, rtol=rtol, max_iter=max_iter, raise_on_notconv=False)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t)
            sv.close()
            sec = min(times) + setup
            trials.append({"levels": lv, "nu1": nu1, "nu2": nu2, "seconds": sec, "setup_seconds": setup,
                           "iterations": its, "relres": rr})
            if rr <= rtol and (best is None or sec < best["seconds"]):
                best = trials[-1]
    if best is None:
        best = dict(default_schedule(n), seconds=None, iterations=None, relres=None)
    best = dict(best, probe_E=E, trials=trials)
    if cache_path:
        cache = _load(cache_path)
        cache[key] = best
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best


class BatchSolver:
    """Setup handles (one stream each) for a list of Problems; solve() runs them together."""

    def __init__(self, problems, schedules: dict | None = None, n_b: int = 3, precision: int = 1,
                 krylov_restart: int = 20):
        import torch
        self.problems = list(problems)
        self.solvers = []
        for prob in self.problems:
            sch = (schedules or {}).get(prob.nx) or default_schedule(prob.nx)
            p = M.params_for(prob, levels=sch["levels"], nu1=sch["nu1"], nu2=sch["nu2"], n_b=n_b,
                             krylov_restart=krylov_restart, precision=precision)
            self.solvers.append(M.Solver(p, prob.v1, prob.v2, prob.v12, stream=torch.cuda.Stream(),
                                         reuse_states=True))
        self.f = [torch.as_tensor(prob.f).to("cuda") for prob in self.problems]
        self.u = [torch.zeros_like(f) for f in self.f]

    @property
    def unknowns(self) -> int:
        return sum(p.n_unknowns for p in self.problems)

    def solve(self, rtol: float = 1e-10, max_iter: int = 2000, zero: bool = True):
        import torch
        if zero:
            for u in self.u:
                u.zero_()
            torch.cuda.synchronize()
        return M.mgcccs_batch_solve(self.solvers, self.u, self.f, rtol=rtol, max_iter=max_iter)

    def graph(self, stream=None) -> "M.Batch":
        """The device-driven batch graph over this batch's handles and buffers."""
        return M.Batch(self.solvers, self.u, self.f, stream=stream)

    def close(self):
        for s in self.solvers:
            s.close()
