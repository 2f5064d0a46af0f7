"""Batched MG-CCCS solves of many (grid, energy) problems on one GPU, with an autotuned
multigrid schedule per grid size.

Every problem gets its own setup handle and CUDA stream.  Two drivers run them together:
a batch graph (mgcccs_batch_create / _run: every problem's device-driven solve as an
independent branch of one CUDA graph, launched once) and the host lock-step driver
(mgcccs_batch_solve: GMRES cycles of all problems advanced together, each Arnoldi step
a replayed graph on the problem's stream).  Either way small grids overlap on the GPU
instead of running one by one.

The autotuner picks, by a coarse grid search and then coordinate descent on the batch
itself, the level count (from the deepest hierarchy to the shallowest whose coarsest grid
has at most 64 cells) and the pre/post smoothing sweep counts (nu1, nu2) with the shortest
measured setup + solve time, then the tile height of the stencil passes on the small
levels (2, 4 or 8 rows per block: a batch of many small grids runs most of its launches on
those levels) by solve time, and caches the choice in a JSON file keyed by the batch's
grids, the precision and the GPU name.  The fine-level tiles stay fixed (32 x 8, chosen for
the FP64 pipe and HBM).
"""
from __future__ import annotations

import concurrent.futures
import json
import math
import os
import time

from . import inputs
from . import mgcccs as M

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
SWEEPS = ((1, 1), (2, 1), (1, 2), (2, 2))
TILE_ROWS = (2, 4, 8)
SETUP_THREADS = 4          # host threads that set problems of a batch up concurrently


def level_candidates(n: int, coarsest_min: int = 8, coarsest_max: int = 64) -> list[int]:
    """Level counts whose coarsest grid has n / 2^(levels-1) cells per side in
    [coarsest_min, coarsest_max]: up to 31^2 unknowns the coarsest solve applies a dense
    inverse, beyond that (rows of at most 63 nodes) block cyclic reduction."""
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
    return {"levels": lv[-1] if lv else 1, "nu1": 1, "nu2": 1, "tile_rows": 0}


def _cache_key(problems, precision: int, gpu: str) -> str:
    sig = ",".join(f"{p.nx}x{p.ny}" for p in problems)
    return f"{len(problems)}|{sig}|{'mixed' if precision else 'fp64'}|{gpu}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _run_batch(problems, sched, n_b, precision, krylov_restart, rtol, max_iter, repeats, tile_rows=None):
    """Setup seconds, best solve seconds over `repeats`, Arnoldi steps and convergence of
    one schedule on the whole batch (one batch graph launch per solve)."""
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    bs = BatchSolver(problems, sched, n_b=n_b, precision=precision, krylov_restart=krylov_restart)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t
    out = []
    for rows in (tile_rows or (None,)):
        if rows is not None:
            for sv in bs.solvers:
                sv.set_tile_rows(rows)
        g = bs.graph()
        g.run(rtol=rtol, max_iter=5)                      # instantiate the batch graph
        times, its, rr, st = [], [], [math.inf], []
        for _ in range(repeats):
            for u in bs.u:
                u.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            its, rr, st = g.run(rtol=rtol, max_iter=max_iter)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        g.close()
        ok = all(x == M.OK for x in st) and max(rr) <= rtol
        out.append((rows, min(times), int(sum(its)), ok))
    bs.close()
    return setup, out


def autotune(problems, precision: int = 1, n_b: int = 3, krylov_restart: int = 20, rtol: float = 1e-10,
             max_iter: int = 2000, cache_path: str | None = DEFAULT_CACHE, repeats: int = 2,
             force: bool = False) -> dict:
    """Schedules {n: {levels, nu1, nu2, tile_rows}} for a batch of problems, by coordinate
    descent on the batch itself, each knob the same for every grid size: (1) V(1,1) and
    V(2,2) on every depth (the deepest hierarchy, one, two ... levels less: more sweeps can
    make up for a shallower hierarchy and the reverse), (2) on the best depth the other
    sweep pairs (nu1, nu2), (3) on that schedule the tile height of the small levels'
    passes.  Cost is the measured setup + solve time for (1) (each energy needs its own
    setup; the bound states, which every schedule shares, are left out) and the solve time
    alone for (2) and (3), which setup does not depend on.  Cached unless force.
    The batch is its own probe because a batch shares the GPU between its problems:
    throughput decides, and a schedule with cheaper but more Arnoldi steps that wins a
    solve on its own (where launch latency decides) can lose in the batch."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _cache_key(problems, precision, gpu)
    cache = _load(cache_path) if cache_path else {}
    if key in cache and not force:
        return {int(n): sch for n, sch in cache[key]["schedules"].items()}
    sizes = sorted({p.nx for p in problems})
    # bound states are shared by every candidate (same grids and potentials): solve them
    # once, so that the setup time below is the part a schedule changes
    BatchSolver(problems, None, n_b=n_b, precision=precision, krylov_restart=krylov_restart).close()
    run = dict(n_b=n_b, precision=precision, krylov_restart=krylov_restart, rtol=rtol, max_iter=max_iter,
               repeats=repeats)
    trials = []

    def schedule(drop, nu1, nu2):
        sched = {}
        for n in sizes:
            lv = level_candidates(n)
            sched[n] = {"levels": lv[max(len(lv) - 1 - drop, 0)] if lv else 1, "nu1": nu1, "nu2": nu2}
        return sched

    def cost(drop, nu1, nu2, with_setup=True):
        setup, ((_, sec, steps, ok),) = _run_batch(problems, schedule(drop, nu1, nu2), **run)
        trials.append({"drop_levels": drop, "nu1": nu1, "nu2": nu2, "seconds": sec, "setup_seconds": setup,
                       "steps": steps, "converged": ok})
        return (setup + sec if with_setup else sec) if ok else math.inf

    max_drop = max(len(level_candidates(n)) for n in sizes) - 1
    corner = (SWEEPS[0], SWEEPS[-1])          # V(1,1) and V(2,2)
    best = min(((cost(drop, nu1, nu2), drop, nu1, nu2) for drop in range(max_drop + 1) for nu1, nu2 in corner),
               key=lambda x: x[0])
    # on one depth the setup does not depend on the sweeps: compare solve times only (the
    # setup's own timing noise, several host threads, would otherwise decide close calls)
    best_solve = [t for t in trials if (t["drop_levels"], t["nu1"], t["nu2"]) == best[1:]][0]["seconds"]
    best = (best_solve, best[1], best[2], best[3])
    for nu1, nu2 in SWEEPS:
        if (nu1, nu2) in corner:
            continue
        c = cost(best[1], nu1, nu2, with_setup=False)
        if c < best[0]:
            best = (c, best[1], nu1, nu2)
    schedules = schedule(best[1], best[2], best[3]) if math.isfinite(best[0]) else \
        {n: default_schedule(n) for n in sizes}
    _, per_rows = _run_batch(problems, schedules, tile_rows=TILE_ROWS, **run)
    best_rows = None
    for rows, sec, steps, ok in per_rows:
        trials.append({"tile_rows": rows, "seconds": sec, "steps": steps, "converged": ok})
        if ok and (best_rows is None or sec < best_rows[0]):
            best_rows = (sec, rows)
    for n in schedules:
        schedules[n] = dict(schedules[n], tile_rows=best_rows[1] if best_rows else 0)
    if cache_path:
        cache = _load(cache_path)
        cache[key] = {"schedules": {str(n): sch for n, sch in schedules.items()}, "trials": trials}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return schedules


class BatchSolver:
    """Setup handles (one stream each) for a list of Problems; solve() runs them together."""

    def __init__(self, problems, schedules: dict | None = None, n_b: int = 3, precision: int = 1,
                 krylov_restart: int = 20, setup_threads: int = SETUP_THREADS):
        import torch
        self.problems = list(problems)
        dev = torch.cuda.current_device()

        def make(prob):
            with torch.cuda.device(dev):
                sch = (schedules or {}).get(prob.nx) or default_schedule(prob.nx)
                p = M.params_for(prob, levels=sch["levels"], nu1=sch["nu1"], nu2=sch["nu2"], n_b=n_b,
                                 krylov_restart=krylov_restart, precision=precision)
                sv = M.Solver(p, prob.v1, prob.v2, prob.v12, stream=torch.cuda.Stream(), reuse_states=True)
                if sch.get("tile_rows"):
                    sv.set_tile_rows(sch["tile_rows"])
                return sv

        # the first problem of each grid computes the grid's bound states (then shared); the
        # other setups run from several host threads, each on its own stream, so that their
        # kernels (a setup alone fills few SMs) overlap on the GPU
        first = {}
        for k, prob in enumerate(self.problems):
            first.setdefault((prob.nx, prob.ny, prob.Lx, prob.Ly, prob.R0x, prob.R0y, prob.theta,
                              prob.v1.tobytes(), prob.v2.tobytes()), k)
        self.solvers = [None] * len(self.problems)

        def put(k):
            self.solvers[k] = make(self.problems[k])

        try:
            for k in first.values():
                put(k)
            rest = [k for k in range(len(self.problems)) if self.solvers[k] is None]
            if setup_threads > 1 and len(rest) > 1:
                with concurrent.futures.ThreadPoolExecutor(max_workers=setup_threads) as ex:
                    for fut in [ex.submit(put, k) for k in rest]:
                        fut.result()
            else:
                for k in rest:
                    put(k)
        except BaseException:
            # a failed setup leaves no half-built batch: release the handles made so far
            for sv in self.solvers:
                if sv is not None:
                    sv.close()
            raise
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
