"""Host logic of the batching form (no GPU): the level candidates of the autotuner, the
default schedule, the batching workload recipe (R15) and the cache key of a batch."""
import numpy as np

from paper_1412_1953_gb300 import batch as BT
from paper_1412_1953_gb300 import inputs


def test_level_candidates_keep_the_coarsest_grid_between_8_and_64_cells():
    for n in (64, 128, 256, 384, 512, 768, 1024, 2048):
        cands = BT.level_candidates(n)
        assert cands == sorted(cands) and cands
        for lv in cands:
            step = 1 << (lv - 1)
            assert n % step == 0 and 8 <= n // step <= 64
        # no deeper hierarchy keeps the coarsest grid at 8 cells or more
        lv = cands[-1] + 1
        assert n % (1 << (lv - 1)) or n // (1 << (lv - 1)) < 8
    assert BT.level_candidates(384) == [4, 5, 6]      # coarsest grids of 48, 24 and 12 cells
    assert BT.level_candidates(1024) == [5, 6, 7, 8]  # 64 (block cyclic reduction) ... 8 cells
    assert BT.default_schedule(1024) == {"levels": 8, "nu1": 1, "nu2": 1, "tile_rows": 0}


def test_batching_recipe_and_cache_key():
    probs = inputs.batching_problems(count=64)
    assert len(probs) == 64
    sizes = {p.nx for p in probs}
    assert sizes <= {256, 384, 512, 768, 1024} and len(sizes) > 1
    E = np.array([p.E for p in probs])
    assert np.allclose(E, np.linspace(0.1, 2.0, 64))
    for p in probs:
        assert p.nx == p.ny and abs(p.Lx - 30.0 * p.nx / 512) < 1e-12 and abs(p.R0x - 2 * p.Lx / 3) < 1e-12
    k1 = BT._cache_key(probs, 1, "gpu")
    assert k1 == BT._cache_key(inputs.batching_problems(count=64), 1, "gpu")
    assert k1 != BT._cache_key(probs, 0, "gpu") and k1 != BT._cache_key(probs[:63], 1, "gpu")
