"""The FP64 throughput probe the benchmark uses for the attainable FP64 rate: every block
writes the sum of its threads' recurrences a <- a m + b, which the closed form
m^n a0 + b (1 - m^n) / (1 - m) fixes; bad arguments launch nothing."""
import numpy as np
import pytest

from paper_1412_1953_gb300 import build
from paper_1412_1953_gb300 import mgcccs as M

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_probe_blocks_sum_the_recurrences():
    build.build()
    blocks, iters, m, b = 5, 64, 0.999, 1e-3
    out = torch.full((blocks + 1,), -1.0, dtype=torch.float64, device="cuda")
    ops = M.mgcccs_fp64_probe(blocks, iters, out, m=m, b=b)
    torch.cuda.synchronize()
    assert ops == blocks * 256 * iters * M.PROBE_CHAINS
    t = np.arange(256)[:, None]
    c = np.arange(M.PROBE_CHAINS)[None, :]
    a0 = 1.0 + 1e-3 * (t + 7 * c)
    an = m ** iters * a0 + b * (1 - m ** iters) / (1 - m)
    ref = an.sum()
    got = out.cpu().numpy()
    assert np.all(np.abs(got[:blocks] - ref) <= 1e-12 * abs(ref))
    assert got[blocks] == -1.0                       # nothing beyond the blocks written
    assert M.lib().mgcccs_fp64_probe(0, 1, 1.0, 0.0, out.data_ptr(), None) == M.EINVAL
    assert M.lib().mgcccs_fp64_probe(1, 0, 1.0, 0.0, out.data_ptr(), None) == M.EINVAL
    assert M.lib().mgcccs_fp64_probe(1, 1, 1.0, 0.0, None, None) == M.EINVAL
