"""Serving on the GPU: every job's result is the same alone and in the mix.

Jobs of different image sizes, visibility and channel counts and both kinds run (1) one at a
time with plain launches and (2) through the continuous-batching server (concurrent streams,
CUDA-graph replays, admission by footprint, Poisson arrivals). The outputs must agree to 1e-6
relative L2: the PSF convolution is deterministic; the gridder's atomic flushes may reorder
floating-point additions between runs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# powers of two, and sides on 3 2^k / 5 2^k grids or with a grid above sigma = 2 (100 -> 256)
@pytest.mark.parametrize("sizes", [(64, 128, 256), (96, 160, 100)])
def test_results_alone_equal_results_in_the_mix(sizes):
    from paper_2406_09144_gb300 import build
    from paper_2406_09144_gb300.serve import (GpuExecutor, Scheduler, _copy_requests,
                                              estimate_bytes, make_requests, poisson_arrivals,
                                              run_sequential)
    build.build()
    base = make_requests(12, seed=300, sizes=sizes, nvis_range=(2e3, 6e4), nchan_max=3,
                         ncalls=3)
    alone = run_sequential(_copy_requests(base))
    mix = poisson_arrivals(_copy_requests(base), rate_per_s=400.0, seed=1)
    budget = 3 * max(estimate_bytes(r) for r in base)
    ex = GpuExecutor(graphs=True)
    sch = Scheduler(ex, budget, max_active=4)
    sch.run(mix)
    torch.cuda.synchronize()
    ex.close_finished()
    assert sch.peak_bytes <= budget and sch.peak_active >= 2
    for a, b in zip(alone, mix):
        assert a.rid == b.rid and a.result.shape == b.result.shape
        d = np.linalg.norm(a.result - b.result) / np.linalg.norm(a.result)
        assert d <= 1e-6, (a.rid, a.kind, d)
        assert b.arrival <= b.t_admit <= b.t_done
