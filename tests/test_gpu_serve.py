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


def test_grouped_psf_convolution_equals_per_plan_calls():
    """fr_psf_apply_group: the PSF convolutions of several plans (equal image size and padding,
    different PSFs, sky counts and batches) in one launch per pass equal each plan's own
    fr_psf_apply."""
    from paper_2406_09144_gb300 import build, synth
    from paper_2406_09144_gb300.binding import (FastResolveError, Plan, psf_apply_group,
                                                psf_group_scratch_bytes)
    build.build()
    nx, ny = 96, 64
    plans, skies = [], []
    for j, (nchan, mfs, batch) in enumerate([(1, True, 2), (3, False, 1), (2, True, 3)]):
        obs = synth.random_observation(900 + 100 * j, nchan, nx, ny, 2e-3, seed=90 + j)
        p = Plan(obs.uvw, obs.freqs, nx, ny, obs.pixsize, weights=obs.weights, eps=1e-5, mfs=mfs)
        plans.append(p)
        skies.append(torch.tensor(synth.random_skies(batch * p.nsky, nx, ny, seed=20 + j)
                                  .reshape(batch, p.nsky, nx, ny), dtype=torch.float32,
                                  device="cuda"))
    need = psf_group_scratch_bytes(plans, [s.shape[0] for s in skies])
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    outs = [torch.full_like(s, float("nan")) for s in skies]
    psf_apply_group(plans, skies, outs, scratch)
    for p, s, o in zip(plans, skies, outs):
        ref = p.psf_apply(s)
        d = (torch.linalg.vector_norm((o - ref).double()) / torch.linalg.vector_norm(ref.double()))
        assert float(d) <= 1e-6, float(d)
    # plans of another image size cannot share the launches
    obs = synth.random_observation(500, 1, 64, 64, 2e-3, seed=99)
    other = Plan(obs.uvw, obs.freqs, 64, 64, obs.pixsize, eps=1e-5)
    sk = torch.zeros((1, 1, 64, 64), device="cuda")
    with pytest.raises(FastResolveError):
        psf_apply_group([plans[0], other], [skies[0], sk], [outs[0], sk.clone()], scratch)


def test_server_shares_psf_launches_across_jobs():
    """PSF-convolution calls that jobs of one image size issue together run as one shared
    launch per pass (one grouped call for all of them), with results equal to the jobs run
    alone; then the jobs go on through the scheduler."""
    from paper_2406_09144_gb300 import build
    from paper_2406_09144_gb300.serve import (GpuExecutor, _copy_requests, make_requests,
                                              run_sequential)
    build.build()
    base = [r for r in make_requests(24, seed=500, sizes=(128,), nvis_range=(2e3, 2e4),
                                     nchan_max=2, ncalls=4) if r.kind == "psf"]
    assert 4 <= len(base) <= 16
    alone = run_sequential(_copy_requests(base))
    mix = _copy_requests(base)
    ex = GpuExecutor(graphs=True)
    hs = [ex.admit(r) for r in mix]
    while not all(ex.ready(h) for h in hs):
        pass
    for h in hs:  # every job issues its first call in the same round
        ex.issue(h)
    ex.flush()
    assert ex.stats["group_calls"] == 1 and ex.stats["group_jobs"] == len(base), ex.stats
    for r, h in zip(mix, hs):  # the remaining calls through the scheduler's loop
        for _ in range(r.ncalls - 1):
            while not ex.ready(h):
                ex.flush()
            ex.issue(h)
        while not ex.ready(h):
            ex.flush()
        ex.finish(h)
    torch.cuda.synchronize()
    ex.close_finished()
    assert ex.stats["group_jobs"] == sum(r.ncalls for r in base)
    for a, b in zip(alone, mix):
        d = np.linalg.norm(a.result - b.result) / np.linalg.norm(a.result)
        assert d <= 1e-6, (a.rid, d)
