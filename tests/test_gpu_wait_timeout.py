"""The error path of the bounded device waits, exercised without a fault.

Every spin on an mbarrier in the library's kernels gives up after a bounded number of polls,
records ST_TIMEOUT in the plan's status word and returns with nothing in flight; fr_plan_check
then reports FR_ETIMEOUT. fr_selftest_wait_timeout launches one CTA that arms its barrier for a
transfer the way the degridder does but issues no copy, so the wait runs out (a flag that
nothing sets). The test checks the status, that it is cleared, and that the context still
runs the operators correctly afterwards.
"""
import numpy as np
import pytest

from paper_2406_09144_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    from paper_2406_09144_gb300 import build
    from paper_2406_09144_gb300.binding import FR_ETIMEOUT, FastResolveError, Plan, load
    build.build()
    lib = load()
    obs = synth.random_observation(600, 1, 32, 32, 2e-3, seed=80, wmax_cycles=1.0)
    plan = Plan(obs.uvw, obs.freqs, 32, 32, obs.pixsize, weights=obs.weights, eps=1e-5)
    sky = torch.tensor(synth.random_skies(1, 32, 32, seed=1), dtype=torch.float32, device="cuda")
    before = plan.grid(plan.degrid(sky)).cpu().numpy()
    plan.check()  # nothing recorded yet
    stream = torch.cuda.current_stream()
    import ctypes
    assert lib.fr_selftest_wait_timeout(plan._h, ctypes.c_void_p(stream.cuda_stream)) == 0
    with pytest.raises(FastResolveError) as e:
        plan.check()
    assert e.value.code == FR_ETIMEOUT
    plan.check()  # the status word was cleared
    after = plan.grid(plan.degrid(sky)).cpu().numpy()
    torch.cuda.synchronize()
    assert np.linalg.norm(after - before) <= 1e-6 * np.linalg.norm(before)
