"""One small run of the operators on a preset workload, for profiler captures.

    python -m paper_2406_09144_gb300.profile_case [--workload meerkat1] [--calls 1] [--psf] [--prof]

builds one plan of the workload (synth.observation), then calls R (degrid), R^dag N^-1 (grid)
and, with --psf, the PSF likelihood and gradient, `--calls` times. With --prof it prints the
library's per-class times, algorithmic bytes and launch counts (fr_profile_*).
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="meerkat1")
    ap.add_argument("--calls", type=int, default=1)
    ap.add_argument("--psf", action="store_true")
    ap.add_argument("--prof", action="store_true")
    a = ap.parse_args()
    import torch
    from . import binding as B
    from . import synth
    B.load()
    obs = synth.observation(a.workload)
    plan = B.Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize,
                  weights=obs.weights.astype(np.float32), eps=1e-5, wterm=obs.wterm,
                  nterm=True, mfs=not obs.per_channel_sky, no_psf=not a.psf)
    sky = torch.from_numpy(synth.random_skies(obs.nsky, obs.nx, obs.ny, seed=0)
                           .astype(np.float32)).cuda()
    if a.prof:
        B.profile_enable(True)
    d = None
    for _ in range(a.calls):
        vis = plan.degrid(sky)
        d = plan.grid(vis)
        if a.psf:
            plan.likelihood_grad(sky[None], d[None], want_value=False)
    torch.cuda.synchronize()
    if a.prof:
        print({k: tuple(v) for k, v in B.profile_read().items()})
    print("ok", float(d.abs().max()))


if __name__ == "__main__":
    main()
