#!/usr/bin/env python
"""Benchmark of the fast-resolve measurement-operator hot path on synthetic data.

Default workload: MeerKAT-like multi-channel, 8 channels of 4096^2 skies at 2" (64 antennas,
856-1712 MHz, 8 h at 8 s = 58,060,800 visibilities, w-terms, natural weights, eps = 1e-5;
PSF convolutions on 8192^2 padded grids). One step is
    R          (degrid the 8 skies to model visibilities)
    R^dag N^-1 (grid the data visibilities to 8 dirty images)
    the PSF likelihood and its gradient (8 PSF convolutions on the padded grids).
Inputs are resident in HBM before timing; L2 is flushed (512 MB write) between timed steps,
outside the timed events. value = grid+degrid Mvis/s = N_vis / (t_degrid + t_grid) over the
whole job. With --gpus N the channels are split over the ranks (per-channel skies are
independent imaging problems, so nothing is exchanged; strong scaling: the job is the same at
every N, N = 1 included); a single-channel workload runs one copy per rank (weak scaling).

Side legs on the same JSON line: the PSF passes against the HBM roofline, the fast-resolve
likelihood and one exact major cycle, reduced PSF padding, FR_DETERMINISTIC gridding, Tab. 2's
3600^2 field, a bounded serving run (p50/p99 latency and throughput against plain per-request
launches), the end-to-end rate through host buffers, and the FP64 oracle on the host cores.

--impl reference times the FP64 CPU oracle (direct sums) on the host cores on a bounded
sample of the same workload and reports the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid+degrid Mvis/s"
UNIT = "Mvis/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fastresolve", choices=["fastresolve", "reference"])
    ap.add_argument("--workload", default="meerkat", choices=["meerkat", "vla", "small", "meerkat1"])
    ap.add_argument("--no-serving", action="store_true", help="skip the bounded serving leg")
    ap.add_argument("--serving-jobs", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the 3600^2 (non-power-of-two) side measurement")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_desc(obs, name):
    return {
        "workload": {
            "vla": "VLA-like single channel: 1024^2 sky at 0.1 arcsec, 27 antennas (351 baselines), "
                   "8 h at 2 s, 5,054,400 complex64 visibilities with w-terms, natural weights, "
                   "FP32 NUFFT eps 1e-5; PSF convolution on the 2048^2 padded grid",
            "small": "plain method, small: 128^2 sky, 1 channel at 1.4 GHz, 27 antennas, 4 h at 10 s "
                     "(505,440 visibilities), w = 0; PSF on the 256^2 padded grid",
            "meerkat": "MeerKAT-like multi-channel: 4096^2 sky per channel at 2 arcsec, 64 antennas, "
                       "8 channels 856-1712 MHz, 8 h at 8 s (58,060,800 visibilities), w-terms; "
                       "PSF convolution on 8192^2 padded grids",
            "meerkat1": "MeerKAT-like top channel alone: 4096^2 sky at 2 arcsec, 64 antennas, "
                        "1658.5 MHz, 8 h at 8 s (7,257,600 visibilities), w-terms; PSF convolution "
                        "on the 8192^2 padded grid",
        }[name],
        "nx": obs.nx, "ny": obs.ny, "nchan": obs.nchan, "nrow": obs.nrow, "nvis": obs.nvis,
        "pixsize_rad": obs.pixsize, "eps": 1e-5,
        "step": "R (degrid) + R^dag N^-1 (grid) + PSF likelihood/gradient",
        "l2": "flushed between timed steps (512 MB write, outside the timed events)",
    }


# ------------------------------------------------------------------------------ CPU oracle
def cpu_psf_fft_rate(nx, ny, psf, sky, reps=3):
    """CPU comparison of the PSF convolution: FP64 scipy.fft on all host cores, the padded
    2nx x 2ny real transforms of Sec. 3.3.2 (transfer function precomputed, as in the plan).
    Returns (Mpix/s, cores)."""
    import scipy.fft as sf
    cores = os.cpu_count() or 1
    P = np.asarray(psf, dtype=np.float64)
    T = sf.rfft2(np.fft.ifftshift(P), workers=cores)
    s = np.asarray(sky, dtype=np.float64)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        out = sf.irfft2(T * sf.rfft2(s, s=(2 * nx, 2 * ny), workers=cores),
                        s=(2 * nx, 2 * ny), workers=cores)[:nx, :ny]
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    del out
    return nx * ny / best / 1e6, cores


def oracle_rate(obs, sky, seconds, seed=0):
    """Time the FP64 direct-sum oracle on a bounded sample; return (Mvis/s, sample text, cores).

    Degridding one visibility costs one O(N_pix) sum; gridding one pixel costs one O(N_vis)
    sum. The whole-job rate is N_vis / (N_vis * tau_vis + N_pix * tau_pix)."""
    from oracle import cdft
    cdft.build()
    rng = np.random.default_rng(seed)
    npix = obs.nx * obs.ny
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    from paper_2406_09144_gb300 import synth
    vis = synth.complex_gaussian((obs.nrow, obs.nchan), seed=1)
    w32 = obs.weights.astype(np.float32)

    def measure(nv, npx):
        rows = rng.integers(0, obs.nrow, nv)
        chans = rng.integers(0, obs.nchan, nv)
        t0 = time.perf_counter()
        cdft.degrid_at(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, rows, chans,
                       wterm=obs.wterm)
        tv = time.perf_counter() - t0
        pix = rng.integers(0, npix, npx)
        imgs = rng.integers(0, obs.nsky, npx)
        t0 = time.perf_counter()
        cdft.grid_at(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, obs.nx, obs.ny, imgs, pix,
                     weights=w32, nsky=obs.nsky, wterm=obs.wterm)
        tp = time.perf_counter() - t0
        return tv / nv, tp / npx

    # a small pilot sizes the sample to about `seconds` of CPU work, split between directions
    tau_v, tau_p = measure(16, 2)
    nv = max(16, int(0.5 * seconds / max(tau_v, 1e-9)))
    npx = max(2, int(0.5 * seconds / max(tau_p, 1e-9)))
    tau_v, tau_p = measure(nv, npx)
    total = obs.nvis * tau_v + npix * tau_p
    rate = obs.nvis / total / 1e6
    # direct-DFT terms per second (one term = one visibility-pixel phase and product)
    terms = {"degrid_terms_per_s": npix / tau_v, "grid_terms_per_s": obs.nvis / tau_p}
    sample = (f"{nv} visibilities (each a {npix}-pixel FP64 direct sum) and {npx} pixels (each a "
              f"{obs.nvis}-visibility sum) of the workload; rate = N_vis / (N_vis t_vis + N_pix t_pix); "
              f"direct-DFT terms/s: degrid {terms['degrid_terms_per_s']:.3g}, "
              f"grid {terms['grid_terms_per_s']:.3g}")
    return rate, sample, cores


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_digest():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2406_09144_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(category, workload):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(category)
    if not e or e.get("source") != source_digest():
        return None
    return float(e["dram_bytes_per_launch"])


# ------------------------------------------------------------------------------ reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_2406_09144_gb300 import synth
    obs = synth.observation(args.workload)
    sky = synth.random_skies(obs.nsky, obs.nx, obs.ny, seed=0)
    rates = []
    per = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup):
        oracle_rate(obs, sky, per, seed=100 + i)
    t0 = time.perf_counter()
    sample = cores = None
    for i in range(args.steps):
        r, sample, cores = oracle_rate(obs, sky, per, seed=i)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = float(statistics.median(rates))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True,
        "scaling": "strong" if obs.per_channel_sky and obs.nchan >= ws else "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_desc(obs, args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step: {sample}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2406_09144_gb300 import build, synth
    from paper_2406_09144_gb300 import binding as B
    build.build()
    B.load()

    from paper_2406_09144_gb300 import shard
    obs_full = synth.observation(args.workload)
    # per-channel skies split by channel over the ranks (no exchange); a single-channel
    # workload runs one copy per rank
    sharded = ws > 1 and obs_full.per_channel_sky and obs_full.nchan >= ws
    # the multi-channel job is fixed whatever the rank count (strong scaling, N = 1 included)
    fixed_job = obs_full.per_channel_sky and obs_full.nchan >= ws
    if sharded:
        c0, c1 = shard.channel_shard(obs_full.nchan, ws, rank)
        obs = shard.channel_slice(obs_full, c0, c1)
        job_vis, job_pix = obs_full.nvis, obs_full.nsky * obs_full.nx * obs_full.ny
    else:
        obs = obs_full
        job_vis, job_pix = ws * obs.nvis, ws * obs.nsky * obs.nx * obs.ny
    w32 = obs.weights.astype(np.float32)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = B.Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=w32, eps=1e-5,
                  wterm=obs.wterm, nterm=True, mfs=not obs.per_channel_sky)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    info = plan.info()

    sky_h = synth.random_skies(obs.nsky, obs.nx, obs.ny, seed=0).astype(np.float32)
    vis_h = synth.complex_gaussian((obs.nrow, obs.nchan), seed=1).astype(np.complex64)
    sky = torch.from_numpy(sky_h).to(dev)
    vis = torch.from_numpy(vis_h).to(dev)
    model = torch.empty(plan.vis_shape, dtype=torch.complex64, device=dev)
    dirty = plan.grid(vis)
    grad = torch.empty_like(dirty)
    resid = torch.empty_like(dirty)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step(evs):
        evs[0].record(stream)
        plan.degrid(sky, out=model)
        evs[1].record(stream)
        plan.grid(vis, out=resid)
        evs[2].record(stream)
        plan.likelihood_grad(sky, dirty, grad=grad, want_value=False)
        evs[3].record(stream)

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(args.warmup):
        flush.zero_()
        step(mk())
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    B.profile_enable(True)
    B.launch_count(reset=True)
    events = []
    for _ in range(args.steps):
        flush.zero_()
        e = mk()
        step(e)
        events.append(e)
    torch.cuda.synchronize()
    launches = B.launch_count()
    if ws > 1:
        dist.barrier()
    cats = B.profile_read()
    B.profile_enable(False)
    clk = clocks.stop()

    t_deg = sum(e[0].elapsed_time(e[1]) for e in events)
    t_grd = sum(e[1].elapsed_time(e[2]) for e in events)
    t_psf = sum(e[2].elapsed_time(e[3]) for e in events)
    t_step = sum(e[0].elapsed_time(e[3]) for e in events)
    times = torch.tensor([t_deg + t_grd, t_psf, t_step], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
    t_dg, t_psf, t_step = (float(x) for x in times.cpu())
    value = job_vis * args.steps / (t_dg * 1e-3) / 1e6
    psf_mpix = job_pix * args.steps / (t_psf * 1e-3) / 1e6

    # roofline of the dominant kernel class
    dom = max(cats, key=lambda k: cats[k][0])
    dms, dby, dn = cats[dom]
    peak, peak_kind = measured_peaks()
    achieved = (dby / dn) / (dms / dn * 1e-3) / 1e9 if dn else 0.0
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dom, args.workload),
                "algorithmic_bytes_per_launch": dby / max(dn, 1),
                "avg_launch_ms": dms / max(dn, 1), "launches": int(dn),
                "share_of_step": dms / max(t_step, 1e-9)}
    # the PSF path (P1/P2/P3 of the likelihood call in the step) against the same HBM peak,
    # with the bytes it moves per sky pixel against the 16 B/px minimum of a PSF convolution
    psf_ms = sum(cats[k][0] for k in ("psf_rows", "psf_cols") if k in cats)
    psf_by = sum(cats[k][1] for k in ("psf_rows", "psf_cols") if k in cats)
    psf_ach = psf_by / (psf_ms * 1e-3) / 1e9 if psf_ms else 0.0
    roofline_psf = {"bound": "hbm", "kernel": "PSF passes P1, P2, P3 (likelihood and gradient)",
                    "achieved": psf_ach, "peak": peak, "peak_source": f"{peak_kind} hbm_gbs",
                    "unit": "GB/s", "frac": psf_ach / peak,
                    "bytes_per_px": psf_by / (obs.nsky * obs.nx * obs.ny * args.steps),
                    "min_bytes_per_px": 16.0, "passes_ms_per_step": psf_ms / args.steps}
    # the visibility kernels are bound by FP32 issue, not HBM: their multiply-add rate against
    # the FP32 peak (152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s, nominal unit counts
    # and the maximum SM clock). Flops: 4 per footprint cell (a complex times a real weight,
    # two FMAs) for every term or w-plane a visibility visits.
    visits = info["wplanes_max"] if info["dw"] == 0.0 else info["support"]
    cells = info["support"] ** 2
    alu = {}
    for k in ("grid", "degrid"):
        if k in cats and cats[k][2]:
            flops = obs.nvis * visits * cells * 4.0
            tf = flops / (cats[k][0] / args.steps * 1e-3) / 1e12
            alu[k] = {"bound": "alu", "achieved": tf, "peak": 80.5, "unit": "TFLOP/s",
                      "frac": tf / 80.5, "flops_per_step": flops,
                      "peak_source": "nominal FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz"}
    kernels = {k: {"ms": v[0] / args.steps, "launches": int(v[2]) // args.steps,
                   "GBps": (v[1] / (v[0] * 1e-3) / 1e9) if v[0] > 0 else None}
               for k, v in cats.items() if v[2]}

    # the fast-resolve minor-cycle likelihood (Eq. ham_new): noise kernel fitted once (untimed),
    # then value + gradient per call; and one exact major cycle (Alg. 1) for comparison
    eps_noise = 1e-4 * float(w32.astype(np.float64).sum()) / obs.nchan
    plan.noise_fit(eps_noise)
    fgrad = torch.empty_like(dirty)
    for _ in range(2):
        plan.fast_likelihood_grad(sky, dirty, grad=fgrad, want_value=False)
        plan.major_cycle(sky, dirty, want_resid=True)
    torch.cuda.synchronize()
    t_fast = t_major = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        plan.fast_likelihood_grad(sky, dirty, grad=fgrad, want_value=False)
        b.record(stream)
        plan.major_cycle(sky, dirty, want_resid=True)
        c.record(stream)
        c.synchronize()
        t_fast += a.elapsed_time(b)
        t_major += b.elapsed_time(c)
    minor_major = {"fast_likelihood_ms": t_fast / args.steps,
                   "fast_likelihood_mpix_s": obs.nsky * obs.nx * obs.ny / (t_fast / args.steps * 1e-3) / 1e6,
                   "major_cycle_ms": t_major / args.steps,
                   "eps_noise": eps_noise}

    # reduced padding (Sec. 3.3.2): the PSF likelihood on lx x ly padded grids, the PSF
    # truncated to the window they hold, against the full 2nx x 2ny padding; a batch of skies
    # larger than L2, rate and bytes of the PSF passes, and the truncation error
    reduced = None
    if rank == 0:
        nb = max(1, 32 // obs.nsky)
        skies = torch.from_numpy(np.stack([synth.sky_image(obs.nx, obs.ny, seed=100 + i)
                                           for i in range(nb)]).astype(np.float32)[:, None]
                                 .repeat(obs.nsky, axis=1)).to(dev)
        dirt = skies.flip(-1).contiguous()
        gb = torch.empty_like(skies)
        rows = []
        ref_out = None
        lengths = [(L, L2) for L, L2 in zip(B.padded_lengths(obs.nx), B.padded_lengths(obs.ny))]
        for lx, ly in reversed(lengths):  # full padding first: the reference output
            plan.set_psf_padding(lx, ly)
            out = plan.psf_apply(skies)
            for _ in range(3):
                plan.likelihood_grad(skies, dirt, grad=gb, want_value=False)
            torch.cuda.synchronize()
            B.profile_enable(True)
            t = 0.0
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                plan.likelihood_grad(skies, dirt, grad=gb, want_value=False)
                b.record(stream)
                b.synchronize()
                t += a.elapsed_time(b)
            pc = B.profile_read()
            B.profile_enable(False)
            pms = sum(pc[k][0] for k in ("psf_rows", "psf_cols") if k in pc)
            pby = sum(pc[k][1] for k in ("psf_rows", "psf_cols") if k in pc)
            npx_all = nb * obs.nsky * obs.nx * obs.ny * args.steps
            if ref_out is None:
                ref_out = out.clone()
            err = float(torch.linalg.vector_norm((out - ref_out).double()) /
                        torch.linalg.vector_norm(ref_out.double()))
            ms = t / args.steps
            rows.append({"lx": lx, "ly": ly,
                         "window": [min(lx - obs.nx, obs.nx - 1), min(ly - obs.ny, obs.ny - 1)],
                         "likelihood_ms": ms,
                         "mpix_s": nb * obs.nsky * obs.nx * obs.ny / (ms * 1e-3) / 1e6,
                         "psf_passes_GBps": pby / (pms * 1e-3) / 1e9 if pms else None,
                         "psf_passes_frac_of_measured_hbm": (pby / (pms * 1e-3) / 1e9 / peak)
                         if pms else None,
                         "rel_err_vs_full_padding": err,
                         # bytes the three passes move per sky pixel, against the 16 B/px
                         # minimum of a PSF convolution (4 in, 4 out, 8 transfer)
                         "psf_bytes_per_px": pby / npx_all if npx_all else None})
        plan.set_psf_padding(2 * obs.nx, 2 * obs.ny)
        # library comparison (not the product path): the same batch of PSF convolutions with
        # cuFFT through torch.fft on the 2nx x 2ny padded grid, against fr_psf_apply
        Pimg = plan.dirty_psf(want_dirty=False)[1]
        Tc = torch.fft.rfft2(torch.fft.ifftshift(Pimg, dim=(-2, -1)))
        outp = torch.empty_like(skies)

        def cufft_apply():
            F = torch.fft.rfft2(skies, s=(2 * obs.nx, 2 * obs.ny))
            return torch.fft.irfft2(F * Tc, s=(2 * obs.nx, 2 * obs.ny))[..., :obs.nx, :obs.ny]

        cmp = {}
        for name, fn in (("fr_psf_apply", lambda: plan.psf_apply(skies, out=outp)),
                         ("cufft_torch", cufft_apply)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            t = 0.0
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = fn()
                b.record(stream)
                b.synchronize()
                t += a.elapsed_time(b)
            cmp[name + "_ms"] = t / args.steps
        cmp["rel_diff"] = float(torch.linalg.vector_norm((outp - r).double()) /
                                torch.linalg.vector_norm(r.double()))
        reduced = {"batch": nb, "sky": "point+blob skies, one per batch element",
                   "rows": rows, "psf_apply_vs_cufft": cmp}
        del skies, dirt, gb, out, ref_out
        torch.cuda.synchronize()

    # FR_DETERMINISTIC on the same workload: R^dag with fixed-point accumulation (bitwise
    # reproducible) against the default float atomics
    det = None
    if rank == 0:
        pd = B.Plan(obs.uvw, obs.freqs, obs.nx, obs.ny, obs.pixsize, weights=w32, eps=1e-5,
                    wterm=obs.wterm, nterm=True, mfs=not obs.per_channel_sky, no_psf=True,
                    deterministic=True)
        dd = torch.empty_like(dirty)
        for _ in range(2):
            pd.grid(vis, out=dd)
        torch.cuda.synchronize()
        tdet = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pd.grid(vis, out=dd)
            b.record(stream)
            b.synchronize()
            tdet += a.elapsed_time(b)
        ref = plan.grid(vis)
        det = {"grid_ms": tdet / args.steps, "default_grid_ms": t_grd / args.steps,
               "rel_diff_vs_default": float(torch.linalg.vector_norm((dd - ref).double()) /
                                            torch.linalg.vector_norm(ref.double()))}
        del pd, dd, ref
        torch.cuda.synchronize()

    # an image side that is not a power of two: Tab. 2's field, 3600^2 pixels of 2", with the
    # MeerKAT-like top channel (7,257,600 visibilities, w-stacking) on an 8192^2 grid
    tab2 = None
    if rank == 0 and not args.no_sizes:
        o3 = synth.observation("meerkat1", npix=3600)
        t0 = time.perf_counter()
        p3 = B.Plan(o3.uvw, o3.freqs, o3.nx, o3.ny, o3.pixsize, weights=o3.weights, eps=1e-5,
                    wterm=o3.wterm, mfs=not o3.per_channel_sky)
        torch.cuda.synchronize()
        p3_s = time.perf_counter() - t0
        i3 = p3.info()
        s3 = torch.from_numpy(synth.random_skies(o3.nsky, o3.nx, o3.ny, seed=3)
                              .astype(np.float32)).to(dev)
        v3 = torch.from_numpy(synth.complex_gaussian((o3.nrow, o3.nchan), seed=4)
                              .astype(np.complex64)).to(dev)
        m3 = torch.empty(p3.vis_shape, dtype=torch.complex64, device=dev)
        d3 = torch.empty(p3.sky_shape, dtype=torch.float32, device=dev)
        c3 = torch.empty_like(d3)
        for _ in range(2):
            p3.degrid(s3, out=m3)
            p3.grid(v3, out=d3)
            p3.psf_apply(s3, out=c3)
        torch.cuda.synchronize()
        td = tg = tp = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            p3.degrid(s3, out=m3)
            e[1].record(stream)
            p3.grid(v3, out=d3)
            e[2].record(stream)
            p3.psf_apply(s3, out=c3)
            e[3].record(stream)
            e[3].synchronize()
            td += e[0].elapsed_time(e[1])
            tg += e[1].elapsed_time(e[2])
            tp += e[2].elapsed_time(e[3])
        k = args.steps
        tab2 = {"workload": "MeerKAT-like top channel (1658.5 MHz, 7,257,600 visibilities, w-terms) "
                            "imaged at 3600^2 pixels of 2 arcsec (Tab. 2's field)",
                "grid": [i3["grid_nu"], i3["grid_nv"]], "psf_padding": list(p3.psf_padding),
                "wplanes_total": i3["wplanes_total"], "plan_s": p3_s,
                "degrid_ms": td / k, "grid_ms": tg / k,
                "mvis_s": o3.nvis / ((td + tg) / k * 1e-3) / 1e6,
                "psf_apply_ms": tp / k,
                "psf_apply_mpix_s": o3.nsky * o3.nx * o3.ny / (tp / k * 1e-3) / 1e6}
        del p3, s3, v3, m3, d3, c3
        torch.cuda.synchronize()

    # end to end through the C ABI with host buffers: H2D sky + vis, R and R^dag, D2H results
    e2e = None
    if True:
        sky_p = torch.from_numpy(sky_h).pin_memory()
        vis_p = torch.from_numpy(vis_h).pin_memory()
        model_p = torch.empty(plan.vis_shape, dtype=torch.complex64).pin_memory()
        dirty_p = torch.empty(plan.sky_shape, dtype=torch.float32).pin_memory()
        sky_d = torch.empty_like(sky)
        vis_d = torch.empty_like(vis)
        out_d = torch.empty_like(dirty)

        # copies overlap the kernels on a second stream: the visibilities upload while R runs,
        # and R's model visibilities download while R^dag runs
        copy_s = torch.cuda.Stream(device=dev)

        def e2e_step():
            sky_d.copy_(sky_p, non_blocking=True)
            copy_s.wait_stream(stream)
            with torch.cuda.stream(copy_s):
                vis_d.copy_(vis_p, non_blocking=True)
            vis_ready = torch.cuda.Event()
            vis_ready.record(copy_s)
            plan.degrid(sky_d, out=model)
            model_ready = torch.cuda.Event()
            model_ready.record(stream)
            stream.wait_event(vis_ready)
            plan.grid(vis_d, out=out_d)
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(model_ready)
                model_p.copy_(model, non_blocking=True)
            dirty_p.copy_(out_d, non_blocking=True)
            stream.wait_stream(copy_s)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        tt = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            tt += a.elapsed_time(b)
        tt_t = torch.tensor([tt], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(tt_t, op=dist.ReduceOp.MAX)
        tt = float(tt_t.item())
        e2e = {"value": job_vis * args.steps / (tt * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(sky_h.nbytes + vis_h.nbytes),
               "d2h_bytes_per_step": int(model.numel() * 8 + dirty.numel() * 4),
               "path": "pinned host sky + visibilities -> fr_degrid, fr_grid -> pinned host model "
                       "visibilities + dirty image; the visibility upload and the model download "
                       "overlap the kernels on a second stream"}

    # serving (continuous batching): a bounded mix of imaging jobs through the server against
    # plain per-request launches, closed-loop throughput and p50/p99 latency under Poisson
    # arrivals at 80 % of the per-request capacity
    serving = None
    if rank == 0 and not args.no_serving:
        from paper_2406_09144_gb300 import serve
        del model, grad, resid
        torch.cuda.empty_cache()
        sv = serve.bench(args.serving_jobs, max_active=16, workers=4, sizes=(256, 512, 1024, 2048),
                          nvis_range=(1e4, 5e6))
        pa = sv["server_poisson"]
        serving = {"workload": sv["workload"], "throughput_gain": sv["throughput_gain"],
                   "server_jobs_per_s": sv["server_closed"]["req_per_s"],
                   "per_request_jobs_per_s": sv["sequential"]["req_per_s"],
                   "p50_ms": pa.get("p50_ms"), "p99_ms": pa.get("p99_ms"),
                   "arrival_rate_per_s": sv["arrival_rate_per_s"],
                   "max_rel_diff_alone_vs_mix": sv["max_rel_diff_alone_vs_mix"], "detail": sv}
        torch.cuda.synchronize()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        r, sample, cores = oracle_rate(obs, sky_h.astype(np.float64), args.cpu_seconds)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        psf_np = plan.dirty_psf(want_dirty=False)[1][0].cpu().numpy()
        pr, pc_ = cpu_psf_fft_rate(obs.nx, obs.ny, psf_np, sky_h[0])
        cpu["psf_apply_fft"] = {"value": pr, "unit": "Mpix/s", "cores": pc_,
                                "kind": "FP64 scipy.fft on the padded grid (comparison)",
                                "sample": f"one {obs.nx}x{obs.ny} sky, best of 3"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step / args.steps, "higher_is_better": True,
            "scaling": "strong" if fixed_job else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded antenna layout, Earth-rotation tracks, point+blob skies, "
                    "Gaussian visibilities)",
            "config": workload_desc(obs, args.workload),
            "psf_apply_mpix_s": psf_mpix,
            "degrid_ms": t_deg / args.steps if ws == 1 else None,
            "grid_ms": t_grd / args.steps if ws == 1 else None,
            "psf_likelihood_ms": t_psf / args.steps,
            "plan_s": plan_s,
            "plan": {k: info[k] for k in ("support", "wplanes_total", "work_items", "grid_nu")},
            "minor_major": minor_major, "psf_reduced_padding": reduced, "size_3600": tab2,
            "deterministic": det,
            "roofline_alu": alu,
            "roofline": roofline, "roofline_psf": roofline_psf, "serving": serving,
            "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
