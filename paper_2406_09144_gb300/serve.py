"""Continuous-batching imaging server on one GPU.

Requests are imaging jobs of different image sizes, visibility counts and channel counts, of two
kinds, matching the two operator calls of the fast-resolve scheme (Algorithm 1):
  * "psf":   minor-cycle work, the PSF convolution of a batch of skies (Sec. 3.3.2);
  * "major": major-cycle work, R^dagger N^-1 R of a sky (Eq. clean), degridding then gridding.
Each job makes `ncalls` operator applications.

Scheduler (host logic, `Scheduler`):
  * arrivals join a FIFO wait queue;
  * a job is admitted as soon as an execution slot is free and its estimated HBM footprint fits
    the remaining budget (admission by footprint); jobs that arrive while others run are
    admitted as slots and memory free up (continuous batching, not a queue in front of a
    single worker);
  * admitted jobs run concurrently, one CUDA stream per slot, so their work overlaps on the
    device; a finished job releases its slot and memory immediately.

GPU executor (`GpuExecutor`): at admission it builds the job's plan (sorted visibilities, PSF
transfer function; resident until the job retires) and uploads the inputs.
  * PSF-convolution jobs share launches: the calls issued in one scheduling round by jobs with
    the same image size and PSF padding are run together, up to 16 jobs per call, by one
    fr_psf_apply_group (three kernel launches for the whole group instead of three per job),
    on a stream of their own with a caller-owned scratch buffer;
  * major-cycle jobs (degridding then gridding, many launches per call over the w-planes)
    reserve their per-stream workspace without computing (fr_plan_prepare) and capture one call
    into a CUDA graph, so every call is one graph launch on the job's own stream.
`run_sequential` is the baseline: one job at a time, plain per-call launches, one stream.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                      # "psf" or "major"
    uvw: np.ndarray                # [nrow, 3] metres
    freqs: np.ndarray              # [nchan] Hz
    weights: Optional[np.ndarray]  # [nrow, nchan] or None
    nx: int
    ny: int
    pixsize: float
    sky: np.ndarray                # psf: [batch, nsky, nx, ny]; major: [nsky, nx, ny]
    mfs: bool = False
    ncalls: int = 1
    arrival: float = 0.0           # seconds after the start of the run
    # filled in by the scheduler
    t_admit: float = math.nan
    t_done: float = math.nan
    result: Optional[np.ndarray] = None

    @property
    def nvis(self) -> int:
        return self.uvw.shape[0] * len(self.freqs)

    @property
    def nsky(self) -> int:
        return 1 if self.mfs else len(self.freqs)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def estimate_bytes(req: Request) -> int:
    """HBM footprint of a job while it is admitted: plan-resident data, the per-stream workspace,
    the inputs and outputs, and the PSF-build transients during plan creation."""
    from .binding import fft_len_at_least
    n = req.nx * req.ny
    m = req.nvis
    # oversampled grid and PSF-build grid cells (4 n and 16 n for sides of FFT form, more when
    # the grid rounds up to the next transform length)
    g = fft_len_at_least(2 * req.nx) * fft_len_at_least(2 * req.ny)
    gp = fft_len_at_least(4 * req.nx) * fft_len_at_least(4 * req.ny)
    plan = m * 28 + n * 8 + req.nsky * (4 * n * 4 + 2 * n * 4)     # sorted vis, tables, PSF, T
    work = g * 8 + n * 4 * 8 + m * 8                               # grid, half planes, vis buffer
    work += 2 * 4 * g * 8                                          # small-w expansion term grids
    build = gp * 8 + 8 * n * 8 + m * 32                            # PSF-build grid and sort temps
    io = req.sky.size * 4 * 2 + (m * 8 * 2 if req.kind == "major" else 0)
    if req.kind == "psf":
        work += req.sky.shape[0] * req.nsky * n * 8 * 2            # half spectra
    return int(plan + work + max(build, 0) + io)


class Scheduler:
    """FIFO admission by HBM footprint into a fixed number of concurrent slots.

    The executor provides admit(req) -> handle, issue(handle) -> None (launch the next call),
    ready(handle) -> bool (previous work finished), finish(handle) -> None (collect the result
    and release device memory). `clock` is a monotonic time source in seconds.
    """

    def __init__(self, executor, budget_bytes: int, max_active: int = 8,
                 clock: Callable[[], float] = time.perf_counter, realtime: bool = True):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.clock = clock
        self.realtime = realtime
        self.peak_bytes = 0
        self.peak_active = 0
        self.log = []

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            if estimate_bytes(r) > self.budget:
                raise ValueError(f"request {r.rid} needs {estimate_bytes(r)} bytes, budget is {self.budget}")
        pending = collections.deque(reqs)
        waiting = collections.deque()
        active = {}
        used = 0
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            if not self.realtime and not waiting and not active and pending:
                now = max(now, pending[0].arrival)
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # admission: FIFO, while a slot is free and the footprint fits
            while waiting and len(active) < self.max_active and \
                    used + estimate_bytes(waiting[0]) <= self.budget:
                r = waiting.popleft()
                r.t_admit = self.clock() - t0
                h = self.ex.admit(r)
                est = estimate_bytes(r)
                active[r.rid] = [r, h, 0, est]
                used += est
                self.peak_bytes = max(self.peak_bytes, used)
                self.peak_active = max(self.peak_active, len(active))
                self.log.append(("admit", r.rid, r.t_admit, used))
                progressed = True
            # issue the next call of every job whose previous call finished (calls that the
            # executor batches are launched together by flush() below)
            for rid in list(active):
                r, h, done, est = active[rid]
                if not self.ex.ready(h):
                    continue
                if done < r.ncalls:
                    self.ex.issue(h)
                    active[rid][2] = done + 1
                    progressed = True
                else:
                    self.ex.finish(h)
                    r.t_done = self.clock() - t0
                    used -= est
                    del active[rid]
                    self.log.append(("done", rid, r.t_done, used))
                    progressed = True
            flush = getattr(self.ex, "flush", None)
            if flush is not None:
                flush()
            if not progressed:
                if self.realtime and not active and not waiting and pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - (self.clock() - t0))))
                else:
                    time.sleep(0.0002 if self.realtime else 0.0)
        return reqs


def summarize(reqs, wall_s: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    nvis = sum(r.nvis * r.ncalls for r in reqs if r.kind == "major")
    npix = sum(r.sky.size * r.ncalls for r in reqs if r.kind == "psf")
    return {"requests": len(reqs), "wall_s": wall_s, "req_per_s": len(reqs) / wall_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "major_mvis_s": nvis / wall_s / 1e6,
            "psf_mpix_s": npix / wall_s / 1e6}


# ------------------------------------------------------------------------------ GPU executor
class CaptureGate:
    """Keeps device-synchronising cleanup (freeing plans and graphs) apart from stream captures.

    Freeing device memory synchronises the whole device, and a synchronisation while another
    thread is capturing a CUDA graph invalidates that capture. Captures enter shared; cleanup
    enters exclusive, waits for the captures in progress and holds new ones back meanwhile.
    """

    def __init__(self):
        import threading
        self._cv = threading.Condition()
        self._capturing = 0
        self._exclusive = False

    def capture(self):
        return _GateSection(self, exclusive=False)

    def exclusive(self):
        return _GateSection(self, exclusive=True)

    def _enter(self, exclusive: bool):
        with self._cv:
            if exclusive:
                while self._exclusive:
                    self._cv.wait()
                self._exclusive = True
                while self._capturing:
                    self._cv.wait()
            else:
                while self._exclusive:
                    self._cv.wait()
                self._capturing += 1

    def _exit(self, exclusive: bool):
        with self._cv:
            if exclusive:
                self._exclusive = False
            else:
                self._capturing -= 1
            self._cv.notify_all()


class _GateSection:
    def __init__(self, gate: CaptureGate, exclusive: bool):
        self.gate, self.ex = gate, exclusive

    def __enter__(self):
        self.gate._enter(self.ex)
        return self

    def __exit__(self, *exc):
        self.gate._exit(self.ex)
        return False


_PENDING = object()  # a grouped call queued for the next flush


class GpuExecutor:
    """Runs admitted jobs on their own CUDA streams (major cycles: one captured CUDA graph per
    call) and batches the PSF-convolution calls of compatible jobs into shared launches."""

    def __init__(self, device="cuda", graphs: bool = True, eps: float = 1e-5, workers: int = 2,
                 group_psf: bool = True):
        import concurrent.futures
        import threading
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device(self.device.type, torch.cuda.current_device())
        self.graphs = graphs
        self.eps = eps
        self.streams = []
        self.lock = threading.Lock()
        # plan building is host work (validation, uploads, sort); worker threads overlap it with
        # the device work of the jobs already admitted
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=workers)
        self.graveyard = []
        self.graveyard_bytes = 0
        self.graveyard_limit = 32 << 30
        self.gate = CaptureGate()
        self.group_psf = group_psf
        self.pending_psf = []
        # jobs of each PSF group key that have issued calls and not finished: a key's queued
        # calls wait (at most group_wait_s) while another of its jobs still has a call in
        # flight, so jobs that started apart fall into step and share launches
        self.group_members = collections.defaultdict(dict)
        self.group_wait_s = 2e-3
        self.group_stream = None
        self.scratch = None
        # kernel launches per operator call: grouped PSF calls and their jobs, graph kernels
        self.stats = {"group_calls": 0, "group_jobs": 0, "group_kernels": 0,
                      "graph_calls": 0, "graph_kernels": 0}

    def _stream(self):
        with self.lock:
            if self.streams:
                return self.streams.pop()
        return self.torch.cuda.Stream(device=self.device)

    def admit(self, r: Request):
        return {"future": self.pool.submit(self._build, r), "ready": None}

    def _build(self, r: Request):
        torch = self.torch
        from .binding import Plan, launch_count
        torch.cuda.set_device(self.device)
        s = self._stream()
        h = {"req": r, "stream": s, "event": None, "graph": None, "grouped": False, "key": None,
             "graph_kernels": 0}
        with torch.cuda.stream(s):
            plan = Plan(r.uvw, r.freqs, r.nx, r.ny, r.pixsize, weights=r.weights, eps=self.eps,
                        mfs=r.mfs, stream=s)
            sky = torch.as_tensor(np.ascontiguousarray(r.sky), dtype=torch.float32).to(self.device,
                                                                                      non_blocking=True)
            if r.kind == "psf":
                out = torch.empty_like(sky)

                def call():
                    plan.psf_apply(sky, out=out, stream=s)
                if self.group_psf:
                    h["grouped"] = True
                    h["key"] = (r.nx, r.ny) + tuple(plan.psf_padding)
                else:
                    plan.prepare(sky.shape[0], stream=s)
            else:
                vis = torch.empty(plan.vis_shape, dtype=torch.complex64, device=self.device)
                out = torch.empty(plan.sky_shape, dtype=torch.float32, device=self.device)

                def call():
                    plan.degrid(sky, out=vis, stream=s)
                    plan.grid(vis, out=out, stream=s)
                # the per-stream workspace, sized without computing: nothing allocates later
                plan.prepare(1, stream=s)
            if self.graphs and not h["grouped"]:
                g = torch.cuda.CUDAGraph()
                # thread-local capture: other threads keep building plans meanwhile; plan and
                # graph destruction (device-synchronising) waits for the capture to end
                k0 = launch_count()
                with self.gate.capture():
                    g.capture_begin(capture_error_mode="thread_local")
                    try:
                        call()
                    finally:
                        g.capture_end()
                h["graph"] = g
                h["graph_kernels"] = launch_count() - k0
        h.update(plan=plan, sky=sky, out=out, call=call)
        ev = torch.cuda.Event()
        ev.record(s)
        h["event"] = ev
        return h

    def _handle(self, h):
        if h["ready"] is None:
            if not h["future"].done():
                return None
            h["ready"] = h["future"].result()
        return h["ready"]

    def ready(self, hh) -> bool:
        h = self._handle(hh)
        if h is None or h["event"] is _PENDING:
            return False
        return h["event"] is None or h["event"].query()

    def issue(self, hh):
        torch = self.torch
        h = self._handle(hh)
        if h["grouped"]:
            h["event"] = _PENDING  # runs with the other queued PSF calls at a flush
            h["pending_since"] = time.perf_counter()
            self.group_members[h["key"]][id(h)] = h
            self.pending_psf.append(h)
            return
        s = h["stream"]
        with torch.cuda.stream(s):
            if h["graph"] is not None:
                h["graph"].replay()
                self.stats["graph_calls"] += 1
                self.stats["graph_kernels"] += h["graph_kernels"]
            else:
                h["call"]()
            ev = torch.cuda.Event()
            ev.record(s)
            h["event"] = ev

    def flush(self):
        """Runs the queued PSF calls: one grouped call per (image size, PSF padding) and up to
        16 jobs, on the executor's group stream. Every queued job's previous work has finished
        (the scheduler issues a call only once ready() says so), so the group needs no waits."""
        if not self.pending_psf:
            return
        torch = self.torch
        from .binding import psf_apply_group, psf_group_scratch_bytes
        groups = collections.OrderedDict()
        for h in self.pending_psf:
            groups.setdefault(h["key"], []).append(h)
        now = time.perf_counter()
        keep = []
        for key in list(groups):
            hs = groups[key]
            in_flight = any(m["event"] is not _PENDING and m["event"] is not None and
                            not m["event"].query() for m in self.group_members[key].values())
            oldest = min(h["pending_since"] for h in hs)
            if in_flight and len(hs) < 16 and now - oldest < self.group_wait_s:
                keep.extend(hs)  # wait for the job in flight to join
                del groups[key]
        self.pending_psf = keep
        if self.group_stream is None:
            self.group_stream = torch.cuda.Stream(device=self.device)
        gs = self.group_stream
        for hs in groups.values():
            for i in range(0, len(hs), 16):
                part = hs[i:i + 16]
                plans = [h["plan"] for h in part]
                need = psf_group_scratch_bytes(plans, [h["sky"].shape[0] for h in part])
                with torch.cuda.stream(gs):
                    if self.scratch is None or self.scratch.numel() < need:
                        self.scratch = torch.empty(need, dtype=torch.uint8, device=self.device)
                    for h in part:  # used on this stream too: keep them alive until it is done
                        h["sky"].record_stream(gs)
                        h["out"].record_stream(gs)
                    psf_apply_group(plans, [h["sky"] for h in part], [h["out"] for h in part],
                                    self.scratch, stream=gs)
                    ev = torch.cuda.Event()
                    ev.record(gs)
                for h in part:
                    h["event"] = ev
                self.stats["group_calls"] += 1
                self.stats["group_jobs"] += len(part)
                self.stats["group_kernels"] += 3

    def finish(self, hh):
        h = self._handle(hh)
        h["event"].synchronize()
        if h["grouped"]:
            self.group_members[h["key"]].pop(id(h), None)
        h["req"].result = h["out"].cpu().numpy()
        # destroying a plan frees device memory, which synchronises the whole device; finished
        # plans are parked and destroyed together once enough of them accumulate (or at close)
        self.graveyard.append((h["plan"], h["graph"]))
        self.graveyard_bytes += estimate_bytes(h["req"])
        if self.graveyard_bytes > self.graveyard_limit:
            self.close_finished()
        for k in ("graph", "plan", "sky", "out", "call"):
            h[k] = None
        with self.lock:
            self.streams.append(h["stream"])

    def close_finished(self):
        with self.gate.exclusive():
            for plan, _ in self.graveyard:
                plan.close()
            self.graveyard = []  # the graphs are released here too, inside the exclusive section
            self.graveyard_bytes = 0


def run_sequential(requests, device="cuda", eps=1e-5, stats=None):
    """Baseline: each job alone, in arrival order, plain launches on one stream. With a dict
    `stats`, counts the operator calls and their kernel launches."""
    import torch
    from .binding import Plan, launch_count
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        r.t_admit = time.perf_counter() - t0
        plan = Plan(r.uvw, r.freqs, r.nx, r.ny, r.pixsize, weights=r.weights, eps=eps, mfs=r.mfs)
        sky = torch.as_tensor(np.ascontiguousarray(r.sky), dtype=torch.float32).to(device)
        k0 = launch_count()
        for _ in range(r.ncalls):
            if r.kind == "psf":
                out = plan.psf_apply(sky)
            else:
                out = plan.grid(plan.degrid(sky))
        if stats is not None:
            key = "psf" if r.kind == "psf" else "major"
            stats[key + "_calls"] = stats.get(key + "_calls", 0) + r.ncalls
            stats[key + "_kernels"] = stats.get(key + "_kernels", 0) + launch_count() - k0
        r.result = out.cpu().numpy()
        plan.close()
        r.t_done = time.perf_counter() - t0
    return reqs


# ------------------------------------------------------------------------------ workload
def make_requests(n: int, seed: int = 100, sizes=(256, 512, 1024, 2048, 4096),
                  nvis_range=(1e4, 2e7), nchan_max: int = 8, ncalls: int = 8,
                  psf_batch: int = 2) -> list:
    """Serving workload: image sizes uniform over `sizes`, visibility counts log-uniform over
    `nvis_range`, 1..nchan_max channels, half PSF-convolution and half major-cycle jobs, arrays
    and tracks as the VLA-like and MeerKAT-like observations (seeded per request: 100 + i)."""
    from . import synth
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        nx = int(rng.choice(sizes))
        nvis = float(np.exp(rng.uniform(math.log(nvis_range[0]), math.log(nvis_range[1]))))
        nchan = int(rng.integers(1, nchan_max + 1))
        meerkat = bool(rng.integers(0, 2))
        enu = synth.meerkat_like_enu(seed + i) if meerkat else synth.vla_like_enu(seed + i)
        nbl = len(enu) * (len(enu) - 1) // 2
        ntime = max(1, int(round(nvis / nchan / nbl)))
        hours = 8.0
        uvw = synth.earth_rotation_uvw(enu, -30.7 if meerkat else 34.08,
                                       -60.5 if meerkat else 40.7, hours, hours * 3600.0 / ntime)
        f0 = 0.9e9 if meerkat else 1.4e9
        freqs = f0 * (1.0 + 0.1 * np.arange(nchan))
        umax = float(np.max(np.abs(uvw[:, :2]))) * freqs.max() / synth.C_LIGHT
        pix = 1.0 / (2.6 * umax)
        kind = "psf" if rng.integers(0, 2) == 0 else "major"
        mfs = bool(rng.integers(0, 2))
        nsky = 1 if mfs else nchan
        if kind == "psf":
            sky = synth.random_skies(psf_batch * nsky, nx, nx, seed=seed + i).reshape(psf_batch, nsky, nx, nx)
        else:
            sky = synth.random_skies(nsky, nx, nx, seed=seed + i)
        wt = rng.uniform(0.5, 2.0, (uvw.shape[0], nchan)).astype(np.float32)
        out.append(Request(rid=i, kind=kind, uvw=uvw, freqs=freqs, weights=wt, nx=nx, ny=nx,
                           pixsize=pix, sky=sky.astype(np.float32), mfs=mfs, ncalls=ncalls))
    return out


def poisson_arrivals(reqs, rate_per_s: float, seed: int = 7):
    rng = np.random.default_rng(seed)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1.0 / rate_per_s)
        r.arrival = t
    return reqs


# ------------------------------------------------------------------------------ benchmark
def _copy_requests(reqs):
    return [dataclasses.replace(r, result=None, t_admit=math.nan, t_done=math.nan) for r in reqs]


def bench(n: int = 64, max_active: int = 8, budget_gb: float = 96.0, load: float = 0.8,
          seed: int = 100, workers: int = 2, **kw) -> dict:
    """Serving benchmark: (1) plain per-request launches, one job at a time, all jobs present
    at t = 0 -> capacity; (2) the continuous-batching server on the same jobs at t = 0 ->
    throughput; (3) the server under Poisson arrivals at `load` x the sequential capacity ->
    p50 / p99 latency. Returns one dict."""
    import torch
    from .binding import load as load_lib
    load_lib()
    base = make_requests(n, seed=seed, **kw)
    budget = int(budget_gb * 2 ** 30)
    # warm-up: one small job of each kind through both paths (module load, kernel attributes)
    warm = make_requests(2, seed=seed + 10 ** 6, sizes=(64,), nvis_range=(1e3, 2e3), nchan_max=1)
    run_sequential(_copy_requests(warm))
    ex0 = GpuExecutor()
    Scheduler(ex0, budget, max_active).run(_copy_requests(warm))
    ex0.close_finished()
    torch.cuda.synchronize()

    seq = _copy_requests(base)
    seq_stats = {}
    t0 = time.perf_counter()
    run_sequential(seq, stats=seq_stats)
    torch.cuda.synchronize()
    seq_wall = time.perf_counter() - t0
    srv = _copy_requests(base)
    ex1 = GpuExecutor(graphs=True, workers=workers)
    sch = Scheduler(ex1, budget, max_active)
    t0 = time.perf_counter()
    sch.run(srv)
    torch.cuda.synchronize()
    srv_wall = time.perf_counter() - t0
    ex1.close_finished()
    worst = 0.0
    for a, b in zip(seq, srv):
        d = float(np.linalg.norm(a.result - b.result) / max(np.linalg.norm(a.result), 1e-30))
        worst = max(worst, d)
    rate = load * n / seq_wall
    arr = poisson_arrivals(_copy_requests(base), rate, seed=seed)
    ex2 = GpuExecutor(graphs=True, workers=workers)
    sch2 = Scheduler(ex2, budget, max_active)
    t0 = time.perf_counter()
    sch2.run(arr)
    torch.cuda.synchronize()
    arr_wall = time.perf_counter() - t0
    ex2.close_finished()
    s_seq = summarize(seq, seq_wall)
    s_srv = summarize(srv, srv_wall)
    s_arr = summarize(arr, arr_wall)
    st = ex1.stats
    launches = {
        "per_request_psf_kernels_per_call": seq_stats.get("psf_kernels", 0) / max(seq_stats.get("psf_calls", 0), 1),
        "server_psf_kernels_per_call": st["group_kernels"] / max(st["group_jobs"], 1),
        "server_psf_jobs_per_shared_launch": st["group_jobs"] / max(st["group_calls"], 1),
        "per_request_major_kernels_per_call": seq_stats.get("major_kernels", 0) / max(seq_stats.get("major_calls", 0), 1),
        "server_major_kernels_per_call": st["graph_kernels"] / max(st["graph_calls"], 1),
        "server_major_host_launches_per_call": 1.0,
    }
    return {
        "launches": launches,
        "workload": f"{n} jobs, images {kw.get('sizes', (256, 512, 1024, 2048, 4096))}, "
                    f"visibilities log-uniform {kw.get('nvis_range', (1e4, 2e7))}, 1-"
                    f"{kw.get('nchan_max', 8)} channels, half PSF-convolution / half major-cycle, "
                    f"{kw.get('ncalls', 8)} calls per job",
        "sequential": s_seq, "server_closed": s_srv, "server_poisson": s_arr,
        "arrival_rate_per_s": rate, "max_active": max_active, "budget_bytes": budget,
        "peak_admitted_bytes": sch.peak_bytes, "peak_active": sch.peak_active,
        "throughput_gain": s_srv["req_per_s"] / s_seq["req_per_s"],
        "max_rel_diff_alone_vs_mix": worst,
    }


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--workers", type=int, default=2)
    ap.add_argument("--budget-gb", type=float, default=96.0)
    ap.add_argument("--max-size", type=int, default=4096)
    ap.add_argument("--max-nvis", type=float, default=2e7)
    a = ap.parse_args()
    sizes = tuple(s for s in (256, 512, 1024, 2048, 4096) if s <= a.max_size)
    print(json.dumps(bench(a.n, a.max_active, a.budget_gb, sizes=sizes, workers=a.workers,
                           nvis_range=(1e4, a.max_nvis))))
