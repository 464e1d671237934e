#!/usr/bin/env python
"""Throughput of the RadioLensfit hot path on GB300.

One step is one pass of the whole chain over the workload: sky model of the
catalogue, extraction of every facet, likelihood fit of every facet, sky-model
update with the measured shapes (rlf_run, captured as one CUDA graph).  Default
workload: 197 antennas (19306 baselines) x 480 time steps x 16 channels =
148,270,080 visibilities and 1000 sources (the paper's 9,266,880 uv points per
channel), all sources in one chunk, split-phase precision.  Inputs are synthetic
and resident in HBM before the timed region (they exceed L2, so no flush is
needed); the data visibilities are made with the library's own sky-model call at
the catalogue's true shapes and scalelengths plus seeded Gaussian noise.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on every host core instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

ARC = math.pi / 648000.0
METRIC = "source fits/sec (end-to-end: sky model + facet extraction + likelihood fit + sky update)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--chunk", type=int, default=0, help="sources per extract/fit/update step (0: all)")
    ap.add_argument("--precision", default="split", choices=["split", "mixed", "fp64"])
    ap.add_argument("--update-mode", type=int, default=1)
    ap.add_argument("--profile", default="exponential", choices=["exponential", "gaussian"],
                    help="source brightness profile (data and fit)")
    ap.add_argument("--estimator", default="grid", choices=["grid", "adaptive"],
                    help="ellipticity estimator: the fixed grid, or adaptive sampling around the maximum")
    ap.add_argument("--sigma-scale", type=float, default=1.0, help="noise per visibility x this")
    ap.add_argument("--n-pos", type=int, default=1, choices=[1, 3, 5],
                    help="position marginal: offsets per axis (1: catalogue positions exact)")
    ap.add_argument("--pos-step", type=float, default=0.1, help="position marginal: offset step, arcsec")
    ap.add_argument("--pos-error", type=float, default=0.0,
                    help="catalogue positions off the true ones by a seeded uniform offset of up to this, arcsec")
    ap.add_argument("--refit-bad", action="store_true",
                    help="fit the bad fits again after the whole catalogue (times rlf_run calls: not capturable)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time rlf_run calls instead of the captured graph")
    ap.add_argument("--no-tune", action="store_true", help="library default launch shapes")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra lines (the mid workload, and the FP64-phase precision form)")
    ap.add_argument("--mlp-sigma", type=float, default=1e-2,
                    help="noise per visibility component (Jy) of the learned-proposal comparison's data")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mlp", action="store_true", help="skip the learned-proposal comparison")
    ap.add_argument("--n-src", type=int, default=0, help="use only the first N sources (profiling cases)")
    ap.add_argument("--extract-waves", type=int, default=0,
                    help="CTA waves of the extraction (0: the autotuner's choice, or the library default "
                         "with --no-tune or --only)")
    ap.add_argument("--only", default="", choices=["", "sky_model", "extract", "fit", "update", "mlp"],
                    help="run only this entry point --steps times after one warm-up, or only the "
                         "learned-proposal comparison (for ncu captures)")
    ap.add_argument("--mlp-steps", type=int, default=2000, help="training steps of the learned proposal")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (every rank gets it); the job's clock is the slowest replica."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_src: int, world: int, ms: float) -> float:
    """Fits per second of the whole job: every replica fits n_src sources per step."""
    return n_src * world / (ms * 1e-3)


# ---------------------------------------------------------------------------------------------
# CPU arm: the FP64 oracle on a bounded sample


def oracle_chain_sample(wl, obs, cat, params, n_threads, sky_row_stride=194, ext_time_stride=16):
    """CPU cost of the chain on this workload, from a bounded sample, on n_threads host threads.

    The FP64 oracle as it stands (OpenMP over rows for the sky model, one source per
    thread for extraction and fit):
      - sky model of every source on every `sky_row_stride`-th row, scaled by the row ratio;
      - extraction of n_threads sources (evenly spaced in the flux order) on every
        `ext_time_stride`-th time step (all baselines), scaled by the step ratio, and the
        fit of those facets, both scaled to all sources by n_src / n_threads;
      - the sky update counted as two sky models (the new and the old shape of every source).
    Returns (fits/s of the whole chain at full size, seconds of the full chain, wall
    seconds of the sample, description)."""
    import concurrent.futures as cf

    import oracle
    R, C, n = obs.n_rows, obs.n_chan, cat.n_src
    al = np.array([oracle.alpha_med(f) for f in cat.flux_jy]) * ARC
    z = np.zeros(n)
    t_start = time.perf_counter()
    rows = np.arange(0, R, sky_row_stride)
    t0 = time.perf_counter()
    oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, z, z, nu_ref=wl.nu_ref_hz,
                     rows=rows, n_threads=n_threads)
    t_sky = (time.perf_counter() - t0) * R / rows.size
    n_bl = obs.n_bl if obs.n_bl > 0 and R % obs.n_bl == 0 else R
    steps = np.arange(0, R // n_bl, ext_time_stride)
    er = (steps[:, None] * n_bl + np.arange(n_bl)[None, :]).reshape(-1)
    u, v, w = obs.u[er], obs.v[er], obs.w[er]
    rng = np.random.default_rng(5)
    data = rng.standard_normal((er.size, C, 2)).astype(np.float32) * np.float32(1e-5)
    sky = np.zeros_like(data)
    n_sample = max(1, min(n, n_threads))
    picks = np.unique(np.linspace(0, n - 1, n_sample).round().astype(int))

    def extract(i):
        du = oracle.facet_du(cat.flux_jy[i], 0.0, params)
        return oracle.extract_facet(u, v, w, obs.freq_hz, data, sky, cat.l[i], cat.m[i], cat.flux_jy[i], al[i],
                                    0.0, 0.0, du, params), du

    with cf.ThreadPoolExecutor(max_workers=n_threads) as ex:
        t0 = time.perf_counter()
        facets = list(ex.map(extract, picks))
        t_ext = time.perf_counter() - t0
        t0 = time.perf_counter()
        list(ex.map(lambda j: oracle.fit_facet(facets[j][0], facets[j][1], cat.flux_jy[picks[j]], params),
                    range(len(picks))))
        t_fit = time.perf_counter() - t0
    wall = time.perf_counter() - t_start
    scale = n / len(picks)
    total = t_sky + (t_ext * (R / er.size) + t_fit) * scale + 2.0 * t_sky
    desc = ("FP64 oracle on %d host threads: sky model of all %d sources on every %dth row (x%d), "
            "extraction of %d sources evenly spaced in flux on every %dth time step (x%.0f) and their fits, "
            "scaled to %d sources; sky update = 2 sky models; fits/s of the full chain"
            % (n_threads, n, sky_row_stride, sky_row_stride, len(picks), ext_time_stride, R / er.size, n))
    return n / total, total, wall, desc


def oracle_small_full(n_threads):
    """The whole chain of the 10-source, 120,960-visibility workload in full, FP64 oracle: fits/s."""
    import oracle
    wl = synth.workload("small")
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    al = cat.alpha_arcsec * ARC
    d = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                         nu_ref=wl.nu_ref_hz, n_threads=n_threads)
    data = (np.stack([d.real, d.imag], -1) + synth.noise(obs.n_rows, obs.n_chan, wl.sigma_jy, wl.seed,
                                                          dtype=np.float64)).astype(np.float32)
    p = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy, chunk=0, update_mode=1)
    t0 = time.perf_counter()
    oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, data, cat.l, cat.m, cat.flux_jy, None, p, n_threads=n_threads)
    wall = time.perf_counter() - t0
    return {"workload": "small", "n_vis": obs.n_rows * obs.n_chan, "n_src": cat.n_src, "wall_s": wall,
            "fits_per_s": cat.n_src / wall, "cores": n_threads}


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    wl = synth.workload(args.workload)
    obs = synth.make_observation(wl)
    cat = synth.make_catalogue(wl)
    params = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy, n_pos=args.n_pos,
                                   pos_step_arcsec=args.pos_step)
    oracle.build()
    nt = host_threads()
    for _ in range(args.warmup):
        oracle_chain_sample(wl, obs, cat, params, nt)
    vals, walls, fulls = [], [], []
    desc = ""
    for _ in range(args.steps):
        v, full, wall, desc = oracle_chain_sample(wl, obs, cat, params, nt)
        vals.append(v)
        walls.append(wall)
        fulls.append(full)
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "n_vis": obs.n_rows * obs.n_chan, "n_src": cat.n_src,
                       "n_pos": args.n_pos},
            "step": "one bounded sample of the workload per step (ms_per_step is the sample's wall time)",
            "full_chain_s_extrapolated": float(np.mean(fulls)),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "fits/s", "cores": nt, "sample": desc},
            "e2e": {"value": value, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm

TUNE_CACHE = os.path.join(ROOT, "paper_2203_14071_gb300", "_build", "tune_cache.json")


def setup_workload(rlf, torch, dev, name, args, prec, rank, stream, n_src=None):
    """Device inputs of a workload: baselines, catalogue (circular shapes), and data =
    the library's sky model at the true shapes and scalelengths plus seeded noise."""
    wl = synth.workload(name)
    obs_np = synth.make_observation(wl)
    cat_np = synth.make_catalogue(wl, n_src if n_src else (args.n_src if args.n_src > 0 else None))
    R, C, n = obs_np.n_rows, obs_np.n_chan, cat_np.n_src
    t64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    obs = rlf.Observation(t64(obs_np.u), t64(obs_np.v), t64(obs_np.w), obs_np.freq_hz, obs_np.n_bl)
    zeros = torch.zeros(n, dtype=torch.float64, device=dev)
    # the catalogue the chain is given; its positions may be off the true ones (position marginal)
    pos_err = getattr(args, "pos_error", 0.0) * math.pi / 648000.0
    off = np.random.default_rng(4321).uniform(-1.0, 1.0, size=(2, n)) * pos_err
    cat = rlf.Catalogue(t64(cat_np.l + off[0]), t64(cat_np.m + off[1]), t64(cat_np.flux_jy), zeros.clone(),
                        zeros.clone())
    truth = rlf.Catalogue(t64(cat_np.l), t64(cat_np.m), cat.flux_jy, t64(cat_np.e1), t64(cat_np.e2),
                          t64(cat_np.alpha_arcsec))
    sigma = wl.sigma_jy * getattr(args, "sigma_scale", 1.0)
    params = rlf.params_default(nu_ref_hz=wl.nu_ref_hz, sigma_jy=sigma, chunk=args.chunk,
                                precision=prec, update_mode=args.update_mode,
                                profile=rlf.PROFILE_GAUSSIAN if args.profile == "gaussian" else 0,
                                estimator=rlf.ESTIMATOR_ADAPTIVE if getattr(args, "estimator", "grid") == "adaptive"
                                else rlf.ESTIMATOR_GRID, refit_bad=1 if getattr(args, "refit_bad", False) else 0,
                                n_pos=getattr(args, "n_pos", 1), pos_step_arcsec=getattr(args, "pos_step", 0.1))
    ws = rlf.alloc_workspace(R, C, n, params, rlf.WS_RUN, device=dev)
    data = torch.empty(R * C * 2, dtype=torch.float32, device=dev)
    rlf.sky_model(obs, truth, params, data, ws, stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    data += torch.randn(R * C * 2, generator=gen, device=dev, dtype=torch.float32) * sigma
    sky = torch.empty_like(data)
    out = rlf.Results(n, dev)
    return {"wl": wl, "obs_np": obs_np, "cat_np": cat_np, "obs": obs, "cat": cat, "truth": truth,
            "params": params, "ws": ws, "data": data, "sky": sky, "out": out}


def graph_steps_ms(rlf, torch, dev, W, params, stream, steps):
    """ms per step of the captured chain on a workload's resident inputs (after one launch)."""
    g = rlf.Graph(W["obs"], W["data"], W["cat"], params, W["out"], W["sky"], W["ws"], stream)
    g.launch(stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        g.launch(stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    g.close()
    return a.elapsed_time(b) / steps


def extra_workload_line(rlf, torch, dev, args, prec, rank, stream, name, steps=5):
    """Another workload's whole chain (all facets per step, one graph, autotuned shapes)."""
    W = setup_workload(rlf, torch, dev, name, args, prec, rank, stream, n_src=0)
    p = W["params"]
    rlf.autotune(W["obs"], W["data"], W["cat"], p, W["out"], W["sky"], W["ws"], TUNE_CACHE, stream)
    ms = graph_steps_ms(rlf, torch, dev, W, p, stream, steps)
    n = W["cat_np"].n_src
    nv = W["obs_np"].n_rows * W["obs_np"].n_chan
    return {"workload": name, "n_vis": nv, "n_src": n, "ms_per_step": ms, "fits_per_s": n / (ms * 1e-3),
            "tuning": {f: int(getattr(p, f)) for f in rlf.TUNE_FIELDS}, "steps": steps}


def precision_line(rlf, torch, dev, W, stream, prec, steps=5):
    """The same workload and inputs in another precision form (its own workspace and tuned
    launch shapes): ms per step of the captured chain, and the fitted shapes' largest
    difference from the headline run."""
    p = rlf.Params.from_buffer_copy(W["params"])
    p.precision = prec
    R, C, n = W["obs_np"].n_rows, W["obs_np"].n_chan, W["cat_np"].n_src
    ws = rlf.alloc_workspace(R, C, n, p, rlf.WS_RUN, device=dev)
    out = rlf.Results(n, dev)
    V = dict(W, ws=ws, out=out)
    rlf.autotune(W["obs"], W["data"], W["cat"], p, out, W["sky"], ws, TUNE_CACHE, stream)
    ms = graph_steps_ms(rlf, torch, dev, V, p, stream, steps)
    a, b = out.numpy(), W["out"].numpy()
    de = float(np.max(np.maximum(np.abs(a["e1"] - b["e1"]), np.abs(a["e2"] - b["e2"]))))
    del ws
    return {"precision": {0: "fp64", 1: "mixed", 2: "split"}[prec], "ms_per_step": ms,
            "fits_per_s": n / (ms * 1e-3), "max_abs_de_vs_headline": de, "steps": steps,
            "tuning": {f: int(getattr(p, f)) for f in rlf.TUNE_FIELDS}}


def data_at(rlf, torch, dev, W, sigma, seed, stream):
    """Data visibilities of the workload's true sky with noise sigma per component (device)."""
    data = torch.empty_like(W["data"])
    rlf.sky_model(W["obs"], W["truth"], W["params"], data, W["ws"], stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    data += torch.randn(data.numel(), generator=gen, device=dev, dtype=torch.float32) * sigma
    return data


def mlp_line(rlf, torch, dev, W, stream, sigma, train_steps=2000, batch=256, lr=1e-3, lr_min=5e-5, chunk=25,
             reps=5):
    """The learned proposal on this workload: data of the true sky with noise `sigma` per
    component; train the network on facets simulated from the workload's own coverage
    (every source's facet as a template, random shapes, scalelengths from the Eq. 4
    prior; cosine learning-rate decay), then fit the real facets with the narrowed grid
    and with the full grid, timed with CUDA events on the same stream.  The random draws
    of `chunk` steps are made at once."""
    obs, cat, ws, sky = (W[k] for k in ("obs", "cat", "ws", "sky"))
    p = rlf.Params.from_buffer_copy(W["params"])
    p.sigma_jy = sigma
    data = data_at(rlf, torch, dev, W, sigma, 777, stream)
    n = W["cat_np"].n_src
    rlf.sky_model(obs, cat, p, sky, ws, stream)
    fac = torch.empty(rlf.facets_size(n, p) // 8, dtype=torch.float64, device=dev)
    rlf.extract_facets(obs, data, sky, cat, 0, n, p, fac, ws, stream)
    m = rlf.Mlp(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4321)
    m.init(torch.randn(m.P, generator=gen, device=dev), stream)
    ws_t = rlf.mlp_workspace(batch, dev)
    x16 = torch.empty(batch, 8192, dtype=torch.float16, device=dev)
    y = torch.empty(batch, 3, device=dev)
    losses = torch.zeros(train_steps, device=dev)
    flux = cat.flux_jy

    def draws(k):
        tidx = torch.randint(0, n, (k, batch), generator=gen, device=dev, dtype=torch.int32)
        e = torch.randn(k, batch, 2, generator=gen, device=dev, dtype=torch.float64) * 0.3
        e = e * torch.clamp(0.75 / torch.linalg.norm(e, dim=2, keepdim=True), max=1.0)
        lna = p.add + p.esp * torch.log(flux[tidx.long()] * 1e6) + p.r_std * torch.randn(
            k, batch, generator=gen, device=dev, dtype=torch.float64)
        al = torch.clamp(torch.exp(lna), p.r_min_arcsec, p.r_max_arcsec)
        z = torch.randn(k, batch, 2, 4096, generator=gen, device=dev)
        return tidx, e[..., 0].contiguous(), e[..., 1].contiguous(), al, z

    # untimed warm-up on a throwaway network: the first use of the sampling ops and of
    # the training kernels in a fresh process carries one-time costs (seconds) that the
    # timed run must not include
    m_w = rlf.Mlp(dev)
    m_w.init(torch.randn(m_w.P, generator=torch.Generator(device=dev).manual_seed(1), device=dev), stream)
    gen_state = gen.get_state()
    tw, e1w, e2w, alw, zw = draws(2)
    gen.set_state(gen_state)   # the timed run draws what it drew without the warm-up
    for j in range(2):
        rlf.mlp_simulate(fac, flux, tw[j], e1w[j], e2w[j], alw[j], zw[j], p, x16, y, stream)
        rlf.mlp_train_step(m_w, x16, y, lr, j + 1, None, ws_t, stream)
    del m_w
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for c0 in range(0, train_steps, chunk):
        tidx, e1, e2, al, z = draws(min(chunk, train_steps - c0))
        for j in range(tidx.shape[0]):
            s = c0 + j + 1
            lr_s = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * (s - 1) / train_steps))
            rlf.mlp_simulate(fac, flux, tidx[j], e1[j], e2[j], al[j], z[j], p, x16, y, stream)
            rlf.mlp_train_step(m, x16, y, lr_s, s, losses[s - 1:s], ws_t, stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    train_ms = a.elapsed_time(b)
    tail = losses[-min(100, train_steps):].mean().item()
    full, narrow = rlf.Results(n, dev), rlf.Results(n, dev)
    nfb = torch.zeros(1, dtype=torch.int32, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1_.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1_) / reps

    t_full = timed(lambda: rlf.fit_sources(fac, cat, 0, n, p, full, ws, stream))
    t_mlp = timed(lambda: rlf.fit_sources_mlp(fac, cat, 0, n, p, m, narrow, ws, nfb, stream))
    F, G = full.numpy(), narrow.numpy()
    de = np.maximum(np.abs(F["e1"] - G["e1"]), np.abs(F["e2"] - G["e2"]))
    nv = W["obs_np"].n_rows * W["obs_np"].n_chan
    snr = W["cat_np"].flux_jy * math.sqrt(nv) / sigma
    del data, fac
    return {"train": {"steps": train_steps, "batch": batch, "lr": [lr, lr_min], "ms": train_ms,
                      "samples_per_s": train_steps * batch / (train_ms * 1e-3), "nll_last_100": tail},
            "sigma_jy": sigma, "snr_range": [float(snr.min()), float(snr.max())],
            "fit_full_ms": t_full, "fit_mlp_ms": t_mlp, "fit_speedup": t_full / t_mlp,
            "fits_per_s_full": n / (t_full * 1e-3), "fits_per_s_mlp": n / (t_mlp * 1e-3),
            "fallbacks": int(nfb.item()), "n_src": n, "agree_1e-4": float(np.mean(de <= 1e-4)),
            "max_abs_de": float(de.max()), "n_bad_full": int(np.sum(F["flag"] & 1)), "box": [7, 7, 5]}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist

    import paper_2203_14071_gb300 as rlf
    from paper_2203_14071_gb300 import build_ext

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        build_ext.build()
    if world > 1:
        dist.barrier()
    rlf.lib()

    stream = torch.cuda.Stream(dev)    # a non-default stream: the chain is captured as a CUDA graph
    torch.cuda.set_stream(stream)
    prec = {"split": rlf.PREC_MIXED_SPLIT, "mixed": rlf.PREC_MIXED, "fp64": rlf.PREC_FP64}[args.precision]
    W = setup_workload(rlf, torch, dev, args.workload, args, prec, rank, stream)
    obs_np, cat_np, obs, cat, params, ws, data, sky, out = (W[k] for k in (
        "obs_np", "cat_np", "obs", "cat", "params", "ws", "data", "sky", "out"))
    n_src, R, C = cat_np.n_src, obs_np.n_rows, obs_np.n_chan
    n_vis = R * C
    wl_head = W["wl"]

    if args.only == "mlp":
        print(json.dumps({"only": "mlp", "mlp_proposal": mlp_line(rlf, torch, dev, W, stream, args.mlp_sigma,
                                                                    train_steps=args.mlp_steps)}))
        return
    if args.only:
        profile_only(args, rlf, torch, obs, data, cat, params, ws, sky, out, stream, dev, n_src)
        return

    tuning = None if args.no_tune else rlf.autotune(obs, data, cat, params, out, sky, ws, TUNE_CACHE, stream)
    if args.extract_waves > 0:
        params.tune_extract_waves = args.extract_waves
    graph = None if (args.no_graph or args.refit_bad) else rlf.Graph(obs, data, cat, params, out, sky, ws, stream)

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            rlf.run(obs, data, cat, params, out, sky, ws, stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    code, status = rlf.read_status(ws, stream)
    if code != rlf.RLF_OK:
        raise RuntimeError(f"device status {status}: {rlf.strerror(code)}")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    res = out.numpy()          # the chain's results (the entry-point timings below reuse `out`)

    # per-kernel timing of the dominant phases (same stream, CUDA events), and e2e
    comp = component_times(rlf, torch, obs, data, cat, params, ws, sky, out, stream, dev, args, n_src)
    clocks.stop()
    ms = max_over_ranks(ms, world, dev)

    e2e = None if args.no_e2e else e2e_time(rlf, torch, obs_np, data, cat, params, ws, sky, out, stream, dev, args)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = rlf.peaks_measure(stream)
    value = whole_job_value(n_src, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f64", 1: "f32+f64", 2: "f32 (phase as f32 pairs)"}[prec], "data": "synthetic",
        "config": {"workload": args.workload, "n_ant": obs_np.n_ant, "n_baselines": obs_np.n_bl,
                   "n_time": obs_np.n_time, "n_chan": C, "n_vis": n_vis, "n_src": n_src,
                   "facet_n": params.facet_n, "grid": [params.n_e, params.n_e, params.n_alpha],
                   "chunk": args.chunk if args.chunk > 0 else n_src, "precision": args.precision,
                   "update_mode": args.update_mode, "profile": args.profile, "estimator": args.estimator,
                   "sigma_jy": params.sigma_jy, "refit_bad": bool(args.refit_bad),
                   "n_pos": args.n_pos, "pos_step_arcsec": args.pos_step, "pos_error_arcsec": args.pos_error,
                   "l2": "inputs larger than L2 (no flush)"},
        "sky_model_gvis_s": comp["sky_gvis_s"],
        "fit_only_fits_per_s": n_src / (comp["phases_ms"]["fit"] * 1e-3),
        "phases_ms": comp["phases_ms"],
        "mean_cells_per_facet": comp["mean_cells_per_facet"],
        "gpu_launches": (comp["launches_per_step"] + refit_launches(params, res, n_src)) * args.steps,
        "clocks": clocks.summary(),
        "measured_unit_peaks": peaks,
        "fits": {"n_bad": int(np.sum(res["flag"] & 1)), "n_invalid": int(np.sum(res["flag"] & 2)),
                 "refinements": np.bincount((res["flag"] >> 8) & 15, minlength=6).tolist(),
                 "n_refit": int(np.sum((res["flag"] & 8) != 0))},
    }
    line["roofline"], line["rooflines"] = roofline(comp, peaks, params, n_vis, n_src, R, C, workload=args.workload)
    line["launch"] = {"graph": graph is not None, "tuning": None if tuning is None else
                      {f: int(getattr(params, f)) for f in rlf.TUNE_FIELDS}}
    if graph is not None:
        graph.close()
    if not args.no_extra and world == 1 and prec == rlf.PREC_MIXED_SPLIT:
        # the FP64-phase form (FP64 phase argument, tile-sum accumulation and normalisation)
        line["precision_mixed"] = precision_line(rlf, torch, dev, W, stream, rlf.PREC_MIXED)
    if not args.no_mlp and world == 1 and args.n_pos == 1:
        line["mlp_proposal"] = mlp_line(rlf, torch, dev, W, stream, args.mlp_sigma, train_steps=args.mlp_steps)
    if not args.no_extra and world == 1 and args.workload != "mid":
        del ws, data, sky, W
        torch.cuda.empty_cache()
        line["mid_workload"] = extra_workload_line(rlf, torch, dev, args, prec, rank, stream, "mid")
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl_head, obs_np, cat_np, args.n_pos, args.pos_step)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profile_only(args, rlf, torch, obs, data, cat, params, ws, sky, out, stream, dev, n_src):
    """One entry point alone (after the chain ran once), for profiler captures."""
    if args.extract_waves > 0:
        params.tune_extract_waves = args.extract_waves
    facets = torch.empty(rlf.facets_size(n_src, params) // 8, dtype=torch.float64, device=dev)
    ws_fit = rlf.alloc_workspace(obs.n_rows, obs.n_chan, n_src, params, rlf.WS_FIT, device=dev)
    rlf.run(obs, data, cat, params, out, sky, ws, stream)
    rlf.extract_facets(obs, data, sky, cat, 0, n_src, params, facets, ws, stream)
    calls = {"sky_model": lambda: rlf.sky_model(obs, cat, params, sky, ws, stream),
             "extract": lambda: rlf.extract_facets(obs, data, sky, cat, 0, n_src, params, facets, ws, stream),
             "fit": lambda: rlf.fit_sources(facets, cat, 0, n_src, params, out, ws_fit, stream),
             "update": lambda: rlf.sky_update(obs, cat, 0, n_src, out.e1, out.e2, None, params, sky, ws, stream)}
    fn = calls[args.only]
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    print(json.dumps({"only": args.only, "n_src": n_src, "ms_per_call": a.elapsed_time(b) / args.steps}))


def component_times(rlf, torch, obs, data, cat, params, ws, sky, out, stream, dev, args, n_src):
    """Each entry point timed alone with CUDA events on the launching stream."""
    reps = max(3, args.steps)
    facets = torch.empty(rlf.facets_size(n_src, params) // 8, dtype=torch.float64, device=dev)
    ws_fit = rlf.alloc_workspace(obs.n_rows, obs.n_chan, n_src, params, rlf.WS_FIT, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    sky_ms = timed(lambda: rlf.sky_model(obs, cat, params, sky, ws, stream))
    ext_ms = timed(lambda: rlf.extract_facets(obs, data, sky, cat, 0, n_src, params, facets, ws, stream))
    fit_ms = timed(lambda: rlf.fit_sources(facets, cat, 0, n_src, params, out, ws_fit, stream))
    # likelihood evaluations of the fit: valid grid points x non-empty cells, per source
    nn = params.facet_n * params.facet_n
    n_cells = (facets.view(n_src, 4, nn)[:, 2, :] > 0).sum(dim=1).double()
    ge = -params.e_max + np.arange(params.n_e) * (2.0 * params.e_max / (params.n_e - 1))
    n_valid = int((np.add.outer(ge ** 2, ge ** 2) < 1.0).sum()) * params.n_alpha
    fit_evals = float(n_cells.sum().item()) * n_valid
    in_window = float(facets.view(n_src, 4, nn)[:, 2, :].sum().item())
    upd_ms = timed(lambda: rlf.sky_update(obs, cat, 0, n_src, out.e1, out.e2, None, params, sky, ws, stream))
    chunk = params.chunk if params.chunk > 0 else n_src
    n_chunks = (n_src + chunk - 1) // chunk
    # kernels of one rlf_run step: prepare + sky model; outside FP64 mode the baseline extents,
    # their order (rows = time x baselines) and the split baselines (split mode); per chunk:
    # residual (batched chunks only; several chunks in mixed modes keep the residual resident:
    # one difference before the chunks and one after), window reach per source (outside FP64 mode), extraction,
    # partial reduce, compaction, LPT order, persistent fit, prepare + sky update (one chunk:
    # prepare of the committed shapes + their sky model instead; memsets and copies are not
    # kernels of ours)
    mixed = params.precision != 0
    is_ordered = obs.n_baselines > 0 and obs.n_rows % obs.n_baselines == 0
    track = n_chunks > 1 and mixed and (obs.n_rows * obs.n_chan) % 2 == 0
    per_chunk = (7 + (1 if chunk >= 3 and mixed and not track else 0) + (1 if mixed else 0) + (1 if n_chunks == 1 else 0)
                 + (1 if params.estimator == 1 else 0))
    launches = (2 + (1 if mixed else 0) + (1 if mixed and is_ordered else 0)
                + (1 if params.precision == 2 else 0) + (2 if track else 0) + n_chunks * per_chunk)
    return {"phases_ms": {"sky_model": sky_ms, "extract": ext_ms, "fit": fit_ms, "update": upd_ms},
            "sky_gvis_s": obs.n_rows * obs.n_chan / (sky_ms * 1e-3) / 1e9, "launches_per_step": launches,
            "fit_evals": fit_evals, "mean_cells_per_facet": float(n_cells.mean().item()),
            "in_window_pairs": in_window}


# Algorithmic operation counts per unit of work: FP32 ops and MUFU ops per unit, plus
# per (row, source) overheads of the phase argument (its float-pair form).  Per unit:
#   sky-model term: 1 sin + 1 cos of the phase and 1 rsqrt of the profile (3 MUFU), ~10 FP32;
#   update term: the new and the old model (2 rsqrt) and one phase (sin, cos): 4 MUFU, ~13 FP32;
#   extraction pair (a visibility inside the source's window): the shift's sin + cos and
#     the model's rsqrt (3 MUFU), ~16 FP32;
#   likelihood evaluation (grid point x cell): 1 rsqrt, ~6 FP32.
OPS = {
    "sky_model": {"fp32": 10.0, "mufu": 3.0, "fp32_rs": 50.0, "mufu_rs": 4.0, "unit": "Gterm/s"},
    "update": {"fp32": 13.0, "mufu": 4.0, "fp32_rs": 50.0, "mufu_rs": 4.0, "unit": "Gterm/s"},
    "extract": {"fp32": 16.0, "mufu": 3.0, "fp32_rs": 50.0, "mufu_rs": 4.0, "unit": "Gpair/s"},
    "fit": {"fp32": 6.0, "mufu": 1.0, "fp32_rs": 0.0, "mufu_rs": 0.0, "unit": "Geval/s"},
}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# per (kernel, workload), kept in the profile summaries; valid while the kernel's source files
# hash to the recorded value, otherwise the bench reports null.
TRAFFIC = {
    ("extract", "batched"): (("csrc/extract.cu", "csrc/rlf_internal.cuh"), "7cc6a69279ac7e5f", 14.137e9 + 380.73e6),
}


def source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2203_14071_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_of(name, workload=None):
    key = (name, workload)
    if key not in TRAFFIC:
        return None
    files, digest, nbytes = TRAFFIC[key]
    return nbytes if source_hash(files) == digest else None


def refit_launches(params, res, n_src):
    """Kernels of the refit pass: the bad list, then per chunk of refitted sources: prepare,
    residual (three or more sources, when the sky model is not resident as a residual),
    window reach, extraction, partial reduce, compaction, LPT order, persistent fit
    (+ adaptive sampling), scatter, prepare + sky update."""
    if not params.refit_bad:
        return 0
    nb = int(np.sum((res["flag"] & 8) != 0))
    if nb == 0:
        return 1
    chunk = params.chunk if params.chunk > 0 else n_src
    per = 11 + (1 if params.estimator == 1 else 0)
    launches = 1
    for first in range(0, nb, chunk):
        cnt = min(chunk, nb - first)
        launches += per + (1 if cnt >= 3 and chunk >= n_src else 0)
    return launches


def roofline_one(name, t_ms, units, row_src, peaks, fp32=None, workload=None):
    """ALU roofline: the shortest time the FP32 and MUFU budgets allow for the
    algorithmic op counts, against the measured unit rates."""
    o = dict(OPS[name])
    if fp32 is not None:
        o["fp32"] = fp32
    fp32_rate = max(peaks["fp32_fma_per_s"], peaks.get("fp32x2_fma_per_s", 0.0))
    mufu_rate = min(peaks["mufu_rsqrt_per_s"], peaks["mufu_sin_per_s"])
    t_fp32 = (o["fp32"] * units + o["fp32_rs"] * row_src) / fp32_rate
    t_mufu = (o["mufu"] * units + o["mufu_rs"] * row_src) / mufu_rate
    t_min = max(t_fp32, t_mufu)
    t = t_ms * 1e-3
    traffic = traffic_of(name, workload)
    line = {"kernel": name, "bound": "alu", "limiting_unit": "fp32" if t_fp32 >= t_mufu else "mufu",
            "unit": o["unit"], "achieved": units / t / 1e9, "peak": units / t_min / 1e9, "frac": t_min / t,
            "units_per_launch": units, "traffic": traffic,
            "peak_basis": "measured FP32 %.3g FMA/s and MUFU %.3g op/s (rlf_peaks_measure)" % (fp32_rate, mufu_rate)}
    # the memory side beside it: the captured DRAM bytes per launch over this launch's time,
    # against the measured copy bandwidth
    hbm = hbm_peak_gbs()
    if traffic is not None and hbm:
        line["dram_gb_s"] = traffic / t / 1e9
        line["hbm_frac_of_measured"] = traffic / t / 1e9 / hbm
    return line


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def roofline(comp, peaks, params, n_vis, n_src, R, C, workload=None):
    ph = comp["phases_ms"]
    out = {}
    for name in ("sky_model", "update"):
        out[name] = roofline_one(name, ph[name], float(n_vis) * n_src, float(R) * n_src, peaks, workload=workload)
    # extraction: the algorithmic work is the terms that enter a facet (visibility-source pairs
    # inside the source's window); pairs outside need no arithmetic, and the (row, source)
    # phase work is counted in the same proportion
    frac_in = comp["in_window_pairs"] / (float(n_vis) * n_src)
    out["extract"] = roofline_one("extract", ph["extract"], comp["in_window_pairs"], float(R) * n_src * frac_in, peaks,
                                  workload=workload)
    # the fit's FP32 ops per evaluation: the brightness (3), a (2) and one b per position offset
    nj = params.n_pos * params.n_pos if params.n_pos > 1 else 1
    out["fit"] = roofline_one("fit", ph["fit"], float(comp["fit_evals"]), 0.0, peaks, fp32=5.0 + nj, workload=workload)
    dom = max(ph, key=ph.get)
    return out[dom], out


def e2e_time(rlf, torch, obs_np, data, cat, params, ws, sky, out, stream, dev, args):
    """Same step through the public API with host buffers: every step uploads its inputs
    from pinned host memory and reads the fitted shapes back.  Two device input buffers
    and a copy stream: the upload of step k + 1 runs during the chain of step k (each
    upload waits for the timed region's start, and for the step that last used its
    buffer), so the timed region holds every step's copies and the copies overlap the
    compute."""
    n = cat.n_src
    h_data = data.cpu().pin_memory()
    h_uvw = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (obs_np.u, obs_np.v, obs_np.w)]
    # the catalogue (positions, fluxes, the initial circular shapes) is uploaded every step too
    h_cat = [x.cpu().pin_memory() for x in (cat.l, cat.m, cat.flux_jy, cat.e1, cat.e2)]
    bufs = []
    for _ in range(2):
        d_uvw = [torch.empty_like(x, device=dev) for x in h_uvw]
        d_data = torch.empty_like(data)
        d_cat = [torch.empty_like(x, device=dev) for x in h_cat]
        bufs.append((d_uvw, d_data, rlf.Observation(d_uvw[0], d_uvw[1], d_uvw[2], obs_np.freq_hz, obs_np.n_bl),
                     d_cat, rlf.Catalogue(*d_cat)))
    h_out = torch.empty((2, n), dtype=torch.float64).pin_memory()
    # the chain of each input buffer as a captured graph (rlf_graph_*), else rlf_run calls
    graphs = None
    if not (args.no_graph or params.refit_bad):
        graphs = [rlf.Graph(bf[2], bf[1], bf[4], params, out, sky, ws, stream) for bf in bufs]
    copy_stream = torch.cuda.Stream(dev)
    ev_copy = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(i, after):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(after)
            for h, d in zip(h_uvw, bufs[i][0]):
                d.copy_(h, non_blocking=True)
            for h, d in zip(h_cat, bufs[i][3]):
                d.copy_(h, non_blocking=True)
            bufs[i][1].copy_(h_data, non_blocking=True)
            ev_copy[i].record(copy_stream)

    def run_steps(k_steps, start):
        upload(0, start)
        if k_steps > 1:
            upload(1, start)
        for k in range(k_steps):
            i = k % 2
            stream.wait_event(ev_copy[i])
            if graphs:
                graphs[i].launch(stream)
            else:
                rlf.run(bufs[i][2], bufs[i][1], bufs[i][4], params, out, sky, ws, stream)
            h_out[0].copy_(out.e1, non_blocking=True)
            h_out[1].copy_(out.e2, non_blocking=True)
            ev_done[i].record(stream)
            if k + 2 < k_steps:
                upload(i, ev_done[i])

    w = torch.cuda.Event()
    w.record(stream)
    run_steps(2, w)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run_steps(args.steps, a)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.steps
    if graphs:
        for g in graphs:
            g.close()
    h2d = h_data.numel() * 4 + sum(x.numel() * 8 for x in h_uvw) + sum(x.numel() * 8 for x in h_cat)
    return {"value": n / (ms * 1e-3), "unit": "fits/s", "ms_per_step": ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 2 * n * 8, "graph": graphs is not None,
            "inputs": "data visibilities, u/v/w and the catalogue (l, m, flux, initial shapes) uploaded every "
                      "step from pinned host memory; the fitted e1, e2 read back",
            "overlap": "uploads on a second stream, two input buffers"}


def cpu_baseline(wl, obs_np, cat_np, n_pos=1, pos_step=0.1):
    import oracle
    params = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy, n_pos=n_pos,
                                   pos_step_arcsec=pos_step)
    oracle.build()
    nt = host_threads()
    value, full, wall, desc = oracle_chain_sample(wl, obs_np, cat_np, params, nt)
    return {"value": value, "unit": "fits/s", "cores": nt, "kind": "oracle", "wall_s": wall,
            "full_chain_s_extrapolated": full, "sample": desc, "small_workload_in_full": oracle_small_full(nt)}


if __name__ == "__main__":
    main()
