#!/usr/bin/env python
"""Wall-clock timings of the FP64 oracle on the host's cores (test infrastructure:
the CPU reference of the method, not a product path).

    python oracle/time_oracle.py [--threads N]

small: the whole chain (sky model, every facet, every fit, update), one thread and
N threads.  mid: the whole chain on N threads; one thread on 4 sources (extraction
and fit) plus one source's sky-model term, scaled per source.  batched: the sky
model on every 97th row for all sources, and extraction + fit of 50 sources on
every row, N threads; rates per term and per source.  Prints one JSON line.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

ARC = np.pi / 648000.0


def data_of(wl, obs, cat, n_threads):
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    true = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, cat.alpha_arcsec * ARC,
                            cat.e1, cat.e2, nu_ref=wl.nu_ref_hz, n_threads=n_threads)
    d = np.stack([true.real, true.imag], -1) + synth.noise(obs.n_rows, obs.n_chan, wl.sigma_jy, wl.seed,
                                                          dtype=np.float64)
    return d.astype(np.float32), al


def chain(wl, obs, cat, data, n_threads):
    p = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy, update_mode=1)
    t0 = time.perf_counter()
    oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, data, cat.l, cat.m, cat.flux_jy, None, p,
                    n_threads=n_threads)
    return time.perf_counter() - t0


def per_source_single(wl, obs, cat, data, al, k):
    """One thread: extraction + fit of k sources and one source's sky-model term, per source."""
    p = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy)
    t0 = time.perf_counter()
    for i in range(k):
        du = oracle.facet_du(cat.flux_jy[i], 0.0, p)
        acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, data, np.zeros_like(data), cat.l[i], cat.m[i],
                                   cat.flux_jy[i], al[i], 0.0, 0.0, du, p)
        oracle.fit_facet(acc, du, cat.flux_jy[i], p)
    t1 = time.perf_counter()
    oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l[:1], cat.m[:1], cat.flux_jy[:1], al[:1], np.zeros(1),
                     np.zeros(1), nu_ref=wl.nu_ref_hz, n_threads=1)
    t2 = time.perf_counter()
    # per source: its extraction and fit, plus three model terms (sky model, and the update's two)
    return (t1 - t0) / k + 3 * (t2 - t1)


def main():
    n_threads = int(sys.argv[sys.argv.index("--threads") + 1]) if "--threads" in sys.argv else os.cpu_count()
    oracle.build()
    out = {"host_threads": n_threads}
    # small, in full
    wl = synth.workload("small")
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    data, al = data_of(wl, obs, cat, n_threads)
    t1 = chain(wl, obs, cat, data, 1)
    tn = chain(wl, obs, cat, data, n_threads)
    out["small"] = {"n_src": cat.n_src, "chain_s_1thread": t1, "chain_s_all": tn,
                    "fits_per_s_1thread": cat.n_src / t1, "fits_per_s_all": cat.n_src / tn}
    # mid: in full on every thread; one thread on a sample of sources
    wl = synth.workload("mid")
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    data, al = data_of(wl, obs, cat, n_threads)
    tn = chain(wl, obs, cat, data, n_threads)
    s1 = per_source_single(wl, obs, cat, data, al, 4)
    out["mid"] = {"n_src": cat.n_src, "chain_s_all": tn, "fits_per_s_all": cat.n_src / tn,
                  "s_per_source_1thread_sampled": s1, "fits_per_s_1thread_sampled": 1.0 / s1,
                  "sample_1thread": "4 sources' extraction and fit, one source's sky-model term x 3"}
    del data
    # batched: fixed subsets
    wl = synth.workload("batched")
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    rows = np.arange(0, obs.n_rows, 97)
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    t0 = time.perf_counter()
    oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                     nu_ref=wl.nu_ref_hz, rows=rows, n_threads=n_threads)
    ts = time.perf_counter() - t0
    terms = rows.size * obs.n_chan * cat.n_src
    # extraction + fit of 50 sources over every row, from pure noise (the cost does not depend on the data)
    p = oracle.default_params(nu_ref_hz=wl.nu_ref_hz, sigma_jy=wl.sigma_jy, chunk=0, update_mode=1)
    noise = synth.noise(obs.n_rows, obs.n_chan, wl.sigma_jy, wl.seed)
    sub = slice(0, 50)
    t0 = time.perf_counter()
    oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, noise, cat.l[sub], cat.m[sub], cat.flux_jy[sub], None, p,
                    n_threads=n_threads)
    tp = time.perf_counter() - t0
    out["batched"] = {"sky_model_terms_per_s_all": terms / ts, "sky_model_sample": "every 97th row, all 1000 sources",
                      "chain_50_sources_s_all": tp, "fits_per_s_all_50_sources": 50 / tp,
                      "chain_sample": "50 sources on every row: sky model of those 50, their facets, fits, update"}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
