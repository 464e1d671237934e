#!/usr/bin/env python
"""Write mid_precision_oracle.json: the FP64 oracle's estimates for every source of the
37,067,520-visibility, 200-source workload, for the two noise levels the precision
table uses: sigma = 1 uJy per component, and sigma set so the faintest source has an
SNR of about 10.

Data = the oracle's sky model at the true shapes + seeded Gaussian noise, rounded
to complex64; the chain runs with all sources in one chunk (extraction from the
circular sky model, Sec. 3.1) and update mode 1.  Only oracle/, synth and the test
input builders are called.  Takes a few minutes on 8 cores:

    python tests/golden/make_mid_precision.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from tests import cases  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mid_precision_oracle.json")


def main():
    c = cases.build(synth.workload("mid"), with_data=False)
    t0 = time.time()
    true = cases.true_sky(c)
    print(f"true sky {time.time() - t0:.0f} s", flush=True)
    out = {"workload": "mid", "n_rows": int(c.obs.n_rows), "n_chan": int(c.obs.n_chan),
           "n_src": int(c.cat.n_src), "chunk": 0, "update_mode": 1,
           "fields": ["e1", "e2", "sig1", "sig2", "alpha_arcsec", "flux_jy", "flag", "e1_smooth", "e2_smooth",
                      "logl_max", "thresh_margin", "map_index", "n_cells"],
           "variants": {}}
    for name, sigma in (("sigma_1uJy", c.wl.sigma_jy), ("snr10", cases.snr10_sigma(c.obs, c.cat))):
        data = cases.data_from(true, sigma, c.wl.seed)
        t0 = time.time()
        est = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, data, c.cat.l, c.cat.m, c.cat.flux_jy,
                              None, c.oracle_params(sigma_jy=sigma, chunk=0, update_mode=1))
        print(f"{name}: sigma {sigma:.4g} Jy, pipeline {time.time() - t0:.0f} s", flush=True)
        out["variants"][name] = {"sigma_jy": sigma, "fingerprint": cases.fingerprint(data),
                                 "est": [[float(f"{x:.17g}") for x in row] for row in est]}
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
