#!/usr/bin/env python
"""Write batched_chain_oracle.json: the FP64 oracle's chain on the 148,270,080-visibility,
1000-source workload (9,266,880 rows x 16 channels), for two noise levels: sigma = 1 uJy
per component (the benchmark's), and sigma set so the faintest source has an SNR of
about 10.

Data = the oracle's sum of Eq. 1 at the true shapes and scalelengths (simulate_vis, the
sky model arranged for speed; pinned against sky_model) + seeded Gaussian noise, rounded
to complex64.  The chain is the one-chunk form with update mode 1 (Sec. 3.1): every
facet is extracted from the circular sky model (sky_model with e = 0 and the Eq. 4
scalelengths), every facet is fitted (fit_facet), and the final sky model holds every
measured shape; for one chunk this is oracle.pipeline's chain (pinned in
test_oracle_order_pins.py), written out here so that the final sky model is evaluated
only at the 300 sampled rows the test compares.  Only oracle/, synth and the test input
builders are called.  Beside each estimate the script stores the source's two best e
nodes by the alpha-marginal likelihood, their ln L gap, and b^2/(2a) at the MAP point:
at sigma = 1 uJy (source SNR ~1e5) the posterior sits on one node and the precision
form's FP32 model can flip a near-tie between two nodes, which the test then accepts
only within that form's error.  About two and a half hours on 8 cores:

    python tests/golden/make_batched_chain.py
"""
import concurrent.futures as cf
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batched_chain_oracle.json")
N_ROWS_SAMPLED = 300
ROW_SEED = 41


def sampled_rows(n_rows: int) -> np.ndarray:
    return np.sort(np.random.default_rng(ROW_SEED).choice(n_rows, N_ROWS_SAMPLED, replace=False))


def true_data(c) -> np.ndarray:
    """The true sky of the batched workload, [R, C, 2] float64 (all host threads)."""
    return oracle.simulate_vis(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                               c.cat.alpha_arcsec * cases.ARC, c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz)


def data_from_true(true: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    d = true + synth.noise(true.shape[0], true.shape[1], sigma, seed, dtype=np.float64)
    return d.astype(np.float32)


def top_two(fit, qp):
    """The two e nodes (flat index e1 * n_e + e2) of largest alpha-marginal likelihood
    L(e) = sum_k qp_k exp(ln L(e, alpha_k)), ln L(best) - ln L(second), and b^2/(2a) at the
    MAP grid point (the scale of the log-likelihood)."""
    lg = fit.loglike
    fin = np.isfinite(lg)
    if not fin.any():
        return [-1.0, -1.0, 0.0, 0.0]
    # ln L(e) by a log-sum-exp over the scalelength nodes of each e node (no underflow between nodes)
    w = np.where(fin, lg + np.log(qp)[None, None, :], -np.inf)
    m = w.max(axis=2)
    ok = np.isfinite(m)
    lnL = np.full(m.shape, -np.inf)
    lnL[ok] = m[ok] + np.log(np.exp(w[ok] - m[ok][:, None]).sum(axis=1))
    lnL = lnL.reshape(-1)
    order = np.argsort(-lnL, kind="stable")
    b1, b2 = int(order[0]), int(order[1])
    gap = float(lnL[b1] - lnL[b2]) if np.isfinite(lnL[b2]) else 1e300
    g = int(fit.est[oracle.MAP_INDEX])
    a, b = fit.a.reshape(-1)[g], fit.b.reshape(-1)[g]
    return [float(b1), float(b2), gap, float(b * b / (2.0 * a)) if a > 0 else 0.0]


def main():
    c = cases.build(synth.workload("batched"), with_data=False)
    n = c.cat.n_src
    al = c.alpha_med_rad()
    rows = sampled_rows(c.obs.n_rows)
    t0 = time.time()
    true = true_data(c)
    print(f"true sky {time.time() - t0:.0f} s", flush=True)
    t0 = time.time()
    z = np.zeros(n)
    s0 = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy, al, z, z,
                          nu_ref=c.wl.nu_ref_hz)
    sky0 = np.stack([s0.real, s0.imag], -1)
    del s0
    print(f"circular sky model {time.time() - t0:.0f} s", flush=True)
    out = {"workload": "batched", "n_rows": int(c.obs.n_rows), "n_chan": int(c.obs.n_chan), "n_src": int(n),
           "chunk": 0, "update_mode": 1, "rows": rows.tolist(),
           "fields": ["e1", "e2", "sig1", "sig2", "alpha_arcsec", "flux_jy", "flag", "e1_smooth", "e2_smooth",
                      "logl_max", "thresh_margin", "map_index", "n_cells"],
           "variants": {}}
    for name, sigma in (("sigma_1uJy", c.wl.sigma_jy), ("snr10", cases.snr10_sigma(c.obs, c.cat))):
        data = data_from_true(true, sigma, c.wl.seed)
        p = c.oracle_params(sigma_jy=sigma, chunk=0, update_mode=1)
        t0 = time.time()

        def one(i):
            du = oracle.facet_du(c.cat.flux_jy[i], 0.0, p)
            acc = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, data, sky0, c.cat.l[i],
                                       c.cat.m[i], c.cat.flux_jy[i], al[i], 0.0, 0.0, du, p)
            fit = oracle.fit_facet(acc, du, c.cat.flux_jy[i], p)
            return fit.est, top_two(fit, oracle.alpha_weight(p, c.cat.flux_jy[i]))

        with cf.ThreadPoolExecutor(max_workers=os.cpu_count()) as ex:
            res = list(ex.map(one, range(n)))
        est = np.array([r[0] for r in res])
        top2 = [r[1] for r in res]
        print(f"{name}: sigma {sigma:.4g} Jy, extraction and fit {time.time() - t0:.0f} s", flush=True)
        fin, fin_abs = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                                        al, est[:, oracle.E1], est[:, oracle.E2], nu_ref=c.wl.nu_ref_hz,
                                        rows=rows, with_abs=True)
        out["variants"][name] = {
            "sigma_jy": sigma, "fingerprint": cases.fingerprint(data),
            "est": [[float(f"{x:.17g}") for x in row] for row in est],
            "top2_fields": ["best_e_node", "second_e_node", "lnl_gap", "b2_over_2a"],
            "top2": [[float(f"{x:.17g}") for x in row] for row in top2],
            "sky_final_re": [[float(f"{x:.17g}") for x in r] for r in fin.real],
            "sky_final_im": [[float(f"{x:.17g}") for x in r] for r in fin.imag],
            "sky_final_abs": [[float(f"{x:.17g}") for x in r] for r in fin_abs]}
        del data
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
