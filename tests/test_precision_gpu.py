"""Per-source error table of the GPU chain against the FP64 oracle on the
37,067,520-visibility, 200-source workload, for the three precision forms (FP64;
FP32 model with FP64 phase and sums; FP32 model with the phase as FP32 pairs).

The oracle's estimates come from tests/golden/mid_precision_oracle.json (written by
make_mid_precision.py beside it, which calls only the oracle).  The data visibilities
are rebuilt here from the oracle's sky model and the seeded noise, and checked
against the fingerprint stored with the estimates.  Set RLF_REPORT_DIR to also write
the per-source table as CSV.
"""
import csv
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import cases

pytestmark = pytest.mark.gpu

GOLD_PATH = os.path.join(os.path.dirname(__file__), "golden", "mid_precision_oracle.json")
N_VIS_ROWS = 512


@pytest.fixture(scope="module")
def rlf():
    import torch
    assert torch.cuda.is_available()
    import paper_2203_14071_gb300 as m
    from paper_2203_14071_gb300 import build_ext
    build_ext.build()
    m.lib()
    return m


@pytest.fixture(scope="module")
def gold():
    with open(GOLD_PATH) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def mid_true():
    c = cases.build(synth.workload("mid"), with_data=False)
    return c, cases.true_sky(c)


def _precs(rlf):
    return {"fp64": rlf.PREC_FP64, "mixed": rlf.PREC_MIXED, "split": rlf.PREC_MIXED_SPLIT}


@pytest.fixture(scope="module")
def vis_errors(rlf, mid_true):
    """max over sampled rows and channels of |V_gpu - V_oracle| / S for each source's own
    model (true shape and scalelength), per precision form."""
    import torch
    c, _ = mid_true
    rows = np.sort(np.random.default_rng(31).choice(c.obs.n_rows, N_VIS_ROWS, replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    obs, _ = cases.to_device(c)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    R, C, n = c.obs.n_rows, c.obs.n_chan, c.cat.n_src
    out = {}
    vis = torch.empty(R * C * 2, dtype=torch.float32, device="cuda")
    for name, prec in _precs(rlf).items():
        p = rlf.params_default(nu_ref_hz=c.wl.nu_ref_hz, precision=prec)
        ws = rlf.alloc_workspace(R, C, 1, p, rlf.WS_SKY)
        err = np.zeros(n)
        for j in range(n):
            cj = rlf.Catalogue(t(c.cat.l[j:j + 1]), t(c.cat.m[j:j + 1]), t(c.cat.flux_jy[j:j + 1]),
                               t(c.cat.e1[j:j + 1]), t(c.cat.e2[j:j + 1]), t(c.cat.alpha_arcsec[j:j + 1]))
            rlf.sky_model(obs, cj, p, vis, ws)
            got = vis.view(R, C, 2)[rows_t].cpu().numpy().astype(np.float64)
            ref = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l[j:j + 1], c.cat.m[j:j + 1],
                                   c.cat.flux_jy[j:j + 1], c.cat.alpha_arcsec[j:j + 1] * cases.ARC,
                                   c.cat.e1[j:j + 1], c.cat.e2[j:j + 1], nu_ref=c.wl.nu_ref_hz, rows=rows)
            err[j] = np.max(np.abs(got[..., 0] + 1j * got[..., 1] - ref)) / c.cat.flux_jy[j]
        out[name] = err
        del ws
    return out


@pytest.mark.parametrize("variant", ["snr10", "sigma_1uJy"])
def test_precision_table(rlf, gold, mid_true, vis_errors, variant):
    import torch
    c, true = mid_true
    g = gold["variants"][variant]
    sigma = g["sigma_jy"]
    data = cases.data_from(true, sigma, c.wl.seed)
    fp, gfp = cases.fingerprint(data), g["fingerprint"]
    # sampled values bit for bit; the float64 sums to 1e-9 (numpy's pairwise summation
    # groups terms differently on different SIMD widths)
    assert fp["values"] == gfp["values"]
    assert math.isclose(fp["sum"], gfp["sum"], rel_tol=1e-9, abs_tol=1e-9)
    assert math.isclose(fp["sum_sq"], gfp["sum_sq"], rel_tol=1e-9)
    est = np.array(g["est"])
    R, C, n = c.obs.n_rows, c.obs.n_chan, c.cat.n_src
    d = cases.vis_tensor(data)
    table, summary = [], {}
    for name, prec in _precs(rlf).items():
        obs, cat = cases.to_device(c)
        p = rlf.params_default(nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=sigma, precision=prec, chunk=0, update_mode=1)
        ws = rlf.alloc_workspace(R, C, n, p, rlf.WS_RUN)
        out = rlf.Results(n, "cuda")
        sky = torch.empty(R * C * 2, dtype=torch.float32, device="cuda")
        rlf.run(obs, d, cat, p, out, sky, ws)
        res = out.numpy()
        del ws, sky
        de = np.array([cases.est_matches(res, i, est[i]) for i in range(n)])
        da = np.abs(res["alpha_arcsec"] - est[:, oracle.ALPHA])
        ds = np.abs(res["flux_jy"] - est[:, oracle.FLUX]) / est[:, oracle.FLUX]
        flag_same = (res["flag"] & 1) == (est[:, oracle.FLAG] != 0)
        for i in range(n):
            table.append({"variant": variant, "precision": name, "source": i, "flux_jy": c.cat.flux_jy[i],
                          "e1_oracle": est[i, oracle.E1], "e2_oracle": est[i, oracle.E2],
                          "e1": res["e1"][i], "e2": res["e2"][i], "abs_de": de[i],
                          "alpha_oracle": est[i, oracle.ALPHA], "abs_dalpha": da[i], "rel_dflux": ds[i],
                          "flag_same": bool(flag_same[i]), "thresh_margin": est[i, oracle.THRESH_MARGIN],
                          "vis_err_rel": vis_errors[name][i]})
        summary[name] = {"max_de": float(de.max()), "median_de": float(np.median(de)),
                         "n_de_gt_1e-4": int(np.sum(de > 1e-4)), "max_abs_dalpha": float(da.max()),
                         "max_rel_dflux": float(ds.max()), "n_flag_diff": int(np.sum(~flag_same)),
                         "max_vis_err_rel": float(vis_errors[name].max()),
                         "n_bad": int(np.sum(res["flag"] & 1))}
    print(f"\n{variant} (sigma {sigma:.4g} Jy):")
    for name, s in summary.items():
        print(f"  {name:6s} {json.dumps(s)}")
    rd = os.environ.get("RLF_REPORT_DIR")
    if rd:
        os.makedirs(rd, exist_ok=True)
        with open(os.path.join(rd, f"precision_mid_{variant}.csv"), "w", newline="") as f:
            w = csv.DictWriter(f, fieldnames=list(table[0]))
            w.writeheader()
            w.writerows(table)
        with open(os.path.join(rd, f"precision_mid_{variant}.json"), "w") as f:
            json.dump({"sigma_jy": sigma, "summary": summary}, f, indent=1)
    for name, s in summary.items():
        assert s["n_de_gt_1e-4"] == 0, (name, s)
        # one source's |V| <= S (nu/nu_ref)^beta < 1.05 S: the FP64 path is limited by the complex64
        # rounding of its output, the mixed forms by the 1e-5 sky-model tolerance
        assert s["max_vis_err_rel"] <= (2e-7 if name == "fp64" else 1.1e-5), (name, s)
