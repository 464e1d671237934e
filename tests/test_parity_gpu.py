"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small workloads are compared element by element; the 37M-visibility, 200-source
workload is run in full on the GPU, in the launch configuration the benchmark
times, and compared on sampled rows and sources that the oracle computes one by
one.  Tolerances:
  visibilities  per value |dV| <= 1e-5 sum_j |term_j| and normwise 1e-5 (mixed),
                1e-10 (FP64 path), plus the complex64 rounding of the output
  facets        counts exact; sums within 3e-5 sum |x| (mixed), 1e-9 (FP64)
  fits          |de1|, |de2| <= 1e-4
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

pytestmark = pytest.mark.gpu

PRECS = {"split": 2, "mixed": 1, "fp64": 0}
VIS_TOL = {"split": 1e-5, "mixed": 1e-5, "fp64": 1e-10}
FACET_TOL = {"split": 3e-5, "mixed": 3e-5, "fp64": 1e-9}


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
def small():
    return small_case(True)


def _torch():
    import torch
    return torch


def _sky_gpu(rlf, case, prec, e1, e2, alpha=None, vis_out=None):
    torch = _torch()
    obs, cat = cases.to_device(case, e1, e2, alpha)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=case.wl.nu_ref_hz)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_SKY)
    vis = vis_out if vis_out is not None else torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32,
                                                           device="cuda")
    rlf.sky_model(obs, cat, p, vis, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK and status == 0
    return vis.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)


def _check_vis(got, ref, ab, tol):
    # the output is complex64: its rounding (2^-24 per component) comes on top of the path's error
    g = got[..., 0] + 1j * got[..., 1]
    err = np.abs(g - ref)
    out_round = 2.0 ** -24 * np.sqrt(2.0) * np.abs(ref)
    assert np.all(err <= tol * ab + out_round + 1e-30), float(np.max((err - out_round) / (ab + 1e-300)))
    assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref) + 2.0 ** -24 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
def test_sky_model_small_full(rlf, small, prec):
    c = small
    al = c.cat.alpha_arcsec
    got = _sky_gpu(rlf, c, prec, c.cat.e1, c.cat.e2, alpha=al)
    ref, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                               al * cases.ARC, c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz, with_abs=True)
    _check_vis(got, ref, ab, VIS_TOL[prec])


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
@pytest.mark.parametrize("n_chan,uniform", [(1, True), (2, True), (3, True), (8, True), (13, True), (5, False)])
def test_sky_model_channels_and_tiles(rlf, prec, n_chan, uniform):
    # 300 sources: three shared-memory tiles with a ragged last one; channel groups with ragged tails
    wl = synth.tiny(seed=30 + n_chan, n_ant=20, n_time=13, n_chan=n_chan, n_src=300, r_max_m=20000.0)
    c = cases.build(wl, with_data=False)
    if not uniform:
        c.obs.freq_hz = c.obs.freq_hz * (1 + 0.01 * np.arange(n_chan) ** 2 / n_chan ** 2)
    got = _sky_gpu(rlf, c, prec, c.cat.e1, c.cat.e2)
    al = c.alpha_med_rad()
    ref, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy, al,
                               c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz, with_abs=True)
    _check_vis(got, ref, ab, VIS_TOL[prec])


def test_sky_update_equals_model_of_new_shapes(rlf):
    torch = _torch()
    wl = synth.tiny(seed=41, n_ant=16, n_time=11, n_chan=4, n_src=37, r_max_m=8000.0)
    c = cases.build(wl, with_data=False)
    obs, cat = cases.to_device(c)  # circular shapes
    p = rlf.params_default(nu_ref_hz=wl.nu_ref_hz)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_SKY)
    vis = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.sky_model(obs, cat, p, vis, ws)
    first, count = 5, 20
    e1n = torch.from_numpy(c.cat.e1[first:first + count].copy()).cuda()
    e2n = torch.from_numpy(c.cat.e2[first:first + count].copy()).cuda()
    flag = torch.zeros(count, dtype=torch.int32, device="cuda")
    flag[3] = rlf.FLAG_BAD    # a bad fit stays circular in the paper's update rule
    rlf.sky_update(obs, cat, first, count, e1n, e2n, flag, p, vis, ws)
    got = vis.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    e1 = np.zeros(c.cat.n_src)
    e2 = np.zeros(c.cat.n_src)
    sel = np.arange(first, first + count) != first + 3
    e1[first:first + count][sel] = c.cat.e1[first:first + count][sel]
    e2[first:first + count][sel] = c.cat.e2[first:first + count][sel]
    ref, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                               c.alpha_med_rad(), e1, e2, nu_ref=wl.nu_ref_hz, with_abs=True)
    _check_vis(got, ref, ab, 2e-5)


def _extract_gpu(rlf, case, prec, e1, e2, data, sky, first=0, count=None, facet_n=64):
    torch = _torch()
    count = case.cat.n_src - first if count is None else count
    obs, cat = cases.to_device(case, e1, e2)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=case.wl.nu_ref_hz, facet_n=facet_n)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_EXTRACT)
    fac = torch.empty(rlf.facets_size(count, p) // 8, dtype=torch.float64, device="cuda")
    rlf.extract_facets(obs, cases.vis_tensor(data), cases.vis_tensor(sky), cat, first, count, p, fac, ws)
    torch.cuda.synchronize()
    return fac.view(count, 4, facet_n * facet_n).cpu().numpy()


def _check_facet(got, ref, ab, tol):
    assert np.array_equal(got[2], ref[2]), np.argwhere(got[2] != ref[2])[:5]
    assert np.all(np.abs(got[0] - ref[0]) <= tol * ab + 1e-300)
    assert np.all(np.abs(got[1] - ref[1]) <= tol * ab + 1e-300)
    assert np.all(np.abs(got[3] - ref[3]) <= 1e-5 * ref[3] + 1e-300)


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
def test_extract_small_full(rlf, small, prec):
    c = small
    e1 = c.cat.e1 * 0.5   # shapes currently in the sky model (non-zero: the added-back model uses them)
    e2 = c.cat.e2 * 0.5
    al = c.alpha_med_rad()
    sky = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy, al, e1, e2,
                           nu_ref=c.wl.nu_ref_hz)
    sky2 = np.stack([sky.real, sky.imag], -1).astype(np.float32)
    got = _extract_gpu(rlf, c, prec, e1, e2, c.data, sky2)
    p = c.oracle_params()
    for i in range(c.cat.n_src):
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, p)
        ref, ab = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, sky2, c.cat.l[i], c.cat.m[i],
                                       c.cat.flux_jy[i], al[i], e1[i], e2[i], du, p, with_abs=True)
        assert ref[2].sum() > 1000
        _check_facet(got[i], ref, ab, FACET_TOL[prec])


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
def test_extract_multichannel_ragged(rlf, prec):
    wl = synth.tiny(seed=52, n_ant=24, n_time=17, n_chan=11, n_src=6, r_max_m=6000.0)
    c = cases.build(wl, snr10=True)
    got = _extract_gpu(rlf, c, prec, None, None, c.data, c.sky0, first=2, count=3, facet_n=16)
    p = c.oracle_params(facet_n=16)
    al = c.alpha_med_rad()
    for t in range(3):
        i = 2 + t
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, p)
        ref, ab = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.sky0, c.cat.l[i],
                                       c.cat.m[i], c.cat.flux_jy[i], al[i], 0.0, 0.0, du, p, with_abs=True)
        assert ref[2].sum() > 100
        _check_facet(got[t], ref, ab, FACET_TOL[prec])


@pytest.mark.parametrize("prec", ["split", "mixed"])
@pytest.mark.parametrize("n_chan,uniform", [(2, True), (5, False), (16, True), (40, True)])
@pytest.mark.parametrize("count", [1, 3])
def test_extract_channel_lanes(rlf, prec, n_chan, uniform, count):
    # every channel-lane layout of the extraction: 2 and 16 channels fill their lanes, 5 leaves
    # three of eight idle (uneven spacing: no phase step), 40 splits into groups of 32 and 8;
    # one source reads data and sky model separately, three the formed residual
    wl = synth.tiny(seed=60 + n_chan, n_ant=20, n_time=37, n_chan=n_chan, n_src=4, r_max_m=5000.0)
    c = cases.build(wl, snr10=True)
    if not uniform:
        c.obs.freq_hz = c.obs.freq_hz * (1 + 0.02 * np.arange(n_chan) ** 2 / n_chan ** 2)
        c = cases.Case(c.wl, c.obs, c.cat, c.sigma)
        c.data = cases.data_from(cases.true_sky(c), c.sigma, wl.seed)
        z = np.zeros(c.cat.n_src)
        s0 = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                              c.alpha_med_rad(), z, z, nu_ref=wl.nu_ref_hz)
        c.sky0 = np.stack([s0.real, s0.imag], -1).astype(np.float32)
    got = _extract_gpu(rlf, c, prec, None, None, c.data, c.sky0, first=1, count=count, facet_n=32)
    p = c.oracle_params(facet_n=32)
    al = c.alpha_med_rad()
    for t in range(count):
        i = 1 + t
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, p)
        ref, ab = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.sky0, c.cat.l[i],
                                       c.cat.m[i], c.cat.flux_jy[i], al[i], 0.0, 0.0, du, p, with_abs=True)
        assert ref[2].sum() > 100
        _check_facet(got[t], ref, ab, FACET_TOL[prec])


def _fit_gpu(rlf, case, prec, facets_np, first=0, **pk):
    torch = _torch()
    count = facets_np.shape[0]
    obs, cat = cases.to_device(case)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=case.wl.nu_ref_hz, sigma_jy=case.sigma, **pk)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(count, "cuda")
    fac = torch.from_numpy(np.ascontiguousarray(facets_np)).cuda()
    rlf.fit_sources(fac, cat, first, count, p, out, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    return out.numpy()


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
@pytest.mark.parametrize("snr10", [True, False])
def test_fit_small_from_oracle_facets(rlf, prec, snr10):
    c = small_case(snr10)
    p = c.oracle_params()
    al = c.alpha_med_rad()
    facets, ests = [], []
    for i in range(c.cat.n_src):
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, p)
        acc = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.sky0, c.cat.l[i], c.cat.m[i],
                                   c.cat.flux_jy[i], al[i], 0.0, 0.0, du, p)
        facets.append(acc)
        ests.append(oracle.fit_facet(acc, du, c.cat.flux_jy[i], p).est)
    got = _fit_gpu(rlf, c, prec, np.stack(facets))
    for i, est in enumerate(ests):
        assert cases.est_matches(got, i, est) <= 1e-4, (i, got["e1"][i], est[oracle.E1])
        assert got["flag"][i] & 1 == int(est[oracle.FLAG])
        if est[oracle.THRESH_MARGIN] > 1e-3:
            assert abs(got["sig1"][i] - est[oracle.SIG1]) <= 1e-4 + 1e-3 * est[oracle.SIG1]
            assert abs(got["alpha_arcsec"][i] - est[oracle.ALPHA]) <= 1e-3
        assert abs(got["flux_jy"][i] - est[oracle.FLUX]) <= 1e-4 * abs(est[oracle.FLUX])


_SMALL = {}


def small_case(snr10: bool):
    if snr10 not in _SMALL:
        _SMALL[snr10] = cases.build(synth.workload("small"), snr10=snr10)
    return _SMALL[snr10]


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
@pytest.mark.parametrize("chunk,update_mode", [(1, 1), (0, 1), (3, 0)])
def test_run_small_pipeline(rlf, prec, chunk, update_mode):
    torch = _torch()
    c = small_case(True)
    p_or = c.oracle_params(chunk=chunk, update_mode=update_mode)
    est, sky_ref = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.cat.l, c.cat.m,
                                   c.cat.flux_jy, None, p_or, want_sky=True)
    obs, cat = cases.to_device(c)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, chunk=chunk,
                           update_mode=update_mode)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.run(obs, cases.vis_tensor(c.data), cat, p, out, sky, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    got = out.numpy()
    for i in range(c.cat.n_src):
        assert cases.est_matches(got, i, est[i]) <= 1e-4, (i, got["e1"][i], est[i, oracle.E1], got["e2"][i],
                                                           est[i, oracle.E2])
    # the sky model after the chain's updates (Sec. 3.1).  The two sides' fitted shapes may
    # differ by up to 1e-4 and one term moves by at most about 1.5 S per unit of e, so the
    # bound is 2e-5 sum S (FP32 model) + 1.5e-4 sum S; a missed or wrong update moves terms
    # by ~0.1 S
    g = sky.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    dv = np.abs(g[..., 0] + 1j * g[..., 1] - sky_ref)
    assert dv.max() <= (2e-5 + 1.5e-4) * c.cat.flux_jy.sum(), dv.max() / c.cat.flux_jy.sum()


@pytest.mark.parametrize("chunk", [0, 3])
def test_run_rows_without_baseline_order(rlf, chunk):
    # rows given without their baseline count (n_baselines = 0): no baseline order, the
    # split baselines in row order for the extraction and the sky kernels; same results
    torch = _torch()
    c = small_case(True)
    est, sky_ref = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.cat.l, c.cat.m,
                                   c.cat.flux_jy, None, c.oracle_params(chunk=chunk, update_mode=1), want_sky=True)
    obs, cat = cases.to_device(c)
    obs = rlf.Observation(obs.u, obs.v, obs.w, c.obs.freq_hz, 0)
    p = rlf.params_default(precision=PRECS["split"], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, chunk=chunk,
                           update_mode=1)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.run(obs, cases.vis_tensor(c.data), cat, p, out, sky, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    got = out.numpy()
    for i in range(c.cat.n_src):
        assert cases.est_matches(got, i, est[i]) <= 1e-4, (i, got["e1"][i], est[i, oracle.E1])
    g = sky.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    assert np.abs(g[..., 0] + 1j * g[..., 1] - sky_ref).max() <= (2e-5 + 1.5e-4) * c.cat.flux_jy.sum()


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
def test_gaussian_profile_sky_model_and_chain(rlf, prec):
    # the Gaussian source profile (footnote to Sec. 2.2) through the sky model and the whole
    # chain: data from the oracle's Gaussian sky model, every step on the GPU with profile 1
    torch = _torch()
    c = cases.build(synth.workload("small"), snr10=True, profile=1)
    obs, cat = cases.to_device(c, c.cat.e1, c.cat.e2, c.cat.alpha_arcsec)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma,
                           profile=rlf.PROFILE_GAUSSIAN)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_SKY)
    vis = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.sky_model(obs, cat, p, vis, ws)
    got = vis.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    ref, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                               c.cat.alpha_arcsec * cases.ARC, c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz,
                               with_abs=True, profile=1)
    _check_vis(got, ref, ab, 1e-10 if prec == "fp64" else 1e-5)
    # the whole chain from a circular catalogue
    obs, cat = cases.to_device(c)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, update_mode=1,
                           profile=rlf.PROFILE_GAUSSIAN)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.run(obs, cases.vis_tensor(c.data), cat, p, out, sky, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    est, sky_ref = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.cat.l, c.cat.m,
                                   c.cat.flux_jy, None, c.oracle_params(chunk=0, update_mode=1), want_sky=True)
    res = out.numpy()
    for i in range(c.cat.n_src):
        assert cases.est_matches(res, i, est[i]) <= 1e-4, (i, res["e1"][i], est[i, oracle.E1])
    g = sky.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    assert np.abs(g[..., 0] + 1j * g[..., 1] - sky_ref).max() <= (2e-5 + 1.5e-4) * c.cat.flux_jy.sum()
    # the profile changes the answer: the exponential model fits these data differently
    p0 = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, update_mode=1)
    out0 = rlf.Results(cat.n_src, "cuda")
    rlf.run(obs, cases.vis_tensor(c.data), cat, p0, out0, sky, ws)
    r0 = out0.numpy()
    assert np.max(np.abs(r0["alpha_arcsec"] - res["alpha_arcsec"])) > 0.05


@pytest.mark.parametrize("prec,profile", [("split", 0), ("mixed", 0), ("fp64", 0), ("split", 1)])
def test_adaptive_estimator_matches_oracle(rlf, prec, profile):
    # adaptive sampling around the maximum (Sec. 2.4) on facets whose posteriors are
    # narrower than the grid: the brightest source at SNR ~100; the oracle's facets in,
    # the number of halvings and the estimates compared with the oracle's (profile 1:
    # the Gaussian source profile, data and fit)
    torch = _torch()
    c0 = cases.build(synth.workload("small"), with_data=False)
    snr_max = c0.cat.flux_jy.max() * math.sqrt(c0.obs.n_rows * c0.obs.n_chan) / c0.cat.flux_jy.min()
    c = cases.build(synth.workload("small"), sigma=cases.snr10_sigma(c0.obs, c0.cat) * snr_max / 100.0,
                    profile=profile)
    po = c.oracle_params(estimator=1)
    al = c.alpha_med_rad()
    facets, ests = [], []
    for i in range(c.cat.n_src):
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, po)
        acc = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.sky0, c.cat.l[i], c.cat.m[i],
                                   c.cat.flux_jy[i], al[i], 0.0, 0.0, du, po)
        facets.append(acc)
        ests.append(oracle.fit_facet_adaptive(acc, du, c.cat.flux_jy[i], po))
    levels = np.array([int(e[oracle.LEVELS]) for e in ests])
    assert levels.max() >= 2 and levels.min() == 0        # both kinds of posterior are present
    obs, cat = cases.to_device(c)
    p = rlf.params_default(nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, precision=PRECS[prec],
                           estimator=rlf.ESTIMATOR_ADAPTIVE, profile=profile)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    rlf.fit_sources(torch.from_numpy(np.stack(facets)).cuda(), cat, 0, cat.n_src, p, out, ws)
    got = out.numpy()
    for i, est in enumerate(ests):
        if est[oracle.NKEPT] == 0:
            # no estimate: the likelihood vanishes on the oracle's last lattice (a posterior
            # pushed against |e| = 1, where the Gaussian brightness underflows FP32 on the
            # GPU a halving or two before FP64 does); both sides flag the fit bad
            assert int(got["flag"][i]) & rlf.FLAG_BAD, i
            assert cases.est_matches(got, i, est) <= 1e-4, (i, got["e1"][i], got["e2"][i])   # (0, 0): no samples kept
            continue
        assert (int(got["flag"][i]) >> rlf.FLAG_LEVELS_SHIFT) & 15 == levels[i], i
        assert cases.est_matches(got, i, est) <= 1e-4, (i, levels[i], got["e1"][i], est[oracle.E1])
        assert abs(got["sig1"][i] - est[oracle.SIG1]) <= 1e-4 + 1e-3 * est[oracle.SIG1]
        assert (int(got["flag"][i]) & rlf.FLAG_BAD != 0) == (est[oracle.FLAG] != 0)


@pytest.mark.parametrize("chunk,update_mode", [(0, 1), (3, 0)])
def test_refit_pass_matches_oracle(rlf, chunk, update_mode):
    # sigma = 1 uJy: every first-pass posterior collapses onto one grid node (bad), so every
    # source is fitted again after the whole catalogue (Sec. 2.4)
    torch = _torch()
    c = small_case(False)
    est, sky_ref = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, c.cat.l, c.cat.m,
                                   c.cat.flux_jy, None, c.oracle_params(chunk=chunk, update_mode=update_mode,
                                                                        refit_bad=1), want_sky=True)
    assert np.all(est[:, oracle.REFIT] == 1)
    obs, cat = cases.to_device(c)
    p = rlf.params_default(precision=PRECS["split"], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, chunk=chunk,
                           update_mode=update_mode, refit_bad=1)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    data = cases.vis_tensor(c.data)
    rlf.run(obs, data, cat, p, out, sky, ws)
    got = out.numpy()
    assert np.all(got["flag"] & rlf.FLAG_REFIT)
    for i in range(c.cat.n_src):
        assert cases.est_matches(got, i, est[i]) <= 1e-4, (i, got["e1"][i], est[i, oracle.E1])
    g = sky.view(obs.n_rows, obs.n_chan, 2).cpu().numpy().astype(np.float64)
    assert np.abs(g[..., 0] + 1j * g[..., 1] - sky_ref).max() <= (2e-5 + 1.5e-4) * c.cat.flux_jy.sum()
    # the refit pass reads a count on the host: not capturable
    with pytest.raises(RuntimeError):
        rlf.Graph(obs, data, cat, p, out, sky, ws, torch.cuda.Stream())


@pytest.mark.parametrize("n_pos,estimator", [(1, 0), (3, 0), (1, 1), (3, 1)])
def test_invalid_and_empty_sources_are_flagged(rlf, n_pos, estimator):
    # estimator 1: adaptive sampling after the grid (the cluster form at n_pos 1, one CTA
    # per facet at n_pos 3): an empty facet is not refined
    torch = _torch()
    wl = synth.tiny(seed=61, n_ant=12, n_time=9, n_chan=2, n_src=4, r_max_m=3000.0)
    c = cases.build(wl, snr10=True)
    obs, cat = cases.to_device(c)
    cat.flux_jy[1] = -1.0                 # invalid flux
    cat.e1[2] = 0.9
    cat.e2[2] = 0.6                       # |e| >= 1
    # K = 1e6 makes the cells ~0.1 wavelength wide: no baseline falls in the facet window
    p = rlf.params_default(nu_ref_hz=wl.nu_ref_hz, sigma_jy=c.sigma, facet_n=8, psf_nat=1.0e6, n_pos=n_pos,
                           estimator=estimator)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    rlf.run(obs, cases.vis_tensor(c.data), cat, p, out, sky, ws)
    code, status = rlf.read_status(ws)
    assert status & rlf.DEV_INVALID_SOURCE
    f = out.numpy()["flag"]
    assert f[1] & rlf.FLAG_INVALID and f[2] & rlf.FLAG_INVALID
    for i in (0, 3):
        assert not (f[i] & rlf.FLAG_INVALID) and f[i] & rlf.FLAG_EMPTY
        assert (int(f[i]) >> rlf.FLAG_LEVELS_SHIFT) & 15 == 0   # no lattice refinement of an empty facet
    # an empty facet is not a numerical failure (no non-finite likelihood reported)
    assert not (status & rlf.DEV_NONFINITE)


# ---- full-size workload (37M visibilities, 200 sources), sampled ----------------------------

@pytest.fixture(scope="module")
def mid():
    wl = synth.workload("mid")
    return cases.build(wl, with_data=False)


@pytest.mark.parametrize("prec", ["split", "mixed"])
def test_sky_model_mid_sampled(rlf, mid, prec):
    c = mid
    got = _sky_gpu(rlf, c, prec, c.cat.e1, c.cat.e2)
    rng = np.random.default_rng(123)
    rows = np.sort(rng.choice(c.obs.n_rows, 1500, replace=False))
    ref, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                               c.alpha_med_rad(), c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz, rows=rows,
                               with_abs=True, n_threads=0)
    _check_vis(got[rows], ref, ab, 1e-5)


@pytest.mark.parametrize("prec", ["split", "mixed"])
def test_extract_and_fit_mid_sampled(rlf, mid, prec):
    # data = an arbitrary sky array plus noise; the sources' current shapes are non-zero, so
    # every facet holds that source's model plus noise and the fit has a known answer
    torch = _torch()
    c = mid
    R, C = c.obs.n_rows, c.obs.n_chan
    rng = np.random.default_rng(7)
    sky = (rng.standard_normal((R, C, 2), dtype=np.float32) * np.float32(1e-4))
    sigma = 3e-3
    data = sky + synth.noise(R, C, sigma, 99)
    e1, e2 = c.cat.e1, c.cat.e2
    got_f = _extract_gpu(rlf, c, prec, e1, e2, data, sky)
    # fit the GPU facets on the GPU
    obs, cat = cases.to_device(c, e1, e2)
    p = rlf.params_default(nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=sigma, precision=PRECS[prec])
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    rlf.fit_sources(torch.from_numpy(got_f).cuda(), cat, 0, cat.n_src, p, out, ws)
    res = out.numpy()
    po = c.oracle_params(sigma_jy=sigma)
    al = c.alpha_med_rad()
    for i in (0, 117, c.cat.n_src - 1):
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, po)
        ref, ab = oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, data, sky, c.cat.l[i], c.cat.m[i],
                                       c.cat.flux_jy[i], al[i], e1[i], e2[i], du, po, with_abs=True)
        _check_facet(got_f[i], ref, ab, FACET_TOL[prec])
        est = oracle.fit_facet(ref, du, c.cat.flux_jy[i], po).est
        assert cases.est_matches(res, i, est) <= 1e-4, (i, res["e1"][i], est[oracle.E1])
