"""GPU parity of the position marginal (Sec. 2.4) with the oracle.

The data hold the small workload's sources at their true positions; the catalogue
the chain is given has every position moved by a seeded offset of up to 0.25 arcsec
per axis, so the likelihood has to find the source within the offset grid.  Facets
come from the oracle (extracted at the catalogue positions) or from the GPU chain;
estimates are compared with the oracle's at the same n_pos and step.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import cases

pytestmark = pytest.mark.gpu

PRECS = {"split": 2, "mixed": 1, "fp64": 0}
STEP = 0.1


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
def displaced():
    c = cases.build(synth.workload("small"), snr10=True)
    rng = np.random.default_rng(71)
    off = rng.uniform(-0.25, 0.25, size=(2, c.cat.n_src)) * cases.ARC
    l_cat, m_cat = c.cat.l + off[0], c.cat.m + off[1]
    z = np.zeros(c.cat.n_src)
    s0 = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, l_cat, m_cat, c.cat.flux_jy, c.alpha_med_rad(),
                          z, z, nu_ref=c.wl.nu_ref_hz)
    sky0 = np.stack([s0.real, s0.imag], -1).astype(np.float32)
    return c, l_cat, m_cat, sky0


def _catalogue(rlf, c, l_cat, m_cat):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    z = np.zeros(c.cat.n_src)
    obs, _ = cases.to_device(c)
    return obs, rlf.Catalogue(t(l_cat), t(m_cat), t(c.cat.flux_jy), t(z), t(z), None)


def _oracle_facets(c, l_cat, m_cat, sky0, po):
    al = c.alpha_med_rad()
    out = []
    for i in range(c.cat.n_src):
        du = oracle.facet_du(c.cat.flux_jy[i], 0.0, po)
        out.append((oracle.extract_facet(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, sky0, l_cat[i], m_cat[i],
                                         c.cat.flux_jy[i], al[i], 0.0, 0.0, du, po), du))
    return out


def _compare(rlf, got, ests, check_levels=False):
    for i, est in enumerate(ests):
        assert cases.est_matches(got, i, est) <= 1e-4, (i, got["e1"][i], est[oracle.E1], got["e2"][i], est[oracle.E2])
        assert (int(got["flag"][i]) & rlf.FLAG_BAD != 0) == (est[oracle.FLAG] != 0), i
        if est[oracle.THRESH_MARGIN] > 1e-3:
            assert abs(got["sig1"][i] - est[oracle.SIG1]) <= 1e-4 + 1e-3 * est[oracle.SIG1]
            assert abs(got["alpha_arcsec"][i] - est[oracle.ALPHA]) <= 1e-3
        assert abs(got["flux_jy"][i] - est[oracle.FLUX]) <= 1e-4 * abs(est[oracle.FLUX]), i
        if check_levels:
            assert (int(got["flag"][i]) >> rlf.FLAG_LEVELS_SHIFT) & 15 == int(est[oracle.LEVELS]), i


@pytest.mark.parametrize("prec", ["split", "mixed", "fp64"])
@pytest.mark.parametrize("n_pos", [3, 5])
def test_position_fit_from_oracle_facets(rlf, displaced, prec, n_pos):
    import torch
    c, l_cat, m_cat, sky0 = displaced
    po = c.oracle_params(n_pos=n_pos, pos_step_arcsec=STEP)
    facets = _oracle_facets(c, l_cat, m_cat, sky0, po)
    ests = [oracle.fit_facet(acc, du, c.cat.flux_jy[i], po).est for i, (acc, du) in enumerate(facets)]
    obs, cat = _catalogue(rlf, c, l_cat, m_cat)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, n_pos=n_pos,
                           pos_step_arcsec=STEP)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    fac = torch.from_numpy(np.ascontiguousarray(np.stack([f for f, _ in facets]))).cuda()
    rlf.fit_sources(fac, cat, 0, cat.n_src, p, out, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    _compare(rlf, out.numpy(), ests)
    # the marginal changes the answer: with the position taken as exact the same facets
    # give other estimates
    exact = [oracle.fit_facet(acc, du, c.cat.flux_jy[i], c.oracle_params()).est for i, (acc, du) in enumerate(facets)]
    assert max(abs(e[oracle.FLUX] - x[oracle.FLUX]) / x[oracle.FLUX] for e, x in zip(exact, ests)) > 1e-3


@pytest.mark.parametrize("prec", ["split", "fp64"])
@pytest.mark.parametrize("profile,flux_prior", [(1, 0), (0, 1)])
def test_position_fit_gaussian_profile_and_real_line_prior(rlf, displaced, prec, profile, flux_prior):
    # the Gaussian profile's brightness and the real-line flux prior through the
    # position-marginal grid (the best offset is then the largest |b|)
    import torch
    c, l_cat, m_cat, sky0 = displaced
    po = c.oracle_params(n_pos=3, pos_step_arcsec=STEP, profile=profile, flux_prior=flux_prior)
    facets = _oracle_facets(c, l_cat, m_cat, sky0, po)
    ests = [oracle.fit_facet(acc, du, c.cat.flux_jy[i], po).est for i, (acc, du) in enumerate(facets)]
    obs, cat = _catalogue(rlf, c, l_cat, m_cat)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, n_pos=3,
                           pos_step_arcsec=STEP, profile=profile, flux_prior=flux_prior)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    fac = torch.from_numpy(np.ascontiguousarray(np.stack([f for f, _ in facets]))).cuda()
    rlf.fit_sources(fac, cat, 0, cat.n_src, p, out, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    _compare(rlf, out.numpy(), ests)


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_position_adaptive_from_oracle_facets(rlf, displaced, prec):
    # adaptive sampling around the maximum with the position marginal at every sample: a
    # brighter copy of the data (noise scaled down) so that posteriors are narrow enough
    # for the lattices to be refined
    import torch
    c, l_cat, m_cat, sky0 = displaced
    snr_max = c.cat.flux_jy.max() * math.sqrt(c.obs.n_rows * c.obs.n_chan) / c.sigma
    cb = cases.build(synth.workload("small"), sigma=c.sigma * snr_max / 100.0)
    po = cb.oracle_params(n_pos=3, pos_step_arcsec=STEP, estimator=1)
    facets = _oracle_facets(cb, l_cat, m_cat, sky0, po)
    ests = [oracle.fit_facet_adaptive(acc, du, cb.cat.flux_jy[i], po) for i, (acc, du) in enumerate(facets)]
    assert max(int(e[oracle.LEVELS]) for e in ests) >= 1
    obs, cat = _catalogue(rlf, cb, l_cat, m_cat)
    p = rlf.params_default(precision=PRECS[prec], nu_ref_hz=cb.wl.nu_ref_hz, sigma_jy=cb.sigma, n_pos=3,
                           pos_step_arcsec=STEP, estimator=rlf.ESTIMATOR_ADAPTIVE)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    fac = torch.from_numpy(np.ascontiguousarray(np.stack([f for f, _ in facets]))).cuda()
    rlf.fit_sources(fac, cat, 0, cat.n_src, p, out, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    _compare(rlf, out.numpy(), ests, check_levels=True)


@pytest.mark.parametrize("chunk,update_mode", [(0, 1), (3, 0)])
def test_position_chain_matches_oracle(rlf, displaced, chunk, update_mode):
    # the whole chain (Sec. 2) from the displaced catalogue with the position marginal
    import torch
    c, l_cat, m_cat, _ = displaced
    po = c.oracle_params(chunk=chunk, update_mode=update_mode, n_pos=3, pos_step_arcsec=STEP)
    est, sky_ref = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.data, l_cat, m_cat, c.cat.flux_jy,
                                   None, po, want_sky=True)
    obs, cat = _catalogue(rlf, c, l_cat, m_cat)
    p = rlf.params_default(precision=PRECS["split"], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, chunk=chunk,
                           update_mode=update_mode, n_pos=3, pos_step_arcsec=STEP)
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


def test_position_marginal_rejected_by_the_learned_proposal(rlf, displaced):
    import torch
    c, l_cat, m_cat, _ = displaced
    obs, cat = _catalogue(rlf, c, l_cat, m_cat)
    p = rlf.params_default(nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, n_pos=3, facet_n=64)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_FIT)
    out = rlf.Results(cat.n_src, "cuda")
    fac = torch.zeros((cat.n_src, 4, 64 * 64), dtype=torch.float64, device="cuda")
    with pytest.raises(rlf.RlfError) as e:
        rlf.fit_sources_mlp(fac, cat, 0, cat.n_src, p, rlf.Mlp(), out, ws)
    assert e.value.code == rlf.RLF_EUNSUPPORTED


def test_position_graph_replay_and_refit(rlf, displaced):
    # the chain with the position marginal captured as a CUDA graph replays the run's
    # results; and the refit of bad fits (Sec. 2.4) with the marginal matches the oracle
    import torch
    c, l_cat, m_cat, _ = displaced
    obs, cat = _catalogue(rlf, c, l_cat, m_cat)
    data = cases.vis_tensor(c.data)
    p = rlf.params_default(precision=PRECS["split"], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=c.sigma, update_mode=1,
                           n_pos=3, pos_step_arcsec=STEP)
    ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_RUN)
    out = rlf.Results(cat.n_src, "cuda")
    sky = torch.empty(obs.n_rows * obs.n_chan * 2, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        rlf.run(obs, data, cat, p, out, sky, ws, stream)
        stream.synchronize()
        ref = out.numpy()
        g = rlf.Graph(obs, data, cat, p, out, sky, ws, stream)
        out.e1.zero_()
        out.e2.zero_()
        g.launch(stream)
        stream.synchronize()
        got = out.numpy()
        g.close()
    for f in ("e1", "e2", "sig1", "sig2", "flux_jy"):
        assert np.allclose(got[f], ref[f], rtol=1e-5, atol=1e-5), f
    # refit pass: sigma = 1 uJy collapses every first-pass posterior onto one node (bad)
    sigma = c.wl.sigma_jy
    dat1 = cases.data_from(cases.true_sky(c), sigma, c.wl.seed)
    po = c.oracle_params(chunk=0, update_mode=1, refit_bad=1, n_pos=3, pos_step_arcsec=STEP, sigma_jy=sigma)
    est = oracle.pipeline(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, dat1, l_cat, m_cat, c.cat.flux_jy, None, po)
    assert np.all(est[:, oracle.REFIT] == 1)
    p1 = rlf.params_default(precision=PRECS["split"], nu_ref_hz=c.wl.nu_ref_hz, sigma_jy=sigma, update_mode=1,
                            refit_bad=1, n_pos=3, pos_step_arcsec=STEP)
    rlf.run(obs, cases.vis_tensor(dat1), cat, p1, out, sky, ws)
    code, status = rlf.read_status(ws)
    assert code == rlf.RLF_OK, status
    got = out.numpy()
    assert np.all(got["flag"] & rlf.FLAG_REFIT)
    for i in range(c.cat.n_src):
        assert cases.est_matches(got, i, est[i]) <= 1e-4, (i, got["e1"][i], est[i, oracle.E1])
