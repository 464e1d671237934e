"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks one oracle routine against something other than itself: a
closed form, a numerical transform or integral computed a different way, a
brute-force loop on a tiny input, or a number printed in the paper.  The
oracle is the reference the CUDA path is compared with, so these run first and
on the CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C = 299792458.0
ARC = math.pi / 648000.0


def test_default_params_are_the_papers():
    p = oracle.default_params()
    assert p.add == GOLD["ADD"]["value"] and p.esp == GOLD["ESP"]["value"]
    assert p.beta == GOLD["beta"]["value"]
    assert p.r_std == GOLD["R_STD"]["value"]
    assert p.r_min_arcsec == GOLD["RMIN_arcsec"]["value"]
    assert p.r_max_arcsec == GOLD["RMAX_arcsec"]["value"]
    assert p.psf_nat == GOLD["PSF_NAT_K"]["value"]
    assert p.thresh_frac == GOLD["threshold_fraction"]["value"]
    assert p.var_sigma_min == GOLD["sigma_e_min"]["value"]
    assert p.var_det_min == GOLD["sqrt_det_cov_min"]["value"]


def test_eq4_scale_flux_relation():
    # ln(alpha/arcsec) is linear in ln(S/uJy) with the printed slope and intercept
    s = np.array([1e-6, 10e-6, 200e-6])
    la = np.log([oracle.alpha_med(x) for x in s])
    slope = np.diff(la) / np.diff(np.log(s * 1e6))
    assert np.allclose(slope, GOLD["ESP"]["value"], rtol=0, atol=1e-12)
    assert abs(la[0] - GOLD["ADD"]["value"]) < 1e-12


# ---- Eq. 1 -------------------------------------------------------------------

def test_p1_zero_spacing_gives_flux():
    # k = 0: the visibility is the flux times the spectral factor, phase 0 at the centre
    for nu in (0.9e9, 1.0e9, 1.3e9):
        v = oracle.model_vis(0.0, 0.0, 0.0, nu, 0.0, 0.0, 1.3e-4, 2e-6, 0.3, -0.4, -0.7, 1.0e9)
        assert abs(v - 1.3e-4 * (nu / 1e9) ** -0.7) < 1e-18


def test_p2_point_source_limit_ignores_shape():
    vals = [oracle.model_vis(1234.5, -987.0, 12.0, 1.1e9, 1e-3, -2e-3, 1e-4, 0.0, e1, e2)
            for e1, e2 in ((0, 0), (0.5, 0.2), (-0.3, 0.6))]
    assert max(abs(v - vals[0]) for v in vals) < 1e-19
    assert abs(abs(vals[0]) - 1e-4 * 1.1 ** -0.7) < 1e-18


def test_p3_circular_profile_is_hankel_transform():
    # circular exponential I(r) = exp(-r/alpha)/(2 pi alpha^2): F(k) = 2 pi int r I J0(2 pi k r) dr
    alpha = 1.0
    for k in (0.02, 0.1, 0.35, 1.0):
        f = lambda r: 2 * math.pi * r * math.exp(-r / alpha) / (2 * math.pi * alpha ** 2) * special.j0(2 * math.pi * k * r)
        val, err = integrate.quad(f, 0, 80 * alpha, limit=2000, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - oracle.shape(k, 0.0, alpha, 0.0, 0.0)) < 1e-9


@pytest.fixture(scope="module")
def pixel_grid():
    L, h = 40.0, 0.04
    x = np.arange(-L, L, h) + h / 2
    X, Y = np.meshgrid(x, x, indexing="ij")
    return X, Y, h


def _sheared_image(X, Y, e1, e2):
    # the circular profile evaluated at A x, A the shear matrix of Eq. 2, flux-normalised
    A = np.array([[1 - e1, -e2], [-e2, 1 + e1]])
    ax = A[0, 0] * X + A[0, 1] * Y
    ay = A[1, 0] * X + A[1, 1] * Y
    return abs(np.linalg.det(A)) / (2 * np.pi) * np.exp(-np.hypot(ax, ay))


def test_p4_sheared_image_fourier_transform(pixel_grid):
    X, Y, h = pixel_grid
    for e1, e2 in ((0.3, -0.2), (-0.45, 0.1), (0.0, 0.55)):
        f = _sheared_image(X, Y, e1, e2)
        for ku, kv in ((0.05, 0.0), (0.0, 0.12), (0.1, 0.07), (0.25, -0.15)):
            F = (f * np.cos(2 * np.pi * (ku * X + kv * Y))).sum() * h * h
            assert abs(F - oracle.shape(ku, kv, 1.0, e1, e2)) < 2e-5, (e1, e2, ku, kv)


def test_p4_eq3_axis_ratio_and_position_angle(pixel_grid):
    # second moments of the sheared image give (a-b)/(a+b) e^{2 i theta} = e1 + i e2 (Eq. 3)
    X, Y, h = pixel_grid
    for e1, e2 in ((0.3, -0.2), (0.5, 0.0), (-0.1, 0.4)):
        f = _sheared_image(X, Y, e1, e2)
        q11, q22, q12 = (f * X * X).sum(), (f * Y * Y).sum(), (f * X * Y).sum()
        chi = complex(q11 - q22, 2 * q12) / (q11 + q22)
        eps = chi / (1 + math.sqrt(1 - abs(chi) ** 2))
        assert abs(eps - complex(e1, e2)) < 1e-4


def test_p5_hermitian():
    a = oracle.model_vis(3e3, -1.2e3, 40.0, 1.2e9, 2e-3, 1e-3, 1e-4, 5e-6, 0.2, 0.3)
    b = oracle.model_vis(-3e3, 1.2e3, -40.0, 1.2e9, 2e-3, 1e-3, 1e-4, 5e-6, 0.2, 0.3)
    assert abs(a - b.conjugate()) < 1e-18


def test_p6_rotation_covariance():
    rng = np.random.default_rng(3)
    for _ in range(20):
        ku, kv = rng.normal(0, 2e4, 2)
        e = complex(*rng.uniform(-0.5, 0.5, 2))
        psi = rng.uniform(0, math.pi)
        kr = complex(ku, kv) * complex(math.cos(psi), math.sin(psi))
        er = e * complex(math.cos(2 * psi), math.sin(2 * psi))
        a = oracle.shape(ku, kv, 4e-6, e.real, e.imag)
        b = oracle.shape(kr.real, kr.imag, 4e-6, er.real, er.imag)
        assert abs(a - b) < 1e-13


# ---- sky model -----------------------------------------------------------------

def test_p7_sky_model_is_sum_of_sources():
    wl = synth.tiny(n_src=5)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    al = cat.alpha_arcsec * ARC
    full = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2)
    parts = sum(oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l[j:j + 1], cat.m[j:j + 1],
                                 cat.flux_jy[j:j + 1], al[j:j + 1], cat.e1[j:j + 1], cat.e2[j:j + 1])
                for j in range(cat.n_src))
    assert np.max(np.abs(full - parts)) < 1e-17
    # row subsets give the same values as the full evaluation
    rows = np.array([0, 5, obs.n_rows - 1])
    sub = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                           rows=rows)
    assert np.array_equal(sub, full[rows])


def test_p14_earth_rotation_geometry_and_dataset_size():
    wl = synth.workload("batched")
    obs = synth.make_observation(wl)
    assert obs.n_bl == 197 * 196 // 2
    assert obs.n_rows == GOLD["uv_points_ska1_1000"]["value"]
    assert obs.n_time == GOLD["observation_hours"]["value"] * 3600 // GOLD["integration_s"]["value"]
    # |uvw| is the baseline length at every hour angle
    L = np.sqrt(obs.u ** 2 + obs.v ** 2 + obs.w ** 2).reshape(obs.n_time, obs.n_bl)
    assert np.max(np.abs(L - L[0:1])) < 1e-6 * np.max(L)
    assert obs.n_chan == 16 and abs(obs.freq_hz.mean() - 1.4e9) < 1


# ---- extraction ------------------------------------------------------------------

def _facet_case(n_src=3, seed=11):
    wl = synth.tiny(seed=seed, n_src=n_src, n_chan=3, n_ant=10, n_time=7)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    return wl, obs, cat


def test_p10_binning_brute_force():
    # flux 0 at the phase centre: the facet is the plain cell average of D - V
    wl, obs, cat = _facet_case()
    p = oracle.default_params(facet_n=8, nu_ref_hz=wl.nu_ref_hz)
    rng = np.random.default_rng(5)
    data = rng.normal(size=(obs.n_rows, obs.n_chan, 2)).astype(np.float32)
    sky = rng.normal(size=(obs.n_rows, obs.n_chan, 2)).astype(np.float32)
    du = 2500.0
    acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, data, sky, 0.0, 0.0, 0.0, 1e-6,
                               0.0, 0.0, du, p)
    N = 8
    ref = np.zeros((4, N * N))
    for r in range(obs.n_rows):
        for c in range(obs.n_chan):
            ku = obs.u[r] * obs.freq_hz[c] / C
            kv = obs.v[r] * obs.freq_hz[c] / C
            hit = [(iu, iv) for iu in range(N) for iv in range(N)
                   if (iu - N // 2) * du <= ku < (iu - N // 2 + 1) * du and (iv - N // 2) * du <= kv < (iv - N // 2 + 1) * du]
            if not hit:
                continue
            (iu, iv), = hit
            cell = iv * N + iu
            ref[0, cell] += float(data[r, c, 0]) - float(sky[r, c, 0])
            ref[1, cell] += float(data[r, c, 1]) - float(sky[r, c, 1])
            ref[2, cell] += 1
            ref[3, cell] += (obs.freq_hz[c] / wl.nu_ref_hz) ** -0.7
    assert ref[2].sum() > 20
    assert np.allclose(acc, ref, rtol=1e-13, atol=1e-13)


def test_p8_isolation_removes_every_other_source():
    # noise-free data equal to the sky model: each facet holds only its own source,
    # real and positive after the phase shift, S s M(k) per visibility
    wl, obs, cat = _facet_case(n_src=4)
    p = oracle.default_params(facet_n=16, nu_ref_hz=wl.nu_ref_hz)
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    sky = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                           nu_ref=wl.nu_ref_hz)
    sky2 = np.stack([sky.real, sky.imag], -1)
    for i in range(cat.n_src):
        du = oracle.facet_du(cat.flux_jy[i], 0.0, p)
        acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, sky2.astype(np.float32), sky2,
                                   cat.l[i], cat.m[i], cat.flux_jy[i], al[i], cat.e1[i], cat.e2[i], du, p)
        # expected: per-vis S s M(k), binned
        N = 16
        exp_re = np.zeros(N * N)
        for r in range(obs.n_rows):
            for c in range(obs.n_chan):
                ku = obs.u[r] * obs.freq_hz[c] / C
                kv = obs.v[r] * obs.freq_hz[c] / C
                iu, iv = math.floor(ku / du) + N // 2, math.floor(kv / du) + N // 2
                if 0 <= iu < N and 0 <= iv < N:
                    exp_re[iv * N + iu] += cat.flux_jy[i] * (obs.freq_hz[c] / wl.nu_ref_hz) ** -0.7 * \
                        oracle.shape(ku, kv, al[i], cat.e1[i], cat.e2[i])
        # float32 rounding of the data is the only difference: bounded by the sky magnitude
        scale = np.abs(sky).max() * 1e-6 * max(acc[2].max(), 1)
        assert np.max(np.abs(acc[0] - exp_re)) < scale
        assert np.max(np.abs(acc[1])) < scale
        assert acc[2].sum() > 0


def _cell_centre_observation(N, du, nu, iuv):
    u = np.array([(iu - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    v = np.array([(iv - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    w = np.linspace(-300.0, 450.0, len(iuv))
    return u, v, w


def test_p9_isolated_source_at_cell_centres_is_recovered_exactly():
    N, nu = 16, 1.0e9
    p = oracle.default_params(facet_n=N, nu_ref_hz=nu, n_e=11, e_max=0.5, n_alpha=6, sigma_jy=1e-7)
    ge, ga = oracle.grid_e(p), oracle.grid_alpha(p)
    flux = 1.2e-4
    du = oracle.facet_du(flux, 0.0, p)
    rng = np.random.default_rng(9)
    iuv = sorted({(int(a), int(b)) for a, b in rng.integers(2, N - 2, size=(60, 2))})
    u, v, w = _cell_centre_observation(N, du, nu, iuv)
    l, m = 1.5e-3, -0.8e-3
    i1, i2, k = 7, 3, 2
    e1, e2, al = ge[i1], ge[i2], ga[k] * ARC
    data = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l, m, flux, al, e1, e2, -0.7, nu)]
                     for r in range(len(u))])
    sky0 = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l, m, flux, al, 0.0, 0.0, -0.7, nu)]
                     for r in range(len(u))])
    d2 = np.stack([data.real, data.imag], -1)
    s2 = np.stack([sky0.real, sky0.imag], -1)
    acc = oracle.extract_facet(u, v, w, np.array([nu]), d2.astype(np.float32), s2, l, m, flux, al, 0.0, 0.0,
                               du, p)
    # float32 data: compare in double on a float64 copy too
    acc64 = oracle.extract_facet(u, v, w, np.array([nu]), d2.astype(np.float32), s2, l, m, flux, al, 0.0, 0.0,
                                 du, p)
    n = acc[2]
    assert n.sum() == len(iuv)
    for (iu, iv) in iuv:
        cell = iv * N + iu
        ku, kv = (iu - N // 2 + 0.5) * du, (iv - N // 2 + 0.5) * du
        assert abs(acc[0, cell] - flux * oracle.shape(ku, kv, al, e1, e2)) < 1e-7 * flux
        assert abs(acc[1, cell]) < 1e-7 * flux
    fit = oracle.fit_facet(acc64, du, flux, p)
    g = int(fit.est[oracle.MAP_INDEX])
    assert g == (i1 * p.n_e + i2) * p.n_alpha + k
    assert abs(fit.est[oracle.E1] - e1) < 1e-12 and abs(fit.est[oracle.E2] - e2) < 1e-12
    assert abs(fit.est[oracle.FLUX] / flux - 1) < 1e-6
    assert fit.est[oracle.FLAG] == 1.0   # a single node above threshold has zero spread


# ---- likelihood ------------------------------------------------------------------

@pytest.mark.parametrize("a,b,cc", [(2.5, 1.7, 3.0), (0.7, -0.9, 1.1), (50.0, 400.0, 3300.0),
                                    (2.0, -40.0, 10.0), (2.0, -100.0, 5.0), (1e4, -3e6, 1.0)])
def test_p11_flux_marginal_equals_quadrature(a, b, cc):
    # int_0^inf exp(-chi2(S)/2) dS with chi2 = C - 2 S b + S^2 a, done numerically
    s_peak = max(b / a, 0.0)
    scale = min(1 / math.sqrt(a), 1 / abs(b)) if b < 0 else 1 / math.sqrt(a)
    f = lambda s: math.exp(-0.5 * (cc - 2 * s * b + s * s * a) + 0.5 * cc - (0.5 * b * b / a if b > 0 else 0))
    val, _ = integrate.quad(f, 0, s_peak + 60 * scale, points=[s_peak] if s_peak > 0 else None,
                            epsabs=0, epsrel=1e-12, limit=500)
    ref = math.log(val) - 0.5 * cc + (0.5 * b * b / a if b > 0 else 0)
    assert abs(oracle.flux_marginal(a, b, cc, 0) - ref) < 1e-9 * max(1, abs(ref))
    # real-line prior: the Gaussian integral
    ref2 = -0.5 * cc + b * b / (2 * a) + 0.5 * math.log(2 * math.pi / a)
    assert abs(oracle.flux_marginal(a, b, cc, 1) - ref2) < 1e-12 * max(1, abs(ref2))


def _tiny_facet(N=8):
    acc = np.zeros((4, N * N))
    cells = [(3, 4, 2.0e-4, 1.0e-5, 3, 2.9), (5, 2, 0.6e-4, -2.0e-5, 1, 1.05), (1, 6, 1.1e-4, 0.5e-5, 2, 1.8)]
    for iu, iv, sre, sim, n, ss in cells:
        c = iv * N + iu
        acc[:, c] = [sre, sim, n, ss]
    return acc, cells


def test_p12_grid_likelihood_brute_force():
    N = 8
    p = oracle.default_params(facet_n=N, n_e=3, e_max=0.4, n_alpha=2, r_min_arcsec=0.5, r_max_arcsec=2.0,
                              sigma_jy=2e-5)
    du = 3.0e4
    acc, cells = _tiny_facet(N)
    lg, a, b, nc = oracle.like_grid(acc, du, p)
    assert nc == 3
    for i1, e1 in enumerate((-0.4, 0.0, 0.4)):
        for i2, e2 in enumerate((-0.4, 0.0, 0.4)):
            A = np.array([[1 - e1, -e2], [-e2, 1 + e1]])
            T = np.linalg.inv(A).T
            for k, al_as in enumerate((0.5, 2.0)):
                al = al_as * ARC
                terms = []
                for iu, iv, sre, sim, n, ss in cells:
                    kk = T @ np.array([(iu - N // 2 + 0.5) * du, (iv - N // 2 + 0.5) * du])
                    M = (1 + 4 * math.pi ** 2 * al ** 2 * kk @ kk) ** -1.5
                    terms.append((n / p.sigma_jy ** 2, sre / n, sim / n, ss / n, M))

                def chi2(S):
                    return sum(w * ((dr - S * s * M) ** 2 + di ** 2) for w, dr, di, s, M in terms)
                s0 = sum(w * s * M * dr for w, dr, di, s, M in terms) / sum(w * s * s * M * M for w, dr, di, s, M in terms)
                c0 = chi2(max(s0, 0))
                width = 1 / math.sqrt(sum(w * s * s * M * M for w, dr, di, s, M in terms))
                val, _ = integrate.quad(lambda S: math.exp(-0.5 * (chi2(S) - c0)), 0, max(s0, 0) + 60 * width,
                                        points=[max(s0, 0)], epsabs=0, epsrel=1e-11, limit=400)
                ref = math.log(val) - 0.5 * c0
                assert abs(lg[i1, i2, k] - ref) < 1e-8 * max(1, abs(ref)), (e1, e2, al_as)


def test_grid_nodes_and_validity():
    p = oracle.default_params()
    ge = oracle.grid_e(p)
    assert np.allclose(ge, -0.8 + 0.08 * np.arange(21), atol=1e-15)
    assert int((np.add.outer(ge ** 2, ge ** 2) < 1).sum()) == 417
    ga = oracle.grid_alpha(p)
    assert ga[0] == 0.3 and abs(ga[-1] - 3.5) < 1e-15
    assert np.all(np.diff(np.diff(ga)) > 0)   # quadratic spacing: widening steps
    assert np.allclose(np.diff(np.sqrt(ga - 0.3)), math.sqrt(3.2) / 19)


# ---- scalelength marginal and estimator ---------------------------------------------

@pytest.mark.parametrize("flux", [50e-6, 100e-6, 200e-6, 15e-6])
def test_p13_alpha_prior_mass_and_mean(flux):
    p = oracle.default_params()
    w = oracle.alpha_weight(p, flux)
    mu, s = -0.93 + 0.33 * math.log(flux * 1e6), 0.3136
    lo, hi = math.log(0.3), math.log(3.5)
    mass = stats.norm.cdf((hi - mu) / s) - stats.norm.cdf((lo - mu) / s)
    mean = math.exp(mu + s * s / 2) * (stats.norm.cdf((hi - mu - s * s) / s) - stats.norm.cdf((lo - mu - s * s) / s)) / mass
    # through the estimator: logL independent of alpha
    lg = np.zeros((p.n_e, p.n_e, p.n_alpha))
    ge = oracle.grid_e(p)
    f = -((ge[:, None] - 0.1) ** 2 + (ge[None, :] + 0.2) ** 2) / (2 * 0.2 ** 2)
    lg += f[:, :, None]
    lg[np.add.outer(ge ** 2, ge ** 2) >= 1] = -np.inf
    est, Le = oracle.estimate(lg, np.ones_like(lg), np.ones_like(lg), flux, p)
    i, j = 11, 7
    assert abs(Le[i, j] / math.exp(f[i, j] - f.max()) / mass - 1) < 5e-3
    assert abs(est[oracle.ALPHA] / mean - 1) < 2e-3
    assert abs(w.sum() / mass - 1) < 5e-3


def test_p15_smooth_mean_of_gaussian_likelihood():
    # a Gaussian logL in e, wide against the 0.08 step: the grid mean is the centre
    p = oracle.default_params()
    ge = oracle.grid_e(p)
    mu1, mu2, s = 0.1, -0.05, 0.15
    f = -((ge[:, None] - mu1) ** 2 + (ge[None, :] - mu2) ** 2) / (2 * s * s)
    lg = np.repeat(f[:, :, None], p.n_alpha, axis=2)
    lg[np.add.outer(ge ** 2, ge ** 2) >= 1] = -np.inf
    est, Le = oracle.estimate(lg, np.ones_like(lg), np.ones_like(lg), 1e-4, p)
    assert abs(est[oracle.E1_SMOOTH] - mu1) < 2e-5 and abs(est[oracle.E2_SMOOTH] - mu2) < 2e-5
    # thresholded moments by a plain loop over the grid
    E1, E2 = np.meshgrid(ge, ge, indexing="ij")
    L = np.exp(f - f.max())
    keep = L >= 0.05 * L.max()
    W = L[keep].sum()
    m1, m2 = (L * E1)[keep].sum() / W, (L * E2)[keep].sum() / W
    v1 = (L * (E1 - m1) ** 2)[keep].sum() / W
    assert abs(est[oracle.E1] - m1) < 1e-12 and abs(est[oracle.E2] - m2) < 1e-12
    assert abs(est[oracle.SIG1] - math.sqrt(v1)) < 1e-12
    assert est[oracle.FLAG] == 0.0
    # the thresholded mean stays close to the centre for a wide posterior
    assert abs(est[oracle.E1] - mu1) < 0.02


def test_bad_fit_flag_on_narrow_posterior():
    p = oracle.default_params()
    ge = oracle.grid_e(p)
    f = -((ge[:, None] - 0.16) ** 2 + (ge[None, :] - 0.0) ** 2) / (2 * 0.005 ** 2)
    lg = np.repeat(f[:, :, None], p.n_alpha, axis=2)
    est, _ = oracle.estimate(lg, np.ones_like(lg), np.ones_like(lg), 1e-4, p)
    assert est[oracle.FLAG] == 1.0
    assert abs(est[oracle.E1] - 0.16) < 1e-12 and est[oracle.SIG1] == 0.0


@pytest.mark.parametrize("profile", [0, 1])
def test_pipeline_recovers_isolated_shapes_small_noise(profile):
    # end-to-end on a tiny case: a single source, data simulated with Eq. 1 (or its Gaussian
    # variant) at the true shape, moderate noise; the estimate lies near the truth
    wl = synth.tiny(seed=21, n_src=1, n_ant=24, n_time=24, n_chan=2, r_max_m=1500.0)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    p = oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=2e-5, update_mode=1, profile=profile)
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    d = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                         nu_ref=wl.nu_ref_hz, profile=profile)
    d2 = np.stack([d.real, d.imag], -1).astype(np.float32)
    est, sky = oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, d2, cat.l, cat.m, cat.flux_jy, None, p,
                               want_sky=True)
    assert abs(est[0, oracle.E1] - cat.e1[0]) < 0.1 and abs(est[0, oracle.E2] - cat.e2[0]) < 0.1
    # after the update the sky model holds the measured shape
    upd = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al,
                           est[:, oracle.E1], est[:, oracle.E2], nu_ref=wl.nu_ref_hz, profile=profile)
    assert np.max(np.abs(sky - upd)) < 1e-15


def _sigma_of_equal_fwhm(alpha):
    # the exponential profile's half-maximum radius, then the Gaussian width with the same one
    # (footnote to Sec. 2.2: FWHM = 2 alpha ln 2 and 2 sigma sqrt(2 ln 2)), both solved numerically
    from scipy.optimize import brentq
    r_half = brentq(lambda r: math.exp(-r / alpha) - 0.5, 0.0, 10 * alpha, xtol=1e-15)
    return brentq(lambda sg: math.exp(-r_half ** 2 / (2 * sg * sg)) - 0.5, 1e-3 * alpha, 10 * alpha, xtol=1e-15)


def test_gaussian_profile_is_hankel_transform_of_equal_fwhm_gaussian():
    # circular Gaussian I(r) = exp(-r^2 / (2 sigma^2)) / (2 pi sigma^2): F(k) = 2 pi int r I J0(2 pi k r) dr
    alpha = 1.0
    sg = _sigma_of_equal_fwhm(alpha)
    for k in (0.02, 0.1, 0.35, 0.7):
        f = lambda r: r * math.exp(-r * r / (2 * sg * sg)) / (sg * sg) * special.j0(2 * math.pi * k * r)
        val, err = integrate.quad(f, 0, 40 * sg, limit=2000, epsabs=1e-14, epsrel=1e-12)
        assert abs(val - oracle.shape(k, 0.0, alpha, 0.0, 0.0, 1)) < 1e-9
    # the two profiles differ away from k = 0 and agree at it
    assert oracle.shape(0.0, 0.0, alpha, 0.3, 0.1, 1) == 1.0
    assert abs(oracle.shape(0.3, 0.0, alpha, 0.0, 0.0, 1) - oracle.shape(0.3, 0.0, alpha, 0.0, 0.0, 0)) > 0.01


def test_gaussian_sheared_image_fourier_transform(pixel_grid):
    X, Y, h = pixel_grid
    sg = _sigma_of_equal_fwhm(1.0)
    for e1, e2 in ((0.3, -0.2), (-0.45, 0.1), (0.0, 0.55)):
        A = np.array([[1 - e1, -e2], [-e2, 1 + e1]])
        ax = A[0, 0] * X + A[0, 1] * Y
        ay = A[1, 0] * X + A[1, 1] * Y
        f = abs(np.linalg.det(A)) / (2 * np.pi * sg * sg) * np.exp(-(ax * ax + ay * ay) / (2 * sg * sg))
        for ku, kv in ((0.05, 0.0), (0.0, 0.12), (0.1, 0.07), (0.25, -0.15)):
            F = (f * np.cos(2 * np.pi * (ku * X + kv * Y))).sum() * h * h
            assert abs(F - oracle.shape(ku, kv, 1.0, e1, e2, 1)) < 1e-9, (e1, e2, ku, kv)


# ---- adaptive sampling around the maximum (Sec. 2.4) ----------------------------------

def test_adaptive_sampling_stops_at_the_grid_when_it_has_enough_samples():
    # np_max = 0: the fixed grid already holds enough samples above the threshold, so the
    # adaptive estimate is the grid estimate itself
    wl = synth.tiny(seed=31, n_src=1, n_ant=24, n_time=24, n_chan=2, r_max_m=1500.0)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    p = oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=3e-5)
    al = oracle.alpha_med(cat.flux_jy[0]) * ARC
    d = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, np.array([al]), cat.e1,
                         cat.e2, nu_ref=wl.nu_ref_hz)
    d2 = (np.stack([d.real, d.imag], -1) + synth.noise(obs.n_rows, obs.n_chan, 3e-5, 5)).astype(np.float32)
    du = oracle.facet_du(cat.flux_jy[0], 0.0, p)
    acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, d2, np.zeros_like(d2), cat.l[0], cat.m[0],
                               cat.flux_jy[0], al, 0.0, 0.0, du, p)
    grid = oracle.fit_facet(acc, du, cat.flux_jy[0], p).est
    p.estimator, p.np_max = 1, 0
    ad = oracle.fit_facet_adaptive(acc, du, cat.flux_jy[0], p)
    assert ad[oracle.LEVELS] == 0 and ad[oracle.STEP] == pytest.approx(0.08)
    for f in range(oracle.NC + 1):
        assert ad[f] == grid[f], f


def test_adaptive_sampling_resolves_an_off_grid_source():
    # a noise-free source sampled at cell centres whose shape lies between grid nodes: the
    # fixed grid can only return nodes, the adaptive lattices close in on the true shape
    N, nu = 16, 1.0e9
    p = oracle.default_params(facet_n=N, nu_ref_hz=nu, sigma_jy=1e-7)
    ga = oracle.grid_alpha(p)
    flux = 1.2e-4
    du = oracle.facet_du(flux, 0.0, p)
    rng = np.random.default_rng(19)
    iuv = sorted({(int(a), int(b)) for a, b in rng.integers(1, N - 1, size=(90, 2))})
    u, v, w = _cell_centre_observation(N, du, nu, iuv)
    l, m = 1.1e-3, 0.4e-3
    e1, e2, al = 0.123, -0.057, ga[6] * ARC
    data = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l, m, flux, al, e1, e2, -0.7, nu)] for r in range(len(u))])
    d2 = np.stack([data.real, data.imag], -1)
    # the sky model holds the source at its current shape, so the facet holds its model alone
    acc = oracle.extract_facet(u, v, w, np.array([nu]), d2.astype(np.float32), d2, l, m, flux, al,
                               e1, e2, du, p)
    grid = oracle.fit_facet(acc, du, flux, p).est
    assert max(abs(grid[oracle.E1] - e1), abs(grid[oracle.E2] - e2)) > 0.01
    p.estimator = 1
    ad = oracle.fit_facet_adaptive(acc, du, flux, p)
    assert ad[oracle.LEVELS] >= 1
    assert ad[oracle.STEP] == pytest.approx(0.08 / 2 ** ad[oracle.LEVELS])
    assert ad[oracle.NKEPT] >= p.np_max or ad[oracle.STEP] <= p.e_res          # the stopping rule
    assert abs(ad[oracle.E1] - e1) < p.e_res and abs(ad[oracle.E2] - e2) < p.e_res
    assert abs(ad[oracle.FLUX] / flux - 1) < 1e-2


def test_adaptive_sampling_of_a_resolved_posterior_stops_early():
    # a broad posterior (low SNR) keeps more than np_max grid samples above the threshold:
    # no refinement
    wl = synth.tiny(seed=33, n_src=1, n_ant=24, n_time=24, n_chan=2, r_max_m=1500.0)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    p = oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=5e-4, estimator=1)
    al = oracle.alpha_med(cat.flux_jy[0]) * ARC
    d2 = synth.noise(obs.n_rows, obs.n_chan, 5e-4, 8).astype(np.float32)
    du = oracle.facet_du(cat.flux_jy[0], 0.0, p)
    acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, d2, np.zeros_like(d2), cat.l[0], cat.m[0],
                               cat.flux_jy[0], al, 0.0, 0.0, du, p)
    ad = oracle.fit_facet_adaptive(acc, du, cat.flux_jy[0], p)
    assert ad[oracle.LEVELS] == 0 and ad[oracle.NKEPT] >= p.np_max


# ---- refit of the bad fits after the whole catalogue (Sec. 2.4) --------------------------

def _refit_case(sigma):
    wl = synth.tiny(seed=41, n_src=3, n_ant=24, n_time=24, n_chan=2, r_max_m=1500.0)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    d = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                         nu_ref=wl.nu_ref_hz)
    d2 = (np.stack([d.real, d.imag], -1) + synth.noise(obs.n_rows, obs.n_chan, sigma, 7)).astype(np.float32)
    return wl, obs, cat, al, d2


def test_refit_changes_nothing_without_bad_fits():
    wl, obs, cat, al, d2 = _refit_case(3e-4)
    p = oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=3e-4, update_mode=1)
    est0 = oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, d2, cat.l, cat.m, cat.flux_jy, None, p)
    assert np.all(est0[:, oracle.FLAG] == 0)
    p.refit_bad = 1
    est1 = oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, d2, cat.l, cat.m, cat.flux_jy, None, p)
    assert np.array_equal(est0, est1) and np.all(est1[:, oracle.REFIT] == 0)


def test_refit_fits_bad_sources_against_the_final_sky_model():
    # every fit is bad (the posteriors collapse onto grid nodes): each source is fitted once
    # more against the sky model that holds every main-pass shape; rebuilt here from the
    # oracle's sky model, extraction and fit
    wl, obs, cat, al, d2 = _refit_case(1e-7)
    p = oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=1e-7, update_mode=1)
    main = oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, d2, cat.l, cat.m, cat.flux_jy, None, p)
    assert np.all(main[:, oracle.FLAG] != 0)
    p.refit_bad = 1
    est = oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, d2, cat.l, cat.m, cat.flux_jy, None, p)
    assert np.all(est[:, oracle.REFIT] == 1)
    sky = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, main[:, oracle.E1],
                           main[:, oracle.E2], nu_ref=wl.nu_ref_hz)
    s2 = np.stack([sky.real, sky.imag], -1)
    for i in range(cat.n_src):
        du = oracle.facet_du(cat.flux_jy[i], 0.0, p)
        acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, d2, s2, cat.l[i], cat.m[i], cat.flux_jy[i],
                                   al[i], main[i, oracle.E1], main[i, oracle.E2], du, p)
        ref = oracle.fit_facet(acc, du, cat.flux_jy[i], p).est
        for f in (oracle.E1, oracle.E2, oracle.SIG1, oracle.SIG2, oracle.FLUX, oracle.FLAG):
            assert abs(est[i, f] - ref[f]) <= 1e-12 * max(1.0, abs(ref[f])), (i, f)


@pytest.mark.parametrize("profile", [0, 1])
@pytest.mark.parametrize("uniform", [True, False])
def test_simulated_data_equals_sky_model(profile, uniform):
    # the data generator of large observations is the sky model's sum arranged for speed
    # (per-row-source terms hoisted, channel phases by the step's rotation): it must agree
    # with the plain double loop to rounding, on uniform and uneven channel sets
    wl = synth.tiny(seed=3, n_src=7, n_chan=5)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    freq = obs.freq_hz if uniform else np.array([0.95e9, 0.97e9, 1.0e9, 1.06e9, 1.2e9])
    args = (obs.u, obs.v, obs.w, freq, cat.l, cat.m, cat.flux_jy, cat.alpha_arcsec * ARC, cat.e1, cat.e2)
    ref, ab = oracle.sky_model(*args, nu_ref=wl.nu_ref_hz, with_abs=True, profile=profile)
    got = oracle.simulate_vis(*args, nu_ref=wl.nu_ref_hz, profile=profile)
    assert np.max(np.abs(got[..., 0] + 1j * got[..., 1] - ref) / ab) < 1e-12
