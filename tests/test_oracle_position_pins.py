"""Pins of the oracle's position marginalisation (Sec. 2.4: the likelihood is
marginalised over the source position with a uniform prior, semi-analytically).

Reading: the prior is uniform over an n_pos x n_pos grid of offsets x0 around the
catalogue position (step pos_step_arcsec).  An offset source's facet model is the
centred model times exp(+2 pi i k.x0) (Eq. 1 after the facet's phase shift), so the
marginal is the mean over offsets of the flux-marginalised likelihood.  The pins:
brute force of that definition (complex residuals, flux integral by quadrature), a
source displaced in the visibilities and extracted at the catalogue position, the
zero-step limit, and the parameter checks.  The offset grid is symmetric about the
catalogue position, so the outputs are invariant under x0 -> -x0 and l <-> m: the
sign of the phase and the order of the offsets are fixed by no output and need no pin.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

C = 299792458.0
ARC = math.pi / 648000.0


def _offsets(n_pos, step_arcsec):
    h = (n_pos - 1) // 2
    return [((i - h) * step_arcsec * ARC, (j - h) * step_arcsec * ARC) for i in range(n_pos) for j in range(n_pos)]


def _complex_facet(N=8):
    # a few cells with complex means: sum Re, sum Im, count, sum spectral factor
    acc = np.zeros((4, N * N))
    cells = [(3, 4, 2.0e-4, 0.9e-4, 3, 2.9), (5, 2, 0.6e-4, -1.1e-4, 1, 1.05), (1, 6, 1.1e-4, 0.5e-4, 2, 1.8),
             (6, 5, -0.4e-4, 0.7e-4, 4, 3.7)]
    for iu, iv, sre, sim, n, ss in cells:
        acc[:, iv * N + iu] = [sre, sim, n, ss]
    return acc, cells


@pytest.mark.parametrize("n_pos,step,flux_prior,profile", [(3, 0.7, 0, 0), (5, 0.45, 0, 0), (3, 0.7, 1, 0),
                                                             (3, 0.7, 0, 1)])
def test_position_marginal_brute_force(n_pos, step, flux_prior, profile):
    # mean over offsets of int exp(-chi2(S, x0)/2) dS (S >= 0, or the real line with
    # flux_prior 1), with chi2 the sum of complex residuals |D_c - S s_c M_c
    # exp(2 pi i k_c.x0)|^2 w_c, done by quadrature; both source profiles
    N = 8
    p = oracle.default_params(facet_n=N, n_e=3, e_max=0.4, n_alpha=2, r_min_arcsec=0.5, r_max_arcsec=2.0,
                              sigma_jy=4e-5, n_pos=n_pos, pos_step_arcsec=step, flux_prior=flux_prior,
                              profile=profile)
    du = 3.0e4
    acc, cells = _complex_facet(N)
    lg, a, b, nc = oracle.like_grid(acc, du, p)
    assert nc == len(cells)
    for i1, e1 in enumerate((-0.4, 0.0, 0.4)):
        for i2, e2 in enumerate((-0.4, 0.0, 0.4)):
            for k, al_as in enumerate((0.5, 2.0)):
                al = al_as * ARC
                terms = []
                for iu, iv, sre, sim, n, ss in cells:
                    ku, kv = (iu - N // 2 + 0.5) * du, (iv - N // 2 + 0.5) * du
                    terms.append((n / p.sigma_jy ** 2, (sre + 1j * sim) / n, ss / n,
                                  oracle.shape(ku, kv, al, e1, e2, profile=profile), ku, kv))
                vals, peaks = [], []
                for dl, dm in _offsets(n_pos, step):
                    ph = [np.exp(2j * math.pi * (ku * dl + kv * dm)) for *_, ku, kv in terms]

                    def chi2(S):
                        return sum(w * abs(d - S * s * M * z) ** 2 for (w, d, s, M, _, _), z in zip(terms, ph))
                    aa = sum(w * s * s * M * M for w, d, s, M, _, _ in terms)
                    bb = sum(w * s * M * (d * np.conj(z)).real for (w, d, s, M, _, _), z in zip(terms, ph))
                    s0 = bb / aa if flux_prior == 1 else max(bb / aa, 0.0)
                    c0 = chi2(s0)
                    lo = s0 - 60 / math.sqrt(aa) if flux_prior == 1 else 0.0
                    val, _ = integrate.quad(lambda S: math.exp(-0.5 * (chi2(S) - c0)), lo, s0 + 60 / math.sqrt(aa),
                                            points=[s0], epsabs=0, epsrel=1e-11, limit=400)
                    vals.append(math.log(val) - 0.5 * c0)
                    peaks.append(bb)
                vals = np.array(vals)
                ref = vals.max() + math.log(np.mean(np.exp(vals - vals.max())))
                assert abs(lg[i1, i2, k] - ref) < 1e-8 * max(1, abs(ref)), (e1, e2, al_as)
                # b reported at the best offset
                assert b[i1, i2, k] == pytest.approx(peaks[int(np.argmax(vals))], rel=1e-12)


def test_displaced_source_is_recovered_at_its_offset():
    # a noise-free source whose true position is off the catalogue position by a grid
    # offset (+1 step in l, -2 steps in m), sampled at cell centres with w = 0 and
    # extracted at the catalogue position: with the position marginal the chi^2 at the
    # true node and offset is zero, so the flux comes back exactly and the shape is the
    # true node; taking the position as exact loses flux at the true node (the model
    # and data are out of phase) and moves the estimate off it
    N, nu = 16, 1.0e9
    step = 1.0
    p = oracle.default_params(facet_n=N, nu_ref_hz=nu, n_e=11, e_max=0.5, n_alpha=6, sigma_jy=1e-7,
                              n_pos=5, pos_step_arcsec=step)
    ge, ga = oracle.grid_e(p), oracle.grid_alpha(p)
    flux = 1.2e-4
    du = oracle.facet_du(flux, 0.0, p)
    rng = np.random.default_rng(23)
    iuv = sorted({(int(a), int(b)) for a, b in rng.integers(2, N - 2, size=(70, 2))})
    u = np.array([(iu - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    v = np.array([(iv - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    w = np.zeros(len(iuv))
    l0, m0 = 1.5e-3, -0.8e-3
    dl, dm = 1 * step * ARC, -2 * step * ARC
    i1, i2, k = 7, 3, 2
    e1, e2, al = ge[i1], ge[i2], ga[k] * ARC
    data = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l0 + dl, m0 + dm, flux, al, e1, e2, -0.7, nu)]
                     for r in range(len(u))])
    # the sky model holds the catalogue source (catalogue position, current shape e = 0), which
    # extraction subtracts and adds back: the facet holds the displaced data alone
    sky = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l0, m0, flux, al, 0.0, 0.0, -0.7, nu)]
                    for r in range(len(u))])
    d2 = np.stack([data.real, data.imag], -1)
    s2 = np.stack([sky.real, sky.imag], -1)
    acc = oracle.extract_facet(u, v, w, np.array([nu]), d2.astype(np.float32), s2, l0, m0, flux, al, 0.0, 0.0,
                               du, p)
    fit = oracle.fit_facet(acc, du, flux, p)
    g = int(fit.est[oracle.MAP_INDEX])
    assert g == (i1 * p.n_e + i2) * p.n_alpha + k
    assert abs(fit.est[oracle.E1] - e1) < 1e-12 and abs(fit.est[oracle.E2] - e2) < 1e-12
    assert abs(fit.est[oracle.FLUX] / flux - 1) < 1e-6       # float32 data
    # the best offset's b is the true one: b = S a at the true node
    assert fit.b.reshape(-1)[g] == pytest.approx(flux * fit.a.reshape(-1)[g], rel=1e-6)
    p.n_pos = 1
    exact = oracle.fit_facet(acc, du, flux, p)
    assert exact.b.reshape(-1)[g] < 0.99 * flux * exact.a.reshape(-1)[g]
    assert int(exact.est[oracle.MAP_INDEX]) != g
    assert exact.loglike.max() < fit.loglike.max()


def test_zero_step_reduces_to_the_exact_position():
    # every offset coincides: the mean of n_pos^2 equal likelihoods is that likelihood
    N = 8
    acc, _ = _complex_facet(N)
    base = dict(facet_n=N, n_e=5, e_max=0.6, n_alpha=3, sigma_jy=4e-5)
    lg1, a1, b1, _ = oracle.like_grid(acc, 3.0e4, oracle.default_params(**base))
    lg3, a3, b3, _ = oracle.like_grid(acc, 3.0e4, oracle.default_params(n_pos=3, pos_step_arcsec=0.0, **base))
    ok = np.isfinite(lg1)
    assert np.array_equal(ok, np.isfinite(lg3))
    assert np.max(np.abs(lg3[ok] - lg1[ok])) < 1e-12 * np.max(np.abs(lg1[ok]))
    assert np.array_equal(a1, a3) and np.max(np.abs(b3 - b1)) <= 1e-15 * np.max(np.abs(b1))


def test_one_offset_is_the_exact_position_bit_for_bit():
    N = 8
    acc, _ = _complex_facet(N)
    base = dict(facet_n=N, n_e=5, e_max=0.6, n_alpha=3, sigma_jy=4e-5)
    r1 = oracle.like_grid(acc, 3.0e4, oracle.default_params(**base))
    r2 = oracle.like_grid(acc, 3.0e4, oracle.default_params(n_pos=1, pos_step_arcsec=5.0, **base))
    for x, y in zip(r1[:3], r2[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n_pos", [2, 4, 9])
def test_unsupported_offset_grids_give_nan(n_pos):
    N = 8
    acc, _ = _complex_facet(N)
    lg, a, b, _ = oracle.like_grid(acc, 3.0e4, oracle.default_params(facet_n=N, n_e=3, n_alpha=2, n_pos=n_pos))
    assert np.all(np.isnan(lg[np.isfinite(lg) | np.isnan(lg)]))


def test_adaptive_sampling_with_the_position_marginal():
    # a noise-free source off the e grid and displaced by a grid offset: adaptive sampling
    # with the position marginal closes in on the true shape, as it does for an undisplaced
    # source without the marginal
    N, nu = 16, 1.0e9
    step = 0.5
    p = oracle.default_params(facet_n=N, nu_ref_hz=nu, sigma_jy=1e-7, n_pos=3, pos_step_arcsec=step, estimator=1)
    ga = oracle.grid_alpha(p)
    flux = 1.2e-4
    du = oracle.facet_du(flux, 0.0, p)
    rng = np.random.default_rng(29)
    iuv = sorted({(int(a), int(b)) for a, b in rng.integers(1, N - 1, size=(90, 2))})
    u = np.array([(iu - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    v = np.array([(iv - N // 2 + 0.5) * du * C / nu for iu, iv in iuv])
    w = np.zeros(len(iuv))
    l0, m0 = 1.1e-3, 0.4e-3
    e1, e2, al = 0.123, -0.057, ga[6] * ARC
    data = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l0 - step * ARC, m0 + step * ARC, flux, al, e1, e2,
                                       -0.7, nu)] for r in range(len(u))])
    sky = np.array([[oracle.model_vis(u[r], v[r], w[r], nu, l0, m0, flux, al, 0.0, 0.0, -0.7, nu)]
                    for r in range(len(u))])
    d2 = np.stack([data.real, data.imag], -1)
    s2 = np.stack([sky.real, sky.imag], -1)
    acc = oracle.extract_facet(u, v, w, np.array([nu]), d2.astype(np.float32), s2, l0, m0, flux, al, 0.0, 0.0,
                               du, p)
    ad = oracle.fit_facet_adaptive(acc, du, flux, p)
    assert ad[oracle.LEVELS] >= 1
    assert abs(ad[oracle.E1] - e1) < p.e_res and abs(ad[oracle.E2] - e2) < p.e_res
    assert abs(ad[oracle.FLUX] / flux - 1) < 1e-2
    # without the marginal the displaced source's estimate is off by more than E_RES
    p.n_pos = 1
    ex = oracle.fit_facet_adaptive(acc, du, flux, p)
    assert max(abs(ex[oracle.E1] - e1), abs(ex[oracle.E2] - e2)) > p.e_res


def test_flux_marginal_grows_with_b():
    # the position marginal's best offset is the one with the largest b (S >= 0 prior) or
    # the largest |b| (real-line prior): for fixed a and C, d ln L / d b is the posterior
    # mean of S, positive when S >= 0, and with S on the real line ln L = b^2/(2a) + const;
    # checked on random pairs
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a = 10 ** rng.uniform(-2, 12)
        scale = math.sqrt(a)
        b1, b2 = np.sort(rng.normal(0.0, 1.0, 2) * scale * 10 ** rng.uniform(-3, 2))
        if b1 == b2:
            continue
        cc = 1.0
        assert oracle.flux_marginal(a, b2, cc, 0) >= oracle.flux_marginal(a, b1, cc, 0), (a, b1, b2)
        l1, l2 = oracle.flux_marginal(a, b1, cc, 1), oracle.flux_marginal(a, b2, cc, 1)
        assert (l2 >= l1) == (abs(b2) >= abs(b1)) or l1 == l2, (a, b1, b2)
