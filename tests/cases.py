"""Shared builders for the GPU parity tests: seeded inputs, oracle references,
device copies.  Inputs come from ``synth`` and expected values from ``oracle``;
nothing here is computed by the CUDA path."""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import oracle
import synth

ARC = math.pi / 648000.0


@dataclasses.dataclass
class Case:
    wl: synth.Workload
    obs: synth.Observation
    cat: synth.Catalogue
    sigma: float
    data: np.ndarray | None = None      # [R, C, 2] float32
    sky0: np.ndarray | None = None      # [R, C, 2] float32 (circular sky model)
    profile: int = 0                    # 0 exponential (Eq. 1), 1 Gaussian of equal FWHM

    def oracle_params(self, **kw):
        kw.setdefault("nu_ref_hz", self.wl.nu_ref_hz)
        kw.setdefault("sigma_jy", self.sigma)
        kw.setdefault("profile", self.profile)
        return oracle.default_params(**kw)

    def alpha_med_rad(self):
        return np.array([oracle.alpha_med(s) for s in self.cat.flux_jy]) * ARC


def snr10_sigma(obs: synth.Observation, cat: synth.Catalogue) -> float:
    """Noise per component that gives the faintest source an SNR of about 10."""
    return float(cat.flux_jy.min() * math.sqrt(obs.n_rows * obs.n_chan) / 10.0)


def build(wl: synth.Workload, sigma: float | None = None, with_data: bool = True, snr10: bool = False,
          n_src: int | None = None, profile: int = 0) -> Case:
    obs = synth.make_observation(wl)
    cat = synth.make_catalogue(wl, n_src)
    if snr10:
        sigma = snr10_sigma(obs, cat)
    sigma = wl.sigma_jy if sigma is None else sigma
    c = Case(wl, obs, cat, sigma, profile=profile)
    if with_data:
        c.data = data_from(true_sky(c), sigma, wl.seed)
        z = np.zeros(cat.n_src)
        s0 = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, c.alpha_med_rad(), z, z,
                              nu_ref=wl.nu_ref_hz, profile=profile)
        c.sky0 = np.stack([s0.real, s0.imag], -1).astype(np.float32)
    return c


def true_sky(c: Case) -> np.ndarray:
    """The oracle's sky model at the catalogue's true shapes and scalelengths, complex128 [R, C]."""
    return oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                            c.cat.alpha_arcsec * ARC, c.cat.e1, c.cat.e2, nu_ref=c.wl.nu_ref_hz, profile=c.profile)


def data_from(true: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Data visibilities: true sky plus seeded Gaussian noise, rounded to complex64 ([R, C, 2] float32)."""
    d = np.stack([true.real, true.imag], -1)
    d += synth.noise(true.shape[0], true.shape[1], sigma, seed, dtype=np.float64)
    return d.astype(np.float32)


def fingerprint(data: np.ndarray) -> dict:
    """A few numbers that identify a data array (sums in float64 and sampled values)."""
    flat = data.reshape(-1).astype(np.float64)
    idx = np.linspace(0, flat.size - 1, 16).astype(np.int64)
    return {"sum": float(flat.sum()), "sum_sq": float(np.dot(flat, flat)), "idx": idx.tolist(),
            "values": flat[idx].tolist()}


def to_device(case: Case, e1=None, e2=None, alpha_arcsec=None, device="cuda"):
    import torch

    import paper_2203_14071_gb300 as rlf
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    obs = rlf.Observation(t(case.obs.u), t(case.obs.v), t(case.obs.w), case.obs.freq_hz, case.obs.n_bl)
    z = np.zeros(case.cat.n_src)
    cat = rlf.Catalogue(t(case.cat.l), t(case.cat.m), t(case.cat.flux_jy), t(z if e1 is None else e1),
                        t(z if e2 is None else e2), None if alpha_arcsec is None else t(alpha_arcsec))
    return obs, cat


def vis_tensor(a: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)


def est_matches(got: dict, i: int, est: np.ndarray, tol_e: float = 1e-4, margin_min: float = 1e-3):
    """Compare one source's GPU result with the oracle's estimate record.

    When a grid point's marginal lies within `margin_min` (in ln L) of the
    threshold, a rounding difference may flip it in or out of the kept set, so
    the threshold-free mean is compared instead."""
    if est[oracle.THRESH_MARGIN] < margin_min:
        d1 = abs(got["e1_smooth"][i] - est[oracle.E1_SMOOTH])
        d2 = abs(got["e2_smooth"][i] - est[oracle.E2_SMOOTH])
    else:
        d1 = abs(got["e1"][i] - est[oracle.E1])
        d2 = abs(got["e2"][i] - est[oracle.E2])
    return max(d1, d2)
