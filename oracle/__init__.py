"""FP64 CPU oracle of the RadioLensfit hot path (arXiv 2203.14071).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports this package and shares no code with it.

The arithmetic lives in ``rlf_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Functions and the passages they follow:

    model_vis        Eq. 1 + Eq. 2 (Sec. 2.2)
    alpha_med        Eq. 4 (Sec. 2.2)
    sky_model        sum of Eq. 1 over the catalogue (Sec. 2.2)
    simulate_vis     the same sum arranged for speed (test data of large observations)
    extract_facet    Sec. 2.3 (residual, phase shift, facet of K * alpha)
    fit_facet        Sec. 2.4 (chi^2, flux, scalelength and position marginals,
                     estimate)
    fit_facet_adaptive  Sec. 2.4 (adaptive sampling around the maximum)
    pipeline         Sec. 2 and Sec. 3.1 (chunked sky-model update), Sec. 2.4
                     (refit of bad fits)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librlf_oracle.so")
_lock = threading.Lock()
_lib = None

NEST = 17
(E1, E2, SIG1, SIG2, ALPHA, FLUX, FLAG, E1_SMOOTH, E2_SMOOTH, LOGL_MAX, THRESH_MARGIN, MAP_INDEX, NC,
 LEVELS, STEP, NKEPT, REFIT) = range(NEST)
C_LIGHT = 299792458.0
ARCSEC = np.pi / 648000.0


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, OpenMP).  Expressions are
    evaluated as written (no FMA contraction), so the oracle gives the same results on
    x86-64 and aarch64."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Algorithm parameters; defaults are the paper's values (Sec. 2.2-2.4, Sec. 4.1-4.2)."""
    _fields_ = [("add", ctypes.c_double), ("esp", ctypes.c_double), ("psf_nat", ctypes.c_double),
                ("beta", ctypes.c_double), ("nu_ref_hz", ctypes.c_double), ("sigma_jy", ctypes.c_double),
                ("e_max", ctypes.c_double), ("r_min_arcsec", ctypes.c_double),
                ("r_max_arcsec", ctypes.c_double), ("r_std", ctypes.c_double),
                ("thresh_frac", ctypes.c_double), ("var_sigma_min", ctypes.c_double),
                ("var_det_min", ctypes.c_double), ("facet_n", ctypes.c_int32), ("n_e", ctypes.c_int32),
                ("n_alpha", ctypes.c_int32), ("flux_prior", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("update_mode", ctypes.c_int32), ("profile", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("e_res", ctypes.c_double), ("np_max", ctypes.c_int32), ("estimator", ctypes.c_int32),
                ("refit_bad", ctypes.c_int32), ("pad2", ctypes.c_int32), ("pos_step_arcsec", ctypes.c_double),
                ("n_pos", ctypes.c_int32), ("pad3", ctypes.c_int32)]


def default_params(**kw) -> Params:
    p = Params(add=-0.93, esp=0.33, psf_nat=38.0, beta=-0.7, nu_ref_hz=1.0e9, sigma_jy=1e-6,
               e_max=0.8, r_min_arcsec=0.3, r_max_arcsec=3.5, r_std=0.3136,
               thresh_frac=0.05, var_sigma_min=5e-3, var_det_min=5e-5,
               facet_n=64, n_e=21, n_alpha=20, flux_prior=0, chunk=0, update_mode=0, profile=0, pad=0,
               e_res=0.003, np_max=30, estimator=0, refit_bad=0, pad2=0, pos_step_arcsec=0.1, n_pos=1, pad3=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            L.rlfo_nest.restype = ctypes.c_int
            L.rlfo_params_size.restype = ctypes.c_int
            L.rlfo_alpha_med.restype = d
            L.rlfo_alpha_med.argtypes = [d, d, d]
            L.rlfo_shape.restype = d
            L.rlfo_shape.argtypes = [d, d, d, d, d, ctypes.c_int]
            L.rlfo_model_vis.restype = None
            L.rlfo_model_vis.argtypes = [d] * 12 + [ctypes.c_int, vp, vp]
            L.rlfo_sky_model.restype = None
            L.rlfo_sky_model.argtypes = [i64, i32, vp, vp, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp, vp,
                                         d, d, ctypes.c_int, vp, vp, ctypes.c_int]
            L.rlfo_simulate_vis.restype = None
            L.rlfo_simulate_vis.argtypes = [i64, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp,
                                            d, d, ctypes.c_int, vp, ctypes.c_int]
            L.rlfo_extract_facet.restype = None
            L.rlfo_extract_facet.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, vp] + [d] * 8 + \
                                            [ctypes.c_int, d, i32, vp, vp]
            L.rlfo_flux_marginal.restype = d
            L.rlfo_flux_marginal.argtypes = [d, d, d, ctypes.c_int]
            L.rlfo_grid_e.restype = d
            L.rlfo_grid_e.argtypes = [vp, ctypes.c_int]
            L.rlfo_grid_alpha.restype = d
            L.rlfo_grid_alpha.argtypes = [vp, ctypes.c_int]
            L.rlfo_fit_facet_adaptive.restype = None
            L.rlfo_fit_facet_adaptive.argtypes = [vp, d, d, vp, vp]
            L.rlfo_fit_facet.restype = None
            L.rlfo_fit_facet.argtypes = [vp, d, d, vp, vp, vp, vp, vp]
            L.rlfo_like_grid.restype = ctypes.c_int
            L.rlfo_like_grid.argtypes = [vp, d, vp, vp, vp, vp]
            L.rlfo_estimate.restype = None
            L.rlfo_estimate.argtypes = [vp, vp, vp, d, ctypes.c_int, vp, vp, vp]
            L.rlfo_alpha_weight.restype = d
            L.rlfo_alpha_weight.argtypes = [vp, d, ctypes.c_int]
            L.rlfo_facet_du.restype = d
            L.rlfo_facet_du.argtypes = [d, d, vp]
            L.rlfo_pipeline.restype = ctypes.c_int
            L.rlfo_pipeline.argtypes = [i64, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp,
                                        vp, ctypes.c_int]
            assert L.rlfo_nest() == NEST
            assert L.rlfo_params_size() == ctypes.sizeof(Params)
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def alpha_med(flux_jy: float, add: float = -0.93, esp: float = 0.33) -> float:
    """Eq. 4: median scalelength in arcsec."""
    return lib().rlfo_alpha_med(flux_jy, add, esp)


def shape(ku, kv, alpha_rad, e1, e2, profile: int = 0) -> float:
    """Eq. 1 brightness factor; profile 0 exponential, 1 Gaussian of equal FWHM."""
    return lib().rlfo_shape(ku, kv, alpha_rad, e1, e2, profile)


def model_vis(u, v, w, freq, l, m, flux, alpha_rad, e1, e2, beta=-0.7, nu_ref=1.0e9, profile: int = 0) -> complex:
    """Eq. 1 for one source at one baseline (metres) and frequency (Hz)."""
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().rlfo_model_vis(u, v, w, freq, l, m, flux, alpha_rad, e1, e2, beta, nu_ref, profile,
                         ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def sky_model(u, v, w, freq, l, m, flux, alpha_rad, e1, e2, beta=-0.7, nu_ref=1.0e9,
              rows=None, with_abs=False, n_threads=0, profile: int = 0):
    """Sky model (Sec. 2.2) as complex128 [n_out, n_chan]; optionally also sum |term|."""
    u, v, w, freq = _f64(u), _f64(v), _f64(w), _f64(freq)
    l, m, flux, alpha_rad, e1, e2 = map(_f64, (l, m, flux, alpha_rad, e1, e2))
    n_rows, n_chan = u.shape[0], freq.shape[0]
    rows_a = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    n_out = n_rows if rows_a is None else rows_a.shape[0]
    out = np.zeros((n_out, n_chan, 2), dtype=np.float64)
    ab = np.zeros((n_out, n_chan), dtype=np.float64) if with_abs else None
    lib().rlfo_sky_model(n_rows, n_chan, _p(u), _p(v), _p(w), _p(freq), _p(rows_a), n_out,
                         l.shape[0], _p(l), _p(m), _p(flux), _p(alpha_rad), _p(e1), _p(e2),
                         beta, nu_ref, profile, _p(out), _p(ab), n_threads)
    vis = out[..., 0] + 1j * out[..., 1]
    return (vis, ab) if with_abs else vis


def simulate_vis(u, v, w, freq, l, m, flux, alpha_rad, e1, e2, beta=-0.7, nu_ref=1.0e9, profile: int = 0,
                 n_threads=0) -> np.ndarray:
    """Data visibilities of a synthetic observation, [n_rows, n_chan, 2] float64: the sum of
    Eq. 1 over the catalogue (as sky_model), arranged for speed; test inputs only."""
    u, v, w, freq = _f64(u), _f64(v), _f64(w), _f64(freq)
    l, m, flux, alpha_rad, e1, e2 = map(_f64, (l, m, flux, alpha_rad, e1, e2))
    out = np.empty((u.shape[0], freq.shape[0], 2), dtype=np.float64)
    lib().rlfo_simulate_vis(u.shape[0], freq.shape[0], _p(u), _p(v), _p(w), _p(freq), l.shape[0], _p(l), _p(m),
                            _p(flux), _p(alpha_rad), _p(e1), _p(e2), beta, nu_ref, profile, _p(out), n_threads)
    return out


def facet_du(flux_jy: float, alpha_cat_arcsec: float, params: Params) -> float:
    return lib().rlfo_facet_du(flux_jy, alpha_cat_arcsec, ctypes.byref(params))


def extract_facet(u, v, w, freq, data, sky, l, m, flux, alpha_sky_rad, e1_cur, e2_cur, du,
                  params: Params, with_abs=False):
    """Facet of one source (Sec. 2.3): [4, N*N] = sum Re, sum Im, count, sum spectral factor.

    data, sky: [n_rows, n_chan, 2] float32 (complex64 layout); sky may be float64.
    """
    u, v, w, freq = _f64(u), _f64(v), _f64(w), _f64(freq)
    data = _f32(data)
    sky_f = sky_d = None
    if sky.dtype == np.float64:
        sky_d = np.ascontiguousarray(sky)
    else:
        sky_f = _f32(sky)
    N = params.facet_n
    acc = np.zeros((4, N * N), dtype=np.float64)
    ab = np.zeros(N * N, dtype=np.float64) if with_abs else None
    lib().rlfo_extract_facet(u.shape[0], freq.shape[0], _p(u), _p(v), _p(w), _p(freq), _p(data),
                             _p(sky_f), _p(sky_d), l, m, flux, alpha_sky_rad, e1_cur, e2_cur,
                             params.beta, params.nu_ref_hz, params.profile, du, N, _p(acc), _p(ab))
    return (acc, ab) if with_abs else acc


@dataclasses.dataclass
class Fit:
    loglike: np.ndarray   # [n_e, n_e, n_alpha]
    a: np.ndarray
    b: np.ndarray
    est: np.ndarray       # [NEST]


def fit_facet_adaptive(acc, du, flux_cat, params: Params) -> np.ndarray:
    """Estimate of one facet by adaptive sampling around the maximum (Sec. 2.4):
    the fixed grid, then halved lattices around the kept samples until np_max of
    them or a step of e_res.  Returns est [NEST] (LEVELS, STEP, NKEPT filled)."""
    est = np.zeros(NEST)
    lib().rlfo_fit_facet_adaptive(_p(_f64(acc)), du, flux_cat, ctypes.byref(params), _p(est))
    return est


def fit_facet(acc, du, flux_cat, params: Params) -> Fit:
    """Likelihood grid, marginals and estimate of one facet (Sec. 2.4)."""
    acc = _f64(acc)
    ne, na = params.n_e, params.n_alpha
    lg = np.zeros((ne, ne, na))
    a = np.zeros_like(lg)
    b = np.zeros_like(lg)
    est = np.zeros(NEST)
    lib().rlfo_fit_facet(_p(acc), du, flux_cat, ctypes.byref(params), _p(lg), _p(a), _p(b), _p(est))
    return Fit(lg, a, b, est)


def like_grid(acc, du, params: Params):
    """Likelihood grid (Sec. 2.4): (loglike, a, b, n_cells), each grid [n_e, n_e, n_alpha]."""
    acc = _f64(acc)
    ne, na = params.n_e, params.n_alpha
    lg = np.zeros((ne, ne, na))
    a = np.zeros_like(lg)
    b = np.zeros_like(lg)
    nc = lib().rlfo_like_grid(_p(acc), du, ctypes.byref(params), _p(lg), _p(a), _p(b))
    return lg, a, b, nc


def estimate(loglike, a, b, flux_cat, params: Params, ncell=1):
    """Estimate from a likelihood grid (Sec. 2.4): (est [NEST], L(e) [n_e, n_e])."""
    lg, a, b = _f64(loglike), _f64(a), _f64(b)
    est = np.zeros(NEST)
    Le = np.zeros((params.n_e, params.n_e))
    lib().rlfo_estimate(_p(lg), _p(a), _p(b), flux_cat, ncell, ctypes.byref(params), _p(est), _p(Le))
    return est, Le


def alpha_weight(params: Params, flux_cat: float) -> np.ndarray:
    """Trapezoid weight times log-normal prior density at each scalelength node."""
    return np.array([lib().rlfo_alpha_weight(ctypes.byref(params), flux_cat, k)
                     for k in range(params.n_alpha)])


def flux_marginal(a, b, cc, flux_prior=0) -> float:
    return lib().rlfo_flux_marginal(a, b, cc, flux_prior)


def grid_e(params: Params) -> np.ndarray:
    return np.array([lib().rlfo_grid_e(ctypes.byref(params), k) for k in range(params.n_e)])


def grid_alpha(params: Params) -> np.ndarray:
    return np.array([lib().rlfo_grid_alpha(ctypes.byref(params), k) for k in range(params.n_alpha)])


def pipeline(obs_u, obs_v, obs_w, freq, data, l, m, flux, alpha_cat_arcsec, params: Params,
             want_sky=False, n_threads=0):
    """Whole chain (Sec. 2, Sec. 3.1) -> est [n_src, NEST] (and the final sky model)."""
    u, v, w, freq = _f64(obs_u), _f64(obs_v), _f64(obs_w), _f64(freq)
    data = _f32(data)
    l, m, flux = _f64(l), _f64(m), _f64(flux)
    ac = None if alpha_cat_arcsec is None else _f64(alpha_cat_arcsec)
    n = l.shape[0]
    est = np.zeros((n, NEST))
    sky = np.zeros((u.shape[0], freq.shape[0], 2)) if want_sky else None
    rc = lib().rlfo_pipeline(u.shape[0], freq.shape[0], _p(u), _p(v), _p(w), _p(freq), _p(data), n,
                             _p(l), _p(m), _p(flux), _p(ac), ctypes.byref(params), _p(est), _p(sky),
                             n_threads)
    if rc != 0:
        raise MemoryError("oracle pipeline allocation failed")
    if want_sky:
        return est, sky[..., 0] + 1j * sky[..., 1]
    return est
