"""GB300 (sm_103a) RadioLensfit hot path: Python binding of librlf.so.

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels of ``csrc/`` behind the C ABI declared in ``include/rlf.h``; PyTorch
supplies device memory and streams.  Importing this package does not need a
GPU, but calling a compute entry point does, and there is no CPU fallback: if
``_build/librlf.so`` is missing the calls raise.

Names follow the C ABI without the ``rlf_`` prefix:
``sky_model``, ``sky_update``, ``extract_facets``, ``fit_sources``, ``run``,
``workspace_size``, ``facets_size``, ``params_default``, ``read_status``.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librlf.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
HEADER = os.path.join(INCLUDE, "rlf.h")

RLF_OK, RLF_EINVAL, RLF_ECUDA, RLF_ENOSPACE, RLF_ETIMEOUT, RLF_ENUMERIC, RLF_EUNSUPPORTED = range(7)
PREC_FP64, PREC_MIXED, PREC_MIXED_SPLIT = 0, 1, 2
PROFILE_EXPONENTIAL, PROFILE_GAUSSIAN = 0, 1
ESTIMATOR_GRID, ESTIMATOR_ADAPTIVE = 0, 1
FLAG_LEVELS_SHIFT = 8
FLAG_BAD, FLAG_INVALID, FLAG_EMPTY, FLAG_REFIT = 1, 2, 4, 8
DEV_INVALID_SOURCE, DEV_NONFINITE, DEV_TIMEOUT = 1, 2, 4
WS_SKY, WS_EXTRACT, WS_FIT, WS_RUN = range(4)
MAX_CHAN, MAX_FACET_N, STATIC_MAX_SRC, MAX_POS = 128, 64, 4096, 5

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


class RlfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class Uvw(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_chan", ctypes.c_int32), ("n_baselines", ctypes.c_int32),
                ("u", _vp), ("v", _vp), ("w", _vp), ("freq_hz", _vp)]


class Sources(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int32), ("reserved", ctypes.c_int32), ("l", _vp), ("m", _vp),
                ("flux_jy", _vp), ("alpha_arcsec", _vp), ("e1", _vp), ("e2", _vp)]


class Params(ctypes.Structure):
    _fields_ = [("add", ctypes.c_double), ("esp", ctypes.c_double), ("psf_nat", ctypes.c_double),
                ("beta", ctypes.c_double), ("nu_ref_hz", ctypes.c_double), ("sigma_jy", ctypes.c_double),
                ("e_max", ctypes.c_double), ("r_min_arcsec", ctypes.c_double),
                ("r_max_arcsec", ctypes.c_double), ("r_std", ctypes.c_double),
                ("thresh_frac", ctypes.c_double), ("var_sigma_min", ctypes.c_double),
                ("var_det_min", ctypes.c_double), ("facet_n", ctypes.c_int32), ("n_e", ctypes.c_int32),
                ("n_alpha", ctypes.c_int32), ("flux_prior", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("update_mode", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tune_fit_ag", ctypes.c_int32), ("tune_fit_blocks", ctypes.c_int32),
                ("tune_extract_waves", ctypes.c_int32), ("tune_sky_blocks", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("e_res", ctypes.c_double), ("np_max", ctypes.c_int32),
                ("estimator", ctypes.c_int32), ("refit_bad", ctypes.c_int32), ("n_pos", ctypes.c_int32),
                ("pos_step_arcsec", ctypes.c_double)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_per_s", ctypes.c_double), ("fp32x2_fma_per_s", ctypes.c_double),
                ("fp64_fma_per_s", ctypes.c_double),
                ("mufu_rsqrt_per_s", ctypes.c_double), ("mufu_sin_per_s", ctypes.c_double),
                ("sm_count", ctypes.c_int)]


class FitOut(ctypes.Structure):
    _fields_ = [("e1", _vp), ("e2", _vp), ("sig1", _vp), ("sig2", _vp), ("alpha_arcsec", _vp),
                ("flux_jy", _vp), ("e1_smooth", _vp), ("e2_smooth", _vp), ("flag", _vp)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load librlf.so (built by build_ext.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run paper_2203_14071_gb300.build_ext.build())")
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            P = ctypes.POINTER
            L.rlf_params_default.argtypes = [P(Params)]
            L.rlf_params_default.restype = None
            L.rlf_workspace_size.argtypes = [i64, i32, i32, P(Params), i32]
            L.rlf_workspace_size.restype = sz
            L.rlf_facets_size.argtypes = [i32, P(Params)]
            L.rlf_facets_size.restype = sz
            L.rlf_strerror.argtypes = [ctypes.c_int]
            L.rlf_strerror.restype = ctypes.c_char_p
            L.rlf_sky_model.argtypes = [P(Uvw), P(Sources), P(Params), _vp, _vp, sz, _vp]
            L.rlf_sky_update.argtypes = [P(Uvw), P(Sources), i32, i32, _vp, _vp, _vp, P(Params), _vp, _vp,
                                         sz, _vp]
            L.rlf_extract_facets.argtypes = [P(Uvw), _vp, _vp, P(Sources), i32, i32, P(Params), _vp, sz,
                                             _vp, sz, _vp]
            L.rlf_fit_sources.argtypes = [_vp, P(Sources), i32, i32, P(Params), P(FitOut), _vp, sz, _vp]
            L.rlf_run.argtypes = [P(Uvw), _vp, P(Sources), P(Params), P(FitOut), _vp, _vp, sz, _vp]
            L.rlf_read_status.argtypes = [_vp, P(ctypes.c_int32), _vp]
            L.rlf_graph_create.argtypes = [P(Uvw), _vp, P(Sources), P(Params), P(FitOut), _vp, _vp, sz, _vp,
                                           P(_vp)]
            L.rlf_graph_create.restype = ctypes.c_int
            L.rlf_graph_launch.argtypes = [_vp, _vp]
            L.rlf_graph_launch.restype = ctypes.c_int
            L.rlf_graph_destroy.argtypes = [_vp]
            L.rlf_graph_destroy.restype = None
            L.rlf_autotune.argtypes = [P(Uvw), _vp, P(Sources), P(Params), P(FitOut), _vp, _vp, sz, _vp,
                                       P(ctypes.c_float)]
            L.rlf_autotune.restype = ctypes.c_int
            L.rlf_mlp_weights_size.argtypes = []
            L.rlf_mlp_weights_size.restype = sz
            L.rlf_mlp_n_params.argtypes = []
            L.rlf_mlp_n_params.restype = i64
            L.rlf_mlp_workspace_size.argtypes = [i32]
            L.rlf_mlp_workspace_size.restype = sz
            L.rlf_mlp_init.argtypes = [_vp, _vp, _vp]
            L.rlf_mlp_simulate.argtypes = [_vp, _vp, i32, _vp, _vp, _vp, _vp, _vp, i32, P(Params), _vp, _vp, _vp]
            L.rlf_mlp_train_step.argtypes = [_vp, _vp, _vp, i32, ctypes.c_float, i32, _vp, _vp, sz, _vp]
            L.rlf_mlp_forward.argtypes = [_vp, _vp, i32, _vp, _vp, sz, _vp]
            L.rlf_mlp_encode.argtypes = [_vp, P(Sources), i32, i32, P(Params), _vp, _vp, sz, _vp]
            L.rlf_mlp_propose.argtypes = [_vp, P(Sources), i32, i32, P(Params), _vp, _vp, _vp, _vp, sz, _vp]
            L.rlf_fit_sources_mlp.argtypes = [_vp, P(Sources), i32, i32, P(Params), _vp, P(FitOut), _vp, _vp, sz,
                                              _vp]
            for f in ("rlf_mlp_init", "rlf_mlp_simulate", "rlf_mlp_train_step", "rlf_mlp_forward",
                      "rlf_mlp_encode", "rlf_mlp_propose", "rlf_fit_sources_mlp"):
                getattr(L, f).restype = ctypes.c_int
            L.rlf_sky_model_static.argtypes = [P(Uvw), P(Sources), P(Params), _vp, _vp]
            L.rlf_sky_model_static.restype = ctypes.c_int
            L.rlf_peaks_measure.argtypes = [_vp, sz, _vp, P(Peaks)]
            L.rlf_peaks_measure.restype = ctypes.c_int
            for f in ("rlf_sky_model", "rlf_sky_update", "rlf_extract_facets", "rlf_fit_sources", "rlf_run",
                      "rlf_read_status"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def header_functions():
    """Names of the functions the headers in include/ declare."""
    names = set()
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(rlf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def strerror(code: int) -> str:
    return lib().rlf_strerror(code).decode()


def _check(code: int, where: str):
    if code != RLF_OK:
        raise RlfError(code, where)


def params_default(**overrides) -> Params:
    p = Params()
    lib().rlf_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def workspace_size(n_rows: int, n_chan: int, n_src: int, params: Params, which: int = WS_RUN) -> int:
    return int(lib().rlf_workspace_size(n_rows, n_chan, n_src, ctypes.byref(params), which))


def facets_size(count: int, params: Params) -> int:
    return int(lib().rlf_facets_size(count, ctypes.byref(params)))


# ---- marshalling helpers (torch tensors -> raw pointers) -------------------------------

def _ptr(t) -> int | None:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Observation:
    """Device baselines plus the host channel table, as the C ABI wants them."""

    def __init__(self, u, v, w, freq_hz, n_baselines: int = 0):
        self.u, self.v, self.w = u, v, w
        self.freq_hz = np.ascontiguousarray(freq_hz, dtype=np.float64)
        self.struct = Uvw(n_rows=int(u.shape[0]), n_chan=int(self.freq_hz.shape[0]), n_baselines=int(n_baselines),
                          u=_ptr(u), v=_ptr(v), w=_ptr(w),
                          freq_hz=self.freq_hz.ctypes.data_as(ctypes.c_void_p).value)

    @property
    def n_rows(self):
        return self.struct.n_rows

    @property
    def n_chan(self):
        return self.struct.n_chan

    @property
    def n_baselines(self):
        return self.struct.n_baselines


class Catalogue:
    """Device catalogue arrays (float64), sorted by decreasing flux."""

    def __init__(self, l, m, flux_jy, e1, e2, alpha_arcsec=None):
        self.l, self.m, self.flux_jy, self.e1, self.e2, self.alpha_arcsec = l, m, flux_jy, e1, e2, alpha_arcsec
        self.struct = Sources(n_src=int(l.shape[0]), reserved=0, l=_ptr(l), m=_ptr(m), flux_jy=_ptr(flux_jy),
                              alpha_arcsec=_ptr(alpha_arcsec), e1=_ptr(e1), e2=_ptr(e2))

    @property
    def n_src(self):
        return self.struct.n_src


class Results:
    """Device result arrays for `count` sources."""

    FIELDS = ("e1", "e2", "sig1", "sig2", "alpha_arcsec", "flux_jy", "e1_smooth", "e2_smooth")

    def __init__(self, count: int, device):
        import torch
        for f in self.FIELDS:
            setattr(self, f, torch.zeros(count, dtype=torch.float64, device=device))
        self.flag = torch.zeros(count, dtype=torch.int32, device=device)
        self.struct = FitOut(**{f: _ptr(getattr(self, f)) for f in self.FIELDS}, flag=_ptr(self.flag))

    def numpy(self):
        d = {f: getattr(self, f).cpu().numpy() for f in self.FIELDS}
        d["flag"] = self.flag.cpu().numpy()
        return d


def sky_model(obs: Observation, cat: Catalogue, params: Params, vis_sky, workspace, stream=None):
    _check(lib().rlf_sky_model(ctypes.byref(obs.struct), ctypes.byref(cat.struct), ctypes.byref(params),
                               _ptr(vis_sky), _ptr(workspace), workspace.numel() * workspace.element_size(),
                               _stream(stream)), "rlf_sky_model")


def sky_update(obs: Observation, cat: Catalogue, first: int, count: int, e1_new, e2_new, flag,
               params: Params, vis_sky, workspace, stream=None):
    _check(lib().rlf_sky_update(ctypes.byref(obs.struct), ctypes.byref(cat.struct), first, count,
                                _ptr(e1_new), _ptr(e2_new), _ptr(flag), ctypes.byref(params), _ptr(vis_sky),
                                _ptr(workspace), workspace.numel() * workspace.element_size(),
                                _stream(stream)), "rlf_sky_update")


def extract_facets(obs: Observation, vis_data, vis_sky, cat: Catalogue, first: int, count: int,
                   params: Params, facets, workspace, stream=None):
    _check(lib().rlf_extract_facets(ctypes.byref(obs.struct), _ptr(vis_data), _ptr(vis_sky),
                                    ctypes.byref(cat.struct), first, count, ctypes.byref(params), _ptr(facets),
                                    facets.numel() * facets.element_size(), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _stream(stream)),
           "rlf_extract_facets")


def fit_sources(facets, cat: Catalogue, first: int, count: int, params: Params, out: Results, workspace,
                stream=None):
    _check(lib().rlf_fit_sources(_ptr(facets), ctypes.byref(cat.struct), first, count, ctypes.byref(params),
                                 ctypes.byref(out.struct), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), _stream(stream)),
           "rlf_fit_sources")


def run(obs: Observation, vis_data, cat: Catalogue, params: Params, out: Results, vis_sky, workspace,
        stream=None):
    _check(lib().rlf_run(ctypes.byref(obs.struct), _ptr(vis_data), ctypes.byref(cat.struct),
                         ctypes.byref(params), ctypes.byref(out.struct), _ptr(vis_sky), _ptr(workspace),
                         workspace.numel() * workspace.element_size(), _stream(stream)), "rlf_run")


def sky_model_static(obs: Observation, cat: Catalogue, params: Params, vis_sky, stream=None):
    """rlf_sky_model_static: the sky model with no workspace (for callers that cannot allocate)."""
    _check(lib().rlf_sky_model_static(ctypes.byref(obs.struct), ctypes.byref(cat.struct), ctypes.byref(params),
                                      _ptr(vis_sky), _stream(stream)), "rlf_sky_model_static")


class Graph:
    """rlf_graph_create / rlf_graph_launch / rlf_graph_destroy: the whole chain as a CUDA graph.

    The graph records the buffers it was created with; keep them alive and update
    their contents in place between launches."""

    def __init__(self, obs: Observation, vis_data, cat: Catalogue, params: Params, out: Results, vis_sky,
                 workspace, stream):
        self._keep = (obs, vis_data, cat, params, out, vis_sky, workspace)
        self.handle = ctypes.c_void_p()
        _check(lib().rlf_graph_create(ctypes.byref(obs.struct), _ptr(vis_data), ctypes.byref(cat.struct),
                                      ctypes.byref(params), ctypes.byref(out.struct), _ptr(vis_sky),
                                      _ptr(workspace), workspace.numel() * workspace.element_size(),
                                      _stream(stream), ctypes.byref(self.handle)), "rlf_graph_create")

    def launch(self, stream=None):
        _check(lib().rlf_graph_launch(self.handle, _stream(stream)), "rlf_graph_launch")

    def close(self):
        if self.handle:
            lib().rlf_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNE_FIELDS = ("tune_sky_blocks", "tune_extract_waves", "tune_fit_ag", "tune_fit_blocks")


def tuning_key(obs: Observation, n_src: int, params: Params) -> str:
    """Cache key: workload shape, grid, precision, chunk, profile, position offsets, the
    GPU's SM count and the tuner's candidate sets (TUNER_VERSION)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return "v%d_rows%d_chan%d_bl%d_src%d_N%d_e%d_a%d_prec%d_chunk%d_prof%d_pos%d_sm%d" % (
        TUNER_VERSION, obs.n_rows, obs.n_chan, obs.struct.n_baselines, n_src, params.facet_n, params.n_e,
        params.n_alpha, params.precision, params.chunk, params.profile, params.n_pos, sms)


# bumped whenever rlf_autotune's candidate sets change, so that cached choices are redone
TUNER_VERSION = 3


def autotune(obs: Observation, vis_data, cat: Catalogue, params: Params, out: Results, vis_sky, workspace,
             cache_path: str | None = None, stream=None) -> dict:
    """rlf_autotune with a JSON cache keyed by tuning_key(); fills params.tune_* in place."""
    import json
    key = tuning_key(obs, cat.n_src, params)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        for f in TUNE_FIELDS:
            setattr(params, f, int(cache[key][f]))
        return dict(cache[key], cached=True)
    ms = (ctypes.c_float * 3)()
    _check(lib().rlf_autotune(ctypes.byref(obs.struct), _ptr(vis_data), ctypes.byref(cat.struct),
                              ctypes.byref(params), ctypes.byref(out.struct), _ptr(vis_sky), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream), ms), "rlf_autotune")
    entry = {f: int(getattr(params, f)) for f in TUNE_FIELDS}
    entry["phase_ms"] = [float(x) for x in ms]
    if cache_path:
        cache[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(entry, cached=False)


def read_status(workspace, stream=None) -> tuple[int, int]:
    v = ctypes.c_int32(0)
    code = lib().rlf_read_status(_ptr(workspace), ctypes.byref(v), _stream(stream))
    return code, int(v.value)


def alloc_workspace(n_rows: int, n_chan: int, n_src: int, params: Params, which: int = WS_RUN, device="cuda"):
    import torch
    n = workspace_size(n_rows, n_chan, n_src, params, which)
    if n == 0:
        raise RlfError(RLF_EINVAL, "rlf_workspace_size")
    return torch.empty(n, dtype=torch.uint8, device=device)


def peaks_measure(stream=None) -> dict:
    """Measured FP32/FP64 FMA and MUFU rsqrt/sin throughputs (per second) on the current GPU."""
    import torch
    out = Peaks()
    scratch = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    code = lib().rlf_peaks_measure(_ptr(scratch), scratch.numel(), _stream(stream), ctypes.byref(out))
    if code != 0:
        raise RuntimeError(f"rlf_peaks_measure failed ({code})")
    return {f: getattr(out, f) for f, _ in Peaks._fields_}


# ---- learned proposal ------------------------------------------------------------------

MLP_IN, MLP_HIDDEN, MLP_OUT = 8192, 256, 8


def mlp_offsets() -> dict:
    """Parameter offsets inside the weights blob (see include/rlf.h)."""
    o = {"W1": 0}
    o["b1"] = o["W1"] + MLP_IN * MLP_HIDDEN
    o["W2"] = o["b1"] + MLP_HIDDEN
    o["b2"] = o["W2"] + MLP_HIDDEN * MLP_HIDDEN
    o["W3"] = o["b2"] + MLP_HIDDEN
    o["b3"] = o["W3"] + MLP_HIDDEN * MLP_OUT
    o["P"] = o["b3"] + MLP_OUT
    return o


class Mlp:
    """A weights blob on the device with views of its sections."""

    def __init__(self, device="cuda"):
        import torch
        n = int(lib().rlf_mlp_weights_size())
        self.blob = torch.zeros(n, dtype=torch.uint8, device=device)
        self.P = int(lib().rlf_mlp_n_params())
        o = mlp_offsets()
        assert o["P"] == self.P
        f32 = self.blob[: 4 * self.P * 4].view(torch.float32)
        self.w, self.m, self.v, self.g = (f32[i * self.P:(i + 1) * self.P] for i in range(4))
        self.h = self.blob[4 * self.P * 4:].view(torch.float16)
        self.off = o

    def section(self, vec, name):
        o = self.off
        shapes = {"W1": (MLP_IN, MLP_HIDDEN), "b1": (MLP_HIDDEN,), "W2": (MLP_HIDDEN, MLP_HIDDEN),
                  "b2": (MLP_HIDDEN,), "W3": (MLP_HIDDEN, MLP_OUT), "b3": (MLP_OUT,)}
        n = int(np.prod(shapes[name]))
        return vec[o[name]:o[name] + n].view(*shapes[name])

    def half(self, name):
        sizes = {"W1": MLP_IN * MLP_HIDDEN, "W2": MLP_HIDDEN * MLP_HIDDEN, "W3": MLP_HIDDEN * MLP_OUT}
        start = {"W1": 0, "W2": sizes["W1"], "W3": sizes["W1"] + sizes["W2"]}[name]
        shape = {"W1": (MLP_IN, MLP_HIDDEN), "W2": (MLP_HIDDEN, MLP_HIDDEN), "W3": (MLP_HIDDEN, MLP_OUT)}[name]
        return self.h[start:start + sizes[name]].view(*shape)

    def init(self, normals, stream=None):
        _check(lib().rlf_mlp_init(_ptr(self.blob), _ptr(normals), _stream(stream)), "rlf_mlp_init")


def mlp_workspace(max_batch: int, device="cuda"):
    import torch
    return torch.empty(int(lib().rlf_mlp_workspace_size(max_batch)), dtype=torch.uint8, device=device)


def mlp_simulate(templates, template_flux, tidx, e1, e2, alpha_arcsec, normals, params: Params, x16, y,
                 stream=None):
    _check(lib().rlf_mlp_simulate(_ptr(templates), _ptr(template_flux), int(template_flux.numel()), _ptr(tidx),
                                  _ptr(e1), _ptr(e2), _ptr(alpha_arcsec), _ptr(normals), int(tidx.numel()),
                                  ctypes.byref(params), _ptr(x16), _ptr(y), _stream(stream)), "rlf_mlp_simulate")


def mlp_train_step(mlp: Mlp, x16, y, lr: float, step: int, loss, workspace, stream=None):
    _check(lib().rlf_mlp_train_step(_ptr(mlp.blob), _ptr(x16), _ptr(y), int(y.shape[0]), float(lr), int(step),
                                    _ptr(loss), _ptr(workspace), workspace.numel(), _stream(stream)),
           "rlf_mlp_train_step")


def mlp_forward(mlp: Mlp, x16, out, workspace, stream=None):
    _check(lib().rlf_mlp_forward(_ptr(mlp.blob), _ptr(x16), int(out.shape[0]), _ptr(out), _ptr(workspace),
                                 workspace.numel(), _stream(stream)), "rlf_mlp_forward")


def mlp_encode(facets, cat: Catalogue, first: int, count: int, params: Params, x16, workspace, stream=None):
    _check(lib().rlf_mlp_encode(_ptr(facets), ctypes.byref(cat.struct), first, count, ctypes.byref(params),
                                _ptr(x16), _ptr(workspace), workspace.numel(), _stream(stream)), "rlf_mlp_encode")


def mlp_propose(facets, cat: Catalogue, first: int, count: int, params: Params, mlp: Mlp, origin, workspace,
                wide=None, stream=None):
    """rlf_mlp_propose: the network's 7 x 7 x 5 sub-box origin per facet (origin: int32 [count, 3])
    and, optionally, its too-wide flag (wide: int32 [count])."""
    _check(lib().rlf_mlp_propose(_ptr(facets), ctypes.byref(cat.struct), first, count, ctypes.byref(params),
                                 _ptr(mlp.blob), _ptr(origin), _ptr(wide), _ptr(workspace), workspace.numel(),
                                 _stream(stream)), "rlf_mlp_propose")


def fit_sources_mlp(facets, cat: Catalogue, first: int, count: int, params: Params, mlp: Mlp, out: Results,
                    workspace, n_fallback=None, stream=None):
    _check(lib().rlf_fit_sources_mlp(_ptr(facets), ctypes.byref(cat.struct), first, count, ctypes.byref(params),
                                     _ptr(mlp.blob), ctypes.byref(out.struct), _ptr(n_fallback), _ptr(workspace),
                                     workspace.numel(), _stream(stream)), "rlf_fit_sources_mlp")
