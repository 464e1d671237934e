"""rlf_sky_model_static: the sky model for callers that cannot allocate device memory.

Such callers (code running where cudaMalloc is not allowed, a real-time loop that
must not allocate after start-up, a plugin handed only input and output buffers)
cannot supply the workspace rlf_sky_model needs; this entry point keeps its
per-source table in a fixed device array inside the library instead.  The test
calls it twice in a row through the C ABI, with different catalogues, and checks
each result against rlf_sky_model's and against the FP64 oracle with the
per-visibility bound of the parity tests (1e-5 of the summed moduli of the terms,
plus the complex64 rounding of the output).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests import cases

pytestmark = pytest.mark.gpu


def test_static_sky_model_matches_workspace_entry_point():
    import torch

    import paper_2203_14071_gb300 as rlf
    from paper_2203_14071_gb300 import build_ext
    build_ext.build()
    L = rlf.lib()
    wl = synth.tiny(seed=77, n_ant=24, n_time=15, n_chan=8, n_src=300, r_max_m=20000.0)
    c = cases.build(wl, with_data=False)
    stream = torch.cuda.current_stream()
    for call, shrink in enumerate((1.0, 0.5)):
        e1, e2 = c.cat.e1 * shrink, c.cat.e2 * shrink
        obs, cat = cases.to_device(c, e1, e2)
        p = rlf.params_default(nu_ref_hz=wl.nu_ref_hz, precision=rlf.PREC_MIXED_SPLIT)
        n = obs.n_rows * obs.n_chan * 2
        ws = rlf.alloc_workspace(obs.n_rows, obs.n_chan, cat.n_src, p, rlf.WS_SKY)
        ref = torch.empty(n, dtype=torch.float32, device="cuda")
        rlf.sky_model(obs, cat, p, ref, ws, stream)
        got = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        code = L.rlf_sky_model_static(ctypes.byref(obs.struct), ctypes.byref(cat.struct), ctypes.byref(p),
                                      got.data_ptr(), int(stream.cuda_stream))
        assert code == rlf.RLF_OK, (call, rlf.strerror(code))
        torch.cuda.synchronize()
        g = got.view(-1, 2).cpu().numpy().astype(np.float64)
        r = ref.view(-1, 2).cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(g)), call
        orc, ab = oracle.sky_model(c.obs.u, c.obs.v, c.obs.w, c.obs.freq_hz, c.cat.l, c.cat.m, c.cat.flux_jy,
                                   c.alpha_med_rad(), e1, e2, nu_ref=wl.nu_ref_hz, with_abs=True)
        orc, ab = orc.reshape(-1), ab.reshape(-1)
        gz, rz = g[:, 0] + 1j * g[:, 1], r[:, 0] + 1j * r[:, 1]
        rnd = 2.0 ** -24 * np.sqrt(2.0) * np.abs(orc)
        # against the workspace entry point: both within the parity bound of the oracle
        assert np.all(np.abs(gz - rz) <= 2e-5 * ab + 2 * rnd + 1e-30), (call, float(np.max(np.abs(gz - rz) / ab)))
        # against the FP64 oracle, as the parity tests bound rlf_sky_model
        assert np.all(np.abs(gz - orc) <= 1e-5 * ab + rnd + 1e-30), (call, float(np.max(np.abs(gz - orc) / ab)))


def test_static_sky_model_rejects_too_many_sources():
    import paper_2203_14071_gb300 as rlf
    L = rlf.lib()
    fake = 0x1000
    freq = np.array([1.0e9], dtype=np.float64)
    uvw = rlf.Uvw(n_rows=4, n_chan=1, n_baselines=0, u=fake, v=fake, w=fake,
                  freq_hz=freq.ctypes.data_as(ctypes.c_void_p).value)
    src = rlf.Sources(n_src=rlf.STATIC_MAX_SRC + 1, reserved=0, l=fake, m=fake, flux_jy=fake, alpha_arcsec=None,
                      e1=fake, e2=fake)
    p = rlf.params_default()
    assert L.rlf_sky_model_static(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), fake, None) == \
        rlf.RLF_ENOSPACE
