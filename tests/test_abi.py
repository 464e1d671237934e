"""The C ABI library builds, loads and exports what include/rlf.h declares.

CPU only: these tests call nothing that reaches the GPU.  Argument errors are
found on the host before any CUDA call, so they are checked here too.
"""
import ctypes
import subprocess

import numpy as np
import pytest

import paper_2203_14071_gb300 as rlf
from paper_2203_14071_gb300 import build_ext


@pytest.fixture(scope="module")
def L():
    build_ext.build()
    return rlf.lib()


def test_every_declared_function_is_exported(L):
    names = rlf.header_functions()
    assert {"rlf_sky_model", "rlf_sky_update", "rlf_extract_facets", "rlf_fit_sources", "rlf_run",
            "rlf_workspace_size", "rlf_facets_size", "rlf_params_default", "rlf_read_status",
            "rlf_strerror"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", rlf.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_build_targets_sm103a_only():
    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_struct_sizes_match_header():
    # pointers and 64-bit fields must land where the C compiler puts them
    assert ctypes.sizeof(rlf.Uvw) == 8 + 4 + 4 + 4 * 8
    assert ctypes.sizeof(rlf.Sources) == 4 + 4 + 6 * 8
    assert ctypes.sizeof(rlf.Params) == 15 * 8 + 16 * 4
    assert ctypes.sizeof(rlf.FitOut) == 9 * 8


def test_params_default_is_the_papers(L):
    p = rlf.params_default()
    assert (p.add, p.esp, p.psf_nat, p.beta) == (-0.93, 0.33, 38.0, -0.7)
    assert (p.r_min_arcsec, p.r_max_arcsec, p.r_std) == (0.3, 3.5, 0.3136)
    assert (p.thresh_frac, p.var_sigma_min, p.var_det_min) == (0.05, 5e-3, 5e-5)
    assert (p.facet_n, p.n_e, p.n_alpha, p.precision) == (64, 21, 20, rlf.PREC_MIXED)


def test_sizes(L):
    p = rlf.params_default()
    assert rlf.facets_size(3, p) == 3 * 4 * 64 * 64 * 8
    assert rlf.facets_size(0, p) == 0
    sky = rlf.workspace_size(1000, 8, 200, p, rlf.WS_SKY)
    fit = rlf.workspace_size(1000, 8, 200, p, rlf.WS_FIT)
    run = rlf.workspace_size(1000, 8, 200, p, rlf.WS_RUN)
    assert 0 < sky < fit <= run
    # a smaller chunk needs less fit scratch in the whole-chain driver
    p1 = rlf.params_default(chunk=1)
    assert rlf.workspace_size(1000, 8, 200, p1, rlf.WS_RUN) < run
    bad = rlf.params_default(facet_n=63)
    assert rlf.workspace_size(1000, 8, 200, bad, rlf.WS_RUN) == 0
    # the position marginal keeps one B per offset and cell, padded to a multiple of four:
    # 28 values per cell for 25 offsets instead of one
    pos = rlf.params_default(n_pos=5)
    grow = rlf.workspace_size(1000, 8, 200, pos, rlf.WS_FIT) - fit
    assert grow == 27 * 200 * 64 * 64 * 8
    assert rlf.params_default().n_pos == 1 and rlf.params_default().pos_step_arcsec == 0.1
    assert rlf.workspace_size(1000, 8, 0, p, rlf.WS_RUN) == 0


def test_strerror(L):
    assert rlf.strerror(rlf.RLF_OK) == "ok"
    assert "workspace" in rlf.strerror(rlf.RLF_ENOSPACE)


def _fake_structs(n_rows=10, n_chan=2, n_src=3, freq=None):
    # pointers that are never dereferenced: the host checks reject the call first
    fake = 0x1000
    freq = np.array([1.0e9, 1.1e9][:n_chan] if freq is None else freq, dtype=np.float64)
    uvw = rlf.Uvw(n_rows=n_rows, n_chan=n_chan, n_baselines=0, u=fake, v=fake, w=fake,
                  freq_hz=freq.ctypes.data_as(ctypes.c_void_p).value)
    src = rlf.Sources(n_src=n_src, reserved=0, l=fake, m=fake, flux_jy=fake, alpha_arcsec=None, e1=fake, e2=fake)
    return uvw, src, freq


def test_host_argument_checks(L):
    p = rlf.params_default()
    uvw, src, keep = _fake_structs()
    ws = ctypes.c_void_p(0x2000)
    f = L.rlf_sky_model
    # null workspace, null output
    assert f(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), 0x3000, None, 10, None) == rlf.RLF_EINVAL
    assert f(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), None, ws, 10, None) == rlf.RLF_EINVAL
    # workspace too small
    assert f(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), 0x3000, ws, 16, None) == rlf.RLF_ENOSPACE
    # bad sizes
    uvw0, _, k0 = _fake_structs(n_rows=0)
    assert f(ctypes.byref(uvw0), ctypes.byref(src), ctypes.byref(p), 0x3000, ws, 1 << 40, None) == rlf.RLF_EINVAL
    # channels not increasing
    uvw1, _, k1 = _fake_structs(freq=[1.1e9, 1.0e9])
    assert f(ctypes.byref(uvw1), ctypes.byref(src), ctypes.byref(p), 0x3000, ws, 1 << 40, None) == rlf.RLF_EINVAL
    # too many channels
    many = np.linspace(1e9, 2e9, rlf.MAX_CHAN + 1)
    uvw2, _, k2 = _fake_structs(n_chan=many.size, freq=many)
    assert f(ctypes.byref(uvw2), ctypes.byref(src), ctypes.byref(p), 0x3000, ws, 1 << 40, None) == rlf.RLF_EUNSUPPORTED
    # parameters out of range
    for bad in (dict(facet_n=65), dict(facet_n=7), dict(n_e=1), dict(n_e=33), dict(sigma_jy=0.0),
                dict(precision=4), dict(r_min_arcsec=2.0, r_max_arcsec=1.0), dict(thresh_frac=0.0),
                dict(n_pos=2), dict(n_pos=7), dict(n_pos=-1), dict(n_pos=3, pos_step_arcsec=0.0),
                dict(n_pos=5, pos_step_arcsec=float("nan"))):
        pb = rlf.params_default(**bad)
        assert f(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(pb), 0x3000, ws, 1 << 40, None) == rlf.RLF_EINVAL
    # source range checks
    g = L.rlf_extract_facets
    fac = 0x4000
    nf = rlf.facets_size(2, p)
    assert g(ctypes.byref(uvw), 0x5000, 0x6000, ctypes.byref(src), 2, 2, ctypes.byref(p), fac, nf, ws, 1 << 40,
             None) == rlf.RLF_EINVAL
    assert g(ctypes.byref(uvw), 0x5000, 0x6000, ctypes.byref(src), 0, 2, ctypes.byref(p), fac, nf - 8, ws,
             1 << 40, None) == rlf.RLF_ENOSPACE
    out = rlf.FitOut()
    h = L.rlf_fit_sources
    assert h(fac, ctypes.byref(src), 0, 2, ctypes.byref(p), ctypes.byref(out), ws, 1 << 40, None) == rlf.RLF_EINVAL


def test_no_cpu_fallback_and_no_oracle_in_the_product():
    # without the built library every compute call raises; the package never loads the oracle
    code = ("import sys, paper_2203_14071_gb300 as r\n"
            "assert 'oracle' not in sys.modules\n"
            "r.LIB_PATH = '/nonexistent/librlf.so'\n"
            "r._lib = None\n"
            "try:\n"
            "    r.lib()\n"
            "except RuntimeError as e:\n"
            "    assert 'not built' in str(e)\n"
            "    print('raised')\n")
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "raised"


def test_static_sky_model_checks_arguments_as_the_workspace_entry_point(L):
    # an out-of-range profile (or estimator) is rejected by both sky-model entry points before
    # anything is enqueued
    fake = 0x1000
    freq = np.array([1.0e9], dtype=np.float64)
    uvw = rlf.Uvw(n_rows=4, n_chan=1, n_baselines=0, u=fake, v=fake, w=fake,
                  freq_hz=freq.ctypes.data_as(ctypes.c_void_p).value)
    src = rlf.Sources(n_src=3, reserved=0, l=fake, m=fake, flux_jy=fake, alpha_arcsec=None, e1=fake, e2=fake)
    for field, bad in (("profile", 7), ("estimator", 9), ("n_pos", 4), ("tune_sky_blocks", -1)):
        p = rlf.params_default()
        setattr(p, field, bad)
        assert L.rlf_sky_model_static(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), fake, None) == \
            rlf.RLF_EINVAL, field
        assert L.rlf_sky_model(ctypes.byref(uvw), ctypes.byref(src), ctypes.byref(p), fake, fake, 1 << 40,
                               None) == rlf.RLF_EINVAL, field
