"""Pins of the oracle's chain order and update rule (Sec. 2.2, Sec. 2.4, Sec. 3.1).

``oracle.pipeline`` runs the chain in chunks of sources: every facet of a chunk is
extracted from the sky model as it stands when the chunk starts, the chunk's
sources are fitted, and only then are their shapes replaced in the sky model
(chunk = 1 is the paper's serial order; a chunk holding every source extracts all
facets from the initial circular model).  With update_mode 0 a fit flagged bad
leaves its source's shape in the sky model as it was (Sec. 2.4: bad fits are not
removed from the sky model; they keep the initial circular model).

Here the same chains are built by hand from the separately pinned building blocks
(``sky_model``, ``extract_facet``, ``fit_facet``), rebuilding the sky model from
scratch after every chunk instead of updating it incrementally, and compared with
``oracle.pipeline`` field by field.  The case (three overlapping sources, the
brightest flagged bad at this noise level) is chosen so that a wrong order or
rule changes the estimates by far more than the tolerance; the tests assert that
too.
"""
import math

import numpy as np
import pytest

import oracle
import synth

ARC = math.pi / 648000.0
SIGMA = 3e-4
FIELDS = (oracle.E1, oracle.E2, oracle.SIG1, oracle.SIG2, oracle.ALPHA, oracle.FLUX, oracle.FLAG,
          oracle.E1_SMOOTH, oracle.E2_SMOOTH)


@pytest.fixture(scope="module")
def case():
    wl = synth.tiny(seed=5, n_src=3, n_ant=16, n_time=12, n_chan=2, r_max_m=2000.0)
    obs, cat = synth.make_observation(wl), synth.make_catalogue(wl)
    # one bright source (its posterior collapses onto a node: a bad fit) and two faint
    # neighbours whose facets see its residual
    cat.flux_jy[:] = [2e-3, 1.2e-4, 1.0e-4]
    cat.l[:] = [0.0, 2.5e-4, -2e-4]
    cat.m[:] = [0.0, 1.5e-4, 2.2e-4]
    al = np.array([oracle.alpha_med(s) for s in cat.flux_jy]) * ARC
    d = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, cat.e1, cat.e2,
                         nu_ref=wl.nu_ref_hz)
    data = (np.stack([d.real, d.imag], -1) + synth.noise(obs.n_rows, obs.n_chan, SIGMA, 9)).astype(np.float32)
    return wl, obs, cat, al, data


def _params(wl, chunk, update_mode):
    return oracle.default_params(facet_n=32, nu_ref_hz=wl.nu_ref_hz, sigma_jy=SIGMA, chunk=chunk,
                                 update_mode=update_mode)


def _sky(obs, cat, al, e1, e2, wl):
    s = oracle.sky_model(obs.u, obs.v, obs.w, obs.freq_hz, cat.l, cat.m, cat.flux_jy, al, e1, e2,
                         nu_ref=wl.nu_ref_hz)
    return np.stack([s.real, s.imag], -1)


def hand_chain(case, chunk, update_mode, update_bad=False, extract_mid_chunk=False):
    """The chain written out: per chunk, extract and fit each source against the sky model
    of the shapes committed so far, then commit the chunk's shapes by the update rule and
    rebuild the sky model from scratch.  The two switches plant the mistakes the pins must
    catch: committing bad fits under update_mode 0, and extracting a chunk's later sources
    from a model already updated with its earlier ones."""
    wl, obs, cat, al, data = case
    p = _params(wl, chunk, update_mode)
    n = cat.n_src
    e1c, e2c = np.zeros(n), np.zeros(n)
    sky = _sky(obs, cat, al, e1c, e2c, wl)
    est = np.zeros((n, oracle.NEST))
    for first in range(0, n, chunk):
        for i in range(first, min(n, first + chunk)):
            du = oracle.facet_du(cat.flux_jy[i], 0.0, p)
            acc = oracle.extract_facet(obs.u, obs.v, obs.w, obs.freq_hz, data, sky, cat.l[i], cat.m[i],
                                       cat.flux_jy[i], al[i], e1c[i], e2c[i], du, p)
            est[i] = oracle.fit_facet(acc, du, cat.flux_jy[i], p).est
            if extract_mid_chunk:
                if update_mode == 1 or est[i, oracle.FLAG] == 0:
                    e1c[i], e2c[i] = est[i, oracle.E1], est[i, oracle.E2]
                sky = _sky(obs, cat, al, e1c, e2c, wl)
        for i in range(first, min(n, first + chunk)):
            if update_mode == 1 or update_bad or est[i, oracle.FLAG] == 0:
                e1c[i], e2c[i] = est[i, oracle.E1], est[i, oracle.E2]
        sky = _sky(obs, cat, al, e1c, e2c, wl)
    return est, sky, (e1c, e2c)


def _pipeline(case, chunk, update_mode):
    wl, obs, cat, al, data = case
    return oracle.pipeline(obs.u, obs.v, obs.w, obs.freq_hz, data, cat.l, cat.m, cat.flux_jy, None,
                           _params(wl, chunk, update_mode), want_sky=True)


def _max_field_diff(a, b):
    return max(float(np.max(np.abs(a[:, f] - b[:, f]))) for f in (oracle.E1, oracle.E2))


def test_case_has_one_bad_and_two_good_fits(case):
    est, _ = _pipeline(case, 1, 0)
    assert list(est[:, oracle.FLAG]) == [1.0, 0.0, 0.0]


@pytest.mark.parametrize("chunk,update_mode", [(1, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 1)])
def test_pipeline_equals_hand_built_chain(case, chunk, update_mode):
    est, sky = _pipeline(case, chunk, update_mode)
    ref, ref_sky, (e1c, e2c) = hand_chain(case, chunk, update_mode)
    for f in FIELDS:
        assert np.allclose(est[:, f], ref[:, f], rtol=1e-9, atol=1e-11), (f, est[:, f], ref[:, f])
    # the final sky model holds the committed shapes: measured ones, and the initial
    # circular shape for bad fits under update_mode 0
    s2 = np.stack([sky.real, sky.imag], -1)
    assert np.max(np.abs(s2 - ref_sky)) <= 1e-13 * np.max(np.abs(ref_sky))
    if update_mode == 0:
        assert e1c[0] == 0.0 and e2c[0] == 0.0


def test_serial_order_differs_from_one_chunk(case):
    # the serial order sees its predecessors' measured shapes; one chunk sees the circular model
    serial, _ = _pipeline(case, 1, 1)
    batched, _ = _pipeline(case, 3, 1)
    assert _max_field_diff(serial, batched) > 1e-2


@pytest.mark.parametrize("chunk", [1, 2])
def test_planted_update_of_bad_fits_is_caught(case, chunk):
    est, _ = _pipeline(case, chunk, 0)
    wrong, _, _ = hand_chain(case, chunk, 0, update_bad=True)
    assert _max_field_diff(est, wrong) > 1e-2


def test_planted_extraction_from_a_model_updated_mid_chunk_is_caught(case):
    est, _ = _pipeline(case, 2, 1)
    wrong, _, _ = hand_chain(case, 2, 1, extract_mid_chunk=True)
    assert _max_field_diff(est, wrong) > 1e-2
