"""Pins of the learned-proposal oracle (oracle/mlp.py) on the CPU.

The analytic backward is checked against central finite differences of the loss,
the loss against its Gaussian definition, Adam against a hand-computed step, the
simulator against the likelihood's facet model, and the proposal rule against
its definition on hand-made cases."""
import math

import numpy as np

import oracle
from oracle import mlp


def _net(rng, n_in=12, n_h=7):
    W1 = rng.normal(0, 0.3, (n_in, n_h)); b1 = rng.normal(0, 0.1, n_h)
    W2 = rng.normal(0, 0.3, (n_h, n_h)); b2 = rng.normal(0, 0.1, n_h)
    W3 = rng.normal(0, 0.3, (n_h, 6)); b3 = rng.normal(0, 0.1, 6)
    return [W1, b1, W2, b2, W3, b3]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = _net(rng)
    x = rng.normal(0, 1, (5, 12))
    y = rng.normal(0, 0.5, (5, 3))
    o, cache = mlp.forward(x, *P)
    grads = mlp.backward(cache, P[2], P[4], mlp.nll_grad(o, y))
    h = 1e-6
    for pi, g in zip(range(6), grads):
        flat = P[pi].reshape(-1)
        for j in rng.choice(flat.size, min(6, flat.size), replace=False):
            old = flat[j]
            flat[j] = old + h
            lp = mlp.nll(mlp.forward(x, *P)[0], y)
            flat[j] = old - h
            lm = mlp.nll(mlp.forward(x, *P)[0], y)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g.reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (pi, j)


def test_nll_is_the_gaussian_negative_log_likelihood():
    # 1/2 (logvar + r^2/var) = -log N(y; mu, var) - 1/2 log(2 pi)
    o = np.array([[0.1, -0.2, 0.3, math.log(0.04), math.log(0.09), math.log(0.25)]])
    y = np.array([[0.15, -0.1, 0.0]])
    var = np.exp(o[0, 3:])
    ref = sum(-(-0.5 * math.log(2 * math.pi * v) - 0.5 * (yy - m) ** 2 / v) - 0.5 * math.log(2 * math.pi)
              for yy, m, v in zip(y[0], o[0, :3], var))
    assert abs(mlp.nll(o, y) - ref) < 1e-12


def test_adam_first_step_is_lr_times_sign():
    # with bias correction the first step moves every weight by lr * g / (|g| + eps)
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.001, 2.0])
    w1, m, v = mlp.adam(w, g, np.zeros(3), np.zeros(3), 1, 1e-3)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_simulated_facet_is_the_likelihood_model():
    # noise-free simulation equals S s M(k_c) / S from the oracle's Eq. 1 factor
    N, du = 8, 4000.0
    counts = np.zeros(N * N); counts[[3, 10, 27, 44]] = [2, 5, 1, 7]
    sbar = np.where(counts > 0, 0.97, 0.0)
    x = mlp.simulate(counts, sbar, du, 0.2, -0.3, 1.3, 0.0, np.zeros((2, N * N)), N=N)
    for c in (3, 10, 27, 44):
        iu, iv = c % N, c // N
        M = oracle.shape((iu - N // 2 + 0.5) * du, (iv - N // 2 + 0.5) * du, 1.3 * mlp.ARC, 0.2, -0.3)
        assert abs(x[c] - 0.97 * M) < 1e-14 and x[N * N + c] == 0.0
    assert np.count_nonzero(x) == 4
    # the Gaussian profile's facet model
    x = mlp.simulate(counts, sbar, du, 0.2, -0.3, 1.3, 0.0, np.zeros((2, N * N)), N=N, profile=1)
    for c in (3, 10, 27, 44):
        iu, iv = c % N, c // N
        M = oracle.shape((iu - N // 2 + 0.5) * du, (iv - N // 2 + 0.5) * du, 1.3 * mlp.ARC, 0.2, -0.3, 1)
        assert abs(x[c] - 0.97 * M) < 1e-14


def test_proposal_box_and_fallback_rules():
    p = oracle.default_params()
    ge, ga = oracle.grid_e(p), oracle.grid_alpha(p)
    # e1 = 0.17 -> node 12 (0.16), e2 = -0.79 -> node 0, alpha = 1.0" -> node 9 (1.018")
    origin, wide = mlp.propose(np.array([0.17, -0.79, math.log(1.0)]), np.log([1e-4, 1e-4, 1e-2]), ge, ga)
    assert origin == (9, 0, 7) and not wide
    # clamped at the top end of the grid
    origin, _ = mlp.propose(np.array([0.8, 0.0, math.log(3.5)]), np.zeros(3) - 9, ge, ga)
    assert origin == (14, 7, 15)
    # a predicted spread above three node spacings asks for the full grid
    _, wide = mlp.propose(np.array([0.0, 0.0, 0.0]), np.log([0.25 ** 2, 1e-4, 1e-4]), ge, ga)
    assert wide
    ne, na, box = 21, 20, (7, 7, 5)
    flat = lambda a, b, k: (a * ne + b) * na + k
    assert mlp.on_inner_boundary(flat(9, 3, 9), (9, 0, 7), box, ne, na)        # lower e1 face, inside the grid
    assert not mlp.on_inner_boundary(flat(12, 0, 9), (9, 0, 7), box, ne, na)   # e2 face is the grid's edge
    assert mlp.on_inner_boundary(flat(12, 6, 9), (9, 0, 7), box, ne, na)       # upper e2 face
    assert mlp.on_inner_boundary(flat(12, 3, 11), (9, 0, 7), box, ne, na)      # upper alpha face
    assert not mlp.on_inner_boundary(flat(12, 3, 9), (9, 0, 7), box, ne, na)


def test_simulated_noise_has_the_cell_variance():
    # the noise of a cell mean of n_c visibilities with per-component sigma, over S:
    # variance sigma^2 / (S^2 n_c) on Re and Im, zero mean (Sec. 2.4 weights w_c = n_c / sigma^2)
    N, du, sig_rel = 4, 4000.0, 0.5
    counts = np.array([1, 4, 9, 16] + [0] * (N * N - 4), dtype=float)
    sbar = np.where(counts > 0, 1.0, 0.0)
    rng = np.random.default_rng(3)
    draws = np.stack([mlp.simulate(counts, sbar, du, 0.0, 0.0, 1.0, sig_rel, rng.standard_normal((2, N * N)), N=N)
                      for _ in range(20000)])
    M = np.array([oracle.shape((c % N - N // 2 + 0.5) * du, (c // N - N // 2 + 0.5) * du, mlp.ARC, 0.0, 0.0)
                  for c in range(4)])
    for c in range(4):
        want = sig_rel ** 2 / counts[c]
        for part, mean in ((draws[:, c], M[c]), (draws[:, N * N + c], 0.0)):
            assert abs(part.mean() - mean) < 5 * math.sqrt(want / 20000)
            assert abs(part.var() / want - 1.0) < 0.05
    assert np.all(draws[:, 4:N * N] == 0.0)


def test_forward_of_a_hand_computed_network():
    # a 3-2-2-6 network with small exact weights, worked out by hand:
    #   x = (1, -2, 1/2):  z1 = (1 - 1 + 1 + 1/4, 1/2 + 2 + 1/2 - 1/2) = (5/4, 5/2), h1 = z1
    #                      z2 = (5/4 - 5/4 + 1/2, -5/4 + 5/8) = (1/2, -5/8), h2 = (1/2, 0)
    #                      o  = (1/2)(1..6) + b3
    #   x = (-1, 1, 1):    z1 = (-1 + 1/2 + 2 + 1/4, -1/2 - 1 + 1 - 1/2) = (7/4, -1), h1 = (7/4, 0)
    #                      z2 = (7/4 + 1/2, -7/4) = (9/4, -7/4), h2 = (9/4, 0)
    #                      o  = (9/4)(1..6) + b3
    # Dropping either ReLU, or transposing W1 or W2, changes every output.
    W1 = np.array([[1.0, 0.5], [0.5, -1.0], [2.0, 1.0]])
    b1 = np.array([0.25, -0.5])
    W2 = np.array([[1.0, -1.0], [-0.5, 0.25]])
    b2 = np.array([0.5, 0.0])
    W3 = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0], [7.0, 8.0, 9.0, 10.0, 11.0, 12.0]])
    b3 = np.array([0.0, 0.5, -1.0, 1.0, 0.0, -0.5])
    x = np.array([[1.0, -2.0, 0.5], [-1.0, 1.0, 1.0]])
    o, (_, z1, h1, z2, h2) = mlp.forward(x, W1, b1, W2, b2, W3, b3)
    assert np.array_equal(z1, [[1.25, 2.5], [1.75, -1.0]])
    assert np.array_equal(h1, [[1.25, 2.5], [1.75, 0.0]])
    assert np.array_equal(z2, [[0.5, -0.625], [2.25, -1.75]])
    assert np.array_equal(h2, [[0.5, 0.0], [2.25, 0.0]])
    assert np.array_equal(o, [[0.5, 1.5, 0.5, 3.0, 2.5, 2.5], [2.25, 5.0, 5.75, 10.0, 11.25, 13.0]])


def test_encode_of_a_hand_made_facet():
    # a 2 x 2 window: cells 0..3 with counts (2, 0, 3, 1); x = [sum Re / n / S, sum Im / n / S],
    # real parts first, the empty cell 0 (not 0/0)
    S = 0.5
    acc = np.array([[1.0, 0.0, -3.0, 0.25],     # sum Re x
                    [0.5, 0.0, 1.5, -0.5],      # sum Im x
                    [2.0, 0.0, 3.0, 1.0],       # count
                    [2.0, 0.0, 3.3, 0.9]])      # sum of the spectral factor (unused)
    x = mlp.encode(acc, S, N=2)
    assert np.array_equal(x, [1.0, 0.0, -2.0, 0.5, 0.5, 0.0, 1.0, -1.0])


def test_box_fallback_rule_on_hand_made_grids():
    # a 7 x 7 x 5 box at origin (7, 7, 7) of a 21 x 21 x 20 grid, flat prior weights; the
    # log-likelihood is a narrow bump at a chosen (e1, e2, alpha) node, -inf outside the box
    ne, na, box, origin = 21, 20, (7, 7, 5), (7, 7, 7)
    qp = np.ones(na)
    m = mlp.box_mask(origin, box, ne, na)
    i1, i2, k = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(na), indexing="ij")

    def grid(c1, c2, ck, w_e, w_a):
        lg = -0.5 * (((i1 - c1) / w_e) ** 2 + ((i2 - c2) / w_e) ** 2 + ((k - ck) / w_a) ** 2)
        return np.where(m, lg, -np.inf)
    fb = lambda lg: mlp.box_needs_full_grid(lg, qp, origin, box, 0.05, ne, na)
    # centred and narrow in every direction: the box stands for the grid
    assert not fb(grid(10, 10, 9, 0.7, 0.3))
    # wide in e: the inner e faces (3 nodes off the centre) carry L above 2.5 % of the maximum
    assert fb(grid(10, 10, 9, 2.0, 0.3))
    # narrow in e but wide in alpha: the alpha faces carry more than 1e-6 of L(e)
    assert fb(grid(10, 10, 9, 0.7, 1.5))
    # at the grid's own edge a box face is not an inner face: a bump on e1 node 0 with the box
    # at origin 0 does not fail on that face
    o0 = (0, 7, 7)
    m0 = mlp.box_mask(o0, box, ne, na)
    lg0 = np.where(m0, -0.5 * ((i1 / 0.7) ** 2 + ((i2 - 10) / 0.7) ** 2 + ((k - 9) / 0.3) ** 2), -np.inf)
    assert not mlp.box_needs_full_grid(lg0, qp, o0, box, 0.05, ne, na)
    # the same bump against an inner face (box at origin 1: e1 node 1 is its lower face)
    o1 = (1, 7, 7)
    m1 = mlp.box_mask(o1, box, ne, na)
    lg1 = np.where(m1, -0.5 * (((i1 - 1) / 0.7) ** 2 + ((i2 - 10) / 0.7) ** 2 + ((k - 9) / 0.3) ** 2), -np.inf)
    assert mlp.box_needs_full_grid(lg1, qp, o1, box, 0.05, ne, na)
