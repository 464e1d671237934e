"""FP64 oracle of the learned proposal (test infrastructure only).

The network proposes where on the (e1, e2, alpha) grid the likelihood of a facet
should be evaluated.  Everything here is the plain definition, in numpy float64:

  encode      x = [Re D_c / S, Im D_c / S] over the N x N window (empty cells 0)
  forward     h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), o = h2 W3 + b3,
              mu = o[0:3] (e1, e2, ln(alpha / arcsec)), logvar = o[3:6]
  nll         mean over the batch of 1/2 sum_j (lv_j + (y_j - mu_j)^2 exp(-lv_j)), with
              lv = logvar clamped to [-8, 8] (zero gradient outside): a predicted
              spread below e^-4 = 0.018 is finer than the grid needs, and the clamp
              keeps the f16 gradients of the GPU kernels finite
  backward    the chain rule of the three layers, written out
  adam        Kingma & Ba (2015), bias-corrected moments
  simulate    D_c / S = s_c M(k_c; e, alpha) + (sigma / S) z / sqrt(n_c) per component,
              the facet model of the likelihood (Sec. 2.4) at the cell centres of a
              given coverage (counts n_c, mean spectral factors s_c)
  propose     the 7 x 7 x 5 sub-box of the grid centred on the node nearest mu,
              clamped inside the grid, and the fallback rules: the full grid when the
              predicted spread is wide, when the box's MAP point lies on an inner face,
              or when a point near the estimate's threshold touches an inner face
              (box_needs_full_grid)
"""
from __future__ import annotations

import math

import numpy as np

ARC = math.pi / 648000.0
N_IN, N_H, N_OUT = 8192, 256, 6


def encode(acc: np.ndarray, flux: float, N: int = 64) -> np.ndarray:
    """Network input of one facet ([4, N*N] accumulators): cell means over S."""
    n = acc[2]
    x = np.zeros(2 * N * N)
    on = n > 0
    x[:N * N][on] = acc[0][on] / n[on] / flux
    x[N * N:][on] = acc[1][on] / n[on] / flux
    return x


def forward(x, W1, b1, W2, b2, W3, b3):
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3 + b3
    return o, (x, z1, h1, z2, h2)


LV_MIN, LV_MAX = -8.0, 8.0


def nll(o, y):
    mu, lv = o[:, :3], np.clip(o[:, 3:6], LV_MIN, LV_MAX)
    return float(np.mean(0.5 * np.sum(lv + (y - mu) ** 2 * np.exp(-lv), axis=1)))


def nll_grad(o, y):
    """d nll / d o."""
    B = o.shape[0]
    raw = o[:, 3:6]
    mu, lv = o[:, :3], np.clip(raw, LV_MIN, LV_MAX)
    r = y - mu
    g = np.zeros_like(o)
    g[:, :3] = -r * np.exp(-lv) / B
    inside = (raw > LV_MIN) & (raw < LV_MAX)
    g[:, 3:6] = np.where(inside, 0.5 * (1.0 - r * r * np.exp(-lv)) / B, 0.0)
    return g


def backward(cache, W2, W3, go):
    x, z1, h1, z2, h2 = cache
    dW3 = h2.T @ go
    db3 = go.sum(0)
    dh2 = (go @ W3.T) * (z2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (z1 > 0)
    dW1 = x.T @ dh1
    db1 = dh1.sum(0)
    return dW1, db1, dW2, db2, dW3, db3


def adam(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def shape_factor(cu, cv, du, e1, e2, alpha_rad, profile=0):
    """Eq. 1 brightness factor at cell centres (cu, cv in units of du); profile 1 is the
    Gaussian of the same FWHM, sigma = alpha sqrt(ln 2 / 2) (footnote to Sec. 2.2)."""
    A = np.array([[1 - e1, -e2], [-e2, 1 + e1]])
    T = np.linalg.inv(A).T
    ku, kv = cu * du, cv * du
    x = T[0, 0] * ku + T[0, 1] * kv
    y = T[1, 0] * ku + T[1, 1] * kv
    if profile == 1:
        return np.exp(-2.0 * math.pi ** 2 * alpha_rad ** 2 * math.log(2.0) / 2.0 * (x * x + y * y))
    return (1.0 + 4.0 * math.pi ** 2 * alpha_rad ** 2 * (x * x + y * y)) ** -1.5


def simulate(counts, sbar, du, e1, e2, alpha_arcsec, sigma_rel, z, N: int = 64, profile: int = 0) -> np.ndarray:
    """One simulated network input: counts, sbar over the N*N cells (iv*N + iu), z [2, N*N] normals."""
    iu = np.arange(N * N) % N
    iv = np.arange(N * N) // N
    cu = iu - N // 2 + 0.5
    cv = iv - N // 2 + 0.5
    M = shape_factor(cu, cv, du, e1, e2, alpha_arcsec * ARC, profile)
    x = np.zeros(2 * N * N)
    on = counts > 0
    sq = np.sqrt(np.where(on, counts, 1.0))
    x[:N * N][on] = (sbar * M + sigma_rel * z[0] / sq)[on]
    x[N * N:][on] = (sigma_rel * z[1] / sq)[on]
    return x


def propose(mu, logvar, grid_e, grid_alpha, box=(7, 7, 5), max_sigma_nodes=3.0):
    """Sub-box origin (i1, i2, k) and whether to fall back to the full grid."""
    ne, na = grid_e.size, grid_alpha.size
    de = grid_e[1] - grid_e[0]
    i1 = int(np.argmin(np.abs(grid_e - mu[0])))
    i2 = int(np.argmin(np.abs(grid_e - mu[1])))
    k = int(np.argmin(np.abs(grid_alpha - math.exp(mu[2]))))
    o1 = min(max(i1 - box[0] // 2, 0), ne - box[0])
    o2 = min(max(i2 - box[1] // 2, 0), ne - box[1])
    ok = min(max(k - box[2] // 2, 0), na - box[2])
    sig = np.exp(0.5 * np.asarray(logvar[:2]))
    wide = bool(np.any(sig > max_sigma_nodes * de))
    return (o1, o2, ok), wide


def on_inner_boundary(g, origin, box, ne, na):
    """True when flat grid index g lies on a face of the sub-box that is not a face of the grid."""
    i1, rem = divmod(g, ne * na)
    i2, k = divmod(rem, na)
    o1, o2, ok = origin
    faces = [(i1, o1, box[0], ne), (i2, o2, box[1], ne), (k, ok, box[2], na)]
    for idx, o, b, n in faces:
        if idx == o and o > 0:
            return True
        if idx == o + b - 1 and o + b < n:
            return True
    return False


def box_needs_full_grid(lg_box, qp, origin, box, thresh_frac, ne, na, alpha_tail=1e-6) -> bool:
    """Whether a sub-box fit cannot stand for the full grid (the second fallback rule).

    lg_box is the log-likelihood grid [ne, ne, na] with -inf outside the box, qp the
    trapezoid weight times the prior density of each scalelength node.  With
    t(e, k) = qp_k exp(lg(e, k) - max lg) and the alpha marginal L(e) = sum_k t(e, k), the
    points that can enter the thresholded estimate are those with L(e) >= thresh_frac
    max L / 2.  The box fails if one of them lies on a face of the box that is not a face
    of the grid (e directions), or if its alpha profile at such a face is above
    alpha_tail L(e) (alpha direction)."""
    fin = np.isfinite(lg_box)
    lmax = lg_box[fin].max()
    t = np.where(fin, qp[None, None, :] * np.exp(np.where(fin, lg_box, lmax) - lmax), 0.0)
    L = t.sum(axis=2)
    near = (L > 0.0) & (L >= 0.5 * thresh_frac * L.max())
    o1, o2, ok = origin
    face = np.zeros((ne, ne), dtype=bool)
    for o, b, axis in ((o1, box[0], 0), (o2, box[1], 1)):
        for idx in ([o] if o > 0 else []) + ([o + b - 1] if o + b < ne else []):
            if axis == 0:
                face[idx, :] = True
            else:
                face[:, idx] = True
    if np.any(near & face):
        return True
    for kf in ([ok] if ok > 0 else []) + ([ok + box[2] - 1] if ok + box[2] < na else []):
        if np.any(near & (t[:, :, kf] > alpha_tail * L)):
            return True
    return False


def box_mask(origin, box, ne, na) -> np.ndarray:
    m = np.zeros((ne, ne, na), dtype=bool)
    o1, o2, ok = origin
    m[o1:o1 + box[0], o2:o2 + box[1], ok:ok + box[2]] = True
    return m
