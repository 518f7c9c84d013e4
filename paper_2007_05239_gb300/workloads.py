"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws point clouds; it holds none of the method's arithmetic
(no kernel, no Fourier coefficient, no window).  Both the CUDA path's tests and
the CPU oracle take their inputs from here, so the two sides see the same
points.  The paper's datasets (the beach images, Pavia centre, the small
multilayer sets) are not available; these generators stand in for them with
the same sizes, dimensions and value structure (Sec. 7 feature grouping;
Sec. 8.2 image workload, Sec. 8.4 hyperspectral workload).

All generators use numpy's PCG64 with an explicit seed and return float64
arrays of shape (n, d_t), one per layer (the block model: n x n weight
matrices, one per layer).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_cube",
    "uniform_ball",
    "image_voronoi_layers",
    "image_discs_layers",
    "gmm_band_layers",
    "block_model_layers",
    "cloud_for_mlp",
    "WORKLOADS",
]


def uniform_cube(n: int = 2000, d: int = 3, half: float = 0.25, seed: int = 1) -> np.ndarray:
    """n points i.i.d. uniform in [-half, half]^d."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-half, half, size=(n, d))


def uniform_ball(n: int = 2000, d: int = 3, radius: float = 1.0, seed: int = 1) -> np.ndarray:
    """n points i.i.d. uniform in the d-ball of the given radius (a Gaussian
    direction scaled by radius * U^(1/d))."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    X /= np.linalg.norm(X, axis=1)[:, None]
    return radius * X * rng.random(n)[:, None] ** (1.0 / d)


def _smooth_texture(h: int, w: int, rng: np.random.Generator, terms: int = 6) -> np.ndarray:
    """A seeded smooth random field on an h x w pixel grid with values in [0, 1].

    Sum of a few low-frequency plane waves with random directions and phases,
    then affinely mapped onto [0, 1].  It carries no class information.
    """
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64) / max(h, w),
                         np.arange(w, dtype=np.float64) / max(h, w), indexing="ij")
    f = np.zeros((h, w))
    for _ in range(terms):
        kx, ky = rng.uniform(-6.0, 6.0, size=2)
        ph = rng.uniform(0.0, 2 * np.pi)
        f += rng.uniform(0.5, 1.0) * np.cos(2 * np.pi * (kx * xx + ky * yy) + ph)
    f -= f.min()
    f /= max(f.max(), 1e-300)
    return f


def _box3(img: np.ndarray) -> np.ndarray:
    """3x3 box filter of an (h, w, c) image with edge replication."""
    p = np.pad(img, ((1, 1), (1, 1), (0, 0)), mode="edge")
    out = np.zeros_like(img)
    h, w = img.shape[:2]
    for dy in range(3):
        for dx in range(3):
            out += p[dy:dy + h, dx:dx + w]
    return out / 9.0


def image_voronoi_layers(h: int = 1000, w: int = 1000, regions: int = 8, noise: float = 0.02,
                         seed: int = 2, third_layer: bool = True, return_labels: bool = False):
    """Image-like multilayer graph (stands in for the 9.7 MP beach image, Sec. 8.2).

    The image is split into `regions` Voronoi cells of seeded sites; each cell
    has a colour drawn U[0,1]^3, plus N(0, noise^2) per channel and pixel.
    Layer 1 = RGB (d=3); layer 2 = (x/w, y/w, texture) (d=3) with a seeded
    smooth texture field in [0,1]; layer 3 (optional) = RGB of the 3x3
    box-filtered image (d=3).  Pixels are vectorised row-major.  With
    return_labels, also the Voronoi region of every pixel (the ground truth
    of a segmentation).
    """
    rng = np.random.default_rng(seed)
    sites = rng.uniform(0.0, 1.0, size=(regions, 2)) * np.array([w, h])
    colours = rng.uniform(0.0, 1.0, size=(regions, 3))
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    best = np.full((h, w), np.inf)
    label = np.zeros((h, w), dtype=np.int64)
    for r in range(regions):
        dist = (xx - sites[r, 0]) ** 2 + (yy - sites[r, 1]) ** 2
        m = dist < best
        best[m] = dist[m]
        label[m] = r
    img = colours[label] + rng.normal(0.0, noise, size=(h, w, 3))
    tex = _smooth_texture(h, w, rng)
    layers = [img.reshape(-1, 3).copy(),
              np.stack([xx.ravel() / w, yy.ravel() / w, tex.ravel()], axis=1)]
    if third_layer:
        layers.append(_box3(img).reshape(-1, 3).copy())
    if return_labels:
        return layers, label.ravel().copy()
    return layers


def image_discs_layers(h: int = 2500, w: int = 4000, discs: int = 5, noise: float = 0.02, seed: int = 4):
    """Large single image (stands in for the 9,734,400-pixel image, Sec. 8.2).

    `discs` uniform-colour discs with seeded centres and radii over a
    background colour, plus N(0, noise^2) per channel.  Layer 1 = RGB,
    layer 2 = (x/w, y/w, texture).
    """
    rng = np.random.default_rng(seed)
    bg = rng.uniform(0.0, 1.0, size=3)
    img = np.empty((h, w, 3))
    img[...] = bg
    yy, xx = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    for _ in range(discs):
        cx, cy = rng.uniform(0.0, w), rng.uniform(0.0, h)
        rad = rng.uniform(0.05, 0.25) * min(h, w)
        col = rng.uniform(0.0, 1.0, size=3)
        img[(xx - cx) ** 2 + (yy - cy) ** 2 <= rad * rad] = col
    img += rng.normal(0.0, noise, size=img.shape)
    tex = _smooth_texture(h, w, rng)
    return [img.reshape(-1, 3).copy(),
            np.stack([xx.ravel() / w, yy.ravel() / w, tex.ravel()], axis=1)]


def gmm_band_layers(n: int = 250_000, features: int = 104, components: int = 12, seed: int = 3,
                    group: int = 2):
    """Hyperspectral-like data (stands in for Pavia centre, Sec. 8.4).

    n samples of a seeded `components`-component Gaussian mixture in
    R^features with equal weights, means U[0,1]^features and per-dimension
    standard deviations U[0.02, 0.08].  Features are grouped into layers the
    way the paper pairs bands: layer t = features (t, t + features/group, ...),
    giving features/group layers of dimension `group`.
    Returns (layers, labels).
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.0, 1.0, size=(components, features))
    stds = rng.uniform(0.02, 0.08, size=(components, features))
    labels = rng.integers(0, components, size=n)
    X = means[labels] + stds[labels] * rng.standard_normal(size=(n, features))
    T = features // group
    layers = [np.ascontiguousarray(X[:, [t + j * T for j in range(group)]]) for t in range(T)]
    return layers, labels


def known_labels(truth: np.ndarray, fraction: float, seed: int) -> np.ndarray:
    """Semi-supervised input: a seeded `fraction` of the nodes keep their
    ground-truth class, the others get -1 (at least one node per class)."""
    rng = np.random.default_rng(seed)
    n = len(truth)
    lab = -np.ones(n, dtype=np.int32)
    pick = rng.choice(n, size=max(1, int(round(fraction * n))), replace=False)
    lab[pick] = truth[pick]
    for c in np.unique(truth):
        if not (lab == c).any():
            i = rng.choice(np.nonzero(truth == c)[0])
            lab[i] = c
    return lab


def block_model_layers(sizes, p_in, p_out, seed: int):
    """Multilayer stochastic block model (Holland, Laskey, Leinhardt 1983), the
    synthetic graphs of the paper's Sec. 9 examples.

    Nodes are grouped into classes of the given sizes.  Layer t connects two
    distinct nodes of one class with probability p_in[t] and of different
    classes with p_out[t], independently per node pair; the layer's weight
    matrix is the symmetric 0/1 adjacency with zero diagonal.  Returns
    (list of n x n float64 matrices, class of each node)."""
    rng = np.random.default_rng(seed)
    truth = np.repeat(np.arange(len(sizes)), sizes).astype(np.int32)
    n = len(truth)
    same = truth[:, None] == truth[None, :]
    layers = []
    for pi, po in zip(p_in, p_out):
        A = np.triu((rng.uniform(size=(n, n)) < np.where(same, pi, po)).astype(np.float64), 1)
        layers.append(A + A.T)
    return layers, truth


def cloud_for_mlp(index: int, n_min: int = 10_000, n_max: int = 1_000_000):
    """One seeded point cloud for the parameter-selection model's data set.

    Seed 10000 + index.  n log-uniform in [n_min, n_max], d in {1,2,3}; the
    distribution is one of: uniform box, Gaussian mixture, piecewise-constant
    values plus noise.  sigma is log-uniform over 0.02..0.5 times the box size.
    Returns (points, sigma).
    """
    rng = np.random.default_rng(10_000 + index)
    n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
    d = int(rng.integers(1, 4))
    kind = int(rng.integers(0, 3))
    if kind == 0:
        X = rng.uniform(0.0, 1.0, size=(n, d))
    elif kind == 1:
        c = int(rng.integers(2, 10))
        mu = rng.uniform(0.0, 1.0, size=(c, d))
        sd = rng.uniform(0.01, 0.1, size=(c, d))
        lab = rng.integers(0, c, size=n)
        X = mu[lab] + sd[lab] * rng.standard_normal(size=(n, d))
    else:
        c = int(rng.integers(2, 10))
        lev = rng.uniform(0.0, 1.0, size=(c, d))
        lab = rng.integers(0, c, size=n)
        X = lev[lab] + rng.normal(0.0, 0.02, size=(n, d))
    box = float(np.max(X.max(axis=0) - X.min(axis=0)))
    sigma = box * float(np.exp(rng.uniform(np.log(0.02), np.log(0.5))))
    return X, sigma


# Named workloads: name -> dict(kind, params, sigma per layer, precision, k, ...)
WORKLOADS = {
    "single_n2000_d3": dict(n=2000, T=1, d=3, sigma=0.1, prec="f64", k=10, b=1),
    "image_voronoi_n1e6_T3": dict(n=1_000_000, T=3, d=3, sigma=0.2, prec="f64", k=20, p=-1.0, b=1),
    "gmm_n250k_T52_d2": dict(n=250_000, T=52, d=2, sigma="half_range", prec="f32", k=10, b=8),
    "image_discs_n1e7_T2": dict(n=10_000_000, T=2, d=3, sigma=0.15, prec="f32+f64", k=10, b=1),
}
