"""Seeded synthetic inputs for separable dictionary learning.

This module only *makes data*: random dictionaries, planted sparse codes,
synthetic images, patches and hyperspectral mixtures.  It holds none of the
learning method's arithmetic (no sparse coding, no dictionary update), so both
the FP64 oracle and the CUDA path can be fed from it without sharing code.

Array conventions (mathematical indexing, float64 unless stated):
  Y    (N, p1, p2)   signal k is the p1 x p2 matrix Y[k]
  D1   (p1, n1)      left dictionary, unit-norm columns
  D2   (p2, n2)      right dictionary, unit-norm columns
The C-ABI wants each signal column-major; ``to_colmajor`` does that reshuffle.

The paper's experiments use the USC-SIPI images and the Indian Pines cube
(Sec. IV); neither is available here, so the generators below stand in for
them with the same shapes and value ranges.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "unit_columns", "random_dictionary", "init_dictionaries", "kron_model", "kron_model3",
    "synthetic_image", "random_patches", "all_patches", "hyperspectral",
    "to_colmajor", "dict_to_colmajor",
]


def unit_columns(A: np.ndarray) -> np.ndarray:
    """Scale every column of A to unit Euclidean norm (the constraint of Eq. (1))."""
    return A / np.linalg.norm(A, axis=0, keepdims=True)


def random_dictionary(p: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """p x n dictionary with N(0,1) entries and unit-norm columns."""
    return unit_columns(rng.standard_normal((p, n)))


def init_dictionaries(p1: int, p2: int, n1: int, n2: int, seed: int = 1):
    """Initial (D1, D2): N(0,1) entries, unit columns, drawn from one seed."""
    rng = np.random.default_rng(seed)
    D1 = random_dictionary(p1, n1, rng)
    D2 = random_dictionary(p2, n2, rng)
    return D1, D2


def kron_model(N: int, p1: int, p2: int, n1: int, n2: int, s: int,
               snr_db: float | None = 20.0, seed: int = 11,
               dict_seeds: tuple[int, int] | None = None):
    """Signals from the separable generative model Y_k = D1* X_k D2*^T + noise.

    X_k holds s distinct atom pairs (i, j) drawn uniformly from the n1*n2 pairs,
    with N(0,1) values.  Noise is white Gaussian with a per-signal variance set
    so that ||clean_k||^2 / ||noise_k||^2 = 10^(snr_db/10) in expectation.
    snr_db=None gives noiseless signals.

    Returns (Y, D1_true, D2_true, support_true, coef_true); support holds the
    pair index q = i + n1*j.
    """
    if dict_seeds is None:
        dict_seeds = (seed, seed + 1)
    D1t = random_dictionary(p1, n1, np.random.default_rng(dict_seeds[0]))
    D2t = random_dictionary(p2, n2, np.random.default_rng(dict_seeds[1]))
    rng = np.random.default_rng(seed + 1000)
    nq = n1 * n2
    # s distinct pairs per signal: the s smallest of nq uniform keys pick a
    # uniformly random subset (in key order)
    keys = rng.random((N, nq), dtype=np.float32)
    part = np.argpartition(keys, s - 1, axis=1)[:, :s]
    order = np.argsort(np.take_along_axis(keys, part, axis=1), axis=1)
    support = np.take_along_axis(part, order, axis=1).astype(np.int64)
    coef = rng.standard_normal((N, s))
    ii, jj = support % n1, support // n1                  # q = i + n1*j
    clean = np.empty((N, p1, p2))
    for a in range(0, N, 65536):                          # memory only
        b = slice(a, a + 65536)
        clean[b] = np.einsum("kl,akl,bkl->kab", coef[b], D1t[:, ii[b]], D2t[:, jj[b]],
                             optimize=True)
    Y = clean
    if snr_db is not None:
        energy = np.einsum("kab,kab->k", clean, clean)
        sigma2 = energy / (p1 * p2 * 10.0 ** (snr_db / 10.0))
        Y = clean + rng.standard_normal(clean.shape) * np.sqrt(sigma2)[:, None, None]
    return Y, D1t, D2t, support, coef


def kron_model3(N: int, p: tuple, n: tuple, s: int, snr_db: float | None = 20.0,
                seed: int = 81):
    """Three-mode signals Y_k = X_k x_1 D1* x_2 D2* x_3 D3* + noise (the
    generative model of the three-mode generalisation): D_m* (p_m x n_m)
    N(0,1) with unit columns from seeds seed, seed+1, seed+2; s distinct atom
    triples per signal (q = i + n1 j + n1 n2 l) with N(0,1) values; white noise
    at snr_db per signal.  Returns (Y (N, p1, p2, p3), [D1*, D2*, D3*],
    support, coef)."""
    Ds = [random_dictionary(p[m], n[m], np.random.default_rng(seed + m)) for m in range(3)]
    rng = np.random.default_rng(seed + 1000)
    Q = n[0] * n[1] * n[2]
    keys = rng.random((N, Q), dtype=np.float32)
    part = np.argpartition(keys, s - 1, axis=1)[:, :s]
    order = np.argsort(np.take_along_axis(keys, part, axis=1), axis=1)
    support = np.take_along_axis(part, order, axis=1).astype(np.int64)
    coef = rng.standard_normal((N, s))
    ii, jj, ll = support % n[0], (support // n[0]) % n[1], support // (n[0] * n[1])
    Y = np.empty((N,) + tuple(p))
    for a in range(0, N, 32768):                          # memory only
        b = slice(a, a + 32768)
        Y[b] = np.einsum("km,akm,bkm,ckm->kabc", coef[b], Ds[0][:, ii[b]], Ds[1][:, jj[b]],
                         Ds[2][:, ll[b]], optimize=True)
    if snr_db is not None:
        energy = np.einsum("kabc,kabc->k", Y, Y)
        sigma2 = energy / (np.prod(p) * 10.0 ** (snr_db / 10.0))
        Y = Y + rng.standard_normal(Y.shape) * np.sqrt(sigma2)[:, None, None, None]
    return Y, Ds, support, coef


def synthetic_image(seed: int, size: int = 512, n_regions: int = 24,
                    n_edges: int = 8, texture_std: float = 6.0) -> np.ndarray:
    """Seeded piecewise-smooth test image in [0, 255] (stand-in for a SIPI photo).

    Voronoi regions with planar intensity ramps, plus straight edges (a step
    offset on one side of a random line), plus a 1/f spectral-synthesis
    texture, clipped to [0, 255].
    """
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    cy = rng.uniform(0, size, n_regions)
    cx = rng.uniform(0, size, n_regions)
    label = np.zeros((size, size), dtype=np.int64)
    best = np.full((size, size), np.inf)
    for r in range(n_regions):
        d = (yy - cy[r]) ** 2 + (xx - cx[r]) ** 2
        closer = d < best
        best[closer] = d[closer]
        label[closer] = r
    base = rng.uniform(40, 215, n_regions)
    gy = rng.uniform(-0.15, 0.15, n_regions)
    gx = rng.uniform(-0.15, 0.15, n_regions)
    img = base[label] + gy[label] * (yy - cy[label]) + gx[label] * (xx - cx[label])
    for _ in range(n_edges):
        theta = rng.uniform(0, np.pi)
        off = rng.uniform(0.2 * size, 0.8 * size)
        side = (np.cos(theta) * xx + np.sin(theta) * yy) > off
        img = img + side * rng.uniform(-40, 40)
    f = np.fft.fftfreq(size)
    fr = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    fr[0, 0] = 1.0
    spec = np.fft.fft2(rng.standard_normal((size, size))) / fr
    spec[0, 0] = 0.0
    tex = np.real(np.fft.ifft2(spec))
    tex *= texture_std / tex.std()
    return np.clip(img + tex, 0.0, 255.0)


def random_patches(images: np.ndarray, N: int, p: int, seed: int,
                   remove_mean: bool = True) -> np.ndarray:
    """N p x p patches at seeded uniform positions of a stack of images.

    Y[k, a, b] = img[r + a, c + b]: rows of the patch are the p1 index.
    """
    rng = np.random.default_rng(seed)
    n_img, H, W = images.shape
    which = rng.integers(0, n_img, N)
    r = rng.integers(0, H - p + 1, N)
    c = rng.integers(0, W - p + 1, N)
    a = np.arange(p)
    Y = images[which[:, None, None], r[:, None, None] + a[None, :, None],
               c[:, None, None] + a[None, None, :]]
    if remove_mean:
        Y = Y - Y.mean(axis=(1, 2), keepdims=True)
    return Y


def all_patches(img: np.ndarray, p: int):
    """Every stride-1 p x p patch of one image, raster order (row of the
    top-left corner major).  Returns (patches (M, p, p), means (M,))."""
    H, W = img.shape
    win = np.lib.stride_tricks.sliding_window_view(img, (p, p))
    Y = win.reshape((H - p + 1) * (W - p + 1), p, p).astype(np.float64)
    means = Y.mean(axis=(1, 2))
    return Y - means[:, None, None], means


def hyperspectral(N: int, pixels: int = 16, bands: int = 64, n_end: int = 8,
                  snr_db: float = 30.0, seed: int = 31) -> np.ndarray:
    """Hyperspectral-shaped 2D signals: Y_k = A_k S + noise, pixels x bands.

    S holds n_end smooth random spectra (each a sum of 3 positive Gaussian
    bumps over the bands); every pixel's abundances A_k[a, :] ~ Dirichlet(1);
    per-signal white noise at snr_db.
    """
    rng = np.random.default_rng(seed)
    b = np.arange(bands, dtype=np.float64)
    S = np.zeros((n_end, bands))
    for e in range(n_end):
        for _ in range(3):
            mu = rng.uniform(0, bands)
            w = rng.uniform(bands / 16, bands / 4)
            S[e] += rng.uniform(0.2, 1.0) * np.exp(-0.5 * ((b - mu) / w) ** 2)
    A = rng.dirichlet(np.ones(n_end), size=(N, pixels))
    clean = A @ S
    energy = np.einsum("kab,kab->k", clean, clean)
    sigma2 = energy / (pixels * bands * 10.0 ** (snr_db / 10.0))
    return clean + rng.standard_normal(clean.shape) * np.sqrt(sigma2)[:, None, None]


def to_colmajor(Y: np.ndarray, dtype=np.float32) -> np.ndarray:
    """(N, p1, p2) -> contiguous buffer where element (a, b, k) sits at
    a + p1*b + p1*p2*k (each signal column-major, signals back to back)."""
    return np.ascontiguousarray(np.asarray(Y).transpose(0, 2, 1), dtype=dtype)


def dict_to_colmajor(D: np.ndarray, dtype=np.float32) -> np.ndarray:
    """p x n dictionary -> column-major buffer (shape (n, p) in C order)."""
    return np.ascontiguousarray(np.asarray(D).T, dtype=dtype)
