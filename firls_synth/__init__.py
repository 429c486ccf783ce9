"""Seeded synthetic inputs for FIRLS reconstructions (CS-MRI style).

This module generates the *inputs* of a reconstruction and nothing else:
ellipse phantoms, smooth phase maps, variable-density Cartesian sampling
masks, noisy undersampled k-space measurements and wavelet parent-child
(tree) group maps.  It holds none of the reconstruction method's arithmetic
(no weights, no preconditioners, no PCG) and is shared by the FP64 oracle
and the CUDA path so that both see exactly the same problem.

The paper's test images (Sec. 5: Brain/Cardiac/Chest/Shoulder MR images, the
SRI24 atlas) are not available; seeded phantoms with the same shapes (n x n
images, 15-30 % variable-density sampling, Sec. 5.4) stand in for them.

Random numbers come from numpy's PCG64 generator seeded with
``[seed, substream]`` so that phantom, phase, mask and noise of one instance
are independent streams and every instance is reproducible from its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PHANTOM, PHASE, MASK, NOISE, PARAMS = 0, 1, 2, 3, 4

PSI_HAAR = 1
PSI_DB4 = 2
PSI_TV = 4
PSI_TV_ANISO = 8   # l1 (anisotropic) TV


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def ellipse_phantom(n: int, seed: int, n_ellipses: int = 10) -> np.ndarray:
    """Real n x n phantom: sum of ``n_ellipses`` random filled ellipses.

    Coordinates are pixel centres on [-1, 1]^2 (row index -> v, column -> u).
    Each ellipse: centre U[-0.7, 0.7]^2, semi-axes U[0.05, 0.45], angle
    U[0, pi), intensity U[0, 1].
    """
    rng = _rng(seed, PHANTOM)
    t = (2.0 * (np.arange(n) + 0.5) / n) - 1.0
    v, u = np.meshgrid(t, t, indexing="ij")
    img = np.zeros((n, n), dtype=np.float64)
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.7, 0.7, size=2)
        ax, ay = rng.uniform(0.05, 0.45, size=2)
        th = rng.uniform(0.0, math.pi)
        inten = rng.uniform(0.0, 1.0)
        du, dv = u - cx, v - cy
        ct, st = math.cos(th), math.sin(th)
        pu = ct * du + st * dv
        pv = -st * du + ct * dv
        inside = (pu / ax) ** 2 + (pv / ay) ** 2 <= 1.0
        img[inside] += inten
    return img


def smooth_phase(n: int, seed: int) -> np.ndarray:
    """Phase map phi = pi * sum_{p+q<=2} a_pq u^p v^q with a_pq ~ U[-0.5, 0.5]."""
    rng = _rng(seed, PHASE)
    t = (2.0 * (np.arange(n) + 0.5) / n) - 1.0
    v, u = np.meshgrid(t, t, indexing="ij")
    phi = np.zeros((n, n))
    for p in range(3):
        for q in range(3 - p):
            phi += rng.uniform(-0.5, 0.5) * u ** p * v ** q
    return math.pi * phi


def complex_phantom(n: int, seed: int) -> np.ndarray:
    """Complex phantom: ellipse magnitude times exp(i * smooth phase)."""
    return ellipse_phantom(n, seed) * np.exp(1j * smooth_phase(n, seed))


def vd_mask(n: int, ratio: float, seed: int) -> np.ndarray:
    """Variable-density random Cartesian sampling mask, uint8 [n][n].

    Unshifted FFT order (DC at [0][0]; index k >= n/2 stands for k - n).
    Exactly round(ratio * n^2) points are drawn without replacement by
    weighted sampling (Efraimidis-Spirakis keys u^(1/w), largest keys win,
    ties to the lower flat index) with weight w = (1 - r/r_max)^4 + 0.02,
    r the distance to DC; DC is always kept.  Denser at low frequencies, as
    in the paper's CS-MRI experiments (Sec. 5.4).
    """
    N = n * n
    m = int(round(ratio * N))
    m = max(1, min(N, m))
    rng = _rng(seed, MASK)
    k = np.arange(n)
    k = np.where(k >= n // 2, k - n, k).astype(np.float64)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    r = np.sqrt(kx ** 2 + ky ** 2)
    rmax = r.max()
    w = (1.0 - r / rmax) ** 4 + 0.02
    u = rng.random(N)
    keys = u ** (1.0 / w.ravel())
    keys[0] = np.inf  # DC always kept
    order = np.argsort(-keys, kind="stable")
    mask = np.zeros(N, dtype=np.uint8)
    mask[order[:m]] = 1
    return mask.reshape(n, n)


def measurements(x0: np.ndarray, mask: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Undersampled noisy k-space b = mask * (F x0 + noise), complex128 [n][n].

    F is the unitary 2-D DFT; the noise is i.i.d. N(0, sigma^2) on the real and
    on the imaginary part of every sampled entry.  Entries off the mask are 0.
    """
    n = x0.shape[0]
    rng = _rng(seed, NOISE)
    y = np.fft.fft2(x0, norm="ortho")
    noise = sigma * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return (mask.astype(np.float64)) * (y + noise)


def tree_groups(n: int, levels: int) -> np.ndarray:
    """Parent-child wavelet tree groups of size 2, int32 [n_groups][2].

    One group per detail coefficient c of an ``levels``-level Mallat layout
    (flat row-major index into the n x n coefficient array): (c, parent(c)).
    The parent of a detail coefficient at level l (local position (i, j) of
    its subband) is the coefficient of the same subband one level coarser at
    (i // 2, j // 2); for the coarsest detail level it is the co-located
    approximation (LL) coefficient.  Groups are ordered by the flat index of
    c.  A quadtree parent has 4 children, so detail coefficients of levels
    2..L belong to 5 groups, the finest ones to 1 and LL ones to 3.
    """
    if n % (1 << levels):
        raise ValueError("n must be divisible by 2^levels")
    child, parent = [], []
    for lvl in range(1, levels + 1):
        h = n >> lvl
        i, j = np.meshgrid(np.arange(h), np.arange(h), indexing="ij")
        for br, bc in ((0, 1), (1, 0), (1, 1)):
            r, c = br * h + i, bc * h + j
            if lvl < levels:
                hp = h // 2
                pr, pc = br * hp + i // 2, bc * hp + j // 2
            else:
                pr, pc = i, j
            child.append((r * n + c).ravel())
            parent.append((pr * n + pc).ravel())
    child = np.concatenate(child)
    parent = np.concatenate(parent)
    order = np.argsort(child, kind="stable")
    return np.stack([child[order], parent[order]], axis=1).astype(np.int32)


@dataclass
class Problem:
    """One reconstruction problem (inputs only)."""
    n: int
    mask: np.ndarray            # uint8 [n][n]
    b: np.ndarray               # complex128 [n][n] (zero off the mask)
    x0: np.ndarray              # ground truth (real or complex)
    real: bool                  # unknown is real (config with a real phantom)
    psi: int                    # bitmask of PSI_HAAR / PSI_DB4 / PSI_TV
    levels: int                 # wavelet levels
    lam: float                  # wavelet lambda (or the only lambda)
    lam_tv: float               # TV lambda (0 if no TV)
    groups: np.ndarray | None = None   # int32 [n_groups][g] or None = singletons
    seed: int = 0
    meta: dict = field(default_factory=dict)


def make_problem(n, ratio, sigma, seed, *, real, psi, levels, lam, lam_tv=0.0, tree=False):
    x0 = ellipse_phantom(n, seed) if real else complex_phantom(n, seed)
    mask = vd_mask(n, ratio, seed)
    b = measurements(x0, mask, sigma, seed)
    groups = tree_groups(n, levels) if tree else None
    return Problem(n=n, mask=mask, b=b, x0=x0, real=real, psi=psi, levels=levels,
                   lam=lam, lam_tv=lam_tv, groups=groups, seed=seed,
                   meta=dict(ratio=ratio, sigma=sigma))


# --- multi-contrast cross sections (joint sparsity / joint TV) --------------

CONTRAST = 5   # substream of the per-contrast intensities


def contrast_phantoms(n: int, contrasts: int, seed: int, n_ellipses: int = 10) -> list:
    """Complex phantoms of one cross section seen with several contrasts: the
    ellipse geometry (centres, semi-axes, angles) of ``seed`` is shared, the
    intensity of every ellipse is drawn per contrast (U[0, 1], substream
    CONTRAST, one draw per contrast and ellipse), and every contrast gets its
    own smooth phase map (seed * 1000 + t)."""
    geo = _rng(seed, PHANTOM)
    shapes = []
    for _ in range(n_ellipses):
        cx, cy = geo.uniform(-0.7, 0.7, size=2)
        ax, ay = geo.uniform(0.05, 0.45, size=2)
        th = geo.uniform(0.0, math.pi)
        geo.uniform(0.0, 1.0)  # the single-contrast intensity draw, unused here
        shapes.append((cx, cy, ax, ay, th))
    inten = _rng(seed, CONTRAST).uniform(0.0, 1.0, size=(contrasts, n_ellipses))
    t = (2.0 * (np.arange(n) + 0.5) / n) - 1.0
    v, u = np.meshgrid(t, t, indexing="ij")
    out = []
    for c in range(contrasts):
        img = np.zeros((n, n))
        for e, (cx, cy, ax, ay, th) in enumerate(shapes):
            du, dv = u - cx, v - cy
            ct, st = math.cos(th), math.sin(th)
            inside = ((ct * du + st * dv) / ax) ** 2 + ((-st * du + ct * dv) / ay) ** 2 <= 1.0
            img[inside] += inten[c, e]
        out.append(img * np.exp(1j * smooth_phase(n, seed * 1000 + c)))
    return out


def multi_contrast(n: int, contrasts: int, ratio: float, sigma: float, seed: int, *, psi: int, levels: int,
                   lam: float, lam_tv: float = 0.0) -> list:
    """One multi-contrast cross section: a Problem per contrast with its own
    variable-density mask and noise (seeds seed * 1000 + t)."""
    out = []
    for c, x0 in enumerate(contrast_phantoms(n, contrasts, seed)):
        s = seed * 1000 + c
        mask = vd_mask(n, ratio, s)
        out.append(Problem(n=n, mask=mask, b=measurements(x0, mask, sigma, s), x0=x0, real=False, psi=psi,
                           levels=levels, lam=lam, lam_tv=lam_tv, groups=None, seed=s,
                           meta=dict(ratio=ratio, sigma=sigma, contrast=c)))
    return out


# --- the five workloads -----------------------------------------------------

def haar_l1_64(seed: int = 1) -> Problem:
    """64x64 real phantom, 25 % mask, sigma 0.01, 3-level Haar, l1, lambda 1e-3."""
    return make_problem(64, 0.25, 0.01, seed, real=True, psi=PSI_HAAR, levels=3, lam=1e-3)


def tv_db4_256(seed: int = 2, n: int = 256) -> Problem:
    """256x256 complex, 20 % mask, sigma 0.01, isotropic TV (lambda_TV 1e-3)
    plus 4-level Daubechies-4 l1 (lambda_W 5e-4)."""
    return make_problem(n, 0.20, 0.01, seed, real=False, psi=PSI_TV | PSI_DB4, levels=4,
                        lam=5e-4, lam_tv=1e-3)


def tree_db4_512(seed: int = 3, n: int = 512) -> Problem:
    """512x512 complex, 15 % mask, sigma 0.005, 5-level D4 with parent-child
    tree groups of size 2 (overlapping), lambda 2e-4."""
    return make_problem(n, 0.15, 0.005, seed, real=False, psi=PSI_DB4, levels=5, lam=2e-4, tree=True)


UNEVEN_SIZES = (128, 192, 256, 320)


def uneven_batch(first_seed: int = 1000, per_size: int = 16) -> list[Problem]:
    """Slices of uneven size (per_size each at 128, 192, 256, 320), TV + D4.

    Per slice: mask ratio U[0.15, 0.30], lambda_TV log-uniform in [1e-4, 1e-3],
    lambda_W = lambda_TV / 2, sigma 0.01; seeds first_seed, first_seed+1, ...
    """
    out = []
    s = first_seed
    for n in UNEVEN_SIZES:
        for _ in range(per_size):
            rng = _rng(s, PARAMS)
            ratio = float(rng.uniform(0.15, 0.30))
            lam_tv = float(10.0 ** rng.uniform(-4.0, -3.0))
            out.append(make_problem(n, ratio, 0.01, s, real=False, psi=PSI_TV | PSI_DB4, levels=4,
                                    lam=lam_tv / 2, lam_tv=lam_tv))
            s += 1
    return out


def mt_db4_256(seed: int = 1, n: int = 256) -> list[Problem]:
    """Multi-contrast cross section (joint sparsity, FIRLS_MT): 3 contrasts at
    256x256, 25 % variable-density masks (one per contrast), sigma 0.01, joint
    4-level Daubechies-4 sparsity, lambda 1e-3."""
    return multi_contrast(n, 3, 0.25, 0.01, seed, psi=PSI_DB4, levels=4, lam=1e-3)


# --- dense random projections (Sec. 5.2-5.3) ---------------------------------

DENSE = 6


@dataclass
class DenseProblem:
    """One sparse-recovery problem with a dense sensing matrix (inputs only)."""
    A: np.ndarray               # float64 [M][N]
    b: np.ndarray               # float64 [M]
    x0: np.ndarray              # float64 [N], the sparse ground truth
    lam: float
    seed: int = 0


def dense_l1(seed: int, N: int = 4000, M: int = 800, density: float = 0.1, sigma: float = 0.01,
             lam: float = 0.05) -> DenseProblem:
    """The 1-D random-projection workload of Sec. 5.3 (length 4000, 10 %
    non-zeros, 800 measurements): A with i.i.d. N(0, 1/M) entries (substream
    DENSE, row-major draws), round(density N) non-zeros at uniformly random
    positions with N(0, 1) values (substream PHANTOM), b = A x0 + sigma e with
    e ~ N(0, I) (substream NOISE)."""
    A = _rng(seed, DENSE).standard_normal((M, N)) / math.sqrt(M)
    g = _rng(seed, PHANTOM)
    k = int(round(density * N))
    x0 = np.zeros(N)
    x0[g.choice(N, size=k, replace=False)] = g.standard_normal(k)
    b = A @ x0 + sigma * _rng(seed, NOISE).standard_normal(M)
    return DenseProblem(A=A, b=b, x0=x0, lam=lam, seed=seed)


def dense_l1_shared(seed: int, problems: int, N: int = 4000, M: int = 800, density: float = 0.1,
                    sigma: float = 0.01, lam: float = 0.05):
    """Several signals measured by one projection (the workload of Sec. 5.3
    with A shared): A as in ``dense_l1(seed)``; signal p has the non-zeros and
    the noise of ``dense_l1(seed + p)`` (substreams PHANTOM and NOISE of
    seed + p), so problem 0 is ``dense_l1(seed)`` itself.  Returns
    (A [M][N], B [problems][M], X0 [problems][N], lam), float64."""
    A = _rng(seed, DENSE).standard_normal((M, N)) / math.sqrt(M)
    k = int(round(density * N))
    X0 = np.zeros((problems, N))
    B = np.empty((problems, M))
    for p in range(problems):
        g = _rng(seed + p, PHANTOM)
        X0[p, g.choice(N, size=k, replace=False)] = g.standard_normal(k)
        B[p] = A @ X0[p] + sigma * _rng(seed + p, NOISE).standard_normal(M)
    return A, B, X0, lam


# --- learned warm start: architecture and seeded initial weights ------------

CNN_CHANNELS = (3, 32, 32, 32, 32, 32, 2)   # input: Re A^H b, Im A^H b, mask


def cnn_init_weights(seed: int = 0):
    """He-normal initial weights of the 6-layer 3x3 CNN, float32.

    Returns a list of (w [3][3][c_in][c_out], b [c_out]); the last layer starts
    at zero so that the untrained network returns A^H b unchanged.
    """
    rng = _rng(seed, PARAMS + 1)
    out = []
    layers = len(CNN_CHANNELS) - 1
    for l in range(layers):
        cin, cout = CNN_CHANNELS[l], CNN_CHANNELS[l + 1]
        std = math.sqrt(2.0 / (9 * cin))
        w = (rng.standard_normal((3, 3, cin, cout)) * std).astype(np.float32)
        if l == layers - 1:
            w[:] = 0.0
        out.append((w, np.zeros(cout, dtype=np.float32)))
    return out


def cnn_input(atb: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Network input [n][n][3]: Re A^H b, Im A^H b, mask (as float)."""
    return np.stack([atb.real, atb.imag, mask.astype(np.float64)], axis=-1)
