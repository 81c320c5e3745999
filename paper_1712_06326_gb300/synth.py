"""Seeded synthetic workloads for the exemplar-inpainting patch search.

This module only *generates inputs*: images/volumes, known-masks and the set of
query centres.  It holds none of the search arithmetic (no cost, projection,
key or sort), so both the CUDA path and the CPU oracle can read the buffers it
produces without sharing any of the method's code.

The paper evaluates on photographs with text masks (Sec. II.I); those are not
available, so these generators stand in for them with the shapes and value
ranges of the synthetic configurations:

* ``sines2d``   -- 128x128 grey image, 6 random sinusoids + noise, centred hole.
* ``voronoi2d`` -- RGB image of Voronoi regions with gradients, texture and
                   noise; disc-shaped holes covering ~10 % of the pixels.
* ``spheres3d`` -- grey volume of blurred random spheres + noise; a fraction of
                   aligned cubic blocks is missing.

Layout of every grid: float32, C-contiguous, shape (Y, X, ch) in 2-D and
(Z, Y, X, ch) in 3-D (x fastest, channel innermost).  Masks: uint8, shape (Y, X)
or (Z, Y, X), 1 = known.  Query centres: int32 array (Q, ndim) holding (x, y)
or (x, y, z).

RNG: numpy PCG64 seeded with ``1712063260 + config number`` (plus an image
index where several images are drawn).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1712063260


def rng_for(cfg: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + cfg, sub])


# ----------------------------------------------------------------------------
# 2-D grey sinusoids (small plain-method case)
# ----------------------------------------------------------------------------
def sines2d(size: int = 128, hole: tuple[int, int] | None = None, seed_sub: int = 0):
    """Grey image 0.5 + sum of 6 random-orientation sinusoids + N(0, 0.05^2),
    clamped to [0, 1]; centred square hole ([52, 76)^2 for 128x128)."""
    rng = rng_for(1, seed_sub)
    a = rng.uniform(0.05, 0.12, 6)
    f = rng.uniform(2.0, 12.0, 6)
    th = rng.uniform(0.0, math.pi, 6)
    ph = rng.uniform(0.0, 2.0 * math.pi, 6)
    y, x = np.mgrid[0:size, 0:size].astype(np.float64)
    img = np.full((size, size), 0.5)
    for i in range(6):
        img += a[i] * np.sin(2.0 * math.pi * f[i] * (x * math.cos(th[i]) + y * math.sin(th[i])) / size + ph[i])
    img += rng.normal(0.0, 0.05, (size, size))
    img = np.clip(img, 0.0, 1.0).astype(np.float32)
    mask = np.ones((size, size), np.uint8)
    if hole is None:
        h = (size * 24) // 128
        lo = (size - h) // 2
        hole = (lo, lo + h)
    mask[hole[0]:hole[1], hole[0]:hole[1]] = 0
    return np.ascontiguousarray(img[..., None]), mask


# ----------------------------------------------------------------------------
# 2-D RGB Voronoi regions (paper-scale 2-D case)
# ----------------------------------------------------------------------------
def voronoi2d(width: int = 1024, height: int | None = None, cfg: int = 2, seed_sub: int = 0,
              coverage: float = 0.10, seeds: int = 64):
    """RGB image of Voronoi regions, each with a base colour U(0.2, 0.8)^3, a
    linear gradient (up to +-0.3 over 1024 px), a sinusoidal texture
    (amplitude 0.05) and N(0, 0.02^2) noise, clamped to [0, 1].  Mask = union
    of seeded discs (radius U{24..64} scaled by min(W, H)/1024, >= 4) added
    until >= ``coverage`` of the pixels are unknown."""
    height = width if height is None else height
    rng = rng_for(cfg, seed_sub)
    W, H = width, height
    sx = rng.uniform(0, W, seeds)
    sy = rng.uniform(0, H, seeds)
    base = rng.uniform(0.2, 0.8, (seeds, 3))
    gth = rng.uniform(0, 2 * math.pi, seeds)
    gamp = rng.uniform(-0.3, 0.3, (seeds, 3))
    tf = rng.uniform(4.0, 40.0, seeds)
    tth = rng.uniform(0, math.pi, seeds)
    tph = rng.uniform(0, 2 * math.pi, seeds)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    best = np.full((H, W), np.inf)
    lab = np.zeros((H, W), np.int64)
    for s in range(seeds):
        d = (x - sx[s]) ** 2 + (y - sy[s]) ** 2
        m = d < best
        best[m] = d[m]
        lab[m] = s
    img = np.empty((H, W, 3))
    u = ((x - sx[lab]) * np.cos(gth[lab]) + (y - sy[lab]) * np.sin(gth[lab])) / 1024.0
    tex = 0.05 * np.sin(2 * math.pi * tf[lab] * (x * np.cos(tth[lab]) + y * np.sin(tth[lab])) / 1024.0 + tph[lab])
    for c in range(3):
        img[..., c] = base[lab, c] + gamp[lab, c] * u + tex
    img += rng.normal(0.0, 0.02, (H, W, 3))
    img = np.clip(img, 0.0, 1.0).astype(np.float32)

    mask = np.ones((H, W), np.uint8)
    scale = min(W, H) / 1024.0
    target = coverage * W * H
    unknown = 0
    while unknown < target:
        rad = max(4.0, rng.integers(24, 65) * scale)
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        x0, x1 = max(0, int(cx - rad) - 1), min(W, int(cx + rad) + 2)
        y0, y1 = max(0, int(cy - rad) - 1), min(H, int(cy + rad) + 2)
        yy, xx = np.mgrid[y0:y1, x0:x1]
        disc = (xx - cx) ** 2 + (yy - cy) ** 2 <= rad * rad
        sub = mask[y0:y1, x0:x1]
        sub[disc] = 0
        unknown = int((mask == 0).sum())
    return np.ascontiguousarray(img), mask


# ----------------------------------------------------------------------------
# 3-D grey spheres (sparse-scan microscopy style)
# ----------------------------------------------------------------------------
def _blur1d(v: np.ndarray, axis: int, sigma: float, radius: int) -> np.ndarray:
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    out = np.zeros_like(v)
    n = v.shape[axis]
    for i, w in enumerate(k):
        o = i - radius
        src = np.take(v, np.clip(np.arange(n) + o, 0, n - 1), axis=axis)
        out += w * src
    return out


def spheres3d(size: int = 256, cfg: int = 3, fill: float = 0.30, block: int = 8, missing: float = 0.15,
              noise: float = 0.03, salt: float = 0.0, seed_sub: int = 0):
    """Grey volume: background 0.5, random spheres (radius U[3, 20] scaled by
    size/256, grey U(0, 1), later spheres overwrite) until ~``fill`` of the
    voxels are covered, separable Gaussian blur (sigma 1 voxel, radius 3),
    N(0, noise^2), optional salt-and-pepper outliers, clamped to [0, 1].
    Mask: ``missing`` of the aligned ``block``^3 blocks, chosen by a seeded
    shuffle, are unknown."""
    rng = rng_for(cfg, seed_sub)
    S = size
    vol = np.full((S, S, S), 0.5, np.float64)
    covered = np.zeros((S, S, S), bool)
    sc = S / 256.0
    goal = fill * S ** 3
    ncov = 0
    while ncov < goal:
        r = rng.uniform(3.0, 20.0) * sc
        c = rng.uniform(0, S, 3)
        g = rng.uniform(0.0, 1.0)
        lo = np.maximum(0, np.floor(c - r).astype(int))
        hi = np.minimum(S, np.ceil(c + r).astype(int) + 1)
        zz, yy, xx = np.mgrid[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = g
        csub = covered[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        ncov += int((inside & ~csub).sum())
        csub[inside] = True
    for ax in range(3):
        vol = _blur1d(vol, ax, 1.0, 3)
    vol += rng.normal(0.0, noise, vol.shape)
    if salt > 0:
        hit = rng.random(vol.shape) < salt
        vol[hit] = (rng.random(int(hit.sum())) < 0.5).astype(np.float64)
    vol = np.clip(vol, 0.0, 1.0).astype(np.float32)
    nb = S // block
    blocks = nb ** 3
    kill = rng.permutation(blocks)[: int(round(missing * blocks))]
    mask = np.ones((S, S, S), np.uint8)
    for b in kill:
        bz, rem = divmod(int(b), nb * nb)
        by, bx = divmod(rem, nb)
        mask[bz * block:(bz + 1) * block, by * block:(by + 1) * block, bx * block:(bx + 1) * block] = 0
    return np.ascontiguousarray(vol[..., None]), mask


# ----------------------------------------------------------------------------
# batched workload: many images of uneven size
# ----------------------------------------------------------------------------
def batch_sizes(count: int = 256, cfg: int = 4, lo: int = 256, hi: int = 2048, seed_sub: int = 0):
    """(width, height) of ``count`` images, each side round(2^U(log2 lo, log2 hi))
    independently (log-uniform); image i is voronoi2d(width, height, cfg,
    seed_sub=1 + i) with its 10 % disc mask."""
    rng = rng_for(cfg, seed_sub)
    w = np.round(2.0 ** rng.uniform(math.log2(lo), math.log2(hi), count)).astype(int)
    h = np.round(2.0 ** rng.uniform(math.log2(lo), math.log2(hi), count)).astype(int)
    return [(int(a), int(b)) for a, b in zip(w, h)]


def batch_image(i: int, size, cfg: int = 4):
    """Image i of the batched workload (grid, mask)."""
    return voronoi2d(size[0], size[1], cfg=cfg, seed_sub=1 + i)


def batch_case(i: int, size, K: int, cap: int, cfg: int = 4):
    """Image i of the batched workload with its queries: (grid, mask, front
    targets capped at ``cap`` with sub-seed 100 + i)."""
    g, m = batch_image(i, size, cfg)
    return g, m, front_targets(m, K, cap=cap, cfg=cfg, seed_sub=100 + i)


# ----------------------------------------------------------------------------
# query centres: known pixels next to the hole (the targets a fill loop meets)
# ----------------------------------------------------------------------------
def front_targets(mask: np.ndarray, K: int, cap: int | None = None, cfg: int = 0, seed_sub: int = 7) -> np.ndarray:
    """Centres of target patches for a batch of queries: every known pixel with
    an axis-neighbour (4- or 6-connected) that is unknown, moved inside the
    valid centre range [r, ext-1-r], de-duplicated and sorted in raster order.
    If more than ``cap`` remain, a seeded subset of ``cap`` is kept (still in
    raster order).  Returns int32 (Q, ndim) with columns (x, y[, z])."""
    r = K // 2
    known = mask.astype(bool)
    unk = ~known
    near = np.zeros_like(known)
    for ax in range(mask.ndim):
        n = mask.shape[ax]
        sl_a = [slice(None)] * mask.ndim
        sl_b = [slice(None)] * mask.ndim
        sl_a[ax] = slice(0, n - 1)
        sl_b[ax] = slice(1, n)
        near[tuple(sl_a)] |= unk[tuple(sl_b)]
        near[tuple(sl_b)] |= unk[tuple(sl_a)]
    front = known & near
    idx = np.argwhere(front)  # (.., z, y, x) order of numpy axes
    coords = idx[:, ::-1].copy()  # -> (x, y[, z])
    ext = np.array(mask.shape[::-1])
    coords = np.clip(coords, r, ext - 1 - r)
    lin = np.zeros(len(coords), np.int64)
    mul = 1
    for a in range(mask.ndim):
        lin += coords[:, a] * mul
        mul *= int(ext[a])
    lin = np.unique(lin)
    if cap is not None and len(lin) > cap:
        rng = rng_for(cfg, seed_sub)
        lin = np.sort(rng.choice(lin, size=cap, replace=False))
    out = np.empty((len(lin), mask.ndim), np.int32)
    rem = lin.copy()
    for a in range(mask.ndim):
        out[:, a] = rem % int(ext[a])
        rem //= int(ext[a])
    return out


def random_targets(mask: np.ndarray, K: int, count: int, cfg: int = 0, seed_sub: int = 11) -> np.ndarray:
    """``count`` seeded query centres drawn uniformly from the valid centre
    range (they may sit anywhere, known or not); int32 (count, ndim)."""
    r = K // 2
    rng = rng_for(cfg, seed_sub)
    ext = mask.shape[::-1]
    cols = [rng.integers(r, e - r, count) for e in ext]
    return np.stack(cols, axis=1).astype(np.int32)
