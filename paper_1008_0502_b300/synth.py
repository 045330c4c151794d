"""Seeded synthetic video and graph inputs.

This module produces INPUTS only: RGB8 frames, ground-truth object masks and
random integer capacities.  It holds none of the segmentation method's
arithmetic (no saliency, prior, term or cut computation) and is the one module
that both the CUDA path's tests/bench and the CPU oracle draw inputs from.

The paper's own clips (Sec. 8.1: ten hand-labelled 5-10 s clips at 12 fps) are
not available; these scenes stand in for them with the shapes of the workloads
the method is measured on:

* ``clip_small`` -- 160x120, 10 frames: low-passed grey noise background in
  [40, 90] with one saturated red disk (r = 15) doing a random walk (steps of at
  most 3 px per axis).
* ``clip_vga`` -- 640x480, 300 frames: textured grey background panned by
  1 px/frame; a yellow ellipse (semi-axes 40x25) moving at (2, 1) px/frame and
  reflecting at the borders; a static 96x96 grating patch (period 8 px at 45
  degrees, grey level 65 +- 40); a light-grey disk (r = 30) that fades out
  linearly over the clip.

Seeds are 10080502 + k for the k-th workload.  Random numbers come from
numpy's PCG64 generator.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

SEED_BASE = 10080502


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def noise_background(rng: np.random.Generator, H: int, W: int, sigma: float = 4.0,
                     lo: float = 40.0, hi: float = 90.0) -> np.ndarray:
    """Grey texture: U(0,1) noise, Gaussian low-pass (reflect), mapped onto [lo, hi]."""
    u = rng.random((H, W))
    b = ndimage.gaussian_filter(u, sigma, mode="reflect")
    b = (b - b.min()) / max(b.max() - b.min(), 1e-12) * (hi - lo) + lo
    return np.rint(b).astype(np.uint8)


def _disk(H: int, W: int, cy: float, cx: float, r: float) -> np.ndarray:
    yy, xx = np.mgrid[0:H, 0:W]
    return (yy - cy) ** 2 + (xx - cx) ** 2 <= r * r


def _ellipse(H: int, W: int, cy: float, cx: float, ry: float, rx: float) -> np.ndarray:
    yy, xx = np.mgrid[0:H, 0:W]
    return ((yy - cy) / ry) ** 2 + ((xx - cx) / rx) ** 2 <= 1.0


def clip_small(n_frames: int = 10, H: int = 120, W: int = 160, seed: int = SEED_BASE + 1,
               radius: int = 15, step: int = 3):
    """Grey low-passed background + saturated red disk on a clamped random walk.

    Returns ``(frames[n,H,W,3] uint8, gt[n,H,W] uint8)``.
    """
    rng = _rng(seed)
    bg = noise_background(rng, H, W)
    cy = int(rng.integers(radius, H - radius))
    cx = int(rng.integers(radius, W - radius))
    frames = np.empty((n_frames, H, W, 3), np.uint8)
    gt = np.empty((n_frames, H, W), np.uint8)
    for t in range(n_frames):
        if t > 0:
            dy, dx = rng.integers(-step, step + 1, size=2)
            cy = int(np.clip(cy + dy, radius, H - 1 - radius))
            cx = int(np.clip(cx + dx, radius, W - 1 - radius))
        f = np.repeat(bg[:, :, None], 3, axis=2)
        m = _disk(H, W, cy, cx, radius)
        f[m] = (255, 0, 0)
        frames[t] = f
        gt[t] = m
    return frames, gt


def clip_vga(n_frames: int = 300, H: int = 480, W: int = 640, seed: int = SEED_BASE + 2):
    """Panned texture + moving yellow ellipse + static grating + fading grey disk.

    Returns ``(frames[n,H,W,3] uint8, gt[n,H,W] uint8)``.  Frames are generated
    one at a time by :func:`clip_vga_frames`; this helper stacks them.
    """
    frames = np.empty((n_frames, H, W, 3), np.uint8)
    gt = np.empty((n_frames, H, W), np.uint8)
    for t, (f, g) in enumerate(clip_vga_frames(n_frames, H, W, seed)):
        frames[t] = f
        gt[t] = g
    return frames, gt


def clip_vga_frames(n_frames: int = 300, H: int = 480, W: int = 640, seed: int = SEED_BASE + 2,
                    pan: int = 1):
    """Generator form of :func:`clip_vga` (one frame at a time, low memory)."""
    rng = _rng(seed)
    canvas = noise_background(rng, H, W + pan * max(n_frames - 1, 0) + 1)
    # static grating patch, 96x96, period 8 px along the 45-degree direction
    gs = 96
    gy0 = int(rng.integers(0, H - gs))
    gx0 = int(rng.integers(0, W - gs))
    py, px = np.mgrid[0:gs, 0:gs]
    phase = (px * np.cos(np.pi / 4) + py * np.sin(np.pi / 4)) / 8.0
    grating = np.rint(65.0 + 40.0 * np.cos(2.0 * np.pi * phase)).astype(np.uint8)
    # fading light-grey disk
    dr = 30
    dcy = int(rng.integers(dr, H - dr))
    dcx = int(rng.integers(dr, W - dr))
    disk = _disk(H, W, dcy, dcx, dr)
    # moving yellow ellipse
    ry, rx = 25, 40
    ecy = float(rng.integers(ry, H - ry))
    ecx = float(rng.integers(rx, W - rx))
    vy, vx = 1.0, 2.0
    for t in range(n_frames):
        bg = canvas[:, pan * t:pan * t + W]
        f = np.repeat(bg[:, :, None], 3, axis=2).astype(np.float64)
        f[gy0:gy0 + gs, gx0:gx0 + gs, :] = grating[:, :, None]
        alpha = 1.0 - t / max(n_frames - 1, 1)
        f[disk] = alpha * 220.0 + (1.0 - alpha) * f[disk]
        ell = _ellipse(H, W, ecy, ecx, ry, rx)
        f[ell] = (230.0, 210.0, 40.0)
        g = ell.copy()
        g[gy0:gy0 + gs, gx0:gx0 + gs] = True
        if alpha >= 0.5:
            g |= disk
        yield np.rint(f).astype(np.uint8), g.astype(np.uint8)
        # constant-velocity motion, reflecting at the frame borders
        ecy += vy
        ecx += vx
        if ecy - ry < 0 or ecy + ry > H - 1:
            vy = -vy
            ecy += 2 * vy
        if ecx - rx < 0 or ecx + rx > W - 1:
            vx = -vx
            ecx += 2 * vx


def random_frame(H: int, W: int, seed: int) -> np.ndarray:
    """Uniform random RGB8 frame (worst-case texture)."""
    return _rng(seed).integers(0, 256, size=(H, W, 3), dtype=np.uint8)


def constant_frame(H: int, W: int, rgb=(97, 97, 97)) -> np.ndarray:
    f = np.empty((H, W, 3), np.uint8)
    f[...] = rgb
    return f


def random_grid_caps(H: int, W: int, nbr: int, seed: int, tmax: int = 1000, nmax: int = 300,
                     p_zero: float = 0.0):
    """Random int32 grid graph: source caps, sink caps and undirected n-link caps.

    ``ncap`` has ``nbr // 2`` planes ordered E, S[, SE, SW]; entries whose
    neighbour lies outside the grid are zero.
    """
    rng = _rng(seed)
    cs = rng.integers(0, tmax + 1, size=(H, W)).astype(np.int32)
    ct = rng.integers(0, tmax + 1, size=(H, W)).astype(np.int32)
    ncap = rng.integers(0, nmax + 1, size=(nbr // 2, H, W)).astype(np.int32)
    if p_zero > 0:
        ncap[rng.random(ncap.shape) < p_zero] = 0
    ncap[0, :, W - 1] = 0                       # E
    ncap[1, H - 1, :] = 0                       # S
    if nbr == 8:
        ncap[2, H - 1, :] = 0                   # SE
        ncap[2, :, W - 1] = 0
        ncap[3, H - 1, :] = 0                   # SW
        ncap[3, :, 0] = 0
    return cs, ct, ncap


def blob_grid_caps(H: int, W: int, nbr: int, seed: int, n_blobs: int = 3, scale: int = 1000,
                   ncap_val: int = 400):
    """Vision-like grid: smooth blobs prefer the source, the rest the sink.

    Produces long residual paths (object interiors far from the sink), the
    structure push-relabel finds hardest.
    """
    rng = _rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    field = np.zeros((H, W))
    for _ in range(n_blobs):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        r = rng.uniform(0.1, 0.3) * min(H, W)
        field += np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * r * r))
    field += 0.3 * rng.standard_normal((H, W))
    d = (field - 0.5) * scale
    cs = np.clip(d, 0, None).astype(np.int32)
    ct = np.clip(-d, 0, None).astype(np.int32)
    ncap = rng.integers(ncap_val // 2, ncap_val + 1, size=(nbr // 2, H, W)).astype(np.int32)
    ncap[0, :, W - 1] = 0
    ncap[1, H - 1, :] = 0
    if nbr == 8:
        ncap[2, H - 1, :] = 0
        ncap[2, :, W - 1] = 0
        ncap[3, H - 1, :] = 0
        ncap[3, :, 0] = 0
    return cs, ct, ncap
