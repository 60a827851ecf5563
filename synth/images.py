"""Seeded synthetic count images for search workloads (inputs only).

A RICI row is a step function of the circle radius: the intersection count stays constant
between radii where a circle starts or stops crossing the surface (Section 3.1).  These
generators produce uint16 images with that structure directly, so that search tests and
benchmarks can use millions of images without generating them from meshes:

* each row starts at a non-negative base count and changes at a few random columns;
* changes are small non-zero integers (|delta| <= ``small``);
* ``add_plateaus`` raises (clutter, Fig. intersectioncounts) or shifts (heavy tails) the
  count over random column ranges of random rows, which leaves deltas unchanged except at
  the two ends of each range.

No distance, rank or delta encoding is computed here.
"""
from __future__ import annotations

import numpy as np


def rici_like_images(rng: np.random.Generator, n: int, N: int, changes_per_row: float = 3.0,
                     small: int = 8, base_hi: int = 4, chunk: int = 8192) -> np.ndarray:
    out = np.empty((n, N, N), dtype=np.uint16)
    p = min(1.0, changes_per_row / max(1, N - 1))
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        steps = np.zeros((m, N, N), dtype=np.int32)
        hit = rng.random((m, N, N - 1)) < p
        mag = rng.integers(1, small + 1, size=(m, N, N - 1), dtype=np.int32)
        sign = np.where(rng.random((m, N, N - 1)) < 0.5, -1, 1).astype(np.int32)
        steps[:, :, 1:] = hit * mag * sign
        row = np.cumsum(steps, axis=2, dtype=np.int32)
        base = -row.min(axis=2, keepdims=True) + rng.integers(0, base_hi + 1, size=(m, N, 1),
                                                               dtype=np.int32)
        out[s:s + m] = np.clip(row + base, 0, 65535).astype(np.uint16)
    return out


def heavy_tail_heights(rng: np.random.Generator, size, kmax: int = 300) -> np.ndarray:
    """Signed integers with P(|v| = k) proportional to k^-2 for k in 1..kmax."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    p = k ** -2.0
    p /= p.sum()
    mag = rng.choice(np.arange(1, kmax + 1), size=size, p=p)
    sign = np.where(rng.random(size) < 0.5, -1, 1)
    return (mag * sign).astype(np.int64)


def add_plateaus(rng: np.random.Generator, images: np.ndarray, image_fraction: float,
                 row_fraction: float, heights=None, positive_only: bool = False,
                 kmax: int = 300) -> np.ndarray:
    """Add a constant over a random column range [c1, c2) of selected rows (in place).

    heights: None draws heavy-tailed heights (``heavy_tail_heights``); an int gives a fixed
    height.  Results are clipped to the uint16 range.
    """
    n, N, _ = images.shape
    sel = np.nonzero(rng.random(n) < image_fraction)[0]
    for i in sel:
        rows = np.nonzero(rng.random(N) < row_fraction)[0]
        if rows.size == 0:
            rows = np.array([int(rng.integers(0, N))])
        for r in rows:
            c1 = int(rng.integers(0, N - 1))
            c2 = int(rng.integers(c1 + 1, N + 1))
            if heights is None:
                v = int(heavy_tail_heights(rng, 1, kmax)[0])
                if positive_only:
                    v = abs(v)
            else:
                v = int(heights)
            seg = images[i, r, c1:c2].astype(np.int64) + v
            images[i, r, c1:c2] = np.clip(seg, 0, 65535).astype(np.uint16)
    return images


def needle_haystack_set(rng: np.random.Generator, num_needles: int, num_haystack: int, N: int,
                        clutter_fraction: float = 0.3, tail_image_fraction: float = 0.02,
                        tail_row_fraction: float = 0.03, kmax: int = 300):
    """Haystack pool with heavy tails; needles are copies taken before clutter is added.

    Returns (needles uint16 [Q,N,N], haystack uint16 [H,N,N], true_match int64 [Q]).
    """
    hay = rici_like_images(rng, num_haystack, N)
    add_plateaus(rng, hay, tail_image_fraction, tail_row_fraction, kmax=kmax)
    match = rng.choice(num_haystack, size=num_needles, replace=False).astype(np.int64)
    needles = hay[match].copy()
    add_plateaus(rng, hay, clutter_fraction, 0.1, heights=2)
    return needles, hay, match


def needle_haystack_set_torch(seed: int, num_needles: int, num_haystack: int, N: int, device,
                              clutter_fraction: float = 0.3, tail_image_fraction: float = 0.02,
                              tail_row_fraction: float = 0.03, kmax: int = 300,
                              changes_per_row: float = 3.0, small: int = 8, chunk: int = 65536):
    """The recipe of ``needle_haystack_set`` drawn with a seeded torch generator on ``device``.

    Used for image sets of a million images and more (drawing them with numpy on the host would
    take minutes).  Returns (needles, haystack, true_match) as torch tensors on ``device``
    (uint16 [Q,N,N], uint16 [H,N,N], int64 [Q]).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    p = min(1.0, changes_per_row / max(1, N - 1))
    # uint16 storage handled through an int16 view (indexing ops lack uint16 kernels)
    hay16 = torch.empty((num_haystack, N, N), dtype=torch.int16, device=device)
    k = torch.arange(1, kmax + 1, dtype=torch.float64, device=device)
    tail_p = (k ** -2.0) / (k ** -2.0).sum()

    def to16(v):  # int values in [0, 65535] -> int16 bit pattern
        return torch.where(v > 32767, v - 65536, v).to(torch.int16)

    def plateaus(ims, image_fraction, row_fraction, height):
        n = ims.shape[0]
        pick = torch.rand((n, 1), generator=g, device=device) < image_fraction
        rows = (torch.rand((n, N), generator=g, device=device) < row_fraction) & pick
        idx = rows.nonzero()
        if idx.numel() == 0:
            return
        c1 = torch.randint(0, N - 1, (idx.shape[0],), generator=g, device=device)
        span = torch.rand((idx.shape[0],), generator=g, device=device)
        c2 = c1 + 1 + (span * (N - 1 - c1).to(torch.float32)).floor().to(torch.int64)
        if height is None:
            mag = torch.multinomial(tail_p, idx.shape[0], replacement=True, generator=g) + 1
            sign = torch.where(torch.rand((idx.shape[0],), generator=g, device=device) < 0.5, -1, 1)
            h = mag * sign
        else:
            h = torch.full((idx.shape[0],), int(height), dtype=torch.int64, device=device)
        cols = torch.arange(N, device=device)[None, :]
        add = ((cols >= c1[:, None]) & (cols < c2[:, None])).to(torch.int64) * h[:, None]
        cur = ims[idx[:, 0], idx[:, 1]].to(torch.int64) & 0xFFFF
        ims[idx[:, 0], idx[:, 1]] = to16((cur + add).clamp(0, 65535))

    for s in range(0, num_haystack, chunk):
        m = min(chunk, num_haystack - s)
        hit = torch.rand((m, N, N - 1), generator=g, device=device) < p
        mag = torch.randint(1, small + 1, (m, N, N - 1), generator=g, device=device, dtype=torch.int32)
        sign = torch.where(torch.rand((m, N, N - 1), generator=g, device=device) < 0.5, -1, 1)
        steps = torch.zeros((m, N, N), dtype=torch.int32, device=device)
        steps[:, :, 1:] = hit.to(torch.int32) * mag * sign.to(torch.int32)
        row = torch.cumsum(steps, dim=2, dtype=torch.int32)
        base = -row.min(dim=2, keepdim=True).values + torch.randint(
            0, 5, (m, N, 1), generator=g, device=device, dtype=torch.int32)
        hay16[s:s + m] = to16((row + base).clamp(0, 65535))
        plateaus(hay16[s:s + m], tail_image_fraction, tail_row_fraction, None)
    match = torch.randperm(num_haystack, generator=g, device=device)[:num_needles].to(torch.int64)
    needles16 = hay16[match].clone()
    for s in range(0, num_haystack, chunk):
        plateaus(hay16[s:s + min(chunk, num_haystack - s)], clutter_fraction, 0.1, 2)
    return needles16.view(torch.uint16), hay16.view(torch.uint16), match
