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


def plateau_list(rng: np.random.Generator, n_images: int, N: int, image_fraction: float,
                 row_fraction: float, heights=None, kmax: int = 300):
    """A seeded list of plateaus: (image, row, c1, c2, height) arrays, one entry per selected row
    of each selected image (every selected image gets at least one row), adding ``height`` to
    columns [c1, c2) of that row.  heights: None draws heavy-tailed signed heights
    (``heavy_tail_heights``), an int gives a fixed height.  Within one list every (image, row)
    pair appears at most once, so the entries can be applied in any order."""
    imgs = np.nonzero(rng.random(n_images) < image_fraction)[0]
    rows = rng.random((imgs.size, N)) < row_fraction
    none = np.nonzero(~rows.any(axis=1))[0]
    rows[none, rng.integers(0, N, none.size)] = True
    ii, rr = np.nonzero(rows)
    img = imgs[ii].astype(np.int64)
    c1 = rng.integers(0, N - 1, img.size)
    c2 = c1 + 1 + np.floor(rng.random(img.size) * (N - c1)).astype(np.int64)
    if heights is None:
        h = heavy_tail_heights(rng, img.size, kmax)
    else:
        h = np.full(img.size, int(heights), np.int64)
    return {"image": img, "row": rr.astype(np.int64), "c1": c1, "c2": c2, "height": h}


def apply_plateaus(images: np.ndarray, plist, chunk: int = 1 << 18) -> np.ndarray:
    """Apply a ``plateau_list`` to uint16 [n, N, N] images in place (results clipped to the
    uint16 range)."""
    N = images.shape[2]
    cols = np.arange(N)[None, :]
    for s in range(0, plist["image"].size, chunk):
        sl = slice(s, s + chunk)
        i, r = plist["image"][sl], plist["row"][sl]
        add = ((cols >= plist["c1"][sl, None]) & (cols < plist["c2"][sl, None])) * \
            plist["height"][sl, None]
        images[i, r] = np.clip(images[i, r].astype(np.int64) + add, 0, 65535).astype(np.uint16)
    return images


def apply_plateaus_torch(images16, plist, chunk: int = 1 << 18):
    """``apply_plateaus`` for a torch uint16 tensor (any device), in place."""
    import torch

    dev = images16.device
    ims = images16.view(torch.int16)
    N = ims.shape[2]
    cols = torch.arange(N, device=dev)[None, :]
    for s in range(0, plist["image"].size, chunk):
        sl = slice(s, s + chunk)
        t = {k: torch.from_numpy(np.ascontiguousarray(v[sl])).to(dev) for k, v in plist.items()}
        add = ((cols >= t["c1"][:, None]) & (cols < t["c2"][:, None])).to(torch.int64) * \
            t["height"][:, None]
        cur = ims[t["image"], t["row"]].to(torch.int64) & 0xFFFF
        v = (cur + add).clamp(0, 65535)
        ims[t["image"], t["row"]] = torch.where(v > 32767, v - 65536, v).to(torch.int16)
    return images16


def precision_form_recipe(seed: int, num_images: int, num_needles: int, N: int,
                          tail_image_fraction: float = 0.02, tail_row_fraction: float = 0.03,
                          clutter_fraction: float = 0.3, clutter_row_fraction: float = 0.1,
                          clutter_height: int = 2, kmax: int = 300):
    """Everything but the base images of the precision-form set: heavy-tailed plateaus (2 % of
    the images, 3 % of their rows, P(|v| = k) ~ k^-2 up to 300), the needle indices (distinct,
    taken after the tails and before clutter) and clutter plateaus (+2 in 10 % of the rows of
    30 % of the haystack images).  The base images are RICI images of seeded scenes
    (``synth.scenes.precision_form_scenes``), computed by whichever side uses the recipe."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tails = plateau_list(rng, num_images, N, tail_image_fraction, tail_row_fraction, None, kmax)
    needles = rng.choice(num_images, size=num_needles, replace=False).astype(np.int64)
    clutter = plateau_list(rng, num_images, N, clutter_fraction, clutter_row_fraction,
                           clutter_height)
    return tails, needles, clutter
