"""Seeded synthetic segmentation workloads.

This module only builds inputs: an image I, the per-label data costs derived
from it, and the TV weight alpha.  It contains none of the solver's arithmetic,
so both the CUDA path and the FP64 CPU oracle can consume the same arrays.

The paper's own test images (Sec. 4, Tables 1-2) are not available, so these
generators stand in for them with segmentation-like shapes:

* ``binary_disk``     -- a disk on a flat background plus Gaussian noise,
                         costs C_s=|I-0.2|, C_t=|I-0.8| (the two-label model,
                         Eq. seg:chanvese).
* ``binary_shapes``   -- random disks / axis-aligned rectangles, same costs,
                         optional edge weight alpha(x)=a0*exp(-10|grad I|).
* ``potts_voronoi``   -- a Voronoi partition whose cells carry one of L grey
                         levels c_i, costs C_i=(I-c_i)^2 (the Potts model,
                         Eq. potts-model).
* ``batch_instances`` -- many instances of uneven size and label count.

All values are generated in float64 and rounded once to float32; the float32
arrays are what both sides receive (the oracle upcasts them), so both solve
exactly the same discrete problem.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    """One segmentation problem.

    ``costs`` is float32 of shape (2, H, W) for the binary model (C_s, C_t) or
    (L, H, W) for the Potts model (C_1..C_L).  ``alpha`` is either a Python
    float (constant weight) or a float32 (H, W) field.
    """

    kind: str                       # "binary" or "potts"
    image: np.ndarray               # float64 (H, W), the noisy image
    costs: np.ndarray               # float32 (2|L, H, W)
    alpha: object                   # float or float32 (H, W)
    levels: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return int(self.costs.shape[1])

    @property
    def W(self) -> int:
        return int(self.costs.shape[2])

    @property
    def L(self) -> int:
        return 2 if self.kind == "binary" else int(self.costs.shape[0])

    def alpha_field(self) -> np.ndarray:
        """alpha as a float32 (H, W) array (broadcasting a constant)."""
        if isinstance(self.alpha, np.ndarray):
            return self.alpha
        return np.full((self.H, self.W), np.float32(self.alpha), dtype=np.float32)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _edge_weight(image: np.ndarray, base: float) -> np.ndarray:
    """alpha(x) = base * exp(-10 |grad I(x)|), forward differences, zero
    difference on the far boundary.  This is input preparation (an edge
    detector on the image), not part of the solver."""
    dx = np.zeros_like(image)
    dy = np.zeros_like(image)
    dx[:, :-1] = image[:, 1:] - image[:, :-1]
    dy[:-1, :] = image[1:, :] - image[:-1, :]
    mag = np.sqrt(dx * dx + dy * dy)
    return (base * np.exp(-10.0 * mag)).astype(np.float32)


def _binary_costs(image: np.ndarray) -> np.ndarray:
    cs = np.abs(image - 0.2)
    ct = np.abs(image - 0.8)
    return np.stack([cs, ct]).astype(np.float32)


def binary_disk(H: int = 64, W: int = 64, seed: int = 1, sigma: float = 0.1,
                alpha: float = 0.5) -> Instance:
    """Disk of radius 20 (scaled by min(H,W)/64) centred in the grid, value 0.8
    on 0.2, plus N(0, sigma^2) noise."""
    rng = _rng(seed)
    radius = 20.0 * min(H, W) / 64.0
    ci, cj = (H - 1) / 2.0, (W - 1) / 2.0
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = np.where((ii - ci) ** 2 + (jj - cj) ** 2 <= radius * radius, 0.8, 0.2)
    img = img + rng.normal(0.0, sigma, size=(H, W))
    return Instance("binary", img, _binary_costs(img), float(alpha),
                    meta={"recipe": "disk", "seed": seed, "sigma": sigma})


def _paint_shapes(rng: np.random.Generator, H: int, W: int, n_shapes: int,
                  values, background: float = 0.2) -> np.ndarray:
    """Flat ``background``; each shape painted with a value drawn by
    ``values`` (a callable taking rng)."""
    scale = min(H, W) / 1024.0
    img = np.full((H, W), background)
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for _ in range(n_shapes):
        is_disk = rng.random() < 0.5
        ci = rng.uniform(0, H)
        cj = rng.uniform(0, W)
        r = rng.uniform(32.0, 160.0) * scale
        v = values(rng)
        if is_disk:
            mask = (ii - ci) ** 2 + (jj - cj) ** 2 <= r * r
        else:
            mask = (np.abs(ii - ci) <= r) & (np.abs(jj - cj) <= r)
        img[mask] = v
    return img


def binary_shapes(H: int = 1024, W: int = 1024, seed: int = 2, n_shapes: int = 8,
                  sigma: float = 0.15, alpha_base: float = 0.5,
                  edge_weighted: bool = True) -> Instance:
    """Eight random disks / axis rectangles (value 0.8 on 0.2) plus noise;
    radius or half-side uniform in [32,160] scaled by min(H,W)/1024."""
    rng = _rng(seed)
    img = _paint_shapes(rng, H, W, n_shapes, lambda r: 0.8)
    img = img + rng.normal(0.0, sigma, size=(H, W))
    alpha = _edge_weight(img, alpha_base) if edge_weighted else float(alpha_base)
    return Instance("binary", img, _binary_costs(img), alpha,
                    meta={"recipe": "shapes", "seed": seed, "sigma": sigma})


def _voronoi_labels(rng: np.random.Generator, H: int, W: int, n_seeds: int) -> np.ndarray:
    from scipy.spatial import cKDTree

    pts = np.stack([rng.uniform(0, H, n_seeds), rng.uniform(0, W, n_seeds)], axis=1)
    ii, jj = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    _, cell = cKDTree(pts).query(np.stack([ii.ravel(), jj.ravel()], axis=1))
    return cell.reshape(H, W)


def potts_voronoi(H: int = 2048, W: int = 2048, L: int = 4, n_seeds: int = 64,
                  sigma: float = 0.1, seed: int = 3, alpha_base: float = 0.3,
                  edge_weighted: bool = False, levels=None) -> Instance:
    """Voronoi partition of n_seeds uniform seeds; each cell takes one of L
    levels uniformly; plus N(0, sigma^2) noise; C_i = (I - c_i)^2."""
    rng = _rng(seed)
    if levels is None:
        if L == 4:
            levels = (0.1, 0.4, 0.6, 0.9)
        else:
            levels = tuple(i / (L - 1) for i in range(L))
    levels = tuple(float(v) for v in levels)
    assert len(levels) == L
    cell = _voronoi_labels(rng, H, W, n_seeds)
    cell_level = rng.integers(0, L, size=n_seeds)
    img = np.asarray(levels)[cell_level[cell]]
    img = img + rng.normal(0.0, sigma, size=(H, W))
    costs = np.stack([(img - c) ** 2 for c in levels]).astype(np.float32)
    alpha = _edge_weight(img, alpha_base) if edge_weighted else float(alpha_base)
    return Instance("potts", img, costs, alpha, levels=levels,
                    meta={"recipe": "voronoi", "seed": seed, "sigma": sigma,
                          "n_seeds": n_seeds})


def potts_shapes(H: int, W: int, L: int, seed: int, n_shapes: int = 8,
                 sigma: float = 0.15, alpha_base: float = 0.5) -> Instance:
    """The binary_shapes geometry painted with L levels c_i=0.1+0.8 i/(L-1):
    background level 0, each shape a uniformly drawn level 1..L-1;
    C_i=(I-c_i)^2 and an edge-weighted alpha."""
    rng = _rng(seed)
    levels = tuple(0.1 + 0.8 * i / (L - 1) for i in range(L))
    img = _paint_shapes(rng, H, W, n_shapes, lambda r: levels[int(r.integers(1, L))],
                        background=levels[0])
    img = img + rng.normal(0.0, sigma, size=(H, W))
    costs = np.stack([(img - c) ** 2 for c in levels]).astype(np.float32)
    return Instance("potts", img, costs, _edge_weight(img, alpha_base), levels=levels,
                    meta={"recipe": "shapes-potts", "seed": seed, "sigma": sigma})


def batch_instances(n: int = 256, side_lo: int = 64, side_hi: int = 1024,
                    label_choices=(2, 3, 4, 8), seed0: int = 4) -> list:
    """n instances; square side uniform in [side_lo, side_hi], L uniform in
    label_choices, instance k generated with seed seed0+k.  L=2 uses the
    binary generator, L>2 the painted-shapes Potts generator."""
    out = []
    for k in range(n):
        rng = _rng(seed0 + k)
        side = int(rng.integers(side_lo, side_hi + 1))
        L = int(label_choices[int(rng.integers(0, len(label_choices)))])
        if L == 2:
            out.append(binary_shapes(side, side, seed=seed0 + k))
        else:
            out.append(potts_shapes(side, side, L, seed=seed0 + k))
    return out


def random_binary(H: int, W: int, seed: int, alpha=0.5, field_alpha: bool = False) -> Instance:
    """Unstructured small problems for unit tests: uniform costs in [0,1]."""
    rng = _rng(seed)
    costs = rng.uniform(0.0, 1.0, size=(2, H, W)).astype(np.float32)
    a = rng.uniform(0.0, 2.0 * alpha, size=(H, W)).astype(np.float32) if field_alpha else float(alpha)
    return Instance("binary", np.zeros((H, W)), costs, a, meta={"recipe": "uniform", "seed": seed})


def random_potts(H: int, W: int, L: int, seed: int, alpha=0.3, field_alpha: bool = False) -> Instance:
    rng = _rng(seed)
    costs = rng.uniform(0.0, 1.0, size=(L, H, W)).astype(np.float32)
    a = rng.uniform(0.0, 2.0 * alpha, size=(H, W)).astype(np.float32) if field_alpha else float(alpha)
    return Instance("potts", np.zeros((H, W)), costs, a, meta={"recipe": "uniform", "seed": seed})


# Named workloads (sizes from the benchmark configurations).
def config1() -> Instance:
    """Binary 64x64 disk, alpha=0.5 (pADMMI, 200 iterations)."""
    return binary_disk(64, 64, seed=1)


def config2(H: int = 1024, W: int = 1024, seed: int = 2) -> Instance:
    """Binary 1024^2 shapes, edge-weighted alpha (run to gap 1e-4)."""
    return binary_shapes(H, W, seed=seed)


def config3(H: int = 2048, W: int = 2048) -> Instance:
    """Potts L=4 2048^2 Voronoi (64 seeds), alpha=0.3."""
    n_seeds = max(4, int(round(64 * (H * W) / (2048 * 2048)))) if H * W < 2048 * 2048 else 64
    return potts_voronoi(H, W, L=4, n_seeds=n_seeds, sigma=0.1, seed=3, alpha_base=0.3)


def config5(H: int = 4096, W: int = 4096, seed: int = 5) -> Instance:
    """Potts L=16 4096^2 Voronoi (512 seeds), 16 levels i/15, edge-weighted alpha."""
    n_seeds = max(8, int(round(512 * (H * W) / (4096 * 4096)))) if H * W < 4096 * 4096 else 512
    return potts_voronoi(H, W, L=16, n_seeds=n_seeds, sigma=0.05, seed=seed, alpha_base=0.3,
                         edge_weighted=True)
