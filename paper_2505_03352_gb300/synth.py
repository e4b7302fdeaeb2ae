"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  This module holds no step of the permittivity chain: it only
draws control arrays and complex field arrays with the shapes and value
distributions of the five workloads below (all host-side numpy, float32 /
complex64, reproducible from the seeds).

Workloads (controls at 10 nm pitch, 2 x 2 subpixels per 20 nm Yee cell,
eps_Si = 12.11, eps_SiO2 = 2.085, an 11-cell (220 nm) slab, eta = 0.5):

  cfg1  64 x 64 controls ~ U[0, 1); R = 3, beta = 8; Yee 32 x 32 x 16; one
        wavelength.
  cfg2  600 x 600 SOI-like layout (Gaussian-smoothed noise, sigma = 4 px,
        thresholded at its median, plus U(-0.1, 0.1) noise, clipped to
        [0, 1]); R = 6, beta = 16; Yee 300 x 300 x 24; one wavelength.
  cfg3  2000 x 2000, same layout generator; R = 6, beta = 16;
        Yee 1000 x 1000 x 32; three wavelengths (1500 / 1550 / 1600 nm).
  cfg4  64 regions, square sides drawn log-uniformly in [64, 1024]
        controls (rounded to even), R uniform in {2..8}, beta uniform in
        {4, 8, 16, 32}, Yee z = 24; one wavelength per region.
  cfg5  3000 x 3000, same layout generator; R = 6, beta = 16;
        Yee 1500 x 1500 x 32; eight wavelengths spanning 1500-1600 nm.

Seeds: C uses 1000 + cfg; E_F of wavelength l uses 2000 + 10 cfg + l and
E_A uses 3000 + 10 cfg + l.  Fields have N(0, 1) real and imaginary parts.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EPS_SI = 12.11
EPS_SIO2 = 2.085
SLAB_NK = 11


@dataclass
class Workload:
    name: str
    mx: int
    my: int
    nz: int
    radius: float
    beta: float
    n_lambda: int
    eta: float = 0.5
    eps_core: float = EPS_SI
    eps_clad: float = EPS_SIO2
    slab_nk: int = SLAB_NK
    sub: int = 2
    bc: int = 0
    cfg: int = 0
    layout: str = "soi"           # "uniform" or "soi"
    extra: dict = field(default_factory=dict)

    @property
    def nx(self):
        return self.mx // self.sub

    @property
    def ny(self):
        return self.my // self.sub

    @property
    def voxels(self):
        return self.nx * self.ny * self.nz


WORKLOADS = {
    1: Workload("cfg1_64x64_R3_b8_nz16", 64, 64, 16, 3.0, 8.0, 1, cfg=1, layout="uniform"),
    2: Workload("cfg2_600x600_R6_b16_nz24", 600, 600, 24, 6.0, 16.0, 1, cfg=2),
    3: Workload("cfg3_2000x2000_R6_b16_nz32_w3", 2000, 2000, 32, 6.0, 16.0, 3, cfg=3),
    5: Workload("cfg5_3000x3000_R6_b16_nz32_w8", 3000, 3000, 32, 6.0, 16.0, 8, cfg=5),
}


def _gauss_kernel(sigma: float):
    r = int(np.ceil(4 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum(), r


def _blur_axis(a, k, r, axis):
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad, mode="reflect")
    out = np.zeros_like(a)
    n = a.shape[axis]
    for t, kt in enumerate(k):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(t, t + n)
        out += kt * ap[tuple(sl)]
    return out


def soi_layout(mx: int, my: int, seed: int, sigma: float = 4.0, noise: float = 0.1):
    """Binary blob layout with small noise: clip(1[G_sigma * U > median] +
    U(-noise, noise), 0, 1), float32."""
    rng = np.random.default_rng(seed)
    base = rng.random((mx, my))
    k, r = _gauss_kernel(sigma)
    sm = _blur_axis(_blur_axis(base, k, r, 0), k, r, 1)
    binary = (sm > np.median(sm)).astype(np.float64)
    c = binary + rng.uniform(-noise, noise, size=(mx, my))
    return np.clip(c, 0.0, 1.0).astype(np.float32)


def uniform_controls(mx: int, my: int, seed: int):
    return np.random.default_rng(seed).random((mx, my), dtype=np.float32)


def controls(w: Workload, seed: int | None = None):
    seed = 1000 + w.cfg if seed is None else seed
    if w.layout == "uniform":
        return uniform_controls(w.mx, w.my, seed)
    return soi_layout(w.mx, w.my, seed)


def complex_field(shape, seed: int):
    """complex64 array of `shape` with N(0, 1) real and imaginary parts
    (interleaved re, im in memory)."""
    rng = np.random.default_rng(seed)
    ri = rng.standard_normal(tuple(shape) + (2,), dtype=np.float32)
    return ri.view(np.complex64)[..., 0]


def field_shape(w: Workload):
    return (3, w.nx, w.ny, w.nz)


def fields(w: Workload, n_lambda: int | None = None):
    """Lists (E_F, E_A) of complex64 [3, nx, ny, nz] arrays, one per
    wavelength."""
    n = w.n_lambda if n_lambda is None else n_lambda
    EF = [complex_field(field_shape(w), 2000 + 10 * w.cfg + l) for l in range(n)]
    EA = [complex_field(field_shape(w), 3000 + 10 * w.cfg + l) for l in range(n)]
    return EF, EA


def batched_regions(n: int = 64, seed: int = 1004, lo: int = 64, hi: int = 1024,
                    nz: int = 24):
    """The cfg4 region table: list of Workload, one per region."""
    rng = np.random.default_rng(seed)
    regs = []
    for r in range(n):
        side = int(2 * round(np.exp(rng.uniform(np.log(lo), np.log(hi))) / 2))
        side = max(side, 4)
        radius = float(rng.integers(2, 9))
        beta = float(rng.choice([4.0, 8.0, 16.0, 32.0]))
        regs.append(Workload(f"cfg4_region{r}", side, side, nz, radius, beta, 1,
                             cfg=4, extra={"region": r}))
    return regs


def region_inputs(w: Workload, region: int):
    """C, E_F, E_A for one cfg4 region (seeds offset by the region index)."""
    C = soi_layout(w.mx, w.my, 1004 * 1000 + region)
    EF = [complex_field(field_shape(w), 2040 * 1000 + region)]
    EA = [complex_field(field_shape(w), 3040 * 1000 + region)]
    return C, EF, EA
