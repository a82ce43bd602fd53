"""Seeded synthetic dirty-snapshot stacks (inputs only).

This module makes the inputs that both the CUDA path and the FP64 oracle are
fed.  It holds none of the detection arithmetic (no differences, ratios, tile
statistics, transforms or thresholds): it only synthesises images.

The paper evaluates on OSKAR/WSClean simulations and on a MeerKAT measurement
set (Sec. 3, "Real Dataset Evaluation" and "Parameters and Experimental
Settings"); neither is available, so the stacks are built from the same
ingredients in sigma units:

* a dirty beam (PSF) from a seeded antenna layout: every baseline (both signs)
  is gridded to its nearest uv cell, multiplied by a Gaussian uv taper whose
  image-domain main lobe has a FWHM of ``fwhm_px`` pixels (2 px = critical
  Nyquist sampling), inverse transformed and normalised to a peak of 1;
* i.i.d. N(0, 1) noise per snapshot, convolved with the PSF and rescaled to unit
  standard deviation (a circular convolution of unit white noise with the PSF
  has standard deviation ||PSF||_2, so the white noise is divided by it);
* steady point sources (PSF at integer pixels, amplitude = peak in sigma);
* pulsed point sources that are on for one snapshot per period, as the
  on/off pulsars of Sec. 3 (a ULP pulsar is visible in one snapshot of a
  three-snapshot unit).

Random numbers for positions and amplitudes come from NumPy's PCG64 so they do
not depend on the device; noise comes from a torch generator on the device that
synthesises the stack.  Everything is deterministic for a given (seed, device).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


@dataclasses.dataclass
class StackSpec:
    """Shape and content of one synthetic field."""

    nsnap: int
    ny: int
    nx: int
    layout: str = "uniform_disc"        # uniform_disc | meerkat_like | ska_aa2_like
    n_ant: int = 32
    fwhm_px: float = 2.0
    n_steady: int = 20
    steady_lo: float = 5.0
    steady_hi: float = 100.0
    steady_dist: str = "uniform"        # uniform | loguniform
    n_pulsed: int = 1
    pulse_amp: Optional[float] = 8.0    # fixed amplitude, or None: companion/ratio
    pulse_period: Tuple[int, int] = (4, 4)   # inclusive range of periods
    companion_min: float = 160.0        # companion steady source floor (sigma)
    companion_ratio: float = 20.0       # companion / pulsar flux
    companion_dist_px: Tuple[float, float] = (2.0, 6.0)
    edge_margin: int = 4


# The five workload shapes the trigger is measured on (sizes in pixels).
C1 = StackSpec(nsnap=16, ny=512, nx=512, layout="uniform_disc", n_ant=32,
               n_steady=20, steady_lo=5, steady_hi=100, steady_dist="uniform",
               n_pulsed=1, pulse_amp=8.0, pulse_period=(4, 4))
C2 = StackSpec(nsnap=64, ny=4096, nx=4096, layout="meerkat_like", n_ant=64,
               n_steady=500, steady_lo=5, steady_hi=500, steady_dist="loguniform",
               n_pulsed=10, pulse_amp=None, pulse_period=(3, 16))


C3 = StackSpec(nsnap=8, ny=50000, nx=50000, layout="meerkat_like", n_ant=64,
               n_steady=10000, steady_lo=5, steady_hi=500, steady_dist="loguniform",
               n_pulsed=50, pulse_amp=None, pulse_period=(3, 16))


def batched_fields(seed: int = 11, nfields: int = 256) -> List[Tuple[int, int]]:
    """(nsnap, side) of the batched workload: square fields of side U{1024..8192}
    with U{16..128} snapshots each (SKA-AA2-like PSF, see :func:`batched_spec`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = rng.integers(1024, 8193, nfields)
    nsnaps = rng.integers(16, 129, nfields)
    return [(int(L), int(s)) for L, s in zip(nsnaps, sides)]


def batched_spec(nsnap: int, side: int) -> StackSpec:
    return small_spec(nsnap, side, side, layout="ska_aa2_like", n_ant=68)


def serving_sides(seed: int = 7, nfields: int = 32) -> List[int]:
    """Square field sides of the serving workload, U{2048..16384}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(v) for v in rng.integers(2048, 16385, nfields)]


def small_spec(nsnap: int, ny: int, nx: int, **kw) -> StackSpec:
    """A C2-like field of arbitrary size with source counts scaled by area."""
    area = ny * nx / float(4096 * 4096)
    base = dict(layout="meerkat_like", n_ant=64, steady_lo=5, steady_hi=500,
                steady_dist="loguniform", pulse_amp=None, pulse_period=(3, 16),
                n_steady=max(4, int(round(500 * area))),
                n_pulsed=max(1, int(round(10 * area))))
    base.update(kw)
    return StackSpec(nsnap=nsnap, ny=ny, nx=nx, **base)


def antenna_layout(kind: str, n: int, seed: int) -> np.ndarray:
    """Seeded antenna (station) positions, arbitrary length units, shape (n, 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "uniform_disc":
        r = np.sqrt(rng.uniform(0.0, 1.0, n))
        th = rng.uniform(0.0, 2 * np.pi, n)
    elif kind == "meerkat_like":
        n_core = int(round(0.7 * n))
        r_core = np.sqrt(rng.uniform(0.0, 1.0, n_core))          # 1 km core
        r_out = np.exp(rng.uniform(0.0, np.log(8.0), n - n_core))  # out to 8 km
        r = np.concatenate([r_core, r_out])
        th = rng.uniform(0.0, 2 * np.pi, n)
    elif kind == "ska_aa2_like":
        n_core = n - 3 * (n // 4)
        r_core = 0.5 * np.sqrt(rng.uniform(0.0, 1.0, n_core))
        th_core = rng.uniform(0.0, 2 * np.pi, n_core)
        per_arm = (n - n_core) // 3
        rs, ths = [r_core], [th_core]
        for arm in range(3):
            ra = np.exp(np.linspace(np.log(0.7), np.log(10.0), per_arm))
            ra = ra * rng.uniform(0.95, 1.05, per_arm)
            ta = arm * 2 * np.pi / 3 + 1.2 * np.log(ra) + rng.normal(0, 0.03, per_arm)
            rs.append(ra)
            ths.append(ta)
        r = np.concatenate(rs)
        th = np.concatenate(ths)
        n = r.size
    else:
        raise ValueError(f"unknown layout {kind!r}")
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def dirty_beam(kind: str, n_ant: int, ny: int, nx: int, seed: int,
               fwhm_px: float = 2.0, umax: float = 0.45) -> np.ndarray:
    """PSF on an origin-centred (circular) ny x nx grid, peak normalised to 1.

    Every ordered antenna pair gives a baseline; the longest is scaled to
    ``umax`` cycles/pixel and each is gridded to its nearest uv cell.
    """
    pos = antenna_layout(kind, n_ant, seed)
    b = (pos[:, None, :] - pos[None, :, :]).reshape(-1, 2)
    b = b[np.any(b != 0.0, axis=1)]
    b = b * (umax / np.max(np.hypot(b[:, 0], b[:, 1])))
    iu = np.rint(b[:, 0] * nx).astype(np.int64) % nx
    iv = np.rint(b[:, 1] * ny).astype(np.int64) % ny
    grid = np.zeros((ny, nx), dtype=np.float64)
    np.add.at(grid, (iv, iu), 1.0)
    fu = np.fft.fftfreq(nx)[None, :]
    fv = np.fft.fftfreq(ny)[:, None]
    sig_x = fwhm_px * FWHM_TO_SIGMA
    sig_u = 1.0 / (2 * np.pi * sig_x)
    grid *= np.exp(-(fu ** 2 + fv ** 2) / (2 * sig_u ** 2))
    psf = np.real(np.fft.ifft2(grid))
    return psf / psf[0, 0]


@dataclasses.dataclass
class Truth:
    steady: List[Tuple[int, int, float]]            # (x, y, amplitude)
    pulsed: List[Tuple[int, int, float, int, int]]  # (x, y, amplitude, period, phase)

    def pulse_on(self, k: int) -> List[Tuple[int, int, float]]:
        return [(x, y, a) for (x, y, a, p, ph) in self.pulsed if k % p == ph]


def draw_sources(spec: StackSpec, seed: int) -> Truth:
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    m = spec.edge_margin
    xs = rng.integers(m, spec.nx - m, spec.n_steady)
    ys = rng.integers(m, spec.ny - m, spec.n_steady)
    if spec.steady_dist == "loguniform":
        amps = np.exp(rng.uniform(np.log(spec.steady_lo), np.log(spec.steady_hi), spec.n_steady))
    else:
        amps = rng.uniform(spec.steady_lo, spec.steady_hi, spec.n_steady)
    steady = [(int(x), int(y), float(a)) for x, y, a in zip(xs, ys, amps)]
    pulsed = []
    bright = [s for s in steady if s[2] >= spec.companion_min]
    for _ in range(spec.n_pulsed):
        p = int(rng.integers(spec.pulse_period[0], spec.pulse_period[1] + 1))
        ph = int(rng.integers(0, p))
        if spec.pulse_amp is None and bright:
            cx, cy, ca = bright[int(rng.integers(0, len(bright)))]
            d = rng.uniform(*spec.companion_dist_px)
            th = rng.uniform(0, 2 * np.pi)
            x = int(np.clip(np.rint(cx + d * np.cos(th)), m, spec.nx - m - 1))
            y = int(np.clip(np.rint(cy + d * np.sin(th)), m, spec.ny - m - 1))
            amp = ca / spec.companion_ratio
        else:
            x = int(rng.integers(m, spec.nx - m))
            y = int(rng.integers(m, spec.ny - m))
            amp = float(spec.pulse_amp if spec.pulse_amp is not None else 8.0)
        pulsed.append((x, y, float(amp), p, ph))
    return Truth(steady=steady, pulsed=pulsed)


def beam_transfer(kind: str, n_ant: int, ny: int, nx: int, seed: int, fwhm_px: float = 2.0,
                  umax: float = 0.45, device: str = "cpu") -> Tuple[torch.Tensor, float]:
    """The dirty beam's transfer function on the rfft half-plane and ||psf||_2.

    The tapered uv grid G is real and symmetric (both signs of every baseline),
    so the beam psf = ifft2(G) / psf[0,0] has rfft2(psf) = G / psf[0,0] with
    psf[0,0] = sum(G) / (nx ny); no transform of the beam is needed, which
    keeps very large fields cheap.  Same beam as :func:`dirty_beam`.
    """
    pos = antenna_layout(kind, n_ant, seed)
    b = (pos[:, None, :] - pos[None, :, :]).reshape(-1, 2)
    b = b[np.any(b != 0.0, axis=1)]
    b = b * (umax / np.max(np.hypot(b[:, 0], b[:, 1])))
    iu = np.rint(b[:, 0] * nx).astype(np.int64) % nx
    iv = np.rint(b[:, 1] * ny).astype(np.int64) % ny
    half = nx // 2 + 1
    keep = iu < half
    dev = torch.device(device)
    grid = torch.zeros(ny, half, dtype=torch.float64, device=dev)
    idx_v = torch.from_numpy(iv[keep]).to(dev)
    idx_u = torch.from_numpy(iu[keep]).to(dev)
    grid.index_put_((idx_v, idx_u), torch.ones(idx_v.numel(), dtype=torch.float64, device=dev),
                    accumulate=True)
    sig_u = 1.0 / (2 * np.pi * fwhm_px * FWHM_TO_SIGMA)
    fu = torch.arange(half, dtype=torch.float64, device=dev) / nx
    fv = torch.fft.fftfreq(ny, dtype=torch.float64, device=dev)
    grid *= torch.exp(-(fv[:, None] ** 2) / (2 * sig_u ** 2))
    grid *= torch.exp(-(fu[None, :] ** 2) / (2 * sig_u ** 2))
    # weights of the half-plane columns in full-plane sums (Hermitian symmetry)
    wcol = torch.full((half,), 2.0, dtype=torch.float64, device=dev)
    wcol[0] = 1.0
    if nx % 2 == 0:
        wcol[-1] = 1.0
    n = float(nx) * float(ny)
    peak = float((grid * wcol).sum()) / n
    H = grid / peak
    norm = float(np.sqrt(float((H * H * wcol).sum()) / n))   # Parseval
    return H.to(torch.float32), norm


def iter_stack(spec: StackSpec, seed: int, device: str = "cpu"):
    """Yield (k, snapshot) one FP32 snapshot at a time (same values as
    make_stack), so that very large stacks never exist twice in memory."""
    H, norm = beam_transfer(spec.layout, spec.n_ant, spec.ny, spec.nx, seed, spec.fwhm_px,
                            device=device)
    truth = draw_sources(spec, seed)
    dev = torch.device(device)
    steady = torch.zeros(spec.ny, spec.nx, dtype=torch.float32, device=dev)
    if truth.steady:
        sx, sy, sa = (torch.tensor(c, device=dev) for c in zip(*truth.steady))
        steady.index_put_((sy.long(), sx.long()), sa.float(), accumulate=True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 7919 + 17)
    for k in range(spec.nsnap):
        img = torch.randn(spec.ny, spec.nx, generator=gen, device=dev, dtype=torch.float32)
        img.mul_(1.0 / norm).add_(steady)
        for x, y, a in truth.pulse_on(k):
            img[y, x] += a
        spec_k = torch.fft.rfft2(img)
        del img
        spec_k *= H
        snap = torch.fft.irfft2(spec_k, s=(spec.ny, spec.nx))
        del spec_k
        yield k, snap


def make_stack(spec: StackSpec, seed: int, device: str = "cpu",
               dtype: torch.dtype = torch.float32) -> Tuple[torch.Tensor, Truth]:
    """Synthesize an (nsnap, ny, nx) stack on ``device``.

    Each snapshot is ``(white/||psf||_2 + sources) (*) psf`` (circular
    convolution by FFT), so the noise has unit standard deviation and a source
    of amplitude A peaks at A.
    """
    H, norm = beam_transfer(spec.layout, spec.n_ant, spec.ny, spec.nx, seed, spec.fwhm_px,
                            device=device)
    truth = draw_sources(spec, seed)
    dev = torch.device(device)
    steady = torch.zeros(spec.ny, spec.nx, dtype=torch.float32, device=dev)
    if truth.steady:
        sx, sy, sa = (torch.tensor(c, device=dev) for c in zip(*truth.steady))
        steady.index_put_((sy.long(), sx.long()), sa.float(), accumulate=True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) * 7919 + 17)
    out = torch.empty(spec.nsnap, spec.ny, spec.nx, dtype=dtype, device=dev)
    for k in range(spec.nsnap):
        img = torch.randn(spec.ny, spec.nx, generator=gen, device=dev, dtype=torch.float32)
        img.mul_(1.0 / norm).add_(steady)
        for x, y, a in truth.pulse_on(k):
            img[y, x] += a
        spec_k = torch.fft.rfft2(img)
        del img
        spec_k *= H
        out[k].copy_(torch.fft.irfft2(spec_k, s=(spec.ny, spec.nx)))
        del spec_k
    return out, truth


def gaussian_noise_stack(nsnap: int, ny: int, nx: int, seed: int,
                         device: str = "cpu") -> torch.Tensor:
    """Plain N(0,1) images, the paper's timing input (Sec. 3.2)."""
    gen = torch.Generator(device=torch.device(device))
    gen.manual_seed(int(seed))
    return torch.randn(nsnap, ny, nx, generator=gen, device=device, dtype=torch.float32)


def periodic_tile_stack(nsnap: int, ny: int, nx: int, w: int, period: int, phase: int,
                        tile: Tuple[int, int], amp: float, seed: int,
                        noise: float = 1.0) -> np.ndarray:
    """White noise plus a pulse filling one tile in snapshots k = phase (mod period).

    Used to exercise period recovery of the frequency branch.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    x = noise * rng.standard_normal((nsnap, ny, nx))
    ty, tx = tile
    for k in range(nsnap):
        if k % period == phase:
            x[k, ty * w:(ty + 1) * w, tx * w:(tx + 1) * w] += amp
    return x.astype(np.float32)


def random_stack(nsnap: int, ny: int, nx: int, seed: int, kind: str = "normal") -> np.ndarray:
    """Small adversarial stacks: normal, integer-valued (ties), or with zeros."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "normal":
        x = rng.standard_normal((nsnap, ny, nx))
    elif kind == "integers":
        x = rng.integers(-3, 4, (nsnap, ny, nx)).astype(np.float64)
    elif kind == "zeros":
        x = rng.standard_normal((nsnap, ny, nx))
        x[rng.uniform(size=x.shape) < 0.2] = 0.0
    elif kind == "positive":
        x = np.abs(rng.standard_normal((nsnap, ny, nx))) + 0.01
    else:
        raise ValueError(kind)
    return x.astype(np.float32)
