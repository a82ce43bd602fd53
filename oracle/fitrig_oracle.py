"""FP64 CPU oracle for the FITrig trigger path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA library and imports nothing from it.

Every step is written straight from the paper's definitions, in float64, by
whole-array NumPy operations and plain loops; there is no fusion, blocking or
reordering beyond what the definitions state.

Paper sections used (arXiv 2509.21754, "FITrig"):

* Sec. 2.2.4 (Mathematics): Eq. (tLISI), the difference image D (Eq. 3), the
  ratio r (Eq. 4) and the guarded reference intensity x-hat (Eq. 5), C = 1e-6.
* Sec. 2.3 (GPU-accelerated tLISI): Eq. (tLISI kernel form) -- the mean is a
  sum over the tile divided by its pixel count; M is one scalar for the stack.
* Sec. 2.4.1 (image-domain detection): Eq. (z-score) and the selected set
  {t | z_t > tau}.
* Sec. 2.4.2 (image-frequency detection): the tLISI cube, Eq. (eta) with h =
  maximum spectral magnitude (the paper's own conservative choice in Sec. 3.4.3),
  the z-score of eta and the selected set.  h may instead be an incoherent
  harmonic sum (Sec. 2.4.2 names harmonic summing as a choice of h and the real-data evaluation of Sec. 3
  applies it to the real data, without defining it; see ``harmonic_sum``).

Readings where the paper is silent or ambiguous (each is an option here):

* rmode "abs": x-hat = |x^(s+1)| (C if zero) so that r lies in [0, 1] as the
  paper requires of tLISI; "signed" keeps the literal Eq. 4/5.
* edge "partial": ceil(n/w) tiles, edge tiles averaged over their own pixel
  count; "drop": the image is cropped to whole tiles first.
* M is the maximum over every finite pixel of every analysed snapshot, floored
  at C (mmode "global"); the real-time reading (mmode "running") takes unit
  s's maximum over snapshots 0..s+2 only.  Non-finite pixels invalidate the
  tiles they touch.
* standard deviation is the population one; the robust scale is
  1.482602218505602 x MAD with lower medians (index floor((n-1)/2)).
* tiles are merged into 8-connected components per unit; one candidate per
  component at its maximum-z tile (ties: smallest row-major tile index); the
  image-branch pixel is the tile's arg-max of Delta (ties: smallest row-major
  pixel), the frequency-branch pixel is the tile centre, refined by a parabola
  through the eta values of the neighbouring tiles.
* the transform is the unnormalised DFT of exact length n = L - 2, bins
  k = 1..floor(n/2).
* harmonic summing (parity with the paper unpinned: the paper gives no
  formula): the classic incoherent sum of the magnitudes at the first m
  harmonics of a fundamental bin k, scaled by 1/sqrt(m), maximised over
  m = 1, 2, 4, .., m_max and over the k with m k <= floor(n/2); m_max = 1 is
  the maximum magnitude.  The bin reported is the fundamental k.  Ties go to
  the smaller m, then the smaller k.
* the spline interpolation of eta (Sec. 2.4.2 and the real-data evaluation of Sec. 3; parity with the paper
  unpinned, no formula given): per axis, the Catmull-Rom cubic through the
  peak tile's eta and two neighbours on each side, maximised within half a
  tile (``cubic_offset``); the default refine is the three-point parabola.
* a sliding-window mode (not in the paper, whose tiles partition the image)
  evaluates the tile statistic over the odd w x w window centred on each pixel,
  clipped at the border, and then treats pixels as 1 x 1 tiles.
* snapshot accumulation (Sec. 3.3.2): the paper sums adjacent snapshots
  "progressively until there is enough difference" without a criterion; the
  reading here sums fixed, non-overlapping blocks of K consecutive snapshots.
* difference-coded half storage (not in the paper; the precision form of the
  trigger): snapshot 0 is kept in FP32 and every later snapshot as the
  BF16/FP16-rounded difference from the previous *decoded* snapshot, so that
  the steady sky, which cancels in Eq. 3, is not rounded to 8 or 11
  significant bits.  ``delta_encode`` and ``delta_decode`` define the stored
  form; the trigger then runs on the decoded FP32 stack.

All pins of this module live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

C = 1e-6                       # Eq. 5 guard constant
MAD_TO_SIGMA = 1.482602218505602   # 1 / Phi^-1(3/4)

BRANCH_IMAGE = 1
BRANCH_FREQ = 2
BRANCH_BOTH = 3


# --------------------------------------------------------------------------
# Snapshot accumulation (Sec. 3.3.2, Fig. "Snapshots accumulation")
# --------------------------------------------------------------------------
def accumulate(raw: np.ndarray, k: int) -> np.ndarray:
    """Stack of sums of K consecutive raw snapshots: snapshot j of the result
    is the sum of raw snapshots jK .. jK+K-1 (an incomplete last block is
    dropped).  K = 1 returns the raw stack."""
    raw = np.asarray(raw, dtype=np.float64)
    if k < 1:
        raise ValueError("k must be >= 1")
    n = raw.shape[0] // k
    out = np.zeros((n,) + raw.shape[1:], dtype=np.float64)
    for j in range(n):
        for i in range(k):
            out[j] += raw[j * k + i]
    return out


# --------------------------------------------------------------------------
# Half-precision storage: rounding and difference coding
# --------------------------------------------------------------------------
def round_half(x: np.ndarray, fmt: str) -> np.ndarray:
    """FP32 values rounded to the nearest BF16 ("bf16") or IEEE binary16
    ("f16") number, ties to even, returned as FP32.  BF16 keeps the upper 16
    bits of the FP32 pattern: adding 0x7FFF plus the lowest kept bit and
    truncating rounds to nearest with ties to the even pattern (an overflow
    carries into the infinity pattern); NaN stays NaN."""
    x = np.asarray(x, dtype=np.float32)
    if fmt == "f16":
        with np.errstate(over="ignore"):
            return x.astype(np.float16).astype(np.float32)
    if fmt != "bf16":
        raise ValueError(fmt)
    bits = x.view(np.uint32).astype(np.uint64)
    kept = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    out = (kept & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(x), np.float32(np.nan), out)


def delta_encode(stack: np.ndarray, fmt: str) -> Tuple[np.ndarray, np.ndarray]:
    """Difference coding of a (L, ny, nx) FP32 stack, closed loop.

    key = x^(0) in FP32.  The coder keeps the decoded previous snapshot xt
    (FP32, starting at key); for s >= 1 it stores
        q^(s)  = round_half(fl32(x^(s) - xt), fmt)
        xt     = fl32(xt + q^(s))
    so each decoded snapshot carries the rounding of one difference only, which
    does not accumulate.  A non-finite input (or a difference that overflows
    the half format) makes q non-finite, and then xt and every later decoded
    value of that pixel are NaN or infinite: a difference stream has nothing
    to restart from without a new key frame.  Returns (key, q) with q[0] = 0
    and q holding half values as FP32."""
    x = np.asarray(stack, dtype=np.float32)
    key = x[0].copy()
    q = np.zeros_like(x)
    xt = key.copy()
    with np.errstate(invalid="ignore", over="ignore"):
        for s in range(1, x.shape[0]):
            q[s] = round_half(x[s] - xt, fmt)          # FP32 difference, then rounded
            xt = xt + q[s]                             # FP32 sum (numpy float32)
    return key, q


def delta_decode(key: np.ndarray, q: np.ndarray) -> np.ndarray:
    """The decoded FP32 stack of a difference-coded one: snapshot 0 is the key,
    snapshot s the FP32 sum of snapshot s-1 and q^(s), in order."""
    key = np.asarray(key, dtype=np.float32)
    q = np.asarray(q, dtype=np.float32)
    out = np.empty(q.shape, dtype=np.float32)
    out[0] = key
    with np.errstate(invalid="ignore", over="ignore"):
        for s in range(1, q.shape[0]):
            out[s] = out[s - 1] + q[s]
    return out


# --------------------------------------------------------------------------
# Tiling (Sec. 2.1: non-overlapping tiles, same shape across time)
# --------------------------------------------------------------------------
def tiling(ny: int, nx: int, w: int, edge: str = "partial") -> Tuple[int, int, int, int]:
    """Return (Ty, Tx, ny_used, nx_used)."""
    if edge == "partial":
        return -(-ny // w), -(-nx // w), ny, nx
    if edge == "drop":
        Ty, Tx = ny // w, nx // w
        return Ty, Tx, Ty * w, Tx * w
    raise ValueError(edge)


def tile_extent(t_index: int, n_used: int, w: int) -> int:
    """Number of pixels of tile row/column ``t_index`` along one axis."""
    return min(w, n_used - t_index * w)


# --------------------------------------------------------------------------
# Normaliser M (Eq. tLISI denominator; a single scalar, Sec. 2.3)
# --------------------------------------------------------------------------
def normaliser_M(stack: np.ndarray) -> float:
    """M = max(max_s max_i x_i^(s), C) over finite pixels."""
    x = np.asarray(stack, dtype=np.float64)
    fin = x[np.isfinite(x)]
    m = float(fin.max()) if fin.size else -np.inf
    return max(m, C)


def normaliser_M_running(stack: np.ndarray) -> np.ndarray:
    """Real-time reading of M (Sec. 2.2.4: in real time the maximum is taken
    over the snapshots seen so far, at least three): M_s for unit s is the
    maximum over every finite pixel of snapshots 0..s+2, floored at C."""
    x = np.asarray(stack, dtype=np.float64)
    L = x.shape[0]
    return np.array([normaliser_M(x[:s + 3]) for s in range(L - 2)])


# --------------------------------------------------------------------------
# Per-pixel terms of one three-snapshot unit (Eq. 3, Eq. 4, Eq. 5)
# --------------------------------------------------------------------------
def unit_terms(x_s: np.ndarray, x_s1: np.ndarray, x_s2: np.ndarray,
               rmode: str = "abs") -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Delta = |D^(s) - D^(s+1)|, r (Eq. 4) and a mask of fully finite pixels."""
    a = np.asarray(x_s, dtype=np.float64)
    b = np.asarray(x_s1, dtype=np.float64)
    c = np.asarray(x_s2, dtype=np.float64)
    finite = np.isfinite(a) & np.isfinite(b) & np.isfinite(c)
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        D_s = np.abs(b - a)            # D^(s)   = |x^(s+1) - x^(s)|
        D_s1 = np.abs(c - b)           # D^(s+1) = |x^(s+2) - x^(s+1)|
        delta = np.abs(D_s - D_s1)
        ref = np.abs(b) if rmode == "abs" else b
        x_hat = np.where(b == 0.0, C, ref)      # Eq. 5
        ratio = delta / x_hat
        r = np.where(ratio < 1.0, ratio, 1.0)   # Eq. 4
    delta = np.where(finite, delta, 0.0)
    r = np.where(finite, r, 0.0)
    return delta, r, finite


@dataclass
class UnitTiles:
    S1: np.ndarray       # sum of Delta per tile           (Ty, Tx)
    S2: np.ndarray       # max of Delta per tile
    S3: np.ndarray       # sum of r per tile
    n: np.ndarray        # pixel count per tile
    valid: np.ndarray    # tile has only finite pixels
    arg_y: np.ndarray    # pixel row of the first max of Delta
    arg_x: np.ndarray    # pixel column of the first max of Delta

    @property
    def numerator(self) -> np.ndarray:
        """mean(Delta) * max(Delta) * mean(r): the Eq. tLISI numerator."""
        with np.errstate(invalid="ignore"):
            v = (self.S1 / self.n) * self.S2 * (self.S3 / self.n)
        return np.where(self.valid, v, np.nan)


def tile_reduce(delta: np.ndarray, r: np.ndarray, finite: np.ndarray, w: int,
                Ty: int, Tx: int) -> UnitTiles:
    """Per-tile sum/max/sum over an image whose origin is a tile corner."""
    ny, nx = delta.shape
    H, W = Ty * w, Tx * w
    pd_sum = np.zeros((H, W))
    pd_max = np.full((H, W), -np.inf)
    pr = np.zeros((H, W))
    pf = np.ones((H, W), dtype=bool)
    h, wd = min(ny, H), min(nx, W)
    pd_sum[:h, :wd] = delta[:h, :wd]
    pd_max[:h, :wd] = delta[:h, :wd]
    pr[:h, :wd] = r[:h, :wd]
    pf[:h, :wd] = finite[:h, :wd]
    blk = lambda a: a.reshape(Ty, w, Tx, w).transpose(0, 2, 1, 3).reshape(Ty, Tx, w * w)
    S1 = blk(pd_sum).sum(axis=2)
    dm = blk(pd_max)
    S2 = dm.max(axis=2)
    idx = dm.argmax(axis=2)                  # first occurrence: smallest row-major
    S3 = blk(pr).sum(axis=2)
    valid = blk(pf).all(axis=2)
    hy = np.array([tile_extent(t, h, w) for t in range(Ty)])
    wx = np.array([tile_extent(t, wd, w) for t in range(Tx)])
    n = (hy[:, None] * wx[None, :]).astype(np.float64)
    ty = np.arange(Ty)[:, None]
    tx = np.arange(Tx)[None, :]
    arg_y = ty * w + idx // w
    arg_x = tx * w + idx % w
    return UnitTiles(S1, S2, S3, n, valid, arg_y, arg_x)


def unit_tiles(stack: np.ndarray, s: int, w: int, rmode: str = "abs",
               edge: str = "partial") -> UnitTiles:
    """Tile statistics of unit s, which spans snapshots (s, s+1, s+2)."""
    L, ny, nx = stack.shape
    Ty, Tx, nyu, nxu = tiling(ny, nx, w, edge)
    a, b, c = (stack[s + i, :nyu, :nxu] for i in range(3))
    delta, r, fin = unit_terms(a, b, c, rmode)
    return tile_reduce(delta, r, fin, w, Ty, Tx)


def window_stats(delta: np.ndarray, r: np.ndarray, finite: np.ndarray, w: int) -> UnitTiles:
    """Sliding-window statistics: for every pixel p, the sums of Delta and r and
    the maximum of Delta over the w x w window centred on p (w odd), clipped at
    the image border (n_p = number of in-image pixels).  Accumulates the w*w
    shifted copies of the maps one offset at a time.  The arg-max fields hold
    the pixel itself (the pixel is the location in this mode)."""
    if w % 2 != 1:
        raise ValueError("sliding windows need an odd size")
    ny, nx = delta.shape
    h = w // 2
    S1 = np.zeros((ny, nx))
    S2 = np.full((ny, nx), -np.inf)
    S3 = np.zeros((ny, nx))
    n = np.zeros((ny, nx))
    valid = np.ones((ny, nx), dtype=bool)
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            # window pixel q = p + (dy, dx); rows/cols of p for which q is inside
            py0, py1 = max(0, -dy), min(ny, ny - dy)
            px0, px1 = max(0, -dx), min(nx, nx - dx)
            if py0 >= py1 or px0 >= px1:
                continue
            q = (slice(py0 + dy, py1 + dy), slice(px0 + dx, px1 + dx))
            p = (slice(py0, py1), slice(px0, px1))
            S1[p] += delta[q]
            S2[p] = np.maximum(S2[p], delta[q])
            S3[p] += r[q]
            n[p] += 1.0
            valid[p] &= finite[q]
    yy, xx = np.mgrid[0:ny, 0:nx]
    return UnitTiles(S1, S2, S3, n, valid, yy, xx)


def unit_windows(stack: np.ndarray, s: int, w: int, rmode: str = "abs") -> UnitTiles:
    """Per-pixel sliding-window statistics of unit s (the 'local window' mode)."""
    a, b, c = (stack[s + i] for i in range(3))
    delta, r, fin = unit_terms(a, b, c, rmode)
    return window_stats(delta, r, fin, w)


def tlisi_from_tiles(ut: UnitTiles, M: float) -> np.ndarray:
    """Eq. tLISI: 1 - mean(Delta) max(Delta) mean(r) / (M * M); NaN if invalid."""
    with np.errstate(invalid="ignore"):
        t = 1.0 - (ut.S1 / ut.n) * ut.S2 * (ut.S3 / ut.n) / (M * M)
    return np.where(ut.valid, t, np.nan)


def sampled_tiles(stack: np.ndarray, w: int, tiles: Sequence[Tuple[int, int]],
                  rmode: str = "abs", edge: str = "partial") -> Dict[str, np.ndarray]:
    """Tile statistics of selected tiles for every unit (tiles are independent).

    Returns arrays of shape (units, len(tiles)).
    """
    L, ny, nx = stack.shape
    Ty, Tx, nyu, nxu = tiling(ny, nx, w, edge)
    U = L - 2
    out = {k: np.zeros((U, len(tiles))) for k in ("S1", "S2", "S3", "n", "numerator")}
    out["valid"] = np.zeros((U, len(tiles)), dtype=bool)
    out["arg_y"] = np.zeros((U, len(tiles)), dtype=np.int64)
    out["arg_x"] = np.zeros((U, len(tiles)), dtype=np.int64)
    for j, (ty, tx) in enumerate(tiles):
        y0, x0 = ty * w, tx * w
        y1, x1 = min(y0 + w, nyu), min(x0 + w, nxu)
        sub = np.asarray(stack[:, y0:y1, x0:x1], dtype=np.float64)
        for s in range(U):
            d, r, f = unit_terms(sub[s], sub[s + 1], sub[s + 2], rmode)
            ut = tile_reduce(d, r, f, w, 1, 1)
            for k in ("S1", "S2", "S3", "n"):
                out[k][s, j] = getattr(ut, k)[0, 0]
            out["numerator"][s, j] = ut.numerator[0, 0]
            out["valid"][s, j] = ut.valid[0, 0]
            out["arg_y"][s, j] = y0 + ut.arg_y[0, 0]
            out["arg_x"][s, j] = x0 + ut.arg_x[0, 0]
    return out


# --------------------------------------------------------------------------
# Noise estimates (Sec. 2.4.1 mean/std; robust median/MAD reading)
# --------------------------------------------------------------------------
def lower_median(values: np.ndarray) -> float:
    v = np.sort(np.asarray(values, dtype=np.float64).ravel())
    return float(v[(v.size - 1) // 2])


def noise_meanstd(values: np.ndarray) -> Tuple[float, float, int]:
    v = np.asarray(values, dtype=np.float64).ravel()
    v = v[np.isfinite(v)]
    if v.size == 0:
        return float("nan"), 0.0, 0
    return float(v.mean()), float(v.std()), int(v.size)


def noise_medmad(values: np.ndarray) -> Tuple[float, float, int]:
    v = np.asarray(values, dtype=np.float64).ravel()
    v = v[np.isfinite(v)]
    if v.size == 0:
        return float("nan"), 0.0, 0
    med = lower_median(v)
    mad = lower_median(np.abs(v - med))
    return med, MAD_TO_SIGMA * mad, int(v.size)


def zscore_image(tlisi: np.ndarray, noise: str = "meanstd") -> Tuple[np.ndarray, float, float]:
    """Eq. (z-score): z = (mu - tLISI) / sigma over the tiles of one unit.

    The robust mode applies the same form to the complement v = 1 - tLISI:
    z = (v - median(v)) / (1.4826 MAD(v)).  Returns (z, centre, scale), where
    the centre/scale are those of the complement v in both modes.
    """
    if noise == "meanstd":
        mu, sigma, _ = noise_meanstd(tlisi)
        with np.errstate(invalid="ignore", divide="ignore"):
            z = (mu - tlisi) / sigma if sigma > 0 else np.full(tlisi.shape, np.nan)
        return z, 1.0 - mu, sigma
    v = 1.0 - tlisi
    med, scale, _ = noise_medmad(v)
    with np.errstate(invalid="ignore", divide="ignore"):
        z = (v - med) / scale if scale > 0 else np.full(tlisi.shape, np.nan)
    return z, med, scale


def zscore_map(values: np.ndarray, noise: str = "meanstd") -> Tuple[np.ndarray, float, float]:
    """z = (value - centre) / scale, used for eta (Sec. 2.4.2) and plain maps."""
    centre, scale, _ = noise_meanstd(values) if noise == "meanstd" else noise_medmad(values)
    with np.errstate(invalid="ignore", divide="ignore"):
        z = (values - centre) / scale if scale > 0 else np.full(np.shape(values), np.nan)
    return z, centre, scale


# --------------------------------------------------------------------------
# Selection and 8-connected components
# --------------------------------------------------------------------------
def select(z: np.ndarray, tau: float) -> np.ndarray:
    """{t | z_t > tau} as a boolean mask (strict inequality)."""
    with np.errstate(invalid="ignore"):
        return np.asarray(z > tau) & np.isfinite(z)


def components(mask: np.ndarray) -> List[List[Tuple[int, int]]]:
    """8-connected components of a boolean (Ty, Tx) mask, by breadth-first search."""
    Ty, Tx = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    comps = []
    for ty, tx in zip(*np.nonzero(mask)):
        if seen[ty, tx]:
            continue
        comp = []
        q = deque([(int(ty), int(tx))])
        seen[ty, tx] = True
        while q:
            cy, cx = q.popleft()
            comp.append((cy, cx))
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ny_, nx_ = cy + dy, cx + dx
                    if 0 <= ny_ < Ty and 0 <= nx_ < Tx and mask[ny_, nx_] and not seen[ny_, nx_]:
                        seen[ny_, nx_] = True
                        q.append((ny_, nx_))
        comps.append(comp)
    return comps


def component_peak(comp: List[Tuple[int, int]], z: np.ndarray) -> Tuple[int, int]:
    """Maximum-z tile of a component; ties go to the smallest row-major index."""
    return max(comp, key=lambda p: (z[p], -p[0], -p[1]))


# --------------------------------------------------------------------------
# Image-frequency branch (Sec. 2.4.2)
# --------------------------------------------------------------------------
def dft_magnitudes(series: np.ndarray) -> np.ndarray:
    """|F[y - mean(y)]|_k for k = 1..floor(n/2), unnormalised DFT of length n.

    ``series`` has shape (..., n).  The twiddle matrix exp(-2 pi i k s / n) is
    applied by a matrix product (naive O(n^2) DFT).
    """
    y = np.asarray(series, dtype=np.float64)
    n = y.shape[-1]
    yc = y - y.mean(axis=-1, keepdims=True)
    k = np.arange(1, n // 2 + 1)
    s = np.arange(n)
    ang = 2.0 * np.pi * ((np.outer(s, k) % n) / n)
    X = yc @ np.cos(ang) - 1j * (yc @ np.sin(ang))
    return np.abs(X)


def harmonic_sum(mags: np.ndarray, m_max: int) -> Tuple[np.ndarray, np.ndarray]:
    """h of Eq. (eta) as an incoherent harmonic sum.

    ``mags`` has shape (tiles, K) and holds |X_k| for k = 1..K.  For every
    m = 1, 2, 4, .., m_max and every fundamental k with m k <= K,
    S_m(k) = (|X_k| + |X_2k| + .. + |X_mk|) / sqrt(m); the result is the
    largest S_m(k) per tile and its fundamental k (ties: smaller m, then
    smaller k).  With m_max = 1 it is max_k |X_k| (the maximum magnitude).
    """
    a = np.asarray(mags, dtype=np.float64)
    ntile, K = a.shape
    best = np.full(ntile, -np.inf)
    kbin = np.ones(ntile, dtype=np.int64)
    m = 1
    while m <= m_max:
        for k in range(1, K // m + 1):
            total = np.zeros(ntile)
            for j in range(1, m + 1):
                total = total + a[:, j * k - 1]
            S = total / np.sqrt(m)
            better = S > best
            best = np.where(better, S, best)
            kbin = np.where(better, k, kbin)
        m *= 2
    return best, kbin


def spectrum(cube: np.ndarray, harmonics: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """eta_t = h(|X_k|) and its bin per tile: h = max_k |X_k| (smallest k on
    ties) when ``harmonics`` is 1, else ``harmonic_sum`` with m_max =
    ``harmonics``.

    ``cube`` is the tLISI cube with shape (L-2, Ty, Tx); tiles with a
    non-finite entry get eta = NaN and bin = -1.
    """
    U, Ty, Tx = cube.shape
    series = np.moveaxis(cube, 0, -1).reshape(Ty * Tx, U)
    ok = np.all(np.isfinite(series), axis=1)
    mags = dft_magnitudes(np.where(ok[:, None], series, 0.0))
    if harmonics == 1:
        eta = mags.max(axis=1)
        kbin = mags.argmax(axis=1) + 1
    else:
        eta, kbin = harmonic_sum(mags, harmonics)
    eta = np.where(ok, eta, np.nan).reshape(Ty, Tx)
    kbin = np.where(ok, kbin, -1).reshape(Ty, Tx)
    return eta, kbin


def parabolic_offset(left: float, centre: float, right: float) -> float:
    """Vertex offset (in grid steps) of the parabola through three samples."""
    if not (np.isfinite(left) and np.isfinite(right) and np.isfinite(centre)):
        return 0.0
    den = left - 2.0 * centre + right
    if not den < 0.0:
        return 0.0
    d = 0.5 * (left - right) / den
    return float(min(0.5, max(-0.5, d)))


def cubic_offset(m2: float, m1: float, c: float, p1: float, p2: float) -> float:
    """Peak offset (in grid steps, within [-0.5, 0.5]) of the Catmull-Rom cubic
    spline through the samples at -2, -1, 0, +1, +2 (the "spline
    interpolation" of eta, Sec. 2.4.2 and the real-data evaluation of Sec. 3; our reading).

    On the segment between samples a (at 0) and b (at 1) with outer neighbours
    z (at -1) and d (at 2) the spline is
        f(t) = a + t (b - z) / 2 + t^2 (2z - 5a + 4b - d) / 2
               + t^3 (-z + 3a - 3b + d) / 2.
    The maximum over [0, 0.5] (segment 0..1, t in [0, 0.5]) and [-0.5, 0]
    (segment -1..0, t in [0.5, 1]) is taken among, in this order, the offset
    0, the right segment's interior roots of f' (ascending) and +0.5, then the
    left segment's interior roots (ascending) and -0.5; the first of equal
    values is kept.  A side whose neighbour at +-1 is missing (outside the map or not
    finite) is not searched; a missing sample at +-2 is extended linearly
    (2 f(+-1) - f(0)).  A non-finite centre gives 0.
    """
    fin = np.isfinite
    if not fin(c):
        return 0.0
    best_x, best_f = 0.0, float(c)

    def consider(x: float, f: float):
        nonlocal best_x, best_f
        if f > best_f:
            best_x, best_f = x, f

    def segment(z, a, b, d, lo, hi, shift):
        # f on t in [lo, hi]; offset x = t + shift
        k1 = 0.5 * (b - z)
        k2 = 0.5 * (2 * z - 5 * a + 4 * b - d)
        k3 = 0.5 * (-z + 3 * a - 3 * b + d)
        f = lambda t: a + t * (k1 + t * (k2 + t * k3))
        # roots of f'(t) = A t^2 + B t + C by the cancellation-free form
        # q = -(B + sign(B) sqrt(B^2 - 4AC)) / 2, t = q / A and C / q (a
        # near-zero A, as for a quadratic, leaves the linear root intact)
        A, B, C_ = 3.0 * k3, 2.0 * k2, k1
        roots = []
        disc = B * B - 4.0 * A * C_
        if disc >= 0.0:
            q = -0.5 * (B + np.copysign(np.sqrt(disc), B))
            if A != 0.0:
                roots.append(q / A)
            if q != 0.0:
                roots.append(C_ / q)
            roots.sort()
        for t in roots:
            if lo < t < hi:
                consider(t + shift, f(t))
        end = hi if shift == 0.0 else lo
        consider(end + shift, f(end))

    if fin(p1):
        d = p2 if fin(p2) else 2.0 * p1 - c
        segment(m1 if fin(m1) else 2.0 * c - p1, c, p1, d, 0.0, 0.5, 0.0)
    if fin(m1):
        z = m2 if fin(m2) else 2.0 * m1 - c
        segment(z, m1, c, p1 if fin(p1) else 2.0 * c - m1, 0.5, 1.0, -1.0)
    return float(best_x)


# --------------------------------------------------------------------------
# Whole trigger
# --------------------------------------------------------------------------
@dataclass
class Candidate:
    snapshot: int
    y: int
    x: int
    significance: float
    branch: int
    freq_bin: int
    xf: float
    yf: float

    def key(self):
        return (self.snapshot, self.y, self.x)


@dataclass
class Detection:
    candidates: List[Candidate]
    M: float
    Ty: int
    Tx: int
    tlisi: Optional[np.ndarray] = None       # (U, Ty, Tx)
    z: Optional[np.ndarray] = None           # (U, Ty, Tx)
    centre: Optional[np.ndarray] = None      # (U,) of the complement v
    scale: Optional[np.ndarray] = None       # (U,)
    units: Optional[List[UnitTiles]] = None
    eta: Optional[np.ndarray] = None
    eta_bin: Optional[np.ndarray] = None
    eta_z: Optional[np.ndarray] = None
    eta_centre: float = float("nan")
    eta_scale: float = float("nan")
    M_units: Optional[np.ndarray] = None     # (U,) normaliser of each unit


def image_candidates(units: List[UnitTiles], z: np.ndarray, tau: float,
                     forced: Optional[Dict[Tuple[int, int, int], bool]] = None) -> List[Candidate]:
    out = []
    for s, ut in enumerate(units):
        mask = select(z[s], tau)
        if forced:
            for (fs, ty, tx), val in forced.items():
                if fs == s:
                    mask[ty, tx] = val
        for comp in components(mask):
            ty, tx = component_peak(comp, z[s])
            out.append(Candidate(s, int(ut.arg_y[ty, tx]), int(ut.arg_x[ty, tx]),
                                 float(z[s, ty, tx]), BRANCH_IMAGE, -1,
                                 float(ut.arg_x[ty, tx]), float(ut.arg_y[ty, tx])))
    return out


def freq_candidates(eta: np.ndarray, kbin: np.ndarray, z: np.ndarray, tau: float,
                    w: int, nyu: int, nxu: int,
                    forced: Optional[Dict[Tuple[int, int], bool]] = None,
                    refine: str = "parabolic") -> List[Candidate]:
    """One candidate per component of the selected eta tiles, at the peak
    tile's centre; the refined position uses ``parabolic_offset`` (three
    samples) or ``cubic_offset`` (the spline through five) along each axis."""
    Ty, Tx = eta.shape
    mask = select(z, tau)
    if forced:
        for (ty, tx), val in forced.items():
            mask[ty, tx] = val
    out = []
    for comp in components(mask):
        ty, tx = component_peak(comp, z)
        hy, wx = tile_extent(ty, nyu, w), tile_extent(tx, nxu, w)
        cx = tx * w + (wx - 1) / 2.0
        cy = ty * w + (hy - 1) / 2.0
        gx = lambda j: eta[ty, j] if 0 <= j < Tx else np.nan
        gy = lambda j: eta[j, tx] if 0 <= j < Ty else np.nan
        if refine == "cubic":
            dx = cubic_offset(gx(tx - 2), gx(tx - 1), eta[ty, tx], gx(tx + 1), gx(tx + 2))
            dy = cubic_offset(gy(ty - 2), gy(ty - 1), eta[ty, tx], gy(ty + 1), gy(ty + 2))
        else:
            dx = parabolic_offset(gx(tx - 1), eta[ty, tx], gx(tx + 1))
            dy = parabolic_offset(gy(ty - 1), eta[ty, tx], gy(ty + 1))
        out.append(Candidate(-1, ty * w + (hy - 1) // 2, tx * w + (wx - 1) // 2,
                             float(z[ty, tx]), BRANCH_FREQ, int(kbin[ty, tx]),
                             float(cx + dx * w), float(cy + dy * w)))
    return out


def detect(stack: np.ndarray, w: int, tau: float, branch: int = BRANCH_IMAGE,
           noise: str = "meanstd", rmode: str = "abs", edge: str = "partial",
           forced_image=None, forced_freq=None, stride: str = "tile",
           mmode: str = "global", harmonics: int = 1, refine: str = "parabolic") -> Detection:
    """Run the trigger on a (L, ny, nx) stack and return the sorted candidates.

    stride "tile" is the paper's tiling; "sliding" evaluates the same statistic
    over a w x w window centred on every pixel, after which every pixel plays
    the part of a 1 x 1 tile in the z-score, selection and components.
    mmode "global" normalises every unit by the one M of the whole stack;
    "running" normalises unit s by M_s over snapshots 0..s+2 (real time).
    ``Detection.M`` is the global M in both modes, ``Detection.M_units`` the
    normaliser of each unit.  ``harmonics`` is m_max of the frequency branch's
    h (1: maximum magnitude).
    """
    x = np.asarray(stack)
    L, ny, nx = x.shape
    if stride == "sliding":
        region = x
        units = [unit_windows(x, s, w, rmode) for s in range(L - 2)]
        Ty, Tx, nyu, nxu, w = ny, nx, ny, nx, 1
    else:
        Ty, Tx, nyu, nxu = tiling(ny, nx, w, edge)
        region = x[:, :nyu, :nxu]
        units = [unit_tiles(x, s, w, rmode, edge) for s in range(L - 2)]
    M = normaliser_M(region)
    Ms = normaliser_M_running(region) if mmode == "running" else np.full(L - 2, M)
    tl = np.stack([tlisi_from_tiles(u, Ms[s]) for s, u in enumerate(units)])
    det = Detection([], M, Ty, Tx, tlisi=tl, units=units, M_units=Ms)
    cands: List[Candidate] = []
    if branch & BRANCH_IMAGE:
        zs, cs, ss = [], [], []
        for s in range(L - 2):
            z, c, sc = zscore_image(tl[s], noise)
            zs.append(z)
            cs.append(c)
            ss.append(sc)
        det.z = np.stack(zs)
        det.centre = np.array(cs)
        det.scale = np.array(ss)
        cands += image_candidates(units, det.z, tau, forced_image)
    if branch & BRANCH_FREQ:
        eta, kbin = spectrum(tl, harmonics)
        ez, ec, es = zscore_map(eta, noise)
        det.eta, det.eta_bin, det.eta_z = eta, kbin, ez
        det.eta_centre, det.eta_scale = ec, es
        cands += freq_candidates(eta, kbin, ez, tau, w, nyu, nxu, forced_freq, refine)
    cands.sort(key=Candidate.key)
    det.candidates = cands
    return det


def freq_window(stack: np.ndarray, w: int, tau: float, n: int, noise: str = "meanstd",
                forced: Optional[Dict[Tuple[int, int], bool]] = None, harmonics: int = 1,
                refine: str = "parabolic"):
    """Real-time image-frequency branch: the Sec. 2.4.2 statistic over the last
    ``n`` units of the stack only (units L-2-n .. L-3), each normalised by its
    running M_s (the real-time reading of Sec. 2.2.4).  Returns (candidates,
    eta, kbin, z) for the window ending at the stack's last unit; the
    candidates' snapshot is that unit.  With n = L - 2 and a running maximum
    that is already global at the first unit this is ``detect(...,
    BRANCH_FREQ)`` exactly."""
    x = np.asarray(stack)
    L, ny, nx = x.shape
    if not 1 <= n <= L - 2:
        raise ValueError("window longer than the units of the stack")
    Ty, Tx, nyu, nxu = tiling(ny, nx, w)
    region = x[:, :nyu, :nxu]
    Ms = normaliser_M_running(region)
    first = L - 2 - n
    tl = np.stack([tlisi_from_tiles(unit_tiles(x, s, w), Ms[s]) for s in range(first, L - 2)])
    eta, kbin = spectrum(tl, harmonics)
    z, _, _ = zscore_map(eta, noise)
    cands = freq_candidates(eta, kbin, z, tau, w, nyu, nxu, forced, refine)
    for c in cands:
        c.snapshot = L - 3
    return cands, eta, kbin, z


def threshold_count(values: np.ndarray, tau: float, noise: str = "meanstd") -> int:
    """Number of entries of a plain map whose z-score exceeds tau."""
    z, _, _ = zscore_map(np.asarray(values, dtype=np.float64), noise)
    return int(np.count_nonzero(select(z, tau)))
