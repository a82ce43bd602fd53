"""Parity rule between a candidate list and the FP64 oracle.

TEST INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and
bench.py's CPU legs).

A tile is *ambiguous* when its oracle z lies within ``REL_TOL * tau`` of the
threshold.  Ambiguous tiles take the decision of the implementation under test
(passed in as ``decide``) and the oracle's components are rebuilt with that
forced mask; outside them the masks must agree exactly.  Each oracle component
must then be matched by exactly one candidate that

* sits in a tile of that component whose oracle z is within REL_TOL of the
  component's maximum z (a near tie may pick either tile),
* reports a significance within REL_TOL (relative) of that tile's oracle z,
* for the image branch, is a pixel whose oracle Delta is within the FP32
  rounding bound of the tile's maximum Delta (ties may pick either pixel),
* for the frequency branch, is the tile centre, with a DFT bin whose oracle
  magnitude is within REL_TOL of the tile's maximum, and a refined position
  within ``XF_TOL_TILES`` tiles of the oracle's.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from . import fitrig_oracle as O

REL_TOL = 1e-4
XF_TOL_TILES = 0.05
U32 = 2.0 ** -24


def _near_peak(comp, z, tol):
    zmax = max(z[p] for p in comp)
    return {p for p in comp if z[p] >= zmax - tol * max(1.0, abs(zmax))}


def _pixels_ok(stack: np.ndarray, s: np.ndarray, y: np.ndarray, x: np.ndarray,
               ty: np.ndarray, tx: np.ndarray, w: int, nyu: int, nxu: int, rmode: str,
               chunk: int = 65536) -> np.ndarray:
    """For each image candidate (unit s, pixel (y, x), peak tile (ty, tx)):
    whether the pixel lies in the tile and its oracle Delta is within the FP32
    rounding bound of the tile's maximum Delta (so near ties may pick either
    pixel).  Vectorised over candidates; ragged edge tiles are masked."""
    n = len(s)
    ok = np.zeros(n, dtype=bool)
    off = np.arange(w)
    for i0 in range(0, n, chunk):
        sl = slice(i0, min(n, i0 + chunk))
        ss, yy, xx, tyy, txx = s[sl], y[sl], x[sl], ty[sl], tx[sl]
        rows = tyy[:, None] * w + off[None, :]                  # (m, w)
        cols = txx[:, None] * w + off[None, :]
        inside = (rows[:, :, None] < nyu) & (cols[:, None, :] < nxu)
        rc = np.minimum(rows, nyu - 1)
        cc = np.minimum(cols, nxu - 1)
        a, b, c = (np.asarray(stack[(ss + k)[:, None, None], rc[:, :, None], cc[:, None, :]],
                              dtype=np.float64) for k in range(3))
        d, _, _ = O.unit_terms(a, b, c, rmode)
        d = np.where(inside, d, -np.inf)
        mag = np.where(inside, np.abs(a) + 2 * np.abs(b) + np.abs(c), 0.0)
        bound = 8 * U32 * mag.reshape(len(ss), -1).max(axis=1) + 1e-300
        dmax = d.reshape(len(ss), -1).max(axis=1)
        iy, ix = yy - tyy * w, xx - txx * w
        inr = (iy >= 0) & (iy < w) & (ix >= 0) & (ix < w) & (yy < nyu) & (xx < nxu)
        m = np.arange(len(ss))
        dv = d[m, np.clip(iy, 0, w - 1), np.clip(ix, 0, w - 1)]
        ok[sl] = inr & (dv >= dmax - bound)
    return ok


def compare(cands: np.ndarray, stack: np.ndarray, w: int, tau: float, branch: int,
            noise: str = "meanstd", rmode: str = "abs", edge: str = "partial",
            decide_image: Optional[Callable[[int, int, int], bool]] = None,
            decide_freq: Optional[Callable[[int, int], bool]] = None,
            det: Optional[O.Detection] = None,
            harmonics: int = 1, refine: str = "parabolic",
            cut_top: bool = False, cut_bottom: bool = False) -> List[str]:
    """Return a list of parity violations (empty when the lists agree).

    ``harmonics`` is m_max of the frequency branch's h (1: maximum magnitude);
    a frequency candidate's bin must then be a fundamental whose best harmonic
    sum is within the tolerance of the tile's largest.  Every candidate is
    checked, including the arg-max pixel of every image candidate.

    ``cut_top`` / ``cut_bottom`` say that ``stack`` is a strip of whole tile
    rows cut out of a larger field at its first / last tile row: components
    that touch a cut row may continue beyond the strip, so they and the
    candidates inside them are skipped; every other component and candidate
    is checked as usual.
    """
    errs: List[str] = []
    L, ny, nx = stack.shape
    Ty, Tx, nyu, nxu = O.tiling(ny, nx, w, edge)
    if det is None:
        det = O.detect(stack, w, tau, branch, noise, rmode, edge, harmonics=harmonics,
                       refine=refine)
    band = REL_TOL * tau
    names = cands.dtype.names
    cols = {k: cands[k].tolist() for k in names}
    got = [dict(zip(names, row)) for row in zip(*(cols[k] for k in names))]

    def check_groups(groups, branch_id):
        # groups: list of (label, z_map, comps, snapshot)
        by_tile = {}
        for k, gc in enumerate(got):
            if gc["branch"] == branch_id:
                key = (int(gc["snapshot"]), int(gc["y"]) // w, int(gc["x"]) // w)
                if key in by_tile:
                    errs.append(f"two candidates in one tile: {gc}")
                by_tile[key] = k
        used = set()
        for label, zmap, comps, snap in groups:
            for comp in comps:
                hits = [by_tile[(snap,) + t] for t in comp if (snap,) + t in by_tile]
                if any((cut_top and t[0] == 0) or (cut_bottom and t[0] == Ty - 1)
                       for t in comp):
                    used.update(hits)   # may continue beyond the strip
                    continue
                if len(hits) != 1:
                    errs.append(f"{label}: oracle component at {sorted(comp)[:4]} has "
                                f"{len(hits)} candidates")
                    used.update(hits)
                    continue
                k = hits[0]
                used.add(k)
                gc = got[k]
                t = (int(gc["y"]) // w, int(gc["x"]) // w)
                near = _near_peak(comp, zmap, REL_TOL)
                if t not in near:
                    errs.append(f"{label}: candidate tile {t} is not a peak tile {sorted(near)[:4]}")
                zt = zmap[t]
                if abs(gc["significance"] - zt) > REL_TOL * max(1.0, abs(zt)):
                    errs.append(f"{label}: significance {gc['significance']} vs oracle {zt}")
                yield gc, t, snap
        for k, gc in enumerate(got):
            if gc["branch"] == branch_id and k not in used:
                errs.append(f"extra candidate {gc}")

    if branch & O.BRANCH_IMAGE:
        groups = []
        for s in range(L - 2):
            z = det.z[s]
            with np.errstate(invalid="ignore"):
                amb = np.isfinite(z) & (np.abs(z - tau) <= band)
            mask = O.select(z, tau)
            for ty, tx in zip(*np.nonzero(amb)):
                if decide_image is None:
                    errs.append(f"unit {s}: ambiguous tile {(ty, tx)} and no decision callback")
                else:
                    mask[ty, tx] = bool(decide_image(s, int(ty), int(tx)))
            groups.append((f"unit {s}", z, O.components(mask), s))
        matched = list(check_groups(groups, O.BRANCH_IMAGE))
        if matched:
            arr = lambda f: np.array([f(m) for m in matched], dtype=np.int64)
            ok = _pixels_ok(stack, arr(lambda m: m[2]), arr(lambda m: int(m[0]["y"])),
                            arr(lambda m: int(m[0]["x"])), arr(lambda m: m[1][0]),
                            arr(lambda m: m[1][1]), w, nyu, nxu, rmode)
            for (gc, _, s) in (matched[i] for i in np.nonzero(~ok)[0]):
                errs.append(f"unit {s}: pixel {(gc['y'], gc['x'])} is not an arg-max of Delta")

    if branch & O.BRANCH_FREQ:
        z = det.eta_z
        with np.errstate(invalid="ignore"):
            amb = np.isfinite(z) & (np.abs(z - tau) <= band)
        mask = O.select(z, tau)
        for ty, tx in zip(*np.nonzero(amb)):
            if decide_freq is None:
                errs.append(f"freq: ambiguous tile {(ty, tx)} and no decision callback")
            else:
                mask[ty, tx] = bool(decide_freq(int(ty), int(tx)))
        comps = O.components(mask)
        ref = {}
        for c in O.freq_candidates(det.eta, det.eta_bin, z, tau, w, nyu, nxu,
                                   forced={(int(a), int(b)): bool(mask[a, b])
                                           for a, b in zip(*np.nonzero(amb))},
                                   refine=refine):
            ref[(c.y // w, c.x // w)] = c
        series = det.tlisi
        for gc, (ty, tx), _ in check_groups([("freq", z, comps, -1)], O.BRANCH_FREQ):
            hy, wx = O.tile_extent(ty, nyu, w), O.tile_extent(tx, nxu, w)
            if (gc["y"], gc["x"]) != (ty * w + (hy - 1) // 2, tx * w + (wx - 1) // 2):
                errs.append(f"freq: candidate {(gc['y'], gc['x'])} is not the centre of {(ty, tx)}")
            mags = O.dft_magnitudes(series[:, ty, tx])
            k = int(gc["freq_bin"])
            if not bin_is_a_maximum(mags, k, harmonics):
                errs.append(f"freq: bin {k} is not a maximum of tile {(ty, tx)}")
            oc = ref.get((ty, tx))
            if oc is not None:
                if abs(gc["xf"] - oc.xf) > XF_TOL_TILES * w or abs(gc["yf"] - oc.yf) > XF_TOL_TILES * w:
                    errs.append(f"freq: refined {(gc['yf'], gc['xf'])} vs oracle {(oc.yf, oc.xf)}")
    return errs


def bin_is_a_maximum(mags: np.ndarray, k: int, harmonics: int = 1) -> bool:
    """Whether fundamental k attains, within REL_TOL, the largest value of h
    over the magnitudes |X_1..X_K| (largest over m of the harmonic sums at k)."""
    K = mags.size
    if not 1 <= k <= K:
        return False
    top = O.harmonic_sum(mags[None, :], harmonics)[0][0]
    val, m = -np.inf, 1
    while m <= harmonics and m * k <= K:
        val = max(val, sum(mags[j * k - 1] for j in range(1, m + 1)) / np.sqrt(m))
        m *= 2
    return bool(val >= top * (1 - REL_TOL))


def tile_value_bound(stack: np.ndarray, s: int, w: int, rmode: str = "abs",
                     edge: str = "partial", stride: str = "tile") -> np.ndarray:
    """Per tile of unit s, an upper bound on |v - v_exact| for an implementation
    that computes the tile statistic v = mean(Delta) max(Delta) mean(r) in
    FP32 (unit roundoff u = 2^-24) from the stored values, where v_exact is
    the FP64 value of the same definition on the same inputs.

    Per pixel: D^(s) = fl|b - a| and D^(s+1) = fl|c - b| are each one rounding
    and Delta one more, so |Delta - Delta_exact| <= e_D = u (D1 + D2 + Delta)
    (1 + 1/64): the error is relative to the differences, not to Delta, which
    can be far smaller when D1 and D2 nearly cancel (a pulse in the middle
    snapshot).  The ratio Delta / |b| takes an approximate reciprocal (relative
    error <= 2u) and a product (u), and min(., 1) does not enlarge errors, so
    |r - r_exact| <= min(1, (e_D + 3u (Delta + e_D)) / |b|), and 0 where both
    sides are certainly clipped at 1.  Tile sums of m terms add (m - 1) u times
    the sum of magnitudes; the maximum moves by at most the largest e_D; the
    two divisions by the pixel count and the two products add 8u.  The bound
    on v follows from the perturbed factors.  With stride "sliding" the sums
    run over the window centred on each pixel instead of over tiles."""
    u = 2.0 ** -24
    L, ny, nx = stack.shape
    Ty, Tx, nyu, nxu = O.tiling(ny, nx, w, edge) if stride == "tile" else (ny, nx, ny, nx)
    a, b, c = (np.asarray(stack[s + i, :nyu, :nxu], dtype=np.float64) for i in range(3))
    delta, r, fin = O.unit_terms(a, b, c, rmode)
    with np.errstate(invalid="ignore", over="ignore"):
        d1 = np.abs(b - a)
        d2 = np.abs(c - b)
        eD = u * (d1 + d2 + delta) * (1.0 + 1.0 / 64)
        xh = np.where(b == 0.0, O.C, np.abs(b))
        ratio = delta / xh
        er = (eD + 3 * u * (delta + eD)) / xh
        er = np.where(ratio - er >= 1.0, 0.0, np.minimum(er, 1.0))
    eD = np.where(fin, eD, 0.0)
    er = np.where(fin, er, 0.0)
    if stride == "tile":
        ut = O.tile_reduce(delta, r, fin, w, Ty, Tx)
        eu = O.tile_reduce(eD, er, fin, w, Ty, Tx)
    else:
        ut = O.window_stats(delta, r, fin, w)
        eu = O.window_stats(eD, er, fin, w)
    m = ut.n
    S1 = ut.S1 + eu.S1 + (m - 1) * u * (ut.S1 + eu.S1)
    S2 = ut.S2 + eu.S2
    S3 = ut.S3 + eu.S3 + (m - 1) * u * (ut.S3 + eu.S3)
    hi = (S1 / m) * S2 * (S3 / m) * (1 + 8 * u)
    return np.where(ut.valid, hi - ut.numerator, np.nan)


def values_within_bound(gpu: np.ndarray, ref: np.ndarray, bound: np.ndarray,
                        slack: float = 2.0) -> Tuple[bool, float]:
    """|gpu - ref| <= slack * bound elementwise (NaNs must coincide); returns
    (ok, worst ratio of error to bound)."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    if not np.array_equal(np.isnan(g), np.isnan(r)):
        return False, float("inf")
    m = np.isfinite(r)
    if not m.any():
        return True, 0.0
    err = np.abs(g[m] - r[m])
    b = np.asarray(bound, dtype=np.float64)[m]
    ratio = err / np.maximum(b, 1e-300)
    return bool(np.all(err <= slack * b)), float(ratio.max())


def values_close(gpu: np.ndarray, ref: np.ndarray, rel: float = 1e-5,
                 abs_scale: float = 1e-6) -> Tuple[bool, float]:
    """Elementwise |gpu - ref| <= rel |ref| + abs_scale * mean|ref|, NaNs must coincide."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    if not np.array_equal(np.isnan(g), np.isnan(r)):
        return False, float("inf")
    m = np.isfinite(r)
    if not m.any():
        return True, 0.0
    scale = float(np.mean(np.abs(r[m]))) if m.any() else 0.0
    err = np.abs(g[m] - r[m])
    ok = bool(np.all(err <= rel * np.abs(r[m]) + abs_scale * scale))
    worst = float(np.max(err / (np.abs(r[m]) + abs_scale * scale + 1e-300)))
    return ok, worst


def library_decisions(res: dict, tau: float):
    """Threshold decisions of the implementation under test, from its dumped
    tile values and noise parameters (centre, scale): a tile is selected when
    (double)v > centre + tau * scale.  Used only for the ambiguous tiles of
    ``compare`` (those whose oracle z lies within the tolerance band of tau).
    Returns (image(s, ty, tx), freq(ty, tx))."""
    def image(s, ty, tx):
        c, sc = res["noise"][s]
        return sc > 0 and float(res["values"][s, ty, tx]) > c + tau * sc

    def freq(ty, tx):
        c, sc = res["eta_noise"]
        return sc > 0 and float(res["eta"][ty, tx]) > c + tau * sc
    return image, freq
