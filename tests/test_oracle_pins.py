"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an invariant the paper
states or implies, a hand-derived worked example, a library routine that the
definition reduces to, or brute force on tiny inputs, so that a dropped term,
a wrong sign/index or a transposed operand in the oracle fails at least one.
"""
import json
import math
import os
import statistics
from fractions import Fraction

import numpy as np
import pytest

from oracle import fitrig_oracle as O
from paper_2509_21754_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac_eval(expr: str) -> float:
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _worked_example_stack():
    g = json.load(open(os.path.join(GOLDEN, "pulse_worked_example.json")))
    b = g["background"]
    x = np.zeros((5, 6, 8), dtype=np.float32)
    for k, bk in enumerate(b):
        x[k] = bk
    p = g["pulse"]
    x[p["snapshot"], p["y"], p["x"]] += p["amp"]
    return g, x


# ---------------------------------------------------------------- worked example
def test_worked_example_tlisi_values():
    """Hand-derived tLISI of every tile of every unit (Eq. tLISI, Eq. 3-5)."""
    g, x = _worked_example_stack()
    det = O.detect(x, g["w"], g["tau"], noise="meanstd")
    assert det.M == 6.0
    assert (det.Ty, det.Tx) == (2, 3)
    for s in range(3):
        want = np.array([[_frac_eval(e) for e in row] for row in g["tlisi"][str(s)]])
        np.testing.assert_allclose(det.tlisi[s], want, rtol=0, atol=1e-15)
    a0 = g["argmax_unit0_tile01"]
    assert (det.units[0].arg_y[0, 1], det.units[0].arg_x[0, 1]) == (a0["y"], a0["x"])
    a2 = g["argmax_unit2_tile01"]
    assert (det.units[2].arg_y[0, 1], det.units[2].arg_x[0, 1]) == (a2["y"], a2["x"])


def test_worked_example_candidates():
    g, x = _worked_example_stack()
    det = O.detect(x, g["w"], g["tau"], noise="meanstd")
    got = [(c.snapshot, c.y, c.x) for c in det.candidates]
    want = [(c["snapshot"], c["y"], c["x"]) for c in g["candidates_meanstd"]]
    assert got == want
    assert det.candidates[0].significance == pytest.approx(math.sqrt(5.0), rel=1e-12)
    det_r = O.detect(x, g["w"], g["tau"], noise="medmad")
    assert det_r.candidates == []


# ---------------------------------------------------------------- invariants
def test_identical_snapshots_give_no_change_value():
    """tLISI = 1 when the two difference images are the same (Sec. 2.1)."""
    x = np.repeat(synth.random_stack(1, 17, 23, 3), 6, axis=0)
    det = O.detect(x, 4, 3.0)
    assert np.all(det.tlisi == 1.0)
    assert np.all(det.scale == 0.0)
    assert det.candidates == []


def test_constant_offset_pair_gives_one():
    """x^(s+2) = x^(s) makes D^(s) = D^(s+1), whatever x^(s+1) is."""
    x = synth.random_stack(3, 12, 15, 5)
    x[2] = x[0]
    ut = O.unit_tiles(x, 0, 3)
    assert np.all(O.tlisi_from_tiles(ut, O.normaliser_M(x)) == 1.0)


def test_tlisi_in_unit_interval_for_nonnegative_images():
    """tLISI lies in [0, 1] (Sec. 2.1) for non-negative snapshots."""
    x = synth.random_stack(6, 20, 21, 7, kind="positive") * 5.0
    det = O.detect(x, 3, 3.0)
    assert np.all(det.tlisi >= 0.0) and np.all(det.tlisi <= 1.0)


def test_scale_invariance():
    """x -> a x scales D, Delta and M by a; r is unchanged; so are tLISI and z."""
    x = synth.random_stack(7, 24, 30, 11)
    x[np.abs(x) < 1e-3] = 0.5
    a = 3.75
    d1 = O.detect(x.astype(np.float64), 4, 2.0, branch=O.BRANCH_BOTH)
    d2 = O.detect(x.astype(np.float64) * a, 4, 2.0, branch=O.BRANCH_BOTH)
    np.testing.assert_allclose(d1.tlisi, d2.tlisi, rtol=0, atol=1e-13)
    np.testing.assert_allclose(d1.z, d2.z, rtol=1e-9, atol=1e-9)
    assert [c.key() for c in d1.candidates] == [c.key() for c in d2.candidates]


def test_z_does_not_depend_on_M():
    """M is one scalar for the whole stack, so it cancels in the z-score."""
    x = synth.random_stack(5, 30, 30, 13)
    ut = O.unit_tiles(x, 1, 5)
    M = O.normaliser_M(x)
    z1, _, _ = O.zscore_image(O.tlisi_from_tiles(ut, M))
    z2, _, _ = O.zscore_image(O.tlisi_from_tiles(ut, 7.0 * M))
    np.testing.assert_allclose(z1, z2, rtol=1e-6, atol=1e-6)


def test_M_is_global_over_the_stack():
    x = np.zeros((4, 4, 4), dtype=np.float32)
    x[3, 2, 2] = 9.0
    x[0, 0, 0] = -20.0
    assert O.normaliser_M(x) == 9.0
    assert O.normaliser_M(-np.ones((3, 2, 2))) == O.C


def test_single_pixel_tiles_closed_form():
    """w = 1: tLISI_i = 1 - Delta_i * Delta_i * r_i / M^2 per pixel."""
    x = synth.random_stack(3, 5, 6, 17).astype(np.float64)
    M = O.normaliser_M(x)
    ut = O.unit_tiles(x, 0, 1)
    t = O.tlisi_from_tiles(ut, M)
    for y in range(5):
        for xx in range(6):
            a, b, c = x[0, y, xx], x[1, y, xx], x[2, y, xx]
            d = abs(abs(c - b) - abs(b - a))
            xh = O.C if b == 0 else abs(b)
            r = min(d / xh, 1.0)
            assert t[y, xx] == pytest.approx(1.0 - d * d * r / (M * M), abs=1e-15)


def test_single_outlier_z_is_samuelson_bound():
    """Population std: one odd tile among T equal ones has z = sqrt(T - 1)."""
    v = np.full((7, 9), 0.25)
    v[3, 4] = 0.1
    z, _, _ = O.zscore_image(v)
    assert z[3, 4] == pytest.approx(math.sqrt(v.size - 1), rel=1e-12)
    assert z[0, 0] == pytest.approx(-1.0 / math.sqrt(v.size - 1), rel=1e-12)
    rng = np.random.default_rng(0)
    z2, _, _ = O.zscore_image(rng.uniform(size=(13, 11)))
    assert np.max(np.abs(z2)) <= math.sqrt(13 * 11 - 1) + 1e-12


def test_pulse_in_noise_seen_in_units_k_and_k_minus_2():
    """A pulse in snapshot k lights the units (k, k+1, k+2) and (k-2, k-1, k) but
    not (k-1, k, k+1), where both differences contain it (Sec. 2.1)."""
    rng = np.random.default_rng(5)
    L, n, w = 9, 40, 4
    x = rng.standard_normal((L, n, n))
    k, py, px = 4, 21, 13
    x[k, py, px] += 60.0
    det = O.detect(x, w, 5.0)
    hits = {c.snapshot for c in det.candidates if (c.y, c.x) == (py, px)}
    assert hits == {k - 2, k}
    near = [c for c in det.candidates if c.snapshot == k - 1
            and abs(c.y - py) < w and abs(c.x - px) < w]
    assert near == []


def test_ratio_clip_and_zero_guard():
    """r <= 1 always (Eq. 4); a zero reference uses C (Eq. 5)."""
    a = np.array([[0.0, 1.0, 5.0]])
    b = np.array([[0.0, 0.0, 1.0]])
    c = np.array([[0.0, 3e-7, 0.0]])
    d, r, f = O.unit_terms(a, b, c)
    # pixel 0: all zero -> Delta 0, r 0; pixel 1: Delta=|3e-7-1| over C -> clipped 1;
    # pixel 2: D0=4, D1=1, Delta=3 over |1| -> clipped 1
    np.testing.assert_allclose(d[0], [0.0, 1.0 - 3e-7, 3.0])
    np.testing.assert_allclose(r[0], [0.0, 1.0, 1.0])
    d2, r2, _ = O.unit_terms(np.array([[0.0]]), np.array([[0.0]]), np.array([[5e-7]]))
    assert r2[0, 0] == pytest.approx(0.5)
    assert f.all()


def test_signed_reading_follows_literal_eq4():
    _, r, _ = O.unit_terms(np.array([[0.0]]), np.array([[-2.0]]), np.array([[-2.5]]))
    # D0 = 2, D1 = 0.5, Delta = 1.5, Delta / x-hat = 1.5 / -2 = -0.75 < 1
    _, rs, _ = O.unit_terms(np.array([[0.0]]), np.array([[-2.0]]), np.array([[-2.5]]), "signed")
    assert r[0, 0] == pytest.approx(0.75)
    assert rs[0, 0] == pytest.approx(-0.75)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("kind", ["normal", "integers", "zeros"])
@pytest.mark.parametrize("shape,w", [((4, 7, 9), 3), ((5, 8, 8), 4), ((3, 5, 11), 2), ((4, 6, 6), 6)])
def test_tiles_against_pixel_loops(kind, shape, w):
    """Vectorised tiling (padding, transposes, arg-max mapping) against loops."""
    x = synth.random_stack(*shape, seed=sum(shape) + w, kind=kind).astype(np.float64)
    L, ny, nx = shape
    for s in range(L - 2):
        ut = O.unit_tiles(x, s, w)
        Ty, Tx = -(-ny // w), -(-nx // w)
        for ty in range(Ty):
            for tx in range(Tx):
                S1 = S3 = 0.0
                best, by, bx, cnt = -1.0, -1, -1, 0
                for y in range(ty * w, min(ny, ty * w + w)):
                    for xx in range(tx * w, min(nx, tx * w + w)):
                        a, b, c = x[s, y, xx], x[s + 1, y, xx], x[s + 2, y, xx]
                        dd = abs(abs(c - b) - abs(b - a))
                        xh = O.C if b == 0 else abs(b)
                        rr = dd / xh if dd / xh < 1 else 1.0
                        S1 += dd
                        S3 += rr
                        cnt += 1
                        if dd > best:
                            best, by, bx = dd, y, xx
                assert ut.S1[ty, tx] == pytest.approx(S1, abs=1e-12)
                assert ut.S2[ty, tx] == best
                assert ut.S3[ty, tx] == pytest.approx(S3, abs=1e-12)
                assert ut.n[ty, tx] == cnt
                assert (ut.arg_y[ty, tx], ut.arg_x[ty, tx]) == (by, bx)


def test_nonfinite_pixels_invalidate_their_tiles():
    x = synth.random_stack(5, 8, 8, 21)
    x[2, 1, 6] = np.nan
    x[4, 7, 0] = np.inf
    det = O.detect(x, 4, 2.0)
    # unit s touches snapshots s..s+2
    for s in range(3):
        assert np.isnan(det.tlisi[s, 0, 1]) == (s <= 2)
        assert np.isnan(det.tlisi[s, 1, 0]) == (s == 2)
    assert np.isfinite(det.tlisi[:, 1, 1]).all()
    assert np.isfinite(det.M)


def test_drop_edge_crops_to_whole_tiles():
    x = synth.random_stack(4, 10, 11, 23)
    d = O.detect(x, 3, 2.0, edge="drop")
    ref = O.detect(x[:, :9, :9], 3, 2.0)
    np.testing.assert_array_equal(d.tlisi, ref.tlisi)


# ---------------------------------------------------------------- noise / threshold
def test_lower_median_and_mad_constant():
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 10, 101, 1000):
        v = rng.standard_normal(n)
        assert O.lower_median(v) == statistics.median_low(v.tolist())
    from scipy.stats import norm
    assert O.MAD_TO_SIGMA == pytest.approx(1.0 / norm.ppf(0.75), rel=1e-15)


def test_medmad_scale_of_gaussian():
    rng = np.random.default_rng(4)
    med, scale, n = O.noise_medmad(rng.standard_normal(400_001))
    assert abs(med) < 0.01 and abs(scale - 1.0) < 0.01


@pytest.mark.parametrize("noise", ["meanstd", "medmad"])
@pytest.mark.parametrize("tau", [3.0, 4.0])
def test_gaussian_tail_false_positive_rate(noise, tau):
    """Exceedances of z > tau on N(0,1) match Q(tau) within a 4-sigma interval."""
    from scipy.special import erfc
    n = 20_000_000
    v = np.random.default_rng(int(tau * 10) + len(noise)).standard_normal(n)
    k = O.threshold_count(v, tau, noise)
    q = 0.5 * erfc(tau / math.sqrt(2.0))
    mean, sd = n * q, math.sqrt(n * q * (1 - q))
    slack = 4 * sd + (0.002 * n * q if noise == "medmad" else 0.0)
    assert abs(k - mean) <= slack, (k, mean, sd)


def test_strict_threshold():
    z = np.array([[2.0, 2.0000001, np.nan]])
    np.testing.assert_array_equal(O.select(z, 2.0), [[False, True, False]])


# ---------------------------------------------------------------- components
def test_components_match_scipy_label():
    from scipy import ndimage
    rng = np.random.default_rng(9)
    for trial in range(20):
        m = rng.uniform(size=(23, 31)) < (0.05 + 0.02 * trial)
        comps = O.components(m)
        lab, n = ndimage.label(m, structure=np.ones((3, 3), dtype=int))
        assert len(comps) == n
        for comp in comps:
            labels = {lab[p] for p in comp}
            assert len(labels) == 1
            assert len(comp) == int(np.count_nonzero(lab == labels.pop()))


def test_component_peak_tie_breaks_to_smallest_index():
    z = np.zeros((3, 3))
    z[1, 2] = z[2, 0] = 5.0
    assert O.component_peak([(2, 0), (1, 2), (1, 1)], z) == (1, 2)


# ---------------------------------------------------------------- frequency branch
def test_dft_matches_numpy_fft():
    rng = np.random.default_rng(12)
    for n in (4, 7, 62, 64, 127):
        y = rng.standard_normal((5, n))
        want = np.abs(np.fft.rfft(y - y.mean(axis=1, keepdims=True), axis=1))[:, 1:n // 2 + 1]
        np.testing.assert_allclose(O.dft_magnitudes(y), want, rtol=1e-11, atol=1e-11)


def test_dft_removes_dc_and_ignores_offsets():
    y = np.arange(10.0)
    np.testing.assert_allclose(O.dft_magnitudes(y), O.dft_magnitudes(y + 123.0), atol=1e-10)


@pytest.mark.parametrize("period,phase", [(4, 1), (8, 3), (16, 0)])
def test_period_recovery(period, phase):
    """A tile pulsing once per period P (P | n) peaks at a multiple of n/P."""
    L = 66
    n = L - 2
    x = synth.periodic_tile_stack(L, 24, 24, 4, period, phase, (2, 3), 40.0, seed=period)
    det = O.detect(x, 4, 5.0, branch=O.BRANCH_FREQ)
    ty, tx = 2, 3
    assert det.eta_z[ty, tx] == np.nanmax(det.eta_z)
    assert det.eta_bin[ty, tx] % (n // period) == 0
    top = max(det.candidates, key=lambda c: c.significance)
    assert (top.y // 4, top.x // 4) == (ty, tx)
    assert top.snapshot == -1 and top.branch == O.BRANCH_FREQ


def test_parabolic_offset_finds_vertex():
    for v in (-0.4, -0.1, 0.0, 0.25, 0.49):
        f = lambda t: 3.0 - 2.0 * (t - v) ** 2
        assert O.parabolic_offset(f(-1), f(0), f(1)) == pytest.approx(v, abs=1e-12)
    assert O.parabolic_offset(1.0, 1.0, 1.0) == 0.0
    assert O.parabolic_offset(np.nan, 2.0, 1.0) == 0.0


def test_freq_candidate_is_tile_centre():
    x = synth.periodic_tile_stack(34, 20, 26, 5, 4, 2, (1, 4), 50.0, seed=2)
    # 24 tiles: a lone outlier reaches at most z = sqrt(23) ~ 4.8
    det = O.detect(x, 5, 3.0, branch=O.BRANCH_FREQ)
    top = max(det.candidates, key=lambda c: c.significance)
    # tile (1, 4) spans rows 5..9 and columns 20..24: centre (7, 22)
    assert (top.y, top.x) == (7, 22)
    assert abs(top.xf - 22.0) <= 2.5 and abs(top.yf - 7.0) <= 2.5


# ---------------------------------------------------------------- sliding windows
@pytest.mark.parametrize("shape,w", [((4, 7, 9), 3), ((3, 6, 5), 5), ((5, 9, 8), 1), ((3, 4, 11), 7)])
def test_sliding_windows_against_pixel_loops(shape, w):
    x = synth.random_stack(*shape, seed=w + 100, kind="zeros").astype(np.float64)
    L, ny, nx = shape
    h = w // 2
    for s in range(L - 2):
        ut = O.unit_windows(x, s, w)
        for y in range(ny):
            for xx in range(nx):
                S1 = S3 = 0.0
                best, cnt = -1.0, 0
                for qy in range(max(0, y - h), min(ny, y + h + 1)):
                    for qx in range(max(0, xx - h), min(nx, xx + h + 1)):
                        a, b, c = x[s, qy, qx], x[s + 1, qy, qx], x[s + 2, qy, qx]
                        dd = abs(abs(c - b) - abs(b - a))
                        xh = O.C if b == 0 else abs(b)
                        S1 += dd
                        S3 += dd / xh if dd / xh < 1 else 1.0
                        best = max(best, dd)
                        cnt += 1
                assert ut.S1[y, xx] == pytest.approx(S1, abs=1e-12)
                assert ut.S2[y, xx] == best
                assert ut.S3[y, xx] == pytest.approx(S3, abs=1e-12)
                assert ut.n[y, xx] == cnt


def test_sliding_w1_is_the_single_pixel_tiling():
    x = synth.random_stack(5, 13, 17, 41)
    a = O.detect(x, 1, 3.0, O.BRANCH_BOTH, stride="sliding")
    b = O.detect(x, 1, 3.0, O.BRANCH_BOTH)
    np.testing.assert_array_equal(a.tlisi, b.tlisi)
    assert [c.key() for c in a.candidates] == [c.key() for c in b.candidates]


def test_sliding_window_counts_are_clipped_at_the_border():
    delta = np.ones((6, 9))
    ut = O.window_stats(delta, delta * 0.5, np.ones((6, 9), bool), 5)
    assert ut.n[0, 0] == 9 and ut.n[0, 4] == 15 and ut.n[3, 4] == 25 and ut.n[5, 8] == 9
    np.testing.assert_allclose(ut.numerator, 0.5)   # mean 1 * max 1 * mean 0.5


def test_sliding_pulse_lights_the_windows_around_it():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((6, 40, 40)) * 0.01
    x[3, 20, 25] += 50.0
    det = O.detect(x, 5, 5.0, stride="sliding")
    # every window holding the pulse has about the same statistic, so the peak
    # of the plateau lies anywhere within the window radius of the pulse
    assert sorted(c.snapshot for c in det.candidates) == [1, 3]
    for c in det.candidates:
        assert abs(c.y - 20) <= 2 and abs(c.x - 25) <= 2


# ---------------------------------------------------------------- running M (real-time reading)
def _spiked_stack(L=7, ny=12, nx=15, amps=None, seed=4):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, (L, ny, nx)).clip(-4.0, 4.0)
    for k, a in enumerate(amps or []):
        x[k, 0, 0] = a
    return x


def test_running_M_is_the_cumulative_maximum():
    amps = [10.0 + k for k in range(7)]            # the spike grows every snapshot
    det = O.detect(_spiked_stack(amps=amps), 3, 3.0, mmode="running")
    # unit s sees snapshots 0..s+2, whose largest pixel is the spike of s+2
    assert list(det.M_units) == [amps[s + 2] for s in range(5)]
    assert det.M == amps[-1]
    glob = O.detect(_spiked_stack(amps=amps), 3, 3.0)
    assert list(glob.M_units) == [amps[-1]] * 5


def test_running_equals_global_when_the_maximum_comes_first():
    x = _spiked_stack(amps=[0.0, 50.0])            # the stack's maximum is in snapshot 1
    a = O.detect(x, 3, 2.5, O.BRANCH_BOTH, mmode="running")
    b = O.detect(x, 3, 2.5, O.BRANCH_BOTH)
    assert np.array_equal(a.tlisi, b.tlisi, equal_nan=True)
    assert [c.key() for c in a.candidates] == [c.key() for c in b.candidates]


def test_running_M_leaves_image_candidates_unchanged():
    # z uses one unit's tiles, so a per-unit constant M_s cancels (Sec. 2.4.1)
    x = _spiked_stack(L=9, ny=30, nx=33, amps=[5.0 + 2 * k for k in range(9)], seed=9)
    a = O.detect(x, 3, 2.0, mmode="running")
    b = O.detect(x, 3, 2.0)
    assert [c.key() for c in a.candidates] == [c.key() for c in b.candidates]
    for ca, cb in zip(a.candidates, b.candidates):
        assert ca.significance == pytest.approx(cb.significance, rel=1e-9)


def test_running_M_series_spectrum_closed_form():
    """Six snapshots give a 4-point series per tile; its DFT bins are
    X1 = (y0 - y2) - i (y1 - y3) and X2 = y0 - y1 + y2 - y3."""
    amps = [10.0, 10.5, 11.0, 12.0, 13.5, 15.0]
    x = _spiked_stack(L=6, ny=9, nx=9, amps=amps, seed=21)
    for mmode in ("global", "running"):
        det = O.detect(x, 3, 1.0, O.BRANCH_FREQ, mmode=mmode)
        for ty in range(3):
            for tx in range(3):
                y = det.tlisi[:, ty, tx]
                x1 = math.hypot(y[0] - y[2], y[1] - y[3])
                x2 = abs(y[0] - y[1] + y[2] - y[3])
                assert det.eta[ty, tx] == pytest.approx(max(x1, x2), rel=1e-12, abs=1e-15)
                assert det.eta_bin[ty, tx] == (1 if x1 >= x2 else 2)


def test_running_M_brings_out_a_steady_tile_in_the_spectrum():
    """A tile whose statistic v is the same in every unit has a flat series
    under the global M (eta = 0) but not when M grows between units."""
    L, w = 6, 2
    x = np.full((L, 2, 4), 1.0)
    x[:, 0, 2] = [0.0, 1.0, 1.0, 0.0, 0.0, 1.0]    # tile (0, 1): Delta = r = 1 in every unit
    x[:, 1, 0] = [4.0, 4.0, 5.0, 6.0, 7.0, 8.0]    # tile (0, 0) carries the growing maximum
    g = O.detect(x, w, 1.0, O.BRANCH_FREQ)
    r = O.detect(x, w, 1.0, O.BRANCH_FREQ, mmode="running")
    v = np.array([u.numerator[0, 1] for u in g.units])
    assert np.all(v == v[0]) and v[0] > 0
    assert g.eta[0, 1] == 0.0
    assert list(r.M_units) == [5.0, 6.0, 7.0, 8.0]
    assert r.eta[0, 1] > 0.0


# ---------------------------------------------------------------- accumulation
def test_accumulate_block_sums_closed_form():
    """Sec. 3.3.2: snapshot j of the accumulated stack is the sum of raw
    snapshots jK .. jK+K-1; with raw snapshot r = r everywhere the sum is
    K^2 j + K(K-1)/2, and an incomplete last block is dropped."""
    raw = np.broadcast_to(np.arange(23, dtype=np.float64)[:, None, None], (23, 3, 4)).copy()
    for k in (1, 2, 5, 7):
        acc = O.accumulate(raw, k)
        assert acc.shape == (23 // k, 3, 4)
        for j in range(acc.shape[0]):
            assert np.all(acc[j] == k * k * j + k * (k - 1) // 2)
    assert np.array_equal(O.accumulate(raw, 1), raw)


def test_accumulate_of_repeated_snapshots_is_scaled_stack():
    """Raw snapshots each repeated K times sum to K x the stack: the same
    candidates and z-scores (the statistic's scale invariance)."""
    stack, _ = synth.make_stack(synth.small_spec(8, 60, 64, n_steady=5, n_pulsed=2,
                                                 pulse_period=(3, 4)), seed=4, device="cpu")
    x = stack.numpy().astype(np.float64)
    raw = np.repeat(x, 4, axis=0)
    acc = O.accumulate(raw, 4)
    assert np.array_equal(acc, 4.0 * x)
    a = O.detect(x, 5, 3.0)
    b = O.detect(acc, 5, 3.0)
    assert [(c.snapshot, c.y, c.x) for c in a.candidates] == \
        [(c.snapshot, c.y, c.x) for c in b.candidates]
    for ca, cb in zip(a.candidates, b.candidates):
        assert cb.significance == pytest.approx(ca.significance, rel=1e-9)


def test_accumulation_reveals_pulse_too_faint_per_snapshot():
    """The paper's case for accumulation: a pulse of 3 sigma lasting K = 16
    raw snapshots once every 48 is never selected among the raw snapshots,
    whose neighbours barely differ; summed in blocks of 16 it stands at 12
    sigma in one accumulated snapshot of every three and is selected at its
    pixel, only in units that hold it at their first or last snapshot."""
    rs = np.random.default_rng(5)
    k, n_acc, ny, nx, w = 16, 12, 48, 48, 4
    raw = rs.standard_normal((n_acc * k, ny, nx))
    py, px = 21, 30
    on = (np.arange(n_acc * k) % (3 * k)) < k
    raw[on, py, px] += 3.0
    plain = O.detect(raw, w, 6.0, O.BRANCH_IMAGE, "meanstd")
    assert not [c for c in plain.candidates if (c.y, c.x) == (py, px)]
    acc = O.detect(O.accumulate(raw, k), w, 6.0, O.BRANCH_IMAGE, "meanstd")
    units = {c.snapshot for c in acc.candidates if (c.y, c.x) == (py, px)}
    assert units <= {0, 1, 3, 4, 6, 7, 9} and len(units) >= 5


# ---------------------------------------------------------------- real-time frequency window
def test_freq_window_over_all_units_is_the_batch_frequency_branch():
    """With the window covering every unit, and the stack's maximum in its
    first three snapshots (so the running M is the global M at every unit),
    the real-time window gives the batch frequency branch exactly."""
    x = synth.periodic_tile_stack(26, 40, 43, 4, 4, 1, (2, 3), 6.0, seed=31)
    x[0, 0, 0] = 10.0 * np.abs(x).max()   # the maximum comes first
    cands, eta, kbin, z = O.freq_window(x, 4, 4.0, 24, "medmad")
    det = O.detect(x, 4, 4.0, O.BRANCH_FREQ, "medmad")
    assert np.array_equal(eta, det.eta) and np.array_equal(kbin, det.eta_bin)
    assert [(c.y, c.x, c.freq_bin) for c in cands] == \
        [(c.y, c.x, c.freq_bin) for c in det.candidates]
    assert all(c.snapshot == 23 for c in cands)


def test_spectrum_magnitudes_ignore_circular_time_shifts():
    """|X_k| of a circularly shifted series equals that of the series (the
    shift multiplies X_k by a phase): a ring of unit maps in any rotation has
    the same eta and bin."""
    rs = np.random.default_rng(17)
    cube = rs.random((14, 6, 7))
    eta, kbin = O.spectrum(cube)
    for r in (1, 5, 13):
        e2, k2 = O.spectrum(np.roll(cube, r, axis=0))
        np.testing.assert_allclose(e2, eta, rtol=1e-12, atol=0)
        assert np.array_equal(k2, kbin)


def test_freq_window_recovers_period_of_recent_pulses():
    """A pulse of period 4 in the last 16 units of a 30-unit stack shows at bin
    16/4 = 4 of a 16-unit window, at its tile."""
    rs = np.random.default_rng(3)
    L, ny, nx, w = 32, 24, 24, 4
    x = 5.0 + 0.01 * rs.standard_normal((L, ny, nx))
    for s in range(L - 18, L):
        if s % 4 == 1:
            x[s, 10, 14] += 3.0
    cands, eta, kbin, z = O.freq_window(x, w, 4.0, 16, "meanstd")
    assert kbin[10 // w, 14 // w] % 4 == 0
    assert any((c.y // w, c.x // w) == (10 // w, 14 // w) for c in cands)


# ---------------------------------------------------------------- harmonic summing
def _one_tile_cube(series):
    return np.asarray(series, dtype=np.float64)[:, None, None]


@pytest.mark.parametrize("amps,k0,m_max,want_eta,want_k", [
    # y_s = sum_j a_j cos(2 pi j k0 s / n), n = 64: |X_(j k0)| = n a_j / 2 exactly
    # (want_k None: equal sums at several bins, which rounding orders)
    ([1, 1, 1, 1], 2, 1, 32.0, None),
    ([1, 1, 1, 1], 2, 2, 64.0 / math.sqrt(2), None),
    ([1, 1, 1, 1], 2, 4, 64.0, 2),
    ([1, 1, 1, 1], 2, 16, 64.0, 2),
    ([1.0, 0.5, 0.25, 0.0], 3, 4, 48.0 / math.sqrt(2), 3),   # S_2 = 48/sqrt 2 beats S_1, S_4
    ([1.0, 0.3, 0.1, 0.0], 3, 4, 32.0, 3),                   # S_1 = 32 beats S_2, S_4
    ([0.2, 1.0, 1.0, 1.0], 2, 4, (6.4 + 96.0) / 2, 2),       # the weak fundamental counts
])
def test_harmonic_sum_of_cosines_closed_form(amps, k0, m_max, want_eta, want_k):
    n = 64
    s = np.arange(n)
    y = sum(a * np.cos(2 * np.pi * (j + 1) * k0 * s / n) for j, a in enumerate(amps))
    eta, kbin = O.spectrum(_one_tile_cube(y), harmonics=m_max)
    assert eta[0, 0] == pytest.approx(want_eta, rel=1e-12, abs=1e-9)
    if want_k is not None:
        assert kbin[0, 0] == want_k


@pytest.mark.parametrize("m_max,want_eta,want_k", [(1, 8.0, 8), (2, 16 / math.sqrt(2), 8),
                                                   (4, 16.0, 8), (8, 16.0, 8)])
def test_harmonic_sum_of_pulse_comb_includes_nyquist(m_max, want_eta, want_k):
    """A comb of period 8 over n = 64 has |X_k| = 8 at k = 8, 16, 24, 32 (32 =
    Nyquist) and 0 elsewhere; four harmonics of k = 8 give 4 * 8 / 2 = 16."""
    n = 64
    y = (np.arange(n) % 8 == 0).astype(np.float64)
    eta, kbin = O.spectrum(_one_tile_cube(y), harmonics=m_max)
    assert eta[0, 0] == pytest.approx(want_eta, rel=1e-12)
    assert kbin[0, 0] == want_k


def test_harmonic_sum_with_one_harmonic_is_the_maximum_magnitude():
    rng = np.random.default_rng(4)
    cube = rng.standard_normal((37, 5, 6))
    e1, k1 = O.spectrum(cube, harmonics=1)
    mags = O.dft_magnitudes(np.moveaxis(cube, 0, -1).reshape(30, 37))
    e, k = O.harmonic_sum(mags, 1)
    assert np.array_equal(e.reshape(5, 6), e1) and np.array_equal(k.reshape(5, 6), k1)


def test_harmonic_sum_grows_with_m_max_and_is_bounded():
    """More harmonics only add candidates to the maximum, and each S_m(k) is at
    most sqrt(m) times the largest magnitude."""
    rng = np.random.default_rng(9)
    cube = rng.standard_normal((126, 4, 4))
    mags = O.dft_magnitudes(np.moveaxis(cube, 0, -1).reshape(16, 126))
    prev = None
    for m_max in (1, 2, 4, 8, 16, 32):
        e, _ = O.spectrum(cube, harmonics=m_max)
        if prev is not None:
            assert np.all(e >= prev)
        assert np.all(e.ravel() <= math.sqrt(m_max) * mags.max(axis=1) * (1 + 1e-12))
        prev = e


def test_harmonic_sum_brute_force_on_tiny_spectra():
    """Every (m, k) written out for K = 6 against a hand enumeration."""
    mags = np.array([[3.0, 1.0, 2.0, 4.0, 0.5, 2.5]])
    cands = {(1, k): mags[0, k - 1] for k in range(1, 7)}
    cands.update({(2, 1): (3 + 1) / math.sqrt(2), (2, 2): (1 + 4) / math.sqrt(2),
                  (2, 3): (2 + 2.5) / math.sqrt(2)})
    cands.update({(4, 1): (3 + 1 + 2 + 4) / 2.0})
    best = max(cands.items(), key=lambda kv: (kv[1], -kv[0][0], -kv[0][1]))
    e, k = O.harmonic_sum(mags, 8)
    assert e[0] == pytest.approx(best[1], rel=1e-15) and k[0] == best[0][1] == 1
    e, k = O.harmonic_sum(mags, 2)
    assert e[0] == pytest.approx(4.0) and k[0] == 4


def test_harmonic_summing_finds_a_pulse_train_missed_by_the_maximum():
    """A narrow periodic pulse spreads its power over many harmonics, so the
    harmonic sum raises the pulsar tile's eta more than a noise tile's."""
    rng = np.random.default_rng(11)
    n, P = 128, 16
    cube = rng.standard_normal((n, 8, 8))
    cube[np.arange(n) % P == 3, 2, 5] += 2.0
    z1 = O.zscore_map(O.spectrum(cube, 1)[0])[0][2, 5]
    z8 = O.zscore_map(O.spectrum(cube, 8)[0])[0][2, 5]
    assert z8 > z1 + 1.0


# ---------------------------------------------------------------- spline refine of eta
@pytest.mark.parametrize("x0", [-0.5, -0.37, -0.1, 0.0, 0.23, 0.41, 0.5])
def test_cubic_refine_reproduces_a_parabola(x0):
    """Catmull-Rom splines reproduce quadratics, so samples of a parabola refine
    to its vertex exactly, as the three-point parabola does."""
    q = lambda x: 7.0 - 3.0 * (x - x0) ** 2
    s = [q(x) for x in (-2, -1, 0, 1, 2)]
    assert O.cubic_offset(*s) == pytest.approx(x0, abs=1e-12)
    assert O.parabolic_offset(s[1], s[2], s[3]) == pytest.approx(x0, abs=1e-12)


def test_cubic_refine_against_a_hermite_spline():
    """The same spline as scipy's cubic Hermite interpolant with Catmull-Rom
    (central-difference) tangents, maximised on a dense grid over [-0.5, 0.5]."""
    from scipy.interpolate import CubicHermiteSpline
    rng = np.random.default_rng(17)
    grid = np.linspace(-0.5, 0.5, 200001)
    checked = 0
    for _ in range(400):
        y = rng.standard_normal(5)
        y[2] += 1.5                       # a peak near the centre, as for a selected tile
        yi = y[1:4]
        m = 0.5 * (y[2:5] - y[0:3])       # tangents at -1, 0, 1
        f = CubicHermiteSpline([-1.0, 0.0, 1.0], yi, m)(grid)
        top = np.sort(f)[-1]
        # skip near ties between two separate maxima (either answer is right)
        far = np.abs(grid - grid[np.argmax(f)]) > 0.02
        if far.any() and f[far].max() > top - 1e-9:
            continue
        x = O.cubic_offset(*y)
        assert x == pytest.approx(grid[np.argmax(f)], abs=2e-5)
        checked += 1
    assert checked > 350


def test_cubic_refine_edges_and_degenerate_samples():
    assert O.cubic_offset(1.0, 2.0, 3.0, 2.0, 1.0) == 0.0            # symmetric
    assert O.cubic_offset(0.0, 1.0, 2.0, 3.0, 4.0) == 0.5            # rising line: right end
    assert O.cubic_offset(4.0, 3.0, 2.0, 1.0, 0.0) == -0.5           # falling line: left end
    assert O.cubic_offset(1.0, 5.0, 3.0, np.nan, np.nan) < 0.0       # no right neighbour
    assert O.cubic_offset(np.nan, np.nan, 3.0, 5.0, 1.0) > 0.0       # no left neighbour
    assert O.cubic_offset(np.nan, np.nan, 3.0, np.nan, np.nan) == 0.0
    assert O.cubic_offset(1.0, 2.0, np.nan, 2.0, 1.0) == 0.0
    # a missing outer sample is the linear extension 2 f(+-1) - f(0)
    a = O.cubic_offset(0.3, 2.0, 3.0, 2.6, np.nan)
    b = O.cubic_offset(0.3, 2.0, 3.0, 2.6, 2 * 2.6 - 3.0)
    assert a == b


def test_cubic_refine_moves_a_freq_candidate_towards_the_source():
    """A pulsed source off the tile centre leaks into the neighbouring tiles;
    both refines move the candidate from the centre towards it."""
    w = 8
    x = synth.periodic_tile_stack(40, 48, 48, w, 4, 1, (2, 2), 0.0, seed=3, noise=0.3)
    x[np.arange(40) % 4 == 1, 20:26, 21:29] += 6.0     # straddles tiles (2, 2) and (2, 3)
    for refine in ("parabolic", "cubic"):
        det = O.detect(x, w, 4.0, O.BRANCH_FREQ, refine=refine)
        c = [c for c in det.candidates if (c.y // w, c.x // w) == (2, 2) or (c.y // w, c.x // w) == (2, 3)]
        assert c, refine
        assert c[0].xf != c[0].x


@pytest.mark.parametrize("harmonics,refine", [(4, "parabolic"), (8, "cubic"), (1, "cubic")])
def test_freq_window_matches_the_batch_branch_with_harmonics_and_refine(harmonics, refine):
    """The real-time window over every unit equals the batch frequency branch
    for the harmonic sum and the spline refine too (same eta, bins, candidate
    positions)."""
    x = synth.periodic_tile_stack(34, 40, 43, 4, 4, 1, (2, 3), 6.0, seed=37)
    x[0, 0, 0] = 10.0 * np.abs(x).max()
    cands, eta, kbin, z = O.freq_window(x, 4, 4.0, 32, "meanstd", harmonics=harmonics,
                                        refine=refine)
    det = O.detect(x, 4, 4.0, O.BRANCH_FREQ, "meanstd", harmonics=harmonics, refine=refine)
    assert np.array_equal(eta, det.eta) and np.array_equal(kbin, det.eta_bin)
    assert [(c.y, c.x, c.freq_bin, c.xf, c.yf) for c in cands] == \
        [(c.y, c.x, c.freq_bin, c.xf, c.yf) for c in det.candidates]
    assert cands


# ---------------------------------------------------------------- sampled tiles
def _tile_by_pixel_loops(x, s, w, ty, tx, nyu, nxu):
    """S1, S2, S3, n, valid and the first arg-max of Delta of one tile of unit
    s, by a loop over its pixels (Eq. 3-5 written out per pixel)."""
    S1 = S3 = 0.0
    best, by, bx, cnt, valid = -1.0, -1, -1, 0, True
    for y in range(ty * w, min(nyu, ty * w + w)):
        for xx in range(tx * w, min(nxu, tx * w + w)):
            a, b, c = (float(x[s + i, y, xx]) for i in range(3))
            cnt += 1
            if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
                valid = False
                continue
            dd = abs(abs(c - b) - abs(b - a))
            xh = O.C if b == 0 else abs(b)
            rr = dd / xh if dd / xh < 1 else 1.0
            S1 += dd
            S3 += rr
            if dd > best:
                best, by, bx = dd, y, xx
    return S1, best, S3, cnt, valid, by, bx


@pytest.mark.parametrize("edge", ["partial", "drop"])
@pytest.mark.parametrize("kind", ["normal", "integers", "zeros"])
@pytest.mark.parametrize("shape,w", [((5, 13, 17), 4), ((4, 9, 10), 3), ((6, 11, 7), 5)])
def test_sampled_tiles_against_pixel_loops_and_unit_tiles(edge, kind, shape, w):
    """The per-tile sampler that checks the library at full size: every tile's
    S1, S2, S3, n, numerator, validity and absolute arg-max pixel equal a pixel
    loop over that tile, and equal the whole-image tiling, on ragged grids
    (the last tile row and column are partial under EDGE_PARTIAL), ties and
    zeros, with a non-finite pixel in one tile."""
    x = synth.random_stack(*shape, seed=sum(shape) * 7 + w, kind=kind).astype(np.float64)
    x[2, shape[1] // 2, shape[2] - 1] = np.nan
    L, ny, nx = shape
    Ty, Tx, nyu, nxu = O.tiling(ny, nx, w, edge)
    tiles = [(ty, tx) for ty in range(Ty) for tx in range(Tx)]
    rng = np.random.default_rng(len(tiles))
    tiles = [tiles[i] for i in rng.permutation(len(tiles))]   # order must not matter
    got = O.sampled_tiles(x, w, tiles, edge=edge)
    for s in range(L - 2):
        ut = O.unit_tiles(x, s, w, edge=edge)
        for j, (ty, tx) in enumerate(tiles):
            S1, S2, S3, n, valid, by, bx = _tile_by_pixel_loops(x, s, w, ty, tx, nyu, nxu)
            assert got["n"][s, j] == n == ut.n[ty, tx]
            assert got["valid"][s, j] == valid == ut.valid[ty, tx]
            if not valid:
                assert np.isnan(got["numerator"][s, j])
                continue
            assert got["S1"][s, j] == pytest.approx(S1, rel=1e-13, abs=1e-300)
            assert got["S2"][s, j] == S2
            assert got["S3"][s, j] == pytest.approx(S3, rel=1e-13, abs=1e-300)
            assert (got["arg_y"][s, j], got["arg_x"][s, j]) == (by, bx)
            assert (got["arg_y"][s, j], got["arg_x"][s, j]) == (ut.arg_y[ty, tx], ut.arg_x[ty, tx])
            want_v = (S1 / n) * S2 * (S3 / n)
            assert got["numerator"][s, j] == pytest.approx(want_v, rel=1e-12, abs=1e-300)
            assert got["numerator"][s, j] == pytest.approx(ut.numerator[ty, tx], rel=1e-12,
                                                           abs=1e-300)


# ---------------------------------------------------------------- difference-coded half storage
_UH = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}   # half unit roundoff (8 / 11 significant bits)
_U32 = 2.0 ** -24


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_round_half_is_torch_round_to_nearest_even(fmt):
    """round_half equals torch's FP32 -> BF16/FP16 conversion (round to
    nearest, ties to even) on random values, exact ties, the largest finite
    values, subnormals, infinities and NaN."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.normal(size=20000) * 10.0 ** rng.uniform(-8, 8, size=20000),
        # halfway between neighbouring BF16 numbers (odd and even kept patterns)
        (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32),
        # halfway between neighbouring FP16 numbers near 1
        1.0 + (np.arange(1, 200) + 0.5) * 2.0 ** -10,
        [65504.0, 65519.0, 65520.0, 3.3e38, 3.4028235e38, 1e-40, -1e-42, 6e-8, 3e-8,
         np.inf, -np.inf, 0.0, -0.0],
    ]).astype(np.float32)
    tdt = torch.bfloat16 if fmt == "bf16" else torch.float16
    want = torch.from_numpy(x).to(tdt).to(torch.float32).numpy()
    got = O.round_half(x, fmt)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.isnan(O.round_half(np.array([np.nan], np.float32), fmt)[0])


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_delta_coding_exact_when_differences_are_representable(fmt):
    """Integer snapshots whose frame-to-frame differences fit in the half
    format (|d| <= 256) decode to themselves bit for bit, whatever the
    absolute level (up to 2^20 here, far beyond the half formats)."""
    rng = np.random.default_rng(4)
    base = rng.integers(-2 ** 20, 2 ** 20, size=(1, 9, 11))
    steps = rng.integers(-256, 257, size=(12, 9, 11))
    steps[0] = 0
    x = (base + np.cumsum(steps, axis=0)).astype(np.float32)
    key, q = O.delta_encode(x, fmt)
    assert np.array_equal(key, x[0])
    assert np.array_equal(q[1:], np.diff(x, axis=0))
    assert np.array_equal(O.delta_decode(key, q), x)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_delta_coding_error_is_one_rounding_per_snapshot(fmt):
    """Closed loop: every decoded snapshot is within one half rounding of its
    own frame-to-frame difference (plus FP32 roundings) of the original, on a
    300-snapshot random walk on a 500-sigma sky, so the error does not grow
    with the snapshot index (an open-loop coder of x^(s) - x^(s-1) drifts)."""
    rng = np.random.default_rng(5)
    L = 300
    sky = rng.uniform(-20, 500, size=(16, 16))
    x = (sky + np.cumsum(rng.normal(size=(L, 16, 16)), axis=0) * 0.1
         + rng.normal(size=(L, 16, 16))).astype(np.float32)
    key, q = O.delta_encode(x, fmt)
    xt = O.delta_decode(key, q)
    assert np.array_equal(xt[0], x[0])
    prev = xt[0].astype(np.float64)
    for s in range(1, L):
        d = x[s].astype(np.float64) - prev
        bound = (_UH[fmt] + _U32) * np.abs(d) * 1.0001 + _U32 * np.abs(xt[s]) * 1.0001
        err = np.abs(xt[s].astype(np.float64) - x[s].astype(np.float64))
        assert np.all(err <= bound), (s, float((err / bound).max()))
        prev = xt[s].astype(np.float64)
    # the open-loop alternative (rounding x^(s) - x^(s-1) itself) does drift
    qo = np.zeros_like(x)
    qo[1:] = O.round_half(np.diff(x, axis=0), fmt)
    drift = np.abs(O.delta_decode(key, qo).astype(np.float64) - x).max()
    assert drift > 4 * np.abs(xt.astype(np.float64) - x).max()


def test_delta_coding_of_a_steady_stack_stores_zeros():
    x = np.repeat(np.random.default_rng(6).normal(size=(1, 7, 9)).astype(np.float32) * 300, 6, 0)
    for fmt in ("bf16", "f16"):
        key, q = O.delta_encode(x, fmt)
        assert not q.any()
        assert np.array_equal(O.delta_decode(key, q), x)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_delta_coding_non_finite_pixel_poisons_only_its_later_snapshots(fmt):
    rng = np.random.default_rng(7)
    x = (rng.normal(size=(8, 5, 6)) + 40).astype(np.float32)
    y = x.copy()
    y[3, 2, 4] = np.nan
    y[5, 0, 1] = np.inf
    dx = O.delta_decode(*O.delta_encode(x, fmt))
    ky = O.delta_decode(*O.delta_encode(y, fmt))
    bad = np.zeros(x.shape, dtype=bool)
    bad[3:, 2, 4] = True
    bad[5:, 0, 1] = True
    assert np.all(~np.isfinite(ky[bad]))
    assert np.array_equal(ky[~bad], dx[~bad])


@pytest.mark.parametrize("fmt,p99_max", [("bf16", 2e-2), ("f16", 3e-3)])
def test_delta_coding_keeps_the_tile_statistic_accurate(fmt, p99_max):
    """On a dirty-image stack with steady sources up to 500 sigma, the tile
    statistic of the decoded stack stays within a fraction of a percent of
    the FP32 original's (p99 of the relative error), while rounding the
    values themselves to the half format is off by whole multiples."""
    spec = synth.small_spec(10, 200, 200, n_steady=40, n_pulsed=3, pulse_period=(3, 5))
    x, _ = synth.make_stack(spec, seed=8, device="cpu")
    x = x.numpy().astype(np.float32)

    def v(stack):
        return np.stack([O.unit_tiles(stack.astype(np.float64), s, 5).numerator
                         for s in range(stack.shape[0] - 2)])

    ref = v(x)
    key, q = O.delta_encode(x, fmt)
    rel_delta = np.abs(v(O.delta_decode(key, q)) - ref) / np.abs(ref)
    rel_value = np.abs(v(O.round_half(x, fmt)) - ref) / np.abs(ref)
    p99d, p99v = np.percentile(rel_delta, 99), np.percentile(rel_value, 99)
    assert p99d < p99_max, p99d
    assert p99v > 10 * p99d, (p99v, p99d)
