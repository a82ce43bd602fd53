"""The candidate-list parity rule (oracle/compare.py) on the CPU.

The rule is what every GPU parity test relies on, so it is checked here
against lists whose right answer is known: the oracle's own candidates pass,
and each planted mistake (a moved pixel, a dropped, extra or duplicated
candidate, a wrong significance, bin or tile) is reported.
"""
import numpy as np
import pytest

from oracle import compare as C
from oracle import fitrig_oracle as O
from paper_2509_21754_gb300 import synth

# the library's 32-byte candidate record, as a NumPy structured type
CAND = np.dtype([("x", np.int32), ("y", np.int32), ("snapshot", np.int32),
                 ("significance", np.float32), ("branch", np.int32),
                 ("freq_bin", np.int32), ("xf", np.float32), ("yf", np.float32)])

W, TAU = 4, 3.0


def as_records(cands):
    out = np.zeros(len(cands), dtype=CAND)
    for i, c in enumerate(cands):
        out[i] = (c.x, c.y, c.snapshot, c.significance, c.branch, c.freq_bin, c.xf, c.yf)
    return out


@pytest.fixture(scope="module")
def case():
    spec = synth.small_spec(12, 61, 58)
    stack, _ = synth.make_stack(spec, seed=5, device="cpu")
    x = stack.numpy().astype(np.float32)
    det = O.detect(x, W, TAU, O.BRANCH_BOTH, "medmad")
    img = [c for c in det.candidates if c.branch == O.BRANCH_IMAGE]
    frq = [c for c in det.candidates if c.branch == O.BRANCH_FREQ]
    assert len(img) > 5 and len(frq) >= 1
    return x, det


def run(x, det, recs):
    return C.compare(recs, x, W, TAU, O.BRANCH_BOTH, "medmad", det=det,
                     decide_image=lambda s, ty, tx: bool(det.z[s, ty, tx] > TAU),
                     decide_freq=lambda ty, tx: bool(det.eta_z[ty, tx] > TAU))


def test_oracle_list_passes(case):
    x, det = case
    assert run(x, det, as_records(det.candidates)) == []


def _first_image(recs):
    return int(np.nonzero(recs["branch"] == O.BRANCH_IMAGE)[0][0])


def test_moved_pixel_is_reported(case):
    x, det = case
    recs = as_records(det.candidates)
    i = _first_image(recs)
    s, y, xx = int(recs[i]["snapshot"]), int(recs[i]["y"]), int(recs[i]["x"])
    ty, tx = y // W, xx // W
    # move to another pixel of the same tile whose Delta is clearly smaller
    d, _, _ = O.unit_terms(*(x[s + k, ty * W:ty * W + W, tx * W:tx * W + W].astype(np.float64)
                             for k in range(3)))
    iy, ix = np.unravel_index(np.argmin(d), d.shape)
    assert d[iy, ix] < d.max() * 0.99
    recs[i]["y"], recs[i]["x"] = ty * W + iy, tx * W + ix
    errs = run(x, det, recs)
    assert any("not an arg-max of Delta" in e for e in errs), errs


def test_dropped_extra_and_duplicate_candidates_are_reported(case):
    x, det = case
    recs = as_records(det.candidates)
    i = _first_image(recs)
    assert any("has 0 candidates" in e for e in run(x, det, np.delete(recs, i)))
    extra = recs[i].copy()
    extra["snapshot"] = (int(extra["snapshot"]) + 1) % (x.shape[0] - 2)
    extra["y"] = (int(extra["y"]) + 2 * W) % x.shape[1]
    errs = run(x, det, np.concatenate([recs, [extra]]))
    assert errs, "an extra candidate passed"
    errs = run(x, det, np.concatenate([recs, recs[i:i + 1]]))
    assert any("two candidates in one tile" in e for e in errs)


def test_wrong_significance_and_bin_are_reported(case):
    x, det = case
    recs = as_records(det.candidates)
    i = _first_image(recs)
    recs[i]["significance"] *= 1.01
    assert any("significance" in e for e in run(x, det, recs))
    recs = as_records(det.candidates)
    j = int(np.nonzero(recs["branch"] == O.BRANCH_FREQ)[0][0])
    ty, tx = int(recs[j]["y"]) // W, int(recs[j]["x"]) // W
    mags = O.dft_magnitudes(det.tlisi[:, ty, tx])
    recs[j]["freq_bin"] = int(np.argmin(mags)) + 1
    assert any("is not a maximum" in e for e in run(x, det, recs))


def test_candidate_off_the_peak_tile_is_reported(case):
    x, det = case
    # a multi-tile component: report a tile that is not its maximum
    for s in range(det.z.shape[0]):
        for comp in O.components(O.select(det.z[s], TAU)):
            if len(comp) < 2:
                continue
            pk = O.component_peak(comp, det.z[s])
            other = [t for t in comp if det.z[s][t] < det.z[s][pk] * 0.99]
            if not other:
                continue
            recs = as_records(det.candidates)
            k = [i for i, r in enumerate(recs) if r["branch"] == O.BRANCH_IMAGE and
                 int(r["snapshot"]) == s and (int(r["y"]) // W, int(r["x"]) // W) == pk][0]
            ty, tx = other[0]
            recs[k]["y"], recs[k]["x"] = ty * W, tx * W
            recs[k]["significance"] = det.z[s][other[0]]
            errs = run(x, det, recs)
            assert any("is not a peak tile" in e for e in errs), errs
            return
    pytest.skip("no multi-tile component with distinct z in this stack")


def strip_view(det, a, b):
    """The oracle's detection restricted to tile rows a..b-1 (z-scores keep the
    whole field's noise parameters)."""
    d = O.Detection([], det.M, b - a, det.Tx, tlisi=det.tlisi[:, a:b], z=det.z[:, a:b])
    d.eta, d.eta_bin, d.eta_z = det.eta[a:b], det.eta_bin[a:b], det.eta_z[a:b]
    return d


def strip_records(recs, a, b):
    ty = recs["y"] // W
    out = recs[(ty >= a) & (ty < b)].copy()
    out["y"] -= a * W
    out["yf"] -= a * W
    return out


@pytest.mark.parametrize("a,b", [(0, 6), (4, 11), (9, 15)])
def test_strip_rule_passes_the_oracle_list_and_skips_cut_components(case, a, b):
    x, det = case
    Ty = det.Ty
    b = min(b, Ty)
    recs = strip_records(as_records(det.candidates), a, b)
    xs = x[:, a * W:b * W]
    d = strip_view(det, a, b)
    kw = dict(det=d, cut_top=a > 0, cut_bottom=b < Ty,
              decide_image=lambda s, ty, tx: bool(d.z[s, ty, tx] > TAU),
              decide_freq=lambda ty, tx: bool(d.eta_z[ty, tx] > TAU))
    assert C.compare(recs, xs, W, TAU, O.BRANCH_BOTH, "medmad", **kw) == []
    # without the cut flags, components cut by the strip edge would be
    # checked as whole ones; a planted mistake inside the strip is still found
    i = _first_image(recs)
    bad = recs.copy()
    bad[i]["significance"] *= 1.01
    ty0 = int(bad[i]["y"]) // W
    errs = C.compare(bad, xs, W, TAU, O.BRANCH_BOTH, "medmad", **kw)
    cut = (a > 0 and ty0 == 0) or (b < Ty and ty0 == b - a - 1)
    assert cut or any("significance" in e for e in errs), errs


def _fp32_tile_statistic(x32: np.ndarray, s: int, w: int) -> np.ndarray:
    """The tile statistic computed the way an FP32 implementation does: every
    difference, ratio, sum (sequential over the tile) and product rounded to
    FP32 (NumPy float32 arithmetic is IEEE round-to-nearest-even)."""
    f = np.float32
    a, b, c = x32[s], x32[s + 1], x32[s + 2]
    d1 = np.abs(b - a)
    d2 = np.abs(c - b)
    delta = np.abs(d1 - d2)
    xh = np.where(b == 0, f(O.C), np.abs(b)).astype(f)
    r = np.minimum(delta * (f(1) / xh), f(1))
    ny, nx = a.shape
    Ty, Tx = -(-ny // w), -(-nx // w)
    out = np.zeros((Ty, Tx), dtype=f)
    for ty in range(Ty):
        for tx in range(Tx):
            sl = (slice(ty * w, ty * w + w), slice(tx * w, tx * w + w))
            S1, S3, S2 = f(0), f(0), f(-1)
            for dv, rv in zip(delta[sl].ravel(), r[sl].ravel()):
                S1 = f(S1 + dv)
                S3 = f(S3 + rv)
                S2 = max(S2, dv)
            n = f(delta[sl].size)
            out[ty, tx] = f(f(f(S1 / n) * S2) * f(S3 / n))
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_tile_value_bound_covers_fp32_arithmetic(seed):
    """The derived FP32 error bound of the tile statistic holds for an FP32
    emulation of the tile arithmetic on stacks with the hard cases: a pulse in
    the middle snapshot of a unit (the two differences nearly cancel in
    Delta), bright steady sky, faint reference pixels and exact zeros; and it
    is tight enough to be a meaningful test (median bound ~1e-7 relative)."""
    rng = np.random.default_rng(seed)
    L, ny, nx, w = 6, 40, 45, 5
    x = rng.standard_normal((L, ny, nx))
    x[:, :10, :] += 300.0 * rng.uniform(0, 1, (1, 10, nx))   # bright steady sky
    x[2, 10:30, :] += 25.0                                   # pulse in snapshot 2
    x[3, 30:, :20] += 400.0                                  # brighter pulse
    x[:, 35:, 40:] *= 1e-3                                   # faint references
    x[1, 5, 5] = 0.0
    x32 = x.astype(np.float32)
    worst = 0.0
    rels = []
    for s in range(L - 2):
        ref = O.unit_tiles(x32, s, w).numerator
        bound = C.tile_value_bound(x32, s, w)
        got = _fp32_tile_statistic(x32, s, w).astype(np.float64)
        ok, ratio = C.values_within_bound(got, ref, bound, slack=1.0)
        assert ok, (s, ratio)
        worst = max(worst, ratio)
        rels.append(np.median(bound / np.abs(ref)))
    assert np.median(rels) < 1e-5
    # the cancellation case needs the bound: the plain 1e-5 relative rule fails
    ok_plain = all(C.values_close(_fp32_tile_statistic(x32, s, w), O.unit_tiles(x32, s, w).numerator,
                                  rel=1e-7, abs_scale=0.0)[0] for s in range(L - 2))
    assert not ok_plain
