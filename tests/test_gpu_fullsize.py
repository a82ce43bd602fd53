"""Parity at the benchmark's full size: 64 snapshots of 4096 x 4096 FP32,
both branches, window 5, 6 sigma, median/MAD noise (the configuration bench.py
times, in its launch configuration).

The FP64 oracle runs the whole trigger on the whole stack (about a minute of
one host core), and:

* the library's candidate list is compared with the oracle's own list by the
  parity rule (oracle/compare.py): every component, every peak tile, every
  significance and every image candidate's arg-max pixel;
* every tile statistic of every unit (within twice its FP32 rounding bound),
  every eta and every noise parameter is compared with the oracle's;
* as a second, independent check of the post-march stages, the oracle's
  z-score, selection and component steps run on the library's own tile values
  and must reproduce its candidates, and the median/MAD must be bit-exact on
  the library's own values.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import compare as C  # noqa: E402
from oracle import fitrig_oracle as O  # noqa: E402
from paper_2509_21754_gb300 import fitrig as F  # noqa: E402
from paper_2509_21754_gb300 import synth  # noqa: E402

W, TAU = 5, 6.0


@pytest.fixture(scope="module")
def run():
    stack, truth = synth.make_stack(synth.C2, seed=2026, device="cuda")
    res = F.detect_stack(stack, W, TAU, F.BRANCH_BOTH, noise=F.NOISE_MEDMAD)
    x = stack.cpu().numpy()
    del stack
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    det = O.detect(x, W, TAU, O.BRANCH_BOTH, "medmad")
    print(f"oracle on 64 x 4096^2: {time.perf_counter() - t0:.1f} s, "
          f"{len(det.candidates)} candidates")
    return res, x, truth, det


def test_candidates_equal_the_oracle_list(run):
    """The whole candidate list against the oracle's own detect: exact outside
    the 1e-4 tau band, with every arg-max pixel checked."""
    res, x, _, det = run
    di, dfq = C.library_decisions(res, TAU)
    errs = C.compare(res["candidates"], x, W, TAU, O.BRANCH_BOTH, "medmad",
                     decide_image=di, decide_freq=dfq, det=det)
    assert not errs, errs[:10]
    assert len(res["candidates"]) > 1000


def test_every_tile_statistic(run):
    """Every tile of every unit within twice the FP32 rounding bound of the
    tile arithmetic (oracle/compare.py: tile_value_bound; where the two
    differences of a pixel nearly cancel in Delta, e.g. a pulse in the middle
    snapshot, the bound is relative to the differences, not to Delta)."""
    res, x, truth, det = run
    ref = np.stack([u.numerator for u in det.units])
    worst = 0.0
    for s in range(ref.shape[0]):
        bound = C.tile_value_bound(x, s, W)
        ok, ratio = C.values_within_bound(res["values"][s], ref[s], bound)
        assert ok, (s, ratio)
        worst = max(worst, ratio)
    print(f"largest error / FP32 bound over all tiles: {worst:.3f}")
    assert res["M"] == det.M
    # the pulsars' tiles are among the compared ones (not only quiet sky)
    for (px, py, *_r) in truth.pulsed:
        assert np.isfinite(ref[:, py // W, px // W]).all()


def test_noise_parameters_against_the_oracle(run):
    """The library's FP32 tile values round the FP64 ones by ~1e-7, so the
    order statistics agree to that (exactness on the library's own values is
    the next test)."""
    res, _, _, det = run
    M2 = det.M * det.M
    for s in range(det.z.shape[0]):
        c, sc = res["noise"][s]
        assert c == pytest.approx(det.centre[s] * M2, rel=1e-5)
        assert sc == pytest.approx(det.scale[s] * M2, rel=1e-5)
    c, sc = res["eta_noise"]
    assert c == pytest.approx(det.eta_centre * M2, rel=2e-5)
    assert sc == pytest.approx(det.eta_scale * M2, rel=2e-5)


def test_noise_is_exact_on_own_values(run):
    res, _, _, _ = run
    v = res["values"]
    for s in range(v.shape[0]):
        a = v[s].ravel()
        a = a[np.isfinite(a)]
        med = np.sort(a)[(a.size - 1) // 2]
        mad = np.sort(np.abs(a - med))[(a.size - 1) // 2]
        assert res["noise"][s][0] == float(med)
        assert res["noise"][s][1] == 1.482602218505602 * float(mad)


def test_candidate_stages_on_own_values(run):
    """Selection, components and candidates equal the oracle's steps applied to
    the library's tile values (exact outside the tolerance band)."""
    res, x, _, _ = run
    M = res["M"]
    U = res["values"].shape[0]
    tl = 1.0 - res["values"].astype(np.float64) / (M * M)
    det = O.Detection([], M, *res["grid"], tlisi=tl)
    det.z = np.stack([O.zscore_image(tl[s], "medmad")[0] for s in range(U)])
    det.eta, det.eta_bin = O.spectrum(tl)
    det.eta_z, det.eta_centre, det.eta_scale = O.zscore_map(det.eta, "medmad")
    di, dfq = C.library_decisions(res, TAU)
    errs = C.compare(res["candidates"], x, W, TAU, O.BRANCH_BOTH, "medmad",
                     decide_image=di, decide_freq=dfq, det=det)
    assert not errs, errs[:10]


def test_every_spectrum_tile(run):
    """eta of every tile against the oracle's DFT of its own FP64 series (the
    scale M^2 cancels: the library's eta is of the M-free statistic)."""
    res, _, _, det = run
    M2 = det.M * det.M
    eta_ref = det.eta * M2
    m = np.isfinite(eta_ref)
    assert np.array_equal(m, np.isfinite(res["eta"]))
    np.testing.assert_allclose(res["eta"][m], eta_ref[m], rtol=5e-5,
                               atol=1e-6 * float(np.median(eta_ref[m])))
    # the bin reaches the maximum magnitude of the library's own series
    v = res["values"].astype(np.float64)
    Ty, Tx = res["grid"]
    rng = np.random.default_rng(1)
    pick = rng.integers(0, Ty * Tx, 5000)
    mags = O.dft_magnitudes(v.reshape(v.shape[0], -1)[:, pick].T)
    kb = res["bin"].ravel()[pick]
    top = mags[np.arange(pick.size), kb - 1]
    assert np.all(top >= mags.max(axis=1) * (1 - 1e-4))
