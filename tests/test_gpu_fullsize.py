"""Parity at the benchmark's full size: 64 snapshots of 4096 x 4096 FP32,
both branches, window 5, 6 sigma, median/MAD noise (the configuration bench.py
times).  The oracle cannot run every tile of every unit here, so:

* tile statistics are compared on a sample of tiles (random ones, the ragged
  last row/column, and the tiles of every injected pulsar) for all 62 units;
* the noise, selection, component and candidate stages are checked by running
  the oracle's own steps on the library's tile values (so the stages must agree
  exactly, up to the stated tolerance band), with the candidate pixels checked
  against the oracle's arg-max of Delta on a sample;
* the spectrum is compared tile by tile against the oracle's DFT of the same
  series.
"""
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
    return res, x, truth


def test_sampled_tiles(run):
    res, x, truth = run
    Ty, Tx = res["grid"]
    rng = np.random.default_rng(0)
    tiles = {(int(a), int(b)) for a, b in zip(rng.integers(0, Ty, 200), rng.integers(0, Tx, 200))}
    tiles |= {(Ty - 1, t) for t in range(0, Tx, 97)} | {(t, Tx - 1) for t in range(0, Ty, 97)}
    tiles |= {(Ty - 1, Tx - 1)}
    tiles |= {(py // W, px // W) for (px, py, *_r) in truth.pulsed}
    tiles = sorted(tiles)
    ref = O.sampled_tiles(x, W, tiles)
    got = np.stack([res["values"][:, ty, tx] for ty, tx in tiles], axis=1)
    ok, worst = C.values_close(got, ref["numerator"])
    assert ok, worst
    assert res["M"] == O.normaliser_M(x)


def test_noise_is_exact_on_own_values(run):
    res, _, _ = run
    v = res["values"]
    for s in range(v.shape[0]):
        a = v[s].ravel()
        a = a[np.isfinite(a)]
        med = np.sort(a)[(a.size - 1) // 2]
        mad = np.sort(np.abs(a - med))[(a.size - 1) // 2]
        assert res["noise"][s][0] == float(med)
        assert res["noise"][s][1] == 1.482602218505602 * float(mad)


def test_candidate_stages(run):
    """Selection, components and candidates equal the oracle's steps applied to
    the library's tile values (exact outside the tolerance band)."""
    res, x, _ = run
    M = res["M"]
    U = res["values"].shape[0]
    tl = 1.0 - res["values"].astype(np.float64) / (M * M)
    det = O.Detection([], M, *res["grid"], tlisi=tl)
    det.z = np.stack([O.zscore_image(tl[s], "medmad")[0] for s in range(U)])
    det.eta, det.eta_bin = O.spectrum(tl)
    det.eta_z, det.eta_centre, det.eta_scale = O.zscore_map(det.eta, "medmad")
    cands = res["candidates"]
    # pixels: the arg-max check reads the stack, so it runs on a sample
    errs = C.compare(cands, x, W, TAU, O.BRANCH_BOTH, "medmad",
                     decide_image=F.decisions(res, TAU)[0],
                     decide_freq=F.decisions(res, TAU)[1], det=det, pixel_sample=3000)
    assert not errs, errs[:10]


def test_spectrum_tiles(run):
    res, _, _ = run
    M = res["M"]
    v = res["values"].astype(np.float64)
    Ty, Tx = res["grid"]
    rng = np.random.default_rng(1)
    pick = rng.integers(0, Ty * Tx, 3000)
    series = v.reshape(v.shape[0], -1)[:, pick].T
    mags = O.dft_magnitudes(series)
    eta = res["eta"].ravel()[pick]
    np.testing.assert_allclose(eta, mags.max(axis=1), rtol=2e-5, atol=1e-6 * np.median(eta))
    kb = res["bin"].ravel()[pick]
    top = mags[np.arange(pick.size), kb - 1]
    assert np.all(top >= mags.max(axis=1) * (1 - 1e-4))
