"""Frequency branch beyond the short series: harmonic summing (every spectrum
kernel) and long series (the warp-per-tile transform, up to 4096 points),
against the FP64 oracle through the C ABI."""
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

NOISE = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}


def run(x, w, tau, hmax, noise="meanstd"):
    res = F.detect_stack(torch.from_numpy(x).cuda(), w, tau, F.BRANCH_FREQ, F.F32, NOISE[noise],
                         harmonics=hmax)
    det = O.detect(x, w, tau, F.BRANCH_FREQ, noise, harmonics=hmax)
    return res, det


def check(res, det, x, w, tau, hmax, noise):
    di, dfq = C.library_decisions(res, tau)
    errs = C.compare(res["candidates"], x, w, tau, F.BRANCH_FREQ, noise, decide_image=di,
                     decide_freq=dfq, det=det, harmonics=hmax)
    assert not errs, errs[:10]
    ok, worst = C.values_close(res["eta"], det.eta * det.M ** 2, rel=1e-4)
    assert ok, worst
    # every tile's bin attains h (the bin of a near tie may differ from the oracle's)
    Ty, Tx = det.eta.shape
    for ty in range(Ty):
        for tx in range(Tx):
            mags = O.dft_magnitudes(det.tlisi[:, ty, tx])
            assert C.bin_is_a_maximum(mags, int(res["bin"][ty, tx]), hmax), (ty, tx)


# n = L - 2 picks the kernel: even <= 66 and odd <= 65 thread-per-tile, the rest
# (and every harmonic sum beyond 66 points) one warp per tile
@pytest.mark.parametrize("L,side,w,period,hmax", [
    (64, 120, 5, 4, 8),      # n = 62, even kernel
    (65, 96, 4, 8, 4),       # n = 63, odd kernel
    (34, 64, 4, 8, 32),      # n = 32, m_max above K / 2
    (122, 64, 4, 8, 16),     # n = 120, warp-per-tile with harmonics
    (302, 48, 4, 16, 8),     # n = 300
    (302, 48, 4, 16, 1),     # n = 300, maximum magnitude
    (259, 40, 4, 7, 1),      # n = 257, odd, first length past the direct kernel
    (1026, 32, 4, 32, 8),    # n = 1024 (the paper's L = 1026)
    (1500, 24, 4, 19, 8),    # n = 1498 (the paper's end-to-end run)
    (4098, 16, 4, 64, 32),   # n = 4096, the longest series
])
def test_spectrum_parity(L, side, w, period, hmax):
    x = synth.periodic_tile_stack(L, side, side + 3, w, period, 1, (2, 3), 4.0, seed=L + side)
    for noise in ("meanstd", "medmad"):
        res, det = run(x, w, 4.0, hmax, noise)
        check(res, det, x, w, 4.0, hmax, noise)


@pytest.mark.parametrize("seed", [21, 22])
def test_harmonic_sum_recovers_the_fundamental(seed):
    """A one-snapshot pulse every 16 snapshots over n = 128 units: the largest
    single magnitude sits on a high harmonic, the harmonic sum on the
    fundamental bin n / 16 = 8 (the spin frequency, as in the real-data evaluation of Sec. 3)."""
    x = synth.periodic_tile_stack(130, 64, 64, 4, 16, 3, (5, 7), 3.0, seed=seed)
    bins = {}
    for hmax in (1, 16):
        res, det = run(x, 4, 4.0, hmax)
        check(res, det, x, 4, 4.0, hmax, "meanstd")
        bins[hmax] = int(res["bin"][5, 7])
    assert bins[16] == 8
    assert bins[1] % 8 == 0 and bins[1] > 8


def test_harmonics_option_and_graph_replay():
    """The option is checked, settable between detects, and a captured graph
    of the old setting is not replayed."""
    x = synth.periodic_tile_stack(66, 64, 67, 4, 8, 1, (2, 3), 4.0, seed=5)
    want = F.detect_stack(torch.from_numpy(x).cuda(), 4, 4.0, F.BRANCH_FREQ, harmonics=8)
    with F.Plan(67, 64, 66, 4, 4.0, F.BRANCH_FREQ) as p:
        for bad in (0, 3, 64, -1):
            with pytest.raises(F.FitrigError) as e:
                F.fitrig_plan_set(p.h, F.OPT_HARMONICS, bad)
            assert e.value.status == F.EINVAL
        p.push_stack(torch.from_numpy(x).cuda())
        for _ in range(3):   # the second detect captures, the third replays
            p.detect()
        F.fitrig_plan_set(p.h, F.OPT_HARMONICS, 8)
        for _ in range(3):
            rc, c = p.detect()
            eta, kbin = F.fitrig_spectrum(p.h)
            assert c.tobytes() == want["candidates"].tobytes()
            assert np.array_equal(eta, want["eta"]) and np.array_equal(kbin, want["bin"])


def test_series_length_limit():
    h = F.fitrig_plan_create(16, 16, 4098, 4, 4.0, F.BRANCH_FREQ)
    F.fitrig_plan_destroy(h)
    with pytest.raises(F.FitrigError) as e:
        F.fitrig_plan_create(16, 16, 4099, 4, 4.0, F.BRANCH_FREQ)
    assert e.value.status == F.EUNSUPPORTED
    h = F.fitrig_plan_create(16, 16, 5000, 4, 4.0, F.BRANCH_IMAGE)   # image branch: no limit
    F.fitrig_plan_destroy(h)


@pytest.mark.parametrize("refine", ["parabolic", "cubic"])
@pytest.mark.parametrize("seed", [3, 4])
def test_refined_positions_follow_the_oracle(refine, seed):
    """Frequency candidates' sub-tile positions (parabola or spline through the
    eta map) within 0.05 tiles of the oracle's: a pulsed source that straddles
    two tiles, one at the map edge and one off-centre inside a tile."""
    w = 8
    code = {"parabolic": F.REFINE_PARABOLIC, "cubic": F.REFINE_CUBIC}[refine]
    x = synth.periodic_tile_stack(42, 128, 128, w, 4, 1, (2, 2), 0.0, seed=seed, noise=0.3)
    x[np.arange(42) % 4 == 1, 44:50, 60:70] += 6.0
    x[np.arange(42) % 4 == 2, 2:8, 121:127] += 5.0
    x[np.arange(42) % 5 == 0, 90:97, 33:36] += 6.0
    res = F.detect_stack(torch.from_numpy(x).cuda(), w, 4.0, F.BRANCH_FREQ, refine=code)
    det = O.detect(x, w, 4.0, F.BRANCH_FREQ, refine=refine)
    di, dfq = C.library_decisions(res, 4.0)
    errs = C.compare(res["candidates"], x, w, 4.0, F.BRANCH_FREQ, decide_image=di,
                     decide_freq=dfq, det=det, refine=refine)
    assert not errs, errs[:10]
    assert len(res["candidates"]) >= 3
    with F.Plan(128, 128, 42, w, 4.0, F.BRANCH_FREQ) as p:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_plan_set(p.h, F.OPT_REFINE, 2)
        assert e.value.status == F.EINVAL
