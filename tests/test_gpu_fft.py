"""The radix FFT of the image-frequency branch (Sec. 2.4.2, Eq. eta) for
series lengths n = 2^m (the paper makes L - 2 a power of two), through the C
ABI's fitrig_spectrum_map on seeded cubes, against the FP64 oracle:

* eta within 2e-5 relative of the oracle's h of its own DFT magnitudes, for
  the maximum magnitude and for harmonic sums m_max = 2..32;
* every bin a fundamental that attains h within 1e-4;
* the radix and the direct O(n^2) kernel agree on the same cube;
* ragged tile counts (not a multiple of the tiles per CTA), a padded stride,
  non-finite series (eta NaN, bin -1), and pure tones whose bin is known;
* a plan's frequency branch at L - 2 = 256 and 2048 against the oracle's
  candidates (the plan takes the radix kernel for these lengths).
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


def cube(n, T, stride, seed, kind="skewed"):
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(n, stride, device="cuda", generator=g)
    if kind == "skewed":   # positive, right-skewed like the tile statistic
        x = x.abs() * x.abs() + 0.5
    x[:, T:] = float("nan")   # padding beyond T is never read
    return x.contiguous()


def run(x, n, T, stride, harmonics, method):
    eta = torch.full((T,), -7.0, device="cuda")
    kb = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    ms = F.fitrig_spectrum_map(x, n, T, stride, harmonics, eta, kb, method)
    return eta.cpu().numpy(), kb.cpu().numpy(), ms


def oracle(x, n, T, harmonics):
    series = x[:, :T].double().cpu().numpy().T     # (T, n)
    ok = np.all(np.isfinite(series), axis=1)
    mags = O.dft_magnitudes(np.where(ok[:, None], series, 0.0))
    eta, kb = (mags.max(axis=1), mags.argmax(axis=1) + 1) if harmonics == 1 else \
        O.harmonic_sum(mags, harmonics)
    return np.where(ok, eta, np.nan), np.where(ok, kb, -1), mags


@pytest.mark.parametrize("n,T", [(128, 1003), (256, 999), (512, 517), (1024, 301),
                                 (2048, 203), (4096, 91)])
@pytest.mark.parametrize("harmonics", [1, 4, 32])
def test_radix_against_the_oracle(n, T, harmonics):
    stride = T + 13
    x = cube(n, T, stride, seed=n + harmonics)
    x[:, 5] = x[:, 5] * 0 + 2.0            # a constant series: all |X_k| = 0
    x[n // 3, 7] = float("inf")            # a non-finite series
    eta, kb, _ = run(x, n, T, stride, harmonics, F.SPECTRUM_RADIX)
    ref, rkb, mags = oracle(x, n, T, harmonics)
    assert np.array_equal(np.isnan(eta), np.isnan(ref))
    assert kb[7] == -1 and np.isnan(eta[7])
    m = np.isfinite(ref)
    scale = float(np.median(ref[m]))
    np.testing.assert_allclose(eta[m], ref[m], rtol=2e-5, atol=1e-6 * scale)
    for t in np.nonzero(m)[0]:
        if t == 5:
            continue
        assert C.bin_is_a_maximum(mags[t], int(kb[t]), harmonics), (t, kb[t], rkb[t])


@pytest.mark.parametrize("n", [512, 2048, 4096])
@pytest.mark.parametrize("harmonics", [1, 8])
def test_radix_equals_direct(n, harmonics):
    T = 257
    x = cube(n, T, T, seed=3 * n + harmonics)
    e1, k1, _ = run(x, n, T, T, harmonics, F.SPECTRUM_RADIX)
    e2, k2, _ = run(x, n, T, T, harmonics, F.SPECTRUM_DIRECT)
    np.testing.assert_allclose(e1, e2, rtol=2e-5, atol=0)
    same = k1 == k2
    # a differing bin must be a near tie of the two values
    assert np.all(same | (np.abs(e1 - e2) <= 2e-5 * np.abs(e2))), (k1[~same], k2[~same])


@pytest.mark.parametrize("n", [128, 1024, 4096])
def test_pure_tones(n):
    """y_s = cos(2 pi k0 s / n) + 0.3 cos(2 pi k1 s / n): |X_k0| = n/2 exactly,
    the maximum, found at k0 (including the Nyquist bin)."""
    T = 6
    s = np.arange(n)
    rows = []
    for k0, k1 in [(1, 7), (n // 2, 3), (n // 4 - 1, n // 8), (37, 36), (n // 2 - 1, 1), (5, 5)]:
        rows.append(np.cos(2 * np.pi * k0 * s / n) + 0.3 * np.cos(2 * np.pi * k1 * s / n) + 4.0)
    x = torch.tensor(np.stack(rows, axis=1), dtype=torch.float32, device="cuda").contiguous()
    eta, kb, _ = run(x, n, T, T, 1, F.SPECTRUM_RADIX)
    want_k = [1, n // 2, n // 4 - 1, 37, n // 2 - 1, 5]
    want_eta = [n / 2, n, n / 2, n / 2, n / 2, 1.3 * n / 2]
    assert list(kb) == want_k
    np.testing.assert_allclose(eta, want_eta, rtol=1e-4)


def test_arguments_are_checked():
    x = torch.zeros(100, 8, device="cuda")
    e = torch.zeros(8, device="cuda")
    b = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FitrigError):
        F.fitrig_spectrum_map(x, 100, 8, 8, 1, e, b, F.SPECTRUM_RADIX)    # not a power of 2
    with pytest.raises(F.FitrigError):
        F.fitrig_spectrum_map(x, 64, 8, 8, 3, e, b)                       # harmonics not 2^k
    with pytest.raises(F.FitrigError):
        F.fitrig_spectrum_map(x, 64, 8, 4, 1, e, b)                       # stride < T


@pytest.mark.parametrize("L,w,harmonics", [(258, 16, 1), (2050, 64, 4)])
def test_plan_frequency_branch_at_power_of_two_lengths(L, w, harmonics):
    """A plan whose series are 2^m long (L - 2 = 256, 2048) takes the radix
    kernel; its frequency candidates match the oracle's."""
    size = 96 if L < 1000 else 64 * 3
    spec = synth.small_spec(L, size, size + w // 2, n_pulsed=2, pulse_period=(4, 8))
    stack, _ = synth.make_stack(spec, seed=L, device="cuda")
    res = F.detect_stack(stack, w, 4.0, F.BRANCH_FREQ, noise=F.NOISE_MEDMAD, harmonics=harmonics)
    x = stack.cpu().numpy()
    di, dfq = C.library_decisions(res, 4.0)
    errs = C.compare(res["candidates"], x, w, 4.0, O.BRANCH_FREQ, "medmad", decide_freq=dfq,
                     harmonics=harmonics)
    assert not errs, errs[:10]
    det = O.detect(x, w, 4.0, O.BRANCH_FREQ, "medmad", harmonics=harmonics)
    M2 = det.M * det.M
    m = np.isfinite(det.eta)
    np.testing.assert_allclose(res["eta"][m], det.eta[m] * M2, rtol=5e-5,
                               atol=1e-6 * float(np.median(det.eta[m] * M2)))
