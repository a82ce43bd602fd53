"""fitrig_noise_static: the noise estimate for callers that cannot allocate
device memory (its working memory is a fixed array inside the library).

Checked through the C ABI on two calls in a row with different data, so that
the array's leftover contents from the first call cannot leak into the
second:

* against the allocating entry point fitrig_threshold_map on the same maps;
* against a NumPy sort of the same FP32 values (the median/MAD is an exact
  order statistic: bit-equal) and NumPy's FP64 mean and population std;
* on maps small enough for the cluster kernels and on one map above 8 Mi
  values, which takes the grid-wide radix select whose histogram and select
  state live in the fixed array and are cleared by every call.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2509_21754_gb300 import fitrig as F  # noqa: E402

MAD_TO_SIGMA = 1.482602218505602


def maps(groups, n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.randn(groups * n, device="cuda", generator=g).abs() * 3.0 + 0.5
    v[::997] = float("nan")   # skipped entries
    return v


def reference(v, groups, n, mode, stream):
    out = []
    for k in range(groups):
        _, c, s = F.fitrig_threshold_map(v[k * n:(k + 1) * n], 3.0, mode, stream)
        out.append((c, s))
    return np.array(out)


def numpy_estimate(a: np.ndarray, mode: int):
    """Lower median and 1.4826 MAD (|v - median| rounded to FP32, as the
    library computes it), or mean and population std, of the finite values."""
    a = a[np.isfinite(a)]
    if mode == F.NOISE_MEDMAD:
        med = np.sort(a)[(a.size - 1) // 2]
        dev = np.abs(a - med).astype(np.float32)
        mad = np.sort(dev)[(dev.size - 1) // 2]
        return float(med), MAD_TO_SIGMA * float(mad)
    d = a.astype(np.float64)
    return float(d.mean()), float(d.std())


@pytest.mark.parametrize("groups,n", [(1, 250_001), (5, 200_003), (64, 4_097), (1, 8_400_001)])
def test_static_noise_matches_allocating_entry_point_and_numpy(groups, n):
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        v = maps(groups, n, seed=7 + call)
        host = v.cpu().numpy().reshape(groups, n)
        for mode in (F.NOISE_MEDMAD, F.NOISE_MEANSTD):
            want = reference(v, groups, n, mode, stream)
            out = torch.full((2 * groups,), -1.0, dtype=torch.float64, device="cuda")
            rc = F.fitrig_noise_static(v, groups, n, mode, out, stream)
            assert rc == F.OK
            torch.cuda.synchronize()
            got = out.cpu().numpy().reshape(groups, 2)
            npy = np.array([numpy_estimate(host[k], mode) for k in range(groups)])
            if mode == F.NOISE_MEDMAD:
                # exact integer selection on the same values: bit-equal
                assert np.array_equal(got, want)
                assert np.array_equal(got, npy)
            else:
                # same estimator; with groups > 1 the blocks split each map
                # differently, and FP32 squared deviations are rounded per
                # term, so the sums agree to ~1e-10 (parity tests allow 1e-5)
                np.testing.assert_allclose(got, want, rtol=1e-9, atol=0)
                np.testing.assert_allclose(got, npy, rtol=1e-6, atol=0)


def test_static_noise_rejects_too_many_groups():
    v = torch.ones(65 * 10, device="cuda")
    out = torch.zeros(130, dtype=torch.float64, device="cuda")
    assert F.fitrig_noise_static(v, 65, 10, F.NOISE_MEDMAD, out, 0) == F.EINVAL
    assert F.fitrig_noise_static(v, 0, 10, F.NOISE_MEDMAD, out, 0) == F.EINVAL
    lib = F.load()
    assert lib.fitrig_noise_static(None, 1, 10, F.NOISE_MEDMAD, ctypes.c_void_p(out.data_ptr()),
                                   0) == F.EINVAL
