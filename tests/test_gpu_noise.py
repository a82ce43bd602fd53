"""Median/MAD noise estimate on device maps, through the C ABI, against the
definition (lower median of the finite values; lower median of |v - median|
in FP32; scale = 1.482602218505602 MAD) evaluated by sorting in NumPy.

The maps cover every way the library selects the order statistics: the
bracketed cluster form of fitrig_noise_static (maps of up to 2 Mi values,
including ones whose bracket cannot hold the copies and fall back to the
multi-pass cluster form), the multi-pass form alone (larger maps), and the
split form that plans and fitrig_threshold_map use (a sample bracket, a
counting and copying pass and an exact selection for the median, then the
same for the MAD; its misses fall back to the cluster form too)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2509_21754_gb300 import fitrig as F  # noqa: E402

MAD_TO_SIGMA = 1.482602218505602


def definition(v: np.ndarray):
    v = v[np.isfinite(v)].astype(np.float32)
    if v.size == 0:
        return float("nan"), 0.0
    k = (v.size - 1) // 2
    med = np.sort(v)[k]
    mad = np.sort(np.abs(v - med))[k]          # FP32 arithmetic, as on the device
    return float(med), MAD_TO_SIGMA * float(mad)


def run(v: torch.Tensor, groups: int, n: int):
    out = torch.full((2 * groups,), -7.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert F.fitrig_noise_static(v, groups, n, F.NOISE_MEDMAD, out, stream) == F.OK
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(groups, 2)


def run_split(v: torch.Tensor, groups: int, n: int):
    """The allocating single-map entry point (the split form up to 2 Mi
    values), one map at a time."""
    stream = torch.cuda.current_stream().cuda_stream
    out = np.zeros((groups, 2))
    for g in range(groups):
        _, c, s = F.fitrig_threshold_map(v[g * n:(g + 1) * n], 3.0, F.NOISE_MEDMAD, stream)
        out[g] = (c, s)
    return out


def check(v: torch.Tensor, groups: int, n: int):
    host = v.cpu().numpy().reshape(groups, n)
    for form, got in (("static", run(v, groups, n)), ("split", run_split(v, groups, n))):
        for g in range(groups):
            med, sc = definition(host[g])
            if np.isnan(med):
                assert np.isnan(got[g, 0]) and got[g, 1] == 0.0, (form, g)
            else:
                assert got[g, 0] == med and got[g, 1] == sc, (form, g, got[g], med, sc)


def gen(seed):
    return torch.Generator(device="cuda").manual_seed(seed)


@pytest.mark.parametrize("groups,n", [(3, 672_401), (2, 672_400), (4, 131_072), (1, 2_097_152),
                                      (2, 3_000_000), (7, 33), (1, 1), (2, 5)])
def test_gaussian_and_skewed_maps(groups, n):
    g = gen(n + groups)
    v = torch.randn(groups * n, device="cuda", generator=g)
    v = v.view(groups, n)
    v[1::2] = torch.exp(2.0 * v[1::2])     # right-skewed groups, like the tile statistic
    v = v.reshape(-1).contiguous()
    if n > 64:
        v[5::389] = float("nan")
        v[11::1009] = float("inf")
    check(v, groups, n)


def test_repeated_value_falls_back_exactly():
    """60% of the values equal: the bracket around the median holds far more
    values than the copy buffer, so the group is finished by the multi-pass
    form; the MAD is then 0 (a degenerate scale)."""
    n = 500_000
    g = gen(3)
    v = torch.randn(2 * n, device="cuda", generator=g)
    v[: int(0.6 * n)] = 1.0
    v[n: n + int(0.3 * n)] = 2.5            # second group: 30% equal, MAD > 0
    check(v, 2, n)


def test_sampled_runs_unrepresentative():
    """Values that change every 32 entries with a long period, so that the
    evenly spread sample sees a different mix than the map: whatever the
    bracket, the result is the exact order statistic."""
    n = 1_000_003
    idx = torch.arange(n, device="cuda", dtype=torch.float64)
    v = torch.where(((idx // 32) % 61) < 29, idx * 1e-6, 5.0 + idx * 1e-7).float()
    check(v, 1, n)


def test_constant_and_empty_groups():
    n = 100_000
    v = torch.full((3 * n,), 4.25, device="cuda")
    v[n:2 * n] = float("nan")                 # no finite value: (nan, 0)
    v[2 * n:] = torch.linspace(-1.0, 1.0, n, device="cuda")
    check(v, 3, n)


@pytest.mark.parametrize("seed", range(4))
def test_split_form_on_shifted_and_asymmetric_maps(seed):
    """Maps whose median and MAD sit where a sample bracket is easily wrong
    (a cluster of values just above the median, a long one-sided tail, a gap
    at the median, quantised values with many ties): every count stays
    exact, whichever form finishes the map."""
    n = 672_401
    g = gen(100 + seed)
    v = torch.randn(n, device="cuda", generator=g)
    if seed == 0:
        v[: n // 40] = 0.0312                      # a spike just above the median
    elif seed == 1:
        v = torch.exp(3.0 * v)                     # heavy right tail
    elif seed == 2:
        v = torch.where(v.abs() < 0.05, v + 0.1 * torch.sign(v), v)   # a gap at the median
    else:
        v = torch.round(v * 64.0) / 64.0          # quantised values: many ties
    check(v.contiguous(), 1, n)
