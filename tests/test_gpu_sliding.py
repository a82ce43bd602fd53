"""Sliding-window mode (odd window centred on every pixel) against the oracle."""
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


def run(stack, w, tau, branch, noise="meanstd", storage=F.F32, tdt=torch.float32):
    res = F.detect_stack(stack.cuda().to(tdt), w, tau, branch, storage,
                         F.NOISE_MEDMAD if noise == "medmad" else F.NOISE_MEANSTD,
                         stride=F.STRIDE_SLIDING)
    x = stack.to(tdt).float().cpu().numpy()
    det = O.detect(x, w, tau, branch, noise, stride="sliding")
    di, dfq = C.library_decisions(res, tau)
    errs = C.compare(res["candidates"], x, 1, tau, branch, noise, decide_image=di,
                     decide_freq=dfq, det=det)
    assert not errs, errs[:8]
    if branch & F.BRANCH_IMAGE:
        for s, u in enumerate(det.units):
            bound = C.tile_value_bound(x, s, w, stride="sliding")
            ok, worst = C.values_within_bound(res["values"][s], u.numerator, bound)
            assert ok, (s, worst)
    return res, det


@pytest.mark.parametrize("L,ny,nx,w", [(5, 37, 53, 3), (6, 64, 130, 5), (4, 33, 40, 1),
                                       (5, 70, 300, 7), (4, 50, 61, 11), (3, 40, 45, 31),
                                       (4, 140, 129, 9)])
def test_sliding_parity(L, ny, nx, w):
    spec = synth.small_spec(L, ny, nx, n_steady=5, n_pulsed=2, pulse_period=(3, 4))
    stack, _ = synth.make_stack(spec, seed=ny + nx + w, device="cuda")
    run(stack.cpu(), w, 4.0, F.BRANCH_IMAGE)


def test_sliding_large_map_crosses_many_blocks():
    """1024 x 1100 pixels: windows straddle the march's CTA boxes and the
    selection's blocks on every side, with pulsars and bright steady sky."""
    spec = synth.small_spec(6, 1024, 1100, pulse_period=(3, 4))
    stack, _ = synth.make_stack(spec, seed=21, device="cuda")
    run(stack.cpu(), 5, 5.0, F.BRANCH_IMAGE, "medmad")


def test_sliding_both_branches_medmad():
    spec = synth.small_spec(20, 96, 100, n_steady=6, n_pulsed=2, pulse_period=(3, 5))
    stack, _ = synth.make_stack(spec, seed=3, device="cuda")
    run(stack.cpu(), 5, 5.0, F.BRANCH_BOTH, "medmad")


def test_sliding_half_storage():
    spec = synth.small_spec(6, 80, 90)
    stack, _ = synth.make_stack(spec, seed=4, device="cuda")
    run(stack.cpu(), 5, 4.0, F.BRANCH_IMAGE, storage=F.F16, tdt=torch.float16)


def test_sliding_rejects_even_windows():
    h = F.fitrig_plan_create(32, 32, 5, 4, 3.0)
    try:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_plan_set(h, F.OPT_STRIDE, F.STRIDE_SLIDING)
        assert e.value.status == F.EINVAL
    finally:
        F.fitrig_plan_destroy(h)
