"""Difference-coded half storage (FITRIG_CODING_DELTA) through the C ABI.

* The stored form (FP32 key frame, half differences) equals the oracle's
  closed-loop coder bit for bit, for host, device and block pushes.
* The trigger on a difference-coded plan equals the FP64 oracle run on the
  decoded stack (the same parity rule as every other plan), over the windows
  the coded march supports, both branches, both noise modes, the signed r
  reading, the running M, cropped edges and non-finite pixels.
* Pushing already-encoded differences gives the same detection; the coder
  refuses FP32 pushes after them; unsupported combinations are refused.
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

FMT = {F.BF16: "bf16", F.F16: "f16"}
TDT = {F.BF16: torch.bfloat16, F.F16: torch.float16}
NOISE = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}


class _DeviceArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                         "typestr": typestr, "version": 2, "strides": None}


def stored_form(plan, L, ny, nx, storage):
    """(key, q) as the plan holds them, as FP32 numpy arrays (q[0] = 0)."""
    kp, kpitch = F.fitrig_stack_device_ptr(plan, 0)
    key = torch.as_tensor(_DeviceArray(kp, (ny, kpitch), "<f4"), device="cuda")[:, :nx]
    q = np.zeros((L, ny, nx), dtype=np.float32)
    for s in range(1, L):
        p, pitch = F.fitrig_stack_device_ptr(plan, s)
        raw = torch.as_tensor(_DeviceArray(p, (ny, pitch), "<i2"), device="cuda")
        q[s] = raw.view(TDT[storage])[:, :nx].float().cpu().numpy()
    return key.cpu().numpy(), q


def same_bits(a, b):
    """Bit-equal FP32 arrays, except that any NaN matches any NaN."""
    na, nb = np.isnan(a), np.isnan(b)
    return np.array_equal(na, nb) and np.array_equal(a[~na].view(np.uint32),
                                                     b[~nb].view(np.uint32))


def make(L, ny, nx, seed, **kw):
    spec = synth.small_spec(L, ny, nx, **kw)
    stack, _ = synth.make_stack(spec, seed=seed, device="cuda")
    return stack


@pytest.mark.parametrize("storage", [F.BF16, F.F16])
@pytest.mark.parametrize("how", ["host", "device", "block"])
def test_stored_differences_are_the_oracle_coder(storage, how):
    L, ny, nx = 9, 203, 230
    stack = make(L, ny, nx, seed=21)
    stack[4, 17, 33] = float("nan")            # poisons that pixel from snapshot 4 on
    x = stack.cpu().numpy()
    with F.Plan(nx, ny, L, 5, 4.0, storage=storage, coding=F.CODING_DELTA) as p:
        if how == "host":
            h = stack.cpu().pin_memory()
            for k in range(L):
                F.fitrig_push_snapshot(p.h, h[k])
        elif how == "device":
            for k in range(L):
                F.fitrig_push_snapshot(p.h, stack[k])
        else:
            F.fitrig_push_snapshots(p.h, stack.cpu().pin_memory())
        torch.cuda.synchronize()
        key, q = stored_form(p.h, L, ny, nx, storage)
    want_key, want_q = O.delta_encode(x, FMT[storage])
    assert same_bits(key, want_key)
    assert same_bits(q[1:], want_q[1:])
    dec = O.delta_decode(key, q)
    assert np.all(np.isnan(dec[4:, 17, 33]))


def run_pair(stack, w, tau, branch, storage, noise="meanstd", rmode="abs", edge="partial",
             mmode="global"):
    res = F.detect_stack(stack, w, tau, branch, storage, NOISE[noise],
                         F.RMODE_SIGNED if rmode == "signed" else F.RMODE_ABS,
                         F.EDGE_DROP if edge == "drop" else F.EDGE_PARTIAL,
                         mmode=F.MMODE_RUNNING if mmode == "running" else F.MMODE_GLOBAL,
                         coding=F.CODING_DELTA)
    torch.cuda.synchronize()
    x = O.delta_decode(*O.delta_encode(stack.cpu().numpy(), FMT[storage]))
    det = O.detect(x, w, tau, branch, noise, rmode, edge, mmode=mmode)
    return res, det, x


def assert_parity(res, det, x, w, tau, branch, noise, rmode="abs", edge="partial"):
    di, dfq = C.library_decisions(res, tau)
    errs = C.compare(res["candidates"], x, w, tau, branch, noise, rmode, edge, di, dfq, det)
    assert not errs, errs[:10]
    if branch & F.BRANCH_IMAGE:
        ref = np.stack([u.numerator for u in det.units])
        ok, worst = C.values_close(res["values"], ref, rel=1e-5)
        assert ok, f"tile values differ, worst relative error {worst}"
    assert res["M"] == det.M


@pytest.mark.parametrize("storage", [F.BF16, F.F16])
@pytest.mark.parametrize("L,ny,nx,w", [(10, 256, 256, 5), (7, 131, 157, 3), (6, 97, 150, 4),
                                       (8, 123, 101, 6), (6, 140, 260, 8), (5, 150, 270, 16),
                                       (5, 200, 300, 32), (4, 260, 190, 64)])
def test_parity_on_the_decoded_stack(storage, L, ny, nx, w):
    stack = make(L, ny, nx, seed=L * 100 + w, n_steady=12, n_pulsed=3, pulse_period=(3, 4))
    res, det, x = run_pair(stack, w, 3.5, F.BRANCH_IMAGE, storage)
    assert_parity(res, det, x, w, 3.5, F.BRANCH_IMAGE, "meanstd")


@pytest.mark.parametrize("noise", ["meanstd", "medmad"])
def test_parity_both_branches(noise):
    stack = make(34, 256, 240, seed=5)
    res, det, x = run_pair(stack, 5, 4.0, F.BRANCH_BOTH, F.BF16, noise)
    assert_parity(res, det, x, 5, 4.0, F.BRANCH_BOTH, noise)
    ok, worst = C.values_close(res["eta"], det.eta * det.M ** 2, rel=1e-4)
    assert ok, worst


@pytest.mark.parametrize("rmode,edge,mmode", [("signed", "partial", "global"),
                                              ("abs", "drop", "global"),
                                              ("abs", "partial", "running")])
def test_parity_options(rmode, edge, mmode):
    stack = make(9, 123, 118, seed=3, n_steady=10, n_pulsed=3, pulse_period=(3, 5))
    res, det, x = run_pair(stack, 5, 3.5, F.BRANCH_IMAGE, F.F16, "medmad", rmode, edge, mmode)
    assert_parity(res, det, x, 5, 3.5, F.BRANCH_IMAGE, "medmad", rmode, edge)
    if mmode == "running":
        assert np.array_equal(res["M_units"], det.M_units)


def test_parity_with_non_finite_pixels():
    stack = make(8, 120, 130, seed=9)
    stack[2, 40, 41] = float("nan")
    stack[5, 100, 7] = float("inf")
    res, det, x = run_pair(stack, 5, 3.5, F.BRANCH_IMAGE, F.BF16)
    assert res["status"] == F.ENONFINITE
    assert_parity(res, det, x, 5, 3.5, F.BRANCH_IMAGE, "meanstd")


@pytest.mark.parametrize("storage", [F.BF16, F.F16])
def test_already_encoded_pushes_give_the_same_detection(storage):
    L, ny, nx = 12, 256, 256     # 256 columns of 2 bytes: unpadded rows, one block copy
    stack = make(L, ny, nx, seed=13)
    key, q = O.delta_encode(stack.cpu().numpy(), FMT[storage])
    enc = torch.from_numpy(q[1:]).to(TDT[storage]).pin_memory()
    outs = []
    for pre in (False, True):
        with F.Plan(nx, ny, L, 5, 3.5, storage=storage, coding=F.CODING_DELTA) as p:
            if pre:
                F.fitrig_push_snapshot(p.h, torch.from_numpy(key).pin_memory())
                F.fitrig_push_snapshots(p.h, enc)
            else:
                F.fitrig_push_snapshots(p.h, stack)
            outs.append(p.detect()[1].tobytes())
            if pre:
                F.fitrig_plan_reset(p.h)
                F.fitrig_push_snapshot(p.h, stack[0])
                F.fitrig_push_snapshot(p.h, enc[0])        # already encoded
                with pytest.raises(F.FitrigError) as e:
                    F.fitrig_push_snapshot(p.h, stack[2])  # the coder's state is behind
                assert e.value.status == F.ESTATE
    assert outs[0] == outs[1]


@pytest.mark.parametrize("kw,status", [
    (dict(storage=F.F32), F.EUNSUPPORTED),
    (dict(storage=F.BF16, window=7), F.EUNSUPPORTED),
    (dict(storage=F.BF16, stride=F.STRIDE_SLIDING), F.EUNSUPPORTED),
    (dict(storage=F.BF16, accumulate=2), F.EUNSUPPORTED)])
def test_unsupported_combinations_are_refused(kw, status):
    w = kw.pop("window", 5)
    with F.Plan(64, 48, 5, w, 3.0, coding=F.CODING_DELTA, **kw) as p:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_push_snapshot(p.h, torch.zeros(48, 64, device="cuda"))
        assert e.value.status == status
    with F.Plan(64, 48, 5, 5, 3.0) as p:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_plan_set(p.h, F.OPT_CODING, 7)
        assert e.value.status == F.EINVAL


def test_batch_with_a_difference_coded_plan_equals_single_plans():
    """A batch that holds a difference-coded plan beside plain ones marches
    plan by plan (no persistent launch) and gives every plan its own detect
    result, bit for bit."""
    specs = [(8, 300, 280, F.CODING_DELTA), (7, 256, 256, F.CODING_VALUE),
             (9, 200, 230, F.CODING_DELTA)]
    plans, single = [], []
    try:
        for k, (L, ny, nx, coding) in enumerate(specs):
            st = make(L, ny, nx, seed=70 + k)
            p = F.Plan(nx, ny, L, 5, 3.5, F.BRANCH_BOTH, F.BF16, F.NOISE_MEDMAD, coding=coding)
            p.push_stack(st)
            plans.append(p)
            single.append(p.detect()[1].tobytes())
        b = F.fitrig_batch_create([p.h for p in plans])
        try:
            for _ in range(2):
                rc, n = F.fitrig_batch_detect(b, len(plans))
                assert rc in (F.OK, F.ENONFINITE)
                for k, p in enumerate(plans):
                    assert F.fitrig_candidates(p.h, int(n[k])).tobytes() == single[k]
        finally:
            F.fitrig_batch_destroy(b)
    finally:
        for p in plans:
            p.close()
