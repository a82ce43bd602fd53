"""CUDA path against the FP64 oracle, element by element and candidate by
candidate, on seeded synthetic stacks.  All calls go through the C ABI."""
import ctypes
import math
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

NOISE = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}
RMODE = {"abs": F.RMODE_ABS, "signed": F.RMODE_SIGNED}
EDGE = {"partial": F.EDGE_PARTIAL, "drop": F.EDGE_DROP}
STORAGE = {"f32": (F.F32, torch.float32), "bf16": (F.BF16, torch.bfloat16),
           "f16": (F.F16, torch.float16)}


def stored(stack_t, storage):
    """The values the library stores (half formats round to nearest even)."""
    tdt = STORAGE[storage][1]
    return stack_t.to(tdt).to(torch.float32).cpu().numpy()


def run_both(stack_t, w, tau, branch=F.BRANCH_IMAGE, noise="meanstd", rmode="abs",
             edge="partial", storage="f32"):
    res = F.detect_stack(stack_t.cuda(), w, tau, branch, STORAGE[storage][0], NOISE[noise],
                         RMODE[rmode], EDGE[edge])
    torch.cuda.synchronize()
    x = stored(stack_t, storage)
    det = O.detect(x, w, tau, branch, noise, rmode, edge)
    return res, det, x


def assert_parity(res, det, x, w, tau, branch, noise="meanstd", rmode="abs", edge="partial",
                  rel=1e-5):
    di, dfq = C.library_decisions(res, tau)
    errs = C.compare(res["candidates"], x, w, tau, branch, noise, rmode, edge, di, dfq, det)
    assert not errs, errs[:10]
    if branch & F.BRANCH_IMAGE:
        ref = np.stack([u.numerator for u in det.units])
        ok, worst = C.values_close(res["values"], ref, rel=rel)
        assert ok, f"tile values differ, worst relative error {worst}"
        assert res["M"] == det.M


# ---------------------------------------------------------------- workloads
def test_config1_full_parity_both_noise_modes():
    """16 snapshots of 512 x 512, window 5, 6 sigma (the small workload)."""
    stack, truth = synth.make_stack(synth.C1, seed=1, device="cuda")
    for noise in ("meanstd", "medmad"):
        res, det, x = run_both(stack, 5, 6.0, F.BRANCH_IMAGE, noise)
        assert_parity(res, det, x, 5, 6.0, F.BRANCH_IMAGE, noise)
        # noise parameters of every unit: same estimator on the same values
        for s in range(x.shape[0] - 2):
            c, sc = res["noise"][s]
            assert sc == pytest.approx(det.scale[s] * det.M ** 2, rel=1e-5)
            assert c == pytest.approx(det.centre[s] * det.M ** 2, rel=1e-5)


@pytest.mark.parametrize("L,ny,nx,w", [
    (5, 37, 53, 4), (6, 64, 70, 7), (4, 33, 33, 33), (3, 20, 31, 1), (8, 100, 90, 16),
    (5, 130, 141, 32), (4, 200, 150, 64), (3, 129, 300, 128), (7, 61, 45, 3), (5, 90, 97, 9),
    (4, 77, 200, 20), (3, 50, 50, 50),
])
def test_ragged_shapes_and_tile_sizes(L, ny, nx, w):
    spec = synth.small_spec(L, ny, nx, n_steady=6, n_pulsed=2, pulse_period=(3, 4))
    stack, _ = synth.make_stack(spec, seed=ny * 7 + nx + w, device="cuda")
    tau = 3.0
    res, det, x = run_both(stack, w, tau)
    assert_parity(res, det, x, w, tau, F.BRANCH_IMAGE)


@pytest.mark.parametrize("rmode", ["abs", "signed"])
@pytest.mark.parametrize("edge", ["partial", "drop"])
@pytest.mark.parametrize("noise", ["meanstd", "medmad"])
def test_options(rmode, edge, noise):
    spec = synth.small_spec(9, 123, 118, n_steady=10, n_pulsed=3, pulse_period=(3, 5))
    stack, _ = synth.make_stack(spec, seed=3, device="cuda")
    res, det, x = run_both(stack, 5, 3.5, F.BRANCH_IMAGE, noise, rmode, edge)
    assert_parity(res, det, x, 5, 3.5, F.BRANCH_IMAGE, noise, rmode, edge)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_half_storage_parity(storage):
    """Half storage: the oracle sees the same rounded values."""
    stack, _ = synth.make_stack(synth.small_spec(10, 256, 256), seed=5, device="cuda")
    res, det, x = run_both(stack, 5, 4.0, F.BRANCH_BOTH, storage=storage)
    assert_parity(res, det, x, 5, 4.0, F.BRANCH_BOTH)


@pytest.mark.parametrize("L,n,w,period", [(64, 120, 5, 4), (66, 96, 4, 8), (32, 64, 8, 3),
                                          (5, 40, 4, 2), (130, 48, 6, 16)])
def test_frequency_branch_parity(L, n, w, period):
    x = synth.periodic_tile_stack(L, n, n + 3, w, period, 1, (2, 3), 6.0, seed=L + n)
    stack = torch.from_numpy(x)
    for noise in ("meanstd", "medmad"):
        res, det, xs = run_both(stack, w, 4.0, F.BRANCH_FREQ, noise)
        assert_parity(res, det, xs, w, 4.0, F.BRANCH_FREQ, noise)
        ok, worst = C.values_close(res["eta"], det.eta / 1.0 * det.M ** 2, rel=1e-4)
        assert ok, worst


def test_both_branches_c2_like():
    spec = synth.small_spec(64, 512, 512)
    stack, _ = synth.make_stack(spec, seed=11, device="cuda")
    res, det, x = run_both(stack, 5, 6.0, F.BRANCH_BOTH, "medmad")
    assert_parity(res, det, x, 5, 6.0, F.BRANCH_BOTH, "medmad")


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("w", [3, 5, 6, 8])
def test_zero_reference_guard(storage, w):
    """Eq. 5: where the reference pixel x^(s+1) is 0, x-hat = C, also when
    0 < Delta < C (r = Delta / C < 1) and when Delta = 0 (r = 0).  The values
    are exact in every storage type (2^-17 and 2^-17 + 2^-22)."""
    spec = synth.small_spec(7, 96, 101, n_steady=4, n_pulsed=1, pulse_period=(3, 4))
    stack, _ = synth.make_stack(spec, seed=40 + w, device="cuda")
    a = 2.0 ** -17
    rs = np.random.default_rng(w)
    for k in range(60):
        s, y, xx = int(rs.integers(0, 5)), int(rs.integers(0, 96)), int(rs.integers(0, 101))
        stack[s, y, xx] = a
        stack[s + 1, y, xx] = 0.0
        stack[s + 2, y, xx] = (a + 2.0 ** -22, a, 3.0)[k % 3]
    res, det, x = run_both(stack, w, 3.0, F.BRANCH_IMAGE, storage=storage)
    assert_parity(res, det, x, w, 3.0, F.BRANCH_IMAGE)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_snapshot_accumulation(storage, k):
    """Sec. 3.3.2: K raw snapshots pushed per stack snapshot are summed in FP32
    in push order and stored in the plan's type; the oracle runs on those
    stored sums."""
    spec = synth.small_spec(7 * k, 96, 101, n_steady=6, n_pulsed=2, pulse_period=(3, 5))
    raw, _ = synth.make_stack(spec, seed=50 + k, device="cuda")
    rawh = raw.cpu()
    res = F.detect_stack(raw, 5, 3.5, F.BRANCH_BOTH, STORAGE[storage][0], accumulate=k)
    x = rawh.numpy().astype(np.float32)
    sums = x[0::k].copy()
    for i in range(1, k):
        sums = (sums + x[i::k]).astype(np.float32)   # FP32, in push order
    stored = torch.from_numpy(sums).to(STORAGE[storage][1]).to(torch.float32).numpy()
    det = O.detect(stored, 5, 3.5, O.BRANCH_BOTH)
    assert_parity(res, det, stored, 5, 3.5, F.BRANCH_BOTH)
    if k > 1:
        assert np.array_equal(O.accumulate(x.astype(np.float64), k).astype(np.float32).shape,
                              stored.shape)


def test_accumulation_pushes_and_reset():
    """Raw pushes (host and device alternating) complete a stack snapshot
    every K; pushing past the stack is refused; a reset starts a new block."""
    k = 3
    raw = torch.randn(3 * k + 1, 40, 44, device="cuda")
    with F.Plan(44, 40, 3, 4, 4.0, accumulate=k) as p:
        for r in range(3 * k):
            F.fitrig_push_snapshot(p.h, raw[r] if r % 2 else raw[r].cpu().numpy())
        lib = F.load()
        rc = lib.fitrig_push_snapshot(p.h, ctypes.c_void_p(raw[3 * k].data_ptr()), F.F32, 1, 0)
        assert rc == F.ESTATE
        rc1, _ = p.detect()
        assert rc1 in F.SOFT
        v1 = F.fitrig_unit_values(p.h, 0).copy()
        F.fitrig_plan_reset(p.h)
        for r in range(3 * k):
            F.fitrig_push_snapshot(p.h, raw[r])
        p.detect()
        assert np.array_equal(F.fitrig_unit_values(p.h, 0), v1)
        assert F.load().fitrig_plan_set(p.h, F.OPT_ACCUMULATE, 2) == F.ESTATE


# ---------------------------------------------------------------- properties
def test_medmad_is_bit_exact_on_own_values():
    spec = synth.small_spec(12, 300, 257)
    stack, _ = synth.make_stack(spec, seed=13, device="cuda")
    res = F.detect_stack(stack, 3, 5.0, F.BRANCH_BOTH, noise=F.NOISE_MEDMAD)
    for s in range(10):
        v = res["values"][s].ravel()
        v = v[np.isfinite(v)]
        med = np.sort(v)[(v.size - 1) // 2]
        mad = np.sort(np.abs(v - med))[(v.size - 1) // 2]   # float32 arithmetic
        c, sc = res["noise"][s]
        assert np.float32(c) == med and c == float(med)
        assert sc == 1.482602218505602 * float(mad)
    e = res["eta"].ravel()
    med = np.sort(e)[(e.size - 1) // 2]
    mad = np.sort(np.abs(e - med))[(e.size - 1) // 2]
    assert res["eta_noise"][0] == float(med)
    assert res["eta_noise"][1] == 1.482602218505602 * float(mad)


def test_identical_snapshots_give_no_candidates():
    one = torch.randn(1, 64, 80, generator=torch.Generator().manual_seed(1))
    stack = one.repeat(6, 1, 1)
    res = F.detect_stack(stack.cuda(), 4, 3.0, F.BRANCH_BOTH)
    assert len(res["candidates"]) == 0
    assert np.all(res["values"] == 0.0)
    assert np.all(res["noise"][:, 1] == 0.0)


def test_nonfinite_pixels_invalidate_tiles():
    spec = synth.small_spec(6, 60, 64, n_steady=4, n_pulsed=1)
    stack, _ = synth.make_stack(spec, seed=17, device="cuda")
    stack[2, 10, 11] = float("nan")
    stack[4, 40, 50] = float("inf")
    stack[0, 5, 5] = float("-inf")
    res, det, x = run_both(stack, 4, 3.0, F.BRANCH_BOTH)
    assert res["status"] == F.ENONFINITE
    assert np.array_equal(np.isnan(res["values"]), np.isnan(det.tlisi))
    assert_parity(res, det, x, 4, 3.0, F.BRANCH_BOTH)


def test_injected_pulse_found_at_its_pixel():
    """A pulse in snapshot k is reported at its pixel in units k and k-2."""
    g = torch.Generator().manual_seed(5)
    stack = torch.randn(9, 96, 96, generator=g)
    k, py, px = 5, 41, 67
    stack[k, py, px] += 60.0
    res = F.detect_stack(stack.cuda(), 4, 5.0)
    hits = {int(c["snapshot"]) for c in res["candidates"] if (c["y"], c["x"]) == (py, px)}
    assert hits == {k - 2, k}


def test_scale_invariance_of_candidates():
    spec = synth.small_spec(8, 128, 128)
    stack, _ = synth.make_stack(spec, seed=19, device="cuda")
    r1 = F.detect_stack(stack, 5, 4.0, F.BRANCH_BOTH)
    r2 = F.detect_stack(stack * 4.0, 5, 4.0, F.BRANCH_BOTH)   # a power of two: exact
    assert np.array_equal(r1["candidates"][["x", "y", "snapshot"]],
                          r2["candidates"][["x", "y", "snapshot"]])
    assert r2["M"] == 4.0 * r1["M"]


def test_graph_replay_matches_eager():
    """Repeated detects of one state replay a captured graph (the second
    captures, the third replays); candidates, tile values, spectrum, noise,
    stage timings and launch counts match the eager detects."""
    spec = synth.small_spec(20, 300, 310, n_steady=10, n_pulsed=3, pulse_period=(3, 6))
    stack, _ = synth.make_stack(spec, seed=21, device="cuda")
    with F.Plan(310, 300, 20, 5, 4.0, F.BRANCH_BOTH, noise=F.NOISE_MEDMAD) as p:
        p.push_stack(stack)
        runs = []
        for graph in (0, 1, 1, 1, 0):
            F.fitrig_plan_set(p.h, F.OPT_GRAPH, graph)
            n0 = F.fitrig_launch_count()
            rc, c = p.detect()
            launches = F.fitrig_launch_count() - n0
            eta, kbin = F.fitrig_spectrum(p.h)
            runs.append((rc, c.tobytes(), F.fitrig_unit_values(p.h, 7).tobytes(), eta.tobytes(),
                         kbin.tobytes(), F.fitrig_noise_params(p.h, 3), launches))
            for k in (F.KERNEL_STACK, F.KERNEL_NOISE, F.KERNEL_SELECT, F.KERNEL_SPECTRUM):
                ms = F.fitrig_kernel_ms(p.h, k)
                assert 0.0 < ms < 100.0, (graph, k, ms)
        assert len(runs[0][1]) > 0
        for r in runs[1:]:
            assert r == runs[0]


def test_determinism():
    stack, _ = synth.make_stack(synth.small_spec(20, 300, 310), seed=23, device="cuda")
    a = F.detect_stack(stack, 5, 4.0, F.BRANCH_BOTH, noise=F.NOISE_MEANSTD)
    b = F.detect_stack(stack, 5, 4.0, F.BRANCH_BOTH, noise=F.NOISE_MEANSTD)
    assert a["candidates"].tobytes() == b["candidates"].tobytes()
    assert a["values"].tobytes() == b["values"].tobytes()
    assert np.array_equal(a["noise"], b["noise"])
    assert a["eta"].tobytes() == b["eta"].tobytes()


def test_tlisi_report_matches_oracle():
    stack, _ = synth.make_stack(synth.small_spec(6, 100, 100), seed=29, device="cuda")
    x = stack.cpu().numpy()
    det = O.detect(x, 5, 4.0)
    with F.Plan(100, 100, 6, 5, 4.0) as p:
        p.push_stack(stack)
        p.detect()
        for s in range(4):
            t = F.fitrig_tlisi(p.h, s)
            np.testing.assert_allclose(t, det.tlisi[s], rtol=0, atol=1e-6)


@pytest.mark.parametrize("noise", ["meanstd", "medmad"])
@pytest.mark.parametrize("tau", [3.0, 4.0])
def test_threshold_stage_gaussian_tail(noise, tau):
    """Exceedances of a pure N(0,1) map match Q(tau) within 4 binomial sigma."""
    from scipy.special import erfc
    n = 100_000_000
    g = torch.Generator(device="cuda").manual_seed(int(tau))
    v = torch.randn(n, device="cuda", generator=g)
    k, c, s = F.fitrig_threshold_map(v, tau, NOISE[noise], torch.cuda.current_stream().cuda_stream)
    q = 0.5 * erfc(tau / math.sqrt(2.0))
    sd = math.sqrt(n * q * (1 - q))
    slack = 4 * sd + (0.002 * n * q if noise == "medmad" else 0.0)
    assert abs(k - n * q) <= slack, (k, n * q)
    assert abs(c) < 1e-3 and abs(s - 1.0) < 1e-3


def test_push_conversions_and_pitches():
    """fp32 input into half storage, host input, and padded row pitch."""
    stack, _ = synth.make_stack(synth.small_spec(5, 70, 90), seed=31, device="cuda")
    ref = F.detect_stack(stack.to(torch.bfloat16), 5, 3.0, storage=F.BF16)
    with F.Plan(90, 70, 5, 5, 3.0, storage=F.BF16) as p:
        big = torch.zeros(5, 70, 128, device="cuda")
        big[:, :, :90] = stack
        for k in range(5):
            if k % 2:
                F.fitrig_push_snapshot(p.h, big[k, :, :90])          # device, pitch 128
            else:
                F.fitrig_push_snapshot(p.h, stack[k].cpu().numpy())  # host fp32
        rc, c = p.detect()
        vals = np.stack([F.fitrig_unit_values(p.h, s) for s in range(3)])
    assert vals.tobytes() == ref["values"].tobytes()
    assert c.tobytes() == ref["candidates"].tobytes()


def test_state_errors():
    with F.Plan(32, 32, 4, 4, 3.0) as p:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_detect(p.h)
        assert e.value.status == F.ESTATE
        x = torch.randn(4, 32, 32, device="cuda")
        p.push_stack(x)
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_push_snapshot(p.h, x[0])
        assert e.value.status == F.ESTATE
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_plan_set(p.h, F.OPT_STORAGE, F.BF16)
        assert e.value.status == F.ESTATE
        p.detect()
        F.fitrig_plan_reset(p.h)
        p.push_stack(x)
        rc, _ = p.detect()
        assert rc == F.OK


@pytest.mark.parametrize("storage", [F.F32, F.BF16])
def test_autotuned_shape_gives_identical_results(storage):
    """The autotuner only changes the CTA shape, never a tile's arithmetic."""
    tby, ns, ms = F.fitrig_autotune(5, storage)
    assert tby in (2, 4, 8) and 2 <= ns <= 6 and ms > 0
    stack, _ = synth.make_stack(synth.small_spec(12, 333, 250), seed=37, device="cuda")
    tdt = torch.float32 if storage == F.F32 else torch.bfloat16
    a = F.detect_stack(stack.to(tdt), 5, 4.0, F.BRANCH_BOTH, storage=storage)
    b = F.detect_stack(stack.to(tdt), 5, 4.0, F.BRANCH_BOTH, storage=storage, autotune=True)
    assert a["values"].tobytes() == b["values"].tobytes()
    assert a["candidates"].tobytes() == b["candidates"].tobytes()


def test_selection_capacity_truncates_loudly():
    """A detect that selects more tiles than MAX_SELECTED returns ETRUNC; with
    room for them the same stack gives the full candidate list."""
    stack, _ = synth.make_stack(synth.small_spec(10, 200, 200), seed=5, device="cuda")
    L, ny, nx = stack.shape
    with F.Plan(nx, ny, L, 4, 2.0, F.BRANCH_IMAGE, noise=F.NOISE_MEDMAD) as p:
        p.push_stack(stack)
        rc, full = p.detect()
        assert rc in (F.OK, F.ENONFINITE) and len(full) > 8
    with F.Plan(nx, ny, L, 4, 2.0, F.BRANCH_IMAGE, noise=F.NOISE_MEDMAD, max_selected=8) as p:
        p.push_stack(stack)
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_detect(p.h)
        assert e.value.status == F.ETRUNC and e.value.needed > 8
        # resize in place to the reported need and detect again
        F.fitrig_plan_set(p.h, F.OPT_MAX_SELECTED, e.value.needed)
        rc, again = p.detect()
        assert again.tobytes() == full.tobytes()
    with F.Plan(nx, ny, L, 4, 2.0) as p:
        with pytest.raises(F.FitrigError) as e:
            F.fitrig_plan_set(p.h, F.OPT_MAX_SELECTED, -1)
        assert e.value.status == F.EINVAL


class _DeviceArray:
    """A borrowed device buffer seen through the CUDA array interface."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                         "typestr": typestr, "version": 2, "strides": None}


def device_view(ptr, pitch, rows, tdt):
    if tdt == torch.bfloat16:   # no array-interface code for bfloat16: view its bits
        t = torch.as_tensor(_DeviceArray(ptr, (rows, pitch), "<i2"), device="cuda")
        return t.view(torch.bfloat16)
    code = {torch.float32: "<f4", torch.float16: "<f2"}[tdt]
    return torch.as_tensor(_DeviceArray(ptr, (rows, pitch), code), device="cuda")


@pytest.mark.parametrize("storage,host_dtype,pad", [(F.F32, torch.float32, 0),
                                                   (F.F32, torch.float32, 96),
                                                   (F.BF16, torch.float32, 0),
                                                   (F.F16, torch.float16, 40)])
def test_large_host_pushes_land_exactly(storage, host_dtype, pad):
    """Snapshots of >= 32 MB from host memory go in row bands over several
    streams; the stored stack equals the device-side conversion of the input."""
    ny, nx, L = 4200, 4001, 3   # >= 32 MiB per snapshot in every case
    x = torch.randn(L, ny, nx + pad, dtype=torch.float32).to(host_dtype).pin_memory()
    tdt = {F.F32: torch.float32, F.BF16: torch.bfloat16, F.F16: torch.float16}[storage]
    with F.Plan(nx, ny, L, 5, 4.0, storage=storage) as p:
        for k in range(L):
            F.fitrig_push_snapshot(p.h, x[k, :, :nx], row_pitch_elems=nx + pad)
        torch.cuda.synchronize()
        for k in range(L):
            got = device_view(*F.fitrig_stack_device_ptr(p.h, k), ny, tdt)
            want = x[k, :, :nx].cuda().to(tdt)
            assert torch.equal(got[:, :nx], want), k


@pytest.mark.parametrize("storage,host_dtype,nx,pad,k,dev", [
    (F.F32, torch.float32, 2048, 0, 1, 0),     # contiguous: one banded transfer
    (F.F32, torch.float32, 2001, 0, 1, 0),     # padded device rows
    (F.F32, torch.float32, 2048, 64, 1, 0),    # padded host rows
    (F.BF16, torch.float32, 2048, 0, 1, 0),    # converted on the device
    (F.F32, torch.float32, 1000, 0, 2, 0),     # accumulation, K = 2
    (F.F16, torch.float16, 1000, 8, 1, 1)])    # device block
def test_block_push_equals_single_pushes(storage, host_dtype, nx, pad, k, dev):
    """fitrig_push_snapshots stores exactly what one push per snapshot stores
    and gives the same candidates."""
    ny, L = 1100, 6
    x = torch.randn(L * k, ny, nx + pad, dtype=torch.float32).to(host_dtype)
    x = x.cuda() if dev else x.pin_memory()
    tdt = {F.F32: torch.float32, F.BF16: torch.bfloat16, F.F16: torch.float16}[storage]
    out = []
    for block in (False, True):
        with F.Plan(nx, ny, L, 5, 4.0, storage=storage, accumulate=k) as p:
            if block:
                F.fitrig_push_snapshots(p.h, x[:2 * k + 1, :, :nx])   # ragged: one partial slot
                F.fitrig_push_snapshots(p.h, x[2 * k + 1:, :, :nx])
                with pytest.raises(F.FitrigError) as e:
                    F.fitrig_push_snapshots(p.h, x[:1, :, :nx])
                assert e.value.status == F.ESTATE
            else:
                for r in range(L * k):
                    F.fitrig_push_snapshot(p.h, x[r, :, :nx])
            torch.cuda.synchronize()
            st = torch.stack([device_view(*F.fitrig_stack_device_ptr(p.h, s), ny, tdt)[:, :nx]
                              for s in range(L)]).clone()
            rc, c = p.detect()
            out.append((st, c))
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1].tobytes() == out[1][1].tobytes()
    if k == 1 and storage == F.F32 and host_dtype == torch.float32:
        assert torch.equal(out[1][0].cpu(), x[:, :, :nx].cpu())


def test_block_push_rejects_bad_arguments():
    with F.Plan(64, 32, 4, 4, 3.0) as p:
        x = torch.randn(4, 32, 64, device="cuda")
        lib = F.load()
        assert lib.fitrig_push_snapshots(p.h, ctypes.c_void_p(x.data_ptr()), -1, F.F32, 1, 0, 0) == F.EINVAL
        assert lib.fitrig_push_snapshots(p.h, ctypes.c_void_p(x.data_ptr()), 2, F.F32, 1, 0, 100) == F.EINVAL
        assert lib.fitrig_push_snapshots(p.h, ctypes.c_void_p(x.data_ptr()), 5, F.F32, 1, 0, 0) == F.ESTATE
        assert lib.fitrig_push_snapshots(p.h, ctypes.c_void_p(x.data_ptr()), 0, F.F32, 1, 0, 0) == F.OK
        F.fitrig_push_snapshots(p.h, x)
        rc, _ = p.detect()
        assert rc in (F.OK,)


def test_candidates_into_a_caller_buffer():
    """A reused (pinned) output buffer gets the same candidates; a short one
    the first of them."""
    stack, _ = synth.make_stack(synth.small_spec(8, 96, 128), seed=5, device="cuda")
    with F.Plan(128, 96, 8, 5, 2.0, branch=F.BRANCH_BOTH) as p:
        p.push_stack(stack)
        rc, want = p.detect()
        assert len(want) > 2
        raw = torch.empty((len(want) + 3) * F.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8,
                          pin_memory=True)
        buf = raw.numpy().view(F.CANDIDATE_DTYPE)
        got = F.fitrig_candidates(p.h, out=buf)
        assert got.tobytes() == want.tobytes()
        assert got.ctypes.data == buf.ctypes.data
        assert F.fitrig_candidates(p.h, out=buf[:2]).tobytes() == want[:2].tobytes()


def test_selection_lists_grow_automatically():
    """A detect that selects more tiles than the starting capacity grows the
    lists and gives the same result as a plan sized for every tile."""
    stack = torch.randn(40, 2048, 2048, device="cuda")
    L, ny, nx = stack.shape
    w, tau = 2, 0.25
    U, T = L - 2, (ny // w) * (nx // w)
    with F.Plan(nx, ny, L, w, tau, F.BRANCH_IMAGE, noise=F.NOISE_MEDMAD) as p:
        p.push_stack(stack)
        rc, auto = p.detect()
        rc2, again = p.detect()       # now within the grown capacity
        selected = 0
        for s in range(U):
            c, sc = F.fitrig_noise_params(p.h, s)
            v = F.fitrig_unit_values(p.h, s).astype(np.float64)
            selected += int(np.count_nonzero(v > c + tau * sc))
    assert selected > (4 << 20) + U * T // 12      # beyond the starting capacity
    with F.Plan(nx, ny, L, w, tau, F.BRANCH_IMAGE, noise=F.NOISE_MEDMAD,
                max_selected=U * T) as p:
        p.push_stack(stack)
        rc3, full = p.detect()
    assert rc == rc2 == rc3
    assert auto.tobytes() == full.tobytes() == again.tobytes()


@pytest.mark.parametrize("stride", ["tile", "sliding"])
def test_running_M_reading(stride):
    """Real-time normaliser: unit s divided by the maximum of snapshots 0..s+2.
    M_s, the reported tLISI, eta and both branches' candidates against the
    oracle run with the same reading."""
    spec = synth.small_spec(12, 150, 170, n_pulsed=3, pulse_period=(3, 4))
    stack, _ = synth.make_stack(spec, seed=77, device="cuda")
    ramp = torch.linspace(100.0, 700.0, stack.shape[0], device="cuda")
    stack[:, 5, 7] = ramp                      # the maximum grows snapshot by snapshot
    w, tau = (5, 3.0) if stride == "tile" else (3, 4.0)
    st = F.STRIDE_TILE if stride == "tile" else F.STRIDE_SLIDING
    res = F.detect_stack(stack, w, tau, F.BRANCH_BOTH, noise=F.NOISE_MEDMAD, stride=st,
                         mmode=F.MMODE_RUNNING)
    x = stack.cpu().numpy()
    det = O.detect(x, w, tau, F.BRANCH_BOTH, "medmad", stride=stride, mmode="running")
    assert list(res["M_units"]) == list(det.M_units)
    assert len(set(det.M_units)) > 3           # the reading really differs from one M
    assert res["M"] == det.M
    di, dfq = C.library_decisions(res, tau)
    if stride == "tile":
        errs = C.compare(res["candidates"], x, w, tau, F.BRANCH_BOTH, "medmad", "abs",
                         "partial", di, dfq, det)
        assert not errs, errs[:10]
    ok, worst = C.values_close(res["eta"], det.eta * det.M ** 2, rel=1e-4)
    assert ok, worst
    glob = F.detect_stack(stack, w, tau, F.BRANCH_IMAGE, noise=F.NOISE_MEDMAD, stride=st)
    img = res["candidates"][res["candidates"]["snapshot"] >= 0]
    assert img.tobytes() == glob["candidates"].tobytes()   # z does not see M_s
    with F.Plan(170, 150, 12, w, tau, F.BRANCH_IMAGE, stride=st, mmode=F.MMODE_RUNNING) as p:
        p.push_stack(stack)
        p.detect()
        for s in (0, 4, 9):
            t = F.fitrig_tlisi(p.h, s)
            ok, worst = C.values_close(t, det.tlisi[s], rel=1e-6)
            assert ok, (s, worst)


def test_device_pushes_wait_for_their_producer():
    """Snapshots computed on the default stream and pushed straight away (their
    memory is reused right after) land intact in the plan's stack."""
    L, ny, nx = 8, 2048, 2048
    kept = []
    with F.Plan(nx, ny, L, 5, 4.0, storage=F.BF16) as p:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        for k in range(L):
            img = torch.randn(ny, nx, generator=gen, device="cuda")
            snap = torch.fft.irfft2(torch.fft.rfft2(img) * 0.5, s=(ny, nx))   # a few kernels
            F.fitrig_push_snapshot(p.h, snap)
            kept.append(snap.to(torch.bfloat16).cpu())
            del img, snap
        torch.cuda.synchronize()
        for k in range(L):
            got = device_view(*F.fitrig_stack_device_ptr(p.h, k), ny, torch.bfloat16)
            assert torch.equal(got[:, :nx].cpu(), kept[k]), k


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """Failure detection without a fault: one device wait, bounded exactly as
    the trigger's TMA waits are, on an mbarrier that nothing ever completes
    gives up after its bound and reports ETIMEOUT; the context stays usable
    (a detect right after equals one made before)."""
    stack, _ = synth.make_stack(synth.small_spec(8, 200, 210), seed=78, device="cuda")
    before = F.detect_stack(stack, 5, 4.0, F.BRANCH_BOTH, dumps=False)
    lib = F.load()
    t0 = time.perf_counter()
    assert lib.fitrig_wait_probe(20_000_000, 0) == F.ETIMEOUT   # 20 ms bound
    assert time.perf_counter() - t0 < 5.0
    after = F.detect_stack(stack, 5, 4.0, F.BRANCH_BOTH, dumps=False)
    assert after["candidates"].tobytes() == before["candidates"].tobytes()
