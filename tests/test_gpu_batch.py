"""Batches: many fields of uneven size and snapshot count, one persistent stack
march and one CUDA graph, must give each plan exactly its own detect result."""
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


def fields(n, seed, storage=torch.bfloat16):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(rng.integers(96, 700))
        L = int(rng.integers(5, 40))
        spec = synth.small_spec(L, side, side + int(rng.integers(-40, 40)), layout="ska_aa2_like",
                                n_ant=68)
        st, _ = synth.make_stack(spec, seed=seed * 100 + k, device="cuda")
        out.append(st.to(storage))
    return out


@pytest.mark.parametrize("storage,tdt,noise,branch", [
    (F.BF16, torch.bfloat16, F.NOISE_MEDMAD, F.BRANCH_BOTH),
    (F.F32, torch.float32, F.NOISE_MEANSTD, F.BRANCH_IMAGE),
])
def test_batch_equals_single_plans(storage, tdt, noise, branch):
    stacks = fields(9, seed=3, storage=tdt)
    plans = []
    try:
        for st in stacks:
            L, ny, nx = st.shape
            p = F.Plan(nx, ny, L, 5, 4.0, branch, storage, noise)
            p.push_stack(st)
            plans.append(p)
        single = []
        for p in plans:
            rc, c = p.detect()
            single.append((c.copy(), [F.fitrig_unit_values(p.h, s).tobytes()
                                      for s in range(p.nsnap - 2)]))
        b = F.fitrig_batch_create(plans)
        try:
            for rep in range(3):   # first call captures the graph, then replays
                rc, n = F.fitrig_batch_detect(b, len(plans))
                assert rc in (F.OK, F.ENONFINITE)
                for k, p in enumerate(plans):
                    c = F.fitrig_candidates(p.h, int(n[k]))
                    assert c.tobytes() == single[k][0].tobytes()
                    vals = [F.fitrig_unit_values(p.h, s).tobytes() for s in range(p.nsnap - 2)]
                    assert vals == single[k][1]
            assert F.fitrig_batch_ms(b) > 0
        finally:
            F.fitrig_batch_destroy(b)
    finally:
        for p in plans:
            p.close()


def test_batch_field_against_oracle():
    stacks = fields(4, seed=5, storage=torch.float32)
    plans = []
    try:
        for st in stacks:
            L, ny, nx = st.shape
            p = F.Plan(nx, ny, L, 5, 4.0, F.BRANCH_BOTH)
            p.push_stack(st)
            plans.append(p)
        b = F.fitrig_batch_create(plans)
        try:
            rc, n = F.fitrig_batch_detect(b, len(plans))
        finally:
            F.fitrig_batch_destroy(b)
        k = 2
        x = stacks[k].cpu().numpy()
        det = O.detect(x, 5, 4.0, O.BRANCH_BOTH)
        p = plans[k]
        res = {"values": np.stack([F.fitrig_unit_values(p.h, s) for s in range(x.shape[0] - 2)]),
               "noise": np.array([F.fitrig_noise_params(p.h, s) for s in range(x.shape[0] - 2)])}
        res["eta"], res["bin"] = F.fitrig_spectrum(p.h)
        res["eta_noise"] = F.fitrig_noise_params(p.h, -1)
        di, dfq = C.library_decisions(res, 4.0)
        errs = C.compare(F.fitrig_candidates(p.h, int(n[k])), x, 5, 4.0, O.BRANCH_BOTH,
                         decide_image=di, decide_freq=dfq, det=det)
        assert not errs, errs[:8]
    finally:
        for p in plans:
            p.close()


def test_batch_of_c4_sized_fields_against_oracle():
    """The batched workload's recipe at a size the oracle finishes in seconds:
    six SKA-AA2-like fields of 1024..4096 pixels square and 16..40 snapshots,
    BF16 storage, both branches, median/MAD, window 5, 6 sigma, in one
    persistent march and graph; every field's candidate list equals the
    oracle's on the stored values by the parity rule."""
    rng = np.random.default_rng(44)
    shapes = [(16, 4096), (40, 1024), (24, 1536), (16, 2048), (33, 1280), (20, 1100)]
    stacks, plans = [], []
    try:
        for k, (L, side) in enumerate(shapes):
            spec = synth.small_spec(L, side, side + int(rng.integers(-16, 17)),
                                    layout="ska_aa2_like", n_ant=68)
            st, _ = synth.make_stack(spec, seed=4400 + k, device="cuda")
            st = st.to(torch.bfloat16)
            p = F.Plan(st.shape[2], st.shape[1], L, 5, 6.0, F.BRANCH_BOTH, F.BF16, F.NOISE_MEDMAD)
            p.push_stack(st)
            stacks.append(st)
            plans.append(p)
        b = F.fitrig_batch_create(plans)
        try:
            F.fitrig_batch_detect(b, len(plans))
            rc, n = F.fitrig_batch_detect(b, len(plans))   # the captured graph
            assert rc in (F.OK, F.ENONFINITE)
        finally:
            F.fitrig_batch_destroy(b)
        for k, p in enumerate(plans):
            x = stacks[k].float().cpu().numpy()
            L = x.shape[0]
            det = O.detect(x, 5, 6.0, O.BRANCH_BOTH, "medmad")
            res = {"values": np.stack([F.fitrig_unit_values(p.h, s) for s in range(L - 2)]),
                   "noise": np.array([F.fitrig_noise_params(p.h, s) for s in range(L - 2)])}
            res["eta"], res["bin"] = F.fitrig_spectrum(p.h)
            res["eta_noise"] = F.fitrig_noise_params(p.h, -1)
            di, dfq = C.library_decisions(res, 6.0)
            cands = F.fitrig_candidates(p.h, int(n[k]))
            errs = C.compare(cands, x, 5, 6.0, O.BRANCH_BOTH, "medmad", decide_image=di,
                             decide_freq=dfq, det=det)
            assert not errs, (k, errs[:8])
            assert len(cands) > 0
    finally:
        for p in plans:
            p.close()
