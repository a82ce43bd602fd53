"""Serving: snapshots stream in per field; every arrival completes one unit.

* each unit's result equals what the batch trigger gives for that unit;
* a field's results are the same alone and mixed with other fields pushed
  concurrently from several threads (their work overlaps on the device);
* admission queues fields that do not fit the HBM budget, FIFO.
"""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2509_21754_gb300 import fitrig as F  # noqa: E402
from paper_2509_21754_gb300 import synth  # noqa: E402


def field_stack(L, ny, nx, seed):
    spec = synth.small_spec(L, ny, nx, n_pulsed=3, pulse_period=(3, 5))
    st, _ = synth.make_stack(spec, seed=seed, device="cuda")
    return st.cpu()


def serve(server, fid, stack, tdt):
    host = stack.to(tdt).contiguous()
    for k in range(host.shape[0]):
        assert F.fitrig_server_push(server, fid, host[k], time.monotonic_ns()) == F.OK


def collect(server):
    F.fitrig_server_drain(server)
    res, cands = F.fitrig_server_poll(server)
    out = {}
    for r in res:
        c = cands[r["cand_offset"]:r["cand_offset"] + r["ncand"]]
        out[(int(r["field"]), int(r["unit"]))] = (r, c)
    return out


@pytest.mark.parametrize("storage,tdt,noise,w", [(F.BF16, torch.bfloat16, F.NOISE_MEDMAD, 5),
                                                 (F.F32, torch.float32, F.NOISE_MEANSTD, 9)])
def test_units_equal_batch_trigger(storage, tdt, noise, w):
    stack = field_stack(11, 300, 283, seed=1)
    L, ny, nx = stack.shape
    ref = F.detect_stack(stack.to(tdt).cuda(), w, 4.0, F.BRANCH_IMAGE, storage, noise, dumps=False)
    srv = F.fitrig_server_create(8 << 30, 4)
    try:
        rc, fid = F.fitrig_server_admit(srv, nx, ny, w, 4.0, storage, noise)
        assert rc == F.OK and F.fitrig_server_field_state(srv, fid) == F.FIELD_ACTIVE
        serve(srv, fid, stack, tdt)
        got = collect(srv)
        assert sorted(u for (_, u) in got) == list(range(L - 2))
        for s in range(L - 2):
            r, c = got[(fid, s)]
            want = ref["candidates"][ref["candidates"]["snapshot"] == s]
            assert r["status"] in (F.OK, F.ENONFINITE)
            assert c.tobytes() == want.tobytes(), s
            assert r["t_done_ns"] >= r["t_arrival_ns"]
    finally:
        F.fitrig_server_destroy(srv)


def test_alone_equals_mixed():
    stacks = [field_stack(9, 256 + 40 * k, 240 + 31 * k, seed=10 + k) for k in range(4)]

    def run(fields):
        srv = F.fitrig_server_create(16 << 30, 8)
        try:
            ids = []
            for st in fields:
                rc, fid = F.fitrig_server_admit(srv, st.shape[2], st.shape[1], 5, 4.0, F.BF16,
                                                F.NOISE_MEDMAD)
                assert rc == F.OK
                ids.append(fid)
            threads = [threading.Thread(target=serve, args=(srv, fid, st, torch.bfloat16))
                       for fid, st in zip(ids, fields)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            return ids, collect(srv)
        finally:
            F.fitrig_server_destroy(srv)

    ids_alone, alone = run(stacks[:1])
    ids_mix, mixed = run(stacks)
    assert len(mixed) == sum(st.shape[0] - 2 for st in stacks)
    for s in range(stacks[0].shape[0] - 2):
        ra, ca = alone[(ids_alone[0], s)]
        rm, cm = mixed[(ids_mix[0], s)]
        assert ca.tobytes() == cm.tobytes()
        assert ra["status"] == rm["status"]


def test_admission_is_fifo_under_the_budget():
    probe = F.fitrig_server_create(1 << 40, 8)
    try:
        rc, f0 = F.fitrig_server_admit(probe, 512, 512, 5, 4.0, F.F32, F.NOISE_MEDMAD)
        one, _, _ = F.fitrig_server_usage(probe)
    finally:
        F.fitrig_server_destroy(probe)
    srv = F.fitrig_server_create(int(2.5 * one), 8)   # room for two such fields
    try:
        states = [F.fitrig_server_admit(srv, 512, 512, 5, 4.0, F.F32, F.NOISE_MEDMAD) for _ in range(4)]
        assert [rc for rc, _ in states] == [F.OK, F.OK, F.EBUSY, F.EBUSY]
        used, active, waiting = F.fitrig_server_usage(srv)
        assert (active, waiting) == (2, 2) and used == 2 * one
        x = torch.randn(512, 512)
        assert F.fitrig_server_push(srv, states[2][1], x, 0) == F.EBUSY
        F.fitrig_server_retire(srv, states[0][1])
        assert F.fitrig_server_field_state(srv, states[2][1]) == F.FIELD_ACTIVE
        assert F.fitrig_server_field_state(srv, states[3][1]) == F.FIELD_QUEUED
        assert F.fitrig_server_field_state(srv, states[0][1]) == F.FIELD_RETIRED
        assert F.fitrig_server_push(srv, states[2][1], x, 0) == F.OK
    finally:
        F.fitrig_server_destroy(srv)
