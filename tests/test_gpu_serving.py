"""Serving: snapshots stream in per field; every arrival completes one unit.

* each unit's result equals what the batch trigger gives for that unit;
* a field's results are the same alone and mixed with other fields pushed
  concurrently from several threads (their work overlaps on the device);
* admission queues fields that do not fit the HBM budget, FIFO.
"""
import ctypes
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
            # the latency accounting is ordered and its device times are sane
            assert r["t_arrival_ns"] <= r["t_push_ns"] <= r["t_enqueued_ns"] <= r["t_done_ns"]
            assert 0.0 <= r["copy_ms"] < 1e3 and 0.0 < r["trigger_ms"] < 1e3
            assert r["copy_ms"] + r["trigger_ms"] <= (r["t_done_ns"] - r["t_push_ns"]) / 1e6 + 1.0
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


@pytest.mark.parametrize("nwin,noise", [(14, F.NOISE_MEDMAD), (9, F.NOISE_MEANSTD)])
def test_realtime_frequency_window(nwin, noise):
    """A field admitted with the real-time frequency branch: before its ring of
    nwin units is full a unit has image candidates only; from then on it also
    has the frequency candidates of the last nwin units (tile statistic over
    the running M_s^2), equal to the oracle's on that window: the same tiles
    except where the oracle's z lies within 1e-4 tau of tau, significance to
    1e-4.  Its image candidates equal those of an image-only field."""
    from oracle import fitrig_oracle as O
    L, ny, nx, w, tau = nwin + 8, 120, 131, 4, 4.0
    x = synth.periodic_tile_stack(L, ny, nx, w, 4, 2, (11, 7), 6.0, seed=nwin)
    stack = torch.from_numpy(x)
    srv = F.fitrig_server_create(8 << 30, 4)
    try:
        rc, fid = F.fitrig_server_admit_freq(srv, nx, ny, w, tau, F.F32, noise, nwin)
        rc2, fid2 = F.fitrig_server_admit(srv, nx, ny, w, tau, F.F32, noise)
        assert rc == F.OK and rc2 == F.OK
        serve(srv, fid, stack, torch.float32)
        serve(srv, fid2, stack, torch.float32)
        got = collect(srv)
    finally:
        F.fitrig_server_destroy(srv)
    name = "medmad" if noise == F.NOISE_MEDMAD else "meanstd"
    found_pulse = 0
    for u in range(L - 2):
        r, c = got[(fid, u)]
        assert r["status"] in (F.OK, F.ENONFINITE)
        img, fq = c[c["branch"] == F.BRANCH_IMAGE], c[c["branch"] == F.BRANCH_FREQ]
        assert img.tobytes() == got[(fid2, u)][1].tobytes()
        if u < nwin - 1:
            assert fq.size == 0
            continue
        want, eta, kbin, z = O.freq_window(x[:u + 3], w, tau, nwin, name)
        amb = np.abs(z - tau) <= 1e-4 * tau
        g = {(int(a["y"]) // w, int(a["x"]) // w): a for a in fq}
        o = {(c_.y // w, c_.x // w): c_ for c_ in want}
        for t in set(g) ^ set(o):
            assert amb[t], (u, t)
        for t in set(g) & set(o):
            assert g[t]["snapshot"] == u and o[t].snapshot == u
            assert (int(g[t]["y"]), int(g[t]["x"])) == (o[t].y, o[t].x)
            assert g[t]["significance"] == pytest.approx(o[t].significance, rel=1e-4)
            assert 1 <= g[t]["freq_bin"] <= nwin // 2
        found_pulse += (11, 7) in g
    assert found_pulse >= 1


@pytest.mark.parametrize("nwin", [0, 6])
def test_field_checkpoint_resumes_exactly(nwin):
    """A field exported after 10 of 20 snapshots and imported into another
    server gives, for the next snapshots, byte-identical results to the
    original field (image and real-time frequency candidates, unit numbers)."""
    stack = field_stack(20, 150, 161, seed=40 + nwin)
    srv_a = F.fitrig_server_create(8 << 30, 4)
    srv_b = F.fitrig_server_create(8 << 30, 4)
    try:
        admit = (lambda srv: F.fitrig_server_admit_freq(srv, 161, 150, 5, 4.0, F.F32,
                                                        F.NOISE_MEDMAD, nwin)) if nwin else \
                (lambda srv: F.fitrig_server_admit(srv, 161, 150, 5, 4.0, F.F32, F.NOISE_MEDMAD))
        rc, fa = admit(srv_a)
        assert rc == F.OK
        serve(srv_a, fa, stack[:10], torch.float32)
        collect(srv_a)
        size = ctypes.c_int64()
        lib = F.load()
        assert lib.fitrig_server_field_export(srv_a, fa, None, 0, ctypes.byref(size)) == F.ETRUNC
        image = F.fitrig_server_field_export(srv_a, fa)
        assert len(image) == size.value
        rc, fb = F.fitrig_server_field_import(srv_b, image)
        assert rc == F.OK and F.fitrig_server_field_state(srv_b, fb) == F.FIELD_ACTIVE
        bad = bytearray(image)
        bad[0] ^= 1
        assert lib.fitrig_server_field_import(srv_b, bytes(bad), len(bad),
                                              ctypes.byref(ctypes.c_int32())) == F.EINVAL
        serve(srv_a, fa, stack[10:], torch.float32)
        serve(srv_b, fb, stack[10:], torch.float32)
        ra, rb = collect(srv_a), collect(srv_b)
        assert sorted(u for (_, u) in rb) == list(range(8, 18))
        for u in range(8, 18):
            (r1, c1), (r2, c2) = ra[(fa, u)], rb[(fb, u)]
            assert c1.tobytes() == c2.tobytes(), u
            assert r1["status"] == r2["status"]
    finally:
        F.fitrig_server_destroy(srv_a)
        F.fitrig_server_destroy(srv_b)
