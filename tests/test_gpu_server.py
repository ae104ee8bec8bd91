"""Serving loop (elas_server_*): requests of mixed shapes from several
simulated cameras are admitted into resident slots and run in overlapping
waves of batched launches.  Every result must equal the oracle's for that
pair and the per-pair path's (the same pair alone), whatever else ran in its
wave, under a tight HBM budget (slots released and re-created), and in the
plain one-at-a-time mode."""
import ctypes as C
import time

import numpy as np
import pytest

import oracle
from paper_1802_07210_gb300 import synth
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _B():
    from paper_1802_07210_gb300 import binding
    return binding


def _cameras():
    ragged = synth.scaled_workload(203, 117, 48)
    ragged.params["disp_min"] = 3
    mid = synth.scaled_workload(400, 300, 128)
    return [("small", synth.SMALL_320, 1), ("ragged", ragged, 7), ("mid", mid, 4)]


CAMS = _cameras()


@pytest.fixture(scope="module")
def requests():
    """12 requests: 4 per camera, seeded; oracle maps for the first of each."""
    out = []
    rid = 0
    for ci, (name, wl, cfg) in enumerate(CAMS):
        for k in range(4):
            L, R, _ = synth.workload_pair(wl, k, cfg)
            prm = dict(wl.params)
            post = (k % 2 == 1)
            if post:
                prm.update(ipol_gap_width=3, filter_adaptive_mean=1)
            ref = oracle.pipeline(L, R, prm, postprocess_on=post) if k < 2 else None
            out.append(dict(id=rid, cam=name, L=L, R=R, prm=prm, post=post, ref=ref))
            rid += 1
    return out


def _alone(req):
    """The per-pair path's maps for one request."""
    B = _B()
    h, w = req["L"].shape
    pl = B.Pipeline(w, h, req["prm"])
    dL = torch.empty((h, w), dtype=torch.int16, device="cuda")
    post = torch.empty((h, w), dtype=torch.float32, device="cuda") if req["post"] else None
    pl.run(dev(req["L"]), dev(req["R"]), dL, None, post)
    res = host(dL), (host(post) if post is not None else None)
    pl.close()
    return res


@pytest.fixture(scope="module")
def alone(requests):
    return {r["id"]: _alone(r) for r in requests}


def _serve(srv, reqs, stagger_s=0.0):
    bufs = {}
    for i, r in enumerate(reqs):
        h, w = r["L"].shape
        bufs[r["id"]] = dict(
            L=torch.from_numpy(r["L"]).pin_memory(), R=torch.from_numpy(r["R"]).pin_memory(),
            dL=torch.full((h, w), -7, dtype=torch.int16).pin_memory(),
            post=torch.zeros((h, w), dtype=torch.float32).pin_memory() if r["post"] else None)
    results = {}
    for i, r in enumerate(reqs):
        b = bufs[r["id"]]
        srv.submit(r["id"], b["L"], b["R"], b["dL"], r["prm"], b["post"])
        if stagger_s:
            time.sleep(stagger_s)
        for res in srv.poll(64, 0):
            results[res["id"]] = res
    t0 = time.time()
    while len(results) < len(reqs):
        for res in srv.poll(64, 200):
            results[res["id"]] = res
        assert time.time() - t0 < 120, "server did not finish"
    return results, bufs


def _check(reqs, results, bufs, alone):
    for r in reqs:
        res = results[r["id"]]
        assert res["status"] == 0, (r["cam"], res)
        b = bufs[r["id"]]
        aL, apost = alone[r["id"]]
        np.testing.assert_array_equal(b["dL"].numpy(), aL, err_msg="request %d (%s)" % (r["id"], r["cam"]))
        if r["post"]:
            np.testing.assert_array_equal(b["post"].numpy(), apost)
        if r["ref"] is not None:
            np.testing.assert_array_equal(b["dL"].numpy(), r["ref"]["lrL"])
            assert res["n_support"] == len(r["ref"]["list"])
            if r["post"]:
                assert np.abs(b["post"].numpy() - r["ref"]["post"]).max() <= 1e-4
        assert res["t_submit_ms"] <= res["t_start_ms"] <= res["t_done_ms"]


def test_burst_matches_oracle_and_alone(requests, alone):
    B = _B()
    srv = B.Server(lanes=3, max_wave=8)
    results, bufs = _serve(srv, requests)
    _check(requests, results, bufs, alone)
    st = srv.stats()
    assert st["completed"] == len(requests) and st["max_wave_seen"] >= 2
    srv.close()


def test_arrivals_during_waves_overlap(requests, alone):
    """Requests that arrive while waves run are queued and join later waves
    on the other lanes; those waves overlap on the device."""
    B = _B()
    srv = B.Server(lanes=3, max_wave=4)
    reqs = requests * 2
    reqs = [dict(r, id=i) for i, r in enumerate(reqs)]
    al = {i: alone[requests[i % len(requests)]["id"]] for i in range(len(reqs))}
    results, bufs = _serve(srv, reqs)
    _check(reqs, results, bufs, al)
    spans = sorted((r["t_start_ms"], r["t_done_ms"]) for r in results.values())
    overlap = any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    assert overlap, "no wave started while another was in flight"
    assert max(r["wave_size"] for r in results.values()) > 1
    assert srv.stats()["waves"] >= len(reqs) // 4
    srv.close()


def test_tight_budget_releases_and_recreates_slots(requests, alone):
    B = _B()
    sizes = {}
    for r in requests:
        h, w = r["L"].shape
        sizes[r["cam"]] = B.lib().elas_slot_device_bytes(w, h, C.byref(B.as_params(r["prm"])))
    assert all(v > 0 for v in sizes.values())
    budget = max(sizes.values()) + min(sizes.values())  # never room for every shape at once
    srv = B.Server(lanes=2, max_wave=4, hbm_budget_bytes=budget)
    results, bufs = _serve(srv, requests)
    _check(requests, results, bufs, alone)
    st = srv.stats()
    assert st["slots_released"] > 0
    assert st["slot_bytes"] <= budget
    srv.close()


def test_plain_mode_is_identical(requests, alone):
    B = _B()
    srv = B.Server(plain=True)
    results, bufs = _serve(srv, requests)
    _check(requests, results, bufs, alone)
    assert all(r["wave_size"] == 1 for r in results.values())
    srv.close()


def test_request_errors(requests):
    B = _B()
    r = requests[0]
    h, w = r["L"].shape
    srv = B.Server(lanes=1, max_wave=2, hbm_budget_bytes=1 << 20)  # 1 MiB: no slot fits
    L = torch.from_numpy(r["L"]).pin_memory()
    R = torch.from_numpy(r["R"]).pin_memory()
    dL = torch.empty((h, w), dtype=torch.int16).pin_memory()
    with pytest.raises(B.ElasError):
        srv.submit(1, L, R, dL, dict(r["prm"], disp_max=5000))
    srv.submit(2, L, R, dL, r["prm"])
    got = []
    t0 = time.time()
    while not got and time.time() - t0 < 30:
        got = srv.poll(4, 200)
    assert got and got[0]["id"] == 2 and got[0]["status"] == 5  # ELAS_ERR_NO_MEMORY
    srv.close()


def _one(srv, rid, r):
    h, w = r["L"].shape
    bufs = dict(L=torch.from_numpy(r["L"]).pin_memory(), R=torch.from_numpy(r["R"]).pin_memory(),
                dL=torch.full((h, w), -7, dtype=torch.int16).pin_memory())
    srv.submit(rid, bufs["L"], bufs["R"], bufs["dL"], r["prm"])
    got = []
    t0 = time.time()
    while not got:
        got = srv.poll(4, 200)
        assert time.time() - t0 < 60, "no result"
    return got[0], bufs


def test_refused_allocation_releases_idle_slots(requests, alone):
    """A slot allocation the device refuses (injected on the host, as when
    other users hold the memory) releases an idle slot of another shape and
    retries; with nothing idle and nothing running the request fails with
    ELAS_ERR_NO_MEMORY instead of waiting forever, and the server goes on."""
    B = _B()
    srv = B.Server(lanes=1, max_wave=2)
    a, b, c = requests[0], requests[4], requests[8]  # three shapes
    res, bufs = _one(srv, 1, a)
    assert res["status"] == 0
    np.testing.assert_array_equal(bufs["dL"].numpy(), alone[a["id"]][0])
    # one refusal: the idle slot of a's shape is released, b's is then created
    srv.inject_alloc_failures(1)
    res, bufs = _one(srv, 2, b)
    assert res["status"] == 0
    np.testing.assert_array_equal(bufs["dL"].numpy(), alone[b["id"]][0])
    st = srv.stats()
    assert st["slots_released"] >= 1 and st["slots_in_use"] == 1
    # refusals beyond every idle slot: c fails with ELAS_ERR_NO_MEMORY
    srv.inject_alloc_failures(100)
    res, _ = _one(srv, 3, c)
    assert res["status"] == 5  # ELAS_ERR_NO_MEMORY
    assert srv.stats()["slots_in_use"] == 0
    # the server still serves once allocations succeed again
    srv.inject_alloc_failures(0)
    res, bufs = _one(srv, 4, c)
    assert res["status"] == 0
    np.testing.assert_array_equal(bufs["dL"].numpy(), alone[c["id"]][0])
    srv.close()


def test_drain_times_out_then_completes(requests):
    """elas_server_drain returns ELAS_ERR_TIMEOUT while requests are still in
    flight, and ELAS_OK once every result is in."""
    B = _B()
    srv = B.Server(lanes=1, max_wave=1)
    keep = []
    for i in range(24):
        r = requests[8 + i % 4]
        h, w = r["L"].shape
        bufs = (torch.from_numpy(r["L"]).pin_memory(), torch.from_numpy(r["R"]).pin_memory(),
                torch.empty((h, w), dtype=torch.int16).pin_memory())
        keep.append(bufs)
        srv.submit(i, bufs[0], bufs[1], bufs[2], r["prm"])
    with pytest.raises(B.ElasError) as ei:
        srv.drain(0)
    assert ei.value.status == 4  # ELAS_ERR_TIMEOUT
    srv.drain(60000)
    got = []
    while len(got) < 24:
        got += srv.poll(64, 200)
    assert all(g["status"] == 0 for g in got)
    srv.close()
