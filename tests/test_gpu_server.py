"""Serving loop: requests of mixed kinds and sizes against several resident
indexes, admitted as slots and memory free up.  Each result must be
identical to the same request run alone through cg_radius_count/fill or
cg_knn (integer results: bit-exact), and a sample must equal the oracle."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _clouds():
    a = cloudgen.als_uniform(60_000, extent=(60.0, 60.0), seed=41)
    b = cloudgen.adversarial_cloud(25_000, seed=42)
    c = cloudgen.als_uniform(40_000, extent=(25.0, 25.0), seed=43)
    return [a, b, c]


def _requests(clouds, n, seed, nq_hi=40_000, use=None):
    rng = np.random.default_rng(seed)
    use = list(range(len(clouds))) if use is None else use
    reqs = []
    for i in range(n):
        idx = int(rng.choice(use))
        xyz = clouds[idx]
        nq = int(np.exp(rng.uniform(np.log(500), np.log(nq_hi))))
        r = float(rng.uniform(0.25, 3.0))
        if idx == 1:  # the 8 m adversarial cube: keep rows and outputs moderate
            nq, r = min(nq, 4000), min(r, 1.0)
        q = xyz[rng.integers(0, len(xyz), nq)] + rng.normal(0, 0.2, (nq, 3))
        if rng.random() < 0.5:
            reqs.append(("radius", idx, np.ascontiguousarray(q), r, int(rng.integers(0, 2))))
        else:
            reqs.append(("knn", idx, np.ascontiguousarray(q), int(rng.choice([8, 16, 32])), None))
    return reqs


def _alone(indexes, reqs):
    out = []
    for kind, idx, q, p, kern in reqs:
        qd = torch.from_numpy(q).to(DEV)
        if kind == "radius":
            off, ind = indexes[idx].radius_search(qd, p, kern)
            out.append((off.cpu().numpy(), ind.cpu().numpy()))
        else:
            i, d = indexes[idx].knn(qd, p)
            out.append((i.cpu().numpy(), d.cpu().numpy()))
    return out


def _submit(srv, reqs):
    ids, keep = [], []
    for kind, idx, q, p, kern in reqs:
        qd = torch.from_numpy(q).to(DEV)
        keep.append(qd)
        ids.append(srv.submit_radius(idx, qd, p, kern) if kind == "radius" else srv.submit_knn(idx, qd, p))
    torch.cuda.synchronize()
    return ids, keep


def _same(res, ref, kind):
    if kind == "radius":
        assert np.array_equal(res["offsets"].cpu().numpy(), ref[0])
        assert np.array_equal(res["indices"].cpu().numpy(), ref[1])
    else:
        assert np.array_equal(res["idx"].cpu().numpy(), ref[0])
        assert np.array_equal(res["d2"].cpu().numpy(), ref[1])


def test_mixed_requests_equal_alone_and_oracle():
    clouds = _clouds()
    indexes = [cg.Index(torch.from_numpy(x).to(DEV), 1.0) for x in clouds]
    reqs = _requests(clouds, 36, seed=1)
    ref = _alone(indexes, reqs)
    srv = cg.Server(indexes, slots=4)
    ids, keep = _submit(srv, reqs)
    for rid, (kind, idx, q, p, kern), r in zip(ids, reqs, ref):
        res = srv.wait(rid)
        _same(res, r, kind)
        assert res["latency_ms"] >= res["queue_ms"] >= 0
        srv.release(rid)
    st = srv.stats()
    assert st["requests_done"] == 36 and st["requests_failed"] == 0
    assert st["max_in_flight"] > 1  # requests overlapped on the device
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["queries_per_s"] > 0
    assert st["memory_in_use"] == 0
    srv.close()
    # a sample against the oracle directly
    for (kind, idx, q, p, kern), r in list(zip(reqs, ref))[:6]:
        o = oracle.Index(clouds[idx], 1.0)
        if kind == "radius":
            oo, oi = o.radius_search(q, p, kern, threads=8)
            assert np.array_equal(r[0], oo) and np.array_equal(r[1], oi)
        else:
            oi, od = o.knn(q, p, threads=8)
            assert np.array_equal(r[0], oi) and np.array_equal(r[1], od)
    for ix in indexes:
        ix.close()


def test_memory_budget_admission_and_oversize_request():
    clouds = _clouds()
    indexes = [cg.Index(torch.from_numpy(x).to(DEV), 1.0) for x in clouds]
    reqs = _requests(clouds, 20, seed=2, nq_hi=8_000, use=[0, 2])
    ref = _alone(indexes, reqs)
    budget = 96 << 20
    srv = cg.Server(indexes, slots=6, memory_budget=budget)
    ids, keep = _submit(srv, reqs)
    # one request far larger than the whole budget (30M output indices)
    xyz = clouds[0]
    big = torch.from_numpy(np.repeat(xyz[:1], 200_000, axis=0) + 0.0).to(DEV)
    bid = srv.submit_radius(0, big, 3.0)
    # drain in completion order, releasing each result (its memory lets the
    # waiting requests in)
    pos = {rid: i for i, rid in enumerate(ids)}
    seen = set()
    for _ in range(len(ids) + 1):
        rid = srv.wait_any(timeout_s=120.0)
        seen.add(rid)
        if rid == bid:
            with pytest.raises(cg.CheeseError) as ei:
                srv.wait(bid)
            assert ei.value.code == 2  # CG_ERR_OOM
        else:
            kind = reqs[pos[rid]][0]
            _same(srv.wait(rid), ref[pos[rid]], kind)
        srv.release(rid)
    assert seen == set(ids) | {bid}
    st = srv.stats()
    assert st["memory_peak"] <= budget and st["memory_in_use"] == 0
    assert st["requests_done"] == 20 and st["requests_failed"] == 1
    srv.close()
    for ix in indexes:
        ix.close()


def test_results_survive_until_release_and_empty_requests():
    xyz = cloudgen.als_uniform(20_000, extent=(30.0, 30.0), seed=44)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    srv = cg.Server([ix], slots=2)
    q = torch.from_numpy(xyz[:3000].copy()).to(DEV)
    empty = torch.empty((0, 3), dtype=torch.float64, device=DEV)
    a = srv.submit_radius(0, q, 1.0)
    b = srv.submit_knn(0, q, 8)
    c = srv.submit_radius(0, empty, 1.0)
    d = srv.submit_knn(0, empty, 4)
    ra = srv.wait(a, copy=False)
    rb = srv.wait(b, copy=False)
    assert srv.wait(c)["offsets"].cpu().tolist() == [0]
    assert srv.wait(d)["idx"].shape == (0, 4)
    off, ind = ix.radius_search(q, 1.0)
    i8, d8 = ix.knn(q, 8)
    assert torch.equal(ra["offsets"], off) and torch.equal(ra["indices"], ind)
    assert torch.equal(rb["idx"], i8) and torch.equal(rb["d2"], d8)
    for rid in (a, b, c, d):
        srv.release(rid)
    with pytest.raises(cg.CheeseError):
        srv.release(a)
    srv.close()
    ix.close()


def test_bad_requests_rejected():
    xyz = cloudgen.als_uniform(5_000, extent=(20.0, 20.0), seed=45)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    srv = cg.Server([ix], slots=1)
    q = torch.from_numpy(xyz[:10].copy()).to(DEV)
    with pytest.raises(cg.CheeseError):
        srv.submit_radius(1, q, 1.0)
    with pytest.raises(cg.CheeseError):
        srv.submit_radius(0, q, -1.0)
    with pytest.raises(cg.CheeseError):
        srv.submit_knn(0, q, 0)
    with pytest.raises(cg.CheeseError):
        srv.submit_knn(0, q, 65)
    srv.close()
    ix.close()
