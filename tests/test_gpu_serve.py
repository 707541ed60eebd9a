"""Serving engine (fmt_server_*) on the GPU: each request's result is the
same when it runs alone and when it shares batches with others (FP64 within
1e-10 max|f|, mixed within 1e-6 max|f|), batches form from requests that
queue up while others run, and the device-memory budget is enforced."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_01353_gb300 import fmt as F
from paper_1511_01353_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def requests(k, seed_offset=0):
    b = W.batch(n_problems=k, n_min=400, n_max=12000, deg_min=4, deg_max=9, targets_per_problem=300,
                seed=W.SEED_BASE + 40 + seed_offset)
    out = []
    for i in range(k):
        s, e = int(b.offsets[i]), int(b.offsets[i + 1])
        ts, te = int(b.toff[i]), int(b.toff[i + 1])
        prec = F.FMT_MIXED if i % 2 else F.FMT_FP64
        p = F.make_params(int(b.degrees[i]), b.max_depth, b.min_pts, b.tol_rel, precision=prec)
        out.append((p, b.x[s:e], b.y[s:e], b.z[s:e], b.f[s:e], b.xq[ts:te], b.yq[ts:te], b.zq[ts:te]))
    return out


def blocker(seed=0):
    # a request large enough (4e5 points, degree 8) to keep a worker busy for
    # far longer than the test takes to submit the others, so that they queue
    # behind it and form batches whatever the timing of the submissions
    rng = np.random.default_rng(1000 + seed)
    x, y, z = rng.uniform(0, 1, (3, 400_000))
    q = rng.uniform(0, 1, (3, 10))
    return (F.make_params(8, 3, 1, 1e-3), x, y, z, np.sin(3 * x) * y + z, *q)


def tol_of(req):
    rel = 1e-10 if req[0].precision == F.FMT_FP64 else 1e-6
    return rel * np.max(np.abs(req[4]))


def test_each_result_same_alone_and_in_the_mix():
    reqs = requests(10)
    alone = []
    sv = F.Server(slots=1)
    for r in reqs:
        t = sv.submit(*r)
        out, info = sv.wait(t)
        assert info["status"] == F.FMT_OK and info["batch_requests"] == 1
        alone.append(out)
    sv.close()
    sv = F.Server(slots=2, max_batch_points=60000)
    held = [sv.submit(*blocker(k)) for k in range(2)]  # both workers busy while the requests queue
    tickets = [sv.submit(*r) for r in reqs]
    mixed_batches = 0
    for r, t, a in zip(reqs, tickets, alone):
        out, info = sv.wait(t)
        assert info["status"] == F.FMT_OK
        mixed_batches = max(mixed_batches, info["batch_requests"])
        assert np.max(np.abs(out - a)) <= tol_of(r), (r[0].precision, np.max(np.abs(out - a)))
    for t in held:
        assert sv.wait(t)[1]["status"] == F.FMT_OK
    sv.close()
    assert mixed_batches > 1  # requests were batched together


def test_served_fp64_result_matches_the_oracle():
    reqs = [r for r in requests(6, 1) if r[0].precision == F.FMT_FP64][:2]
    sv = F.Server(slots=2)
    tickets = [sv.submit(*r) for r in reqs]
    for r, t in zip(reqs, tickets):
        out, info = sv.wait(t)
        p = r[0]
        T = O.fit(r[1], r[2], r[3], r[4], p.degree, p.max_depth, p.min_pts, p.tol_rel)
        ref, _ = T.evaluate(r[5], r[6], r[7])
        # at fresh targets of a clustered cloud a high-degree fit extrapolates
        # between sparse data, so the bar here is the mixed one
        assert np.max(np.abs(out - ref)) <= 1e-6 * T.maxabs
    sv.close()


def test_budget_rejects_a_request_that_can_never_fit():
    rng = np.random.default_rng(3)
    small = rng.uniform(0, 1, (4, 200))
    big = rng.uniform(0, 1, (4, 20000))
    q = rng.uniform(0, 1, (3, 10))
    sv = F.Server(slots=1, budget_bytes=40e6)
    t_big = sv.submit(F.make_params(8, 2, 1, 1e-6), *big, *q)
    t_small = sv.submit(F.make_params(2, 2, 1, 1e-6), *small, *q)
    _, info = sv.wait(t_big)
    assert info["status"] == F.FMT_ENOMEM
    out, info = sv.wait(t_small)
    assert info["status"] == F.FMT_OK and np.all(np.isfinite(out))
    sv.close()


def test_requests_arriving_during_a_batch_join_the_next_one():
    reqs = requests(8, 2)
    sv = F.Server(slots=1)
    first = sv.submit(*blocker())
    later = [sv.submit(*r) for r in reqs]  # queued while the first batch runs
    _, i0 = sv.wait(first)
    infos = [sv.wait(t)[1] for t in later]
    sv.close()
    assert all(i["status"] == F.FMT_OK for i in infos)
    assert max(i["batch_requests"] for i in infos) > 1
    assert min(i["t_start"] for i in infos) >= i0["t_start"]


def test_resident_tree_serves_evaluate_only_requests():
    # a fit request that keeps its tree: evaluate-only requests against it
    # give exactly what the fit's own evaluation gave at the same targets, and
    # its memory stays admitted until it is released
    reqs = requests(4, 3)
    sv = F.Server(slots=2, budget_bytes=20e9)
    t_keep = sv.submit(*reqs[0], keep=True)
    t_other = sv.submit(*reqs[1])
    out_fit, info = sv.wait(t_keep)
    assert info["status"] == F.FMT_OK and info["resident_id"] > 0
    sv.wait(t_other)
    rid = info["resident_id"]
    mem = sv.memory()
    assert mem["resident_trees"] == 1 and mem["admitted"] > 0
    xq, yq, zq = reqs[0][5:8]
    tickets = [sv.submit_eval(rid, xq, yq, zq) for _ in range(2)]
    for t in tickets:
        out, ie = sv.wait(t)
        assert ie["status"] == F.FMT_OK and ie["resident_id"] == rid
        assert np.array_equal(out, out_fit)
    # another request's targets on the same tree: the same polynomial (sum of
    # the first half of the targets evaluated alone equals the full evaluation's)
    out_half, _ = sv.wait(sv.submit_eval(rid, xq[:50], yq[:50], zq[:50]))
    assert np.array_equal(out_half, out_fit[:50])
    sv.release(rid)
    mem = sv.memory()
    assert mem["resident_trees"] == 0 and mem["admitted"] == 0.0
    assert mem["peak_admitted"] <= 20e9
    with pytest.raises(F.FmtError):
        sv.submit_eval(rid, xq, yq, zq)
    sv.close()


def test_admitted_memory_stays_within_the_budget():
    # many requests, some kept: the admitted bytes (running batches plus
    # resident trees) never exceed the budget, and return to zero at the end
    reqs = requests(8, 4)
    budget = 2.0e9
    sv = F.Server(slots=2, budget_bytes=budget, max_batch_points=30000)
    tickets = [sv.submit(*r, keep=(i % 3 == 0)) for i, r in enumerate(reqs)]
    kept = []
    for t in tickets:
        _, info = sv.wait(t)
        assert info["status"] == F.FMT_OK
        if info["resident_id"] > 0:
            kept.append(info["resident_id"])
    assert len(kept) == 3
    assert sv.memory()["peak_admitted"] <= budget
    for rid in kept:
        sv.release(rid)
    assert sv.memory()["admitted"] == 0.0
    sv.close()
