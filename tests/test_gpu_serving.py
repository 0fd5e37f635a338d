"""Continuous-batching server on the GPU: requests of different sizes overlap
on the device, cached hierarchies skip setup, and each result is the same
alone and in the mix (bit-identical: every kernel is deterministic)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import gen
    import paper_2602_05686_gb300 as sa
    sa.build()
    return torch, gen, sa


def _setup(torch, gen, nreq=24, seed=3):
    ops, reqs = gen.serving_requests(nreq, seed=seed, max2d=96, max3d=20, min_el=12)
    probs = {}
    for k, o in enumerate(ops):
        probs[k] = gen.layered_serving(o["dim"], o["n_el"], o["contrast"])
    rhs = []
    for r in reqs:
        p = probs[r["op"]]
        st = gen.Stream(1000 + r["rhs_seed"], 9)
        b = st.normal(p["n"])
        b[p["dir_mask"] == 1] = 0.0
        rhs.append(torch.from_numpy(b))
    return ops, reqs, probs, rhs


def _options(op):
    return dict(theta=0.05, measure="material", precision="fp32", max_coarse=200)


def test_alone_equals_mix(env):
    torch, gen, sa = env
    from paper_2602_05686_gb300.serving import Request, Server
    ops, reqs, probs, rhs = _setup(torch, gen)

    def run(slots, gaps, group=False, batch=8):
        srv = Server(lambda op: probs[op], _options, slots=slots, hbm_budget=8 << 30, group_solves=group,
                     batch=batch)
        rs = []
        t = 0.0
        for k, r in enumerate(reqs):
            t += r["gap"] * gaps
            rs.append(Request(rid=k, op=r["op"], arrival=t, rhs=rhs[k].clone()))
        out = srv.serve(rs, realtime=gaps > 0)
        res = {r.rid: (r.result.cpu().numpy(), r.info["iters"], r.status) for r in rs}
        srv.close()
        return out, res

    alone = {}
    for k, r in enumerate(reqs):
        srv = Server(lambda op: probs[op], _options, slots=1, hbm_budget=8 << 30)
        rq = Request(rid=k, op=r["op"], arrival=0.0, rhs=rhs[k].clone())
        srv.serve([rq], realtime=False)
        alone[k] = (rq.result.cpu().numpy(), rq.info["iters"], rq.status)
        srv.close()
    out, mix = run(slots=4, gaps=0.002)
    assert out["failed"] == 0 and out["setups"] <= len(ops)
    assert out["hits"] + out["setups"] == len(reqs)  # no duplicated setups
    for k in alone:
        assert alone[k][2] == 0 and mix[k][2] == 0
        assert alone[k][1] == mix[k][1]
        assert np.array_equal(alone[k][0], mix[k][0]), k
    assert out["p50_s"] <= out["p99_s"]
    # everything waiting at once: same-operator requests share multi-RHS jobs
    out0, mix0 = run(slots=2, gaps=0.0)
    assert out0["failed"] == 0 and out0["batched"] > 0 and out0["jobs"] < len(reqs)
    for k in alone:
        assert alone[k][1] == mix0[k][1] and np.array_equal(alone[k][0], mix0[k][0]), k
    # different operators in shared launches (group solves): still bitwise
    # the request alone
    outg, mixg = run(slots=6, gaps=0.0, group=True, batch=1)
    assert outg["failed"] == 0 and outg["grouped"] == len(reqs) and outg["max_group"] > 1
    for k in alone:
        assert alone[k][1] == mixg[k][1] and np.array_equal(alone[k][0], mixg[k][0]), k
    outr, mixr = run(slots=4, gaps=0.002, group=True)
    assert outr["failed"] == 0
    for k in alone:
        assert alone[k][1] == mixr[k][1] and np.array_equal(alone[k][0], mixr[k][0]), k


def test_small_budget_evicts_but_stays_correct(env):
    torch, gen, sa = env
    from paper_2602_05686_gb300.serving import Request, Server
    ops, reqs, probs, rhs = _setup(torch, gen, nreq=16, seed=5)
    srv = Server(lambda op: probs[op], _options, slots=2, hbm_budget=24 << 20)
    rs = [Request(rid=k, op=r["op"], arrival=0.0, rhs=rhs[k].clone()) for k, r in enumerate(reqs)]
    out = srv.serve(rs, realtime=False)
    srv.close()
    assert out["failed"] == 0
    for r in rs:
        assert r.info["rel_res"] <= 1e-8
