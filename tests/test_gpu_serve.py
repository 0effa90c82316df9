"""Solve server with continuous batching: results are the same alone and in the mix, requests
overlap on the device, admission respects the HBM budget, bad requests are rejected.

Tolerance for "the same alone and in the mix": 1e-14 relative (the solves are deterministic and
share no work space, so the results are in fact bitwise identical).
"""
import numpy as np
import pytest

from tests.gpu_common import gpu

pytestmark = pytest.mark.gpu

SCHED = {3: (3, 1), 5: (5, 3, 1), 7: (7, 3, 1)}


def stream_specs():
    """10 requests on 5 distinct meshes (keys reused), p in {3, 5, 7}, varied right-hand sides."""
    meshes = [((3, 3, 3), 3, 11), ((4, 3, 3), 5, 12), ((3, 3, 2), 7, 13), ((5, 4, 4), 3, 14),
              ((3, 2, 3), 5, 15)]
    order = [0, 1, 2, 0, 3, 1, 4, 2, 0, 3]
    return [(meshes[k], k, ((i % 3) + 1, (i % 2) + 1, 1), 0.5 + 0.1 * i) for i, k in enumerate(order)]


def run_stream(se, specs, slots, precision, budget=32 << 30, serial=False, op_df=0):
    S = se.se_serve_create(budget, slots, operator_df64=op_df)
    try:
        xs, tickets, keep = [], [], []
        for (nel, p, seed), key, modes, amp in specs:
            L = nel[0] * nel[1] * nel[2] * (p + 1) ** 3
            x = np.full(L, np.nan)
            md = se.mesh_desc(nel, p, perturb_frac=0.05, seed=seed)
            pd = se.pmg_desc(SCHED[p], se.SE_SMOOTH_RAS, 2, precision=precision)
            q = se.make_request(md, key, pd, modes=modes, amplitude=amp, x_host=x, tol=1e-8)
            keep.append(q)
            t = se.se_serve_submit(S, q)
            if serial:
                se.se_serve_wait(S, t)
            xs.append(x)
            tickets.append(t)
        results = [se.se_serve_wait(S, t) for t in tickets]
        return xs, results, se.se_serve_stats(S)
    finally:
        se.se_serve_destroy(S)


@pytest.mark.parametrize("precision,op_df", [(0, 0), (1, 0), (1, 1)])
def test_same_alone_and_in_the_mix(precision, op_df):
    """op_df = 1: the outer operators in df64 (the p = 3, 5, 7 meshes all have df64 kernels)."""
    torch, se = gpu()
    specs = stream_specs()
    x_mix, r_mix, st = run_stream(se, specs, slots=4, precision=precision, op_df=op_df)
    x_one, r_one, _ = run_stream(se, specs, slots=1, precision=precision, serial=True, op_df=op_df)
    for a, b, ra, rb in zip(x_mix, x_one, r_mix, r_one):
        assert ra.status == 0 and rb.status == 0
        assert ra.rel_residual <= 1e-8 and ra.iterations == rb.iterations
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))
    assert st.completed == len(specs) and st.meshes_created == 5 and st.mesh_reuses == 5
    assert st.max_concurrent >= 2          # requests did overlap on the device
    assert st.p99_ms >= st.p50_ms > 0


def test_budget_refusal_and_eviction():
    torch, se = gpu()
    md = se.mesh_desc((4, 4, 4), 5, perturb_frac=0.05, seed=3)
    pd = se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32)
    need = se.se_mesh_footprint_bytes(md, pd)
    assert need > 0
    S = se.se_serve_create(need // 2, 2)
    try:
        with pytest.raises(se.SeError) as e:
            se.se_serve_submit(S, se.make_request(md, 1, pd))
        assert e.value.code == se.SE_EREFUSED
        bad = se.make_request(md, 2, pd)
        bad.tol = -1.0
        with pytest.raises(se.SeError) as e:
            se.se_serve_submit(S, bad)
        assert e.value.code == se.SE_EINVAL
        with pytest.raises(se.SeError):
            se.se_serve_wait(S, 12345)
        assert se.se_serve_stats(S).refused == 1
    finally:
        se.se_serve_destroy(S)
    # room for one mesh and a half: distinct meshes force evictions, all still complete
    S = se.se_serve_create(int(1.5 * need), 1)
    try:
        ts = []
        for k in range(4):
            mk = se.mesh_desc((4, 4, 4), 5, perturb_frac=0.05, seed=20 + k)
            ts.append(se.se_serve_submit(S, se.make_request(mk, 100 + k, pd)))
        res = [se.se_serve_wait(S, t) for t in ts]
        assert all(r.status == 0 and r.rel_residual <= 1e-8 for r in res)
        st = se.se_serve_stats(S)
        assert st.evictions >= 1 and st.resident_bytes <= 1.5 * need
    finally:
        se.se_serve_destroy(S)


def test_cancel_queued_request():
    """A request still in the queue is removed by se_serve_cancel (result SE_ECANCELED, no solve);
    one that has started is not interrupted (SE_EBUSY) and completes; finished or unknown tickets
    are rejected (SE_EINVAL).  One slot: the first request's mesh set-up holds it while the
    others wait in the queue."""
    import time
    torch, se = gpu()
    pd = se.pmg_desc((7, 3, 1), se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32)
    pd9 = se.pmg_desc((9, 5, 1), se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32)
    big = se.mesh_desc((40, 40, 40), 9, perturb_frac=0.05, seed=41)  # set-up about 0.4 s
    small = [se.mesh_desc((4, 4, 4), 7, perturb_frac=0.05, seed=42 + k) for k in range(2)]
    S = se.se_serve_create(se.se_mesh_footprint_bytes(big, pd9) * 4, 1)
    try:
        t1 = se.se_serve_submit(S, se.make_request(big, 301, pd9))
        t2 = se.se_serve_submit(S, se.make_request(small[0], 302, pd))
        t3 = se.se_serve_submit(S, se.make_request(small[1], 303, pd))
        assert se.se_serve_cancel(S, t3) == se.SE_OK
        r3 = se.se_serve_wait(S, t3, allow=(se.SE_ECANCELED,))
        assert r3.status == se.SE_ECANCELED and r3.iterations == 0
        time.sleep(0.1)  # the scheduler admits within milliseconds; the set-up takes longer
        assert se.se_serve_cancel(S, t1) == se.SE_EBUSY
        r1, r2 = se.se_serve_wait(S, t1), se.se_serve_wait(S, t2)
        assert r1.status == 0 and r1.rel_residual <= 1e-8
        assert r2.status == 0 and r2.rel_residual <= 1e-8
        for t in (t1, t3, 987654):
            with pytest.raises(se.SeError) as e:
                se.se_serve_cancel(S, t)
            assert e.value.code == se.SE_EINVAL
        st = se.se_serve_stats(S)
        assert st.cancelled == 1 and st.completed == 2 and st.pending == 0
    finally:
        se.se_serve_destroy(S)


def test_projection_in_the_server():
    """Requests on one resident mesh with right-hand sides from a small space: with projection
    (proj_vectors = 4) later requests start from the projected guess and need (almost) no
    iterations; every result meets the tolerance relative to ||b|| and agrees with the solve
    from zero to the accuracy the tolerance gives."""
    torch, se = gpu()
    md = se.mesh_desc((3, 3, 3), 5, perturb_frac=0.05, seed=5)
    pd = se.pmg_desc((5, 3, 1), se.SE_SMOOTH_RAS, 2, precision=se.SE_FP32)
    L = 27 * 6 ** 3
    modes = [(1, 1, 1), (2, 1, 1), (1, 1, 1), (2, 1, 1), (1, 1, 1), (1, 1, 1)]
    amps = [1.0, 0.6, 1.7, 1.2, 0.4, 2.0]
    out = {}
    for nv in (0, 4):
        S = se.se_serve_create(32 << 30, 2, proj_vectors=nv)
        try:
            xs, its = [], []
            for k, a in zip(modes, amps):
                x = np.full(L, np.nan)
                q = se.make_request(md, 77, pd, modes=k, amplitude=a, x_host=x, tol=1e-8)
                r = se.se_serve_wait(S, se.se_serve_submit(S, q))   # one at a time, in order
                assert r.status == 0 and r.rel_residual <= 1e-8
                xs.append(x)
                its.append(r.iterations)
            out[nv] = (xs, its, se.se_serve_stats(S))
        finally:
            se.se_serve_destroy(S)
    xs0, its0, st0 = out[0]
    xs4, its4, st4 = out[4]
    assert st0.projected == 0 and st4.projected == len(modes) - 1
    assert its4[0] == its0[0]
    assert all(i <= 1 for i in its4[2:])        # b in the span of prior right-hand sides
    for a, b in zip(xs4, xs0):
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
