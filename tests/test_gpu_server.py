"""Serving layer: continuous batching of Stokes solves through the C ABI.

A request's result must not depend on what else runs: the same request solved alone and in
a mix of concurrent requests of other shapes gives the bitwise-identical solution."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


def layouts(level, n_r):
    P = (2 ** level + 4) // 4 * 4
    n0 = 10 * n_r * (2 ** level + 1) * P
    P1 = (2 ** (level - 1) + 4) // 4 * 4
    n1 = 10 * ((n_r - 1) // 2 + 1) * (2 ** (level - 1) + 1) * P1
    return n0, n1


def valid_mask(level, n_r):
    N = 2 ** level
    P = (N + 4) // 4 * 4
    j = np.arange(10 * n_r * (N + 1) * P) % P
    return j <= N


@pytest.mark.parametrize("eta_storage,hg_kappa,quad", [(0, 0.0, 1), (1, 0.3, 1), (1, 0.0, 2)])
def test_same_request_alone_and_in_a_mix(tn, eta_storage, hg_kappa, quad):
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=4, keep_solutions=1, eta_storage=eta_storage,
                                                        hg_kappa=hg_kappa, radial_quad_points=quad))
    try:
        ref = dict(lateral_level=3, radial_layers=9, E=math.log(100.0), Ra=7e3, t_degree=3, t_order=2,
                   t_amplitude=0.03)
        t0 = tn.tn_server_submit(srv, **ref)
        r0 = tn.tn_server_wait(srv, t0)
        assert r0["status"] == tn.TN_OK and r0["rel_residual"] <= 1e-8
        u0, p0 = tn.tn_server_solution(srv, t0, *layouts(3, 9))
        mix = [dict(lateral_level=4, radial_layers=17, E=math.log(1e3), Ra=7e3, t_degree=4, t_order=4, t_amplitude=0.02),
               ref,
               dict(lateral_level=3, radial_layers=17, E=0.0, Ra=1e4, t_degree=2, t_order=0, t_amplitude=0.05),
               dict(lateral_level=4, radial_layers=9, E=math.log(10.0), Ra=7e3, t_degree=6, t_order=3,
                    t_amplitude=0.01),
               ref]
        tickets = [tn.tn_server_submit(srv, **q) for q in mix]
        results = [tn.tn_server_wait(srv, t) for t in tickets]
        for q, r in zip(mix, results):
            assert r["status"] == tn.TN_OK, (q, r)
            assert r["rel_residual"] <= 1e-8
            assert r["t_submit"] <= r["t_start"] <= r["t_end"]
        v = valid_mask(3, 9)
        for t in (tickets[1], tickets[4]):
            u1, p1 = tn.tn_server_solution(srv, t, *layouts(3, 9))
            assert np.array_equal(u1[:, v], u0[:, v])
            pv = valid_mask(2, 5)
            assert np.array_equal(p1[pv], p0[pv])
        # several solves overlapped: some request started before another one ended
        spans = sorted((r["t_start"], r["t_end"]) for r in results)
        assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
        st = tn.tn_server_stats(srv)
        assert st["queued"] == 0 and st["running"] == 0 and st["resident"] >= 3
    finally:
        tn.tn_server_destroy(srv)


def test_admission_and_invalid_requests(tn):
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=2, memory_fraction=1e-4))
    try:
        # larger than the whole memory budget: completes at once with TN_ENOMEM
        t = tn.tn_server_submit(srv, 6, 65, math.log(10.0), 7e3, 3, 2, 0.01)
        r = tn.tn_server_wait(srv, t)
        assert r["status"] == tn.TN_ENOMEM and r["state"] == 2
        with pytest.raises(tn.TnError) as e:
            tn.tn_server_submit(srv, 3, 8, 0.0, 7e3, 3, 2, 0.01)  # radial_layers - 1 must be even
        assert e.value.status == tn.TN_EINVAL
        with pytest.raises(tn.TnError):
            tn.tn_server_submit(srv, 3, 9, 0.0, 7e3, 2, 3, 0.01)  # order > degree
    finally:
        tn.tn_server_destroy(srv)


def test_same_shape_requests_batched_in_lockstep(tn):
    """max_batch = 4: queued requests of one shape are solved in lockstep (tn_stokes_solve_batch, their
    V-cycles from one graph launch).  A request's solution is bitwise the same alone and inside such
    a batch, and batches do form."""
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=1, keep_solutions=1, max_batch=4, hg_kappa=0.3,
                                                        eta_storage=1, mode=tn.TN_SOLVE_F64_PREC32))
    try:
        ref = dict(lateral_level=3, radial_layers=9, E=math.log(100.0), Ra=7e3, t_degree=3, t_order=2,
                   t_amplitude=0.03)
        t0 = tn.tn_server_submit(srv, **ref)
        r0 = tn.tn_server_wait(srv, t0)
        assert r0["status"] == tn.TN_OK and r0["batch"] == 0
        u0, p0 = tn.tn_server_solution(srv, t0, *layouts(3, 9))
        # one worker: while it solves the first request, the others queue up and the next take batches
        mix = [dict(ref, E=math.log(1e3)), ref, dict(ref, t_degree=5, t_order=3), dict(ref, E=0.0), ref,
               dict(ref, t_amplitude=0.05), dict(ref, lateral_level=4, radial_layers=9)]
        tickets = [tn.tn_server_submit(srv, **q) for q in mix]
        results = [tn.tn_server_wait(srv, t) for t in tickets]
        for q, r in zip(mix, results):
            assert r["status"] == tn.TN_OK and r["rel_residual"] <= 1e-8, (q, r)
        assert max(r["batch"] for r in results) >= 2, [r["batch"] for r in results]
        v, pv = valid_mask(3, 9), valid_mask(2, 5)
        for t in (tickets[1], tickets[4]):
            u1, p1 = tn.tn_server_solution(srv, t, *layouts(3, 9))
            assert np.array_equal(u1[:, v], u0[:, v]) and np.array_equal(p1[pv], p0[pv])
    finally:
        tn.tn_server_destroy(srv)
