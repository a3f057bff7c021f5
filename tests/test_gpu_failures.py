"""Failure handling of the solver and the server, with every failure made on the host.

Nothing here faults or hangs the GPU: the bad values are planted in host-prepared fields (a NaN
temperature, a NaN viscosity, an overflowing viscosity law), the unreachable tolerance is an
option, and cancellation and shutdown are host calls.  Each case must end in bounded time with a
status code, and the server must free the slot of a failed request."""
import math
import threading
import time

import numpy as np
import pytest

from oracle.mesh import ShellMesh
from paper_2609_21633_gb300 import inputs
from tests.layout import LayoutMap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_21633_gb300 as tn
    tn.lib()
    return tn


def _problem(tn, level, n_r, T_edit=None, eta_edit=None):
    """Mesh with the prescribed temperature (optionally edited) or an explicit viscosity (edited),
    and its buoyancy right-hand side."""
    om = ShellMesh(level, n_r, 0.55, 1.0)
    m = tn.tn_mesh_create(level, n_r, 0.55, 1.0)
    info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
    mp = LayoutMap(info, om)
    T = inputs.temperature(om.node_xyz(), 0.55, 1.0)
    if T_edit is not None:
        T_edit(T)
    Td = torch.tensor(mp.to_layout(T), device="cuda")
    tn.tn_set_temperature(m, Td, math.log(10.0))
    if eta_edit is not None:
        eta = inputs.lognormal_viscosity(om.n_wedges, 3, 0.5)
        eta_edit(eta)
        tn.tn_set_viscosity(m, torch.tensor(mp.wedges_to_layout(eta), device="cuda"))
    f = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
    tn.tn_buoyancy(m, Td, 7e3, f)
    u = [torch.zeros_like(f[0]) for _ in range(3)]
    p = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
    return m, f, u, p


def _solve_status(tn, m, f, u, p, **opts):
    o = tn.tn_solve_default_opts(**opts)
    st = tn.tn_solve_stats()
    import ctypes
    pf, _a = tn._lib._ptrs(f)
    pu, _b = tn._lib._ptrs(u)
    s = tn.lib().tn_stokes_solve(m, ctypes.byref(o), pf, None, pu, tn._lib._ptr(p), ctypes.byref(st),
                                 tn._lib._stream(None))
    return s, {k: getattr(st, k) for k, _ in tn.tn_solve_stats._fields_}, tn.lib().tn_last_error().decode()


def test_nan_in_the_temperature_field_returns_before_iterating(tn):
    """A NaN planted at one node of the host-prepared temperature makes the buoyancy right-hand
    side non-finite: the solve returns TN_ENOTCONVERGED without a single iteration."""
    def plant(T):
        T[len(T) // 2] = np.nan
    m, f, u, p = _problem(tn, 3, 9, T_edit=plant)
    try:
        s, st, msg = _solve_status(tn, m, f, u, p)
        assert s == tn.TN_ENOTCONVERGED and st["iterations"] == 0 and st["converged"] == 0, (s, st, msg)
        assert "non-finite" in msg
    finally:
        tn.tn_mesh_destroy(m)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_nan_viscosity_stops_fgmres_within_one_restart(tn, mode):
    """A NaN viscosity on one wedge (finite right-hand side) poisons the operator: FGMRES must stop
    at the first non-finite Hessenberg column, within the first restart, in every solve mode."""
    def plant(eta):
        eta[len(eta) // 3] = np.nan
    m, f, u, p = _problem(tn, 3, 9, eta_edit=plant)
    try:
        t0 = time.perf_counter()
        s, st, msg = _solve_status(tn, m, f, u, p, mode=mode, restart=10)
        assert s == tn.TN_ENOTCONVERGED and st["converged"] == 0, (s, st, msg)
        assert st["iterations"] <= 10 and "non-finite" in msg, (st, msg)
        assert time.perf_counter() - t0 < 60
    finally:
        tn.tn_mesh_destroy(m)


def test_unreachable_tolerance_stops_as_stagnation(tn):
    """rtol = 1e-17 lies below FP64 rounding of the residual: FGMRES(10) stops after five restarts
    without progress instead of running all 2000 iterations."""
    m, f, u, p = _problem(tn, 3, 9)
    try:
        s, st, msg = _solve_status(tn, m, f, u, p, rtol=1e-17, restart=10, max_iters=2000)
        assert s == tn.TN_ENOTCONVERGED and "stagnation" in msg, (s, st, msg)
        assert st["iterations"] < 2000 and st["rel_residual"] < 1e-12, st
    finally:
        tn.tn_mesh_destroy(m)


def test_failed_request_frees_its_slot(tn):
    """A viscosity law that overflows (E = 2000: exp(+-1000)) breaks the request's solve down; it
    completes with TN_ENOTCONVERGED, the server holds nothing for it, and the next request runs."""
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=1))
    try:
        bad = tn.tn_server_submit(srv, 3, 9, 2000.0, 7e3, 3, 2, 0.03)
        good = tn.tn_server_submit(srv, 3, 9, math.log(10.0), 7e3, 3, 2, 0.03)
        rb, rg = tn.tn_server_wait(srv, bad), tn.tn_server_wait(srv, good)
        assert rb["status"] == tn.TN_ENOTCONVERGED and rb["state"] == 2, rb
        assert rg["status"] == tn.TN_OK and rg["rel_residual"] <= 1e-8, rg
        st = tn.tn_server_stats(srv)
        assert st["running"] == 0 and st["queued"] == 0
        with pytest.raises(tn.TnError) as e:  # non-finite parameters never get a slot
            tn.tn_server_submit(srv, 3, 9, 0.0, 7e3, 3, 2, float("nan"))
        assert e.value.status == tn.TN_EINVAL
    finally:
        tn.tn_server_destroy(srv)


def test_cancel_queued_and_running_requests(tn):
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=1, mode=tn.TN_SOLVE_F64))
    try:
        long = tn.tn_server_submit(srv, 5, 33, math.log(1e4), 7e3, 3, 2, 0.03)
        queued = tn.tn_server_submit(srv, 3, 9, math.log(10.0), 7e3, 3, 2, 0.03)
        tn.tn_server_cancel(srv, queued)
        rq = tn.tn_server_wait(srv, queued)
        assert rq["status"] == tn.TN_ECANCELED and rq["iterations"] == 0
        deadline = time.time() + 60
        while tn.tn_server_poll(srv, long)[1]["state"] != 1 and time.time() < deadline:
            time.sleep(0.01)
        time.sleep(0.5)
        t0 = time.perf_counter()
        tn.tn_server_cancel(srv, long)
        rl = tn.tn_server_wait(srv, long)
        assert rl["status"] in (tn.TN_ECANCELED, tn.TN_OK), rl  # TN_OK only if it finished first
        assert time.perf_counter() - t0 < 30
        st = tn.tn_server_stats(srv)
        assert st["running"] == 0 and st["queued"] == 0
        with pytest.raises(tn.TnError):
            tn.tn_server_cancel(srv, 12345)
        again = tn.tn_server_submit(srv, 3, 9, math.log(10.0), 7e3, 3, 2, 0.03)
        assert tn.tn_server_wait(srv, again)["status"] == tn.TN_OK
    finally:
        tn.tn_server_destroy(srv)


def test_destroy_with_queued_requests_returns(tn):
    """tn_server_destroy finishes the queued requests and returns (checked from a watcher thread
    with a time limit, so a hang fails the test instead of blocking the run)."""
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=1))
    for k in range(6):
        tn.tn_server_submit(srv, 3, 9, math.log(10.0 + k), 7e3, 3, 2, 0.03)
    done = []
    th = threading.Thread(target=lambda: done.append(tn.tn_server_destroy(srv)), daemon=True)
    th.start()
    th.join(timeout=300)
    assert done == [None], "tn_server_destroy did not return"
