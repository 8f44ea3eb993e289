"""Continuous-batching server: each request's result is the same alone and in
a mix (bit for bit: the batched kernel steps every tile with the same code
whatever else is in the table), it matches the single-grid tile path within
the storage precision, admission waits for memory, failures stay local, and a
served request matches the FP64 oracle."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RB = dict(tau=0.05, tau_g=0.05, beta=2e-4, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)


def _requests():
    # different sizes, Rayleigh numbers (through beta) and step counts
    return [
        dict(rid=1, nsteps=37, nx=40, ny=40, sy=1, stretch_y=2.0, bcy=1, dt=0.1, amp=1e-2, seed=1, **RB),
        dict(rid=2, nsteps=58, nx=96, ny=64, sy=1, stretch_y=2.0, bcy=1, dt=0.1, amp=1e-2, seed=2,
             **{**RB, "beta": 5e-4}),
        dict(rid=3, nsteps=21, nx=64, ny=64, bcy=1, dt=0.2, amp=1e-2, seed=3, **{**RB, "tau": 0.1, "tau_g": 0.1}),
    ]


def _alone_on_grid(lb, req, store):
    """The same request through an ordinary grid with the tile schedule."""
    kw = dict(req)
    rid, nsteps = kw.pop("rid"), kw.pop("nsteps")
    grid_keys = ("nx", "ny", "lx", "ly", "sx", "sy", "stretch_x", "stretch_y", "bcx", "bcy")
    gk = {k: kw.pop(k) for k in list(kw) if k in grid_keys}
    g = lb.Grid(thermal=True, store=store, **gk)
    g.init(kind=lb.LB_INIT_RB, **kw)
    # the server's batched kernels use the (paired) tile decomposition
    g.set_fv_schedule(lb.LB_FV_PTILE if store != "f64" else lb.LB_FV_TILE)
    g.step_fv(nsteps)
    return g.nusselt(), g.conservation()[0]


def _drain(server):
    out = {}
    while True:
        active, pending = server.pump()
        for r in server.results():
            out[r["id"]] = r
        if active == 0 and pending == 0:
            for r in server.results():
                out[r["id"]] = r
            return out


@pytest.mark.parametrize("policy", [0, 1, 2], ids=["share", "shortest", "arrival"])
@pytest.mark.parametrize("store", ["f32", "f16dev"])
def test_alone_equals_mix(lbgpu, store, policy):
    lb = lbgpu
    reqs = _requests()
    mix = lb.Server(store=store, thermal=True, steps_per_launch=8, policy=policy)
    for r in reqs:
        mix.submit(**r)
    got = _drain(mix)
    assert set(got) == {1, 2, 3}
    tol = 1e-7 if store == "f32" else 1e-5  # plate Nu amplifies rounding by ~H * 20
    for r in reqs:
        res = got[r["rid"]]
        assert res["status"] == lb.LB_OK and res["steps"] == r["nsteps"]
        mixed = (res["nu_vol"], res["nu_bot"], res["nu_top"], res["mass"])
        # alone through its own server: identical bits
        one = lb.Server(store=store, thermal=True, steps_per_launch=8)
        one.submit(**r)
        alone = _drain(one)[r["rid"]]
        assert (alone["nu_vol"], alone["nu_bot"], alone["nu_top"], alone["mass"]) == mixed
        # the ordinary grid path (separately compiled): within storage precision
        nu, mass = _alone_on_grid(lb, r, store)
        for a, b in zip(mixed, nu + (mass,)):
            assert abs(a - b) <= tol * abs(b)
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]


def test_table_growth_recaptures_the_graph(lbgpu):
    """The server replays a captured graph of its batched launches, which
    holds the device tables' addresses.  When the request table outgrows its
    capacity (64) while the tile table does not, both tables are
    reallocated, and the next pump must capture a new graph.  Seventy
    one-tile requests join after three pumps of the first one; every result
    equals the request's solo run."""
    lb = lbgpu
    small = dict(nx=16, ny=16, bcy=1, dt=0.2, amp=1e-2, **{**RB, "tau": 0.1, "tau_g": 0.1})
    s = lb.Server(store="f32", thermal=True, steps_per_launch=2)
    s.submit(rid=0, nsteps=40, seed=100, **small)
    out = {}
    for _ in range(3):  # plain launches, a captured graph, a replay
        s.pump()
        out.update({r["id"]: r for r in s.results()})
    for i in range(1, 71):
        s.submit(rid=i, nsteps=6, seed=100 + i, **small)
    out.update(_drain(s))
    assert len(out) == 71 and all(r["status"] == lb.LB_OK for r in out.values())
    for i in (0, 1, 35, 70):
        one = lb.Server(store="f32", thermal=True, steps_per_launch=2)
        one.submit(rid=i, nsteps=40 if i == 0 else 6, seed=100 + i, **small)
        alone = _drain(one)[i]
        assert (alone["nu_vol"], alone["nu_bot"], alone["mass"]) == (out[i]["nu_vol"], out[i]["nu_bot"],
                                                                     out[i]["mass"])


def test_admission_waits_for_memory(lbgpu):
    """A budget that holds one request at a time: they run one after another."""
    lb = lbgpu
    reqs = _requests()
    s = lb.Server(store="f32", thermal=True, hbm_budget=1_258_291, steps_per_launch=8)
    for r in reqs[:2]:
        s.submit(**r)
    got = _drain(s)
    a, b = got[1], got[2]
    assert a["status"] == b["status"] == lb.LB_OK
    assert b["t_admit"] >= a["t_done"] - 1e-6
    with pytest.raises(lb.LBError) as e:
        s.submit(rid=9, nsteps=1, nx=2048, ny=2048, **RB)
    assert e.value.status == lb.LB_ERR_ARG


def test_unstable_request_fails_alone(lbgpu):
    """A request far beyond the stability limit ends with LB_ERR_UNSTABLE; the
    request batched with it is unaffected."""
    lb = lbgpu
    good = _requests()[0]
    s = lb.Server(store="f32", thermal=True, steps_per_launch=8)
    s.submit(**good)
    bad = dict(good, rid=7, dt=40.0, nsteps=200, amp=0.5)
    s.submit(**bad)
    got = _drain(s)
    assert got[7]["status"] == lb.LB_ERR_UNSTABLE
    assert got[1]["status"] == lb.LB_OK
    one = lb.Server(store="f32", thermal=True, steps_per_launch=8)
    one.submit(**good)
    alone = _drain(one)[1]
    assert (got[1]["nu_vol"], got[1]["nu_bot"], got[1]["nu_top"]) == (alone["nu_vol"], alone["nu_bot"],
                                                                       alone["nu_top"])


def test_served_request_matches_oracle(lbgpu, oracle):
    """FP64 server: the batched kernel's Nusselt numbers equal the oracle's."""
    lb = lbgpu
    oracle.set_threads(os.cpu_count() or 1)
    r = _requests()[1]
    s = lb.Server(store="f64", thermal=True, steps_per_launch=6)
    s.submit(**r)
    res = _drain(s)[2]
    ref = oracle.RefGrid(r["nx"], r["ny"], sy=r["sy"], stretch_y=r["stretch_y"], bcy=r["bcy"], thermal=True)
    ref.set_params(tau=r["tau"], dt=r["dt"], tau_g=r["tau_g"], beta=r["beta"], grav=r["grav"], T0=r["T0"],
                   T_bot=r["T_bot"], T_top=r["T_top"])
    ref.init_preset(oracle.INIT_RB, amp=r["amp"], seed=r["seed"])
    ref.step_fv(r["nsteps"])
    for a, b in zip((res["nu_vol"], res["nu_bot"], res["nu_top"]), ref.nusselt()):
        assert abs(a - b) <= 1e-10 * max(1.0, abs(b))


@pytest.mark.parametrize("store,tol", [("f32", 1e-6), ("f16dev", 1e-3)])
def test_served_mix_matches_oracle_reduced_precision(lbgpu, oracle, store, tol):
    """FP32 arithmetic in the paired batched kernel (k_fv_ptile_batched), with
    FP32 and FP16 deviation storage: each request of a three-request mix has
    Nusselt numbers within the storage's bar of the FP64 oracle's (1e-6
    relative for FP32, 1e-3 for FP16 storage), as on a single grid."""
    lb = lbgpu
    oracle.set_threads(os.cpu_count() or 1)
    reqs = _requests()
    s = lb.Server(store=store, thermal=True, steps_per_launch=8)
    for r in reqs:
        s.submit(**r)
    got = _drain(s)
    for r in reqs:
        assert got[r["rid"]]["status"] == lb.LB_OK
        ref = oracle.RefGrid(r["nx"], r["ny"], sy=r.get("sy", 0), stretch_y=r.get("stretch_y", 0.0),
                             bcy=r["bcy"], thermal=True)
        ref.set_params(tau=r["tau"], dt=r["dt"], tau_g=r["tau_g"], beta=r["beta"], grav=r["grav"],
                       T0=r["T0"], T_bot=r["T_bot"], T_top=r["T_top"])
        ref.init_preset(oracle.INIT_RB, amp=r["amp"], seed=r["seed"])
        ref.step_fv(r["nsteps"])
        res = got[r["rid"]]
        for a, b in zip((res["nu_vol"], res["nu_bot"], res["nu_top"]), ref.nusselt()):
            assert abs(a / b - 1.0) < tol, (r["rid"], a, b)


def test_arrival_policy_is_first_come_first_served(lbgpu):
    """LB_SERVE_ARRIVAL: when every request alone fills the GPU (a 1024^2
    grid is far more than two waves of tiles), they run one at a time in
    submission order; LB_SERVE_SHORTEST lets a later, smaller one overtake."""
    lb = lbgpu
    big = dict(nx=1024, ny=1024, sy=1, stretch_y=2.0, bcy=1, dt=0.1, amp=1e-3, **RB)
    small = dict(nx=512, ny=512, sy=1, stretch_y=2.0, bcy=1, dt=0.1, amp=1e-3, **RB)
    order = {}
    for policy in (lb.LB_SERVE_ARRIVAL, lb.LB_SERVE_SHORTEST):
        s = lb.Server(store="f16dev", thermal=True, steps_per_launch=4, policy=policy)
        s.submit(rid=1, nsteps=12, seed=1, **big)
        s.submit(rid=2, nsteps=12, seed=2, **big)
        s.submit(rid=3, nsteps=12, seed=3, **small)
        got = _drain(s)
        assert all(got[i]["status"] == lb.LB_OK for i in (1, 2, 3))
        order[policy] = sorted(got, key=lambda i: got[i]["t_done"])
    assert order[lb.LB_SERVE_ARRIVAL] == [1, 2, 3]
    assert order[lb.LB_SERVE_SHORTEST][0] == 3
