"""D3Q19 kernels (include/lb3.h) against the FP64 3-D oracle: FV and ST
steps element by element from random states (FP64 to 1e-13, FP32 to 2e-6 of
the deviation scale), periodic boxes, walls and plates on stretched grids,
axes of one cell; the observables; the Rayleigh-Benard workload of Table rb
at its full size on sampled planes."""
import numpy as np
import pytest

from tests import inputs

pytestmark = pytest.mark.gpu

CASES = [
    dict(nx=9, ny=7, nz=6),
    dict(nx=8, ny=6, nz=10, sz=2, stretch_z=4.0, bcz=1, thermal=True),
    dict(nx=5, ny=12, nz=8, sy=1, stretch_y=1.5, bcy=1, sz=3, bcz=1),
    dict(nx=1, ny=10, nz=8, lx=1.0, sz=1, stretch_z=2.0, bcz=1, thermal=True),
    dict(nx=33, ny=9, nz=4, bcx=1),
    # the smallest z extents: every plane is a ghost source (walls need two cells)
    dict(nx=5, ny=4, nz=2, bcx=1, bcz=1),
    dict(nx=7, ny=3, nz=1),
    # even nx: the paired FP32 collision and star passes, with a partial last
    # warp in x, and a three-plane thermal grid whose planes all feed ghosts
    dict(nx=130, ny=5, nz=4, bcy=1),
    dict(nx=6, ny=4, nz=3, bcz=1, thermal=True),
]


def _ids(c):
    return "-".join(f"{k}{v}" for k, v in c.items())


def _pair(lb, oracle, case, store, **kw):
    gk = {k: v for k, v in case.items() if k not in ("nx", "ny", "nz")}
    g = lb.Grid3(case["nx"], case["ny"], case["nz"], store=store, **gk).init(**kw)
    r = oracle.RefGrid3(case["nx"], case["ny"], case["nz"], **gk).set_params(**kw)
    return g, r


def oracle_weights3():
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return w[:, None, None, None]


def _params(th):
    kw = dict(tau=0.3, dt=0.05, ax=2e-4, ay=-1e-4, az=5e-5)
    if th:
        kw.update(tau_g=0.25, beta=1e-2, grav=1.0, T0=1.0, T_bot=1.3, T_top=0.8)
    return kw


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_fv3_step(lbgpu, oracle, case, store):
    lb = lbgpu
    th = case.get("thermal", False)
    g, r = _pair(lb, oracle, case, lb.STORE_NAMES[store], **_params(th))
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    f = inputs.random_populations3(nx, ny, nz, seed=nx + 7 * nz, amp=0.2)
    gg = inputs.random_populations3(nx, ny, nz, seed=5, amp=0.2) if th else None
    g.set_pops(f, gg)
    f, gg = g.get_pops()
    r.set_pops(f, gg)
    g.step_fv(3)
    r.step_fv(3)
    w = oracle.lattice3()[3][:, None, None, None]
    fg, gg2 = g.get_pops()
    fr, gr = r.get_pops()
    tol = 1e-13 if store == "f64" else 2e-6 * np.abs(f - w).max()
    assert np.abs(fg - fr).max() <= tol
    if th:
        assert np.abs(gg2 - gr).max() <= (1e-13 if store == "f64" else 2e-6 * np.abs(gg - w).max())


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("case", [dict(nx=9, ny=7, nz=6), dict(nx=8, ny=6, nz=10, bcz=1, thermal=True),
                                  dict(nx=6, ny=5, nz=7, bcy=1, bcz=1), dict(nx=1, ny=10, nz=8, bcz=1, thermal=True),
                                  # even widths take the paired kernel: whole warps, a partial
                                  # last warp, periodic wrap at the row ends, plates on z
                                  dict(nx=130, ny=9, nz=5), dict(nx=64, ny=6, nz=7, bcz=1, thermal=True),
                                  dict(nx=2, ny=4, nz=3)],
                         ids=_ids)
def test_st3_step(lbgpu, oracle, case, store):
    lb = lbgpu
    th = case.get("thermal", False)
    kw = _params(th)
    kw["dt"] = 1.0
    g, r = _pair(lb, oracle, case, lb.STORE_NAMES[store], **kw)
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    f = inputs.random_populations3(nx, ny, nz, seed=11 + nx, amp=0.2)
    gg = inputs.random_populations3(nx, ny, nz, seed=6, amp=0.2) if th else None
    g.set_pops(f, gg)
    f, gg = g.get_pops()
    r.set_pops(f, gg)
    g.step_st(4)
    r.step_st(4)
    w = oracle.lattice3()[3][:, None, None, None]
    tol = 1e-13 if store == "f64" else 2e-6 * np.abs(f - w).max()
    assert np.abs(g.get_pops()[0] - r.get_pops()[0]).max() <= tol
    if th:
        assert np.abs(g.get_pops()[1] - r.get_pops()[1]).max() <= (
            1e-13 if store == "f64" else 2e-6 * np.abs(gg - w).max())


@pytest.mark.parametrize("kind", ["tgv", "shear", "rb"])
def test_presets_and_observables(lbgpu, oracle, kind):
    """Presets, moments, conservation sums and Nusselt numbers equal the
    oracle's (FP64) before and after 20 FV steps."""
    lb = lbgpu
    if kind == "rb":
        case = dict(nx=8, ny=6, nz=12, lz=12.0, sz=2, stretch_z=4.0, bcz=1, thermal=True)
        kw = dict(tau=0.1, tau_g=0.1, dt=0.1, beta=1e-3, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
        init = dict(kind=lb.LB_INIT_RB, amp=1e-2, seed=1234)
        okind = oracle.INIT_RB
    else:
        case = dict(nx=12, ny=10, nz=8)
        kw = dict(tau=0.3, dt=0.5)
        init = dict(kind=lb.LB_INIT_TGV, u0=0.02) if kind == "tgv" else dict(kind=lb.LB_INIT_SHEAR, amp=0.01, mode=2)
        okind = oracle.INIT_TGV if kind == "tgv" else oracle.INIT_SHEAR
    gk = {k: v for k, v in case.items() if k not in ("nx", "ny", "nz")}
    g = lb.Grid3(case["nx"], case["ny"], case["nz"], store=lb.LB_STORE_F64, **gk).init(**kw, **init)
    r = oracle.RefGrid3(case["nx"], case["ny"], case["nz"], **gk).set_params(**kw)
    r.init_preset(okind, u0=init.get("u0", 0.0), amp=init.get("amp", 0.0), mode=init.get("mode", 1),
                  seed=init.get("seed", 0))
    for steps in (0, 20):
        g.step_fv(steps)
        r.step_fv(steps)
        fields = list(zip(g.moments(), r.moments()))
        for a, b in fields if kind == "rb" else fields[:4]:  # T is defined on thermal grids only
            assert np.abs(a - b).max() < 1e-13
        nc = 5 if kind == "rb" else 4  # heat is defined on thermal grids only
        # momenta cancel to rounding (~1e-14) on these symmetric states
        assert np.allclose(g.conservation()[:nc], r.conservation()[:nc], rtol=1e-12, atol=1e-12)
        if kind == "rb":
            assert np.allclose(g.nusselt(), r.nusselt(), rtol=1e-10, atol=1e-10)


def test_errors_and_states(lbgpu):
    lb = lbgpu
    with pytest.raises(lb.LBError):
        lb.Grid3(4, 4, 4, bcx=lb.LB_BC_WALLS, thermal=True)
    with pytest.raises(lb.LBError):
        lb.Grid3(4, 4, 5, sz=lb.LB_AXIS_SINH, stretch_z=2.0)
    with pytest.raises(lb.LBError):
        lb.Grid3(4, 4, 4, store=lb.LB_STORE_F16DEV)
    g = lb.Grid3(4, 4, 4)
    with pytest.raises(lb.LBError) as e:
        g.step_fv(1)
    assert e.value.status == lb.LB_ERR_STATE
    g.init(tau=0.3, dt=0.5)
    with pytest.raises(lb.LBError) as e:
        g.step_st(1)
    assert e.value.status == lb.LB_ERR_ARG
    with pytest.raises(lb.LBError) as e:
        g.nusselt()
    assert e.value.status == lb.LB_ERR_STATE


def test_rb_table_grid_sampled(lbgpu, oracle):
    """The FV workload of Table rb at its full size (128 x 128 x 64, sinh z
    grid, H = 640, L = 1280, dt = 4, tau = tau_g = 0.5) in FP32: after 2 steps
    from the seeded RB state the GPU equals the FP64 oracle on every cell to
    2e-6 of the deviation scale, and mass is conserved (heat is not: it
    crosses the isothermal plates)."""
    lb = lbgpu
    from paper_1505_03271_gb300 import configs as cfg
    w = cfg.rb3d_table("fv")
    gk = dict(w.grid)
    store = gk.pop("store")
    g = lb.Grid3(store=store, **gk).init(**w.params, **w.init)
    r = oracle.RefGrid3(**gk).set_params(**w.params)
    oracle.set_threads(8)
    r.init_preset(oracle.INIT_RB, amp=w.init["amp"], seed=w.init["seed"])
    f0, g0 = g.get_pops()
    r.set_pops(f0, g0)
    m0 = g.conservation()
    g.step_fv(2)
    r.step_fv(2)
    fg, tg = g.get_pops()
    fr, tr = r.get_pops()
    wts = oracle.lattice3()[3][:, None, None, None]
    assert np.abs(fg - fr).max() <= 2e-6 * np.abs(f0 - wts).max()
    assert np.abs(tg - tr).max() <= 2e-6 * np.abs(g0 - wts).max()
    m1 = g.conservation()
    assert abs(m1[0] / m0[0] - 1) < 1e-8


# grids the staged flux passes serve: x and y periodic, nx a power of two with
# 16-byte rows; ragged y tiles (ny not a multiple of the tile), z chunks with
# a short last chunk, z walls and plates on stretched grids
STAGED_CASES = [
    dict(nx=8, ny=6, nz=10, sz=2, stretch_z=4.0, bcz=1, thermal=True),
    dict(nx=16, ny=12, nz=20),
    dict(nx=32, ny=10, nz=12, sz=1, stretch_z=1.5, bcz=1, thermal=True),
    dict(nx=4, ny=3, nz=5, sy=1, stretch_y=1.2),
    dict(nx=64, ny=20, nz=17, sz=1, stretch_z=2.0, bcz=1),
    # a single z plane (periodic), a single y row, and two and three plates-bounded planes
    dict(nx=8, ny=6, nz=1),
    dict(nx=8, ny=1, nz=6, sz=1, stretch_z=1.5, bcz=1),
    dict(nx=4, ny=5, nz=2, bcz=1, thermal=True),
    dict(nx=16, ny=3, nz=3, bcz=1, thermal=True),
]


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("case", STAGED_CASES, ids=_ids)
def test_fv3_staged_step(lbgpu, oracle, case, store):
    """The staged flux passes (shared-memory z-plane ring filled by bulk
    copies) against the FP64 oracle, 3 steps from a random state."""
    lb = lbgpu
    th = case.get("thermal", False)
    g, r = _pair(lb, oracle, case, lb.STORE_NAMES[store], **_params(th))
    g.set_fv_schedule(lb.LB3_FV_STAGED)
    assert g.fv_schedule == lb.LB3_FV_STAGED
    nx, ny, nz = case["nx"], case["ny"], case["nz"]
    f = inputs.random_populations3(nx, ny, nz, seed=3 * nx + nz, amp=0.2)
    gg = inputs.random_populations3(nx, ny, nz, seed=9, amp=0.2) if th else None
    g.set_pops(f, gg)
    f, gg = g.get_pops()
    r.set_pops(f, gg)
    g.step_fv(3)
    r.step_fv(3)
    w = oracle.lattice3()[3][:, None, None, None]
    fg, tg = g.get_pops()
    fr, tr = r.get_pops()
    assert np.abs(fg - fr).max() <= (1e-13 if store == "f64" else 2e-6 * np.abs(f - w).max())
    if th:
        assert np.abs(tg - tr).max() <= (1e-13 if store == "f64" else 2e-6 * np.abs(gg - w).max())


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_fv3_staged_matches_plain(lbgpu, store):
    """Both flux schedules give the same 5 steps on a thermal RB grid, up to
    the rounding of the folded face weights."""
    lb = lbgpu
    case = dict(nx=32, ny=24, nz=18, lz=18.0, sz=2, stretch_z=3.0, bcz=1, thermal=True)
    kw = dict(tau=0.2, tau_g=0.2, dt=0.2, beta=1e-2, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    out = []
    for sched in (lb.LB3_FV_PLAIN, lb.LB3_FV_STAGED):
        gk = {k: v for k, v in case.items() if k not in ("nx", "ny", "nz")}
        g = lb.Grid3(case["nx"], case["ny"], case["nz"], store=lb.STORE_NAMES[store], **gk)
        g.init(**kw, kind=lb.LB_INIT_RB, amp=1e-2, seed=7).set_fv_schedule(sched)
        assert g.fv_schedule == sched
        g.step_fv(5)
        out.append(g.get_pops())
    # relative to the deviation scale: FP64 rounding, or a few FP32 ulps per step
    wts = oracle_weights3()
    for q in range(2):
        scale = np.abs(out[0][q] - wts * (1.0 if q == 0 else kw["T0"])).max()
        assert np.abs(out[0][q] - out[1][q]).max() <= (1e-12 if store == "f64" else 1e-5) * scale


def test_fv3_schedule_rules(lbgpu):
    """AUTO resolves to the staged passes exactly where they serve the grid;
    asking for them elsewhere is LB_ERR_ARG and leaves the grid as it was."""
    lb = lbgpu
    assert lb.Grid3(16, 8, 8).fv_schedule == lb.LB3_FV_STAGED
    for kw in (dict(nx=12, ny=8, nz=8), dict(nx=16, ny=8, nz=8, bcy=lb.LB_BC_WALLS),
               dict(nx=2, ny=8, nz=8), dict(nx=512, ny=2, nz=2)):
        g = lb.Grid3(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), **kw)
        assert g.fv_schedule == lb.LB3_FV_PLAIN
        with pytest.raises(lb.LBError) as e:
            g.set_fv_schedule(lb.LB3_FV_STAGED)
        assert e.value.status == lb.LB_ERR_ARG
        assert g.fv_schedule == lb.LB3_FV_PLAIN
    g = lb.Grid3(2, 8, 8, store=lb.LB_STORE_F64)  # 16-byte FP64 rows
    assert g.fv_schedule == lb.LB3_FV_STAGED
    with pytest.raises(lb.LBError):
        g.set_fv_schedule(7)


def test_fv3_staged_wait_timeout(lbgpu, oracle):
    """The bounded waits of the staged passes: with the test hook on, each
    CTA announces a copy group it never starts, its wait runs out (2 ms) and
    the step reports LB_ERR_TIMEOUT on the next sync; the grid is poisoned
    until lb3_init, after which the same context steps correctly again."""
    lb = lbgpu
    case = dict(nx=16, ny=8, nz=6)
    kw = dict(tau=0.3, dt=0.25, ax=1e-4)
    g, r = _pair(lb, oracle, case, lb.LB_STORE_F32, **kw)
    g.drop_copies(True)
    g.step_fv(1)
    with pytest.raises(lb.LBError) as e:
        g.sync()
    assert e.value.status == lb.LB_ERR_TIMEOUT
    with pytest.raises(lb.LBError) as e:
        g.step_fv(1)
    assert e.value.status == lb.LB_ERR_STATE
    g.drop_copies(False)
    g.init(**kw)
    f = inputs.random_populations3(16, 8, 6, seed=4, amp=0.2)
    g.set_pops(f)
    f, _ = g.get_pops()
    r.set_pops(f)
    g.step_fv(2).sync()
    r.step_fv(2)
    w = oracle.lattice3()[3][:, None, None, None]
    assert np.abs(g.get_pops()[0] - r.get_pops()[0]).max() <= 2e-6 * np.abs(f - w).max()


def test_fv3_staged_shapes(lbgpu):
    """Rows per tile, z planes per CTA and copies in flight change the
    schedule of the staged passes, not their arithmetic: the state after 3
    steps is bitwise the same for every shape; shapes out of range are
    LB_ERR_ARG."""
    lb = lbgpu
    kw = dict(tau=0.2, tau_g=0.2, dt=0.2, beta=1e-2, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    ref = None
    for shape in ((0, 0, 0), (1, 1, 1), (3, 5, 6), (16, 64, 12), (2, 7, 2)):
        g = lb.Grid3(16, 12, 20, lz=20.0, sz=lb.LB_AXIS_TANH, stretch_z=1.5, bcz=lb.LB_BC_WALLS, thermal=True)
        g.init(**kw, kind=lb.LB_INIT_RB, amp=1e-2, seed=3).set_staged_shape(*shape).step_fv(3)
        f, t = g.get_pops()
        if ref is None:
            ref = (f, t)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(t, ref[1]), shape
    g = lb.Grid3(16, 12, 20)
    for bad in ((65, 0, 0), (0, 300, 0), (0, 0, 13), (-1, 0, 0)):
        with pytest.raises(lb.LBError) as e:
            g.set_staged_shape(*bad)
        assert e.value.status == lb.LB_ERR_ARG


def test_fv3_autotune(lbgpu):
    """The 3-D autotuner restores the state bit for bit and keeps one of its
    candidates: stepping afterwards equals stepping a grid set to the picked
    schedule and shape by hand."""
    lb = lbgpu
    kw = dict(tau=0.2, tau_g=0.2, dt=0.2, beta=1e-2, grav=1.0, T0=1.0, T_bot=1.5, T_top=0.5)
    geo = dict(lz=20.0, sz=lb.LB_AXIS_TANH, stretch_z=1.5, bcz=lb.LB_BC_WALLS, thermal=True)

    def grid():
        return lb.Grid3(32, 16, 20, **geo).init(**kw, kind=lb.LB_INIT_RB, amp=1e-2, seed=11)

    g = grid()
    f0, t0 = g.get_pops()
    g.autotune_fv(2)
    f1, t1 = g.get_pops()
    assert np.array_equal(f0, f1) and np.array_equal(t0, t1)
    sched, shape = g.fv_schedule, g.staged_shape
    assert sched in (lb.LB3_FV_PLAIN, lb.LB3_FV_STAGED)
    g.step_fv(3)
    h = grid().set_fv_schedule(sched)
    if sched == lb.LB3_FV_STAGED:
        h.set_staged_shape(*shape)
    h.step_fv(3)
    for a, b in zip(g.get_pops(), h.get_pops()):
        assert np.array_equal(a, b)
    with pytest.raises(lb.LBError):
        g.autotune_fv(0)
