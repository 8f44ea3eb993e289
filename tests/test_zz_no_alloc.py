"""lb_conservation_noalloc: the conservation sums for callers that cannot
allocate device memory (their memory belongs to their own pool, or an
allocation would stall a latency-critical path).  It must give the same sums
as lb_conservation on the same state, call after call, while its scratch
lives in a fixed array inside the library.  This file is collected last so
that a failure here stops a -x run only after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _device_copy(torch, pops, offset, nx, ny, pitch):
    """Caller-owned FP32 buffer [9][ny][pitch] holding pops - w * offset."""
    buf = torch.zeros((9, ny, pitch), dtype=torch.float32, device="cuda")
    dev = (pops - W[:, None, None] * offset).astype(np.float32)
    buf[:, :, :nx] = torch.from_numpy(dev).cuda()
    return buf


def test_noalloc_matches_lb_conservation(lbgpu):
    import torch
    lb = lbgpu
    nx, ny, pitch = 300, 200, 320
    T0 = 1.0
    params = dict(tau=0.3, dt=0.5, tau_g=0.25, ax=1e-5, ay=2e-6, beta=1e-3, grav=1.0, T0=T0)
    g = lb.Grid(nx, ny, thermal=True, store="f32")
    g.init(kind=lb.LB_INIT_TGV, u0=0.02, amp=0.01, mode=2, **params)
    dx = torch.ones(nx, dtype=torch.float64, device="cuda")
    dy = torch.ones(ny, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row, on two different states
        g.step_fv(3)
        ref = np.array(g.conservation())
        f, gg = g.get_pops()
        fd = _device_copy(torch, f, 1.0, nx, ny, pitch)
        gd = _device_copy(torch, gg, T0, nx, ny, pitch)
        out.fill_(float("nan"))
        lb.lb_conservation_noalloc(fd.data_ptr(), gd.data_ptr(), nx, ny, pitch, dx.data_ptr(),
                                   dy.data_ptr(), params["dt"], params["ax"], params["ay"],
                                   params["beta"] * params["grav"], T0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-15), (call, got, ref)


def test_noalloc_flow_only_and_size_limit(lbgpu):
    import torch
    lb = lbgpu
    nx, ny = 64, 48
    g = lb.Grid(nx, ny, store="f32")
    g.init(tau=0.3, dt=1.0, ax=1e-5, kind=lb.LB_INIT_TGV, u0=0.02)
    g.step_st(4)
    ref = np.array(g.conservation())
    f, _ = g.get_pops()
    fd = _device_copy(torch, f, 1.0, nx, ny, nx)
    one_x = torch.ones(nx, dtype=torch.float64, device="cuda")
    one_y = torch.ones(ny, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        lb.lb_conservation_noalloc(fd.data_ptr(), None, nx, ny, nx, one_x.data_ptr(),
                                   one_y.data_ptr(), 1.0, 1e-5, 0.0, 0.0, 1.0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got[:3] - ref[:3]) <= 1e-12 * np.abs(ref[:3]) + 1e-15)
    # beyond the fixed scratch: rejected before any work is queued
    with pytest.raises(lb.LBError) as e:
        lb.lb_conservation_noalloc(fd.data_ptr(), None, 4096, 4096, 4096, one_x.data_ptr(),
                                   one_y.data_ptr(), 1.0, 0.0, 0.0, 0.0, 1.0, out.data_ptr(), stream)
    assert e.value.status == lb.LB_ERR_ARG
    assert "8388608" in lb.lb_last_error()


def test_noalloc_stretched_grid_volume_weights(lbgpu, oracle):
    """A tanh-refined y axis and a sinh-refined x axis with nx != ny: the
    volume weight V = dx[i] * dy[j] varies along both axes, so a swapped or
    mis-indexed width changes every sum.  The cell widths are the grid's own
    (Eq. (grids)), passed as device FP64 arrays; the state is random fields
    stepped twice, so mass, momentum and heat all vary from cell to cell."""
    import torch
    from tests import inputs
    lb = lbgpu
    nx, ny = 96, 70
    T0 = 1.0
    g = lb.Grid(nx, ny, sx=lb.LB_AXIS_SINH, sy=lb.LB_AXIS_TANH, stretch_x=3.0, stretch_y=2.0,
                thermal=True, store="f32")
    params = dict(tau=0.2, dt=0.05, tau_g=0.2, ax=1e-5, ay=-2e-6, beta=1e-3, grav=1.0, T0=T0)
    rho, ux, uy, T = inputs.random_fields(nx, ny, seed=21, T_amp=0.05, T0=T0)
    g.init(rho=rho, ux=ux, uy=uy, T=T, **params)
    g.step_fv(2)
    ref = np.array(g.conservation())
    f, gg = g.get_pops()
    fd = _device_copy(torch, f, 1.0, nx, ny, nx)
    gd = _device_copy(torch, gg, T0, nx, ny, nx)
    wx = np.diff(oracle.faces(nx, float(nx), oracle.SINH, 3.0))
    wy = np.diff(oracle.faces(ny, float(ny), oracle.TANH, 2.0))
    assert np.ptp(wx) > 0.1 and np.ptp(wy) > 0.1
    dx = torch.from_numpy(wx).cuda()
    dy = torch.from_numpy(wy).cuda()
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        lb.lb_conservation_noalloc(fd.data_ptr(), gd.data_ptr(), nx, ny, nx, dx.data_ptr(),
                                   dy.data_ptr(), params["dt"], params["ax"], params["ay"],
                                   params["beta"] * params["grav"], T0, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-15), (got, ref)
