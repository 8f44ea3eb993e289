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
