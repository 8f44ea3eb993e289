"""The accuracy and stability studies (Figs. POI2, POI3, KOL3) through the C
ABI: their building blocks agree with the FP64 oracle run the same way."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_stability_verdicts_match_oracle(lbgpu, oracle):
    """The GPU stability probe (shear wave + seeded noise, 3000 steps) gives
    the oracle's verdicts at points on both sides of each scheme's limit."""
    import torch

    from paper_1505_03271_gb300 import studies
    probes = [("euler", 0.25, 0.45), ("semi", 0.25, 0.45), ("semi", 0.25, 0.65), ("heun", 0.25, 0.65),
              ("semi", 0.125, 1.2), ("heun", 0.125, 1.2), ("euler", 0.25, 0.3), ("heun", 0.5, 1.2)]
    got = studies.stable_many(lbgpu, torch, probes)
    sch = {"euler": oracle.FV_EULER, "semi": oracle.FV_SEMI, "heun": oracle.FV_HEUN}
    oracle.set_threads(1)
    for s, tau, dt in probes:
        r = oracle.RefGrid(1, 64, lx=1.0, ly=64.0).set_scheme(sch[s]).set_params(tau=tau, dt=dt)
        r.init_preset(oracle.INIT_SHEAR, amp=1e-5)
        f, _ = r.get_pops()
        rng = np.random.default_rng(1)
        r.set_pops(f + 1e-6 * studies.W[:, None, None] * rng.standard_normal(f.shape))
        k0, ok = None, True
        for _ in range(30):
            r.step_fv(100)
            _, ux, uy, _ = r.moments()
            k = float((ux**2 + uy**2).sum())
            k0 = k if k0 is None else k0
            if not math.isfinite(k) or k > 10 * k0:
                ok = False
                break
        assert got[(s, tau, dt)] == ok, (s, tau, dt)


@pytest.mark.parametrize("method,n", [("fv-tanh", 16), ("fv-cheb", 12), ("fv-sinh", 16), ("st", 16)])
def test_poiseuille_case_matches_oracle(lbgpu, oracle, method, n):
    """One Poiseuille run of the refinement study (shortened to one decay
    time) gives the oracle's error to 1e-9 relative."""
    import torch

    from paper_1505_03271_gb300 import studies
    case = studies.Poiseuille(method, n, 64.0, relax=1.0)
    got = studies.run_poiseuille(lbgpu, torch, [case])[case]
    grid, params, U, steps, xi, L, scheme = case.spec()
    r = oracle.RefGrid(grid["nx"], grid["ny"], lx=grid["lx"], ly=grid["ly"], sy=grid.get("sy", 0),
                       stretch_y=grid.get("stretch_y", 0.0), bcy=grid["bcy"]).set_params(**params)
    r.init_preset(oracle.INIT_POISEUILLE, u0=U)
    oracle.set_threads(1)
    (r.step_st if scheme == "st" else r.step_fv)(steps)
    err = case.error(r.moments()[1][:, 0], xi, L, U)
    assert abs(got["err"] - err) <= 1e-9 * err
    assert got["steps"] == steps and 0 < err < 0.1
