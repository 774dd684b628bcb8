"""Continuous batching: results are the same alone and in the mix (GPU)."""
import numpy as np
import pytest

from paper_2410_06657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _requests(prec):
    """Four small freezing runs of different sizes and parameters; later
    ones arrive while earlier ones are running (virtual clock below)."""
    shapes = [(64, 32, 10.0, 80.0, 0.3, 2.0, 5.0, 0.9), (96, 48, 15.0, 110.0, 0.1, 0.5, 2.0, 0.6),
              (64, 32, 10.0, 100.0, 0.0, 5.0, 9.5, 1.0), (48, 24, 7.5, 70.0, 0.5, 2.0, 0.5, 0.8)]
    from paper_2410_06657_gb300.serving import Request
    out = []
    for i, (nx, ny, R, th, ca, rs, se, ste) in enumerate(shapes):
        p = W.params(nx=nx, ny=ny, R0=R, theta_deg=th, CaE=ca, R_sigma=rs, S_eps=se, Ste=ste,
                     alpha_l=0.1, precision=prec)
        xc, yc = W.sessile_center(nx, R, th)
        out.append(Request(id=i, arrival=0.0 + i * 1.0, params=p, R=R, xc=xc, yc=yc))
    return out


class TickClock:
    """Virtual clock: one unit per tick, so admissions are deterministic."""
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.5
        return self.t


@pytest.mark.parametrize("prec", [W.FP64, W.FP32], ids=["fp64", "fp32"])
def test_results_same_alone_and_in_the_mix(prec):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_06657_gb300.serving import Server, footprint_bytes, run_alone
    reqs = _requests(prec)
    budget = sum(footprint_bytes(r.params) for r in reqs[:3])   # the fourth waits for memory
    srv = Server(budget, chunk=100, clock=TickClock())
    res = srv.run(reqs)
    assert [r.id for r in res] == [0, 1, 2, 3]
    assert all(r.frozen for r in res)
    admitted = sorted(r.admitted for r in res)
    assert len(set(admitted)) > 1          # admissions happened at different times
    for req, r in zip(reqs, res):
        alone = run_alone(req, chunk=100)
        if prec == W.FP64:
            assert r.steps == alone["step"] and r.t_fre == alone["t_fre"]
        else:   # a rounding-level difference may move the detection by one chunk
            assert abs(r.steps - alone["step"]) <= 100 and abs(r.t_fre - alone["t_fre"]) <= 100
        for k in ("frozen_fraction", "mass", "height", "width", "aspect"):
            if prec == W.FP64:
                assert r.obs[k] == alone[k], (req.id, k)
            elif r.steps == alone["step"]:
                assert abs(r.obs[k] - alone[k]) <= 5e-3 * max(abs(alone[k]), 1.0), (req.id, k)
