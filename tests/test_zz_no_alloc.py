"""The allocation-free observables entry point against the regular one.

lbm_observables_noalloc serves callers that cannot call cudaMalloc (a
runtime that already owns the device memory pool, or a latency-critical loop
that must not synchronise the device).  It reads a caller-held state and
writes a caller-provided device lbm_obs, with its scratch in a fixed array of
the library.  Here the state is a snapshot body uploaded by the test (the
test itself may allocate; the entry point must not), and the result must
equal what lbm_observables reports for the same state, on three calls in a
row, and the calls after the first must not change the device's free memory.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2410_06657_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER_BYTES = 64   # snapshot header before the arrays


def _setup(lbm):
    L = lbm.load()
    L.lbm_observables_noalloc.argtypes = [C.POINTER(lbm.Params), C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_int64, C.c_void_p, C.c_void_p]
    return L


@pytest.mark.parametrize("prec", [W.FP64, W.FP32, W.FP16S])
def test_noalloc_observables_match_lbm_observables(prec):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_06657_gb300 import lbm
    L = _setup(lbm)
    nx, ny, R = 100, 45, 14.0
    p = W.params(nx=nx, ny=ny, R0=R, theta_deg=80.0, precision=prec, k_e=2)
    stream = torch.cuda.current_stream()
    sim = lbm.Simulation(p, stream)
    xc, yc = W.sessile_center(nx, R, 80.0)
    sim.init_droplet(R, xc, yc, 5)
    pitch = (nx + 31) // 32 * 32
    elem = {W.FP64: 8, W.FP32: 4, W.FP16S: 2}[prec]
    f_elem = 8 if prec == W.FP64 else 4      # half storage keeps f in single precision
    aux_elem = 8 if prec == W.FP64 else 4
    plane = pitch * ny
    pop_bytes, aux_bytes = 9 * plane * f_elem + 23 * plane * elem, 7 * plane * aux_elem

    out = torch.zeros(C.sizeof(lbm.Obs), dtype=torch.uint8, device="cuda")
    init = lbm.Obs()
    init.t_fre = -1
    init.Fo_fre = -1.0
    out.copy_(torch.frombuffer(bytearray(bytes(init)), dtype=torch.uint8))
    cp = lbm.make_params(p)
    for call in range(3):
        sim.step(60 if call == 0 else 25)
        want = sim.observables()
        snap = sim.export_state()
        body = torch.from_numpy(snap[HEADER_BYTES:HEADER_BYTES + pop_bytes + aux_bytes].copy()).cuda()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = L.lbm_observables_noalloc(C.byref(cp), C.c_void_p(body.data_ptr()),
                                       C.c_void_p(body.data_ptr() + pop_bytes), pitch, sim.t,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0, L.lbm_last_error()
        torch.cuda.synchronize()
        # the first call may load the library's module on this device; after
        # it, a call must leave the device's free memory exactly as it was
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free_before, call
        got = lbm.Obs.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()
        for k, v in want.items():
            if isinstance(v, float):
                assert abs(got[k] - v) <= 1e-12 * max(abs(v), 1.0), (call, k, got[k], v)
            else:
                assert got[k] == v, (call, k, got[k], v)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_06657_gb300 import lbm
    L = _setup(lbm)
    p = lbm.make_params(W.params(nx=64, ny=5000, precision=W.FP32))
    rc = L.lbm_observables_noalloc(C.byref(p), C.c_void_p(16), C.c_void_p(16), 64, 0, C.c_void_p(16), None)
    assert rc == lbm.ERR_BADPARAM
    assert b"scratch" in L.lbm_last_error()
