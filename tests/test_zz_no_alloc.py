"""swe_step_noalloc: the one entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc while they run (code being
captured into a CUDA graph, real-time loops that cannot take cudaMalloc's
device-wide synchronisation, applications whose own allocator owns all device
memory).  Its working memory is a fixed array inside the library, so the
test checks that two calls in a row reproduce the ordinary handle-based path
(swe_create / swe_set_state / swe_step) within the FP32 per-step tolerance of
the parity tests.  This file sorts last so a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 4e-5  # FP32 per-step tolerance of tests/test_gpu_parity.py


def test_noalloc_two_steps_match_handle_path():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe

    L = swe.load_library()
    L.swe_step_noalloc.argtypes = [ctypes.POINTER(swe.Params), ctypes.c_double, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    L.swe_step_noalloc.restype = ctypes.c_int

    n, dx, nman = 512, 5.0, 0.035
    sc = I.half_wet(n, dx=dx, seed=5)
    H, Hu, Hv, b = (np.ascontiguousarray(a, dtype=np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b))
    rng = I.rng(6)
    wet = H > 1e-4
    Hu = np.where(wet, rng.normal(0, 0.3, H.shape).astype(np.float32) * H, 0).astype(np.float32)
    Hv = np.where(wet, rng.normal(0, 0.3, H.shape).astype(np.float32) * H, 0).astype(np.float32)

    # the ordinary path through a handle
    S = swe.Solver(n, n, dx, precision="fp32")
    S.set_manning(np.array([[nman]]), block=n)
    S.set_state(H, Hu, Hv, b)
    dt_ref = [S.step()]
    ref = [np.stack(S.get_state(np.float32), -1)]
    dt_ref.append(S.step())
    ref.append(np.stack(S.get_state(np.float32), -1))
    S.close()

    # the allocation-free path on caller-owned AoS buffers
    p = swe.Params()
    assert L.swe_params_default(ctypes.byref(p), n, n, dx) == swe.SWE_OK
    bufs = [torch.from_numpy(np.stack([H, Hu, Hv, b], -1)).cuda().contiguous()]
    bufs += [torch.empty_like(bufs[0]) for _ in range(2)]
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for k in range(2):
        dt = ctypes.c_double(0.0)
        st = L.swe_step_noalloc(ctypes.byref(p), nman, ctypes.c_void_p(bufs[k].data_ptr()),
                                ctypes.c_void_p(bufs[k + 1].data_ptr()), ctypes.c_void_p(stream),
                                ctypes.byref(dt))
        assert st == swe.SWE_OK, st
        got = bufs[k + 1].cpu().numpy()
        assert dt.value == pytest.approx(dt_ref[k], rel=1e-12)
        err = np.abs(got.astype(np.float64) - ref[k].astype(np.float64)).max()
        assert err <= TOL, (k, err)


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe

    L = swe.load_library()
    L.swe_step_noalloc.argtypes = [ctypes.POINTER(swe.Params), ctypes.c_double, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    L.swe_step_noalloc.restype = ctypes.c_int
    p = swe.Params()
    L.swe_params_default(ctypes.byref(p), 64, 1 << 22, 1.0)   # too many rows for the fixed array
    a = torch.zeros(16, device="cuda")
    bb = torch.zeros(16, device="cuda")
    assert L.swe_step_noalloc(ctypes.byref(p), 0.03, ctypes.c_void_p(a.data_ptr()),
                              ctypes.c_void_p(bb.data_ptr()), None, None) == swe.SWE_EINVAL
    L.swe_params_default(ctypes.byref(p), 8, 8, 1.0)
    p.precision = swe.SWE_FP64
    assert L.swe_step_noalloc(ctypes.byref(p), 0.03, ctypes.c_void_p(a.data_ptr()),
                              ctypes.c_void_p(bb.data_ptr()), None, None) == swe.SWE_EINVAL
