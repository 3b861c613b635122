"""swe_step_noalloc: the one entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc while they run: real-time
loops that cannot take cudaMalloc's device-wide synchronisation, and
applications whose own allocator owns all device memory.  Its working memory
is a fixed array inside the library that every call shares, so the test
checks that consecutive calls reproduce the ordinary handle-based path
(swe_create, swe_set_state, swe_step from the same input) bit for bit: the
two run the same kernels with the same constants.  A call on a grid of
another size, with dry blocks, sits between the two compared calls, so a
census, skip flag or block list left over in the shared array would show.
This file sorts last so a stop-at-first-failure run has already run every
other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe
    return swe, swe.load_library()


def _state(nx, ny, seed, wet_fraction, x0=0):
    side = max(nx + x0, ny)
    sc = I.half_wet(side, dx=5.0, seed=seed, wet_fraction=wet_fraction)
    H = np.ascontiguousarray(sc.H[:ny, x0:x0 + nx], dtype=np.float32)
    b = np.ascontiguousarray(sc.b[:ny, x0:x0 + nx], dtype=np.float32)
    rng = I.rng(seed + 1)
    wet = H > 1e-4
    Hu = np.where(wet, rng.normal(0, 0.3, H.shape).astype(np.float32) * H, 0).astype(np.float32)
    Hv = np.where(wet, rng.normal(0, 0.3, H.shape).astype(np.float32) * H, 0).astype(np.float32)
    return np.stack([H, Hu, Hv, b], -1)


def _handle_step(swe, aos, nman):
    """The existing path: a solver handle, swe_set_state, one swe_step."""
    ny, nx = aos.shape[:2]
    S = swe.Solver(nx, ny, 5.0, precision="fp32")
    S.set_manning(np.full((ny, nx), nman), block=0)
    S.set_state(*(aos[..., q] for q in range(4)))
    dt = S.step()
    out = np.stack(S.get_state(np.float32), -1)
    census = S.census()
    S.close()
    return out, dt, census


def _noalloc(swe, L, aos_dev, out_dev, nman):
    import torch
    ny, nx = aos_dev.shape[:2]
    p = swe.Params()
    assert L.swe_params_default(ctypes.byref(p), nx, ny, 5.0) == swe.SWE_OK
    dt = ctypes.c_double(0.0)
    st = L.swe_step_noalloc(ctypes.byref(p), nman, ctypes.c_void_p(aos_dev.data_ptr()),
                            ctypes.c_void_p(out_dev.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(dt))
    assert st == swe.SWE_OK, st
    return dt.value


def test_noalloc_consecutive_calls_match_the_handle_path_bit_for_bit():
    import torch
    swe, L = _lib()
    nman = 0.035
    a0 = _state(512, 512, 5, 0.5)           # grid A: 3 x 16 blocks
    dry = _state(300, 700, 9, 0.02, x0=400)  # grid B: 2 x 22 blocks, 19 of them dry

    bufs = [torch.from_numpy(a0).cuda().contiguous()]
    bufs += [torch.empty_like(bufs[0]) for _ in range(2)]
    db = [torch.from_numpy(dry).cuda().contiguous(), None]
    db[1] = torch.empty_like(db[0])
    torch.cuda.synchronize()

    # call 1 on grid A
    ref1, dt1, _ = _handle_step(swe, a0, nman)
    d1 = _noalloc(swe, L, bufs[0], bufs[1], nman)
    got1 = bufs[1].cpu().numpy()
    assert d1 == dt1
    assert np.array_equal(got1, ref1)

    # a call on grid B in between: another block grid, dry blocks skipped
    refB, dtB, cenB = _handle_step(swe, dry, nman)
    assert np.any(cenB == 0) and np.any(cenB > 0)
    dB = _noalloc(swe, L, db[0], db[1], nman)
    assert dB == dtB
    assert np.array_equal(db[1].cpu().numpy(), refB)

    # call 2 on grid A, from call 1's output
    ref2, dt2, _ = _handle_step(swe, got1, nman)
    d2 = _noalloc(swe, L, bufs[1], bufs[2], nman)
    assert d2 == dt2
    assert np.array_equal(bufs[2].cpu().numpy(), ref2)
    assert not np.array_equal(ref2, ref1)


def test_noalloc_rejects_what_it_cannot_do():
    import torch
    swe, L = _lib()
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
