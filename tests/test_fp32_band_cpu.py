"""The FP32 comparison band around the Shamov gate (tests/fp32_band.py): its
edges switch the gate only for velocities within a few 1e-6 of the critical
velocity of Eq. 5, and leave every other cell's result unchanged."""
import math

import numpy as np

from fp32_band import C_SH_BAND, band_error, band_params


def _frozen(orc, v0, p_kw=None):
    nx, dx = 32, 2.0
    x = (np.arange(nx) + 0.5) * dx
    b = 0.05 * np.cos(2 * math.pi * x / (nx * dx))[None, :]
    H = np.ones((1, nx))
    st = orc.State(H, 0 * H, H * v0, b)
    return st, orc.Params(nx=nx, ny=1, dx=dx, frozen_hydro=1, A_J=0.002, tile_x=nx, tile_y=1, **(p_kw or {}))


def test_band_edges_switch_the_gate_only_near_the_critical_velocity(orc):
    p0 = orc.Params(nx=1, ny=1)
    vk = p0.C_Sh * p0.d50 ** (1 / 3)          # H = 1
    # just below v_k: off at the threshold, on at the lower band edge
    st, p = _frozen(orc, vk * (1 - 2e-6))
    res = [orc.step(pp, st, 0.03)[0] for pp in band_params(p)]
    assert np.array_equal(res[0].b, st.b)
    assert not np.array_equal(res[1].b, st.b)
    assert np.array_equal(res[2].b, st.b)
    # well below: off everywhere in the band; well above: the same result
    for v in (vk * (1 - 1e-4), vk * 1.5):
        st, p = _frozen(orc, v)
        res = [orc.step(pp, st, 0.03)[0].arrays() for pp in band_params(p)]
        for r in res[1:]:
            for a, b in zip(r, res[0]):
                assert np.array_equal(a, b)
    assert C_SH_BAND * 6 < 1e-4


def test_band_error_takes_the_nearest_result():
    a = [np.zeros((2, 2))] * 4
    b = [np.full((2, 2), 1e-3)] * 4
    got = np.full((2, 2), 1e-3, dtype=np.float32)
    excess, plain = band_error(got, [a, b], 3)
    assert np.all(excess <= 0) and np.all(plain > 4e-5)
    excess, _ = band_error(got, [a], 3)
    assert np.all(excess > 0)
