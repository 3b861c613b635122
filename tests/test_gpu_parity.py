"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
  * FP64 build, per step from identical inputs: relative L-infinity <= 1e-11
    (H against max|H|, momenta against max|H| sqrt(g max|H|), b against
    max(max|b|, 1e-3)); dt to 1e-13; census bit-exact.
  * FP32 build after a config's full run: relative L1 <= 1e-4 on H and b,
    and <= 5e-4 on the bed change b - b0 (the Grass load is cubic in the
    velocity: ~3x the water state's relative error).
  * FP32 single step at full size, sampled windows: the per-step bound derived
    from FP32 rounding of the largest intermediate (the free surface
    eta <= ~25 m: ulp 2e-6) times the ~10 roundings on its path: 4e-5 m on H
    and b, 4e-5 m^2/s + 2e-5 |Hu| on momenta.  Per element, against the
    oracle at the Shamov threshold or at the edges of the FP32 decision band
    around it (tests/fp32_band.py).
"""
import math
import os
import time

import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I
from fp32_band import band_error, band_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe
    swe.load_library()
    return swe


def _rel_linf(g, o, H_ref):
    gH, gU, gV, gb = g
    oH, oU, oV, ob = o
    hs = max(np.abs(H_ref).max(), 1e-12)
    ms = hs * math.sqrt(9.81 * hs)
    bs = max(np.abs(ob).max(), 1e-3)
    return (np.abs(gH - oH).max() / hs, np.abs(gU - oU).max() / ms,
            np.abs(gV - oV).max() / ms, np.abs(gb - ob).max() / bs)


def _fp64_solver(gpu, sc, bw=128, th=32, **kw):
    S = gpu.Solver(sc.nx, sc.ny, sc.dx, precision="fp64", block_cols=bw, tile_rows=th, **kw)
    if sc.manning_block > 1:
        S.set_manning(sc.manning, block=sc.manning_block)
    else:
        S.set_manning(np.broadcast_to(sc.manning, (sc.ny, sc.nx)).copy(), block=0)
    if sc.src is not None:
        S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
    S.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
    return S


def _per_step_parity(gpu, orc, sc, nsteps, bw=128, th=32, tol=1e-11, check_census=True, qb=None, rain=None,
                     beta=None, **kw):
    S = _fp64_solver(gpu, sc, bw=bw, th=th, **kw)
    if qb is not None:
        S.set_bed_source(qb)
    if rain is not None:
        S.set_rain(rain)
    if beta is not None:
        S.set_infiltration(beta)
    d = S.diag()
    p = orc.Params(nx=sc.nx, ny=sc.ny, dx=sc.dx, tile_x=d["tile_x"], tile_y=d["tile_y"], **kw)
    n_cell = sc.manning_per_cell()
    hydro = orc.Hydrograph(sc.hydro_t, sc.hydro_Q) if sc.src is not None else None
    st = orc.State(*S.get_state())
    t = 0.0
    worst = np.zeros(4)
    for it in range(nsteps):
        o, info = orc.step(p, st, n_cell, src=sc.src, qb=qb, hydro=hydro, t=t, rain=rain, beta=beta)
        dt = S.step()
        g = S.get_state()
        assert dt == pytest.approx(info.dt, rel=1e-13, abs=0), it
        err = np.array(_rel_linf(g, o.arrays(), o.H))
        worst = np.maximum(worst, err)
        assert np.all(err <= tol), (it, err)
        if check_census:
            cg = S.census()
            co = orc.census(p, g[0], sc.src)
            assert np.array_equal(cg, co), it
        st = orc.State(*g)
        t = t + info.dt
    S.close()
    return worst


def test_fp64_parity_dam_break_128(gpu, orc):
    """The 128^2 dam break over the noisy erodible bed, 500 steps."""
    sc = I.dam_break(128, 128, seed=1)
    worst = _per_step_parity(gpu, orc, sc, 500, bw=128, th=32)
    print("fp64 dam break worst rel Linf (H, Hu, Hv, b):", worst)


def test_fp64_parity_flood_channel_ragged_tiles(gpu, orc):
    """Initially dry fractal terrain, inflow hydrograph, partially dry fronts,
    HGS skipping on, grid not a multiple of the block (200 x 176 cells with
    120 x 32 blocks)."""
    sc = I.flood_channel(200, dx=5.0, seed=2, peak=300.0)
    sc2 = I.Scenario(200, 176, 5.0, sc.H[:176], sc.Hu[:176], sc.Hv[:176], sc.b[:176],
                     sc.manning, manning_block=64, src=sc.src[:176], hydro_t=sc.hydro_t,
                     hydro_Q=sc.hydro_Q)
    # start from a wetted state: run the oracle a little first to get fronts
    p0 = orc.Params(nx=200, ny=176, dx=5.0)
    st, t, _ = orc.run(p0, orc.State(sc2.H, sc2.Hu, sc2.Hv, sc2.b), sc2.manning_per_cell(), 150,
                       src=sc2.src, hydro=orc.Hydrograph(sc2.hydro_t, sc2.hydro_Q))
    sc2.H, sc2.Hu, sc2.Hv, sc2.b = st.H, st.Hu, st.Hv, st.b
    assert (st.H > 1e-4).sum() > 20
    worst = _per_step_parity(gpu, orc, sc2, 200, bw=128, th=32)
    print("fp64 flood channel worst rel Linf:", worst)


def test_fp64_parity_tall_strips(gpu, orc):
    """Blocks of the benchmark's height (120 x 256 cells) on a 300 x 560
    half-wet fractal grid moving across every side: 3 column bands (the last
    60 columns wide) x 3 strips (the last 48 rows high), so most sweep
    positions run the copy without row-range tests; per step against the
    oracle to 1e-11 relative, 40 steps."""
    nx, ny = 300, 560
    base = I.half_wet(max(nx, ny), dx=5.0, seed=61, wet_fraction=0.5, dtype=np.float64)
    H = np.ascontiguousarray(base.H[:ny, :nx])
    sc = I.Scenario(nx, ny, 5.0, H, 0.4 * H, -0.25 * H, np.ascontiguousarray(base.b[:ny, :nx]),
                    np.full((1, 1), 0.03), manning_block=1024)
    worst = _per_step_parity(gpu, orc, sc, 40, bw=128, th=256, A_J=0.01)
    print("fp64 tall strips worst rel Linf (H, Hu, Hv, b):", worst)


@pytest.mark.parametrize("knots", [1, 2, 4, 7])
def test_fp64_parity_hydrograph_knots(gpu, orc, knots):
    """Inflow hydrographs of 1, 2, 4 (read into registers in one batch) and 7
    (read knot by knot) knots within the first 12 s, about a step apart, so
    the steps start before the first knot, cross knots and run past the last:
    the source increment, hence H, and dt match the oracle per step."""
    sc = I.flood_channel(64, dx=5.0, seed=2, peak=300.0)
    g = I.rng(50 + knots)
    sc.hydro_t = np.sort(g.uniform(0.5, 12.0, knots))
    sc.hydro_Q = g.uniform(5.0, 80.0, knots)
    _per_step_parity(gpu, orc, sc, 30, bw=128, th=32)


@pytest.mark.parametrize("shape", [(1, 9), (9, 1), (3, 5), (4, 4), (130, 3)])
def test_fp64_parity_tiny_and_thin_grids(gpu, orc, shape):
    ny, nx = shape
    g = I.rng(31)
    H = 1.0 + g.uniform(0, 0.5, (ny, nx))
    Hu = g.normal(0, 0.3, (ny, nx))
    Hv = g.normal(0, 0.3, (ny, nx))
    b = g.uniform(-0.05, 0.05, (ny, nx))
    sc = I.Scenario(nx, ny, 1.0, H, Hu, Hv, b, np.full((1, 1), 0.03), manning_block=256)
    _per_step_parity(gpu, orc, sc, 20, bw=128, th=32, A_J=0.05)


def _moving_sediment_case(side=96, seed=41):
    """Half-wet terrain with a 2 m dam-break step and an inflow hydrograph,
    per-cell Manning n."""
    sc = I.ensemble_scenario(side, seed=seed, manning=0.03, peak=200.0, d50_scale=1.0)
    sc = I.Scenario(side, side, sc.dx, sc.H, sc.Hu, sc.Hv, sc.b, np.full((side, side), 0.03),
                    manning_block=1, src=sc.src, hydro_t=sc.hydro_t, hydro_Q=sc.hydro_Q)
    return sc


@pytest.mark.parametrize("opts", [
    {"sediment_on": 0},
    {"aj_mode": 1},
    {"dt_literal_D": 1, "A_J": 0.05},
    {"hgs_skip": 0, "A_J": 0.02},
    {"bed_source": True},
    {"bc_w": 1, "bc_e": 1, "bc_s": 1, "bc_n": 1},
    {"bc_e": 1, "bc_n": 1, "A_J": 0.02},
    {"rain": True},
    {"infiltration": True},
], ids=["exner_off", "aj_from_eq4", "literal_D", "hgs_off", "bed_source", "open_all", "open_mixed", "rain",
        "infiltration"])
def test_fp64_parity_options(gpu, orc, opts):
    """The step's options against the oracle, per step: the Exner coupling
    off (the surrogate's water-only steps), A_J from Eq. 4, the printed Eq. 7
    D term, HGS skipping off, and a bed source field, with per-cell Manning
    and an inflow hydrograph on partially wet terrain; open (zero-gradient)
    boundaries on all or some sides; a per-cell rain field."""
    sc = _moving_sediment_case()
    kw = {k: v for k, v in opts.items() if k not in ("bed_source", "rain", "infiltration")}
    qb = rain = beta = None
    if opts.get("bed_source"):
        g = I.rng(43)
        qb = g.normal(0.0, 1e-4, (sc.ny, sc.nx))
    if opts.get("rain"):
        g = I.rng(44)
        rain = g.uniform(0.0, 2e-4, (sc.ny, sc.nx))
    if opts.get("infiltration"):
        g = I.rng(45)
        beta = g.uniform(0.0, 5e-3, (sc.ny, sc.nx))     # drains thin films within the run
    p0 = orc.Params(nx=sc.nx, ny=sc.ny, dx=sc.dx, **kw)
    st, t, _ = orc.run(p0, orc.State(sc.H, sc.Hu, sc.Hv, sc.b), sc.manning_per_cell(), 40, src=sc.src,
                       qb=qb, hydro=orc.Hydrograph(sc.hydro_t, sc.hydro_Q), rain=rain, beta=beta)
    sc.H, sc.Hu, sc.Hv, sc.b = st.H, st.Hu, st.Hv, st.b
    worst = _per_step_parity(gpu, orc, sc, 30, bw=128, th=16, qb=qb, rain=rain, beta=beta, **kw)
    print("fp64 options", opts, "worst rel Linf:", worst)


@pytest.mark.parametrize("bw", [256, 128])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)], ids=["walls", "open"])
def test_fp32_ragged_multi_tile_per_step(gpu, orc, bc, bw):
    """FP32 state, element by element against the FP64 oracle one step at a
    time from the same inputs, on a 333 x 271 grid (2 x 9 blocks of 248 x 32,
    or 3 x 9 of 120 x 32 -- the kernels compiled for three and for six blocks
    per SM -- with ragged right and bottom edges), walls or open sides: the
    per-step FP32 bound of the full-size test (4e-5 m on H and b, 4e-5 m^2/s +
    2e-5 |Hu| on momenta)."""
    nx, ny = 333, 271
    side = max(nx, ny)
    base = I.ensemble_scenario(side, seed=48, manning=0.035, peak=300.0, d50_scale=1.0)
    H, b = base.H[:ny, :nx].astype(np.float64), base.b[:ny, :nx].astype(np.float64)
    Hu, Hv = 0.5 * H, -0.3 * H          # a drift across every side, so the boundaries matter
    sides = dict(bc_w=bc[0], bc_e=bc[1], bc_s=bc[2], bc_n=bc[3])
    S = gpu.Solver(nx, ny, base.dx, precision="fp32", block_cols=bw, tile_rows=32, **sides)
    S.set_manning(np.full((ny, nx), 0.035), block=0)
    S.set_state(H, Hu, Hv, b)
    p = orc.Params(nx=nx, ny=ny, dx=base.dx, **sides)
    ncell = np.full((ny, nx), 0.035)
    worst = np.zeros(4)
    outflow = 0.0
    for it in range(25):
        st = orc.State(*S.get_state(np.float32))
        st = orc.State(*(a.astype(np.float64) for a in st.arrays()))
        o, info = orc.step(p, st, ncell)
        outs = [o.arrays()] + [orc.step(pp, st, ncell)[0].arrays() for pp in band_params(p)[1:]]
        outflow += info.outflow_vol
        dt = S.step()
        assert dt == pytest.approx(info.dt, rel=1e-5), it
        got = S.get_state(np.float32)
        for q in range(4):
            excess, e = band_error(got[q], outs, q)
            worst[q] = max(worst[q], e.max())
            assert np.all(excess <= 0), (it, q, e.max(), int((excess > 0).sum()))
    S.close()
    assert (outflow != 0.0) if bc[0] else (outflow == 0.0)   # water crosses open sides (both ways)
    print("fp32 ragged per-step", bc, "worst abs err (H, Hu, Hv, b):", worst, "outflow m^3:", outflow)


@pytest.mark.parametrize("bw", [256, 128])
@pytest.mark.parametrize("variant", ["inflow", "rain_infiltration", "general_laws"])
def test_fp32_kernel_variants_per_step(gpu, orc, variant, bw):
    """The FP32 step kernel's other compiled variants, element by element
    against the FP64 oracle one step at a time from the same inputs on the
    ragged 333 x 271 grid, in 256- and 128-column blocks: inflow cells with a
    hydrograph (the source-term variant), rain and infiltration fields on
    top, and the general transport laws (A_J from Eq. 4, m = 2.5).  Same
    per-step FP32 bound as above."""
    nx, ny = 333, 271
    base = I.ensemble_scenario(max(nx, ny), seed=52, manning=0.035, peak=300.0, d50_scale=1.0)
    H, b = base.H[:ny, :nx].astype(np.float64), base.b[:ny, :nx].astype(np.float64)
    Hu, Hv = 0.4 * H, -0.2 * H
    kw = dict(A_J=0.01)
    src = rain = beta = hydro = None
    if variant in ("inflow", "rain_infiltration"):
        src = np.ascontiguousarray(base.src[:ny, :nx])
        assert src.sum() > 0
        hydro = orc.Hydrograph(base.hydro_t, base.hydro_Q)
    if variant == "rain_infiltration":
        rng = np.random.default_rng(52)
        rain = rng.uniform(0.0, 2e-3, (ny, nx))
        beta = rng.uniform(0.0, 1e-3, (ny, nx))
    if variant == "general_laws":
        kw.update(aj_mode=1, m_exp=2.5)
    S = gpu.Solver(nx, ny, base.dx, precision="fp32", block_cols=bw, tile_rows=32, **kw)
    S.set_manning(np.full((ny, nx), 0.035), block=0)
    if src is not None:
        S.set_sources(src, base.hydro_t, base.hydro_Q)
    S.set_state(H, Hu, Hv, b)
    if rain is not None:
        S.set_rain(rain)
        S.set_infiltration(beta)
    p = orc.Params(nx=nx, ny=ny, dx=base.dx, **kw)
    ncell = np.full((ny, nx), 0.035)
    worst = np.zeros(4)
    for it in range(20):
        t = S.diag()["t"]
        st = orc.State(*(a.astype(np.float64) for a in S.get_state(np.float32)))
        kw_o = dict(src=src, hydro=hydro, t=t, rain=rain, beta=beta)
        o, info = orc.step(p, st, ncell, **kw_o)
        outs = [o.arrays()] + [orc.step(pp, st, ncell, **kw_o)[0].arrays() for pp in band_params(p)[1:]]
        dt = S.step()
        assert dt == pytest.approx(info.dt, rel=1e-5), it
        got = S.get_state(np.float32)
        for q in range(4):
            excess, e = band_error(got[q], outs, q)
            worst[q] = max(worst[q], e.max())
            if np.any(excess > 0):
                bad = np.argwhere(excess > 0)[0]
                ex = [np.abs(got[q][tuple(bad)] - oo[q][tuple(bad)]) for oo in outs]
                print("variant", variant, "step", it, "q", q, "cell", bad, "err vs threshold/band edges", ex,
                      "H", outs[0][0][tuple(bad)], "b0", st.b[tuple(bad)])
            assert np.all(excess <= 0), (it, q, e.max(), int((excess > 0).sum()))
    S.close()
    print("fp32 variant", variant, "worst abs err (H, Hu, Hv, b):", worst)


def test_fp32_tall_strips_per_step(gpu, orc):
    """The benchmark's block shape (128 threads, 120 x 256 cells, six blocks
    per SM) on a 610 x 530 grid with inflow: 6 column bands (the last 10
    columns wide) x 3 strips (the last 18 rows high), so most sweep positions
    run the copy without row-range tests, and the strip ends, the grid's
    bottom ghost rows and the ragged band all occur.  FP32 state element by
    element against the FP64 oracle one step at a time from the same inputs,
    within the per-step FP32 bound of the ragged-grid tests."""
    nx, ny = 610, 530
    base = I.ensemble_scenario(max(nx, ny), seed=57, manning=0.035, peak=400.0, d50_scale=1.0)
    H, b = base.H[:ny, :nx].astype(np.float64), base.b[:ny, :nx].astype(np.float64)
    Hu, Hv = 0.6 * H, 0.35 * H
    src = np.ascontiguousarray(base.src[:ny, :nx])
    assert src.sum() > 0
    kw = dict(A_J=0.01)
    S = gpu.Solver(nx, ny, base.dx, precision="fp32", block_cols=128, tile_rows=256, **kw)
    S.set_manning(np.full((ny, nx), 0.03), block=0)
    S.set_sources(src, base.hydro_t, base.hydro_Q)
    S.set_state(H, Hu, Hv, b)
    assert S.tile == (120, 256)
    p = orc.Params(nx=nx, ny=ny, dx=base.dx, **kw)
    ncell = np.full((ny, nx), 0.03)
    hydro = orc.Hydrograph(base.hydro_t, base.hydro_Q)
    worst = np.zeros(4)
    moved = 0.0
    for it in range(10):
        t = S.diag()["t"]
        st = orc.State(*(a.astype(np.float64) for a in S.get_state(np.float32)))
        o, info = orc.step(p, st, ncell, src=src, hydro=hydro, t=t)
        outs = [o.arrays()] + [orc.step(pp, st, ncell, src=src, hydro=hydro, t=t)[0].arrays()
                               for pp in band_params(p)[1:]]
        dt = S.step()
        assert dt == pytest.approx(info.dt, rel=1e-5), it
        got = S.get_state(np.float32)
        moved = max(moved, np.abs(o.b - st.b).max())
        for q in range(4):
            excess, e = band_error(got[q], outs, q)
            worst[q] = max(worst[q], e.max())
            assert np.all(excess <= 0), (it, q, e.max(), int((excess > 0).sum()))
    S.close()
    assert moved > 1e-7   # the Exner update is exercised
    print("fp32 tall strips worst abs err (H, Hu, Hv, b):", worst)


@pytest.mark.parametrize("shape", [(1, 9), (9, 1), (3, 5), (130, 3)])
@pytest.mark.parametrize("bc", [(1, 0, 0, 1), (0, 1, 1, 0), (1, 1, 1, 1)], ids=["open_wn", "open_es", "open_all"])
def test_fp64_parity_tiny_grids_open_boundaries(gpu, orc, shape, bc):
    """Grids narrower than the stencil with open and wall sides mixed: the
    ghost rule (mirror at walls, repeat at open sides, composed across both
    ends) must agree with the oracle's."""
    ny, nx = shape
    g = I.rng(33)
    H = 1.0 + g.uniform(0, 0.5, (ny, nx))
    Hu = g.normal(0, 0.3, (ny, nx))
    Hv = g.normal(0, 0.3, (ny, nx))
    b = g.uniform(-0.05, 0.05, (ny, nx))
    sc = I.Scenario(nx, ny, 1.0, H, Hu, Hv, b, np.full((1, 1), 0.03), manning_block=256)
    _per_step_parity(gpu, orc, sc, 20, bw=128, th=32, A_J=0.05,
                     bc_w=bc[0], bc_e=bc[1], bc_s=bc[2], bc_n=bc[3])


def test_fp64_advance_lands_on_t_end(gpu, orc):
    sc = I.dam_break(64, 48, x_dam=30, seed=3)
    S = _fp64_solver(gpu, sc, bw=128, th=16)
    n = S.advance(2.5)
    assert S.t == 2.5
    g = S.get_state()
    p = orc.Params(nx=64, ny=48, dx=1.0)
    st, t, infos = orc.run(p, orc.State(sc.H, sc.Hu, sc.Hv, sc.b), 0.03, 10000, t_end=2.5)
    assert t == 2.5 and len(infos) == n
    err = _rel_linf(g, st.arrays(), st.H)
    assert max(err) < 1e-10, err


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hgs_skip_is_bit_exact_on_gpu(gpu, precision):
    """Skipping dry blocks (and not even copying blocks dry twice in a row)
    gives bit-identical states to computing every block."""
    sc = I.flood_channel(512, dx=5.0, seed=2, peak=500.0)
    res = []
    for hgs in (1, 0):
        S = gpu.Solver(512, 512, 5.0, precision=precision, hgs_skip=hgs, tile_rows=32)
        S.set_manning(sc.manning, block=64)
        S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
        S.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
        S.run_steps(400)
        S.sync()
        res.append((S.get_state(np.float64), S.diag()))
        S.close()
    (a, da), (b, db) = res
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert da["t"] == db["t"]
    assert da["active_tiles"] < da["total_tiles"]
    assert da["wet_cells"] > 0


def test_fp32_flood_channel_2048_full_run(gpu):
    """The 2048^2 flood channel: FP32 state vs the FP64 oracle after 10^4 steps, at the
    oracle's final time: relative L1 <= 1e-4 on H and b.  The oracle's final
    state is stored by tests/golden/make_flood2048_reference.py (oracle only)."""
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "flood2048_oracle.npz"))
    sc = I.flood_channel(2048, dx=5.0, seed=2, peak=500.0)
    assert sc.b.sum() == pytest.approx(float(ref["b0_sum"]), rel=1e-12)
    assert sc.manning.sum() == pytest.approx(float(ref["n_sum"]), rel=1e-12)
    t_ref = float(ref["t"])
    S = gpu.Solver(2048, 2048, 5.0, precision="fp32")
    S.set_manning(sc.manning, block=64)
    S.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
    S.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
    n_gpu = S.advance(t_ref)
    g = S.get_state()
    d = S.diag()
    H_ref = ref["H"]
    b_ref = sc.b + ref["db"]
    relH = np.abs(g[0] - H_ref).sum() / np.abs(H_ref).sum()
    relb = np.abs(g[3] - b_ref).sum() / np.abs(b_ref).sum()
    db_o = ref["db"]
    rel_db = np.abs((g[3] - sc.b) - db_o).sum() / max(np.abs(db_o).sum(), 1e-30)
    print(f"flood 2048^2: steps gpu {n_gpu} oracle {int(ref['steps'])} t={t_ref:.3f} relL1 H {relH:.3e} "
          f"b {relb:.3e} bed-change {rel_db:.3e} wet {(H_ref > 1e-4).sum()} "
          f"vol gpu {d['water_volume']:.6e} oracle {H_ref.sum() * 25.0:.6e} inflow gpu {d['inflow_volume']:.6e} "
          f"oracle {float(ref['inflow']):.6e}")
    assert abs(n_gpu - int(ref["steps"])) <= 2
    assert relH <= 1e-4 and relb <= 1e-4
    # The bed change carries the Exner physics (relative L1 of b is dominated
    # by the 0-20 m terrain and cannot see it).  Its bound: the Grass load is
    # cubic in the velocity, so its relative error is ~3x that of the water
    # state (bounded by 1e-4 above); 5e-4 also covers the few cells whose
    # Shamov gate switches one step apart.  A wrong Exner term gives O(1).
    assert rel_db <= 5e-4, rel_db
    S.close()


def test_fp32_full_size_step_sampled(gpu, orc):
    """16384^2 half-wet fractal terrain in the benchmark's launch
    configuration: one FP32 step, compared on sampled windows (interior,
    corners, edges, wet/dry fronts) with the oracle evaluated window by window
    at the oracle's own dt."""
    n = int(os.environ.get("SWE_FULL_N", "16384"))
    sc = I.half_wet(n, dx=5.0, seed=3)
    S = gpu.Solver(n, n, 5.0, precision="fp32")
    S.set_manning(sc.manning, block=64)
    S.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
    dt_gpu = S.step()
    g = S.get_state(np.float32)
    S.close()
    H = sc.H.astype(np.float64)
    b = sc.b.astype(np.float64)
    Z = np.zeros_like(H)
    st = orc.State(H, Z, Z.copy(), b)
    ncell = np.ascontiguousarray(sc.manning_per_cell(), dtype=np.float64)
    p = orc.Params(nx=n, ny=n, dx=5.0)
    dt_o, _ = orc.dt_from_terms(p, *orc.dt_terms(p, st, ncell))
    assert dt_gpu == pytest.approx(dt_o, rel=1e-6)
    rng = I.rng(99)
    w = 24
    wet = H > 1e-4
    front = np.argwhere(wet[1:-1, 1:-1] != wet[2:, 1:-1])
    picks = [(0, 0), (0, n - w), (n - w, 0), (n - w, n - w), (n // 2 - w // 2, 0), (0, n // 2 - w // 2)]
    picks += [tuple(rng.integers(0, n - w, 2)) for _ in range(8)]
    picks += [tuple(np.clip(front[i] - w // 2, 0, n - w)) for i in rng.integers(0, len(front), 8)]
    worst = np.zeros(4)
    for (y0, x0) in picks:
        y0, x0 = int(y0), int(x0)
        outs = []
        for pp in band_params(p):
            out, bad = orc.step_rect(pp, st, ncell, dt_o, (x0, y0, x0 + w, y0 + w))
            assert bad == 0
            outs.append(out)
        for q in range(4):
            excess, e = band_error(g[q][y0:y0 + w, x0:x0 + w], outs, q)
            worst[q] = max(worst[q], e.max())
            assert np.all(excess <= 0), (q, (y0, x0), e.max())
    print("full-size sampled worst abs err (H, Hu, Hv, b):", worst)


def test_error_paths(gpu):
    """Out-of-order calls, bad arguments and a host-injected NaN are reported
    as status codes, and the handle stays usable."""
    S = gpu.Solver(32, 32, 1.0, precision="fp32")
    with pytest.raises(gpu.SweError) as e:
        S.step()
    assert e.value.status == gpu.SWE_ESTATE
    with pytest.raises(gpu.SweError) as e:
        S.set_manning(np.full(4, -1.0), block=16)
    assert e.value.status == gpu.SWE_EINVAL
    H = np.ones((32, 32))
    H[5, 7] = np.nan
    Z = np.zeros_like(H)
    with pytest.raises(gpu.SweError) as e:
        S.set_state(H, Z, Z, Z)
        S.step()
    assert e.value.status == gpu.SWE_ENUMERIC
    H[5, 7] = 1.0
    S.set_state(H, Z, Z, Z)   # a fresh state clears the status
    S.step()
    S.close()


def test_autotune_restores_the_state_and_changes_no_result(gpu):
    """swe_autotune times block shapes on the current state, keeps the
    fastest and restores state and time exactly; the steps after it equal,
    bit for bit, those of a solver with the default shape (results do not
    depend on the block shape)."""
    sc = I.half_wet(640, dx=5.0, seed=5, wet_fraction=0.5)
    args = [np.ascontiguousarray(a, dtype=np.float32) for a in (sc.H, sc.Hu, sc.Hv, sc.b)]

    def solver():
        S = gpu.Solver(640, 640, 5.0, precision="fp32")
        S.set_manning(sc.manning, block=64)
        S.set_state(*args)
        S.run_steps(3)
        S.sync()
        return S

    A = solver()
    before = A.get_state(np.float32)
    t_before = A.diag()["t"]
    bw, th = A.autotune(3)
    assert bw in (128, 256) and th % 8 == 0 and 16 <= th <= 256
    assert A.tile == (bw - 8, th)
    for a, r in zip(A.get_state(np.float32), before):
        assert np.array_equal(a, r)
    assert A.diag()["t"] == t_before
    A.run_steps(20)
    B = solver()
    B.run_steps(20)
    for a, r in zip(A.get_state(np.float32), B.get_state(np.float32)):
        assert np.array_equal(a, r)
    A.close()
    B.close()


def _sparse_grid():
    import torch
    return 2 * torch.cuda.get_device_properties(0).multi_processor_count


def test_fp64_parity_sparse_lake_region_level(gpu, orc):
    """HGS region level and the sparse launch (Sec. 3, Fig. 2: regions of 8 x 8
    blocks above the blocks): a lake spreading over mostly dry terrain,
    1024 x 2048 cells in blocks of 120 x 16 (9 x 128 blocks, 2 x 16 regions),
    the lake straddling the corner of four regions.  After the first step only
    a few blocks are active, so the steps launch one wave of CUDA blocks that
    walk the block list found by the region-level compaction.  Per step: FP64
    parity (1e-11) with the oracle and the block census bit-exact, every block
    included (blocks never examined keep census 0)."""
    sc = I.sparse_lake(1024, 2048)
    S = _fp64_solver(gpu, sc, bw=128, th=16)
    d = S.diag()
    assert d["total_tiles"] > _sparse_grid()
    S.close()
    worst = _per_step_parity(gpu, orc, sc, 12, bw=128, th=16)
    assert np.all(worst <= 1e-11)
    # the same steps run sparse: few blocks active
    S = _fp64_solver(gpu, sc, bw=128, th=16)
    for _ in range(3):
        S.step()
    d = S.diag()
    assert 0 < d["active_tiles"] <= _sparse_grid(), d
    S.close()


def test_sparse_launch_and_regions_are_bit_exact_against_no_skip(gpu):
    """FP32, 240 steps of the sparse lake through the step graphs (the launch
    picked from the last replay's active-block count: sparse here) with the
    dry-block skip on, against the same steps with it off: bit-identical
    states and times."""
    sc = I.sparse_lake(1024, 2048)
    res = []
    for hgs in (1, 0):
        S = gpu.Solver(sc.nx, sc.ny, sc.dx, precision="fp32", hgs_skip=hgs, block_cols=128, tile_rows=16)
        S.set_manning(sc.manning, block=0)
        S.set_state(sc.H, sc.Hu, sc.Hv, sc.b)
        for _ in range(8):
            S.run_steps(30)
        S.sync()
        res.append((S.get_state(np.float32), S.diag()))
        S.close()
    (a, da), (b, db) = res
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert da["t"] == db["t"]
    assert 0 < da["active_tiles"] <= _sparse_grid()
    assert da["cells_computed"] < db["cells_computed"] / 10
