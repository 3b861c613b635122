"""Batched ensembles (one persistent launch advancing many scenarios, work
scheduled by dataflow): each scenario must evolve bit for bit as it does
alone, the autotuner must keep that true, the members must match the oracle
step by step, and the launch's bounded waits must give up cleanly."""
import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I
from fp32_band import band_error, band_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe as S
    S.load_library()
    return S


SIDES = [64, 200, 256, 128, 96, 312]


def _scenarios():
    out = []
    g = I.rng(77)
    for k, side in enumerate(SIDES):
        sc = I.ensemble_scenario(side, seed=500 + k, manning=float(g.uniform(0.02, 0.06)),
                                 peak=float(g.uniform(50, 1000)), d50_scale=float(g.uniform(0.5, 2.0)))
        out.append(sc)
    return out


def _spec(sc):
    return dict(nx=sc.nx, ny=sc.ny, dx=sc.dx, d50=sc.d50)


def _load(m, sc):
    m.set_manning(sc.manning, block=sc.manning_block)
    m.set_sources(sc.src, sc.hydro_t, sc.hydro_Q)
    m.set_state(sc.H, sc.Hu, sc.Hv, sc.b)


def _standalone(swe, sc, nsteps, bw, th):
    S = swe.Solver(sc.nx, sc.ny, sc.dx, precision="fp32", block_cols=bw, tile_rows=th, d50=sc.d50)
    _load(S, sc)
    S.run_steps(nsteps)
    S.sync()
    out = S.get_state(np.float32), S.t
    S.close()
    return out


@pytest.mark.parametrize("bw", [256, 128])
def test_ensemble_matches_standalone_runs(swe, bw):
    """Every member after 120 steps of one persistent launch equals the same
    scenario run alone, bit for bit, in 256- and 128-thread blocks (the
    latter six per SM); blocks take items of other scenarios whenever their
    own scenario's next item would wait, which must not change any result."""
    scs = _scenarios()
    E = swe.Ensemble([_spec(s) for s in scs], block_cols=bw, tile_rows=32)
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    E.run(120)
    for k, (m, sc) in enumerate(zip(E.members, scs)):
        got, t = m.get_state(np.float32), m.t
        ref, t_ref = _standalone(swe, sc, 120, bw, 32)
        assert t == t_ref, k
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), k
        d = m.diag()
        assert d["steps"] == 120 and d["status"] == 0
    E.close()


def test_ensemble_autotune_keeps_results(swe):
    scs = _scenarios()
    E = swe.Ensemble([_spec(s) for s in scs])
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    bw, th = E.autotune(4)
    assert bw in (128, 256) and th in (16, 32, 64, 96, 128, 192, 256)
    for m in E.members:
        assert m.t == 0.0
    E.run(40)
    for k, (m, sc) in enumerate(zip(E.members, scs)):
        ref, t_ref = _standalone(swe, sc, 40, bw, th)
        got = m.get_state(np.float32)
        assert m.t == t_ref
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), k
    E.close()


def test_ensemble_wait_gives_up_with_a_status(swe):
    """Every scenario step is made to wait for one work item that does not
    exist: every block stops after the time limit, the host reads
    SWE_ETIMEOUT, and the ensemble works again once the limit is back to
    normal."""
    scs = _scenarios()[:3]
    E = swe.Ensemble([_spec(s) for s in scs], block_cols=256, tile_rows=32)
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    E.set_timeout(0.2, extra_arrivals=1)
    with pytest.raises(swe.SweError) as e:
        E.run(3)   # the second step's items wait for the first step, which never completes
    assert e.value.status == swe.SWE_ETIMEOUT
    E.set_timeout(2.0, 0)
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    E.run(10)
    for k, (m, sc) in enumerate(zip(E.members, scs)):
        ref, _ = _standalone(swe, sc, 10, 256, 32)
        for a, b in zip(m.get_state(np.float32), ref):
            assert np.array_equal(a, b), k
    E.close()


def test_ensemble_members_match_the_oracle_per_step(swe, orc):
    """Each member of one persistent ensemble launch against the FP64 oracle,
    one step at a time from the member's own FP32 state, element by element,
    within the per-step FP32 bound of the single-grid parity tests (4e-5 m on
    H and b, 4e-5 m^2/s + 2e-5 |Hu| on momenta; the oracle at the Shamov
    threshold or at the edges of its FP32 decision band); dt (Eq. 7) per member.
    Members of uneven size: a ragged 333 x 271 grid with inflow (2 x 9 blocks
    of 248 x 32, ragged right and bottom), a 200 x 200 grid without sources,
    a tall 96 x 312 grid with inflow, a 64 x 64 grid; every one drifts so the
    Grass load (Eq. 3) and the Exner update run."""
    shapes = [(333, 271, True, (0.8, -0.3)), (200, 200, False, (-0.6, 0.7)), (96, 312, True, (0.3, 0.9)),
              (64, 64, False, (0.9, 0.2))]
    members = []
    for k, (nx, ny, inflow, (ux, uy)) in enumerate(shapes):
        base = I.ensemble_scenario(max(nx, ny), seed=610 + k, manning=0.03 + 0.005 * k, peak=400.0,
                                   d50_scale=0.7 + 0.2 * k)
        H = np.ascontiguousarray(base.H[:ny, :nx], dtype=np.float64)
        b = np.ascontiguousarray(base.b[:ny, :nx], dtype=np.float64)
        src = None
        if inflow:
            src = np.ascontiguousarray(base.src[:ny, :nx])
            assert src.sum() > 0
        members.append(dict(nx=nx, ny=ny, dx=base.dx, d50=base.d50, n=0.03 + 0.005 * k, H=H, Hu=ux * H,
                            Hv=uy * H, b=b, src=src, ht=base.hydro_t, hq=base.hydro_Q))
    E = swe.Ensemble([dict(nx=m["nx"], ny=m["ny"], dx=m["dx"], d50=m["d50"], A_J=0.01) for m in members],
                     block_cols=256, tile_rows=32)
    for h, m in zip(E.members, members):
        h.set_manning(np.full((m["ny"], m["nx"]), m["n"]), block=0)
        if m["src"] is not None:
            h.set_sources(m["src"], m["ht"], m["hq"])
        h.set_state(m["H"], m["Hu"], m["Hv"], m["b"])
    worst = np.zeros((len(members), 4))
    moved = np.zeros(len(members))
    for it in range(12):
        before = [(orc.State(*(a.astype(np.float64) for a in h.get_state(np.float32))), h.t) for h in E.members]
        E.run(1)
        for k, (h, m) in enumerate(zip(E.members, members)):
            st, t = before[k]
            p = orc.Params(nx=m["nx"], ny=m["ny"], dx=m["dx"], d50=m["d50"], A_J=0.01)
            hydro = orc.Hydrograph(m["ht"], m["hq"]) if m["src"] is not None else None
            ncell = np.full((m["ny"], m["nx"]), m["n"])
            o, info = orc.step(p, st, ncell, src=m["src"], hydro=hydro, t=t)
            outs = [o.arrays()] + [orc.step(pp, st, ncell, src=m["src"], hydro=hydro, t=t)[0].arrays()
                                   for pp in band_params(p)[1:]]
            assert h.t - t == pytest.approx(info.dt, rel=1e-5), (it, k)
            got = h.get_state(np.float32)
            moved[k] = max(moved[k], np.abs(o.b - st.b).max())
            for q in range(4):
                excess, e = band_error(got[q], outs, q)
                worst[k, q] = max(worst[k, q], e.max())
                assert np.all(excess <= 0), (it, k, q, e.max())
    E.close()
    assert np.all(moved > 1e-7), moved   # the bed moves in every member
    print("ensemble vs oracle, worst abs err per member (H, Hu, Hv, b):", worst.tolist())
