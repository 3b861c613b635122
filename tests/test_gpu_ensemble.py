"""Batched ensembles (one persistent launch advancing many scenarios): each
scenario must evolve bit for bit as it does alone, the autotuner must keep
that true, and the launch's bounded grid barrier must give up cleanly."""
import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I

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


def test_ensemble_matches_standalone_runs(swe):
    scs = _scenarios()
    E = swe.Ensemble([_spec(s) for s in scs], block_cols=256, tile_rows=32)
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    E.run(120)
    for k, (m, sc) in enumerate(zip(E.members, scs)):
        got, t = m.get_state(np.float32), m.t
        ref, t_ref = _standalone(swe, sc, 120, 256, 32)
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
    assert bw in (128, 256) and th in (16, 32, 64, 128)
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


def test_ensemble_barrier_gives_up_with_a_status(swe):
    """The barrier is made to wait for one block that does not exist: every
    block stops after the time limit, the host reads SWE_ETIMEOUT, and the
    ensemble works again once the limit is back to normal."""
    scs = _scenarios()[:3]
    E = swe.Ensemble([_spec(s) for s in scs], block_cols=256, tile_rows=32)
    for m, sc in zip(E.members, scs):
        _load(m, sc)
    E.set_timeout(0.2, extra_arrivals=1)
    with pytest.raises(swe.SweError) as e:
        E.run(1)
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
