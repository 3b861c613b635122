"""The library's checked variant (built with -DSWE_CHECKED): every global
index of the step kernel (state loads and stores, Manning tables, source
lists, rain and infiltration fields, census, work list, copied blocks) is
tested against its buffer, and an index outside sets device status bit 8 and
skips the access.  Step-kernel cases with tiny, thin and ragged grids, open
and wall sides, every source term and both transport laws run on it without
a single index outside, and give the production build's results bit for
bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_15196_gb300 import swe
    swe.load_library(checked=True)
    return swe


def _case(nx, ny, seed, open_sides=(0, 0, 0, 0)):
    rng = np.random.default_rng(seed)
    b = rng.uniform(0.0, 0.6, (ny, nx))
    eta = 0.8 + 0.4 * (np.arange(nx)[None, :] < nx // 2)
    H = np.maximum(eta - b, 0.0)
    H[rng.random((ny, nx)) < 0.15] = 0.0           # dry patches: wet/dry fronts everywhere
    wet = H > 1e-4
    Hu = np.where(wet, H * rng.normal(0.0, 0.3, (ny, nx)), 0.0)
    Hv = np.where(wet, H * rng.normal(0.0, 0.3, (ny, nx)), 0.0)
    kw = dict(bc_w=open_sides[0], bc_e=open_sides[1], bc_s=open_sides[2], bc_n=open_sides[3], A_J=0.02)
    return (H, Hu, Hv, b), kw, rng


def _run(swe, precision, checked, nx, ny, state, kw, extras, nsteps, bw, th):
    S = swe.Solver(nx, ny, 1.0, precision=precision, checked=checked, block_cols=bw, tile_rows=th, **kw)
    S.set_manning(extras["manning"], block=extras["mblock"])
    if "src" in extras:
        S.set_sources(extras["src"], np.array([0.0, 1e6]), np.array([2.0, 2.0]))
    S.set_state(*state)
    if "rain" in extras:
        S.set_rain(extras["rain"])
    if "beta" in extras:
        S.set_infiltration(extras["beta"])
    S.run_steps(nsteps)
    S.sync()
    d = S.diag()
    out = S.get_state(np.float64)
    S.close()
    return out, d["status"]


CASES = [
    # nx, ny, precision, block columns, rows, open sides, extras
    (9, 1, "fp64", 128, 8, (0, 1, 0, 0), ()),
    (1, 9, "fp64", 128, 8, (0, 0, 1, 1), ()),
    (3, 5, "fp32", 128, 8, (1, 0, 0, 1), ()),
    (130, 3, "fp32", 128, 8, (1, 1, 0, 0), ("src",)),
    (333, 271, "fp32", 256, 32, (0, 1, 1, 0), ("src", "rain", "beta")),
    (333, 271, "fp32", 256, 32, (0, 0, 0, 0), ("src", "gen")),
    (300, 140, "fp64", 128, 16, (1, 0, 0, 1), ("src", "rain", "beta", "gen")),
]


@pytest.mark.parametrize("nx,ny,precision,bw,th,open_sides,what", CASES)
def test_checked_build_finds_no_index_outside(swe, nx, ny, precision, bw, th, open_sides, what):
    state, kw, rng = _case(nx, ny, seed=nx * 1000 + ny, open_sides=open_sides)
    extras = {"manning": rng.uniform(0.02, 0.05, ((ny + 7) // 8, (nx + 7) // 8)), "mblock": 8}
    if "src" in what:
        m = np.zeros((ny, nx), dtype=np.uint8)
        m[ny // 2, 0] = 1
        m[ny - 1, nx - 1] = 1
        extras["src"] = m
    if "rain" in what:
        extras["rain"] = rng.uniform(0.0, 1e-3, (ny, nx))
    if "beta" in what:
        extras["beta"] = rng.uniform(0.0, 5e-4, (ny, nx))
    if "gen" in what:
        kw = dict(kw, aj_mode=1, m_exp=2.5)
    ref, st_ref = _run(swe, precision, False, nx, ny, state, kw, extras, 12, bw, th)
    got, st = _run(swe, precision, True, nx, ny, state, kw, extras, 12, bw, th)
    assert st == 0 and st_ref == 0, (st, st_ref)
    for a, r in zip(got, ref):
        assert np.array_equal(a, r)


def test_checked_build_ensemble(swe):
    """The persistent ensemble kernel on the checked build: scenarios of
    different sizes (a 1-column one among them), inflow and walls/open
    sides, 10 steps; no index outside, members bit-identical to the
    production build's ensemble."""
    sizes = [(1, 40), (37, 23), (300, 140), (130, 3)]

    def run(checked):
        specs = [dict(nx=nx, ny=ny, dx=1.0, A_J=0.02, bc_e=k % 2) for k, (nx, ny) in enumerate(sizes)]
        E = swe.Ensemble(specs, checked=checked, block_cols=128, tile_rows=16)
        outs = []
        for k, (m, (nx, ny)) in enumerate(zip(E.members, sizes)):
            state, kw, rng = _case(nx, ny, seed=77 + k)
            m.set_manning(np.array([[0.03]]), block=1 << 14)
            src = np.zeros((ny, nx), dtype=np.uint8)
            src[ny // 2, 0] = 1
            m.set_sources(src, np.array([0.0, 1e6]), np.array([1.0, 1.0]))
            m.set_state(*state)
        E.run(10)
        for m in E.members:
            m.sync()
            outs.append((m.get_state(np.float64), m.diag()["status"]))
        E.close()
        return outs

    ref, got = run(False), run(True)
    for (a, st_a), (r, st_r) in zip(got, ref):
        assert st_a == 0 and st_r == 0, (st_a, st_r)
        for x, y in zip(a, r):
            assert np.array_equal(x, y)
