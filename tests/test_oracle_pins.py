"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself:
closed forms, analytic solutions, invariants, symmetries and textbook special
cases.  Each test names what would fail if the oracle had a dropped term, a
wrong sign or index, or a transposed operand.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2103_15196_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _state(O, H, Hu=None, Hv=None, b=None):
    z = np.zeros_like(H)
    return O.State(np.array(H, float), np.array(z if Hu is None else Hu, float),
                   np.array(z if Hv is None else Hv, float), np.array(z if b is None else b, float))


# ------------------------------------------------------------------ HLL / K7

def test_hll_textbook_identities(orc):
    """HLL (Harten-Lax-van Leer): upwind states when both bounds share a sign;
    consistency F(U, U) = F(U); for the advective problem with the two
    velocities as bounds, converging flow gives F_L + F_R and diverging flow
    with equal states gives zero."""
    h = orc.hll
    assert h(1.0, 2.0, 3.0, 5.0, 0.5, 2.0) == 3.0          # both bounds >= 0 -> F_L
    assert h(1.0, 2.0, 3.0, 5.0, -2.0, -0.5) == 5.0        # both bounds <= 0 -> F_R
    assert h(1.5, 1.5, 0.7, 0.7, -3.0, 2.0) == pytest.approx(0.7, abs=1e-15)
    H, uL, uR = 1.3, 0.8, -0.5                             # converging
    assert h(H, H, H * uL, H * uR, uR, uL) == pytest.approx(H * uL + H * uR, abs=1e-15)
    uL, uR = -0.4, 0.9                                     # diverging
    assert h(H, H, H * uL, H * uR, uL, uR) == pytest.approx(0.0, abs=1e-15)
    # the generic formula against a worked value: sL=-1, sR=2, FL=1, FR=4, UL=0, UR=3
    # (2*1 - (-1)*4 + (-1*2)*(3-0)) / 3 = (2 + 4 - 6)/3 = 0
    assert h(0.0, 3.0, 1.0, 4.0, -1.0, 2.0) == pytest.approx(0.0, abs=1e-15)


def test_minmod_is_the_median_with_zero(orc):
    """The limiter of the K7 reconstruction: minmod(a, b) is 0 when the two
    slopes differ in sign (or one is 0) and the one of smaller magnitude
    otherwise; equivalently the median of (a, b, 0).  Checked on the
    textbook cases and against that characterisation on random pairs
    spanning signs, ties and magnitudes."""
    m = orc.minmod
    assert m(1.0, 2.0) == 1.0 and m(2.0, 1.0) == 1.0
    assert m(-1.0, -2.0) == -1.0 and m(-2.0, -1.0) == -1.0
    assert m(1.0, -2.0) == 0.0 and m(-1.0, 2.0) == 0.0
    assert m(0.0, 3.0) == 0.0 and m(3.0, 0.0) == 0.0
    assert m(0.75, 0.75) == 0.75 and m(-0.75, -0.75) == -0.75
    rng = np.random.default_rng(17)
    a = rng.normal(size=2000) * 10.0 ** rng.integers(-6, 4, size=2000)
    b = rng.normal(size=2000) * 10.0 ** rng.integers(-6, 4, size=2000)
    b[::7] = a[::7]
    b[::11] = -a[::11]
    for x, y in zip(a, b):
        assert m(x, y) == float(np.median([x, y, 0.0]))


def test_hydrograph_integral_closed_form(orc):
    """Area under the triangular hydrograph 0 -> 500 (t=1200) -> 0 (t=3600)."""
    hg = orc.Hydrograph([0.0, 1200.0, 3600.0], [0.0, 500.0, 0.0])
    assert hg.integral(0.0, 3600.0) == pytest.approx(0.5 * 3600 * 500, rel=1e-15)
    assert hg.integral(0.0, 600.0) == pytest.approx(0.5 * 600 * 250, rel=1e-15)
    # straddling the peak: 1000..1500 -> trapezoids 1000..1200 and 1200..1500
    q1000, q1500 = 500 * 1000 / 1200, 500 * (3600 - 1500) / 2400
    exp = 0.5 * (q1000 + 500) * 200 + 0.5 * (500 + q1500) * 300
    assert hg.integral(1000.0, 1500.0) == pytest.approx(exp, rel=1e-14)
    assert hg.integral(3600.0, 4000.0) == 0.0


# ------------------------------------------------------------------ Eq. 7

def test_dt_golden_cases(orc):
    """Eq. 7 on uniform states whose three terms were evaluated by hand
    (tests/golden/dt_cases.json): which term binds, and the value."""
    with open(os.path.join(GOLDEN, "dt_cases.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        p = orc.Params(nx=4, ny=4, dx=c["dx"], cfl_K=c["K"], A_J=c["A_J"], C_J=c["C_J"],
                       psi=c["psi"], sediment_on=c["sediment_on"], dt_literal_D=c.get("literal_D", 0))
        H = np.full((4, 4), c["H"])
        st = _state(orc, H, H * c["u"], H * c["v"])
        vp, vs, jm = orc.dt_terms(p, st, 0.03)
        dt, which = orc.dt_from_terms(p, vp, vs, jm)
        assert which == c["binding"], c["name"]
        assert dt == pytest.approx(c["dt"], rel=1e-12), c["name"]


def test_dt_sediment_never_larger(orc):
    """The Exner term can only tighten the step (the paper's point at Eq. 7)."""
    g = I.rng(5)
    for _ in range(20):
        H = g.uniform(0.0, 3.0, (8, 8))
        st = _state(orc, H, H * g.normal(0, 2, (8, 8)), H * g.normal(0, 2, (8, 8)))
        pa = orc.Params(nx=8, ny=8, A_J=0.05)
        pb = orc.Params(nx=8, ny=8, A_J=0.05, sediment_on=0)
        dta, _ = orc.dt_from_terms(pa, *orc.dt_terms(pa, st, 0.03))
        dtb, _ = orc.dt_from_terms(pb, *orc.dt_terms(pb, st, 0.03))
        assert dta <= dtb


# ----------------------------------------------------------- invariants

def test_lake_at_rest_noisy_bed(orc):
    """A flat free surface over the +-1 cm noisy bed stays at rest to roundoff
    (forces K2/K5 and the hydrostatic HLL in K7 must cancel exactly)."""
    sc = I.dam_break(64, 64, noise=0.01, seed=1)
    H = 2.0 - sc.b
    st0 = _state(orc, H, b=sc.b)
    p = orc.Params(nx=64, ny=64, dx=1.0)
    st, t, infos = orc.run(p, st0, 0.03, 400)
    assert np.abs(st.H + st.b - 2.0).max() < 1e-13
    assert np.abs(st.Hu).max() < 1e-13 and np.abs(st.Hv).max() < 1e-13
    assert np.array_equal(st.b, sc.b)


def test_lake_at_rest_partially_dry(orc):
    """Fractal terrain filled to its median level: half the cells dry, with
    dry cells above the water line acting as walls; nothing moves."""
    n = 64
    b = I.fractal_dem(n, n, seed=7, relief=10.0)
    eta = float(np.median(b))
    H = np.maximum(eta - b, 0.0)
    st0 = _state(orc, H, b=b)
    p = orc.Params(nx=n, ny=n, dx=5.0, tile_x=16, tile_y=16)
    st, t, infos = orc.run(p, st0, 0.04, 300)
    wet = H > 1e-4
    assert 0.3 < wet.mean() < 0.7
    assert np.abs(st.H - H).max() < 1e-12
    assert np.abs(st.Hu).max() < 1e-13 and np.abs(st.Hv).max() < 1e-13
    assert np.array_equal(st.b, b)


def test_conservation_walls(orc):
    """Water and sediment volume are conserved with walls and no sources
    (flux-form update of Eq. 6 rows 1 and 4, zero wall fluxes)."""
    sc = I.dam_break(128, 128, seed=1)
    st0 = _state(orc, sc.H, b=sc.b)
    p = orc.Params(nx=128, ny=128, dx=1.0, A_J=0.01)
    st, t, infos = orc.run(p, st0, 0.03, 300)
    assert abs(st.H.sum() - sc.H.sum()) / sc.H.sum() < 1e-13
    assert abs(st.b.sum() - sc.b.sum()) < 1e-13 * np.abs(sc.b).sum() + 1e-15 * sc.b.size
    assert np.abs(st.b - sc.b).max() > 1e-6        # the bed did move
    assert sum(i.n_bad for i in infos) == 0


def test_inflow_volume_budget(orc):
    """With an inflow hydrograph the water volume grows by exactly the integral
    of Q over the simulated time (sigma of Eq. 6 row 1)."""
    sc = I.flood_channel(64, dx=5.0, seed=2, peak=50.0)
    p = orc.Params(nx=64, ny=64, dx=5.0, tile_x=16, tile_y=16)
    st0 = _state(orc, sc.H, b=sc.b)
    hg = orc.Hydrograph(sc.hydro_t, sc.hydro_Q)
    st, t, infos = orc.run(p, st0, sc.manning_per_cell(), 400, src=sc.src, hydro=hg)
    vol = st.H.sum() * 25.0
    # closed form of the triangle area up to t (t < 1200 s: rising limb)
    assert t < 1200.0
    exact = 0.5 * t * (50.0 * t / 1200.0)
    assert vol == pytest.approx(exact, rel=1e-11)
    assert sum(i.inflow_vol for i in infos) == pytest.approx(exact, rel=1e-11)


# -------------------------------------------------------- symmetries

def _run_case(orc, st0, p, nsteps=40, n=0.03):
    st, t, infos = orc.run(p, st0, n, nsteps)
    return st


def test_mirror_symmetry_exact(orc):
    """Mirroring x (and negating Hu) mirrors the result bit for bit."""
    g = I.rng(11)
    n = 32
    b = g.uniform(-0.05, 0.05, (n, n))
    H = np.where(g.uniform(size=(n, n)) < 0.15, 0.0, 1.0 + g.uniform(0, 0.5, (n, n)))
    Hu = np.where(H > 0, g.normal(0, 0.5, (n, n)), 0.0)
    Hv = np.where(H > 0, g.normal(0, 0.5, (n, n)), 0.0)
    p = orc.Params(nx=n, ny=n, dx=1.0, A_J=0.01, tile_x=8, tile_y=8)
    a = _run_case(orc, _state(orc, H, Hu, Hv, b), p)
    m = _run_case(orc, _state(orc, H[:, ::-1], -Hu[:, ::-1], Hv[:, ::-1], b[:, ::-1]), p)
    assert np.array_equal(a.H, m.H[:, ::-1])
    assert np.array_equal(a.Hu, -m.Hu[:, ::-1])
    assert np.array_equal(a.Hv, m.Hv[:, ::-1])
    assert np.array_equal(a.b, m.b[:, ::-1])


def test_transpose_symmetry_exact(orc):
    """Swapping x and y (and Hu with Hv) transposes the result bit for bit."""
    g = I.rng(12)
    n = 32
    b = g.uniform(-0.05, 0.05, (n, n))
    H = np.where(g.uniform(size=(n, n)) < 0.15, 0.0, 1.0 + g.uniform(0, 0.5, (n, n)))
    Hu = np.where(H > 0, g.normal(0, 0.5, (n, n)), 0.0)
    Hv = np.where(H > 0, g.normal(0, 0.5, (n, n)), 0.0)
    p = orc.Params(nx=n, ny=n, dx=1.0, A_J=0.01, tile_x=8, tile_y=8)
    a = _run_case(orc, _state(orc, H, Hu, Hv, b), p)
    t = _run_case(orc, _state(orc, H.T, Hv.T, Hu.T, b.T), p)
    assert np.array_equal(a.H, t.H.T)
    assert np.array_equal(a.Hu, t.Hv.T)
    assert np.array_equal(a.Hv, t.Hu.T)
    assert np.array_equal(a.b, t.b.T)


def test_strip_rows_identical(orc):
    """A 1D problem on an N x 4 strip keeps its rows identical."""
    sc = I.dam_break(64, 4, x_dam=32, noise=0.0)
    p = orc.Params(nx=64, ny=4, dx=1.0, tile_x=16, tile_y=4)
    st, t, _ = orc.run(p, _state(orc, sc.H), 0.03, 60)
    assert np.array_equal(st.H, np.broadcast_to(st.H[0], st.H.shape))


# ----------------------------------------------------- analytic solutions

def _stoker(x, t, hL, hR, x0, g=9.81):
    """Textbook exact 1D dam break on a flat frictionless bed: rarefaction
    into the left state, a constant middle state (h_m, u_m) found by Newton on
    2(c_L - c_m) = (h_m - h_R) sqrt(g (h_m + h_R) / (2 h_m h_R)), and a shock
    with speed h_m u_m / (h_m - h_R); for h_R = 0 the Ritter solution."""
    cL = math.sqrt(g * hL)
    xi = (x - x0) / t
    if hR <= 0.0:
        h = np.where(xi < -cL, hL, np.where(xi < 2 * cL, (2 * cL - xi) ** 2 / (9 * g), 0.0))
        return h
    hm = 0.5 * (hL + hR)
    for _ in range(60):
        def f(h):
            return 2 * (cL - math.sqrt(g * h)) - (h - hR) * math.sqrt(g * (h + hR) / (2 * h * hR))
        d = (f(hm * (1 + 1e-8)) - f(hm)) / (hm * 1e-8)
        hm -= f(hm) / d
    cm = math.sqrt(g * hm)
    um = 2 * (cL - cm)
    s = hm * um / (hm - hR)
    return np.where(xi < -cL, hL, np.where(xi < um - cm, (2 * cL - xi) ** 2 / (9 * g),
                                           np.where(xi < s, hm, hR)))


@pytest.mark.parametrize("hR", [0.5, 0.0], ids=["stoker_wet_bed", "ritter_dry_bed"])
def test_dam_break_converges_to_analytic(orc, hR):
    """Relative L1 error of H against the exact dam break falls with
    refinement (rate >= 0.7, the shock-limited first order) and is below 2 %
    at N = 1024 (frictionless, sediment off, flat bed, t = 5 s)."""
    errs = []
    Ns = [128, 256, 512, 1024]
    for N in Ns:
        dx = 128.0 / N
        x = (np.arange(N) + 0.5) * dx
        H = np.where(x < 64.0, 2.0, hR) * np.ones((4, 1))
        p = orc.Params(nx=N, ny=4, dx=dx, sediment_on=0, tile_x=256, tile_y=4)
        st, t, _ = orc.run(p, _state(orc, H), 0.0, 100000, t_end=5.0)
        assert t == pytest.approx(5.0, abs=1e-12)
        he = _stoker(x, t, 2.0, hR, 64.0)
        errs.append(np.abs(st.H[0] - he).sum() / np.abs(he).sum())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.7), (errs, rates)
    assert errs[-1] < 0.02


def test_manning_friction_ode(orc):
    """Uniform flow on a flat bed decays by Manning friction alone:
    dv/dt = -g n^2 v|v| / H^(4/3), v(t) = v0 / (1 + c v0 t).  The point-implicit
    Lagrangian update must converge to it at first order in dt (K halved)."""
    v0, H0, nman, T = 1.5, 0.8, 0.05, 4.0
    c = 9.81 * nman ** 2 / H0 ** (4.0 / 3.0)
    errs = []
    for K in [0.4, 0.2, 0.1]:
        N = 2400
        H = np.full((1, N), H0)
        p = orc.Params(nx=N, ny=1, dx=1.0, cfl_K=K, sediment_on=0, tile_x=N, tile_y=1)
        st, t, _ = orc.run(p, _state(orc, H, H * v0), nman, 100000, t_end=T)
        v = st.Hu[0, N // 2] / st.H[0, N // 2]
        assert st.H[0, N // 2] == H0
        errs.append(abs(v - v0 / (1 + c * v0 * t)))
    assert errs[0] / errs[1] > 1.7 and errs[1] / errs[2] > 1.7, errs
    assert errs[2] / v0 < 2e-3


# ----------------------------------------------------- Exner (Eq. 1-5)

def _exner_decay_case(orc, v0, aj_mode=0, nman=0.03, H0=1.0, m_wave=3, nx=64, m_exp=2.0):
    """Frozen uniform flow along y on a 1-row grid, bed b = eps cos(k x):
    the x-direction Exner flux is pure slope diffusion C_J |J0| db/dx, so each
    Fourier mode decays by 1 - 4 (C_J |J0| dt / ((1-psi) h^2)) sin^2(k h / 2)."""
    dx = 2.0
    x = (np.arange(nx) + 0.5) * dx
    k = math.pi * m_wave / (nx * dx)
    b = 0.05 * np.cos(k * x)[None, :]
    H = np.full((1, nx), H0)
    st0 = _state(orc, H, 0 * H, H * v0, b)
    p = orc.Params(nx=nx, ny=1, dx=dx, frozen_hydro=1, aj_mode=aj_mode, A_J=0.002, m_exp=m_exp,
                   tile_x=nx, tile_y=1)
    st, info = orc.step(p, st0, nman)
    return p, st0, st, info, k


def test_exner_diffusion_mode_decay(orc):
    for aj_mode in (0, 1):
        v0, H0, nman = 1.2, 1.0, 0.03
        p, st0, st, info, k = _exner_decay_case(orc, v0, aj_mode=aj_mode, nman=nman, H0=H0)
        if aj_mode == 0:
            AJ = p.A_J                                                 # Eq. 3 constant
        else:
            AJ = 0.05 * nman ** 3 / ((p.s_rel - 1.0) * math.sqrt(p.g * H0) * p.d50)  # Eq. 4
        J0 = AJ * v0 ** 3                                              # Eq. 3, m = 2
        D = p.C_J * J0 / (1.0 - p.psi)
        r = 1.0 - 4.0 * D * info.dt / p.dx ** 2 * math.sin(k * p.dx / 2) ** 2
        assert np.allclose(st.b, r * st0.b, rtol=0, atol=1e-15), (aj_mode, r)
        assert r < 1.0 - 1e-6


@pytest.mark.parametrize("m", [1.5, 2.5, 3.0])
def test_exner_diffusion_mode_decay_grass_exponent(orc, m):
    """The Grass exponent m of Eq. 3 away from the default m = 2: a uniform
    speed v0 carries |J0| = A_J v0^(m+1), so the cosine bed mode decays by the
    closed-form factor with D = C_J A_J v0^(m+1) / (1 - psi).  dt itself is
    checked against Eq. 7 written out with that D."""
    v0, H0 = 1.7, 1.0
    p, st0, st, info, k = _exner_decay_case(orc, v0, H0=H0, m_exp=m)
    J0 = p.A_J * v0 ** (m + 1.0)
    D = p.C_J * J0 / (1.0 - p.psi)
    dt = p.cfl_K * min(p.dx / (2 * v0), p.dx / (v0 + math.sqrt(p.g * H0)), p.dx ** 2 / (2 * D), p.dt_max / p.cfl_K)
    assert info.dt == pytest.approx(dt, rel=1e-14, abs=0), (m, info.dt, dt)
    r = 1.0 - 4.0 * D * info.dt / p.dx ** 2 * math.sin(k * p.dx / 2) ** 2
    assert np.allclose(st.b, r * st0.b, rtol=0, atol=1e-15), (m, r)
    assert r < 1.0 - 1e-6
    # a different exponent gives a measurably different decay: the pin sees m
    r2 = 1.0 - 4.0 * (p.C_J * p.A_J * v0 ** 3 / (1.0 - p.psi)) * info.dt / p.dx ** 2 * math.sin(k * p.dx / 2) ** 2
    assert not np.allclose(st.b, r2 * st0.b, rtol=0, atol=1e-12)


def test_exner_shamov_gate(orc):
    """Below the Shamov critical velocity (Eq. 5) no sediment moves."""
    p = orc.Params(nx=1, ny=1)
    vk = p.C_Sh * p.d50 ** (1 / 3) * 1.0 ** (1 / 6)
    _, st0, st, _, _ = _exner_decay_case(orc, 0.999 * vk)
    assert np.array_equal(st.b, st0.b)
    _, st0, st, _, _ = _exner_decay_case(orc, 1.001 * vk)
    assert not np.array_equal(st.b, st0.b)


@pytest.mark.parametrize("m", [2.0, 1.5, 2.5], ids=["m2", "m1.5", "m2.5"])
@pytest.mark.parametrize("q", [2.0, -2.0], ids=["flow_+x", "flow_-x"])
def test_exner_advection_is_upwind(orc, q, m):
    """Frozen steady flow q = const over a bed hump with C_J = 0 reduces the
    Exner update (Eq. 1) to first-order upwind differencing of the Grass load
    J0 = A_J v|v|^m (Eq. 3) with v = q/H: backward differences for q > 0,
    forward ones for q < 0.  The hump's centroid moves downstream and the
    bed volume is conserved."""
    nx, dx = 200, 1.0
    x = (np.arange(nx) + 0.5) * dx
    b = 0.2 * np.exp(-((x - 100.0) / 8.0) ** 2)[None, :]
    eta0 = 2.0
    H = eta0 - b
    st0 = _state(orc, H, q + 0 * H, 0 * H, b)
    p = orc.Params(nx=nx, ny=1, dx=dx, frozen_hydro=1, C_J=0.0, A_J=0.01, m_exp=m, tile_x=nx, tile_y=1)
    st, info = orc.step(p, st0, 0.03)
    v = q / H[0]
    J = p.A_J * v * np.abs(v) ** m
    db = st.b[0] - b[0]
    c = info.dt / (dx * (1.0 - p.psi))
    inner = slice(5, nx - 5)
    if q > 0:
        exp = -c * (J - np.roll(J, 1))
    else:
        exp = -c * (np.roll(J, -1) - J)
    assert np.allclose(db[inner], exp[inner], rtol=1e-12, atol=1e-18)
    for _ in range(50):
        st, info = orc.step(p, st, 0.03)
    c0 = (x * b[0]).sum() / b[0].sum()
    inner_b = st.b[0][20:-20]
    ci = (x[20:-20] * inner_b).sum() / inner_b.sum()
    assert (ci - c0) * np.sign(q) > 0.05
    assert abs(st.b.sum() - b.sum()) < 1e-13


# ------------------------------------------------------------- K1 / HGS

def test_census_brute_force(orc):
    g = I.rng(21)
    H = np.where(g.uniform(size=(50, 70)) < 0.9, 0.0, 1.0) * g.uniform(0, 1e-3, (50, 70))
    src = (g.uniform(size=(50, 70)) < 0.01).astype(np.uint8)
    p = orc.Params(nx=70, ny=50, tile_x=16, tile_y=8)
    c = orc.census(p, H, src)
    for ty in range(c.shape[0]):
        for tx in range(c.shape[1]):
            blk = (H[ty * 8:(ty + 1) * 8, tx * 16:(tx + 1) * 16] > 1e-4) | \
                  (src[ty * 8:(ty + 1) * 8, tx * 16:(tx + 1) * 16] > 0)
            assert c[ty, tx] == blk.sum()


def test_hgs_skip_does_not_change_results(orc):
    """Skipping dry tiles (K1 + the Eulerian 4-neighbour rule) is exact."""
    sc = I.flood_channel(96, dx=5.0, seed=2, peak=200.0)
    hg = orc.Hydrograph(sc.hydro_t, sc.hydro_Q)
    res = []
    for skip in (1, 0):
        p = orc.Params(nx=96, ny=96, dx=5.0, hgs_skip=skip, tile_x=16, tile_y=8)
        st, t, infos = orc.run(p, _state(orc, sc.H, b=sc.b), sc.manning_per_cell(), 150,
                               src=sc.src, hydro=hg)
        res.append((st, t, infos))
    (a, ta, ia), (b, tb, ib) = res
    assert ta == tb
    for x, y in zip(a.arrays(), b.arrays()):
        assert np.array_equal(x, y)
    assert min(i.active_tiles for i in ia) < 96 * 96 // (16 * 8)   # something was skipped


# ------------------------------------------- open boundaries and rain (widening)

@pytest.mark.parametrize("u", [2.0, 5.0], ids=["subcritical", "supercritical"])
def test_open_boundaries_keep_uniform_flow(orc, u):
    """A uniform flow on a flat frictionless bed has no gradients; with open
    (zero-gradient) boundaries on all four sides its ghost cells equal the
    interior, so it must stay uniform to roundoff (with walls it cannot)."""
    ny, nx = 12, 20
    H = np.full((ny, nx), 1.0)
    st0 = _state(orc, H, Hu=u * H, Hv=0.5 * H)
    p = orc.Params(nx=nx, ny=ny, dx=1.0, bc_w=1, bc_e=1, bc_s=1, bc_n=1)
    st, _, _ = orc.run(p, st0, 0.0, 40)
    for a, a0 in zip(st.arrays(), st0.arrays()):
        assert np.abs(a - a0).max() < 1e-12
    pw = orc.Params(nx=nx, ny=ny, dx=1.0)
    sw, _, _ = orc.run(pw, st0, 0.0, 40)
    assert np.abs(sw.H - 1.0).max() > 1e-3


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (0, 1, 1, 0)], ids=["all_open", "mixed"])
def test_open_boundary_volume_budget(orc, bc):
    """Water volume plus the water that left through open sides is constant
    to roundoff (the boundary fluxes are the update's own fluxes), water does
    leave, and wall sides pass none."""
    ny, nx = 40, 48
    g = I.rng(61)
    y, x = np.mgrid[0:ny, 0:nx] + 0.5
    b = g.uniform(-0.02, 0.02, (ny, nx))
    H = 1.0 + 0.6 * np.exp(-((x - 30) ** 2 + (y - 14) ** 2) / 40.0) - b
    p = orc.Params(nx=nx, ny=ny, dx=2.0, bc_w=bc[0], bc_e=bc[1], bc_s=bc[2], bc_n=bc[3], tile_x=16, tile_y=16)
    st = _state(orc, H, b=b)
    v0 = st.H.sum() * p.dx ** 2
    out = 0.0
    for _ in range(150):
        st, info = orc.step(p, st, 0.02)
        out += info.outflow_vol
    v1 = st.H.sum() * p.dx ** 2
    assert out > 1e-3 * v0
    assert abs(v0 - v1 - out) < 1e-12 * v0


def test_open_boundary_lets_a_dry_bed_dam_break_flow_out(orc):
    """Ritter's dry-bed dam break on a domain that ends 32 m past the dam:
    the flow there is supercritical (u - c = (x - x0)/t > 0), so the exact
    solution is unaffected by what lies beyond, and an open boundary must
    reproduce it after the front has left (t = 8 s: 0.27 m of water crossing
    the end, the rarefaction head still 29 m from the left wall); a wall
    reflects the flow as a bore and cannot."""
    N, L, x0 = 768, 96.0, 64.0
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    H = np.where(x < x0, 2.0, 0.0) * np.ones((4, 1))
    errs = {}
    for name, bce in (("open", 1), ("wall", 0)):
        p = orc.Params(nx=N, ny=4, dx=dx, sediment_on=0, bc_e=bce, tile_x=256, tile_y=4)
        st, t, _ = orc.run(p, _state(orc, H), 0.0, 100000, t_end=8.0)
        he = _stoker(x, t, 2.0, 0.0, x0)
        errs[name] = np.abs(st.H[0] - he).sum() / np.abs(he).sum()
    assert errs["open"] < 0.01, errs
    assert errs["wall"] > 5 * errs["open"], errs


@pytest.mark.parametrize("sigma", [2e-3, -1e-3], ids=["rain", "evaporation"])
def test_rain_raises_a_lake_uniformly(orc, sigma):
    """A uniform source sigma (m/s) on a lake at rest over a noisy bed in a
    closed basin: the free surface stays flat and at rest, and the volume
    changes by exactly sigma x area x elapsed time."""
    ny, nx = 24, 32
    g = I.rng(62)
    b = g.uniform(-0.05, 0.05, (ny, nx))
    H = 1.5 - b
    p = orc.Params(nx=nx, ny=ny, dx=1.0)
    st = _state(orc, H, b=b)
    v0 = st.H.sum()
    rv, t = 0.0, 0.0
    for _ in range(30):
        st, info = orc.step(p, st, 0.03, rain=np.full((ny, nx), sigma))
        rv += info.rain_vol
        t += info.dt
    eta = st.H + st.b
    assert eta.max() - eta.min() < 1e-12
    assert np.abs(st.Hu).max() < 1e-12 and np.abs(st.Hv).max() < 1e-12
    assert rv == pytest.approx(sigma * nx * ny * t, rel=1e-12)
    assert st.H.sum() - v0 == pytest.approx(rv, rel=1e-10)


def test_infiltration_drains_a_lake_at_its_rate_and_stops_at_zero(orc):
    """A flat lake at rest, uniform absorption rate beta: the depth falls by
    exactly beta dt per step while water lasts, never below zero, the lake
    stays at rest, and the infiltrated volume is what the lake lost."""
    ny, nx, beta, H0 = 10, 14, 2e-3, 0.05
    H = np.full((ny, nx), H0)
    p = orc.Params(nx=nx, ny=ny, dx=1.0, sediment_on=0)
    st = _state(orc, H)
    lost, t = 0.0, 0.0
    for _ in range(400):
        st, info = orc.step(p, st, 0.03, beta=beta)
        lost += info.infil_vol
        t += info.dt
        assert st.H.min() >= 0.0
        expect = max(H0 - beta * t, 0.0)
        assert np.abs(st.H - expect).max() < 1e-12 * max(1.0, t)
        assert not st.Hu.any() and not st.Hv.any()
        if expect == 0.0:
            break
    assert st.H.max() == 0.0, "the lake must drain completely"
    assert lost == pytest.approx(H0 * nx * ny, rel=1e-12)


def test_infiltration_keeps_the_velocity_of_a_uniform_flow(orc):
    """Infiltration takes its share of momentum: a uniform flow with open
    boundaries loses depth uniformly while its velocity stays unchanged."""
    ny, nx = 8, 12
    H = np.full((ny, nx), 1.0)
    p = orc.Params(nx=nx, ny=ny, dx=1.0, bc_w=1, bc_e=1, bc_s=1, bc_n=1)
    st = _state(orc, H, Hu=1.5 * H, Hv=-0.5 * H)
    for _ in range(20):
        st, _ = orc.step(p, st, 0.0, beta=1e-3)
    assert st.H.max() < 1.0 and np.ptp(st.H) < 1e-13
    assert np.abs(st.Hu / st.H - 1.5).max() < 1e-12 and np.abs(st.Hv / st.H + 0.5).max() < 1e-12
