"""Seeded synthetic inputs shaped like the paper's flood workloads.

The paper runs on the Volga-Akhtuba floodplain DEM (Sec. 3), which is not
available; these generators stand in for it.  They hold none of the method's
arithmetic: they only build terrains, initial states, Manning fields, source
masks and hydrographs, all from a numpy ``Generator(PCG64(seed))``.

Recipes (sizes in cells, lengths in metres):
  * dam break: H = h_left for x < x_dam, h_right otherwise, v = 0, flat bed
    plus uniform noise (+-amp), walls.
  * fractal DEM: spectral synthesis, amplitude |k|^(-beta/2) with random phases,
    rescaled to a given relief (max - min).
  * channel: a sinusoidal meander from x = 0 to the far edge, `width` metres
    wide, its bed 2 m below the local terrain minimum along the path and made
    monotone downhill.
  * Manning n: uniform random per block (e.g. 64 x 64 cells).
  * hydrograph: triangular inflow on the cells of the channel head.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Scenario:
    """A complete input set: state (H, Hu, Hv, b) [ny, nx] float64, Manning n
    (per cell or per block), optional source mask and hydrograph."""
    nx: int
    ny: int
    dx: float
    H: np.ndarray
    Hu: np.ndarray
    Hv: np.ndarray
    b: np.ndarray
    manning: np.ndarray          # [ny, nx] per cell, or [nby, nbx] per block
    manning_block: int = 0       # 0: per cell, else block edge in cells (power of two)
    src: np.ndarray | None = None  # uint8 [ny, nx]
    hydro_t: np.ndarray | None = None
    hydro_Q: np.ndarray | None = None
    name: str = ""

    def manning_per_cell(self) -> np.ndarray:
        if self.manning_block <= 1:
            return np.broadcast_to(self.manning, (self.ny, self.nx))
        B = self.manning_block
        return np.repeat(np.repeat(self.manning, B, axis=0), B, axis=1)[: self.ny, : self.nx]


def canonical_dry(H, Hu, Hv, eps=1e-4):
    """Dry cells (H <= eps) carry no momentum."""
    dry = ~(H > eps)
    Hu = np.where(dry, 0.0, Hu)
    Hv = np.where(dry, 0.0, Hv)
    return Hu, Hv


def dam_break(nx=128, ny=128, dx=1.0, x_dam=64, h_left=2.0, h_right=0.5, noise=0.01,
              manning=0.03, seed=1) -> Scenario:
    """Dam break over a flat erodible bed with uniform +-noise (walls)."""
    g = rng(seed)
    b = g.uniform(-noise, noise, (ny, nx)) if noise > 0 else np.zeros((ny, nx))
    H = np.where(np.arange(nx)[None, :] < x_dam, h_left, h_right) * np.ones((ny, 1))
    Hu = np.zeros_like(H)
    Hv = np.zeros_like(H)
    return Scenario(nx, ny, dx, H, Hu, Hv, b, np.full((1, 1), manning), manning_block=max(nx, ny),
                    name=f"dam_break_{nx}x{ny}")


def fractal_dem(nx: int, ny: int, seed: int, beta: float = 2.0, relief: float = 20.0,
                dtype=np.float64) -> np.ndarray:
    """Spectral-synthesis fractal surface with power spectrum ~ |k|^-beta,
    rescaled to `relief` metres (min 0)."""
    g = rng(seed)
    # float64 spectra up to 4096^2 (the result rounded to float32 is then the
    # same on every platform to the last bit, practically); float32 above that
    # to bound host memory
    wide = nx * ny <= 4096 * 4096
    ft = np.float64 if wide else np.float32
    ky = np.fft.fftfreq(ny).astype(ft)[:, None]
    kx = np.fft.rfftfreq(nx).astype(ft)[None, :]
    kk = np.sqrt(kx * kx + ky * ky)
    kk[0, 0] = 1.0
    amp = kk ** ft(-beta / 2.0)
    amp[0, 0] = 0.0
    del kk
    phase = g.uniform(0.0, 2.0 * np.pi, size=amp.shape).astype(ft)
    spec = (amp * np.exp(1j * phase)).astype(np.complex128 if wide else np.complex64)
    del amp, phase
    try:
        import scipy.fft as sfft
        z = sfft.irfft2(spec, s=(ny, nx), workers=-1)
    except Exception:  # pragma: no cover - numpy fallback
        z = np.fft.irfft2(spec, s=(ny, nx))
    del spec
    z = np.asarray(z, dtype=ft)
    lo, hi = float(z.min()), float(z.max())
    z -= lo
    z *= ft(relief / (hi - lo))
    # quantise to float32 so both sides of a comparison see the same terrain
    return z.astype(np.float32).astype(dtype, copy=False)


def carve_channel(b: np.ndarray, dx: float, width_m: float = 40.0, depth_m: float = 2.0,
                  meander_amp_frac: float = 0.125, wavelength_frac: float = 0.5):
    """Carves a sinusoidal meander from x = 0 to x = nx-1 into b (in place).
    Returns the (rows, cols) of the channel head cells at x = 0."""
    ny, nx = b.shape
    wc = max(1, int(round(width_m / dx)))
    x = np.arange(nx)
    yc = ny / 2 + meander_amp_frac * ny * np.sin(2 * np.pi * x / (wavelength_frac * nx))
    y0 = np.clip(np.round(yc - wc / 2).astype(np.int64), 0, ny - wc)
    rows = y0[None, :] + np.arange(wc)[:, None]           # [wc, nx]
    cols = np.broadcast_to(x[None, :], rows.shape)
    local_min = b[rows, cols].min(axis=0) - depth_m
    z = np.minimum.accumulate(local_min)                  # monotone downhill along x
    b[rows, cols] = np.broadcast_to(z[None, :], rows.shape).astype(b.dtype)
    return rows[:, 0].copy(), np.zeros(wc, dtype=np.int64)


def manning_blocks(nx: int, ny: int, block: int, lo: float, hi: float, seed: int) -> np.ndarray:
    g = rng(seed)
    nbx = -(-nx // block)
    nby = -(-ny // block)
    return g.uniform(lo, hi, (nby, nbx))


def triangular_hydrograph(peak: float, t_peak: float = 1200.0, t_end: float = 3600.0):
    return np.array([0.0, t_peak, t_end]), np.array([0.0, peak, 0.0])


def flood_channel(n: int = 2048, dx: float = 5.0, seed: int = 2, peak: float = 500.0,
                  n_lo: float = 0.02, n_hi: float = 0.05, block: int = 64,
                  relief: float = 20.0) -> Scenario:
    """Initially dry fractal terrain with a carved 40 m channel and an inflow
    hydrograph on the channel head cells; Manning n per block."""
    b = fractal_dem(n, n, seed, relief=relief)
    rows, cols = carve_channel(b, dx)
    H = np.zeros_like(b)
    src = np.zeros((n, n), dtype=np.uint8)
    src[rows, cols] = 1
    ht, hq = triangular_hydrograph(peak)
    man = manning_blocks(n, n, block, n_lo, n_hi, seed + 1000)
    return Scenario(n, n, dx, H, np.zeros_like(b), np.zeros_like(b), b, man, manning_block=block,
                    src=src, hydro_t=ht, hydro_Q=hq, name=f"flood_channel_{n}")


def half_wet(n: int = 16384, dx: float = 5.0, seed: int = 3, wet_fraction: float = 0.5,
             step_m: float = 2.0, block: int = 64, dtype=np.float32, relief: float = 20.0) -> Scenario:
    """Fractal terrain with a carved channel, filled to a level eta0 (+ step_m
    on x < n/2, a dam-break step so fronts move) chosen by bisection so that the
    wet fraction is `wet_fraction`; H = max(eta - b, 0), v = 0."""
    b = fractal_dem(n, n, seed, relief=relief, dtype=np.float32)
    carve_channel(b, dx)
    half = n // 2
    sub = b[::8, ::8]
    left = sub[:, : sub.shape[1] // 2]
    right = sub[:, sub.shape[1] // 2:]

    def frac(e0):
        return 0.5 * float((left < e0 + step_m).mean()) + 0.5 * float((right < e0).mean())

    lo, hi = float(b.min()) - step_m, float(b.max()) + step_m
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if frac(mid) < wet_fraction:
            lo = mid
        else:
            hi = mid
    eta0 = 0.5 * (lo + hi)
    H = np.empty_like(b)
    np.subtract(np.float32(eta0 + step_m), b[:, :half], out=H[:, :half])
    np.subtract(np.float32(eta0), b[:, half:], out=H[:, half:])
    np.maximum(H, np.float32(0.0), out=H)
    man = manning_blocks(n, n, block, 0.02, 0.05, seed + 1000)
    zeros = np.zeros_like(b)
    sc = Scenario(n, n, dx, H.astype(dtype, copy=False), zeros, zeros.copy(), b.astype(dtype, copy=False),
                  man, manning_block=block, name=f"half_wet_{n}")
    sc.eta0 = eta0
    return sc


def ensemble_specs(n_scen: int = 64, seed: int = 4, side_lo: int = 256, side_hi: int = 2048):
    """Per-scenario parameters of a batched flood ensemble: square sides
    32*U{8..64} (256..2048), Manning n ~ U[0.02, 0.06], inflow peak ~ U[50, 1000],
    grain-size scale ~ U[0.5, 2]."""
    g = rng(seed)
    sides = 32 * g.integers(side_lo // 32, side_hi // 32 + 1, n_scen)
    return [dict(side=int(sides[k]), seed=int(1000 + k), manning=float(g.uniform(0.02, 0.06)),
                 peak=float(g.uniform(50.0, 1000.0)), d50_scale=float(g.uniform(0.5, 2.0)))
            for k in range(n_scen)]


def ensemble_scenario(side: int, seed: int, manning: float, peak: float, d50_scale: float,
                      dx: float = 5.0, wet_fraction: float = 0.5) -> Scenario:
    """One member of a flood ensemble: fractal terrain with a carved channel,
    filled half wet with a dam-break step, plus an inflow hydrograph of the
    given peak on the channel head; uniform Manning n.  The grain-size scale
    multiplies d50 (returned as the attribute d50)."""
    sc = half_wet(side, dx=dx, seed=seed, wet_fraction=wet_fraction, dtype=np.float64)
    b = sc.b
    wc = max(1, int(round(40.0 / dx)))
    yc = side / 2
    rows = np.clip(np.round(yc - wc / 2).astype(np.int64), 0, side - wc) + np.arange(wc)
    src = np.zeros((side, side), dtype=np.uint8)
    src[rows, 0] = 1
    ht, hq = triangular_hydrograph(peak)
    out = Scenario(side, side, dx, sc.H, sc.Hu, sc.Hv, b, np.full((1, 1), manning), manning_block=1 << 14,
                   src=src, hydro_t=ht, hydro_Q=hq, name=f"ensemble_{side}_{seed}")
    out.d50 = 5e-4 * d50_scale
    return out



def sparse_lake(nx: int, ny: int, dx: float = 5.0, seed: int = 11, center=(128, 960), radius: int = 40,
                rise: float = 1.5) -> Scenario:
    """Mostly dry fractal terrain with one lake released from a circular
    reservoir: water level `rise` metres above the terrain's highest point
    inside a disc of `radius` cells at `center` (row, column), dry elsewhere,
    at rest; uniform Manning n 0.03.  The lake's edge spreads across the
    HGS blocks and regions around it while most of the domain stays dry."""
    b = fractal_dem(nx, ny, seed)
    yy, xx = np.mgrid[0:ny, 0:nx]
    disc = (yy - center[0]) ** 2 + (xx - center[1]) ** 2 <= radius ** 2
    eta = b[disc].max() + rise
    H = np.where(disc, eta - b, 0.0)
    Z = np.zeros_like(H)
    return Scenario(nx, ny, dx, H, Z, Z.copy(), b, np.full((ny, nx), 0.03), manning_block=0,
                    name=f"sparse_lake_{nx}x{ny}")
