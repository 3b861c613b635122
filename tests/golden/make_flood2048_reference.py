"""Writes tests/golden/flood2048_oracle.npz: the FP64 CPU oracle's state after
10^4 steps of the 2048^2 flood-channel workload (fractal DEM seed 2, 40 m
channel, 500 m^3/s triangular hydrograph, Manning n per 64x64 block, psi 0.4,
K 0.4).  Calls only the oracle and the seeded input generators.

Stored: final H, the bed change b - b0, t and the step count, plus input
checksums so a consumer can verify it regenerated the same inputs.
Usage: python tests/golden/make_flood2048_reference.py [nsteps]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2103_15196_gb300 import inputs as I  # noqa: E402


def main(nsteps=10000):
    sc = I.flood_channel(2048, dx=5.0, seed=2, peak=500.0)
    p = O.Params(nx=2048, ny=2048, dx=5.0, tile_x=64, tile_y=64)
    O.set_threads(os.cpu_count() or 1)
    n = np.ascontiguousarray(sc.manning_per_cell(), dtype=np.float64)
    st = O.State(sc.H, sc.Hu, sc.Hv, sc.b)
    t0 = time.time()
    st, t, infos = O.run(p, st, n, nsteps, src=sc.src, hydro=O.Hydrograph(sc.hydro_t, sc.hydro_Q))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flood2048_oracle.npz")
    np.savez_compressed(out, H=st.H, db=st.b - sc.b, Hu=st.Hu, Hv=st.Hv, t=t, steps=len(infos),
                        b0_sum=float(sc.b.sum()), n_sum=float(sc.manning.sum()),
                        inflow=float(sum(i.inflow_vol for i in infos)))
    print(f"{len(infos)} steps, t = {t:.6f} s, {time.time() - t0:.0f} s, wet {(st.H > 1e-4).sum()}, "
          f"-> {out} ({os.path.getsize(out) / 1e6:.1f} MB)")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 10000)
