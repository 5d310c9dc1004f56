"""Write the stored oracle sample of the 64^3 3-D cavity (cavity3d_tanh64.npz).

The FP64 oracle (oracle/islbm_oracle.py) runs the 3-D side-heated cavity
(D3Q19 + D3Q7, Sec. 4) on the 64^3 tanh-stretched mesh (a = 1.5) at Ra = 1e6,
Pr = 0.71 from rest with the seeded temperature noise for 1000 steps (about
eight minutes on one core).  The GPU test compares the 3-D step kernels with
this run on several tiles per axis without running the oracle itself.
Stored: T, u, v, w at 6000 nodes drawn with numpy's PCG64 (seed 64), the
largest |T| and speed over all nodes (the normalisers of the field-relative
error), and the reductions.

    python tests/golden/make_cavity3d_tanh64.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import islbm_oracle as O  # noqa: E402
from synthetic import temperature_noise  # noqa: E402

N, A, RA, STEPS, SAMPLES = 64, 1.5, 1e6, 1000, 6000


def main():
    xi = O.mesh_tanh(N, A)
    cav = O.Cavity(xi, xi, xi, params=O.Params(Ra=RA))
    cav.init_fields(temperature_noise(cav.shape, 1e-6, seed=0))
    cav.step(STEPS)
    rho, u, T = cav.fields()
    red = cav.reductions()
    idx = np.random.default_rng(64).choice(T.size, SAMPLES, replace=False)
    idx.sort()
    speed = np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    keys = [k for k in ("Nu", "Nu_hot", "Nu_cold", "Re", "Re_uv", "mass") if k in red]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity3d_tanh64.npz")
    np.savez_compressed(
        out, n=N, a=A, Ra=RA, steps=STEPS, index=idx,
        T=T.ravel()[idx], u=u[0].ravel()[idx], v=u[1].ravel()[idx], w=u[2].ravel()[idx],
        T_absmax=np.abs(T).max(), u_absmax=np.abs(u).max(), speed_max=speed.max(),
        red_keys=np.array(keys), red_values=np.array([red[k] for k in keys]))
    print(out, {k: red[k] for k in keys})


if __name__ == "__main__":
    main()
