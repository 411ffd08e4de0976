"""Writes cube_channel_256_10000.json: the FP64 oracle on the 2x downscaled copy
of the porous-cube channel (256 x 128 x 128 nodes, centred cube of side 64 with
eps = 0.4 and kappa = 1e-4 64^2, F = 0.55, free fluid elsewhere; velocity inlet
0.05 at x = 0, pressure outlet rho = 1 at x = 255, halfway bounce-back walls in y
and z; nu = 0.032, Re = 100 on the cube side), 10,000 steps from rest.  Stored:
the Darcy-Forchheimer drag along x summed over all nodes, the through-cube flow
fraction at mid-cube, the mean velocity, the largest speed and the velocity at
512 nodes drawn with numpy's default_rng(256), for the GPU parity test of the
channel at its downscaled size.  Calls only oracle/.  About four hours on eight
cores.

    python tests/golden/make_cube_channel_256.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2606_29619_b300 import workloads  # noqa: E402

NX, NY, NZ, SIDE, STEPS = 256, 128, 128, 64, 10000
U, NU, F = 0.05, 0.032, 0.55


def main():
    eps, kap = workloads.cube_channel(NX, NY, NZ, side=SIDE, eps_cube=0.4, Da=1e-4)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=NU, wall=(2, 1, 1), forch=F, v_in=(U, 0, 0), rho_out=1.0).init()
    o.step(STEPS)
    rho, v = o.moments()
    muD, muF, _, _ = o.static()
    speed = np.sqrt((v**2).sum(axis=0))
    drag = float((rho * (muD + muF * speed) * v[0]).sum())
    x0, y0, z0 = (NX - SIDE) // 2, (NY - SIDE) // 2, (NZ - SIDE) // 2
    vx = v[0, :, :, NX // 2]
    frac = float(vx[z0:z0 + SIDE, y0:y0 + SIDE].sum() / vx.sum())
    rng = np.random.default_rng(256)
    idx = np.stack([rng.integers(0, NZ, 512), rng.integers(0, NY, 512), rng.integers(0, NX, 512)], axis=1)
    out = {"steps": STEPS, "shape": [NZ, NY, NX], "side": SIDE, "nu": NU, "U": U, "forchheimer": F,
           "drag_x": drag, "flow_fraction": frac, "mean_v": [float(v[a].mean()) for a in range(3)],
           "max_speed": float(speed.max()), "nodes": idx.tolist(),
           "v_nodes": [[float(v[a][z, y, x]) for a in range(3)] for z, y, x in idx]}
    with open(os.path.join(HERE, "cube_channel_256_10000.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
