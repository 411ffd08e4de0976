"""Writes porous_box_64_5000.json: the FP64 oracle on the 64^3 copy of the
porous-box benchmark (Gaussian random field porosity, correlation length 16,
seed 2; Carman-Kozeny permeability d = 2, Ergun F, nu = 0.02, b = 6e-4 along x),
5,000 steps from rest.  Stored: the domain-mean superficial velocity, the sum of
|v|^2 and the velocity at 512 nodes drawn with numpy's default_rng(64), for the
GPU parity test of the workload at its own step count.  Calls only oracle/.

    python tests/golden/make_porous_box_64.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2606_29619_b300 import workloads  # noqa: E402

STEPS = 5000


def main():
    eps, kap = workloads.porous_box((64, 64, 64), ell=16.0, seed=2)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=0.02, b=(6e-4, 0.0, 0.0), forch=-1.0).init()
    o.step(STEPS)
    _, v = o.moments()
    rng = np.random.default_rng(64)
    idx = rng.integers(0, 64, size=(512, 3))  # (z, y, x)
    out = {"steps": STEPS, "shape": [64, 64, 64], "mean_v": [float(v[a].mean()) for a in range(3)],
           "v2_sum": float((v**2).sum()), "max_speed": float(np.sqrt((v**2).sum(axis=0)).max()),
           "nodes": idx.tolist(), "v_nodes": [[float(v[a][z, y, x]) for a in range(3)] for z, y, x in idx]}
    with open(os.path.join(HERE, "porous_box_64_5000.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
