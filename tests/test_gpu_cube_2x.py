"""The porous-cube channel of the benchmark (config: velocity inlet, pressure
outlet, bounce-back side walls, a sharp porous cube, Re = 100) on its 2x
downscaled copy at 10,000 steps, against the oracle's stored result."""
import json
import os

import numpy as np
import pytest

import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import workloads
from test_gpu_parity import TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_29619_b300 import build

    build.build()


def test_cube_channel_downscaled_2x_against_stored_oracle():
    """The porous-cube channel on its 2x downscaled copy (256 x 128 x 128, cube
    of side 64, nu = 0.032, Re = 100) at 10,000 steps against the oracle's result
    stored in tests/golden/cube_channel_256_10000.json (written by
    tests/golden/make_cube_channel_256.py, which calls only the oracle).  The
    GPU FP64 path must match to 1e-12 at the 512 sampled nodes and in the drag;
    FP32 and FP16 storage are held to their parity bars at the sampled nodes
    (the sharp cube violates the C2 porosity the method asks for, R9: a form
    that misses its bar is reported xfailed with its error) and to 1e-3 in the
    drag and the through-cube flow fraction."""
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "cube_channel_256_10000.json")))
    nz, ny, nx = g["shape"]
    side = g["side"]
    eps, kap = workloads.cube_channel(nx, ny, nz, side=side, eps_cube=0.4, Da=1e-4)
    x0, y0, z0 = (nx - side) // 2, (ny - side) // 2, (nz - side) // 2
    errs, bad = {}, {}
    for storage, kernel in (("fp64", "sweep"), ("fp32", "split"), ("fp16", "split")):
        s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel=kernel, bc=("inflow_outflow", "wall", "wall"),
                           viscosity=g["nu"], forchheimer=g["forchheimer"], inlet_v=(g["U"], 0, 0), outlet_rho=1.0)
        s.step(g["steps"])
        _, v = s.moments()
        st = s.reduce()
        s.close()
        vn = np.array([[v[a][z, y, x] for a in range(3)] for z, y, x in g["nodes"]])
        err = float(np.max(np.sqrt(((vn - np.array(g["v_nodes"])) ** 2).sum(axis=1)))) / g["max_speed"]
        vx = v[0, :, :, nx // 2]
        frac = float(vx[z0:z0 + side, y0:y0 + side].sum() / vx.sum())
        drag_err = abs(st["drag"][0] - g["drag_x"]) / abs(g["drag_x"])
        errs[storage] = (err, drag_err, abs(frac - g["flow_fraction"]))
        if storage == "fp64":
            assert err <= TOL["fp64"] and drag_err <= 1e-12, errs
        else:
            assert drag_err <= 1e-3 and abs(frac - g["flow_fraction"]) <= 1e-3, errs
            if err > TOL[storage]:
                bad[storage] = err
    if bad:
        pytest.xfail(f"sharp cube, 2x copy: reduced storage beyond its bar {bad} (all: {errs})")
