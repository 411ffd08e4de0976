"""The library's FP64 reductions (lbm_reduce) and long runs, against the oracle.

* Reductions: the mass, mean superficial velocity, |v|^2 sum, the residual of
  Eq. (SS_convergence_L2) over a k-step gap, the Darcy-Forchheimer drag
  sum rho (mu_D + mu_F |v|) v and the apparent permeability nu_f <v> / b are
  computed here with NumPy from the ORACLE's populations, rho, v and drag
  coefficients and compared with lbm_reduce on the sweep, split (two arrays
  and in place) and fused paths at FP64, FP32 and FP16, with walls and with a
  porous cube.
* The 64^3 copy of the porous-box benchmark (Gaussian random field,
  correlation length 16, seed 2) over 1,000 steps.
* The porous-cube channel with its sharp-edged cube, on an 8x downscaled copy
  (64 x 32 x 32, cube of side 16, Re = 100) that the oracle runs in seconds.
"""
import numpy as np
import pytest

import oracle
import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import workloads
from test_gpu_parity import TOL, assert_parity, vel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_29619_b300 import build

    build.build()


def oracle_reductions(o, b, nu_f, v_ref=None):
    """The quantities lbm_reduce reports, from the oracle's state."""
    rho, v = o.moments()
    muD, muF, _, _ = o.static()
    nv = np.sqrt((v**2).sum(axis=0))
    out = {"mass": float(o.get_f().sum()), "mean_v": [float(v[a].mean()) for a in range(3)],
           "v2_sum": float((v**2).sum()),
           "drag": [float((rho * (muD + muF * nv) * v[a]).sum()) for a in range(3)],
           "k_app": [nu_f * float(v[a].mean()) / b[a] if b[a] != 0 else 0.0 for a in range(3)]}
    if v_ref is not None:
        out["residual"] = float(np.sqrt(((v - v_ref) ** 2).sum() / (v_ref**2).sum()))
    return out, v


REL = {"fp64": 1e-11, "fp32": 2e-5, "fp16": 2e-3}


@pytest.mark.parametrize("storage,kernel,streaming", [("fp64", "sweep", "auto"), ("fp32", "split", "two_arrays"),
                                                      ("fp32", "split", "in_place"), ("fp16", "split", "in_place"),
                                                      ("fp32", "fused", "auto")])
@pytest.mark.parametrize("case", ["box", "walls_cube"])
def test_reductions_match_oracle(storage, kernel, streaming, case):
    if case == "box":
        shape = (10, 12, 32)
        eps = workloads.random_smooth_porosity(shape, seed=51, lo=0.45, hi=0.95)
        kap = workloads.carman_kappa(eps, 2.0)
        walls = (0, 0, 0)
        b = (6e-4, 2e-4, 1e-4)
    else:
        # bounce-back walls on y and z around a porous cube (smoothed edges:
        # the C2 porosity the method requires) in a channel driven along x
        eps, kap = workloads.cube_channel(32, 16, 16, side=8, eps_cube=0.4, Da=1e-2, smooth=2)
        walls = (0, 1, 1)
        b = (8e-4, 0.0, 0.0)
    nu = 0.03
    bc = tuple("wall" if w else "periodic" for w in walls)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=nu, b=b, forch=-1.0, wall=walls).init()
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel=kernel, bc=bc, viscosity=nu, force=b,
                       forchheimer=lbm.F_ERGUN, streaming=streaming)
    # a transient that still moves: the residual over the gap is O(0.1-1)
    o.step(21)
    s.step(21)
    _, v_ref = o.moments()
    s.reduce(snapshot=True)
    o.step(30)
    s.step(30)
    ref, _ = oracle_reductions(o, b, nu, v_ref)
    got = s.reduce()
    rel = REL[storage]
    assert got["steps"] == 51
    assert got["mass"] == pytest.approx(ref["mass"], rel=rel * 1e-2)
    assert got["v2_sum"] == pytest.approx(ref["v2_sum"], rel=3 * rel)
    assert got["residual"] == pytest.approx(ref["residual"], rel=10 * rel)
    assert 0.05 < ref["residual"] < 5
    vmax = max(abs(x) for x in ref["mean_v"])
    for a in range(3):
        assert got["mean_v"][a] == pytest.approx(ref["mean_v"][a], rel=rel, abs=rel * vmax)
        dmax = max(abs(x) for x in ref["drag"])
        assert got["drag"][a] == pytest.approx(ref["drag"][a], rel=rel, abs=rel * dmax)
        if b[a] != 0:
            assert got["k_app"][a] == pytest.approx(ref["k_app"][a], rel=rel)
        else:
            assert got["k_app"][a] == 0.0
    # the drag is not negligible (porous nodes carry flow)
    assert abs(ref["drag"][0]) > 1e-3 * abs(ref["mean_v"][0]) * eps.size


def test_porous_box_64_copy_1000_steps():
    """The 64^3 copy of the benchmark box (same recipe: correlation length 16,
    seed 2), 1,000 steps: FP32 on both streaming forms and FP16 in place."""
    eps, kap = workloads.porous_box((64, 64, 64), ell=16.0, seed=2)
    kw = dict(nu_f=0.02, b=(6e-4, 0.0, 0.0), forch=-1.0)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init()
    o.step(1000)
    ro, vo = o.moments()
    for storage, streaming in (("fp32", "two_arrays"), ("fp32", "in_place"), ("fp16", "in_place")):
        s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel="split", viscosity=0.02, force=kw["b"],
                           forchheimer=lbm.F_ERGUN, streaming=streaming)
        s.step(1000)
        _, vg = s.moments()
        assert_parity(vel_err(vg, vo), storage)
        # the mean flow rate of the configuration
        assert s.reduce()["mean_v"][0] == pytest.approx(float(vo[0].mean()), rel=TOL[storage])
        s.close()


def test_sharp_cube_channel_downscaled_copy():
    """The porous-cube channel with a SHARP cube (eps = 0.4 inside, 1 outside,
    Da = 1e-4 on the cube side, F = 0.55, velocity inlet 0.05, pressure outlet,
    bounce-back side walls, Re = 100 on the cube side) on the 8x downscaled
    copy, 2,000 steps.  FP64 must match the oracle to 1e-12.  FP32 and FP16 are
    held to their parity bars: at the one-node porosity jump the
    finite-difference Delta_nu makes the step stiff (the method asks for C2
    porosity, Sec. 3.5) and amplifies storage rounding; a form that misses its
    bar is reported xfailed with its error."""
    nx, ny, nz, side = 64, 32, 32, 16
    eps, kap = workloads.cube_channel(nx, ny, nz, side=side, eps_cube=0.4, Da=1e-4)
    U, nu = 0.05, 0.05 * side / 100.0
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=nu, wall=(2, 1, 1), forch=0.55, v_in=(U, 0, 0),
                      rho_out=1.0).init()
    o.step(2000)
    _, vo = o.moments()
    errs = {}
    for storage, kernel in (("fp64", "sweep"), ("fp32", "split"), ("fp16", "split")):
        s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel=kernel, bc=("inflow_outflow", "wall", "wall"),
                           viscosity=nu, forchheimer=0.55, inlet_v=(U, 0, 0), outlet_rho=1.0)
        s.step(2000)
        errs[storage] = vel_err(s.moments()[1], vo)
        s.close()
    assert errs["fp64"] <= TOL["fp64"]
    bad = {k: v for k, v in errs.items() if k != "fp64" and v > TOL[k]}
    assert all(v < 1e-1 for v in errs.values()), errs
    if bad:
        pytest.xfail(f"sharp cube: reduced storage beyond its bar {bad} (all errors {errs})")


@pytest.mark.parametrize("storage,streaming", [("fp32", "two_arrays"), ("fp32", "in_place"), ("fp16", "two_arrays"),
                                               ("fp16", "in_place"), ("bf16", "two_arrays")])
def test_porous_box_64_copy_5000_steps_against_stored_oracle(storage, streaming):
    """The 64^3 copy of the benchmark box at the workload's own 5,000 steps
    against the oracle's result stored in tests/golden/porous_box_64_5000.json
    (written by tests/golden/make_porous_box_64.py, which calls only the
    oracle): the velocity at 512 sampled nodes within the storage form's parity
    bar (normalised by the oracle's largest speed) and the mean flow rate."""
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "porous_box_64_5000.json")))
    eps, kap = workloads.porous_box((64, 64, 64), ell=16.0, seed=2)
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel="split", viscosity=0.02, force=(6e-4, 0.0, 0.0),
                       forchheimer=lbm.F_ERGUN, streaming=streaming)
    s.step(g["steps"])
    _, v = s.moments()
    st = s.reduce()
    s.close()
    vn = np.array([[v[a][z, y, x] for a in range(3)] for z, y, x in g["nodes"]])
    err = float(np.max(np.sqrt(((vn - np.array(g["v_nodes"])) ** 2).sum(axis=1)))) / g["max_speed"]
    assert st["mean_v"][0] == pytest.approx(g["mean_v"][0], rel=TOL[storage] if storage != "bf16" else 1e-2)
    assert_parity(err, storage)

