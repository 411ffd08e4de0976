"""The split step with in-place (AA-pattern) streaming (LBM_STREAM_IN_PLACE:
one population array), called through the C ABI and checked against the FP64
oracle on the same seeded inputs.

The stored layout alternates between steps, so every check runs at odd and
even step counts.  Tolerances are those of test_gpu_parity (velocity error
E = max |v - v_oracle| / max |v_oracle|).
"""
import os

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


def _sim(eps, kap, storage, kernel="split", walls=(0, 0, 0), **kw):
    bc = tuple("wall" if w else "periodic" for w in walls)
    streaming = "in_place" if kernel == "split" else "auto"
    return lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel=kernel, bc=bc, viscosity=kw["nu_f"],
                          force=kw.get("b", (0, 0, 0)), forchheimer=kw.get("forch", 0.0), streaming=streaming,
                          **kw.get("extra", {}))


# ragged tiles: nx = 72 is one full 64-node tile row plus 8; ny = 10 leaves two rows of the last 4-row tile
BOX = (12, 10, 72)


@pytest.mark.parametrize("storage,steps", [("fp32", 1), ("fp32", 2), ("fp32", 7), ("fp32", 40), ("fp16", 39),
                                           ("fp16", 40), ("bf16", 39), ("bf16", 40)])
def test_inplace_porous_box_matches_oracle(storage, steps):
    """Reduced-precision storage is compared after ~40 steps: a few steps from
    rest |v| is still ~1e-4 and FP16 rounding of the initial populations alone
    is ~1e-3 of it."""
    eps = workloads.random_smooth_porosity(BOX, seed=41, lo=0.4, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    kw = dict(nu_f=0.02, b=(6e-4, 2e-4, -1e-4), forch=-1.0)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init()
    s = _sim(eps, kap, storage, **kw)
    assert s.info()["kernel"] == "split" and s.info()["in_place"]
    o.step(steps)
    s.step(steps)
    ro, vo = o.moments()
    rg, vg = s.moments()
    assert_parity(vel_err(vg, vo), storage)
    if storage == "fp32":
        np.testing.assert_allclose(rg, ro, rtol=1e-6)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_inplace_walls_matches_oracle(storage):
    """Halfway bounce-back walls on y and z: reflected populations stay in the
    node's own slots in both layouts."""
    shape = (16, 12, 40)
    eps = workloads.random_smooth_porosity(shape, seed=43, lo=0.45, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    kw = dict(nu_f=0.04, b=(5e-4, 0, 0), forch=-1.0)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, wall=(0, 1, 1), **kw).init()
    s = _sim(eps, kap, storage, walls=(0, 1, 1), **kw)
    for n in (3, 30):
        o.step(n)
        s.step(n)
        _, vo = o.moments()
        _, vg = s.moments()
        assert_parity(vel_err(vg, vo), storage)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_inplace_cube_channel_inlet_outlet(storage):
    """Inlet / outlet planes (rebuilt after every step in the current layout)
    with bounce-back side walls on the smoothed cube channel."""
    eps, kap = workloads.cube_channel(48, 24, 24, side=12, eps_cube=0.4, Da=1e-4, smooth=4)
    kw = dict(nu_f=0.02, forch=0.55)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, wall=(2, 1, 1), v_in=(0.05, 0, 0), rho_out=1.0, **kw).init()
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel="split", streaming="in_place", bc=("inflow_outflow", "wall", "wall"),
                       viscosity=0.02, forchheimer=0.55, inlet_v=(0.05, 0, 0), outlet_rho=1.0)
    for n in (25, 75):
        o.step(n)
        s.step(n)
        _, vo = o.moments()
        _, vg = s.moments()
        assert_parity(vel_err(vg, vo), storage)


def test_inplace_moving_walls_bounce_back_density():
    """Moving wet-node walls on y with the bounce-back density, which reads the
    reflected outgoing populations in the unknown slots (AA layout 1 keeps
    them in the node's slot i)."""
    nz, ny, nx = 8, 24, 24
    eps = workloads.random_smooth_porosity((nz, ny, nx), seed=44, lo=0.5, hi=0.95)
    eps[:, :3, :] = 0.7
    eps[:, -3:, :] = 0.7
    kap = workloads.carman_kappa(eps, 2.0)
    wv = ((-0.02, 0.0, 0.0), (0.02, 0.0, 0.0))
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=0.05, wall=(0, 3, 0), b=(0, -5e-4, 0), forch=-1.0, wall_v=wv,
                      plane_density=lbm.DENSITY["bounce_back"]).init()
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp32", kernel="split", streaming="in_place", bc=("periodic", "moving_walls", "periodic"),
                       viscosity=0.05, force=(0, -5e-4, 0), forchheimer=-1.0, wall_v=wv, plane_density="bounce_back")
    m0 = s.reduce()["mass"]
    for n in (11, 50):
        o.step(n)
        s.step(n)
        _, vo = o.moments()
        _, vg = s.moments()
        assert vel_err(vg, vo) <= TOL["fp32"]
    # the closed channel keeps its mass (FP32 storage rounding only)
    assert abs(s.reduce()["mass"] / m0 - 1) < 1e-6


def test_inplace_checkpoint_and_populations_at_odd_parity(tmp_path):
    eps = workloads.random_smooth_porosity(BOX, seed=45, lo=0.4, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    kw = dict(nu_f=0.02, b=(6e-4, 0, 0), forch=-1.0)
    a = _sim(eps, kap, "fp32", **kw)
    a.step(7)  # odd: the in-place layout is the shifted one
    path = os.fspath(tmp_path / "odd.ckpt")
    a.save(path)
    b = lbm.Simulation.load(path)
    assert b.info()["in_place"]
    f7 = a.get_populations()
    np.testing.assert_array_equal(b.get_populations(), f7)
    # setting the populations it just read changes nothing
    c = _sim(eps, kap, "fp32", **kw)
    c.step(7)
    c.set_populations(f7)
    for s in (a, b, c):
        s.step(5)
    fa = a.get_populations()
    np.testing.assert_array_equal(b.get_populations(), fa)
    np.testing.assert_array_equal(c.get_populations(), fa)
    # and the state is the oracle's
    o = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init().step(12)
    assert vel_err(a.moments()[1], o.moments()[1]) <= TOL["fp32"]


def test_inplace_allocates_one_population_array():
    """The sweep path double-buffers; the in-place split path holds one
    population array (plus its padded porosity for the tiled copies)."""
    import torch

    shape = (16, 16, 64)
    eps = workloads.random_smooth_porosity(shape, seed=46, lo=0.4, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    kw = dict(nu_f=0.02, b=(6e-4, 0, 0), forch=-1.0)
    used = {}
    for kernel in ("split", "sweep"):
        s = _sim(eps, kap, "fp32", kernel=kernel, **kw)
        used[kernel] = sum(s._alloc.live.values())
        s.close()
        torch.cuda.synchronize()
    nz, ny, nx = shape
    pop = 27 * eps.size * 4
    pad = (nx + 8) * (ny + 2) * (nz + 2) * 4
    assert used["sweep"] - used["split"] == pop - pad


def test_inplace_bounded_wait_runs_out_and_is_sticky():
    """The test-only probe makes one block wait on a barrier that no copy will
    complete; the wait gives up after ~20 us (no fault, nothing in flight), the
    step reports LBM_E_TIMEOUT, and the context keeps reporting it."""
    eps = workloads.random_smooth_porosity((8, 8, 64), seed=47, lo=0.5, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp32", kernel="split", viscosity=0.02, force=(1e-4, 0, 0),
                       forchheimer=-1.0, wait_probe=True, streaming="in_place")
    s.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        s.sync()
    assert ei.value.code == -6
    with pytest.raises(lbm.LbmError) as ei:
        s.step(1)
    assert ei.value.code == -6
    # a context without the probe on the same device still works
    t = lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp32", kernel="split", viscosity=0.02, force=(1e-4, 0, 0),
                       forchheimer=-1.0, streaming="in_place")
    t.step(3).sync()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_inplace_full_size_porous_box_one_step(storage):
    """256^3 porous box in the launch configuration bench.py times: from the GPU
    state after 21 steps (odd: the shifted layout), one more GPU step matches
    one oracle step from the same populations at every node."""
    shape = (256, 256, 256)
    eps, kap = workloads.porous_box(shape, ell=16.0, seed=2)
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel="split", viscosity=0.02, force=(6e-4, 0, 0),
                       forchheimer=-1.0, streaming="in_place")
    s.step(21)
    f0 = s.get_populations()
    s.step(1)
    _, vg = s.moments()
    o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=0.02, b=(6e-4, 0, 0), forch=-1.0)
    o.set_f(f0)
    del f0
    o.step(1)
    _, vo = o.moments()
    assert_parity(vel_err(vg, vo), storage)


def test_streaming_choice():
    """AUTO streams in place only when two population arrays would crowd the
    device; TWO_ARRAYS and IN_PLACE are honoured; IN_PLACE needs nx even."""
    eps = workloads.random_smooth_porosity((8, 8, 64), seed=48, lo=0.5, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    kw = dict(storage="fp32", kernel="split", viscosity=0.02, force=(1e-4, 0, 0), forchheimer=-1.0)
    assert not lbm.Simulation(lbm.D3Q27, eps, kap, **kw).info()["in_place"]
    assert not lbm.Simulation(lbm.D3Q27, eps, kap, streaming="two_arrays", **kw).info()["in_place"]
    assert lbm.Simulation(lbm.D3Q27, eps, kap, streaming="in_place", **kw).info()["in_place"]
    odd = workloads.random_smooth_porosity((8, 8, 63), seed=48, lo=0.5, hi=0.95)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Simulation(lbm.D3Q27, odd, workloads.carman_kappa(odd, 2.0), streaming="in_place", **kw)
    assert ei.value.code == -5
