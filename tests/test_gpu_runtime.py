"""Runtime features on the GPU: checkpoint / resume."""
import numpy as np
import pytest

import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("storage,kernel", [("fp64", "sweep"), ("fp32", "fused"), ("fp16", "fused")])
def test_checkpoint_resume_is_bitwise(tmp_path, storage, kernel):
    """2n steps equal n steps, save, load, n steps, bit for bit."""
    shape = (20, 18, 30)
    eps, kap = workloads.porous_box(shape, ell=6.0, seed=3)
    kw = dict(viscosity=0.02, force=(6e-4, 0, 0), forchheimer=lbm.F_ERGUN, storage=storage, kernel=kernel,
              bc=("periodic", "wall", "periodic"))
    a = lbm.Simulation(lbm.D3Q27, eps, kap, **kw)
    a.step(40)
    b = lbm.Simulation(lbm.D3Q27, eps, kap, **kw)
    b.step(20)
    path = str(tmp_path / "ck.plbm")
    b.save(path)
    b.close()
    c = lbm.Simulation.load(path)
    assert c.reduce()["steps"] == 20
    c.step(20)
    np.testing.assert_array_equal(c.get_populations(), a.get_populations())
    ra, va = a.moments()
    rc, vc = c.moments()
    np.testing.assert_array_equal(vc, va)


@pytest.mark.parametrize("case", ["cavity", "cylinder"])
def test_checkpoint_keeps_boundary_options(tmp_path, case):
    """The checkpoint carries the boundary options (wet side walls, regularised
    lid, bounce-back density; Poiseuille inlet, zero-gradient outlet): a
    reloaded context continues bit for bit."""
    if case == "cavity":
        eps, kap = workloads.porous_cavity(L=31, D=17.0, eps_core=0.5)
        kw = dict(viscosity=0.05, forchheimer=lbm.F_ERGUN, storage="fp32", kernel="split",
                  bc=("moving_walls", "moving_walls", "periodic"), wall_v=((0, 0, 0), (0.05, 0, 0)),
                  lid_profile="regularised", lid_delta=0.1, plane_density="bounce_back")
    else:
        eps, kap = workloads.porous_cylinder(D=6, eps_core=0.5, L_over_D=22.5)
        kw = dict(viscosity=0.03, forchheimer=lbm.F_ERGUN, storage="fp32", kernel="split",
                  bc=("inflow_outflow", "moving_walls", "periodic"), inlet_v=(0.05, 0, 0),
                  inlet_profile="poiseuille", outlet="zero_gradient")
    e3 = np.ascontiguousarray(np.broadcast_to(eps, (4,) + eps.shape[1:]))
    k3 = np.ascontiguousarray(np.broadcast_to(kap, (4,) + kap.shape[1:]))
    a = lbm.Simulation(lbm.D3Q27, e3, k3, **kw)
    a.step(40)
    b = lbm.Simulation(lbm.D3Q27, e3, k3, **kw)
    b.step(20)
    path = str(tmp_path / "ck.plbm")
    b.save(path)
    b.close()
    c = lbm.Simulation.load(path)
    c.step(20)
    np.testing.assert_array_equal(c.get_populations(), a.get_populations())


def case_bytes(shape, storage_bytes):
    """The device footprint the server charges a case (one population array,
    porosity, permeability, 22 scratch values, the residual snapshot, the
    padded porosity of the tiled copies and 4 MiB of small buffers)."""
    nz, ny, nx = shape
    return nx * ny * nz * (27 * storage_bytes + 25 * 4) + (nx + 8) * (ny + 2) * (nz + 2) * 4 + 4 * 2**20


def _cases():
    out = []
    for k, shape in enumerate([(16, 16, 16), (24, 20, 24), (12, 28, 32)]):
        eps = workloads.random_smooth_porosity(shape, seed=40 + k, lo=0.5, hi=0.95, ell=3.0)
        out.append((eps, workloads.carman_kappa(eps, 2.0)))
    return out


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_server_results_equal_alone_and_in_the_mix(storage):
    """Continuous batching: each case's result is bitwise the same when it runs
    alone and in a mix of uneven cases (same batched kernels), and bitwise the
    same as a single-case in-place simulation stepped the same number of steps."""
    kw = dict(viscosity=0.05, force=(1e-4, 0, 0), forchheimer=lbm.F_ERGUN, tol=1e-4, max_steps=20000)
    mix = lbm.Server(storage=storage, hbm_cap_bytes=4e9, check_every=100)
    ids = [mix.submit(e, k, **kw) for e, k in _cases()]
    done = {}
    while len(done) < len(ids):
        res, active, queued = mix.run(batches=1)
        for r in res:
            done[r["id"]] = r
    mix.close()
    for (e, k), i in zip(_cases(), ids):
        r = done[i]
        assert r["status"] in (0, 1)  # below tol, or at the storage noise floor
        assert r["residual"] < (1e-4 if r["status"] == 0 else 2e-3)
        alone = lbm.Server(storage=storage, hbm_cap_bytes=4e9, check_every=100)
        j = alone.submit(e, k, **kw)
        ra = None
        while ra is None:
            res, _, _ = alone.run(batches=1)
            ra = next((x for x in res if x["id"] == j), None)
        alone.close()
        assert ra["steps"] == r["steps"]
        assert ra["mean_v"] == r["mean_v"]
        # the batched kernels do the single-case in-place split kernels' arithmetic
        sim = lbm.Simulation(lbm.D3Q27, e, k, viscosity=0.05, force=(1e-4, 0, 0), forchheimer=lbm.F_ERGUN,
                             storage=storage, kernel="split", streaming="in_place")
        sim.step(r["steps"])
        assert sim.reduce()["mean_v"] == r["mean_v"]
        assert r["k_app"] == pytest.approx(0.05 * r["mean_v"][0] / 1e-4, rel=1e-12)


def test_server_admission_respects_the_memory_cap():
    """With a cap that holds one case at a time, cases run one after another."""
    kw = dict(viscosity=0.05, force=(1e-4, 0, 0), forchheimer=lbm.F_ERGUN, tol=1e-4, max_steps=20000)
    cases = _cases()
    cap = 1.5 * max(case_bytes(e.shape, 2) for e, _ in cases)
    srv = lbm.Server(storage="fp16", hbm_cap_bytes=cap, check_every=100)
    for e, k in cases:
        srv.submit(e, k, **kw)
    seen_active = 0
    finished = 0
    while finished < len(cases):
        res, active, queued = srv.run(batches=1)
        seen_active = max(seen_active, active)
        finished += len(res)
        assert srv.stats()["used_bytes"] <= cap
    assert seen_active == 1
    srv.close()


def test_server_large_case_runs_its_own_kernels_with_the_same_result():
    """A case of 2^20 nodes or more runs the single-case kernels inside the
    batch's graph while the small cases share the batched kernels; every
    result is bitwise that of a single-case in-place simulation stepped the
    same number of steps, and a batch with both kinds issues one launch of
    each batched kernel plus the large case's own three per step."""
    kw = dict(viscosity=0.05, force=(1e-4, 0, 0), forchheimer=lbm.F_ERGUN, tol=1e-4, max_steps=3000)
    big = (64, 128, 128)  # 2^20 nodes
    eb = workloads.random_smooth_porosity(big, seed=77, lo=0.5, hi=0.95, ell=4.0)
    cases = _cases()[:2] + [(eb, workloads.carman_kappa(eb, 2.0))]
    srv = lbm.Server(storage="fp16", hbm_cap_bytes=8e9, check_every=100)
    ids = [srv.submit(e, k, **kw) for e, k in cases]
    done = {}
    res, active, queued = srv.run(batches=1)
    assert active == 3 and srv.stats()["kernel_launches"] == 3 * 100 * 2
    for r in res:
        done[r["id"]] = r
    while len(done) < len(ids):
        res, active, queued = srv.run(batches=1)
        for r in res:
            done[r["id"]] = r
    srv.close()
    for (e, k), i in zip(cases, ids):
        r = done[i]
        assert r["status"] in (0, 1, -1)
        sim = lbm.Simulation(lbm.D3Q27, e, k, viscosity=0.05, force=(1e-4, 0, 0), forchheimer=lbm.F_ERGUN,
                             storage="fp16", kernel="split", streaming="in_place")
        sim.step(r["steps"])
        assert sim.reduce()["mean_v"] == r["mean_v"]
        sim.close()
