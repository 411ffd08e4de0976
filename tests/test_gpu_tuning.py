"""The autotuner of the split kernels' tile height (rows of 64 nodes per block).

* Every candidate height computes the same arithmetic per node: populations
  after several steps are bitwise equal to those of the default height, on
  both streaming forms and at FP32 and FP16, with ragged x and y tiles.
* Each candidate height passes parity against the FP64 oracle.
* autotune=True times the candidates, keeps the fastest, caches the choice in
  a JSON-lines file and restores the initial state; a second context with the
  same cache file takes the stored choice without timing.
* A forced height on a grid the heights do not apply to (walls) is refused.
"""
import json
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


def box(shape=(12, 36, 48), seed=7):
    eps = workloads.random_smooth_porosity(shape, seed=seed, lo=0.45, hi=0.95)
    return eps, workloads.carman_kappa(eps, 2.0)


def sim(eps, kap, storage, streaming, **kw):
    return lbm.Simulation(lbm.D3Q27, eps, kap, storage=storage, kernel="split", viscosity=0.03,
                          force=(6e-4, 2e-4, -1e-4), forchheimer=lbm.F_ERGUN, streaming=streaming, **kw)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("streaming", ["two_arrays", "in_place"])
@pytest.mark.parametrize("tile_y", [2, 8])
def test_tile_heights_are_bitwise_equal(storage, streaming, tile_y):
    # nx = 48: one ragged 64-node x tile; ny = 36: ragged for 8 rows
    eps, kap = box()
    ref = sim(eps, kap, storage, streaming)
    s = sim(eps, kap, storage, streaming, tile_y=tile_y)
    assert ref.tuning()["tile_y"] == 4 and s.tuning()["tile_y"] == tile_y
    ref.step(7)
    s.step(7)
    assert np.array_equal(s.get_populations(), ref.get_populations())
    ref.close()
    s.close()


@pytest.mark.parametrize("tile_y", [2, 4, 8])
def test_tile_heights_pass_oracle_parity(tile_y):
    eps, kap = box((10, 24, 32), seed=9)
    kw = dict(nu_f=0.03, b=(6e-4, 2e-4, -1e-4), forch=-1.0)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init()
    o.step(30)
    for storage in ("fp32", "fp16"):
        s = sim(eps, kap, storage, "auto", tile_y=tile_y)
        s.step(30)
        assert_parity(vel_err(s.moments()[1], o.moments()[1]), storage)
        s.close()


def test_autotune_times_caches_and_restores(tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    eps, kap = box((32, 64, 64), seed=3)
    fresh = sim(eps, kap, "fp32", "two_arrays")
    f0 = fresh.get_populations()
    fresh.step(5)
    f5 = fresh.get_populations()
    fresh.close()
    s = sim(eps, kap, "fp32", "two_arrays", autotune=True, tune_cache=cache)
    t = s.tuning()
    assert t["source"] == "timed"
    assert sorted(t["candidates"]) == [2, 4, 8]
    assert t["tile_y"] == min(t["candidates"], key=t["candidates"].get)
    assert all(ms > 0 for ms in t["candidates"].values())
    # the timed steps left no trace: the state is the initial one and steps like a fresh context
    assert np.array_equal(s.get_populations(), f0)
    s.step(5)
    assert np.array_equal(s.get_populations(), f5)
    assert s.reduce()["steps"] == 5
    s.close()
    lines = [json.loads(x) for x in open(cache).read().splitlines()]
    assert len(lines) == 1 and lines[0]["tile_y"] == t["tile_y"] and lines[0]["candidates"] == [2, 4, 8]
    key = lines[0]["key"]
    assert key.startswith("D3Q27/fp32/two_arrays/2^17/")
    assert lbm.tune_cache_lookup(cache, key) == t["tile_y"]
    s2 = sim(eps, kap, "fp32", "two_arrays", autotune=True, tune_cache=cache)
    t2 = s2.tuning()
    assert t2["source"] == "cache" and t2["tile_y"] == t["tile_y"] and t2["candidates"] == {}
    s2.close()
    # another streaming form is another key: timed again
    s3 = sim(eps, kap, "fp32", "in_place", autotune=True, tune_cache=cache)
    assert s3.tuning()["source"] == "timed"
    s3.close()
    assert len(open(cache).read().splitlines()) == 2


def test_forced_tile_height_needs_a_periodic_grid():
    eps, kap = box()
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp32", kernel="split", bc=("periodic", "wall", "periodic"),
                       viscosity=0.03, tile_y=8)
    assert e.value.code == -5
    # walls: the heights do not apply and the default is reported
    s = lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp32", kernel="split", bc=("periodic", "wall", "periodic"),
                       viscosity=0.03, autotune=True)
    assert s.tuning() == {"tile_y": 4, "candidates": {}, "source": "default"}
    s.close()
