"""The allocation-free population sums, called through the C ABI.

lbm_population_sums_noalloc serves callers that may not allocate device memory
(inside a CUDA stream capture, or under a memory pool that forbids library
allocations).  Its mass must equal the mass lbm_reduce reports for the same
state, on consecutive calls that reuse the fixed scratch array.  This file is
collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes

import numpy as np
import pytest

import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import workloads

pytestmark = pytest.mark.gpu


def _sums(torch, lattice, f_host, stream):
    lib = lbm.load_library()
    f_dev = torch.from_numpy(np.ascontiguousarray(f_host.reshape(f_host.shape[0], -1))).to("cuda:0")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda:0")
    n = f_dev.shape[1]
    rc = lib.lbm_population_sums_noalloc(lattice, n, ctypes.c_void_p(f_dev.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("lattice,shape", [(lbm.D3Q27, (12, 14, 16)), (lbm.D2Q9, (1, 40, 30))])
def test_noalloc_sums_match_reduce_on_consecutive_calls(lattice, shape):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps = workloads.random_smooth_porosity(shape, seed=9, lo=0.45, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    walls = ("periodic", "wall", "periodic")
    sim = lbm.Simulation(lattice, eps, kap, storage="fp64", viscosity=0.03, force=(2e-4, 1e-4, 5e-5),
                         forchheimer=lbm.F_ERGUN, bc=walls)
    stream = torch.cuda.Stream()
    c = np.array([[i % 3 - 1, (i // 3) % 3 - 1, (i // 9 - 1) if lattice == lbm.D3Q27 else 0]
                  for i in range(sim.Q)], dtype=np.float64)
    for call in range(2):
        sim.step(25)
        f = sim.get_populations()
        mass = sim.reduce()["mass"]
        out = _sums(torch, lattice, f, stream)
        assert out[0] == pytest.approx(mass, rel=1e-12)
        mom = c.T @ f.reshape(sim.Q, -1).sum(axis=1)
        np.testing.assert_allclose(out[1:], mom, rtol=1e-10, atol=1e-12 * mass)


def test_noalloc_rejects_sizes_beyond_the_limit():
    lib = lbm.load_library()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.lbm_population_sums_noalloc(lbm.D3Q27, (1 << 24) + 1, dummy, dummy, None) == -1
    assert lib.lbm_population_sums_noalloc(lbm.D3Q27, 0, dummy, dummy, None) == -1
    assert lib.lbm_population_sums_noalloc(7, 10, dummy, dummy, None) == -1


def test_noalloc_sums_inside_a_captured_graph():
    """The documented capture pattern: one call outside any capture (it looks
    up the partial-sum array's device address), then calls captured into a CUDA
    graph on the caller's stream.  Replaying the graph after the populations
    change gives the new state's sums, equal to lbm_reduce's mass."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = lbm.load_library()
    shape = (10, 12, 16)
    eps = workloads.random_smooth_porosity(shape, seed=4, lo=0.45, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    sim = lbm.Simulation(lbm.D3Q27, eps, kap, storage="fp64", viscosity=0.03, force=(2e-4, 1e-4, 5e-5),
                         forchheimer=lbm.F_ERGUN)
    n = sim.N
    f_dev = torch.from_numpy(np.ascontiguousarray(sim.get_populations().reshape(sim.Q, -1))).to("cuda:0")
    outs = [torch.full((4,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in range(2)]
    stream = torch.cuda.Stream()

    def call(out):
        return lib.lbm_population_sums_noalloc(lbm.D3Q27, n, ctypes.c_void_p(f_dev.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))

    assert call(outs[0]) == 0
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        assert call(outs[0]) == 0
        assert call(outs[1]) == 0
    for _ in range(2):
        sim.step(20)
        f_dev.copy_(torch.from_numpy(np.ascontiguousarray(sim.get_populations().reshape(sim.Q, -1))))
        for o in outs:
            o.fill_(float("nan"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        mass = sim.reduce()["mass"]
        for o in outs:
            assert o[0].item() == pytest.approx(mass, rel=1e-12)
    sim.close()
