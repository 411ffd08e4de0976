"""Slab decomposition along z on CPU ranks (gloo): the host reference of the
multi-GPU exchange.

Each rank owns a z-slab of one periodic D3Q27 domain and steps it with the
three halo exchanges of np_slab (m after the moments, rho and v_z after the
velocity, the crossing populations after collide and stream), sent to its
neighbours with torch.distributed point-to-point messages.  After the steps
every rank's planes must equal the single-domain FP64 oracle's, node by node.
"""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(walls):
    rng = np.random.default_rng(11)
    shape = (10, 5, 6)
    eps = rng.uniform(0.45, 0.95, shape)
    kap = rng.uniform(0.5, 5.0, shape)
    kap[rng.random(shape) < 0.3] = np.inf
    kw = dict(nu_f=0.05, b=(3e-3, -1e-3, 2e-3), forch=-1.0, RT=0.3, J_nu=1.2, J_eta=0.8, wall=walls)
    rho0 = rng.uniform(0.95, 1.05, shape)
    v0 = rng.uniform(-0.02, 0.02, (3,) + shape)
    return eps, kap, kw, rho0, v0


def _rank(rank, world, port, walls, steps, out):
    sys.path.insert(0, HERE)
    sys.path.insert(0, os.path.dirname(HERE))
    import torch
    import torch.distributed as dist

    import oracle
    from np_lbm import NpLBM
    from np_slab import Slab, slab_bounds

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    eps, kap, kw, rho0, v0 = _problem(walls)
    glob = NpLBM(3, eps, kap, **kw).init(rho0, v0)
    z0, z1 = slab_bounds(eps.shape[0], world)[rank]
    slab = Slab(glob, glob.f, z0, z1)
    below, above = (rank - 1) % world, (rank + 1) % world

    def swap(kind, to_below, to_above):
        # tag 0: towards the rank below, tag 1: towards the rank above
        recv_below = torch.empty(to_above.shape, dtype=torch.float64)
        recv_above = torch.empty(to_below.shape, dtype=torch.float64)
        reqs = [dist.isend(torch.from_numpy(np.ascontiguousarray(to_below)), below, tag=0),
                dist.isend(torch.from_numpy(np.ascontiguousarray(to_above)), above, tag=1),
                dist.irecv(recv_below, below, tag=1), dist.irecv(recv_above, above, tag=0)]
        for r in reqs:
            r.wait()
        return recv_below.numpy(), recv_above.numpy()

    from np_slab import step_slab

    for _ in range(steps):
        step_slab(slab, swap)
    o = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init(rho0, v0).step(steps)
    ref = o.get_f()[:, z0:z1]
    out[rank] = float(np.abs(slab.f - ref).max() / np.abs(ref).max())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("walls", [(0, 0, 0), (1, 1, 0)])
def test_slab_decomposition_matches_single_domain(world, walls):
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, walls, 4, out), nprocs=world, join=True)
        errs = dict(out)
    assert sorted(errs) == list(range(world))
    for r, e in errs.items():
        assert e < 1e-14, f"rank {r}: relative difference {e:.2e}"
