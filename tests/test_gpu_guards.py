"""No kernel writes outside the device memory the library allocated.

A test allocator, passed through the ABI's allocator callbacks, pads every
allocation with guard bands of a known byte pattern on both sides.  Every
kernel path runs on tiny and ragged grids (periodic and walled, inlet/outlet
planes, two population arrays and in-place streaming at both parities, every
storage form and tile height, the sweep, split and fused kernels, D2Q9 and
D3Q27), and every guard band must still hold its pattern when the buffer is
freed.  Reads beyond an allocation are not seen by this check; writes are.
"""
import numpy as np
import pytest

import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import workloads

pytestmark = pytest.mark.gpu

GUARD = 1 << 18  # bytes on each side (a multiple of 512: allocations stay aligned)
PATTERN = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_29619_b300 import build

    build.build()


class GuardedAllocator:
    """ALLOC_FN / FREE_FN callbacks over torch tensors with guard bands."""

    def __init__(self):
        import torch

        self.torch = torch
        self.live = {}
        self.violations = []
        self.allocations = 0

        def _alloc(nbytes, _user):
            t = torch.full((int(nbytes) + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda:0")
            ptr = t.data_ptr() + GUARD
            self.live[ptr] = (t, int(nbytes))
            self.allocations += 1
            return ptr

        def _free(ptr, _user):
            if ptr:
                self.check(int(ptr))
                self.live.pop(int(ptr), None)

        self.alloc = lbm.ALLOC_FN(_alloc)
        self.free = lbm.FREE_FN(_free)

    def check(self, ptr):
        t, n = self.live[ptr]
        self.torch.cuda.synchronize()
        lo, hi = t[:GUARD], t[GUARD + n:]
        for name, band in (("below", lo), ("above", hi)):
            bad = (band != PATTERN).nonzero()
            if bad.numel():
                self.violations.append((n, name, int(bad.numel())))

    def check_all(self):
        for ptr in list(self.live):
            self.check(ptr)


def _box(shape, seed):
    eps = workloads.random_smooth_porosity(shape, seed=seed, lo=0.45, hi=0.95, ell=2.0)
    return eps, workloads.carman_kappa(eps, 2.0)


CASES = [
    # (lattice, shape (z, y, x), storage, kernel, streaming, bc, extra)
    (lbm.D3Q27, (6, 5, 16), "fp32", "split", "two_arrays", ("periodic",) * 3, {}),
    (lbm.D3Q27, (6, 5, 16), "fp16", "split", "in_place", ("periodic",) * 3, {}),
    (lbm.D3Q27, (6, 5, 16), "bf16", "split", "two_arrays", ("periodic",) * 3, {"tile_y": 2}),
    (lbm.D3Q27, (5, 9, 16), "fp32", "split", "in_place", ("periodic",) * 3, {"tile_y": 8}),
    (lbm.D3Q27, (5, 7, 10), "fp32", "split", "two_arrays", ("periodic",) * 3, {}),
    (lbm.D3Q27, (5, 7, 9), "fp16", "split", "two_arrays", ("periodic",) * 3, {}),
    (lbm.D3Q27, (6, 6, 16), "fp32", "split", "two_arrays", ("periodic", "wall", "wall"), {}),
    (lbm.D3Q27, (6, 6, 16), "fp16", "split", "in_place", ("wall", "wall", "periodic"), {}),
    (lbm.D3Q27, (6, 6, 16), "fp32", "split", "two_arrays", ("inflow_outflow", "wall", "wall"),
     {"inlet_v": (0.02, 0, 0)}),
    (lbm.D3Q27, (6, 6, 16), "fp16", "split", "in_place", ("inflow_outflow", "wall", "wall"),
     {"inlet_v": (0.02, 0, 0)}),
    (lbm.D3Q27, (5, 6, 8), "fp64", "sweep", "auto", ("periodic", "wall", "periodic"), {}),
    (lbm.D3Q27, (6, 8, 16), "fp32", "fused", "auto", ("periodic",) * 3, {}),
    (lbm.D2Q9, (1, 7, 9), "fp64", "sweep", "auto", ("periodic", "wall", "periodic"), {}),
    (lbm.D2Q9, (1, 6, 10), "fp32", "sweep", "auto", ("inflow_outflow", "wall", "periodic"),
     {"inlet_v": (0.02, 0, 0)}),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_no_write_outside_the_allocations(case):
    lattice, shape, storage, kernel, streaming, bc, extra = CASES[case]
    eps, kap = _box(shape, seed=300 + case)
    if bc[0] == "inflow_outflow":
        # the planes need uniform porosity and permeability over three layers (free fluid here)
        for sl in (slice(0, 3), slice(-3, None)):
            eps[..., sl] = 1.0
            kap[..., sl] = np.inf
    if lattice == lbm.D2Q9:
        eps, kap = eps[0], kap[0]
    g = GuardedAllocator()
    s = lbm.Simulation(lattice, eps, kap, storage=storage, kernel=kernel, streaming=streaming, bc=bc, viscosity=0.04,
                       force=(4e-4, 1e-4, 0.0), forchheimer=lbm.F_ERGUN, allocator=g, **extra)
    for n in (1, 2, 4):  # odd and even step counts: both in-place layouts
        s.step(n)
        s.moments()
        s.reduce(snapshot=True)
    f = s.get_populations()
    s.set_populations(f)
    s.step(3)
    g.check_all()
    s.close()
    assert g.allocations > 0
    assert not g.violations, g.violations
    assert np.isfinite(f).all()


class FailingAllocator(GuardedAllocator):
    """Refuses the k-th request (returns NULL), serves the others."""

    def __init__(self, fail_at):
        super().__init__()
        inner = self.alloc
        self.requests = 0

        def _alloc(nbytes, user):
            self.requests += 1
            if self.requests == fail_at:
                return None
            return inner(nbytes, user)

        self.alloc = lbm.ALLOC_FN(_alloc)


@pytest.mark.parametrize("kernel,streaming,storage", [("split", "two_arrays", "fp32"), ("split", "in_place", "fp16"),
                                                      ("sweep", "auto", "fp64")])
def test_allocator_failure_is_reported_and_frees_everything(kernel, streaming, storage):
    """A NULL from the allocator callback at any of creation's requests makes
    lbm_create return LBM_E_NOMEM with every buffer it already had handed back
    (host-injected fault: nothing fails on the device)."""
    eps, kap = _box((6, 6, 16), seed=9)
    kw = dict(storage=storage, kernel=kernel, streaming=streaming, viscosity=0.04, force=(4e-4, 0, 0),
              forchheimer=lbm.F_ERGUN)
    counting = GuardedAllocator()
    s = lbm.Simulation(lbm.D3Q27, eps, kap, allocator=counting, **kw)
    s.close()
    n = counting.allocations
    assert n >= 3 and not counting.live
    for k in range(1, n + 1):
        g = FailingAllocator(k)
        with pytest.raises(lbm.LbmError) as e:
            lbm.Simulation(lbm.D3Q27, eps, kap, allocator=g, **kw)
        assert e.value.code == -3, (k, e.value)
        assert not g.live, f"request {k} refused: {len(g.live)} buffers not freed"
        assert not g.violations
