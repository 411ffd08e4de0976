"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects invalid input before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2606_29619_b300 as lbm
from paper_2606_29619_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)) - {"lbm_alloc_fn", "lbm_free_fn"})


def test_header_declares_binding_exports():
    assert sorted(lbm.EXPORTS) == declared_symbols()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_default_params(lib):
    p = lbm.LbmParams()
    lib.lbm_default_params(ctypes.byref(p))
    assert p.storage == lbm.STORAGE["fp32"]
    assert p.RT == pytest.approx(1 / 3)
    assert p.J_nu == 1.0 and p.J_eta == 1.0 and p.rho0 == 1.0
    assert p.corrections == lbm.CORR_FULL
    assert list(p.bc) == [0, 0, 0]
    assert p.outlet == 0 and p.inlet_profile == 0


def test_error_codes_match_header():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    codes = {int(v): k for k, v in re.findall(r"#define (LBM_E_[A-Z_]+) \((-\d+)\)", text)}
    assert codes == lbm.ERRORS


def test_params_layout_matches_header(tmp_path):
    """The ctypes mirror of lbm_params has the C struct's size and field offsets
    (a small C program compiled against include/lbm.h prints them)."""
    names = [f[0] for f in lbm.LbmParams._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(lbm_params));']
    lines += [f'  printf("%zu\\n", offsetof(lbm_params, {n}));' for n in names]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(lbm.LbmParams)
    for n, off in zip(names, out[1:]):
        assert getattr(lbm.LbmParams, n).offset == off, n


def _create(lib, eps, kap, lattice=1, dims=None, visc=0.1, forch=0.0, params=None):
    eps = np.ascontiguousarray(eps, np.float64)
    kap = np.ascontiguousarray(kap, np.float64)
    nz, ny, nx = dims if dims else eps.shape
    h = ctypes.c_void_p()
    f = np.zeros(3)
    P = ctypes.POINTER(ctypes.c_double)
    rc = lib.lbm_create(ctypes.byref(h), lattice, nx, ny, nz, eps.ctypes.data_as(P), kap.ctypes.data_as(P),
                        forch, visc, f.ctypes.data_as(P), ctypes.byref(params) if params else None)
    return rc, h, lib.lbm_last_error().decode()


@pytest.mark.parametrize("case", ["eps0", "eps_gt1", "kappa_neg", "kappa_nan", "visc0", "nz_d2q9", "small_axis",
                                  "bad_storage", "bad_lattice", "bad_outlet", "outlet_without_planes",
                                  "bad_inlet_profile", "poiseuille_without_walls"])
def test_invalid_inputs_rejected(lib, case):
    shape = (4, 4, 4)
    eps = np.full(shape, 0.5)
    kap = np.full(shape, 1.0)
    kw = {}
    p = lbm.LbmParams()
    lib.lbm_default_params(ctypes.byref(p))
    if case == "eps0":
        eps[1, 1, 1] = 0.0
    elif case == "eps_gt1":
        eps[0, 0, 0] = 1.01
    elif case == "kappa_neg":
        kap[2, 2, 2] = -1.0
    elif case == "kappa_nan":
        kap[2, 2, 2] = np.nan
    elif case == "visc0":
        kw["visc"] = 0.0
    elif case == "nz_d2q9":
        kw["lattice"] = 0
    elif case == "small_axis":
        p.bc[1] = 1  # a wall axis needs 4 nodes
        eps, kap = eps[:, :3], kap[:, :3]
    elif case == "bad_storage":
        p.storage = 9
    elif case == "bad_lattice":
        kw["lattice"] = 5
    elif case == "bad_outlet":
        p.outlet = 2
    elif case == "outlet_without_planes":
        p.outlet = 1
    elif case == "bad_inlet_profile":
        p.inlet_profile = 7
    elif case == "poiseuille_without_walls":
        p.inlet_profile = 1
    rc, h, msg = _create(lib, eps, kap, params=p, **kw)
    assert rc == -1, msg
    assert not h.value
    assert msg


def test_destroy_null_is_noop(lib):
    lib.lbm_destroy(None)


def test_tune_cache_roundtrip(lib, tmp_path):
    """The autotuner's JSON-lines cache: absent file and key give 0, the last
    line of a key wins, unparsable lines are skipped, other keys are kept apart."""
    import json

    path = str(tmp_path / "tune.jsonl")
    assert lbm.tune_cache_lookup(path, "D3Q27/fp32/two_arrays/2^24/B300") == 0
    lbm.tune_cache_store(path, "D3Q27/fp32/two_arrays/2^24/B300", 4, {2: 1.25, 4: 1.125, 8: 1.5})
    lbm.tune_cache_store(path, "D3Q27/fp16/in_place/2^24/B300", 2)
    with open(path, "a") as fh:
        fh.write('{"key": "D3Q27/fp32/two_arrays/2^24/B300", "tile_y": \n')  # torn line
        fh.write("not json at all\n")
    assert lbm.tune_cache_lookup(path, "D3Q27/fp32/two_arrays/2^24/B300") == 4
    assert lbm.tune_cache_lookup(path, "D3Q27/fp16/in_place/2^24/B300") == 2
    assert lbm.tune_cache_lookup(path, "D3Q27/fp16/in_place/2^24/B30") == 0
    lbm.tune_cache_store(path, "D3Q27/fp32/two_arrays/2^24/B300", 8, {8: 0.9})
    assert lbm.tune_cache_lookup(path, "D3Q27/fp32/two_arrays/2^24/B300") == 8
    first = json.loads(open(path).read().splitlines()[0])
    assert first == {"key": "D3Q27/fp32/two_arrays/2^24/B300", "tile_y": 4, "candidates": [2, 4, 8],
                     "ms_per_step": [1.25, 1.125, 1.5]}


@pytest.mark.parametrize("key,tile", [('bad"key', 4), ("bad\\key", 4), ("", 4), ("ok", 3), ("ok", 16)])
def test_tune_cache_rejects_bad_arguments(lib, tmp_path, key, tile):
    with pytest.raises(lbm.LbmError) as e:
        lbm.tune_cache_store(str(tmp_path / "t.jsonl"), key, tile)
    assert e.value.code == -1


def test_create_rejects_bad_tile_height(lib):
    eps = np.full((4, 8, 8), 0.8)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(lbm.D3Q27, eps, np.ones_like(eps), viscosity=0.1, tile_y=3, torch_allocator=False)
    assert e.value.code == -1
