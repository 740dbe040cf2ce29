"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
symbol that include/nbcore.h declares.  No compute calls (no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    hdr = open(os.path.join(ROOT, "include", "nbcore.h")).read()
    return re.findall(r"^(?:const char\*|nb_status|void|int64_t|int32_t)\s+(\w+)\s*\(", hdr, re.M)


def test_header_declares_the_hot_path_calls():
    names = set(header_functions())
    for n in ("nl_build", "nonbonded_forces", "pme_spread", "pme_gather", "md_step", "hmc_trajectory",
              "hmc_trajectory_backward", "nonbonded_force_vjp"):
        assert n in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2503_20541_b300 import build, nbcore
    try:
        build.build()
    except RuntimeError as e:  # no toolkit on this machine
        pytest.skip(str(e))
    lib = nbcore.load()
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(set(names)) == sorted(nbcore.EXPORTS)
    assert lib.nb_status_str(2) == b"periodic box edge smaller than 2 r_nl"


def test_create_rejects_bad_arguments_without_a_gpu():
    """Argument validation happens on the host before any device call."""
    from paper_2503_20541_b300 import nbcore
    lib = nbcore.load()
    d = (nbcore.SystemDesc * 1)()
    d[0].n_atoms = 10
    d[0].periodic = 1
    for k in range(3):
        d[0].box[k] = 4.0
    d[0].r_cut = 2.5
    d[0].r_skin = 0.3
    d[0].r_switch = -1.0
    sig = np.ones(10, np.float32)
    h = ctypes.c_void_p()
    st = lib.nb_create(ctypes.byref(h), d, 1, sig.ctypes.data, sig.ctypes.data, None, None, None)
    assert st == 2  # NB_ERR_BOX_TOO_SMALL: 4 < 2 * 2.8
    for k in range(3):
        d[0].box[k] = 10.0
    d[0].pme_grid[0] = 16  # partial PME mesh
    st = lib.nb_create(ctypes.byref(h), d, 1, sig.ctypes.data, sig.ctypes.data, None, None, None)
    assert st == 1
    d[0].pme_grid[0] = 0
    opt = nbcore.Options(0, 12, 0, 0)  # stencil_tile must be a multiple of 64 in [256, 4096]
    st = lib.nb_create(ctypes.byref(h), d, 1, sig.ctypes.data, sig.ctypes.data, None, None, ctypes.byref(opt))
    assert st == 1


def test_workload_scalars_are_fp32_exact():
    from paper_2503_20541_b300 import workloads as wl
    for s in (wl.water_box(), wl.lj_fcc(), wl.lj_random(500)):
        for v in list(s.box) + [s.r_cut, s.r_skin, s.alpha, s.ke]:
            assert float(np.float32(v)) == v


@pytest.mark.parametrize("mesh", [(1 << 22, 1 << 21, 1 << 21), (1 << 21, 1 << 21, 1 << 21), (2048, 1024, 1024),
                                  (1 << 30, 4, 4), (4, 4, (1 << 20) + 1)])
def test_static_spread_refuses_oversized_meshes_before_any_gpu_work(mesh):
    """pme_spread_static checks every mesh size against its static capacity before it
    multiplies them (a product of three int32 sizes can wrap to 0) and before any device
    call, so the refusal needs no GPU; the pointers are never dereferenced."""
    from paper_2503_20541_b300 import nbcore
    lib = nbcore.load()
    box = np.array([10.0, 10.0, 10.0])
    m = np.array(mesh, np.int32)
    dummy = ctypes.c_void_p(16)
    assert lib.pme_spread_static(dummy, 4, box.ctypes.data, m.ctypes.data, dummy, None) == 1
