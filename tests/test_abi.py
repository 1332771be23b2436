"""The C-ABI library builds, loads and exports every symbol include/gbmd.h declares;
host-side argument checks run without a GPU (no compute is launched here)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbmd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1308_5587_gb300 import _build, gbmd
    _build.build()
    return gbmd


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gbmd_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("gbmd_create", "gbmd_step", "gbmd_get_forces", "gbmd_get_thermo",
                 "gbmd_get_state", "gbmd_set_state", "gbmd_get_neighbors",
                 "gbmd_footprint_bytes", "gbmd_batch_create", "gbmd_batch_add",
                 "gbmd_batch_remove", "gbmd_batch_step", "gbmd_autotune", "gbmd_destroy",
                 "gbmd_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared() if not hasattr(so, n)]
    assert not missing, missing
    assert set(declared()) <= set(lib._SIGS)


def test_abi_version(lib):
    assert lib.gbmd_abi_version() == 6


def _desc(lib, **over):
    n = over.pop("n", 4)
    pos = over.pop("pos", np.zeros((n, 3)))
    vel = np.zeros((n, 3))
    kw = dict(box=over.pop("box", 20.0), types=over.pop("types", None), eps=over.pop("eps", 1.0),
              sigma=over.pop("sigma", 1.0), rcut=over.pop("rcut", 2.5), r_buff=0.4,
              dt=over.pop("dt", 0.005),
              mass=1.0, precision=over.pop("precision", "mixed"))
    return lib.make_desc(n, kw["box"], pos, vel, kw["types"], kw["eps"], kw["sigma"], kw["rcut"],
                         kw["r_buff"], kw["dt"], kw["mass"], kw["precision"], **over)


@pytest.mark.parametrize("bad,status", [
    (dict(dt=0.0), "BAD_ARG"),
    (dict(dt=-1.0), "BAD_ARG"),
    (dict(box=5.0), "BOX_TOO_SMALL"),
    (dict(rcut=-1.0), "BAD_ARG"),
    (dict(precision=7), "BAD_ARG"),
    (dict(types=np.array([0, 1, 0, 0], np.int32)), "BAD_ARG"),      # type >= ntypes
    (dict(pos=np.full((4, 3), np.nan)), "BAD_ARG"),
    (dict(threads_per_particle=3), "BAD_ARG"),
    (dict(force_path=2), "BAD_ARG"),
    (dict(n=0), "BAD_ARG"),                                           # empty system
    (dict(integrator=1, kT=0.0, tau=1.0), "BAD_ARG"),                 # NVT without kT
    (dict(integrator=1, kT=1.0, tau=-1.0), "BAD_ARG"),
    (dict(integrator=2), "BAD_ARG"),
    (dict(eps=np.array([[1.0, 2.0], [1.5, 1.0]])), "BAD_ARG"),     # not symmetric
    (dict(potential=5), "BAD_ARG"),
    (dict(potential="mie"), "BAD_ARG"),                               # no exponents
    (dict(potential="mie", mie_n=6.0, mie_m=6.0), "BAD_ARG"),         # needs n > m
    (dict(potential="mie", mie_n=12.0, mie_m=0.0), "BAD_ARG"),
    (dict(potential="yukawa"), "BAD_ARG"),                            # no kappa
    (dict(potential="yukawa", kappa=-1.0), "BAD_ARG"),
    (dict(potential="yukawa", kappa=1.0, eps=0.0), "BAD_ARG"),
    (dict(potential="yukawa", kappa=np.array([[1.0, 2.0], [1.0, 1.0]]),
          eps=np.ones((2, 2))), "BAD_ARG"),                           # kappa not symmetric
    (dict(potential="gauss", sigma=None), "BAD_ARG"),
    (dict(potential="wca", sigma=None, rcut=None), "BAD_ARG"),
    (dict(potential="lj", rcut=None), "BAD_ARG"),
    (dict(potential="mie", mie_n=12.0, mie_m=6.0, eps=-1.0), "BAD_ARG"),
    (dict(potential="wca", rcut=None, box=3.0), "BOX_TOO_SMALL"),     # 2 (2^(1/6) + 0.4) > 3
    (dict(nlist=2), "BAD_ARG"),
    (dict(nlist="tree", types=np.array([0, 1, 0, 0], np.int32)), "BAD_ARG"),
])
def test_create_rejects_bad_arguments_on_the_host(lib, bad, status):
    d, keep = _desc(lib, **bad)
    with pytest.raises(lib.GbmdError) as e:
        lib.gbmd_create(d)
    assert e.value.status == status
    assert lib.gbmd_last_error()


def test_null_arguments(lib):
    L = lib.load()
    import ctypes
    assert L.gbmd_create(None, ctypes.byref(ctypes.c_void_p())) == -1
    assert L.gbmd_step(None, 1) == -1
    assert L.gbmd_destroy(None) == -1
    assert "NULL" in lib.gbmd_last_error()


def test_footprint_is_host_side_and_monotone(lib):
    a, k1 = _desc(lib, n=1000, box=12.0)
    b, k2 = _desc(lib, n=8000, box=24.0)
    fa, fb = lib.gbmd_footprint_bytes(a), lib.gbmd_footprint_bytes(b)
    assert 0 < fa < fb
    # about 0.7-1.2 KB per particle for the default capacity at liquid density
    assert 300 < fb / 8000 < 3000


def test_footprint_follows_the_potential_cut(lib):
    """WCA reads no rcut table: its cut is 2^(1/6) sigma, so its list is shorter."""
    lj, k1 = _desc(lib, n=8000, box=24.0)
    wca, k2 = _desc(lib, n=8000, box=24.0, potential="wca", rcut=None)
    yuk, k3 = _desc(lib, n=8000, box=24.0, potential="yukawa", sigma=None, kappa=1.0)
    f_lj, f_wca = lib.gbmd_footprint_bytes(lj), lib.gbmd_footprint_bytes(wca)
    assert 0 < f_wca < f_lj
    assert lib.gbmd_footprint_bytes(yuk) == f_lj   # same r_cut, same layout


def test_footprint_of_the_tree_list(lib):
    """The tree list's cells only order the particles (finer grid, type-major bins)
    and it holds its boxes, sort keys and leaf copies: about 56 bytes per particle more."""
    cell, k1 = _desc(lib, n=8000, box=24.0)
    tree, k2 = _desc(lib, n=8000, box=24.0, nlist="tree")
    fc, ft = lib.gbmd_footprint_bytes(cell), lib.gbmd_footprint_bytes(tree)
    assert 8000 * 40 < ft - fc < 8000 * 80


def test_probe_rejects_bad_arguments_before_any_launch(lib):
    for kind, iters in ((7, 10), (-1, 10), (0, 0), (1, -5)):
        with pytest.raises(lib.GbmdError) as e:
            lib.gbmd_probe_arith(kind, iters)
        assert e.value.status == "BAD_ARG"


@pytest.mark.parametrize("over,msg", [
    (dict(n_ghost=-1), "n_ghost"),
    (dict(n_ghost=4), "n_ghost"),
    (dict(n_ghost=1, integrator="nvt", kT=1.0, tau=1.0), "ghosts need"),
    (dict(n_ghost=1, force_path="staged"), "ghosts need"),
])
def test_ghost_arguments_are_checked_on_the_host(lib, over, msg):
    d, keep = _desc(lib, **over)
    with pytest.raises(lib.GbmdError) as e:
        lib.gbmd_create(d)
    assert e.value.status == "BAD_ARG" and msg in str(e.value)


def test_ghost_calls_reject_null_arguments(lib):
    with pytest.raises(lib.GbmdError):
        lib.gbmd_set_ghost_positions(None, np.zeros((1, 3)))
    import ctypes
    so = lib.load()
    assert so.gbmd_get_positions(None, None, 0, None, 0) == -1
