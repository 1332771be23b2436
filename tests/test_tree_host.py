"""The tree of the tree neighbour list (csrc/tree_core.cuh) on the CPU: built over
fixed-point coordinates in several orders (cell-like, random, sorted on one axis),
in cubic and elongated boxes, with particles crowding the periodic faces, every
pair within r is found -- against the oracle's brute-force pair search.

The header is compiled for the host with g++ (tests/host/tree_pairs.cpp); the
kernels in k_tree.cu call the same functions on the device."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("tree") / "libtree_pairs.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    os.path.join(HERE, "host", "tree_pairs.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.tree_pairs.restype = C.c_longlong
    lib.tree_pairs.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                               C.c_longlong, C.c_void_p]
    return lib


def fixed(pos, box):
    """positions -> 32-bit fixed point of x/L on [0, 2^32) (the box [-L/2, L/2))"""
    q = np.rint(pos / box * 2.0 ** 32).astype(np.int64)
    return ((q & 0xFFFFFFFF) ^ 0x80000000).astype(np.uint32)


def tree_pairs(lib, u, order, box, r):
    n = u.shape[0]
    u = np.ascontiguousarray(u, np.uint32)
    order = np.ascontiguousarray(order, np.int32)
    box = np.ascontiguousarray(box, np.float64)
    cap = n * (n - 1) // 2 + 16
    pairs = np.zeros((cap, 2), np.int32)
    cnt = lib.tree_pairs(n, u.ctypes.data, order.ctypes.data, box.ctypes.data, r, cap,
                         pairs.ctypes.data)
    assert 0 <= cnt <= cap
    return {(int(a), int(b)) for a, b in pairs[:cnt]}


@pytest.mark.parametrize("n,box,r", [(1000, (10.0, 10.0, 10.0), 2.9), (777, (6.0, 9.0, 12.0), 2.9),
                                     (3000, (30.0, 8.0, 8.0), 1.5), (5, (6.0, 6.0, 6.0), 2.9),
                                     (1, (6.0, 6.0, 6.0), 2.9)])
@pytest.mark.parametrize("how", ["cells", "random", "x_sorted"])
def test_tree_finds_every_pair(lib, n, box, r, how):
    box = np.array(box)
    rng = np.random.default_rng(n)
    pos = rng.uniform(-0.5, 0.5, (n, 3)) * box
    # half the particles crowd the faces x = +-L/2 (pairs across the boundary)
    k = n // 2
    pos[:k, 0] = np.where(rng.random(k) < 0.5, -0.5, 0.5) * box[0] + rng.uniform(-0.3, 0.3, k)
    pos -= box * np.floor(pos / box + 0.5)
    u = fixed(pos, box)
    if how == "cells":   # the order the cell sort gives: by cell, then index
        c = np.floor((pos / box + 0.5) * np.maximum(1, np.floor(box / r))).astype(int)
        order = np.lexsort((np.arange(n), c[:, 0], c[:, 1], c[:, 2]))
    elif how == "random":
        order = rng.permutation(n)
    else:
        order = np.argsort(u[:, 0], kind="stable")
    mine = tree_pairs(lib, u, order, box, r)
    # the oracle at the positions the fixed point represents
    q = (u.astype(np.int64) ^ 0x80000000).astype(np.int64)
    q = np.where(q >= 2 ** 31, q - 2 ** 32, q)
    x = q / 2.0 ** 32 * box
    ref, rr = oracle.neighbors(x, box, None, np.array([[r]]))
    band = np.abs(rr - r) < 1e-9
    want = {(int(a), int(b)) for a, b in ref[~band]}
    amb = {(int(a), int(b)) for a, b in ref[band]}
    assert want <= mine          # nothing missed
    assert mine - want <= amb    # nothing extra outside the 1e-9 band
