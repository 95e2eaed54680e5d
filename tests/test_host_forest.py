"""The library's host block tree (csrc/forest.cpp), built with g++ behind a small C shim, against
the oracle's forest: treecodes, block order, slots, neighbour tables, adaptation passes, grading
and tiling checks bit-exact; the leaf map against a dictionary.  No GPU is needed."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.forest import Forest as OForest
from paper_1912_05371_gb300.workloads import random_graded_leaves

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1912_05371_gb300", "csrc")

I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("hostforest") / "libhostforest.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, os.path.join(CSRC, "forest.cpp"),
                    os.path.join(HERE, "host", "forest_shim.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    L.hf_create.restype = C.c_void_p
    L.hf_create.argtypes = [C.c_int] * 6 + [C.c_int64]
    L.hf_destroy.argtypes = [C.c_void_p]
    L.hf_apply_pass.argtypes = [C.c_void_p, C.c_int] + [I32] * 4 + [C.c_int] + [I32] * 4 + [I32]
    L.hf_take_slots.argtypes = [C.c_void_p, C.c_int, I32, C.c_int, I32]
    L.hf_n.restype = C.c_int64
    L.hf_n.argtypes = [C.c_void_p]
    L.hf_sorted.argtypes = [C.c_void_p] + [I32] * 5 + [np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")]
    L.hf_is_graded.argtypes = [C.c_void_p]
    L.hf_tiles_domain.argtypes = [C.c_void_p]
    L.hf_neighbour_table.argtypes = [C.c_void_p, I32, np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")]
    L.hm_create.restype = C.c_void_p
    L.hm_create.argtypes = [C.c_int64]
    L.hm_destroy.argtypes = [C.c_void_p]
    L.hm_put.argtypes = [C.c_void_p] + [C.c_int32] * 5
    L.hm_erase.argtypes = [C.c_void_p] + [C.c_int32] * 4
    L.hm_get.restype = C.c_int32
    L.hm_get.argtypes = [C.c_void_p] + [C.c_int32] * 4
    L.hm_size.restype = C.c_int64
    L.hm_size.argtypes = [C.c_void_p]
    return L


def _arr(boxes):
    a = np.array(boxes, dtype=np.int32).reshape(-1, 4)
    return [np.ascontiguousarray(a[:, k]) for k in range(4)]


class Host:
    def __init__(self, L, nroot, Bs, Jmin, Jmax, max_blocks):
        self.L = L
        self.h = L.hf_create(*nroot, Bs, Jmin, Jmax, max_blocks)

    def apply_pass(self, removed, created):
        r, c = _arr(removed), _arr(created)
        out = np.zeros(len(created), np.int32)
        ok = self.L.hf_apply_pass(self.h, len(removed), *r, len(created), *c, out)
        return out if ok else None

    def sorted(self):
        n = self.L.hf_n(self.h)
        a = [np.zeros(n, np.int32) for _ in range(5)]
        code = np.zeros(n, np.uint64)
        self.L.hf_sorted(self.h, *a, code)
        return a, code

    def table(self):
        n = self.L.hf_n(self.h)
        nbr = np.zeros(n * 56, np.int32)
        rel = np.zeros(n * 26, np.int8)
        self.L.hf_neighbour_table(self.h, nbr, rel)
        return nbr.reshape(n, 56), rel.reshape(n, 26)

    def close(self):
        self.L.hf_destroy(self.h)


def _compare(host, fo):
    (J, x, y, z, slot), code = host.sorted()
    tc, lv, sl, nbr, rel = fo.topology()
    order = fo.sorted_leaves()
    assert np.array_equal(code, tc) and np.array_equal(J, lv.astype(np.int32)) and np.array_equal(slot, sl)
    assert [tuple(v) for v in zip(J, x, y, z)] == [tuple(l) for l in order]
    hn, hr = host.table()
    assert np.array_equal(hn, nbr) and np.array_equal(hr, rel)


@pytest.mark.parametrize("seed,nroot,J0,Jmax,n", [(1, (1, 1, 1), 1, 3, 60), (2, (2, 1, 1), 1, 3, 90),
                                                  (3, (1, 2, 2), 0, 3, 50), (4, (3, 1, 1), 1, 2, 40)])
def test_layout_topology_is_the_oracles(lib, seed, nroot, J0, Jmax, n):
    leaves = random_graded_leaves(seed, nroot=nroot, J0=J0, Jmax=Jmax, n_target=n)
    fo = OForest(nroot=nroot, root_len=1.0, Bs=9, Jmin=0, Jmax=Jmax + 1, max_blocks=4096)
    fo.set_leaves(leaves)
    host = Host(lib, nroot, 9, 0, Jmax + 1, 4096)
    slots = host.apply_pass([], leaves)
    assert slots is not None
    _compare(host, fo)
    assert lib.hf_is_graded(host.h) == 1 and lib.hf_tiles_domain(host.h) == 1
    # a refinement pass of every leaf below the finest level, then a coarsening pass of every
    # complete sister group: the same slots as the oracle's passes
    parents = [l for l in fo.sorted_leaves() if l[0] <= Jmax]
    kids = [k for p in parents for k in OForest.children_of(p)]
    fo.apply_pass(parents, kids)
    assert host.apply_pass(parents, kids) is not None
    _compare(host, fo)
    groups = fo.sister_groups()
    removed = [k for p in groups for k in OForest.children_of(p)]
    fo.apply_pass(removed, groups)
    assert host.apply_pass(removed, groups) is not None
    _compare(host, fo)
    host.close()


def test_grading_and_capacity(lib):
    nroot = (1, 1, 1)
    leaves = [(1, x, y, z) for z in range(2) for y in range(2) for x in range(2) if (x, y, z) != (1, 0, 0)]
    kids = OForest.children_of((1, 1, 0, 0))
    grand = OForest.children_of(kids[0])                    # level 3 next to level-1 leaves
    layout = leaves + kids[1:] + grand
    fo = OForest(nroot=nroot, root_len=1.0, Bs=9, Jmin=0, Jmax=4, max_blocks=64)
    fo.set_leaves(layout)
    host = Host(lib, nroot, 9, 0, 4, 64)
    assert host.apply_pass([], layout) is not None
    assert fo.covers_domain_exactly() and lib.hf_tiles_domain(host.h) == 1
    assert not fo.is_graded() and lib.hf_is_graded(host.h) == 0
    host.close()
    # a pass that needs more slots than the pool holds changes nothing
    host = Host(lib, nroot, 9, 0, 4, 8)
    uni = [(1, x, y, z) for z in range(2) for y in range(2) for x in range(2)]
    assert host.apply_pass([], uni) is not None
    (J, x, y, z, slot0), _ = host.sorted()
    assert host.apply_pass([uni[0]], OForest.children_of(uni[0])) is None
    (J2, x2, y2, z2, slot1), _ = host.sorted()
    assert np.array_equal(slot0, slot1) and np.array_equal(J, J2)
    host.close()


def test_take_slots_gives_the_lowest_free_slots(lib):
    host = Host(lib, (1, 1, 1), 9, 0, 3, 64)
    uni = [(2, x, y, z) for z in range(4) for y in range(4) for x in range(4)]
    slots = host.apply_pass([], uni)
    assert sorted(slots.tolist()) == list(range(64))          # the pool is full
    out = np.zeros(2, np.int32)
    assert lib.hf_take_slots(host.h, 3, np.array([40, 9, 5], np.int32), 2, out) == 1
    assert out.tolist() == [5, 9]                               # released first, lowest first
    two = np.zeros(2, np.int32)
    assert lib.hf_take_slots(host.h, 0, np.zeros(0, np.int32), 2, two) == 0   # only slot 40 is free
    one = np.zeros(1, np.int32)
    assert lib.hf_take_slots(host.h, 0, np.zeros(0, np.int32), 1, one) == 1 and one.tolist() == [40]
    host.close()


def test_leaf_map_against_a_dictionary(lib):
    rng = np.random.default_rng(5)
    m = lib.hm_create(4096)
    ref = {}
    for _ in range(20000):
        k = (int(rng.integers(0, 6)), int(rng.integers(0, 40)), int(rng.integers(0, 40)), int(rng.integers(0, 40)))
        op = rng.integers(0, 3)
        if op == 0 and (len(ref) < 4000 or k in ref):
            s = int(rng.integers(0, 1 << 20))
            lib.hm_put(m, *k, s)
            ref[k] = s
        elif op == 1:
            assert lib.hm_erase(m, *k) == (1 if k in ref else 0)
            ref.pop(k, None)
        else:
            assert lib.hm_get(m, *k) == ref.get(k, -1)
        assert lib.hm_size(m) == len(ref)
    for k, s in ref.items():
        assert lib.hm_get(m, *k) == s
    lib.hm_destroy(m)
