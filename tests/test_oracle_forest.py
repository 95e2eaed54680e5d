"""Pins of the oracle's block forest (Sec. 4.1 treecodes and neighbours, Sec. 3.5 grading)."""
import numpy as np
import pytest

from oracle.forest import DIRECTIONS, Forest, brute_force_adjacency, group_start
from paper_1912_05371_gb300.workloads import random_graded_leaves
from tests.golden_util import load_golden


def test_treecode_hand_computed():
    fo = Forest(nroot=(2, 1, 1), Bs=17)
    # level 2, global block (5, 2, 3): root 1, local (1, 2, 3);
    # level-1 digit from the high bits (0, 1, 1) -> 0 + 2 + 4 = 6, level-2 digit (1, 0, 1) -> 5
    code = fo.treecode(2, (5, 2, 3))
    assert code == (1 << 56) | (6 << 51) | (5 << 48)
    assert fo.decode(code, 2) == (5, 2, 3)


def test_treecode_roundtrip_and_jmax():
    gold = load_golden("paper_constants.txt")
    fo = Forest(nroot=(3, 2, 2), Bs=17)
    rng = np.random.default_rng(0)
    for _ in range(500):
        J = int(rng.integers(0, int(gold["jmax_limit"]) + 1))
        g = tuple(int(rng.integers(0, n << J)) for n in fo.nroot)
        code = fo.treecode(J, g)
        assert code < (1 << 64)
        assert fo.decode(code, J) == g


def test_key_order_is_depth_first_morton():
    fo = Forest(nroot=(1, 1, 1), Bs=9)
    fo.init_uniform(1)
    leaf = (1, 1, 0, 0)
    fo.apply_pass([leaf], Forest.children_of(leaf))
    order = fo.sorted_leaves()
    # child 0 of (1,1,0,0) follows (1,0,0,0) and precedes (1,0,1,0)
    assert order[0] == (1, 0, 0, 0)
    assert order[1:9] == Forest.children_of(leaf)
    assert order[9] == (1, 0, 1, 0)


def test_slot_allocation_rule():
    fo = Forest(nroot=(1, 1, 1), Bs=9, max_blocks=32)
    fo.init_uniform(1)
    assert [fo.leaves[l] for l in fo.sorted_leaves()] == list(range(8))
    leaf = (1, 1, 1, 0)                # slot 3
    assert fo.leaves[leaf] == 3
    new = fo.apply_pass([leaf], Forest.children_of(leaf))
    # slot 3 is returned first, then children in key order take 3, 8, 9, ...
    kids = sorted(new, key=fo.key)
    assert [new[k] for k in kids] == [3, 8, 9, 10, 11, 12, 13, 14]
    # merging gives back the lowest free slot
    new = fo.apply_pass(kids, [leaf])
    assert new[leaf] == 3
    with pytest.raises(MemoryError):
        fo.apply_pass([], [(3, i, 0, 0) for i in range(40)])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_neighbour_table_matches_brute_force(seed):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=60)
    fo = Forest(nroot=(2, 1, 1), Bs=9, max_blocks=4096)
    fo.set_leaves(leaves)
    assert fo.is_graded() and fo.covers_domain_exactly()
    order = fo.sorted_leaves()
    nbr, rel = fo.neighbour_table(order)
    adj = brute_force_adjacency(fo)
    slot2leaf = {s: l for l, s in fo.leaves.items()}
    for i, leaf in enumerate(order):
        listed = {slot2leaf[s] for s in nbr[i] if s >= 0}
        listed.discard(leaf)
        truth = set(adj[leaf])
        assert listed == truth, (leaf, listed ^ truth)
        for k, d in enumerate(DIRECTIONS):
            s0, n = group_start(k)
            ents = [slot2leaf[s] for s in nbr[i, s0:s0 + n] if s >= 0]
            assert ents, "every direction has a neighbour on a periodic graded grid"
            for e in ents:
                assert e[0] - leaf[0] == rel[i, k]
            if rel[i, k] == 1:
                assert len(ents) == n
            else:
                assert len(ents) == 1


def test_random_layouts_are_graded():
    for seed in range(4):
        leaves = random_graded_leaves(seed, nroot=(1, 1, 1), J0=1, Jmax=4, n_target=200)
        fo = Forest(Bs=9, max_blocks=1 << 14)
        fo.set_leaves(leaves)
        assert fo.is_graded()
        assert fo.covers_domain_exactly()
        for leaf in leaves:
            for other in brute_force_adjacency(fo)[leaf] if seed == 0 and len(leaves) < 120 else []:
                assert abs(other[0] - leaf[0]) <= 1
