"""Pins for the oracle's clustering inside the linear BVH's subtrees
(oracle.subtree_cluster; CPU only): with cap 1 it is the linear BVH itself, numbering
included; with a cap of at least n it is greedy agglomerative clustering of all
leaves; a hand-worked five-box case fixes the merges and the root's children; tree
invariants, boxes and a surface-area cost below the linear BVH's on the workloads'
kinds of input."""
import numpy as np
import pytest

import oracle
import scenegen
from test_oracle_ploc import _boxes, _greedy_sets, _tree_sets

LEAF = -0x80000000


def _check(cl, cr, pi, pl, n):
    """A binary tree over n leaves with root 0: every node and leaf the child of exactly
    one node (the root of none), parent links consistent, node numbers 0..n-2 each used."""
    assert cl.shape == (n - 1,) and cr.shape == (n - 1,) and pi[0] == -1
    seen_leaf = np.zeros(n, np.int64)
    seen_node = np.zeros(n - 1, np.int64)
    for q in range(n - 1):
        for side, c in enumerate((cl[q], cr[q])):
            if c < 0:
                k = int(c) & 0x7FFFFFFF
                seen_leaf[k] += 1
                assert pl[k] == q
            else:
                seen_node[c] += 1
                assert pi[c] == q
    assert np.all(seen_leaf == 1) and seen_node[0] == 0 and np.all(seen_node[1:] == 1)
    # every node reaches the root
    for q in range(1, n - 1):
        steps, x = 0, q
        while x != 0:
            x = int(pi[x])
            steps += 1
            assert steps < n
    return True


def _run(lo, hi, cap, bits=10):
    c = 0.5 * (lo + hi)
    return oracle.subtree_cluster(lo, hi, c.astype(np.float32), bits, cap)


@pytest.mark.parametrize("n", [2, 3, 17, 300])
def test_cap_one_is_the_linear_bvh(n):
    """With cap 1 every node merges its two children's single clusters, taking its own
    number: the linear BVH's topology and numbering exactly."""
    lo, hi = _boxes(n, seed=n)
    ref = _run(lo, hi, 1)
    assert np.array_equal(ref["childL"], ref["lbvh_childL"]) and np.array_equal(ref["childR"], ref["lbvh_childR"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cap_at_least_n_is_greedy_clustering(seed):
    """With a cap of n no node below the root merges anything, and the root clusters all
    leaves by mutual nearest neighbours over the whole list: the greedy agglomerative
    result (Walter et al. 2008), compared as sets of leaf sets."""
    n = 40
    lo, hi = _boxes(n, seed=100 + seed)
    want = _greedy_sets(lo, hi)
    if want is None:
        pytest.skip("near-tie between candidate pairs")
    ref = _run(lo, hi, n)
    order = ref["order"]
    got = _tree_sets(ref["childL"], ref["childR"], n)
    assert {frozenset(int(order[k]) for k in s) for s in got} == want


def test_hand_worked_five_boxes():
    """Five boxes of size 0.5 x 1 x 1 at x = 0, 1, 9.5, 11, 12. Their Morton order is
    their order in x; the linear BVH splits {0, 1} | {2, 3, 4}, then {2} | {3, 4}. With
    cap 2 the two-leaf nodes keep their leaves; node {2, 3, 4} holds three clusters and
    merges its mutual pair (3, 4) (union areas 2(x y + y z + z x) / 2: 4 for (3, 4), 5 for
    (2, 3), 7 for (2, 4)); the root holds [0, 1, 2, {3, 4}] and merges (0, 1) and
    (2, {3, 4}), then the two groups, taking number 0."""
    xs = np.array([0, 1, 9.5, 11, 12], np.float32)
    lo = np.stack([xs, np.zeros(5), np.zeros(5)], axis=1).astype(np.float32)
    hi = (lo + np.array([0.5, 1, 1], np.float32)).astype(np.float32)
    ref = _run(lo, hi, 2)
    n = 5
    assert np.array_equal(ref["order"], np.arange(5))
    assert _check(ref["childL"], ref["childR"], ref["parent_internal"], ref["parent_leaf"], n)
    got = {frozenset(int(k) for k in s) for s in _tree_sets(ref["childL"], ref["childR"], n)}
    assert got == {frozenset({0, 1}), frozenset({3, 4}), frozenset({2, 3, 4}), frozenset(range(5))}
    # the root's children: the group {0, 1} on the left (it came first in the list)
    left, right = ref["childL"][0], ref["childR"][0]
    assert left >= 0 and right >= 0
    assert {int(c) & 0x7FFFFFFF for c in (ref["childL"][left], ref["childR"][left])} == {0, 1}
    assert all(c < 0 for c in (ref["childL"][left], ref["childR"][left]))


@pytest.mark.parametrize("cap", [2, 8, 16])
def test_tree_invariants_and_boxes(cap):
    m = scenegen.terrain(cells=24, amplitude=0.2)
    lo, hi, c = oracle.triangle_aabbs(m.vertices, m.indices)
    ref = oracle.subtree_cluster(lo, hi, c, 10, cap)
    n = lo.shape[0]
    assert _check(ref["childL"], ref["childR"], ref["parent_internal"], ref["parent_leaf"], n)
    # every box holds its children's boxes; the root holds every leaf
    nlo, nhi = ref["node_lo"], ref["node_hi"]
    for q in range(n - 1):
        for ch in (ref["childL"][q], ref["childR"][q]):
            clo = ref["leaf_lo"][ch & 0x7FFFFFFF] if ch < 0 else nlo[ch]
            chi = ref["leaf_hi"][ch & 0x7FFFFFFF] if ch < 0 else nhi[ch]
            assert np.all(nlo[q] <= clo) and np.all(nhi[q] >= chi)
    assert np.array_equal(nlo[0], ref["leaf_lo"].min(axis=0)) and np.array_equal(nhi[0], ref["leaf_hi"].max(axis=0))


@pytest.mark.parametrize("kind", ["terrain", "soup"])
def test_cost_below_linear_bvh(kind):
    """Surface-area cost (Sec. 6.2) at cap 16 at least 10% below the linear BVH's on a
    height field and on a clustered triangle soup."""
    if kind == "terrain":
        m = scenegen.terrain(cells=64, amplitude=0.2)
    else:
        m = scenegen.soup_scene(3, seed=7, nmin=20_000, nmax=20_000).mesh
    lo, hi, c = oracle.triangle_aabbs(m.vertices, m.indices)
    ref = oracle.subtree_cluster(lo, hi, c, 10, 16)
    base = oracle.lbvh(lo, hi, c, 10)
    cost = oracle.sah_cost(ref["node_lo"], ref["node_hi"])
    base_cost = oracle.sah_cost(base["node_lo"], base["node_hi"])
    assert cost < 0.9 * base_cost, (cost, base_cost)


def test_equal_boxes_terminate():
    """5,000 identical boxes (every area ties): hashes break the ties and the build ends
    with a valid tree."""
    lo = np.zeros((5000, 3), np.float32)
    hi = np.ones((5000, 3), np.float32)
    ref = _run(lo, hi, 16)
    assert _check(ref["childL"], ref["childR"], ref["parent_internal"], ref["parent_leaf"], 5000)
