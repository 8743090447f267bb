"""Pins for the oracle's LBVH build steps (CPU only).

Each check ties the oracle to something other than its own code: hand-computed
Morton codes, a hand-derived hierarchy, Python's stable sort, and structural
invariants that any correct binary BVH over sorted leaves must satisfy."""
import os

import numpy as np
import pytest

import oracle
import scenegen

LEAF = np.int32(-2147483648)


def _q(bits=10):
    return 1 << bits


# ---------------------------------------------------------------- Morton codes
def test_morton_hand_values_30bit():
    # bounds [0, 1024]^3 make q = floor(c) exactly
    lo = np.zeros(3, np.float32)
    hi = np.full(3, 1024.0, np.float32)
    c = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [2, 0, 0], [3, 0, 0],
                  [0, 3, 0], [1023, 1023, 1023], [1024, 1024, 1024], [512, 0, 0]], np.float32)
    codes = oracle.morton(c, lo, hi, 10)
    # x occupies bit 3k+2, y bit 3k+1, z bit 3k. expand(1)=1, expand(2)=0b1000=8, expand(3)=9
    expected = [0, 4, 2, 1, 7, 8 << 2, 9 << 2, 9 << 1, (1 << 30) - 1, (1 << 30) - 1, 1 << 29]
    assert codes.tolist() == expected


def test_morton_hand_values_63bit():
    lo = np.zeros(3, np.float32)
    hi = np.full(3, float(1 << 21), np.float32)
    c = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [2, 0, 0], [(1 << 21) - 1] * 3, [1 << 20, 0, 0]], np.float32)
    codes = oracle.morton(c, lo, hi, 21)
    assert codes.tolist() == [0, 4, 1, 32, (1 << 63) - 1, 1 << 62]


def test_morton_quantisation_edges():
    lo = np.array([0, 5, -1], np.float32)
    hi = np.array([1, 5, 1], np.float32)  # zero extent in y
    c = np.array([[0.5, 5, 0], [1.0, 5, 1], [np.nextafter(np.float32(1), np.float32(0)), 5, -1]], np.float32)
    codes = oracle.morton(c, lo, hi, 10)
    # (0.5 -> 512, y -> 0, z: 1/2 -> 512); (1 -> clamp 1023, 0, 1023); (just below 1 -> 1023, 0, 0)
    def code(x, y, z):
        out = 0
        for k in range(9, -1, -1):
            out = (out << 3) | (((x >> k) & 1) << 2) | (((y >> k) & 1) << 1) | ((z >> k) & 1)
        return out

    assert codes.tolist() == [code(512, 0, 512), code(1023, 0, 1023), code(1023, 0, 0)]


def test_morton_order_is_z_order_on_a_grid():
    # On a 2x2x2 grid of cells the codes must enumerate the octants in z-order
    lo = np.zeros(3, np.float32)
    hi = np.full(3, 2.0, np.float32)
    pts = np.array([[x, y, z] for x in (0.5, 1.5) for y in (0.5, 1.5) for z in (0.5, 1.5)], np.float32)
    codes = oracle.morton(pts, lo, hi, 10)
    order = np.argsort(codes, kind="stable")
    assert order.tolist() == list(range(8))  # x major, then y, then z


# ---------------------------------------------------------------- sort
def test_stable_sort_matches_python_sorted():
    rng = np.random.default_rng(1)
    codes = rng.integers(0, 50, 2000).astype(np.uint64)
    sk, order = oracle.stable_sort(codes)
    ref = sorted(range(len(codes)), key=lambda i: int(codes[i]))
    assert order.tolist() == ref
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)


# ---------------------------------------------------------------- topology
def _read_tree(path):
    keys, nodes = None, {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "keys":
            keys = [int(x) for x in parts[1:]]
        else:
            nodes[int(parts[1])] = parts[2:]
    return keys, nodes


def _enc(s):
    return (int(s[1:]) | -2147483648) if s[0] == "L" else int(s[1:])


def test_topology_hand_derived_example(golden_dir):
    keys, nodes = _read_tree(os.path.join(golden_dir, "karras_example_tree.txt"))
    cl, cr, pi, pl = oracle.topology(np.array(keys, np.uint64), 32)
    for k, (l, r) in nodes.items():
        assert cl[k] == np.int32(_enc(l)) and cr[k] == np.int32(_enc(r)), k


def test_topology_duplicate_keys_split_by_index():
    cl, cr, pi, pl = oracle.topology(np.zeros(5, np.uint64), 32)
    # indices 0..4: highest differing bit of 0 and 4 is bit 2 -> [0,3] | [4]
    assert (cl[0], cr[0]) == (3, np.int32(4 | -2147483648))
    assert (cl[3], cr[3]) == (1, 2)
    assert (cl[1], cr[1]) == (np.int32(0 | -2147483648), np.int32(1 | -2147483648))


def _check_invariants(cl, cr, pi, pl, n):
    assert cl.shape == (n - 1,) and cr.shape == (n - 1,)
    leaf_seen = np.zeros(n, int)
    node_seen = np.zeros(n - 1, int)
    rng_lo = np.full(n - 1, -1)
    rng_hi = np.full(n - 1, -1)
    # ranges by a top-down walk
    stack = [(0, 0, n - 1)]
    while stack:
        k, a, b = stack.pop()
        rng_lo[k], rng_hi[k] = a, b
        assert k in (a, b), "Karras: a node's index is one end of its range"
        ends = []
        for c in (cl[k], cr[k]):
            if c < 0:
                leaf_seen[c & 0x7FFFFFFF] += 1
                ends.append((c & 0x7FFFFFFF, c & 0x7FFFFFFF))
            else:
                node_seen[c] += 1
                ends.append(None)
        # children partition [a,b] into [a,g] and [g+1,b]
        g = None
        if cl[k] < 0:
            g = cl[k] & 0x7FFFFFFF
            assert g == a
        else:
            g = cl[k]
        if cr[k] < 0:
            assert (cr[k] & 0x7FFFFFFF) == b and (cr[k] & 0x7FFFFFFF) == g + 1
        else:
            assert cr[k] == g + 1
        if cl[k] >= 0:
            stack.append((cl[k], a, g))
        if cr[k] >= 0:
            stack.append((cr[k], g + 1, b))
    assert (leaf_seen == 1).all(), "every primitive in exactly one leaf"
    assert node_seen[0] == 0 and (node_seen[1:] == 1).all(), "every non-root node has one parent"
    assert pi[0] == -1
    for k in range(n - 1):
        for c in (cl[k], cr[k]):
            if c < 0:
                assert pl[c & 0x7FFFFFFF] == k
            else:
                assert pi[c] == k
    return rng_lo, rng_hi


@pytest.mark.parametrize("n,maxkey", [(2, 5), (3, 1), (17, 4), (1000, 1 << 30), (4096, 64)])
def test_topology_invariants(n, maxkey):
    rng = np.random.default_rng(n)
    keys = np.sort(rng.integers(0, maxkey, n).astype(np.uint64))
    cl, cr, pi, pl = oracle.topology(keys, 32)
    _check_invariants(cl, cr, pi, pl, n)


def test_topology_split_is_highest_differing_bit():
    # brute force the split rule on every internal node of a random tree
    rng = np.random.default_rng(7)
    n = 300
    keys = np.sort(rng.integers(0, 1 << 12, n).astype(np.uint64))
    cl, cr, pi, pl = oracle.topology(keys, 32)
    lo, hi = _check_invariants(cl, cr, pi, pl, n)
    aug = [(int(keys[i]) << 32) | i for i in range(n)]
    for k in range(n - 1):
        a, b = lo[k], hi[k]
        bit = (aug[a] ^ aug[b]).bit_length() - 1
        g = cl[k] & 0x7FFFFFFF if cl[k] < 0 else cl[k]
        assert all(((aug[m] >> bit) & 1) == 0 for m in range(a, g + 1))
        assert all(((aug[m] >> bit) & 1) == 1 for m in range(g + 1, b + 1))


# ---------------------------------------------------------------- fit
def test_fit_boxes_are_unions_of_leaf_ranges():
    mesh = scenegen.icosphere(2)
    lo, hi, c = oracle.triangle_aabbs(mesh.vertices, mesh.indices)
    r = oracle.lbvh(lo, hi, c, 10)
    n = lo.shape[0]
    rl, rh = _check_invariants(r["childL"], r["childR"], r["parent_internal"], r["parent_leaf"], n)
    for k in range(n - 1):
        a, b = rl[k], rh[k]
        assert np.array_equal(r["node_lo"][k], r["leaf_lo"][a:b + 1].min(axis=0))
        assert np.array_equal(r["node_hi"][k], r["leaf_hi"][a:b + 1].max(axis=0))
    # the root is the union of every primitive box, and it contains the unit sphere's mesh
    assert np.array_equal(r["node_lo"][0], lo.min(axis=0))
    assert np.array_equal(r["node_hi"][0], hi.max(axis=0))


def test_triangle_aabbs_and_centroids():
    v = np.array([[0, 0, 0], [2, -1, 4], [1, 3, -2]], np.float32)
    lo, hi, c = oracle.triangle_aabbs(v, np.array([[0, 1, 2]], np.uint32))
    assert lo[0].tolist() == [0, -1, -2] and hi[0].tolist() == [2, 3, 4]
    assert c[0].tolist() == [1, 1, 1]


def test_sah_cost_of_two_unit_boxes():
    # root [0,2]x[0,1]x[0,1] area 10; two unit children are leaves: cost = 10/10 = 1
    assert oracle.sah_cost(np.array([[0, 0, 0]], np.float32), np.array([[2, 1, 1]], np.float32)) == 1.0


# ---------------------------------------------------------------- 4-wide nodes
def _tree_dict(cl, cr, leaf_lo, leaf_hi):
    nlo, nhi = oracle.fit(cl, cr, leaf_lo, leaf_hi)
    return dict(childL=cl, childR=cr, node_lo=nlo, node_hi=nhi, leaf_lo=leaf_lo, leaf_hi=leaf_hi)


def test_wide_nodes_hand_derived():
    # five equal keys: node 0 = (node 3, leaf 4), node 3 = (node 1, node 2),
    # node 1 = (leaf 0, leaf 1), node 2 = (leaf 2, leaf 3) (see the duplicate-key test)
    cl, cr, _, _ = oracle.topology(np.zeros(5, np.uint64), 32)
    leaf_lo = np.array([[i, 0, 0] for i in range(5)], np.float32)
    leaf_hi = leaf_lo + np.float32(0.5)
    lo, hi, child = oracle.wide_nodes(_tree_dict(cl, cr, leaf_lo, leaf_hi))
    L = 0x80000000
    E = 0xFFFFFFFF
    assert child.tolist() == [[1, 2, L | 4, E], [L | 0, E, L | 1, E], [L | 2, E, L | 3, E],
                              [L | 0, L | 1, L | 2, L | 3]]
    # node 0: slot 0 = node 1 = leaves 0-1, slot 1 = node 2 = leaves 2-3, slot 2 = leaf 4
    assert lo[0, 0].tolist() == [0, 0, 0] and hi[0, 0].tolist() == [1.5, 0.5, 0.5]
    assert lo[0, 1].tolist() == [2, 0, 0] and hi[0, 1].tolist() == [3.5, 0.5, 0.5]
    assert lo[0, 2].tolist() == [4, 0, 0] and hi[0, 2].tolist() == [4.5, 0.5, 0.5]
    assert np.all(lo[0, 3] == np.inf) and np.all(hi[0, 3] == -np.inf)
    assert lo[3, 3].tolist() == [3, 0, 0] and hi[3, 3].tolist() == [3.5, 0.5, 0.5]


def test_wide_nodes_single_primitive():
    d = dict(leaf_lo=np.array([[1, 2, 3]], np.float32), leaf_hi=np.array([[4, 5, 6]], np.float32))
    lo, hi, child = oracle.wide_nodes(d)
    assert child.tolist() == [[0x80000000, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]]
    assert lo[0, 0].tolist() == [1, 2, 3] and hi[0, 0].tolist() == [4, 5, 6]
    assert np.all(lo[0, 1:] == np.inf) and np.all(hi[0, 1:] == -np.inf)


@pytest.mark.parametrize("level", [1, 3])
def test_wide_nodes_invariants(level):
    mesh = scenegen.icosphere(level)
    tlo, thi, c = oracle.triangle_aabbs(mesh.vertices, mesh.indices)
    r = oracle.lbvh(tlo, thi, c, 10)
    n = tlo.shape[0]
    lo, hi, child = oracle.wide_nodes(r)
    assert child.shape == (n - 1, 4)
    for k in range(n - 1):
        used = child[k] != 0xFFFFFFFF
        # the slots cover exactly the binary node's box
        assert np.array_equal(lo[k][used].min(axis=0), r["node_lo"][k])
        assert np.array_equal(hi[k][used].max(axis=0), r["node_hi"][k])
        # an empty slot is always the second of a pair whose first is a leaf
        for j in (1, 3):
            if not used[j]:
                assert child[k, j - 1] & 0x80000000
        assert used[0] and used[2]
    # a walk from wide node 0 reaches every leaf exactly once, through the wide nodes of
    # binary nodes at even depth only
    seen = np.zeros(n, int)
    visited = []
    stack = [0]
    while stack:
        k = stack.pop()
        visited.append(k)
        for cc in child[k]:
            if cc == 0xFFFFFFFF:
                continue
            if cc & 0x80000000:
                seen[cc & 0x7FFFFFFF] += 1
            else:
                stack.append(int(cc))
    assert (seen == 1).all()
    parent = np.full(n - 1, -1)
    for k in range(n - 1):
        for cc in (r["childL"][k], r["childR"][k]):
            if cc >= 0:
                parent[cc] = k
    for k in visited:  # even depth: the number of binary edges up to the root
        d, x = 0, k
        while parent[x] >= 0:
            x, d = parent[x], d + 1
        assert d % 2 == 0


# ---------------------------------------------------------------- quantised 4-wide nodes
def _golden_quantized(golden_dir):
    nodes, slots = [], []
    with open(os.path.join(golden_dir, "quantized_wide_nodes.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "slot":
                slots.append(([float(x) for x in t[1:4]], [float(x) for x in t[4:7]], int(t[7], 16)))
            elif t[0] == "words":
                nodes.append((slots, [int(w, 16) for w in t[1:]]))
                slots = []
    return nodes


def test_quantized_nodes_hand_derived(golden_dir):
    """Three nodes worked by hand (tests/golden/quantized_wide_nodes.txt): an origin at 0
    with a different exponent per axis and a flat slot, a negative origin, and planes near
    1e6 where the float32 rounding of p + q 2^e (ties to even) decides the exponent and
    the bytes."""
    cases = _golden_quantized(golden_dir)
    assert len(cases) == 3
    for slots, words in cases:
        lo = np.full((1, 4, 3), np.inf, np.float32)
        hi = np.full((1, 4, 3), -np.inf, np.float32)
        child = np.full((1, 4), oracle.NONE, np.uint32)
        for j, (l, h, c) in enumerate(slots):
            lo[0, j], hi[0, j], child[0, j] = l, h, c
        got = oracle.quantized_wide_nodes(lo, hi, child)
        assert [int(w) for w in got[0]] == words


def _wide_of(kind, seed=0):
    if kind == "terrain":
        m = scenegen.terrain(cells=24, amplitude=0.2)
        lo, hi, c = oracle.triangle_aabbs(m.vertices, m.indices)
    elif kind == "spheres":
        s = scenegen.spheres(3000, half=50.0, rmin=0.01, rmax=1.0, config=5)
        b = scenegen.sphere_aabbs(s)
        lo, hi = b[:, 0:3].copy(), b[:, 3:6].copy()
        c = oracle.box_centroids(b)
    elif kind == "far":  # tiny boxes far from the origin, both signs
        rng = np.random.default_rng(seed)
        ctr = rng.uniform(-1, 1, (800, 3)) * np.array([3e5, 1e4, 7e6]) + np.array([1e6, -5e3, 2e7])
        ext = rng.uniform(0, 0.05, (800, 3))
        lo, hi = (ctr - ext).astype(np.float32), (ctr + ext).astype(np.float32)
        c = (0.5 * (lo + hi)).astype(np.float32)
    elif kind == "flat":  # zero extent on y, boxes touching zero from both sides
        rng = np.random.default_rng(seed)
        x = rng.uniform(-1e-3, 1e-3, (500, 1))
        lo = np.concatenate([x, np.zeros((500, 1)), -np.abs(x)], axis=1).astype(np.float32)
        hi = np.concatenate([x + 1e-4, np.zeros((500, 1)), np.abs(x)], axis=1).astype(np.float32)
        c = (0.5 * (lo + hi)).astype(np.float32)
    else:  # clustered soup
        m = scenegen.soup_scene(2, seed=9, nmin=3000, nmax=3000).mesh
        lo, hi, c = oracle.triangle_aabbs(m.vertices, m.indices)
    return oracle.wide_nodes(oracle.lbvh(lo, hi, c, 10))


@pytest.mark.parametrize("kind", ["terrain", "spheres", "far", "flat", "soup"])
def test_quantized_nodes_conservative_and_tight(kind):
    """Every decoded slot box contains the slot's exact box (traversal stays
    conservative), one step tighter on any plane would cut into it, the exponent is the
    least that reaches the node's top, empty slots decode inverted (255 / 0) and the
    child words are copied. The decoding here is numpy float32 arithmetic, not the
    oracle's C code."""
    wlo, whi, ch = _wide_of(kind, seed=3)
    q = oracle.quantized_wide_nodes(wlo, whi, ch)
    dlo, dhi = oracle.dequantize_wide_nodes(q)
    used = ch != oracle.NONE
    assert np.all(dlo[used] <= wlo[used]) and np.all(dhi[used] >= whi[used])
    assert np.array_equal(q[:, 10:14], ch) and not q[:, 14:16].any()
    p = q[:, 0:3].copy().view(np.float32)
    e = np.stack([(q[:, 3] >> (8 * a)) & 0xFF for a in range(3)], axis=1).astype(np.int64) - 127
    assert ((e >= -126) & (e <= 127)).all() and not (q[:, 3] >> 24).any()
    m = q.shape[0]
    for a in range(3):
        lo_a = np.where(used, wlo[:, :, a], np.inf).min(axis=1)
        top_a = np.where(used, whi[:, :, a], -np.inf).max(axis=1)
        assert np.array_equal(p[:, a], lo_a.astype(np.float32))
        dec = lambda qq, ee: (p[:, a] + np.float32(qq) * np.ldexp(np.float32(1), ee).astype(np.float32)).astype(np.float32)
        # the least exponent: one less no longer reaches the top
        smaller = e[:, a] > -126
        ee = np.maximum(e[:, a] - 1, -126)
        assert np.all(dec(255, ee)[smaller] < top_a[smaller])
        step = np.ldexp(np.float32(1), e[:, a]).astype(np.float32)
        for j in range(4):
            ql = ((q[:, 4 + 2 * a] >> (8 * j)) & 0xFF).astype(np.float32)
            qh = ((q[:, 5 + 2 * a] >> (8 * j)) & 0xFF).astype(np.float32)
            u = used[:, j]
            assert np.all(ql[~u] == 255) and np.all(qh[~u] == 0)
            up = u & (ql < 255)
            assert np.all((p[:, a] + (ql + 1) * step).astype(np.float32)[up] > wlo[up, j, a])
            dn = u & (qh > 0)
            assert np.all((p[:, a] + (qh - 1) * step).astype(np.float32)[dn] < whi[dn, j, a])
    assert m == wlo.shape[0]


def test_quantized_single_primitive_and_degenerate_node():
    """A one-primitive geometry's node (leaf in slot 0, three empty slots) and a point
    box: the origin is the box's corner, a zero extent takes the least exponent, and the
    point decodes exactly."""
    d = dict(leaf_lo=np.array([[1, 2, 3]], np.float32), leaf_hi=np.array([[4, 2, 3]], np.float32))
    lo, hi, child = oracle.wide_nodes(d)
    q = oracle.quantized_wide_nodes(lo, hi, child)
    assert q[0, 0:3].view(np.float32).tolist() == [1, 2, 3]
    assert [(int(q[0, 3]) >> (8 * a)) & 0xFF for a in range(3)] == [127 - 6, 1, 1]  # 255/64 >= 3 > 255/128
    dlo, dhi = oracle.dequantize_wide_nodes(q)
    assert dlo[0, 0].tolist() == [1, 2, 3] and dhi[0, 0].tolist() == [4, 2, 3]
    assert q[0, 10] == 0x80000000 and (q[0, 11:14] == oracle.NONE).all()


# ---------------------------------------------------------------- 8-wide nodes
def test_wide8_nodes_hand_derived(golden_dir):
    """Karras's eight-key example (tests/golden/karras_example_tree.txt): node 0 =
    (N3, N4), N3 = (N1, N2), N1 = (L0, L1), N2 = (L2, L3), N4 = (L4, N5), N5 = (N6, L7),
    N6 = (L5, L6). Three levels below node 0: N3's grandchildren L0-L3 fill slots 0-3;
    N4's children are L4 (slot 4, slot 5 empty) and N5, whose children N6 and L7 fill
    slots 6 and 7. N6 (depth 3) holds its leaf children L5 in slot 0 and L6 in slot 4."""
    keys, _ = _read_tree(os.path.join(golden_dir, "karras_example_tree.txt"))
    cl, cr, _, _ = oracle.topology(np.array(keys, np.uint64), 32)
    leaf_lo = np.array([[i, 0, 0] for i in range(8)], np.float32)
    leaf_hi = leaf_lo + np.float32(0.5)
    lo, hi, child = oracle.wide8_nodes(_tree_dict(cl, cr, leaf_lo, leaf_hi))
    L, E = 0x80000000, 0xFFFFFFFF
    assert child[0].tolist() == [L | 0, L | 1, L | 2, L | 3, L | 4, E, 6, L | 7]
    assert child[6].tolist() == [L | 5, E, E, E, L | 6, E, E, E]
    assert lo[0, 6].tolist() == [5, 0, 0] and hi[0, 6].tolist() == [6.5, 0.5, 0.5]  # N6 = leaves 5-6
    assert lo[0, 7].tolist() == [7, 0, 0] and np.all(lo[0, 5] == np.inf) and np.all(hi[0, 5] == -np.inf)


def test_wide8_nodes_single_primitive():
    d = dict(leaf_lo=np.array([[1, 2, 3]], np.float32), leaf_hi=np.array([[4, 5, 6]], np.float32))
    lo, hi, child = oracle.wide8_nodes(d)
    assert child.tolist() == [[0x80000000] + [0xFFFFFFFF] * 7]
    assert lo[0, 0].tolist() == [1, 2, 3] and np.all(lo[0, 1:] == np.inf)


@pytest.mark.parametrize("level", [1, 3])
def test_wide8_nodes_invariants(level):
    """Used slots cover exactly the binary node's box; a walk from node 0 reaches every
    leaf exactly once, through nodes of binary depth divisible by 3 only."""
    mesh = scenegen.icosphere(level)
    tlo, thi, c = oracle.triangle_aabbs(mesh.vertices, mesh.indices)
    r = oracle.lbvh(tlo, thi, c, 10)
    n = tlo.shape[0]
    lo, hi, child = oracle.wide8_nodes(r)
    assert child.shape == (n - 1, 8)
    for k in range(n - 1):
        used = child[k] != 0xFFFFFFFF
        assert np.array_equal(lo[k][used].min(axis=0), r["node_lo"][k])
        assert np.array_equal(hi[k][used].max(axis=0), r["node_hi"][k])
        assert used[0] and used[4]
    parent = np.full(n - 1, -1)
    for k in range(n - 1):
        for cc in (r["childL"][k], r["childR"][k]):
            if cc >= 0:
                parent[cc] = k
    seen = np.zeros(n, int)
    stack = [0]
    while stack:
        k = stack.pop()
        d, x = 0, k
        while parent[x] >= 0:
            x, d = parent[x], d + 1
        assert d % 3 == 0
        for cc in child[k]:
            if cc == 0xFFFFFFFF:
                continue
            if cc & 0x80000000:
                seen[cc & 0x7FFFFFFF] += 1
            else:
                stack.append(int(cc))
    assert (seen == 1).all()
