"""The oracle's spatial splits of triangles (split_ref.cpp; the paper's high-quality
option, Sec. 8, made before the build after Karras and Aila, HPG 2013), pinned by
hand-derived cases, the budget arithmetic the method fixes, and geometric facts any
correct split has: every point of a triangle lies in one of its references' boxes, and
no reference box leaves the triangle's own box."""
import os

import numpy as np
import pytest

import oracle


def _num(x: str) -> float:
    return float.fromhex(x) if "x" in x else float(x)


def _golden(golden_dir):
    cases, cur = [], None
    with open(os.path.join(golden_dir, "split_triangles.txt")) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "case":
                cur = dict(name=w[1], budget=int(w[3]), tris=[], refs=[])
            elif w[0] == "tri":
                cur["tris"].append([_num(x) for x in w[1:10]])
            elif w[0] == "splits":
                cur["splits"] = [int(x) for x in w[1:]]
            elif w[0] == "ref":
                cur["refs"].append(([_num(x) for x in w[1:7]], int(w[7]), int(w[8])))
            elif w[0] == "end":
                cases.append(cur)
    return cases


def _mesh(tris):
    v = np.asarray(tris, np.float32).reshape(-1, 3)
    return v, np.arange(v.shape[0], dtype=np.uint32).reshape(-1, 3)


def test_split_hand_derived_cases(golden_dir):
    """Four cases worked by hand (tests/golden/split_triangles.txt): a grid-line cut with
    widened crossings, a second cut on another axis after the narrowing of the box,
    the remainder of a zero total weight, and the midpoint cut of a box inside one cell."""
    cases = _golden(golden_dir)
    assert [c["name"] for c in cases] == ["single", "diagonal", "degenerate", "midpoint"]
    for c in cases:
        v, idx = _mesh(c["tris"])
        lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, c["budget"])
        want = np.array([r[0] for r in c["refs"]], np.float32)
        assert splits.tolist() == c["splits"], c["name"]
        assert np.array_equal(np.concatenate([lo, hi], axis=1), want), c["name"]
        assert prim.tolist() == [r[1] for r in c["refs"]], c["name"]
        assert owner.astype(int).tolist() == [r[2] for r in c["refs"]], c["name"]


def _soup(n, seed, big=0.3):
    """Triangles of log-uniform size (up to `big`) at random places and orientations."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (n, 1, 3))
    size = np.exp(rng.uniform(np.log(1e-3), np.log(big), (n, 1, 1)))
    v = (c + size * rng.normal(size=(n, 3, 3))).astype(np.float32).reshape(-1, 3)
    return v, np.arange(3 * n, dtype=np.uint32).reshape(n, 3)


def test_zero_budget_gives_the_triangle_boxes():
    v, idx = _soup(500, 1)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, 0)
    tlo, thi, _ = oracle.triangle_aabbs(v, idx)
    assert np.array_equal(lo, tlo) and np.array_equal(hi, thi)
    assert np.array_equal(prim, np.arange(500)) and owner.all() and not splits.any()


@pytest.mark.parametrize("factor", [0.1, 0.5, 1.0])
def test_budget_is_spent_exactly(factor):
    """n + floor(factor n) references, numbered triangle by triangle, one owner (the
    first) per triangle, split counts summing to the budget and the per-triangle cap
    (31 by priority, +1 from the remainder) respected."""
    n = 1500
    v, idx = _soup(n, 2)
    S = oracle.split_budget(n, factor)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, S)
    assert lo.shape[0] == n + S and int(splits.sum()) == S and splits.max() <= oracle.SPLIT_MAX + 1
    counts = np.bincount(prim, minlength=n)
    assert np.array_equal(counts, splits + 1)
    assert np.all(np.diff(prim.astype(np.int64)) >= 0)
    first = np.r_[True, prim[1:] != prim[:-1]]
    assert np.array_equal(owner, first)


def test_split_budget_rounding():
    assert oracle.split_budget(10, 0.0) == 5 and oracle.split_budget(11, 0.0) == 5
    assert oracle.split_budget(3, 1.0) == 3 and oracle.split_budget(7, 0.25) == 1
    # the factor is a float32: 0.1f is a little above 0.1
    assert oracle.split_budget(10, 0.1) == 1 and oracle.split_budget(1000, 0.3) == 300


def test_cap_and_remainder():
    """31 flat segments (weight 0: a box with two zero extents has no area to save) and one
    large triangle that holds the whole weight: with budget 32 it takes the cap of 31, and
    the one split left over goes to triangle 0."""
    seg = [[0, 0, 0, 1, 0, 0, 1, 0, 0]] * 31
    tris = seg + [[0, 0, 0, 4, 3, 1, 1, 4, 2]]
    v, idx = _mesh(tris)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, 32)
    assert splits[31] == 31 and splits[0] == 1 and splits[1:31].sum() == 0
    assert lo.shape[0] == 64


def _inside_some_reference(v, idx, lo, hi, prim, samples):
    """For each triangle and barycentric sample, whether the point (double) lies in one of
    the triangle's reference boxes (closed, float bounds)."""
    tri = v[idx].astype(np.float64)  # (n,3,3)
    pts = np.einsum("kj,njc->nkc", samples, tri)  # (n,K,3)
    p = pts[prim]  # (m,K,3)
    inside = np.all((p >= lo[:, None, :].astype(np.float64)) & (p <= hi[:, None, :].astype(np.float64)), axis=2)
    start = np.flatnonzero(np.r_[True, prim[1:] != prim[:-1]])
    return np.logical_or.reduceat(inside, start, axis=0)  # (n,K)


def _samples(k=16):
    """Barycentric weights i/k, j/k, (k-i-j)/k with k a power of two: the sample points of
    float32 vertices are then exact in double (no rounding can move one off a box face)."""
    b = [(i / k, j / k, (k - i - j) / k) for i in range(k + 1) for j in range(k + 1 - i)]
    return np.array(b, np.float64)


@pytest.mark.parametrize("seed,factor", [(3, 0.5), (4, 1.0), (5, 0.2)])
def test_references_cover_their_triangle_and_stay_in_its_box(seed, factor):
    n = 800
    v, idx = _soup(n, seed, big=0.8)
    S = oracle.split_budget(n, factor)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, S)
    assert splits.max() >= 2  # the large triangles are cut more than once
    assert np.all(lo <= hi), "empty reference box"
    tlo, thi, _ = oracle.triangle_aabbs(v, idx)
    assert np.all(lo >= tlo[prim]) and np.all(hi <= thi[prim]), "reference outside its triangle's box"
    cover = _inside_some_reference(v, idx, lo, hi, prim, _samples())
    assert cover.all(), np.argwhere(~cover)[:5]


@pytest.mark.parametrize("scale,offset", [(1e-38, 0.0), (1e25, 0.0), (1.0, 3e6), (1e-3, 100.0)])
def test_references_stay_conservative_at_extreme_scales(scale, offset):
    """Tiny, huge and far-off coordinates: the widening scales with the endpoints'
    magnitude (plus 2^-140 for subnormals), so coverage holds; at the extreme scales the
    float32 areas of the priority leave the range, the weights vanish and the budget goes
    by the remainder rule (one cut each), which is still a valid split."""
    v, idx = _soup(800, 31, big=0.8)
    v = (v.astype(np.float64) * scale + offset).astype(np.float32)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, oracle.split_budget(800, 1.0))
    tlo, thi, _ = oracle.triangle_aabbs(v, idx)
    assert np.all(lo <= hi) and np.all(lo >= tlo[prim]) and np.all(hi <= thi[prim])
    assert _inside_some_reference(v, idx, lo, hi, prim, _samples()).all()


def test_axis_aligned_grid_mesh_is_covered():
    """A flat grid of right triangles whose vertices and edge crossings fall on grid lines
    (the exact coincidences the widening and the narrowing are for)."""
    k = 16
    xs = np.linspace(0.0, 1.0, k + 1, dtype=np.float32)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    v = np.stack([X.ravel(), np.zeros(X.size, np.float32), Z.ravel()], axis=1)
    q = np.arange(k)
    a = (q[:, None] * (k + 1) + q[None, :]).ravel()
    idx = np.concatenate([np.stack([a, a + 1, a + k + 2], 1), np.stack([a, a + k + 2, a + k + 1], 1)]).astype(np.uint32)
    S = oracle.split_budget(idx.shape[0], 1.0)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, S)
    assert np.all(lo <= hi)
    assert _inside_some_reference(v, idx, lo, hi, prim, _samples()).all()


def test_splits_lower_the_leaf_area_and_the_tree_cost():
    """Long thin diagonal triangles: cutting them shrinks the summed leaf surface area,
    and the linear BVH over the references costs less (surface-area heuristic) than the
    one over whole triangles."""
    rng = np.random.default_rng(7)
    n = 600
    a = rng.uniform(-1, 1, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    e = rng.normal(size=(n, 3)) * 0.01
    v = np.stack([a, a + 0.8 * d, a + 0.8 * d + e], axis=1).astype(np.float32).reshape(-1, 3)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)

    def area(lo, hi):
        s = (hi - lo).astype(np.float64)
        return float(np.sum(s[:, 0] * s[:, 1] + s[:, 1] * s[:, 2] + s[:, 2] * s[:, 0]))

    tlo, thi, tc = oracle.triangle_aabbs(v, idx)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, oracle.split_budget(n, 1.0))
    assert area(lo, hi) < 0.75 * area(tlo, thi)
    base = oracle.lbvh(tlo, thi, tc, 10)
    cut = oracle.lbvh(lo, hi, oracle.box_centroids(np.concatenate([lo, hi], axis=1)), 10)
    assert oracle.sah_cost(cut["node_lo"], cut["node_hi"]) < 0.95 * oracle.sah_cost(base["node_lo"], base["node_hi"])


def test_priority_prefers_large_diagonal_triangles():
    """100 long diagonal triangles among 2,000 small ones, budget 10%: the priority (area
    the box wastes, weighted by the level of the grid lines it crosses) sends nearly all
    the splits (80%) to the long ones, while a small one gets at most one (the
    rounding of its share, which is far below one)."""
    rng = np.random.default_rng(11)
    a = rng.uniform(-1, 1, (100, 3))
    big = np.stack([a, a + 0.5, a + [0.5, 0.5, 0.52]], axis=1)
    c = rng.uniform(-1, 1, (2000, 1, 3))
    small = c + 0.002 * rng.normal(size=(2000, 3, 3))
    v = np.concatenate([big, small]).astype(np.float32).reshape(-1, 3)
    idx = np.arange(v.shape[0], dtype=np.uint32).reshape(-1, 3)
    S = oracle.split_budget(2100, 0.1)
    _, _, _, _, splits = oracle.split_triangles(v, idx, S)
    assert splits[:100].sum() >= 0.8 * S and splits[:100].min() >= 1 and splits[100:].max() <= 1


def _mt(o, d, v0, v1, v2):
    """Moller-Trumbore in double for one ray against triangles (arrays (k,3)): t, or inf."""
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = o - v0
    u = np.einsum("ij,ij->i", s, p) * inv
    q = np.cross(s, e1)
    w = (q @ d) * inv
    t = np.einsum("ij,ij->i", e2, q) * inv
    hit = ok & (u >= 0) & (w >= 0) & (u + w <= 1) & (t >= 0)
    return np.where(hit, t, np.inf)


def test_closest_hits_through_the_split_tree_equal_brute_force():
    """End to end on the CPU: the linear BVH over the split references (the oracle's own
    build), walked with a plain slab test, finds for every ray the same closest triangle
    and t as testing all triangles: no cut loses a part of a triangle that a ray can hit."""
    n = 300
    v, idx = _soup(n, 21, big=0.9)
    lo, hi, prim, owner, splits = oracle.split_triangles(v, idx, oracle.split_budget(n, 1.0))
    assert splits.max() >= 3
    ref = oracle.lbvh(lo, hi, oracle.box_centroids(np.concatenate([lo, hi], axis=1)), 10)
    order, cl, cr = ref["order"], ref["childL"].view(np.uint32), ref["childR"].view(np.uint32)
    nlo, nhi = ref["node_lo"].astype(np.float64), ref["node_hi"].astype(np.float64)
    llo, lhi = ref["leaf_lo"].astype(np.float64), ref["leaf_hi"].astype(np.float64)
    tri = v[idx].astype(np.float64)
    rng = np.random.default_rng(22)
    eps = 1e-9

    def enters(o, inv, blo, bhi):
        t0, t1 = (blo - eps - o) * inv, (bhi + eps - o) * inv
        return np.minimum(t0, t1).max() <= max(np.maximum(t0, t1).min(), 0.0) and np.maximum(t0, t1).min() >= 0

    for _ in range(400):
        o = rng.uniform(-1.5, 1.5, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        inv = 1.0 / np.where(d == 0, 1e-300, d)
        tb = _mt(o, d, tri[:, 0], tri[:, 1], tri[:, 2])
        want = (tb.min(), int(np.argmin(tb))) if np.isfinite(tb.min()) else (np.inf, -1)
        cand, stack = set(), [0]
        while stack:
            k = stack.pop()
            for c in (cl[k], cr[k]):
                if c & 0x80000000:
                    leaf = int(c & 0x7FFFFFFF)
                    if enters(o, inv, llo[leaf], lhi[leaf]):
                        cand.add(int(prim[order[leaf]]))
                else:
                    if enters(o, inv, nlo[c], nhi[c]):
                        stack.append(int(c))
        got = (np.inf, -1)
        if cand:
            c = np.array(sorted(cand))
            tc = _mt(o, d, tri[c, 0], tri[c, 1], tri[c, 2])
            if np.isfinite(tc.min()):
                got = (tc.min(), int(c[np.argmin(tc)]))
        assert got == want, (got, want)
