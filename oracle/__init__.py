"""CPU oracle for BVH build and ray tracing (FP64). TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg may import
this package. It shares no code with the CUDA library: its C++ sources
(build_ref.cpp, trace_ref.cpp, shade_ref.cpp) are compiled by `build()` into
`_liboracle.so` with g++ and called through ctypes. Every function restates a
definition from the paper ("Ray Tracing using HIP": Sec. 3.1 ray/triangle, Sec. 3.2
camera, Sec. 4 ambient occlusion, Sec. 6.2 BVH construction, refit, traversal and
two-level instancing) or from the published methods the LBVH build uses (Karras
2012; Moller-Trumbore 1997), in plain sequential form.

Pins (tests/test_oracle_*.py) tie each function to something other than itself:
hand-computed Morton codes, closed-form sphere/plane/quad hits, brute force vs the
oracle's BVH, the paper's plane/edge formula vs Moller-Trumbore, BVH invariants.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["build_ref.cpp", "trace_ref.cpp", "shade_ref.cpp", "lambert_ref.cpp", "split_ref.cpp"]
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF
LEAF_BIT = 0x80000000


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2, no fused multiply-add) into _liboracle.so."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    if not force and os.path.exists(_LIB_PATH):
        mt = os.path.getmtime(_LIB_PATH)
        deps = srcs + [os.path.join(_HERE, "oracle_math.h")]
        if all(os.path.getmtime(s) <= mt for s in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.oracle_scene_new.restype = P
            L.oracle_scene_free.argtypes = [P]
            L.oracle_scene_add_mesh.argtypes = [P, P, i64, P, i64]
            L.oracle_scene_add_spheres.argtypes = [P, P, i64]
            L.oracle_scene_add_discs.argtypes = [P, P, i64]
            L.oracle_min_disc_margin.argtypes = [P, P]
            L.oracle_min_disc_margin.restype = ctypes.c_double
            L.oracle_scene_add_instance.argtypes = [P, ctypes.c_int, P]
            L.oracle_scene_build.argtypes = [P]
            L.oracle_trace.argtypes = [P, P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, P, P, P,
                                       P, P]
            L.oracle_scene_set_instance_mask.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_scene_set_prim_filter.argtypes = [P, ctypes.c_int, P]
            L.oracle_path_trace.argtypes = [P, P, i64, P, P, P, P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                            P, ctypes.c_int, P]
            L.oracle_all_hits.argtypes = [P, P, i64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, i64, P, P, P, P, P,
                                          P]
            L.oracle_intersect_prim.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, P, P, P]
            L.oracle_min_edge_margin.argtypes = [P, P]
            L.oracle_min_edge_margin.restype = ctypes.c_double
            L.oracle_min_sphere_margin.argtypes = [P, P]
            L.oracle_min_sphere_margin.restype = ctypes.c_double
            L.oracle_plane_edge_test.argtypes = [P, P, P, P, P]
            L.oracle_mt_test.argtypes = [P, P, P, P, P]
            L.oracle_instance_frames.argtypes = [P, ctypes.c_uint32, P, P]
            L.oracle_world_triangle.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, P]
            L.oracle_triangle_aabbs.argtypes = [P, i64, P, P, P, P]
            L.oracle_box_centroids.argtypes = [P, i64, P]
            L.oracle_morton.argtypes = [P, i64, P, P, ctypes.c_int, P]
            L.oracle_centroid_bounds.argtypes = [P, i64, P, P]
            L.oracle_stable_sort.argtypes = [P, i64, P, P]
            L.oracle_topology.argtypes = [P, i64, ctypes.c_int, P, P, P, P]
            L.oracle_fit.argtypes = [P, P, i64, P, P, P, P]
            L.oracle_ploc.argtypes = [P, P, i64, ctypes.c_int, P, P, P, P, P]
            L.oracle_subtree_cluster.argtypes = [P, P, i64, ctypes.c_int, P, P, P, P, P, P]
            L.oracle_sah_cost.argtypes = [P, P, i64]
            L.oracle_sah_cost.restype = ctypes.c_double
            L.oracle_quantize_wide.argtypes = [P, P, P, i64, P]
            L.oracle_split_triangles.argtypes = [P, i64, ctypes.c_uint32, ctypes.c_int, P, P, P, P, P]
            L.oracle_split_triangles.restype = ctypes.c_int64
            L.oracle_xi.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            L.oracle_xi.restype = ctypes.c_double
            L.oracle_camera_rays.argtypes = [P, i64, i64, P]
            L.oracle_uniform_rays.argtypes = [P, P, ctypes.c_uint64, i64, ctypes.c_float, ctypes.c_float, P]
            L.oracle_sample_hemisphere.argtypes = [ctypes.c_double, ctypes.c_double, P]
            L.oracle_ao_rays.argtypes = [P, P, P, P, i64, ctypes.c_int, ctypes.c_uint64, ctypes.c_float, P]
            L.oracle_lambert_forward.argtypes = [P, i64, P, i64, P, P, P, i64, P, P, P, P, P]
            L.oracle_lambert_gradient.argtypes = [P, i64, P, i64, P, P, P, i64, P, P, P, P]
            L.oracle_lambert_gradient.restype = ctypes.c_double
            L.oracle_lambert_gradient_l1.argtypes = [P, i64, P, i64, P, P, P, i64, P, P, P, P]
            L.oracle_lambert_fd.argtypes = [P, i64, P, i64, P, P, P, i64, P, P, i64, ctypes.c_double, P, P, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------------
# Build steps (bit-exact definitions)
# ----------------------------------------------------------------------------------
def triangle_aabbs(vertices: np.ndarray, indices: np.ndarray):
    """Per-triangle AABB lo, hi and centroid 0.5*(lo+hi), float32 (n,3) each."""
    v = _c(vertices, np.float32)
    idx = _c(indices, np.uint32)
    n = idx.shape[0]
    lo = np.empty((n, 3), np.float32)
    hi = np.empty((n, 3), np.float32)
    c = np.empty((n, 3), np.float32)
    lib().oracle_triangle_aabbs(_p(idx), n, _p(v), _p(lo), _p(hi), _p(c))
    return lo, hi, c


def box_centroids(boxes: np.ndarray) -> np.ndarray:
    b = _c(boxes, np.float32).reshape(-1, 6)
    c = np.empty((b.shape[0], 3), np.float32)
    lib().oracle_box_centroids(_p(b), b.shape[0], _p(c))
    return c


def centroid_bounds(centroids: np.ndarray):
    c = _c(centroids, np.float32).reshape(-1, 3)
    lo = np.empty(3, np.float32)
    hi = np.empty(3, np.float32)
    lib().oracle_centroid_bounds(_p(c), c.shape[0], _p(lo), _p(hi))
    return lo, hi


def morton(centroids: np.ndarray, lo, hi, bits_per_axis: int) -> np.ndarray:
    """Morton codes (uint64 holding 30 or 63 bits)."""
    c = _c(centroids, np.float32).reshape(-1, 3)
    out = np.empty(c.shape[0], np.uint64)
    lib().oracle_morton(_p(c), c.shape[0], _p(_c(lo, np.float32)), _p(_c(hi, np.float32)), bits_per_axis, _p(out))
    return out


def stable_sort(codes: np.ndarray):
    """(sorted codes, order) with equal codes kept in input order."""
    k = _c(codes, np.uint64)
    sk = np.empty_like(k)
    order = np.empty(k.shape[0], np.uint32)
    lib().oracle_stable_sort(_p(k), k.shape[0], _p(sk), _p(order))
    return sk, order


def topology(sorted_keys: np.ndarray, keybits: int):
    """Karras-numbered binary hierarchy: (childL, childR, parent_internal, parent_leaf).
    Leaf children carry bit 31 (as int32, negative)."""
    k = _c(sorted_keys, np.uint64)
    n = k.shape[0]
    m = max(n - 1, 0)
    cl = np.full(m, -1, np.int32)
    cr = np.full(m, -1, np.int32)
    pi = np.full(m, -1, np.int32)
    pl = np.full(n, -1, np.int32)
    if n >= 2:
        lib().oracle_topology(_p(k), n, keybits, _p(cl), _p(cr), _p(pi), _p(pl))
    return cl, cr, pi, pl


def fit(childL, childR, leaf_lo, leaf_hi):
    """Internal-node boxes (lo, hi), float32 (n-1,3)."""
    cl = _c(childL, np.int32)
    cr = _c(childR, np.int32)
    lo = _c(leaf_lo, np.float32)
    hi = _c(leaf_hi, np.float32)
    n = lo.shape[0]
    nlo = np.empty((max(n - 1, 0), 3), np.float32)
    nhi = np.empty((max(n - 1, 0), 3), np.float32)
    if n >= 2:
        lib().oracle_fit(_p(cl), _p(cr), n, _p(lo), _p(hi), _p(nlo), _p(nhi))
    return nlo, nhi


SPLIT_MAX = 31  # splits a triangle takes from the budget by priority (one more may come from the remainder)


def split_budget(count: int, factor: float) -> int:
    """Extra references of a split build of `count` triangles: floor(factor * count) in
    double, factor the float32 split factor (0 selects 0.5)."""
    f = float(np.float32(factor)) if factor else 0.5
    return int(math.floor(f * float(count)))


def split_triangles(vertices: np.ndarray, indices: np.ndarray, budget: int, max_splits: int = SPLIT_MAX):
    """Spatial splits of the triangles before a build (split_ref.cpp): (lo, hi) float32
    (m,3) reference boxes, prim uint32 (m,), owner bool (m,) and the per-triangle split
    counts, with m = n + budget references numbered triangle by triangle."""
    v = _c(vertices, np.float32)
    idx = _c(indices, np.uint32)
    n = idx.shape[0]
    tris = np.ascontiguousarray(v[idx.reshape(-1)].reshape(n, 9), np.float32)
    m = n + int(budget)
    lo = np.empty((m, 3), np.float32)
    hi = np.empty((m, 3), np.float32)
    prim = np.empty(m, np.uint32)
    owner = np.empty(m, np.uint8)
    splits = np.empty(n, np.uint32)
    got = lib().oracle_split_triangles(_p(tris), n, int(budget), int(max_splits), _p(lo), _p(hi), _p(prim),
                                       _p(owner), _p(splits))
    if got != m:
        raise ValueError("split budget above the triangle count")
    return lo, hi, prim, owner.astype(bool), splits


def sah_cost(node_lo, node_hi) -> float:
    lo = _c(node_lo, np.float32)
    hi = _c(node_hi, np.float32)
    return float(lib().oracle_sah_cost(_p(lo), _p(hi), lo.shape[0]))


def lbvh(leaf_lo, leaf_hi, centroids, bits_per_axis: int):
    """The whole LBVH reference: bounds, Morton, stable sort, topology, fit. Returns a dict."""
    clo, chi = centroid_bounds(centroids)
    codes = morton(centroids, clo, chi, bits_per_axis)
    sk, order = stable_sort(codes)
    keybits = 32 if bits_per_axis == 10 else 64
    cl, cr, pi, pl = topology(sk, keybits)
    slo = np.ascontiguousarray(np.asarray(leaf_lo)[order])
    shi = np.ascontiguousarray(np.asarray(leaf_hi)[order])
    nlo, nhi = fit(cl, cr, slo, shi)
    return dict(centroid_lo=clo, centroid_hi=chi, codes=codes, sorted_codes=sk, order=order, childL=cl,
                childR=cr, parent_internal=pi, parent_leaf=pl, node_lo=nlo, node_hi=nhi, leaf_lo=slo,
                leaf_hi=shi)


def ploc_topology(leaf_lo, leaf_hi, radius: int):
    """Clustering hierarchy over leaves in sorted order: (childL, childR, parent_internal,
    parent_leaf, iterations), in the format of topology()."""
    lo = _c(leaf_lo, np.float32)
    hi = _c(leaf_hi, np.float32)
    n = lo.shape[0]
    m = max(n - 1, 0)
    cl = np.full(m, -1, np.int32)
    cr = np.full(m, -1, np.int32)
    pi = np.full(m, -1, np.int32)
    pl = np.full(n, -1, np.int32)
    it = np.zeros(1, np.int64)
    if n >= 2:
        lib().oracle_ploc(_p(lo), _p(hi), n, int(radius), _p(cl), _p(cr), _p(pi), _p(pl), _p(it))
    return cl, cr, pi, pl, int(it[0])


def ploc(leaf_lo, leaf_hi, centroids, bits_per_axis: int, radius: int):
    """The whole clustering-build reference: the LBVH's Morton order (bounds, codes,
    stable sort), then clustering with the given search radius, then the fit. Returns a
    dict with the keys of lbvh() plus 'iterations'."""
    clo, chi = centroid_bounds(centroids)
    codes = morton(centroids, clo, chi, bits_per_axis)
    sk, order = stable_sort(codes)
    slo = np.ascontiguousarray(np.asarray(leaf_lo)[order])
    shi = np.ascontiguousarray(np.asarray(leaf_hi)[order])
    cl, cr, pi, pl, iters = ploc_topology(slo, shi, radius)
    nlo, nhi = fit(cl, cr, slo, shi)
    return dict(centroid_lo=clo, centroid_hi=chi, codes=codes, sorted_codes=sk, order=order, childL=cl,
                childR=cr, parent_internal=pi, parent_leaf=pl, node_lo=nlo, node_hi=nhi, leaf_lo=slo,
                leaf_hi=shi, iterations=iters)


def subtree_cluster_topology(leaf_lo, leaf_hi, lbvh_childL, lbvh_childR, cap: int):
    """Clustering inside the LBVH's subtrees (oracle_subtree_cluster): (childL, childR,
    parent_internal, parent_leaf) in the format of topology()."""
    lo = _c(leaf_lo, np.float32)
    hi = _c(leaf_hi, np.float32)
    n = lo.shape[0]
    m = max(n - 1, 0)
    cl = np.full(m, -1, np.int32)
    cr = np.full(m, -1, np.int32)
    pi = np.full(m, -1, np.int32)
    pl = np.full(n, -1, np.int32)
    if n >= 2:
        L0, R0 = _c(lbvh_childL, np.int32), _c(lbvh_childR, np.int32)
        lib().oracle_subtree_cluster(_p(lo), _p(hi), n, int(cap), _p(L0), _p(R0), _p(cl), _p(cr), _p(pi), _p(pl))
    return cl, cr, pi, pl


def subtree_cluster(leaf_lo, leaf_hi, centroids, bits_per_axis: int, cap: int):
    """The whole subtree-clustering build reference: the LBVH (bounds, codes, stable sort,
    Karras topology), clustering inside its subtrees with cluster cap `cap`, then the
    fit. Returns a dict with the keys of lbvh() plus lbvh_childL / lbvh_childR."""
    ref = lbvh(leaf_lo, leaf_hi, centroids, bits_per_axis)
    cl, cr, pi, pl = subtree_cluster_topology(ref["leaf_lo"], ref["leaf_hi"], ref["childL"], ref["childR"], cap)
    nlo, nhi = fit(cl, cr, ref["leaf_lo"], ref["leaf_hi"])
    return dict(ref, lbvh_childL=ref["childL"], lbvh_childR=ref["childR"], childL=cl, childR=cr, parent_internal=pi,
                parent_leaf=pl, node_lo=nlo, node_hi=nhi)


def wide_nodes(ref):
    """4-wide nodes from a binary LBVH (the dict of lbvh()), by definition: wide node k has
    binary node k's two children, each internal child replaced by its own two children.
    Slots 2s and 2s+1 come from child s: its two children, or the leaf itself and an
    empty slot (index 0xFFFFFFFF, box lo = +inf, hi = -inf). Returns lo, hi (m, 4, 3)
    float32 and child (m, 4) uint32, m = max(n - 1, 1). Child words use the binary
    format: bit 31 set = leaf, low bits = sorted position."""
    n = ref["leaf_lo"].shape[0]
    m = max(n - 1, 1)
    lo = np.full((m, 4, 3), np.inf, np.float32)
    hi = np.full((m, 4, 3), -np.inf, np.float32)
    child = np.full((m, 4), NONE, np.uint32)
    if n == 1:  # a single primitive: one node, the leaf in slot 0
        lo[0, 0], hi[0, 0], child[0, 0] = ref["leaf_lo"][0], ref["leaf_hi"][0], LEAF_BIT
        return lo, hi, child
    cl = ref["childL"].view(np.uint32)
    cr = ref["childR"].view(np.uint32)
    all_lo = np.concatenate([ref["node_lo"], ref["leaf_lo"]])  # internal nodes, then leaves
    all_hi = np.concatenate([ref["node_hi"], ref["leaf_hi"]])
    for s_, c in enumerate((cl, cr)):
        leaf = (c & LEAF_BIT) != 0
        inner = np.where(leaf, 0, c & 0x7FFFFFFF)
        first = np.where(leaf, c, cl[inner])  # the leaf itself, or the child's two children
        second = np.where(leaf, np.uint32(NONE), cr[inner])
        for j, g in enumerate((first, second)):
            used = g != NONE
            row = np.where(g & LEAF_BIT, n - 1 + (g & 0x7FFFFFFF), g).astype(np.int64)
            lo[used, 2 * s_ + j] = all_lo[row[used]]
            hi[used, 2 * s_ + j] = all_hi[row[used]]
            child[:, 2 * s_ + j] = g
    return lo, hi, child


# ----------------------------------------------------------------------------------
# Scenes and traces
# ----------------------------------------------------------------------------------
def wide8_nodes(ref):
    """8-wide nodes from a binary LBVH (the dict of lbvh()), by definition: wide node k has
    binary node k's descendants three levels down. Slots 4s..4s+3 come from child s: if it
    is a leaf, slot 4s holds it and 4s+1..4s+3 are empty; otherwise each of its children t
    fills slots 4s+2t and 4s+2t+1 with its own two children, or with itself (a leaf) and
    an empty slot. Empty slots: index 0xFFFFFFFF, box lo = +inf, hi = -inf. Returns lo, hi
    (m, 8, 3) float32 and child (m, 8) uint32, m = max(n - 1, 1). Child words use the
    binary format (bit 31 set = leaf, low bits = sorted position). A walk from node 0 only
    meets the nodes of binary depth divisible by 3."""
    n = ref["leaf_lo"].shape[0]
    m = max(n - 1, 1)
    lo = np.full((m, 8, 3), np.inf, np.float32)
    hi = np.full((m, 8, 3), -np.inf, np.float32)
    child = np.full((m, 8), NONE, np.uint32)
    if n == 1:  # a single primitive: one node, the leaf in slot 0
        lo[0, 0], hi[0, 0], child[0, 0] = ref["leaf_lo"][0], ref["leaf_hi"][0], LEAF_BIT
        return lo, hi, child
    cl = ref["childL"].view(np.uint32)
    cr = ref["childR"].view(np.uint32)
    all_lo = np.concatenate([ref["node_lo"], ref["leaf_lo"]])  # internal nodes, then leaves
    all_hi = np.concatenate([ref["node_hi"], ref["leaf_hi"]])

    def put(k, slot, w):
        child[k, slot] = w
        row = n - 1 + (w & 0x7FFFFFFF) if w & LEAF_BIT else w
        lo[k, slot], hi[k, slot] = all_lo[row], all_hi[row]

    for k in range(n - 1):
        for s_, c in enumerate((int(cl[k]), int(cr[k]))):
            if c & LEAF_BIT:
                put(k, 4 * s_, c)
                continue
            for t, g in enumerate((int(cl[c]), int(cr[c]))):
                if g & LEAF_BIT:
                    put(k, 4 * s_ + 2 * t, g)
                else:
                    put(k, 4 * s_ + 2 * t, int(cl[g]))
                    put(k, 4 * s_ + 2 * t + 1, int(cr[g]))
    return lo, hi, child


def quantized_wide_nodes(lo, hi, child) -> np.ndarray:
    """Quantised 4-wide nodes (oracle_quantize_wide) of the wide nodes (lo, hi (m, 4, 3)
    float32, child (m, 4) uint32) that wide_nodes returns: (m, 16) uint32 words per node,
    p.xyz, biased exponents, the six plane words (slot j in byte j), the child words."""
    lo, hi = _c(lo, np.float32), _c(hi, np.float32)
    child = _c(child, np.uint32)
    m = lo.shape[0]
    out = np.zeros((m, 16), np.uint32)
    if m:
        lib().oracle_quantize_wide(_p(lo), _p(hi), _p(child), m, _p(out))
    return out


def dequantize_wide_nodes(q: np.ndarray):
    """Decoded slot boxes of quantised nodes: plane = fl32(p + byte * 2^e), per axis.
    Returns lo, hi (m, 4, 3) float32 (empty slots decode to whatever their bytes say)."""
    q = np.asarray(q, np.uint32)
    m = q.shape[0]
    p = q[:, 0:3].copy().view(np.float32)  # (m, 3)
    e = np.stack([(q[:, 3] >> (8 * a)) & 0xFF for a in range(3)], axis=1).astype(np.int32) - 127
    step = np.ldexp(np.float32(1.0), e).astype(np.float32)  # (m, 3)
    lo = np.zeros((m, 4, 3), np.float32)
    hi = np.zeros((m, 4, 3), np.float32)
    for a in range(3):
        for j in range(4):
            ql = ((q[:, 4 + 2 * a] >> (8 * j)) & 0xFF).astype(np.float32)
            qh = ((q[:, 5 + 2 * a] >> (8 * j)) & 0xFF).astype(np.float32)
            with np.errstate(over="ignore"):
                lo[:, j, a] = p[:, a] + ql * step[:, a]
                hi[:, j, a] = p[:, a] + qh * step[:, a]
    return lo, hi


class Hits:
    """Hit records in FP64: inst, prim (uint32; NONE on a miss), t (+inf on miss), u, v."""

    def __init__(self, n: int):
        self.inst = np.full(n, NONE, np.uint32)
        self.prim = np.full(n, NONE, np.uint32)
        self.t = np.full(n, np.inf)
        self.u = np.zeros(n)
        self.v = np.zeros(n)

    def __len__(self):
        return self.prim.shape[0]


class Scene:
    """An oracle scene: geometries (meshes or spheres) and instances with SRT frames."""

    def __init__(self):
        self._L = lib()
        self._h = ctypes.c_void_p(self._L.oracle_scene_new())
        self._keep = []

    def __del__(self):
        try:
            if self._h:
                self._L.oracle_scene_free(self._h)
                self._h = None
        except Exception:
            pass

    def add_mesh(self, vertices, indices) -> int:
        v = _c(vertices, np.float32)
        i = _c(indices, np.uint32)
        return int(self._L.oracle_scene_add_mesh(self._h, _p(v), v.shape[0], _p(i), i.shape[0]))

    def add_spheres(self, spheres) -> int:
        s = _c(spheres, np.float32).reshape(-1, 4)
        return int(self._L.oracle_scene_add_spheres(self._h, _p(s), s.shape[0]))

    def add_discs(self, discs) -> int:
        """Discs as float32 (n, 8): centre xyz, radius, normal xyz, unused (a custom
        primitive; the oracle normalises the normal in FP64)."""
        d = _c(discs, np.float32).reshape(-1, 8)
        self._keep.append(d)
        return self._L.oracle_scene_add_discs(self._h, _p(d), d.shape[0])

    def add_instance(self, geom: int, frame=None):
        if frame is None:
            self._L.oracle_scene_add_instance(self._h, geom, None)
        else:
            f = _c(frame, np.float32).reshape(10)
            self._L.oracle_scene_add_instance(self._h, geom, _p(f))

    def set_prim_filter(self, geom: int, bits):
        """Intersection filter (Sec. 7.6) of geometry `geom` as a primitive mask: hits on
        primitive i stand only when bit i of `bits` (uint32 words, word i // 32) is set."""
        b = _c(bits, np.uint32)
        self._keep.append(b)
        self._L.oracle_scene_set_prim_filter(self._h, geom, _p(b))

    def set_instance_mask(self, inst: int, mask: int):
        """Instance `inst`'s 32-bit visibility mask (Sec. 7.5; default all bits set): a ray
        sees the instance only when the mask ANDed with the ray's mask is nonzero."""
        self._L.oracle_scene_set_instance_mask(self._h, inst, mask & 0xFFFFFFFF)

    def build(self):
        self._L.oracle_scene_build(self._h)

    def trace(self, rays, any_hit: bool = False, bvh: bool = True, threads: int = 0,
              ray_mask: int = 0xFFFFFFFF) -> Hits:
        r = _c(rays, np.float32).reshape(-1, 8)
        h = Hits(r.shape[0])
        self._L.oracle_trace(self._h, _p(r), r.shape[0], int(any_hit), int(bvh), threads, ray_mask & 0xFFFFFFFF,
                             _p(h.inst), _p(h.prim), _p(h.t), _p(h.u), _p(h.v))
        return h

    def all_hits(self, rays, max_hits: int, bvh: bool = True, threads: int = 0, ray_mask: int = 0xFFFFFFFF):
        """Every hit of each ray (Sec. 7.5), sorted by (t, instance, primitive): arrays
        inst, prim, t, u, v of shape (n, max_hits) (misses after the last hit) and the
        number of hits per ray (n,), which may exceed max_hits."""
        r = _c(rays, np.float32).reshape(-1, 8)
        n = r.shape[0]
        inst = np.empty((n, max_hits), np.uint32)
        prim = np.empty((n, max_hits), np.uint32)
        t = np.empty((n, max_hits))
        u = np.empty((n, max_hits))
        v = np.empty((n, max_hits))
        cnt = np.empty(n, np.int64)
        self._L.oracle_all_hits(self._h, _p(r), n, int(bvh), threads, ray_mask & 0xFFFFFFFF, max_hits, _p(inst),
                                _p(prim), _p(t), _p(u), _p(v), _p(cnt))
        return inst, prim, t, u, v, cnt

    def path_trace(self, rays, albedo, emission, mat_offset, lights, max_depth: int, spp: int, seed: int, sky,
                   threads: int = 0) -> np.ndarray:
        """Path tracing with next event estimation (Sec. 5) from the given float32 rays:
        the mean radiance over `spp` samples, (n, 3) FP64. albedo / emission: (M, 3)
        per material entry, entry mat_offset[instance] + primitive; lights: (K, 2)
        (instance, primitive) pairs of emitting triangles; sky: radiance of escaping
        rays. The steps are listed at oracle_path_trace (trace_ref.cpp)."""
        r = _c(rays, np.float32).reshape(-1, 8)
        a = _c(albedo, np.float32).reshape(-1, 3)
        e = _c(emission, np.float32).reshape(-1, 3)
        mo = _c(mat_offset, np.uint32)
        li = _c(lights, np.uint32).reshape(-1, 2)
        sk = _c(sky, np.float32).reshape(3)
        out = np.empty((r.shape[0], 3))
        self._L.oracle_path_trace(self._h, _p(r), r.shape[0], _p(a), _p(e), _p(mo), _p(li), li.shape[0], max_depth,
                                  spp, seed, _p(sk), threads, _p(out))
        return out

    def intersect_prim(self, ray, inst: int, prim: int):
        """(hit, t, u, v) of one (instance, primitive) in FP64."""
        r = _c(ray, np.float32).reshape(8)
        t = ctypes.c_double()
        u = ctypes.c_double()
        v = ctypes.c_double()
        ok = self._L.oracle_intersect_prim(self._h, _p(r), inst, prim, ctypes.byref(t), ctypes.byref(u),
                                           ctypes.byref(v))
        return bool(ok), t.value, u.value, v.value

    def min_edge_margin(self, ray) -> float:
        r = _c(ray, np.float32).reshape(8)
        return float(self._L.oracle_min_edge_margin(self._h, _p(r)))

    def min_disc_margin(self, ray) -> float:
        r = _c(ray, np.float32).reshape(8)
        return float(self._L.oracle_min_disc_margin(self._h, _p(r)))

    def min_sphere_margin(self, ray) -> float:
        r = _c(ray, np.float32).reshape(8)
        return float(self._L.oracle_min_sphere_margin(self._h, _p(r)))

    def instance_frames(self, inst: int):
        f = np.empty(12)
        g = np.empty(12)
        self._L.oracle_instance_frames(self._h, inst, _p(f), _p(g))
        return f.reshape(3, 4), g.reshape(3, 4)

    def world_triangle(self, inst: int, prim: int) -> np.ndarray:
        out = np.empty(9)
        ok = self._L.oracle_world_triangle(self._h, inst, prim, _p(out))
        if not ok:
            raise ValueError("not a triangle")
        return out.reshape(3, 3)


def mt_test(ray, tri):
    r = _c(ray, np.float32).reshape(8)
    t9 = _c(tri, np.float32).reshape(9)
    t = ctypes.c_double()
    u = ctypes.c_double()
    v = ctypes.c_double()
    ok = lib().oracle_mt_test(_p(r), _p(t9), ctypes.byref(t), ctypes.byref(u), ctypes.byref(v))
    return bool(ok), t.value, u.value, v.value


def plane_edge_test(ray, tri):
    r = _c(ray, np.float32).reshape(8)
    t9 = _c(tri, np.float32).reshape(9)
    t = ctypes.c_double()
    u = ctypes.c_double()
    v = ctypes.c_double()
    ok = lib().oracle_plane_edge_test(_p(r), _p(t9), ctypes.byref(t), ctypes.byref(u), ctypes.byref(v))
    return bool(ok), t.value, u.value, v.value


# ----------------------------------------------------------------------------------
# Ray generation
# ----------------------------------------------------------------------------------
def camera_rays(camera_packed, width: int, height: int) -> np.ndarray:
    """Pinhole camera rays (paper Sec. 3.2) at pixel centres, float32 (W*H, 8)."""
    cam = _c(camera_packed, np.float32).reshape(9)
    out = np.empty((width * height, 8), np.float32)
    lib().oracle_camera_rays(_p(cam), width, height, _p(out))
    return out


def uniform_rays(lo, hi, seed: int, count: int, tmin: float = 0.0, tmax: float = float("inf")) -> np.ndarray:
    """count rays, origins uniform in the box [lo, hi], directions uniform on the unit
    sphere (FP64, rounded to float32), from the splitmix64 stream `seed`."""
    out = np.empty((count, 8), np.float32)
    lib().oracle_uniform_rays(_p(_c(lo, np.float32).reshape(3)), _p(_c(hi, np.float32).reshape(3)),
                              ctypes.c_uint64(seed), count, ctypes.c_float(tmin), ctypes.c_float(tmax), _p(out))
    return out


def xi(seed: int, pixel: int, sample: int, dim: int) -> float:
    return float(lib().oracle_xi(seed, pixel, sample, dim))


def sample_hemisphere(xi0: float, xi1: float) -> np.ndarray:
    out = np.empty(3)
    lib().oracle_sample_hemisphere(xi0, xi1, _p(out))
    return out


def ao_rays(scene: Scene, primary_rays, hits: Hits, spp: int, seed: int, length: float) -> np.ndarray:
    """Ambient-occlusion rays (paper Sec. 4) for each pixel's oracle primary hit."""
    r = _c(primary_rays, np.float32).reshape(-1, 8)
    n = r.shape[0]
    tri = np.zeros((n, 9))
    for p in np.nonzero(hits.prim != NONE)[0]:
        tri[p] = scene.world_triangle(int(hits.inst[p]), int(hits.prim[p])).ravel()
    out = np.empty((n * spp, 8), np.float32)
    lib().oracle_ao_rays(_p(r), _p(tri), _p(_c(hits.prim, np.uint32)), _p(_c(hits.t, np.float64)), n, spp,
                         ctypes.c_uint64(seed), ctypes.c_float(length), _p(out))
    return out


# ----------------------------------------------------------------------------------
# Lambertian shading and its gradient (FP64, brute-force visibility)
# ----------------------------------------------------------------------------------
class LambertResult:
    def __init__(self, n: int):
        self.image = np.zeros((n, 3))
        self.prim = np.full(n, -1, np.int32)
        self.vis = np.zeros(n, np.int8)
        self.sign = np.zeros(n, np.int8)
        self.tuv = np.zeros((n, 3))


def lambert_forward(vertices, indices, colours, light, rays) -> LambertResult:
    """Image I = V * max(0, n_f . l) * c(u,v) per pixel (see lambert_ref.cpp)."""
    v = _c(vertices, np.float64)
    i = _c(indices, np.uint32)
    c = _c(colours, np.float64)
    l = _c(light, np.float64).reshape(3)
    r = _c(rays, np.float32).reshape(-1, 8)
    R = LambertResult(r.shape[0])
    lib().oracle_lambert_forward(_p(v), v.shape[0], _p(i), i.shape[0], _p(c), _p(l), _p(r), r.shape[0], _p(R.image),
                                 _p(R.prim), _p(R.vis), _p(R.sign), _p(R.tuv))
    return R


def lambert_gradient(vertices, indices, colours, light, rays, target):
    """(loss, dL/dcolours (V,3), dL/dlight (3,), dL/dpositions (V,3)) of L = sum (I - I*)^2."""
    v = _c(vertices, np.float64)
    i = _c(indices, np.uint32)
    c = _c(colours, np.float64)
    l = _c(light, np.float64).reshape(3)
    r = _c(rays, np.float32).reshape(-1, 8)
    t = _c(target, np.float64).reshape(-1, 3)
    dc = np.zeros_like(c)
    dl = np.zeros(3)
    dp = np.zeros_like(v)
    loss = lib().oracle_lambert_gradient(_p(v), v.shape[0], _p(i), i.shape[0], _p(c), _p(l), _p(r), r.shape[0], _p(t),
                                         _p(dc), _p(dl), _p(dp))
    return float(loss), dc, dl, dp


def lambert_gradient_l1(vertices, indices, colours, light, rays, target):
    """Per-parameter sums over pixels of |the pixel's term of the analytic gradient|:
    (colours (V,3), light (3,), positions (V,3)). How much a gradient's terms cancel:
    the accuracy a sum of rounded terms can reach is relative to these, not to the sum."""
    v = _c(vertices, np.float64)
    i = _c(indices, np.uint32)
    c = _c(colours, np.float64)
    l = _c(light, np.float64).reshape(3)
    r = _c(rays, np.float32).reshape(-1, 8)
    t = _c(target, np.float64).reshape(-1, 3)
    ac = np.zeros_like(c)
    al = np.zeros(3)
    ap = np.zeros_like(v)
    lib().oracle_lambert_gradient_l1(_p(v), v.shape[0], _p(i), i.shape[0], _p(c), _p(l), _p(r), r.shape[0], _p(t),
                                     _p(ac), _p(al), _p(ap))
    return ac, al, ap


class LambertScene:
    """Lambert shading of a two-level scene (instances under SRT frames, Sec. 6.2) by the
    plain oracle in world space. One object-space mesh (vertices, indices); instance i
    is its triangles [tri_offset[i], tri_offset[i] + tri_count[i]) under frames[i]
    (quaternion xyzw, scale, translation; the oracle's FP64 frame). The world mesh holds,
    for each instance, every object vertex mapped by the instance's frame; shading,
    visibility (every instance occludes) and the analytic gradient are the plain
    oracle's on it. Gradients come back to object space: colours add up over instances,
    positions as M_i^T g (M_i the linear part of instance i's frame)."""

    def __init__(self, vertices, indices, tri_offset, tri_count, frames):
        v = np.asarray(vertices, np.float64).reshape(-1, 3)
        idx = np.asarray(indices, np.uint32).reshape(-1, 3)
        self.nv = v.shape[0]
        S = Scene()
        g = S.add_mesh(v.astype(np.float32), idx)
        frames = np.asarray(frames, np.float32).reshape(-1, 10)
        for f in frames:
            S.add_instance(g, f)
        self.fwd = [S.instance_frames(i)[0] for i in range(frames.shape[0])]
        self.world_vertices = np.concatenate([v @ F[:, :3].T + F[:, 3] for F in self.fwd])
        tris, inst, prim = [], [], []
        for i, (off, cnt) in enumerate(zip(tri_offset, tri_count)):
            tris.append(idx[off:off + cnt].astype(np.int64) + i * self.nv)
            inst.append(np.full(cnt, i, np.int64))
            prim.append(np.arange(cnt, dtype=np.int64))
        self.world_indices = np.concatenate(tris).astype(np.uint32)
        self.tri_inst = np.concatenate(inst)
        self.tri_prim = np.concatenate(prim)
        self.ninst = frames.shape[0]

    def _colours(self, colours):
        return np.tile(np.asarray(colours, np.float64).reshape(-1, 3), (self.ninst, 1))

    def forward(self, colours, light, rays):
        """LambertResult with .inst and .iprim (instance and primitive within it, -1 on a
        miss) added; .prim stays the world-mesh triangle."""
        R = lambert_forward(self.world_vertices, self.world_indices, self._colours(colours), light, rays)
        hit = R.prim >= 0
        R.inst = np.where(hit, self.tri_inst[np.maximum(R.prim, 0)], -1)
        R.iprim = np.where(hit, self.tri_prim[np.maximum(R.prim, 0)], -1)
        return R

    def _fold(self, dcw, dpw, absolute=False):
        dc = sum(dcw[i * self.nv:(i + 1) * self.nv] for i in range(self.ninst))
        dp = sum(dpw[i * self.nv:(i + 1) * self.nv] @ (np.abs(F[:, :3]) if absolute else F[:, :3])
                 for i, F in enumerate(self.fwd))
        return dc, dp

    def gradient(self, colours, light, rays, target):
        """(loss, dL/dcolours (V,3), dL/dlight (3,), dL/dpositions (V,3), object space)."""
        loss, dcw, dl, dpw = lambert_gradient(self.world_vertices, self.world_indices, self._colours(colours), light,
                                              rays, target)
        dc, dp = self._fold(dcw, dpw)
        return loss, dc, dl, dp

    def gradient_l1(self, colours, light, rays, target):
        """Bounds on the L1 norms of the per-pixel terms of gradient(): per instance the
        world terms' norms mapped by |M_i|^T (a bound on the norm of the mapped terms)."""
        acw, al, apw = lambert_gradient_l1(self.world_vertices, self.world_indices, self._colours(colours), light,
                                           rays, target)
        ac, ap = self._fold(acw, apw, absolute=True)
        return ac, al, ap


def lambert_fd(vertices, indices, colours, light, rays, target, params, h: float = 1e-4, exclude=None,
               return_unstable: bool = False):
    """Central differences (masked loss) for parameter ids: [0,3V) colours, [3V,3V+3) light,
    [3V+3, 6V+3) positions. Returns (fd, analytic gradient of the masked pixels, masked counts)
    and, with return_unstable, the per-pixel mask of pixels unstable for some parameter.
    exclude (bool per pixel) removes pixels from every parameter's loss."""
    v = _c(vertices, np.float64)
    i = _c(indices, np.uint32)
    c = _c(colours, np.float64)
    l = _c(light, np.float64).reshape(3)
    r = _c(rays, np.float32).reshape(-1, 8)
    t = _c(target, np.float64).reshape(-1, 3)
    q = _c(params, np.int64)
    fd = np.zeros(q.shape[0])
    ma = np.zeros(q.shape[0])
    mc = np.zeros(q.shape[0], np.int64)
    ex = None if exclude is None else _c(exclude, np.uint8)
    un = np.zeros(r.shape[0], np.uint8)
    lib().oracle_lambert_fd(_p(v), v.shape[0], _p(i), i.shape[0], _p(c), _p(l), _p(r), r.shape[0], _p(t), _p(q),
                            q.shape[0], h, _p(fd), _p(ma), _p(mc), None if ex is None else _p(ex), _p(un))
    if return_unstable:
        return fd, ma, mc, un.astype(bool)
    return fd, ma, mc
