"""Pins for the oracle's path tracer with next event estimation (Sec. 5), CPU only.

Closed forms: a flat plane under a uniform sky returns albedo x sky after one bounce;
an emitter seen directly returns its emission; a plane under a parallel square light
converges, with direct lighting by next event estimation only, to albedo x emission x
the configuration factor of a parallel rectangle (Howell's catalogue, the
differential-element-to-parallel-rectangle case, summed over four corner rectangles)."""
import math

import numpy as np
import pytest

import oracle
import scenegen

NONE = oracle.NONE


def _rays(o, d, tmin=0.0, tmax=np.inf):
    o = np.atleast_2d(np.asarray(o, np.float64))
    d = np.atleast_2d(np.asarray(d, np.float64))
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    n = max(o.shape[0], d.shape[0])
    r = np.empty((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


def _quad(half, y):
    """Two triangles of the square [-half, half]^2 at height y (x, z plane)."""
    v = np.array([[-half, y, -half], [half, y, -half], [half, y, half], [-half, y, half]], np.float32)
    return v, np.array([[0, 1, 2], [0, 2, 3]], np.uint32)


def test_flat_plane_under_a_uniform_sky():
    plane = scenegen.terrain(cells=16, amplitude=0.0)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(plane.vertices, plane.indices))
    S.build()
    nt = plane.indices.shape[0]
    rho = np.array([0.5, 0.6, 0.7], np.float32)
    sky = np.array([1.0, 2.0, 3.0], np.float32)
    rng = np.random.default_rng(5)
    tgt = np.c_[rng.uniform(-0.9, 0.9, 500), np.zeros(500), rng.uniform(-0.9, 0.9, 500)]
    org = tgt + np.c_[rng.uniform(-1, 1, 500), np.full(500, 3.0), rng.uniform(-1, 1, 500)]
    rays = np.concatenate([_rays(org, tgt - org), _rays([[0, 3, 0]], [[0, 1, 0]])])  # the last ray escapes
    alb = np.tile(rho, (nt, 1))
    emi = np.zeros((nt, 3), np.float32)
    for depth in (2, 3):
        L = S.path_trace(rays, alb, emi, [0], np.zeros((0, 2)), depth, 2, 11, sky)
        assert np.allclose(L[:-1], rho.astype(np.float64) * sky, rtol=1e-12)  # one bounce, then the sky
        assert np.allclose(L[-1], sky)
    L1 = S.path_trace(rays, alb, emi, [0], np.zeros((0, 2)), 1, 2, 11, sky)
    assert np.all(L1[:-1] == 0.0)  # the path ends at its first vertex without light


def test_emitter_seen_directly_and_not_counted_again():
    v, i = _quad(0.5, 1.0)
    S = oracle.Scene()
    g = S.add_mesh(v, i)
    S.add_instance(g)
    S.build()
    Le = np.array([4.0, 5.0, 6.0], np.float32)
    rays = _rays([[0.1, 3.0, 0.2], [0.1, -3.0, -0.1]], [[0, -1, 0], [0, 1, 0]])
    L = S.path_trace(rays, np.full((2, 3), 0.5, np.float32), np.tile(Le, (2, 1)), [0], [[0, 0], [0, 1]], 4, 3, 2,
                     np.zeros(3, np.float32))
    assert np.allclose(L, Le.astype(np.float64)[None, :], rtol=1e-12)


def _corner_factor(x, y):
    """Configuration factor from a differential element to a parallel rectangle of
    sides x, y (in units of the height) with one corner above the element."""
    if x <= 0 or y <= 0:
        return 0.0
    a, b = x / math.sqrt(1 + x * x), y / math.sqrt(1 + y * y)
    return (a * math.atan(y / math.sqrt(1 + x * x)) + b * math.atan(x / math.sqrt(1 + y * y))) / (2 * math.pi)


@pytest.mark.parametrize("h", [0.5, 1.0])
def test_next_event_estimation_matches_the_parallel_square_form_factor(h):
    plane = scenegen.terrain(cells=16, amplitude=0.0)
    lv, li = _quad(0.5, h)
    S = oracle.Scene()
    S.add_instance(S.add_mesh(plane.vertices, plane.indices))
    S.add_instance(S.add_mesh(lv, li))
    S.build()
    nt = plane.indices.shape[0]
    rho = np.array([0.8, 0.5, 0.25], np.float32)
    Le = np.array([2.0, 3.0, 4.0], np.float32)
    alb = np.concatenate([np.tile(rho, (nt, 1)), np.zeros((2, 3), np.float32)])
    emi = np.concatenate([np.zeros((nt, 3), np.float32), np.tile(Le, (2, 1))])
    p = np.array([0.0371, 0.0, -0.0213])  # inside a cell, under the light
    org = p + np.array([2.5, 0.3 * h, 0.4])  # an oblique ray that passes below the light
    rays = _rays([org], [p - org])
    L = S.path_trace(rays, alb, emi, [0, nt], [[1, 0], [1, 1]], 1, 40000, 7, np.zeros(3, np.float32))[0]
    # four corner rectangles of the square around the point's foot
    dx, dz = 0.5 - p[0], 0.5 - p[2]
    ex, ez = 0.5 + p[0], 0.5 + p[2]
    F = sum(_corner_factor(a / h, b / h) for a, b in ((dx, dz), (dx, ez), (ex, dz), (ex, ez)))
    expect = rho.astype(np.float64) * Le * F
    assert np.allclose(L, expect, rtol=0.02), (L, expect, F)
