"""Seeded synthetic inputs: meshes, sphere sets, instance frames and random rays.

This module produces INPUT DATA only. It holds none of the ray-tracing method's
arithmetic (no intersection, no camera model, no hemisphere sampling, no BVH
step); both the CUDA library and the CPU oracle consume what it returns.

Every random number comes from a counter-based splitmix64 stream
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), so a given (seed, stream, counter) gives the same value on every
machine and numpy version.

Workloads (the problem sizes the paper's method is exercised on):
  * icosphere(3): 642 vertices, 1,280 triangles, radius 1 (the smallest scene).
  * terrain(256): 257x257 grid, 131,072 triangles, 4-octave value-noise heights
    of amplitude 0.2, instanced 64 times under random SRT frames.
  * spheres(1M): centres U[-50,50]^3, radii log-uniform [0.01,1], as an AABB list.
  * random rays in a box with directions uniform on the sphere.
  * triangle soups with Gaussian-cluster centroids (many uneven scenes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20260301

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied elementwise to uint64 state values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(*parts: int) -> int:
    """Derive a 64-bit stream key from integers (seed, config, purpose, ...)."""
    k = np.uint64(0)
    with np.errstate(over="ignore"):
        for p in parts:
            k = _mix64(np.uint64(k + np.uint64(p & 0xFFFFFFFFFFFFFFFF) + _GOLDEN))
    return int(k)


def u64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """n counter-based 64-bit words of stream `key` (counters offset..offset+n-1)."""
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(np.uint64(key) + ctr * _GOLDEN)


def uniform(key: int, n: int, offset: int = 0) -> np.ndarray:
    """n float64 values uniform in [0, 1) with 53 random bits each."""
    return (u64(key, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def log_uniform(key: int, n: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * uniform(key, n))


def normal(key: int, n: int) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniform streams."""
    u1 = uniform(key, n, 0)
    u2 = uniform(key, n, n)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
    return r * np.cos(2.0 * math.pi * u2)


def unit_vectors(key: int, n: int) -> np.ndarray:
    """n directions uniform on the unit sphere (float64, shape (n,3))."""
    z = 1.0 - 2.0 * uniform(key, n, 0)
    phi = 2.0 * math.pi * uniform(key, n, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    d = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# ----------------------------------------------------------------------------------
# Meshes
# ----------------------------------------------------------------------------------
@dataclass
class Mesh:
    vertices: np.ndarray  # float32 (V,3)
    indices: np.ndarray   # uint32 (T,3)

    @property
    def num_triangles(self) -> int:
        return int(self.indices.shape[0])


def icosphere(level: int = 3, radius: float = 1.0) -> Mesh:
    """Subdivided icosahedron. Faces split 1->4 (three corner children, then the
    centre child); edge midpoints are shared; vertices are pushed to the sphere in
    float64 and rounded to float32. Faces are counter-clockwise seen from outside.
    level 3 -> 642 vertices, 1,280 faces."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0),
         (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi),
         (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    # make every face CCW seen from outside (normal along the centroid direction)
    fixed = []
    for a, b, c in faces:
        n = np.cross(verts[b] - verts[a], verts[c] - verts[a])
        fixed.append((a, b, c) if np.dot(n, verts[a] + verts[b] + verts[c]) > 0 else (a, c, b))
    faces = fixed
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    vv = (np.array(verts) * radius).astype(np.float32)
    return Mesh(vv, np.array(faces, dtype=np.uint32))


def _value_noise(key: int, octave: int, x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Value noise on a (4*2^octave)-cell lattice over [-1,1]^2: lattice values
    uniform in [-1,1] hashed from (key, octave, ix, iz); bilinear with smoothstep."""
    cells = 4 * (1 << octave)
    gx = (x + 1.0) * 0.5 * cells
    gz = (z + 1.0) * 0.5 * cells
    ix = np.clip(np.floor(gx).astype(np.int64), 0, cells - 1)
    iz = np.clip(np.floor(gz).astype(np.int64), 0, cells - 1)
    fx = gx - ix
    fz = gz - iz
    sx = fx * fx * (3.0 - 2.0 * fx)
    sz = fz * fz * (3.0 - 2.0 * fz)
    okey = stream_key(key, octave)

    def lat(i, j):
        h = _mix64(np.uint64(okey) + (i.astype(np.uint64) * np.uint64(cells + 1) + j.astype(np.uint64) + np.uint64(1)) * _GOLDEN)
        return (h >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0

    v00, v10 = lat(ix, iz), lat(ix + 1, iz)
    v01, v11 = lat(ix, iz + 1), lat(ix + 1, iz + 1)
    a = v00 + (v10 - v00) * sx
    b = v01 + (v11 - v01) * sx
    return a + (b - a) * sz


def terrain(cells: int = 256, amplitude: float = 0.2, seed: int = MASTER_SEED, octaves: int = 4) -> Mesh:
    """Height field on [-1,1]^2 in (x,z), (cells+1)^2 vertices, 2*cells^2 triangles.
    Vertex (i,j) has index j*(cells+1)+i. Cell (i,j) gives triangles 2*(j*cells+i)+{0,1},
    split along (i,j)-(i+1,j+1), counter-clockwise seen from +y.
    height = amplitude * sum_o 0.5^o N_o(x,z) / sum_o 0.5^o."""
    n = cells + 1
    i = np.arange(n, dtype=np.float64)
    xs = -1.0 + 2.0 * i / cells
    X, Z = np.meshgrid(xs, xs, indexing="xy")  # X[j,i], Z[j,i]
    X = X.ravel()
    Z = Z.ravel()
    h = np.zeros_like(X)
    norm = 0.0
    if amplitude != 0.0:
        key = stream_key(seed, 0x7E44A1)
        for o in range(octaves):
            h += (0.5 ** o) * _value_noise(key, o, X, Z)
            norm += 0.5 ** o
        h = amplitude * h / norm
    verts = np.stack([X, h, Z], axis=1).astype(np.float32)
    ci, cj = np.meshgrid(np.arange(cells), np.arange(cells), indexing="xy")
    ci = ci.ravel().astype(np.int64)
    cj = cj.ravel().astype(np.int64)
    a = cj * n + ci
    b = a + 1
    c = a + n + 1
    d = a + n
    t0 = np.stack([a, c, b], axis=1)
    t1 = np.stack([a, d, c], axis=1)
    idx = np.empty((cells * cells * 2, 3), dtype=np.int64)
    idx[0::2] = t0
    idx[1::2] = t1
    return Mesh(verts, idx.astype(np.uint32))


# ----------------------------------------------------------------------------------
# Custom primitives
# ----------------------------------------------------------------------------------
def _round_down_f32(x: np.ndarray) -> np.ndarray:
    f = x.astype(np.float32)
    return np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f).astype(np.float32)


def _round_up_f32(x: np.ndarray) -> np.ndarray:
    f = x.astype(np.float32)
    return np.where(f.astype(np.float64) < x, np.nextafter(f, np.float32(np.inf)), f).astype(np.float32)


def spheres(n: int = 1_000_000, half: float = 50.0, rmin: float = 0.01, rmax: float = 1.0,
            seed: int = MASTER_SEED, config: int = 3) -> np.ndarray:
    """float32 (n,4): centre xyz uniform in [-half,half]^3, radius log-uniform."""
    key = stream_key(seed, config, 0x5B4E)
    c = -half + 2.0 * half * uniform(stream_key(key, 1), 3 * n).reshape(n, 3)
    r = log_uniform(stream_key(key, 2), n, rmin, rmax)
    return np.concatenate([c, r[:, None]], axis=1).astype(np.float32)


def sphere_aabbs(sph: np.ndarray) -> np.ndarray:
    """Boxes (n,6) = lo.xyz, hi.xyz enclosing each float32 sphere, rounded outward
    so the float32 box contains the exact sphere (the AABB-list input)."""
    c = sph[:, :3].astype(np.float64)
    r = sph[:, 3:4].astype(np.float64)
    return np.concatenate([_round_down_f32(c - r), _round_up_f32(c + r)], axis=1).astype(np.float32)


# ----------------------------------------------------------------------------------
# Instances, frames and rays
# ----------------------------------------------------------------------------------
@dataclass
class Frames:
    rotation: np.ndarray     # float32 (n,4) unit quaternion x,y,z,w
    scale: np.ndarray        # float32 (n,3)
    translation: np.ndarray  # float32 (n,3)

    def packed(self) -> np.ndarray:
        """(n,10) float32 rows: rotation xyzw, scale xyz, translation xyz."""
        return np.concatenate([self.rotation, self.scale, self.translation], axis=1).astype(np.float32)


def random_frames(n: int, seed: int = MASTER_SEED, config: int = 2, scale_lo: float = 0.5,
                  scale_hi: float = 2.0, half: float = 10.0) -> Frames:
    """Uniform random rotations (Shoemake 1992 subgroup algorithm), per-axis scale
    uniform in [scale_lo, scale_hi], translation uniform in [-half, half]^3."""
    key = stream_key(seed, config, 0xF4A3)
    u = uniform(stream_key(key, 1), 3 * n).reshape(n, 3)
    u1, u2, u3 = u[:, 0], u[:, 1], u[:, 2]
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * math.pi * u2), a * np.cos(2 * math.pi * u2),
                  b * np.sin(2 * math.pi * u3), b * np.cos(2 * math.pi * u3)], axis=1)
    s = scale_lo + (scale_hi - scale_lo) * uniform(stream_key(key, 2), 3 * n).reshape(n, 3)
    t = -half + 2.0 * half * uniform(stream_key(key, 3), 3 * n).reshape(n, 3)
    return Frames(q.astype(np.float32), s.astype(np.float32), t.astype(np.float32))


def quat_to_matrix64(q: np.ndarray) -> np.ndarray:
    """Rotation matrices (n,3,3) of unit quaternions x,y,z,w (normalised first), float64.
    Used only to place the camera and measure scene extent for input setup."""
    q = q.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    x, y, z, w = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], axis=1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], axis=1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], axis=1),
    ], axis=1)


def world_bounds(meshes: list, geom_of_instance: np.ndarray, frames: Frames) -> tuple[np.ndarray, np.ndarray]:
    """Exact float64 AABB of all instanced vertices (world = T + R*S*x)."""
    R = quat_to_matrix64(frames.rotation)
    lo = np.full(3, np.inf)
    hi = np.full(3, -np.inf)
    for i, g in enumerate(geom_of_instance):
        v = meshes[g].vertices.astype(np.float64) * frames.scale[i].astype(np.float64)
        w = v @ R[i].T + frames.translation[i].astype(np.float64)
        lo = np.minimum(lo, w.min(axis=0))
        hi = np.maximum(hi, w.max(axis=0))
    return lo, hi


def random_rays(n: int, lo, hi, seed: int = MASTER_SEED, config: int = 3, tmin: float = 0.0,
                tmax: float = np.inf) -> np.ndarray:
    """float32 (n,8) rays {origin.xyz, minT, direction.xyz, maxT}: origins uniform in
    the box [lo,hi], unit directions uniform on the sphere."""
    key = stream_key(seed, config, 0xA7A7)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    o = lo + (hi - lo) * uniform(stream_key(key, 1), 3 * n).reshape(n, 3)
    d = unit_vectors(stream_key(key, 2), n)
    r = np.empty((n, 8), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


@dataclass
class Camera:
    """Pinhole camera parameters in the paper's form: lens position, half-width
    vector `right` and half-height vector `up` of the film at distance 1."""
    origin: np.ndarray
    right: np.ndarray
    up: np.ndarray
    width: int
    height: int

    def packed(self) -> np.ndarray:
        return np.concatenate([self.origin, self.right, self.up]).astype(np.float32)


def look_down_z_camera(eye, width: int, height: int, vfov_deg: float = 60.0) -> Camera:
    """Camera at `eye` looking along -z with the given vertical field of view:
    up = (0, tan(fov/2), 0), right = (aspect*tan(fov/2), 0, 0)."""
    th = math.tan(math.radians(vfov_deg) * 0.5)
    aspect = width / height
    return Camera(np.asarray(eye, dtype=np.float32), np.array([aspect * th, 0, 0], dtype=np.float32),
                  np.array([0, th, 0], dtype=np.float32), width, height)


def look_at_camera(eye, target, width: int, height: int, vfov_deg: float = 60.0, world_up=(0.0, 1.0, 0.0)) -> Camera:
    """Camera at `eye` looking at `target` with the given vertical field of view: right
    and up span the film at distance 1 (their cross product up x right points along the
    view direction, the pinhole model's forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, dtype=np.float64))
    if np.linalg.norm(r) < 1e-6:  # looking along the world up: any perpendicular right
        r = np.cross(f, [1.0, 0.0, 0.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(vfov_deg) * 0.5)
    return Camera(eye.astype(np.float32), (r * (width / height) * th).astype(np.float32),
                  (u * th).astype(np.float32), width, height)


# ----------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------
@dataclass
class InstancedScene:
    meshes: list
    geom_of_instance: np.ndarray  # int32 (I,)
    frames: Frames
    lo: np.ndarray
    hi: np.ndarray

    @property
    def extent(self) -> float:
        return float(np.max(self.hi - self.lo))

    @property
    def centre(self) -> np.ndarray:
        return 0.5 * (self.lo + self.hi)


def terrain_instances(num_instances: int = 64, cells: int = 256, amplitude: float = 0.2,
                      seed: int = MASTER_SEED) -> InstancedScene:
    """The two-level ambient-occlusion workload: one terrain mesh under random SRT frames."""
    mesh = terrain(cells, amplitude, seed)
    fr = random_frames(num_instances, seed)
    g = np.zeros(num_instances, dtype=np.int32)
    lo, hi = world_bounds([mesh], g, fr)
    return InstancedScene([mesh], g, fr, lo, hi)


def overview_camera(scene: InstancedScene, width: int, height: int) -> Camera:
    """Camera at scene centre + (0,0,1.5*extent), looking at the centre, 60 deg vertical."""
    eye = scene.centre + np.array([0.0, 0.0, 1.5 * scene.extent])
    return look_down_z_camera(eye, width, height)


def close_camera(scene: InstancedScene, width: int, height: int, distance: float = 0.35) -> Camera:
    """The overview camera moved to scene centre + (0,0,distance*extent): at 0.35 about
    56% of a 1920x1080 image hits the 64-terrain scene (5.8% from 1.5 extent)."""
    eye = scene.centre + np.array([0.0, 0.0, distance * scene.extent])
    return look_down_z_camera(eye, width, height)


@dataclass
class ShadingProblem:
    mesh: Mesh
    camera: Camera
    colours: np.ndarray         # float32 (V,3), uniform in [0,1]
    light: np.ndarray           # float32 (3,), normalize(1,1,1)
    target_colours: np.ndarray  # colours + U[-0.1, 0.1], unclamped
    target_light: np.ndarray    # light rotated by U[0,5] degrees about a random perpendicular axis


def shading_problem(width: int = 1920, height: int = 1080, seed: int = MASTER_SEED, config: int = 4,
                    level: int = 3) -> ShadingProblem:
    """The differentiable-shading workload: the icosphere seen by the (0,0,3) camera with
    per-vertex colours and one directional light, plus the perturbed target parameters."""
    mesh = icosphere(level)
    key = stream_key(seed, config, 0x5AD)
    nv = mesh.vertices.shape[0]
    cols = uniform(stream_key(key, 1), 3 * nv).reshape(nv, 3)
    tcols = cols + (-0.1 + 0.2 * uniform(stream_key(key, 2), 3 * nv).reshape(nv, 3))
    light = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    u = unit_vectors(stream_key(key, 3), 1)[0]
    axis = np.cross(light, u)
    axis /= np.linalg.norm(axis)
    ang = math.radians(5.0 * float(uniform(stream_key(key, 4), 1)[0]))
    tlight = light * math.cos(ang) + np.cross(axis, light) * math.sin(ang)
    cam = look_down_z_camera([0, 0, 3], width, height)
    return ShadingProblem(mesh, cam, cols.astype(np.float32), light.astype(np.float32), tcols.astype(np.float32),
                          tlight.astype(np.float32))


@dataclass
class Soup:
    mesh: Mesh
    num_rays: int
    camera: Camera
    random_rays: np.ndarray
    lo: np.ndarray
    hi: np.ndarray


def soup_scene(index: int, seed: int = MASTER_SEED, config: int = 5, nmin: int = 1000, nmax: int = 2_000_000,
               rmin: int = 4096, rmax: int = 1 << 20) -> Soup:
    """Triangle soup `index` of the many-uneven-scenes workload: N log-uniform in
    [nmin,nmax], centroids from an 8-component Gaussian mixture in the unit cube
    [-0.5,0.5]^3 (means U[-0.4,0.4]^3, sigma log-U[0.02,0.1], Dirichlet(1) weights),
    edge lengths log-U[1e-3,1e-1], vertices at 120 degrees in a random plane.
    Rays: R log-uniform in [rmin,rmax]; half camera rays (returned as a camera with
    W*H = R/2), half random rays (origin in the AABB, direction uniform)."""
    key = stream_key(seed, config, index)
    n = int(round(float(log_uniform(stream_key(key, 1), 1, nmin, nmax)[0])))
    R = int(round(float(log_uniform(stream_key(key, 2), 1, rmin, rmax)[0])))
    means = -0.4 + 0.8 * uniform(stream_key(key, 3), 24).reshape(8, 3)
    sig = log_uniform(stream_key(key, 4), 8, 0.02, 0.1)
    w = -np.log1p(-uniform(stream_key(key, 5), 8))
    w = w / w.sum()
    comp = np.searchsorted(np.cumsum(w), uniform(stream_key(key, 6), n), side="right")
    comp = np.minimum(comp, 7)
    c = means[comp] + sig[comp, None] * normal(stream_key(key, 7), 3 * n).reshape(n, 3)
    e = log_uniform(stream_key(key, 8), n, 1e-3, 1e-1)
    a = unit_vectors(stream_key(key, 9), n)  # plane normal
    helper = np.where(np.abs(a[:, 0:1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    b1 = np.cross(a, helper)
    b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
    b2 = np.cross(a, b1)
    ang0 = 2 * math.pi * uniform(stream_key(key, 10), n)
    verts = np.empty((n, 3, 3))
    for k in range(3):
        ang = ang0 + k * 2 * math.pi / 3
        verts[:, k, :] = c + (e / math.sqrt(3.0))[:, None] * (np.cos(ang)[:, None] * b1 + np.sin(ang)[:, None] * b2)
    v32 = verts.reshape(-1, 3).astype(np.float32)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    lo = v32.min(axis=0).astype(np.float64)
    hi = v32.max(axis=0).astype(np.float64)
    ncam = R // 2
    side = max(1, int(round(math.sqrt(ncam))))
    centroid = c.mean(axis=0)
    cam = look_down_z_camera(centroid + np.array([0, 0, 1.5]), side, side)
    rr = random_rays(R - side * side, lo, hi, seed, config * 1000 + index)
    return Soup(Mesh(v32, idx), R, cam, rr, lo, hi)
