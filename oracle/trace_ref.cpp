// ORACLE (test infrastructure only; never linked into the library): closest-hit and
// any-hit queries in FP64.
//
// Definitions followed:
//  * ray R(t) = o + t d with t in [minT, maxT] (paper Eq. 1 and Sec. 7.5's ray
//    fields); both ends inclusive;
//  * triangles are double-sided with inclusive edges (Sec. 3.1 rejects only a
//    negative edge function and tests no orientation). Two formulas are provided:
//    Moller-Trumbore ("Fast, Minimum Storage Ray/Triangle Intersection", 1997) and
//    the paper's plane-then-three-edge-tests form of Sec. 3.1, which a test uses to
//    cross-check the first; barycentrics follow p = (1-u-v) v0 + u v1 + v v2;
//  * a custom sphere primitive is the smallest root of |o + t d - c|^2 = r^2 in
//    [minT, maxT], with u = v = 0;
//  * closest hit: the valid hit with the smallest t; ties go to the smaller
//    instance ID, then the smaller primitive ID (brute force over every primitive,
//    as in Sec. 3.3's linear search). any-hit: whether a valid hit exists;
//  * two levels (Sec. 6.2 "Two-Level Hierarchy and Instancing"): instance frame
//    M = T R S maps object to world space; the ray is taken to object space by
//    M^-1 without renormalising the direction, so t is the same in both spaces.
//    R is the rotation of the unit quaternion (x,y,z,w), normalised here.
//
// The oracle's own acceleration structure is a top-down median-split BVH in FP64
// (the top-down construction of Sec. 6.2) over each geometry, with boxes padded by
// a relative 1e-9 so that rounding in the slab test never culls a primitive that the
// exact test hits; a stack traversal (Sec. 6.2 "BVH Traversal") visits it. A test
// checks it against brute force.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

#include "oracle_math.h"

using namespace oracle;

namespace {
const double PI = 3.14159265358979323846;

const uint32_t NONE = 0xFFFFFFFFu;

struct RayD {
    V3 o, d;
    double tmin, tmax;
};

struct HitD {
    uint32_t inst = NONE, prim = NONE;
    double t = INFINITY, u = 0, v = 0;
};

// Moller-Trumbore in FP64, double-sided, inclusive edges.
bool mt(const RayD& r, V3 v0, V3 v1, V3 v2, double& t, double& u, double& v) {
    const V3 e1 = v1 - v0, e2 = v2 - v0;
    const V3 P = cross(r.d, e2);
    const double det = dot(e1, P);
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const V3 T = r.o - v0;
    u = dot(T, P) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const V3 Q = cross(T, e1);
    v = dot(r.d, Q) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    t = dot(e2, Q) * inv;
    return t >= r.tmin && t <= r.tmax;
}

// Plane + three edge functions (paper Sec. 3.1) in FP64. Returns the plane hit's
// barycentrics even when outside (inside == all three edge values >= 0).
bool plane_edges(const RayD& r, V3 v0, V3 v1, V3 v2, double& t, double& u, double& v, bool& inside) {
    const V3 e0 = v1 - v0, e1 = v2 - v1, e2 = v0 - v2;
    const V3 n = cross(e0, e1);
    const double nd = dot(n, r.d);
    if (nd == 0.0) return false;
    t = dot(v0 - r.o, n) / nd;
    const V3 p = r.o + r.d * t;
    const double a = dot(n, cross(e0, p - v0));  // weight of v2
    const double b = dot(n, cross(e1, p - v1));  // weight of v0
    const double c = dot(n, cross(e2, p - v2));  // weight of v1
    const double s = a + b + c;
    if (s == 0.0) return false;
    u = c / s;
    v = a / s;
    inside = a >= 0.0 && b >= 0.0 && c >= 0.0;
    return true;
}

bool sphere(const RayD& r, V3 c, double rad, double& t) {
    const V3 f = r.o - c;
    const double a = dot(r.d, r.d);
    const double b = dot(f, r.d);
    const double cc = dot(f, f) - rad * rad;
    const double disc = b * b - a * cc;
    if (disc < 0.0 || a == 0.0) return false;
    const double sq = std::sqrt(disc);
    const double t0 = (-b - sq) / a, t1 = (-b + sq) / a;
    if (t0 >= r.tmin && t0 <= r.tmax) {
        t = t0;
        return true;
    }
    if (t1 >= r.tmin && t1 <= r.tmax) {
        t = t1;
        return true;
    }
    return false;
}

// Disc (a custom primitive): centre c, unit normal n, radius rad. The ray meets the
// disc's plane at t = ((c - o) . n) / (d . n) and hits the disc when that point lies
// within rad of c (the rim included) and t is in range; a ray parallel to the plane
// misses.
bool disc(const RayD& r, V3 c, V3 n, double rad, double& t) {
    const double den = dot(r.d, n);
    if (den == 0.0) return false;
    const double th = dot(c - r.o, n) / den;
    if (!(th >= r.tmin && th <= r.tmax)) return false;
    const V3 q = (r.o + r.d * th) - c;
    if (dot(q, q) > rad * rad) return false;
    t = th;
    return true;
}

struct Box {
    V3 lo{INFINITY, INFINITY, INFINITY}, hi{-INFINITY, -INFINITY, -INFINITY};
    void grow(V3 p) {
        lo = {std::min(lo.x, p.x), std::min(lo.y, p.y), std::min(lo.z, p.z)};
        hi = {std::max(hi.x, p.x), std::max(hi.y, p.y), std::max(hi.z, p.z)};
    }
    void grow(const Box& b) {
        grow(b.lo);
        grow(b.hi);
    }
    void pad() {
        const double m = 1e-9 * (std::max({std::fabs(lo.x), std::fabs(lo.y), std::fabs(lo.z), std::fabs(hi.x),
                                           std::fabs(hi.y), std::fabs(hi.z)}) +
                                 1e-30);
        lo = lo - v3(m, m, m);
        hi = hi + v3(m, m, m);
    }
};

// Slab test with explicit handling of zero direction components.
bool box_hit(const Box& b, const RayD& r, double tmax) {
    double t0 = r.tmin, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        const double o = comp(r.o, a), d = comp(r.d, a), lo = comp(b.lo, a), hi = comp(b.hi, a);
        if (d == 0.0) {
            if (o < lo || o > hi) return false;
            continue;
        }
        double ta = (lo - o) / d, tb = (hi - o) / d;
        if (ta > tb) std::swap(ta, tb);
        t0 = std::max(t0, ta);
        t1 = std::min(t1, tb);
        if (t0 > t1 * (1.0 + 1e-12) + 1e-300) return false;
    }
    return true;
}

struct Geom {
    int kind = 0;  // 0 triangles, 1 spheres, 2 discs
    std::vector<V3> a, b, c;  // triangle vertices (object space)
    std::vector<V3> centre, normal;
    std::vector<double> radius;
    size_t count() const { return kind == 0 ? a.size() : centre.size(); }
    Box prim_box(size_t i) const {
        Box bx;
        if (kind == 0) {
            bx.grow(a[i]);
            bx.grow(b[i]);
            bx.grow(c[i]);
        } else if (kind == 1) {
            const double r = radius[i];
            bx.grow(centre[i] - v3(r, r, r));
            bx.grow(centre[i] + v3(r, r, r));
        } else {
            // the disc spans rad * sqrt(1 - n_a^2) along axis a
            const double r = radius[i];
            const V3 n = normal[i];
            const V3 e = v3(r * std::sqrt(std::max(0.0, 1.0 - n.x * n.x)), r * std::sqrt(std::max(0.0, 1.0 - n.y * n.y)),
                            r * std::sqrt(std::max(0.0, 1.0 - n.z * n.z)));
            bx.grow(centre[i] - e);
            bx.grow(centre[i] + e);
        }
        return bx;
    }
    // Intersection filter (Sec. 7.6) as a primitive mask: bit i of keep (word i / 32)
    // says whether hits on primitive i stand; empty = every hit stands.
    std::vector<uint32_t> keep;
    bool accepts(size_t i) const { return keep.empty() || ((keep[i >> 5] >> (i & 31)) & 1u); }
    bool intersect(const RayD& r, size_t i, double& t, double& u, double& v) const {
        if (!accepts(i)) return false;
        if (kind == 0) return mt(r, a[i], b[i], c[i], t, u, v);
        u = v = 0.0;
        if (kind == 2) return disc(r, centre[i], normal[i], radius[i], t);
        return sphere(r, centre[i], radius[i], t);
    }
    // FP64 median-split BVH: nodes hold a box and either two children or a prim range.
    struct Node {
        Box box;
        int32_t left = -1, right = -1;
        uint32_t first = 0, count = 0;
    };
    std::vector<Node> nodes;
    std::vector<uint32_t> prims;
    void build() {
        const size_t n = count();
        prims.resize(n);
        for (size_t i = 0; i < n; ++i) prims[i] = (uint32_t)i;
        nodes.clear();
        if (n == 0) return;
        std::vector<Box> pb(n);
        std::vector<V3> cen(n);
        for (size_t i = 0; i < n; ++i) {
            pb[i] = prim_box(i);
            pb[i].pad();
            cen[i] = (pb[i].lo + pb[i].hi) * 0.5;
        }
        struct Item {
            int32_t node;
            uint32_t first, count;
        };
        nodes.push_back(Node{});
        std::vector<Item> st{{0, 0, (uint32_t)n}};
        while (!st.empty()) {
            Item it = st.back();
            st.pop_back();
            Box bx, cb;
            for (uint32_t k = it.first; k < it.first + it.count; ++k) {
                bx.grow(pb[prims[k]]);
                cb.grow(cen[prims[k]]);
            }
            nodes[it.node].box = bx;
            if (it.count <= 4) {
                nodes[it.node].first = it.first;
                nodes[it.node].count = it.count;
                continue;
            }
            const V3 ext = cb.hi - cb.lo;
            const int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
            const uint32_t half = it.count / 2;
            std::nth_element(prims.begin() + it.first, prims.begin() + it.first + half,
                             prims.begin() + it.first + it.count,
                             [&](uint32_t p, uint32_t q) { return comp(cen[p], axis) < comp(cen[q], axis); });
            const int32_t l = (int32_t)nodes.size();
            nodes.push_back(Node{});
            nodes.push_back(Node{});
            nodes[it.node].left = l;
            nodes[it.node].right = l + 1;
            st.push_back({l, it.first, half});
            st.push_back({l + 1, it.first + half, it.count - half});
        }
    }
};

struct Instance {
    int geom = 0;
    Affine fwd, inv;
    Box world;
    uint32_t mask = 0xFFFFFFFFu;  // visibility mask (Sec. 7.5): tested against the ray mask with AND
};

struct Scene {
    std::vector<Geom> geoms;
    std::vector<Instance> inst;
    bool built = false;
};

Affine srt(const float* q4, const float* s3, const float* t3, Affine* inverse) {
    double x = q4[0], y = q4[1], z = q4[2], w = q4[3];
    const double nq = std::sqrt(x * x + y * y + z * z + w * w);
    x /= nq, y /= nq, z /= nq, w /= nq;
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)},
                            {2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)},
                            {2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)}};
    const double S[3] = {s3[0], s3[1], s3[2]};
    const double T[3] = {t3[0], t3[1], t3[2]};
    Affine f{};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) f.m[i][j] = R[i][j] * S[j];
        f.m[i][3] = T[i];
    }
    // inverse: S^-1 R^T (x - T)
    Affine g{};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) g.m[i][j] = R[j][i] / S[i];
        g.m[i][3] = -(g.m[i][0] * T[0] + g.m[i][1] * T[1] + g.m[i][2] * T[2]);
    }
    *inverse = g;
    return f;
}

RayD load_ray(const float* r) {
    return RayD{v3(r[0], r[1], r[2]), v3(r[4], r[5], r[6]), (double)r[3], (double)r[7]};
}

// Closest (any=false) or any hit over one geometry for an object-space ray.
void trace_geom(const Geom& g, const RayD& r, bool any, bool use_bvh, uint32_t inst, HitD& best) {
    auto consider = [&](uint32_t p) -> bool {
        double t, u, v;
        if (!g.intersect(r, p, t, u, v)) return false;
        if (t < best.t || (t == best.t && (inst < best.inst || (inst == best.inst && p < best.prim)))) {
            best.t = t;
            best.u = u;
            best.v = v;
            best.inst = inst;
            best.prim = p;
        }
        return true;
    };
    if (!use_bvh) {
        for (size_t p = 0; p < g.count(); ++p)
            if (consider((uint32_t)p) && any) return;
        return;
    }
    if (g.nodes.empty()) return;
    std::vector<int32_t> st{0};
    while (!st.empty()) {
        const int32_t k = st.back();
        st.pop_back();
        const auto& nd = g.nodes[(size_t)k];
        const double tlim = any ? r.tmax : std::min(r.tmax, best.t);
        if (!box_hit(nd.box, r, tlim)) continue;
        if (nd.left < 0) {
            for (uint32_t i = nd.first; i < nd.first + nd.count; ++i)
                if (consider(g.prims[i]) && any) return;
        } else {
            st.push_back(nd.left);
            st.push_back(nd.right);
        }
    }
}

void trace_one(const Scene& S, const RayD& wr, bool any, bool use_bvh, uint32_t ray_mask, HitD& best) {
    for (size_t i = 0; i < S.inst.size(); ++i) {
        const Instance& I = S.inst[i];
        if ((I.mask & ray_mask) == 0) continue;  // the instance is invisible to this ray
        if (use_bvh && !box_hit(I.world, wr, any ? wr.tmax : std::min(wr.tmax, best.t))) continue;
        RayD r{I.inv.point(wr.o), I.inv.vector(wr.d), wr.tmin, wr.tmax};
        trace_geom(S.geoms[(size_t)I.geom], r, any, use_bvh, (uint32_t)i, best);
        if (any && best.prim != NONE) return;
    }
}

// Every valid intersection of one world ray: (instance, primitive, t, u, v) for each
// primitive of each visible instance whose exact intersection lies in [tmin, tmax].
struct HitRec {
    double t, u, v;
    uint32_t inst, prim;
};
void all_hits_one(const Scene& S, const RayD& wr, bool use_bvh, uint32_t ray_mask, std::vector<HitRec>& out) {
    for (size_t i = 0; i < S.inst.size(); ++i) {
        const Instance& I = S.inst[i];
        if ((I.mask & ray_mask) == 0) continue;
        if (use_bvh && !box_hit(I.world, wr, wr.tmax)) continue;
        const RayD r{I.inv.point(wr.o), I.inv.vector(wr.d), wr.tmin, wr.tmax};
        const Geom& g = S.geoms[(size_t)I.geom];
        auto consider = [&](uint32_t p) {
            double t, u, v;
            if (g.intersect(r, p, t, u, v)) out.push_back(HitRec{t, u, v, (uint32_t)i, p});
        };
        if (!use_bvh) {
            for (size_t p = 0; p < g.count(); ++p) consider((uint32_t)p);
            continue;
        }
        if (g.nodes.empty()) continue;
        std::vector<int32_t> st{0};
        while (!st.empty()) {
            const auto& nd = g.nodes[(size_t)st.back()];
            st.pop_back();
            if (!box_hit(nd.box, r, r.tmax)) continue;
            if (nd.left < 0) {
                for (uint32_t k = nd.first; k < nd.first + nd.count; ++k) consider(g.prims[k]);
            } else {
                st.push_back(nd.left);
                st.push_back(nd.right);
            }
        }
    }
    std::sort(out.begin(), out.end(), [](const HitRec& a, const HitRec& b) {
        if (a.t != b.t) return a.t < b.t;
        if (a.inst != b.inst) return a.inst < b.inst;
        return a.prim < b.prim;
    });
}

template <class F>
void parallel_for(int64_t n, int threads, F f) {
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    if (n < 256 || threads == 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < threads; ++w)
        pool.emplace_back([&]() {
            for (;;) {
                const int64_t s = next.fetch_add(256);
                if (s >= n) break;
                const int64_t e = std::min(n, s + 256);
                for (int64_t i = s; i < e; ++i) f(i);
            }
        });
    for (auto& t : pool) t.join();
}

}  // namespace

extern "C" {

void* oracle_scene_new() { return new Scene(); }
void oracle_scene_free(void* s) { delete (Scene*)s; }

// Adds an indexed triangle mesh; returns its geometry index.
int oracle_scene_add_mesh(void* s, const float* verts, int64_t nv, const uint32_t* idx, int64_t nt) {
    Scene* S = (Scene*)s;
    Geom g;
    g.kind = 0;
    g.a.resize((size_t)nt), g.b.resize((size_t)nt), g.c.resize((size_t)nt);
    for (int64_t i = 0; i < nt; ++i) {
        const uint32_t* t = idx + 3 * i;
        auto V = [&](uint32_t k) { return v3(verts[3 * k], verts[3 * k + 1], verts[3 * k + 2]); };
        g.a[(size_t)i] = V(t[0]);
        g.b[(size_t)i] = V(t[1]);
        g.c[(size_t)i] = V(t[2]);
    }
    (void)nv;
    S->geoms.push_back(std::move(g));
    S->built = false;
    return (int)S->geoms.size() - 1;
}

// Adds discs given as 8 floats each: centre xyz, radius, normal xyz (normalised here in
// FP64), unused.
int oracle_scene_add_discs(void* s, const float* d, int64_t n) {
    Scene* S = (Scene*)s;
    Geom g;
    g.kind = 2;
    g.centre.resize((size_t)n);
    g.normal.resize((size_t)n);
    g.radius.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const float* e = d + 8 * i;
        g.centre[(size_t)i] = v3(e[0], e[1], e[2]);
        g.radius[(size_t)i] = e[3];
        const V3 nn = v3(e[4], e[5], e[6]);
        g.normal[(size_t)i] = nn * (1.0 / std::sqrt(dot(nn, nn)));
    }
    S->geoms.push_back(std::move(g));
    S->built = false;
    return (int)S->geoms.size() - 1;
}

// Adds spheres given as float4 (centre xyz, radius).
int oracle_scene_add_spheres(void* s, const float* sph, int64_t n) {
    Scene* S = (Scene*)s;
    Geom g;
    g.kind = 1;
    g.centre.resize((size_t)n);
    g.radius.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        g.centre[(size_t)i] = v3(sph[4 * i], sph[4 * i + 1], sph[4 * i + 2]);
        g.radius[(size_t)i] = sph[4 * i + 3];
    }
    S->geoms.push_back(std::move(g));
    S->built = false;
    return (int)S->geoms.size() - 1;
}

// Adds an instance of geometry `geom`. frame: rotation quaternion xyzw, scale xyz,
// translation xyz (10 floats), or NULL for the identity. Instance IDs count from 0 in
// insertion order.
void oracle_scene_add_instance(void* s, int geom, const float* frame) {
    Scene* S = (Scene*)s;
    Instance I;
    I.geom = geom;
    const float ident[10] = {0, 0, 0, 1, 1, 1, 1, 0, 0, 0};
    const float* f = frame ? frame : ident;
    I.fwd = srt(f, f + 4, f + 7, &I.inv);
    S->inst.push_back(I);
    S->built = false;
}

// Gives geometry `geom` a primitive-mask filter: hits on primitive i stand only when bit
// i of `bits` (word i / 32, bit i % 32) is set.
void oracle_scene_set_prim_filter(void* s, int geom, const uint32_t* bits) {
    Scene* S = (Scene*)s;
    Geom& g = S->geoms[(size_t)geom];
    g.keep.assign(bits, bits + (g.count() + 31) / 32);
}

// Sets instance `inst`'s 32-bit visibility mask (default: all bits set).
void oracle_scene_set_instance_mask(void* s, uint32_t inst, uint32_t mask) {
    Scene* S = (Scene*)s;
    if (inst < S->inst.size()) S->inst[inst].mask = mask;
}

void oracle_scene_build(void* s) {
    Scene* S = (Scene*)s;
    for (auto& g : S->geoms) g.build();
    for (auto& I : S->inst) {
        const Geom& g = S->geoms[(size_t)I.geom];
        Box w;
        for (size_t p = 0; p < g.count(); ++p) {
            Box b = g.prim_box(p);
            for (int c = 0; c < 8; ++c)
                w.grow(I.fwd.point(v3((c & 1) ? b.hi.x : b.lo.x, (c & 2) ? b.hi.y : b.lo.y, (c & 4) ? b.hi.z : b.lo.z)));
        }
        w.pad();
        I.world = w;
    }
    S->built = true;
}

// rays: n x 8 float32 {o.xyz, minT, d.xyz, maxT}. Only instances whose mask ANDed
// with ray_mask is nonzero take part. Outputs per ray: instance ID, prim ID (NONE on a
// miss), t (+inf on a miss), u, v.
void oracle_trace(void* s, const float* rays, int64_t n, int any, int use_bvh, int threads, uint32_t ray_mask,
                  uint32_t* inst_out, uint32_t* prim_out, double* t_out, double* u_out, double* v_out) {
    Scene* S = (Scene*)s;
    if (use_bvh && !S->built) oracle_scene_build(s);
    parallel_for(n, threads, [&](int64_t i) {
        HitD h;
        trace_one(*S, load_ray(rays + 8 * i), any != 0, use_bvh != 0, ray_mask, h);
        inst_out[i] = h.inst;
        prim_out[i] = h.prim;
        t_out[i] = h.t;
        u_out[i] = h.u;
        v_out[i] = h.v;
    });
}

// All hits of each ray (Sec. 7.5), sorted by (t, instance, primitive): the first
// max_hits of ray i go to rows [i * max_hits, ...) of the outputs (misses after them),
// count_out[i] gets how many there are.
void oracle_all_hits(void* s, const float* rays, int64_t n, int use_bvh, int threads, uint32_t ray_mask,
                     int64_t max_hits, uint32_t* inst_out, uint32_t* prim_out, double* t_out, double* u_out,
                     double* v_out, int64_t* count_out) {
    Scene* S = (Scene*)s;
    if (use_bvh && !S->built) oracle_scene_build(s);
    parallel_for(n, threads, [&](int64_t i) {
        std::vector<HitRec> h;
        all_hits_one(*S, load_ray(rays + 8 * i), use_bvh != 0, ray_mask, h);
        count_out[i] = (int64_t)h.size();
        for (int64_t j = 0; j < max_hits; ++j) {
            const int64_t o = i * max_hits + j;
            const bool ok = j < (int64_t)h.size();
            inst_out[o] = ok ? h[(size_t)j].inst : NONE;
            prim_out[o] = ok ? h[(size_t)j].prim : NONE;
            t_out[o] = ok ? h[(size_t)j].t : INFINITY;
            u_out[o] = ok ? h[(size_t)j].u : 0.0;
            v_out[o] = ok ? h[(size_t)j].v : 0.0;
        }
    });
}

double oracle_xi(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim);
void oracle_sample_hemisphere(double xi0, double xi1, double* out3);

// Path tracing with next event estimation (Sec. 5), in FP64, one path per (ray,
// sample) starting from the given float32 ray. Per path vertex (depth 0 .. max_depth-1):
//  * closest hit; a miss adds T * sky and ends the path;
//  * a hit on an emitting triangle (emission != 0) adds T * emission only at depth 0
//    (later vertices count emitters through next event estimation) and ends the path;
//  * otherwise, with n the face normal turned toward the ray, tangent normalize(v1-v0),
//    p' = p + 1e-4 n: one light triangle l = floor(xi_a * L) (in integers on the 24-bit
//    xi), a uniform point q on it (s = sqrt(xi_b): (1-s) a + s(1-xi_c) b + s xi_c c); if
//    cos_s = n.w > 0 and cos_l = |n_l.w| > 0 with w = (q - p') / dist, and an any-hit
//    ray from p' along w over [0, dist (1 - 1e-4)] finds nothing, add
//    T * (albedo / pi) * cos_s cos_l / dist^2 * emission_l * L * area_l;
//  * the next ray leaves p' along a cosine-weighted direction (xi_d, xi_e) around n
//    (tangent frame as for ambient occlusion), and T *= albedo.
// Random numbers: xi(seed, ray, j, dim) with j = (sample * max_depth + depth) * 3 + k:
// (k, dim) = (0,0) a, (0,1) b, (1,0) c, (1,1) d, (2,0) e. Materials: entry
// mat_offset[instance] + primitive of albedo / emission (3 floats each). lights: (instance,
// primitive) pairs. out: the mean over samples, 3 doubles per ray.
void oracle_path_trace(void* s, const float* rays, int64_t n, const float* albedo, const float* emission,
                       const uint32_t* mat_offset, const uint32_t* lights, int64_t light_count, int max_depth,
                       int spp, uint64_t seed, const float* sky, int threads, double* out) {
    Scene* S = (Scene*)s;
    if (!S->built) oracle_scene_build(s);
    auto world_tri = [&](uint32_t inst, uint32_t prim, V3& a, V3& b, V3& c) {
        const Instance& I = S->inst[inst];
        const Geom& g = S->geoms[(size_t)I.geom];
        a = I.fwd.point(g.a[prim]);
        b = I.fwd.point(g.b[prim]);
        c = I.fwd.point(g.c[prim]);
    };
    auto col = [](const float* f, size_t m) { return v3(f[3 * m], f[3 * m + 1], f[3 * m + 2]); };
    const V3 skyL = v3(sky[0], sky[1], sky[2]);
    parallel_for(n, threads, [&](int64_t p) {
        V3 acc = v3(0, 0, 0);
        for (int smp = 0; smp < spp; ++smp) {
            RayD ray = load_ray(rays + 8 * p);
            V3 T = v3(1, 1, 1), L = v3(0, 0, 0);
            for (int depth = 0; depth < max_depth; ++depth) {
                HitD h;
                trace_one(*S, ray, false, true, 0xFFFFFFFFu, h);
                if (h.prim == NONE) {
                    L = L + v3(T.x * skyL.x, T.y * skyL.y, T.z * skyL.z);
                    break;
                }
                const size_t m = (size_t)mat_offset[h.inst] + h.prim;
                const V3 Le = col(emission, m);
                if (Le.x != 0.0 || Le.y != 0.0 || Le.z != 0.0) {
                    if (depth == 0) L = L + v3(T.x * Le.x, T.y * Le.y, T.z * Le.z);
                    break;
                }
                V3 v0, v1, v2;
                world_tri(h.inst, h.prim, v0, v1, v2);
                V3 nrm = normalize(cross(v1 - v0, v2 - v0));
                if (dot(nrm, ray.d) > 0.0) nrm = -nrm;
                const V3 tg = normalize(v1 - v0);
                const V3 bt = cross(nrm, tg);
                const V3 org = (ray.o + ray.d * h.t) + nrm * 1e-4;
                const uint32_t j = (uint32_t)((smp * max_depth + depth) * 3);
                const V3 rho = col(albedo, m);
                if (light_count > 0) {
                    const uint64_t ka = (uint64_t)(oracle_xi(seed, (uint64_t)p, j, 0) * 16777216.0);
                    const int64_t li = (int64_t)((ka * (uint64_t)light_count) >> 24);
                    const uint32_t linst = lights[2 * li], lprim = lights[2 * li + 1];
                    V3 a, b, c;
                    world_tri(linst, lprim, a, b, c);
                    const V3 cr = cross(b - a, c - a);
                    const double area = 0.5 * length(cr);
                    const V3 nl = normalize(cr);
                    const double su = std::sqrt(oracle_xi(seed, (uint64_t)p, j, 1));
                    const double xc = oracle_xi(seed, (uint64_t)p, j + 1, 0);
                    const V3 q = a * (1.0 - su) + b * (su * (1.0 - xc)) + c * (su * xc);
                    V3 w = q - org;
                    const double dist = length(w);
                    w = w * (1.0 / dist);
                    const double cs = dot(nrm, w), cl = std::fabs(dot(nl, w));
                    if (cs > 0.0 && cl > 0.0) {
                        HitD sh;
                        trace_one(*S, RayD{org, w, 0.0, dist * (1.0 - 1e-4)}, true, true, 0xFFFFFFFFu, sh);
                        if (sh.prim == NONE) {
                            const V3 El = col(emission, (size_t)mat_offset[linst] + lprim);
                            const double k = cs * cl / (dist * dist) * (double)light_count * area / PI;
                            L = L + v3(T.x * rho.x * El.x * k, T.y * rho.y * El.y * k, T.z * rho.z * El.z * k);
                        }
                    }
                }
                double hs[3];
                oracle_sample_hemisphere(oracle_xi(seed, (uint64_t)p, j + 1, 1), oracle_xi(seed, (uint64_t)p, j + 2, 0),
                                         hs);
                const V3 dir = tg * hs[0] + bt * hs[2] + nrm * hs[1];
                T = v3(T.x * rho.x, T.y * rho.y, T.z * rho.z);
                ray = RayD{org, dir, 0.0, INFINITY};
            }
            acc = acc + L;
        }
        out[3 * p] = acc.x / spp;
        out[3 * p + 1] = acc.y / spp;
        out[3 * p + 2] = acc.z / spp;
    });
}

// Intersects ray i with one (instance, prim) in FP64. Returns 1 on a valid hit.
int oracle_intersect_prim(void* s, const float* ray, uint32_t inst, uint32_t prim, double* t, double* u, double* v) {
    Scene* S = (Scene*)s;
    if (inst >= S->inst.size()) return 0;
    const Instance& I = S->inst[inst];
    const Geom& g = S->geoms[(size_t)I.geom];
    if (prim >= g.count()) return 0;
    const RayD w = load_ray(ray);
    RayD r{I.inv.point(w.o), I.inv.vector(w.d), w.tmin, w.tmax};
    return g.intersect(r, prim, *t, *u, *v) ? 1 : 0;
}

// Smallest |min(u, v, 1-u-v)| over every triangle whose plane is crossed at a t in
// [minT, maxT] (inside or outside the triangle); +inf if none. A value near 0 marks a
// ray that grazes an edge or vertex.
double oracle_min_edge_margin(void* s, const float* ray) {
    Scene* S = (Scene*)s;
    const RayD w = load_ray(ray);
    double best = INFINITY;
    for (const Instance& I : S->inst) {
        const Geom& g = S->geoms[(size_t)I.geom];
        if (g.kind != 0) continue;
        RayD r{I.inv.point(w.o), I.inv.vector(w.d), w.tmin, w.tmax};
        for (size_t p = 0; p < g.count(); ++p) {
            double t, u, v;
            bool inside;
            if (!plane_edges(r, g.a[p], g.b[p], g.c[p], t, u, v, inside)) continue;
            if (!(t >= r.tmin && t <= r.tmax)) continue;
            best = std::min(best, std::fabs(std::min({u, v, 1.0 - u - v})));
        }
    }
    return best;
}

// Smallest relative gap |r^2 - p^2| / (|f|^2 + r^2) over every sphere, where p is the
// distance from the sphere's centre to the ray's line and f the offset from the ray
// origin to the centre (object space), for spheres whose closest approach lies at a t
// in [minT, maxT]; +inf if none. A value near 0 marks a ray grazing a silhouette.
double oracle_min_sphere_margin(void* s, const float* ray) {
    Scene* S = (Scene*)s;
    const RayD w = load_ray(ray);
    double best = INFINITY;
    for (const Instance& I : S->inst) {
        const Geom& g = S->geoms[(size_t)I.geom];
        if (g.kind != 1) continue;
        RayD r{I.inv.point(w.o), I.inv.vector(w.d), w.tmin, w.tmax};
        const double a = dot(r.d, r.d);
        for (size_t p = 0; p < g.count(); ++p) {
            const V3 f = g.centre[p] - r.o;
            const double along = dot(f, r.d) / a;
            if (!(along >= r.tmin && along <= r.tmax)) continue;
            const V3 l = f - r.d * along;
            const double r2 = g.radius[p] * g.radius[p];
            best = std::min(best, std::fabs(r2 - dot(l, l)) / (dot(f, f) + r2));
        }
    }
    return best;
}

// Smallest relative rim gap | |p - c|^2 / rad^2 - 1 | over every disc whose plane the ray
// meets at a t in [minT, maxT] (p that plane point), +inf if none; near 0 marks a ray
// grazing a disc's rim. A ray within 1e-9 of parallel to a disc's plane counts as 0.
double oracle_min_disc_margin(void* s, const float* ray) {
    Scene* S = (Scene*)s;
    const RayD w = load_ray(ray);
    double best = INFINITY;
    for (const Instance& I : S->inst) {
        const Geom& g = S->geoms[(size_t)I.geom];
        if (g.kind != 2) continue;
        RayD r{I.inv.point(w.o), I.inv.vector(w.d), w.tmin, w.tmax};
        const double dl = std::sqrt(dot(r.d, r.d));
        for (size_t p = 0; p < g.count(); ++p) {
            const double den = dot(r.d, g.normal[p]);
            if (std::fabs(den) <= 1e-9 * dl) {
                best = 0.0;
                continue;
            }
            const double th = dot(g.centre[p] - r.o, g.normal[p]) / den;
            if (!(th >= r.tmin && th <= r.tmax)) continue;
            const V3 q = (r.o + r.d * th) - g.centre[p];
            best = std::min(best, std::fabs(dot(q, q) / (g.radius[p] * g.radius[p]) - 1.0));
        }
    }
    return best;
}

// The paper's plane + edge-test formula on one triangle (cross-check of MT).
int oracle_plane_edge_test(const float* ray, const float* tri, double* t, double* u, double* v) {
    RayD r = load_ray(ray);
    bool inside = false;
    const V3 v0 = v3(tri[0], tri[1], tri[2]), v1 = v3(tri[3], tri[4], tri[5]), v2 = v3(tri[6], tri[7], tri[8]);
    if (!plane_edges(r, v0, v1, v2, *t, *u, *v, inside)) return 0;
    return (inside && *t >= r.tmin && *t <= r.tmax) ? 1 : 0;
}

// Moller-Trumbore on one triangle (float32 inputs, FP64 arithmetic).
int oracle_mt_test(const float* ray, const float* tri, double* t, double* u, double* v) {
    RayD r = load_ray(ray);
    const V3 v0 = v3(tri[0], tri[1], tri[2]), v1 = v3(tri[3], tri[4], tri[5]), v2 = v3(tri[6], tri[7], tri[8]);
    return mt(r, v0, v1, v2, *t, *u, *v) ? 1 : 0;
}

// Forward and inverse 3x4 frames of an instance (row-major, FP64).
void oracle_instance_frames(void* s, uint32_t inst, double* fwd12, double* inv12) {
    Scene* S = (Scene*)s;
    const Instance& I = S->inst[inst];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) {
            fwd12[4 * i + j] = I.fwd.m[i][j];
            inv12[4 * i + j] = I.inv.m[i][j];
        }
}

// World-space vertices of triangle `prim` of instance `inst` (9 doubles, FP64).
int oracle_world_triangle(void* s, uint32_t inst, uint32_t prim, double* out9) {
    Scene* S = (Scene*)s;
    if (inst >= S->inst.size()) return 0;
    const Instance& I = S->inst[inst];
    const Geom& g = S->geoms[(size_t)I.geom];
    if (g.kind != 0 || prim >= g.count()) return 0;
    const V3 w[3] = {I.fwd.point(g.a[prim]), I.fwd.point(g.b[prim]), I.fwd.point(g.c[prim])};
    for (int k = 0; k < 3; ++k) out9[3 * k] = w[k].x, out9[3 * k + 1] = w[k].y, out9[3 * k + 2] = w[k].z;
    return 1;
}

}  // extern "C"
