// ORACLE (test infrastructure only; never linked into the library): spatial splits of
// triangles ahead of a build, written out as plain sequential code.
//
// The paper names spatial splits (SBVH, Stich, Friedrich and Dietrich 2009) for its
// high-quality build option (Sec. 8): a triangle may be referenced by several leaves,
// each bounding the part of it inside one region, so that the boxes of long or
// diagonal triangles stop covering empty space. This restates the splitting done
// before a build, after Karras and Aila ("Fast Parallel Construction of High-Quality
// Bounding Volume Hierarchies", HPG 2013, Sec. 4.1): a budget of extra references is
// shared out by a per-triangle priority, and each triangle is cut recursively at the
// most important plane of the scene's Morton grid that crosses its box.
//
// Steps, in this order (every operation is float32, rounded to nearest; compile with
// -ffp-contract=off so no multiply-add is fused):
//  1. B_t = the box of triangle t's vertices; G = the union of all B_t.
//  2. Grid: per axis a, ext_a = G.hi_a - G.lo_a, inv_a = 1024 / ext_a, q(x) = (x - G.lo_a)
//     inv_a. A box [lo, hi] spans the cells cl = floor(q(lo + d)) to ch = max(cl,
//     ceil(q(hi - d)) - 1), clamped to [0, 1023] (all 0 on an axis of zero extent), where
//     d = 2^-18 max(|lo|, |hi|) narrows the box by more than the widening of step 5: a box
//     that ends on a grid line, or a crossing widened past one, does not reach the next
//     cell. The level of a box is the largest bit length over the axes of cl xor ch (0..10).
//  3. Priority: A(B) = (dx dy + dy dz) + dz dx (half the surface area); the triangle's own
//     A_tri = ((|c.x| + |c.y|) + |c.z|) / 2 with c = (v1 - v0) x (v2 - v0) (its three axis
//     projections, which no set of covering boxes can undercut); excess = max(0, A(B_t) -
//     A_tri); r_t = (excess / A(G)) 2^level(B_t) (<= 1024); the priority is the published
//     r_t^(1/3) (X = 2, Y = 1/3), taken exactly as the weight w_t = the integer cube root
//     of r_t 2^53 (the largest w with w^3 <= it; < 2^21), so the total W is an exact integer.
//  4. Splits: with C_t = w_0 + ... + w_{t-1} (C_n = W), triangle t's share of the budget S
//     is s_t = min(maxSplits, floor(S C_{t+1} / W) - floor(S C_t / W)): each gets its fair
//     share S w_t / W rounded down or up, and the shares add up to S (Karras and Aila
//     round every share down and leave the rest unspent). What a cap (or W = 0) leaves
//     over, R = S - sum s_t, goes one each to triangles 0..R-1. Triangle t gets s_t + 1
//     (+1) references, so there are exactly n + S of them, numbered triangle by triangle.
//  5. Splitting a box B with s splits left: none left -> emit B. Otherwise pick the plane:
//     per axis the highest bit b where cl and ch differ names the grid line j = (ch >> b)
//     << b, inside the box, at G.lo + j (ext / 1024); the axis with the largest b wins
//     (ties: the longer extent hi - lo of B, then the lower axis). If no grid line crosses
//     B, cut the longest axis at (lo + hi) / 2. Each side's box is the box of the
//     triangle's vertices on that side (<= / >= the plane), then of the points where its
//     edges cross the plane, intersected with B. A crossing of edge a-e is t = (P - a_k) /
//     (e_k - a_k), q_c = a_c + (e_c - a_c) t on the other axes (P itself on the cut axis),
//     widened to [q_c - pad, q_c + pad] with pad = max(|a_c|, |e_c|) 2^-19 + 2^-140: the
//     rounding errors of q_c stay below 12 units in the last place of that magnitude (and
//     of the widening subtraction below one more), so the interval holds the exact
//     crossing. An empty side takes a copy of the other side's box and no further splits.
//     The s - 1 splits left go to the sides in proportion to their longest extents w:
//     the left side takes floor((s - 1) wL / (wL + wR) + 0.5) ((s - 1) / 2 when both are
//     0); the left side's references come first (depth first).
//  6. The first reference of each triangle is its owner (the one a primitive-to-leaf
//     map points at).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace {

struct FBox {
    float lo[3], hi[3];
};

struct Grid {
    float lo[3], ext[3], inv[3];
    int cell(float x, int a, bool end) const {
        if (inv[a] == 0.0f) return 0;
        const float q = (x - lo[a]) * inv[a];
        const float f = end ? std::ceil(q) - 1.0f : std::floor(q);
        if (!(f >= 0.0f)) return 0;
        if (f > 1023.0f) return 1023;
        return (int)f;
    }
    // first and last cell of the box's extent on axis a (narrowed by d at each end)
    void span(const FBox& b, int a, int* cl, int* ch) const {
        const float d = std::max(std::fabs(b.lo[a]), std::fabs(b.hi[a])) * 0x1p-18f;
        *cl = cell(b.lo[a] + d, a, false);
        *ch = std::max(*cl, cell(b.hi[a] - d, a, true));
    }
};

// Largest w with w^3 <= N (N < 2^64).
uint32_t integer_cube_root(uint64_t N) {
    uint64_t w = (uint64_t)std::cbrt((double)N);
    while (w > 0 && w * w * w > N) --w;
    while ((w + 1) * (w + 1) * (w + 1) <= N) ++w;
    return (uint32_t)w;
}

int bit_length(uint32_t x) {
    int n = 0;
    while (x) ++n, x >>= 1;
    return n;
}

int level(const Grid& g, const FBox& b) {
    int L = 0;
    for (int a = 0; a < 3; ++a) {
        int cl, ch;
        g.span(b, a, &cl, &ch);
        L = std::max(L, bit_length((uint32_t)(cl ^ ch)));
    }
    return L;
}

float half_area(const FBox& b) {
    const float dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
    return (dx * dy + dy * dz) + dz * dx;
}

float longest(const FBox& b) {
    float w = 0.0f;
    for (int a = 0; a < 3; ++a) w = std::max(w, b.hi[a] - b.lo[a]);
    return w;
}

bool empty(const FBox& b) { return b.lo[0] > b.hi[0] || b.lo[1] > b.hi[1] || b.lo[2] > b.hi[2]; }

// The plane that cuts box b: axis and coordinate (step 5).
void choose_plane(const Grid& g, const FBox& b, int* axis, float* plane) {
    int best = -1, bestBit = -1, bestJ = 0;
    float bestExt = -1.0f;
    for (int a = 0; a < 3; ++a) {
        int cl, ch;
        g.span(b, a, &cl, &ch);
        if (cl == ch) continue;
        const int bit = bit_length((uint32_t)(cl ^ ch)) - 1;
        const float e = b.hi[a] - b.lo[a];
        if (bit > bestBit || (bit == bestBit && e > bestExt)) best = a, bestBit = bit, bestExt = e, bestJ = (ch >> bit) << bit;
    }
    if (best >= 0) {
        *axis = best;
        *plane = g.lo[best] + (float)bestJ * (g.ext[best] * 0x1p-10f);
        return;
    }
    int a0 = 0;
    float e0 = b.hi[0] - b.lo[0];
    for (int a = 1; a < 3; ++a) {
        const float e = b.hi[a] - b.lo[a];
        if (e > e0) a0 = a, e0 = e;
    }
    *axis = a0;
    *plane = 0.5f * (b.lo[a0] + b.hi[a0]);
}

// Box of the part of triangle v on one side of the plane x_axis = P, intersected with b.
FBox clip_side(const float v[3][3], int axis, float P, bool left, const FBox& b) {
    FBox r;
    for (int c = 0; c < 3; ++c) r.lo[c] = INFINITY, r.hi[c] = -INFINITY;
    for (int i = 0; i < 3; ++i) {
        const bool in = left ? v[i][axis] <= P : v[i][axis] >= P;
        if (!in) continue;
        for (int c = 0; c < 3; ++c) r.lo[c] = std::min(r.lo[c], v[i][c]), r.hi[c] = std::max(r.hi[c], v[i][c]);
    }
    for (int i = 0; i < 3; ++i) {
        const float* a = v[i];
        const float* e = v[(i + 1) % 3];
        const bool crosses = (a[axis] < P && e[axis] > P) || (a[axis] > P && e[axis] < P);
        if (!crosses) continue;
        const float t = (P - a[axis]) / (e[axis] - a[axis]);
        for (int c = 0; c < 3; ++c) {
            if (c == axis) {
                r.lo[c] = std::min(r.lo[c], P), r.hi[c] = std::max(r.hi[c], P);
                continue;
            }
            const float q = a[c] + (e[c] - a[c]) * t;
            const float pad = std::max(std::fabs(a[c]), std::fabs(e[c])) * 0x1p-19f + 0x1p-140f;
            r.lo[c] = std::min(r.lo[c], q - pad);
            r.hi[c] = std::max(r.hi[c], q + pad);
        }
    }
    for (int c = 0; c < 3; ++c) r.lo[c] = std::max(r.lo[c], b.lo[c]), r.hi[c] = std::min(r.hi[c], b.hi[c]);
    return r;
}

void split_box(const Grid& g, const float v[3][3], const FBox& b, int s, std::vector<FBox>& out) {
    if (s == 0) {
        out.push_back(b);
        return;
    }
    int axis;
    float P;
    choose_plane(g, b, &axis, &P);
    FBox L = clip_side(v, axis, P, true, b), R = clip_side(v, axis, P, false, b);
    const int rest = s - 1;
    int sL;
    if (empty(L) && empty(R)) {
        L = R = b;
        sL = 0;
    } else if (empty(L)) {
        L = R;
        sL = 0;
    } else if (empty(R)) {
        R = L;
        sL = rest;
    } else {
        const float wL = longest(L), wR = longest(R);
        if (wL + wR > 0.0f)
            sL = (int)std::floor((float)rest * wL / (wL + wR) + 0.5f);
        else
            sL = rest / 2;
        sL = std::min(sL, rest);
    }
    split_box(g, v, L, sL, out);
    split_box(g, v, R, rest - sL, out);
}

}  // namespace

extern "C" {

// tris: n x 9 floats (v0, v1, v2). Writes n + budget references (lo, hi: 3 floats each;
// prim: the triangle; owner: 1 on each triangle's first reference) and each triangle's
// split count; returns the reference count (n + budget), or -1 if budget > n.
int64_t oracle_split_triangles(const float* tris, int64_t n, uint32_t budget, int max_splits, float* out_lo,
                               float* out_hi, uint32_t* out_prim, uint8_t* out_owner, uint32_t* out_splits) {
    if ((int64_t)budget > n) return -1;
    if (n == 0) return 0;
    std::vector<FBox> box(n);
    FBox G;
    for (int c = 0; c < 3; ++c) G.lo[c] = INFINITY, G.hi[c] = -INFINITY;
    for (int64_t t = 0; t < n; ++t) {
        const float* v = tris + 9 * t;
        for (int c = 0; c < 3; ++c) {
            box[t].lo[c] = std::min(std::min(v[c], v[3 + c]), v[6 + c]);
            box[t].hi[c] = std::max(std::max(v[c], v[3 + c]), v[6 + c]);
            G.lo[c] = std::min(G.lo[c], box[t].lo[c]);
            G.hi[c] = std::max(G.hi[c], box[t].hi[c]);
        }
    }
    Grid g;
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = G.lo[a];
        g.ext[a] = G.hi[a] - G.lo[a];
        g.inv[a] = g.ext[a] > 0.0f ? 1024.0f / g.ext[a] : 0.0f;
    }
    const float areaG = half_area(G);
    std::vector<uint32_t> w(n);
    uint64_t W = 0;
    for (int64_t t = 0; t < n; ++t) {
        const float* v = tris + 9 * t;
        const float e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        const float e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        const float cx = e1[1] * e2[2] - e1[2] * e2[1];
        const float cy = e1[2] * e2[0] - e1[0] * e2[2];
        const float cz = e1[0] * e2[1] - e1[1] * e2[0];
        const float tri = 0.5f * ((std::fabs(cx) + std::fabs(cy)) + std::fabs(cz));
        float excess = half_area(box[t]) - tri;
        if (!(excess > 0.0f)) excess = 0.0f;
        const float r = areaG > 0.0f ? (excess / areaG) * (float)(1u << level(g, box[t])) : 0.0f;
        w[t] = integer_cube_root((uint64_t)(r * 0x1p53f));
        W += w[t];
    }
    std::vector<uint32_t> s(n, 0);
    uint64_t used = 0, C = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (W) {
            const uint64_t before = (uint64_t)((unsigned __int128)budget * C / W);
            const uint64_t after = (uint64_t)((unsigned __int128)budget * (C + w[t]) / W);
            s[t] = (uint32_t)std::min<uint64_t>((uint64_t)max_splits, after - before);
        }
        C += w[t];
        used += s[t];
    }
    const uint64_t left = (uint64_t)budget - used;
    int64_t m = 0;
    std::vector<FBox> refs;
    for (int64_t t = 0; t < n; ++t) {
        if ((uint64_t)t < left) s[t] += 1;
        out_splits[t] = s[t];
        float v[3][3];
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) v[i][c] = tris[9 * t + 3 * i + c];
        refs.clear();
        split_box(g, v, box[t], (int)s[t], refs);
        for (size_t k = 0; k < refs.size(); ++k, ++m) {
            for (int c = 0; c < 3; ++c) out_lo[3 * m + c] = refs[k].lo[c], out_hi[3 * m + c] = refs[k].hi[c];
            out_prim[m] = (uint32_t)t;
            out_owner[m] = k == 0 ? 1 : 0;
        }
    }
    return m;
}

}  // extern "C"
