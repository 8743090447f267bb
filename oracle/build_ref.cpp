// ORACLE (test infrastructure only; never linked into the library): the LBVH build
// steps written out as plain sequential code.
//
//  * primitive AABB and centroid: componentwise min/max of the triangle's vertices
//    (or the given box), centroid = 0.5*(lo+hi) in float32;
//  * Morton codes (30-bit: 10 bits per axis; 63-bit: 21 bits per axis), quantised in
//    float32 with a fixed operation order so that the result is exact and shared by
//    any IEEE-754 implementation that follows the same steps;
//  * the sort: std::stable_sort of primitive indices by code (equal codes keep the
//    input order, the result of a stable LSD radix sort);
//  * the hierarchy: a recursive top-down split of the sorted range at the highest
//    bit where the (code, index) concatenation changes (Karras, "Maximizing
//    Parallelism in the Construction of BVHs, Octrees, and k-d Trees", HPG 2012,
//    Sec. 3-4, which proves its parallel per-node emission yields this same tree),
//    with Karras's numbering: root 0, an internal left child is numbered by the
//    last leaf of its range, an internal right child by the first;
//  * the fit: each internal box is the union of its children's boxes (the bottom-up
//    refit from child volumes of the paper's Sec. 6.2 "BVH Construction");
//  * the clustering build (bottom-up, Sec. 6.2; PLOC of Meister and Bittner, "Parallel
//    Locally-Ordered Clustering for Bounding Volume Hierarchy Construction", TVCG 2018),
//    one iteration at a time over a plain array of clusters.
//
// Compile with -ffp-contract=off so no multiply-add is fused.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "oracle_math.h"

namespace {

// Leading equal bits of two words of `bits` width, counted from the top bit.
int leading_equal_bits(uint64_t a, uint64_t b, int bits) {
    int n = 0;
    for (int k = bits - 1; k >= 0; --k) {
        if (((a >> k) & 1ull) != ((b >> k) & 1ull)) break;
        ++n;
    }
    return n;
}

// Common-prefix length of the concatenations key||index for sorted positions i, j.
int prefix(const uint64_t* keys, int keybits, int64_t i, int64_t j) {
    if (keys[i] != keys[j]) return leading_equal_bits(keys[i], keys[j], keybits);
    return keybits + leading_equal_bits((uint64_t)(uint32_t)i, (uint64_t)(uint32_t)j, 32);
}

const int32_t LEAF = (int32_t)0x80000000u;

uint32_t quantise(float c, float lo, float hi, int bits) {
    // x = (c - lo) / (hi - lo) in float32; x = 0 when the extent is zero
    volatile float ext = hi - lo;
    float x;
    if (ext == 0.0f) {
        x = 0.0f;
    } else {
        volatile float num = c - lo;
        volatile float q = num / ext;
        x = q;
    }
    volatile float s = x * (float)(1u << bits);  // power-of-two scaling
    double f = std::floor((double)s);
    const double top = (double)((1u << bits) - 1u);
    if (!(f >= 0.0)) f = 0.0;  // also maps NaN to 0
    if (f > top) f = top;
    return (uint32_t)f;
}

// Half the surface area of the union of boxes a and b, float32, in the order
// (dx*dy + dy*dz) + dz*dx, plus +0 so a zero area is +0.
float union_area(const float* alo, const float* ahi, const float* blo, const float* bhi) {
    float d[3];
    for (int k = 0; k < 3; ++k) d[k] = std::fmax(ahi[k], bhi[k]) - std::fmin(alo[k], blo[k]);
    float a = d[0] * d[1] + d[1] * d[2];
    a = a + d[2] * d[0];
    return a + 0.0f;
}

// MurmurHash3's 32-bit finaliser (fmix32, Appleby).
uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

}  // namespace

extern "C" {

// Prim AABB + centroid for an indexed triangle mesh (float32, exact min/max).
// idx: 3*n uint32, verts: 3*nv float32. lo/hi/centroid: 3*n float32 out.
void oracle_triangle_aabbs(const uint32_t* idx, int64_t n, const float* verts, float* lo, float* hi,
                           float* centroid) {
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            float mn = verts[3 * (int64_t)idx[3 * i + 0] + a];
            float mx = mn;
            for (int k = 1; k < 3; ++k) {
                float v = verts[3 * (int64_t)idx[3 * i + k] + a];
                mn = std::min(mn, v);
                mx = std::max(mx, v);
            }
            lo[3 * i + a] = mn;
            hi[3 * i + a] = mx;
            volatile float s = mn + mx;
            centroid[3 * i + a] = 0.5f * s;
        }
    }
}

// Centroids of given boxes (lo.xyz, hi.xyz per prim).
void oracle_box_centroids(const float* boxes, int64_t n, float* centroid) {
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            volatile float s = boxes[6 * i + a] + boxes[6 * i + 3 + a];
            centroid[3 * i + a] = 0.5f * s;
        }
}

// Morton codes of centroids within [lo, hi] (the centroid bounds). bits = 10 or 21 per
// axis. Code bit 3k+2 holds bit k of x, 3k+1 of y, 3k of z.
void oracle_morton(const float* centroid, int64_t n, const float* lo, const float* hi, int bits,
                   uint64_t* codes) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) q[a] = quantise(centroid[3 * i + a], lo[a], hi[a], bits);
        uint64_t code = 0;
        for (int k = bits - 1; k >= 0; --k) {
            code = (code << 1) | ((q[0] >> k) & 1u);
            code = (code << 1) | ((q[1] >> k) & 1u);
            code = (code << 1) | ((q[2] >> k) & 1u);
        }
        codes[i] = code;
    }
}

// Centroid bounds (min/max of centroids).
void oracle_centroid_bounds(const float* centroid, int64_t n, float* lo, float* hi) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], centroid[3 * i + a]);
            hi[a] = std::max(hi[a], centroid[3 * i + a]);
        }
}

// Stable sort of (code, index) by code. order[k] = primitive at sorted position k.
void oracle_stable_sort(const uint64_t* codes, int64_t n, uint64_t* sorted_codes, uint32_t* order) {
    std::vector<uint32_t> idx((size_t)n);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return codes[a] < codes[b]; });
    for (int64_t k = 0; k < n; ++k) {
        order[k] = idx[(size_t)k];
        sorted_codes[k] = codes[idx[(size_t)k]];
    }
}

// Hierarchy over n >= 2 sorted keys of `keybits` width (32 for 30-bit codes held in
// 32-bit words, 64 for 63-bit codes). childL/childR: n-1 entries, leaf children
// carry the top bit. parent_internal: n-1 (root gets -1); parent_leaf: n.
void oracle_topology(const uint64_t* sorted_keys, int64_t n, int keybits, int32_t* childL, int32_t* childR,
                     int32_t* parent_internal, int32_t* parent_leaf) {
    if (n < 2) return;
    parent_internal[0] = -1;
    // explicit work list instead of deep recursion for long chains
    struct Item {
        int64_t a, b;
        int32_t id;
    };
    std::vector<Item> stack;
    stack.push_back({0, n - 1, 0});
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        const int64_t a = it.a, b = it.b;
        const int32_t id = it.id;
        const int p = prefix(sorted_keys, keybits, a, b);
        int64_t gamma = a;
        for (int64_t m = a; m < b; ++m)
            if (prefix(sorted_keys, keybits, a, m) > p) gamma = m;
        if (gamma == a) {
            childL[id] = LEAF | (int32_t)a;
            parent_leaf[a] = id;
        } else {
            childL[id] = (int32_t)gamma;
            parent_internal[gamma] = id;
            stack.push_back({a, gamma, (int32_t)gamma});
        }
        if (gamma + 1 == b) {
            childR[id] = LEAF | (int32_t)b;
            parent_leaf[b] = id;
        } else {
            childR[id] = (int32_t)(gamma + 1);
            parent_internal[gamma + 1] = id;
            stack.push_back({gamma + 1, b, (int32_t)(gamma + 1)});
        }
    }
}

// Boxes of all internal nodes as unions of their children. leaf_lo/hi: 3*n float32
// in SORTED order. node_lo/hi: 3*(n-1) out. Children are visited before parents by
// a post-order walk.
void oracle_fit(const int32_t* childL, const int32_t* childR, int64_t n, const float* leaf_lo,
                const float* leaf_hi, float* node_lo, float* node_hi) {
    if (n < 2) return;
    std::vector<std::pair<int32_t, int>> st;
    st.push_back({0, 0});
    while (!st.empty()) {
        auto& top = st.back();
        const int32_t id = top.first;
        if (top.second == 0) {
            top.second = 1;
            for (int32_t c : {childL[id], childR[id]})
                if (!(c & LEAF)) st.push_back({c, 0});
            continue;
        }
        for (int a = 0; a < 3; ++a) {
            float mn = INFINITY, mx = -INFINITY;
            for (int32_t c : {childL[id], childR[id]}) {
                const float* clo = (c & LEAF) ? &leaf_lo[3 * (int64_t)(c & 0x7fffffff)] : &node_lo[3 * (int64_t)c];
                const float* chi = (c & LEAF) ? &leaf_hi[3 * (int64_t)(c & 0x7fffffff)] : &node_hi[3 * (int64_t)c];
                mn = std::min(mn, clo[a]);
                mx = std::max(mx, chi[a]);
            }
            node_lo[3 * (int64_t)id + a] = mn;
            node_hi[3 * (int64_t)id + a] = mx;
        }
        st.pop_back();
    }
}

// Clustering build over n >= 2 leaves in sorted order (boxes leaf_lo/hi, 3*n float32).
// Clusters start as the leaves. One iteration:
//   1. nearest neighbour of each cluster i among positions i-radius..i+radius (not i):
//      smallest union area; equal areas by the pair hash fmix32(fmix32(a) + b) of the
//      two positions a < b; then the lower position;
//   2. each pair that are each other's nearest neighbour merges; the new internal node
//      has the lower position's cluster as left child and takes that position;
//   3. the remaining clusters close ranks in their order.
// The m-th merge of the build (iterations in order, merges within one by position)
// is internal node n-2-m, so the last one is the root, 0. Output in the format of
// oracle_topology; *iterations = number of iterations run.
void oracle_ploc(const float* leaf_lo, const float* leaf_hi, int64_t n, int radius, int32_t* childL,
                 int32_t* childR, int32_t* parent_internal, int32_t* parent_leaf, int64_t* iterations) {
    *iterations = 0;
    if (n < 2) return;
    struct Cluster {
        float lo[3], hi[3];
        int32_t id;  // leaf: LEAF | sorted position; internal: node index
    };
    std::vector<Cluster> cur((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        for (int a = 0; a < 3; ++a) {
            cur[(size_t)k].lo[a] = leaf_lo[3 * k + a];
            cur[(size_t)k].hi[a] = leaf_hi[3 * k + a];
        }
        cur[(size_t)k].id = LEAF | (int32_t)k;
    }
    auto link = [&](int32_t child, int32_t parent) {
        if (child & LEAF)
            parent_leaf[child & 0x7fffffff] = parent;
        else
            parent_internal[child] = parent;
    };
    int64_t merges = 0;
    while (cur.size() > 1) {
        const int64_t m = (int64_t)cur.size();
        std::vector<int64_t> nearest((size_t)m);
        for (int64_t i = 0; i < m; ++i) {
            uint64_t best_key = ~0ull;
            int64_t best = -1;
            for (int64_t j = std::max<int64_t>(0, i - radius); j <= std::min<int64_t>(m - 1, i + radius); ++j) {
                if (j == i) continue;
                const Cluster &a = cur[(size_t)i], &b = cur[(size_t)j];
                const float area = union_area(a.lo, a.hi, b.lo, b.hi);
                uint32_t bits;
                std::memcpy(&bits, &area, 4);
                const uint32_t lo = (uint32_t)std::min(i, j), hi = (uint32_t)std::max(i, j);
                const uint64_t key = ((uint64_t)bits << 32) | fmix32(fmix32(lo) + hi);
                if (key < best_key) best_key = key, best = j;  // j ascends: ties keep the lower j
            }
            nearest[(size_t)i] = best;
        }
        std::vector<Cluster> next;
        for (int64_t i = 0; i < m; ++i) {
            const int64_t j = nearest[(size_t)i];
            const bool mutual = nearest[(size_t)j] == i;
            if (mutual && j < i) continue;  // merged into the cluster at j
            if (!mutual) {
                next.push_back(cur[(size_t)i]);
                continue;
            }
            const int32_t q = (int32_t)(n - 2 - merges);
            ++merges;
            const Cluster &a = cur[(size_t)i], &b = cur[(size_t)j];
            childL[q] = a.id;
            childR[q] = b.id;
            link(a.id, q);
            link(b.id, q);
            Cluster u;
            for (int k = 0; k < 3; ++k) u.lo[k] = std::fmin(a.lo[k], b.lo[k]), u.hi[k] = std::fmax(a.hi[k], b.hi[k]);
            u.id = q;
            next.push_back(u);
        }
        cur.swap(next);
        ++*iterations;
    }
    parent_internal[0] = -1;
}

// Clustering inside the linear BVH's subtrees, bottom up (a one-pass form of the
// locally-ordered clustering the paper names as HIPRT's balanced build, Sec. 8). Input:
// n >= 2 leaves in sorted order (boxes) and the LBVH over them (lbvhL/lbvhR as from
// oracle_topology). Every LBVH node p, children first, turns its children's cluster
// lists into its own:
//   1. L = the left child's clusters, then the right child's (a leaf child is the one
//      cluster of that leaf); F = the unused internal-node numbers of both children and
//      p itself, in descending order;
//   2. while L holds more than `cap` clusters (more than 1 at the root, node 0): every
//      cluster's nearest neighbour in L by union area, equal areas by the pair hash
//      fmix32(fmix32(a) + b) of the list positions a < b, then the lower position; each
//      mutual pair (a, b), a < b, becomes the internal node numbered by the next entry
//      of F (pairs in order of a) with left child a, and takes position a; the others
//      close ranks in order;
//   3. L and the unused rest of F go to p's parent.
// F always holds |L| - 1 numbers, so the root's last merge takes its own number 0.
// Output in the format of oracle_topology.
void oracle_subtree_cluster(const float* leaf_lo, const float* leaf_hi, int64_t n, int cap, const int32_t* lbvhL,
                            const int32_t* lbvhR, int32_t* childL, int32_t* childR, int32_t* parent_internal,
                            int32_t* parent_leaf) {
    if (n < 2) return;
    struct Cluster {
        float lo[3], hi[3];
        int32_t id;  // leaf: LEAF | sorted position; internal: node number
    };
    struct Out {
        std::vector<Cluster> list;
        std::vector<int32_t> free_ids;
    };
    auto link = [&](int32_t child, int32_t parent) {
        if (child & LEAF)
            parent_leaf[child & 0x7fffffff] = parent;
        else
            parent_internal[child] = parent;
    };
    auto leaf = [&](int32_t k) {
        Out o;
        Cluster c;
        for (int a = 0; a < 3; ++a) c.lo[a] = leaf_lo[3 * (int64_t)k + a], c.hi[a] = leaf_hi[3 * (int64_t)k + a];
        c.id = LEAF | k;
        o.list.push_back(c);
        return o;
    };
    std::vector<Out> done((size_t)(n - 1));
    // children-first order: an explicit post-order walk of the LBVH from the root
    std::vector<std::pair<int32_t, bool>> st{{0, false}};
    while (!st.empty()) {
        const auto [p, expanded] = st.back();
        st.pop_back();
        if (!expanded) {
            st.push_back({p, true});
            if (!(lbvhR[p] & LEAF)) st.push_back({lbvhR[p], false});
            if (!(lbvhL[p] & LEAF)) st.push_back({lbvhL[p], false});
            continue;
        }
        Out a = (lbvhL[p] & LEAF) ? leaf(lbvhL[p] & 0x7fffffff) : std::move(done[(size_t)lbvhL[p]]);
        Out b = (lbvhR[p] & LEAF) ? leaf(lbvhR[p] & 0x7fffffff) : std::move(done[(size_t)lbvhR[p]]);
        std::vector<Cluster> L = a.list;
        L.insert(L.end(), b.list.begin(), b.list.end());
        std::vector<int32_t> F = a.free_ids;
        F.insert(F.end(), b.free_ids.begin(), b.free_ids.end());
        F.push_back(p);
        std::sort(F.begin(), F.end(), std::greater<int32_t>());
        size_t next_free = 0;
        const size_t target = p == 0 ? 1 : (size_t)cap;
        while (L.size() > target) {
            const int64_t m = (int64_t)L.size();
            std::vector<int64_t> nearest((size_t)m);
            for (int64_t i = 0; i < m; ++i) {
                uint64_t best_key = ~0ull;
                int64_t best = -1;
                for (int64_t j = 0; j < m; ++j) {
                    if (j == i) continue;
                    const float area = union_area(L[(size_t)i].lo, L[(size_t)i].hi, L[(size_t)j].lo, L[(size_t)j].hi);
                    uint32_t bits;
                    std::memcpy(&bits, &area, 4);
                    const uint32_t lo = (uint32_t)std::min(i, j), hi = (uint32_t)std::max(i, j);
                    const uint64_t key = ((uint64_t)bits << 32) | fmix32(fmix32(lo) + hi);
                    if (key < best_key) best_key = key, best = j;  // j ascends: ties keep the lower j
                }
                nearest[(size_t)i] = best;
            }
            std::vector<Cluster> next;
            for (int64_t i = 0; i < m; ++i) {
                const int64_t j = nearest[(size_t)i];
                const bool mutual = nearest[(size_t)j] == i;
                if (mutual && j < i) continue;  // merged into the cluster at j
                if (!mutual) {
                    next.push_back(L[(size_t)i]);
                    continue;
                }
                const int32_t q = F[next_free++];
                const Cluster &x = L[(size_t)i], &y = L[(size_t)j];
                childL[q] = x.id;
                childR[q] = y.id;
                link(x.id, q);
                link(y.id, q);
                Cluster u;
                for (int k = 0; k < 3; ++k) u.lo[k] = std::fmin(x.lo[k], y.lo[k]), u.hi[k] = std::fmax(x.hi[k], y.hi[k]);
                u.id = q;
                next.push_back(u);
            }
            L.swap(next);
        }
        done[(size_t)p].list = std::move(L);
        done[(size_t)p].free_ids.assign(F.begin() + (std::ptrdiff_t)next_free, F.end());
    }
    parent_internal[0] = -1;
}

// Surface-area cost of a binary BVH: sum over internal nodes of box area, divided by
// the root box area (the quality measure of Sec. 6.2 "BVH Construction").
double oracle_sah_cost(const float* node_lo, const float* node_hi, int64_t n_internal) {
    auto area = [&](int64_t k) {
        double dx = (double)node_hi[3 * k] - node_lo[3 * k];
        double dy = (double)node_hi[3 * k + 1] - node_lo[3 * k + 1];
        double dz = (double)node_hi[3 * k + 2] - node_lo[3 * k + 2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    };
    if (n_internal < 1) return 0.0;
    double s = 0.0;
    for (int64_t k = 0; k < n_internal; ++k) s += area(k);
    double r = area(0);
    return r > 0 ? s / r : 0.0;
}

// Quantised 4-wide nodes: the paper's wide trees (Sec. 6.2, branching factor 4) with
// each child box stored as 8-bit planes relative to the node's own box, the compressed
// wide node of Ylitie, Karras and Laine ("Efficient Incoherent Ray Traversal on GPUs
// Through Compressed Wide BVHs", HPG 2017). Input: m wide nodes as wide_nodes gives
// them (lo, hi: 4 slots x 3 floats each; child: 4 words, 0xFFFFFFFF = empty slot).
// For every node and axis a, over the used slots:
//   p_a  = the smallest slot lo_a,  H_a = the largest slot hi_a;
//   e_a  = the least integer e in [-126, 127] with fl(p_a + 255 * 2^e) >= H_a;
//   a slot's lower plane qlo = the largest q in [0, 255] with fl(p_a + q 2^e_a) <= lo_a,
//   its upper plane   qhi = the smallest q in [0, 255] with fl(p_a + q 2^e_a) >= hi_a,
// fl being float32 rounding to nearest (q 2^e is exact, so each value is rounded once).
// Both conditions are monotone in q and e, so each choice is unique, and the decoded
// box [fl(p + qlo 2^e), fl(p + qhi 2^e)] contains the slot's box. Output: 16 words per
// node: p.x, p.y, p.z; the three biased exponents e_a + 127 in bytes 0-2 of word 3;
// words 4-9 the planes qlo.x, qhi.x, qlo.y, qhi.y, qlo.z, qhi.z, slot j in byte j;
// words 10-13 the child words; words 14-15 zero. An empty slot has qlo = 255, qhi = 0.
// A node without a used slot has p = 0 and e = -126 on every axis.
static float qdecode(float p, int q, int e) {
    const float step = std::ldexp(1.0f, e);
    const float off = (float)q * step;  // exact: q < 2^8 and step a power of two
    return p + off;
}

void oracle_quantize_wide(const float* lo, const float* hi, const uint32_t* child, int64_t m, uint32_t* out) {
    for (int64_t k = 0; k < m; ++k) {
        const float* L = lo + 12 * k;  // [slot][axis]
        const float* Hh = hi + 12 * k;
        const uint32_t* C = child + 4 * k;
        uint32_t* o = out + 16 * k;
        std::memset(o, 0, 16 * sizeof(uint32_t));
        bool used[4];
        int nUsed = 0;
        for (int j = 0; j < 4; ++j) nUsed += (used[j] = C[j] != 0xFFFFFFFFu);
        uint32_t expWord = 0;
        for (int a = 0; a < 3; ++a) {
            float p = 0.0f, top = 0.0f;
            if (nUsed) {
                p = INFINITY, top = -INFINITY;
                for (int j = 0; j < 4; ++j)
                    if (used[j]) p = std::min(p, L[3 * j + a]), top = std::max(top, Hh[3 * j + a]);
            }
            // the least exponent whose 255th step reaches the top of the node's box
            int e = -126;
            if (nUsed) {
                const double ext = (double)top - (double)p;
                if (ext > 0) {
                    int k2 = 0;
                    std::frexp(ext / 255.0, &k2);  // ext / 255 < 2^k2
                    e = std::max(-126, std::min(127, k2));
                }
                while (e > -126 && qdecode(p, 255, e - 1) >= top) --e;
                while (e < 127 && qdecode(p, 255, e) < top) ++e;
            }
            uint32_t qlo = 0, qhi = 0;
            for (int j = 0; j < 4; ++j) {
                int ql = 255, qh = 0;
                if (used[j]) {
                    const float l = L[3 * j + a], h = Hh[3 * j + a];
                    const double step = std::ldexp(1.0, e);
                    ql = (int)std::max(0.0, std::min(255.0, std::floor(((double)l - p) / step)));
                    while (ql > 0 && qdecode(p, ql, e) > l) --ql;
                    while (ql < 255 && qdecode(p, ql + 1, e) <= l) ++ql;
                    qh = (int)std::max(0.0, std::min(255.0, std::ceil(((double)h - p) / step)));
                    while (qh < 255 && qdecode(p, qh, e) < h) ++qh;
                    while (qh > 0 && qdecode(p, qh - 1, e) >= h) --qh;
                }
                qlo |= (uint32_t)ql << (8 * j);
                qhi |= (uint32_t)qh << (8 * j);
            }
            std::memcpy(o + a, &p, 4);
            expWord |= (uint32_t)(e + 127) << (8 * a);
            o[4 + 2 * a] = qlo;
            o[5 + 2 * a] = qhi;
        }
        o[3] = expWord;
        for (int j = 0; j < 4; ++j) o[10 + j] = C[j];
    }
}

}  // extern "C"
