// ORACLE (test infrastructure only; never linked into the library): Lambertian
// shading of one triangle mesh, its analytic gradient, and central finite
// differences, all in FP64 with brute-force visibility.
//
// Forward, per pixel (primary ray o + t d):
//   closest hit (prim, t, u, v) over every triangle (Moller-Trumbore, double-sided);
//   n_f = the face normal normalize((v1-v0) x (v2-v0)), turned to face the ray
//   (Sec. 4.1's normal, oriented toward the viewer);
//   s = max(0, n_f . l), l the light direction used as given (Sec. 4.1 cosine law;
//   the Lambert BRDF c/pi of Sec. 5.2 with the constant pi folded into the loss scale);
//   V = 1 unless the shadow ray p + 1e-4 n_f + t l, t in [0, inf), hits a triangle;
//   c(u,v) = (1-u-v) c[i0] + u c[i1] + v c[i2] per channel (per-vertex colours);
//   I = V s c(u,v); a miss gives I = 0.
// Loss L = sum over pixels and channels of (I - I*)^2.
// Gradient (interior hits; visibility and the hit triangle are piecewise constant):
//   dL/dc_k = sum 2(I-I*) V s w_k, w = (1-u-v, u, v);
//   dL/dl   = sum g_s n_f where g_s = sum_ch 2(I-I*) V c, when n_f . l > 0;
//   dL/dv_k through n_f (m = e1 x e2; ds/dm = sigma (l - n (n.l)) / |m|) and through
//   (u, v) on the fixed ray: d(t,u,v)/dv_k = -w_k A^-1 with A = [-d | e1 | e2].
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include "oracle_math.h"

using namespace oracle;

namespace {

struct Mesh {
    const double* v;    // 3 per vertex
    const uint32_t* i;  // 3 per triangle
    int64_t nt;
    V3 vert(int64_t t, int k) const {
        const double* p = v + 3 * (int64_t)i[3 * t + k];
        return v3(p[0], p[1], p[2]);
    }
};

bool mt(V3 o, V3 d, V3 v0, V3 v1, V3 v2, double tmin, double tmax, double& t, double& u, double& v) {
    const V3 e1 = v1 - v0, e2 = v2 - v0;
    const V3 P = cross(d, e2);
    const double det = dot(e1, P);
    if (det == 0.0) return false;
    const double inv = 1.0 / det;
    const V3 T = o - v0;
    u = dot(T, P) * inv;
    if (u < 0.0 || u > 1.0) return false;
    const V3 Q = cross(T, e1);
    v = dot(d, Q) * inv;
    if (v < 0.0 || u + v > 1.0) return false;
    t = dot(e2, Q) * inv;
    return t >= tmin && t <= tmax;
}

struct PixelState {
    int32_t prim = -1;
    double t = 0, u = 0, v = 0;
    int vis = 0;
    int sign = 0;  // sign of n_f . l
    double s = 0;
    V3 nf{0, 0, 0};
};

PixelState shadePixel(const Mesh& M, const float* ray, V3 l) {
    PixelState S;
    const V3 o = v3(ray[0], ray[1], ray[2]), d = v3(ray[4], ray[5], ray[6]);
    double best = INFINITY;
    for (int64_t p = 0; p < M.nt; ++p) {
        double t, u, v;
        if (mt(o, d, M.vert(p, 0), M.vert(p, 1), M.vert(p, 2), ray[3], ray[7], t, u, v) && t < best) {
            best = t;
            S.prim = (int32_t)p;
            S.t = t, S.u = u, S.v = v;
        }
    }
    if (S.prim < 0) return S;
    const V3 v0 = M.vert(S.prim, 0), v1 = M.vert(S.prim, 1), v2 = M.vert(S.prim, 2);
    V3 n = normalize(cross(v1 - v0, v2 - v0));
    if (dot(n, d) > 0.0) n = -n;
    S.nf = n;
    const double nl = dot(n, l);
    S.sign = nl > 0 ? 1 : (nl < 0 ? -1 : 0);
    S.s = std::max(0.0, nl);
    // shadow ray
    const V3 org = (o + d * S.t) + n * 1e-4;
    S.vis = 1;
    for (int64_t p = 0; p < M.nt; ++p) {
        double t, u, v;
        if (mt(org, l, M.vert(p, 0), M.vert(p, 1), M.vert(p, 2), 0.0, INFINITY, t, u, v)) {
            S.vis = 0;
            break;
        }
    }
    return S;
}

void colourAt(const Mesh& M, const double* col, const PixelState& S, double out[3]) {
    const double w0 = 1.0 - S.u - S.v;
    for (int ch = 0; ch < 3; ++ch) {
        out[ch] = w0 * col[3 * (int64_t)M.i[3 * S.prim + 0] + ch] + S.u * col[3 * (int64_t)M.i[3 * S.prim + 1] + ch] +
                  S.v * col[3 * (int64_t)M.i[3 * S.prim + 2] + ch];
    }
}

template <class F>
void parallel_for(int64_t n, F f) {
    const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < threads; ++w)
        pool.emplace_back([&]() {
            for (;;) {
                const int64_t s = next.fetch_add(64);
                if (s >= n) break;
                for (int64_t i = s; i < std::min(n, s + 64); ++i) f(i);
            }
        });
    for (auto& t : pool) t.join();
}

// Per-pixel gradient contribution of one pixel to every parameter it touches.
struct PixelGrad {
    uint32_t vk[3];
    double dcol[3][3];  // [corner][channel]
    double dl[3];
    double dpos[3][3];  // [corner][axis]
};

PixelGrad pixelGrad(const Mesh& M, const double* col, V3 l, const float* ray, const PixelState& S, const double* target) {
    PixelGrad G{};
    for (int k = 0; k < 3; ++k) G.vk[k] = M.i[3 * S.prim + k];
    double c[3];
    colourAt(M, col, S, c);
    double gI[3];
    for (int ch = 0; ch < 3; ++ch) gI[ch] = 2.0 * (S.vis * S.s * c[ch] - target[ch]);
    const double w[3] = {1.0 - S.u - S.v, S.u, S.v};
    for (int k = 0; k < 3; ++k)
        for (int ch = 0; ch < 3; ++ch) G.dcol[k][ch] = gI[ch] * S.vis * S.s * w[k];
    if (!S.vis) return G;
    // through the shading term
    double gs = 0.0;
    for (int ch = 0; ch < 3; ++ch) gs += gI[ch] * c[ch];
    const V3 v0 = M.vert(S.prim, 0), v1 = M.vert(S.prim, 1), v2 = M.vert(S.prim, 2);
    const V3 e1 = v1 - v0, e2 = v2 - v0;
    V3 dv[3] = {v3(0, 0, 0), v3(0, 0, 0), v3(0, 0, 0)};
    if (S.sign > 0) {
        for (int a = 0; a < 3; ++a) G.dl[a] = gs * comp(S.nf, a);
        const V3 m = cross(e1, e2);
        const double ml = length(m);
        const V3 n = m * (1.0 / ml);
        const double sigma = dot(S.nf, n) > 0 ? 1.0 : -1.0;
        const V3 gm = (l - n * dot(n, l)) * (gs * sigma / ml);
        dv[1] = dv[1] + cross(e2, gm);
        dv[2] = dv[2] + cross(gm, e1);
        dv[0] = dv[0] + cross(e1 - e2, gm);
    }
    // through the barycentrics of the hit point on the fixed ray
    double gu = 0.0, gv = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        const double c0 = col[3 * (int64_t)G.vk[0] + ch], c1 = col[3 * (int64_t)G.vk[1] + ch],
                     c2 = col[3 * (int64_t)G.vk[2] + ch];
        gu += gI[ch] * S.s * (c1 - c0);
        gv += gI[ch] * S.s * (c2 - c0);
    }
    const V3 d = v3(ray[4], ray[5], ray[6]);
    const V3 a1 = -d, a2 = e1, a3 = e2;
    const double det = dot(a1, cross(a2, a3));
    if (det != 0.0) {
        const V3 r2 = cross(a3, a1) * (1.0 / det), r3 = cross(a1, a2) * (1.0 / det);
        const V3 y = r2 * gu + r3 * gv;  // A^-T (0, gu, gv)
        for (int k = 0; k < 3; ++k) dv[k] = dv[k] - y * w[k];
    }
    for (int k = 0; k < 3; ++k) G.dpos[k][0] = dv[k].x, G.dpos[k][1] = dv[k].y, G.dpos[k][2] = dv[k].z;
    return G;
}

}  // namespace

extern "C" {

// Forward render. verts: 3*nv doubles, idx: 3*nt, col: 3*nv, light: 3, rays: n*8 float32.
// Outputs: image (n*3), prim (n; -1 on a miss), vis (n), sign (n), t/u/v (n each, may be NULL).
void oracle_lambert_forward(const double* verts, int64_t nv, const uint32_t* idx, int64_t nt, const double* col,
                            const double* light, const float* rays, int64_t n, double* image, int32_t* prim,
                            int8_t* vis, int8_t* sign, double* tuv) {
    (void)nv;
    const Mesh M{verts, idx, nt};
    const V3 l = v3(light[0], light[1], light[2]);
    parallel_for(n, [&](int64_t p) {
        const PixelState S = shadePixel(M, rays + 8 * p, l);
        prim[p] = S.prim;
        vis[p] = (int8_t)S.vis;
        sign[p] = (int8_t)S.sign;
        if (tuv) tuv[3 * p] = S.t, tuv[3 * p + 1] = S.u, tuv[3 * p + 2] = S.v;
        double c[3] = {0, 0, 0};
        if (S.prim >= 0) colourAt(M, col, S, c);
        for (int ch = 0; ch < 3; ++ch) image[3 * p + ch] = S.prim >= 0 ? S.vis * S.s * c[ch] : 0.0;
    });
}

// Loss and its analytic gradient. target: n*3. dcol/dpos: 3*nv (zeroed here), dl: 3.
double oracle_lambert_gradient(const double* verts, int64_t nv, const uint32_t* idx, int64_t nt, const double* col,
                               const double* light, const float* rays, int64_t n, const double* target, double* dcol,
                               double* dl, double* dpos) {
    const Mesh M{verts, idx, nt};
    const V3 l = v3(light[0], light[1], light[2]);
    std::vector<PixelState> S((size_t)n);
    parallel_for(n, [&](int64_t p) { S[(size_t)p] = shadePixel(M, rays + 8 * p, l); });
    std::fill(dcol, dcol + 3 * nv, 0.0);
    std::fill(dpos, dpos + 3 * nv, 0.0);
    dl[0] = dl[1] = dl[2] = 0.0;
    double loss = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        const PixelState& s = S[(size_t)p];
        double c[3] = {0, 0, 0};
        if (s.prim >= 0) colourAt(M, col, s, c);
        for (int ch = 0; ch < 3; ++ch) {
            const double I = s.prim >= 0 ? s.vis * s.s * c[ch] : 0.0;
            loss += (I - target[3 * p + ch]) * (I - target[3 * p + ch]);
        }
        if (s.prim < 0) continue;
        const PixelGrad G = pixelGrad(M, col, l, rays + 8 * p, s, target + 3 * p);
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                dcol[3 * (int64_t)G.vk[k] + a] += G.dcol[k][a];
                dpos[3 * (int64_t)G.vk[k] + a] += G.dpos[k][a];
            }
        for (int a = 0; a < 3; ++a) dl[a] += G.dl[a];
    }
    return loss;
}

// Per-parameter L1 norms of the per-pixel terms of the analytic gradient: for each
// parameter the sum over hit pixels of |that pixel's term| (the terms
// oracle_lambert_gradient adds up). It measures how much the gradient's terms cancel,
// which sets the accuracy a sum of rounded terms can reach. Outputs as
// oracle_lambert_gradient's (zeroed here).
void oracle_lambert_gradient_l1(const double* verts, int64_t nv, const uint32_t* idx, int64_t nt, const double* col,
                                const double* light, const float* rays, int64_t n, const double* target, double* acol,
                                double* al, double* apos) {
    const Mesh M{verts, idx, nt};
    const V3 l = v3(light[0], light[1], light[2]);
    std::vector<PixelState> S((size_t)n);
    parallel_for(n, [&](int64_t p) { S[(size_t)p] = shadePixel(M, rays + 8 * p, l); });
    std::fill(acol, acol + 3 * nv, 0.0);
    std::fill(apos, apos + 3 * nv, 0.0);
    al[0] = al[1] = al[2] = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        const PixelState& s = S[(size_t)p];
        if (s.prim < 0) continue;
        const PixelGrad G = pixelGrad(M, col, l, rays + 8 * p, s, target + 3 * p);
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                acol[3 * (int64_t)G.vk[k] + a] += std::fabs(G.dcol[k][a]);
                apos[3 * (int64_t)G.vk[k] + a] += std::fabs(G.dpos[k][a]);
            }
        for (int a = 0; a < 3; ++a) al[a] += std::fabs(G.dl[a]);
    }
}

// Central differences of the masked loss for a list of parameters, and the analytic
// gradient of the pixels the mask removes. Parameter ids: [0, 3nv) colours
// (3*vertex + channel), [3nv, 3nv+3) light, [3nv+3, 6nv+3) positions (3*vertex + axis).
// A pixel enters the loss of parameter q only if its (prim, V, sign(n.l)) is the same
// in the renders at q-h, q and q+h. Only pixels that can change are re-rendered:
// colours touch the pixels whose hit triangle uses the vertex; the light touches every
// hit pixel; a position touches the pixels whose primary or shadow ray meets the box
// of the vertex's triangles widened by 4h. exclude (n bytes, may be NULL) removes
// pixels from every parameter's loss; unstable (n bytes, may be NULL) receives 1 for
// each pixel found unstable for some parameter.
void oracle_lambert_fd(const double* verts, int64_t nv, const uint32_t* idx, int64_t nt, const double* col,
                       const double* light, const float* rays, int64_t n, const double* target,
                       const int64_t* params, int64_t nparams, double h, double* fd, double* masked_analytic,
                       int64_t* masked_count, const uint8_t* exclude, uint8_t* unstable) {
    const Mesh M0{verts, idx, nt};
    const V3 l0 = v3(light[0], light[1], light[2]);
    std::vector<PixelState> S0((size_t)n);
    parallel_for(n, [&](int64_t p) { S0[(size_t)p] = shadePixel(M0, rays + 8 * p, l0); });
    // vertex -> triangles
    std::vector<std::vector<int64_t>> vtris((size_t)nv);
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) vtris[idx[3 * t + k]].push_back(t);
    auto pixelLoss = [&](const Mesh& M, const double* c, V3 l, int64_t p, const PixelState& s) {
        double cc[3] = {0, 0, 0};
        if (s.prim >= 0) colourAt(M, c, s, cc);
        double L = 0;
        for (int ch = 0; ch < 3; ++ch) {
            const double I = s.prim >= 0 ? s.vis * s.s * cc[ch] : 0.0;
            L += (I - target[3 * p + ch]) * (I - target[3 * p + ch]);
        }
        return L;
    };
    for (int64_t qi = 0; qi < nparams; ++qi) {
        const int64_t q = params[qi];
        std::vector<double> vp(verts, verts + 3 * (int64_t)std::max<int64_t>(nv, 0)), vm = vp;
        std::vector<double> cp(col, col + 3 * nv), cm = cp;
        V3 lp = l0, lm = l0;
        std::vector<int64_t> cand;
        int kind;
        if (q < 3 * nv) {
            kind = 0;
            cp[(size_t)q] += h, cm[(size_t)q] -= h;
            const int64_t vtx = q / 3;
            for (int64_t p = 0; p < n; ++p) {
                const int32_t pr = S0[(size_t)p].prim;
                if (pr < 0) continue;
                if (idx[3 * pr] == vtx || idx[3 * pr + 1] == vtx || idx[3 * pr + 2] == vtx) cand.push_back(p);
            }
        } else if (q < 3 * nv + 3) {
            kind = 1;
            const int a = (int)(q - 3 * nv);
            if (a == 0) lp.x += h, lm.x -= h;
            if (a == 1) lp.y += h, lm.y -= h;
            if (a == 2) lp.z += h, lm.z -= h;
            for (int64_t p = 0; p < n; ++p)
                if (S0[(size_t)p].prim >= 0) cand.push_back(p);
        } else {
            kind = 2;
            const int64_t r = q - 3 * nv - 3;
            vp[(size_t)r] += h, vm[(size_t)r] -= h;
            const int64_t vtx = r / 3;
            V3 lo = v3(INFINITY, INFINITY, INFINITY), hi = v3(-INFINITY, -INFINITY, -INFINITY);
            for (int64_t t : vtris[(size_t)vtx])
                for (int k = 0; k < 3; ++k) {
                    const V3 x = M0.vert(t, k);
                    lo = v3(std::min(lo.x, x.x), std::min(lo.y, x.y), std::min(lo.z, x.z));
                    hi = v3(std::max(hi.x, x.x), std::max(hi.y, x.y), std::max(hi.z, x.z));
                }
            const double g = 4.0 * h + 1e-9;
            lo = lo - v3(g, g, g);
            hi = hi + v3(g, g, g);
            auto meets = [&](V3 o, V3 d, double tmax) {
                double t0 = 0.0, t1 = tmax;
                for (int a = 0; a < 3; ++a) {
                    const double oa = comp(o, a), da = comp(d, a), la = comp(lo, a), ha = comp(hi, a);
                    if (da == 0.0) {
                        if (oa < la || oa > ha) return false;
                        continue;
                    }
                    double ta = (la - oa) / da, tb = (ha - oa) / da;
                    if (ta > tb) std::swap(ta, tb);
                    t0 = std::max(t0, ta);
                    t1 = std::min(t1, tb);
                    if (t0 > t1) return false;
                }
                return true;
            };
            for (int64_t p = 0; p < n; ++p) {
                const float* ry = rays + 8 * p;
                const V3 o = v3(ry[0], ry[1], ry[2]), d = v3(ry[4], ry[5], ry[6]);
                bool hit = meets(o, d, ry[7]);
                const PixelState& s = S0[(size_t)p];
                if (!hit && s.prim >= 0) hit = meets((o + d * s.t) + s.nf * 1e-4, l0, INFINITY);
                if (hit) cand.push_back(p);
            }
        }
        (void)kind;
        const Mesh Mp{vp.data(), idx, nt}, Mm{vm.data(), idx, nt};
        std::vector<PixelState> Sp(cand.size()), Sm(cand.size());
        parallel_for((int64_t)cand.size(), [&](int64_t j) {
            Sp[(size_t)j] = shadePixel(Mp, rays + 8 * cand[(size_t)j], lp);
            Sm[(size_t)j] = shadePixel(Mm, rays + 8 * cand[(size_t)j], lm);
        });
        double Lp = 0, Lm = 0, ma = 0;
        int64_t masked = 0;
        for (size_t j = 0; j < cand.size(); ++j) {
            const int64_t p = cand[j];
            const PixelState &s0 = S0[(size_t)p], &sp = Sp[j], &sm = Sm[j];
            const bool stable = s0.prim == sp.prim && s0.prim == sm.prim && s0.vis == sp.vis && s0.vis == sm.vis &&
                                s0.sign == sp.sign && s0.sign == sm.sign;
            if (!stable && unstable) unstable[p] = 1;
            if (exclude && exclude[p]) continue;  // left out of every parameter's loss
            if (stable) {
                Lp += pixelLoss(Mp, cp.data(), lp, p, sp);
                Lm += pixelLoss(Mm, cm.data(), lm, p, sm);
            } else if (s0.prim >= 0) {
                ++masked;
                const PixelGrad G = pixelGrad(M0, col, l0, rays + 8 * p, s0, target + 3 * p);
                if (q < 3 * nv) {
                    for (int k = 0; k < 3; ++k)
                        if ((int64_t)G.vk[k] == q / 3) ma += G.dcol[k][q % 3];
                } else if (q < 3 * nv + 3) {
                    ma += G.dl[q - 3 * nv];
                } else {
                    const int64_t r = q - 3 * nv - 3;
                    for (int k = 0; k < 3; ++k)
                        if ((int64_t)G.vk[k] == r / 3) ma += G.dpos[k][r % 3];
                }
            }
        }
        fd[qi] = (Lp - Lm) / (2.0 * h);
        masked_analytic[qi] = ma;
        masked_count[qi] = masked;
    }
}

}  // extern "C"
