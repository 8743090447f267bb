// ORACLE (test infrastructure only; never linked into the library): ray generation
// and ambient-occlusion rays in FP64, rounded to float32 at the end.
//
//  * Camera (paper Sec. 3.2): lens at `origin`, film at distance 1 along
//    forward = normalize(up x right); the film point for normalised coordinates (u,v)
//    is origin + forward + lerp(-right, right, u) + lerp(up, -up, v); the direction is
//    normalised. Pixel (x, y) uses its centre u = (x+1/2)/W, v = (y+1/2)/H; y = 0 is
//    the top row; ray index = y*W + x; minT = 0, maxT = +inf.
//  * Cosine-weighted hemisphere (Sec. 4.1): phi = 2 pi xi0, r = sqrt(xi1),
//    (x, z) = r (cos phi, sin phi), y = sqrt(max(1 - r^2, 0)), Y up.
//  * AO ray frame (Sec. 4.1-4.2): n = the hit triangle's world-space face normal,
//    turned to face the incoming ray; tangent = normalize(v1 - v0) in world space;
//    bitangent = n x tangent; direction = tangent*x + bitangent*z + n*y; origin =
//    p + 1e-4 n with p = o + t d; minT = 0, maxT = the given length.
//  * The random numbers xi come from the splitmix64 generator (Steele, Lea, Flood
//    2014) at counter c = (pixel << 32) | (sample << 1) | dim of stream `seed`:
//    h = mix(seed + (c + 1) * 0x9E3779B97F4A7C15), xi = (h >> 40) * 2^-24.
#include <cmath>
#include <cstdint>

#include "oracle_math.h"

using namespace oracle;

namespace {
const uint32_t NONE = 0xFFFFFFFFu;
const double PI = 3.14159265358979323846;

void store_ray(float* out, V3 o, double tmin, V3 d, double tmax) {
    out[0] = (float)o.x, out[1] = (float)o.y, out[2] = (float)o.z, out[3] = (float)tmin;
    out[4] = (float)d.x, out[5] = (float)d.y, out[6] = (float)d.z, out[7] = (float)tmax;
}
}  // namespace

extern "C" {

double oracle_xi(uint64_t seed, uint64_t pixel, uint32_t sample, uint32_t dim) {
    const uint64_t c = (pixel << 32) | ((uint64_t)sample << 1) | (uint64_t)dim;
    const uint64_t h = mix64(seed + (c + 1ull) * 0x9E3779B97F4A7C15ull);
    return (double)(h >> 40) * (1.0 / 16777216.0);
}

// cam: origin.xyz, right.xyz, up.xyz (9 floats). rays: W*H x 8 float32 out.
void oracle_camera_rays(const float* cam, int64_t W, int64_t H, float* rays) {
    const V3 o = v3(cam[0], cam[1], cam[2]), right = v3(cam[3], cam[4], cam[5]), up = v3(cam[6], cam[7], cam[8]);
    const V3 fwd = normalize(cross(up, right));
    for (int64_t y = 0; y < H; ++y)
        for (int64_t x = 0; x < W; ++x) {
            const double u = (x + 0.5) / (double)W, v = (y + 0.5) / (double)H;
            const V3 lr = (-right) + (right - (-right)) * u;  // lerp(-right, right, u)
            const V3 ud = up + ((-up) - up) * v;               // lerp(up, -up, v)
            const V3 to = o + fwd + lr + ud;
            store_ray(rays + 8 * (y * W + x), o, 0.0, normalize(to - o), INFINITY);
        }
}

// Uniform random rays: origin uniform in the box [lo, hi] (lo + (hi - lo) * xi per
// axis), direction uniform on the unit sphere by Archimedes' hat-box theorem (the
// height z = 1 - 2 xi is uniform in [-1, 1], the azimuth 2 pi xi uniform, the radius
// of the circle at height z is sqrt(1 - z^2)). Numbers: ray i's splitmix64 values at
// (sample, dim) = (0,0), (0,1), (1,0) for the origin, (1,1) for z, (2,0) for the azimuth.
void oracle_uniform_rays(const float* lo, const float* hi, uint64_t seed, int64_t n, float tmin, float tmax,
                         float* rays) {
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t p = (uint64_t)i;
        const V3 o = v3(lo[0] + ((double)hi[0] - lo[0]) * oracle_xi(seed, p, 0, 0),
                        lo[1] + ((double)hi[1] - lo[1]) * oracle_xi(seed, p, 0, 1),
                        lo[2] + ((double)hi[2] - lo[2]) * oracle_xi(seed, p, 1, 0));
        const double z = 1.0 - 2.0 * oracle_xi(seed, p, 1, 1);
        const double phi = 2.0 * PI * oracle_xi(seed, p, 2, 0);
        const double r = std::sqrt(std::fmax(1.0 - z * z, 0.0));
        store_ray(rays + 8 * i, o, (double)tmin, v3(r * std::cos(phi), r * std::sin(phi), z), (double)tmax);
    }
}

// Cosine-weighted hemisphere sample (Y up) for one (xi0, xi1).
void oracle_sample_hemisphere(double xi0, double xi1, double* out3) {
    const double phi = xi0 * 2.0 * PI;
    const double r = std::sqrt(xi1);
    out3[0] = std::cos(phi) * r;
    out3[2] = std::sin(phi) * r;
    out3[1] = std::sqrt(std::fmax(1.0 - r * r, 0.0));
}

// AO rays for n primary hits. world_tri: per pixel the hit triangle's world-space
// vertices (9 doubles; see oracle_world_triangle), primary: the pixel's ray (8 floats),
// prim: NONE marks a miss, t: the primary hit distance. Writes spp rays per pixel;
// a missed pixel gets empty rays (direction 0, minT 0, maxT -1).
void oracle_ao_rays(const float* primary, const double* world_tri, const uint32_t* prim, const double* t,
                    int64_t n, int spp, uint64_t seed, float length, float* out) {
    for (int64_t p = 0; p < n; ++p) {
        if (prim[p] == NONE) {
            for (int s = 0; s < spp; ++s) store_ray(out + 8 * (p * spp + s), v3(0, 0, 0), 0.0, v3(0, 0, 0), -1.0);
            continue;
        }
        const float* r = primary + 8 * p;
        const V3 o = v3(r[0], r[1], r[2]), d = v3(r[4], r[5], r[6]);
        const double* w = world_tri + 9 * p;
        const V3 v0 = v3(w[0], w[1], w[2]), v1 = v3(w[3], w[4], w[5]), v2 = v3(w[6], w[7], w[8]);
        V3 n = normalize(cross(v1 - v0, v2 - v0));
        if (dot(n, d) > 0.0) n = -n;
        const V3 tg = normalize(v1 - v0);
        const V3 bt = cross(n, tg);
        const V3 org = (o + d * t[p]) + n * 1e-4;
        for (int s = 0; s < spp; ++s) {
            double h[3];
            oracle_sample_hemisphere(oracle_xi(seed, (uint64_t)p, (uint32_t)s, 0),
                                     oracle_xi(seed, (uint64_t)p, (uint32_t)s, 1), h);
            const V3 dir = tg * h[0] + bt * h[2] + n * h[1];
            store_ray(out + 8 * (p * spp + s), org, 0.0, dir, (double)length);
        }
    }
}

}  // extern "C"
