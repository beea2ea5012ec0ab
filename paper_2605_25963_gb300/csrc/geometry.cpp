// geometry.cpp -- host-side mesh validation, nesting tree and parity localisation.
//
// Localisation follows the paper's rule (Sec. 2.4.2, Fig. 5): cast a ray from the
// point, count its crossings with every closed solid; an odd count means the
// point is inside that solid; among those, the container is the solid whose
// first crossing is nearest; none means the world.  On the host this is done in
// FP64 with the Moller-Trumbore test; a ray that passes within 1e-9 of a
// triangle edge is discarded and another generic direction is tried, so the
// count is never corrupted by a double-counted edge.
//
// The nesting tree (parent of each solid) is what the GPU uses instead of the
// parity rule at run time: crossing into solid s puts the photon in s, crossing
// out of s puts it in parent(s).  For closed, nested, non-intersecting solids
// both rules give the same region.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <unordered_map>

#include "gadep_internal.h"

namespace gadep {

namespace {
thread_local char g_err[512] = "no error";
}

gadep_status fail(gadep_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

void clear_error() { std::snprintf(g_err, sizeof(g_err), "no error"); }

const char *last_error() { return g_err; }

double solid_volume(const MeshData &m, int32_t s)
{
    double v = 0.0;
    for (int32_t t = 0; t < m.n_tri(); ++t) {
        if (m.tri_solid[t] != s) continue;
        const double *a = &m.xyz[3 * m.tri[3 * t]], *b = &m.xyz[3 * m.tri[3 * t + 1]],
                     *c = &m.xyz[3 * m.tri[3 * t + 2]];
        v += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
             a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    return v / 6.0;
}

int32_t solid_euler(const MeshData &m, int32_t s)
{
    std::unordered_map<uint64_t, int> edges;
    std::unordered_map<int32_t, int> verts;
    int32_t F = 0;
    for (int32_t t = 0; t < m.n_tri(); ++t) {
        if (m.tri_solid[t] != s) continue;
        ++F;
        for (int k = 0; k < 3; ++k) {
            uint32_t a = (uint32_t)m.tri[3 * t + k], b = (uint32_t)m.tri[3 * t + (k + 1) % 3];
            uint64_t key = a < b ? ((uint64_t)a << 32 | b) : ((uint64_t)b << 32 | a);
            edges[key] = 1;
            verts[(int32_t)a] = 1;
        }
    }
    return (int32_t)verts.size() - (int32_t)edges.size() + F;
}

namespace {

struct Box { double lo[3], hi[3]; };

std::vector<Box> solid_boxes(const MeshData &m)
{
    std::vector<Box> b(m.n_solid());
    for (auto &x : b)
        for (int k = 0; k < 3; ++k) { x.lo[k] = INFINITY; x.hi[k] = -INFINITY; }
    for (int32_t t = 0; t < m.n_tri(); ++t) {
        Box &x = b[m.tri_solid[t]];
        for (int j = 0; j < 3; ++j) {
            const double *v = &m.xyz[3 * m.tri[3 * t + j]];
            for (int k = 0; k < 3; ++k) { x.lo[k] = std::min(x.lo[k], v[k]); x.hi[k] = std::max(x.hi[k], v[k]); }
        }
    }
    return b;
}

// Moller-Trumbore in FP64.  Returns 1 for a clean hit (t > 0), 0 for a miss,
// -1 when the ray is too close to an edge or vertex to be counted reliably.
int mt_hit(const double *o, const double *d, const double *a, const double *b, const double *c,
           double *t_out)
{
    const double e1[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
    const double e2[3] = { c[0] - a[0], c[1] - a[1], c[2] - a[2] };
    const double p[3] = { d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0] };
    const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    const double scale = std::sqrt((e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) *
                                   (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
    if (std::fabs(det) <= 1e-12 * scale) return 0;  // ray parallel to the plane
    const double inv = 1.0 / det;
    const double s[3] = { o[0] - a[0], o[1] - a[1], o[2] - a[2] };
    const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
    const double q[3] = { s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0] };
    const double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
    const double t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
    const double eps = 1e-9;
    if (u < -eps || v < -eps || u + v > 1.0 + eps) return 0;
    if (t <= 0.0) return t > -1e-9 ? -1 : 0;
    if (u < eps || v < eps || u + v > 1.0 - eps) return -1;
    *t_out = t;
    return 1;
}

bool ray_box(const double *o, const double *d, const Box &b)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double inv = 1.0 / d[k];
        double a = (b.lo[k] - 1e-9 - o[k]) * inv, c = (b.hi[k] + 1e-9 - o[k]) * inv;
        if (a > c) std::swap(a, c);
        t0 = std::max(t0, a);
        t1 = std::min(t1, c);
        if (t0 > t1) return false;
    }
    return true;
}

// Crossing count and nearest crossing of the ray with one solid; false if ambiguous.
bool count_solid(const MeshData &m, const std::vector<int32_t> &tris, const double *o,
                 const double *d, int *count, double *first)
{
    *count = 0;
    *first = INFINITY;
    for (int32_t t : tris) {
        double th;
        int r = mt_hit(o, d, &m.xyz[3 * m.tri[3 * t]], &m.xyz[3 * m.tri[3 * t + 1]],
                       &m.xyz[3 * m.tri[3 * t + 2]], &th);
        if (r < 0) return false;
        if (r == 1) { ++*count; *first = std::min(*first, th); }
    }
    return true;
}

const double kDirs[8][3] = {
    { 0.5773502, 0.5773603, 0.5773402 },  { -0.3141592, 0.2718281, 0.9098765 },
    { 0.8017837, -0.5345225, 0.2672612 }, { -0.1234567, -0.9876543, 0.0962401 },
    { 0.0731, 0.6154, -0.7848 },          { -0.7001, 0.1003, -0.7069 },
    { 0.3320, -0.3321, 0.8826 },          { 0.9129, 0.3651, 0.1826 },
};

std::vector<std::vector<int32_t>> tris_by_solid(const MeshData &m)
{
    std::vector<std::vector<int32_t>> out(m.n_solid());
    for (int32_t t = 0; t < m.n_tri(); ++t) out[m.tri_solid[t]].push_back(t);
    return out;
}

// Parity rule with precomputed per-solid data.  -2: every direction was ambiguous.
int32_t locate_with(const MeshData &m, const std::vector<std::vector<int32_t>> &by,
                    const std::vector<Box> &boxes, const double p[3])
{
    for (const auto &dd : kDirs) {
        double n = std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        const double d[3] = { dd[0] / n, dd[1] / n, dd[2] / n };
        bool ok = true;
        int32_t best = -1;
        double best_t = INFINITY;
        for (int32_t s = 0; s < m.n_solid() && ok; ++s) {
            if (!ray_box(p, d, boxes[s])) continue;
            int c;
            double f;
            if (!count_solid(m, by[s], p, d, &c, &f)) { ok = false; break; }
            if ((c & 1) && f < best_t) { best_t = f; best = s; }
        }
        if (ok) return best;
    }
    return -2;
}

}  // namespace

int32_t locate_point(const MeshData &m, const double p[3])
{
    return locate_with(m, tris_by_solid(m), solid_boxes(m), p);
}

int32_t locate_point_fixed(const MeshData &m, const double p[3])
{
    // The same parity rule with per-solid counters in fixed arrays: one pass over
    // every triangle per trial direction, no heap memory.
    constexpr int kMax = kLocateMaxSolids;
    if (m.n_solid() > kMax) return -3;
    for (const auto &dd : kDirs) {
        const double n = std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        const double d[3] = { dd[0] / n, dd[1] / n, dd[2] / n };
        int count[kMax] = { 0 };
        double first[kMax];
        for (int s = 0; s < kMax; ++s) first[s] = INFINITY;
        bool ok = true;
        for (int32_t t = 0; t < m.n_tri() && ok; ++t) {
            double th;
            const int r = mt_hit(p, d, &m.xyz[3 * m.tri[3 * t]], &m.xyz[3 * m.tri[3 * t + 1]],
                                 &m.xyz[3 * m.tri[3 * t + 2]], &th);
            if (r < 0) ok = false;
            else if (r == 1) {
                const int32_t s = m.tri_solid[t];
                count[s]++;
                first[s] = std::min(first[s], th);
            }
        }
        if (!ok) continue;
        int32_t best = -1;
        double best_t = INFINITY;
        for (int32_t s = 0; s < m.n_solid(); ++s)
            if ((count[s] & 1) && first[s] < best_t) { best_t = first[s]; best = s; }
        return best;
    }
    return -2;
}

gadep_status validate_and_nest(MeshData &m)
{
    const int32_t ns = m.n_solid();
    if (ns < 1 || m.n_tri() < 4) return fail(GADEP_E_MESH, "mesh: no solids");
    auto by = tris_by_solid(m);
    for (int32_t s = 0; s < ns; ++s) {
        if (by[s].size() < 4) return fail(GADEP_E_MESH, "mesh: solid %d has fewer than 4 triangles", s);
        // closed 2-manifold, consistently oriented: every directed edge once, its reverse once
        std::unordered_map<uint64_t, int> dir_edges;
        dir_edges.reserve(by[s].size() * 3);
        for (int32_t t : by[s]) {
            for (int k = 0; k < 3; ++k) {
                uint32_t a = (uint32_t)m.tri[3 * t + k], b = (uint32_t)m.tri[3 * t + (k + 1) % 3];
                if (a == b) return fail(GADEP_E_MESH, "mesh: degenerate triangle %d", t);
                if (++dir_edges[(uint64_t)a << 32 | b] > 1)
                    return fail(GADEP_E_MESH, "mesh: solid %d is not 2-manifold (edge %u-%u repeated)", s, a, b);
            }
        }
        for (const auto &e : dir_edges) {
            uint64_t rev = (e.first << 32) | (e.first >> 32);
            if (!dir_edges.count(rev))
                return fail(GADEP_E_MESH, "mesh: solid %d is not closed or not consistently oriented", s);
        }
        if (!(solid_volume(m, s) > 0.0))
            return fail(GADEP_E_MESH, "mesh: solid %d has non-positive volume (inward normals)", s);
    }
    // nesting by the parity rule at sample vertices of each solid
    auto boxes = solid_boxes(m);
    std::vector<double> vol(ns);
    for (int32_t s = 0; s < ns; ++s) vol[s] = solid_volume(m, s);
    for (int32_t s = 0; s < ns; ++s) {
        // sample vertices spread over the solid's triangle list
        std::vector<int32_t> samples;
        const size_t nt = by[s].size();
        for (int k = 0; k < 5; ++k) samples.push_back(m.tri[3 * by[s][(nt - 1) * k / 4] + (k % 3)]);
        int32_t parent = -1;
        for (int32_t t = 0; t < ns; ++t) {
            if (t == s) continue;
            int inside = -1;
            for (int32_t v : samples) {
                const double *p = &m.xyz[3 * v];
                int here = 0;
                bool in_box = true;
                for (int k = 0; k < 3; ++k) in_box = in_box && p[k] >= boxes[t].lo[k] && p[k] <= boxes[t].hi[k];
                if (in_box) {
                    bool decided = false;
                    for (const auto &dd : kDirs) {
                        double n = std::sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
                        const double d[3] = { dd[0] / n, dd[1] / n, dd[2] / n };
                        int c;
                        double f;
                        if (count_solid(m, by[t], p, d, &c, &f)) { here = c & 1; decided = true; break; }
                    }
                    if (!decided) return fail(GADEP_E_MESH, "mesh: a vertex of solid %d lies on solid %d", s, t);
                }
                if (inside == -1) inside = here;
                else if (inside != here)
                    return fail(GADEP_E_MESH, "mesh: solids %d and %d intersect", s, t);
            }
            if (inside == 1) {
                if (!(vol[t] > vol[s])) return fail(GADEP_E_MESH, "mesh: solids %d and %d overlap", s, t);
                if (parent < 0 || vol[t] < vol[parent]) parent = t;
            }
        }
        m.solids[s].parent = parent;
    }
    return GADEP_OK;
}

}  // namespace gadep

extern "C" const char *gadep_last_error(void) { return gadep::last_error(); }
extern "C" int32_t gadep_abi_version(void) { return 2; }
