// bvh.cpp -- binned surface-area-heuristic BVH over the detector triangles.
//
// The paper's Gadep keeps its triangles in a bounding volume hierarchy so that
// a ray query touches only nearby facets (Sec. 2.4.3); tripling the facet count
// costs it only 3.5% in run time (Sec. 3.3).  This builder uses the binned SAH
// of Wald (2007): at every node, 32 centroid bins per axis, split where
//   C = C_trav + (A_L N_L + A_R N_R) / A * C_tri
// is smallest; a leaf is kept when N <= max_leaf and N C_tri is not worse.
// Optionally (split_alpha > 0) spatial splits cut triangle references too.
// The costs, the leaf limit and the split threshold are build options
// (gadep_bvh_opts); C_trav = 1.5 C_tri measured fastest on the coaxial meshes.
// The binary tree is then collapsed into the 64-byte 4-wide node layout
// documented in gadep_internal.h (the four child boxes stored in the parent,
// quantised to 7 bits on the node's own grid, depth-first order) with the
// triangles reordered so that every leaf is one contiguous run of 48-byte
// triangles.  A wide node halves the dependent node steps of a query and gives
// each step four independent box tests; quantising its boxes halves the bytes
// each step loads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "gadep_internal.h"

namespace {

constexpr int kBins = 32;          // centroid bins of the object split
constexpr int kSpatialBins = 32;   // slabs of the spatial split
constexpr int kMaxDepth = 60;
constexpr int32_t kClipAutoTris = 1 << 17;   // AUTO early split clipping: meshes at least this large
constexpr float kClipAutoRatio = 8.0f;

struct AABB {
    float lo[3] = { INFINITY, INFINITY, INFINITY };
    float hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    void grow(const float *p) { for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); } }
    void grow(const AABB &b) { for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); } }
    float area() const
    {
        float d[3];
        for (int k = 0; k < 3; ++k) d[k] = std::max(0.0f, hi[k] - lo[k]);
        return 2.0f * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
    }
    bool valid() const { return lo[0] <= hi[0]; }
    bool nonempty() const { return lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2]; }
    static AABB meet(const AABB &a, const AABB &b)
    {
        AABB r;
        for (int k = 0; k < 3; ++k) { r.lo[k] = std::max(a.lo[k], b.lo[k]); r.hi[k] = std::min(a.hi[k], b.hi[k]); }
        return r;
    }
    static AABB join(const AABB &a, const AABB &b) { AABB r = a; r.grow(b); return r; }
};

// A triangle reference: the box of the part of the triangle it stands for (the
// whole triangle unless a spatial split cut it) and that box's centre.
struct Ref { AABB box; float c[3]; int32_t tri; };

Ref make_ref(const AABB &box, int32_t tri)
{
    Ref r;
    r.box = box;
    for (int k = 0; k < 3; ++k) r.c[k] = 0.5f * (box.lo[k] + box.hi[k]);
    r.tri = tri;
    return r;
}

struct BNode {
    AABB box;
    int32_t child[2] = { -1, -1 };   // build-node indices (inner)
    int32_t start = 0, count = 0;    // leaf range in the leaf-ordered references
    bool leaf() const { return child[0] < 0; }
};

// binary32 bounds of an FP64 interval, rounded outward
float round_down(double x) { float f = (float)x; return (double)f > x ? std::nextafter(f, -INFINITY) : f; }
float round_up(double x) { float f = (float)x; return (double)f < x ? std::nextafter(f, INFINITY) : f; }

// Box of the part of triangle v (FP64 copies of its binary32 vertices) with
// lo <= x_k <= hi: the triangle clipped by the two planes (Sutherland-Hodgman),
// its vertices bounded outward in binary32.  Empty (not nonempty()) when the
// triangle misses the slab.
AABB clip_box(const double v[3][3], int k, double lo, double hi)
{
    double poly[8][3], next[8][3];
    int n = 3;
    std::memcpy(poly, v, sizeof(double) * 9);
    for (int side = 0; side < 2 && n > 0; ++side) {
        const double plane = side == 0 ? lo : hi;
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const double *p = poly[i], *q = poly[(i + 1) % n];
            const double dp = side == 0 ? p[k] - plane : plane - p[k];
            const double dq = side == 0 ? q[k] - plane : plane - q[k];
            if (dp >= 0.0) std::memcpy(next[m++], p, sizeof(double) * 3);
            if ((dp >= 0.0) != (dq >= 0.0)) {
                const double s = dp / (dp - dq);
                for (int c = 0; c < 3; ++c) next[m][c] = p[c] + s * (q[c] - p[c]);
                next[m][k] = plane;
                ++m;
            }
        }
        n = m;
        std::memcpy(poly, next, sizeof(double) * 3 * (size_t)n);
    }
    AABB b;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            b.lo[c] = std::min(b.lo[c], round_down(poly[i][c]));
            b.hi[c] = std::max(b.hi[c], round_up(poly[i][c]));
        }
    return b;
}

// Part of triangle v inside the box [lo, hi] (Sutherland-Hodgman against its six
// planes): up to 9 vertices in `poly`, returns the count (0 if none).
int clip_to_box(const double v[3][3], const double lo[3], const double hi[3], double poly[9][3])
{
    double buf[2][9][3];
    int n = 3;
    std::memcpy(buf[0], v, sizeof(double) * 9);
    int cur = 0;
    for (int k = 0; k < 3 && n > 0; ++k)
        for (int side = 0; side < 2 && n > 0; ++side) {
            const double plane = side == 0 ? lo[k] : hi[k];
            double(*in)[3] = buf[cur];
            double(*out)[3] = buf[cur ^ 1];
            int m = 0;
            for (int i = 0; i < n; ++i) {
                const double *p = in[i], *q = in[(i + 1) % n];
                const double dp = side == 0 ? p[k] - plane : plane - p[k];
                const double dq = side == 0 ? q[k] - plane : plane - q[k];
                if (dp >= 0.0 && m < 9) std::memcpy(out[m++], p, sizeof(double) * 3);
                if ((dp >= 0.0) != (dq >= 0.0) && m < 9) {
                    const double t = dp / (dp - dq);
                    for (int c = 0; c < 3; ++c) out[m][c] = p[c] + t * (q[c] - p[c]);
                    out[m][k] = plane;
                    ++m;
                }
            }
            n = m;
            cur ^= 1;
        }
    std::memcpy(poly, buf[cur], sizeof(double) * 3 * (size_t)n);
    return n;
}

// Early split clipping (Ernst and Greiner 2007).  A sliver at an angle to the
// axes -- the centre-fan triangles of a detector's flat end faces run from the
// axis to the rim -- has a bounding box far larger than itself, and every such
// box near the axis contains the axis: a ray crossing the face there would test
// most of the fan.  Such a triangle is stored as several references instead,
// each bounding the part of the triangle inside one half of the previous piece's
// box (halved across its longest axis), until each piece is tight -- its box,
// seen along the triangle's dominant normal axis, at most `ratio` times the
// piece's own projected area -- or the triangle has `max_pieces` pieces.  The
// pieces of a triangle cover it (boxes rounded outward), so the tree still finds
// every hit; a query may meet the same triangle in two leaves, with the same
// distance both times.
void clip_loose(const double v[3][3], int32_t tri, float ratio, int max_pieces, std::vector<Ref> &out)
{
    const double e1[3] = { v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2] };
    const double e2[3] = { v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2] };
    const double nrm[3] = { e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0] };
    const int kz = (std::fabs(nrm[0]) > std::fabs(nrm[1])) ? (std::fabs(nrm[0]) > std::fabs(nrm[2]) ? 0 : 2)
                                                           : (std::fabs(nrm[1]) > std::fabs(nrm[2]) ? 1 : 2);
    const int kx = (kz + 1) % 3, ky = (kz + 2) % 3;
    struct Piece { double lo[3], hi[3]; AABB box; double looseness; };
    // the part of the triangle in [lo, hi]: its outward-rounded box and how loose
    // that box is around it (box area over polygon area, both projected along kz)
    auto make = [&](const double lo[3], const double hi[3], Piece &pc) -> bool {
        double poly[9][3];
        const int n = clip_to_box(v, lo, hi, poly);
        if (n < 3) return false;
        std::memcpy(pc.lo, lo, sizeof(pc.lo));
        std::memcpy(pc.hi, hi, sizeof(pc.hi));
        double plo[3] = { INFINITY, INFINITY, INFINITY }, phi[3] = { -INFINITY, -INFINITY, -INFINITY };
        double area2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const double *p = poly[i], *q = poly[(i + 1) % n];
            area2 += p[kx] * q[ky] - q[kx] * p[ky];
            for (int c = 0; c < 3; ++c) { plo[c] = std::min(plo[c], p[c]); phi[c] = std::max(phi[c], p[c]); }
        }
        for (int c = 0; c < 3; ++c) { pc.box.lo[c] = round_down(plo[c]); pc.box.hi[c] = round_up(phi[c]); }
        const double box_area = (phi[kx] - plo[kx]) * (phi[ky] - plo[ky]);
        const double a = 0.5 * std::fabs(area2);
        pc.looseness = a > 0.0 ? box_area / a : (box_area > 0.0 ? INFINITY : 1.0);
        return true;
    };
    std::vector<Piece> pieces(1);
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(v[0][c], std::min(v[1][c], v[2][c]));
        hi[c] = std::max(v[0][c], std::max(v[1][c], v[2][c]));
    }
    if (!make(lo, hi, pieces[0])) return;
    // split the loosest piece until all are tight or the budget is spent
    while ((int)pieces.size() < max_pieces) {
        size_t w = 0;
        for (size_t i = 1; i < pieces.size(); ++i)
            if (pieces[i].looseness > pieces[w].looseness) w = i;
        if (!(pieces[w].looseness > ratio)) break;
        const Piece p = pieces[w];
        int ax = 0;
        for (int c = 1; c < 3; ++c)
            if (p.box.hi[c] - p.box.lo[c] > p.box.hi[ax] - p.box.lo[ax]) ax = c;
        const double mid = 0.5 * ((double)p.box.lo[ax] + (double)p.box.hi[ax]);
        double llo[3], lhi[3], rlo[3], rhi[3];
        for (int c = 0; c < 3; ++c) {
            llo[c] = rlo[c] = std::max(p.lo[c], (double)p.box.lo[c]);
            lhi[c] = rhi[c] = std::min(p.hi[c], (double)p.box.hi[c]);
        }
        lhi[ax] = mid;
        rlo[ax] = mid;
        Piece a, b;
        const bool ha = make(llo, lhi, a), hb = make(rlo, rhi, b);
        if (!ha || !hb) { pieces[w].looseness = 0.0; continue; }   // a sliver of a piece: keep it whole
        pieces[w] = a;
        pieces.push_back(b);
    }
    for (const Piece &p : pieces) out.push_back(make_ref(p.box, tri));
}

struct Split {
    float cost = INFINITY;
    int axis = -1, bin = -1;
    float pos = 0.0f;            // spatial: the plane x_axis = pos
    AABB l, r;
    int32_t nl = 0, nr = 0;
};

// Top-down builder.  Object splits partition the references by centroid bin
// (binned SAH, Wald 2007).  Where the two children of the best object split
// overlap by more than alpha times the root's surface area, a spatial split is
// tried too (Stich, Friedrich and Dietrich 2009): the node's box is cut into
// slabs along each axis, every reference is clipped into the slabs it spans,
// and a plane between slabs is costed with the references that cross it counted
// on both sides.  A reference that crosses the chosen plane goes to one side
// whole when that is cheaper ("unsplitting"), else it is cut in two.  The
// number of references is capped at max_dup times the triangles.
struct Builder {
    const float *xyz = nullptr;      // binary32 vertex coordinates of the mesh
    const int32_t *tv = nullptr;     // vertex indices of each mesh triangle
    int max_leaf = 4;
    float c_trav = 1.0f, c_tri = 1.0f, alpha = 0.0f;
    int64_t ref_budget = 0, n_refs = 0;
    float root_area = 0.0f;
    std::vector<BNode> nodes;
    std::vector<Ref> leaf_refs;      // references in leaf order
    int max_depth = 0;

    void verts(int32_t t, double v[3][3]) const
    {
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) v[j][c] = (double)xyz[3 * (size_t)tv[3 * (size_t)t + j] + c];
    }

    Split object_split(const std::vector<Ref> &refs, const AABB &cb, float area) const
    {
        Split best;
        for (int ax = 0; ax < 3; ++ax) {
            const float ext = cb.hi[ax] - cb.lo[ax];
            if (!(ext > 0.0f)) continue;
            AABB bb[kBins];
            int cnt[kBins] = { 0 };
            const float scale = kBins / ext;
            for (const Ref &r : refs) {
                int b = std::min(kBins - 1, (int)((r.c[ax] - cb.lo[ax]) * scale));
                cnt[b]++;
                bb[b].grow(r.box);
            }
            AABB rbox[kBins];
            int rcnt[kBins];
            AABB acc;
            int c = 0;
            for (int b = kBins - 1; b > 0; --b) {
                acc.grow(bb[b]); c += cnt[b];
                rbox[b] = acc;
                rcnt[b] = c;
            }
            AABB lacc;
            int lc = 0;
            for (int b = 1; b < kBins; ++b) {
                lacc.grow(bb[b - 1]); lc += cnt[b - 1];
                if (lc == 0 || rcnt[b] == 0) continue;
                const float cost = c_trav + (lacc.area() * lc + rbox[b].area() * rcnt[b]) / area * c_tri;
                if (cost < best.cost) {
                    best.cost = cost; best.axis = ax; best.bin = b;
                    best.l = lacc; best.r = rbox[b]; best.nl = lc; best.nr = rcnt[b];
                }
            }
        }
        return best;
    }

    Split spatial_split(const std::vector<Ref> &refs, const AABB &box, float area) const
    {
        Split best;
        for (int ax = 0; ax < 3; ++ax) {
            const float lo = box.lo[ax], ext = box.hi[ax] - box.lo[ax];
            if (!(ext > 0.0f)) continue;
            float plane[kSpatialBins + 1];
            for (int i = 0; i <= kSpatialBins; ++i) plane[i] = lo + ext * ((float)i / kSpatialBins);
            plane[kSpatialBins] = box.hi[ax];
            const float scale = kSpatialBins / ext;
            auto bin_of = [&](float x) { return std::max(0, std::min(kSpatialBins - 1, (int)((x - lo) * scale))); };
            AABB bb[kSpatialBins];
            int entry[kSpatialBins] = { 0 }, exit[kSpatialBins] = { 0 };
            for (const Ref &r : refs) {
                const int b0 = bin_of(r.box.lo[ax]), b1 = std::max(b0, bin_of(r.box.hi[ax]));
                entry[b0]++;
                exit[b1]++;
                if (b0 == b1) { bb[b0].grow(r.box); continue; }
                double v[3][3];
                verts(r.tri, v);
                for (int b = b0; b <= b1; ++b) {
                    const AABB part = AABB::meet(clip_box(v, ax, plane[b], plane[b + 1]), r.box);
                    if (part.nonempty()) bb[b].grow(part);
                }
            }
            AABB rbox[kSpatialBins];
            int rcnt[kSpatialBins];
            AABB acc;
            int c = 0;
            for (int b = kSpatialBins - 1; b > 0; --b) {
                acc.grow(bb[b]); c += exit[b];
                rbox[b] = acc;
                rcnt[b] = c;
            }
            AABB lacc;
            int lc = 0;
            for (int b = 1; b < kSpatialBins; ++b) {
                lacc.grow(bb[b - 1]); lc += entry[b - 1];
                if (lc == 0 || rcnt[b] == 0 || !lacc.valid() || !rbox[b].valid()) continue;
                const float cost = c_trav + (lacc.area() * lc + rbox[b].area() * rcnt[b]) / area * c_tri;
                if (cost < best.cost) {
                    best.cost = cost; best.axis = ax; best.bin = b; best.pos = plane[b];
                    best.l = lacc; best.r = rbox[b]; best.nl = lc; best.nr = rcnt[b];
                }
            }
        }
        return best;
    }

    // Partition by a spatial split; false when a side would keep every reference
    // (no progress), in which case L and R are left empty.
    bool spatial_partition(const std::vector<Ref> &refs, const Split &s, std::vector<Ref> &L, std::vector<Ref> &R)
    {
        const int ax = s.axis;
        const float al = s.l.area(), ar = s.r.area();
        int64_t added = 0;
        for (const Ref &r : refs) {
            if (r.box.hi[ax] <= s.pos) { L.push_back(r); continue; }
            if (r.box.lo[ax] >= s.pos) { R.push_back(r); continue; }
            const float c_split = al * s.nl + ar * s.nr;
            const float c_left = AABB::join(s.l, r.box).area() * s.nl + ar * (s.nr - 1);
            const float c_right = al * (s.nl - 1) + AABB::join(s.r, r.box).area() * s.nr;
            if (c_left < c_split && c_left <= c_right) { L.push_back(r); continue; }
            if (c_right < c_split) { R.push_back(r); continue; }
            double v[3][3];
            verts(r.tri, v);
            const AABB a = AABB::meet(clip_box(v, ax, -INFINITY, s.pos), r.box);
            const AABB b = AABB::meet(clip_box(v, ax, s.pos, INFINITY), r.box);
            if (a.nonempty() && b.nonempty()) {
                L.push_back(make_ref(a, r.tri));
                R.push_back(make_ref(b, r.tri));
                ++added;
            } else if (a.nonempty()) {
                L.push_back(r);
            } else {
                R.push_back(r);
            }
        }
        if (L.empty() || R.empty() || L.size() >= refs.size() || R.size() >= refs.size()) {
            L.clear(); R.clear();
            return false;
        }
        n_refs += added;
        return true;
    }

    int32_t build(std::vector<Ref> &refs, int depth)
    {
        max_depth = std::max(max_depth, depth);
        BNode n;
        AABB cb;
        for (const Ref &r : refs) { n.box.grow(r.box); cb.grow(r.c); }
        const int32_t N = (int32_t)refs.size();
        const int32_t id = (int32_t)nodes.size();
        nodes.push_back(n);
        const float area = std::max(n.box.area(), 1e-30f);
        if (depth == 0) root_area = area;
        Split os, ss;
        if (N > 1) {
            os = object_split(refs, cb, area);
            if (alpha > 0.0f && n_refs < ref_budget && depth + 1 < kMaxDepth) {
                const AABB ov = os.axis >= 0 ? AABB::meet(os.l, os.r) : n.box;
                const float lambda = ov.nonempty() ? ov.area() : 0.0f;
                if (lambda > alpha * root_area) ss = spatial_split(refs, n.box, area);
            }
        }
        const float best_cost = std::min(os.cost, ss.cost);
        const float leaf_cost = N * c_tri;
        bool make_leaf = (N <= max_leaf && leaf_cost <= best_cost) || N == 1 || depth >= kMaxDepth;
        if (make_leaf && N > max_leaf && depth < kMaxDepth) make_leaf = false;
        if (make_leaf) {
            // pieces of one clipped triangle that meet in a leaf become one record
            // (the leaf box already bounds all of them)
            nodes[id].start = (int32_t)leaf_refs.size();
            for (const Ref &r : refs) {
                bool dup = false;
                for (size_t i = (size_t)nodes[id].start; i < leaf_refs.size() && !dup; ++i) dup = leaf_refs[i].tri == r.tri;
                if (!dup) leaf_refs.push_back(r);
            }
            nodes[id].count = (int32_t)leaf_refs.size() - nodes[id].start;
            return id;
        }
        std::vector<Ref> L, R;
        bool done = ss.cost < os.cost && spatial_partition(refs, ss, L, R);
        if (!done) {
            auto mid = refs.begin() + N / 2;   // all centroids coincide: split the list
            if (os.axis >= 0) {
                const int ax = os.axis, bin = os.bin;
                const float lo = cb.lo[ax], scale = kBins / (cb.hi[ax] - cb.lo[ax]);
                auto it = std::partition(refs.begin(), refs.end(), [&](const Ref &r) {
                    return std::min(kBins - 1, (int)((r.c[ax] - lo) * scale)) < bin;
                });
                if (it != refs.begin() && it != refs.end()) mid = it;
            }
            L.assign(refs.begin(), mid);
            R.assign(mid, refs.end());
        }
        std::vector<Ref>().swap(refs);
        const int32_t l = build(L, depth + 1);
        const int32_t r = build(R, depth + 1);
        nodes[id].child[0] = l;
        nodes[id].child[1] = r;
        return id;
    }
};

// Leaf reference stored in a child word: ~(first << 3 | count), always negative.
int32_t leaf_ref(int32_t first, int32_t count) { return ~((first << 3) | count); }

void pad_box(const AABB &b, float out_lo[3], float out_hi[3])
{
    for (int k = 0; k < 3; ++k) {
        float m = std::max(std::fabs(b.lo[k]), std::fabs(b.hi[k]));
        float pad = 1e-4f + 4e-6f * m;
        out_lo[k] = b.lo[k] - pad;
        out_hi[k] = b.hi[k] + pad;
    }
}

// Word layout of a quantised node (see gadep_internal.h).
constexpr int kWordS[3] = { 3, 14, 15 };      // S per axis
constexpr int kWordLo[3] = { 8, 10, 12 };     // low-plane bytes per axis; high planes follow
constexpr int kQMax = 127;

// Quantise the padded boxes of a node's n children onto the node's own grid
// and write the node's 16 words: per axis the base b (rounded down so that
// b + S lies at or below every low plane), the grid step s (a power of two,
// the smallest with 127 s spanning the children) and per child the low plane
// rounded down and the high plane rounded up to the grid.  All of it is exact
// in FP64 (floats, powers of two and small integer multiples of them).
void quantise_node(int n, const float lo[4][3], const float hi[4][3], const int32_t child[4],
                   float f[kNodeFloats])
{
    uint32_t u[kNodeFloats] = {};
    for (int k = 0; k < 3; ++k) {
        double p = INFINITY, top = -INFINITY;
        for (int c = 0; c < n; ++c) {
            p = std::min(p, (double)lo[c][k]);
            top = std::max(top, (double)hi[c][k]);
        }
        int e = 0;
        std::frexp((top - p) / kQMax, &e);    // 2^e >= (top - p) / 127
        double s, S, base;
        float b;
        for (;;) {
            s = std::ldexp(1.0, e);
            S = 128.0 * s;
            b = round_down(p - S);
            base = (double)b + S;     // the plane of q = 0
            if (base <= p && top - base <= kQMax * s) break;
            ++e;
        }
        const float Sf = (float)S;
        std::memcpy(&u[k], &b, 4);
        std::memcpy(&u[kWordS[k]], &Sf, 4);
        uint32_t wl = 0, wh = 0;
        for (int c = 0; c < 4; ++c) {
            int ql = kQMax, qh = 0;            // empty slot: inverted box
            if (c < n) {
                ql = (int)std::floor(((double)lo[c][k] - base) / s);
                qh = (int)std::ceil(((double)hi[c][k] - base) / s);
                ql = std::max(0, std::min(ql, kQMax));
                qh = std::max(0, std::min(qh, kQMax));
            }
            wl |= (uint32_t)(128 + ql) << (8 * c);
            wh |= (uint32_t)(128 + qh) << (8 * c);
        }
        u[kWordLo[k]] = wl;
        u[kWordLo[k] + 1] = wh;
    }
    std::memcpy(&u[4], child, 16);
    std::memcpy(f, u, sizeof(u));
}

}  // namespace

namespace gadep {

namespace {

struct TreeStats { int32_t leaves = 0, max_leaf = 0, depth = 0; double sah = 0.0; int64_t refs = 0; };

// Build one BVH over the mesh triangles `ids`; append its nodes and its
// leaf-ordered triangle records to `out` and return the root node index.
int32_t append_tree(const detmesh_mesh *m, const std::vector<int32_t> &ids, const gadep_bvh_opts &o,
                    gadep_bvh *out, TreeStats &ts, gadep_status &st)
{
    const MeshData &g = m->geo;
    const int32_t n_ids = (int32_t)ids.size();
    if (n_ids == 0) return -1;
    Builder B;
    B.xyz = m->xyz_f.data();
    B.tv = g.tri.data();
    B.max_leaf = o.max_leaf;
    B.c_trav = o.c_trav;
    B.c_tri = o.c_tri;
    B.alpha = o.split_alpha;
    std::vector<Ref> refs;
    refs.reserve(n_ids);
    for (int32_t i = 0; i < n_ids; ++i) {
        const int32_t t = ids[i];
        if (o.clip_ratio > 0.0f && o.clip_pieces > 1) {
            double v[3][3];
            B.verts(t, v);
            clip_loose(v, t, o.clip_ratio, o.clip_pieces, refs);
            continue;
        }
        AABB box;
        for (int j = 0; j < 3; ++j) box.grow(&m->xyz_f[3 * g.tri[3 * t + j]]);
        refs.push_back(make_ref(box, t));
    }
    B.n_refs = (int64_t)refs.size();
    B.ref_budget = (int64_t)((double)o.max_dup * (double)refs.size());
    B.nodes.reserve(2 * (size_t)n_ids / o.max_leaf + 8);
    B.build(refs, 0);
    if (B.max_depth >= kMaxDepth) {
        st = fail(GADEP_E_MESH, "bvh: depth limit reached (degenerate mesh?)");
        return -1;
    }
    const int32_t nt = (int32_t)B.leaf_refs.size();
    if ((int64_t)out->tris.size() / 12 + nt >= (1 << 27)) {
        st = fail(GADEP_E_INVAL, "bvh: more than 2^27 triangle records");
        return -1;
    }
    ts.depth = std::max(ts.depth, B.max_depth);
    ts.refs += nt;
    const int32_t tri_base = (int32_t)(out->tris.size() / 12);
    const int32_t node_base = (int32_t)(out->nodes.size() / kNodeFloats);
    // triangles in leaf order: (v0, region), (v1, mesh triangle id), (v2, 0)
    for (int32_t i = 0; i < nt; ++i) {
        const int32_t t = B.leaf_refs[i].tri;
        out->tri_orig.push_back(t);
        float rec[12];
        for (int j = 0; j < 3; ++j) {
            const float *v = &m->xyz_f[3 * g.tri[3 * t + j]];
            rec[4 * j + 0] = v[0]; rec[4 * j + 1] = v[1]; rec[4 * j + 2] = v[2]; rec[4 * j + 3] = 0.0f;
        }
        const int32_t region = g.tri_solid[t] + 1;
        std::memcpy(&rec[3], &region, 4);
        std::memcpy(&rec[7], &t, 4);
        out->tris.insert(out->tris.end(), rec, rec + 12);
    }
    // Collapse into 4-wide nodes: a wide node takes the two children of a binary
    // node and opens its largest-area inner child (replacing it by that child's
    // two children) until it holds four children or only leaves.  Wide nodes are
    // stored depth-first; the root of the tree is always a wide node (a root that
    // is a leaf becomes a wide node with one child).
    auto collapse = [&](int32_t bnode, int32_t kids[4]) -> int {
        const BNode &nb = B.nodes[bnode];
        if (nb.leaf()) { kids[0] = bnode; return 1; }
        int n = 0;
        kids[n++] = nb.child[0];
        kids[n++] = nb.child[1];
        while (n < 4) {
            int open = -1;
            float open_area = -1.0f;
            for (int i = 0; i < n; ++i) {
                const BNode &c = B.nodes[kids[i]];
                if (!c.leaf() && c.box.area() > open_area) { open_area = c.box.area(); open = i; }
            }
            if (open < 0) break;
            const BNode &c = B.nodes[kids[open]];
            kids[open] = c.child[0];
            kids[n++] = c.child[1];
        }
        return n;
    };
    std::vector<int32_t> dev_of(B.nodes.size(), -1);
    std::vector<int32_t> order;   // build ids of the wide nodes, depth-first
    {
        std::vector<int32_t> stack{ 0 };
        while (!stack.empty()) {
            const int32_t bn = stack.back();
            stack.pop_back();
            dev_of[bn] = node_base + (int32_t)order.size();
            order.push_back(bn);
            int32_t kids[4];
            const int n = collapse(bn, kids);
            for (int i = n - 1; i >= 0; --i)
                if (kids[i] != bn && !B.nodes[kids[i]].leaf()) stack.push_back(kids[i]);
        }
    }
    const double root_area = std::max((double)B.nodes[0].box.area(), 1e-30);
    for (const int32_t bn : order) {
        int32_t kids[4];
        const int n = collapse(bn, kids);
        int32_t w[4] = { kEmptyChild, kEmptyChild, kEmptyChild, kEmptyChild };
        float lo[4][3], hi[4][3];
        ts.sah += B.nodes[bn].leaf() ? 0.0 : B.nodes[bn].box.area() / root_area * o.c_trav;
        for (int c = 0; c < n; ++c) {
            const BNode &ch = B.nodes[kids[c]];
            pad_box(ch.box, lo[c], hi[c]);
            if (ch.leaf()) {
                w[c] = leaf_ref(tri_base + ch.start, ch.count);
                ts.leaves++;
                ts.max_leaf = std::max(ts.max_leaf, ch.count);
                ts.sah += ch.box.area() / root_area * ch.count * o.c_tri;
            } else {
                w[c] = dev_of[kids[c]];
            }
        }
        float f[kNodeFloats];
        quantise_node(n, lo, hi, w, f);
        out->nodes.insert(out->nodes.end(), f, f + kNodeFloats);
    }
    return node_base;
}

}  // namespace

// Triangle sets: region r = solid r - 1 (0 = world) gets the triangles of its own
// solid and of the solids whose parent it is -- the only surfaces a photon inside
// r can reach first when solids are closed, nested and disjoint (which the mesh
// validation enforces).  One extra tree holds every triangle, for region-free
// nearest-hit queries.
std::vector<std::vector<int32_t>> region_triangle_sets(const MeshData &g)
{
    std::vector<std::vector<int32_t>> sets((size_t)g.n_solid() + 1);
    for (int32_t t = 0; t < g.n_tri(); ++t) {
        const int32_t s = g.tri_solid[t];
        sets[(size_t)s + 1].push_back(t);
        sets[(size_t)g.solids[s].parent + 1].push_back(t);
    }
    return sets;
}

gadep_status build_bvh_host(const detmesh_mesh *m, const gadep_bvh_opts &o, gadep_bvh *out)
{
    const MeshData &g = m->geo;
    const int32_t nt = g.n_tri();
    if (nt >= (1 << 26)) return fail(GADEP_E_INVAL, "bvh: at most 2^26 triangles");
    if (o.max_leaf < 1 || o.max_leaf > 7 || !(o.c_trav >= 0.0f) || !(o.c_tri > 0.0f) || !(o.split_alpha >= 0.0f) ||
        !(o.max_dup >= 1.0f) || !(o.max_dup <= 16.0f) || !(o.clip_ratio <= 0.0f || o.clip_ratio >= 1.0f) ||
        o.clip_pieces < 1 || o.clip_pieces > 256)
        return fail(GADEP_E_INVAL, "bvh: bad options (max_leaf 1..7, c_tri > 0, c_trav >= 0, split_alpha >= 0, "
                                   "max_dup in [1, 16], clip_ratio <= 0 or >= 1, clip_pieces 1..256)");
    // AUTO clipping (clip_ratio < 0): on for meshes of at least kClipAutoTris
    // triangles.  Measured: the 1,012,288-triangle stress mesh traces 1.7x faster
    // with clip_ratio 8 (its 1024-segment centre fans made 53 triangle tests per
    // query, 19 after clipping); on the 13,824-triangle coax the tree fits in L1
    // and the extra nodes cost as much as the triangle tests they save (1-2 %
    // slower), so small meshes keep one reference per triangle.
    gadep_bvh_opts oo = o;
    if (oo.clip_ratio < 0.0f) oo.clip_ratio = nt >= kClipAutoTris ? kClipAutoRatio : 0.0f;
    out->nodes.clear();
    out->tris.clear();
    out->tri_orig.clear();
    gadep_status st = GADEP_OK;
    TreeStats all_ts, reg_ts;
    std::vector<int32_t> all(nt);
    for (int32_t t = 0; t < nt; ++t) all[t] = t;
    out->root_all = append_tree(m, all, oo, out, all_ts, st);
    if (st != GADEP_OK) return st;
    const auto sets = region_triangle_sets(g);
    std::vector<int32_t> roots(sets.size(), -1);
    for (size_t r = 0; r < sets.size(); ++r) {
        roots[r] = append_tree(m, sets[r], oo, out, reg_ts, st);
        if (st != GADEP_OK) return st;
    }
    // regions: 0 = world, s + 1 = solid s; (material, active | (group + 1) << 1, parent, root)
    out->regions.assign(4 * ((size_t)g.n_solid() + 1), 0);
    out->regions[0] = GADEP_MAT_VACUUM; out->regions[1] = 0; out->regions[2] = 0; out->regions[3] = roots[0];
    for (int32_t s = 0; s < g.n_solid(); ++s) {
        const gadep_solid &so = g.solids[s];
        int32_t *r = &out->regions[4 * ((size_t)s + 1)];
        r[0] = so.material;
        r[1] = (so.active ? 1 : 0) | ((so.group + 1) << 1);
        r[2] = so.parent + 1;
        r[3] = roots[(size_t)s + 1];
    }
    // planes of the stored (binary32) triangles, computed in FP64: the transport
    // takes the distance of the hit it selected from these (see plane_t)
    out->planes.assign(4 * (size_t)nt, 0.0f);
    for (int32_t t = 0; t < nt; ++t) {
        double v[3][3];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) v[k][c] = (double)m->xyz_f[3 * (size_t)g.tri[3 * (size_t)t + k] + c];
        const double e1[3] = { v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2] };
        const double e2[3] = { v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2] };
        double n[3] = { e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0] };
        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) return fail(GADEP_E_MESH, "bvh: degenerate triangle %d", t);
        double w = 0.0;
        for (int c = 0; c < 3; ++c) {
            n[c] /= len;
            w += n[c] * (v[0][c] + v[1][c] + v[2][c]) / 3.0;
        }
        for (int c = 0; c < 3; ++c) out->planes[4 * (size_t)t + c] = (float)n[c];
        out->planes[4 * (size_t)t + 3] = (float)w;
    }
    out->geo = g;
    gadep_bvh_stats &stt = out->stats;
    stt.n_nodes = (int32_t)(out->nodes.size() / kNodeFloats);
    stt.n_leaves = all_ts.leaves + reg_ts.leaves;
    stt.max_depth = std::max(all_ts.depth, reg_ts.depth);
    stt.max_leaf_tris = std::max(all_ts.max_leaf, reg_ts.max_leaf);
    stt.n_tri = nt;
    stt.n_region = g.n_solid() + 1;
    stt.sah_cost = all_ts.sah;
    stt.node_bytes = (int64_t)stt.n_nodes * kNodeFloats * 4;
    stt.tri_bytes = (int64_t)(out->tris.size() / 12) * 48;
    stt.n_refs = all_ts.refs + reg_ts.refs;
    stt.opts = oo;
    return GADEP_OK;
}

}  // namespace gadep

namespace gadep {

void decode_node(const float *f, WideNode &out)
{
    uint32_t u[kNodeFloats];
    std::memcpy(u, f, sizeof(u));
    std::memcpy(out.child, &u[4], 16);
    out.n = 0;
    for (int c = 0; c < 4; ++c) out.n += out.child[c] != kEmptyChild;
    for (int k = 0; k < 3; ++k) {
        float b, S;
        std::memcpy(&b, &u[k], 4);
        std::memcpy(&S, &u[kWordS[k]], 4);
        const double s = (double)S / 128.0, base = (double)b + (double)S;
        for (int c = 0; c < 4; ++c) {
            const int ql = (int)((u[kWordLo[k]] >> (8 * c)) & 0xffu) - 128;
            const int qh = (int)((u[kWordLo[k] + 1] >> (8 * c)) & 0xffu) - 128;
            out.lo[c][k] = base + ql * s;
            out.hi[c][k] = base + qh * s;
        }
    }
}

}  // namespace gadep

extern "C" void gadep_bvh_opts_default(gadep_bvh_opts *o)
{
    if (!o) return;
    o->max_leaf = 4;
    o->c_trav = 1.5f;
    o->c_tri = 1.0f;
    o->split_alpha = 0.0f;
    o->max_dup = 2.0f;
    o->clip_ratio = -1.0f;
    o->clip_pieces = 16;
}

extern "C" gadep_status gadep_bvh_get_stats(const gadep_bvh *b, gadep_bvh_stats *out)
{
    gadep::clear_error();
    if (!b || !out) return gadep::fail(GADEP_E_INVAL, "gadep_bvh_get_stats: NULL argument");
    *out = b->stats;
    return GADEP_OK;
}

namespace {

struct LeafBox { int32_t id, rec; float lo[3], hi[3]; };   // mesh triangle, its record

// Walk one tree: every stored child box non-empty, empty slots empty, no
// triangle twice in one leaf, every leaf's box meeting the bounding box of each
// triangle it holds; append (mesh triangle id, box) for every triangle record,
// the box being the intersection of the leaf's box with those of all its
// ancestors (the region a ray must pass every box test of to reach the leaf).
gadep_status walk_tree(const gadep_bvh *b, int32_t root, std::vector<LeafBox> &out)
{
    const int32_t nn = b->stats.n_nodes;
    const int32_t ns = (int32_t)(b->tris.size() / 12);
    struct Item { int32_t node; double lo[3], hi[3]; };
    std::vector<Item> stack;
    stack.push_back(Item{ root, { -INFINITY, -INFINITY, -INFINITY }, { INFINITY, INFINITY, INFINITY } });
    int64_t visited = 0;
    gadep::WideNode wn;
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        if (it.node < 0 || it.node >= nn || ++visited > nn)
            return gadep::fail(GADEP_E_MESH, "bvh: bad node index %d", it.node);
        gadep::decode_node(&b->nodes[(size_t)it.node * kNodeFloats], wn);
        if (wn.n < 1) return gadep::fail(GADEP_E_MESH, "bvh: node %d has no children", it.node);
        for (int c = 0; c < 4; ++c) {
            const int32_t wc = wn.child[c];
            if (c >= wn.n) {
                bool inverted = true;
                for (int k = 0; k < 3; ++k) inverted = inverted && wn.lo[c][k] > wn.hi[c][k];
                if (wc != kEmptyChild || !inverted)
                    return gadep::fail(GADEP_E_MESH, "bvh: empty slot of node %d is not empty", it.node);
                continue;
            }
            double lo[3], hi[3];
            for (int k = 0; k < 3; ++k) {
                if (wn.lo[c][k] > wn.hi[c][k])
                    return gadep::fail(GADEP_E_MESH, "bvh: child box of node %d is empty", it.node);
                lo[k] = std::max(wn.lo[c][k], it.lo[k]);
                hi[k] = std::min(wn.hi[c][k], it.hi[k]);
                if (lo[k] > hi[k])
                    return gadep::fail(GADEP_E_MESH, "bvh: child box of node %d outside its parent", it.node);
            }
            if (wc >= 0) {
                stack.push_back(Item{ wc, { lo[0], lo[1], lo[2] }, { hi[0], hi[1], hi[2] } });
                continue;
            }
            float flo[3], fhi[3];
            for (int k = 0; k < 3; ++k) { flo[k] = round_down(lo[k]); fhi[k] = round_up(hi[k]); }
            const int32_t first = (~wc) >> 3, cnt = (~wc) & 7;
            if (first < 0 || cnt < 1 || first + cnt > ns) return gadep::fail(GADEP_E_MESH, "bvh: bad leaf range");
            for (int32_t t = first; t < first + cnt; ++t) {
                int32_t id;
                std::memcpy(&id, &b->tris[(size_t)t * 12 + 7], 4);
                if (id != b->tri_orig[t]) return gadep::fail(GADEP_E_MESH, "bvh: triangle id mismatch");
                for (int32_t u = first; u < t; ++u)
                    if (b->tri_orig[u] == id) return gadep::fail(GADEP_E_MESH, "bvh: triangle %d twice in a leaf", id);
                for (int k = 0; k < 3; ++k) {
                    float vlo = INFINITY, vhi = -INFINITY;
                    for (int j = 0; j < 3; ++j) {
                        const float v = b->tris[(size_t)t * 12 + 4 * j + k];
                        vlo = std::min(vlo, v);
                        vhi = std::max(vhi, v);
                    }
                    if (vhi < lo[k] || vlo > hi[k]) return gadep::fail(GADEP_E_MESH, "bvh: leaf box misses its triangle");
                }
                out.push_back(LeafBox{ id, t, { flo[0], flo[1], flo[2] }, { fhi[0], fhi[1], fhi[2] } });
            }
        }
    }
    return GADEP_OK;
}

// Every point of a barycentric grid on one triangle (its vertices included)
// lies in one of the leaf boxes [first, last) that hold the triangle.
bool covered(const gadep_bvh *b, const LeafBox *first, const LeafBox *last)
{
    constexpr int kGrid = 8;
    const float *v[3];
    for (int j = 0; j < 3; ++j) v[j] = &b->tris[(size_t)first->rec * 12 + 4 * j];
    for (int i = 0; i <= kGrid; ++i)
        for (int j = 0; i + j <= kGrid; ++j) {
            const int k = kGrid - i - j;
            float p[3];
            for (int c = 0; c < 3; ++c) {
                if (i == kGrid || j == kGrid || k == kGrid) {
                    p[c] = i == kGrid ? v[0][c] : (j == kGrid ? v[1][c] : v[2][c]);
                } else {
                    p[c] = (float)(((double)i * v[0][c] + (double)j * v[1][c] + (double)k * v[2][c]) / kGrid);
                }
            }
            bool in = false;
            for (const LeafBox *lb = first; lb != last && !in; ++lb)
                in = p[0] >= lb->lo[0] && p[0] <= lb->hi[0] && p[1] >= lb->lo[1] && p[1] <= lb->hi[1] &&
                     p[2] >= lb->lo[2] && p[2] <= lb->hi[2];
            if (!in) return false;
        }
    return true;
}

}  // namespace

extern "C" gadep_status gadep_bvh_validate(const gadep_bvh *b)
{
    gadep::clear_error();
    if (!b) return gadep::fail(GADEP_E_INVAL, "gadep_bvh_validate: NULL bvh");
    const gadep::MeshData &g = b->geo;
    auto sets = gadep::region_triangle_sets(g);
    std::vector<int32_t> all(g.n_tri());
    for (int32_t t = 0; t < g.n_tri(); ++t) all[t] = t;
    sets.push_back(all);
    for (size_t r = 0; r < sets.size(); ++r) {
        const int32_t root = r + 1 < sets.size() ? b->regions[4 * r + 3] : b->root_all;
        std::vector<LeafBox> boxes;
        if (root >= 0) {
            gadep_status st = walk_tree(b, root, boxes);
            if (st != GADEP_OK) return st;
        }
        std::sort(boxes.begin(), boxes.end(), [](const LeafBox &x, const LeafBox &y) { return x.id < y.id; });
        std::vector<int32_t> ids;
        for (const LeafBox &lb : boxes)
            if (ids.empty() || ids.back() != lb.id) ids.push_back(lb.id);
        std::vector<int32_t> want = sets[r];
        std::sort(want.begin(), want.end());
        if (ids != want) return gadep::fail(GADEP_E_MESH, "bvh: tree %zu does not hold each of its triangles", r);
        for (size_t i = 0; i < boxes.size();) {
            size_t j = i;
            while (j < boxes.size() && boxes[j].id == boxes[i].id) ++j;
            if (!covered(b, &boxes[i], &boxes[j]))
                return gadep::fail(GADEP_E_MESH, "bvh: leaf boxes of triangle %d do not cover it", boxes[i].id);
            i = j;
        }
    }
    return GADEP_OK;
}
