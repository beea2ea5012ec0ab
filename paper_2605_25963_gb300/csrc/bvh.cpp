// bvh.cpp -- binned surface-area-heuristic BVH over the detector triangles.
//
// The paper's Gadep keeps its triangles in a bounding volume hierarchy so that
// a ray query touches only nearby facets (Sec. 2.4.3); tripling the facet count
// costs it only 3.5% in run time (Sec. 3.3).  This builder uses the binned SAH
// of Wald (2007): at every node, 32 centroid bins per axis, split where
//   C = C_trav + (A_L N_L + A_R N_R) / A * C_tri
// is smallest; a leaf is kept when N <= max_leaf and N C_tri is not worse.
// The tree is then compacted into the 64-byte two-child node layout documented
// in gadep_internal.h (both child boxes stored in the parent, depth-first order,
// the left child of an inner node right after it) with the triangles reordered
// so that every leaf is one contiguous run of 48-byte triangles.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "gadep_internal.h"

namespace {

constexpr int kBins = 32;
constexpr float kCTrav = 1.0f, kCTri = 1.0f;
constexpr int kMaxLeaf = 4;
constexpr int kMaxDepth = 60;

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
};

struct Ref { AABB box; float c[3]; int32_t tri; };

struct BNode {
    AABB box;
    int32_t child[2] = { -1, -1 };   // build-node indices (inner)
    int32_t start = 0, count = 0;    // leaf range in refs
    bool leaf() const { return child[0] < 0; }
};

struct Builder {
    std::vector<Ref> refs;
    std::vector<BNode> nodes;
    int max_depth = 0;

    int32_t build(int32_t start, int32_t end, int depth)
    {
        max_depth = std::max(max_depth, depth);
        BNode n;
        AABB cb;
        for (int32_t i = start; i < end; ++i) { n.box.grow(refs[i].box); cb.grow(refs[i].c); }
        const int32_t N = end - start;
        const int32_t id = (int32_t)nodes.size();
        nodes.push_back(n);
        float best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        const float parent_area = std::max(n.box.area(), 1e-30f);
        if (N > 1) {
            for (int ax = 0; ax < 3; ++ax) {
                const float ext = cb.hi[ax] - cb.lo[ax];
                if (!(ext > 0.0f)) continue;
                AABB bb[kBins];
                int cnt[kBins] = { 0 };
                const float scale = kBins / ext;
                for (int32_t i = start; i < end; ++i) {
                    int b = std::min(kBins - 1, (int)((refs[i].c[ax] - cb.lo[ax]) * scale));
                    cnt[b]++;
                    bb[b].grow(refs[i].box);
                }
                float right_area[kBins];
                int right_cnt[kBins];
                AABB acc;
                int c = 0;
                for (int b = kBins - 1; b > 0; --b) {
                    acc.grow(bb[b]); c += cnt[b];
                    right_area[b] = acc.valid() ? acc.area() : 0.0f;
                    right_cnt[b] = c;
                }
                AABB lacc;
                int lc = 0;
                for (int b = 1; b < kBins; ++b) {
                    lacc.grow(bb[b - 1]); lc += cnt[b - 1];
                    if (lc == 0 || right_cnt[b] == 0) continue;
                    float cost = kCTrav + (lacc.area() * lc + right_area[b] * right_cnt[b]) / parent_area * kCTri;
                    if (cost < best_cost) { best_cost = cost; best_axis = ax; best_bin = b; }
                }
            }
        }
        const float leaf_cost = N * kCTri;
        bool make_leaf = (N <= kMaxLeaf && leaf_cost <= best_cost) || N == 1 || depth >= kMaxDepth;
        if (make_leaf && N > kMaxLeaf && depth < kMaxDepth) make_leaf = false;
        if (make_leaf) {
            nodes[id].start = start;
            nodes[id].count = N;
            return id;
        }
        int32_t mid;
        if (best_axis >= 0) {
            const float ext = cb.hi[best_axis] - cb.lo[best_axis];
            const float scale = kBins / ext;
            const int ax = best_axis, bin = best_bin;
            const float lo = cb.lo[ax];
            auto it = std::partition(refs.begin() + start, refs.begin() + end, [&](const Ref &r) {
                return std::min(kBins - 1, (int)((r.c[ax] - lo) * scale)) < bin;
            });
            mid = (int32_t)(it - refs.begin());
        } else {
            mid = start + N / 2;  // all centroids coincide: split the list
        }
        if (mid == start || mid == end) mid = start + N / 2;
        int32_t l = build(start, mid, depth + 1);
        int32_t r = build(mid, end, depth + 1);
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

}  // namespace

namespace gadep {

namespace {

struct TreeStats { int32_t leaves = 0, max_leaf = 0, depth = 0; double sah = 0.0; };

// Build one BVH over the mesh triangles `ids`; append its nodes and its
// leaf-ordered triangles to `out` and return the root node index.
int32_t append_tree(const detmesh_mesh *m, const std::vector<int32_t> &ids, gadep_bvh *out, TreeStats &ts,
                    gadep_status &st)
{
    const MeshData &g = m->geo;
    const int32_t nt = (int32_t)ids.size();
    if (nt == 0) return -1;
    Builder B;
    B.refs.resize(nt);
    for (int32_t i = 0; i < nt; ++i) {
        Ref &r = B.refs[i];
        const int32_t t = ids[i];
        for (int j = 0; j < 3; ++j) r.box.grow(&m->xyz_f[3 * g.tri[3 * t + j]]);
        for (int k = 0; k < 3; ++k) r.c[k] = 0.5f * (r.box.lo[k] + r.box.hi[k]);
        r.tri = t;
    }
    B.nodes.reserve(2 * (size_t)nt / kMaxLeaf + 8);
    B.build(0, nt, 0);
    if (B.max_depth >= kMaxDepth) {
        st = fail(GADEP_E_MESH, "bvh: depth limit reached (degenerate mesh?)");
        return -1;
    }
    ts.depth = std::max(ts.depth, B.max_depth);
    const int32_t tri_base = (int32_t)(out->tris.size() / 12);
    const int32_t node_base = (int32_t)(out->nodes.size() / 16);
    // triangles in leaf order: (v0, region), (v1, mesh triangle id), (v2, 0)
    for (int32_t i = 0; i < nt; ++i) {
        const int32_t t = B.refs[i].tri;
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
    // compaction: one device node per inner build node (root always a device node)
    std::vector<int32_t> dev_of(B.nodes.size(), -1);
    std::vector<int32_t> order;   // build ids of device nodes, depth-first
    {
        std::vector<int32_t> stack{ 0 };
        while (!stack.empty()) {
            int32_t b = stack.back();
            stack.pop_back();
            dev_of[b] = node_base + (int32_t)order.size();
            order.push_back(b);
            const BNode &n = B.nodes[b];
            if (n.leaf()) continue;
            if (!B.nodes[n.child[1]].leaf()) stack.push_back(n.child[1]);
            if (!B.nodes[n.child[0]].leaf()) stack.push_back(n.child[0]);
        }
    }
    const double root_area = std::max((double)B.nodes[0].box.area(), 1e-30);
    for (size_t di = 0; di < order.size(); ++di) {
        const BNode &n = B.nodes[order[di]];
        float lo[2][3], hi[2][3];
        int32_t child[2];
        if (n.leaf()) {
            // the root is a single leaf: slot 0 holds it, slot 1 is empty
            pad_box(n.box, lo[0], hi[0]);
            child[0] = leaf_ref(tri_base + n.start, n.count);
            for (int k = 0; k < 3; ++k) { lo[1][k] = 1.0f; hi[1][k] = -1.0f; }
            child[1] = leaf_ref(0, 0);
            ts.leaves++; ts.max_leaf = std::max(ts.max_leaf, n.count);
            ts.sah += n.box.area() / root_area * n.count * kCTri;
        } else {
            ts.sah += n.box.area() / root_area * kCTrav;
            for (int c = 0; c < 2; ++c) {
                const BNode &ch = B.nodes[n.child[c]];
                pad_box(ch.box, lo[c], hi[c]);
                if (ch.leaf()) {
                    child[c] = leaf_ref(tri_base + ch.start, ch.count);
                    ts.leaves++; ts.max_leaf = std::max(ts.max_leaf, ch.count);
                    ts.sah += ch.box.area() / root_area * ch.count * kCTri;
                } else {
                    child[c] = dev_of[n.child[c]];
                }
            }
        }
        float f[16];
        f[0] = lo[0][0]; f[1] = hi[0][0]; f[2] = lo[0][1]; f[3] = hi[0][1];
        f[4] = lo[1][0]; f[5] = hi[1][0]; f[6] = lo[1][1]; f[7] = hi[1][1];
        f[8] = lo[0][2]; f[9] = hi[0][2]; f[10] = lo[1][2]; f[11] = hi[1][2];
        const int32_t w[4] = { child[0], child[1], 0, 0 };
        std::memcpy(&f[12], w, 16);
        out->nodes.insert(out->nodes.end(), f, f + 16);
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

gadep_status build_bvh_host(const detmesh_mesh *m, gadep_bvh *out)
{
    const MeshData &g = m->geo;
    const int32_t nt = g.n_tri();
    if (nt >= (1 << 26)) return fail(GADEP_E_INVAL, "bvh: at most 2^26 triangles");
    out->nodes.clear();
    out->tris.clear();
    out->tri_orig.clear();
    gadep_status st = GADEP_OK;
    TreeStats all_ts, reg_ts;
    std::vector<int32_t> all(nt);
    for (int32_t t = 0; t < nt; ++t) all[t] = t;
    out->root_all = append_tree(m, all, out, all_ts, st);
    if (st != GADEP_OK) return st;
    const auto sets = region_triangle_sets(g);
    std::vector<int32_t> roots(sets.size(), -1);
    for (size_t r = 0; r < sets.size(); ++r) {
        roots[r] = append_tree(m, sets[r], out, reg_ts, st);
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
    stt.n_nodes = (int32_t)(out->nodes.size() / 16);
    stt.n_leaves = all_ts.leaves + reg_ts.leaves;
    stt.max_depth = std::max(all_ts.depth, reg_ts.depth);
    stt.max_leaf_tris = std::max(all_ts.max_leaf, reg_ts.max_leaf);
    stt.n_tri = nt;
    stt.n_region = g.n_solid() + 1;
    stt.sah_cost = all_ts.sah;
    stt.node_bytes = (int64_t)stt.n_nodes * 64;
    stt.tri_bytes = (int64_t)(out->tris.size() / 12) * 48;
    return GADEP_OK;
}

}  // namespace gadep

extern "C" gadep_status gadep_bvh_get_stats(const gadep_bvh *b, gadep_bvh_stats *out)
{
    gadep::clear_error();
    if (!b || !out) return gadep::fail(GADEP_E_INVAL, "gadep_bvh_get_stats: NULL argument");
    *out = b->stats;
    return GADEP_OK;
}

namespace {

// Walk one tree: child boxes inside the box the parent stores, leaf boxes contain
// their triangles; return the multiset of mesh triangle ids in its leaves.
gadep_status walk_tree(const gadep_bvh *b, int32_t root, std::vector<int32_t> &ids)
{
    const int32_t nn = b->stats.n_nodes;
    const int32_t ns = (int32_t)(b->tris.size() / 12);
    struct Item { int32_t node; float lo[3], hi[3]; };
    std::vector<Item> stack;
    stack.push_back(Item{ root, { -INFINITY, -INFINITY, -INFINITY }, { INFINITY, INFINITY, INFINITY } });
    int64_t visited = 0;
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        if (it.node < 0 || it.node >= nn || ++visited > nn)
            return gadep::fail(GADEP_E_MESH, "bvh: bad node index %d", it.node);
        const float *f = &b->nodes[(size_t)it.node * 16];
        int32_t w[4];
        std::memcpy(w, &f[12], 16);
        for (int c = 0; c < 2; ++c) {
            const float lo[3] = { f[4 * c + 0], f[4 * c + 2], f[8 + 2 * c] };
            const float hi[3] = { f[4 * c + 1], f[4 * c + 3], f[9 + 2 * c] };
            if (w[c] < 0 && ((~w[c]) & 7) == 0) continue;  // empty leaf slot
            for (int k = 0; k < 3; ++k)
                if (lo[k] < it.lo[k] || hi[k] > it.hi[k] || lo[k] > hi[k])
                    return gadep::fail(GADEP_E_MESH, "bvh: child box of node %d not inside its parent", it.node);
            if (w[c] >= 0) {
                stack.push_back(Item{ w[c], { lo[0], lo[1], lo[2] }, { hi[0], hi[1], hi[2] } });
            } else {
                const int32_t first = (~w[c]) >> 3, cnt = (~w[c]) & 7;
                if (first < 0 || cnt < 1 || first + cnt > ns) return gadep::fail(GADEP_E_MESH, "bvh: bad leaf range");
                for (int32_t t = first; t < first + cnt; ++t) {
                    int32_t id;
                    std::memcpy(&id, &b->tris[(size_t)t * 12 + 7], 4);
                    if (id != b->tri_orig[t]) return gadep::fail(GADEP_E_MESH, "bvh: triangle id mismatch");
                    ids.push_back(id);
                    for (int j = 0; j < 3; ++j)
                        for (int k = 0; k < 3; ++k) {
                            const float v = b->tris[(size_t)t * 12 + 4 * j + k];
                            if (v < lo[k] || v > hi[k])
                                return gadep::fail(GADEP_E_MESH, "bvh: triangle outside its leaf box");
                        }
                }
            }
        }
    }
    return GADEP_OK;
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
        std::vector<int32_t> ids;
        if (root >= 0) {
            gadep_status st = walk_tree(b, root, ids);
            if (st != GADEP_OK) return st;
        }
        std::sort(ids.begin(), ids.end());
        std::vector<int32_t> want = sets[r];
        std::sort(want.begin(), want.end());
        if (ids != want) return gadep::fail(GADEP_E_MESH, "bvh: tree %zu does not hold each of its triangles once", r);
    }
    return GADEP_OK;
}
