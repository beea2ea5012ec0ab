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

gadep_status build_bvh_host(const detmesh_mesh *m, gadep_bvh *out)
{
    const MeshData &g = m->geo;
    const int32_t nt = g.n_tri();
    Builder B;
    B.refs.resize(nt);
    for (int32_t t = 0; t < nt; ++t) {
        Ref &r = B.refs[t];
        for (int j = 0; j < 3; ++j) r.box.grow(&m->xyz_f[3 * g.tri[3 * t + j]]);
        for (int k = 0; k < 3; ++k) r.c[k] = 0.5f * (r.box.lo[k] + r.box.hi[k]);
        r.tri = t;
    }
    B.nodes.reserve(2 * (size_t)nt / kMaxLeaf + 8);
    B.build(0, nt, 0);
    if (B.max_depth >= kMaxDepth)
        return fail(GADEP_E_MESH, "bvh: depth limit reached (degenerate mesh?)");

    // triangles in leaf order
    out->tris.assign((size_t)nt * 12, 0.0f);
    out->tri_orig.resize(nt);
    for (int32_t i = 0; i < nt; ++i) {
        const int32_t t = B.refs[i].tri;
        out->tri_orig[i] = t;
        for (int j = 0; j < 3; ++j) {
            const float *v = &m->xyz_f[3 * g.tri[3 * t + j]];
            float *dst = &out->tris[(size_t)i * 12 + 4 * j];
            dst[0] = v[0]; dst[1] = v[1]; dst[2] = v[2]; dst[3] = 0.0f;
        }
        int32_t region = g.tri_solid[t] + 1;
        std::memcpy(&out->tris[(size_t)i * 12 + 3], &region, 4);
    }

    // compaction: one device node per inner build node (root always a device node)
    std::vector<int32_t> dev_of(B.nodes.size(), -1);
    std::vector<int32_t> order;   // build ids of device nodes, depth-first
    {
        std::vector<int32_t> stack{ 0 };
        while (!stack.empty()) {
            int32_t b = stack.back();
            stack.pop_back();
            dev_of[b] = (int32_t)order.size();
            order.push_back(b);
            const BNode &n = B.nodes[b];
            if (n.leaf()) continue;
            if (!B.nodes[n.child[1]].leaf()) stack.push_back(n.child[1]);
            if (!B.nodes[n.child[0]].leaf()) stack.push_back(n.child[0]);
        }
    }
    out->nodes.assign(order.size() * 16, 0.0f);
    int32_t n_leaves = 0, max_leaf = 0;
    double sah = 0.0;
    const double root_area = std::max((double)B.nodes[0].box.area(), 1e-30);
    for (size_t di = 0; di < order.size(); ++di) {
        const BNode &n = B.nodes[order[di]];
        float lo[2][3], hi[2][3];
        int32_t child[2], count[2];
        if (n.leaf()) {
            // the root is a single leaf: slot 0 holds it, slot 1 is empty
            pad_box(n.box, lo[0], hi[0]);
            child[0] = ~n.start; count[0] = n.count;
            for (int k = 0; k < 3; ++k) { lo[1][k] = 1.0f; hi[1][k] = -1.0f; }
            child[1] = -1; count[1] = 0;
            n_leaves++; max_leaf = std::max(max_leaf, n.count);
            sah += n.box.area() / root_area * n.count * kCTri;
        } else {
            sah += n.box.area() / root_area * kCTrav;
            for (int c = 0; c < 2; ++c) {
                const BNode &ch = B.nodes[n.child[c]];
                pad_box(ch.box, lo[c], hi[c]);
                if (ch.leaf()) {
                    child[c] = ~ch.start; count[c] = ch.count;
                    n_leaves++; max_leaf = std::max(max_leaf, ch.count);
                    sah += ch.box.area() / root_area * ch.count * kCTri;
                } else {
                    child[c] = dev_of[n.child[c]]; count[c] = 0;
                }
            }
        }
        float *f = &out->nodes[di * 16];
        f[0] = lo[0][0]; f[1] = hi[0][0]; f[2] = lo[0][1]; f[3] = hi[0][1];
        f[4] = lo[1][0]; f[5] = hi[1][0]; f[6] = lo[1][1]; f[7] = hi[1][1];
        f[8] = lo[0][2]; f[9] = hi[0][2]; f[10] = lo[1][2]; f[11] = hi[1][2];
        int32_t w[4] = { child[0], child[1], count[0], count[1] };
        std::memcpy(&f[12], w, 16);
    }

    // regions: 0 = world, s + 1 = solid s
    out->regions.assign(4 * ((size_t)g.n_solid() + 1), 0);
    out->regions[0] = GADEP_MAT_VACUUM; out->regions[1] = 0; out->regions[2] = -1; out->regions[3] = 0;
    for (int32_t s = 0; s < g.n_solid(); ++s) {
        const gadep_solid &so = g.solids[s];
        int32_t *r = &out->regions[4 * ((size_t)s + 1)];
        r[0] = so.material; r[1] = so.active; r[2] = so.group; r[3] = so.parent + 1;
    }
    out->geo = g;
    gadep_bvh_stats &st = out->stats;
    st.n_nodes = (int32_t)order.size();
    st.n_leaves = n_leaves;
    st.max_depth = B.max_depth;
    st.max_leaf_tris = max_leaf;
    st.n_tri = nt;
    st.n_region = g.n_solid() + 1;
    st.sah_cost = sah;
    st.node_bytes = (int64_t)order.size() * 64;
    st.tri_bytes = (int64_t)nt * 48;
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

extern "C" gadep_status gadep_bvh_validate(const gadep_bvh *b)
{
    gadep::clear_error();
    if (!b) return gadep::fail(GADEP_E_INVAL, "gadep_bvh_validate: NULL bvh");
    const int32_t nn = b->stats.n_nodes, nt = b->stats.n_tri;
    std::vector<int> seen(nt, 0);
    // walk from the root carrying the box the parent stores for each node
    struct Item { int32_t node; float lo[3], hi[3]; };
    std::vector<Item> stack;
    Item root{ 0, { -INFINITY, -INFINITY, -INFINITY }, { INFINITY, INFINITY, INFINITY } };
    stack.push_back(root);
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
            if (w[c] < 0 && w[2 + c] == 0) continue;  // empty slot
            for (int k = 0; k < 3; ++k)
                if (lo[k] < it.lo[k] || hi[k] > it.hi[k] || lo[k] > hi[k])
                    return gadep::fail(GADEP_E_MESH, "bvh: child box of node %d not inside its parent", it.node);
            if (w[c] >= 0) {
                Item ch{ w[c], { lo[0], lo[1], lo[2] }, { hi[0], hi[1], hi[2] } };
                stack.push_back(ch);
            } else {
                const int32_t first = ~w[c], cnt = w[2 + c];
                if (first < 0 || cnt < 1 || first + cnt > nt)
                    return gadep::fail(GADEP_E_MESH, "bvh: bad leaf range");
                for (int32_t t = first; t < first + cnt; ++t) {
                    seen[t]++;
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
    for (int32_t t = 0; t < nt; ++t)
        if (seen[t] != 1) return gadep::fail(GADEP_E_MESH, "bvh: triangle %d in %d leaves", t, seen[t]);
    return GADEP_OK;
}
