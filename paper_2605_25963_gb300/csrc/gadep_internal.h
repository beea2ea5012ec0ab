// gadep_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "gadep.h"

namespace gadep {

struct WavefrontBuffers;

// Error reporting: every failing C-ABI call records a thread-local message.
gadep_status fail(gadep_status s, const char *fmt, ...);
void clear_error();

// Geometry of a closed, region-labelled triangle soup, FP64 on the host.
struct MeshData {
    std::vector<double> xyz;          // [n_vert][3]
    std::vector<int32_t> tri;         // [n_tri][3]
    std::vector<int32_t> tri_solid;   // [n_tri]
    std::vector<gadep_solid> solids;  // [n_solid]
    int32_t n_vert() const { return (int32_t)(xyz.size() / 3); }
    int32_t n_tri() const { return (int32_t)tri_solid.size(); }
    int32_t n_solid() const { return (int32_t)solids.size(); }
};

// Parity rule of Sec. 2.4.2 on the host: innermost solid with an odd number of
// crossings along a generic ray from p; -1 = world.  Returns -2 when every
// trial ray grazed an edge (cannot happen for points off the surfaces).
int32_t locate_point(const MeshData &m, const double p[3]);
// Same rule without heap memory, for meshes of at most kLocateMaxSolids solids
// (-3 when there are more).
constexpr int kLocateMaxSolids = 63;
int32_t locate_point_fixed(const MeshData &m, const double p[3]);
double solid_volume(const MeshData &m, int32_t s);
int32_t solid_euler(const MeshData &m, int32_t s);
// Validate closedness/orientation and derive the nesting tree (solids[].parent).
gadep_status validate_and_nest(MeshData &m);

}  // namespace gadep

struct detmesh_mesh {
    gadep::MeshData geo;
    std::vector<float> xyz_f;  // FP32 copy handed to the BVH and to callers
};

// Device-side compacted BVH of 4-wide nodes with quantised child boxes (after
// Ylitie, Karras and Laine, HPG 2017).  Node = 4 x 16 bytes (64 B, half an L1
// line), the boxes of the four children stored in the parent on a grid of the
// node's own:
//   f4[0] = (b.x, b.y, b.z, S.x)        i4[1] = (child0, child1, child2, child3)
//   u4[2] = (lo.x, hi.x, lo.y, hi.y)    u4[3] = (lo.z, hi.z, S.y, S.z)
// A plane word holds one byte per child, 128 + q with q in [0, 127]; the plane
// it stands for is b + S (1 + q / 128) on that axis, where S = 128 s is a power
// of two and s the grid step.  Low planes are rounded down and high planes up
// from the padded child box, so the quantised box contains it.  child >= 0:
// inner node index; child < 0: leaf ~(first << 3 | count) holding triangles
// [first, first + count).  Slots past the number of children are empty: child
// ~0 (count 0) and an inverted box (every low plane q = 127, every high plane
// q = 0), which a slab test with near and far planes chosen by the ray's
// direction signs never meets.
// Triangle = 3 x float4: (v0, region id bits), (v1, mesh triangle id bits), (v2, 0)
// with region id = solid + 1 (0 = world).
// Trees: one per region (the triangles of the region's own solid and of its child
// solids) plus one over every triangle; all share the node and triangle arrays.
constexpr int kNodeFloats = 16;
constexpr int32_t kEmptyChild = ~0;   // leaf_ref(0, 0)

namespace gadep {
// One node decoded on the host: the child boxes in FP64 (the planes the device
// approximates), the child words and the number of children in use.
struct WideNode {
    double lo[4][3], hi[4][3];
    int32_t child[4];
    int n;
};
void decode_node(const float *f, WideNode &out);
}  // namespace gadep

struct gadep_bvh {
    int device = 0;
    gadep::MeshData geo;                 // for host-side localisation of sources
    std::vector<float> nodes;            // kNodeFloats floats per node
    std::vector<float> tris;             // 12 floats per triangle slot (leaf order, per tree)
    std::vector<int32_t> tri_orig;       // triangle slot -> mesh triangle index
    std::vector<float> planes;           // per mesh triangle: unit normal, offset n . centroid
    std::vector<int32_t> regions;        // 4 ints per region: material, active | (group + 1) << 1,
                                         // parent region, root node of the region's tree (-1 = none)
    int32_t root_all = -1;               // tree over every triangle
    // Photon-slot buffers of the wavefront transport, kept for reuse by the next
    // run on this mesh (allocating gigabytes per call would dominate short runs).
    std::mutex wf_mutex;
    gadep::WavefrontBuffers *wf_cache = nullptr;
    int wf_cache_slots = 0;
    bool wf_cache_busy = false;
    // device scratch of the plan that holds wf_cache (tables, instances, tallies,
    // spectra, counters): the same addresses run after run, so the kernel
    // arguments repeat and the cached CUDA graph of the wavefront loop is reused
    void *plan_scratch = nullptr;
    size_t plan_scratch_bytes = 0;
    gadep_bvh_stats stats{};
    void *d_nodes = nullptr, *d_tris = nullptr, *d_tri_orig = nullptr, *d_regions = nullptr,
         *d_planes = nullptr;
};

namespace gadep {
std::vector<std::vector<int32_t>> region_triangle_sets(const MeshData &g);
gadep_status upload_bvh(gadep_bvh *b);
void free_bvh_device(gadep_bvh *b);
}  // namespace gadep
