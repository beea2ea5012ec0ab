/*
 * gadep.h -- C ABI of libgadep: DetMesh detector surfaces + GPU photon transport
 * (GB300, sm_103a).
 *
 * Method: DetMesh-Gadep, "Triangulated Surface Modeling and GPU-based Monte Carlo
 * Efficiency Calibration of High-Purity Germanium Detectors" (arXiv 2605.25963).
 * The CPU builds the detector's triangulated surfaces from a parameter array and
 * initialises the transport; the GPU transports photons through the meshes;
 * scoring turns tallies into the full-energy-peak efficiency (Fig. 4).
 *
 * Conventions for every call:
 *   - Returns gadep_status: GADEP_OK (0) or a negative code.  No call aborts,
 *     traps, prints or throws; gadep_last_error() returns a thread-local message
 *     for the last failing call of the calling thread.
 *   - Handles (detmesh_mesh, gadep_bvh, gadep_plan) are owned by the library and
 *     released with the matching *_destroy call.  Input arrays are copied; the
 *     caller may free them when the call returns.
 *   - Units: mm, keV, g/cm^3; attenuation coefficients in mm^-1.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Output buffers documented as "host or device" are inspected with
 *     cudaPointerGetAttributes; device buffers must be on the plan's device.
 */
#ifndef GADEP_H
#define GADEP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GADEP_OK = 0,
    GADEP_E_INVAL = -1,     /* bad argument, size or pointer */
    GADEP_E_MESH = -2,      /* mesh not closed / not manifold / solids overlap */
    GADEP_E_NOMEM = -3,     /* host or device allocation failed */
    GADEP_E_CUDA = -4,      /* CUDA runtime error */
    GADEP_E_TIMEOUT = -5,   /* a bounded device wait ran out */
    GADEP_E_DEVICE = -6     /* the device error word was set (see gadep_result.dev_err) */
} gadep_status;

/* Thread-local description of the last error of this thread (never NULL). */
const char *gadep_last_error(void);
/* ABI version of this header: 2. */
int32_t gadep_abi_version(void);

/* ------------------------------------------------------------------------- */
/* DetMesh: parametric detector surfaces (Sec. 2.2-2.3, Table 2)              */
/* ------------------------------------------------------------------------- */

enum { GADEP_DET_BARE_CYLINDER = 0, GADEP_DET_COAX = 1 };
enum { GADEP_MAT_VACUUM = 0, GADEP_MAT_GE = 1, GADEP_MAT_AL = 2, GADEP_MAT_CU = 3,
       GADEP_MAT_WATER = 4, GADEP_N_MAT_CODES = 5 };

/* Detector parameters.  d[0..9] = d1..d10 and D[0..6] = D1..D7 of Table 2:
 *   d1 endcap (entrance window) outer radius   d2 window thickness
 *   d3 endcap side-wall thickness               d4 crystal cup (holder) wall thickness
 *   d5 vacuum gap window -> crystal front       d6 gap crystal side -> cup inner wall
 *   d7 endcap depth (bottom outer face at z = -d7)
 *   d8 cup depth (outer bottom at z = -d8)      d9 endcap bottom thickness
 *   d10 cup bottom thickness
 *   D1 crystal length  D2 crystal radius  D3 front-edge rounding radius
 *   D4 outer dead-layer thickness  D5 borehole depth  D6 borehole radius
 *   D7 borehole contact-layer thickness
 * Frame: z axis = detector axis, z grows toward the source; the window's outer
 * face is z = 0 (COAX) / the crystal front face is z = 0 (BARE_CYLINDER).
 * n_theta: angular segments theta_i = 2 pi i / n_theta (Sec. 2.2.2);
 * n_phi: rounding subdivisions phi_j = (pi/2) j / n_phi (Sec. 2.2.2);
 * z_slices: axial bands of the crystal side wall (>= 1).
 * sep_delta: separation applied to coincident back faces, per nesting level,
 * innermost shifted most (Sec. 2.4.2, Fig. 6).  cup_rim_drop: cup rim below the
 * crystal front face.  Optional source solid: regular src_n_sides-gon prism of
 * circumradius src_r, z in [src_z0, src_z0 + src_h], water.
 * Solids, in this order (ids are the mesh's solid indices):
 *   BARE_CYLINDER: 0 active Ge crystal (R = D2, L = D1, rounding D3); [1 source]
 *   COAX: 0 endcap Al, 1 endcap vacuum, 2 holder Cu, 3 crystal (dead Ge),
 *         4 active Ge (R_active = D2 - D4, L_active = D1 - D4, Eq. of Sec. 2.3.2),
 *         5 bore contact (dead Ge), 6 bore vacuum, [source], [flange Cu]
 * Density groups: 0 dead layer (COAX solid 3), 1 endcap, 2 active Ge, 3 source
 * matrix; other solids -1. */
typedef struct {
    int32_t kind;
    double  d[10];
    double  D[7];
    int32_t n_theta, n_phi, z_slices;
    double  cup_rim_drop;
    double  sep_delta;
    int32_t has_source_solid;
    double  src_r, src_h, src_z0;
    int32_t src_n_sides;
    /* Stress features of the coax (0 = absent).  Groove: an annular channel of
     * width groove_w and depth groove_d centred at radius groove_r, cut into the
     * crystal's back face; the active volume's back face follows it one
     * separation step inside.  Flange: a flat Cu ring around the holder, radii
     * flange_r_in .. flange_r_out, thickness flange_h, top face at z = flange_z_top,
     * with n_bolt_holes axial through-holes of radius bolt_r (bolt_n_sides-gon
     * walls) centred on the circle of radius bolt_rc, one per angular sector
     * (n_theta must be a multiple of n_bolt_holes). */
    double  groove_r, groove_w, groove_d;
    double  flange_r_in, flange_r_out, flange_h, flange_z_top;
    int32_t n_bolt_holes, bolt_n_sides;
    double  bolt_r, bolt_rc;
} detmesh_params;

/* Per-solid attributes.  parent: innermost solid containing this one, -1 = world
 * (the nesting tree, derived from the paper's parity rule at build time). */
typedef struct {
    int32_t material;   /* GADEP_MAT_* code = row of the attenuation tables */
    int32_t active;     /* 1: deposits count toward the spectrum */
    int32_t group;      /* density-scale group, -1 = none */
    int32_t parent;
} gadep_solid;

typedef struct detmesh_mesh detmesh_mesh;

/* Build the triangulated surfaces on the host (Sec. 2.2-2.3).  Triangles are
 * counter-clockwise seen from outside (normal n = (v1-v0) x (v2-v0) points out,
 * Sec. 2.2.2 Eq. n).  Validates: every solid closed and 2-manifold, positive
 * volume, no two solids overlapping (sampled vertex containment).
 * Errors: GADEP_E_INVAL (bad parameters), GADEP_E_MESH (validation failed). */
gadep_status detmesh_build(const detmesh_params *p, detmesh_mesh **out);

/* Wrap caller triangles (any closed, non-overlapping solids) as a mesh.
 * xyz [n_vert][3] mm, tri [n_tri][3] vertex indices, tri_solid [n_tri] in
 * [0, n_solid); material/active/group [n_solid].  Parents are derived with the
 * parity rule.  Same validation as detmesh_build. */
gadep_status detmesh_from_arrays(const float *xyz, int32_t n_vert, const int32_t *tri,
                                 const int32_t *tri_solid, int32_t n_tri,
                                 const int32_t *material, const int32_t *active,
                                 const int32_t *group, int32_t n_solid, detmesh_mesh **out);

/* Borrowed views into the mesh (valid until detmesh_destroy). Any out pointer may be NULL. */
gadep_status detmesh_get(const detmesh_mesh *m, const float **xyz, int32_t *n_vert,
                         const int32_t **tri, const int32_t **tri_solid, int32_t *n_tri,
                         const gadep_solid **solids, int32_t *n_solid);

/* Signed volume (mm^3, divergence theorem) and Euler characteristic V - E + F of one solid. */
gadep_status detmesh_solid_stats(const detmesh_mesh *m, int32_t solid, double *volume,
                                 int32_t *euler);

/* Region of a point by the parity rule of Sec. 2.4.2: the innermost solid with an
 * odd number of ray crossings (-1 = world).  FP64 on the host. */
gadep_status detmesh_locate(const detmesh_mesh *m, const double p[3], int32_t *solid);

void detmesh_destroy(detmesh_mesh *m);

/* ------------------------------------------------------------------------- */
/* Cross-section tables                                                        */
/* ------------------------------------------------------------------------- */

/* Fill mu[n_mat][3][n_grid] (photoabsorption, Compton, pair; mm^-1) at the
 * n_grid energies E_k = exp(ln E_min + k (ln E_max - ln E_min)/(n_grid - 1))
 * for material codes codes[n_mat], from closed-form synthetic models: Born
 * K-shell photoabsorption x 5/4, Klein-Nishina Compton on free electrons,
 * near-threshold pair production (stand-ins for the evaluated photon data the
 * paper uses, Sec. 2.4.1).  Computed in FP64, stored as FP32. */
gadep_status gadep_xs_build(const int32_t *codes, int32_t n_mat, int32_t n_grid, double E_min,
                            double E_max, float *mu);

/* ------------------------------------------------------------------------- */
/* Acceleration structure                                                      */
/* ------------------------------------------------------------------------- */

typedef struct gadep_bvh gadep_bvh;

/* Build options of the BVH.  The cost model is the surface-area heuristic
 *   C = c_trav + (A_L N_L + A_R N_R) / A * c_tri
 * (a node split where C is smallest; a leaf of N <= max_leaf triangles kept
 * when N c_tri is not worse).  split_alpha > 0 turns on spatial splits (Stich,
 * Friedrich and Dietrich 2009): where the two halves of the best centroid
 * partition overlap by more than split_alpha times the root's surface area, a
 * split plane that cuts triangle references in two is also costed; a cut
 * triangle is stored in both subtrees (a copy of its 48-byte record each), at
 * most max_dup records per triangle of a tree on average.  Long, thin
 * triangles (the side walls of a cylinder) otherwise give every node near them
 * a box as long as the wall.  On the coaxial detector meshes, though, spatial
 * splits trade triangle tests for more node visits and the transport runs
 * slower, so they are off by default; they stay available for meshes with
 * large triangles.
 * clip_ratio > 0 turns on early split clipping (Ernst and Greiner 2007) before
 * the build: a triangle whose bounding box, seen along its dominant normal axis,
 * covers more than clip_ratio times its own projected area (a sliver at an angle
 * to the axes, such as the centre-fan triangles of a flat end face) is stored as
 * up to clip_pieces references, each bounding the part of the triangle in one
 * half of the previous piece's box, so that each reference box fits its piece;
 * each reference is a copy of the 48-byte record. */
typedef struct {
    int32_t max_leaf;   /* 1..7 triangles per leaf at most; default 4 */
    float c_trav;       /* >= 0; default 1.5 */
    float c_tri;        /* > 0; default 1 */
    float split_alpha;  /* >= 0, 0 = no spatial splits; default 0 (1e-5 is the usual value when on) */
    float max_dup;      /* 1..16; default 2 */
    float clip_ratio;   /* 0 = off, >= 1: early split clipping of loose triangles (below);
                           < 0 = AUTO (default): 8 for meshes of at least 2^17 triangles, else off */
    int32_t clip_pieces;/* 1..256 references per triangle at most; default 16 */
} gadep_bvh_opts;
void gadep_bvh_opts_default(gadep_bvh_opts *o);

typedef struct {
    int32_t n_nodes, n_leaves, max_depth, max_leaf_tris, n_tri, n_region;
    double  sah_cost;
    int64_t node_bytes, tri_bytes;
    int64_t n_refs;          /* triangle records over all trees (copies from spatial splits included) */
    gadep_bvh_opts opts;     /* the options the tree was built with */
} gadep_bvh_stats;

/* Binned-SAH BVH over all triangles of the mesh (the tree the paper's Gadep uses
 * to accelerate triangle queries, Sec. 2.4.3), compacted to 64-byte 4-wide nodes
 * (child boxes quantised to 7 bits on each node's own grid, rounded outward) and
 * 48-byte triangle records, copied to `device`: one tree over every triangle and
 * one per region (the triangles a photon in that region can reach first).  The
 * mesh may be destroyed afterwards.  device = -1 builds the host copy only
 * (stats and validation work; transport calls on such a handle fail with
 * GADEP_E_INVAL).  gadep_bvh_build uses the default options;
 * gadep_bvh_build_opts takes them (NULL = defaults; GADEP_E_INVAL when out of
 * range). */
gadep_status gadep_bvh_build(const detmesh_mesh *m, int32_t device, gadep_bvh **out);
gadep_status gadep_bvh_build_opts(const detmesh_mesh *m, const gadep_bvh_opts *opts, int32_t device,
                                  gadep_bvh **out);
gadep_status gadep_bvh_get_stats(const gadep_bvh *b, gadep_bvh_stats *out);
/* Host-side invariant check of every tree, on the decoded (quantised) boxes:
 * each of its triangles held by at least one leaf and never twice by one leaf,
 * every child box non-empty and meeting its parent's, empty slots empty, every
 * leaf box meeting the bounds of the triangles it holds, and, with each leaf's
 * box intersected with those of all its ancestors (the region a ray passes
 * every box test of on its way to the leaf), the leaves of each triangle
 * covering a grid of points on it (vertices included; the whole triangle when
 * it was not cut).  GADEP_E_MESH if violated. */
gadep_status gadep_bvh_validate(const gadep_bvh *b);
void gadep_bvh_destroy(gadep_bvh *b);

/* Nearest-hit queries (the traversal step of the transport, exposed for testing).
 * rays: device float [n][8] = (o.x, o.y, o.z, t_min, d.x, d.y, d.z, exclude) where
 * exclude is a triangle index of the mesh stored as float bits (-1 = none); hits
 * need t > t_min.  regions: optional device int32 [n], the region of each origin
 * (0 = world, s + 1 = solid s): the query then searches only that region's tree
 * (its own solid's and its child solids' triangles, the surfaces a photon there
 * can reach first, Sec. 2.4.2 nesting); NULL searches every triangle.
 * Outputs (device, [n]): t (INFINITY when nothing is hit), mesh triangle index
 * (-1), entering flag (1 when d . n < 0; -2 when the traversal stack overflowed).
 * Asynchronous on `stream`. */
gadep_status gadep_nearest_hit(const gadep_bvh *b, const float *rays, const int32_t *regions,
                               int64_t n, float *t_out, int32_t *tri_out, int32_t *entering_out,
                               void *stream);

/* ------------------------------------------------------------------------- */
/* Transport                                                                   */
/* ------------------------------------------------------------------------- */

/* Attenuation tables on a log grid: mu[n_mat][3][n_grid] host memory (pe, Compton,
 * pair, mm^-1 at unit density), indexed by the solids' material codes.  Linear
 * interpolation in ln E, end intervals clamped; mu_pair is taken as 0 at and below
 * 2 m_e c^2.
 * Charged particles (used only with gadep_opts.e_model = 1): e_range[n_mat][e_n]
 * host memory, the CSDA range in mm at unit density of an electron of kinetic
 * energy T_k = exp(ln T_min + k (ln T_max - ln T_min) / (e_n - 1)), strictly
 * increasing in k, +inf on every row of a material that does not slow charged
 * particles (vacuum); gadep_erange_build fills it.  e_range NULL (e_n 0) when
 * not given. */
typedef struct {
    int32_t n_mat, n_grid;
    double  E_min, E_max;
    const float *mu;
    int32_t e_n;
    double  T_min, T_max;
    const float *e_range;
} gadep_materials;

/* CSDA ranges of electrons for the charged-particle model (e_model 1), the
 * stand-in for the paper's electron transport (Sec. 2.4.1 physics list), whose
 * evaluated data are not available: mass stopping power
 *   S(T) = S_col(T) (1 + Z_r T / 800 MeV),
 * S_col the Bethe formula for electrons in Rohrlich-Carlson form (ICRU Report
 * 37) without the density-effect term, mean excitation energies Ge 350 eV,
 * Al 166 eV, Cu 322 eV, water 75 eV; the radiative share after Attix, with
 * Z_r = sum n Z^2 / sum n Z; R(T) = T_min / S(T_min) + integral from T_min to
 * T of dT' / S(T'), divided by the density.  range[n_mat][e_n] (mm), computed
 * in FP64, stored as FP32; +inf rows for vacuum.  GADEP_E_INVAL for unknown
 * codes, e_n < 2, T_min <= 0 or T_max <= T_min. */
gadep_status gadep_erange_build(const int32_t *codes, int32_t n_mat, int32_t e_n, double T_min, double T_max,
                                float *range);

enum { GADEP_SRC_POINT = 0, GADEP_SRC_DISK = 1, GADEP_SRC_PRISM = 2, GADEP_SRC_PENCIL = 3 };
/* Source: POINT at pos, isotropic.  DISK: uniform in the disk of `radius` centred
 * at pos in the plane z = pos.z, isotropic.  PRISM: uniform in the regular
 * n_sides-gon prism of circumradius `radius`, base centre pos, height `height`
 * (the mesh's source solid `solid`), isotropic.  PENCIL: from pos along dir. */
typedef struct {
    int32_t kind;
    float   pos[3];
    float   dir[3];
    float   radius, height;
    int32_t n_sides;
    int32_t solid;
} gadep_source;

enum { GADEP_VARIANT_AUTO = 0, GADEP_VARIANT_MEGA = 1, GADEP_VARIANT_WAVEFRONT = 2 };
#define GADEP_MAX_GROUPS 8

typedef struct {
    uint64_t seed;            /* Philox key */
    uint64_t history_offset;  /* first history id (runs with disjoint id ranges add up exactly) */
    float    e_cut_keV;       /* photons below this deposit locally (default 10) */
    float    fep_delta_keV;   /* full-energy peak: E0 - E_dep <= fep_delta (default 0.01) */
    float    e_max_keV;       /* spectrum range [0, e_max) (default 3000) */
    int32_t  n_bins;          /* spectrum bins (default 4096) */
    int32_t  step_cap;        /* segments per history before it is ended as an error (1e4) */
    int32_t  variant;         /* GADEP_VARIANT_*; AUTO: the wavefront form when >= 2^18 histories are
                                 expected to reach the scene (the mesh's bounding box), else the
                                 megakernel */
    int32_t  block;           /* threads per block (0 = default) */
    int32_t  chunk;           /* histories a warp takes from the work counter at once (0 = default) */
    int32_t  blocks_per_sm;   /* persistent grid = SMs x this (0 = occupancy maximum) */
    int32_t  n_group;         /* density groups scored by gadep_grad (<= 4) */
    float    group_scale[GADEP_MAX_GROUPS];  /* density scale per group (default 1) */
    int32_t  wf_slots;        /* wavefront variant: photon slots in device memory, 1024..2^26 (0 = from
                                 the run: the smallest power of two >= the histories expected to
                                 reach the scene, within [2^20, 2^25]; ~220 B each) */
    int32_t  e_model;         /* charged particles set in motion by photon interactions:
                                 0 (default) deposit their kinetic energy at the interaction point;
                                 1 run straight ahead in the continuous-slowing-down
                                 approximation, depositing region by region along the
                                 mesh (needs gadep_materials.e_range; not with gadep_grad
                                 or gadep_run_noalloc).  Photoabsorption: one electron of
                                 T = E along the photon; Compton: one electron of T = E - E'
                                 along E d - E' d'; pair: electron and positron of
                                 (E - 2 mc^2) / 2 each along the photon (annihilation at the
                                 interaction point).  Below T_min a particle deposits where
                                 it is; what leaves the mesh escapes. */
} gadep_opts;

/* Fill *o with the defaults above (seed 1, offset 0, variant AUTO, scales 1). */
void gadep_opts_default(gadep_opts *o);

/* Per-instance result.  fepe = n_fep / n_hist; sigma = sqrt(fepe (1 - fepe) / n_hist).
 * dev_err: OR of device error bits (1 step cap, 2 Compton sampler bound,
 * 4 photon lost inside a solid, 8 traversal stack overflow, 16 non-finite state). */
typedef struct {
    uint64_t n_hist, n_fep, n_zero, n_over, n_err;
    uint64_t n_segments, n_interactions;
    uint64_t n_culled;        /* histories born in the world whose first ray misses every solid's box */
    double   fepe, sigma;
    double   sum_dep_active, sum_dep_all, sum_esc;
    uint32_t dev_err;
} gadep_result;

/* One transport instance (the GPU transport and host scoring of Fig. 4, Sec. 2.4;
 * physics of Sec. 2.4.1 with the partial cross-section free flight, region
 * identification of Sec. 2.4.2, BVH traversal of Sec. 2.4.3; FEPE and its sigma
 * as the efficiencies of Sec. 3.2): n_hist histories of energy energy_keV from `src`,
 * history ids opts.history_offset + [0, n_hist), Philox instance id `instance`.
 * spectrum: n_bins uint32 counts, host or device (zeroed by the call).
 * edep_trace: optional device float [n_trace] receiving the active deposit of the
 * first n_trace histories (NULL to skip).  result: host.  Synchronises `stream`
 * before returning.  n_hist < 2^32 (the spectrum counts are 32-bit). */
gadep_status gadep_run(const gadep_bvh *b, const gadep_materials *mat, const gadep_source *src,
                       float energy_keV, uint64_t n_hist, uint32_t instance,
                       const gadep_opts *opts, uint32_t *spectrum, float *edep_trace,
                       uint64_t n_trace, gadep_result *result, void *stream);

/* gadep_run without device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate device memory while
 * they run -- applications whose own allocator (a framework's caching allocator,
 * a memory pool sized at start-up) owns all device memory, and loops that cannot
 * take the device-wide synchronisation that cudaFree implies.
 * It runs the megakernel form (variant AUTO or MEGA; WAVEFRONT is refused with
 * GADEP_E_INVAL, since that form's photon slots are allocated) and computes the
 * same histories as gadep_run with the same arguments (n_trace 0) in that form;
 * it returns the same result as gadep_run whenever gadep_run also runs the
 * megakernel (variant MEGA, or AUTO below its wavefront threshold).
 * Scratch: instead of allocating, the call keeps the staged tables, region table,
 * instance record, tallies and work counter in one fixed device array of 345,472
 * bytes (337 KiB) that every GPU loading the library holds until the process exits.
 * Limits (GADEP_E_INVAL beyond them): at most 63 solids, and (materials with
 * non-zero tables used by the mesh) x n_grid <= 12288, n_grid <= 12288.
 * spectrum_dev: caller's device buffer of opts->n_bins uint32 (zeroed by the call);
 * result: host.  The call copies its inputs from host memory and synchronises
 * `stream` before it returns.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array and leave the last call's contents in
 * it; the call clears what must start at zero.  Calls that overlap on the GPU
 * (different streams or host threads at the same time) race on it. */
gadep_status gadep_run_noalloc(const gadep_bvh *b, const gadep_materials *mat, const gadep_source *src,
                               float energy_keV, uint64_t n_hist, uint32_t instance,
                               const gadep_opts *opts, uint32_t *spectrum_dev, gadep_result *result,
                               void *stream);

/* Batched (the paper runs one energy at a time, Sec. 3.2 / Table 3; here the
 * instances of that loop share one launch, the transport of each being that of
 * gadep_run: Fig. 4, Sec. 2.4, 2.4.1): n_inst instances, each with its own energy, source, history count,
 * Philox instance id and density scales, in one persistent launch drawing
 * histories from a device work counter.  spectra [n_inst][n_bins] host or device;
 * results [n_inst] host. */
typedef struct {
    float        energy_keV;
    gadep_source src;
    uint64_t     n_hist;
    uint32_t     instance;
    float        group_scale[GADEP_MAX_GROUPS];
} gadep_instance;

gadep_status gadep_run_batch(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                             const gadep_instance *inst, const gadep_opts *opts,
                             uint32_t *spectra, gadep_result *results, void *stream);

/* Density-perturbation gradient (no counterpart in the paper: the derivative of
 * the FEPE of Sec. 3.2 with respect to the densities of the materials of Sec. 2.4.1,
 * for the dead-layer characterisation the paper motivates in Sec. 1 and Sec. 4;
 * the transport is gadep_run's): for each instance and group p,
 * dfepe[i][p] = d FEPE_i / d s_p = mean over histories of FEP * score_p with
 * score_p = (collisions in group p)/s_p - sum over segments in group p of
 * mu_unit(E) * length, accumulated on the fly (no stored tracks);
 * dsigma[i][p] its standard error.  Also fills spectra/results like
 * gadep_run_batch (the same histories).  dfepe, dsigma: host [n_inst][opts.n_group]. */
gadep_status gadep_grad(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                        const gadep_instance *inst, const gadep_opts *opts, uint32_t *spectra,
                        gadep_result *results, double *dfepe, double *dsigma, void *stream);

/* Plans: the device-resident form of a batched run, for repeated launches and
 * CUDA-graph capture.  gadep_plan_create uploads tables, regions and instances and
 * allocates tallies; gadep_plan_launch only zeroes the tallies and launches the
 * kernel on `stream` (no allocation, no host copy, no synchronisation);
 * gadep_plan_results copies tallies back, synchronises `stream` and finalises.
 * grad != 0 accumulates the density-perturbation scores. */
typedef struct gadep_plan gadep_plan;
gadep_status gadep_plan_create(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                               const gadep_instance *inst, const gadep_opts *opts, int32_t grad,
                               gadep_plan **out);
/* spectra_dev: device [n_inst][n_bins] uint32, or NULL to use the plan's own buffer. */
gadep_status gadep_plan_launch(gadep_plan *p, uint32_t *spectra_dev, void *stream);
gadep_status gadep_plan_results(gadep_plan *p, uint32_t *spectra_host, gadep_result *results,
                                double *dfepe, double *dsigma, void *stream);
/* Launch shape the plan uses: grid blocks, threads per block, dynamic shared bytes. */
gadep_status gadep_plan_shape(const gadep_plan *p, int32_t *grid, int32_t *block,
                              int32_t *smem_bytes);
void gadep_plan_destroy(gadep_plan *p);

/* Peaks of `device` measured by the library's own microbenchmarks (no
 * counterpart in the paper; denominators for the transport kernels, which are
 * bound by FP32/ALU issue and served from L2): FP32 FMA throughput in TFLOP/s
 * (an FMA counts 2 FLOP) of independent FMA chains on every SM, and the read
 * bandwidth in GB/s of a 64 MB buffer re-read from L2.  Allocates and frees
 * 64 MB of device memory and synchronises the device; either output may be NULL. */
gadep_status gadep_measure_peaks(int32_t device, double *fp32_tflops, double *l2_read_gbs);

/* Kernel launches of a plan since the last reset, per kind: the persistent
 * megakernel, or the kernels of each wavefront iteration (with e_model 1 also the
 * deferred charged-particle tracks, ETRACK) plus the slot-list initialisation.
 * With timing on, gadep_plan_launch records a CUDA event pair on the launching
 * stream around every launch and ms[] sums their elapsed times (device time of
 * the kernels alone, without host gaps).  Entries past the last kind are 0. */
enum { GADEP_KERNEL_MEGA = 0, GADEP_KERNEL_SPAWN = 1, GADEP_KERNEL_TRACE = 2, GADEP_KERNEL_PHYSICS = 3,
       GADEP_KERNEL_GEN = 4, GADEP_KERNEL_CTRL = 5, GADEP_KERNEL_INIT = 6, GADEP_KERNEL_SORT = 7,
       GADEP_KERNEL_ETRACK = 8, GADEP_N_KERNEL_KINDS = 9 };
typedef struct {
    uint64_t launches[16];    /* [GADEP_KERNEL_*] */
    double   ms[16];          /* [GADEP_KERNEL_*], 0 unless timing was on */
} gadep_kernel_stats;
/* on != 0 turns per-launch event timing on for later launches of the plan. */
gadep_status gadep_plan_set_timing(gadep_plan *p, int32_t on);
/* Waits for the timed launches (host synchronisation on their events), writes
 * the statistics to *out (host) and, when reset != 0, clears them. */
gadep_status gadep_plan_kernel_stats(gadep_plan *p, gadep_kernel_stats *out, int32_t reset);

/* Trace queue size of each wavefront iteration of the plan's last launch, in
 * order (the queries its trace kernel launches served), for measurements that
 * need the work of individual launches (no counterpart in the paper).  out: host
 * [max]; *n: entries written (0 for a megakernel plan; the log holds the first
 * 8192 iterations).  Synchronises `stream`. */
gadep_status gadep_plan_queue_sizes(gadep_plan *p, uint32_t *out, int32_t max, int32_t *n, void *stream);

/* Work counters of the traversal for one batch (same histories as gadep_run_batch):
 * 4-wide BVH nodes visited, child boxes tested in them (a node's empty slots not
 * counted) and triangles tested, summed over all segment queries, and the number
 * of queries that found no surface in their region's tree and were relocated
 * through the tree of every triangle (photons a rounding error past a boundary).
 * `relocated` and `boxes_tested` may be NULL.  Runs an instrumented copy of the
 * transport kernels; used to turn the measured time into algorithmic bytes and
 * FLOPs per query.  results: host [n_inst]. */
gadep_status gadep_count_work(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                              const gadep_instance *inst, const gadep_opts *opts,
                              gadep_result *results, uint64_t *nodes_visited,
                              uint64_t *tris_tested, uint64_t *relocated, uint64_t *boxes_tested,
                              void *stream);

/* Philox4x32-10 stream words of one history computed on the GPU (layout:
 * key = (seed lo, seed hi), counter = (block, hid lo, hid hi, instance)).
 * out: device uint32 [n_words].  For testing the device generator. */
gadep_status gadep_philox_words(uint64_t seed, uint64_t hid, uint32_t instance, int32_t n_words,
                                uint32_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
