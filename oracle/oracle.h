/*
 * oracle.h -- plain, slow FP64 CPU oracle for the DetMesh-Gadep photon path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no source, header,
 * table or constant with the CUDA path.
 *
 * What it computes (paper: DetMesh-Gadep, arXiv 2605.25963):
 *   - triangulated detector surfaces from the parametric model of Sec. 2.2-2.3
 *     (angular sampling Eq. theta_i, rounding Eq. rho_j/z_j, active-volume
 *     shrinkage Eq. R_active/L_active, coincident-surface separation Sec. 2.4.2);
 *   - photon transport with the partial cross-section free-flight scheme
 *     (Sec. 2.4.1) and the ray-parity localization rule (Sec. 2.4.2, Fig. 5);
 *   - the pulse-height spectrum of energy deposited in the active germanium
 *     and the full-energy-peak efficiency (FEPE) tallied on the host (Fig. 4).
 * Ingredients the paper leaves to the implementation are restated from their
 * published definitions: Philox4x32-10 (Salmon et al., SC'11), Kahn's
 * rejection sampler for Klein-Nishina scattering (Kahn 1956, as given by
 * Everett & Cashwell 1973), density-perturbation (differential operator)
 * scores for dFEPE/d(density scale).
 *
 * Brute force everywhere: every flight intersects its ray with every triangle
 * (after a per-solid bounding-box test, the paper's "subset filtered by
 * bounding boxes"), and the region of every segment is decided by the
 * literal parity rule.
 */
#ifndef GADEP_ORACLE_H
#define GADEP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- counter-based RNG (Philox4x32-10) ---------------- */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* u = (2*(x >> 9) + 1) * 2^-24, exact in binary32 and binary64, in (0,1) */
double orc_u01(uint32_t x);
/* words of the stream of history `hid` of instance `inst`: n_words values
   starting at draw 0 (block 0 word 0). */
void   orc_stream_words(uint64_t seed, uint64_t hid, uint32_t inst, int n_words, uint32_t *out);

/* ---------------- cross sections (closed-form synthetic models) ---------------- */
enum { ORC_MAT_VACUUM = 0, ORC_MAT_GE = 1, ORC_MAT_AL = 2, ORC_MAT_CU = 3, ORC_MAT_WATER = 4,
       ORC_N_MAT_CODES = 5 };
double orc_sigma_kn(double k);                       /* cm^2 per electron, k = E/mc^2 */
double orc_dsigma_kn_dcos(double k, double c);       /* cm^2 per electron per unit cos(theta) */
double orc_sigma_pe(int Z, double E_keV);            /* cm^2 per atom */
double orc_sigma_pair(int Z, double E_keV);          /* cm^2 per atom */
/* linear attenuation coefficients of a material code at E, mm^-1: out = pe, compton, pair */
int    orc_mu(int code, double E_keV, double out[3]);

/* Tables on a log-energy grid, rounded to binary32 as the transport consumes them.
   mu layout [n_mat][3][n_grid] (pe, compton, pair), mm^-1 at unit density scale. */
typedef struct {
    int n_mat, n_grid;
    double lnE_min, lnE_max;
    float *mu;
    /* charged particles (continuous slowing down, see orc_xs.c): CSDA range in mm
       at unit density scale on e_n log-spaced kinetic energies from ORC_E_TMIN to
       E_max, [n_mat][e_n], FP64; a row of +inf for a material with no stopping
       (vacuum); e_n = 0 when the tables were not built from material codes */
    int e_n;
    double lnT_min, lnT_max;
    double *e_range;
} orc_tables;
orc_tables *orc_tables_build(const int *codes, int n_mat, int n_grid, double E_min, double E_max);
orc_tables *orc_tables_from_array(int n_mat, int n_grid, double E_min, double E_max, const float *mu);
void        orc_tables_free(orc_tables *t);
/* interpolated mu (pe, compton, pair) of material m at E, FP64 arithmetic on the stored values */
void        orc_tables_eval(const orc_tables *t, int m, double E_keV, double out[3]);

/* charged particles: below ORC_E_TMIN a particle deposits where it is */
#define ORC_E_TMIN 1.0   /* keV */
/* mass stopping power of material `code` for an electron of kinetic energy T:
   collision part and total (collision + radiative), MeV cm^2/g; -1 for an
   unknown code, 0 with both zero for vacuum */
int    orc_e_stopping(int code, double T_keV, double *s_col, double *s_tot);
/* CSDA range (mm, unit density scale) of table material m at T; +inf for vacuum */
double orc_e_range(const orc_tables *t, int m, double T_keV);
/* kinetic energy left after a path of L mm (unit density scale) in material m */
double orc_e_energy_after(const orc_tables *t, int m, double T_keV, double L_mm);

/* ---------------- detector meshes (Sec. 2.2-2.3) ---------------- */
enum { ORC_DET_BARE_CYLINDER = 0, ORC_DET_COAX = 1 };
typedef struct {
    int    kind;
    double d[10];      /* Table 2 external group d1..d10 */
    double D[7];       /* Table 2 internal group D1..D7 */
    int    n_theta, n_phi, z_slices;
    double cup_rim_drop;   /* cup rim below the crystal front face */
    double sep_delta;      /* coincident-face separation per nesting level */
    int    has_source_solid;
    double src_r, src_h, src_z0;
    int    src_n_sides;
    /* stress features of the coax (0 = absent): back-face groove, bolted flange */
    double groove_r, groove_w, groove_d;
    double flange_r_in, flange_r_out, flange_h, flange_z_top;
    int    n_bolt_holes, bolt_n_sides;
    double bolt_r, bolt_rc;
} orc_detparams;

typedef struct {
    int     n_vert, n_tri, n_solid;
    double *xyz;           /* [n_vert][3] mm */
    int    *tri;           /* [n_tri][3], counter-clockwise seen from outside */
    int    *tri_solid;     /* [n_tri] */
    int    *solid_material, *solid_active, *solid_group, *solid_parent; /* parent -1 = world */
} orc_mesh;
int       orc_mesh_build(const orc_detparams *p, orc_mesh **out);
orc_mesh *orc_mesh_from_arrays(int n_vert, const double *xyz, int n_tri, const int *tri,
                               const int *tri_solid, int n_solid, const int *material,
                               const int *active, const int *group, const int *parent);
void      orc_mesh_free(orc_mesh *m);
/* signed volume (divergence theorem), area and Euler characteristic of one solid */
double    orc_mesh_volume(const orc_mesh *m, int solid);
double    orc_mesh_area(const orc_mesh *m, int solid);
int       orc_mesh_euler(const orc_mesh *m, int solid);
/* number of directed edges of the solid that are not matched by exactly one opposite edge */
int       orc_mesh_open_edges(const orc_mesh *m, int solid);
/* parity-rule region of a point: innermost solid whose triangle count along +dir is odd */
int       orc_locate(const orc_mesh *m, const double p[3], const double dir[3]);

/* Nearest crossing along o + t d with t > t_min, skipping triangle `exclude`
   (-1 none): brute force over every triangle.  Returns the triangle or -1. */
int       orc_nearest_hit(const orc_mesh *m, const double o[3], const double d[3], double t_min,
                          int exclude, double *t, int *entering);

/* ---------------- sources and sampling ---------------- */
enum { ORC_SRC_POINT = 0, ORC_SRC_DISK = 1, ORC_SRC_PRISM = 2, ORC_SRC_PENCIL = 3 };
typedef struct {
    int    kind;
    double pos[3];     /* point / disk centre / prism base centre / pencil origin */
    double dir[3];     /* pencil direction (unit) */
    double radius;     /* disk radius, prism circumradius */
    double height;     /* prism height */
    int    n_sides;    /* prism polygon sides */
} orc_source;
/* samples birth position and direction of history hid (consumes the stream's first draws) */
void orc_sample_birth(const orc_source *s, uint64_t seed, uint64_t hid, uint32_t inst,
                      double pos[3], double dir[3]);
/* Kahn sampler: n samples of x = E/E' at k = E/mc^2 from one stream per sample */
int  orc_kahn_samples(double k, uint64_t seed, int n, double *x_out);

/* ---------------- transport and tallies ---------------- */
typedef struct {
    uint64_t seed, history_offset;
    uint32_t instance;
    double   energy_keV, e_cut_keV, fep_delta_keV, e_max_keV;
    int      n_bins;
    int      step_cap;             /* segments per history */
    int      n_group;              /* density groups, <= 8 */
    double   group_scale[8];
    int      e_model;              /* 0: charged particles deposit at their birth point;
                                      1: continuous-slowing-down tracks (orc_transport.c) */
} orc_opts;

typedef struct {
    uint64_t n_hist, n_fep, n_zero, n_over, n_err;
    uint64_t n_parity_mismatch;    /* crossings where tree rule != parity rule */
    uint64_t n_dup_hits;           /* coincident same-solid hits merged */
    uint64_t n_segments, n_interactions, n_crossings, n_flights;
    uint64_t n_first_pe, n_first_compton, n_first_pair, n_first_none;
    double   sum_dep_active, sum_dep_all, sum_esc, max_rel_energy_err;
    double   fep_score[8], fep_score_sq[8];
} orc_tally;

/* Transport n_hist histories (ids history_offset .. +n_hist-1) with n_threads
   threads.  spectrum: n_bins uint32 (may be NULL).  edep: optional per-history
   active deposit [n_hist] (may be NULL).  Returns 0 or a negative error. */
int orc_transport(const orc_mesh *m, const orc_tables *t, const orc_source *src,
                  const orc_opts *o, uint64_t n_hist, int n_threads,
                  orc_tally *out, uint32_t *spectrum, double *edep);

/* One charged-particle line of e_model 1 (orc_transport.c): `weight` particles of
   kinetic energy T from p along unit u, born in region `region` (solid index,
   -1 = world), density scales from o.  out = (active deposit, all deposits,
   escaped), keV.  Returns 0, or nonzero on a geometry error. */
int orc_e_track(const orc_mesh *m, const orc_tables *t, const orc_opts *o, const double p[3], const double u[3],
                double T_keV, double weight, int region, double out[3]);

#ifdef __cplusplus
}
#endif
#endif
