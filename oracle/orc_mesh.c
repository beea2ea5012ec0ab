/*
 * orc_mesh.c -- oracle detector surfaces (test infrastructure only).
 *
 * Every solid of the detector models is a solid of revolution, so the oracle
 * builds each one by revolving a closed (rho, z) profile about the z axis in
 * the detector's global frame (z toward the source, window outer face at
 * z = 0).  The angular positions are theta_i = 2 pi i / N_theta (Sec. 2.2.2,
 * angular-equidistant sampling); the front-edge rounding uses
 *   phi_j = (pi/2) j / N_phi,
 *   rho_j = (R - R_ch) + R_ch cos(phi_j),
 *   z_j   = z_front - R_ch (1 - sin(phi_j))
 * (Sec. 2.2.2, written in the global frame where the front face looks toward
 * +z).  A rounding radius equal to the radius gives the hemispherical blind end
 * of the borehole with a single apex vertex (Fig. 10).
 *
 * Profiles are walked with the solid's outward normal on the left of the
 * walking direction (rho to the right, z up); each profile segment becomes a
 * band of N_theta quads (two triangles) or a fan when one end is on the axis.
 * A segment from the axis to a ring in the same plane (a flat end face; the
 * paper does not say how such a face is cut into triangles) is cut into
 * concentric rings instead of a fan of slivers that all meet at the centre:
 * ring k at radius R - k w, w = 4 (2 pi R / N_theta) (four times the arc between
 * the outer ring's vertices), with max(8, round(N_theta (R - k w) / R)) vertices
 * at angles 2 pi i / count, for k = 1, 2, ... while the radius is at least w and
 * the count falls; consecutive rings are joined by walking around them by angle,
 * and the innermost ring closes with a fan at the centre.  The face is the same
 * plane polygon, so volumes and the surface are unchanged.
 *
 * Coaxial detector layout (Table 2 parameters, Sec. 2.3.2):
 *   solid 0  endcap (Al)            cylinder R = d1, z in [-d7, 0]
 *   solid 1  endcap vacuum          cylinder R = d1 - d3, z in [-d7 + d9, -d2]
 *   solid 2  crystal holder (Cu)    cup: inner radius D2 + d6, wall d4, rim at
 *                                   z_front - rim_drop, outer bottom -d8, bottom d10
 *   solid 3  crystal (dead Ge)      R = D2, length D1, rounding D3, front at -(d2 + d5)
 *   solid 4  active Ge              R = D2 - D4, length D1 - D4, rounding D3 - D4
 *                                   (Eq. R_active, L_active: back face not shrunk)
 *   solid 5  bore contact (dead Ge) R = D6 + D7, depth D5 + D7, hemispherical end
 *   solid 6  bore vacuum            R = D6, depth D5, hemispherical end
 *   solid 7  optional source (water prism)
 * The back faces of solids 3..6 coincide; they are separated inside-out
 * (Sec. 2.4.2, Fig. 6): nesting level L is lifted by L * sep_delta.
 *   stress features (optional): an annular groove cut into the crystal's back
 *   face (profile notch; the active volume's back face follows it one sep_delta
 *   inside) and, after the source, a flat Cu flange ring with axial bolt holes.
 *   The flange faces are planar polygons with holes; the oracle triangulates
 *   each angular sector (one hole per sector) by ear clipping after bridging the
 *   hole to the sector boundary.
 *
 * Bare cylinder: solid 0 = active Ge cylinder R = D2, length D1, rounding D3,
 * front face at z = 0; solid 1 = optional source prism.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    int n_vert, cap_vert, n_tri, cap_tri;
    double *xyz; int *tri; int *tri_solid;
} builder;

static int add_vertex(builder *b, double x, double y, double z)
{
    if (b->n_vert == b->cap_vert) {
        b->cap_vert = b->cap_vert ? 2 * b->cap_vert : 1024;
        b->xyz = (double *)realloc(b->xyz, (size_t)b->cap_vert * 3 * sizeof(double));
    }
    b->xyz[3 * b->n_vert + 0] = x;
    b->xyz[3 * b->n_vert + 1] = y;
    b->xyz[3 * b->n_vert + 2] = z;
    return b->n_vert++;
}

static void add_tri(builder *b, int a, int c, int d, int solid)
{
    if (b->n_tri == b->cap_tri) {
        b->cap_tri = b->cap_tri ? 2 * b->cap_tri : 1024;
        b->tri = (int *)realloc(b->tri, (size_t)b->cap_tri * 3 * sizeof(int));
        b->tri_solid = (int *)realloc(b->tri_solid, (size_t)b->cap_tri * sizeof(int));
    }
    b->tri[3 * b->n_tri + 0] = a;
    b->tri[3 * b->n_tri + 1] = c;
    b->tri[3 * b->n_tri + 2] = d;
    b->tri_solid[b->n_tri] = solid;
    b->n_tri++;
}

/* Triangles joining ring A (na vertices from a0) to ring B (nb from b0), both
   starting at angle 0, oriented like the quad band (A_i, B_i, A_i+1),
   (A_i+1, B_i, B_i+1): around the rings by angle, stepping along A unless B's
   next vertex comes strictly first. */
static void join_rings(builder *b, int solid, int a0, int na, int b0, int nb)
{
    int i = 0, j = 0;
    while (i < na || j < nb) {
        int step_a;
        if (i == na) step_a = 0;
        else if (j == nb) step_a = 1;
        else step_a = (double)(i + 1) * nb <= (double)(j + 1) * na;   /* next angle of A <= next of B */
        if (step_a) {
            add_tri(b, a0 + i % na, b0 + j % nb, a0 + (i + 1) % na, solid);
            ++i;
        } else {
            add_tri(b, a0 + i % na, b0 + j % nb, b0 + (j + 1) % nb, solid);
            ++j;
        }
    }
}

/* The inner rings of a flat end face whose outer ring has radius R and N
   vertices (header comment): appends their vertices, stores each ring's first
   vertex and count (at most 64 rings) and returns how many there are. */
static int disk_rings(builder *b, double R, double zf, int N, int *first, int *count)
{
    const double w = 4.0 * (2.0 * ORC_PI * R / (double)N);
    int k_rings = 0, prev = N;
    for (int k = 1; k < 64; ++k) {
        double r = R - (double)k * w;
        long m = lround((double)N * r / R);
        if (m < 8) m = 8;
        if (r < w || m >= prev) break;
        first[k_rings] = b->n_vert;
        count[k_rings] = (int)m;
        for (int i = 0; i < m; ++i) {
            double th = 2.0 * ORC_PI * (double)i / (double)m;
            add_vertex(b, r * cos(th), r * sin(th), zf);
        }
        prev = (int)m;
        ++k_rings;
    }
    return k_rings;
}

/* Revolve a profile of np points (rho, z); rho == 0 marks an axis point. */
static void revolve(builder *b, int solid, const double *rho, const double *z, int np, int N)
{
    int *first = (int *)malloc((size_t)np * sizeof(int));
    for (int k = 0; k < np; ++k) {
        if (rho[k] == 0.0) {
            first[k] = add_vertex(b, 0.0, 0.0, z[k]);
        } else {
            first[k] = b->n_vert;
            for (int i = 0; i < N; ++i) {
                double th = 2.0 * ORC_PI * (double)i / (double)N;
                add_vertex(b, rho[k] * cos(th), rho[k] * sin(th), z[k]);
            }
        }
    }
    for (int k = 0; k + 1 < np; ++k) {
        int ra = rho[k] != 0.0, rb = rho[k + 1] != 0.0;
        if (ra != rb && z[k] == z[k + 1]) {
            /* flat end face: rings from the outer one inward, then the centre fan */
            int rf[64], rc[64];
            const int kr = ra ? k : k + 1, kc = ra ? k + 1 : k;
            const int nr = disk_rings(b, rho[kr], z[kr], N, rf, rc);
            int o0 = first[kr], on = N;
            for (int q = 0; q < nr; ++q) {
                if (ra) join_rings(b, solid, o0, on, rf[q], rc[q]);       /* ring first, then inward */
                else join_rings(b, solid, rf[q], rc[q], o0, on);          /* axis first: inner ring is A */
                o0 = rf[q];
                on = rc[q];
            }
            for (int i = 0; i < on; ++i) {
                int i1 = (i + 1) % on;
                if (ra) add_tri(b, o0 + i, first[kc], o0 + i1, solid);
                else add_tri(b, first[kc], o0 + i, o0 + i1, solid);
            }
            continue;
        }
        for (int i = 0; i < N; ++i) {
            int i1 = (i + 1) % N;
            if (ra && rb) {
                int A0 = first[k] + i, A1 = first[k] + i1;
                int B0 = first[k + 1] + i, B1 = first[k + 1] + i1;
                add_tri(b, A0, B0, A1, solid);
                add_tri(b, A1, B0, B1, solid);
            } else if (!ra && rb) {
                add_tri(b, first[k], first[k + 1] + i, first[k + 1] + i1, solid);
            } else if (ra && !rb) {
                add_tri(b, first[k] + i, first[k + 1], first[k] + i1, solid);
            }
        }
    }
    free(first);
}

/* Profile of a cylinder of radius R from z_front down to z_back with a front
   rounding of radius rch (0 <= rch <= R); rch == R gives a hemispherical end. */
static int rounded_profile(double R, double rch, double z_front, double z_back, int n_phi,
                           int z_slices, double g_in, double g_out, double g_depth, double *rho, double *z)
{
    int n = 0;
    if (rch > 0.0) {
        int hemi = (rch == R);
        /* apex / front-face centre */
        if (!hemi) { rho[n] = 0.0; z[n] = z_front; ++n; }
        for (int j = n_phi; j >= 0; --j) {
            double phi = 0.5 * ORC_PI * (double)j / (double)n_phi;
            double r = (R - rch) + rch * cos(phi);
            double zz = z_front - rch * (1.0 - sin(phi));
            if (hemi && j == n_phi) r = 0.0;  /* single apex vertex */
            rho[n] = r; z[n] = zz; ++n;
        }
    } else {
        rho[n] = 0.0; z[n] = z_front; ++n;
        rho[n] = R;   z[n] = z_front; ++n;
    }
    double z_side_top = z_front - rch;
    if (z_slices < 1) z_slices = 1;
    for (int s = 1; s <= z_slices; ++s) {
        rho[n] = R;
        z[n] = (s == z_slices) ? z_back : z_side_top - (z_side_top - z_back) * (double)s / (double)z_slices;
        ++n;
    }
    if (g_depth > 0.0) {
        /* annular channel g_in < rho < g_out cut g_depth into the back face */
        rho[n] = g_out; z[n] = z_back; ++n;
        rho[n] = g_out; z[n] = z_back + g_depth; ++n;
        rho[n] = g_in;  z[n] = z_back + g_depth; ++n;
        rho[n] = g_in;  z[n] = z_back; ++n;
    }
    rho[n] = 0.0; z[n] = z_back; ++n;
    return n;
}

static void add_rounded_g(builder *b, int solid, double R, double rch, double z_front, double z_back,
                          int N, int n_phi, int z_slices, double g_in, double g_out, double g_depth)
{
    int cap = n_phi + z_slices + 12;
    double *rho = (double *)malloc((size_t)cap * sizeof(double));
    double *z = (double *)malloc((size_t)cap * sizeof(double));
    int np = rounded_profile(R, rch, z_front, z_back, n_phi, z_slices, g_in, g_out, g_depth, rho, z);
    revolve(b, solid, rho, z, np, N);
    free(rho); free(z);
}

static void add_rounded(builder *b, int solid, double R, double rch, double z_front, double z_back,
                        int N, int n_phi, int z_slices)
{
    add_rounded_g(b, solid, R, rch, z_front, z_back, N, n_phi, z_slices, 0.0, 0.0, 0.0);
}

/* ---- flange: planar faces with holes, triangulated by ear clipping ---- */

typedef struct { double x, y; int id; } pt2;

static double cross3(const pt2 *a, const pt2 *b, const pt2 *c)
{
    return (b->x - a->x) * (c->y - a->y) - (b->y - a->y) * (c->x - a->x);
}

static int same_point(const pt2 *a, const pt2 *b) { return a->x == b->x && a->y == b->y; }

/* p inside or on the closed triangle (a, b, c) given counter-clockwise */
static int in_triangle(const pt2 *p, const pt2 *a, const pt2 *b, const pt2 *c)
{
    return cross3(a, b, p) >= 0.0 && cross3(b, c, p) >= 0.0 && cross3(c, a, p) >= 0.0;
}

/* Ear clipping of a counter-clockwise (weakly) simple polygon of n points; emits
   n - 2 counter-clockwise triangles through emit(ids).  Returns 0 on success. */
static int ear_clip(pt2 *poly, int n, builder *b, int solid, int flip)
{
    int *idx = (int *)malloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) idx[i] = i;
    int m = n, guard = 0;
    while (m > 3) {
        int found = 0;
        for (int k = 0; k < m && !found; ++k) {
            const pt2 *a = &poly[idx[(k + m - 1) % m]], *c0 = &poly[idx[k]], *c = &poly[idx[(k + 1) % m]];
            if (cross3(a, c0, c) <= 0.0) continue;          /* reflex or degenerate corner */
            int blocked = 0;
            for (int q = 0; q < m && !blocked; ++q) {
                const pt2 *p = &poly[idx[q]];
                if (same_point(p, a) || same_point(p, c0) || same_point(p, c)) continue;
                if (in_triangle(p, a, c0, c)) blocked = 1;
            }
            if (blocked) continue;
            if (flip) add_tri(b, a->id, c->id, c0->id, solid);
            else add_tri(b, a->id, c0->id, c->id, solid);
            for (int q = k; q + 1 < m; ++q) idx[q] = idx[q + 1];
            --m;
            found = 1;
        }
        if (!found || ++guard > 4 * n) { free(idx); return -1; }
    }
    const pt2 *a = &poly[idx[0]], *c0 = &poly[idx[1]], *c = &poly[idx[2]];
    if (flip) add_tri(b, a->id, c->id, c0->id, solid);
    else add_tri(b, a->id, c0->id, c->id, solid);
    free(idx);
    return 0;
}

/* Flat ring r_in..r_out, z in [z_top - h, z_top], with nh axial holes of radius
   rh (M-gon, M even) centred on radius rc, hole k at angle 2 pi (k + 1/2) / nh.
   N (a multiple of nh, N / nh even) vertices on each circle. */
static int add_flange(builder *b, int solid, double r_in, double r_out, double h, double z_top, int nh,
                      int M, double rh, double rc, int N)
{
    if (nh < 1 || N % nh != 0 || (N / nh) % 2 != 0 || M < 4 || M % 2 != 0) return -1;
    const double zt = z_top, zb = z_top - h;
    const int m = N / nh;
    int ring[4];                       /* inner top, outer top, inner bottom, outer bottom */
    const double rr[4] = { r_in, r_out, r_in, r_out }, zz[4] = { zt, zt, zb, zb };
    for (int q = 0; q < 4; ++q) {
        ring[q] = b->n_vert;
        for (int i = 0; i < N; ++i) {
            double th = 2.0 * ORC_PI * (double)i / (double)N;
            add_vertex(b, rr[q] * cos(th), rr[q] * sin(th), zz[q]);
        }
    }
    int *hole = (int *)malloc((size_t)nh * 2 * sizeof(int));
    for (int k = 0; k < nh; ++k) {
        double tc = 2.0 * ORC_PI * ((double)k + 0.5) / (double)nh;
        double cx = rc * cos(tc), cy = rc * sin(tc);
        for (int f = 0; f < 2; ++f) {
            hole[2 * k + f] = b->n_vert;
            for (int j = 0; j < M; ++j) {
                double a = tc + 2.0 * ORC_PI * (double)j / (double)M;
                add_vertex(b, cx + rh * cos(a), cy + rh * sin(a), f == 0 ? zt : zb);
            }
        }
    }
    /* walls: outer faces +r, inner faces toward the axis, hole walls toward the hole axis */
    for (int i = 0; i < N; ++i) {
        int i1 = (i + 1) % N;
        add_tri(b, ring[1] + i, ring[3] + i, ring[3] + i1, solid);
        add_tri(b, ring[1] + i, ring[3] + i1, ring[1] + i1, solid);
        add_tri(b, ring[0] + i, ring[2] + i1, ring[2] + i, solid);
        add_tri(b, ring[0] + i, ring[0] + i1, ring[2] + i1, solid);
    }
    for (int k = 0; k < nh; ++k) {
        int t = hole[2 * k], u = hole[2 * k + 1];
        for (int j = 0; j < M; ++j) {
            int j1 = (j + 1) % M;
            add_tri(b, t + j, t + j1, u + j1, solid);
            add_tri(b, t + j, u + j1, u + j, solid);
        }
    }
    /* faces: each sector polygon, hole bridged to the inner-arc midpoint */
    int n_poly = 2 * (m + 1) + M + 3;
    pt2 *poly = (pt2 *)malloc((size_t)n_poly * sizeof(pt2));
    int rc_ok = 0;
    for (int f = 0; f < 2 && rc_ok == 0; ++f) {
        int in = ring[f == 0 ? 0 : 2], out = ring[f == 0 ? 1 : 3];
        for (int k = 0; k < nh && rc_ok == 0; ++k) {
            int n = 0;
#define ORC_PUSH(vid) do { int v_ = (vid); poly[n].x = b->xyz[3 * v_]; poly[n].y = b->xyz[3 * v_ + 1]; poly[n].id = v_; ++n; } while (0)
            /* counter-clockwise: outer arc forward, inner arc backward with the bridge */
            for (int i = 0; i <= m; ++i) ORC_PUSH(out + (k * m + i) % N);
            for (int i = m; i >= m / 2; --i) ORC_PUSH(in + (k * m + i) % N);
            int hv = hole[2 * k + f];
            /* around the hole clockwise, from its vertex facing the axis and back */
            for (int j = 0; j <= M; ++j) ORC_PUSH(hv + ((M / 2 - j) % M + M) % M);
            for (int i = m / 2; i >= 0; --i) ORC_PUSH(in + (k * m + i) % N);
#undef ORC_PUSH
            rc_ok = ear_clip(poly, n, b, solid, f == 1);
        }
    }
    free(poly);
    free(hole);
    return rc_ok;
}

static void add_cup(builder *b, int solid, double r_in, double r_out, double z_rim,
                    double z_inner_bottom, double z_outer_bottom, int N)
{
    double rho[6] = { 0.0, r_in, r_in, r_out, r_out, 0.0 };
    double z[6] = { z_inner_bottom, z_inner_bottom, z_rim, z_rim, z_outer_bottom, z_outer_bottom };
    revolve(b, solid, rho, z, 6, N);
}

static orc_mesh *finish(builder *b, int n_solid)
{
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(*m));
    m->n_vert = b->n_vert; m->n_tri = b->n_tri; m->n_solid = n_solid;
    m->xyz = b->xyz; m->tri = b->tri; m->tri_solid = b->tri_solid;
    m->solid_material = (int *)calloc((size_t)n_solid, sizeof(int));
    m->solid_active = (int *)calloc((size_t)n_solid, sizeof(int));
    m->solid_group = (int *)calloc((size_t)n_solid, sizeof(int));
    m->solid_parent = (int *)calloc((size_t)n_solid, sizeof(int));
    return m;
}

static void set_solid(orc_mesh *m, int s, int mat, int active, int group, int parent)
{
    m->solid_material[s] = mat; m->solid_active[s] = active;
    m->solid_group[s] = group; m->solid_parent[s] = parent;
}

int orc_mesh_build(const orc_detparams *p, orc_mesh **out)
{
    builder b;
    memset(&b, 0, sizeof(b));
    int N = p->n_theta, nphi = p->n_phi, zs = p->z_slices < 1 ? 1 : p->z_slices;
    double sep = p->sep_delta;
    *out = NULL;
    if (N < 3 || nphi < 1) return -1;
    if (p->kind == ORC_DET_BARE_CYLINDER) {
        double R = p->D[1], L = p->D[0], rch = p->D[2];
        add_rounded(&b, 0, R, rch, 0.0, -L, N, nphi, zs);
        int n_solid = 1;
        if (p->has_source_solid) {
            double rho[4] = { 0.0, p->src_r, p->src_r, 0.0 };
            double z[4] = { p->src_z0 + p->src_h, p->src_z0 + p->src_h, p->src_z0, p->src_z0 };
            revolve(&b, 1, rho, z, 4, p->src_n_sides);
            n_solid = 2;
        }
        orc_mesh *m = finish(&b, n_solid);
        set_solid(m, 0, ORC_MAT_GE, 1, 2, -1);
        if (n_solid == 2) set_solid(m, 1, ORC_MAT_WATER, 0, 3, -1);
        *out = m;
        return 0;
    }
    if (p->kind != ORC_DET_COAX) return -1;
    const double *d = p->d, *D = p->D;
    double z_front = -(d[1] + d[4]);
    double z_back = z_front - D[0];
    /* 0 endcap, 1 endcap vacuum */
    add_rounded(&b, 0, d[0], 0.0, 0.0, -d[6], N, nphi, 1);
    add_rounded(&b, 1, d[0] - d[2], 0.0, -d[1], -d[6] + d[8], N, nphi, 1);
    /* 2 holder cup */
    double r_in = D[1] + d[5];
    add_cup(&b, 2, r_in, r_in + d[3], z_front - p->cup_rim_drop, -d[7] + d[9], -d[7], N);
    /* 3 crystal, 4 active (Eq. R_active = D2 - D4, L_active = D1 - D4) */
    double gi = p->groove_r - 0.5 * p->groove_w, go = p->groove_r + 0.5 * p->groove_w;
    double gd = p->groove_d > 0.0 ? p->groove_d : 0.0;
    add_rounded_g(&b, 3, D[1], D[2], z_front, z_back, N, nphi, zs, gi, go, gd);
    double rch_a = D[2] - D[3] > 0.0 ? D[2] - D[3] : 0.0;
    add_rounded_g(&b, 4, D[1] - D[3], rch_a, z_front - D[3], z_back + 1.0 * sep, N, nphi, zs, gi - sep, go + sep, gd);
    /* 5 bore contact, 6 bore vacuum: blind end toward the front, depth from the back face */
    double rc = D[5] + D[6];
    add_rounded(&b, 5, rc, rc, z_back + D[4] + D[6], z_back + 2.0 * sep, N, nphi, 1);
    add_rounded(&b, 6, D[5], D[5], z_back + D[4], z_back + 3.0 * sep, N, nphi, 1);
    int n_solid = 7, src_solid = -1, flange_solid = -1;
    if (p->has_source_solid) {
        double rho[4] = { 0.0, p->src_r, p->src_r, 0.0 };
        double z[4] = { p->src_z0 + p->src_h, p->src_z0 + p->src_h, p->src_z0, p->src_z0 };
        src_solid = n_solid++;
        revolve(&b, src_solid, rho, z, 4, p->src_n_sides);
    }
    if (p->flange_h > 0.0) {
        flange_solid = n_solid++;
        if (add_flange(&b, flange_solid, p->flange_r_in, p->flange_r_out, p->flange_h, p->flange_z_top,
                       p->n_bolt_holes, p->bolt_n_sides, p->bolt_r, p->bolt_rc, N) != 0) {
            free(b.xyz); free(b.tri); free(b.tri_solid);
            return -1;
        }
    }
    orc_mesh *m = finish(&b, n_solid);
    set_solid(m, 0, ORC_MAT_AL, 0, 1, -1);
    set_solid(m, 1, ORC_MAT_VACUUM, 0, -1, 0);
    set_solid(m, 2, ORC_MAT_CU, 0, -1, 1);
    set_solid(m, 3, ORC_MAT_GE, 0, 0, 1);
    set_solid(m, 4, ORC_MAT_GE, 1, 2, 3);
    set_solid(m, 5, ORC_MAT_GE, 0, -1, 4);
    set_solid(m, 6, ORC_MAT_VACUUM, 0, -1, 5);
    if (src_solid >= 0) set_solid(m, src_solid, ORC_MAT_WATER, 0, 3, -1);
    if (flange_solid >= 0) set_solid(m, flange_solid, ORC_MAT_CU, 0, -1, 1);
    *out = m;
    return 0;
}

orc_mesh *orc_mesh_from_arrays(int n_vert, const double *xyz, int n_tri, const int *tri,
                               const int *tri_solid, int n_solid, const int *material,
                               const int *active, const int *group, const int *parent)
{
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(*m));
    m->n_vert = n_vert; m->n_tri = n_tri; m->n_solid = n_solid;
    m->xyz = (double *)malloc((size_t)n_vert * 3 * sizeof(double));
    memcpy(m->xyz, xyz, (size_t)n_vert * 3 * sizeof(double));
    m->tri = (int *)malloc((size_t)n_tri * 3 * sizeof(int));
    memcpy(m->tri, tri, (size_t)n_tri * 3 * sizeof(int));
    m->tri_solid = (int *)malloc((size_t)n_tri * sizeof(int));
    memcpy(m->tri_solid, tri_solid, (size_t)n_tri * sizeof(int));
    m->solid_material = (int *)malloc((size_t)n_solid * sizeof(int));
    m->solid_active = (int *)malloc((size_t)n_solid * sizeof(int));
    m->solid_group = (int *)malloc((size_t)n_solid * sizeof(int));
    m->solid_parent = (int *)malloc((size_t)n_solid * sizeof(int));
    memcpy(m->solid_material, material, (size_t)n_solid * sizeof(int));
    memcpy(m->solid_active, active, (size_t)n_solid * sizeof(int));
    memcpy(m->solid_group, group, (size_t)n_solid * sizeof(int));
    memcpy(m->solid_parent, parent, (size_t)n_solid * sizeof(int));
    return m;
}

void orc_mesh_free(orc_mesh *m)
{
    if (!m) return;
    free(m->xyz); free(m->tri); free(m->tri_solid);
    free(m->solid_material); free(m->solid_active); free(m->solid_group); free(m->solid_parent);
    free(m);
}

double orc_mesh_volume(const orc_mesh *m, int solid)
{
    double v = 0.0;
    for (int t = 0; t < m->n_tri; ++t) {
        if (m->tri_solid[t] != solid) continue;
        const double *a = m->xyz + 3 * m->tri[3 * t];
        const double *b = m->xyz + 3 * m->tri[3 * t + 1];
        const double *c = m->xyz + 3 * m->tri[3 * t + 2];
        /* a . (b x c) / 6 */
        v += (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
              a[2] * (b[0] * c[1] - b[1] * c[0])) / 6.0;
    }
    return v;
}

double orc_mesh_area(const orc_mesh *m, int solid)
{
    double s = 0.0;
    for (int t = 0; t < m->n_tri; ++t) {
        if (m->tri_solid[t] != solid) continue;
        const double *a = m->xyz + 3 * m->tri[3 * t];
        const double *b = m->xyz + 3 * m->tri[3 * t + 1];
        const double *c = m->xyz + 3 * m->tri[3 * t + 2];
        double u[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
        double w[3] = { c[0] - a[0], c[1] - a[1], c[2] - a[2] };
        double n[3] = { u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0] };
        s += 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    }
    return s;
}

/* directed edges of one solid, as (from, to) pairs, plain O(E^2) matching */
static int solid_edges(const orc_mesh *m, int solid, int **out)
{
    int n = 0;
    for (int t = 0; t < m->n_tri; ++t) if (m->tri_solid[t] == solid) n += 3;
    int *e = (int *)malloc((size_t)(n > 0 ? n : 1) * 2 * sizeof(int));
    int k = 0;
    for (int t = 0; t < m->n_tri; ++t) {
        if (m->tri_solid[t] != solid) continue;
        for (int j = 0; j < 3; ++j) {
            e[2 * k] = m->tri[3 * t + j];
            e[2 * k + 1] = m->tri[3 * t + (j + 1) % 3];
            ++k;
        }
    }
    *out = e;
    return n;
}

static int cmp_pair(const void *a, const void *b)
{
    const int *x = (const int *)a, *y = (const int *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

int orc_mesh_open_edges(const orc_mesh *m, int solid)
{
    int *e;
    int n = solid_edges(m, solid, &e);
    qsort(e, (size_t)n, 2 * sizeof(int), cmp_pair);
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        /* each directed edge must be unique and its reverse must exist exactly once */
        if (i > 0 && e[2 * i] == e[2 * i - 2] && e[2 * i + 1] == e[2 * i - 1]) { ++bad; continue; }
        int key[2] = { e[2 * i + 1], e[2 * i] };
        void *hit = bsearch(key, e, (size_t)n, 2 * sizeof(int), cmp_pair);
        if (!hit) ++bad;
    }
    free(e);
    return bad;
}

int orc_mesh_euler(const orc_mesh *m, int solid)
{
    int *e;
    int n = solid_edges(m, solid, &e);
    int F = n / 3;
    /* undirected edges: normalise (min, max) and count unique */
    for (int i = 0; i < n; ++i) {
        if (e[2 * i] > e[2 * i + 1]) { int t = e[2 * i]; e[2 * i] = e[2 * i + 1]; e[2 * i + 1] = t; }
    }
    qsort(e, (size_t)n, 2 * sizeof(int), cmp_pair);
    int E = 0;
    for (int i = 0; i < n; ++i)
        if (i == 0 || e[2 * i] != e[2 * i - 2] || e[2 * i + 1] != e[2 * i - 1]) ++E;
    free(e);
    char *used = (char *)calloc((size_t)m->n_vert, 1);
    int V = 0;
    for (int t = 0; t < m->n_tri; ++t) {
        if (m->tri_solid[t] != solid) continue;
        for (int j = 0; j < 3; ++j) {
            int v = m->tri[3 * t + j];
            if (!used[v]) { used[v] = 1; ++V; }
        }
    }
    free(used);
    return V - E + F;
}
