/*
 * orc_transport.c -- oracle photon transport (test infrastructure only).
 *
 * One history = one source photon (plus the annihilation photon a pair
 * production leaves behind).  Steps, in the paper's terms:
 *   birth       position and isotropic direction from the source (Sec. 3.2);
 *   localization   the parity rule of Sec. 2.4.2 / Fig. 5: intersect the ray
 *               along the flight direction with every solid, a solid with an
 *               odd number of crossings contains the particle, the container
 *               is the odd solid whose first crossing is nearest, none = world;
 *   free flight the partial cross-section method of Sec. 2.4.1, read as: one
 *               number of mean free paths lambda = -ln u per flight, consumed
 *               region by region (lambda -= mu * length) until it runs out
 *               inside a region (interaction) or the photon leaves the mesh;
 *   interaction process chosen by partial attenuation coefficients,
 *               photoabsorption (deposit E), Compton (Kahn sampler, deposit
 *               E - E'), pair production (deposit E - 2 mc^2, two 511 keV
 *               photons back to back); charged particles deposit locally
 *               (e_model 0) or run continuous-slowing-down tracks (e_model 1,
 *               below);
 *   scoring     energy deposited in active solids is summed per history and
 *               binned; a history is in the full-energy peak when
 *               E0 - E_dep <= fep_delta (host scoring, Fig. 4).
 *
 * The ray of one flight is a single line, so its intersections with all
 * triangles are enumerated once per flight and reused for every segment and
 * every parity query along it (the same intersections the rule asks for).
 * At each crossing the oracle also evaluates the nesting-tree rule (entering
 * solid s -> s, leaving s -> parent of s) and counts disagreements.
 *
 * Charged-particle tracks (e_model 1; the stand-in for the paper's electron
 * and positron transport, stopping powers and ranges in orc_xs.c).  Each
 * interaction sets particles in motion: photoabsorption one electron of
 * T = E along the photon's direction (binding energy neglected, as in the
 * local deposit); Compton one electron of T = E - E' along E d - E' d'
 * (momentum conservation); pair production an electron and a positron of
 * T = (E - 2 mc^2) / 2 each, both along the photon's direction, so one line
 * carries twice the deposits (the annihilation photons still start at the
 * interaction point).  A particle with T < ORC_E_TMIN deposits at its birth
 * point in the photon's region.  Otherwise it runs straight ahead: the regions
 * along its line come from the same crossings and parity rule as a photon
 * flight; in each region it goes as far as its CSDA range (divided by the
 * region's density scale) allows, depositing T - T' where T' is what is left
 * at the next boundary; it stops when the range runs out (depositing the
 * rest there) or falls below ORC_E_TMIN (depositing the rest in the region it
 * has entered), and what leaves the mesh escapes.  Vacuum takes no energy.
 * The tracks draw no random numbers, so the photon histories are the same in
 * both models.
 *
 * Density-perturbation scores: with mu of every solid of group p scaled by
 * s_p, d ln(track probability)/d s_p = (collisions in p)/s_p
 *                                     - sum over segments in p of mu_unit * length.
 */
#include "oracle.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI   3.14159265358979323846
#define ORC_MEC2 510.99895
#define MAX_SOLIDS 64

typedef struct {
    uint32_t key[2], ctr[4], buf[4];
    int idx;
} rng_t;

static void rng_init(rng_t *r, uint64_t seed, uint64_t hid, uint32_t inst)
{
    r->key[0] = (uint32_t)seed; r->key[1] = (uint32_t)(seed >> 32);
    r->ctr[0] = 0; r->ctr[1] = (uint32_t)hid; r->ctr[2] = (uint32_t)(hid >> 32); r->ctr[3] = inst;
    r->idx = 4;
}

static double rng_u(rng_t *r)
{
    if (r->idx == 4) {
        orc_philox4x32_10(r->ctr, r->key, r->buf);
        r->ctr[0]++;
        r->idx = 0;
    }
    return orc_u01(r->buf[r->idx++]);
}

/* ---------- geometry ---------- */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Line through o along d against triangle (a, b, c): the three edge volumes
   d . ((p - o) x (q - o)) over the directed edges (a,b), (b,c), (c,a) must
   not have opposite signs.  A shared edge is evaluated with its two endpoints
   swapped by the neighbour, which negates the value exactly, so a line never
   slips between two triangles.  t from the plane of the triangle. */
static int ray_tri(const double *o, const double *d, const double *a, const double *b,
                   const double *c, double *t, int *entering)
{
    double pa[3] = { a[0] - o[0], a[1] - o[1], a[2] - o[2] };
    double pb[3] = { b[0] - o[0], b[1] - o[1], b[2] - o[2] };
    double pc[3] = { c[0] - o[0], c[1] - o[1], c[2] - o[2] };
    double x[3];
    cross3(pa, pb, x); double e0 = dot3(d, x);
    cross3(pb, pc, x); double e1 = dot3(d, x);
    cross3(pc, pa, x); double e2 = dot3(d, x);
    int pos = (e0 >= 0 && e1 >= 0 && e2 >= 0), neg = (e0 <= 0 && e1 <= 0 && e2 <= 0);
    if (!pos && !neg) return 0;
    if (e0 == 0 && e1 == 0 && e2 == 0) return 0;
    double u[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
    double w[3] = { c[0] - a[0], c[1] - a[1], c[2] - a[2] };
    double n[3];
    cross3(u, w, n);
    double dn = dot3(d, n);
    if (dn == 0) return 0;
    *t = dot3(pa, n) / dn;
    *entering = dn < 0;
    return 1;
}

typedef struct { double t; int tri, solid, entering; } hit_t;

typedef struct {
    const orc_mesh *m;
    double (*box)[6];    /* per-solid AABB */
    int *order;          /* triangles grouped by solid */
    int *start;          /* [n_solid + 1] */
} scene_t;

static void scene_init(scene_t *s, const orc_mesh *m)
{
    s->m = m;
    s->box = (double (*)[6])malloc((size_t)(m->n_solid > 0 ? m->n_solid : 1) * sizeof(*s->box));
    s->start = (int *)calloc((size_t)m->n_solid + 1, sizeof(int));
    s->order = (int *)malloc((size_t)(m->n_tri > 0 ? m->n_tri : 1) * sizeof(int));
    for (int i = 0; i < m->n_solid; ++i) {
        s->box[i][0] = s->box[i][1] = s->box[i][2] = INFINITY;
        s->box[i][3] = s->box[i][4] = s->box[i][5] = -INFINITY;
    }
    for (int t = 0; t < m->n_tri; ++t) s->start[m->tri_solid[t] + 1]++;
    for (int i = 0; i < m->n_solid; ++i) s->start[i + 1] += s->start[i];
    int *fill = (int *)calloc((size_t)m->n_solid, sizeof(int));
    for (int t = 0; t < m->n_tri; ++t) {
        int so = m->tri_solid[t];
        s->order[s->start[so] + fill[so]++] = t;
        for (int j = 0; j < 3; ++j) {
            const double *v = m->xyz + 3 * m->tri[3 * t + j];
            for (int k = 0; k < 3; ++k) {
                if (v[k] < s->box[so][k]) s->box[so][k] = v[k];
                if (v[k] > s->box[so][3 + k]) s->box[so][3 + k] = v[k];
            }
        }
    }
    free(fill);
    for (int i = 0; i < m->n_solid; ++i)
        for (int k = 0; k < 3; ++k) { s->box[i][k] -= 1e-6; s->box[i][3 + k] += 1e-6; }
}

static void scene_free(scene_t *s)
{
    free(s->box); free(s->start); free(s->order);
}

static int ray_box(const double *o, const double *d, const double *b)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < b[k] || o[k] > b[3 + k]) return 0;
            continue;
        }
        double a = (b[k] - o[k]) / d[k], c = (b[3 + k] - o[k]) / d[k];
        if (a > c) { double x = a; a = c; c = x; }
        if (a > t0) t0 = a;
        if (c < t1) t1 = c;
        if (t0 > t1) return 0;
    }
    return 1;
}

static int cmp_hit(const void *a, const void *b)
{
    const hit_t *x = (const hit_t *)a, *y = (const hit_t *)b;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    if (x->solid != y->solid) return x->solid < y->solid ? -1 : 1;
    return x->tri < y->tri ? -1 : (x->tri > y->tri);
}

/* All crossings t > 0 of the ray, sorted; same-solid same-orientation hits at
   the same point (a line through a shared edge or vertex) count once. */
static int collect_hits(const scene_t *s, const double *o, const double *d, hit_t **buf, int *cap,
                        uint64_t *n_dup)
{
    const orc_mesh *m = s->m;
    int n = 0;
    for (int so = 0; so < m->n_solid; ++so) {
        if (!ray_box(o, d, s->box[so])) continue;
        for (int k = s->start[so]; k < s->start[so + 1]; ++k) {
            int t = s->order[k];
            double th; int ent;
            const double *a = m->xyz + 3 * m->tri[3 * t];
            const double *b = m->xyz + 3 * m->tri[3 * t + 1];
            const double *c = m->xyz + 3 * m->tri[3 * t + 2];
            if (!ray_tri(o, d, a, b, c, &th, &ent) || !(th > 0.0)) continue;
            if (n == *cap) {
                *cap = *cap ? 2 * *cap : 64;
                *buf = (hit_t *)realloc(*buf, (size_t)*cap * sizeof(hit_t));
            }
            (*buf)[n].t = th; (*buf)[n].tri = t; (*buf)[n].solid = so; (*buf)[n].entering = ent;
            ++n;
        }
    }
    hit_t *h = *buf;
    if (n > 1) qsort(h, (size_t)n, sizeof(hit_t), cmp_hit);     /* h is NULL before the first hit */
    int w = 0;
    for (int i = 0; i < n; ++i) {
        int dup = 0;
        for (int j = w - 1; j >= 0 && h[i].t - h[j].t <= 1e-9 * (1.0 + h[i].t); --j) {
            if (h[j].solid == h[i].solid && h[j].entering == h[i].entering) { dup = 1; break; }
        }
        if (dup) { (*n_dup)++; continue; }
        h[w++] = h[i];
    }
    return w;
}

/* parity rule using the crossings h[from..n) that lie ahead of the particle */
static int parity_region(const hit_t *h, int from, int n, int n_solid)
{
    int count[MAX_SOLIDS];
    double first[MAX_SOLIDS];
    for (int i = 0; i < n_solid; ++i) { count[i] = 0; first[i] = INFINITY; }
    for (int i = from; i < n; ++i) {
        count[h[i].solid]++;
        if (h[i].t < first[h[i].solid]) first[h[i].solid] = h[i].t;
    }
    int best = -1;
    double bt = INFINITY;
    for (int i = 0; i < n_solid; ++i)
        if ((count[i] & 1) && first[i] < bt) { bt = first[i]; best = i; }
    return best;
}

int orc_locate(const orc_mesh *m, const double p[3], const double dir[3])
{
    scene_t s;
    scene_init(&s, m);
    hit_t *buf = NULL; int cap = 0; uint64_t nd = 0;
    int n = collect_hits(&s, p, dir, &buf, &cap, &nd);
    int r = parity_region(buf, 0, n, m->n_solid);
    free(buf);
    scene_free(&s);
    return r;
}

int orc_nearest_hit(const orc_mesh *m, const double o[3], const double d[3], double t_min,
                    int exclude, double *t, int *entering)
{
    int best = -1;
    double bt = INFINITY;
    int be = 0;
    for (int k = 0; k < m->n_tri; ++k) {
        if (k == exclude) continue;
        double th; int ent;
        const double *a = m->xyz + 3 * m->tri[3 * k];
        const double *b = m->xyz + 3 * m->tri[3 * k + 1];
        const double *c = m->xyz + 3 * m->tri[3 * k + 2];
        if (!ray_tri(o, d, a, b, c, &th, &ent)) continue;
        if (th > t_min && th < bt) { bt = th; best = k; be = ent; }
    }
    *t = bt;
    *entering = be;
    return best;
}

/* ---------- sampling ---------- */

static void iso_dir(rng_t *r, double d[3])
{
    double c = 2.0 * rng_u(r) - 1.0;
    double phi = 2.0 * ORC_PI * rng_u(r);
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    d[0] = s * cos(phi); d[1] = s * sin(phi); d[2] = c;
}

static void birth(const orc_source *src, rng_t *r, double pos[3], double dir[3])
{
    memcpy(pos, src->pos, 3 * sizeof(double));
    if (src->kind == ORC_SRC_DISK) {
        double rr = src->radius * sqrt(rng_u(r));
        double phi = 2.0 * ORC_PI * rng_u(r);
        pos[0] += rr * cos(phi); pos[1] += rr * sin(phi);
    } else if (src->kind == ORC_SRC_PRISM) {
        /* fan triangle k of the regular polygon, uniform point inside it */
        int N = src->n_sides;
        int k = (int)floor(N * rng_u(r));
        if (k >= N) k = N - 1;
        double s1 = sqrt(rng_u(r)), u3 = rng_u(r);
        double a0 = 2.0 * ORC_PI * k / N, a1 = 2.0 * ORC_PI * ((k + 1) % N) / N;
        double bx = src->radius * cos(a0), by = src->radius * sin(a0);
        double cx = src->radius * cos(a1), cy = src->radius * sin(a1);
        pos[0] += s1 * (1.0 - u3) * bx + s1 * u3 * cx;
        pos[1] += s1 * (1.0 - u3) * by + s1 * u3 * cy;
        pos[2] += src->height * rng_u(r);
    }
    if (src->kind == ORC_SRC_PENCIL) {
        memcpy(dir, src->dir, 3 * sizeof(double));
    } else {
        iso_dir(r, dir);
    }
}

void orc_sample_birth(const orc_source *s, uint64_t seed, uint64_t hid, uint32_t inst,
                      double pos[3], double dir[3])
{
    rng_t r;
    rng_init(&r, seed, hid, inst);
    birth(s, &r, pos, dir);
}

/* Kahn's rejection method for x = E/E' in [1, 1 + 2k] (Everett & Cashwell). */
static int kahn(rng_t *r, double k, double *x_out)
{
    for (int trial = 0; trial < 1000; ++trial) {
        double r1 = rng_u(r), r2 = rng_u(r), r3 = rng_u(r);
        if (r1 <= (1.0 + 2.0 * k) / (9.0 + 2.0 * k)) {
            double x = 1.0 + 2.0 * k * r2;
            if (r3 <= 4.0 * (1.0 / x - 1.0 / (x * x))) { *x_out = x; return 0; }
        } else {
            double x = (1.0 + 2.0 * k) / (1.0 + 2.0 * k * r2);
            double c = 1.0 - (x - 1.0) / k;
            if (r3 <= 0.5 * (c * c + 1.0 / x)) { *x_out = x; return 0; }
        }
    }
    return -1;
}

int orc_kahn_samples(double k, uint64_t seed, int n, double *x_out)
{
    for (int i = 0; i < n; ++i) {
        rng_t r;
        rng_init(&r, seed, (uint64_t)i, 0u);
        if (kahn(&r, k, &x_out[i]) != 0) return -1;
    }
    return 0;
}

/* new direction at polar angle acos(c) and azimuth phi about d */
static void rotate(double d[3], double c, double phi)
{
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    double cp = cos(phi), sp = sin(phi);
    double r = sqrt(d[0] * d[0] + d[1] * d[1]);
    double n[3];
    if (r < 1e-9) {
        n[0] = s * cp; n[1] = s * sp; n[2] = d[2] > 0 ? c : -c;
    } else {
        n[0] = d[0] * c + s * (d[0] * d[2] * cp - d[1] * sp) / r;
        n[1] = d[1] * c + s * (d[1] * d[2] * cp + d[0] * sp) / r;
        n[2] = d[2] * c - s * r * cp;
    }
    double l = sqrt(dot3(n, n));
    d[0] = n[0] / l; d[1] = n[1] / l; d[2] = n[2] / l;
}

/* ---------- one history ---------- */

typedef struct {
    const scene_t *sc;
    const orc_tables *xs;
    const orc_source *src;
    const orc_opts *o;
    hit_t *buf; int cap;
    hit_t *ebuf; int ecap;      /* crossings of a charged-particle line */
} ctx_t;

typedef struct { double edep; int fep, err; } hist_out;

#define ORC_E_MAX_CROSSINGS 256

/* One charged-particle line: `weight` particles of kinetic energy T each from
   p along unit u, born in the photon's region `region0`.  Adds the deposits to
   edep (active regions) and dep_all, what leaves the mesh to esc.  Returns
   nonzero on a geometry error. */
static int e_track(ctx_t *cx, const double p[3], const double u[3], double T, double weight, int region0,
                   double *edep, double *dep_all, double *esc)
{
    const orc_mesh *m = cx->sc->m;
    const orc_opts *o = cx->o;
    if (T < ORC_E_TMIN) {
        *dep_all += weight * T;
        if (region0 >= 0 && m->solid_active[region0]) *edep += weight * T;
        return 0;
    }
    uint64_t dup = 0;
    int n = collect_hits(cx->sc, p, u, &cx->ebuf, &cx->ecap, &dup);
    const hit_t *h = cx->ebuf;
    int region = parity_region(h, 0, n, m->n_solid);
    double t_cur = 0.0;
    for (int i = 0; i <= ORC_E_MAX_CROSSINGS; ++i) {
        int active = region >= 0 && m->solid_active[region];
        if (T < ORC_E_TMIN) {
            *dep_all += weight * T;
            if (active) *edep += weight * T;
            return 0;
        }
        int mat = region >= 0 ? m->solid_material[region] : 0;
        int grp = region >= 0 ? m->solid_group[region] : -1;
        double sc = (grp >= 0 && grp < o->n_group) ? o->group_scale[grp] : 1.0;
        double reach = orc_e_range(cx->xs, mat, T) / sc;
        double t_next = i < n ? h[i].t : INFINITY;
        if (reach < INFINITY && t_next - t_cur >= reach) {   /* stops in this region */
            *dep_all += weight * T;
            if (active) *edep += weight * T;
            return 0;
        }
        if (i == n) {                            /* leaves the mesh (only through vacuum) */
            if (region != -1) return 1;
            *esc += weight * T;
            return 0;
        }
        double T2 = orc_e_energy_after(cx->xs, mat, T, (t_next - t_cur) * sc);
        *dep_all += weight * (T - T2);
        if (active) *edep += weight * (T - T2);
        T = T2;
        t_cur = t_next;
        region = parity_region(h, i + 1, n, m->n_solid);
    }
    return 1;
}

static void run_history(ctx_t *cx, uint64_t hid, orc_tally *T, uint32_t *spec, hist_out *ho)
{
    const orc_mesh *m = cx->sc->m;
    const orc_opts *o = cx->o;
    rng_t r;
    rng_init(&r, o->seed, hid, o->instance);
    double pos[3], dir[3];
    birth(cx->src, &r, pos, dir);
    double E = o->energy_keV, E0 = o->energy_keV;
    double edep = 0.0, dep_all = 0.0, esc = 0.0;
    double score[8] = { 0 };
    int err = 0, segs = 0, first_done = 0;
    int carried = -2;                  /* region carried along by the tree rule; -2 = unknown */
    int has_sec = 0;
    double sec_pos[3], sec_dir[3];
    int sec_region = -1;
    int alive = 1;
    while (alive && !err) {
        /* ---- one flight ---- */
        int n = collect_hits(cx->sc, pos, dir, &cx->buf, &cx->cap, &T->n_dup_hits);
        hit_t *h = cx->buf;
        T->n_flights++;
        int region = parity_region(h, 0, n, m->n_solid);
        if (carried != -2 && carried != region) T->n_parity_mismatch++;
        double lam = -log(rng_u(&r));
        double t_cur = 0.0;
        int i = 0;
        int flight_over = 0;
        while (!flight_over) {
            if (++segs > o->step_cap) { err = 1; break; }
            T->n_segments++;
            double t_next = i < n ? h[i].t : INFINITY;
            int mat = region >= 0 ? m->solid_material[region] : 0;
            int grp = region >= 0 ? m->solid_group[region] : -1;
            double sc = (grp >= 0 && grp < o->n_group) ? o->group_scale[grp] : 1.0;
            double mu3[3] = { 0, 0, 0 };
            if (mat != 0) orc_tables_eval(cx->xs, mat, E, mu3);
            double mu_unit = mu3[0] + mu3[1] + mu3[2];
            double mu = mu_unit * sc;
            if (mu > 0.0) {
                double d_int = lam / mu;
                if (d_int < t_next - t_cur) {
                    /* ---- interaction ---- */
                    if (grp >= 0 && grp < o->n_group) score[grp] += 1.0 / sc - mu_unit * d_int;
                    double tt = t_cur + d_int;
                    double p[3] = { pos[0] + tt * dir[0], pos[1] + tt * dir[1], pos[2] + tt * dir[2] };
                    T->n_interactions++;
                    int active = region >= 0 && m->solid_active[region];
                    double u = rng_u(&r) * mu_unit;
                    int proc;
                    if (u < mu3[0]) proc = 0;
                    else if (u < mu3[0] + mu3[1] || mu3[2] == 0.0) proc = 1;
                    else proc = 2;
                    if (!first_done) {
                        first_done = 1;
                        if (proc == 0) T->n_first_pe++;
                        else if (proc == 1) T->n_first_compton++;
                        else T->n_first_pair++;
                    }
                    double dep = 0.0;
                    /* charged particles of e_model 1: kinetic energy, direction, count */
                    double eT = 0.0, eu[3] = { dir[0], dir[1], dir[2] }, ew = 1.0;
                    if (proc == 0) {
                        if (o->e_model) eT = E;
                        else dep = E;
                        E = 0.0; alive = 0;
                    } else if (proc == 1) {
                        double k = E / ORC_MEC2, x;
                        if (kahn(&r, k, &x) != 0) { err = 1; break; }
                        double c = 1.0 - (x - 1.0) / k;
                        double phi = 2.0 * ORC_PI * rng_u(&r);
                        double Ep = E / x;
                        rotate(dir, c, phi);
                        if (o->e_model) {
                            eT = E - Ep;
                            double q[3] = { E * eu[0] - Ep * dir[0], E * eu[1] - Ep * dir[1], E * eu[2] - Ep * dir[2] };
                            double ql = sqrt(dot3(q, q));
                            if (ql > 0.0) { eu[0] = q[0] / ql; eu[1] = q[1] / ql; eu[2] = q[2] / ql; }
                        } else {
                            dep = E - Ep;
                        }
                        E = Ep;
                        if (E < o->e_cut_keV) { dep += E; E = 0.0; alive = 0; }
                    } else {
                        if (o->e_model) { eT = 0.5 * (E - 2.0 * ORC_MEC2); ew = 2.0; }
                        else dep = E - 2.0 * ORC_MEC2;
                        double nd[3];
                        iso_dir(&r, nd);
                        E = ORC_MEC2;
                        memcpy(dir, nd, sizeof(nd));
                        has_sec = 1;
                        memcpy(sec_pos, p, sizeof(p));
                        sec_dir[0] = -nd[0]; sec_dir[1] = -nd[1]; sec_dir[2] = -nd[2];
                        sec_region = region;
                    }
                    dep_all += dep;
                    if (active) edep += dep;
                    if (eT > 0.0 && e_track(cx, p, eu, eT, ew, region, &edep, &dep_all, &esc) != 0) { err = 1; break; }
                    memcpy(pos, p, sizeof(p));
                    carried = region;
                    flight_over = 1;
                    break;
                }
            }
            if (i == n) {
                /* leaves the mesh: only possible from the world region */
                if (region != -1) { err = 1; break; }
                esc += E; E = 0.0; alive = 0;
                flight_over = 1;
                break;
            }
            double len = t_next - t_cur;
            lam -= mu * len;
            if (grp >= 0 && grp < o->n_group) score[grp] -= mu_unit * len;
            t_cur = t_next;
            int tree = h[i].entering ? h[i].solid : m->solid_parent[h[i].solid];
            ++i;
            region = parity_region(h, i, n, m->n_solid);
            if (tree != region) T->n_parity_mismatch++;
            T->n_crossings++;
        }
        if (!alive && !err && has_sec) {
            has_sec = 0;
            memcpy(pos, sec_pos, sizeof(sec_pos));
            memcpy(dir, sec_dir, sizeof(sec_dir));
            E = ORC_MEC2;
            carried = sec_region;
            alive = 1;
        }
    }
    if (!first_done) T->n_first_none++;
    T->n_hist++;
    if (err) {
        T->n_err++;
        ho->edep = edep; ho->fep = 0; ho->err = 1;
        return;
    }
    double rel = fabs(dep_all + esc - E0) / E0;
    if (rel > T->max_rel_energy_err) T->max_rel_energy_err = rel;
    T->sum_dep_active += edep; T->sum_dep_all += dep_all; T->sum_esc += esc;
    int fep = (E0 - edep) <= o->fep_delta_keV;
    if (fep) {
        T->n_fep++;
        for (int g = 0; g < o->n_group && g < 8; ++g) {
            T->fep_score[g] += score[g];
            T->fep_score_sq[g] += score[g] * score[g];
        }
    }
    if (edep == 0.0) T->n_zero++;
    else if (edep >= o->e_max_keV) T->n_over++;
    else if (spec) {
        long b = (long)floor(edep / (o->e_max_keV / o->n_bins));
        if (b >= o->n_bins) b = o->n_bins - 1;
        spec[b]++;
    }
    ho->edep = edep; ho->fep = fep; ho->err = 0;
}

int orc_e_track(const orc_mesh *m, const orc_tables *t, const orc_opts *o, const double p[3], const double u[3],
                double T_keV, double weight, int region, double out[3])
{
    if (!m || !t || !o || !out || t->e_n < 2 || m->n_solid > MAX_SOLIDS) return -1;
    scene_t sc;
    scene_init(&sc, m);
    ctx_t cx = { &sc, t, NULL, o, NULL, 0, NULL, 0 };
    out[0] = out[1] = out[2] = 0.0;
    int rc = e_track(&cx, p, u, T_keV, weight, region, &out[0], &out[1], &out[2]);
    free(cx.buf);
    free(cx.ebuf);
    scene_free(&sc);
    return rc;
}

/* ---------- threads ---------- */

typedef struct {
    const orc_mesh *m; const scene_t *sc; const orc_tables *xs; const orc_source *src;
    const orc_opts *o;
    uint64_t n_hist; int tid, n_threads;
    orc_tally T; uint32_t *spec; double *edep;
} job_t;

static void *worker(void *arg)
{
    job_t *j = (job_t *)arg;
    ctx_t cx = { j->sc, j->xs, j->src, j->o, NULL, 0, NULL, 0 };
    const uint64_t block = 256;
    for (uint64_t b0 = (uint64_t)j->tid * block; b0 < j->n_hist; b0 += (uint64_t)j->n_threads * block) {
        uint64_t b1 = b0 + block < j->n_hist ? b0 + block : j->n_hist;
        for (uint64_t i = b0; i < b1; ++i) {
            hist_out ho;
            run_history(&cx, j->o->history_offset + i, &j->T, j->spec, &ho);
            if (j->edep) j->edep[i] = ho.edep;
        }
    }
    free(cx.buf);
    free(cx.ebuf);
    return NULL;
}

int orc_transport(const orc_mesh *m, const orc_tables *t, const orc_source *src,
                  const orc_opts *o, uint64_t n_hist, int n_threads,
                  orc_tally *out, uint32_t *spectrum, double *edep)
{
    if (!m || !t || !src || !o || !out || n_threads < 1 || m->n_solid > MAX_SOLIDS) return -1;
    if (o->n_group > 8 || o->n_bins < 1 || o->step_cap < 1) return -1;
    if (o->e_model != 0 && (o->e_model != 1 || t->e_n < 2)) return -1;
    for (int s = 0; s < m->n_solid; ++s)
        if (m->solid_material[s] < 0 || m->solid_material[s] >= t->n_mat) return -1;
    memset(out, 0, sizeof(*out));
    if (spectrum) memset(spectrum, 0, (size_t)o->n_bins * sizeof(uint32_t));
    scene_t sc;
    scene_init(&sc, m);
    job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].m = m; jobs[i].sc = &sc; jobs[i].xs = t; jobs[i].src = src; jobs[i].o = o;
        jobs[i].n_hist = n_hist; jobs[i].tid = i; jobs[i].n_threads = n_threads;
        jobs[i].spec = spectrum ? (uint32_t *)calloc((size_t)o->n_bins, sizeof(uint32_t)) : NULL;
        jobs[i].edep = edep;
        pthread_create(&th[i], NULL, worker, &jobs[i]);
    }
    for (int i = 0; i < n_threads; ++i) {
        pthread_join(th[i], NULL);
        orc_tally *T = &jobs[i].T;
        out->n_hist += T->n_hist; out->n_fep += T->n_fep; out->n_zero += T->n_zero;
        out->n_over += T->n_over; out->n_err += T->n_err;
        out->n_parity_mismatch += T->n_parity_mismatch; out->n_dup_hits += T->n_dup_hits;
        out->n_segments += T->n_segments; out->n_interactions += T->n_interactions;
        out->n_crossings += T->n_crossings; out->n_flights += T->n_flights;
        out->n_first_pe += T->n_first_pe; out->n_first_compton += T->n_first_compton;
        out->n_first_pair += T->n_first_pair; out->n_first_none += T->n_first_none;
        out->sum_dep_active += T->sum_dep_active; out->sum_dep_all += T->sum_dep_all;
        out->sum_esc += T->sum_esc;
        if (T->max_rel_energy_err > out->max_rel_energy_err) out->max_rel_energy_err = T->max_rel_energy_err;
        for (int g = 0; g < 8; ++g) { out->fep_score[g] += T->fep_score[g]; out->fep_score_sq[g] += T->fep_score_sq[g]; }
        if (spectrum) {
            for (int b = 0; b < o->n_bins; ++b) spectrum[b] += jobs[i].spec[b];
            free(jobs[i].spec);
        }
    }
    free(jobs); free(th);
    scene_free(&sc);
    return 0;
}
