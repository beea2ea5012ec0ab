// detmesh.cpp -- DetMesh: parametric detector surfaces (paper Sec. 2.2-2.3).
//
// Structure follows the paper's framework (Fig. 1-2): a PhysicalGeometry
// assembles a detector from Geometry primitives; each primitive generates a
// triangulated surface in its own local frame and is mapped to the global frame
// by relocate (the paper's relocatemesh, stacking components along z).
//
// Local frame of the rounded ("bulletized") cylinder: the front face lies at
// z = Z_base = 0 and the body extends toward +z, which is the frame in which the
// paper writes the rounding vertices
//     phi_j = (pi/2) j / N_phi,  rho_j = (R - R_ch) + R_ch cos(phi_j),
//     z_j   = Z_base + R_ch (1 - sin(phi_j)),
//     x_ij  = rho_j cos(theta_i), y_ij = rho_j sin(theta_i), theta_i = 2 pi i / N_theta.
// relocate mirrors z (the detector looks toward +z in the global frame) and
// translates; every solid's orientation is then fixed by its signed volume so
// that normals n = (v1 - v0) x (v2 - v0) point outward (triprocess, Sec. 2.2.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>

#include "gadep_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Surface {
    std::vector<double> v;            // [n][3]
    std::vector<int32_t> f;           // [m][3]
    int add(double x, double y, double z)
    {
        v.push_back(x); v.push_back(y); v.push_back(z);
        return (int)(v.size() / 3 - 1);
    }
    void tri(int a, int b, int c) { f.push_back(a); f.push_back(b); f.push_back(c); }
};

// Geometry interface: surface generation in the primitive's local frame.
class Geometry {
public:
    virtual ~Geometry() = default;
    virtual Surface generate() const = 0;
};

// Ring of n_theta vertices at (rho, z), or a single axis vertex when rho == 0.
struct Ring { int first; bool axis; };

Ring make_ring(Surface &s, double rho, double z, int n_theta)
{
    if (rho == 0.0) return Ring{ s.add(0.0, 0.0, z), true };
    int first = (int)(s.v.size() / 3);
    for (int i = 0; i < n_theta; ++i) {
        double th = 2.0 * kPi * i / n_theta;
        s.add(rho * std::cos(th), rho * std::sin(th), z);
    }
    return Ring{ first, false };
}

// Triangles between ring P (n_p vertices from p0) and ring Q (n_q from q0), both
// starting at angle 0: walking around by angle, each step takes the ring whose
// next vertex comes first.  With n_p == n_q this is the quad band split along
// (P_i, Q_{i+1}), with the same orientation.
void merge_rings(Surface &s, int p0, int n_p, int q0, int n_q)
{
    int i = 0, j = 0;
    while (i < n_p || j < n_q) {
        const double tp = (double)(i + 1) / n_p, tq = (double)(j + 1) / n_q;
        if (j < n_q && (i == n_p || tq <= tp)) {
            s.tri(p0 + i % n_p, q0 + (j + 1) % n_q, q0 + j % n_q);
            ++j;
        } else {
            s.tri(p0 + i % n_p, p0 + (i + 1) % n_p, q0 + j % n_q);
            ++i;
        }
    }
}

// A flat disk face (axis vertex c and ring r of n vertices in one plane) as
// concentric rings instead of a fan of n slivers meeting at the centre: rings
// inward at a spacing of kDiskAspect times the arc between the outer ring's
// vertices, each with vertices in proportion to its radius (at least
// kDiskMinRing), and a small fan at the centre.  The same surface, without
// n triangles whose boxes all contain the centre.
constexpr double kDiskAspect = 4.0;
constexpr int kDiskMinRing = 8;

void flat_disk(Surface &s, int c, int r0, int n, bool centre_first)
{
    const double z = s.v[3 * (size_t)r0 + 2];
    const double R = std::hypot(s.v[3 * (size_t)r0], s.v[3 * (size_t)r0 + 1]);
    const double w = kDiskAspect * 2.0 * kPi * R / n;
    int prev = r0, n_prev = n;
    for (int k = 1;; ++k) {
        const double rho = R - k * w;
        const int m = std::max(kDiskMinRing, (int)std::lround(n * rho / R));
        if (rho < w || m >= n_prev) break;
        const int first = (int)(s.v.size() / 3);
        for (int i = 0; i < m; ++i) {
            const double th = 2.0 * kPi * i / m;
            s.add(rho * std::cos(th), rho * std::sin(th), z);
        }
        // the outer ring plays the role it has in stitch(): Q (second) when the
        // centre comes first in the profile, P (first) otherwise
        if (centre_first) merge_rings(s, first, m, prev, n_prev);
        else merge_rings(s, prev, n_prev, first, m);
        prev = first;
        n_prev = m;
    }
    for (int i = 0; i < n_prev; ++i) {
        const int j = (i + 1) % n_prev;
        if (centre_first) s.tri(c, prev + j, prev + i);
        else s.tri(prev + i, prev + j, c);
    }
}

// Band of quads between two consecutive rings (a fan if one is an axis vertex;
// a flat disk of concentric rings when the axis vertex and the ring lie in one
// plane).  Quads are split along the (a_i, b_{i+1}) diagonal.
void stitch(Surface &s, const Ring &a, const Ring &b, int n_theta)
{
    if (a.axis != b.axis) {
        const int c = a.axis ? a.first : b.first, r = a.axis ? b.first : a.first;
        if (s.v[3 * (size_t)c + 2] == s.v[3 * (size_t)r + 2]) {
            flat_disk(s, c, r, n_theta, a.axis);
            return;
        }
    }
    for (int i = 0; i < n_theta; ++i) {
        int j = (i + 1) % n_theta;
        if (!a.axis && !b.axis) {
            s.tri(a.first + i, a.first + j, b.first + j);
            s.tri(a.first + i, b.first + j, b.first + i);
        } else if (a.axis && !b.axis) {
            s.tri(a.first, b.first + j, b.first + i);
        } else if (!a.axis && b.axis) {
            s.tri(a.first + i, a.first + j, b.first);
        }
    }
}

// ChamferedCylinder: cylinder of radius R and length L with a front-edge
// rounding of radius r_ch (0 <= r_ch <= R).  r_ch == R closes the front with a
// hemisphere whose apex is a single vertex (the borehole end, Fig. 10).
// Optionally with an annular groove g_in < rho < g_out cut g_depth deep into the
// back face (the contact groove of a stress model).
class ChamferedCylinder : public Geometry {
public:
    ChamferedCylinder(double R, double r_ch, double L, int n_theta, int n_phi, int z_slices,
                      double g_in = 0.0, double g_out = 0.0, double g_depth = 0.0)
        : R_(R), rch_(r_ch), L_(L), nt_(n_theta), np_(n_phi), zs_(std::max(1, z_slices)),
          gi_(g_in), go_(g_out), gd_(g_depth) {}
    Surface generate() const override
    {
        Surface s;
        std::vector<Ring> rings;
        if (rch_ > 0.0) {
            const bool hemi = (rch_ == R_);
            if (!hemi) rings.push_back(make_ring(s, 0.0, 0.0, nt_));  // front face centre
            for (int j = np_; j >= 0; --j) {
                double phi = 0.5 * kPi * j / np_;
                double rho = (R_ - rch_) + rch_ * std::cos(phi);
                double z = rch_ * (1.0 - std::sin(phi));
                if (hemi && j == np_) rho = 0.0;  // apex
                rings.push_back(make_ring(s, rho, z, nt_));
            }
        } else {
            rings.push_back(make_ring(s, 0.0, 0.0, nt_));
            rings.push_back(make_ring(s, R_, 0.0, nt_));
        }
        const double z0 = rch_;
        for (int k = 1; k <= zs_; ++k) {
            double z = (k == zs_) ? L_ : z0 + (L_ - z0) * k / zs_;
            rings.push_back(make_ring(s, R_, z, nt_));
        }
        if (gd_ > 0.0) {
            rings.push_back(make_ring(s, go_, L_, nt_));
            rings.push_back(make_ring(s, go_, L_ - gd_, nt_));
            rings.push_back(make_ring(s, gi_, L_ - gd_, nt_));
            rings.push_back(make_ring(s, gi_, L_, nt_));
        }
        rings.push_back(make_ring(s, 0.0, L_, nt_));               // back face centre
        for (size_t k = 0; k + 1 < rings.size(); ++k) stitch(s, rings[k], rings[k + 1], nt_);
        return s;
    }
private:
    double R_, rch_, L_;
    int nt_, np_, zs_;
    double gi_, go_, gd_;
};

// Cup (crystal holder): open-topped hollow cylinder with a flat bottom.  Local
// frame: rim at z = 0, outer bottom at z = depth.
class Cup : public Geometry {
public:
    Cup(double r_in, double wall, double depth, double bottom, int n_theta)
        : ri_(r_in), w_(wall), h_(depth), b_(bottom), nt_(n_theta) {}
    Surface generate() const override
    {
        Surface s;
        const double ro = ri_ + w_;
        Ring inner_bottom_c = make_ring(s, 0.0, h_ - b_, nt_);
        Ring inner_bottom = make_ring(s, ri_, h_ - b_, nt_);
        Ring inner_rim = make_ring(s, ri_, 0.0, nt_);
        Ring outer_rim = make_ring(s, ro, 0.0, nt_);
        Ring outer_bottom = make_ring(s, ro, h_, nt_);
        Ring outer_bottom_c = make_ring(s, 0.0, h_, nt_);
        Ring seq[6] = { inner_bottom_c, inner_bottom, inner_rim, outer_rim, outer_bottom,
                        outer_bottom_c };
        for (int k = 0; k < 5; ++k) stitch(s, seq[k], seq[k + 1], nt_);
        return s;
    }
private:
    double ri_, w_, h_, b_;
    int nt_;
};

// Flange: flat ring r_in..r_out, thickness h (local z in [0, h]), with nh axial
// bolt holes (M-gon walls of circumradius rh) centred on radius rc, hole k at the
// middle of angular sector k.  Each face of a sector is a polygon with one hole;
// it is triangulated by zipping the sector boundary and the hole polygon in the
// sector's (radius, arc length) coordinates, where the boundary is a rectangle
// and both loops are star-shaped about the hole centre.  generate() fails (empty
// surface) if a triangle comes out with non-positive area in the plane.
class Flange : public Geometry {
public:
    Flange(double r_in, double r_out, double h, int nh, int M, double rh, double rc, int n_theta)
        : ri_(r_in), ro_(r_out), h_(h), nh_(nh), M_(M), rh_(rh), rc_(rc), nt_(n_theta) {}
    Surface generate() const override
    {
        Surface s;
        const int m = nt_ / nh_;
        // rings: inner / outer circle at the two faces; hole polygons at the two faces
        int ring[2][2];                          // [face][inner, outer]
        for (int f = 0; f < 2; ++f)
            for (int q = 0; q < 2; ++q) ring[f][q] = make_ring(s, q ? ro_ : ri_, f ? h_ : 0.0, nt_).first;
        std::vector<int> hole(2 * nh_);
        for (int k = 0; k < nh_; ++k) {
            const double tc = 2.0 * kPi * (k + 0.5) / nh_;
            const double cx = rc_ * std::cos(tc), cy = rc_ * std::sin(tc);
            for (int f = 0; f < 2; ++f) {
                hole[2 * k + f] = (int)(s.v.size() / 3);
                for (int j = 0; j < M_; ++j) {
                    const double a = tc + 2.0 * kPi * j / M_;
                    s.add(cx + rh_ * std::cos(a), cy + rh_ * std::sin(a), f ? h_ : 0.0);
                }
            }
        }
        // side walls, wound with outward normals (outer wall +r, inner wall and
        // hole walls toward their axes)
        for (int i = 0; i < nt_; ++i) {
            const int j = (i + 1) % nt_;
            s.tri(ring[0][1] + i, ring[0][1] + j, ring[1][1] + j);   // outer wall
            s.tri(ring[0][1] + i, ring[1][1] + j, ring[1][1] + i);
            s.tri(ring[0][0] + i, ring[1][0] + j, ring[0][0] + j);   // inner wall
            s.tri(ring[0][0] + i, ring[1][0] + i, ring[1][0] + j);
        }
        for (int k = 0; k < nh_; ++k) {
            const int t = hole[2 * k], u = hole[2 * k + 1];
            for (int j = 0; j < M_; ++j) {
                const int j1 = (j + 1) % M_;
                s.tri(t + j, u + j1, t + j1);
                s.tri(t + j, u + j, u + j1);
            }
        }
        // faces
        for (int f = 0; f < 2; ++f) {
            for (int k = 0; k < nh_; ++k) {
                const double tc = 2.0 * kPi * (k + 0.5) / nh_;
                // sector boundary counter-clockwise in the plane: outer arc forward,
                // radial edge in, inner arc backward, radial edge out
                std::vector<int> outer;
                for (int i = 0; i <= m; ++i) outer.push_back(ring[f][1] + (k * m + i) % nt_);
                for (int i = m; i >= 0; --i) outer.push_back(ring[f][0] + (k * m + i) % nt_);
                std::vector<int> inner;                              // hole, counter-clockwise
                for (int j = 0; j < M_; ++j) inner.push_back(hole[2 * k + f] + j);
                // polar angle about the hole centre in (radius - rc, rc * (theta - tc))
                auto ang = [&](int v) {
                    const double x = s.v[3 * v], y = s.v[3 * v + 1];
                    double th = std::atan2(y, x) - tc;
                    th -= 2.0 * kPi * std::floor((th + kPi) / (2.0 * kPi));
                    return std::atan2(rc_ * th, std::hypot(x, y) - rc_);
                };
                const int no = (int)outer.size(), ni = (int)inner.size();
                std::vector<double> ao(no), ai(ni);
                for (int i = 0; i < no; ++i) ao[i] = ang(outer[i]);
                for (int j = 0; j < ni; ++j) ai[j] = ang(inner[j]);
                const int o0 = (int)(std::min_element(ao.begin(), ao.end()) - ao.begin());
                const double ref = ao[o0];
                auto rel = [&](double a) { double d = a - ref; while (d < 0.0) d += 2.0 * kPi; return d; };
                int i0 = 0;
                for (int j = 1; j < ni; ++j)
                    if (rel(ai[j]) < rel(ai[i0])) i0 = j;
                int io = 0, ii = 0;
                while (io < no || ii < ni) {
                    const int oa = outer[(o0 + io) % no], ia = inner[(i0 + ii) % ni];
                    const double next_o = io + 1 <= no ? (io + 1 == no ? 2.0 * kPi : rel(ao[(o0 + io + 1) % no])) : 1e300;
                    const double next_i = ii + 1 <= ni ? rel(ai[(i0 + ii + 1) % ni]) + (ii + 1 == ni ? 2.0 * kPi : 0.0) : 1e300;
                    if (io < no && (ii >= ni || next_o <= next_i)) {
                        s.tri(oa, outer[(o0 + io + 1) % no], ia);
                        ++io;
                    } else {
                        s.tri(oa, inner[(i0 + ii + 1) % ni], ia);
                        ++ii;
                    }
                }
            }
        }
        // the zipper winds both faces counter-clockwise (normal +z); the face at
        // z = 0 bounds the solid from below, so its outward windings are reversed
        const size_t n_face = (size_t)nh_ * (size_t)(2 * m + 2 + M_) * 3;
        const size_t face0 = s.f.size() - 2 * n_face, face1 = s.f.size() - n_face;
        for (size_t t = face0; t < face1; t += 3) std::swap(s.f[t + 1], s.f[t + 2]);
        // every face triangle must have positive area in its face's winding
        for (size_t t = face0; t < s.f.size(); t += 3) {
            const double *a = &s.v[3 * s.f[t]], *b = &s.v[3 * s.f[t + 1]], *c = &s.v[3 * s.f[t + 2]];
            double cz = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
            if (t < face1) cz = -cz;
            if (!(cz > 0.0)) return Surface{};
        }
        return s;
    }
private:
    double ri_, ro_, h_;
    int nh_, M_;
    double rh_, rc_;
    int nt_;
};

// relocate (the paper's relocatemesh): global = (x, y, z_offset - z_local).
void relocate(Surface &s, double z_offset)
{
    for (size_t i = 2; i < s.v.size(); i += 3) s.v[i] = z_offset - s.v[i];
}

double signed_volume(const Surface &s)
{
    double v = 0.0;
    for (size_t t = 0; t < s.f.size(); t += 3) {
        const double *a = &s.v[3 * s.f[t]], *b = &s.v[3 * s.f[t + 1]], *c = &s.v[3 * s.f[t + 2]];
        v += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
             a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    return v / 6.0;
}

// Outward orientation: flip the winding when the signed volume is negative.
void orient_outward(Surface &s)
{
    if (signed_volume(s) < 0.0)
        for (size_t t = 0; t < s.f.size(); t += 3) std::swap(s.f[t + 1], s.f[t + 2]);
}

struct Assembly {
    gadep::MeshData m;
    void add(Surface s, const gadep_solid &attr)
    {
        orient_outward(s);
        const int32_t base = m.n_vert();
        const int32_t sid = m.n_solid();
        m.xyz.insert(m.xyz.end(), s.v.begin(), s.v.end());
        for (size_t t = 0; t < s.f.size(); t += 3) {
            for (int k = 0; k < 3; ++k) m.tri.push_back(base + s.f[t + k]);
            m.tri_solid.push_back(sid);
        }
        m.solids.push_back(attr);
    }
};

gadep_solid attr(int32_t material, int32_t active, int32_t group)
{
    return gadep_solid{ material, active, group, -1 };
}

// PhysicalGeometry: a detector type builds itself from the standard parameter array.
class PhysicalGeometry {
public:
    virtual ~PhysicalGeometry() = default;
    virtual gadep_status createGeometry(const detmesh_params &p, Assembly &out) const = 0;
};

void add_source_prism(const detmesh_params &p, Assembly &a)
{
    ChamferedCylinder prism(p.src_r, 0.0, p.src_h, p.src_n_sides, 1, 1);
    Surface s = prism.generate();
    relocate(s, p.src_z0 + p.src_h);  // front face (local z = 0) on top
    a.add(std::move(s), attr(GADEP_MAT_WATER, 0, 3));
}

class BareCylinderDetector : public PhysicalGeometry {
public:
    gadep_status createGeometry(const detmesh_params &p, Assembly &a) const override
    {
        const double L = p.D[0], R = p.D[1], rch = p.D[2];
        if (!(L > 0 && R > 0 && rch >= 0 && rch < R && rch <= L))
            return gadep::fail(GADEP_E_INVAL, "bare cylinder: need D1 > 0, D2 > 0, 0 <= D3 < D2");
        ChamferedCylinder crystal(R, rch, L, p.n_theta, p.n_phi, p.z_slices);
        Surface s = crystal.generate();
        relocate(s, 0.0);
        a.add(std::move(s), attr(GADEP_MAT_GE, 1, 2));
        if (p.has_source_solid) add_source_prism(p, a);
        return GADEP_OK;
    }
};

// Single-ended coaxial HPGe in an endcap with a crystal cup, built inside-out
// (Sec. 2.3.2): crystal and active volume, borehole with its contact layer,
// holder, endcap; then all components are relocated into the global frame.
class CoaxDetector : public PhysicalGeometry {
public:
    gadep_status createGeometry(const detmesh_params &p, Assembly &a) const override
    {
        const double *d = p.d, *D = p.D;
        for (int i = 0; i < 10; ++i)
            if (!(d[i] > 0)) return gadep::fail(GADEP_E_INVAL, "coax: d%d must be > 0", i + 1);
        for (int i = 0; i < 7; ++i)
            if (!(D[i] > 0) && i != 2)
                return gadep::fail(GADEP_E_INVAL, "coax: D%d must be > 0", i + 1);
        const double sep = p.sep_delta;
        if (!(sep > 0)) return gadep::fail(GADEP_E_INVAL, "coax: sep_delta must be > 0");
        // adaptive assembly: the crystal front follows the window and the top gap
        const double z_front = -(d[1] + d[4]);
        const double z_back = z_front - D[0];
        const double r_act = D[1] - D[3], l_act = D[0] - D[3];     // Eq. R_active, L_active
        const double rch_act = std::max(D[2] - D[3], 0.0);
        const double r_cup_in = D[1] + d[5];
        const double z_rim = z_front - p.cup_rim_drop;
        // geometric consistency (no overlaps by construction)
        if (!(D[2] < D[1] && r_act > D[5] + D[6] && l_act > D[4] + D[6] + 3 * sep &&
              D[4] > D[5] && r_cup_in + d[3] < d[0] - d[2] && z_rim < z_front &&
              z_rim > -d[7] + d[9] && z_back > -d[7] + d[9] && -d[7] > -d[6] + d[8] &&
              z_front < -d[1] && D[3] < D[0]))
            return gadep::fail(GADEP_E_INVAL, "coax: parameters give overlapping components");
        if (p.groove_d > 0.0 &&
            !(p.groove_w > 0.0 && p.groove_r - 0.5 * p.groove_w - sep > D[5] + D[6] + sep &&
              p.groove_r + 0.5 * p.groove_w + sep < r_act && p.groove_d + 4 * sep < l_act - D[4]))
            return gadep::fail(GADEP_E_INVAL, "coax: the back-face groove must lie between the bore and the side");
        if (p.flange_h > 0.0) {
            const double r_cup_out = r_cup_in + d[3];
            const int nh = p.n_bolt_holes, M = p.bolt_n_sides;
            if (!(nh >= 1 && M >= 4 && M % 2 == 0 && p.n_theta % nh == 0 && (p.n_theta / nh) % 2 == 0 &&
                  p.flange_r_in > r_cup_out && p.flange_r_out < d[0] - d[2] && p.flange_r_in < p.flange_r_out &&
                  p.bolt_r > 0.0 && p.bolt_rc - p.bolt_r > p.flange_r_in && p.bolt_rc + p.bolt_r < p.flange_r_out &&
                  2.0 * p.bolt_r < 2.0 * kPi * (p.bolt_rc - p.bolt_r) / nh &&
                  p.flange_z_top < -d[1] && p.flange_z_top - p.flange_h > -d[6] + d[8]))
                return gadep::fail(GADEP_E_INVAL, "coax: flange must lie between the holder and the endcap wall, "
                                                  "n_theta a multiple of 2 n_bolt_holes, even bolt_n_sides");
        }
        const int nt = p.n_theta, np = p.n_phi;

        // endcap and its vacuum: plain cylinders, top face at local z = 0
        Surface endcap = ChamferedCylinder(d[0], 0.0, d[6], nt, np, 1).generate();
        relocate(endcap, 0.0);
        Surface endvac = ChamferedCylinder(d[0] - d[2], 0.0, d[6] - d[8] - d[1], nt, np, 1).generate();
        relocate(endvac, -d[1]);
        Surface cup = Cup(r_cup_in, d[3], z_rim + d[7], d[9], nt).generate();
        relocate(cup, z_rim);
        // optional back-face groove; the active volume follows it one delta inside
        const double gi = p.groove_r - 0.5 * p.groove_w, go = p.groove_r + 0.5 * p.groove_w;
        const double gd = p.groove_d > 0.0 ? p.groove_d : 0.0;
        Surface crystal = ChamferedCylinder(D[1], D[2], D[0], nt, np, p.z_slices, gi, go, gd).generate();
        relocate(crystal, z_front);
        // active volume: front shrunk by D4, back face kept and separated by one delta
        Surface active = ChamferedCylinder(r_act, rch_act, l_act - sep, nt, np, p.z_slices, gi - sep, go + sep, gd).generate();
        relocate(active, z_front - D[3]);
        // borehole contact and vacuum: hemispherical blind ends toward the front
        const double rc = D[5] + D[6];
        Surface contact = ChamferedCylinder(rc, rc, D[4] + D[6] - 2 * sep, nt, np, 1).generate();
        relocate(contact, z_back + D[4] + D[6]);
        Surface borevac = ChamferedCylinder(D[5], D[5], D[4] - 3 * sep, nt, np, 1).generate();
        relocate(borevac, z_back + D[4]);

        a.add(std::move(endcap), attr(GADEP_MAT_AL, 0, 1));
        a.add(std::move(endvac), attr(GADEP_MAT_VACUUM, 0, -1));
        a.add(std::move(cup), attr(GADEP_MAT_CU, 0, -1));
        a.add(std::move(crystal), attr(GADEP_MAT_GE, 0, 0));
        a.add(std::move(active), attr(GADEP_MAT_GE, 1, 2));
        a.add(std::move(contact), attr(GADEP_MAT_GE, 0, -1));
        a.add(std::move(borevac), attr(GADEP_MAT_VACUUM, 0, -1));
        if (p.has_source_solid) add_source_prism(p, a);
        if (p.flange_h > 0.0) {
            Surface fl = Flange(p.flange_r_in, p.flange_r_out, p.flange_h, p.n_bolt_holes, p.bolt_n_sides, p.bolt_r,
                                p.bolt_rc, nt).generate();
            if (fl.f.empty()) return gadep::fail(GADEP_E_MESH, "coax: flange face triangulation failed");
            relocate(fl, p.flange_z_top);
            a.add(std::move(fl), attr(GADEP_MAT_CU, 0, -1));
        }
        return GADEP_OK;
    }
};

}  // namespace

extern "C" gadep_status detmesh_build(const detmesh_params *p, detmesh_mesh **out)
{
    gadep::clear_error();
    if (!p || !out) return gadep::fail(GADEP_E_INVAL, "detmesh_build: NULL argument");
    *out = nullptr;
    if (p->n_theta < 3 || p->n_theta > 65536 || p->n_phi < 1 || p->n_phi > 4096 ||
        p->z_slices < 1 || p->z_slices > 65536)
        return gadep::fail(GADEP_E_INVAL, "detmesh_build: n_theta in [3, 65536], n_phi in [1, 4096], "
                                          "z_slices in [1, 65536] required");
    if (p->has_source_solid &&
        !(p->src_r > 0 && p->src_h > 0 && p->src_n_sides >= 3 && p->src_n_sides <= 65536))
        return gadep::fail(GADEP_E_INVAL, "detmesh_build: bad source solid");
    std::unique_ptr<PhysicalGeometry> det;
    if (p->kind == GADEP_DET_BARE_CYLINDER) det.reset(new BareCylinderDetector());
    else if (p->kind == GADEP_DET_COAX) det.reset(new CoaxDetector());
    else return gadep::fail(GADEP_E_INVAL, "detmesh_build: unknown detector kind %d", p->kind);
    Assembly a;
    gadep_status st = det->createGeometry(*p, a);
    if (st != GADEP_OK) return st;
    st = gadep::validate_and_nest(a.m);
    if (st != GADEP_OK) return st;
    detmesh_mesh *m = new (std::nothrow) detmesh_mesh();
    if (!m) return gadep::fail(GADEP_E_NOMEM, "detmesh_build: out of host memory");
    m->geo = std::move(a.m);
    m->xyz_f.assign(m->geo.xyz.begin(), m->geo.xyz.end());
    *out = m;
    return GADEP_OK;
}

extern "C" gadep_status detmesh_from_arrays(const float *xyz, int32_t n_vert, const int32_t *tri,
                                            const int32_t *tri_solid, int32_t n_tri,
                                            const int32_t *material, const int32_t *active,
                                            const int32_t *group, int32_t n_solid,
                                            detmesh_mesh **out)
{
    gadep::clear_error();
    if (!out) return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: NULL out");
    *out = nullptr;
    if (!xyz || !tri || !tri_solid || !material || !active || !group || n_vert < 3 || n_tri < 4 ||
        n_solid < 1 || n_solid > 1024)
        return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: bad arguments");
    gadep::MeshData g;
    g.xyz.assign(xyz, xyz + 3 * (size_t)n_vert);
    for (double v : g.xyz)
        if (!std::isfinite(v)) return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: non-finite vertex");
    g.tri.assign(tri, tri + 3 * (size_t)n_tri);
    g.tri_solid.assign(tri_solid, tri_solid + n_tri);
    for (int32_t v : g.tri)
        if (v < 0 || v >= n_vert) return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: vertex index out of range");
    for (int32_t s : g.tri_solid)
        if (s < 0 || s >= n_solid) return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: solid index out of range");
    for (int32_t s = 0; s < n_solid; ++s) {
        if (material[s] < 0 || material[s] >= 1024 || group[s] < -1 || group[s] >= GADEP_MAX_GROUPS)
            return gadep::fail(GADEP_E_INVAL, "detmesh_from_arrays: bad attributes of solid %d", s);
        g.solids.push_back(gadep_solid{ material[s], active[s] ? 1 : 0, group[s], -1 });
    }
    gadep_status st = gadep::validate_and_nest(g);
    if (st != GADEP_OK) return st;
    detmesh_mesh *m = new (std::nothrow) detmesh_mesh();
    if (!m) return gadep::fail(GADEP_E_NOMEM, "detmesh_from_arrays: out of host memory");
    m->geo = std::move(g);
    m->xyz_f.assign(xyz, xyz + 3 * (size_t)n_vert);
    *out = m;
    return GADEP_OK;
}

extern "C" gadep_status detmesh_get(const detmesh_mesh *m, const float **xyz, int32_t *n_vert,
                                    const int32_t **tri, const int32_t **tri_solid, int32_t *n_tri,
                                    const gadep_solid **solids, int32_t *n_solid)
{
    gadep::clear_error();
    if (!m) return gadep::fail(GADEP_E_INVAL, "detmesh_get: NULL mesh");
    if (xyz) *xyz = m->xyz_f.data();
    if (n_vert) *n_vert = m->geo.n_vert();
    if (tri) *tri = m->geo.tri.data();
    if (tri_solid) *tri_solid = m->geo.tri_solid.data();
    if (n_tri) *n_tri = m->geo.n_tri();
    if (solids) *solids = m->geo.solids.data();
    if (n_solid) *n_solid = m->geo.n_solid();
    return GADEP_OK;
}

extern "C" gadep_status detmesh_solid_stats(const detmesh_mesh *m, int32_t solid, double *volume,
                                            int32_t *euler)
{
    gadep::clear_error();
    if (!m || solid < 0 || solid >= m->geo.n_solid())
        return gadep::fail(GADEP_E_INVAL, "detmesh_solid_stats: bad mesh or solid index");
    if (volume) *volume = gadep::solid_volume(m->geo, solid);
    if (euler) *euler = gadep::solid_euler(m->geo, solid);
    return GADEP_OK;
}

extern "C" gadep_status detmesh_locate(const detmesh_mesh *m, const double p[3], int32_t *solid)
{
    gadep::clear_error();
    if (!m || !p || !solid) return gadep::fail(GADEP_E_INVAL, "detmesh_locate: NULL argument");
    int32_t r = gadep::locate_point(m->geo, p);
    if (r == -2) return gadep::fail(GADEP_E_MESH, "detmesh_locate: point lies on a surface");
    *solid = r;
    return GADEP_OK;
}

extern "C" void detmesh_destroy(detmesh_mesh *m) { delete m; }
