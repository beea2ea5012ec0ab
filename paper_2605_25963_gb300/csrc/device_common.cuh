// device_common.cuh -- device building blocks of the photon transport (sm_103a).
//
//   philox4x32_10   counter-based generator (Salmon et al., SC'11), one stream
//                   per history: key = seed, counter = (block, hid lo, hid hi, instance)
//   Stream          4 words per Philox block, u = (2 (x >> 9) + 1) 2^-24
//   Shear, tri_test watertight ray/triangle test of Woop, Benthin & Wald (JCGT
//                   2013): vertices are translated to the ray origin, sheared so
//                   the ray runs along +z', and the 2-D edge functions U, V, W
//                   decide the hit; products are never contracted into FMAs so a
//                   shared edge gives exactly opposite values in its two
//                   triangles, and exact zeros are re-evaluated in FP64.
//   node4_keys      the four box tests of a 4-wide BVH node (child boxes on a
//                   7-bit grid of the node's own), children hit sorted nearest first
//   traverse        nearest hit in the 4-wide BVH with a per-thread stack
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gadep {
namespace dev {

constexpr float kMeC2 = 510.99895f;
constexpr float kTwoMeC2 = 1021.9979f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr int kStack = 64;

// One 32-byte load through the read-only data path (sm_100 and later); p must be
// 32-byte aligned.  A 64-byte BVH node takes two.
__device__ __forceinline__ void ldg256(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

enum : uint32_t { ERR_STEPCAP = 1u, ERR_KAHN = 2u, ERR_LOST = 4u, ERR_STACK = 8u, ERR_NONFINITE = 16u };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

struct Stream {
    uint32_t block, c1, c2, c3;
    uint4 buf;
    int idx;
    __device__ __forceinline__ void init(unsigned long long hid, uint32_t inst)
    {
        block = 0u; c1 = (uint32_t)hid; c2 = (uint32_t)(hid >> 32); c3 = inst; idx = 4;
    }
    __device__ __forceinline__ uint32_t word(uint32_t k0, uint32_t k1)
    {
        if (idx == 4) {
            buf = philox4x32_10(make_uint4(block, c1, c2, c3), k0, k1);
            ++block;
            idx = 0;
        }
        const uint32_t x = idx == 0 ? buf.x : (idx == 1 ? buf.y : (idx == 2 ? buf.z : buf.w));
        ++idx;
        return x;
    }
    __device__ __forceinline__ float u01(uint32_t k0, uint32_t k1)
    {
        return __uint2float_rn(2u * (word(k0, k1) >> 9) + 1u) * 5.9604644775390625e-8f;
    }
};

__device__ __forceinline__ float pick(float x, float y, float z, int k)
{
    return k == 0 ? x : (k == 1 ? y : z);
}

struct Shear {
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ Shear make_shear(float dx, float dy, float dz)
{
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    Shear s;
    s.kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    s.kx = s.kz == 2 ? 0 : s.kz + 1;
    s.ky = s.kx == 2 ? 0 : s.kx + 1;
    const float dkz = pick(dx, dy, dz, s.kz);
    if (dkz < 0.0f) { const int t = s.kx; s.kx = s.ky; s.ky = t; }
    s.Sx = pick(dx, dy, dz, s.kx) / dkz;
    s.Sy = pick(dx, dy, dz, s.ky) / dkz;
    s.Sz = 1.0f / dkz;
    return s;
}

// Watertight test of triangle slot i against the ray (o, shear), skipped when its
// mesh id (v1.w) is `exclude`; on a hit with t_min < t < t_best updates
// t_best / best / entering (entering: d . n < 0).
__device__ __forceinline__ void tri_test(const float4 *__restrict__ tris, int i, int exclude, float ox,
                                         float oy, float oz, const Shear &sh, float t_min, float &t_best,
                                         int &best, bool &entering)
{
    const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
    if (__float_as_int(b.w) == exclude) return;
    const float Ax0 = a.x - ox, Ay0 = a.y - oy, Az0 = a.z - oz;
    const float Bx0 = b.x - ox, By0 = b.y - oy, Bz0 = b.z - oz;
    const float Cx0 = c.x - ox, Cy0 = c.y - oy, Cz0 = c.z - oz;
    const float Akz = pick(Ax0, Ay0, Az0, sh.kz), Bkz = pick(Bx0, By0, Bz0, sh.kz), Ckz = pick(Cx0, Cy0, Cz0, sh.kz);
    const float Ax = fmaf(-sh.Sx, Akz, pick(Ax0, Ay0, Az0, sh.kx));
    const float Ay = fmaf(-sh.Sy, Akz, pick(Ax0, Ay0, Az0, sh.ky));
    const float Bx = fmaf(-sh.Sx, Bkz, pick(Bx0, By0, Bz0, sh.kx));
    const float By = fmaf(-sh.Sy, Bkz, pick(Bx0, By0, Bz0, sh.ky));
    const float Cx = fmaf(-sh.Sx, Ckz, pick(Cx0, Cy0, Cz0, sh.kx));
    const float Cy = fmaf(-sh.Sy, Ckz, pick(Cx0, Cy0, Cz0, sh.ky));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        // products of two binary32 values are exact in binary64: exact signs
        U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        V = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return;
    const float det = U + V + W;
    if (det == 0.0f) return;
    const float T = U * (sh.Sz * Akz) + V * (sh.Sz * Bkz) + W * (sh.Sz * Ckz);
    const float t = T / det;
    if (t > t_min && t < t_best) {
        t_best = t;
        best = i;
        entering = det > 0.0f;
    }
}

// Shear of a ray for the fixed-permutation test below: kz = dominant axis,
// kx = kz + 1 and ky = kx + 1 (mod 3), never swapped; flip = d[kz] < 0.
struct ShearK {
    int kz;
    bool flip;
    float sx, sy, sz;
};

__device__ __forceinline__ ShearK make_shear_k(float dx, float dy, float dz)
{
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    ShearK s;
    s.kz = (ax > ay) ? ((ax > az) ? 0 : 2) : ((ay > az) ? 1 : 2);
    const int kx = s.kz == 2 ? 0 : s.kz + 1;
    const int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = pick(dx, dy, dz, s.kz);
    s.flip = dkz < 0.0f;
    s.sx = pick(dx, dy, dz, kx) / dkz;
    s.sy = pick(dx, dy, dz, ky) / dkz;
    s.sz = 1.0f / dkz;
    return s;
}

template <int K>
__device__ __forceinline__ float comp(float x, float y, float z)
{
    return K == 0 ? x : (K == 1 ? y : z);
}

// tri_test with the axis permutation fixed at compile time (KZ = dominant axis).
// make_shear swaps kx and ky when d[kz] < 0 to keep the winding; that swap
// negates U, V, W, det and T exactly, so t and the hit decision are the same
// and only the sign of det turns, which `flip` undoes for `entering`.
template <int KZ>
__device__ __forceinline__ void tri_test_k(const float4 *__restrict__ tris, int i, int exclude, float ox,
                                           float oy, float oz, const ShearK &sh, float t_min, float &t_best,
                                           int &best, bool &entering)
{
    constexpr int KX = (KZ + 1) % 3, KY = (KX + 1) % 3;
    const float4 a = __ldg(tris + 3 * i), b = __ldg(tris + 3 * i + 1), c = __ldg(tris + 3 * i + 2);
    if (__float_as_int(b.w) == exclude) return;
    const float Akz = comp<KZ>(a.x, a.y, a.z) - comp<KZ>(ox, oy, oz);
    const float Bkz = comp<KZ>(b.x, b.y, b.z) - comp<KZ>(ox, oy, oz);
    const float Ckz = comp<KZ>(c.x, c.y, c.z) - comp<KZ>(ox, oy, oz);
    const float Ax = fmaf(-sh.sx, Akz, comp<KX>(a.x, a.y, a.z) - comp<KX>(ox, oy, oz));
    const float Ay = fmaf(-sh.sy, Akz, comp<KY>(a.x, a.y, a.z) - comp<KY>(ox, oy, oz));
    const float Bx = fmaf(-sh.sx, Bkz, comp<KX>(b.x, b.y, b.z) - comp<KX>(ox, oy, oz));
    const float By = fmaf(-sh.sy, Bkz, comp<KY>(b.x, b.y, b.z) - comp<KY>(ox, oy, oz));
    const float Cx = fmaf(-sh.sx, Ckz, comp<KX>(c.x, c.y, c.z) - comp<KX>(ox, oy, oz));
    const float Cy = fmaf(-sh.sy, Ckz, comp<KY>(c.x, c.y, c.z) - comp<KY>(ox, oy, oz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        V = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return;
    const float det = U + V + W;
    if (det == 0.0f) return;
    const float T = U * (sh.sz * Akz) + V * (sh.sz * Bkz) + W * (sh.sz * Ckz);
    const float t = T / det;
    if (t > t_min && t < t_best) {
        t_best = t;
        best = i;
        entering = (det > 0.0f) != sh.flip;
    }
}

template <int KZ>
__device__ __forceinline__ void leaf_test_k(const float4 *__restrict__ tris, int ref, int exclude, float ox,
                                            float oy, float oz, const ShearK &sh, float t_min, float &t_best,
                                            int &best, bool &ent, uint32_t &ntested)
{
    const int code = ~ref;
    const int first = code >> 3, count = code & 7;
    for (int i = first; i < first + count; ++i) {
        ++ntested;
        tri_test_k<KZ>(tris, i, exclude, ox, oy, oz, sh, t_min, t_best, best, ent);
    }
}

struct TravStats { uint32_t nodes, boxes, tris, relocated; };

// Sort key of a child box met by the ray: its entry distance (non-negative, so
// its bits order as unsigned integers) with the two low mantissa bits replaced
// by the child's slot; kMiss for a box the ray does not meet.  Two distances
// within 4 ulp may swap places, which only changes the visiting order.
constexpr uint32_t kMiss = 0xffffffffu;

// Grid position of child c's plane in a plane word (byte c = 128 + q): the
// float 1 + q / 128, made by placing that byte under the exponent byte 0x3f.
template <int C>
__device__ __forceinline__ float qplane(uint32_t w)
{
    return __uint_as_float(__byte_perm(w, 0x3f000000u, 0x7044u | (C << 8)));
}

// Key of one child from its near-plane and far-plane distances along each axis.
__device__ __forceinline__ uint32_t slab_key(float xn, float xf, float yn, float yf, float zn, float zf, float t_min,
                                             float t_best, uint32_t slot)
{
    const float tn = fmaxf(fmaxf(xn, yn), fmaxf(zn, t_min));
    const float tf = fminf(fminf(xf, yf), fminf(zf, t_best));
    return tn <= tf ? ((__float_as_uint(tn) & 0x7ffffffcu) | slot) : kMiss;
}

// Distances t = f * (S / d) + (b - o) / d of one axis's planes in plane word w
// for children (0, 1) and (2, 3), two per packed FMA.
__device__ __forceinline__ void qplanes(uint32_t w, float2 a, float2 b, float2 &t01, float2 &t23)
{
    t01 = __ffma2_rn(make_float2(qplane<0>(w), qplane<1>(w)), a, b);
    t23 = __ffma2_rn(make_float2(qplane<2>(w), qplane<3>(w)), a, b);
}

__device__ __forceinline__ void cswap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b);
    b = max(a, b);
    a = lo;
}

// The four child boxes of wide node `node` against the ray (o, 1/d) restricted
// to [t_min, t_best]: keys k[0..3] of the children hit, nearest first (kMiss
// after the last), the node's child words and its number of children.  Per
// axis the near plane is the low one for a direction component >= 0 and the
// high one otherwise, so one comparison per axis replaces a min and a max per
// child and axis; an empty slot's inverted box (low above high) is never met.
__device__ __forceinline__ void node4_keys(const float4 *__restrict__ nodes, int node, float ix, float iy,
                                           float iz, float oix, float oiy, float oiz, float t_min, float t_best,
                                           uint32_t &k0, uint32_t &k1, uint32_t &k2, uint32_t &k3, int4 &child,
                                           int &n_child)
{
    float4 base, cw, pxy, pz;
    ldg256(nodes + 4 * node, base, cw);
    ldg256(nodes + 4 * node + 2, pxy, pz);
    child = make_int4(__float_as_int(cw.x), __float_as_int(cw.y), __float_as_int(cw.z), __float_as_int(cw.w));
    n_child = (child.x != ~0) + (child.y != ~0) + (child.z != ~0) + (child.w != ~0);
    const float ax = base.w * ix, ay = pz.z * iy, az = pz.w * iz;
    const float bx = fmaf(base.x, ix, -oix), by = fmaf(base.y, iy, -oiy), bz = fmaf(base.z, iz, -oiz);
    const uint32_t lx = __float_as_uint(pxy.x), hx = __float_as_uint(pxy.y);
    const uint32_t ly = __float_as_uint(pxy.z), hy = __float_as_uint(pxy.w);
    const uint32_t lz = __float_as_uint(pz.x), hz = __float_as_uint(pz.y);
    const bool sx = ix < 0.0f, sy = iy < 0.0f, sz = iz < 0.0f;
    const uint32_t nx = sx ? hx : lx, fx = sx ? lx : hx;
    const uint32_t ny = sy ? hy : ly, fy = sy ? ly : hy;
    const uint32_t nz = sz ? hz : lz, fz = sz ? lz : hz;
    float2 xn01, xn23, xf01, xf23, yn01, yn23, yf01, yf23, zn01, zn23, zf01, zf23;
    const float2 ax2 = make_float2(ax, ax), bx2 = make_float2(bx, bx);
    const float2 ay2 = make_float2(ay, ay), by2 = make_float2(by, by);
    const float2 az2 = make_float2(az, az), bz2 = make_float2(bz, bz);
    qplanes(nx, ax2, bx2, xn01, xn23);
    qplanes(fx, ax2, bx2, xf01, xf23);
    qplanes(ny, ay2, by2, yn01, yn23);
    qplanes(fy, ay2, by2, yf01, yf23);
    qplanes(nz, az2, bz2, zn01, zn23);
    qplanes(fz, az2, bz2, zf01, zf23);
    k0 = slab_key(xn01.x, xf01.x, yn01.x, yf01.x, zn01.x, zf01.x, t_min, t_best, 0u);
    k1 = slab_key(xn01.y, xf01.y, yn01.y, yf01.y, zn01.y, zf01.y, t_min, t_best, 1u);
    k2 = slab_key(xn23.x, xf23.x, yn23.x, yf23.x, zn23.x, zf23.x, t_min, t_best, 2u);
    k3 = slab_key(xn23.y, xf23.y, yn23.y, yf23.y, zn23.y, zf23.y, t_min, t_best, 3u);
    cswap(k0, k1);
    cswap(k2, k3);
    cswap(k0, k2);
    cswap(k1, k3);
    cswap(k1, k2);
}

// Child word of slot s (the low two bits of a key).
__device__ __forceinline__ int child_of(const int4 &c, uint32_t key)
{
    const int a = (key & 1u) ? c.y : c.x;
    const int b = (key & 1u) ? c.w : c.z;
    return (key & 2u) ? b : a;
}

// Distance of the hit on mesh triangle m, taken from the triangle's plane (unit
// normal and offset computed in FP64 from the stored vertices) once the
// watertight test has selected it.  On a sliver triangle the edge-function
// distance loses accuracy as eps |v - o|^2 / width; the plane form keeps about
// eps |o| / |cos|.  The selection (which triangle, entering or leaving) is not
// touched; a plane distance that is not finite or not beyond t_min (a hit within
// rounding of the ray start) keeps the edge-function value.
__device__ __forceinline__ float plane_t(const float4 *__restrict__ planes, int m, float ox, float oy, float oz,
                                         float dx, float dy, float dz, float t_edge, float t_min)
{
    const float4 p = __ldg(planes + m);
    const float dn = fmaf(p.x, dx, fmaf(p.y, dy, p.z * dz));
    const float num = fmaf(-p.x, ox, fmaf(-p.y, oy, fmaf(-p.z, oz, p.w)));
    const float t = num / dn;
    return (isfinite(t) && t > t_min) ? t : t_edge;
}

// Child word of a node: >= 0 inner node index; < 0 leaf ~(first << 3 | count).
constexpr int kSentinel = 0x7fffffff;

__device__ __forceinline__ void leaf_test(const float4 *__restrict__ tris, int ref, int exclude, float ox,
                                          float oy, float oz, const Shear &sh, float t_min, float &t_best,
                                          int &best, bool &ent, uint32_t &ntested)
{
    const int code = ~ref;
    const int first = code >> 3, count = code & 7;
    for (int i = first; i < first + count; ++i) {
        ++ntested;
        tri_test(tris, i, exclude, ox, oy, oz, sh, t_min, t_best, best, ent);
    }
}

// Nearest triangle along o + t d with t_min < t < t_max (exclusive) in the tree
// rooted at `root` (-1: empty), skipping mesh triangle `exclude`.  Returns the
// triangle slot or -1; t_hit / entering set on a hit.  Sets ERR_STACK in err if
// the stack would overflow (query abandoned).
// Loop structure after Aila & Laine (HPG 2009): an inner-node loop that runs
// until every lane of the warp holds a leaf (postponing at most one leaf per
// lane), then a leaf loop, so lanes execute node steps and triangle tests in
// lockstep instead of branching between them at every node.
template <bool COUNT>
__device__ __forceinline__ int traverse(const float4 *__restrict__ nodes,
                                        const float4 *__restrict__ tris,
                                        const float4 *__restrict__ planes, int root, float ox, float oy,
                                        float oz, float dx, float dy, float dz, float t_min,
                                        int exclude, float &t_hit, bool &entering, uint32_t &err,
                                        TravStats &st, float t_max = INFINITY)
{
    if (root < 0) return -1;
    const Shear sh = make_shear(dx, dy, dz);
    const float ix = 1.0f / (fabsf(dx) > 1e-30f ? dx : copysignf(1e-30f, dx));
    const float iy = 1.0f / (fabsf(dy) > 1e-30f ? dy : copysignf(1e-30f, dy));
    const float iz = 1.0f / (fabsf(dz) > 1e-30f ? dz : copysignf(1e-30f, dz));
    const float oix = ox * ix, oiy = oy * iy, oiz = oz * iz;
    float t_best = t_max;
    int best = -1;
    bool ent = false;
    // stack entries: (child word, key of its box); an entry whose box is entered
    // beyond the nearest hit found since it was pushed is dropped when popped
    uint2 stack[kStack];
    stack[0] = make_uint2((uint32_t)kSentinel, 0u);
    int sp = 0;
    int node = root;
    int leaf = 0;
    uint32_t nn = 0, nb = 0, nt = 0;
    auto pop = [&]() -> int {
        uint2 e = stack[sp--];
        while (__uint_as_float(e.y) > t_best) e = stack[sp--];
        return (int)e.x;
    };
    while (node != kSentinel) {
        while ((unsigned)node < (unsigned)kSentinel) {
            uint32_t k0, k1, k2, k3;
            int4 cw;
            int nch;
            node4_keys(nodes, node, ix, iy, iz, oix, oiy, oiz, t_min, t_best, k0, k1, k2, k3, cw, nch);
            ++nn;
            nb += nch;
            if (k0 == kMiss) {
                node = pop();
            } else {
                node = child_of(cw, k0);
                if (k1 != kMiss) {      // push the others, farthest first
                    if (sp + 3 >= kStack) { err |= ERR_STACK; return -1; }
                    if (k3 != kMiss) stack[++sp] = make_uint2((uint32_t)child_of(cw, k3), k3);
                    if (k2 != kMiss) stack[++sp] = make_uint2((uint32_t)child_of(cw, k2), k2);
                    stack[++sp] = make_uint2((uint32_t)child_of(cw, k1), k1);
                }
            }
            if (node < 0 && leaf >= 0) {     // postpone this leaf, keep descending
                leaf = node;
                node = pop();
            }
            if (!__any_sync(__activemask(), leaf >= 0)) break;
        }
        while (leaf < 0) {
            leaf_test(tris, leaf, exclude, ox, oy, oz, sh, t_min, t_best, best, ent, nt);
            leaf = node;
            if (node < 0) node = pop();
        }
    }
    if (COUNT) { st.nodes += nn; st.boxes += nb; st.tris += nt; }
    if (best >= 0) {
        // direction back from its reciprocals, as the wavefront trace kernel does,
        // so that both forms take the same distance
        t_hit = plane_t(planes, __float_as_int(__ldg(&tris[3 * best + 1].w)), ox, oy, oz, __frcp_rn(ix),
                        __frcp_rn(iy), __frcp_rn(iz), t_best, t_min);
        entering = ent;
    }
    return best;
}

}  // namespace dev
}  // namespace gadep
