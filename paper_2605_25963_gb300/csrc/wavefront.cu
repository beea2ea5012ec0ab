// wavefront.cu -- wavefront form of the photon transport (same physics, same
// Philox streams and same tallies as the persistent megakernel in transport.cu).
//
// Photons live in S device-memory slots.  One iteration runs three kernels:
//   birth    every slot on the dead list takes the next history from the work
//            counter (histories born in the world whose first ray misses the
//            scene box end here with nothing deposited) and joins the trace queue;
//   trace    lean persistent traversal: warps take slots from the queue, lanes
//            that finish a query take the next one as soon as too few lanes of
//            the warp are still traversing (dynamic fetch), so the warp is not
//            held by its longest ray;
//   physics  one thread per queued slot applies the segment: free flight,
//            boundary crossing (nesting-tree rule), interaction or escape, and the
//            end-of-history tally; survivors go to the next trace queue, finished
//            slots to the next dead list.
// The host issues iterations and reads the control block every few iterations
// to stop when the work counter is exhausted and no photon is alive.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "gadep_internal.h"
#include "transport_common.cuh"

namespace gadep {
namespace wf {

using namespace gadep::dev;

struct __align__(16) Ray {      // read by trace, written by birth and physics
    float ox, oy, oz, t_cur;
    float dx, dy, dz;
    int last_tri;               // mesh triangle id to skip (-1 none)
    int root;                   // tree of the photon's region
    int pad[3];
};
struct __align__(16) Hit {      // written by trace
    float t;
    int tri;                    // mesh triangle id, -1 = nothing ahead
    int region;                 // region id of the triangle's solid
    int entering;               // 1 entering, 0 leaving, -2 traversal stack overflow
};
struct __align__(16) Phot {
    float E, lam;
    int region, steps;
    float E0, edep, dep_all, esc;
};
struct __align__(16) Rng {
    uint32_t block, idx, c1, c2;
    uint4 buf;
};
struct __align__(16) Hist {
    unsigned long long g_hist;
    int inst;
    uint32_t herr;
    int sec;                    // region of a waiting annihilation photon, -1 = none
    uint32_t n_inter;           // interactions of this history so far
    float sox, soy;
};

// Per-block tallies in shared memory, one record per instance, flushed once per
// launch into the block's tally copy: finished histories of many instances mix
// in every kernel launch, so per-thread accumulators would flush constantly.
struct STally {
    unsigned int hist, fep, zero, over, err, seg, inter, errbits;
    float dep, dep_all, esc, pad;
};

template <bool GRAD>
struct BlockTally {
    STally *t;
    double *sc;                 // GRAD: [n_inst][8] fep score sums and squares
    int n;
    __device__ void init(void *smem, int n_inst)
    {
        t = reinterpret_cast<STally *>(smem);
        sc = reinterpret_cast<double *>(t + n_inst);
        n = n_inst;
        for (int i = threadIdx.x; i < n_inst; i += blockDim.x) t[i] = STally{ 0, 0, 0, 0, 0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f };
        if (GRAD)
            for (int i = threadIdx.x; i < 8 * n_inst; i += blockDim.x) sc[i] = 0.0;
    }
    __device__ void history(int inst, uint32_t segs, uint32_t inter, uint32_t herr, bool fep, float edep,
                            float dep_all, float esc, float e_max, const float *score)
    {
        STally &s = t[inst];
        atomicAdd(&s.hist, 1u);
        atomicAdd(&s.seg, segs);
        if (inter) atomicAdd(&s.inter, inter);
        if (herr) {
            atomicAdd(&s.err, 1u);
            atomicOr(&s.errbits, herr);
            return;
        }
        if (fep) {
            atomicAdd(&s.fep, 1u);
            if (GRAD)
                for (int g = 0; g < 4; ++g) {
                    const double v = (double)score[g];
                    atomicAdd(&sc[8 * inst + g], v);
                    atomicAdd(&sc[8 * inst + 4 + g], v * v);
                }
        }
        if (edep == 0.0f) atomicAdd(&s.zero, 1u);
        else if (edep >= e_max) atomicAdd(&s.over, 1u);
        if (edep != 0.0f) atomicAdd(&s.dep, edep);
        atomicAdd(&s.dep_all, dep_all);
        atomicAdd(&s.esc, esc);
    }
    __device__ void flush(TallyDev *T)
    {
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const STally &s = t[i];
            if (!s.hist && !s.seg) continue;
            TallyDev &d = T[i];
            if (s.hist) atomicAdd(&d.n_hist, (unsigned long long)s.hist);
            if (s.fep) atomicAdd(&d.n_fep, (unsigned long long)s.fep);
            if (s.zero) atomicAdd(&d.n_zero, (unsigned long long)s.zero);
            if (s.over) atomicAdd(&d.n_over, (unsigned long long)s.over);
            if (s.err) { atomicAdd(&d.n_err, (unsigned long long)s.err); atomicOr(&d.err_bits, (unsigned long long)s.errbits); }
            if (s.seg) atomicAdd(&d.n_segments, (unsigned long long)s.seg);
            if (s.inter) atomicAdd(&d.n_interactions, (unsigned long long)s.inter);
            atomicAdd(&d.sum_dep_active, (double)s.dep);
            atomicAdd(&d.sum_dep_all, (double)s.dep_all);
            atomicAdd(&d.sum_esc, (double)s.esc);
            if (GRAD)
                for (int g = 0; g < 4; ++g) {
                    atomicAdd(&d.fep_score[g], sc[8 * i + g]);
                    atomicAdd(&d.fep_score_sq[g], sc[8 * i + 4 + g]);
                }
        }
    }
};

template <bool GRAD>
__host__ __device__ constexpr size_t block_tally_bytes(int n_inst)
{
    return (size_t)n_inst * (sizeof(STally) + (GRAD ? 8 * sizeof(double) : 0));
}

struct Ctrl {
    unsigned int q_count[2];     // trace queue sizes, by iteration parity
    unsigned int dead_count[2];  // dead lists, by iteration parity
    unsigned int trace_head;     // dynamic-fetch cursor of the trace kernel
    unsigned int pad;
    unsigned long long work;     // next global history index
};

struct State {
    Ray *ray;
    Hit *hit;
    Phot *phot;
    Rng *rng;
    Hist *hist;
    float4 *sec;                 // secondary photon: (z, -direction)
    float4 *score;               // GRAD only
    unsigned int *queue[2];
    unsigned int *dead[2];
    Ctrl *ctrl;
    int slots;
};

__device__ __forceinline__ float rng_u01(Rng &r, uint32_t c3, uint32_t k0, uint32_t k1)
{
    if (r.idx == 4) {
        r.buf = philox4x32_10(make_uint4(r.block, r.c1, r.c2, c3), k0, k1);
        ++r.block;
        r.idx = 0;
    }
    const uint32_t x = r.idx == 0 ? r.buf.x : (r.idx == 1 ? r.buf.y : (r.idx == 2 ? r.buf.z : r.buf.w));
    ++r.idx;
    return __uint2float_rn(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f;
}

// Warp-aggregated append of `slot` to list (count at *cnt).
__device__ __forceinline__ void warp_append(bool want, unsigned int slot, unsigned int *list, unsigned int *cnt)
{
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned int)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) list[base + __popc(mask & ((1u << lane) - 1u))] = slot;
}

__global__ void init_kernel(State S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.slots) S.dead[0][i] = (unsigned int)i;
    if (i == 0) {
        S.ctrl->q_count[0] = S.ctrl->q_count[1] = 0;
        S.ctrl->dead_count[0] = (unsigned int)S.slots;
        S.ctrl->dead_count[1] = 0;
        S.ctrl->trace_head = 0;
        S.ctrl->work = 0;
    }
}

// ---------------------------------------------------------------- birth
template <bool GRAD>
__global__ void __launch_bounds__(256) birth_kernel(const Params P, State S, int cur)
{
    const uint32_t FULL = 0xffffffffu;
    const int nxt = cur ^ 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.ctrl->q_count[nxt] = 0;
        S.ctrl->dead_count[nxt] = 0;
        S.ctrl->trace_head = 0;
    }
    extern __shared__ double4 smem_birth[];
    BlockTally<false> bt;               // culled histories carry no score
    bt.init(smem_birth, P.n_inst);
    __syncthreads();
    const unsigned int n_dead = S.ctrl->dead_count[cur];
    const int lane = threadIdx.x & 31;
    const uint32_t k0 = P.key0, k1 = P.key1;
    int inst = 0;
    // warp-uniform loop over the dead list
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n_dead; base += stride) {
        const unsigned int j = base + lane;
        const bool mine = j < n_dead;
        const unsigned int slot = mine ? S.dead[cur][j] : 0u;
        bool need = mine, placed = false;
        // draw histories until the slot holds one that reaches the scene; the warp
        // takes exactly as many history ids as it has lanes in need, so no id is lost
        while (true) {
            const uint32_t needm = __ballot_sync(FULL, need);
            if (!needm) break;
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(&S.ctrl->work, (unsigned long long)__popc(needm));
            b = __shfl_sync(FULL, b, 0);
            if (b >= P.total) break;
            const uint32_t rank = __popc(needm & ((1u << lane) - 1u));
            if (need && b + rank < P.total) {
                const unsigned long long g = b + rank;
                if (g >= P.inst_end[inst]) {
                    // first instance whose end exceeds g (binary search over the prefix sums)
                    int lo = inst + 1, hi = P.n_inst - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (g < P.inst_end[mid]) hi = mid; else lo = mid + 1;
                    }
                    inst = lo;
                }
                const InstDev &I = P.inst[inst];
                const unsigned long long local = g - (inst ? P.inst_end[inst - 1] : 0ull);
                const unsigned long long hid = I.hist_offset + local;
                Rng r;
                r.block = 0u; r.c1 = (uint32_t)hid; r.c2 = (uint32_t)(hid >> 32); r.idx = 4;
                const uint32_t c3 = I.inst_id;
                float ox = I.px, oy = I.py, oz = I.pz, dx, dy, dz;
                if (I.src_kind == GADEP_SRC_DISK) {
                    const float rr = I.radius * sqrtf(rng_u01(r, c3, k0, k1));
                    float sp, cp;
                    sincospif(2.0f * rng_u01(r, c3, k0, k1), &sp, &cp);
                    ox = fmaf(rr, cp, ox); oy = fmaf(rr, sp, oy);
                } else if (I.src_kind == GADEP_SRC_PRISM) {
                    const int N = I.n_sides;
                    int kk = (int)((float)N * rng_u01(r, c3, k0, k1));
                    kk = min(kk, N - 1);
                    const float s1 = sqrtf(rng_u01(r, c3, k0, k1)), u3 = rng_u01(r, c3, k0, k1);
                    float sa, ca, sb, cb;
                    sincospif(2.0f * (float)kk / (float)N, &sa, &ca);
                    sincospif(2.0f * (float)((kk + 1) % N) / (float)N, &sb, &cb);
                    const float wa = s1 * (1.0f - u3), wb = s1 * u3;
                    ox += I.radius * (wa * ca + wb * cb);
                    oy += I.radius * (wa * sa + wb * sb);
                    oz = fmaf(I.height, rng_u01(r, c3, k0, k1), oz);
                }
                if (I.src_kind == GADEP_SRC_PENCIL) {
                    dx = I.dx; dy = I.dy; dz = I.dz;
                } else {
                    const float c = 2.0f * rng_u01(r, c3, k0, k1) - 1.0f;
                    float sp, cp;
                    sincospif(2.0f * rng_u01(r, c3, k0, k1), &sp, &cp);
                    const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
                    dx = s * cp; dy = s * sp; dz = c;
                }
                const int region = I.birth_region;
                if (region == 0 && !ray_hits_box(P.root_lo, P.root_hi, ox, oy, oz, dx, dy, dz)) {
                    bt.history(inst, 1u, 0u, 0u, false, 0.0f, 0.0f, I.E0, P.e_max, nullptr);
                    if (g < P.n_trace) P.edep_trace[g] = 0.0f;
                } else {
                    const float lam = -logf(rng_u01(r, c3, k0, k1));
                    Ray ry;
                    ry.ox = ox; ry.oy = oy; ry.oz = oz; ry.t_cur = 0.0f;
                    ry.dx = dx; ry.dy = dy; ry.dz = dz; ry.last_tri = -1;
                    ry.root = P.regions[region].w;
                    ry.pad[0] = ry.pad[1] = ry.pad[2] = 0;
                    S.ray[slot] = ry;
                    Phot ph;
                    ph.E = I.E0; ph.lam = lam; ph.region = region; ph.steps = 0;
                    ph.E0 = I.E0; ph.edep = 0.0f; ph.dep_all = 0.0f; ph.esc = 0.0f;
                    S.phot[slot] = ph;
                    S.rng[slot] = r;
                    Hist h;
                    h.g_hist = g; h.inst = inst; h.herr = 0u; h.sec = -1; h.n_inter = 0u; h.sox = 0.0f; h.soy = 0.0f;
                    S.hist[slot] = h;
                    if (GRAD) S.score[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    need = false;
                    placed = true;
                }
            }
            if (b + __popc(needm) >= P.total) break;
        }
        warp_append(placed, slot, S.queue[cur], &S.ctrl->q_count[cur]);
    }
    bt.flush(block_tally(P));
}

// ---------------------------------------------------------------- trace
constexpr int kFetchThreshold = 20;   // refill lanes when fewer are still traversing (8, 12, 20 measured)

template <bool COUNT>
__global__ void __launch_bounds__(256) trace_kernel(const float4 *__restrict__ nodes,
                                                    const float4 *__restrict__ tris, State S, int cur,
                                                    unsigned long long *counters)
{
    const uint32_t FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned int n = S.ctrl->q_count[cur];
    const unsigned int *queue = S.queue[cur];
    bool has = false;
    unsigned int slot = 0;
    float ox = 0, oy = 0, oz = 0, t_min = 0, ix = 0, iy = 0, iz = 0, oix = 0, oiy = 0, oiz = 0, t_best = 0;
    int exclude = -1, node = kSentinel, leaf = 0, sp = 0, best = -1;
    bool ent = false;
    Shear sh{ 0, 1, 2, 0.0f, 0.0f, 1.0f };
    int stack[kStack];
    uint32_t nn = 0, nt = 0, err = 0;
    bool drained = false;
    while (true) {
        // ---- dynamic fetch: lanes without a ray take the next queue entries ----
        const uint32_t need = __ballot_sync(FULL, !has);
        if (need && !drained) {
            unsigned int base = 0;
            if (lane == 0) base = atomicAdd(&S.ctrl->trace_head, (unsigned int)__popc(need));
            base = __shfl_sync(FULL, base, 0);
            if (base >= n) drained = true;
            const unsigned int idx = base + __popc(need & ((1u << lane) - 1u));
            if (!has && idx < n) {
                slot = queue[idx];
                const Ray r = S.ray[slot];
                ox = r.ox; oy = r.oy; oz = r.oz; t_min = r.t_cur;
                exclude = r.last_tri;
                sh = make_shear(r.dx, r.dy, r.dz);
                ix = 1.0f / (fabsf(r.dx) > 1e-30f ? r.dx : copysignf(1e-30f, r.dx));
                iy = 1.0f / (fabsf(r.dy) > 1e-30f ? r.dy : copysignf(1e-30f, r.dy));
                iz = 1.0f / (fabsf(r.dz) > 1e-30f ? r.dz : copysignf(1e-30f, r.dz));
                oix = ox * ix; oiy = oy * iy; oiz = oz * iz;
                t_best = INFINITY;
                best = -1;
                ent = false;
                stack[0] = kSentinel;
                sp = 0;
                node = r.root < 0 ? kSentinel : r.root;
                leaf = 0;
                has = true;
            }
        }
        if (__ballot_sync(FULL, has) == 0) break;
        // ---- traversal (while-while), left early when too few lanes remain ----
        while (has) {
            while ((unsigned)node < (unsigned)kSentinel) {
                const float4 n0 = __ldg(nodes + 4 * node + 0);
                const float4 n1 = __ldg(nodes + 4 * node + 1);
                const float4 n2 = __ldg(nodes + 4 * node + 2);
                const int4 n3 = __ldg(reinterpret_cast<const int4 *>(nodes) + 4 * node + 3);
                ++nn;
                const float a0 = fmaf(n0.x, ix, -oix), a1 = fmaf(n0.y, ix, -oix);
                const float a2 = fmaf(n0.z, iy, -oiy), a3 = fmaf(n0.w, iy, -oiy);
                const float a4 = fmaf(n2.x, iz, -oiz), a5 = fmaf(n2.y, iz, -oiz);
                const float b0 = fmaf(n1.x, ix, -oix), b1 = fmaf(n1.y, ix, -oix);
                const float b2 = fmaf(n1.z, iy, -oiy), b3 = fmaf(n1.w, iy, -oiy);
                const float b4 = fmaf(n2.z, iz, -oiz), b5 = fmaf(n2.w, iz, -oiz);
                const float tmin0 = fmaxf(fmaxf(fminf(a0, a1), fminf(a2, a3)), fmaxf(fminf(a4, a5), t_min));
                const float tmax0 = fminf(fminf(fmaxf(a0, a1), fmaxf(a2, a3)), fminf(fmaxf(a4, a5), t_best));
                const float tmin1 = fmaxf(fmaxf(fminf(b0, b1), fminf(b2, b3)), fmaxf(fminf(b4, b5), t_min));
                const float tmax1 = fminf(fminf(fmaxf(b0, b1), fmaxf(b2, b3)), fminf(fmaxf(b4, b5), t_best));
                const bool h0 = tmin0 <= tmax0, h1 = tmin1 <= tmax1;
                if (!h0 && !h1) {
                    node = stack[sp--];
                } else {
                    const bool first0 = h0 && (!h1 || tmin0 <= tmin1);
                    node = first0 ? n3.x : n3.y;
                    if (h0 && h1) {
                        if (sp + 1 >= kStack) { err |= ERR_STACK; node = kSentinel; leaf = 0; best = -1; break; }
                        stack[++sp] = first0 ? n3.y : n3.x;
                    }
                }
                if (node < 0 && leaf >= 0) {
                    leaf = node;
                    node = stack[sp--];
                }
                if (!__any_sync(__activemask(), leaf >= 0)) break;
            }
            while (leaf < 0) {
                leaf_test(tris, leaf, exclude, ox, oy, oz, sh, t_min, t_best, best, ent, nt);
                leaf = node;
                if (node < 0) node = stack[sp--];
            }
            if (node == kSentinel) {
                Hit h;
                h.t = best >= 0 ? t_best : INFINITY;
                h.tri = best >= 0 ? __float_as_int(__ldg(&tris[3 * best + 1].w)) : -1;
                h.region = best >= 0 ? __float_as_int(__ldg(&tris[3 * best].w)) : 0;
                h.entering = best >= 0 ? (ent ? 1 : 0) : ((err & ERR_STACK) ? -2 : 0);
                S.hit[slot] = h;
                err = 0;
                has = false;
            }
            if (__popc(__activemask()) < kFetchThreshold && !drained) break;
        }
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)nn);
        atomicAdd(&counters[1], (unsigned long long)nt);
    }
}

// ---------------------------------------------------------------- physics
template <bool GRAD, bool COUNT>
__global__ void __launch_bounds__(256) physics_kernel(const Params P, State S, int cur,
                                                      unsigned long long *counters)
{
    const uint32_t FULL = 0xffffffffu;
    const int nxt = cur ^ 1;
    // shared: region table (material slot, flags, parent, root), then block tallies
    extern __shared__ int4 s_reg[];
    for (int i = threadIdx.x; i < P.n_region; i += blockDim.x) s_reg[i] = P.regions[i];
    BlockTally<GRAD> bt;
    bt.init(s_reg + P.n_region, P.n_inst);
    __syncthreads();
    const unsigned int n = S.ctrl->q_count[cur];
    const int lane = threadIdx.x & 31;
    const uint32_t k0 = P.key0, k1 = P.key1;
    TravStats ts{ 0u, 0u, 0u };
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const unsigned int j = base + lane;
        const bool mine = j < n;
        const unsigned int slot = mine ? S.queue[cur][j] : 0u;
        bool alive_slot = false, finished = false;
        int inst = 0;
        float edep_out = 0.0f, E0_out = 0.0f;
        unsigned long long g_hist = 0;
        uint32_t herr_out = 0;
        if (mine) {
            Ray ry = S.ray[slot];
            Hit ht = S.hit[slot];
            Phot ph = S.phot[slot];
            Hist hs = S.hist[slot];
            inst = hs.inst;
            g_hist = hs.g_hist;
            uint32_t herr = hs.herr;
            float4 sc4 = GRAD ? S.score[slot] : make_float4(0, 0, 0, 0);
            float score[4] = { sc4.x, sc4.y, sc4.z, sc4.w };
            bool rng_loaded = false;
            Rng r;
            const InstDev &I = P.inst[inst];
            const uint32_t c3 = I.inst_id;
            bool ray_dirty = false;
            if (ht.entering == -2) herr |= ERR_STACK;
            if (++ph.steps > P.step_cap) herr |= ERR_STEPCAP;
            if (herr) {
                finished = true;
            } else {
                int region = ph.region;
                const int4 R = s_reg[region];
                const int group = (R.y >> 1) - 1;
                float t_hit = ht.t;
                int hit_tri = ht.tri, hit_region = ht.region;
                bool entering = ht.entering == 1;
                if (hit_tri < 0 && region != 0) {
                    // not inside the region it carries: relocate through every triangle
                    const int k = traverse<COUNT>(P.nodes, P.tris, P.root_all, ry.ox, ry.oy, ry.oz, ry.dx, ry.dy,
                                                  ry.dz, ry.t_cur, ry.last_tri, t_hit, entering, herr, ts);
                    if (COUNT) ts.relocated++;
                    if (k < 0) {
                        region = 0;
                    } else {
                        hit_tri = __float_as_int(__ldg(&P.tris[3 * k + 1].w));
                        hit_region = __float_as_int(__ldg(&P.tris[3 * k].w));
                    }
                }
                const int hit = hit_tri;
                float pe = 0.0f, co = 0.0f, pa = 0.0f;
                if (R.x >= 0) mu_at(P.xs + (size_t)R.x * P.n_grid, P.n_grid, P.lnE_min, P.inv_dlnE, ph.E, pe, co, pa);
                const float mu_unit = pe + co + pa;
                const float scl = group >= 0 ? I.scale[group] : 1.0f;
                const float mu = mu_unit * scl;
                const float d_int = mu > 0.0f ? ph.lam / mu : INFINITY;
                bool photon_done = false;
                if (herr) {
                    finished = true;
                } else if (d_int < t_hit - ry.t_cur) {
                    // ---- interaction ----
                    hs.n_inter++;
                    r = S.rng[slot];
                    rng_loaded = true;
                    if (GRAD && group >= 0 && group < 4) score[group] += 1.0f / scl - mu_unit * d_int;
                    const float tt = ry.t_cur + d_int;
                    const float px = fmaf(tt, ry.dx, ry.ox), py = fmaf(tt, ry.dy, ry.oy), pz = fmaf(tt, ry.dz, ry.oz);
                    const float u = rng_u01(r, c3, k0, k1) * mu_unit;
                    float dep;
                    float E = ph.E;
                    if (u < pe) {
                        dep = E; E = 0.0f; photon_done = true;
                    } else if (u < pe + co || pa == 0.0f) {
                        const float k = E * (1.0f / kMeC2);
                        const float a2k = 1.0f + 2.0f * k;
                        const float br = a2k / (9.0f + 2.0f * k);
                        float x = 1.0f;
                        bool ok = false;
                        for (int trial = 0; trial < 1000; ++trial) {
                            const float r1 = rng_u01(r, c3, k0, k1), r2 = rng_u01(r, c3, k0, k1),
                                        r3 = rng_u01(r, c3, k0, k1);
                            if (r1 <= br) {
                                x = 1.0f + 2.0f * k * r2;
                                if (r3 <= 4.0f * (1.0f / x - 1.0f / (x * x))) { ok = true; break; }
                            } else {
                                x = a2k / (1.0f + 2.0f * k * r2);
                                const float cc = 1.0f - (x - 1.0f) / k;
                                if (r3 <= 0.5f * (cc * cc + 1.0f / x)) { ok = true; break; }
                            }
                        }
                        if (!ok) {
                            herr |= ERR_KAHN;
                            dep = 0.0f;
                            photon_done = true;
                        } else {
                            const float c = 1.0f - (x - 1.0f) / k;
                            float sp, cp;
                            sincospif(2.0f * rng_u01(r, c3, k0, k1), &sp, &cp);
                            const float Ep = E / x;
                            dep = E - Ep;
                            rotate(ry.dx, ry.dy, ry.dz, c, sp, cp);
                            E = Ep;
                            if (E < P.e_cut) { dep += E; E = 0.0f; photon_done = true; }
                        }
                    } else {
                        dep = E - kTwoMeC2;
                        float nx, ny, nz;
                        const float c = 2.0f * rng_u01(r, c3, k0, k1) - 1.0f;
                        float sp, cp;
                        sincospif(2.0f * rng_u01(r, c3, k0, k1), &sp, &cp);
                        const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
                        nx = s * cp; ny = s * sp; nz = c;
                        E = kMeC2;
                        ry.dx = nx; ry.dy = ny; ry.dz = nz;
                        hs.sec = region;
                        hs.sox = px; hs.soy = py;
                        S.sec[slot] = make_float4(pz, -nx, -ny, -nz);
                    }
                    if (R.y & 1) ph.edep += dep;
                    ph.dep_all += dep;
                    ph.E = E;
                    ry.ox = px; ry.oy = py; ry.oz = pz;
                    ry.t_cur = 0.0f; ry.last_tri = -1;
                    ray_dirty = true;
                    if (herr) finished = true;
                    else if (!photon_done) ph.lam = -logf(rng_u01(r, c3, k0, k1));
                } else if (hit < 0) {
                    if (region != 0) herr |= ERR_LOST;
                    ph.esc += ph.E;
                    ph.E = 0.0f;
                    photon_done = true;
                    if (herr) finished = true;
                } else {
                    // ---- boundary crossing ----
                    const float len = t_hit - ry.t_cur;
                    ph.lam -= mu * len;
                    if (GRAD && group >= 0 && group < 4) score[group] -= mu_unit * len;
                    ry.t_cur = t_hit;
                    ry.last_tri = hit_tri;
                    region = entering ? hit_region : s_reg[hit_region].z;
                    ry.root = s_reg[region].w;
                    ph.region = region;
                    ray_dirty = true;
                }
                if (photon_done && !finished) {
                    if (hs.sec >= 0) {
                        if (!rng_loaded) { r = S.rng[slot]; rng_loaded = true; }
                        const float4 s4 = S.sec[slot];
                        const int sreg = hs.sec;
                        hs.sec = -1;
                        ry.ox = hs.sox; ry.oy = hs.soy; ry.oz = s4.x;
                        ry.dx = s4.y; ry.dy = s4.z; ry.dz = s4.w;
                        ry.t_cur = 0.0f; ry.last_tri = -1;
                        ph.E = kMeC2;
                        ph.region = sreg;
                        ry.root = s_reg[sreg].w;
                        ph.lam = -logf(rng_u01(r, c3, k0, k1));
                        ray_dirty = true;
                    } else {
                        finished = true;
                    }
                }
                if (!finished && !(isfinite(ry.dx) && isfinite(ph.E) && isfinite(ph.lam))) {
                    herr |= ERR_NONFINITE;
                    finished = true;
                }
            }
            hs.herr = herr;
            herr_out = herr;
            edep_out = ph.edep;
            E0_out = ph.E0;
            if (!finished) {
                if (ray_dirty) S.ray[slot] = ry;
                S.phot[slot] = ph;
                if (rng_loaded) S.rng[slot] = r;
                S.hist[slot] = hs;
                if (GRAD) S.score[slot] = make_float4(score[0], score[1], score[2], score[3]);
                alive_slot = true;
            } else {
                const bool fep = !herr && (E0_out - edep_out) <= P.fep_delta;
                bt.history(inst, (uint32_t)ph.steps, hs.n_inter, herr, fep, edep_out, ph.dep_all, ph.esc, P.e_max,
                           score);
                if (g_hist < P.n_trace) P.edep_trace[g_hist] = herr ? -1.0f : edep_out;
            }
        }
        // ---- warp-converged: spectrum atomics, queue / dead-list appends ----
        const bool binned = finished && herr_out == 0u && edep_out > 0.0f && edep_out < P.e_max;
        int bin = 0;
        if (binned) bin = min((int)(edep_out * P.bin_scale), P.n_bins - 1);
        const uint32_t key = binned ? (uint32_t)(inst * P.n_bins + bin) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(FULL, key);
        if (binned && lane == __ffs(peers) - 1)
            atomicAdd(&P.spectra[(size_t)inst * P.n_bins + bin], (uint32_t)__popc(peers));
        warp_append(alive_slot, slot, S.queue[nxt], &S.ctrl->q_count[nxt]);
        warp_append(finished, slot, S.dead[nxt], &S.ctrl->dead_count[nxt]);
    }
    bt.flush(block_tally(P));
    if (COUNT) {
        if (ts.nodes) atomicAdd(&counters[0], (unsigned long long)ts.nodes);
        if (ts.tris) atomicAdd(&counters[1], (unsigned long long)ts.tris);
        if (ts.relocated) atomicAdd(&counters[2], (unsigned long long)ts.relocated);
    }
}

}  // namespace wf

// ---------------------------------------------------------------- host driver

struct WavefrontBuffers {
    wf::State S{};
    void *block = nullptr;
    wf::Ctrl *host_ctrl = nullptr;   // pinned mirror of the control block
    int trace_grid = 0, work_grid = 0;
};

int wavefront_trace_grid(const WavefrontBuffers *w) { return w ? w->trace_grid : 0; }

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

gadep_status wavefront_create(int device, int slots, bool grad, WavefrontBuffers **out)
{
    *out = nullptr;
    if (slots < 1024 || slots > (1 << 24)) return fail(GADEP_E_INVAL, "wavefront: slots must be in [1024, 2^24]");
    WavefrontBuffers *w = new (std::nothrow) WavefrontBuffers();
    if (!w) return fail(GADEP_E_NOMEM, "wavefront: out of host memory");
    const size_t n = (size_t)slots;
    size_t off = 0;
    size_t o_ray = off; off = align_up(off + n * sizeof(wf::Ray));
    size_t o_hit = off; off = align_up(off + n * sizeof(wf::Hit));
    size_t o_phot = off; off = align_up(off + n * sizeof(wf::Phot));
    size_t o_rng = off; off = align_up(off + n * sizeof(wf::Rng));
    size_t o_hist = off; off = align_up(off + n * sizeof(wf::Hist));
    size_t o_sec = off; off = align_up(off + n * sizeof(float4));
    size_t o_score = off; off = align_up(off + n * sizeof(float4));   // always: buffers serve both forms
    (void)grad;
    size_t o_q0 = off; off = align_up(off + n * 4);
    size_t o_q1 = off; off = align_up(off + n * 4);
    size_t o_d0 = off; off = align_up(off + n * 4);
    size_t o_d1 = off; off = align_up(off + n * 4);
    size_t o_ctrl = off; off = align_up(off + sizeof(wf::Ctrl));
    cudaError_t e = cudaMalloc(&w->block, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete w;
        return fail(GADEP_E_NOMEM, "wavefront: cudaMalloc of %zu bytes: %s", off, cudaGetErrorString(e));
    }
    if (cudaHostAlloc((void **)&w->host_ctrl, sizeof(wf::Ctrl), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w->block);
        delete w;
        return fail(GADEP_E_NOMEM, "wavefront: pinned host allocation failed");
    }
    char *b = (char *)w->block;
    w->S.ray = (wf::Ray *)(b + o_ray);
    w->S.hit = (wf::Hit *)(b + o_hit);
    w->S.phot = (wf::Phot *)(b + o_phot);
    w->S.rng = (wf::Rng *)(b + o_rng);
    w->S.hist = (wf::Hist *)(b + o_hist);
    w->S.sec = (float4 *)(b + o_sec);
    w->S.score = (float4 *)(b + o_score);
    w->S.queue[0] = (unsigned int *)(b + o_q0);
    w->S.queue[1] = (unsigned int *)(b + o_q1);
    w->S.dead[0] = (unsigned int *)(b + o_d0);
    w->S.dead[1] = (unsigned int *)(b + o_d1);
    w->S.ctrl = (wf::Ctrl *)(b + o_ctrl);
    w->S.slots = slots;
    int n_sm = 0, bps = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (void *)wf::trace_kernel<false>, 256, 0);
    w->trace_grid = n_sm * std::max(bps, 1);
    w->work_grid = n_sm * 8;
    *out = w;
    return GADEP_OK;
}

void wavefront_destroy(WavefrontBuffers *w)
{
    if (!w) return;
    cudaFree(w->block);
    cudaFreeHost(w->host_ctrl);
    delete w;
}

// Run every history of the plan's Params through the wavefront kernels on `s`.
gadep_status wavefront_run(WavefrontBuffers *w, const dev::Params &P, bool grad, bool count,
                           unsigned long long *counters, cudaStream_t s)
{
    wf::State S = w->S;
    if (P.n_inst > kWavefrontMaxInstances)
        return fail(GADEP_E_INVAL, "wavefront: at most %d instances per run", kWavefrontMaxInstances);
    // dynamic shared memory: block tallies (birth); region table + block tallies (physics)
    const size_t bsm = wf::block_tally_bytes<false>(P.n_inst);
    const size_t rsm = (size_t)P.n_region * sizeof(int4) +
                       (grad ? wf::block_tally_bytes<true>(P.n_inst) : wf::block_tally_bytes<false>(P.n_inst));
    {
        cudaError_t e = cudaSuccess;
        auto set = [&](const void *f, size_t b) {
            if (e == cudaSuccess && b > 48 * 1024)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        };
        set((const void *)wf::birth_kernel<true>, bsm);
        set((const void *)wf::birth_kernel<false>, bsm);
        set((const void *)wf::physics_kernel<true, true>, rsm);
        set((const void *)wf::physics_kernel<true, false>, rsm);
        set((const void *)wf::physics_kernel<false, true>, rsm);
        set((const void *)wf::physics_kernel<false, false>, rsm);
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: shared memory: %s", cudaGetErrorString(e));
    }
    wf::init_kernel<<<(S.slots + 255) / 256, 256, 0, s>>>(S);
    const int check_every = 16;
    const long long max_iter = (long long)P.step_cap * 4 + (long long)(P.total / 1024) + 1000000;
    for (long long it = 0; it < max_iter; ++it) {
        const int cur = (int)(it & 1);
        if (grad) {
            wf::birth_kernel<true><<<w->work_grid, 256, bsm, s>>>(P, S, cur);
        } else {
            wf::birth_kernel<false><<<w->work_grid, 256, bsm, s>>>(P, S, cur);
        }
        if (count) wf::trace_kernel<true><<<w->trace_grid, 256, 0, s>>>(P.nodes, P.tris, S, cur, counters);
        else wf::trace_kernel<false><<<w->trace_grid, 256, 0, s>>>(P.nodes, P.tris, S, cur, counters);
        if (grad) {
            if (count) wf::physics_kernel<true, true><<<w->work_grid, 256, rsm, s>>>(P, S, cur, counters);
            else wf::physics_kernel<true, false><<<w->work_grid, 256, rsm, s>>>(P, S, cur, counters);
        } else {
            if (count) wf::physics_kernel<false, true><<<w->work_grid, 256, rsm, s>>>(P, S, cur, counters);
            else wf::physics_kernel<false, false><<<w->work_grid, 256, rsm, s>>>(P, S, cur, counters);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: launch: %s", cudaGetErrorString(e));
        if (it % check_every == check_every - 1) {
            e = cudaMemcpyAsync(w->host_ctrl, S.ctrl, sizeof(wf::Ctrl), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: control read: %s", cudaGetErrorString(e));
            const int nxt = cur ^ 1;
            if (w->host_ctrl->work >= P.total && w->host_ctrl->q_count[nxt] == 0) return GADEP_OK;
        }
    }
    return fail(GADEP_E_TIMEOUT, "wavefront: iteration bound reached with photons still alive");
}

}  // namespace gadep
