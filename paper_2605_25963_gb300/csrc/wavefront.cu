// wavefront.cu -- wavefront form of the photon transport (same physics, same
// Philox streams and same tallies as the persistent megakernel in transport.cu).
//
// Photons live in device-memory slots.  One iteration runs five kernels on the
// stream, with no host round trip between them:
//   spawn    free slots (popped from a stack) take births from the pending ring
//            (an index map: the i-th popped slot gets the i-th pending history)
//            and join the trace queue after the survivors of the previous iteration;
//   sort     counting sort of the queue by (region, direction class), from the
//            key histogram that physics and spawn accumulate, so that a warp
//            traverses one region's tree with rays of similar direction;
//   trace    lean persistent traversal: warps claim chunks of the queue, lanes
//            that finish a query take the next entry as soon as too few lanes of
//            the warp are still traversing (dynamic fetch), so the warp is not
//            held by its longest ray; the hit is stored by queue position;
//   physics  one thread per queued photon applies the segment: free flight,
//            boundary crossing (nesting-tree rule), interaction or escape, and the
//            end-of-history tally; survivors go to the next trace queue, finished
//            slots back onto the free stack (one global atomic per list, block and pass);
//   gen      history ids in chunks: source point and direction of each id;
//            histories born in the world whose first ray misses the scene box end
//            here with nothing deposited, the others join the pending ring;
//   ctrl     one thread: advances the counters and plans the next iteration.
// The host issues iterations and reads the control block every few iterations
// to stop once the history supply, the ring and the queue are all empty.
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

// Per-slot photon record: 64 bytes, the DRAM fetch unit, in two 32-byte halves
// (DRAM sectors).  The first holds everything a boundary crossing -- three
// visits in four -- reads and changes; the second (flight origin, direction,
// random-number state) is read only at interactions and when a waiting
// annihilation photon starts, and written then.  The trace query reads both and
// leaves a copy of the first in queue order (State::hot), so a physics visit
// reads it in a coalesced stream and writes it back to the slot, one sector.
struct __align__(32) SlotA {
    float4 f;                   // t_cur (distance travelled from the flight origin), tag bits
                                // (last mesh triangle + 1) << 8 | region, E, lam (mean free paths left)
    uint4 u;                    // info (instance, error bits, flags, direction cell), segments so far,
                                // edep (active) bits, dep_all bits
};
struct __align__(32) SlotB {
    float4 o;                   // flight origin, w = Philox words used (bits)
    float4 d;                   // direction, w = history index within the instance (bits)
};
struct __align__(64) Slot {
    SlotA a;                    // read by trace (copied to State::hot), written by every physics visit
    SlotB b;                    // read by trace; read and written by physics at interactions
};
// info word: instance (10 bits; a run has at most 1024), error bits (6), flags (2),
// direction cell of the sort key (14: face and cell of the cube map)
constexpr uint32_t kInstMask = 0x3ffu, kErrShift = 10, kErrMask = 0x3fu, kFlagShift = 16, kFlagMask = 3u,
                   kCellShift = 18;
__device__ __forceinline__ uint32_t info_pack(uint32_t inst, uint32_t err, uint32_t flags, uint32_t cell)
{
    return inst | ((err & kErrMask) << kErrShift) | ((flags & kFlagMask) << kFlagShift) | (cell << kCellShift);
}
struct __align__(16) Hit {      // by queue position, written by trace
    float t;
    int tri;                    // mesh triangle id, -1 = nothing ahead
    int region;                 // region of the triangle's solid
    int entering;               // 1 entering, 0 leaving, -2 traversal stack overflow,
                                // kBeyond: no surface before the sampled interaction point;
                                // + kRelocated when the hit (or tri -1: none) came from the
                                // tree of every triangle (relocation, see trace_kernel)
};
constexpr int kBeyond = -3;
constexpr int kRelocated = 4;
static_assert(sizeof(Slot) == 64 && sizeof(SlotA) == 32, "slot record: two 32-byte DRAM sectors");
// A charged-particle track (e_model 1) whose history goes on after the physics
// visit that set it going: traced by etrack_kernel before the slot's next visit.
struct __align__(16) Track {
    float4 p;                   // start point, w = kinetic energy
    float4 u;                   // unit direction, w = number of particles on the line
    unsigned int slot, tag;     // tag = region | instance << 8
    unsigned int pad[2];
};
struct __align__(32) Sec {      // second annihilation photon, waiting for the first
    float4 p;                   // position
    float4 d;                   // direction, w = region bits
};

constexpr int kMaxFaceBins = 12;    // direction cells per cube-map face and axis, at most
constexpr int kMaxKeys = 8192;      // regions * 6 * face_bins^2 at most

// Face cells per axis for a mesh of n_region regions: the finest that keeps the
// key space within kMaxKeys (one bin at 256 regions).
__host__ __device__ constexpr int face_bins_for(int n_region)
{
    int b = kMaxFaceBins;
    while (b > 1 && n_region * 6 * b * b > kMaxKeys) --b;
    return b;
}
constexpr uint32_t kFlagSec = 1u;   // a second annihilation photon is waiting
constexpr uint32_t kFlagEsc = 2u;   // esc[slot] holds energy this history let escape
constexpr int kTagShift = 8;        // at most 256 regions
constexpr int kMaxTriId = (1 << 23) - 2;

__device__ __forceinline__ uint32_t ray_tag(int last_tri, int region)
{
    return ((uint32_t)(last_tri + 1) << kTagShift) | (uint32_t)region;
}

// Sort key of a ray: its region, then a cube-map cell of its direction -- the
// face (dominant axis and its sign) and a fb x fb cell of the
// other two components divided by the dominant one.  Lanes of a warp then share
// the region's tree and the shear permutation of the triangle test, and descend
// the tree along similar paths.
__device__ __forceinline__ uint32_t dir_cell(int fb, float dx, float dy, float dz)
{
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    const uint32_t kz = (ax > ay) ? ((ax > az) ? 0u : 2u) : ((ay > az) ? 1u : 2u);
    const float m = kz == 0 ? dx : (kz == 1 ? dy : dz);
    const float u = kz == 0 ? dy : dx, w = kz == 2 ? dy : dz;
    const float h = 0.5f * (float)fb / fabsf(m);
    const uint32_t bu = min((uint32_t)fmaxf(fmaf(u, h, 0.5f * (float)fb), 0.0f), (uint32_t)fb - 1u);
    const uint32_t bw = min((uint32_t)fmaxf(fmaf(w, h, 0.5f * (float)fb), 0.0f), (uint32_t)fb - 1u);
    return (kz * 2u + (m < 0.0f ? 1u : 0u)) * (uint32_t)(fb * fb) + bu * (uint32_t)fb + bw;
}

// Sort key from the region and the direction cell (dir_cell, kept in the slot so
// that a crossing, which keeps the direction, needs no direction to key the ray).
__device__ __forceinline__ uint32_t sort_key(int region, int fb, uint32_t cell)
{
    return (uint32_t)region * 6u * (uint32_t)(fb * fb) + cell;
}

// Adds key k to a shared-memory histogram, one atomic per distinct key of the warp.
__device__ __forceinline__ void warp_hist_add(bool want, uint32_t k, unsigned int *h)
{
    const uint32_t peers = __match_any_sync(0xffffffffu, want ? k : 0xffffffffu);
    if (want && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[k], (unsigned int)__popc(peers));
}

// Philox stream resumed from the count of words already used: word k of a
// history is component k mod 4 of block k / 4 (the counter layout of the
// megakernel's Stream, so both forms draw the same numbers).
struct Words {
    uint32_t w, c1, c2, c3;
    uint4 buf;
    bool have;
    __device__ __forceinline__ void init(uint32_t used, unsigned long long hid, uint32_t inst)
    {
        w = used; c1 = (uint32_t)hid; c2 = (uint32_t)(hid >> 32); c3 = inst; have = false;
    }
    __device__ __forceinline__ float u01(uint32_t k0, uint32_t k1)
    {
        if (!have) {
            buf = philox4x32_10(make_uint4(w >> 2, c1, c2, c3), k0, k1);
            have = true;
        }
        const uint32_t i = w & 3u;
        const uint32_t x = i == 0 ? buf.x : (i == 1 ? buf.y : (i == 2 ? buf.z : buf.w));
        ++w;
        if ((w & 3u) == 0) have = false;
        return __uint2float_rn(2u * (x >> 9) + 1u) * 5.9604644775390625e-8f;
    }
};

// Per-block tallies in shared memory, one record per instance, flushed once per
// launch into the block's tally copy: finished histories of many instances mix
// in every launch, so per-thread accumulators would flush constantly.
struct STally {
    unsigned int hist, fep, zero, over, err, seg, inter, errbits;
    float dep, dep_all, esc;
    unsigned int culled;
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
        for (int i = threadIdx.x; i < n_inst; i += blockDim.x) t[i] = STally{ 0, 0, 0, 0, 0, 0, 0, 0, 0.f, 0.f, 0.f, 0u };
        if (GRAD)
            for (int i = threadIdx.x; i < 8 * n_inst; i += blockDim.x) sc[i] = 0.0;
    }
    __device__ void history(int inst, uint32_t segs, uint32_t herr, bool fep, float edep, float dep_all, float esc,
                            float e_max, const float *score)
    {
        STally &s = t[inst];
        atomicAdd(&s.hist, 1u);
        atomicAdd(&s.seg, segs);
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
        if (dep_all != 0.0f) atomicAdd(&s.dep_all, dep_all);
        if (esc != 0.0f) atomicAdd(&s.esc, esc);
    }
    // The finished histories of a warp (every lane calls; fin: this lane finished
    // one): the lanes of one instance are summed in registers and one lane adds
    // the sums, instead of every lane adding its own.
    __device__ void history_warp(bool fin, int inst, uint32_t segs, uint32_t herr, bool fep, float edep,
                                 float dep_all, float esc, float e_max)
    {
        const uint32_t FULL = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        uint32_t todo = __ballot_sync(FULL, fin);
        while (todo) {
            const int src = __ffs(todo) - 1;
            const int gi = __shfl_sync(FULL, inst, src);
            const bool mine = fin && inst == gi;
            const uint32_t grp = __ballot_sync(FULL, mine);
            todo &= ~grp;
            const bool ok = mine && !herr;
            const uint32_t n_err = __popc(__ballot_sync(FULL, mine && herr));
            const uint32_t n_fep = __popc(__ballot_sync(FULL, ok && fep));
            const uint32_t n_zero = __popc(__ballot_sync(FULL, ok && edep == 0.0f));
            const uint32_t n_over = __popc(__ballot_sync(FULL, ok && edep != 0.0f && edep >= e_max));
            const uint32_t seg = __reduce_add_sync(FULL, mine ? segs : 0u);
            const uint32_t eb = __reduce_or_sync(FULL, mine ? herr : 0u);
            float d = ok ? edep : 0.0f, da = ok ? dep_all : 0.0f, e = ok ? esc : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                d += __shfl_xor_sync(FULL, d, o);
                da += __shfl_xor_sync(FULL, da, o);
                e += __shfl_xor_sync(FULL, e, o);
            }
            if (lane == src) {
                STally &s = t[gi];
                atomicAdd(&s.hist, (unsigned int)__popc(grp));
                atomicAdd(&s.seg, seg);
                if (n_err) { atomicAdd(&s.err, n_err); atomicOr(&s.errbits, eb); }
                if (n_fep) atomicAdd(&s.fep, n_fep);
                if (n_zero) atomicAdd(&s.zero, n_zero);
                if (n_over) atomicAdd(&s.over, n_over);
                if (d != 0.0f) atomicAdd(&s.dep, d);
                if (da != 0.0f) atomicAdd(&s.dep_all, da);
                if (e != 0.0f) atomicAdd(&s.esc, e);
            }
        }
    }
    // n histories of instance inst that ended at birth: one segment each, nothing
    // deposited, the source energy escaped
    __device__ void culled(int inst, uint32_t n, float E0)
    {
        STally &s = t[inst];
        atomicAdd(&s.hist, n);
        atomicAdd(&s.seg, n);
        atomicAdd(&s.zero, n);
        atomicAdd(&s.culled, n);
        atomicAdd(&s.esc, (float)n * E0);
    }
    __device__ void flush(TallyDev *T)
    {
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const STally &s = t[i];
            if (!s.hist && !s.seg && !s.inter) continue;
            TallyDev &d = T[i];
            if (s.hist) atomicAdd(&d.n_hist, (unsigned long long)s.hist);
            if (s.fep) atomicAdd(&d.n_fep, (unsigned long long)s.fep);
            if (s.zero) atomicAdd(&d.n_zero, (unsigned long long)s.zero);
            if (s.over) atomicAdd(&d.n_over, (unsigned long long)s.over);
            if (s.err) { atomicAdd(&d.n_err, (unsigned long long)s.err); atomicOr(&d.err_bits, (unsigned long long)s.errbits); }
            if (s.seg) atomicAdd(&d.n_segments, (unsigned long long)s.seg);
            if (s.inter) atomicAdd(&d.n_interactions, (unsigned long long)s.inter);
            if (s.culled) atomicAdd(&d.n_culled, (unsigned long long)s.culled);
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
    // counters
    unsigned int q_count[2];       // trace queue sizes, by iteration parity
    unsigned int free_top;         // free slots: a stack, free_slots[0 .. free_top)
    unsigned int trace_head;       // chunk cursor of the trace kernel
    unsigned int iter;
    unsigned long long work;       // next history index handed to gen (may run past the total)
    unsigned long long pend_add;   // births appended by the running gen launch
    unsigned long long pend_head;  // births consumed so far
    unsigned long long pend_tail;  // births produced so far
    // plan of the next spawn and gen, written by ctrl only
    unsigned int sp_free, sp_filled, sp_q0, done;     // done: 1 finished, 2 iteration bound reached
    unsigned long long sp_head;
    unsigned long long gen_live;   // ring entries left once the next spawn has run
    unsigned long long max_iter;
    unsigned int t_count;          // deferred charged-particle tracks of this iteration
    unsigned int qlog_n;           // iterations whose queue size is in the log
};

struct State {
    Slot *slot;
    Sec *sec;
    float *esc;
    float4 *score;                 // GRAD only
    Hit *hit;                      // by queue position
    SlotA *hot;                    // by queue position: the slot's first half, copied by trace, read by physics
    unsigned int *queue[2];
    unsigned int *qkey[2];         // sort key of each queue entry
    unsigned int *hist[2];         // key histogram of queue[parity]
    unsigned int *fill;            // bucket cursors of the sort
    unsigned int *base;            // bucket starts of the sort
    unsigned int *qsort;           // the queue in key order: what trace and physics walk
    unsigned int *free_slots;      // stack of free slots: spawn pops, physics pushes
    Track *trk;                    // deferred tracks (e_model 1), one per slot at most
    unsigned long long *pend;      // ring of global history indices waiting for a slot
    unsigned long long pend_mask;  // ring size - 1 (a power of two)
    unsigned long long gen_target; // ring fill at which gen stops claiming ids
    Ctrl *ctrl;
    unsigned int *qlog;            // trace queue size of each iteration (the first kQueueLog)
    int slots;
};
constexpr int kQueueLog = 8192;

constexpr int kGenChunk = 2048;    // history ids per gen claim (8 per thread)
constexpr int kTraceChunk = 64;    // queue entries per trace claim

// Instance of global history index g (inst_end: inclusive prefix sums of the
// history counts); `inst` is a guess tried first.
__device__ __forceinline__ int find_inst(const Params &P, unsigned long long g, int inst)
{
    if (g < P.inst_end[inst] && (inst == 0 || g >= P.inst_end[inst - 1])) return inst;
    int lo = 0, hi = P.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (g < P.inst_end[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Source point and direction of a history (the megakernel's draw order).
__device__ __forceinline__ void sample_birth(const InstDev &I, Words &r, uint32_t k0, uint32_t k1, float &ox,
                                             float &oy, float &oz, float &dx, float &dy, float &dz)
{
    ox = I.px; oy = I.py; oz = I.pz;
    if (I.src_kind == GADEP_SRC_DISK) {
        const float rr = I.radius * sqrtf(r.u01(k0, k1));
        float sp, cp;
        sincospif(2.0f * r.u01(k0, k1), &sp, &cp);
        ox = fmaf(rr, cp, ox); oy = fmaf(rr, sp, oy);
    } else if (I.src_kind == GADEP_SRC_PRISM) {
        const int N = I.n_sides;
        int kk = (int)((float)N * r.u01(k0, k1));
        kk = min(kk, N - 1);
        const float s1 = sqrtf(r.u01(k0, k1)), u3 = r.u01(k0, k1);
        float sa, ca, sb, cb;
        sincospif(2.0f * (float)kk / (float)N, &sa, &ca);
        sincospif(2.0f * (float)((kk + 1) % N) / (float)N, &sb, &cb);
        const float wa = s1 * (1.0f - u3), wb = s1 * u3;
        ox += I.radius * (wa * ca + wb * cb);
        oy += I.radius * (wa * sa + wb * sb);
        oz = fmaf(I.height, r.u01(k0, k1), oz);
    }
    if (I.src_kind == GADEP_SRC_PENCIL) {
        dx = I.dx; dy = I.dy; dz = I.dz;
    } else {
        const float c = 2.0f * r.u01(k0, k1) - 1.0f;
        float sp, cp;
        sincospif(2.0f * r.u01(k0, k1), &sp, &cp);
        const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
        dx = s * cp; dy = s * sp; dz = c;
    }
}

__global__ void init_kernel(State S, unsigned long long max_iter)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.slots) S.free_slots[i] = (unsigned int)i;
    for (int k = i; k < kMaxKeys; k += gridDim.x * blockDim.x) {
        S.hist[0][k] = 0u;
        S.hist[1][k] = 0u;
        S.fill[k] = 0u;
    }
    if (i == 0) {
        Ctrl &c = *S.ctrl;
        c.q_count[0] = c.q_count[1] = 0;
        c.free_top = (unsigned int)S.slots;
        c.trace_head = 0;
        c.iter = 0;
        c.work = 0;
        c.pend_add = c.pend_head = c.pend_tail = 0;
        c.sp_free = c.sp_filled = c.sp_q0 = c.done = 0;
        c.sp_head = 0;
        c.gen_live = 0;
        c.max_iter = max_iter;
        c.t_count = 0;
        c.qlog_n = 0;
    }
}

// ---------------------------------------------------------------- ctrl
// One step of the control block: close iteration `cur` (spawn, sort, trace,
// physics and gen have run) and plan the next.
__device__ __forceinline__ void ctrl_step(Ctrl &c, int cur, unsigned long long total)
{
    const int nxt = cur ^ 1;
    c.pend_tail += c.pend_add;
    c.pend_add = 0;
    c.pend_head += c.sp_filled;
    const unsigned long long work = c.work < total ? c.work : total;
    c.work = work;
    const unsigned int n_alive = c.q_count[nxt], n_free = c.free_top;
    const unsigned long long avail = c.pend_tail - c.pend_head;
    const unsigned int filled = (unsigned int)(avail < n_free ? avail : n_free);
    // the next spawn pops the top `filled` free slots; physics then pushes above them
    c.sp_free = n_free - filled;
    c.sp_filled = filled;
    c.sp_q0 = n_alive;
    c.sp_head = c.pend_head;
    c.free_top = n_free - filled;
    c.q_count[nxt] = n_alive + filled;
    c.q_count[cur] = 0;
    c.t_count = 0;                 // etrack has run
    c.trace_head = 0;
    c.gen_live = avail - filled;
    c.iter++;
    if (work >= total && avail == 0 && n_alive == 0) c.done = 1;
    else if (c.iter >= c.max_iter) c.done = 2;
}

// In a graph (in_graph != 0) it also sets the condition of the WHILE node that
// repeats the iterations: 0 once the run is done or the iteration bound is hit.
__global__ void ctrl_kernel(State S, int cur, unsigned long long total, cudaGraphConditionalHandle loop,
                            int in_graph)
{
    for (int k = threadIdx.x; k < kMaxKeys; k += blockDim.x) {
        S.hist[cur][k] = 0u;        // the sort of iteration `cur` is done with it
        S.fill[k] = 0u;
    }
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctrl &c = *S.ctrl;
    if (!c.done) {
        ctrl_step(c, cur, total);
        // queue of the iteration just planned (for measurements per query)
        if (!c.done && c.iter <= (unsigned int)kQueueLog) {
            S.qlog[c.iter - 1] = c.q_count[cur ^ 1];
            c.qlog_n = c.iter;
        }
    }
    if (in_graph) cudaGraphSetConditional(loop, c.done ? 0u : 1u);
}

// ---------------------------------------------------------------- gen
// Blocks claim chunks of history ids while the ring holds fewer than gen_target
// births; each block has at most one chunk in flight, so the fill stays below
// gen_target + blocks x chunk, which the ring size covers.
__global__ void __launch_bounds__(256) gen_kernel(const Params P, State S)
{
    const uint32_t FULL = 0xffffffffu;
    constexpr int kPer = kGenChunk / 256;   // ids per thread and chunk
    Ctrl &c = *S.ctrl;
    if (c.done) return;
    extern __shared__ int4 smem_gen[];     // 16-byte aligned: the tallies hold FP64 sums
    __shared__ unsigned long long s_chunk, s_base;
    __shared__ unsigned int s_warp[8];
    BlockTally<false> bt;               // culled histories carry no score
    bt.init(smem_gen, P.n_inst);
    const unsigned long long live0 = c.gen_live, tail0 = c.pend_tail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t k0 = P.key0, k1 = P.key1;
    int inst = 0;
    // culled histories of instance cull_inst not yet added to the block tally
    uint32_t cull_n = 0;
    int cull_inst = 0;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long added = atomicAdd(&c.pend_add, 0ull);
            s_chunk = live0 + added < S.gen_target ? atomicAdd(&c.work, (unsigned long long)kGenChunk) : ~0ull;
        }
        __syncthreads();
        const unsigned long long chunk = s_chunk;
        if (chunk >= P.total) break;
        uint32_t keep = 0;              // bit k: id chunk + 256 k + threadIdx.x joins the ring
#pragma unroll 1
        for (int k = 0; k < kPer; ++k) {
            const unsigned long long g = chunk + (unsigned long long)(k * 256 + threadIdx.x);
            if (g >= P.total) break;
            inst = find_inst(P, g, inst);
            const InstDev &I = P.inst[inst];
            const unsigned long long local = g - (inst ? P.inst_end[inst - 1] : 0ull);
            Words r;
            r.init(0u, I.hist_offset + local, I.inst_id);
            float ox, oy, oz, dx, dy, dz;
            sample_birth(I, r, k0, k1, ox, oy, oz, dx, dy, dz);
            if (I.birth_region == 0 && !ray_hits_box(P.root_lo, P.root_hi, ox, oy, oz, dx, dy, dz)) {
                if (inst != cull_inst && cull_n) {
                    bt.culled(cull_inst, cull_n, P.inst[cull_inst].E0);
                    cull_n = 0;
                }
                cull_inst = inst;
                ++cull_n;
                if (g < P.n_trace) P.edep_trace[g] = 0.0f;
            } else {
                keep |= 1u << k;
            }
        }
        // block-wide exclusive prefix of the kept counts, one ring reservation per chunk
        const unsigned int cnt = __popc(keep);
        unsigned int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int tot = 0;
            for (int w = 0; w < 8; ++w) { const unsigned int v = s_warp[w]; s_warp[w] = tot; tot += v; }
            s_base = tot ? atomicAdd(&c.pend_add, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        unsigned long long pos = tail0 + s_base + s_warp[warp] + (inc - cnt);
        while (keep) {
            const int k = __ffs(keep) - 1;
            keep &= keep - 1u;
            S.pend[pos & S.pend_mask] = chunk + (unsigned long long)(k * 256 + threadIdx.x);
            ++pos;
        }
    }
    if (cull_n) bt.culled(cull_inst, cull_n, P.inst[cull_inst].E0);
    bt.flush(block_tally(P));
}

// ---------------------------------------------------------------- spawn
// Places history g into `slot` at queue position qpos; returns its sort key.
template <bool GRAD>
__device__ __forceinline__ uint32_t spawn_one(const Params &P, const State &S, int cur, unsigned int slot,
                                              unsigned long long g, unsigned int qpos, uint32_t k0, uint32_t k1,
                                              int &inst)
{
    inst = find_inst(P, g, inst);
    const InstDev &I = P.inst[inst];
    const unsigned long long local = g - (inst ? P.inst_end[inst - 1] : 0ull);
    Words r;
    r.init(0u, I.hist_offset + local, I.inst_id);
    float ox, oy, oz, dx, dy, dz;
    sample_birth(I, r, k0, k1, ox, oy, oz, dx, dy, dz);
    const float lam = -logf(r.u01(k0, k1));
    const uint32_t cell = dir_cell(P.face_bins, dx, dy, dz);
    Slot sl;
    sl.a.f = make_float4(0.0f, __uint_as_float(ray_tag(-1, I.birth_region)), I.E0, lam);
    sl.a.u = make_uint4(info_pack((uint32_t)inst, 0u, 0u, cell), 0u, __float_as_uint(0.0f), __float_as_uint(0.0f));
    sl.b.o = make_float4(ox, oy, oz, __uint_as_float(r.w));
    sl.b.d = make_float4(dx, dy, dz, __uint_as_float((uint32_t)local));
    S.slot[slot] = sl;
    if (GRAD) S.score[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const uint32_t key = sort_key(I.birth_region, P.face_bins, cell);
    S.queue[cur][qpos] = slot;
    S.qkey[cur][qpos] = key;
    return key;
}

template <bool GRAD>
__global__ void __launch_bounds__(256) spawn_kernel(const Params P, State S, int cur)
{
    const Ctrl &c = *S.ctrl;
    const unsigned int first = c.sp_free, filled = c.sp_filled, q0 = c.sp_q0;
    if (filled == 0) return;
    const unsigned long long head = c.sp_head;
    const uint32_t k0 = P.key0, k1 = P.key1;
    const int n_keys = P.n_keys;
    extern __shared__ unsigned int s_hist[];
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x) s_hist[k] = 0u;
    __syncthreads();
    int inst = 0;
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int base = blockIdx.x * blockDim.x; base < filled; base += stride) {   // warp-uniform
        const unsigned int i = base + threadIdx.x;
        const bool born = i < filled;
        uint32_t key = 0;
        if (born)
            key = spawn_one<GRAD>(P, S, cur, S.free_slots[first + i], S.pend[(head + i) & S.pend_mask], q0 + i, k0,
                                  k1, inst);
        warp_hist_add(born, key, s_hist);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x)
        if (s_hist[k]) atomicAdd(&S.hist[cur][k], s_hist[k]);
}

// ---------------------------------------------------------------- sort
constexpr int kSortPerThread = 16;

// Exclusive prefix of the key histogram of queue[cur]: the start of every bucket.
__global__ void __launch_bounds__(1024) sort_prefix_kernel(State S, int cur, int n_keys)
{
    const uint32_t FULL = 0xffffffffu;
    __shared__ unsigned int s_warp[32];
    constexpr int kpt = kMaxKeys / 1024;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int loc[kpt], sum = 0;
#pragma unroll
    for (int q = 0; q < kpt; ++q) {
        const int k = threadIdx.x * kpt + q;
        loc[q] = k < n_keys ? S.hist[cur][k] : 0u;
        sum += loc[q];
    }
    unsigned int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned int t = s_warp[lane];
        unsigned int x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int v = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += v;
        }
        s_warp[lane] = x - t;
    }
    __syncthreads();
    unsigned int pre = s_warp[warp] + inc - sum;
#pragma unroll
    for (int q = 0; q < kpt; ++q) {
        const int k = threadIdx.x * kpt + q;
        if (k < n_keys) S.base[k] = pre;
        pre += loc[q];
    }
}

// Counting sort of queue[cur] into qsort: each block takes a contiguous range,
// counts its keys, reserves room in every bucket it touches with one atomic per
// key and scatters.  Dynamic shared memory: 2 * n_keys words.
__global__ void __launch_bounds__(256) sort_kernel(State S, int cur, int n_keys)
{
    const uint32_t FULL = 0xffffffffu;
    extern __shared__ unsigned int s_sort[];
    unsigned int *s_base = s_sort, *s_cnt = s_sort + n_keys;
    const unsigned int n = S.ctrl->q_count[cur];
    const unsigned int begin = blockIdx.x * (256u * kSortPerThread);
    if (begin >= n) return;
    const unsigned int end = min(begin + 256u * kSortPerThread, n);
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < n_keys; k += 256) s_cnt[k] = 0u;
    __syncthreads();
    for (unsigned int i = begin + threadIdx.x; i < end; i += 256u) atomicAdd(&s_cnt[S.qkey[cur][i]], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < n_keys; k += 256)
        if (s_cnt[k]) {
            s_base[k] = S.base[k] + atomicAdd(&S.fill[k], s_cnt[k]);
            s_cnt[k] = 0u;
        }
    __syncthreads();
    for (unsigned int b = begin; b < end; b += 256u) {   // warp-uniform
        const unsigned int i = b + threadIdx.x;
        const bool valid = i < end;
        const uint32_t key = valid ? S.qkey[cur][i] : 0xffffffffu;
        const uint32_t peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        unsigned int off = 0;
        if (valid && lane == leader) off = atomicAdd(&s_cnt[key], (unsigned int)__popc(peers));
        off = __shfl_sync(FULL, off, leader) + __popc(peers & ((1u << lane) - 1u));
        if (valid) S.qsort[s_base[key] + off] = S.queue[cur][i];
    }
}

// ---------------------------------------------------------------- trace
constexpr int kFetchThreshold = 20;   // refill lanes when fewer are still traversing (8, 12, 20 measured)

// A query looks no further than the photon's sampled interaction point: the
// slot record carries E and lam, so t_best starts at t_cur + lam / mu (with a
// margin of 2^-10 relative + 1 um, above any rounding difference to the physics
// kernel's own d_int and to the plane distance).  Every surface closer than the
// interaction is still found, so physics decides exactly as with an unbounded
// query; when none is, the hit is marked kBeyond (an interaction follows).
template <bool COUNT>
__global__ void __launch_bounds__(256, 4) trace_kernel(const Params P, State S, int cur, unsigned long long *counters)
{
    const uint32_t FULL = 0xffffffffu;
    const float4 *__restrict__ nodes = P.nodes;
    const float4 *__restrict__ tris = P.tris;
    const float4 *__restrict__ planes = P.planes;
    __shared__ int4 s_reg[256];
    for (int i = threadIdx.x; i < P.n_region; i += blockDim.x) s_reg[i] = P.regions[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned int n = S.ctrl->q_count[cur];
    const unsigned int *queue = S.qsort;
    bool has = false;
    unsigned int qidx = 0;
    float ox = 0, oy = 0, oz = 0, t_min = 0, ix = 0, iy = 0, iz = 0, oix = 0, oiy = 0, oiz = 0, t_best = 0;
    int exclude = -1, node = kSentinel, leaf = 0, sp = 0, best = -1;
    bool ent = false, bounded = false, in_solid = false, reloc = false;
    ShearK sh{ 2, false, 0.0f, 0.0f, 1.0f };
    // stack entries: (child word, key of its box); an entry whose box is entered
    // beyond the nearest hit found since it was pushed is dropped when popped
    uint2 stack[kStack];
    uint32_t nn = 0, nb = 0, nt = 0, err = 0;
    auto pop = [&]() -> int {
        uint2 e = stack[sp--];
        while (__uint_as_float(e.y) > t_best) e = stack[sp--];
        return (int)e.x;
    };
    // warp-uniform private range [wb, we) of the queue, refilled a chunk at a time
    unsigned int wb = 0, we = 0;
    bool global_done = false, drained = false;
    while (true) {
        // ---- dynamic fetch: lanes without a ray take the next queue entries ----
        const uint32_t need = __ballot_sync(FULL, !has);
        if (need && !drained) {
            const unsigned int k = __popc(need);
            const unsigned int avail = we - wb;
            unsigned int nb = 0, ne = 0;
            if (avail < k && !global_done) {
                if (lane == 0) nb = atomicAdd(&S.ctrl->trace_head, (unsigned int)kTraceChunk);
                nb = __shfl_sync(FULL, nb, 0);
                if (nb >= n) { global_done = true; nb = ne = n; }
                else ne = min(nb + (unsigned int)kTraceChunk, n);
            }
            const unsigned int rank = __popc(need & ((1u << lane) - 1u));
            unsigned int idx = 0xffffffffu;
            if (rank < avail) idx = wb + rank;
            else if (nb + (rank - avail) < ne) idx = nb + (rank - avail);
            if (avail >= k) wb += k;
            else if (ne > nb) { wb = min(nb + (k - avail), ne); we = ne; }
            else wb = we;
            drained = global_done && wb >= we;
            if (!has && idx != 0xffffffffu) {
                qidx = idx;
                const Slot &sr = S.slot[queue[idx]];
                const SlotA sa = sr.a;
                S.hot[idx] = sa;        // physics reads it here, in queue order
                const float4 af = sa.f;
                const uint32_t pinst = sa.u.x & kInstMask;
                const float4 bo = sr.b.o, bd = sr.b.d;
                const float E = af.z, lam = af.w;
                const uint32_t tag = __float_as_uint(af.y);
                t_min = af.x;
                // the ray runs from the flight origin; surfaces count beyond the
                // distance already travelled along it (t_min)
                ox = bo.x; oy = bo.y; oz = bo.z;
                exclude = (int)(tag >> kTagShift) - 1;
                sh = make_shear_k(bd.x, bd.y, bd.z);
                ix = 1.0f / (fabsf(bd.x) > 1e-30f ? bd.x : copysignf(1e-30f, bd.x));
                iy = 1.0f / (fabsf(bd.y) > 1e-30f ? bd.y : copysignf(1e-30f, bd.y));
                iz = 1.0f / (fabsf(bd.z) > 1e-30f ? bd.z : copysignf(1e-30f, bd.z));
                oix = ox * ix; oiy = oy * iy; oiz = oz * iz;
                const int4 R = s_reg[tag & 255u];
                t_best = INFINITY;
                if (R.x >= 0) {
                    float pe, co, pa;
                    mu_at(P.xs + (size_t)R.x * P.n_grid, P.n_grid, P.lnE_min, P.inv_dlnE, E, pe, co, pa);
                    const int group = (R.y >> 1) - 1;
                    const float scl = group >= 0 ? __ldg(&P.inst[pinst].scale[group]) : 1.0f;
                    const float mu = (pe + co + pa) * scl;
                    if (mu > 0.0f) t_best = fmaf(lam / mu, 1.0f + 1.0f / 1024.0f, t_min) + 1e-3f;
                }
                bounded = t_best < INFINITY;
                in_solid = (tag & 255u) != 0u;
                reloc = false;
                best = -1;
                ent = false;
                stack[0] = make_uint2((uint32_t)kSentinel, 0u);
                sp = 0;
                const int root = R.w;
                node = root < 0 ? kSentinel : root;
                leaf = 0;
                has = true;
            }
        }
        if (__ballot_sync(FULL, has) == 0) break;
        // ---- traversal (while-while), left early when too few lanes remain ----
        while (has) {
            while ((unsigned)node < (unsigned)kSentinel) {
                uint32_t k0, k1, k2, k3;
                int4 cw;
                int nch;
                node4_keys(nodes, node, ix, iy, iz, oix, oiy, oiz, t_min, t_best, k0, k1, k2, k3, cw, nch);
                ++nn;
                if (COUNT) nb += nch;
                if (k0 == kMiss) {
                    node = pop();
                } else {
                    node = child_of(cw, k0);
                    if (k1 != kMiss) {      // push the others, farthest first
                        if (sp + 3 >= kStack) { err |= ERR_STACK; node = kSentinel; leaf = 0; best = -1; break; }
                        if (k3 != kMiss) stack[++sp] = make_uint2((uint32_t)child_of(cw, k3), k3);
                        if (k2 != kMiss) stack[++sp] = make_uint2((uint32_t)child_of(cw, k2), k2);
                        stack[++sp] = make_uint2((uint32_t)child_of(cw, k1), k1);
                    }
                }
                if (node < 0 && leaf >= 0) {
                    leaf = node;
                    node = pop();
                }
                if (!__any_sync(__activemask(), leaf >= 0)) break;
            }
            // the queue is sorted by dominant axis, so lanes of a warp take one branch
            while (leaf < 0) {
                if (sh.kz == 0) leaf_test_k<0>(tris, leaf, exclude, ox, oy, oz, sh, t_min, t_best, best, ent, nt);
                else if (sh.kz == 1) leaf_test_k<1>(tris, leaf, exclude, ox, oy, oz, sh, t_min, t_best, best, ent, nt);
                else leaf_test_k<2>(tris, leaf, exclude, ox, oy, oz, sh, t_min, t_best, best, ent, nt);
                leaf = node;
                if (node < 0) node = pop();
            }
            if (node == kSentinel && best < 0 && !bounded && in_solid && !reloc && !(err & ERR_STACK)) {
                // Inside a solid every ray meets the solid's boundary, so a photon whose
                // region tree has no surface ahead sits a rounding error past it (an
                // interaction point computed in FP32 right at a surface): search the
                // tree of every triangle instead; physics then takes the photon to the
                // region of the surface found, or to the world when there is none.
                reloc = true;
                stack[0] = make_uint2((uint32_t)kSentinel, 0u);
                sp = 0;
                leaf = 0;
                node = P.root_all < 0 ? kSentinel : P.root_all;
            }
            if (node == kSentinel) {
                Hit h;
                h.tri = best >= 0 ? __float_as_int(__ldg(&tris[3 * best + 1].w)) : -1;
                // the direction back from its reciprocals: the plane distance only
                // needs it to a few ulp
                h.t = best >= 0 ? plane_t(planes, h.tri, ox, oy, oz, __frcp_rn(ix), __frcp_rn(iy), __frcp_rn(iz), t_best,
                                          t_min)
                                : INFINITY;
                h.region = best >= 0 ? __float_as_int(__ldg(&tris[3 * best].w)) : 0;
                h.entering = (err & ERR_STACK) ? -2
                           : (best >= 0 ? (ent ? 1 : 0) + (reloc ? kRelocated : 0)
                                        : (reloc ? kRelocated : (bounded ? kBeyond : 0)));
                S.hit[qidx] = h;
                err = 0;
                has = false;
            }
            if (__popc(__activemask()) < kFetchThreshold && !drained) break;
        }
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)nn);
        atomicAdd(&counters[1], (unsigned long long)nt);
        atomicAdd(&counters[3], (unsigned long long)nb);
    }
}

// ---------------------------------------------------------------- physics
// Bounds on registers: with room for three blocks of 256 per SM, ptxas allocates the
// photon-only form without spilling in 64 registers (so four blocks still fit; under a
// four-block bound it spilled a few bytes and ran slower) and the charged-particle form
// in 80; the gradient form would take 69 and drop to three blocks per SM, slower than
// its small spill at four, so it keeps the four-block bound.
template <bool GRAD, bool COUNT, bool EM>
__global__ void __launch_bounds__(256, GRAD ? 4 : 3) physics_kernel(const Params P, State S, int cur,
                                                      unsigned long long *counters)
{
    const uint32_t FULL = 0xffffffffu;
    const int nxt = cur ^ 1;
    // shared: region table (material slot, flags, parent, root), then block tallies
    extern __shared__ int4 s_reg[];
    __shared__ unsigned int s_cnt[3], s_base[3];    // queue, free slots, deferred tracks
    for (int i = threadIdx.x; i < P.n_region; i += blockDim.x) s_reg[i] = P.regions[i];
    BlockTally<GRAD> bt;
    bt.init(s_reg + P.n_region, P.n_inst);
    // key histogram of the next queue, after the block tallies
    unsigned int *s_hist = reinterpret_cast<unsigned int *>(
        reinterpret_cast<char *>(s_reg + P.n_region) + block_tally_bytes<GRAD>(P.n_inst));
    const int n_keys = P.n_keys;
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x) s_hist[k] = 0u;
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const unsigned int n = S.ctrl->q_count[cur];
    const int lane = threadIdx.x & 31;
    const uint32_t k0 = P.key0, k1 = P.key1;
    TravStats ts{};
    uint32_t inter_acc = 0;             // interactions of instance inter_inst not yet tallied
    int inter_inst = 0;
    const unsigned int stride = gridDim.x * blockDim.x;
    for (unsigned int base = blockIdx.x * blockDim.x; base < n; base += stride) {   // block-uniform
        // last queue entry first: the trace kernel handed out its queue from the
        // front, so the records it touched last are the likeliest still in L2
        const unsigned int jf = base + threadIdx.x;
        const bool mine = jf < n;
        const unsigned int j = mine ? n - 1u - jf : 0u;
        const unsigned int slot = mine ? S.qsort[j] : 0u;
        bool alive_slot = false, finished = false;
        uint32_t key = 0;
        int inst = 0;
        float edep_out = 0.0f;
        uint32_t herr_out = 0;
        bool fep_out = false;
        float dep_all_out = 0.0f, esc_out = 0.0f;
        uint32_t segs_out = 0;
        bool defer = false;             // EM: a track left to etrack_kernel
        Track tr;
        if (mine) {
            const Hit ht = S.hit[j];
            // the slot's first half as the trace kernel found it (nothing writes the
            // slot between the two kernels), in queue order: a coalesced read
            const SlotA sa = S.hot[j];
            float t_cur = sa.f.x;
            const uint32_t tag = __float_as_uint(sa.f.y);
            float E = sa.f.z, lam = sa.f.w;
            float edep = __uint_as_float(sa.u.z), dep_all = __uint_as_float(sa.u.w);
            const uint32_t info = sa.u.x;
            inst = (int)(info & kInstMask);
            uint32_t herr = (info >> kErrShift) & kErrMask, flags = (info >> kFlagShift) & kFlagMask;
            uint32_t cell = info >> kCellShift, steps = sa.u.y;
            int region = (int)(tag & 255u);
            int last_tri = (int)(tag >> kTagShift) - 1;
            const float4 sc4 = GRAD ? S.score[slot] : make_float4(0, 0, 0, 0);
            float score[4] = { sc4.x, sc4.y, sc4.z, sc4.w };
            const InstDev &I = P.inst[inst];
            // the slot's second half (flight origin, direction, random-number state),
            // loaded only by an interaction or a waiting annihilation photon
            bool have_b = false;
            float4 bo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), bd = bo;
            uint32_t local = 0;
            Words r;
            auto load_b = [&]() {
                if (have_b) return;
                const SlotB sb = S.slot[slot].b;
                bo = sb.o;
                bd = sb.d;
                local = __float_as_uint(sb.d.w);
                r.init(__float_as_uint(sb.o.w), I.hist_offset + local, I.inst_id);
                have_b = true;
            };
            float esc_now = 0.0f;       // energy escaping in this segment
            if (inst != inter_inst) {
                if (inter_acc) atomicAdd(&bt.t[inter_inst].inter, inter_acc);
                inter_acc = 0;
                inter_inst = inst;
            }
            if (ht.entering == -2) herr |= ERR_STACK;
            if (++steps > (uint32_t)P.step_cap) herr |= ERR_STEPCAP;
            if (herr) {
                finished = true;
            } else {
                const float t_hit = ht.t;
                const int hit_tri = ht.tri, hit_region = ht.region;
                const bool entering = ht.entering == 1 || ht.entering == 1 + kRelocated;
                if (ht.entering >= kRelocated) {
                    // the trace kernel relocated the photon (a rounding error past a
                    // boundary) by the nearest surface of the whole mesh; with none
                    // ahead it is outside every solid
                    if (COUNT) ts.relocated++;
                    if (hit_tri < 0) region = 0;
                }
                // region record: material slot, active | (group + 1) << 1, parent, tree root
                const int4 R = s_reg[region];
                const int group = (R.y >> 1) - 1;
                float pe = 0.0f, co = 0.0f, pa = 0.0f;
                if (R.x >= 0) mu_at(P.xs + (size_t)R.x * P.n_grid, P.n_grid, P.lnE_min, P.inv_dlnE, E, pe, co, pa);
                const float mu_unit = pe + co + pa;
                const float scl = group >= 0 ? I.scale[group] : 1.0f;
                const float mu = mu_unit * scl;
                const float d_int = mu > 0.0f ? lam / mu : INFINITY;
                bool photon_done = false;
                if (herr) {
                    finished = true;
                } else if (d_int < t_hit - t_cur) {
                    // ---- interaction ----
                    load_b();
                    ++inter_acc;
                    if (GRAD && group >= 0 && group < 4) score[group] += 1.0f / scl - mu_unit * d_int;
                    const float tt = t_cur + d_int;
                    const float px = fmaf(tt, bd.x, bo.x), py = fmaf(tt, bd.y, bo.y), pz = fmaf(tt, bd.z, bo.z);
                    const float u = r.u01(k0, k1) * mu_unit;
                    float dep = 0.0f;
                    // charged particles of e_model 1: kinetic energy, direction, count
                    float eT = 0.0f, eux = bd.x, euy = bd.y, euz = bd.z, ew = 1.0f;
                    if (u < pe) {
                        if (EM) eT = E;
                        else dep = E;
                        E = 0.0f; photon_done = true;
                    } else if (u < pe + co || pa == 0.0f) {
                        const float k = E * (1.0f / kMeC2);
                        const float a2k = 1.0f + 2.0f * k;
                        const float br = a2k / (9.0f + 2.0f * k);
                        float x = 1.0f;
                        bool ok = false;
                        for (int trial = 0; trial < 1000; ++trial) {
                            const float r1 = r.u01(k0, k1), r2 = r.u01(k0, k1), r3 = r.u01(k0, k1);
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
                            sincospif(2.0f * r.u01(k0, k1), &sp, &cp);
                            const float Ep = E / x;
                            rotate(bd.x, bd.y, bd.z, c, sp, cp);
                            if (EM) {
                                eT = E - Ep;
                                const float qx = E * eux - Ep * bd.x, qy = E * euy - Ep * bd.y,
                                            qz = E * euz - Ep * bd.z;
                                const float ql = sqrtf(qx * qx + qy * qy + qz * qz);
                                if (ql > 0.0f) { eux = qx / ql; euy = qy / ql; euz = qz / ql; }
                            } else {
                                dep = E - Ep;
                            }
                            E = Ep;
                            if (E < P.e_cut) { dep += E; E = 0.0f; photon_done = true; }
                        }
                    } else {
                        if (EM) { eT = 0.5f * (E - kTwoMeC2); ew = 2.0f; }
                        else dep = E - kTwoMeC2;
                        const float c = 2.0f * r.u01(k0, k1) - 1.0f;
                        float sp, cp;
                        sincospif(2.0f * r.u01(k0, k1), &sp, &cp);
                        const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
                        const float nx = s * cp, ny = s * sp, nz = c;
                        E = kMeC2;
                        bd.x = nx; bd.y = ny; bd.z = nz;
                        flags |= kFlagSec;
                        Sec sc;
                        sc.p = make_float4(px, py, pz, 0.0f);
                        sc.d = make_float4(-nx, -ny, -nz, __int_as_float(region));
                        S.sec[slot] = sc;
                    }
                    if (R.y & 1) edep += dep;
                    dep_all += dep;
                    if (EM && eT > 0.0f && !herr) {
                        if (!photon_done || (flags & kFlagSec)) {
                            // the history goes on: etrack_kernel adds the track's deposits
                            // to the slot before its next visit, with full warps
                            defer = true;
                            tr.p = make_float4(px, py, pz, eT);
                            tr.u = make_float4(eux, euy, euz, ew);
                            tr.slot = slot;
                            tr.tag = (uint32_t)region | ((uint32_t)inst << 8);
                        } else {
                            float e_esc = 0.0f;
                            e_track<COUNT>(P, s_reg, I.scale, px, py, pz, eux, euy, euz, eT, ew, region, edep,
                                           dep_all, e_esc, herr, ts);
                            esc_now += e_esc;
                        }
                    }
                    bo.x = px; bo.y = py; bo.z = pz;
                    t_cur = 0.0f;
                    last_tri = -1;
                    if (herr) finished = true;
                    else if (!photon_done) lam = -logf(r.u01(k0, k1));
                } else if (hit_tri < 0) {
                    if (region != 0) herr |= ERR_LOST;
                    esc_now = E;
                    E = 0.0f;
                    photon_done = true;
                    if (herr) finished = true;
                } else {
                    // ---- boundary crossing ----
                    const float len = t_hit - t_cur;
                    lam -= mu * len;
                    if (GRAD && group >= 0 && group < 4) score[group] -= mu_unit * len;
                    t_cur = t_hit;
                    last_tri = hit_tri;
                    region = entering ? hit_region : s_reg[hit_region].z;
                }
                if (esc_now != 0.0f) {
                    // escaped energy of this history so far, kept in the slot while the
                    // history goes on (a pending annihilation photon, or the photon
                    // itself after a charged particle escaped)
                    if (flags & kFlagEsc) esc_now += S.esc[slot];
                    flags |= kFlagEsc;
                    if (!finished && ((flags & kFlagSec) || !photon_done)) S.esc[slot] = esc_now;
                }
                if (photon_done && !finished) {
                    if (flags & kFlagSec) {
                        load_b();
                        const Sec sc = S.sec[slot];
                        flags &= ~kFlagSec;
                        region = __float_as_int(sc.d.w);
                        bo.x = sc.p.x; bo.y = sc.p.y; bo.z = sc.p.z;
                        t_cur = 0.0f;
                        bd.x = sc.d.x; bd.y = sc.d.y; bd.z = sc.d.z;
                        last_tri = -1;
                        E = kMeC2;
                        lam = -logf(r.u01(k0, k1));
                    } else {
                        finished = true;
                    }
                }
                if (!finished && !((!have_b || isfinite(bd.x)) && isfinite(E) && isfinite(lam))) {
                    herr |= ERR_NONFINITE;
                    finished = true;
                }
            }
            herr_out = herr;
            edep_out = edep;
            if (!finished) {
                // a crossing keeps the direction (and its key cell) and the second half
                if (have_b) cell = dir_cell(P.face_bins, bd.x, bd.y, bd.z);
                SlotA na;
                na.f = make_float4(t_cur, __uint_as_float(ray_tag(last_tri, region)), E, lam);
                na.u = make_uint4(info_pack((uint32_t)inst, herr, flags, cell), steps, __float_as_uint(edep),
                                  __float_as_uint(dep_all));
                S.slot[slot].a = na;
                if (have_b) {
                    SlotB nb;
                    nb.o = make_float4(bo.x, bo.y, bo.z, __uint_as_float(r.w));
                    nb.d = make_float4(bd.x, bd.y, bd.z, __uint_as_float(local));
                    S.slot[slot].b = nb;
                }
                if (GRAD) S.score[slot] = make_float4(score[0], score[1], score[2], score[3]);
                key = sort_key(region, P.face_bins, cell);
                alive_slot = true;
            } else {
                float esc = 0.0f;
                if (flags & kFlagEsc) esc = esc_now != 0.0f ? esc_now : S.esc[slot];
                const bool fep = !herr && (I.E0 - edep) <= P.fep_delta;
                if (GRAD) {
                    bt.history(inst, steps, herr, fep, edep, dep_all, esc, P.e_max, score);
                } else {
                    fep_out = fep; dep_all_out = dep_all; esc_out = esc; segs_out = steps;
                }
                if (P.n_trace) {
                    const uint32_t loc = have_b ? local : __float_as_uint(S.slot[slot].b.d.w);
                    const unsigned long long g = (inst ? P.inst_end[inst - 1] : 0ull) + loc;
                    if (g < P.n_trace) P.edep_trace[g] = herr ? -1.0f : edep;
                }
            }
        }
        if (!GRAD) bt.history_warp(finished, inst, segs_out, herr_out, fep_out, edep_out, dep_all_out, esc_out, P.e_max);
        // ---- spectrum atomics (warp-aggregated per bin) ----
        const bool binned = finished && herr_out == 0u && edep_out > 0.0f && edep_out < P.e_max;
        int bin = 0;
        if (binned) bin = min((int)(edep_out * P.bin_scale), P.n_bins - 1);
        const uint32_t bkey = binned ? (uint32_t)(inst * P.n_bins + bin) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(FULL, bkey);
        if (binned && lane == __ffs(peers) - 1)
            atomicAdd(&P.spectra[(size_t)inst * P.n_bins + bin], (uint32_t)__popc(peers));
        // ---- queue / free-list appends: one global atomic per list, block and pass ----
        const bool dt = EM && defer && alive_slot;     // the history goes on (no error either)
        const uint32_t ma = __ballot_sync(FULL, alive_slot), mf = __ballot_sync(FULL, finished);
        const uint32_t mt = EM ? __ballot_sync(FULL, dt) : 0u;
        unsigned int oa = 0, of = 0, ot = 0;
        if (lane == 0) {
            if (ma) oa = atomicAdd(&s_cnt[0], (unsigned int)__popc(ma));
            if (mf) of = atomicAdd(&s_cnt[1], (unsigned int)__popc(mf));
            if (EM && mt) ot = atomicAdd(&s_cnt[2], (unsigned int)__popc(mt));
        }
        const uint32_t below = (1u << lane) - 1u;
        oa = __shfl_sync(FULL, oa, 0) + __popc(ma & below);
        of = __shfl_sync(FULL, of, 0) + __popc(mf & below);
        if (EM) ot = __shfl_sync(FULL, ot, 0) + __popc(mt & below);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base[0] = s_cnt[0] ? atomicAdd(&S.ctrl->q_count[nxt], s_cnt[0]) : 0u;
            s_base[1] = s_cnt[1] ? atomicAdd(&S.ctrl->free_top, s_cnt[1]) : 0u;
            if (EM) s_base[2] = s_cnt[2] ? atomicAdd(&S.ctrl->t_count, s_cnt[2]) : 0u;
            s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
        }
        __syncthreads();
        if (EM && dt) S.trk[s_base[2] + ot] = tr;
        if (alive_slot) {
            S.queue[nxt][s_base[0] + oa] = slot;
            S.qkey[nxt][s_base[0] + oa] = key;
        }
        if (finished) S.free_slots[s_base[1] + of] = slot;
        warp_hist_add(alive_slot, key, s_hist);
    }
    if (inter_acc) atomicAdd(&bt.t[inter_inst].inter, inter_acc);
    bt.flush(block_tally(P));     // starts with a barrier
    for (int k = threadIdx.x; k < n_keys; k += blockDim.x)
        if (s_hist[k]) atomicAdd(&S.hist[nxt][k], s_hist[k]);
    if (COUNT) {
        if (ts.nodes) atomicAdd(&counters[0], (unsigned long long)ts.nodes);
        if (ts.boxes) atomicAdd(&counters[3], (unsigned long long)ts.boxes);
        if (ts.tris) atomicAdd(&counters[1], (unsigned long long)ts.tris);
        if (ts.relocated) atomicAdd(&counters[2], (unsigned long long)ts.relocated);
    }
}

// ---------------------------------------------------------------- etrack
// The charged-particle tracks physics deferred in this iteration (e_model 1), one
// per thread: their deposits and escapes join the history in its slot, and an
// error of the track becomes the history's, before the slot's next physics visit.
template <bool COUNT>
__global__ void __launch_bounds__(256) etrack_kernel(const Params P, State S, unsigned long long *counters)
{
    __shared__ int4 s_reg[256];
    for (int i = threadIdx.x; i < P.n_region; i += blockDim.x) s_reg[i] = P.regions[i];
    __syncthreads();
    const unsigned int n = S.ctrl->t_count;
    TravStats ts{};
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Track t = S.trk[i];
        const int region = (int)(t.tag & 255u), inst = (int)(t.tag >> 8);
        float edep = 0.0f, dep_all = 0.0f, esc = 0.0f;
        uint32_t herr = 0;
        e_track<COUNT>(P, s_reg, P.inst[inst].scale, t.p.x, t.p.y, t.p.z, t.u.x, t.u.y, t.u.z, t.p.w, t.u.w, region,
                       edep, dep_all, esc, herr, ts);
        SlotA &a = S.slot[t.slot].a;
        uint4 u = a.u;
        u.z = __float_as_uint(__uint_as_float(u.z) + edep);
        u.w = __float_as_uint(__uint_as_float(u.w) + dep_all);
        if (esc != 0.0f) {
            const bool had = ((u.x >> kFlagShift) & kFlagEsc) != 0u;
            S.esc[t.slot] = (had ? S.esc[t.slot] : 0.0f) + esc;
            u.x |= (uint32_t)kFlagEsc << kFlagShift;
        }
        u.x |= (herr & kErrMask) << kErrShift;
        a.u = u;
    }
    if (COUNT) {
        if (ts.nodes) atomicAdd(&counters[0], (unsigned long long)ts.nodes);
        if (ts.boxes) atomicAdd(&counters[3], (unsigned long long)ts.boxes);
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
    // executable graph of the last run launched outside stream capture, and the
    // bytes of the arguments it was built for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> graph_key;
    void *trk = nullptr;             // deferred-track records, allocated by the first e_model 1 run
};

int wavefront_trace_grid(const WavefrontBuffers *w) { return w ? w->trace_grid : 0; }

bool wavefront_supports(int n_region, long long n_mesh_tri)
{
    return n_region >= 1 && n_region <= 256 && n_mesh_tri <= wf::kMaxTriId;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

gadep_status wavefront_create(int device, int slots, bool grad, WavefrontBuffers **out)
{
    *out = nullptr;
    if (slots < 1024 || slots > (1 << 26)) return fail(GADEP_E_INVAL, "wavefront: slots must be in [1024, 2^26]");
    WavefrontBuffers *w = new (std::nothrow) WavefrontBuffers();
    if (!w) return fail(GADEP_E_NOMEM, "wavefront: out of host memory");
    int n_sm = 0, bps = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (void *)wf::trace_kernel<false>, 256, 0);
    w->trace_grid = n_sm * std::max(bps, 1);
    w->work_grid = n_sm * 8;
    // ring of pending births: gen stops claiming once it holds `slots` (the most a
    // spawn can take); every gen block may complete one more chunk after that
    const unsigned long long target = (unsigned long long)slots;
    const unsigned long long need = 2 * target + (unsigned long long)w->work_grid * wf::kGenChunk;
    unsigned long long ring = 1;
    while (ring < need) ring <<= 1;
    const size_t n = (size_t)slots;
    size_t off = 0;
    size_t o_slot = off; off = align_up(off + n * sizeof(wf::Slot));
    size_t o_sec = off; off = align_up(off + n * sizeof(wf::Sec));
    size_t o_esc = off; off = align_up(off + n * sizeof(float));
    size_t o_score = off; off = align_up(off + n * sizeof(float4));   // always: buffers serve both forms
    (void)grad;
    size_t o_hit = off; off = align_up(off + n * sizeof(wf::Hit));
    size_t o_hot = off; off = align_up(off + n * sizeof(wf::SlotA));
    size_t o_q0 = off; off = align_up(off + n * 4);
    size_t o_q1 = off; off = align_up(off + n * 4);
    size_t o_k0 = off; off = align_up(off + n * 4);
    size_t o_k1 = off; off = align_up(off + n * 4);
    size_t o_qs = off; off = align_up(off + n * 4);
    size_t o_h = off; off = align_up(off + 4 * wf::kMaxKeys * 4);
    size_t o_d0 = off; off = align_up(off + n * 4);
    size_t o_pend = off; off = align_up(off + ring * sizeof(unsigned long long));
    size_t o_ctrl = off; off = align_up(off + sizeof(wf::Ctrl));
    size_t o_qlog = off; off = align_up(off + sizeof(unsigned int) * wf::kQueueLog);
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
    w->S.slot = (wf::Slot *)(b + o_slot);
    w->S.sec = (wf::Sec *)(b + o_sec);
    w->S.esc = (float *)(b + o_esc);
    w->S.score = (float4 *)(b + o_score);
    w->S.hit = (wf::Hit *)(b + o_hit);
    w->S.hot = (wf::SlotA *)(b + o_hot);
    w->S.queue[0] = (unsigned int *)(b + o_q0);
    w->S.queue[1] = (unsigned int *)(b + o_q1);
    w->S.qkey[0] = (unsigned int *)(b + o_k0);
    w->S.qkey[1] = (unsigned int *)(b + o_k1);
    w->S.qsort = (unsigned int *)(b + o_qs);
    w->S.hist[0] = (unsigned int *)(b + o_h);
    w->S.hist[1] = w->S.hist[0] + wf::kMaxKeys;
    w->S.fill = w->S.hist[1] + wf::kMaxKeys;
    w->S.base = w->S.fill + wf::kMaxKeys;
    w->S.free_slots = (unsigned int *)(b + o_d0);
    w->S.pend = (unsigned long long *)(b + o_pend);
    w->S.pend_mask = ring - 1;
    w->S.gen_target = target;
    w->S.ctrl = (wf::Ctrl *)(b + o_ctrl);
    w->S.qlog = (unsigned int *)(b + o_qlog);
    w->S.slots = slots;
    *out = w;
    return GADEP_OK;
}

void wavefront_destroy(WavefrontBuffers *w)
{
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    cudaFree(w->trk);
    cudaFree(w->block);
    cudaFreeHost(w->host_ctrl);
    delete w;
}

// Run every history of the plan's Params through the wavefront kernels on `s`.
gadep_status wavefront_run(WavefrontBuffers *w, const dev::Params &P0, bool grad, bool count,
                           unsigned long long *counters, KernelTimer *timer, cudaStream_t s, int slots)
{
    if (P0.e_model && !w->trk) {
        void *t = nullptr;
        if (cudaMalloc(&t, (size_t)w->S.slots * sizeof(wf::Track)) != cudaSuccess) {
            cudaGetLastError();
            return fail(GADEP_E_NOMEM, "wavefront: cudaMalloc of the track records failed");
        }
        w->trk = t;
        w->S.trk = (wf::Track *)t;
    }
    wf::State S = w->S;
    // a run may keep fewer photons in flight than the (cached, largest-seen)
    // buffers hold: its free-slot stack and birth target cover only those slots
    if (slots > 0 && slots < S.slots) {
        S.slots = slots;
        S.gen_target = (unsigned long long)slots;
    }
    dev::Params P = P0;
    P.face_bins = wf::face_bins_for(P.n_region);
    P.n_keys = P.n_region * 6 * P.face_bins * P.face_bins;
    if (P.n_inst > kWavefrontMaxInstances)
        return fail(GADEP_E_INVAL, "wavefront: at most %d instances per run", kWavefrontMaxInstances);
    if (!wavefront_supports(P.n_region, 0)) return fail(GADEP_E_INVAL, "wavefront: too many regions");
    // dynamic shared memory: block tallies (gen); region table + block tallies (physics)
    const size_t gsm = wf::block_tally_bytes<false>(P.n_inst);
    const size_t ksm = (size_t)P.n_keys * sizeof(unsigned int);   // key histogram (spawn)
    const size_t ssm = 2 * ksm;                                    // bucket starts and counts (sort)
    const size_t rsm = (size_t)P.n_region * sizeof(int4) +
                       (grad ? wf::block_tally_bytes<true>(P.n_inst) : wf::block_tally_bytes<false>(P.n_inst)) +
                       (size_t)P.n_keys * sizeof(unsigned int);
    {
        cudaError_t e = cudaSuccess;
        auto set = [&](const void *f, size_t b) {
            if (e == cudaSuccess && b > 40 * 1024)
                e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
        };
        set((const void *)wf::gen_kernel, gsm);
        set((const void *)wf::sort_kernel, ssm);
        set((const void *)wf::physics_kernel<true, true, false>, rsm);
        set((const void *)wf::physics_kernel<true, false, false>, rsm);
        set((const void *)wf::physics_kernel<false, true, false>, rsm);
        set((const void *)wf::physics_kernel<false, false, false>, rsm);
        set((const void *)wf::physics_kernel<false, true, true>, rsm);
        set((const void *)wf::physics_kernel<false, false, true>, rsm);
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: shared memory: %s", cudaGetErrorString(e));
    }
    const unsigned long long max_iter = (unsigned long long)P.step_cap * 4 + P.total / 1024 + 1000000ull;
    const int sort_grid = (S.slots + 256 * wf::kSortPerThread - 1) / (256 * wf::kSortPerThread);
    // the kernels of the run, in order (cur = -1: the pre-loop part)
    const unsigned long long total = P.total;
    const int n_keys = P.n_keys;
    auto launch = [&](int kind, int cur, cudaGraph_t g, const cudaGraphNode_t *dep, size_t n_dep,
                      cudaGraphNode_t *node, cudaGraphConditionalHandle loop, int in_graph) -> cudaError_t {
        const void *fn = nullptr;
        dim3 grid(1), block(256);
        size_t smem = 0;
        int c = cur < 0 ? 1 : cur;
        void *args[8];
        switch (kind) {
        case KK_INIT: fn = (const void *)wf::init_kernel; grid = dim3((S.slots + 255) / 256);
            args[0] = &S; args[1] = (void *)&max_iter; break;
        case KK_GEN: fn = (const void *)wf::gen_kernel; grid = dim3(w->work_grid); smem = gsm;
            args[0] = &P; args[1] = &S; break;
        case KK_CTRL: fn = (const void *)wf::ctrl_kernel;
            args[0] = &S; args[1] = &c; args[2] = (void *)&total; args[3] = &loop; args[4] = &in_graph; break;
        case KK_SPAWN: fn = grad ? (const void *)wf::spawn_kernel<true> : (const void *)wf::spawn_kernel<false>;
            grid = dim3(w->work_grid); smem = ksm; args[0] = &P; args[1] = &S; args[2] = &c; break;
        case KK_SORT: fn = (const void *)wf::sort_kernel; grid = dim3(sort_grid); smem = ssm;
            args[0] = &S; args[1] = &c; args[2] = (void *)&n_keys; break;
        case KK_N: fn = (const void *)wf::sort_prefix_kernel; block = dim3(1024);   // the sort's prefix
            args[0] = &S; args[1] = &c; args[2] = (void *)&n_keys; break;
        case KK_TRACE: fn = count ? (const void *)wf::trace_kernel<true> : (const void *)wf::trace_kernel<false>;
            grid = dim3(w->trace_grid);
            args[0] = &P; args[1] = &S; args[2] = &c; args[3] = &counters; break;
        case KK_PHYSICS:
            if (grad)
                fn = count ? (const void *)wf::physics_kernel<true, true, false>
                           : (const void *)wf::physics_kernel<true, false, false>;
            else if (P.e_model)
                fn = count ? (const void *)wf::physics_kernel<false, true, true>
                           : (const void *)wf::physics_kernel<false, false, true>;
            else
                fn = count ? (const void *)wf::physics_kernel<false, true, false>
                           : (const void *)wf::physics_kernel<false, false, false>;
            grid = dim3(w->work_grid); smem = rsm; args[0] = &P; args[1] = &S; args[2] = &c; args[3] = &counters; break;
        case KK_ETRACK: fn = count ? (const void *)wf::etrack_kernel<true> : (const void *)wf::etrack_kernel<false>;
            grid = dim3(w->work_grid); args[0] = &P; args[1] = &S; args[2] = &counters; break;
        default: return cudaErrorInvalidValue;
        }
        if (!g) return cudaLaunchKernel(fn, grid, block, args, smem, s);
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void *>(fn);
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = (unsigned int)smem;
        kp.kernelParams = args;
        kp.extra = nullptr;
        return cudaGraphAddKernelNode(node, g, dep, n_dep, &kp);
    };
    // the kernels of one iteration; the deferred charged-particle tracks run right
    // after physics
    int kIteration[8] = { KK_SPAWN, KK_N, KK_SORT, KK_TRACE, KK_PHYSICS, KK_GEN, KK_CTRL, KK_CTRL };
    int n_iter = 7;
    if (P.e_model) {
        kIteration[5] = KK_ETRACK;
        kIteration[6] = KK_GEN;
        kIteration[7] = KK_CTRL;
        n_iter = 8;
    }
    KernelTimer none;
    KernelTimer &T = timer ? *timer : none;

    if (!T.timing) {
        // ---- graph: init, gen, ctrl, then WHILE(condition) { two iterations } ----
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: stream query: %s", cudaGetErrorString(e));
        const bool capturing = cap == cudaStreamCaptureStatusActive;
        // graph arguments: the bytes of everything the nodes capture
        std::vector<unsigned char> key(sizeof(P) + sizeof(S) + 16);
        std::memcpy(key.data(), &P, sizeof(P));
        std::memcpy(key.data() + sizeof(P), &S, sizeof(S));
        unsigned char *kx = key.data() + sizeof(P) + sizeof(S);
        kx[0] = grad; kx[1] = count;
        std::memcpy(kx + 8, &counters, sizeof(counters));
        if (!capturing && w->exec && key == w->graph_key) {
            e = cudaGraphLaunch(w->exec, s);
            return e == cudaSuccess ? GADEP_OK : fail(GADEP_E_CUDA, "wavefront: graph launch: %s", cudaGetErrorString(e));
        }
        cudaGraph_t g = nullptr;
        std::vector<cudaGraphNode_t> deps;
        if (capturing) {
            const cudaGraphNode_t *d = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(s, &cap, nullptr, &g, &d, nullptr, &nd);
            if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: capture info: %s", cudaGetErrorString(e));
            deps.assign(d, d + nd);
        } else {
            if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
            if (w->graph) { cudaGraphDestroy(w->graph); w->graph = nullptr; }
            w->graph_key.clear();
            if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess)
                return fail(GADEP_E_CUDA, "wavefront: graph: %s", cudaGetErrorString(e));
            w->graph = g;
        }
        cudaGraphConditionalHandle loop = 0;
        e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNode_t prev = nullptr, node = nullptr;
        const int pre[] = { KK_INIT, KK_GEN, KK_CTRL };
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            if (prev) e = launch(pre[k], -1, g, &prev, 1, &node, loop, 0);
            else e = launch(pre[k], -1, g, deps.data(), deps.size(), &node, loop, 0);
            prev = node;
        }
        cudaGraphNode_t loop_node = nullptr;
        if (e == cudaSuccess) {
            cudaGraphNodeParams cp{};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = loop;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&loop_node, g, &prev, nullptr, 1, &cp);
            if (e == cudaSuccess) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                cudaGraphNode_t bprev = nullptr;
                for (int cur = 0; cur < 2 && e == cudaSuccess; ++cur)
                    for (int k = 0; k < n_iter && e == cudaSuccess; ++k) {
                        e = launch(kIteration[k], cur, body, bprev ? &bprev : nullptr, bprev ? 1 : 0, &node, loop, 1);
                        bprev = node;
                    }
            }
        }
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: graph build: %s", cudaGetErrorString(e));
        if (capturing) {
            e = cudaStreamUpdateCaptureDependencies(s, &loop_node, nullptr, 1, cudaStreamSetCaptureDependencies);
            return e == cudaSuccess ? GADEP_OK : fail(GADEP_E_CUDA, "wavefront: capture: %s", cudaGetErrorString(e));
        }
        if ((e = cudaGraphInstantiate(&w->exec, g, 0)) != cudaSuccess) {
            w->exec = nullptr;
            return fail(GADEP_E_CUDA, "wavefront: graph instantiation: %s", cudaGetErrorString(e));
        }
        w->graph_key = key;
        e = cudaGraphLaunch(w->exec, s);
        return e == cudaSuccess ? GADEP_OK : fail(GADEP_E_CUDA, "wavefront: graph launch: %s", cudaGetErrorString(e));
    }

    // ---- host loop with a CUDA event pair around every kernel (timing) ----
    const int pre[] = { KK_INIT, KK_GEN, KK_CTRL };
    for (int k = 0; k < 3; ++k) {
        T.before(s);
        const cudaError_t e = launch(pre[k], -1, nullptr, nullptr, 0, nullptr, 0, 0);
        T.after(pre[k], s);
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: launch: %s", cudaGetErrorString(e));
    }
    const int check_every = 16;
    for (unsigned long long it = 0;; ++it) {
        const int cur = (int)(it & 1);
        for (int k = 0; k < n_iter; ++k) {
            const int kind = kIteration[k];
            if (kind != KK_SORT) T.before(s);      // the prefix and the sort are timed together
            const cudaError_t e = launch(kind, cur, nullptr, nullptr, 0, nullptr, 0, 0);
            if (kind != KK_N) T.after(kind, s);
            if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: launch: %s", cudaGetErrorString(e));
        }
        if (it % check_every == check_every - 1) {
            cudaError_t e = cudaMemcpyAsync(w->host_ctrl, S.ctrl, sizeof(wf::Ctrl), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: control read: %s", cudaGetErrorString(e));
            if (w->host_ctrl->done == 1) return GADEP_OK;
            if (w->host_ctrl->done == 2)
                return fail(GADEP_E_TIMEOUT, "wavefront: iteration bound reached with photons still alive");
        }
    }
}

// After a run has completed on `s`: the trace queue size of each of its
// iterations (at most `max`, and at most the first kQueueLog); returns the count.
gadep_status wavefront_queue_log(WavefrontBuffers *w, uint32_t *out, int max, int *n, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(w->host_ctrl, w->S.ctrl, sizeof(wf::Ctrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: queue log: %s", cudaGetErrorString(e));
    const int iters = (int)std::min<unsigned int>(w->host_ctrl->qlog_n, (unsigned int)wf::kQueueLog);
    const int k = std::max(0, std::min(iters, max));
    if (k > 0) {
        e = cudaMemcpyAsync(out, w->S.qlog, sizeof(uint32_t) * (size_t)k, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: queue log: %s", cudaGetErrorString(e));
    }
    *n = k;
    return GADEP_OK;
}

// After a run has completed on `s` (the caller synchronised it): the iteration
// bound status of the control block.
gadep_status wavefront_check(WavefrontBuffers *w, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(w->host_ctrl, w->S.ctrl, sizeof(wf::Ctrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GADEP_E_CUDA, "wavefront: control read: %s", cudaGetErrorString(e));
    if (w->host_ctrl->done == 2)
        return fail(GADEP_E_TIMEOUT, "wavefront: iteration bound reached with photons still alive");
    return GADEP_OK;
}

}  // namespace gadep
