// transport_common.cuh -- records and device helpers shared by the transport
// kernels (persistent megakernel and wavefront kernels).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "gadep.h"

namespace gadep {
namespace dev {

struct InstDev {
    float E0;
    int32_t src_kind;
    float px, py, pz;
    float dx, dy, dz;
    float radius, height;
    int32_t n_sides;
    int32_t birth_region;
    uint32_t inst_id;
    uint32_t pad0;
    unsigned long long hist_offset;
    float scale[GADEP_MAX_GROUPS];
};

struct TallyDev {
    unsigned long long n_hist, n_fep, n_zero, n_over, n_err, n_segments, n_interactions, n_culled;
    unsigned long long err_bits;
    double sum_dep_active, sum_dep_all, sum_esc;
    double fep_score[GADEP_MAX_GROUPS], fep_score_sq[GADEP_MAX_GROUPS];
};

struct Params {
    const float4 *nodes;
    const float4 *tris;
    const float4 *planes;             // per mesh triangle: unit normal, offset
    const float4 *xs;                 // [n_mat][n_grid] (pe, compton, pair, 0), mm^-1
    const int4 *regions;              // (material slot or -1, active, group, parent)
    const InstDev *inst;
    const unsigned long long *inst_end;  // inclusive prefix sums of n_hist
    TallyDev *tally;
    uint32_t *spectra;
    unsigned long long *work;
    float *edep_trace;
    unsigned long long n_trace;
    unsigned long long total;
    int n_mat, n_grid, n_region, n_inst;
    float lnE_min, inv_dlnE;
    uint32_t key0, key1;
    float e_cut, fep_delta, e_max, bin_scale;
    int n_bins, step_cap, n_group, chunk;
    int n_stripes;                      // tally copies [n_stripes][n_inst], summed on the host
    float root_lo[3], root_hi[3];       // bounds of every triangle (padded)
    int root_all;                       // tree over every triangle
    int face_bins, n_keys;              // wavefront queue sort: direction cells, key count
    // charged particles (e_model 1): CSDA range of each staged material on e_n
    // log-spaced kinetic energies from e_T_min, mm at unit density
    const float *erange;                // [n_mat][e_n]
    int e_model, e_n;
    float e_T_min, e_lnT_min, e_inv_dlnT;
};

// Slab test of the ray (t >= 0) against an axis-aligned box.
__device__ __forceinline__ bool ray_hits_box(const float lo[3], const float hi[3], float ox, float oy, float oz,
                                             float dx, float dy, float dz)
{
    float t0 = 0.0f, t1 = INFINITY;
    const float o[3] = { ox, oy, oz }, d[3] = { dx, dy, dz };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float inv = 1.0f / (fabsf(d[k]) > 1e-30f ? d[k] : copysignf(1e-30f, d[k]));
        float a = (lo[k] - o[k]) * inv, b = (hi[k] - o[k]) * inv;
        t0 = fmaxf(t0, fminf(a, b));
        t1 = fminf(t1, fmaxf(a, b));
    }
    return t0 <= t1;
}

// Per-lane partial tallies of one instance, flushed on instance change and at exit.
template <bool GRAD>
struct Acc {
    int inst;
    uint32_t hist, fep, zero, over, err, seg, inter, errbits, culled;
    float dep, dep_all, esc;
    double score[GRAD ? 4 : 1], score2[GRAD ? 4 : 1];
    __device__ void reset(int i)
    {
        inst = i; hist = fep = zero = over = err = seg = inter = errbits = culled = 0u;
        dep = dep_all = esc = 0.0f;
#pragma unroll
        for (int g = 0; g < (GRAD ? 4 : 1); ++g) { score[g] = 0.0; score2[g] = 0.0; }
    }
    __device__ void flush_lane(TallyDev *T) const
    {
        if (inst < 0 || (hist == 0 && seg == 0 && inter == 0)) return;
        TallyDev &t = T[inst];
        atomicAdd(&t.n_hist, (unsigned long long)hist);
        if (fep) atomicAdd(&t.n_fep, (unsigned long long)fep);
        if (zero) atomicAdd(&t.n_zero, (unsigned long long)zero);
        if (over) atomicAdd(&t.n_over, (unsigned long long)over);
        if (err) { atomicAdd(&t.n_err, (unsigned long long)err); atomicOr(&t.err_bits, (unsigned long long)errbits); }
        atomicAdd(&t.n_segments, (unsigned long long)seg);
        atomicAdd(&t.n_interactions, (unsigned long long)inter);
        if (culled) atomicAdd(&t.n_culled, (unsigned long long)culled);
        atomicAdd(&t.sum_dep_active, (double)dep);
        atomicAdd(&t.sum_dep_all, (double)dep_all);
        atomicAdd(&t.sum_esc, (double)esc);
        if (GRAD) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                atomicAdd(&t.fep_score[g], score[g]);
                atomicAdd(&t.fep_score_sq[g], score2[g]);
            }
        }
    }
};

// Tally copy of this block: blocks spread their end-of-launch atomics over
// n_stripes copies so they do not all serialise on the same addresses.
__device__ __forceinline__ TallyDev *block_tally(const Params &P)
{
    return P.tally + (size_t)(blockIdx.x % (unsigned)P.n_stripes) * P.n_inst;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool GRAD>
__device__ void flush_warp(const Acc<GRAD> &a, TallyDev *T)
{
    int same = 0;
    __match_all_sync(0xffffffffu, a.inst, &same);
    if (!same || a.inst < 0) { a.flush_lane(T); return; }
    const int lane = threadIdx.x & 31;
    const uint32_t hist = __reduce_add_sync(0xffffffffu, a.hist);
    const uint32_t fep = __reduce_add_sync(0xffffffffu, a.fep);
    const uint32_t zero = __reduce_add_sync(0xffffffffu, a.zero);
    const uint32_t over = __reduce_add_sync(0xffffffffu, a.over);
    const uint32_t err = __reduce_add_sync(0xffffffffu, a.err);
    const uint32_t errbits = __reduce_or_sync(0xffffffffu, a.errbits);
    const uint32_t seg = __reduce_add_sync(0xffffffffu, a.seg);
    const uint32_t inter = __reduce_add_sync(0xffffffffu, a.inter);
    const uint32_t culled = __reduce_add_sync(0xffffffffu, a.culled);
    const double dep = warp_sum((double)a.dep), dep_all = warp_sum((double)a.dep_all),
                 esc = warp_sum((double)a.esc);
    double sc[4] = { 0, 0, 0, 0 }, sc2[4] = { 0, 0, 0, 0 };
    if (GRAD) {
#pragma unroll
        for (int g = 0; g < 4; ++g) { sc[g] = warp_sum(a.score[g]); sc2[g] = warp_sum(a.score2[g]); }
    }
    if (lane == 0 && (hist || seg || inter)) {
        TallyDev &t = T[a.inst];
        atomicAdd(&t.n_hist, (unsigned long long)hist);
        if (fep) atomicAdd(&t.n_fep, (unsigned long long)fep);
        if (zero) atomicAdd(&t.n_zero, (unsigned long long)zero);
        if (over) atomicAdd(&t.n_over, (unsigned long long)over);
        if (err) { atomicAdd(&t.n_err, (unsigned long long)err); atomicOr(&t.err_bits, (unsigned long long)errbits); }
        atomicAdd(&t.n_segments, (unsigned long long)seg);
        atomicAdd(&t.n_interactions, (unsigned long long)inter);
        if (culled) atomicAdd(&t.n_culled, (unsigned long long)culled);
        atomicAdd(&t.sum_dep_active, dep);
        atomicAdd(&t.sum_dep_all, dep_all);
        atomicAdd(&t.sum_esc, esc);
        if (GRAD) {
#pragma unroll
            for (int g = 0; g < 4; ++g) { atomicAdd(&t.fep_score[g], sc[g]); atomicAdd(&t.fep_score_sq[g], sc2[g]); }
        }
    }
}

__device__ __forceinline__ void rotate(float &dx, float &dy, float &dz, float c, float sphi, float cphi)
{
    const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    const float r = sqrtf(dx * dx + dy * dy);
    float nx, ny, nz;
    if (r < 1e-9f) {
        nx = s * cphi; ny = s * sphi; nz = dz > 0.0f ? c : -c;
    } else {
        const float ir = 1.0f / r;
        nx = dx * c + s * (dx * dz * cphi - dy * sphi) * ir;
        ny = dy * c + s * (dy * dz * cphi + dx * sphi) * ir;
        nz = dz * c - s * r * cphi;
    }
    const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
    dx = nx * inv; dy = ny * inv; dz = nz * inv;
}

__device__ __forceinline__ void iso_dir(Stream &rng, uint32_t k0, uint32_t k1, float &dx, float &dy, float &dz)
{
    const float c = 2.0f * rng.u01(k0, k1) - 1.0f;
    float sp, cp;
    sincospif(2.0f * rng.u01(k0, k1), &sp, &cp);
    const float s = sqrtf(fmaxf(0.0f, 1.0f - c * c));
    dx = s * cp; dy = s * sp; dz = c;
}

// Interpolated attenuation (pe, compton, pair) of a staged material at energy E.
__device__ __forceinline__ void mu_at(const float4 *tab, int n_grid, float lnE_min, float inv_dl,
                                      float E, float &pe, float &co, float &pa)
{
    const float g = (logf(E) - lnE_min) * inv_dl;
    int k = (int)floorf(g);
    k = min(max(k, 0), n_grid - 2);
    const float f = fminf(fmaxf(g - (float)k, 0.0f), 1.0f);
    const float4 a = tab[k], b = tab[k + 1];
    pe = fmaf(f, b.x - a.x, a.x);
    co = fmaf(f, b.y - a.y, a.y);
    pa = E > kTwoMeC2 ? fmaf(f, b.z - a.z, a.z) : 0.0f;
}

// CSDA range (mm, unit density) of staged material m at kinetic energy T >= e_T_min:
// linear in ln T between grid points (the last interval extended above the grid).
__device__ __forceinline__ float erange_at(const Params &P, int m, float T)
{
    const float *row = P.erange + (size_t)m * P.e_n;
    const float g = (logf(T) - P.e_lnT_min) * P.e_inv_dlnT;
    const int k = min(max((int)floorf(g), 0), P.e_n - 2);
    const float a = __ldg(row + k), b = __ldg(row + k + 1);
    return fmaf(g - (float)k, b - a, a);
}

// Kinetic energy whose range is `left` mm (the inverse of erange_at): bisection
// over the grid for the interval, then linear in ln T; below the first grid point
// the range is taken proportional to T.
__device__ __forceinline__ float e_energy_for_range(const Params &P, int m, float left)
{
    if (!(left > 0.0f)) return 0.0f;
    const float *row = P.erange + (size_t)m * P.e_n;
    const float r0 = __ldg(row);
    if (left <= r0) return P.e_T_min * (left / r0);
    int lo = 0, hi = P.e_n - 1;            // row[lo] < left; row[hi] >= left unless above the grid
    if (left >= __ldg(row + hi)) {
        lo = P.e_n - 2;
    } else {
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(row + mid) < left) lo = mid;
            else hi = mid;
        }
    }
    const float a = __ldg(row + lo), b = __ldg(row + lo + 1);
    return expf(P.e_lnT_min + ((float)lo + (left - a) / (b - a)) / P.e_inv_dlnT);
}

constexpr int kMaxTrackCrossings = 256;

// One line of `w` identical charged particles (kinetic energy T each) from p along
// unit u, born in `region` (the photon's): continuous slowing down straight ahead,
// region by region through the mesh.  In a region of material m and density
// scale s the particles reach R_m(T) / s; when the next boundary is nearer they
// cross it with the T' of range R_m(T) - s L and deposit T - T' in the region.
// Below e_T_min the rest is deposited where they are; vacuum takes nothing; what
// leaves the mesh escapes.  Active deposits go to edep, all to dep_all.
template <bool COUNT>
__device__ void e_track(const Params &P, const int4 *s_reg, const float *scale, float px, float py, float pz,
                        float ux, float uy, float uz, float T, float w, int region, float &edep, float &dep_all,
                        float &esc, uint32_t &herr, TravStats &ts)
{
    float t_cur = 0.0f;
    int last = -1;
    for (int k = 0; k <= kMaxTrackCrossings; ++k) {
        int4 R = s_reg[region];
        if (T < P.e_T_min) {
            dep_all += w * T;
            if (R.y & 1) edep += w * T;
            return;
        }
        const int group = (R.y >> 1) - 1;
        const float sc = group >= 0 ? scale[group] : 1.0f;
        const float rn = R.x >= 0 ? erange_at(P, R.x, T) : INFINITY;
        const float reach = rn / sc;
        float t_hit = INFINITY;
        bool entering = false;
        int hit = traverse<COUNT>(P.nodes, P.tris, P.planes, R.w, px, py, pz, ux, uy, uz, t_cur, last, t_hit,
                                  entering, herr, ts, t_cur + reach);
        if (herr & ERR_STACK) return;
        if (hit < 0 && reach < INFINITY) {         // stops in this region
            dep_all += w * T;
            if (R.y & 1) edep += w * T;
            return;
        }
        if (hit < 0 && region != 0) {
            // vacuum inside a solid with no surface ahead: the start sits a rounding
            // error past a boundary; relocate by the nearest surface of the mesh
            hit = traverse<COUNT>(P.nodes, P.tris, P.planes, P.root_all, px, py, pz, ux, uy, uz, t_cur, last,
                                  t_hit, entering, herr, ts);
            if (herr & ERR_STACK) return;
        }
        if (hit < 0) {                             // leaves the mesh
            esc += w * T;
            return;
        }
        float T2 = T;
        if (R.x >= 0) T2 = fminf(T, e_energy_for_range(P, R.x, rn - (t_hit - t_cur) * sc));
        dep_all += w * (T - T2);
        if (R.y & 1) edep += w * (T - T2);
        T = T2;
        t_cur = t_hit;
        last = __float_as_int(__ldg(&P.tris[3 * hit + 1].w));
        const int treg = __float_as_int(__ldg(&P.tris[3 * hit].w));
        region = entering ? treg : s_reg[treg].z;
    }
    herr |= ERR_STEPCAP;
}

}  // namespace dev

// Kernel launches of a plan, counted per kind, and optionally timed with CUDA
// events recorded on the launching stream around every launch.
enum KernelKind { KK_MEGA = 0, KK_SPAWN, KK_TRACE, KK_PHYSICS, KK_GEN, KK_CTRL, KK_INIT, KK_SORT, KK_ETRACK, KK_N };
struct KernelTimer {
    bool timing = false;
    unsigned long long launches[KK_N] = {};
    double ms[KK_N] = {};
    struct Pair { int kind; cudaEvent_t a, b; };
    std::vector<Pair> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open = nullptr;
    cudaEvent_t take()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return e;
    }
    void before(cudaStream_t s)
    {
        if (!timing) return;
        open = take();
        if (open && cudaEventRecord(open, s) != cudaSuccess) { cudaGetLastError(); pool.push_back(open); open = nullptr; }
    }
    void after(int kind, cudaStream_t s)
    {
        ++launches[kind];
        if (!timing || !open) return;
        cudaEvent_t b = take();
        if (b && cudaEventRecord(b, s) == cudaSuccess) pending.push_back(Pair{ kind, open, b });
        else { cudaGetLastError(); pool.push_back(open); if (b) pool.push_back(b); }
        open = nullptr;
    }
    // Wait for the recorded launches and add their durations.
    cudaError_t resolve()
    {
        cudaError_t err = cudaSuccess;
        for (const Pair &p : pending) {
            float t = 0.0f;
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
            if (e == cudaSuccess) ms[p.kind] += t;
            else if (err == cudaSuccess) err = e;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        return err;
    }
    void reset()
    {
        for (int k = 0; k < KK_N; ++k) { launches[k] = 0; ms[k] = 0.0; }
    }
    void release()
    {
        resolve();
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

// Wavefront form of the transport (wavefront.cu): photon slots in device memory,
// spawn / sort / trace / physics / gen / ctrl kernels per iteration.
struct WavefrontBuffers;
constexpr int kWavefrontMaxInstances = 1024;   // block tallies live in shared memory
gadep_status wavefront_create(int device, int slots, bool grad, WavefrontBuffers **out);
void wavefront_destroy(WavefrontBuffers *w);
// slots: photon slots the run keeps in flight (at most the buffers' capacity; 0 =
// the capacity).
gadep_status wavefront_run(WavefrontBuffers *w, const dev::Params &P, bool grad, bool count,
                           unsigned long long *counters, KernelTimer *timer, cudaStream_t s, int slots);
int wavefront_trace_grid(const WavefrontBuffers *w);
gadep_status wavefront_check(WavefrontBuffers *w, cudaStream_t s);
gadep_status wavefront_queue_log(WavefrontBuffers *w, uint32_t *out, int max, int *n, cudaStream_t s);
// Whether the wavefront records can address the mesh (region and triangle ids
// share one 32-bit word).
bool wavefront_supports(int n_region, long long n_mesh_tri);

}  // namespace gadep
