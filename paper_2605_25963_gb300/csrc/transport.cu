// transport.cu -- GPU photon transport through the detector mesh (paper Sec. 2.4).
//
// One persistent "megakernel" runs whole histories.  Every warp takes histories
// from a device work counter in chunks (the work queue of a batched run is the
// flattened history range of all instances, so one launch serves any number of
// instances with uneven history counts); a lane whose history ends takes the
// next one at once, so lanes stay busy while long histories continue.
//
// Per history (paper's Gadep step, photon part):
//   birth        source position and isotropic direction (Philox stream of the
//                history), birth region precomputed on the host by the parity rule;
//   flight       partial cross-section free flight (Sec. 2.4.1): one number of
//                mean free paths lambda = -ln u per flight, consumed segment by
//                segment (lambda -= mu * length); the segment ends at the nearest
//                triangle (BVH query, Sec. 2.4.3) or at the interaction point;
//   crossing     region update by the nesting tree: entering solid s -> s,
//                leaving s -> parent(s) (equal to the parity rule of Sec. 2.4.2 for
//                nested closed solids; the tree itself is built with that rule);
//   interaction  process by partial attenuation coefficients: photoabsorption,
//                Compton (Kahn's rejection sampler), pair production (two 511 keV
//                photons back to back, the second one tracked afterwards);
//                charged secondaries deposit their energy locally;
//   tally        energy deposited in active solids per history -> pulse-height
//                spectrum (warp-aggregated atomics), full-energy-peak count,
//                FP64 sums; with GRAD, density-perturbation scores
//                score_p = n_coll,p / s_p - sum_p mu_unit * length per history.
// Cross-section tables (float4 per grid point) are read through L1 from global
// memory; the region table is staged in shared memory per block.  Arithmetic is
// FP32; counts are integers; sums of scores are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "device_common.cuh"
#include "gadep_internal.h"
#include "transport_common.cuh"

namespace gadep {

gadep_status build_bvh_host(const detmesh_mesh *m, const gadep_bvh_opts &o, gadep_bvh *out);

namespace dev {
// EM: charged-particle tracks (e_model 1), a separate instantiation so that the
// photon-only kernels keep their registers.
template <bool GRAD, bool COUNT, bool EM>
// 4 blocks of 256 threads per SM (64 registers): measured faster than 2 or 3
// blocks despite the register spills, as the traversal is latency bound.
__global__ void __launch_bounds__(256, 4) transport_kernel(const Params P, unsigned long long *counters)
{
    // Shared memory holds the region table and the instance prefix sums.  The
    // attenuation tables stay in global memory and are read through L1: staging a
    // copy per block (16 KB per material) took L1 capacity away from the BVH
    // nodes and measured 16 % slower.
    extern __shared__ float4 smem[];
    int4 *s_reg = reinterpret_cast<int4 *>(smem);
    unsigned long long *s_end = reinterpret_cast<unsigned long long *>(s_reg + P.n_region);
    for (int i = threadIdx.x; i < P.n_region; i += blockDim.x) s_reg[i] = P.regions[i];
    for (int i = threadIdx.x; i < P.n_inst; i += blockDim.x) s_end[i] = P.inst_end[i];
    __syncthreads();

    const uint32_t FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t k0 = P.key0, k1 = P.key1;

    unsigned long long pool_next = 0, pool_end = 0;
    bool exhausted = false;
    bool busy = false;
    int inst = 0;
    unsigned long long g_hist = 0;
    Stream rng;
    float ox = 0, oy = 0, oz = 0, dx = 0, dy = 0, dz = 1, E = 0, E0 = 0, lam = 0, t_cur = 0;
    int region = 0, last_tri = -1, steps = 0;
    bool has_sec = false;
    float sox = 0, soy = 0, soz = 0, sdx = 0, sdy = 0, sdz = 0;
    int sreg = 0;
    float edep = 0, dep_all = 0, esc = 0;
    uint32_t herr = 0;
    float score[GRAD ? 4 : 1];
#pragma unroll
    for (int g = 0; g < (GRAD ? 4 : 1); ++g) score[g] = 0.0f;
    Acc<GRAD> acc;
    acc.reset(-1);
    TravStats ts{};

    while (true) {
        // ---------------- refill idle lanes from the work counter ----------------
        uint32_t need = __ballot_sync(FULL, !busy);
        while (need && !exhausted) {
            if (pool_next == pool_end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(P.work, (unsigned long long)P.chunk);
                base = __shfl_sync(FULL, base, 0);
                if (base >= P.total) { exhausted = true; break; }
                pool_next = base;
                pool_end = min(base + (unsigned long long)P.chunk, P.total);
            }
            const uint32_t avail = (uint32_t)(pool_end - pool_next);
            const uint32_t take = min((uint32_t)__popc(need), avail);
            const uint32_t rank = __popc(need & lt_mask);
            if (!busy && rank < take) {
                g_hist = pool_next + rank;
                while (g_hist >= s_end[inst]) ++inst;
                if (acc.inst != inst) { acc.flush_lane(block_tally(P)); acc.reset(inst); }
                const InstDev &I = P.inst[inst];
                const unsigned long long local = g_hist - (inst ? s_end[inst - 1] : 0ull);
                rng.init(I.hist_offset + local, I.inst_id);
                ox = I.px; oy = I.py; oz = I.pz;
                if (I.src_kind == GADEP_SRC_DISK) {
                    const float r = I.radius * sqrtf(rng.u01(k0, k1));
                    float sp, cp;
                    sincospif(2.0f * rng.u01(k0, k1), &sp, &cp);
                    ox = fmaf(r, cp, ox); oy = fmaf(r, sp, oy);
                } else if (I.src_kind == GADEP_SRC_PRISM) {
                    const int N = I.n_sides;
                    int kk = (int)((float)N * rng.u01(k0, k1));
                    kk = min(kk, N - 1);
                    const float s1 = sqrtf(rng.u01(k0, k1)), u3 = rng.u01(k0, k1);
                    float sa, ca, sb, cb;
                    sincospif(2.0f * (float)kk / (float)N, &sa, &ca);
                    sincospif(2.0f * (float)((kk + 1) % N) / (float)N, &sb, &cb);
                    const float wa = s1 * (1.0f - u3), wb = s1 * u3;
                    ox += I.radius * (wa * ca + wb * cb);
                    oy += I.radius * (wa * sa + wb * sb);
                    oz = fmaf(I.height, rng.u01(k0, k1), oz);
                }
                if (I.src_kind == GADEP_SRC_PENCIL) { dx = I.dx; dy = I.dy; dz = I.dz; }
                else iso_dir(rng, k0, k1, dx, dy, dz);
                E = E0 = I.E0;
                region = I.birth_region;
                t_cur = 0.0f; last_tri = -1; steps = 0;
                has_sec = false;
                edep = dep_all = esc = 0.0f;
                herr = 0u;
#pragma unroll
                for (int g = 0; g < (GRAD ? 4 : 1); ++g) score[g] = 0.0f;
                if (region == 0 && !ray_hits_box(P.root_lo, P.root_hi, ox, oy, oz, dx, dy, dz)) {
                    // Born in the world and aimed away from every solid: the one
                    // segment of this history escapes with nothing deposited.  It
                    // ends here so the lane can take the next history at once.
                    acc.hist++; acc.zero++; acc.seg++; acc.culled++;
                    acc.esc += E0;
                    if (g_hist < P.n_trace) P.edep_trace[g_hist] = 0.0f;
                } else {
                    lam = -logf(rng.u01(k0, k1));
                    busy = true;
                }
            }
            pool_next += take;
            need = __ballot_sync(FULL, !busy);
        }
        if (__ballot_sync(FULL, busy) == 0) break;

        // ---------------- one segment of the current photon ----------------
        bool finished = false;
        if (busy) {
            if (++steps > P.step_cap) {
                herr |= ERR_STEPCAP;
                finished = true;
            } else {
                float t_hit = INFINITY;
                bool entering = false;
                // region record: material slot, active | (group + 1) << 1, parent, tree root
                int4 R = s_reg[region];
                int hit = traverse<COUNT>(P.nodes, P.tris, P.planes, R.w, ox, oy, oz, dx, dy, dz, t_cur, last_tri,
                                          t_hit, entering, herr, ts);
                if (hit < 0 && region != 0 && !(herr & ERR_STACK)) {
                    // Inside a solid every ray meets that solid's boundary, so the
                    // photon actually sits a rounding error past it (an interaction
                    // point computed in FP32 right at a surface).  Relocate by the
                    // nearest surface of the whole mesh and the nesting-tree rule;
                    // with no surface ahead it is outside every solid.
                    hit = traverse<COUNT>(P.nodes, P.tris, P.planes, P.root_all, ox, oy, oz, dx, dy, dz, t_cur, last_tri,
                                          t_hit, entering, herr, ts);
                    if (COUNT) ts.relocated++;
                    if (hit < 0) {
                        region = 0;
                        R = s_reg[0];       // the segment runs in the world
                    }
                }
                const int group = (R.y >> 1) - 1;
                float pe = 0.0f, co = 0.0f, pa = 0.0f;
                if (R.x >= 0) mu_at(P.xs + (size_t)R.x * P.n_grid, P.n_grid, P.lnE_min, P.inv_dlnE, E, pe, co, pa);
                const float mu_unit = pe + co + pa;
                const float sc = group >= 0 ? P.inst[inst].scale[group] : 1.0f;
                const float mu = mu_unit * sc;
                const float d_int = mu > 0.0f ? lam / mu : INFINITY;
                acc.seg++;
                if (herr & ERR_STACK) {
                    finished = true;
                } else if (d_int < t_hit - t_cur) {
                    // ---- interaction ----
                    acc.inter++;
                    if (GRAD && group >= 0 && group < 4) score[group] += 1.0f / sc - mu_unit * d_int;
                    const float tt = t_cur + d_int;
                    const float px = fmaf(tt, dx, ox), py = fmaf(tt, dy, oy), pz = fmaf(tt, dz, oz);
                    const float u = rng.u01(k0, k1) * mu_unit;
                    float dep = 0.0f;
                    bool alive = true;
                    // charged particles of e_model 1: kinetic energy, direction, count
                    float eT = 0.0f, eux = dx, euy = dy, euz = dz, ew = 1.0f;
                    if (u < pe) {
                        if (EM) eT = E;
                        else dep = E;
                        E = 0.0f; alive = false;
                    } else if (u < pe + co || pa == 0.0f) {
                        const float k = E * (1.0f / kMeC2);
                        const float a2k = 1.0f + 2.0f * k;
                        const float br = a2k / (9.0f + 2.0f * k);
                        float x = 1.0f;
                        bool ok = false;
                        for (int trial = 0; trial < 1000; ++trial) {
                            const float r1 = rng.u01(k0, k1), r2 = rng.u01(k0, k1), r3 = rng.u01(k0, k1);
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
                            alive = false;
                        } else {
                            const float c = 1.0f - (x - 1.0f) / k;
                            float sp, cp;
                            sincospif(2.0f * rng.u01(k0, k1), &sp, &cp);
                            const float Ep = E / x;
                            rotate(dx, dy, dz, c, sp, cp);
                            if (EM) {
                                eT = E - Ep;
                                const float qx = E * eux - Ep * dx, qy = E * euy - Ep * dy, qz = E * euz - Ep * dz;
                                const float ql = sqrtf(qx * qx + qy * qy + qz * qz);
                                if (ql > 0.0f) { eux = qx / ql; euy = qy / ql; euz = qz / ql; }
                            } else {
                                dep = E - Ep;
                            }
                            E = Ep;
                            if (E < P.e_cut) { dep += E; E = 0.0f; alive = false; }
                        }
                    } else {
                        if (EM) { eT = 0.5f * (E - kTwoMeC2); ew = 2.0f; }
                        else dep = E - kTwoMeC2;
                        float nx, ny, nz;
                        iso_dir(rng, k0, k1, nx, ny, nz);
                        E = kMeC2;
                        dx = nx; dy = ny; dz = nz;
                        has_sec = true;
                        sox = px; soy = py; soz = pz;
                        sdx = -nx; sdy = -ny; sdz = -nz;
                        sreg = region;
                    }
                    if (R.y & 1) edep += dep;
                    dep_all += dep;
                    if (eT > 0.0f && !herr)
                        e_track<COUNT>(P, s_reg, P.inst[inst].scale, px, py, pz, eux, euy, euz, eT, ew, region, edep,
                                       dep_all, esc, herr, ts);
                    if (herr) {
                        finished = true;
                    } else if (alive) {
                        ox = px; oy = py; oz = pz;
                        t_cur = 0.0f; last_tri = -1;
                        lam = -logf(rng.u01(k0, k1));
                    } else if (has_sec) {
                        has_sec = false;
                        ox = sox; oy = soy; oz = soz; dx = sdx; dy = sdy; dz = sdz;
                        E = kMeC2; region = sreg;
                        t_cur = 0.0f; last_tri = -1;
                        lam = -logf(rng.u01(k0, k1));
                    } else {
                        finished = true;
                    }
                } else if (hit < 0) {
                    // leaves the mesh
                    if (region != 0) herr |= ERR_LOST;
                    esc += E;
                    E = 0.0f;
                    if (!herr && has_sec) {
                        has_sec = false;
                        ox = sox; oy = soy; oz = soz; dx = sdx; dy = sdy; dz = sdz;
                        E = kMeC2; region = sreg;
                        t_cur = 0.0f; last_tri = -1;
                        lam = -logf(rng.u01(k0, k1));
                    } else {
                        finished = true;
                    }
                } else {
                    // ---- boundary crossing ----
                    const float len = t_hit - t_cur;
                    lam -= mu * len;
                    if (GRAD && group >= 0 && group < 4) score[group] -= mu_unit * len;
                    t_cur = t_hit;
                    last_tri = __float_as_int(__ldg(&P.tris[3 * hit + 1].w));   // mesh triangle id
                    const int treg = __float_as_int(__ldg(&P.tris[3 * hit].w));
                    region = entering ? treg : s_reg[treg].z;
                }
            }
            if (!finished && !(isfinite(dx) && isfinite(E) && isfinite(lam))) {
                herr |= ERR_NONFINITE;
                finished = true;
            }
        }

        // ---------------- tally of finished histories (warp-converged) ----------------
        const bool binned = finished && herr == 0u && edep > 0.0f && edep < P.e_max;
        int bin = 0;
        if (binned) bin = min((int)(edep * P.bin_scale), P.n_bins - 1);
        const uint32_t key = binned ? (uint32_t)(inst * P.n_bins + bin) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(FULL, key);
        if (binned && lane == __ffs(peers) - 1)
            atomicAdd(&P.spectra[(size_t)inst * P.n_bins + bin], (uint32_t)__popc(peers));
        if (finished) {
            acc.hist++;
            if (herr) {
                acc.err++;
                acc.errbits |= herr;
            } else {
                const bool fep = (E0 - edep) <= P.fep_delta;
                if (fep) {
                    acc.fep++;
                    if (GRAD) {
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const double s = (double)score[g];
                            acc.score[g] += s;
                            acc.score2[g] += s * s;
                        }
                    }
                }
                if (edep == 0.0f) acc.zero++;
                else if (edep >= P.e_max) acc.over++;
                acc.dep += edep; acc.dep_all += dep_all; acc.esc += esc;
            }
            if (g_hist < P.n_trace) P.edep_trace[g_hist] = herr ? -1.0f : edep;
            busy = false;
        }
    }
    flush_warp<GRAD>(acc, block_tally(P));
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)ts.nodes);
        atomicAdd(&counters[1], (unsigned long long)ts.tris);
        atomicAdd(&counters[3], (unsigned long long)ts.boxes);
        if (ts.relocated) atomicAdd(&counters[2], (unsigned long long)ts.relocated);
    }
}

// One query per thread.  region[i] (0 = world, s + 1 = solid s) selects that
// region's tree; without regions, or for an out-of-range id, the tree over every
// triangle is used.
__global__ void nearest_hit_kernel(const float4 *nodes, const float4 *tris, const float4 *planes,
                                   const int32_t *region_roots,
                                   int32_t n_region, int32_t root_all, const int32_t *regions,
                                   const float *rays, long long n, float *t_out, int32_t *tri_out,
                                   int32_t *ent_out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *r = rays + 8 * i;
    const int ex = __float_as_int(r[7]);
    int root = root_all;
    if (regions) {
        const int g = regions[i];
        if (g >= 0 && g < n_region) root = region_roots[g];
    }
    float t = INFINITY;
    bool ent = false;
    uint32_t err = 0;
    TravStats st{};
    const int hit = traverse<false>(nodes, tris, planes, root, r[0], r[1], r[2], r[4], r[5], r[6], r[3], ex, t, ent,
                                    err, st);
    t_out[i] = hit >= 0 ? t : INFINITY;
    tri_out[i] = hit >= 0 ? __float_as_int(__ldg(&tris[3 * hit + 1].w)) : -1;
    ent_out[i] = hit >= 0 ? (ent ? 1 : 0) : (err ? -2 : -1);
}

// FP32 FMA throughput: 8 independent chains per thread, kFmaIters rounds.
constexpr int kFmaIters = 4096;
__global__ void __launch_bounds__(256) fma_peak_kernel(float b, float c, float *out)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

// L2 read bandwidth: `rounds` grid-stride passes of 16-byte loads over n float4.
__global__ void __launch_bounds__(256) l2_read_kernel(const float4 *__restrict__ buf, size_t n, int rounds,
                                                      float *out)
{
    float s = 0.0f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < rounds; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const float4 v = __ldcg(buf + i);
            s += v.x + v.y + v.z + v.w;
        }
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void philox_words_kernel(unsigned long long seed, unsigned long long hid, uint32_t inst,
                                    int n_words, uint32_t *out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * b >= n_words) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)hid, (uint32_t)(hid >> 32), inst),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t v[4] = { w.x, w.y, w.z, w.w };
    for (int k = 0; k < 4 && 4 * b + k < n_words; ++k) out[4 * b + k] = v[k];
}

}  // namespace dev

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

gadep_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(GADEP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <class T>
gadep_status dalloc(T **p, size_t n, const char *what)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? GADEP_E_NOMEM : GADEP_E_CUDA, "%s: cudaMalloc: %s",
                    what, cudaGetErrorString(e));
    }
    return GADEP_OK;
}

int is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return 0; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

gadep_status upload_bvh(gadep_bvh *b)
{
    DeviceGuard g(b->device);
    if (!g.ok) return fail(GADEP_E_CUDA, "gadep_bvh_build: cannot select device %d", b->device);
    gadep_status st;
    if ((st = dalloc((float **)&b->d_nodes, b->nodes.size(), "bvh nodes")) != GADEP_OK) return st;
    if ((st = dalloc((float **)&b->d_tris, b->tris.size(), "bvh triangles")) != GADEP_OK) return st;
    if ((st = dalloc((float **)&b->d_planes, b->planes.size(), "bvh planes")) != GADEP_OK) return st;
    const size_t nr = b->regions.size() / 4;
    std::vector<int32_t> roots(nr);
    for (size_t r = 0; r < nr; ++r) roots[r] = b->regions[4 * r + 3];
    if ((st = dalloc((int32_t **)&b->d_regions, nr, "bvh region roots")) != GADEP_OK) return st;
    cudaError_t e;
    if ((e = cudaMemcpy(b->d_nodes, b->nodes.data(), b->nodes.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_tris, b->tris.data(), b->tris.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_planes, b->planes.data(), b->planes.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_regions, roots.data(), nr * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "gadep_bvh_build: upload");
    return GADEP_OK;
}

void free_bvh_device(gadep_bvh *b)
{
    if (!b->d_nodes && !b->d_tris && !b->d_regions && !b->d_planes) return;
    DeviceGuard g(b->device);
    wavefront_destroy(b->wf_cache);
    b->wf_cache = nullptr;
    cudaFree(b->plan_scratch);
    b->plan_scratch = nullptr;
    b->plan_scratch_bytes = 0;
    cudaFree(b->d_nodes);
    cudaFree(b->d_tris);
    cudaFree(b->d_regions);
    cudaFree(b->d_planes);
    b->d_nodes = b->d_tris = b->d_regions = b->d_planes = nullptr;
}

}  // namespace gadep

using gadep::DeviceGuard;
using gadep::is_device_ptr;

struct gadep_plan {
    const gadep_bvh *bvh = nullptr;
    int device = 0;
    int n_inst = 0;
    bool grad = false;
    gadep_opts opts{};
    int n_bins = 0;
    std::vector<gadep::dev::InstDev> inst;
    std::vector<unsigned long long> inst_end;
    void *scratch = nullptr;                 // one device block holding the buffers below
    bool scratch_cached = false;             // scratch borrowed from the BVH (with wf)
    float4 *d_xs = nullptr;
    float *d_erange = nullptr;
    int4 *d_regions = nullptr;
    gadep::dev::InstDev *d_inst = nullptr;
    unsigned long long *d_end = nullptr;
    gadep::dev::TallyDev *d_tally = nullptr;
    uint32_t *d_spectra = nullptr;
    unsigned long long *d_work = nullptr;
    unsigned long long *d_counters = nullptr;
    gadep::dev::Params P{};
    int grid = 0, block = 256, smem = 0;
    int n_stripes = 1;                        // tally copies per instance
    bool count = false;
    uint32_t *last_spectra = nullptr;
    gadep::WavefrontBuffers *wf = nullptr;   // set when the plan runs the wavefront form
    bool wf_cached = false;                  // wf borrowed from the BVH's cache
    int wf_slots = 0;                        // photon slots the plan keeps in flight
    gadep::KernelTimer timer;                // launch counts and optional event timing
};

namespace {

using gadep::fail;

gadep_status check_opts(const gadep_opts *o)
{
    if (!o) return fail(GADEP_E_INVAL, "NULL opts");
    if (!(o->e_cut_keV >= 0.0f) || !(o->fep_delta_keV >= 0.0f) || !(o->e_max_keV > 0.0f) ||
        o->n_bins < 1 || o->n_bins > (1 << 20) || o->step_cap < 1 || o->n_group < 0 ||
        o->n_group > 4 || o->block < 0 || o->block > 256 || (o->block % 32) != 0 || o->chunk < 0 ||
        o->blocks_per_sm < 0 || o->blocks_per_sm > 32 || o->e_model < 0 || o->e_model > 1)
        return fail(GADEP_E_INVAL, "bad gadep_opts (n_bins in [1, 2^20], step_cap >= 1, n_group <= 4, "
                                   "block a multiple of 32 <= 256, e_model 0 or 1)");
    for (int g = 0; g < GADEP_MAX_GROUPS; ++g)
        if (!(o->group_scale[g] >= 0.0f) || !std::isfinite(o->group_scale[g]))
            return fail(GADEP_E_INVAL, "bad group scale");
    return GADEP_OK;
}

template <bool GRAD, bool COUNT, bool EM>
void *kernel_ptr() { return (void *)gadep::dev::transport_kernel<GRAD, COUNT, EM>; }

void *pick_kernel(bool grad, bool count, bool em)
{
    if (grad) return count ? kernel_ptr<true, true, false>() : kernel_ptr<true, false, false>();
    if (em) return count ? kernel_ptr<false, true, true>() : kernel_ptr<false, false, true>();
    return count ? kernel_ptr<false, true, false>() : kernel_ptr<false, false, false>();
}

}  // namespace

extern "C" void gadep_opts_default(gadep_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->seed = 1;
    o->history_offset = 0;
    o->e_cut_keV = 10.0f;
    o->fep_delta_keV = 0.01f;
    o->e_max_keV = 3000.0f;
    o->n_bins = 4096;
    o->step_cap = 10000;
    o->variant = GADEP_VARIANT_AUTO;
    o->block = 0;
    o->chunk = 0;
    o->blocks_per_sm = 0;
    o->n_group = 0;
    for (int g = 0; g < GADEP_MAX_GROUPS; ++g) o->group_scale[g] = 1.0f;
}

extern "C" gadep_status gadep_bvh_build(const detmesh_mesh *m, int32_t device, gadep_bvh **out)
{
    return gadep_bvh_build_opts(m, nullptr, device, out);
}

extern "C" gadep_status gadep_bvh_build_opts(const detmesh_mesh *m, const gadep_bvh_opts *opts, int32_t device,
                                             gadep_bvh **out)
{
    gadep::clear_error();
    if (!m || !out) return fail(GADEP_E_INVAL, "gadep_bvh_build: NULL argument");
    gadep_bvh_opts o;
    gadep_bvh_opts_default(&o);
    if (opts) o = *opts;
    *out = nullptr;
    if (device != -1) {
        int n_dev = 0;
        if (cudaGetDeviceCount(&n_dev) != cudaSuccess) { cudaGetLastError(); n_dev = 0; }
        if (device < 0 || device >= n_dev) return fail(GADEP_E_INVAL, "gadep_bvh_build: no CUDA device %d", device);
    }
    gadep_bvh *b = new (std::nothrow) gadep_bvh();
    if (!b) return fail(GADEP_E_NOMEM, "gadep_bvh_build: out of host memory");
    b->device = device;
    gadep_status st = gadep::build_bvh_host(m, o, b);
    if (st == GADEP_OK && device >= 0) st = gadep::upload_bvh(b);
    if (st != GADEP_OK) { gadep::free_bvh_device(b); delete b; return st; }
    *out = b;
    return GADEP_OK;
}

extern "C" void gadep_bvh_destroy(gadep_bvh *b)
{
    if (!b) return;
    gadep::free_bvh_device(b);
    delete b;
}

extern "C" gadep_status gadep_nearest_hit(const gadep_bvh *b, const float *rays, const int32_t *regions, int64_t n,
                                          float *t_out, int32_t *tri_out, int32_t *entering_out, void *stream)
{
    gadep::clear_error();
    if (!b || n < 0 || (n > 0 && (!rays || !t_out || !tri_out || !entering_out)))
        return fail(GADEP_E_INVAL, "gadep_nearest_hit: bad arguments");
    if (b->device < 0 || !b->d_nodes) return fail(GADEP_E_INVAL, "gadep_nearest_hit: the BVH has no device copy");
    if (n == 0) return GADEP_OK;
    if (!is_device_ptr(rays) || !is_device_ptr(t_out) || !is_device_ptr(tri_out) || !is_device_ptr(entering_out) ||
        (regions && !is_device_ptr(regions)))
        return fail(GADEP_E_INVAL, "gadep_nearest_hit: rays, regions and outputs must be device memory");
    DeviceGuard g(b->device);
    const int threads = 128;
    const long long blocks = (n + threads - 1) / threads;
    gadep::dev::nearest_hit_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        (const float4 *)b->d_nodes, (const float4 *)b->d_tris, (const float4 *)b->d_planes,
        (const int32_t *)b->d_regions,
        (int32_t)(b->regions.size() / 4), b->root_all, regions, rays, n, t_out, tri_out, entering_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GADEP_OK : gadep::cuda_fail(e, "gadep_nearest_hit");
}

extern "C" gadep_status gadep_philox_words(uint64_t seed, uint64_t hid, uint32_t instance, int32_t n_words,
                                           uint32_t *out, void *stream)
{
    gadep::clear_error();
    if (n_words < 0 || (n_words > 0 && !out)) return fail(GADEP_E_INVAL, "gadep_philox_words: bad arguments");
    if (n_words == 0) return GADEP_OK;
    if (!is_device_ptr(out)) return fail(GADEP_E_INVAL, "gadep_philox_words: out must be device memory");
    const int blocks4 = (n_words + 3) / 4;
    gadep::dev::philox_words_kernel<<<(blocks4 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(seed, hid, instance,
                                                                                          n_words, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GADEP_OK : gadep::cuda_fail(e, "gadep_philox_words");
}

extern "C" void gadep_plan_destroy(gadep_plan *p)
{
    if (!p) return;
    {
        DeviceGuard g(p->device);
        if (!p->scratch_cached) cudaFree(p->scratch);
        p->timer.release();
        if (p->wf_cached) {
            gadep_bvh *bm = const_cast<gadep_bvh *>(p->bvh);
            std::lock_guard<std::mutex> lock(bm->wf_mutex);
            bm->wf_cache_busy = false;
        } else {
            gadep::wavefront_destroy(p->wf);
        }
    }
    delete p;
}

namespace gadep {

// Bounds of every solid seen from the world: the union of the world tree's root
// child boxes (lo > hi when the world tree is empty).
void scene_box(const gadep_bvh *b, float lo[3], float hi[3])
{
    for (int k = 0; k < 3; ++k) { lo[k] = 0.0f; hi[k] = -1.0f; }
    if (b->regions[3] < 0) return;
    WideNode wn;
    decode_node(b->nodes.data() + (size_t)b->regions[3] * kNodeFloats, wn);
    double dlo[3] = { INFINITY, INFINITY, INFINITY }, dhi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int c = 0; c < wn.n; ++c) {
        for (int k = 0; k < 3; ++k) {
            dlo[k] = std::min(dlo[k], wn.lo[c][k]);
            dhi[k] = std::max(dhi[k], wn.hi[c][k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        lo[k] = (float)dlo[k];
        if ((double)lo[k] > dlo[k]) lo[k] = std::nextafter(lo[k], -INFINITY);
        hi[k] = (float)dhi[k];
        if ((double)hi[k] < dhi[k]) hi[k] = std::nextafter(hi[k], INFINITY);
    }
}

// Fraction of an instance's histories whose first ray reaches the scene box
// (the rest end at birth): 1 for sources inside a solid; otherwise estimated
// with 4096 directions on a Fibonacci spiral from the source point (a disk
// source adds 16 points on its area).  Only the choice of transport form and
// the number of photon slots depend on it.
double hit_fraction(const dev::InstDev &d, const float lo[3], const float hi[3])
{
    if (d.birth_region != 0) return 1.0;
    if (!(lo[0] <= hi[0])) return 0.0;
    auto hits = [&](const double o[3], const double dir[3]) {
        double t0 = 0.0, t1 = INFINITY;
        for (int k = 0; k < 3; ++k) {
            if (dir[k] == 0.0) {
                if (o[k] < lo[k] || o[k] > hi[k]) return false;
                continue;
            }
            double a = (lo[k] - o[k]) / dir[k], c = (hi[k] - o[k]) / dir[k];
            if (a > c) std::swap(a, c);
            t0 = std::max(t0, a);
            t1 = std::min(t1, c);
        }
        return t0 <= t1;
    };
    if (d.src_kind == GADEP_SRC_PENCIL) {
        const double o[3] = { d.px, d.py, d.pz }, dir[3] = { d.dx, d.dy, d.dz };
        return hits(o, dir) ? 1.0 : 0.0;
    }
    const int n_dir = 4096, n_pos = d.src_kind == GADEP_SRC_DISK ? 16 : 1;
    const double golden = 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
    long hit = 0;
    for (int q = 0; q < n_pos; ++q) {
        double o[3] = { d.px, d.py, d.pz };
        if (n_pos > 1) {
            const double r = d.radius * std::sqrt((q + 0.5) / n_pos), a = golden * q;
            o[0] += r * std::cos(a);
            o[1] += r * std::sin(a);
        }
        for (int i = 0; i < n_dir; ++i) {
            const double z = 1.0 - (2.0 * i + 1.0) / n_dir, rr = std::sqrt(std::max(0.0, 1.0 - z * z));
            const double dir[3] = { rr * std::cos(golden * i), rr * std::sin(golden * i), z };
            hit += hits(o, dir);
        }
    }
    return (double)hit / ((double)n_dir * n_pos);
}

gadep_status plan_create(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                         const gadep_instance *inst, const gadep_opts *opts, bool grad, bool count,
                         gadep_plan **out)
{
    if (!out) return fail(GADEP_E_INVAL, "plan: NULL out");
    *out = nullptr;
    if (!b || !mat || !inst || n_inst < 1 || n_inst > 4096) return fail(GADEP_E_INVAL, "plan: bad arguments (1 <= n_inst <= 4096)");
    if (b->device < 0 || !b->d_nodes) return fail(GADEP_E_INVAL, "plan: the BVH was built without a device copy");
    gadep_status st = check_opts(opts);
    if (st != GADEP_OK) return st;
    if (!mat->mu || mat->n_mat < 1 || mat->n_mat > 1024 || mat->n_grid < 2 || mat->n_grid > 65536 ||
        !(mat->E_min > 0.0) || !(mat->E_max > mat->E_min))
        return fail(GADEP_E_INVAL, "plan: bad gadep_materials");
    const bool electrons = opts->e_model == 1;
    if (electrons && grad) return fail(GADEP_E_INVAL, "plan: e_model 1 is not available with gradients");
    if (electrons && (!mat->e_range || mat->e_n < 2 || mat->e_n > 65536 || !(mat->T_min > 0.0) ||
                      !(mat->T_max > mat->T_min) || !std::isfinite(mat->T_max)))
        return fail(GADEP_E_INVAL, "plan: e_model 1 needs gadep_materials.e_range (e_n >= 2, 0 < T_min < T_max)");
    const MeshData &geo = b->geo;
    // compact the materials the mesh uses; all-zero tables behave as vacuum (-1),
    // for charged particles too
    const size_t ng = (size_t)mat->n_grid;
    std::vector<int> slot(mat->n_mat, -2);
    std::vector<float4> xs;
    std::vector<float> er;          // charged-particle ranges of the staged materials
    std::vector<int32_t> regions(b->regions);
    for (int32_t r = 0; r < (int32_t)regions.size() / 4; ++r) {
        const int code = regions[4 * r];
        if (code < 0 || code >= mat->n_mat) return fail(GADEP_E_INVAL, "plan: solid material %d has no table", code);
        if (slot[code] == -2) {
            bool any = false;
            for (size_t c = 0; c < 3 * ng; ++c) {
                const float v = mat->mu[(size_t)code * 3 * ng + c];
                if (!(v >= 0.0f) || !std::isfinite(v)) return fail(GADEP_E_INVAL, "plan: negative or non-finite attenuation");
                any = any || v > 0.0f;
            }
            if (!any) {
                slot[code] = -1;
            } else {
                slot[code] = (int)(xs.size() / ng);
                for (size_t g = 0; g < ng; ++g) {
                    const float *m = mat->mu + (size_t)code * 3 * ng;
                    xs.push_back(make_float4(m[g], m[ng + g], m[2 * ng + g], 0.0f));
                }
                if (electrons) {
                    const float *row = mat->e_range + (size_t)code * mat->e_n;
                    for (int32_t g = 0; g < mat->e_n; ++g) {
                        if (!(row[g] > 0.0f) || !std::isfinite(row[g]) || (g > 0 && !(row[g] > row[g - 1])))
                            return fail(GADEP_E_INVAL, "plan: e_range of material %d is not finite, positive "
                                                       "and increasing", code);
                        er.push_back(row[g]);
                    }
                }
            }
        }
        regions[4 * r] = slot[code];
    }
    regions[0] = -1;  // the world region is vacuum whatever the table says
    const int n_mat_c = (int)(xs.size() / ng);
    gadep_plan *p = new (std::nothrow) gadep_plan();
    if (!p) return fail(GADEP_E_NOMEM, "plan: out of host memory");
    p->bvh = b;
    p->device = b->device;
    p->n_inst = n_inst;
    p->grad = grad;
    p->count = count;
    p->opts = *opts;
    p->n_bins = opts->n_bins;
    // instances
    unsigned long long total = 0;
    for (int32_t i = 0; i < n_inst; ++i) {
        const gadep_instance &I = inst[i];
        const gadep_source &s = I.src;
        if (!(I.energy_keV > 0.0f) || !std::isfinite(I.energy_keV) || I.energy_keV > 1e5f) {
            gadep_plan_destroy(p);
            return fail(GADEP_E_INVAL, "plan: instance %d energy must be in (0, 1e5] keV", i);
        }
        if (I.n_hist >= (1ull << 32)) { gadep_plan_destroy(p); return fail(GADEP_E_INVAL, "plan: n_hist must be < 2^32"); }
        dev::InstDev d{};
        d.E0 = I.energy_keV;
        d.src_kind = s.kind;
        d.px = s.pos[0]; d.py = s.pos[1]; d.pz = s.pos[2];
        d.dx = s.dir[0]; d.dy = s.dir[1]; d.dz = s.dir[2];
        d.radius = s.radius; d.height = s.height; d.n_sides = s.n_sides;
        d.inst_id = I.instance;
        d.hist_offset = opts->history_offset;
        for (int g = 0; g < GADEP_MAX_GROUPS; ++g) {
            d.scale[g] = I.group_scale[g];
            if (!(d.scale[g] >= 0.0f) || !std::isfinite(d.scale[g])) { gadep_plan_destroy(p); return fail(GADEP_E_INVAL, "plan: bad group scale"); }
        }
        if (s.kind == GADEP_SRC_PRISM) {
            if (s.solid < 0 || s.solid >= geo.n_solid() || s.n_sides < 3 || !(s.radius > 0) || !(s.height > 0)) {
                gadep_plan_destroy(p);
                return fail(GADEP_E_INVAL, "plan: prism source needs a valid solid, n_sides >= 3, radius, height");
            }
            d.birth_region = s.solid + 1;
        } else if (s.kind == GADEP_SRC_POINT || s.kind == GADEP_SRC_DISK || s.kind == GADEP_SRC_PENCIL) {
            if (s.kind == GADEP_SRC_DISK && !(s.radius > 0)) { gadep_plan_destroy(p); return fail(GADEP_E_INVAL, "plan: disk radius"); }
            if (s.kind == GADEP_SRC_PENCIL) {
                const double n2 = (double)s.dir[0] * s.dir[0] + (double)s.dir[1] * s.dir[1] + (double)s.dir[2] * s.dir[2];
                if (!(std::fabs(n2 - 1.0) < 1e-5)) { gadep_plan_destroy(p); return fail(GADEP_E_INVAL, "plan: pencil direction must be a unit vector"); }
            }
            const double q[3] = { s.pos[0], s.pos[1], s.pos[2] };
            const int32_t r = locate_point(geo, q);
            if (r == -2) { gadep_plan_destroy(p); return fail(GADEP_E_INVAL, "plan: source position lies on a surface"); }
            d.birth_region = r + 1;
        } else {
            gadep_plan_destroy(p);
            return fail(GADEP_E_INVAL, "plan: unknown source kind %d", s.kind);
        }
        p->inst.push_back(d);
        total += I.n_hist;
        p->inst_end.push_back(total);
    }
    // launch shape
    p->block = opts->block ? opts->block : 256;
    const size_t smem = regions.size() * 4 + (size_t)n_inst * 8;
    p->smem = (int)smem;
    DeviceGuard g(p->device);
    if (!g.ok) { gadep_plan_destroy(p); return fail(GADEP_E_CUDA, "plan: cannot select device %d", p->device); }
    int dev_smem = 0, n_sm = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device);
    if (smem > (size_t)dev_smem) {
        gadep_plan_destroy(p);
        return fail(GADEP_E_INVAL, "plan: tables need %zu bytes of shared memory, the device has %d", smem, dev_smem);
    }
    void *kfn = pick_kernel(grad, count, opts->e_model == 1);
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { gadep_plan_destroy(p); return cuda_fail(e, "plan: cudaFuncSetAttribute"); }
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, p->block, smem);
    if (e != cudaSuccess || bps < 1) { gadep_plan_destroy(p); return fail(GADEP_E_CUDA, "plan: kernel does not fit on the device"); }
    if (opts->blocks_per_sm > 0) bps = std::min(bps, opts->blocks_per_sm);
    p->grid = n_sm * bps;
    // form of the transport.  AUTO takes the wavefront kernels when many photons
    // reach the scene (measured faster from a few million histories on), and for
    // very large runs of a distant source, whose histories mostly end at birth
    // (gen culls them faster than the megakernel's lanes); the megakernel
    // otherwise -- with few photons in flight the wavefront's ~0.1 ms per
    // iteration dominates (measured: detector #2, source at 250 mm, 1e7 histories
    // per energy 5x faster in the megakernel, 1e8 per energy 2.5x faster in the
    // wavefront form)
    float box_lo[3], box_hi[3];
    scene_box(b, box_lo, box_hi);
    double reaching = 0.0;   // histories expected to reach the scene
    for (int32_t i = 0; i < n_inst; ++i) reaching += (double)inst[i].n_hist * hit_fraction(p->inst[i], box_lo, box_hi);
    int variant = opts->variant;
    const bool wf_ok = n_inst <= kWavefrontMaxInstances &&
                       wavefront_supports((int)(regions.size() / 4), (long long)b->geo.n_tri());
    // The wavefront form has a fixed cost per run (~2.5 ms: slot set, iterations of
    // small queues) and ~1.5 ns per history that reaches the scene; the megakernel
    // ~1 ms and ~6.7 ns (coax and Table 4 detector at 2e6 .. 1e7 histories per run):
    // break-even near 2.9e5 reaching histories.  Histories that miss the scene cost
    // little in either form.
    if (variant == GADEP_VARIANT_AUTO)
        variant = wf_ok && reaching >= (double)(1u << 18) ? GADEP_VARIANT_WAVEFRONT : GADEP_VARIANT_MEGA;
    if (variant == GADEP_VARIANT_WAVEFRONT && !wf_ok) {
        gadep_plan_destroy(p);
        return fail(GADEP_E_INVAL, "plan: the wavefront form takes at most %d instances, 256 regions and "
                                   "2^23 - 1 triangles", kWavefrontMaxInstances);
    }
    if (variant == GADEP_VARIANT_WAVEFRONT) {
        int slots = opts->wf_slots;
        if (slots <= 0) {
            // every photon that reaches the scene in flight at once where that fits:
            // the sorted queue's buckets fill and the iterations are fewer (coax,
            // 2.5e7 reaching per run: 2^25 slots 4.9 % faster than 2^24)
            slots = 1 << 20;
            while (slots < (1 << 25) && (double)slots < reaching) slots <<= 1;
        }
        p->wf_slots = slots;
        gadep_bvh *bm = const_cast<gadep_bvh *>(b);
        {
            std::lock_guard<std::mutex> lock(bm->wf_mutex);
            if (!bm->wf_cache_busy) {
                // keep the largest buffers seen; a run uses the slots it asked for
                if (bm->wf_cache && bm->wf_cache_slots < slots) {
                    wavefront_destroy(bm->wf_cache);
                    bm->wf_cache = nullptr;
                }
                if (!bm->wf_cache) {
                    st = wavefront_create(p->device, slots, grad, &bm->wf_cache);
                    if (st == GADEP_OK) bm->wf_cache_slots = slots;
                }
                if (bm->wf_cache) {
                    p->wf = bm->wf_cache;
                    p->wf_cached = true;
                    bm->wf_cache_busy = true;
                }
            }
        }
        if (!p->wf && (st = wavefront_create(p->device, slots, grad, &p->wf)) != GADEP_OK) {
            gadep_plan_destroy(p);
            return st;
        }
        p->grid = wavefront_trace_grid(p->wf);
    }
    // device buffers: one block (the BVH's, run after run, when the plan holds the
    // BVH's wavefront buffers)
    p->n_stripes = std::max(1, std::min(256, 65536 / n_inst));
    size_t need = 0;
    auto carve = [&need](size_t bytes) {
        const size_t at = need;
        need += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
        return at;
    };
    const size_t o_xs = carve(xs.size() * sizeof(float4));
    const size_t o_er = carve(er.size() * sizeof(float));
    const size_t o_reg = carve(regions.size() * sizeof(int32_t));
    const size_t o_inst = carve((size_t)n_inst * sizeof(dev::InstDev));
    const size_t o_end = carve((size_t)n_inst * sizeof(unsigned long long));
    const size_t o_tally = carve((size_t)n_inst * p->n_stripes * sizeof(dev::TallyDev));
    const size_t o_spec = carve((size_t)n_inst * p->n_bins * sizeof(uint32_t));
    const size_t o_work = carve(sizeof(unsigned long long));
    const size_t o_cnt = carve(4 * sizeof(unsigned long long));
    if (p->wf_cached) {
        gadep_bvh *bm = const_cast<gadep_bvh *>(b);
        std::lock_guard<std::mutex> lock(bm->wf_mutex);   // this plan holds the cache (busy)
        if (bm->plan_scratch_bytes < need) {
            cudaFree(bm->plan_scratch);
            bm->plan_scratch = nullptr;
            bm->plan_scratch_bytes = 0;
            if ((e = cudaMalloc(&bm->plan_scratch, need)) != cudaSuccess) {
                cudaGetLastError();
                bm->plan_scratch = nullptr;
            } else {
                bm->plan_scratch_bytes = need;
            }
        }
        if (bm->plan_scratch) {
            p->scratch = bm->plan_scratch;
            p->scratch_cached = true;
        }
    }
    if (!p->scratch && (e = cudaMalloc(&p->scratch, need)) != cudaSuccess) {
        cudaGetLastError();
        p->scratch = nullptr;
        gadep_plan_destroy(p);
        return fail(GADEP_E_NOMEM, "plan: cudaMalloc of %zu bytes failed", need);
    }
    {
        char *base = (char *)p->scratch;
        p->d_xs = (float4 *)(base + o_xs);
        p->d_erange = er.empty() ? nullptr : (float *)(base + o_er);
        p->d_regions = (int4 *)(base + o_reg);
        p->d_inst = (dev::InstDev *)(base + o_inst);
        p->d_end = (unsigned long long *)(base + o_end);
        p->d_tally = (dev::TallyDev *)(base + o_tally);
        p->d_spectra = (uint32_t *)(base + o_spec);
        p->d_work = (unsigned long long *)(base + o_work);
        p->d_counters = (unsigned long long *)(base + o_cnt);
    }
    if ((!xs.empty() && (e = cudaMemcpy(p->d_xs, xs.data(), xs.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (!er.empty() && (e = cudaMemcpy(p->d_erange, er.data(), er.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(p->d_regions, regions.data(), regions.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_inst, p->inst.data(), p->inst.size() * sizeof(dev::InstDev), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_end, p->inst_end.data(), p->inst_end.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) {
        gadep_plan_destroy(p);
        return cuda_fail(e, "plan: upload");
    }
    dev::Params &P = p->P;
    P.nodes = (const float4 *)b->d_nodes;
    P.tris = (const float4 *)b->d_tris;
    P.planes = (const float4 *)b->d_planes;
    P.xs = p->d_xs;
    P.regions = p->d_regions;
    P.inst = p->d_inst;
    P.inst_end = p->d_end;
    P.tally = p->d_tally;
    P.spectra = p->d_spectra;
    P.work = p->d_work;
    P.edep_trace = nullptr;
    P.n_trace = 0;
    P.total = total;
    P.n_mat = n_mat_c;
    P.n_grid = mat->n_grid;
    P.n_region = (int)(regions.size() / 4);
    P.n_inst = n_inst;
    P.lnE_min = (float)std::log(mat->E_min);
    P.inv_dlnE = (float)((mat->n_grid - 1) / (std::log(mat->E_max) - std::log(mat->E_min)));
    P.key0 = (uint32_t)opts->seed;
    P.key1 = (uint32_t)(opts->seed >> 32);
    P.e_cut = opts->e_cut_keV;
    P.fep_delta = opts->fep_delta_keV;
    P.e_max = opts->e_max_keV;
    P.bin_scale = (float)opts->n_bins / opts->e_max_keV;
    P.n_bins = opts->n_bins;
    P.step_cap = opts->step_cap;
    P.n_group = opts->n_group;
    P.chunk = opts->chunk > 0 ? opts->chunk : 256;
    P.n_stripes = p->n_stripes;
    P.root_all = b->root_all;
    P.erange = p->d_erange;
    P.e_model = electrons ? 1 : 0;
    P.e_n = electrons ? mat->e_n : 0;
    P.e_T_min = electrons ? (float)mat->T_min : 0.0f;
    P.e_lnT_min = electrons ? (float)std::log(mat->T_min) : 0.0f;
    P.e_inv_dlnT = electrons ? (float)((mat->e_n - 1) / (std::log(mat->T_max) - std::log(mat->T_min))) : 0.0f;
    // scene bounds seen from the world (births outside it whose ray misses it end at once)
    scene_box(b, P.root_lo, P.root_hi);
    *out = p;
    return GADEP_OK;
}

gadep_status plan_launch(gadep_plan *p, uint32_t *spectra_dev, float *edep_trace, uint64_t n_trace,
                         cudaStream_t s)
{
    DeviceGuard g(p->device);
    dev::Params P = p->P;
    if (spectra_dev) P.spectra = spectra_dev;
    P.edep_trace = edep_trace;
    P.n_trace = edep_trace ? n_trace : 0;
    p->last_spectra = P.spectra;
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->d_tally, 0, sizeof(dev::TallyDev) * p->n_inst * p->n_stripes, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.spectra, 0, sizeof(uint32_t) * (size_t)p->n_inst * p->n_bins, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_work, 0, sizeof(unsigned long long), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->d_counters, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(e, "plan launch: memset");
    if (P.total == 0) return GADEP_OK;
    if (p->wf) return wavefront_run(p->wf, P, p->grad, p->count, p->d_counters, &p->timer, s, p->wf_slots);
    p->timer.before(s);
    if (p->grad) {
        if (p->count) dev::transport_kernel<true, true, false><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
        else dev::transport_kernel<true, false, false><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
    } else if (P.e_model) {
        if (p->count) dev::transport_kernel<false, true, true><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
        else dev::transport_kernel<false, false, true><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
    } else {
        if (p->count) dev::transport_kernel<false, true, false><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
        else dev::transport_kernel<false, false, false><<<p->grid, p->block, p->smem, s>>>(P, p->d_counters);
    }
    p->timer.after(KK_MEGA, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? GADEP_OK : cuda_fail(e, "plan launch: kernel");
}

gadep_status plan_results(gadep_plan *p, uint32_t *spectra_host, gadep_result *res, double *dfepe,
                          double *dsigma, unsigned long long *counters, cudaStream_t s)
{
    DeviceGuard g(p->device);
    const size_t n_copies = (size_t)p->n_inst * p->n_stripes;
    std::vector<dev::TallyDev> stripes(n_copies);
    cudaError_t e = cudaMemcpyAsync(stripes.data(), p->d_tally, sizeof(dev::TallyDev) * n_copies,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && spectra_host)
        e = cudaMemcpyAsync(spectra_host, p->last_spectra ? p->last_spectra : p->d_spectra,
                            sizeof(uint32_t) * (size_t)p->n_inst * p->n_bins, cudaMemcpyDeviceToHost, s);
    unsigned long long cnt[4] = { 0, 0, 0, 0 };
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, p->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "plan results");
    if (p->wf) {
        const gadep_status st = wavefront_check(p->wf, s);   // iteration bound of a graph-driven run
        if (st != GADEP_OK) return st;
    }
    if (counters) std::memcpy(counters, cnt, sizeof(cnt));
    // sum the per-block tally copies (integer counts exactly, FP64 sums in stripe order)
    std::vector<dev::TallyDev> T(p->n_inst);
    std::memset(T.data(), 0, sizeof(dev::TallyDev) * T.size());
    for (int k = 0; k < p->n_stripes; ++k) {
        for (int i = 0; i < p->n_inst; ++i) {
            const dev::TallyDev &a = stripes[(size_t)k * p->n_inst + i];
            dev::TallyDev &t = T[i];
            t.n_hist += a.n_hist; t.n_fep += a.n_fep; t.n_zero += a.n_zero; t.n_over += a.n_over;
            t.n_err += a.n_err; t.n_segments += a.n_segments; t.n_interactions += a.n_interactions;
            t.n_culled += a.n_culled;
            t.err_bits |= a.err_bits;
            t.sum_dep_active += a.sum_dep_active; t.sum_dep_all += a.sum_dep_all; t.sum_esc += a.sum_esc;
            for (int g2 = 0; g2 < GADEP_MAX_GROUPS; ++g2) {
                t.fep_score[g2] += a.fep_score[g2];
                t.fep_score_sq[g2] += a.fep_score_sq[g2];
            }
        }
    }
    bool dev_err = false;
    for (int i = 0; i < p->n_inst; ++i) {
        const dev::TallyDev &t = T[i];
        if (res) {
            gadep_result &r = res[i];
            std::memset(&r, 0, sizeof(r));
            r.n_hist = t.n_hist; r.n_fep = t.n_fep; r.n_zero = t.n_zero; r.n_over = t.n_over; r.n_err = t.n_err;
            r.n_segments = t.n_segments; r.n_interactions = t.n_interactions; r.n_culled = t.n_culled;
            r.fepe = t.n_hist ? (double)t.n_fep / (double)t.n_hist : 0.0;
            r.sigma = t.n_hist ? std::sqrt(r.fepe * (1.0 - r.fepe) / (double)t.n_hist) : 0.0;
            r.sum_dep_active = t.sum_dep_active; r.sum_dep_all = t.sum_dep_all; r.sum_esc = t.sum_esc;
            r.dev_err = (uint32_t)t.err_bits;
        }
        if (t.err_bits) dev_err = true;
        if (p->grad) {
            const double n = (double)t.n_hist;
            for (int g2 = 0; g2 < p->opts.n_group; ++g2) {
                const double m1 = n > 0 ? t.fep_score[g2] / n : 0.0;
                const double m2 = n > 0 ? t.fep_score_sq[g2] / n : 0.0;
                if (dfepe) dfepe[(size_t)i * p->opts.n_group + g2] = m1;
                if (dsigma) dsigma[(size_t)i * p->opts.n_group + g2] = n > 0 ? std::sqrt(std::max(m2 - m1 * m1, 0.0) / n) : 0.0;
            }
        }
    }
    if (dev_err) return fail(GADEP_E_DEVICE, "device error word set (see gadep_result.dev_err)");
    return GADEP_OK;
}

}  // namespace gadep

extern "C" gadep_status gadep_plan_create(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                                          const gadep_instance *inst, const gadep_opts *opts, int32_t grad,
                                          gadep_plan **out)
{
    gadep::clear_error();
    return gadep::plan_create(b, mat, n_inst, inst, opts, grad != 0, false, out);
}

extern "C" gadep_status gadep_plan_launch(gadep_plan *p, uint32_t *spectra_dev, void *stream)
{
    gadep::clear_error();
    if (!p) return fail(GADEP_E_INVAL, "gadep_plan_launch: NULL plan");
    if (spectra_dev && !is_device_ptr(spectra_dev)) return fail(GADEP_E_INVAL, "gadep_plan_launch: spectra must be device memory");
    return gadep::plan_launch(p, spectra_dev, nullptr, 0, (cudaStream_t)stream);
}

extern "C" gadep_status gadep_plan_results(gadep_plan *p, uint32_t *spectra_host, gadep_result *results,
                                           double *dfepe, double *dsigma, void *stream)
{
    gadep::clear_error();
    if (!p) return fail(GADEP_E_INVAL, "gadep_plan_results: NULL plan");
    return gadep::plan_results(p, spectra_host, results, dfepe, dsigma, nullptr, (cudaStream_t)stream);
}

extern "C" gadep_status gadep_measure_peaks(int32_t device, double *fp32_tflops, double *l2_read_gbs)
{
    gadep::clear_error();
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess) { cudaGetLastError(); n_dev = 0; }
    if (device < 0 || device >= n_dev) return fail(GADEP_E_INVAL, "gadep_measure_peaks: no CUDA device %d", device);
    DeviceGuard g(device);
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    const size_t n4 = (64u << 20) / sizeof(float4);
    float4 *buf = nullptr;
    float *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&buf, n4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)n_sm * 8 * 256 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, n4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best_fma = INFINITY, best_l2 = INFINITY;
    const int grid = n_sm * 8, rounds = 16;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        float ms = 0.0f;
        e = cudaEventRecord(a);
        gadep::dev::fma_peak_kernel<<<grid, 256>>>(0.999999f, 1e-6f, out);
        if (e == cudaSuccess) e = cudaEventRecord(b);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0) best_fma = std::min(best_fma, ms);
        if (e == cudaSuccess) e = cudaEventRecord(a);
        gadep::dev::l2_read_kernel<<<grid, 256>>>(buf, n4, rounds, out);
        if (e == cudaSuccess) e = cudaEventRecord(b);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0) best_l2 = std::min(best_l2, ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(out);
    if (e != cudaSuccess) return gadep::cuda_fail(e, "gadep_measure_peaks");
    const double flop = 2.0 * 8.0 * gadep::dev::kFmaIters * (double)grid * 256.0;
    if (fp32_tflops) *fp32_tflops = flop / (best_fma * 1e-3) / 1e12;
    if (l2_read_gbs) *l2_read_gbs = (double)rounds * n4 * sizeof(float4) / (best_l2 * 1e-3) / 1e9;
    return GADEP_OK;
}

extern "C" gadep_status gadep_plan_set_timing(gadep_plan *p, int32_t on)
{
    gadep::clear_error();
    if (!p) return fail(GADEP_E_INVAL, "gadep_plan_set_timing: NULL plan");
    p->timer.timing = on != 0;
    return GADEP_OK;
}

extern "C" gadep_status gadep_plan_kernel_stats(gadep_plan *p, gadep_kernel_stats *out, int32_t reset)
{
    gadep::clear_error();
    if (!p || !out) return fail(GADEP_E_INVAL, "gadep_plan_kernel_stats: NULL argument");
    DeviceGuard g(p->device);
    const cudaError_t e = p->timer.resolve();
    std::memset(out, 0, sizeof(*out));
    for (int k = 0; k < gadep::KK_N && k < 16; ++k) {
        out->launches[k] = p->timer.launches[k];
        out->ms[k] = p->timer.ms[k];
    }
    if (reset) p->timer.reset();
    return e == cudaSuccess ? GADEP_OK : gadep::cuda_fail(e, "gadep_plan_kernel_stats: event");
}

extern "C" gadep_status gadep_plan_queue_sizes(gadep_plan *p, uint32_t *out, int32_t max, int32_t *n, void *stream)
{
    gadep::clear_error();
    if (!p || !n || (max > 0 && !out)) return fail(GADEP_E_INVAL, "gadep_plan_queue_sizes: NULL argument");
    *n = 0;
    if (!p->wf) return GADEP_OK;
    DeviceGuard g(p->device);
    int k = 0;
    const gadep_status st = gadep::wavefront_queue_log(p->wf, out, max, &k, (cudaStream_t)stream);
    *n = k;
    return st;
}

extern "C" gadep_status gadep_plan_shape(const gadep_plan *p, int32_t *grid, int32_t *block, int32_t *smem_bytes)
{
    gadep::clear_error();
    if (!p) return fail(GADEP_E_INVAL, "gadep_plan_shape: NULL plan");
    if (grid) *grid = p->grid;
    if (block) *block = p->block;
    if (smem_bytes) *smem_bytes = p->smem;
    return GADEP_OK;
}

namespace {

// run a batch through a temporary plan; spectra may be host or device
gadep_status run_batch(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst, const gadep_instance *inst,
                       const gadep_opts *opts, bool grad, uint32_t *spectra, float *edep_trace, uint64_t n_trace,
                       gadep_result *results, double *dfepe, double *dsigma, unsigned long long *counters,
                       bool count, cudaStream_t s)
{
    if (edep_trace && !is_device_ptr(edep_trace)) return fail(GADEP_E_INVAL, "edep_trace must be device memory");
    gadep_plan *p = nullptr;
    gadep_status st = gadep::plan_create(b, mat, n_inst, inst, opts, grad, count, &p);
    if (st != GADEP_OK) return st;
    const bool dev_spec = spectra && is_device_ptr(spectra);
    st = gadep::plan_launch(p, dev_spec ? spectra : nullptr, edep_trace, n_trace, s);
    if (st == GADEP_OK)
        st = gadep::plan_results(p, dev_spec ? nullptr : spectra, results, dfepe, dsigma, counters, s);
    gadep_plan_destroy(p);
    return st;
}

}  // namespace

extern "C" gadep_status gadep_run(const gadep_bvh *b, const gadep_materials *mat, const gadep_source *src,
                                  float energy_keV, uint64_t n_hist, uint32_t instance, const gadep_opts *opts,
                                  uint32_t *spectrum, float *edep_trace, uint64_t n_trace, gadep_result *result,
                                  void *stream)
{
    gadep::clear_error();
    if (!src || !result) return fail(GADEP_E_INVAL, "gadep_run: NULL source or result");
    gadep_instance I;
    std::memset(&I, 0, sizeof(I));
    I.energy_keV = energy_keV;
    I.src = *src;
    I.n_hist = n_hist;
    I.instance = instance;
    if (opts)
        for (int g = 0; g < GADEP_MAX_GROUPS; ++g) I.group_scale[g] = opts->group_scale[g];
    return run_batch(b, mat, 1, &I, opts, false, spectrum, edep_trace, n_trace, result, nullptr, nullptr,
                     nullptr, false, (cudaStream_t)stream);
}

extern "C" gadep_status gadep_run_batch(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                                        const gadep_instance *inst, const gadep_opts *opts, uint32_t *spectra,
                                        gadep_result *results, void *stream)
{
    gadep::clear_error();
    if (!results) return fail(GADEP_E_INVAL, "gadep_run_batch: NULL results");
    return run_batch(b, mat, n_inst, inst, opts, false, spectra, nullptr, 0, results, nullptr, nullptr, nullptr,
                     false, (cudaStream_t)stream);
}

extern "C" gadep_status gadep_grad(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                                   const gadep_instance *inst, const gadep_opts *opts, uint32_t *spectra,
                                   gadep_result *results, double *dfepe, double *dsigma, void *stream)
{
    gadep::clear_error();
    if (!results || !dfepe || !dsigma) return fail(GADEP_E_INVAL, "gadep_grad: NULL output");
    if (!opts || opts->n_group < 1) return fail(GADEP_E_INVAL, "gadep_grad: opts.n_group must be >= 1");
    return run_batch(b, mat, n_inst, inst, opts, true, spectra, nullptr, 0, results, dfepe, dsigma, nullptr, false,
                     (cudaStream_t)stream);
}

// Work counters of the traversal (nodes visited, boxes and triangles tested) for
// one batch: the COUNT instantiation of the same kernels, used to derive
// algorithmic bytes and FLOPs per segment query.
extern "C" gadep_status gadep_count_work(const gadep_bvh *b, const gadep_materials *mat, int32_t n_inst,
                                         const gadep_instance *inst, const gadep_opts *opts,
                                         gadep_result *results, uint64_t *nodes_visited,
                                         uint64_t *tris_tested, uint64_t *relocated, uint64_t *boxes_tested,
                                         void *stream)
{
    gadep::clear_error();
    if (!results || !nodes_visited || !tris_tested) return fail(GADEP_E_INVAL, "gadep_count_work: NULL output");
    unsigned long long c[4] = { 0, 0, 0, 0 };
    gadep_status st = run_batch(b, mat, n_inst, inst, opts, false, nullptr, nullptr, 0, results, nullptr, nullptr,
                                c, true, (cudaStream_t)stream);
    *nodes_visited = c[0];
    *tris_tested = c[1];
    if (relocated) *relocated = c[2];
    if (boxes_tested) *boxes_tested = c[3];
    return st;
}

// ---------------------------------------------------------------------------
// Single-instance run without any device allocation (gadep_run_noalloc).
//
// For callers that must not allocate device memory during a run: applications
// that hand all device memory to their own allocator and forbid libraries from
// taking more, and loops that cannot afford the device synchronisation cudaFree
// implies.  Everything gadep_run keeps in allocated
// scratch -- the staged attenuation tables, the region table, the instance
// record, the tallies and the work counter -- lives here in one file-scope
// device array of fixed size, owned by every GPU that loads the library until
// the process exits.
// ---------------------------------------------------------------------------

namespace gadep {
namespace noalloc {

constexpr int kMaxTable = 12288;                    // float4 table entries: used materials x grid points
constexpr int kMaxRegions = kLocateMaxSolids + 1;   // world + solids

struct __align__(16) Layout {
    float4 xs[kMaxTable];                // interleaved (pe, compton, pair, 0) tables
    float raw[3 * kMaxTable];            // planar tables as copied from the caller
    int4 regions[kMaxRegions];
    dev::InstDev inst;
    unsigned long long inst_end[2];
    dev::TallyDev tally;
    unsigned long long work;
    unsigned long long counters[4];
};

}  // namespace noalloc
}  // namespace gadep

// 345,472 bytes (337 KiB) on every device that loads the library.
static_assert(sizeof(gadep::noalloc::Layout) == 345472, "scratch size stated in gadep.h");
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(gadep::noalloc::Layout)];

namespace gadep {
namespace noalloc {

__global__ void interleave_tables(const float *raw, int n_mat, int n_grid, float4 *xs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_mat * n_grid) return;
    const int m = i / n_grid, g = i - m * n_grid;
    const float *r = raw + (size_t)m * 3 * n_grid;
    xs[i] = make_float4(r[g], r[n_grid + g], r[2 * n_grid + g], 0.0f);
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
Layout *g_ptr[kMaxDevices] = { nullptr };

// Device address of the scratch array on `device` (current), looked up once.
gadep_status scratch_of(int device, Layout **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(GADEP_E_INVAL, "gadep_run_noalloc: device index %d", device);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(GADEP_E_CUDA, "gadep_run_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        }
        g_ptr[device] = (Layout *)p;
    }
    *out = g_ptr[device];
    return GADEP_OK;
}

}  // namespace noalloc
}  // namespace gadep

extern "C" gadep_status gadep_run_noalloc(const gadep_bvh *b, const gadep_materials *mat, const gadep_source *src,
                                          float energy_keV, uint64_t n_hist, uint32_t instance,
                                          const gadep_opts *opts, uint32_t *spectrum_dev, gadep_result *result,
                                          void *stream)
{
    using namespace gadep;
    using noalloc::Layout;
    clear_error();
    if (!b || !mat || !src || !result || !spectrum_dev)
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: NULL argument");
    if (b->device < 0 || !b->d_nodes) return fail(GADEP_E_INVAL, "gadep_run_noalloc: the BVH has no device copy");
    gadep_status st = check_opts(opts);
    if (st != GADEP_OK) return st;
    if (opts->e_model != 0) return fail(GADEP_E_INVAL, "gadep_run_noalloc: e_model 1 needs gadep_run");
    if (opts->variant == GADEP_VARIANT_WAVEFRONT)
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: the wavefront form needs gadep_run (its photon slots are "
                                   "allocated); this call runs the megakernel");
    if (n_hist >= (1ull << 32)) return fail(GADEP_E_INVAL, "gadep_run_noalloc: n_hist must be < 2^32");
    if (!(energy_keV > 0.0f) || !std::isfinite(energy_keV) || energy_keV > 1e5f)
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: energy must be in (0, 1e5] keV");
    if (!mat->mu || mat->n_mat < 1 || mat->n_mat > 1024 || mat->n_grid < 2 || mat->n_grid > noalloc::kMaxTable ||
        !(mat->E_min > 0.0) || !(mat->E_max > mat->E_min))
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: bad gadep_materials");
    const int n_region = (int)(b->regions.size() / 4);
    if (n_region > noalloc::kMaxRegions)
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: at most %d solids (mesh has %d)", noalloc::kMaxRegions - 1,
                    n_region - 1);
    if (!is_device_ptr(spectrum_dev)) return fail(GADEP_E_INVAL, "gadep_run_noalloc: spectrum must be device memory");
    DeviceGuard g(b->device);
    if (!g.ok) return fail(GADEP_E_CUDA, "gadep_run_noalloc: cannot select device %d", b->device);
    Layout *S = nullptr;
    if ((st = noalloc::scratch_of(b->device, &S)) != GADEP_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t ng = (size_t)mat->n_grid;

    // regions and the materials they use (all-zero tables act as vacuum; the world is vacuum)
    int4 regions[noalloc::kMaxRegions];
    int slot[1024];
    for (int i = 0; i < mat->n_mat; ++i) slot[i] = -2;
    int n_used = 0;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < n_region; ++r) {
        const int code = b->regions[4 * r];
        if (code < 0 || code >= mat->n_mat) return fail(GADEP_E_INVAL, "gadep_run_noalloc: solid material %d has no table", code);
        if (slot[code] == -2) {
            const float *rows = mat->mu + (size_t)code * 3 * ng;
            bool any = false;
            for (size_t c = 0; c < 3 * ng; ++c) {
                if (!(rows[c] >= 0.0f) || !std::isfinite(rows[c]))
                    return fail(GADEP_E_INVAL, "gadep_run_noalloc: negative or non-finite attenuation");
                any = any || rows[c] > 0.0f;
            }
            if (!any) {
                slot[code] = -1;
            } else {
                if ((size_t)(n_used + 1) * ng > (size_t)noalloc::kMaxTable)
                    return fail(GADEP_E_INVAL, "gadep_run_noalloc: tables exceed %d entries (materials x grid points)",
                                noalloc::kMaxTable);
                slot[code] = n_used++;
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S->raw + (size_t)slot[code] * 3 * ng, rows, 3 * ng * sizeof(float),
                                        cudaMemcpyHostToDevice, s);
            }
        }
        regions[r] = make_int4(slot[code], b->regions[4 * r + 1], b->regions[4 * r + 2], b->regions[4 * r + 3]);
    }
    regions[0].x = -1;
    // instance record with its birth region (parity rule for sources outside the mesh)
    dev::InstDev d{};
    d.E0 = energy_keV;
    d.src_kind = src->kind;
    d.px = src->pos[0]; d.py = src->pos[1]; d.pz = src->pos[2];
    d.dx = src->dir[0]; d.dy = src->dir[1]; d.dz = src->dir[2];
    d.radius = src->radius; d.height = src->height; d.n_sides = src->n_sides;
    d.inst_id = instance;
    d.hist_offset = opts->history_offset;
    for (int k = 0; k < GADEP_MAX_GROUPS; ++k) d.scale[k] = opts->group_scale[k];
    if (src->kind == GADEP_SRC_PRISM) {
        if (src->solid < 0 || src->solid >= b->geo.n_solid() || src->n_sides < 3 || !(src->radius > 0) || !(src->height > 0))
            return fail(GADEP_E_INVAL, "gadep_run_noalloc: prism source needs a valid solid, n_sides >= 3, radius, height");
        d.birth_region = src->solid + 1;
    } else if (src->kind == GADEP_SRC_POINT || src->kind == GADEP_SRC_DISK || src->kind == GADEP_SRC_PENCIL) {
        if (src->kind == GADEP_SRC_DISK && !(src->radius > 0)) return fail(GADEP_E_INVAL, "gadep_run_noalloc: disk radius");
        if (src->kind == GADEP_SRC_PENCIL) {
            const double n2 = (double)src->dir[0] * src->dir[0] + (double)src->dir[1] * src->dir[1] +
                              (double)src->dir[2] * src->dir[2];
            if (!(std::fabs(n2 - 1.0) < 1e-5)) return fail(GADEP_E_INVAL, "gadep_run_noalloc: pencil direction must be a unit vector");
        }
        const double q[3] = { src->pos[0], src->pos[1], src->pos[2] };
        const int32_t r = locate_point_fixed(b->geo, q);
        if (r < -1) return fail(GADEP_E_INVAL, "gadep_run_noalloc: source position lies on a surface");
        d.birth_region = r + 1;
    } else {
        return fail(GADEP_E_INVAL, "gadep_run_noalloc: unknown source kind %d", src->kind);
    }
    const unsigned long long ends[2] = { n_hist, n_hist };

    // launch shape: the megakernel with gadep_run's megakernel shape rule
    const int block = opts->block ? opts->block : 256;
    const size_t smem = (size_t)n_region * sizeof(int4) + 8;
    int dev_smem = 0, n_sm = 0, bps = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (smem > (size_t)dev_smem) return fail(GADEP_E_INVAL, "gadep_run_noalloc: tables need too much shared memory");
    void *kfn = (void *)dev::transport_kernel<false, false, false>;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn, block, smem);
    if (e == cudaSuccess && bps < 1) return fail(GADEP_E_CUDA, "gadep_run_noalloc: kernel does not fit on the device");
    if (opts->blocks_per_sm > 0) bps = std::min(bps, opts->blocks_per_sm);

    // stage inputs into the scratch array, clear what must start at zero
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->regions, regions, (size_t)n_region * sizeof(int4), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&S->inst, &d, sizeof(d), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->inst_end, ends, sizeof(ends), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&S->tally, 0, sizeof(S->tally), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&S->work, 0, sizeof(S->work), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->counters, 0, sizeof(S->counters), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(spectrum_dev, 0, sizeof(uint32_t) * (size_t)opts->n_bins, s);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_fail(e, "gadep_run_noalloc: staging"); }
    if (n_used > 0) {
        const int n = n_used * (int)ng;
        noalloc::interleave_tables<<<(n + 255) / 256, 256, 0, s>>>(S->raw, n_used, (int)ng, S->xs);
    }
    dev::Params P{};
    P.nodes = (const float4 *)b->d_nodes;
    P.tris = (const float4 *)b->d_tris;
    P.planes = (const float4 *)b->d_planes;
    P.xs = S->xs;
    P.regions = S->regions;
    P.inst = &S->inst;
    P.inst_end = S->inst_end;
    P.tally = &S->tally;
    P.spectra = spectrum_dev;
    P.work = &S->work;
    P.edep_trace = nullptr;
    P.n_trace = 0;
    P.total = n_hist;
    P.n_mat = n_used;
    P.n_grid = mat->n_grid;
    P.n_region = n_region;
    P.n_inst = 1;
    P.lnE_min = (float)std::log(mat->E_min);
    P.inv_dlnE = (float)((mat->n_grid - 1) / (std::log(mat->E_max) - std::log(mat->E_min)));
    P.key0 = (uint32_t)opts->seed;
    P.key1 = (uint32_t)(opts->seed >> 32);
    P.e_cut = opts->e_cut_keV;
    P.fep_delta = opts->fep_delta_keV;
    P.e_max = opts->e_max_keV;
    P.bin_scale = (float)opts->n_bins / opts->e_max_keV;
    P.n_bins = opts->n_bins;
    P.step_cap = opts->step_cap;
    P.n_group = opts->n_group;
    P.chunk = opts->chunk > 0 ? opts->chunk : 256;
    P.n_stripes = 1;                       // the one tally record of the scratch array
    P.root_all = b->root_all;
    gadep::scene_box(b, P.root_lo, P.root_hi);
    if (n_hist > 0)
        dev::transport_kernel<false, false, false><<<n_sm * bps, block, smem, s>>>(P, S->counters);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gadep_run_noalloc: launch");
    // tallies back to the host, finalise
    dev::TallyDev t;
    e = cudaMemcpyAsync(&t, &S->tally, sizeof(t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gadep_run_noalloc: results");
    std::memset(result, 0, sizeof(*result));
    result->n_hist = t.n_hist; result->n_fep = t.n_fep; result->n_zero = t.n_zero; result->n_over = t.n_over;
    result->n_err = t.n_err; result->n_segments = t.n_segments; result->n_interactions = t.n_interactions;
    result->n_culled = t.n_culled;
    result->fepe = t.n_hist ? (double)t.n_fep / (double)t.n_hist : 0.0;
    result->sigma = t.n_hist ? std::sqrt(result->fepe * (1.0 - result->fepe) / (double)t.n_hist) : 0.0;
    result->sum_dep_active = t.sum_dep_active; result->sum_dep_all = t.sum_dep_all; result->sum_esc = t.sum_esc;
    result->dev_err = (uint32_t)t.err_bits;
    if (t.err_bits) return fail(GADEP_E_DEVICE, "device error word set (see gadep_result.dev_err)");
    return GADEP_OK;
}
