// kernels_reuse_group.cu -- the paper's shared-group reuse (Sec. 5: groups mapped onto warp
// lanes with a subgroup exchange) for power-of-two blocks, and the queued first-hit
// validation (Eq. 7) of its unbiased estimator.
#include <cuda_runtime.h>

#include <atomic>

#include "occ_dens_x2.cuh"
#include "occ_reuse.cuh"

namespace occ {
namespace {

// ---------------------------------------------------------------------------------------
// Warp-cooperative GROUP kernel.  K = GW * GH lanes per group, 32 / K groups per warp
// laid side by side (warp block = (32/K * GW) x GH pixels), OCC_GROUP_WARPS warps side by side
// per CTA.
// ---------------------------------------------------------------------------------------
// Loading the hit-normal plane only for rays that hit saves bytes but adds a dependent
// round trip; OCC_GROUP_EAGER_R1=1 loads it together with the other planes (measured
// slower for AO at 1080p: 32.2 vs 28.8 us).
#ifndef OCC_GROUP_EAGER_R1
#define OCC_GROUP_EAGER_R1 0
#endif
// warps per CTA of the group kernel (side by side) and the load flavour: every byte of
// the G-buffer and records is read exactly once, so streaming loads (evict-first) can be
// used instead of read-only cached loads.
// 4 warps per CTA measured faster than 8 at 1080p (4x2 AO 27.5 against 29.1 us; shadows
// 32.8 against 34.8 us): the finer CTAs fill the SMs' slots left by finished ones sooner.
#ifndef OCC_GROUP_WARPS
#define OCC_GROUP_WARPS 4
#endif
// resident CTAs per SM requested from the register allocator (0: no request)
#ifndef OCC_GROUP_MIN_BLOCKS
#define OCC_GROUP_MIN_BLOCKS 0
#endif
#if OCC_GROUP_MIN_BLOCKS > 0
#define OCC_GROUP_BOUNDS __launch_bounds__(32 * OCC_GROUP_WARPS, OCC_GROUP_MIN_BLOCKS)
#else
#define OCC_GROUP_BOUNDS __launch_bounds__(32 * OCC_GROUP_WARPS)
#endif
#ifndef OCC_GROUP_STREAM_LOADS
#define OCC_GROUP_STREAM_LOADS 0
#endif
// Fire-and-forget bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename T>
__device__ __forceinline__ T group_load(const T* p) {
    if (OCC_GROUP_STREAM_LOADS) return __ldcs(p);
    return __ldg(p);
}

// Densities of candidate (z, n_z) at two members given as float pairs (see occ_dens_x2.cuh).
template <int EFFECT>
__device__ __forceinline__ float2 dens_x2(f32x2 zx, f32x2 zy, f32x2 zz, f32x2 mnx, f32x2 mny,
                                          f32x2 mnz, float2 xs, float2 ys, float2 zs, float2 ns0,
                                          float2 ns1, float2 ns2, float R2s, const RectLight& L) {
    return dens_x2_pairs<EFFECT>(zx, zy, zz, mnx, mny, mnz, pk2(xs.x, xs.y), pk2(ys.x, ys.y),
                                 pk2(zs.x, zs.y), pk2(ns0.x, ns0.y), pk2(ns1.x, ns1.y),
                                 pk2(ns2.x, ns2.y), R2s, L);
}

template <int EFFECT, int EST, int GW, int GH, bool PACKED>
__global__ void OCC_GROUP_BOUNDS k_reuse_group(ReuseArgs a) {
    constexpr int K = GW * GH;
    constexpr int GPW = 32 / K;
    constexpr int BW = GPW * GW;
    // Columns without inline validation rays run on paired FP32 instructions, reading the
    // group's receivers from a structure-of-arrays block (x, y, z and the three receiver
    // terms, rows of K floats); the inline-validation columns read (x, valid) and receiver
    // term float4 slots.
    constexpr bool PAIRED = EST != kUnbiased;
    // receiver exchange buffer; group slots are K + 2 float4 apart so that the groups of a
    // warp reading their k-th member hit different shared-memory banks; the paired blocks
    // are 6K + 4 (K >= 4) or 6K + 2 floats apart for the same reason
    constexpr int GS = K + 2;
    constexpr int SS = 6 * K + (K >= 4 ? 4 : 2);
    __shared__ float4 s_x[OCC_GROUP_WARPS][PAIRED ? 1 : GPW * GS];
    __shared__ float4 s_n[OCC_GROUP_WARPS][PAIRED ? 1 : GPW * GS];
    __shared__ __align__(16) float s_soa[OCC_GROUP_WARPS][PAIRED ? GPW * SS : 4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / K, m = lane % K;
    // the CTA's warps sit side by side: each row of the CTA is contiguous pixels
    const int x = (blockIdx.x * OCC_GROUP_WARPS + warp) * BW + g * GW + m % GW;
    const int y = blockIdx.y * GH + m / GW;
    const bool inside = x < a.gb.W && y < a.gb.H;
    const int i = inside ? y * a.gb.W + x : 0;
    const int gi = inside ? gb_index(a.gb, x, y) : 0;   // G-buffer entry
    RectLight L;
    if (EFFECT == kShadow) L = make_light(a.lp);
    // Prefetch into L2 the rows of the CTA one wave of resident CTAs later (CTAs start in
    // launch order, so its loads then hit L2 instead of waiting for DRAM): one thread per
    // row and plane, one bulk prefetch each.
    if (a.pf_planes > 0 && !a.gb.tiled && threadIdx.x < (unsigned)(GH * a.pf_planes)) {
        constexpr int CW = OCC_GROUP_WARPS * BW;
        const unsigned t = blockIdx.y * gridDim.x + blockIdx.x + (unsigned)a.pf_ahead;
        if (t < gridDim.x * gridDim.y) {
            const int px = (int)(t % gridDim.x) * CW, py = (int)(t / gridDim.x) * GH + (int)threadIdx.x % GH;
            if (py < a.gb.H) {
                const int n = min(CW, a.gb.W - px);
                const int plane = (int)threadIdx.x / GH;
                // G-buffer planes are pitched, record planes dense
                const bool gplane = plane == 0 || (plane == 1 && !PACKED);
                const size_t q = (size_t)py * (gplane ? a.gb.pitch : a.gb.W) + px;
                const float4* base = plane == 0 ? a.gb.pos : plane == 1 ? (PACKED ? a.rec.r0 : a.gb.nrm)
                                   : plane == 2 ? a.rec.r0 : a.rec.r1;
                if (base && !(PACKED && plane >= 2)) prefetch_l2(base + q, (uint32_t)n * 16u);
            }
        }
    }

    float4 P = make_float4(0.0f, 0.0f, 0.0f, 0.0f), N = P;
    float4 R0 = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1)), R1 = P;
    float3 z = make_float3(0.0f, 0.0f, 0.0f), nz = z, nx = z;
    bool valid, hit;
    if (PACKED) {
        // 16 + 16 bytes per pixel: (x, octahedral normal) and the packed record
        if (inside) {
            P = group_load(a.gb.pos + gi);
            R0 = group_load(a.rec.r0 + i);
        }
        valid = inside && __float_as_uint(P.w) != kOctInvalid;
        hit = valid && __float_as_int(R0.w) >= 0;
        if (valid) nx = oct_decode(__float_as_uint(P.w));
        if (hit) rec_unpack(R0, f3(P), &z, &nz);
    } else {
        if (inside) {
            P = group_load(a.gb.pos + gi);
            N = group_load(a.gb.nrm + gi);
            R0 = group_load(a.rec.r0 + i);
            if (OCC_GROUP_EAGER_R1) R1 = group_load(a.rec.r1 + i);
        }
        valid = inside && P.w != 0.0f;
        hit = valid && __float_as_int(R0.w) >= 0;
        // a ray that missed provides no candidate, so its hit normal is not needed
        if (!OCC_GROUP_EAGER_R1 && hit) R1 = group_load(a.rec.r1 + i);
        nx = f3(N);
        z = f3(R0);
        nz = f3(R1);
    }
    // receiver data for the density: AO (x, n); shadow (x, precomputed plane terms)
    const Recv me = make_recv<EFFECT>(f3(P), nx, valid, L);
    if (PAIRED) {
        float* sg = &s_soa[warp][g * SS];
        sg[0 * K + m] = me.x.x;
        sg[1 * K + m] = me.x.y;
        sg[2 * K + m] = me.x.z;
        sg[3 * K + m] = valid ? me.n.x : 0.0f;
        sg[4 * K + m] = valid ? me.n.y : 0.0f;
        sg[5 * K + m] = valid ? me.n.z : 0.0f;
    } else {
        s_x[warp][g * GS + m] = make_float4(me.x.x, me.x.y, me.x.z, valid ? 1.0f : 0.0f);
        s_n[warp][g * GS + m] = make_float4(me.n.x, me.n.y, me.n.z, 0.0f);
    }
    __syncwarp();

    const unsigned gmask = (K == 32 ? 0xFFFFFFFFu : ((1u << K) - 1u)) << (g * K);
    const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid) & gmask;
    const unsigned hmask = __ballot_sync(0xFFFFFFFFu, hit) & gmask;

    // column of candidate z_m: densities at every receiver of the group
    float r[K];
    float Psum = 0.0f;
    uint32_t need = 0;                                     // kUnbCollect: members to validate
    const uint32_t vb = EST == kUnbFinal && hit ? __ldg(a.vbits + i) : 0u;
    if (PAIRED) {
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] = 0.0f;
        if (hit) {
            const float* sg = &s_soa[warp][g * SS];
            const f32x2 zx = bc2(z.x), zy = bc2(z.y), zz = bc2(z.z);
            const f32x2 mnx = bc2(-nz.x), mny = bc2(-nz.y), mnz = bc2(-nz.z);
            float2 q[K / 2];
            if (K >= 4) {
#pragma unroll
                for (int k = 0; k < K; k += 4) {
                    const float4 X = *reinterpret_cast<const float4*>(sg + 0 * K + k);
                    const float4 Y = *reinterpret_cast<const float4*>(sg + 1 * K + k);
                    const float4 Z = *reinterpret_cast<const float4*>(sg + 2 * K + k);
                    const float4 NX = *reinterpret_cast<const float4*>(sg + 3 * K + k);
                    const float4 NY = *reinterpret_cast<const float4*>(sg + 4 * K + k);
                    const float4 NZ = *reinterpret_cast<const float4*>(sg + 5 * K + k);
                    q[k / 2] = dens_x2<EFFECT>(zx, zy, zz, mnx, mny, mnz, make_float2(X.x, X.y),
                                               make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                                               make_float2(NX.x, NX.y), make_float2(NY.x, NY.y),
                                               make_float2(NZ.x, NZ.y), a.R2s, L);
                    q[k / 2 + 1] = dens_x2<EFFECT>(zx, zy, zz, mnx, mny, mnz, make_float2(X.z, X.w),
                                                   make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                                                   make_float2(NX.z, NX.w), make_float2(NY.z, NY.w),
                                                   make_float2(NZ.z, NZ.w), a.R2s, L);
                }
            } else {
                q[0] = dens_x2<EFFECT>(zx, zy, zz, mnx, mny, mnz,
                                       *reinterpret_cast<const float2*>(sg + 0 * K),
                                       *reinterpret_cast<const float2*>(sg + 1 * K),
                                       *reinterpret_cast<const float2*>(sg + 2 * K),
                                       *reinterpret_cast<const float2*>(sg + 3 * K),
                                       *reinterpret_cast<const float2*>(sg + 4 * K),
                                       *reinterpret_cast<const float2*>(sg + 5 * K), a.R2s, L);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float qk = (k & 1) ? q[k / 2].y : q[k / 2].x;
                if (EST == kUnbCollect && qk > 0.0f && k != m) need |= 1u << k;
                if (EST == kUnbFinal && k != m && !((vb >> k) & 1u)) qk = 0.0f;
                r[k] = qk;
                Psum += qk;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < (PAIRED ? 0 : K); ++k) {
        const float4 sx = s_x[warp][g * GS + k];
        const float4 sn = s_n[warp][g * GS + k];
        Recv rk;
        rk.x = f3(sx);
        rk.n = f3(sn);
        float q = 0.0f;
        if (hit && sx.w != 0.0f) q = density<EFFECT>(z, nz, rk, a.R2s, L);
        if (EST == kUnbiased && q > 0.0f && k != m)
            if (!first_hit(a.bvh, rk.x, z, (uint32_t)__float_as_int(R0.w), a.status)) q = 0.0f;
        if (EST == kUnbCollect && q > 0.0f && k != m) need |= 1u << k;
        if (EST == kUnbFinal && k != m && !((vb >> k) & 1u)) q = 0.0f;
        r[k] = q;
        Psum += q;
    }
    if (EST == kUnbCollect) {
        // append (candidate pixel, member) queries: a warp scan and one atomic per warp
        const int cnt = __popc(need);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        uint32_t base = 0;
        if (lane == 31 && incl > 0) base = atomicAdd(a.vcount, (unsigned)incl);
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        uint32_t pos = base + (uint32_t)(incl - cnt);
        while (need) {
            const int k = __ffs(need) - 1;
            need &= need - 1u;
            a.vq[pos++] = ((uint32_t)i << 4) | (uint32_t)k;
        }
        return;
    }
    const float inv = Psum > 0.0f ? 1.0f / Psum : 0.0f;
    if (PAIRED) {
        const f32x2 inv2 = bc2(inv);
#pragma unroll
        for (int k = 0; k < K; k += 2) {
            const float2 v = up2(mul2(pk2(r[k], r[k + 1]), inv2));
            r[k] = v.x;
            r[k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] *= inv;
    }

    // reduce-scatter over the group's lanes: lane m ends with sum_j r_j[m]
#pragma unroll
    for (int h = K / 2; h >= 1; h >>= 1) {
        const bool upper = (m & h) != 0;
#pragma unroll
        for (int e = 0; e < h; ++e) {
            const float keep = upper ? r[e + h] : r[e];
            const float send = upper ? r[e] : r[e + h];
            r[e] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, h);
        }
    }
    if (!inside) return;
    float res = 1.0f;
    if (valid) {
        res = 1.0f - r[0];
        if (EFFECT == kShadow && EST == kBiased && vmask == hmask) res = 0.0f;
    }
    a.out[i] = res;
}

// Eq. 7 for the queued pairs of the group kernel: the closest hit from member k's receiver
// x_k toward the candidate's occluder z (t in (0, 1 + 2^-10] in units of z - x_k, the same
// query as first_hit) must be z's own triangle; a success sets bit k of the candidate's word.
// Persistent: a warp refills its idle lanes from the query list once at least
// OCC_VALIDATE_MIN_IDLE lanes are idle, as in the dynamic trace.
#ifndef OCC_VALIDATE_MIN_IDLE
#define OCC_VALIDATE_MIN_IDLE 16
#endif
__global__ void __launch_bounds__(128, 8)
    k_validate(ReuseArgs a, unsigned* fetch) {
    const uint32_t n = *a.vcount;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int gw = a.pat.gw, gh = a.pat.gh, W = a.gb.W;
    Traversal t;
    StackEntry stack[kStackSize];
    trav_clear(t);
    t.overflow = false;
    t.bad = false;
    bool have = false, exhausted = false, overflow = false, bad = false;
    uint32_t cand = 0, bit = 0, tri = 0;
    for (;;) {
        while (!exhausted) {
            const unsigned need = __ballot_sync(0xFFFFFFFFu, !have);
            if (!need) break;
            if (__popc(need) < OCC_VALIDATE_MIN_IDLE && need != 0xFFFFFFFFu) break;
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(fetch, (unsigned)__popc(need));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base >= n) {
                exhausted = true;
                break;
            }
            if (!have) {
                const uint32_t idx = base + (uint32_t)__popc(need & below);
                if (idx < n) {
                    const uint32_t e = __ldg(a.vq + idx);
                    cand = e >> 4;
                    const int k = (int)(e & 15u);
                    const int x = (int)(cand % (uint32_t)W), y = (int)(cand / (uint32_t)W);
                    const int qm = ((y / gh) * gh + k / gw) * W + (x / gw) * gw + k % gw;
                    float3 xk = make_float3(0.0f, 0.0f, 0.0f), xi = xk, nn = xk, z = xk, nz = xk;
                    gb_fetch(a.gb, qm, &xk, &nn);
                    gb_fetch(a.gb, (int)cand, &xi, &nn);
                    tri = (uint32_t)fetch_cand(a.rec, (int)cand, xi, &z, &nz);
                    bit = 1u << k;
                    trav_init(t, xk, sub3(z, xk), kValidateTmax, 0u);
                    have = true;
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, have)) break;
        if (have) {
            trav_round(t, a.bvh, stack);
            if (trav_done(t)) {
                overflow |= t.overflow;
                bad |= t.bad;
                if (t.best_id == tri) atomicOr(a.vbits + cand, bit);
                have = false;
            }
        }
    }
    if (overflow && a.status) atomicOr(a.status, kStatusStackOverflowBit);
    if (OCC_CHECKS && bad && a.status) atomicOr(a.status, kStatusBadIndexBit);
}

// Resident CTAs of a kernel on this device (computed once per kernel; racing threads
// compute the same value).
template <typename Kern>
int resident_ctas(Kern k, std::atomic<int>& cache) {
    int n = cache.load(std::memory_order_relaxed);
    if (!n) {
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * OCC_GROUP_WARPS, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        n = per_sm * sm_count();
        cache.store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int EFFECT, int EST, int GW, int GH>
void launch_group_t(const ReuseArgs& a_in, cudaStream_t s) {
    constexpr int K = GW * GH;
    constexpr int BW = (32 / K) * GW;
    constexpr int CW = OCC_GROUP_WARPS * BW;
    const dim3 grid((unsigned)((a_in.gb.W + CW - 1) / CW), (unsigned)((a_in.gb.H + GH - 1) / GH));
    ReuseArgs a = a_in;
    static std::atomic<int> cache[2];
    if (a.gb.packed && a.rec.packed) {
        auto k = k_reuse_group<EFFECT, EST, GW, GH, true>;
        if (a.pf_planes) a.pf_ahead = resident_ctas(k, cache[1]);
        k<<<grid, 32 * OCC_GROUP_WARPS, 0, s>>>(a);
    } else if (!a.gb.packed && !a.rec.packed) {
        auto k = k_reuse_group<EFFECT, EST, GW, GH, false>;
        if (a.pf_planes) a.pf_ahead = resident_ctas(k, cache[0]);
        k<<<grid, 32 * OCC_GROUP_WARPS, 0, s>>>(a);
    }
}


template <int EFFECT, int EST>
bool launch_group(const ReuseArgs& a, cudaStream_t s) {
    const int gw = a.pat.gw, gh = a.pat.gh;
    if ((a.gb.packed != 0) != (a.rec.packed != 0)) return false;
    if (gw == 2 && gh == 1) { launch_group_t<EFFECT, EST, 2, 1>(a, s); return true; }
    if (gw == 2 && gh == 2) { launch_group_t<EFFECT, EST, 2, 2>(a, s); return true; }
    if (gw == 4 && gh == 2) { launch_group_t<EFFECT, EST, 4, 2>(a, s); return true; }
    if (gw == 4 && gh == 4) { launch_group_t<EFFECT, EST, 4, 4>(a, s); return true; }
    return false;
}

}  // namespace

bool launch_group_reuse(int effect, int est, const ReuseArgs& a, cudaStream_t s) {
    if (effect == kAO) {
        switch (est) {
            case kBiased: return launch_group<kAO, kBiased>(a, s);
            case kUnbiased: return launch_group<kAO, kUnbiased>(a, s);
            case kUnbCollect: return launch_group<kAO, kUnbCollect>(a, s);
            case kUnbFinal: return launch_group<kAO, kUnbFinal>(a, s);
            default: return false;
        }
    }
    switch (est) {
        case kBiased: return launch_group<kShadow, kBiased>(a, s);
        case kUnbiased: return launch_group<kShadow, kUnbiased>(a, s);
        case kUnbCollect: return launch_group<kShadow, kUnbCollect>(a, s);
        case kUnbFinal: return launch_group<kShadow, kUnbFinal>(a, s);
        default: return false;
    }
}

cudaError_t launch_validate(const ReuseArgs& a, cudaStream_t s) {
    static std::atomic<int> cached{0};   // persistent grid: resident CTAs per SM x SMs
    int ctas = cached.load(std::memory_order_relaxed);
    if (!ctas) {
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_validate, 128, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        ctas = per_sm * sm_count();
        cached.store(ctas, std::memory_order_relaxed);
    }
    k_validate<<<ctas, 128, 0, s>>>(a, a.vcount + 1);
    return cudaGetLastError();
}

}  // namespace occ
