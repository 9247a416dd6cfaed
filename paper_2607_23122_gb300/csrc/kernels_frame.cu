// kernels_frame.cu -- steps 1-3 of Algorithms 1 and 2 in one kernel for shared groups.
//
// The paper's own pass (Sec. 5, "Reuse Implementation") traces the step-1 rays of a
// group in neighbouring lanes and exchanges the occluders among those lanes, so the
// records never travel through device memory.  Here a warp holds (8 / GW) x (4 / GH)
// groups of GW x GH receivers covering an 8 x 4 pixel sub-tile (lane = group * K +
// member, members row-major in the block), each lane traces its own ray, and once every
// ray of a group has finished the group's lanes evaluate the estimate: lane j owns the
// candidate z_j, sums its column P_j = sum_k p(z_j|x_k) (Eq. 12), and a recursive-
// halving shuffle reduce-scatter hands lane i its B_i = sum_j p(z_j|x_i) / P_j
// (Eqs. 17-18, 23-24).  Receiver and occluder data are exchanged through shared memory
// (one float4 slot per lane and quantity, groups padded apart).
//
//  k_frame_group      one CTA per 16 x 8 tile; AO rays start at the warp's start node.
//  k_frame_group_dyn  AO, persistent: a warp refills whole groups from a global counter
//                     once at least OCC_FRAME_DYN_MIN_IDLE lanes belong to finished
//                     groups, and runs the estimate of those groups just before.
//
// The estimate always uses the FP32 occluders held on chip; a record buffer, when given,
// receives a copy of step 1 in its own format.
#include <cuda_runtime.h>

#include <atomic>

#include "occ_device.cuh"
#include "occ_kernels.h"
#include "occ_path.cuh"

#ifndef OCC_TRACE_MIN_BLOCKS
#define OCC_TRACE_MIN_BLOCKS 8
#endif
// Persistent AO path: refill once at least this many lanes belong to finished groups.
#ifndef OCC_FRAME_DYN_MIN_IDLE
#define OCC_FRAME_DYN_MIN_IDLE 24
#endif

namespace occ {
namespace {

struct FrameArgs {
    GBufView gb;
    DevBVH bvh;
    float radius;       // AO
    float R2s;          // AO: R^2 (1 + 2^-16)
    LightParams lp;     // shadow
    uint64_t seed;
    uint32_t sample;
    int32_t est;        // kNoReuse, kBiased, kUnbiased, kBoxMean
    RecView rec;        // r0 == nullptr: step-1 records are not stored
    float* out;
    unsigned* status;
};

// Pixel of lane `lane` in the 8 x 4 sub-tile at (x0, y0).
template <int GW, int GH>
__device__ __forceinline__ void group_pixel(int lane, int x0, int y0, int* x, int* y) {
    constexpr int K = GW * GH, GX = 8 / GW;
    const int g = lane / K, m = lane % K;
    *x = x0 + (g % GX) * GW + m % GW;
    *y = y0 + (g / GX) * GH + m / GW;
}

// Per-lane slots of a CTA: receiver (x, valid), receiver terms of the density, occluder
// (z, triangle id bits, -1 = none), occluder normal.  A group's slots are K + 1 float4
// apart (odd), so the groups of a warp reading their k-th member hit distinct banks.
template <int K>
struct FrameSmem {
    static constexpr int kWarpSlots = 32 + 32 / K;
    float4 x[4 * kWarpSlots], n[4 * kWarpSlots], z[4 * kWarpSlots], nz[4 * kWarpSlots];
    __device__ static int base(int warp) { return warp * kWarpSlots; }
    __device__ static int slot(int warp, int lane) { return warp * kWarpSlots + lane + lane / K; }
};

template <int EFFECT, typename Smem>
__device__ __forceinline__ void put_receiver(Smem& s, int slot, float3 x, float3 n, bool valid,
                                             const RectLight& L) {
    const Recv r = make_recv<EFFECT>(x, n, valid, L);
    s.x[slot] = make_float4(x.x, x.y, x.z, valid ? 1.0f : 0.0f);
    s.n[slot] = make_float4(r.n.x, r.n.y, r.n.z, 0.0f);
    s.z[slot] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
}

// Occluder of the finished ray of `t` (or none) into the lane's slot, and the optional
// record copy.
template <typename Smem>
__device__ __forceinline__ void put_occluder(Smem& s, int slot, const FrameArgs& a, uint32_t p,
                                             float3 o, float3 d, float tbest, uint32_t id,
                                             uint32_t hit_slot) {
    if (id == kNoHit) {
        if (a.rec.r0) write_record(a.rec, p, o, o, o, 0.0f, -1);
        return;
    }
    const float3 nz = hit_normal(a.bvh, hit_slot, d);
    const float3 z = make_float3(fmaf(tbest, d.x, o.x), fmaf(tbest, d.y, o.y), fmaf(tbest, d.z, o.z));
    s.z[slot] = make_float4(z.x, z.y, z.z, __int_as_float((int)id));
    s.nz[slot] = make_float4(nz.x, nz.y, nz.z, 0.0f);
    if (a.rec.r0) write_record(a.rec, p, o, z, nz, tbest, (int)id);
}

// Estimate of every lane from the warp's slots (warp-collective: all 32 lanes call it
// together).  Invalid receivers get 1.
template <int EFFECT, int GW, int GH, bool UNB>
__device__ __forceinline__ float group_estimate(const FrameArgs& a, const RectLight& L,
                                                const FrameSmem<GW * GH>& s, int warp, int lane) {
    constexpr int K = GW * GH;
    const int g = lane / K, m = lane % K;
    const int me = FrameSmem<K>::slot(warp, lane), gb = FrameSmem<K>::base(warp) + g * (K + 1);
    const float4 X = s.x[me], Z = s.z[me];
    const int tri = __float_as_int(Z.w);
    const bool valid = X.w != 0.0f;
    const bool hit = valid && tri >= 0;
    const unsigned gmask = (K == 32 ? 0xFFFFFFFFu : ((1u << K) - 1u)) << (g * K);
    const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid) & gmask;
    const unsigned hmask = __ballot_sync(0xFFFFFFFFu, hit) & gmask;
    if (a.est == kNoReuse) return hit ? 0.0f : 1.0f;
    if (a.est == kBoxMean)
        return valid ? (float)__popc(vmask & ~hmask) / (float)__popc(vmask) : 1.0f;

    const float3 z = f3(Z), nz = f3(s.nz[me]);
    float r[K];
    float Psum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 sx = s.x[gb + k];
        Recv rk;
        rk.x = f3(sx);
        rk.n = f3(s.n[gb + k]);
        float q = 0.0f;
        if (hit && sx.w != 0.0f) q = density<EFFECT>(z, nz, rk, a.R2s, L);
        if (UNB && q > 0.0f && k != m)
            if (!first_hit(a.bvh, rk.x, z, (uint32_t)tri, a.status)) q = 0.0f;
        r[k] = q;
        Psum += q;
    }
    const float inv = Psum > 0.0f ? 1.0f / Psum : 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) r[k] *= inv;
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
    if (!valid) return 1.0f;
    if (EFFECT == kShadow && !UNB && vmask == hmask) return 0.0f;   // all-blocked guard
    return 1.0f - r[0];
}

template <int EFFECT, int GW, int GH, bool UNB>
__global__ void __launch_bounds__(128, OCC_TRACE_MIN_BLOCKS) k_frame_group(FrameArgs a) {
    __shared__ FrameSmem<GW * GH> s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int me = FrameSmem<GW * GH>::slot(warp, lane);
    int x, y;
    group_pixel<GW, GH>(lane, blockIdx.x * 16 + (warp & 1) * 8, blockIdx.y * 8 + (warp >> 1) * 4, &x,
                        &y);
    const bool inside = x < a.gb.W && y < a.gb.H;
    const uint32_t p = inside ? (uint32_t)y * (uint32_t)a.gb.W + (uint32_t)x : 0u;
    float3 xo = make_float3(0.0f, 0.0f, 0.0f), n = xo;
    const bool valid = inside && gb_fetch(a.gb, (int)p, &xo, &n);
    RectLight L;
    if (EFFECT == kShadow) L = make_light(a.lp);
    // AO segments are short: start below the part of the tree they cannot leave
    const uint32_t start = EFFECT == kAO ? warp_start_node(a.bvh, valid, xo, a.radius) : 0u;
    put_receiver<EFFECT>(s, me, xo, n, valid, L);
    if (valid) {
        float tmax;
        const float3 d = step1_ray<EFFECT>(xo, n, p, a.radius, L, a.seed, a.sample, &tmax);
        const Hit h = closest_hit(a.bvh, xo, d, tmax, a.status, start);
        put_occluder(s, me, a, p, xo, d, h.t, h.id, h.slot);
    } else if (inside && a.rec.r0) {
        write_record(a.rec, p, xo, xo, xo, 0.0f, -1);
    }
    __syncwarp();
    const float res = group_estimate<EFFECT, GW, GH, UNB>(a, L, s, warp, lane);
    if (inside) a.out[p] = res;
}

template <int GW, int GH>
__global__ void __launch_bounds__(128, OCC_TRACE_MIN_BLOCKS)
    k_frame_group_dyn(FrameArgs a, unsigned* counter, int tiles_x, uint32_t n_groups) {
    constexpr int K = GW * GH, GPW = 32 / K;
    __shared__ FrameSmem<K> s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int me = FrameSmem<K>::slot(warp, lane);
    const int g = lane / K;
    const unsigned gmask = (K == 32 ? 0xFFFFFFFFu : ((1u << K) - 1u)) << (g * K);
    const unsigned gbelow = (1u << (g * K)) - 1u;
    const RectLight L{};
    Traversal t;
    StackEntry stack[kStackSize];
    trav_clear(t);
    t.overflow = false;
    t.bad = false;
    bool active = false, tracing = false, exhausted = false, overflow = false, bad = false;
    int p = -1;   // the lane's pixel (-1: outside the image)
    for (;;) {
        const unsigned busy = __ballot_sync(0xFFFFFFFFu, tracing);
        const bool done = active && (busy & gmask) == 0;
        const unsigned dmask = __ballot_sync(0xFFFFFFFFu, done);
        const unsigned idle = ~__ballot_sync(0xFFFFFFFFu, active) | dmask;
        const bool refill = !exhausted && (busy == 0 || __popc(idle) >= OCC_FRAME_DYN_MIN_IDLE);
        if (dmask && (refill || busy == 0)) {
            // estimates of the finished groups (slots written by their own lanes)
            __syncwarp();
            const float res = group_estimate<kAO, GW, GH, false>(a, L, s, warp, lane);
            if (done) {
                if (p >= 0) a.out[p] = res;
                active = false;
            }
            __syncwarp();
        }
        if (refill) {
            const unsigned fr = __ballot_sync(0xFFFFFFFFu, !active);
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(counter, (unsigned)(__popc(fr) / K));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (base >= n_groups) exhausted = true;
            if (!active && base < n_groups) {
                const uint32_t gi = base + (uint32_t)(__popc(fr & gbelow) / K);
                if (gi < n_groups) {
                    active = true;
                    const uint32_t sub = gi / GPW, within = gi % GPW;
                    const uint32_t tile = sub >> 2, w = sub & 3u;
                    int x, y;
                    group_pixel<GW, GH>((int)within * K + lane % K,
                                        (int)(tile % (uint32_t)tiles_x) * 16 + (int)(w & 1u) * 8,
                                        (int)(tile / (uint32_t)tiles_x) * 8 + (int)(w >> 1) * 4, &x,
                                        &y);
                    const bool inside = x < a.gb.W && y < a.gb.H;
                    p = inside ? y * a.gb.W + x : -1;
                    float3 xo = make_float3(0.0f, 0.0f, 0.0f), n = xo;
                    const bool valid = inside && gb_fetch(a.gb, p, &xo, &n);
                    put_receiver<kAO>(s, me, xo, n, valid, L);
                    if (valid) {
                        float tmax;
                        const float3 d = step1_ray<kAO>(xo, n, (uint32_t)p, a.radius, L, a.seed,
                                                        a.sample, &tmax);
                        trav_init(t, xo, d, tmax, 0u);
                        tracing = true;
                    } else if (inside && a.rec.r0) {
                        write_record(a.rec, (uint32_t)p, xo, xo, xo, 0.0f, -1);
                    }
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, active)) {
            if (exhausted) break;
            continue;
        }
        if (tracing) {
            trav_round(t, a.bvh, stack);
            if (trav_done(t)) {
                tracing = false;
                overflow |= t.overflow;
                bad |= t.bad;
                put_occluder(s, me, a, (uint32_t)p, t.r.o, t.r.d, t.tbest, t.best_id, t.best_slot);
            }
        }
    }
    if (overflow && a.status) atomicOr(a.status, kStatusStackOverflowBit);
    if (OCC_CHECKS && bad && a.status) atomicOr(a.status, kStatusBadIndexBit);
}

int sms() {
    int dev = 0, n = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

template <int EFFECT, int GW, int GH>
cudaError_t launch_shape(const FrameArgs& a, int mode, unsigned* counter, cudaStream_t s) {
    const unsigned tx = (unsigned)((a.gb.W + 15) / 16), ty = (unsigned)((a.gb.H + 7) / 8);
    if (EFFECT == kAO && mode == 2 && a.est != kUnbiased && counter) {
        constexpr int K = GW * GH;
        // persistent grid: resident CTAs per SM x SMs (computed once; threads that race
        // here compute the same value)
        static std::atomic<int> cached{0};
        int ctas = cached.load(std::memory_order_relaxed);
        if (!ctas) {
            int per_sm = 1;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_frame_group_dyn<GW, GH>, 128,
                                                              0) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            ctas = per_sm * sms();
            cached.store(ctas, std::memory_order_relaxed);
        }
        const uint32_t n_groups = tx * ty * 4u * (uint32_t)(32 / K);
        const unsigned blocks = (unsigned)ctas < tx * ty ? (unsigned)ctas : tx * ty;
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        k_frame_group_dyn<GW, GH><<<blocks, 128, 0, s>>>(a, counter, (int)tx, n_groups);
        return cudaGetLastError();
    }
    const dim3 grid(tx, ty);
    if (a.est == kUnbiased)
        k_frame_group<EFFECT, GW, GH, true><<<grid, 128, 0, s>>>(a);
    else
        k_frame_group<EFFECT, GW, GH, false><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

template <int EFFECT>
cudaError_t launch_effect(const FrameArgs& a, int gw, int gh, int mode, unsigned* counter,
                          cudaStream_t s) {
    if (gw == 2 && gh == 1) return launch_shape<EFFECT, 2, 1>(a, mode, counter, s);
    if (gw == 2 && gh == 2) return launch_shape<EFFECT, 2, 2>(a, mode, counter, s);
    if (gw == 4 && gh == 2) return launch_shape<EFFECT, 4, 2>(a, mode, counter, s);
    if (gw == 4 && gh == 4) return launch_shape<EFFECT, 4, 4>(a, mode, counter, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool frame_group_shape(int gw, int gh) {
    return (gw == 2 && gh == 1) || (gw == 2 && gh == 2) || (gw == 4 && gh == 2) || (gw == 4 && gh == 4);
}

cudaError_t launch_trace_reuse(int effect, int estimator, const GBufView& gb, const DevBVH& bvh,
                               float radius, const LightParams& light, uint64_t seed,
                               uint32_t sample, int gw, int gh, RecView rec, float* out,
                               unsigned* status, cudaStream_t s, unsigned* counter, int mode) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    FrameArgs a;
    a.gb = gb;
    a.bvh = bvh;
    a.radius = radius;
    a.R2s = (float)((double)radius * (double)radius * (1.0 + 1.0 / 65536.0));
    a.lp = light;
    a.seed = seed;
    a.sample = sample;
    a.est = estimator;
    a.rec = rec;
    a.out = out;
    a.status = status;
    return effect == kAO ? launch_effect<kAO>(a, gw, gh, mode == 0 ? 2 : mode, counter, s)
                         : launch_effect<kShadow>(a, gw, gh, 1, counter, s);
}

}  // namespace occ
