// kernels_reuse.cu -- steps 2-3 of Algorithms 1 and 2: occluder-domain reuse with
// balance-heuristic MIS (Eqs. 10-12) for AO (Eqs. 15, 17, 18) and area-light shadows
// (Eqs. 20, 21, 23, 24), plus the no-reuse and box-mean baselines.
//
// Densities are evaluated in FP32 without the constant factors 1/pi and 1/Area,
// which cancel in every ratio p(z_j|x_i) / sum_k p(z_j|x_k).
//
//  k_reuse_group    GROUP patterns with power-of-two blocks (the paper's shared
//                   groups mapped onto warp lanes).  Lane j owns candidate z_j and
//                   evaluates its column p(z_j|x_k) for all K receivers (receiver data
//                   exchanged through shared memory), normalises by P_j, and a
//                   recursive-halving shuffle reduce-scatter (K-1 shuffles) hands lane
//                   i its B_i = sum_j p(z_j|x_i)/P_j.
//  k_reuse_tile     (kernels_reuse_tile.cu) biased box / offset windows with the tile
//                   and its halo staged in shared memory by TMA.
//  k_reuse_generic  any pattern: one thread per receiver, members' receiver data held
//                   in registers, K^2 pair densities (unbiased windows, odd groups).
//  k_reuse_simple   NOREUSE / BOXMEAN.
#include <cuda_runtime.h>

#include "occ_device.cuh"
#include "occ_kernels.h"
#include "occ_path.cuh"

namespace occ {
namespace {

struct ReuseArgs {
    GBufView gb;
    RecView rec;
    PatternParams pat;
    float R2s;          // AO: R^2 (1 + 2^-16)
    LightParams lp;
    DevBVH bvh;         // unbiased only
    float* out;
    unsigned* status;
};

// Receiver data of pixel q, from either G-buffer format.
template <int EFFECT>
__device__ __forceinline__ Recv fetch_recv(const GBufView& gb, int q, const RectLight& L) {
    float3 x = make_float3(0.0f, 0.0f, 0.0f), n = x;
    const bool v = gb_fetch(gb.pos, gb.nrm, gb.packed != 0, q, &x, &n);
    return make_recv<EFFECT>(x, n, v, L);
}

// Candidate of pixel q whose own receiver point is xsrc: occluder point and normal; returns
// the triangle id (< 0: no occluder).  Either record format.
__device__ __forceinline__ int fetch_cand(const RecView& rec, int q, float3 xsrc, float3* z,
                                          float3* nz) {
    const float4 r0 = __ldg(rec.r0 + q);
    const int tri = __float_as_int(r0.w);
    if (tri < 0) return tri;
    if (rec.packed) return rec_unpack(r0, xsrc, z, nz);
    *z = f3(r0);
    *nz = f3(__ldg(rec.r1 + q));
    return tri;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n;
}

__device__ __forceinline__ void tile_pixel(int* x, int* y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    *x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    *y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
}

// Members of N_i in a fixed order (the receiver's own slot returned in *self).
// GROUP: row-major over the block; BOX: row-major over the window; OFFSETS: the
// receiver, then each offset.  Out-of-image and invalid pixels are dropped.
template <int MAXK>
__device__ __forceinline__ int gather_members(const PatternParams& pat, const GBufView& gb, int x,
                                              int y, int* mem, int* self) {
    int n = 0;
    *self = 0;
    for (int a = 0; a < pat.K; ++a) {
        int px, py;
        if (pat.kind == 0) {
            px = (x / pat.gw) * pat.gw + a % pat.gw;
            py = (y / pat.gh) * pat.gh + a / pat.gw;
        } else if (pat.kind == 1) {
            px = x - (pat.gw - 1) / 2 + a % pat.gw;
            py = y - (pat.gh - 1) / 2 + a / pat.gw;
        } else {
            px = x + (a == 0 ? 0 : pat.off[a - 1].x);
            py = y + (a == 0 ? 0 : pat.off[a - 1].y);
        }
        if (px < 0 || py < 0 || px >= gb.W || py >= gb.H) continue;
        const int q = py * gb.W + px;
        if (!gb_valid(gb.pos, gb.packed != 0, q)) continue;
        if (px == x && py == y) *self = n;
        if (n < MAXK) mem[n++] = q;
    }
    return n;
}

// ---------------------------------------------------------------------------------------
// Generic per-receiver kernel (any pattern).
// ---------------------------------------------------------------------------------------
template <int EFFECT, int EST, int MAXK>
__device__ __forceinline__ void reuse_pixel(const ReuseArgs& a, int x, int y) {
    if (x >= a.gb.W || y >= a.gb.H) return;
    const int i = y * a.gb.W + x;
    if (!gb_valid(a.gb.pos, a.gb.packed != 0, i)) {
        a.out[i] = 1.0f;
        return;
    }
    RectLight L;
    if (EFFECT == kShadow) L = make_light(a.lp);
    int mem[MAXK];
    int self;
    const int n = gather_members<MAXK>(a.pat, a.gb, x, y, mem, &self);
    // the receiver first, then the other members in pattern order
#pragma unroll
    for (int b = MAXK - 1; b >= 1; --b)
        if (b <= self) mem[b] = mem[b - 1];
    mem[0] = i;
    // up to 16 slots every slot is evaluated: unused ones carry zero receiver terms, whose
    // densities are 0 (AO: n_x.d = 0; shadow: s_L = 0); larger sets test the member count
    constexpr bool kPadded = MAXK <= 16;
    Recv rk[MAXK];
#pragma unroll
    for (int b = 0; b < MAXK; ++b) {
        if (b < n) {
            rk[b] = fetch_recv<EFFECT>(a.gb, mem[b], L);
        } else {
            rk[b].x = make_float3(0.0f, 0.0f, 0.0f);
            rk[b].n = rk[b].x;
            rk[b].valid = false;
        }
    }
    float B = 0.0f;
    int blocked = 0;
#pragma unroll 1
    for (int c = 0; c < n; ++c) {
        float3 z, nz;
        const int tri = fetch_cand(a.rec, mem[c], f3(__ldg(a.gb.pos + mem[c])), &z, &nz);
        if (tri < 0) continue;
        ++blocked;
        float Psum = 0.0f, pi = 0.0f;
#pragma unroll
        for (int b = 0; b < MAXK; ++b) {
            if (kPadded || b < n) {
                float q = density<EFFECT>(z, nz, rk[b], a.R2s, L);
                if (EST == kUnbiased && q > 0.0f && b != c)
                    if (!first_hit(a.bvh, rk[b].x, z, (uint32_t)tri, a.status)) q = 0.0f;
                Psum += q;
                if (b == 0) pi = q;
            }
        }
        if (pi > 0.0f) B += pi / Psum;
    }
    float res = 1.0f - B;
    if (EFFECT == kShadow && EST == kBiased && blocked == n) res = 0.0f;
    a.out[i] = res;
}

template <int EFFECT, int EST, int MAXK>
__global__ void __launch_bounds__(128) k_reuse_generic(ReuseArgs a) {
    int x, y;
    tile_pixel(&x, &y);
    reuse_pixel<EFFECT, EST, MAXK>(a, x, y);
}

// ---------------------------------------------------------------------------------------
// NOREUSE (Eq. 3 / Eq. 6 with one sample) and BOXMEAN (mean visibility over N_i).
// ---------------------------------------------------------------------------------------
template <int EST>
__device__ __forceinline__ void reuse_simple_pixel(const ReuseArgs& a, int x, int y) {
    if (x >= a.gb.W || y >= a.gb.H) return;
    const int i = y * a.gb.W + x;
    if (!gb_valid(a.gb.pos, a.gb.packed != 0, i)) {
        a.out[i] = 1.0f;
        return;
    }
    if (EST == kNoReuse) {
        a.out[i] = __float_as_int(__ldg(&a.rec.r0[i].w)) < 0 ? 1.0f : 0.0f;
        return;
    }
    int mem[kMaxMembers];
    int self;
    const int n = gather_members<kMaxMembers>(a.pat, a.gb, x, y, mem, &self);
    int vis = 0;
    for (int c = 0; c < n; ++c) vis += __float_as_int(__ldg(&a.rec.r0[mem[c]].w)) < 0 ? 1 : 0;
    a.out[i] = (float)vis / (float)n;
}

template <int EST>
__global__ void __launch_bounds__(128) k_reuse_simple(ReuseArgs a) {
    int x, y;
    tile_pixel(&x, &y);
    reuse_simple_pixel<EST>(a, x, y);
}

// ---------------------------------------------------------------------------------------
// Unbiased light-sample reuse for shadows (Light(N U), Sec. 6.2): receiver i traces a
// segment to every member j's light sample y_j (Eq. 5 with j's random numbers) and
// averages the visibility.  For j = i the segment is i's own step-1 ray (same arithmetic
// as the trace), so N_i = {i} reproduces no reuse.
// ---------------------------------------------------------------------------------------
template <int MAXK>
__global__ void __launch_bounds__(128) k_reuse_light(ReuseArgs a, uint64_t seed, uint32_t sample) {
    int x, y;
    tile_pixel(&x, &y);
    if (x >= a.gb.W || y >= a.gb.H) return;
    const int i = y * a.gb.W + x;
    if (!gb_valid(a.gb.pos, a.gb.packed != 0, i)) {
        a.out[i] = 1.0f;
        return;
    }
    const RectLight L = make_light(a.lp);
    int mem[MAXK];
    int self;
    const int n = gather_members<MAXK>(a.pat, a.gb, x, y, mem, &self);
    const float3 xi = f3(__ldg(a.gb.pos + i));
    int vis = 0;
    for (int c = 0; c < n; ++c) {
        float tmax;
        const float3 d = light_direction(L, xi, uniform_pair(seed, (uint32_t)mem[c], sample, kStreamShadow),
                                         &tmax);
        if (!any_hit(a.bvh, xi, d, tmax, a.status)) ++vis;
    }
    a.out[i] = (float)vis / (float)n;
}

// ---------------------------------------------------------------------------------------
// Batched reuse over views of different sizes, patterns, effects and estimators: the
// persistent counterpart of k_trace_batch (same tile space and view lookup); each tile
// runs the per-receiver evaluation of its view.
// ---------------------------------------------------------------------------------------
template <int MAXK>
__global__ void __launch_bounds__(128) k_reuse_batch(const BatchView* views, int n_views,
                                                     int n_tiles, DevBVH bvh, unsigned* status) {
    __shared__ int s_first[kMaxBatchViews + 1];
    for (int v = threadIdx.x; v <= n_views; v += blockDim.x)
        s_first[v] = v < n_views ? views[v].first_tile : n_tiles;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int lo = 0, hi = n_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        const BatchView* v = views + lo;
        const int t = tile - s_first[lo];
        const int x = (t % v->tiles_x) * 16 + (warp & 1) * 8 + (lane & 7);
        const int y = (t / v->tiles_x) * 8 + (warp >> 1) * 4 + (lane >> 3);
        ReuseArgs a;
        a.gb = v->gb;
        a.rec = v->rec;
        a.pat = v->pat;
        a.R2s = v->R2s;
        a.lp = v->light;
        a.bvh = bvh;
        a.out = v->out;
        a.status = status;
        const int est = v->estimator;
        if (est == kNoReuse) reuse_simple_pixel<kNoReuse>(a, x, y);
        else if (est == kBoxMean) reuse_simple_pixel<kBoxMean>(a, x, y);
        else if (v->effect == kAO) {
            if (est == kBiased) reuse_pixel<kAO, kBiased, MAXK>(a, x, y);
            else reuse_pixel<kAO, kUnbiased, MAXK>(a, x, y);
        } else {
            if (est == kBiased) reuse_pixel<kShadow, kBiased, MAXK>(a, x, y);
            else reuse_pixel<kShadow, kUnbiased, MAXK>(a, x, y);
        }
    }
}

// ---------------------------------------------------------------------------------------
// MIS weights of selected receivers (debug / tests): w[a][b] = p(z_a|x_b) / P_a.
// ---------------------------------------------------------------------------------------
template <int EFFECT, int EST>
__global__ void k_debug_mis(ReuseArgs a, const int32_t* pix, int32_t npix, int32_t* members,
                            float* w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npix) return;
    const int i = pix[t];
    const int x = i % a.gb.W, y = i / a.gb.W;
    RectLight L;
    if (EFFECT == kShadow) L = make_light(a.lp);
    int mem[kMaxMembers];
    int self;
    int n = 0;
    if (gb_valid(a.gb.pos, a.gb.packed != 0, i))
        n = gather_members<kMaxMembers>(a.pat, a.gb, x, y, mem, &self);
    for (int c = 0; c < kMaxMembers; ++c) members[t * kMaxMembers + c] = c < n ? mem[c] : -1;
    float* wt = w + (size_t)t * kMaxMembers * kMaxMembers;
    for (int c = 0; c < n; ++c) {
        float3 z, nz;
        const int tri = fetch_cand(a.rec, mem[c], fetch_recv<EFFECT>(a.gb, mem[c], L).x, &z, &nz);
        float Psum = 0.0f;
        for (int b = 0; b < n; ++b) {
            float q = 0.0f;
            if (tri >= 0) {
                const Recv rk = fetch_recv<EFFECT>(a.gb, mem[b], L);
                q = density<EFFECT>(z, nz, rk, a.R2s, L);
                if (EST == kUnbiased && q > 0.0f && b != c)
                    if (!first_hit(a.bvh, rk.x, z, (uint32_t)tri, a.status)) q = 0.0f;
            }
            wt[c * kMaxMembers + b] = q;
            Psum += q;
        }
        for (int b = 0; b < n; ++b)
            wt[c * kMaxMembers + b] = Psum > 0.0f ? wt[c * kMaxMembers + b] / Psum : 0.0f;
    }
}

// ---------------------------------------------------------------------------------------
// Warp-cooperative GROUP kernel.  K = GW * GH lanes per group, 32 / K groups per warp
// laid side by side (warp block = (32/K * GW) x GH pixels), 8 warps side by side per CTA.
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
#ifndef OCC_GROUP_WARPS
#define OCC_GROUP_WARPS 8
#endif
#ifndef OCC_GROUP_STREAM_LOADS
#define OCC_GROUP_STREAM_LOADS 0
#endif
template <typename T>
__device__ __forceinline__ T group_load(const T* p) {
    if (OCC_GROUP_STREAM_LOADS) return __ldcs(p);
    return __ldg(p);
}

template <int EFFECT, int EST, int GW, int GH, bool PACKED>
__global__ void __launch_bounds__(32 * OCC_GROUP_WARPS) k_reuse_group(ReuseArgs a) {
    constexpr int K = GW * GH;
    constexpr int GPW = 32 / K;
    constexpr int BW = GPW * GW;
    // receiver exchange buffer; group slots are K + 2 float4 apart so that the groups of a
    // warp reading their k-th member hit different shared-memory banks
    constexpr int GS = K + 2;
    __shared__ float4 s_x[OCC_GROUP_WARPS][GPW * GS];
    __shared__ float4 s_n[OCC_GROUP_WARPS][GPW * GS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / K, m = lane % K;
    // the CTA's warps sit side by side: each row of the CTA is contiguous pixels
    const int x = (blockIdx.x * OCC_GROUP_WARPS + warp) * BW + g * GW + m % GW;
    const int y = blockIdx.y * GH + m / GW;
    const bool inside = x < a.gb.W && y < a.gb.H;
    const int i = inside ? y * a.gb.W + x : 0;
    RectLight L;
    if (EFFECT == kShadow) L = make_light(a.lp);

    float4 P = make_float4(0.0f, 0.0f, 0.0f, 0.0f), N = P;
    float4 R0 = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1)), R1 = P;
    float3 z = make_float3(0.0f, 0.0f, 0.0f), nz = z, nx = z;
    bool valid, hit;
    if (PACKED) {
        // 16 + 16 bytes per pixel: (x, octahedral normal) and the packed record
        if (inside) {
            P = group_load(a.gb.pos + i);
            R0 = group_load(a.rec.r0 + i);
        }
        valid = inside && __float_as_uint(P.w) != kOctInvalid;
        hit = valid && __float_as_int(R0.w) >= 0;
        if (valid) nx = oct_decode(__float_as_uint(P.w));
        if (hit) rec_unpack(R0, f3(P), &z, &nz);
    } else {
        if (inside) {
            P = group_load(a.gb.pos + i);
            N = group_load(a.gb.nrm + i);
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
    s_x[warp][g * GS + m] = make_float4(me.x.x, me.x.y, me.x.z, valid ? 1.0f : 0.0f);
    s_n[warp][g * GS + m] = make_float4(me.n.x, me.n.y, me.n.z, 0.0f);
    __syncwarp();

    const unsigned gmask = (K == 32 ? 0xFFFFFFFFu : ((1u << K) - 1u)) << (g * K);
    const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid) & gmask;
    const unsigned hmask = __ballot_sync(0xFFFFFFFFu, hit) & gmask;

    // column of candidate z_m: densities at every receiver of the group
    float r[K];
    float Psum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float4 sx = s_x[warp][g * GS + k];
        const float4 sn = s_n[warp][g * GS + k];
        Recv rk;
        rk.x = f3(sx);
        rk.n = f3(sn);
        float q = 0.0f;
        if (hit && sx.w != 0.0f) q = density<EFFECT>(z, nz, rk, a.R2s, L);
        if (EST == kUnbiased && q > 0.0f && k != m)
            if (!first_hit(a.bvh, rk.x, z, (uint32_t)__float_as_int(R0.w), a.status)) q = 0.0f;
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
    if (!inside) return;
    float res = 1.0f;
    if (valid) {
        res = 1.0f - r[0];
        if (EFFECT == kShadow && EST == kBiased && vmask == hmask) res = 0.0f;
    }
    a.out[i] = res;
}

template <int EFFECT, int EST, int GW, int GH>
void launch_group_t(const ReuseArgs& a, cudaStream_t s) {
    constexpr int K = GW * GH;
    constexpr int BW = (32 / K) * GW;
    constexpr int CW = OCC_GROUP_WARPS * BW;
    const dim3 grid((unsigned)((a.gb.W + CW - 1) / CW), (unsigned)((a.gb.H + GH - 1) / GH));
    if (a.gb.packed && a.rec.packed)
        k_reuse_group<EFFECT, EST, GW, GH, true><<<grid, 32 * OCC_GROUP_WARPS, 0, s>>>(a);
    else if (!a.gb.packed && !a.rec.packed)
        k_reuse_group<EFFECT, EST, GW, GH, false><<<grid, 32 * OCC_GROUP_WARPS, 0, s>>>(a);
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

template <int EFFECT, int EST>
void launch_generic(const ReuseArgs& a, cudaStream_t s) {
    const dim3 grid((unsigned)((a.gb.W + 15) / 16), (unsigned)((a.gb.H + 7) / 8));
    if constexpr (EST != kUnbiased) {
        if (a.pat.K <= 8) {
            k_reuse_generic<EFFECT, EST, 8><<<grid, 128, 0, s>>>(a);
            return;
        }
    }
    if (a.pat.K <= 9)
        k_reuse_generic<EFFECT, EST, 9><<<grid, 128, 0, s>>>(a);
    else if (a.pat.K <= 16)
        k_reuse_generic<EFFECT, EST, 16><<<grid, 128, 0, s>>>(a);
    else
        k_reuse_generic<EFFECT, EST, kMaxMembers><<<grid, 128, 0, s>>>(a);
}

template <int EFFECT>
cudaError_t launch_effect(int est, const ReuseArgs& a, cudaStream_t s, const Tuning& tune) {
    const dim3 grid((unsigned)((a.gb.W + 15) / 16), (unsigned)((a.gb.H + 7) / 8));
    if (est == kNoReuse) {
        k_reuse_simple<kNoReuse><<<grid, 128, 0, s>>>(a);
    } else if (est == kBoxMean) {
        k_reuse_simple<kBoxMean><<<grid, 128, 0, s>>>(a);
    } else if (est == kBiased) {
        if (a.pat.kind != 0) {
            cudaError_t e = cudaSuccess;
            if (tune.window_path != 2 &&
                launch_reuse_tile(EFFECT, a.gb, a.rec, a.pat, a.R2s, a.lp, a.out, a.status, s, &e,
                                  tune.tile_rows, tune.window_path == 3))
                return e;
            launch_generic<EFFECT, kBiased>(a, s);
        } else if (!launch_group<EFFECT, kBiased>(a, s)) {
            launch_generic<EFFECT, kBiased>(a, s);
        }
    } else {
        if (a.pat.kind != 0 || !launch_group<EFFECT, kUnbiased>(a, s)) launch_generic<EFFECT, kUnbiased>(a, s);
    }
    return cudaSuccess;
}

ReuseArgs make_args(const GBufView& gb, const RecView& rec, const PatternParams& pat, float radius,
                    const LightParams& light, const DevBVH* bvh, float* out, unsigned* status) {
    ReuseArgs a;
    a.gb = gb;
    a.rec = rec;
    a.pat = pat;
    a.R2s = (float)((double)radius * (double)radius * (1.0 + 1.0 / 65536.0));
    a.lp = light;
    a.bvh = bvh ? *bvh : DevBVH{nullptr, nullptr};
    a.out = out;
    a.status = status;
    return a;
}

}  // namespace

cudaError_t launch_reuse(int effect, int estimator, const GBufView& gb, const RecView& rec,
                         const PatternParams& pat, float radius, const LightParams& light,
                         const DevBVH* bvh, float* out, unsigned* status, cudaStream_t s,
                         const Tuning& tune, uint64_t seed, uint32_t sample) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    const ReuseArgs a = make_args(gb, rec, pat, radius, light, bvh, out, status);
    if (estimator == kLightUnbiased) {
        const dim3 grid((unsigned)((gb.W + 15) / 16), (unsigned)((gb.H + 7) / 8));
        if (pat.K <= 16)
            k_reuse_light<16><<<grid, 128, 0, s>>>(a, seed, sample);
        else
            k_reuse_light<kMaxMembers><<<grid, 128, 0, s>>>(a, seed, sample);
        return cudaGetLastError();
    }
    const cudaError_t e = effect == kAO ? launch_effect<kAO>(estimator, a, s, tune)
                                        : launch_effect<kShadow>(estimator, a, s, tune);
    const cudaError_t l = cudaGetLastError();
    return e != cudaSuccess ? e : l;
}

cudaError_t launch_reuse_batch(const BatchView* views, int n_views, int n_tiles, int max_k,
                               const DevBVH& bvh, int per_sm_wanted, unsigned* status,
                               cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    auto k = max_k <= 9 ? k_reuse_batch<9> : k_reuse_batch<16>;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm_wanted > 0 && per_sm_wanted < per_sm) per_sm = per_sm_wanted;
    const int ctas = per_sm * sm_count();
    k<<<ctas < n_tiles ? ctas : n_tiles, 128, 0, s>>>(views, n_views, n_tiles, bvh, status);
    return cudaGetLastError();
}

cudaError_t launch_debug_mis(int effect, int estimator, const GBufView& gb, const RecView& rec,
                             const PatternParams& pat, float radius, const LightParams& light,
                             const DevBVH* bvh, const int32_t* pix, int32_t n, int32_t* members,
                             float* w, unsigned* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const ReuseArgs a = make_args(gb, rec, pat, radius, light, bvh, nullptr, status);
    const unsigned blocks = (unsigned)((n + 63) / 64);
    const bool unb = estimator == kUnbiased;
    if (effect == kAO) {
        if (unb) k_debug_mis<kAO, kUnbiased><<<blocks, 64, 0, s>>>(a, pix, n, members, w);
        else k_debug_mis<kAO, kBiased><<<blocks, 64, 0, s>>>(a, pix, n, members, w);
    } else {
        if (unb) k_debug_mis<kShadow, kUnbiased><<<blocks, 64, 0, s>>>(a, pix, n, members, w);
        else k_debug_mis<kShadow, kBiased><<<blocks, 64, 0, s>>>(a, pix, n, members, w);
    }
    return cudaGetLastError();
}

}  // namespace occ
