// kernels_reuse.cu -- steps 2-3 of Algorithms 1 and 2: occluder-domain reuse with
// balance-heuristic MIS (Eqs. 10-12) for AO (Eqs. 15, 17, 18) and area-light shadows
// (Eqs. 20, 21, 23, 24), plus the no-reuse and box-mean baselines.
//
// Densities are evaluated in FP32 without the constant factors 1/pi and 1/Area,
// which cancel in every ratio p(z_j|x_i) / sum_k p(z_j|x_k).
//
//  k_reuse_group    (kernels_reuse_group.cu) GROUP patterns with power-of-two blocks
//                   (the paper's shared groups mapped onto warp lanes).  Lane j owns
//                   candidate z_j and evaluates its column p(z_j|x_k) for all K receivers
//                   (receiver data exchanged through shared memory), normalises by P_j,
//                   and a recursive-halving shuffle reduce-scatter (K-1 shuffles) hands
//                   lane i its B_i = sum_j p(z_j|x_i)/P_j.  Unbiased: the pairs that need
//                   Eq. 7 are queued and traced by the persistent k_validate.
//  k_reuse_tile     (kernels_reuse_tile.cu) biased box / offset windows with the tile
//                   and its halo staged in shared memory by TMA.
//  k_reuse_generic  any pattern: one thread per receiver, members' receiver data held
//                   in registers, K^2 pair densities (unbiased windows, odd groups).
//  k_reuse_simple   NOREUSE / BOXMEAN.
#include <cuda_runtime.h>

#include "occ_reuse.cuh"

namespace occ {
namespace {

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
    if (pat.kind == 3) {
        // per-receiver random offsets: the receiver, then each drawn offset in slot order
        int2 acc[MAXK];
        int nacc = 0;
        const uint32_t pix = (uint32_t)y * (uint32_t)gb.W + (uint32_t)x;
        mem[n++] = (int)pix;   // reuse_pixel calls this for valid receivers only
        for (int s = 1; s < pat.K && s < MAXK; ++s) {
            int2 o;
            if (!random_offset(pat.seed, pix, pat.sample, s, pat.radius, acc, nacc, &o)) continue;
            acc[nacc++] = o;
            const int px = x + o.x, py = y + o.y;
            if (px < 0 || py < 0 || px >= gb.W || py >= gb.H) continue;
            const int q = py * gb.W + px;
            if (!gb_valid(gb, q)) continue;
            mem[n++] = q;
        }
        return n;
    }
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
        if (!gb_valid(gb, q)) continue;
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
    if (!gb_valid(a.gb, i)) {
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
        const int tri = fetch_cand(a.rec, mem[c], gb_point(a.gb, mem[c]), &z, &nz);
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
    if (!gb_valid(a.gb, i)) {
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
    if (!gb_valid(a.gb, i)) {
        a.out[i] = 1.0f;
        return;
    }
    const RectLight L = make_light(a.lp);
    int mem[MAXK];
    int self;
    const int n = gather_members<MAXK>(a.pat, a.gb, x, y, mem, &self);
    const float3 xi = gb_point(a.gb, i);
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
__global__ void __launch_bounds__(128) k_reuse_batch(const BatchView* views, const BatchDyn* dyn,
                                                     int n_views, int n_tiles, DevBVH bvh,
                                                     unsigned* status) {
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
        a.pat.sample = dyn[lo].sample;   // random patterns draw per sample
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
    if (gb_valid(a.gb, i))
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

// Two threads per receiver in the TMA window kernel: on request (window path 3), and by
// default for AO windows of more than 9 members, where one thread's 16 receivers crowd its
// registers (4K, 16 disk offsets: 1.82 against 2.13 ms FP32, 1.89 against 2.74 ms packed;
// shadows and K <= 9 are faster with one thread per receiver).
bool window_pairs(int effect, int K, const Tuning& tune) {
    if (tune.window_path == 3) return true;
    return tune.window_path == 0 && effect == kAO && K > 9;
}

// Planes the group kernel prefetches into L2 (tuning choice group_prefetch: 1 none, 2 the
// G-buffer and record plane 0, 3 also the hit-normal plane; 0 the built-in default).
#ifndef OCC_GROUP_PREFETCH_DEFAULT
#define OCC_GROUP_PREFETCH_DEFAULT 2
#endif
int group_prefetch_planes(const Tuning& tune) {
    const int c = tune.group_prefetch ? tune.group_prefetch : OCC_GROUP_PREFETCH_DEFAULT;
    return c == 2 ? 3 : c == 3 ? 4 : 0;
}

template <int EFFECT>
cudaError_t launch_effect(int est, const ReuseArgs& a_in, cudaStream_t s, const Tuning& tune) {
    ReuseArgs a = a_in;
    a.pf_planes = group_prefetch_planes(tune);
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
                                  tune.tile_rows, window_pairs(EFFECT, a.pat.K, tune)))
                return e;
            launch_generic<EFFECT, kBiased>(a, s);
        } else if (!launch_group_reuse(EFFECT, kBiased, a, s)) {
            launch_generic<EFFECT, kBiased>(a, s);
        }
    } else if (a.pat.kind == 0 && a.vq && launch_group_reuse(EFFECT, kUnbCollect, a, s)) {
        // queued validation: the pairs that need Eq. 7 are traced by the persistent
        // k_validate, then the group kernel estimates with the validated pairs
        const cudaError_t e = launch_validate(a, s);
        if (e != cudaSuccess) return e;
        launch_group_reuse(EFFECT, kUnbFinal, a, s);
    } else {
        if (a.pat.kind != 0 || !launch_group_reuse(EFFECT, kUnbiased, a, s))
            launch_generic<EFFECT, kUnbiased>(a, s);
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
    a.vq = nullptr;
    a.vcount = nullptr;
    a.vbits = nullptr;
    a.pf_planes = 0;
    a.pf_ahead = 0;
    return a;
}

}  // namespace

cudaError_t launch_reuse(int effect, int estimator, const GBufView& gb, const RecView& rec,
                         const PatternParams& pat, float radius, const LightParams& light,
                         const DevBVH* bvh, float* out, unsigned* status, cudaStream_t s,
                         const Tuning& tune, uint64_t seed, uint32_t sample,
                         const ValidateWs* vws) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    ReuseArgs a = make_args(gb, rec, pat, radius, light, bvh, out, status);
    const size_t P = (size_t)gb.W * gb.H;
    if (estimator == kUnbiased && vws && vws->queue && pat.kind == 0 && pat.K <= 16 &&
        P < (1u << 28) && vws->queue_cap >= (size_t)(pat.K - 1) * P && vws->bits_cap >= P) {
        cudaError_t e = cudaMemsetAsync(vws->bits, 0, P * sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(vws->counters, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        a.vq = vws->queue;
        a.vcount = vws->counters;
        a.vbits = vws->bits;
    }
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

cudaError_t launch_reuse_batch(const BatchView* views, const BatchDyn* dyn, int n_views,
                               int n_tiles, int max_k,
                               const DevBVH& bvh, int per_sm_wanted, unsigned* status,
                               cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    auto k = max_k <= 9 ? k_reuse_batch<9> : k_reuse_batch<16>;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm_wanted > 0 && per_sm_wanted < per_sm) per_sm = per_sm_wanted;
    const int ctas = per_sm * sm_count();
    k<<<ctas < n_tiles ? ctas : n_tiles, 128, 0, s>>>(views, dyn, n_views, n_tiles, bvh, status);
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
