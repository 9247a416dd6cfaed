// kernels_reuse_tile.cu -- biased occluder reuse (Eq. 18 AO / Eq. 24 shadow) for window
// patterns (a centred box or shared offsets), with the receiver tile and the halo its
// neighbour sets reach staged in shared memory by the Tensor Memory Accelerator.  Either
// format: FP32 (G-buffer and record planes, four float4 planes) or packed (two 16-byte
// planes, decoded from shared memory).
//
// Persistent CTAs walk the image in TW x TH receiver tiles.  For each tile a producer warp
// (one thread of the CTA's last warp; OCC_TILE_WS) issues four (FP32) or two (packed) 2D
// bulk-tensor copies (cp.async.bulk.tensor) of the G-buffer and record planes -- (TW +
// halo) x (TH + halo) float4 each, zero-filled outside the image -- into one of two
// buffers, completing on an mbarrier; every receiver thread then evaluates its receiver's
// pair densities from shared memory (K receivers held in registers, each candidate record
// that holds an occluder read once), normalises by P_j = sum_k p(z_j|x_k) and writes
// 1 - B_i, and its warp releases the buffer on a second mbarrier.  Missing members carry
// zero receiver terms, whose densities are 0, so the pair loop has no per-member test.
// Waits on the mbarriers are bounded: on expiry the waiter records kStatusWaitTimeoutBit and
// returns, and the producer waits (again bounded) for its own copies before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "occ_dens_x2.cuh"
#include "occ_device.cuh"
#include "occ_f32x2.cuh"
#include "occ_kernels.h"

namespace occ {
namespace {

constexpr float kSupportSlackT = 1.0f + 1.0f / 65536.0f;

// Windows of 4 or 8 member slots evaluate their density columns on paired FP32 instructions
// and walk each receiver's own list of candidates (OCC_TILE_PAIRED=1; 0 keeps the scalar
// column over every slot).
#ifndef OCC_TILE_PAIRED
#define OCC_TILE_PAIRED 1
#endif
// P_j of the paired column as a pairwise tree of paired adds (1) or a slot-order chain (0)
#ifndef OCC_TILE_TREESUM
#define OCC_TILE_TREESUM 0
#endif
// Two candidate columns per step of the paired loop (1) or one (0; 1080p AO 0.099 against
// 0.103 ms with two)
#ifndef OCC_TILE_CAND2
#define OCC_TILE_CAND2 0
#endif
// MIS weight p_i / P_j with the approximate division __fdividef (1: a few ulp, far inside the
// 1e-5 output tolerance; P_j >= p_i > 0 and P_j < 2^126 here) or the IEEE one (0).
// 1080p, 8 disk offsets: AO 0.097 against 0.099 ms, shadows 0.127 against 0.130 ms.
#ifndef OCC_TILE_FASTDIV
#define OCC_TILE_FASTDIV 1
#endif
__device__ __forceinline__ float tile_ratio(float p, float P) {
#if OCC_TILE_FASTDIV
    return __fdividef(p, P);
#else
    return p / P;
#endif
}
// One extra warp issues the bulk-tensor copies and the receiver warps release each staged
// buffer on an mbarrier (1), instead of thread 0 issuing them between CTA-wide barriers (0):
// a warp whose receivers had fewer candidates starts the next tile without waiting for the
// slowest warp of the CTA (1080p, 8 disk offsets, AO: 0.099 against 0.110 ms).  Two ways of
// also balancing the lanes' candidate lists were measured slower and dropped: the producer
// ordering each landed tile's receivers by candidate count (0.18 ms: the ordering, a warp's
// work, sat on the critical path), and a shared per-tile receiver queue refilling idle lanes
// (0.117 ms: receivers then start in small groups, and setting up a receiver's members costs
// about as much as its ~2 candidate columns).
#ifndef OCC_TILE_WS
#define OCC_TILE_WS 1
#endif
constexpr int kTileW = 32;
constexpr uint32_t kWaitSpins = 1u << 24;

struct TileArgs {
    int W, H;
    int TW, TH;            // receivers per tile
    int hx0, hy0;          // halo left / top
    int SW, SH;            // staged extent (pixels)
    int tiles_x, n_tiles;
    int stages;            // 1, or 2 to prefetch the next tile during this one
    int kind, gw, gh, K;   // pattern (kind 1 box, 2 offsets)
    int2 off[kMaxMembers - 1];
    float R2s;
    LightParams lp;
    float* out;
    unsigned* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_init_count(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for phase `parity` of the barrier.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitSpins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ RectLight tile_light(const LightParams& p) {
    RectLight L;
    L.c = make_float3(p.c[0], p.c[1], p.c[2]);
    L.eu = make_float3(p.eu[0], p.eu[1], p.eu[2]);
    L.ev = make_float3(p.ev[0], p.ev[1], p.ev[2]);
    L.n = normalize3(cross3(L.eu, L.ev));
    L.inv_eu2 = 1.0f / dot3(L.eu, L.eu);
    L.inv_ev2 = 1.0f / dot3(L.ev, L.ev);
    L.lim = 0.5f * kSupportSlackT;
    return L;
}

// Receiver terms: AO (x, n); shadow (x, (n_L.(c - x), (x - c).eu, (x - c).ev)).
template <int EFFECT>
__device__ __forceinline__ void recv_terms(float4 P, float4 N, const RectLight& L, float3* x,
                                           float3* t) {
    *x = f3(P);
    if (EFFECT == kAO) {
        *t = f3(N);
    } else {
        const float3 xc = sub3(*x, L.c);
        *t = make_float3(-dot3(L.n, xc), dot3(xc, L.eu), dot3(xc, L.ev));
    }
}

// Biased pair density without 1/pi or 1/Area (they cancel in every ratio).
template <int EFFECT>
__device__ __forceinline__ float pair_density(float3 z, float3 nz, float3 x, float3 t, float R2s,
                                              const RectLight& L) {
    const float3 d = sub3(z, x);
    if (EFFECT == kAO) {
        const float r2 = dot3(d, d);
        const float a = dot3(t, d);
        const float b = -dot3(nz, d);
        const bool ok = (a > 0.0f) & (b > 0.0f) & (r2 > 0.0f) & (r2 <= R2s);
        return ok ? __fdividef(a * b, r2 * r2) : 0.0f;
    } else {
        const float nd = dot3(L.n, d);
        const float cz = -dot3(nz, d);
        // approximate reciprocal (a few ulp): moves s_L and J far less than the 1e-5 output
        // tolerance; only support tests within that margin of their threshold can flip
        const float inv = __fdividef(1.0f, nd);
        const float sL = t.x * inv;
        // every term evaluated, the support tests combined into one select: the lanes of a
        // warp test different pairs and would diverge at each early exit (1080p, 8 disk
        // offsets: 0.150 against 0.162 ms with early exits)
        const float a = fmaf(sL, dot3(d, L.eu), t.y) * L.inv_eu2;
        const float b = fmaf(sL, dot3(d, L.ev), t.z) * L.inv_ev2;
        const bool ok = (nd < 0.0f) & (cz > 0.0f) & (sL > 1.0f) & !(fabsf(a) > L.lim) &
                        !(fabsf(b) > L.lim);
        return ok ? sL * sL * cz * (-inv) : 0.0f;
    }
}

// Offset of member slot s of a window: slot 0 is the receiver; a box lists its other cells
// row-major, an offsets pattern its offsets in order.
__device__ __forceinline__ int2 member_offset(const TileArgs& a, int s) {
    if (a.kind == 1) {
        const int centre = ((a.gh - 1) / 2) * a.gw + (a.gw - 1) / 2;
        const int cell = s == 0 ? centre : (s <= centre ? s - 1 : s);
        return make_int2(cell % a.gw - (a.gw - 1) / 2, cell / a.gw - (a.gh - 1) / 2);
    }
    return s == 0 ? make_int2(0, 0) : a.off[s - 1];
}

// Members of the receiver at (x, y), staged index sc: bit s set when slot s is inside the
// image and a valid receiver.
// Validity of a staged G-buffer entry: FP32 w = 1 / 0; packed w = octahedral code, with
// one code reserved for background.
template <bool PACKED>
__device__ __forceinline__ bool staged_valid(float4 P) {
    return PACKED ? __float_as_uint(P.w) != kOctInvalid : P.w != 0.0f;
}

template <int MAXK, bool PACKED>
__device__ __forceinline__ uint32_t member_mask(const TileArgs& a, const float4* s_pos, int x,
                                                int y, int sc, int* sidx = nullptr) {
    uint32_t vmask = 0;
#pragma unroll
    for (int s = 0; s < MAXK; ++s) {
        if (sidx) sidx[s] = sc;
        if (s < a.K) {
            const int2 o = member_offset(a, s);
            const int px = x + o.x, py = y + o.y;
            const int q = sc + o.y * a.SW + o.x;
            if (px >= 0 && py >= 0 && px < a.W && py < a.H && staged_valid<PACKED>(s_pos[q])) {
                vmask |= 1u << s;
                if (sidx) sidx[s] = q;
            }
        }
    }
    return vmask;
}

struct Staged {
    const float4 *pos, *nrm, *r0, *r1;   // packed: pos and r0 only
};

// Receiver terms of staged pixel q in either format.
template <int EFFECT, bool PACKED>
__device__ __forceinline__ void staged_recv(const Staged& st, int q, const RectLight& L, float3* x,
                                            float3* t) {
    const float4 P = st.pos[q];
    float4 N;
    if (PACKED) {
        const float3 n = oct_decode(__float_as_uint(P.w));
        N = make_float4(n.x, n.y, n.z, 0.0f);
    } else {
        N = st.nrm[q];
    }
    recv_terms<EFFECT>(P, N, L, x, t);
}

// Candidate of staged pixel q whose record word 0 is r0 (triangle id >= 0): occluder point
// and normal in either format.
template <bool PACKED>
__device__ __forceinline__ void staged_cand(const Staged& st, int q, float4 r0, float3* z, float3* nz) {
    if (PACKED) {
        rec_unpack(r0, f3(st.pos[q]), z, nz);
    } else {
        *z = f3(r0);
        *nz = f3(st.r1[q]);
    }
}

// Receiver terms of the member slots of a receiver as lane pairs (slots 2j, 2j + 1); a slot
// outside vmask carries zero terms (its densities are 0).
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void members_x2(const RectLight& L, const Staged& st, const int* sidx,
                                           uint32_t vmask, f32x2 (&px)[MAXK / 2][3],
                                           f32x2 (&pn)[MAXK / 2][3]) {
#pragma unroll
    for (int j = 0; j < MAXK / 2; ++j) {
        float3 x0r, t0, x1r, t1;
        staged_recv<EFFECT, PACKED>(st, sidx[2 * j], L, &x0r, &t0);
        staged_recv<EFFECT, PACKED>(st, sidx[2 * j + 1], L, &x1r, &t1);
        if (!((vmask >> (2 * j)) & 1u)) t0 = make_float3(0.0f, 0.0f, 0.0f);
        if (!((vmask >> (2 * j + 1)) & 1u)) t1 = make_float3(0.0f, 0.0f, 0.0f);
        px[j][0] = pk2(x0r.x, x1r.x);
        px[j][1] = pk2(x0r.y, x1r.y);
        px[j][2] = pk2(x0r.z, x1r.z);
        pn[j][0] = pk2(t0.x, t1.x);
        pn[j][1] = pk2(t0.y, t1.y);
        pn[j][2] = pk2(t0.z, t1.z);
    }
}

// Member slots of a receiver whose staged record holds an occluder.
template <int MAXK>
__device__ __forceinline__ uint32_t hit_slots(const TileArgs& a, const Staged& st, const int* sidx,
                                              uint32_t vmask) {
    uint32_t hm = 0;
#pragma unroll
    for (int c = 0; c < MAXK; ++c)
        if (c < a.K && ((vmask >> c) & 1u) &&
            __float_as_int(reinterpret_cast<const float*>(st.r0 + sidx[c])[3]) >= 0)
            hm |= 1u << c;
    return hm;
}

// Column of candidate slot c of the receiver at staged index sc on paired instructions: the
// receiver's own density (slot 0) and P_c = sum over the slots.
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void column_x2(const TileArgs& a, const RectLight& L, const Staged& st,
                                          const int* s_qoff, int sc, int c,
                                          const f32x2 (&px)[MAXK / 2][3],
                                          const f32x2 (&pn)[MAXK / 2][3], float* pi_out,
                                          float* psum_out) {
    constexpr int NP = MAXK / 2;
    const int q = sc + s_qoff[c];
    const float4 r0 = st.r0[q];
    float3 z, nz;
    staged_cand<PACKED>(st, q, r0, &z, &nz);
    const f32x2 zx = bc2(z.x), zy = bc2(z.y), zz = bc2(z.z);
    const f32x2 mnx = bc2(-nz.x), mny = bc2(-nz.y), mnz = bc2(-nz.z);
    float2 d[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j)
        d[j] = dens_x2_pairs<EFFECT>(zx, zy, zz, mnx, mny, mnz, px[j][0], px[j][1], px[j][2],
                                     pn[j][0], pn[j][1], pn[j][2], a.R2s, L);
    // slot 0 is the receiver: its density is the numerator
    const float pi = d[0].x;
#if OCC_TILE_TREESUM
    // P_c as a pairwise tree on paired adds (depth log2 K instead of K - 1)
    f32x2 s2[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) s2[j] = pk2(d[j].x, d[j].y);
#pragma unroll
    for (int w = NP / 2; w >= 1; w /= 2)
#pragma unroll
        for (int j = 0; j < w; ++j) s2[j] = add2(s2[j], s2[j + w]);
    const float2 sp = up2(s2[0]);
    const float Psum = sp.x + sp.y;
#else
    // P_c sums in slot order
    float Psum = pi + d[0].y;
#pragma unroll
    for (int j = 1; j < NP; ++j) Psum = (Psum + d[j].x) + d[j].y;
#endif
    *pi_out = pi;
    *psum_out = Psum;
}

// One thread per receiver, 4 or 8 member slots: the K receivers are held as lane pairs
// (slots 2j, 2j + 1) and every candidate's column of densities runs on paired FP32
// instructions (half the issue slots of the scalar column, the same results).
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void tile_single_x2(const TileArgs& a, const RectLight& L,
                                               const Staged& st, const int* s_qoff, int x0,
                                               int y0, int lx, int ly) {
    constexpr int NP = MAXK / 2;
    const int x = x0 + lx, y = y0 + ly;
    if (ly >= a.TH || x >= a.W || y >= a.H) return;
    const int sc = (ly + a.hy0) * a.SW + (lx + a.hx0);
    float res = 1.0f;
    if (staged_valid<PACKED>(st.pos[sc])) {
        int sidx[MAXK];
        const uint32_t vmask = member_mask<MAXK, PACKED>(a, st.pos, x, y, sc, sidx);
        f32x2 px[NP][3], pn[NP][3];
        members_x2<EFFECT, MAXK, PACKED>(L, st, sidx, vmask, px, pn);
        // the member slots whose record holds an occluder: each lane walks its own list, so
        // a warp takes as many candidate steps as its busiest lane (lanes whose candidate
        // missed no longer idle through the other lanes' columns)
        uint32_t hm = hit_slots<MAXK>(a, st, sidx, vmask);
        const uint32_t blocked = hm;   // valid members whose record holds an occluder
        float B = 0.0f;
#if OCC_TILE_CAND2
        // two candidate columns per step (independent work for the scheduler); the terms
        // are added in slot order as in the one-column loop
        while (hm) {
            const int c0 = __ffs(hm) - 1;
            hm &= hm - 1u;
            const bool two = hm != 0u;
            const int c1 = two ? __ffs(hm) - 1 : c0;
            hm &= hm - 1u;
            float pi0, P0, pi1, P1;
            column_x2<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, sc, c0, px, pn, &pi0, &P0);
            column_x2<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, sc, c1, px, pn, &pi1, &P1);
            if (pi0 > 0.0f) B += tile_ratio(pi0, P0);
            if (two && pi1 > 0.0f) B += tile_ratio(pi1, P1);
        }
#else
        while (hm) {
            const int c = __ffs(hm) - 1;
            hm &= hm - 1u;
            float pi, Psum;
            column_x2<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, sc, c, px, pn, &pi, &Psum);
            if (pi > 0.0f) B += tile_ratio(pi, Psum);
        }
#endif
        res = 1.0f - B;
        if (EFFECT == kShadow && blocked == vmask) res = 0.0f;   // all-blocked guard
    }
    a.out[y * a.W + x] = res;
}

// One thread per receiver: its K receivers in registers (missing members carry zero
// receiver terms, whose densities are 0, so the pair loop has no per-member test).
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void tile_single(const TileArgs& a, const RectLight& L, const Staged& st,
                                            const int* s_qoff, int x0, int y0, int lx, int ly) {
    // (16 slots held as pairs spill: they keep the scalar column)
    if ((MAXK == 4 || MAXK == 8) && OCC_TILE_PAIRED) {
        tile_single_x2<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, x0, y0, lx, ly);
        return;
    }
    const int x = x0 + lx, y = y0 + ly;
    if (ly >= a.TH || x >= a.W || y >= a.H) return;
    const int sc = (ly + a.hy0) * a.SW + (lx + a.hx0);
    float res = 1.0f;
    if (staged_valid<PACKED>(st.pos[sc])) {
        // staged index of every member slot (the receiver's own for missing members)
        int sidx[MAXK];
        const uint32_t vmask = member_mask<MAXK, PACKED>(a, st.pos, x, y, sc, sidx);
        float3 rx[MAXK], rt[MAXK];
#pragma unroll
        for (int s = 0; s < MAXK; ++s) {
            staged_recv<EFFECT, PACKED>(st, sidx[s], L, &rx[s], &rt[s]);
            if (!((vmask >> s) & 1u)) rt[s] = make_float3(0.0f, 0.0f, 0.0f);
        }
        float B = 0.0f;
        uint32_t blocked = 0;
        auto candidate = [&](int c) {
            if (!((vmask >> c) & 1u)) return;
            const int q = sidx[c];
            const float4 r0 = st.r0[q];
            if (__float_as_int(r0.w) < 0) return;
            blocked |= 1u << c;
            float3 z, nz;
            staged_cand<PACKED>(st, q, r0, &z, &nz);
            // slot 0 is the receiver: its density is the numerator
            const float pi = pair_density<EFFECT>(z, nz, rx[0], rt[0], a.R2s, L);
            float Psum = pi;
#pragma unroll
            for (int s = 1; s < MAXK; ++s) Psum += pair_density<EFFECT>(z, nz, rx[s], rt[s], a.R2s, L);
            if (pi > 0.0f) B += tile_ratio(pi, Psum);
        };
        // AO: the unrolled candidate loop keeps the member indices in registers (1080p,
        // 8 disk offsets: 0.129 against 0.134 ms rolled); shadows measured faster rolled
        // (0.150 against 0.152 ms)
        if (EFFECT == kAO) {
#pragma unroll
            for (int c = 0; c < MAXK; ++c)
                if (c < a.K) candidate(c);
        } else {
#pragma unroll 1
            for (int c = 0; c < a.K; ++c) candidate(c);
        }
        res = 1.0f - B;
        if (EFFECT == kShadow && blocked == vmask) res = 0.0f;   // all-blocked guard
    }
    a.out[y * a.W + x] = res;
}

// Two threads per receiver (twice the resident warps at half the registers each): thread h
// of the pair holds the member slots 2j + h, and the pair adds its halves of P_j with one
// shuffle.  Candidates that no lane of the warp has are skipped warp-uniformly, so every
// lane reaches the shuffle.  The default for AO windows of more than 9 members (4K, 16 disk
// offsets: 1.82 against 2.13 ms); with 8 offsets the doubled candidate loads, member masks
// and shuffles outweigh the extra warps (1080p: 0.179 against 0.137 ms).
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void tile_pairs(const TileArgs& a, const RectLight& L, const Staged& st,
                                           int x0, int y0) {
    constexpr int HALF = (MAXK + 1) / 2;
    const int r = threadIdx.x >> 1, h = threadIdx.x & 1;
    const int lx = r % a.TW, ly = r / a.TW;
    const int x = x0 + lx, y = y0 + ly;
    const bool inside = ly < a.TH && x < a.W && y < a.H;
    const int sc = (min(ly, a.TH - 1) + a.hy0) * a.SW + (lx + a.hx0);
    const bool rvalid = inside && staged_valid<PACKED>(st.pos[sc]);
    const uint32_t vmask = rvalid ? member_mask<MAXK, PACKED>(a, st.pos, x, y, sc) : 0u;
    float3 rx[HALF], rt[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const int s = 2 * j + h;
        const bool v = (vmask >> s) & 1u;
        int q = sc;
        if (v) {
            const int2 o = member_offset(a, s);
            q = sc + o.y * a.SW + o.x;
        }
        staged_recv<EFFECT, PACKED>(st, q, L, &rx[j], &rt[j]);
        if (!v) rt[j] = make_float3(0.0f, 0.0f, 0.0f);
    }
    float B = 0.0f;
    uint32_t blocked = 0;
#pragma unroll 1
    for (int c = 0; c < a.K; ++c) {
        const int2 o = member_offset(a, c);
        const int q = sc + o.y * a.SW + o.x;
        bool cand = (vmask >> c) & 1u;
        float4 r0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (cand) {
            r0 = st.r0[q];
            cand = __float_as_int(r0.w) >= 0;
        }
        if (!__any_sync(0xFFFFFFFFu, cand)) continue;
        blocked |= (uint32_t)cand << c;
        float3 z = make_float3(0.0f, 0.0f, 0.0f), nz = z;
        if (cand) staged_cand<PACKED>(st, q, r0, &z, &nz);
        float pi = 0.0f, part = 0.0f;
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
            const float d = pair_density<EFFECT>(z, nz, rx[j], rt[j], a.R2s, L);
            part += d;
            if (j == 0) pi = d;   // slot 0 (the receiver) on the pair's first thread
        }
        const float Psum = part + __shfl_xor_sync(0xFFFFFFFFu, part, 1);
        if (cand && h == 0 && pi > 0.0f) B += pi / Psum;
    }
    if (h == 0 && inside) {
        float res = 1.0f;
        if (rvalid) {
            res = 1.0f - B;
            if (EFFECT == kShadow && blocked == vmask) res = 0.0f;   // all-blocked guard
        }
        a.out[y * a.W + x] = res;
    }
}

template <int EFFECT, int MAXK, bool PAIRS, bool PACKED>
__device__ __forceinline__ void reuse_tile_body(const CUtensorMap* tm_pos, const CUtensorMap* tm_nrm,
                                                const CUtensorMap* tm_r0, const CUtensorMap* tm_r1,
                                                const TileArgs& a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    // bulk-tensor copies need 128-byte aligned shared destinations: align the base (the
    // launch adds 128 bytes of slack) and round every plane up to a multiple of 128 bytes
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    constexpr int kPlanes = PACKED ? 2 : 4;                   // packed: G-buffer, records
    const int plane = ((a.SW * a.SH + 7) / 8) * 8;          // float4 per plane
    const uint32_t bytes = (uint32_t)kPlanes * (uint32_t)(a.SW * a.SH) * 16u;   // bytes delivered
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
    }
    __syncthreads();
    RectLight L;
    if (EFFECT == kShadow) L = tile_light(a.lp);
    // buffer b holds the G-buffer and record planes of one staged tile
    auto issue = [&](int tile, int b) {
        float4* base = reinterpret_cast<float4*>(smem) + (size_t)b * kPlanes * plane;
        const int x0 = (tile % a.tiles_x) * a.TW, y0 = (tile / a.tiles_x) * a.TH;
        const int gx = 4 * (x0 - a.hx0), gy = y0 - a.hy0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[b], bytes);
        if (PACKED) {
            tma_load_2d(base, tm_pos, gx, gy, &bar[b]);
            tma_load_2d(base + plane, tm_r0, gx, gy, &bar[b]);
        } else {
            tma_load_2d(base, tm_pos, gx, gy, &bar[b]);
            tma_load_2d(base + plane, tm_nrm, gx, gy, &bar[b]);
            tma_load_2d(base + 2 * plane, tm_r0, gx, gy, &bar[b]);
            tma_load_2d(base + 3 * plane, tm_r1, gx, gy, &bar[b]);
        }
    };
    // staged-index offset of every member slot (slot s of the receiver at staged index sc
    // sits at sc + s_qoff[s])
    __shared__ int s_qoff[kMaxMembers];
    if (threadIdx.x < (unsigned)a.K) {
        const int2 o = member_offset(a, (int)threadIdx.x);
        s_qoff[threadIdx.x] = o.y * a.SW + o.x;
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    if (threadIdx.x == 0 && (int)blockIdx.x < a.n_tiles) issue(blockIdx.x, 0);
    int it = 0;
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
        const int b = a.stages == 2 ? (it & 1) : 0;
        if (a.stages == 2 && threadIdx.x == 0 && tile + (int)gridDim.x < a.n_tiles)
            issue(tile + gridDim.x, b ^ 1);   // prefetch: that buffer was released last iteration
        if (!mbar_wait(&bar[b], parity[b])) {
            if (threadIdx.x == 0) atomicOr(a.status, kStatusWaitTimeoutBit);
            mbar_wait(&bar[b], parity[b]);          // let the copies drain (bounded)
            if (a.stages == 2) mbar_wait(&bar[b ^ 1], parity[b ^ 1]);
            return;
        }
        parity[b] ^= 1u;
        Staged st;
        st.pos = reinterpret_cast<const float4*>(smem) + (size_t)b * kPlanes * plane;
        if (PACKED) {
            st.nrm = nullptr;
            st.r0 = st.pos + plane;
            st.r1 = nullptr;
        } else {
            st.nrm = st.pos + plane;
            st.r0 = st.pos + 2 * plane;
            st.r1 = st.pos + 3 * plane;
        }
        const int x0 = (tile % a.tiles_x) * a.TW, y0 = (tile / a.tiles_x) * a.TH;
        if (PAIRS)
            tile_pairs<EFFECT, MAXK, PACKED>(a, L, st, x0, y0);
        else
            tile_single<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, x0, y0, (int)threadIdx.x % a.TW,
                                              (int)threadIdx.x / a.TW);
        __syncthreads();   // buffer b is free for the copies issued next
        if (a.stages == 1 && threadIdx.x == 0 && tile + (int)gridDim.x < a.n_tiles)
            issue(tile + gridDim.x, 0);
    }
}

// The same walk with a producer warp (the CTA's last warp, lane 0) that issues the copies
// of the CTA's tiles into `stages` buffers: full[b] completes when the copies into buffer b
// have landed, empty[b] when every receiver warp has finished with it (one arrival per
// warp).  The producer refills a buffer only after its empty phase; at the end it waits for
// its own last copies, so none is in flight when the CTA exits.  Every wait is bounded: on expiry the waiter records
// kStatusWaitTimeoutBit and stops (the producer issues nothing more; a receiver warp
// returns).
template <int EFFECT, int MAXK, bool PACKED>
__device__ __forceinline__ void reuse_tile_body_ws(const CUtensorMap* tm_pos, const CUtensorMap* tm_nrm,
                                                   const CUtensorMap* tm_r0, const CUtensorMap* tm_r1,
                                                   const TileArgs& a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ int s_qoff[kMaxMembers];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    constexpr int kPlanes = PACKED ? 2 : 4;
    const int plane = ((a.SW * a.SH + 7) / 8) * 8;
    const uint32_t bytes = (uint32_t)kPlanes * (uint32_t)(a.SW * a.SH) * 16u;
    const int S = a.stages;
    const int consumers = a.TW * a.TH;           // receiver threads; the producer warp follows
    const uint32_t cwarps = (uint32_t)(consumers / 32);
    if (threadIdx.x == 0) {
        mbar_init(&full[0]);
        mbar_init(&full[1]);
        mbar_init_count(&empty[0], cwarps);
        mbar_init_count(&empty[1], cwarps);
    }
    if (threadIdx.x < (unsigned)a.K) {
        const int2 o = member_offset(a, (int)threadIdx.x);
        s_qoff[threadIdx.x] = o.y * a.SW + o.x;
    }
    __syncthreads();
    if ((int)threadIdx.x >= consumers) {
        if ((int)threadIdx.x != consumers) return;
        int it = 0, last = -1;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
            const int b = it % S;
            if (it >= S && !mbar_wait(&empty[b], (uint32_t)((it / S - 1) & 1))) {
                atomicOr(a.status, kStatusWaitTimeoutBit);
                break;
            }
            float4* base = reinterpret_cast<float4*>(smem) + (size_t)b * kPlanes * plane;
            const int x0 = (tile % a.tiles_x) * a.TW, y0 = (tile / a.tiles_x) * a.TH;
            const int gx = 4 * (x0 - a.hx0), gy = y0 - a.hy0;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&full[b], bytes);
            tma_load_2d(base, tm_pos, gx, gy, &full[b]);
            if (PACKED) {
                tma_load_2d(base + plane, tm_r0, gx, gy, &full[b]);
            } else {
                tma_load_2d(base + plane, tm_nrm, gx, gy, &full[b]);
                tma_load_2d(base + 2 * plane, tm_r0, gx, gy, &full[b]);
                tma_load_2d(base + 3 * plane, tm_r1, gx, gy, &full[b]);
            }
            last = it;
        }
        // the copies of the last `S` issued tiles may still be landing
        for (int j = last; j >= 0 && j > last - S; --j)
            if (!mbar_wait(&full[j % S], (uint32_t)((j / S) & 1))) atomicOr(a.status, kStatusWaitTimeoutBit);
        return;
    }
    RectLight L;
    if (EFFECT == kShadow) L = tile_light(a.lp);
    const int lane = threadIdx.x & 31;
    int it = 0;
    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
        const int b = it % S;
        if (!mbar_wait(&full[b], (uint32_t)((it / S) & 1))) {
            if (lane == 0) atomicOr(a.status, kStatusWaitTimeoutBit);
            return;
        }
        Staged st;
        st.pos = reinterpret_cast<const float4*>(smem) + (size_t)b * kPlanes * plane;
        if (PACKED) {
            st.nrm = nullptr;
            st.r0 = st.pos + plane;
            st.r1 = nullptr;
        } else {
            st.nrm = st.pos + plane;
            st.r0 = st.pos + 2 * plane;
            st.r1 = st.pos + 3 * plane;
        }
        const int x0 = (tile % a.tiles_x) * a.TW, y0 = (tile / a.tiles_x) * a.TH;
        tile_single<EFFECT, MAXK, PACKED>(a, L, st, s_qoff, x0, y0, (int)threadIdx.x % a.TW,
                                          (int)threadIdx.x / a.TW);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
}

template <int EFFECT, int MAXK, bool PACKED>
__global__ void __launch_bounds__(512, 1)
    k_reuse_tile(const __grid_constant__ CUtensorMap tm_pos, const __grid_constant__ CUtensorMap tm_nrm,
                 const __grid_constant__ CUtensorMap tm_r0, const __grid_constant__ CUtensorMap tm_r1,
                 const __grid_constant__ TileArgs a) {
#if OCC_TILE_WS
    reuse_tile_body_ws<EFFECT, MAXK, PACKED>(&tm_pos, &tm_nrm, &tm_r0, &tm_r1, a);
#else
    reuse_tile_body<EFFECT, MAXK, false, PACKED>(&tm_pos, &tm_nrm, &tm_r0, &tm_r1, a);
#endif
}

template <int EFFECT, int MAXK, bool PACKED>
__global__ void __launch_bounds__(1024, 1)
    k_reuse_tile_pairs(const __grid_constant__ CUtensorMap tm_pos,
                       const __grid_constant__ CUtensorMap tm_nrm,
                       const __grid_constant__ CUtensorMap tm_r0,
                       const __grid_constant__ CUtensorMap tm_r1, const __grid_constant__ TileArgs a) {
    reuse_tile_body<EFFECT, MAXK, true, PACKED>(&tm_pos, &tm_nrm, &tm_r0, &tm_r1, a);
}

// The bounded-wait path of the kernel above, exercised on purpose: one thread polls a barrier
// that no arrival will ever complete, gives up after `spins` polls and records
// kStatusWaitTimeoutBit, as every wait of k_reuse_tile does when it runs out.
__global__ void k_debug_wait_timeout(uint32_t spins, unsigned* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar);
    bool done = false;
    for (uint32_t i = 0; i < spins && !done; ++i) done = mbar_try_wait(&bar, 0u);
    if (!done) atomicOr(status, kStatusWaitTimeoutBit);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2D view of a W x H float4 plane as float32 [H][4W]; box = (4 SW, SH).
// 2D map of a float4 plane of W x H pixels with rows `pitch` pixels apart.
bool make_map(CUtensorMap* m, const void* base, int W, int H, int pitch, int SW, int SH) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)4 * W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 16};
    const cuuint32_t box[2] = {(cuuint32_t)(4 * SW), (cuuint32_t)SH};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EFFECT, int MAXK>
cudaError_t launch_t(const CUtensorMap* maps, const TileArgs& a, size_t smem, int sms, bool pairs,
                     bool packed, cudaStream_t s) {
    auto k = packed ? (pairs ? k_reuse_tile_pairs<EFFECT, MAXK, true> : k_reuse_tile<EFFECT, MAXK, true>)
                    : (pairs ? k_reuse_tile_pairs<EFFECT, MAXK, false> : k_reuse_tile<EFFECT, MAXK, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = a.n_tiles < sms ? a.n_tiles : sms;
    const int threads = pairs ? 2 * a.TW * a.TH : a.TW * a.TH + 32 * OCC_TILE_WS;
    k<<<grid, threads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
    return cudaPeekAtLastError();
}

}  // namespace

// Returns false (nothing launched) when the pattern or the staging does not fit this
// kernel: not a box / offsets pattern, a tiled G-buffer, K > 16, a halo wider than the TMA
// box allows, or a tile that does not fit in shared memory.
cudaError_t launch_debug_wait_timeout(uint32_t spins, unsigned* status, cudaStream_t s) {
    k_debug_wait_timeout<<<1, 32, 0, s>>>(spins, status);
    return cudaGetLastError();
}

bool launch_reuse_tile(int effect, const GBufView& gb, const RecView& rec, const PatternParams& pat,
                       float R2s, const LightParams& light, float* out, unsigned* status,
                       cudaStream_t s, cudaError_t* err, int tile_rows, bool pairs) {
    *err = cudaSuccess;
    if (pat.kind != 1 && pat.kind != 2) return false;
    if ((gb.packed != 0) != (rec.packed != 0)) return false;
    if (gb.tiled) return false;   // the bulk-tensor copies stage row-major boxes
    const bool packed = gb.packed != 0;
    const size_t planes = packed ? 2 : 4;
    if (pat.K > 16) return false;
    const int hx = pat.halo[0] + pat.halo[1], hy = pat.halo[2] + pat.halo[3];
    const int SW = kTileW + hx;
    if (4 * SW > 256) return false;
    int dev = 0, sms = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    // largest tile height whose staging fits; two buffers (prefetch) when they fit.  With a
    // producer warp the tiles are one row shorter (15, 7 or 3 rows) so that the receiver
    // warps and the producer make 512, 256 or 128 threads.
    int TH = (tile_rows == 4 || tile_rows == 8) ? tile_rows : 16, stages = 1;
    size_t smem = 0;
    const bool ws = OCC_TILE_WS && !pairs;
    for (; TH >= 4; TH /= 2) {
        const int rows = ws ? TH - 1 : TH;
        if (hy + rows > 256) continue;
        smem = planes * (((size_t)SW * (rows + hy) + 7) / 8 * 8) * 16;   // 128-byte planes
        if (2 * smem + 1024 <= (size_t)max_smem) {
            stages = 2;
            smem = 2 * smem + 128;
            break;
        }
        if (smem + 1024 <= (size_t)max_smem) {
            smem += 128;
            break;
        }
    }
    if (TH < 4) return false;
    if (ws) --TH;
    TileArgs a;
    a.W = gb.W;
    a.H = gb.H;
    a.TW = kTileW;
    a.TH = TH;
    a.hx0 = pat.halo[0];
    a.hy0 = pat.halo[2];
    a.SW = SW;
    a.SH = TH + hy;
    a.tiles_x = (gb.W + kTileW - 1) / kTileW;
    a.n_tiles = a.tiles_x * ((gb.H + TH - 1) / TH);
    a.stages = stages;
    a.kind = pat.kind;
    a.gw = pat.gw;
    a.gh = pat.gh;
    a.K = pat.K;
    for (int i = 0; i < kMaxMembers - 1; ++i) a.off[i] = pat.off[i];
    a.R2s = R2s;
    a.lp = light;
    a.out = out;
    a.status = status;
    CUtensorMap maps[4];
    if (packed) {
        // the kernel reads the packed G-buffer and record planes only
        if (!make_map(&maps[0], gb.pos, gb.W, gb.H, gb.pitch, a.SW, a.SH) ||
            !make_map(&maps[2], rec.r0, gb.W, gb.H, gb.W, a.SW, a.SH))
            return false;
        maps[1] = maps[0];
        maps[3] = maps[2];
    } else if (!make_map(&maps[0], gb.pos, gb.W, gb.H, gb.pitch, a.SW, a.SH) ||
               !make_map(&maps[1], gb.nrm, gb.W, gb.H, gb.pitch, a.SW, a.SH) ||
               !make_map(&maps[2], rec.r0, gb.W, gb.H, gb.W, a.SW, a.SH) ||
               !make_map(&maps[3], rec.r1, gb.W, gb.H, gb.W, a.SW, a.SH)) {
        return false;
    }
    // slot counts: every slot beyond K costs a density, so the common sizes get their own
    if (effect == kAO)
        *err = pat.K <= 4 ? launch_t<kAO, 4>(maps, a, smem, sms, pairs, packed, s)
               : pat.K <= 8 ? launch_t<kAO, 8>(maps, a, smem, sms, pairs, packed, s)
               : pat.K <= 9 ? launch_t<kAO, 9>(maps, a, smem, sms, pairs, packed, s)
                            : launch_t<kAO, 16>(maps, a, smem, sms, pairs, packed, s);
    else
        *err = pat.K <= 4 ? launch_t<kShadow, 4>(maps, a, smem, sms, pairs, packed, s)
               : pat.K <= 8 ? launch_t<kShadow, 8>(maps, a, smem, sms, pairs, packed, s)
               : pat.K <= 9 ? launch_t<kShadow, 9>(maps, a, smem, sms, pairs, packed, s)
                            : launch_t<kShadow, 16>(maps, a, smem, sms, pairs, packed, s);
    return true;
}

}  // namespace occ
