// occ_path.cuh -- per-receiver device steps shared by the trace, reuse and fused
// trace + reuse kernels: the light frame, the step-1 ray of Alg. 1 / Alg. 2, the record
// writer, the AO start node, and the pair densities of Eq. 15 and Eqs. 20-21 with the
// first-hit test of Eq. 7.
#pragma once

#include "occ_device.cuh"
#include "occ_kernels.h"

namespace occ {

constexpr float kSupportSlack = 1.0f + 1.0f / 65536.0f;

// G-buffer index of pixel p = y W + x (records and outputs use p itself): y pitch + x.
// Entry of pixel (x, y) in a G-buffer plane: row-major with the view's pitch, or the tiled
// layout (8 x 8 tiles in row-major tile order, the tile's pixels in Morton order).
__device__ __forceinline__ int gb_index(const GBufView& gb, int x, int y) {
    if (gb.tiled) {
        const int tiles_x = (gb.W + 7) >> 3;
        const int u = x & 7, v = y & 7;
        const int m = (u & 1) | ((v & 1) << 1) | ((u & 2) << 1) | ((v & 2) << 2) | ((u & 4) << 2) |
                      ((v & 4) << 3);
        return ((y >> 3) * tiles_x + (x >> 3)) * 64 + m;
    }
    return y * gb.pitch + x;
}

// Entry of pixel p = y W + x.
__device__ __forceinline__ int gb_at(const GBufView& gb, int p) {
    if (!gb.tiled && gb.pitch == gb.W) return p;
    const int y = p / gb.W;
    return gb_index(gb, p - y * gb.W, y);
}

// G-buffer entry of pixel p: receiver point, normal, validity.
__device__ __forceinline__ bool gb_fetch(const GBufView& gb, int p, float3* x, float3* n) {
    return gb_fetch(gb.pos, gb.nrm, gb.packed != 0, gb_at(gb, p), x, n);
}

__device__ __forceinline__ bool gb_valid(const GBufView& gb, int p) {
    return gb_valid(gb.pos, gb.packed != 0, gb_at(gb, p));
}

__device__ __forceinline__ float3 gb_point(const GBufView& gb, int p) {
    return f3(__ldg(gb.pos + gb_at(gb, p)));
}
constexpr float kValidateTmax = 1.0f + 1.0f / 1024.0f;

__device__ __forceinline__ RectLight make_light(const LightParams& p) {
    RectLight L;
    L.c = make_float3(p.c[0], p.c[1], p.c[2]);
    L.eu = make_float3(p.eu[0], p.eu[1], p.eu[2]);
    L.ev = make_float3(p.ev[0], p.ev[1], p.ev[2]);
    L.n = normalize3(cross3(L.eu, L.ev));
    L.inv_eu2 = 1.0f / dot3(L.eu, L.eu);
    L.inv_ev2 = 1.0f / dot3(L.ev, L.ev);
    L.lim = 0.5f * kSupportSlack;
    return L;
}

// Step-1 ray of receiver p: origin x, direction, tmax.
template <int EFFECT>
__device__ __forceinline__ float3 step1_ray(float3 x, float3 n, uint32_t p, float radius,
                                            const RectLight& L, uint64_t seed, uint32_t sample,
                                            float* tmax) {
    if (EFFECT == kAO) {
        *tmax = radius;
        return cosine_direction(n, uniform_pair(seed, p, sample, kStreamAO));
    } else {
        return light_direction(L, x, uniform_pair(seed, p, sample, kStreamShadow), tmax);
    }
}

// Record of receiver p (tri < 0: no occluder) in the buffer's format.
__device__ __forceinline__ void write_record(const RecView& rec, uint32_t p, float3 xsrc, float3 z,
                                             float3 nz, float t, int tri) {
    if (rec.packed) {
        rec.r0[p] = rec_pack(xsrc, z, nz, tri);
    } else if (tri < 0) {
        rec.r0[p] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
        rec.r1[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
        rec.r0[p] = make_float4(z.x, z.y, z.z, __int_as_float(tri));
        rec.r1[p] = make_float4(nz.x, nz.y, nz.z, t);
    }
}

// Box holding every AO segment of the warp: the valid origins widened by the radius
// (with slack for the rounding of |direction| and of the box test), reduced over lanes.
__device__ __forceinline__ uint32_t warp_start_node(const DevBVH& bvh, bool valid, float3 x,
                                                    float radius) {
    const float inf = __int_as_float(0x7f800000);
    float lo[3] = {valid ? x.x : inf, valid ? x.y : inf, valid ? x.z : inf};
    float hi[3] = {valid ? x.x : -inf, valid ? x.y : -inf, valid ? x.z : -inf};
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xFFFFFFFFu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xFFFFFFFFu, hi[a], o));
        }
    }
    if (!(lo[0] <= hi[0])) return kEmptyRef;   // no valid receiver in this warp
    const float mag = fmaxf(fmaxf(fmaxf(fabsf(lo[0]), fabsf(hi[0])), fmaxf(fabsf(lo[1]), fabsf(hi[1]))),
                            fmaxf(fabsf(lo[2]), fabsf(hi[2])));
    const float pad = radius * 1.001f + 1e-5f * (1.0f + mag);
    return start_node(bvh, make_float3(lo[0] - pad, lo[1] - pad, lo[2] - pad),
                      make_float3(hi[0] + pad, hi[1] + pad, hi[2] + pad));
}

// Offset of slot s (>= 1) of receiver pixel `pix` in a random pattern (OCC_PAT_RANDOM,
// the per-receiver form of Eq. 8): the first of 32 Philox4x32-10 draws (counter (pix,
// sample, 2, 32 s + a), key = seed) that maps to a lattice point of the disk of radius R
// other than (0, 0) and the slot's earlier offsets acc[0 .. nacc).  Integer arithmetic only;
// false when no attempt qualifies (the slot stays empty).
__device__ __forceinline__ bool random_offset(uint64_t seed, uint32_t pix, uint32_t sample, int s,
                                              int R, const int2* acc, int nacc, int2* out) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t span = 2u * (uint32_t)R + 1u;
    for (int a = 0; a < 32; ++a) {
        const uint4 w = philox4x32_10(make_uint4(pix, sample, 2u, 32u * (uint32_t)s + (uint32_t)a), key);
        const int dx = (int)__umulhi(w.x, span) - R, dy = (int)__umulhi(w.y, span) - R;
        if (dx * dx + dy * dy > R * R || (dx == 0 && dy == 0)) continue;
        bool dup = false;
        for (int q = 0; q < nacc; ++q) dup |= acc[q].x == dx && acc[q].y == dy;
        if (dup) continue;
        *out = make_int2(dx, dy);
        return true;
    }
    return false;
}

// Receiver data needed by the density of each effect.
struct Recv {
    float3 x;
    float3 n;       // AO: normal.  Shadow: (n_L.(c - x), (x - c).eu, (x - c).ev)
    bool valid;
};

template <int EFFECT>
__device__ __forceinline__ Recv make_recv(float3 x, float3 n, bool valid, const RectLight& L) {
    Recv r;
    r.x = x;
    r.valid = valid;
    if (EFFECT == kAO) {
        r.n = n;
    } else {
        const float3 xc = sub3(r.x, L.c);
        r.n = make_float3(-dot3(L.n, xc), dot3(xc, L.eu), dot3(xc, L.ev));
    }
    return r;
}

// Eq. 15 without Occ and 1/pi: max(0, n_x.d) max(0, -n_z.d) / r^4 inside the radius.
__device__ __forceinline__ float dens_ao(float3 z, float3 nz, const Recv& r, float R2s) {
    const float3 d = sub3(z, r.x);
    const float r2 = dot3(d, d);
    const float a = dot3(r.n, d);
    const float b = -dot3(nz, d);
    const bool ok = (a > 0.0f) & (b > 0.0f) & (r2 > 0.0f) & (r2 <= R2s);
    return ok ? __fdividef(a * b, r2 * r2) : 0.0f;
}

// Eqs. 20-21 without Occ and 1/Area: the ray x + s d meets the light plane at
// s_L = n_L.(c - x) / n_L.d (> 1, hitting the emitting side); y' = x + s_L d must lie
// in the rectangle; J = s_L^2 (-n_z.d) / (-n_L.d).
__device__ __forceinline__ float dens_sh(float3 z, float3 nz, const Recv& r, const RectLight& L) {
    const float3 d = sub3(z, r.x);
    const float nd = dot3(L.n, d);
    const float cz = -dot3(nz, d);
    if (!(nd < 0.0f) || !(cz > 0.0f)) return 0.0f;
    // approximate reciprocal (a few ulp): moves s_L and J far less than the 1e-5 output
    // tolerance; only support tests within that margin of their threshold can flip
    const float inv = __fdividef(1.0f, nd);
    const float sL = r.n.x * inv;
    if (!(sL > 1.0f)) return 0.0f;
    const float a = fmaf(sL, dot3(d, L.eu), r.n.y) * L.inv_eu2;
    const float b = fmaf(sL, dot3(d, L.ev), r.n.z) * L.inv_ev2;
    if (fabsf(a) > L.lim || fabsf(b) > L.lim) return 0.0f;
    return sL * sL * cz * (-inv);
}

template <int EFFECT>
__device__ __forceinline__ float density(float3 z, float3 nz, const Recv& r, float R2s,
                                         const RectLight& L) {
    if (EFFECT == kAO) return dens_ao(z, nz, r, R2s);
    return dens_sh(z, nz, r, L);
}

// Eq. 7 for a reused candidate: the closest hit from x toward z (t in (0, 1 + 2^-10]
// in units of z - x) is z's own triangle.
__device__ __forceinline__ bool first_hit(const DevBVH& bvh, float3 x, float3 z, uint32_t tri,
                                          unsigned* status) {
    const Hit h = closest_hit(bvh, x, sub3(z, x), kValidateTmax, status);
    return h.id == tri;
}

}  // namespace occ
