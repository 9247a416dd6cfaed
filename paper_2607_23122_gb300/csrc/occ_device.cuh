// occ_device.cuh -- device-side building blocks shared by the trace and reuse kernels.
//
//  * Philox4x32-10 counter-based generator (Salmon et al., SC'11).
//  * Step-1 ray generation: cosine-weighted AO directions (Eq. 2) with the
//    Duff et al. (JCGT 2017) tangent frame, uniform rectangle-light samples (Eq. 5).
//  * Closest-hit query over the 4-wide BVH with a short per-thread stack and
//    the watertight ray/triangle test of Woop, Benthin and Wald (JCGT 2013)
//    in FP32 (with its FP64 fallback on exactly-zero edge functions).
//    The hit on (0, tmax] with the smallest t wins; equal t goes to the smaller
//    triangle id -- the first intersection of Eq. 7.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "occ_f32x2.cuh"
#include "occ_layout.h"

namespace occ {

// ---------------------------------------------------------------------------------------
// Philox4x32-10.  Round: (x0,x1,x2,x3) -> (hi(B x2)^x1^k0, lo(B x2), hi(A x0)^x3^k1, lo(A x0)),
// A = 0xD2511F53, B = 0xCD9E8D57; key += (0x9E3779B9, 0xBB67AE85) after each round.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hiA = __umulhi(0xD2511F53u, c.x), loA = 0xD2511F53u * c.x;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, c.z), loB = 0xCD9E8D57u * c.z;
        c = make_uint4(hiB ^ c.y ^ k.x, loB, hiA ^ c.w ^ k.y, loA);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

enum : uint32_t { kStreamAO = 0, kStreamShadow = 1 };

// Two uniforms in [0, 1): top 24 bits of the first two words times 2^-24 (exact).
__device__ __forceinline__ float2 uniform_pair(uint64_t seed, uint32_t pix, uint32_t sample,
                                               uint32_t stream) {
    const uint4 w = philox4x32_10(make_uint4(pix, sample, stream, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return make_float2((float)(w.x >> 8) * 0x1p-24f, (float)(w.y >> 8) * 0x1p-24f);
}

// ---------------------------------------------------------------------------------------
// float3 helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) {
    const float inv = 1.0f / sqrtf(dot3(a, a));
    return make_float3(a.x * inv, a.y * inv, a.z * inv);
}

// ---------------------------------------------------------------------------------------
// Packed formats.  Octahedral unit-vector code (Cigolle et al., JCGT 2014): project n
// onto the octahedron |x|+|y|+|z| = 1, fold the lower half over the diagonals, store
// (x, y) as two 16-bit snorms.  0x80008000 (never produced: codes are clamped to
// +-32767) marks an invalid G-buffer pixel.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kOctInvalid = 0x80008000u;

__device__ __forceinline__ float sign_nz(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ uint32_t oct_encode(float3 n) {
    const float inv = 1.0f / (fabsf(n.x) + fabsf(n.y) + fabsf(n.z));
    float px = n.x * inv, py = n.y * inv;
    if (n.z < 0.0f) {
        const float fx = (1.0f - fabsf(py)) * sign_nz(px);
        const float fy = (1.0f - fabsf(px)) * sign_nz(py);
        px = fx;
        py = fy;
    }
    const int qx = __float2int_rn(fminf(fmaxf(px, -1.0f), 1.0f) * 32767.0f);
    const int qy = __float2int_rn(fminf(fmaxf(py, -1.0f), 1.0f) * 32767.0f);
    return ((uint32_t)qx & 0xFFFFu) | ((uint32_t)qy << 16);
}

// The unfolded vector is formed in integers (units of 1/32767): its z, and whether the
// code lies in the folded half, are then exact, so every decoder agrees on the sign of z
// (the tangent frame built from a normal branches on that sign).
__device__ __forceinline__ float3 oct_decode(uint32_t c) {
    int qx = (int)(int16_t)(c & 0xFFFFu), qy = (int)(int16_t)(c >> 16);
    const int qz = 32767 - abs(qx) - abs(qy);
    if (qz < 0) {
        const int tx = qx;
        qx = (32767 - abs(qy)) * (tx >= 0 ? 1 : -1);
        qy = (32767 - abs(tx)) * (qy >= 0 ? 1 : -1);
    }
    const float x = (float)qx, y = (float)qy, z = (float)qz;
    const float inv = rsqrtf(x * x + y * y + z * z);
    return make_float3(x * inv, y * inv, z * inv);
}

// G-buffer entry p: receiver point, normal, validity.
__device__ __forceinline__ bool gb_fetch(const float4* pos, const float4* nrm, bool packed, int p,
                                         float3* x, float3* n) {
    const float4 q = __ldg(pos + p);
    *x = make_float3(q.x, q.y, q.z);
    if (packed) {
        const uint32_t c = __float_as_uint(q.w);
        if (c == kOctInvalid) return false;
        *n = oct_decode(c);
        return true;
    }
    if (q.w == 0.0f) return false;
    const float4 m = __ldg(nrm + p);
    *n = make_float3(m.x, m.y, m.z);
    return true;
}

__device__ __forceinline__ bool gb_valid(const float4* pos, bool packed, int p) {
    const float4 q = __ldg(pos + p);
    return packed ? __float_as_uint(q.w) != kOctInvalid : q.w != 0.0f;
}

// Packed record: words 0-1 = a 64-bit word holding the occluder offset (below) in bits
// 0-62 and bit 63 set; word 2 = octahedral n_z; word 3 = triangle id (-1: no occluder).
// Packed occluder offset d = z - x_source: three 19-bit two's-complement mantissas m with a
// shared exponent E (6 bits), d = m * 2^(E - 60).  E = floor(log2 max|d_i|) + 43, so the
// largest component uses 17-18 bits and every component is rounded to a unit of
// 2^-17..2^-18 of max|d_i|: the precision follows |z - x|, which is what the density
// and support tests are sensitive to.
constexpr int kOffMantBits = 19;
constexpr int kOffMantMax = (1 << (kOffMantBits - 1)) - 1;
constexpr int kOffExpBias = 60;

__device__ __forceinline__ uint64_t pack_offset(float3 d) {
    const float M = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
    if (!(M > 0.0f)) return 0ull;
    const int k = ((__float_as_int(M) >> 23) & 0xFF) - 127;   // floor(log2 M), M normal
    const int E = max(0, min(63, k + 43));
    const float inv_unit = __int_as_float((kOffExpBias - E + 127) << 23);   // 2^(60 - E)
    const int mx = max(-kOffMantMax, min(kOffMantMax, __float2int_rn(d.x * inv_unit)));
    const int my = max(-kOffMantMax, min(kOffMantMax, __float2int_rn(d.y * inv_unit)));
    const int mz = max(-kOffMantMax, min(kOffMantMax, __float2int_rn(d.z * inv_unit)));
    const uint64_t mask = (1ull << kOffMantBits) - 1ull;
    return ((uint64_t)(uint32_t)mx & mask) | (((uint64_t)(uint32_t)my & mask) << 19) |
           (((uint64_t)(uint32_t)mz & mask) << 38) | ((uint64_t)E << 57);
}

// x + m * unit with one rounding (m: the sign-extended 19-bit field, exact as a float)
__device__ __forceinline__ float unpack_coord(uint64_t bits, float unit, float x) {
    const int m = (int)((uint32_t)(bits & 0x7FFFFu) << 13) >> 13;
    return __fmaf_rn((float)m, unit, x);
}

__device__ __forceinline__ float4 rec_pack(float3 xsrc, float3 z, float3 nz, int tri) {
    if (tri < 0) return make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
    const uint64_t w = pack_offset(make_float3(z.x - xsrc.x, z.y - xsrc.y, z.z - xsrc.z)) |
                       (1ull << 63);
    return make_float4(__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)(w >> 32)),
                       __uint_as_float(oct_encode(nz)), __int_as_float(tri));
}

// Unpacks a packed record of a source receiver at xsrc; returns its triangle id.
__device__ __forceinline__ int rec_unpack(float4 r, float3 xsrc, float3* z, float3* nz) {
    const uint64_t w = (uint64_t)__float_as_uint(r.x) | ((uint64_t)__float_as_uint(r.y) << 32);
    const int E = (int)((w >> 57) & 63u);
    const float unit = __int_as_float((E - kOffExpBias + 127) << 23);   // 2^(E - 60)
    *z = make_float3(unpack_coord(w, unit, xsrc.x), unpack_coord(w >> 19, unit, xsrc.y),
                     unpack_coord(w >> 38, unit, xsrc.z));
    *nz = oct_decode(__float_as_uint(r.z));
    return __float_as_int(r.w);
}

// ---------------------------------------------------------------------------------------
// Step-1 rays.
// ---------------------------------------------------------------------------------------
struct RectLight {
    float3 c, eu, ev;   // rectangle c + a eu + b ev, |a|, |b| <= 1/2
    float3 n;           // emitting normal normalize(eu x ev)
    float inv_eu2, inv_ev2, lim;   // 1/|eu|^2, 1/|ev|^2, rectangle half-extent with slack
};

// Eq. 2: Malley's method (r = sqrt(u1), phi = 2 pi u2) lifted onto the hemisphere of n,
// expressed in the branch-free orthonormal basis of Duff et al.
__device__ __forceinline__ float3 cosine_direction(float3 n, float2 u) {
    const float r = sqrtf(u.x);
    float sphi, cphi;
    sincospif(2.0f * u.y, &sphi, &cphi);
    const float lx = r * cphi, ly = r * sphi, lz = sqrtf(fmaxf(0.0f, 1.0f - u.x));
    const float s = copysignf(1.0f, n.z);
    const float a = -1.0f / (s + n.z);
    const float b = n.x * n.y * a;
    const float3 t = make_float3(1.0f + s * n.x * n.x * a, s * b, -s * n.x);
    const float3 bt = make_float3(b, s + n.y * n.y * a, -n.y);
    return make_float3(lx * t.x + ly * bt.x + lz * n.x, lx * t.y + ly * bt.y + lz * n.y,
                       lx * t.z + ly * bt.z + lz * n.z);
}

// Eq. 5: y uniform on the rectangle; unit direction toward y and its distance.
__device__ __forceinline__ float3 light_direction(const RectLight& L, float3 x, float2 u,
                                                  float* dist) {
    const float a = u.x - 0.5f, b = u.y - 0.5f;
    const float3 y = make_float3(L.c.x + a * L.eu.x + b * L.ev.x, L.c.y + a * L.eu.y + b * L.ev.y,
                                 L.c.z + a * L.eu.z + b * L.ev.z);
    const float3 d = sub3(y, x);
    const float len = sqrtf(dot3(d, d));
    *dist = len;
    return make_float3(d.x / len, d.y / len, d.z / len);
}

// ---------------------------------------------------------------------------------------
// Watertight ray / triangle test (Woop, Benthin, Wald 2013).
// The ray is sheared so it runs along +z: for a vertex v relative to the origin,
// (Ax, Ay, Az) = (v[kx] - Sx v[kz], v[ky] - Sy v[kz], Sz v[kz]).  The three rows are
// stored as dense vectors so no per-triangle component selection is needed; the
// projection of a vertex is a fixed function of the vertex, so edges shared by two
// triangles get identical edge functions (watertightness).
// ---------------------------------------------------------------------------------------
// 4-wide node visits evaluate the slab distances of two children per instruction (paired
// FP32), take 3-input min / max, and sort packed (distance, slot) keys (OCC_VISIT_PAIRED=1);
// 0 selects the scalar visit (also used by 8-wide trees).  The paired visit issues ~10 %
// fewer instructions; measured at 1080p it was faster for the shadow trace (0.268 against
// 0.275 ms) and slower for the persistent AO trace (0.378 against 0.371 ms).  Once the scalar
// visit dropped its empty-slot test and full sort, it is the faster one for shadows too
// (0.249 against 0.253 ms), so the paired form is off by default.
#ifndef OCC_VISIT_PAIRED
#define OCC_VISIT_PAIRED 0
#endif
constexpr bool kVisitPaired = OCC_VISIT_PAIRED && kWidth == 4;

struct TraceRay {
    float3 o;
    float3 idir;            // 1 / d with zero components replaced by a tiny value
    float3 oidir;           // o * idir: slab distances are lo * idir - oidir (one FMA)
    f32x2 idir2[3];         // paired visits: (idir.a, idir.a) and (-oidir.a, -oidir.a)
    f32x2 noidir2[3];
    uint32_t nsel;          // bit a set: the high plane of axis a is entered first
    float3 rx, ry, rz;      // shear rows
    float3 d;
};

__device__ __forceinline__ TraceRay make_trace_ray(float3 o, float3 d) {
    TraceRay r;
    r.o = o;
    r.d = d;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = 0;
    float m = ax;
    if (ay > m) { kz = 1; m = ay; }
    if (az > m) { kz = 2; }
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dz = kz == 0 ? d.x : (kz == 1 ? d.y : d.z);
    if (dz < 0.0f) { const int t = kx; kx = ky; ky = t; }
    const float dx = kx == 0 ? d.x : (kx == 1 ? d.y : d.z);
    const float dy = ky == 0 ? d.x : (ky == 1 ? d.y : d.z);
    // One reciprocal serves every triangle of the ray, so its rounding is the same for
    // all of them (watertightness needs consistency, not correct rounding).
    const float Sz = __frcp_rn(dz);
    const float Sx = dx * Sz, Sy = dy * Sz;
    r.rx = make_float3(kx == 0 ? 1.0f : (kz == 0 ? -Sx : 0.0f), kx == 1 ? 1.0f : (kz == 1 ? -Sx : 0.0f),
                       kx == 2 ? 1.0f : (kz == 2 ? -Sx : 0.0f));
    r.ry = make_float3(ky == 0 ? 1.0f : (kz == 0 ? -Sy : 0.0f), ky == 1 ? 1.0f : (kz == 1 ? -Sy : 0.0f),
                       ky == 2 ? 1.0f : (kz == 2 ? -Sy : 0.0f));
    r.rz = make_float3(kz == 0 ? Sz : 0.0f, kz == 1 ? Sz : 0.0f, kz == 2 ? Sz : 0.0f);
    const float tiny = 1e-20f;
    r.idir = make_float3(__frcp_rn(fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                         __frcp_rn(fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                         __frcp_rn(fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    r.oidir = make_float3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
    if (kVisitPaired) {
        r.idir2[0] = bc2(r.idir.x);
        r.idir2[1] = bc2(r.idir.y);
        r.idir2[2] = bc2(r.idir.z);
        r.noidir2[0] = bc2(-r.oidir.x);
        r.noidir2[1] = bc2(-r.oidir.y);
        r.noidir2[2] = bc2(-r.oidir.z);
    }
    // a node holds planes lox, hix, loy, hiy, loz, hiz in that order: for a positive
    // direction component the low plane is entered first.
    r.nsel = (r.idir.x >= 0.0f ? 0u : 1u) | (r.idir.y >= 0.0f ? 0u : 2u) | (r.idir.z >= 0.0f ? 0u : 4u);
    return r;
}

// Tests triangle (v0, v1, v2) with input id `id` against the ray on (0, tbest]; on a
// better hit updates tbest / best_id / best_slot.
__device__ __forceinline__ void triangle_test(const TraceRay& r, float4 v0, float4 v1, float4 v2,
                                              uint32_t slot, float& tbest, uint32_t& best_id,
                                              uint32_t& best_slot) {
    const float3 A = sub3(f3(v0), r.o), B = sub3(f3(v1), r.o), C = sub3(f3(v2), r.o);
    const float Ax = dot3(r.rx, A), Ay = dot3(r.ry, A);
    const float Bx = dot3(r.rx, B), By = dot3(r.ry, B);
    const float Cx = dot3(r.rx, C), Cy = dot3(r.ry, C);
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return;
    const float det = U + V + W;
    if (det == 0.0f) return;
    const float Az = dot3(r.rz, A), Bz = dot3(r.rz, B), Cz = dot3(r.rz, C);
    const float T = fmaf(U, Az, fmaf(V, Bz, W * Cz));
    const float adet = fabsf(det);
    const float aT = det < 0.0f ? -T : T;
    if (!(aT > 0.0f)) return;
    if (aT > tbest * adet * 1.00001f) return;
    const float t = __fdiv_rn(aT, adet);
    if (!(t > 0.0f) || t > tbest) return;
    const uint32_t id = __float_as_uint(v0.w);
    if (t == tbest && id >= best_id) return;
    tbest = t;
    best_id = id;
    best_slot = slot;
}

struct Hit {
    uint32_t id;     // input triangle id, kNoHit if none
    uint32_t slot;   // position in the BVH's triangle array
    float t;
};

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Instrumented build (OCC_COUNTERS): a visit of node n / a test of triangle slot s.
__device__ __forceinline__ void count_node(const DevBVH& bvh, uint32_t n) {
#if OCC_COUNTERS
    if (bvh.ctr) {
        atomicAdd(bvh.ctr + 0, 1ull);
        atomicOr(bvh.node_bits + (n >> 5), 1u << (n & 31u));
    }
#endif
}
__device__ __forceinline__ void count_tri(const DevBVH& bvh, uint32_t s) {
#if OCC_COUNTERS
    if (bvh.ctr) {
        atomicAdd(bvh.ctr + 1, 1ull);
        atomicOr(bvh.tri_bits + (s >> 5), 1u << (s & 31u));
    }
#endif
}

#if !OCC_BVH_CW8
// Traversal stack entries: the node reference alone (4 bytes; a popped node beyond the
// current best hit is culled by its own box test), or with its entry distance so that it
// is skipped without the fetch (OCC_STACK_KEYS=1, 8 bytes).  Measured at 1080p: equal for
// AO, 1.7% faster shadows with 4-byte entries (half the local-memory stack).
#ifndef OCC_STACK_KEYS
#define OCC_STACK_KEYS 0
#endif
#if OCC_STACK_KEYS
using StackEntry = uint2;
__device__ __forceinline__ StackEntry stack_entry(uint32_t ref, float key) {
    return make_uint2(ref, __float_as_uint(key));
}
__device__ __forceinline__ uint32_t entry_ref(StackEntry e) { return e.x; }
__device__ __forceinline__ bool entry_live(StackEntry e, float tbest) {
    return __uint_as_float(e.y) <= tbest;
}
#else
using StackEntry = uint32_t;
__device__ __forceinline__ StackEntry stack_entry(uint32_t ref, float) { return ref; }
__device__ __forceinline__ uint32_t entry_ref(StackEntry e) { return e; }
__device__ __forceinline__ bool entry_live(StackEntry, float) { return true; }
#endif

// Push of a hit child (a full stack drops it and records the overflow).  Storing every
// slot's entry and advancing the top by the hit flag, without branches, measured slower
// (1080p AO trace 0.359 against 0.341 ms).
__device__ __forceinline__ void push_entry(StackEntry* stack, int& sp, bool& overflow, bool hit,
                                           StackEntry e) {
    if (hit) {
        if (sp < kStackSize) stack[sp++] = e;
        else overflow = true;
    }
}

// A visit pushes at most kWidth - 1 entries: with that much room left (OCC_PUSH_ROOM=1) the
// pushes skip the per-entry bound test; 0 tests every push (1080p: AO equal, shadow trace
// 0.253 against 0.256 ms).
#ifndef OCC_PUSH_ROOM
#define OCC_PUSH_ROOM 1
#endif
__device__ __forceinline__ bool push_room(int sp) {
    return OCC_PUSH_ROOM && sp <= kStackSize - (kWidth - 1);
}

// Child reference of slot s (0..3) of a node's reference quad.
__device__ __forceinline__ uint32_t child_of(uint4 ch, uint32_t s) {
    const uint32_t lo = (s & 1u) ? ch.y : ch.x, hi = (s & 1u) ? ch.w : ch.z;
    return (s & 2u) ? hi : lo;
}

// Children of a 4-wide node hit by the ray before tbest, nearest first (see visit_node).
// Slab distances of children (0, 1) and (2, 3) come from paired FMAs (each lane rounds as
// fmaf); entry and exit distances take 3-input max / min.  A hit child's key is its entry
// distance (>= 0, so its bits order like the float) with the slot in the two low bits; a
// missed child's key is +inf with its slot.  The keys are sorted as integers: the order of
// children whose entry distances agree to 3 ulps may differ from a float sort, which moves
// no result (the closest hit and its tie rule do not depend on the visit order).  Empty
// slots hold inverted infinite boxes, which no ray enters.
__device__ __forceinline__ void visit_node4(const DevBVH& bvh, uint32_t cur, const TraceRay& r,
                                            float tbest, StackEntry* stack, int& sp,
                                            bool& overflow, uint32_t* next) {
    const float4* nb = reinterpret_cast<const float4*>(bvh.nodes + cur);
    const uint32_t ix = r.nsel & 1u, iy = 2u + ((r.nsel >> 1) & 1u), iz = 4u + ((r.nsel >> 2) & 1u);
    const float4 nx = __ldg(nb + ix), fx = __ldg(nb + (ix ^ 1u));
    const float4 ny = __ldg(nb + iy), fy = __ldg(nb + (iy ^ 1u));
    const float4 nz = __ldg(nb + iz), fz = __ldg(nb + (iz ^ 1u));
    const uint4 ch = __ldg(reinterpret_cast<const uint4*>(nb + 6));
    const float2 nx01 = up2(fma2(pk2(nx.x, nx.y), r.idir2[0], r.noidir2[0]));
    const float2 nx23 = up2(fma2(pk2(nx.z, nx.w), r.idir2[0], r.noidir2[0]));
    const float2 ny01 = up2(fma2(pk2(ny.x, ny.y), r.idir2[1], r.noidir2[1]));
    const float2 ny23 = up2(fma2(pk2(ny.z, ny.w), r.idir2[1], r.noidir2[1]));
    const float2 nz01 = up2(fma2(pk2(nz.x, nz.y), r.idir2[2], r.noidir2[2]));
    const float2 nz23 = up2(fma2(pk2(nz.z, nz.w), r.idir2[2], r.noidir2[2]));
    const float2 fx01 = up2(fma2(pk2(fx.x, fx.y), r.idir2[0], r.noidir2[0]));
    const float2 fx23 = up2(fma2(pk2(fx.z, fx.w), r.idir2[0], r.noidir2[0]));
    const float2 fy01 = up2(fma2(pk2(fy.x, fy.y), r.idir2[1], r.noidir2[1]));
    const float2 fy23 = up2(fma2(pk2(fy.z, fy.w), r.idir2[1], r.noidir2[1]));
    const float2 fz01 = up2(fma2(pk2(fz.x, fz.y), r.idir2[2], r.noidir2[2]));
    const float2 fz23 = up2(fma2(pk2(fz.z, fz.w), r.idir2[2], r.noidir2[2]));
    const float tn[4] = {max3f(nx01.x, ny01.x, fmaxf(nz01.x, 0.0f)),
                         max3f(nx01.y, ny01.y, fmaxf(nz01.y, 0.0f)),
                         max3f(nx23.x, ny23.x, fmaxf(nz23.x, 0.0f)),
                         max3f(nx23.y, ny23.y, fmaxf(nz23.y, 0.0f))};
    const float tf[4] = {min3f(fx01.x, fy01.x, fminf(fz01.x, tbest)),
                         min3f(fx01.y, fy01.y, fminf(fz01.y, tbest)),
                         min3f(fx23.x, fy23.x, fminf(fz23.x, tbest)),
                         min3f(fx23.y, fy23.y, fminf(fz23.y, tbest))};
    constexpr uint32_t kMissKey = 0x7F800000u;
    uint32_t k[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        k[c] = (tn[c] <= tf[c] ? (__float_as_uint(tn[c]) & ~3u) : kMissKey) | (uint32_t)c;
    // ascending sorting network (0,1)(2,3)(0,2)(1,3)(1,2) on the integer keys
#define OCC_USWAP(a, b)                                  \
    {                                                    \
        const uint32_t lo = min(k[a], k[b]), hi = max(k[a], k[b]); \
        k[a] = lo;                                       \
        k[b] = hi;                                       \
    }
    OCC_USWAP(0, 1) OCC_USWAP(2, 3) OCC_USWAP(0, 2) OCC_USWAP(1, 3) OCC_USWAP(1, 2)
#undef OCC_USWAP
    if (push_room(sp)) {
#pragma unroll
        for (int c = 3; c >= 1; --c)
            if (k[c] < kMissKey) stack[sp++] = stack_entry(child_of(ch, k[c] & 3u), __uint_as_float(k[c] & ~3u));
    } else {
#pragma unroll
        for (int c = 3; c >= 1; --c)
            push_entry(stack, sp, overflow, k[c] < kMissKey,
                       stack_entry(child_of(ch, k[c] & 3u), __uint_as_float(k[c] & ~3u)));
    }
    *next = k[0] < kMissKey ? child_of(ch, k[0] & 3u) : kEmptyRef;
}

// Scalar visit: entry / exit distances by three-input max / min (1) or pairwise (0)
#ifndef OCC_VISIT_MAX3
#define OCC_VISIT_MAX3 1
#endif
// Child slots: 1 also tests the reference of a slot against kEmptyRef; 0 relies on the
// empty slots' inverted boxes alone (1080p AO trace 0.342-0.344 against 0.352-0.353 ms with
// the test and the pairwise max / min)
#ifndef OCC_VISIT_EMPTY_TEST
#define OCC_VISIT_EMPTY_TEST 0
#endif


// Four-wide nodes: 1 sorts the hit children fully; 0 stops after the three comparators
// that find the nearest (the others are pushed in partial order; 1080p AO trace 0.333
// against 0.340 ms with the full sort, shadows keep the paired visit's full sort).
#ifndef OCC_VISIT_FULL_SORT
#define OCC_VISIT_FULL_SORT 0
#endif

// Children of node `cur` hit by the ray before tbest, nearest first: the nearest goes to
// *next, the others are pushed far-to-near.  *next = kEmptyRef if none is hit.
#define OCC_CSWAP(a, b)                                                          \
    if (key[b] < key[a]) {                                                      \
        const float tk = key[a]; key[a] = key[b]; key[b] = tk;                  \
        const uint32_t tr = ref[a]; ref[a] = ref[b]; ref[b] = tr;               \
    }
__device__ __forceinline__ void visit_node(const DevBVH& bvh, uint32_t cur, const TraceRay& r,
                                           float tbest, StackEntry* stack, int& sp, bool& overflow,
                                           uint32_t* next) {
    // Slab test of the children: near / far planes are picked by address (the ray's
    // direction signs), each plane distance is one FMA; boxes are grown at build time so
    // this is conservative.
    const float4* nb = reinterpret_cast<const float4*>(bvh.nodes + cur);
    // plane a of axis k is plane 2k + a; its children 4h .. 4h + 3 sit at float4
    // (2k + a) * kPlaneVecs + h, the far plane is the other one of the axis
    const uint32_t ix = r.nsel & 1u, iy = 2u + ((r.nsel >> 1) & 1u), iz = 4u + ((r.nsel >> 2) & 1u);
    const float inf = __int_as_float(0x7f800000);
    float key[kWidth];
    uint32_t ref[kWidth];
#pragma unroll
    for (int h = 0; h < kPlaneVecs; ++h) {
        const float4 nx = __ldg(nb + ix * kPlaneVecs + h), fx = __ldg(nb + (ix ^ 1u) * kPlaneVecs + h);
        const float4 ny = __ldg(nb + iy * kPlaneVecs + h), fy = __ldg(nb + (iy ^ 1u) * kPlaneVecs + h);
        const float4 nz = __ldg(nb + iz * kPlaneVecs + h), fz = __ldg(nb + (iz ^ 1u) * kPlaneVecs + h);
        const uint4 ch = __ldg(reinterpret_cast<const uint4*>(nb + 6 * kPlaneVecs + h));
        const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, fxs[4] = {fx.x, fx.y, fx.z, fx.w};
        const float nys[4] = {ny.x, ny.y, ny.z, ny.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w};
        const float nzs[4] = {nz.x, nz.y, nz.z, nz.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
        const uint32_t cref[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#if OCC_VISIT_MAX3
            const float tn = max3f(fmaf(nxs[c], r.idir.x, -r.oidir.x), fmaf(nys[c], r.idir.y, -r.oidir.y),
                                   fmaxf(fmaf(nzs[c], r.idir.z, -r.oidir.z), 0.0f));
            const float tf = min3f(fmaf(fxs[c], r.idir.x, -r.oidir.x), fmaf(fys[c], r.idir.y, -r.oidir.y),
                                   fminf(fmaf(fzs[c], r.idir.z, -r.oidir.z), tbest));
#else
            const float tn = fmaxf(fmaxf(fmaf(nxs[c], r.idir.x, -r.oidir.x), fmaf(nys[c], r.idir.y, -r.oidir.y)),
                                   fmaxf(fmaf(nzs[c], r.idir.z, -r.oidir.z), 0.0f));
            const float tf = fminf(fminf(fmaf(fxs[c], r.idir.x, -r.oidir.x), fmaf(fys[c], r.idir.y, -r.oidir.y)),
                                   fminf(fmaf(fzs[c], r.idir.z, -r.oidir.z), tbest));
#endif
            // an empty slot has the box (+inf, -inf): its near distance is +inf and its far
            // distance -inf for every direction, so it never passes (as in visit_node4)
            const bool hit = OCC_VISIT_EMPTY_TEST ? (cref[c] != kEmptyRef && tn <= tf) : tn <= tf;
            key[4 * h + c] = hit ? tn : inf;
            ref[4 * h + c] = cref[c];
        }
    }
    // near-to-far order by a sorting network: 4 keys (0,1)(2,3)(0,2)(1,3)(1,2); 8 keys the
    // 19-comparator network (pairs, quadruples, merge).  The nearest child is visited next,
    // the others are pushed far-to-near so closer ones pop first.
    if (kWidth == 4) {
        OCC_CSWAP(0, 1) OCC_CSWAP(2, 3) OCC_CSWAP(0, 2)
#if OCC_VISIT_FULL_SORT
        OCC_CSWAP(1, 3) OCC_CSWAP(1, 2)
#endif
    } else {
        OCC_CSWAP(0, 2) OCC_CSWAP(1, 3) OCC_CSWAP(4, 6) OCC_CSWAP(5, 7)
        OCC_CSWAP(0, 4) OCC_CSWAP(1, 5) OCC_CSWAP(2, 6) OCC_CSWAP(3, 7)
        OCC_CSWAP(0, 1) OCC_CSWAP(2, 3) OCC_CSWAP(4, 5) OCC_CSWAP(6, 7)
        OCC_CSWAP(2, 4) OCC_CSWAP(3, 5) OCC_CSWAP(1, 4) OCC_CSWAP(3, 6)
        OCC_CSWAP(1, 2) OCC_CSWAP(3, 4) OCC_CSWAP(5, 6)
    }
    if (push_room(sp)) {
#pragma unroll
        for (int c = kWidth - 1; c >= 1; --c)
            if (key[c] != inf) stack[sp++] = stack_entry(ref[c], key[c]);
    } else {
#pragma unroll
        for (int c = kWidth - 1; c >= 1; --c)
            push_entry(stack, sp, overflow, key[c] != inf, stack_entry(ref[c], key[c]));
    }
    *next = key[0] != inf ? ref[0] : kEmptyRef;
}
#undef OCC_CSWAP

// Pops the next entry that can still hold a hit before tbest (kEmptyRef when none).
__device__ __forceinline__ uint32_t pop_next(const StackEntry* stack, int& sp, float tbest) {
    while (sp > 0) {
        const StackEntry e = stack[--sp];
        if (entry_live(e, tbest)) return entry_ref(e);
    }
    return kEmptyRef;
}

__device__ __forceinline__ bool is_leaf_ref(uint32_t ref) { return (ref & kLeafBit) != 0u; }

// Resumable closest-hit traversal of one ray on (0, tmax] (t in units of |d|).  While-while
// order: each round walks internal nodes until every active lane of the warp holds a
// postponed leaf, then all lanes test their leaves together, which keeps the lanes on the
// same code path.  The short stack lives outside the state (thread-local array).
struct Traversal {
    TraceRay r;
    float tbest;
    uint32_t best_id, best_slot;
    uint32_t cur, leaf;
    int sp;
    bool overflow;
    bool bad;               // OCC_CHECKS: an index outside the BVH was met
};

// Starts at `start`: the root (0), any node or leaf reference whose subtree holds every
// triangle the ray can meet, or kEmptyRef when none can be met.
__device__ __forceinline__ void trav_init(Traversal& t, float3 o, float3 d, float tmax,
                                          uint32_t start) {
    t.r = make_trace_ray(o, d);
    t.tbest = tmax;
    t.best_id = kNoHit;
    t.best_slot = kNoHit;
    t.sp = 0;
    t.overflow = false;
    t.bad = false;
    t.cur = start;
    t.leaf = kEmptyRef;
    if (t.cur != kEmptyRef && is_leaf_ref(t.cur)) {
        t.leaf = t.cur;
        t.cur = kEmptyRef;
    }
}

// A traversal with no ray (trav_done is true).
__device__ __forceinline__ void trav_clear(Traversal& t) {
    t.cur = t.leaf = kEmptyRef;
    t.sp = 0;
    t.overflow = false;
    t.bad = false;
}

__device__ __forceinline__ bool trav_done(const Traversal& t) {
    return t.cur == kEmptyRef && t.leaf == kEmptyRef;
}

// One round: internal nodes until the warp's active lanes all hold a leaf (or ran out),
// then the leaves.  Call only while !trav_done.  ANY: stop at the first triangle accepted
// on (0, tmax] (visibility queries need only whether one exists; the acceptance test is
// the closest-hit one, so the answer is the same).
template <bool ANY = false, bool PAIRED = kVisitPaired>
__device__ __forceinline__ void trav_round(Traversal& t, const DevBVH& bvh, StackEntry* stack) {
    // internal references are below kEmptyRef, leaf references above it
    while (t.cur < kEmptyRef) {
#if OCC_CHECKS
        if (t.cur >= bvh.n_nodes) {
            t.bad = true;
            t.cur = t.leaf = kEmptyRef;
            return;
        }
#endif
        uint32_t next;
        count_node(bvh, t.cur);
        if (PAIRED && kVisitPaired)
            visit_node4(bvh, t.cur, t.r, t.tbest, stack, t.sp, t.overflow, &next);
        else
            visit_node(bvh, t.cur, t.r, t.tbest, stack, t.sp, t.overflow, &next);
        t.cur = next != kEmptyRef ? next : pop_next(stack, t.sp, t.tbest);
        if (is_leaf_ref(t.cur) && t.leaf == kEmptyRef) {
            t.leaf = t.cur;   // postpone the leaf and keep walking internal nodes
            t.cur = pop_next(stack, t.sp, t.tbest);
        }
        if (!__any_sync(__activemask(), t.leaf == kEmptyRef)) break;
    }
    while (t.leaf != kEmptyRef) {
        const uint32_t first = t.leaf & kLeafFirstMask;
        const uint32_t count = ((t.leaf & ~kLeafBit) >> kLeafCountShift) + 1u;
#if OCC_CHECKS
        if ((uint64_t)first + count > bvh.n_tris) {
            t.bad = true;
            t.cur = t.leaf = kEmptyRef;
            return;
        }
#endif
        for (uint32_t i = 0; i < count; ++i) {
            const float4* tr = bvh.tris + 3ull * (first + i);
            count_tri(bvh, first + i);
            triangle_test(t.r, __ldg(tr), __ldg(tr + 1), __ldg(tr + 2), first + i, t.tbest,
                          t.best_id, t.best_slot);
            if (ANY && t.best_id != kNoHit) break;
        }
        if (ANY && t.best_id != kNoHit) {
            t.cur = t.leaf = kEmptyRef;
        } else if (is_leaf_ref(t.cur)) {
            t.leaf = t.cur;
            t.cur = pop_next(stack, t.sp, t.tbest);
        } else {
            t.leaf = kEmptyRef;
        }
    }
}

#else  // OCC_BVH_CW8
// ---------------------------------------------------------------------------------------
// Traversal of the compressed 8-wide layout (occ_layout.h).  Per ray the octant (bit a set
// for a negative direction component) orders the children: a node's hit internal children
// become bits 24 + (slot ^ octant) of a node group (child base index, bits | imask), visited
// lowest bit first, and its hit leaf children's triangles bits of a triangle group (triangle
// base index, bits 0..23).  The stack holds node groups, one entry per level at most.
// While-while order: a lane walks nodes until it holds a triangle group (or ran out), then
// the lanes test their triangles together.
// ---------------------------------------------------------------------------------------
using StackEntry = uint2;

struct Traversal {
    TraceRay r;
    float tbest;
    uint32_t best_id, best_slot;
    uint2 ng;               // node group: (child base, hit bits 24..31 | imask bits 0..7)
    uint2 tg;               // triangle group: (triangle base, hit bits 0..23)
    uint32_t oct;           // ray octant
    int sp;
    bool overflow;
    bool bad;               // OCC_CHECKS: an index outside the BVH was met
};

__device__ __forceinline__ void trav_clear(Traversal& t) {
    t.ng = make_uint2(0u, 0u);
    t.tg = make_uint2(0u, 0u);
    t.sp = 0;
    t.overflow = false;
    t.bad = false;
}

// Starts at the root (`start` = kEmptyRef: no triangle can be met, nothing to do).
__device__ __forceinline__ void trav_init(Traversal& t, float3 o, float3 d, float tmax,
                                          uint32_t start) {
    t.r = make_trace_ray(o, d);
    t.tbest = tmax;
    t.best_id = kNoHit;
    t.best_slot = kNoHit;
    trav_clear(t);
    t.oct = t.r.nsel;
    // the root as slot 0 of a one-child group based at node 0
    if (start != kEmptyRef) t.ng = make_uint2(0u, (1u << (24u + t.oct)) | 1u);
}

__device__ __forceinline__ bool trav_done(const Traversal& t) {
    return (t.ng.y >> 24) == 0u && t.tg.y == 0u && t.sp == 0;
}

// Byte b (0..3) of w as the float 2^23 + byte (one byte permutation).
__device__ __forceinline__ float byte_f(uint32_t w, uint32_t b) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | b));
}

// Node visit: slab tests of the 8 children (two per paired FMA), then the groups of the hit
// children.  Plane distance of grid value q on axis a: (p_a + q 2^e_a - o_a) / d_a, taken
// as one FMA of the biased byte value f = 2^23 + q: f (2^e_a / d_a) + (p_a - o_a) / d_a
// - 2^23 (2^e_a / d_a); the rounding of the last term is below half a grid step, which the
// builder's extra step of margin on every side absorbs.
__device__ __forceinline__ void visit_cw(const DevBVH& bvh, uint32_t node, const TraceRay& r,
                                         float tbest, uint32_t oct, uint2* ng, uint2* tg) {
    const float4* nb = reinterpret_cast<const float4*>(bvh.nodes) + 5ull * node;
    const float4 v0 = __ldg(nb), v1 = __ldg(nb + 1), v2 = __ldg(nb + 2), v3 = __ldg(nb + 3),
                 v4 = __ldg(nb + 4);
    const uint32_t eb = __float_as_uint(v0.w);
    const float sx = __uint_as_float((eb & 0xFFu) << 23) * r.idir.x;
    const float sy = __uint_as_float(((eb >> 8) & 0xFFu) << 23) * r.idir.y;
    const float sz = __uint_as_float(((eb >> 16) & 0xFFu) << 23) * r.idir.z;
    const float cx = fmaf(-8388608.0f, sx, (v0.x - r.o.x) * r.idir.x);
    const float cy = fmaf(-8388608.0f, sy, (v0.y - r.o.y) * r.idir.y);
    const float cz = fmaf(-8388608.0f, sz, (v0.z - r.o.z) * r.idir.z);
    // near / far plane words (children 0-3, 4-7) per axis: low planes for positive directions
    const uint32_t lox0 = __float_as_uint(v2.x), lox1 = __float_as_uint(v2.y);
    const uint32_t loy0 = __float_as_uint(v2.z), loy1 = __float_as_uint(v2.w);
    const uint32_t loz0 = __float_as_uint(v3.x), loz1 = __float_as_uint(v3.y);
    const uint32_t hix0 = __float_as_uint(v3.z), hix1 = __float_as_uint(v3.w);
    const uint32_t hiy0 = __float_as_uint(v4.x), hiy1 = __float_as_uint(v4.y);
    const uint32_t hiz0 = __float_as_uint(v4.z), hiz1 = __float_as_uint(v4.w);
    const bool nx = oct & 1u, ny = oct & 2u, nz = oct & 4u;
    const uint32_t nxw[2] = {nx ? hix0 : lox0, nx ? hix1 : lox1}, fxw[2] = {nx ? lox0 : hix0, nx ? lox1 : hix1};
    const uint32_t nyw[2] = {ny ? hiy0 : loy0, ny ? hiy1 : loy1}, fyw[2] = {ny ? loy0 : hiy0, ny ? loy1 : hiy1};
    const uint32_t nzw[2] = {nz ? hiz0 : loz0, nz ? hiz1 : loz1}, fzw[2] = {nz ? loz0 : hiz0, nz ? loz1 : hiz1};
    const f32x2 sx2 = bc2(sx), sy2 = bc2(sy), sz2 = bc2(sz), cx2 = bc2(cx), cy2 = bc2(cy), cz2 = bc2(cz);
    const uint32_t imask = eb >> 24;
    const uint32_t meta[2] = {__float_as_uint(v1.z), __float_as_uint(v1.w)};
    uint32_t bits = 0;
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
        const int h = c >> 2;
        const uint32_t b0 = (uint32_t)(c & 3), b1 = b0 + 1u;
        const float2 tnx = up2(fma2(pk2(byte_f(nxw[h], b0), byte_f(nxw[h], b1)), sx2, cx2));
        const float2 tny = up2(fma2(pk2(byte_f(nyw[h], b0), byte_f(nyw[h], b1)), sy2, cy2));
        const float2 tnz = up2(fma2(pk2(byte_f(nzw[h], b0), byte_f(nzw[h], b1)), sz2, cz2));
        const float2 tfx = up2(fma2(pk2(byte_f(fxw[h], b0), byte_f(fxw[h], b1)), sx2, cx2));
        const float2 tfy = up2(fma2(pk2(byte_f(fyw[h], b0), byte_f(fyw[h], b1)), sy2, cy2));
        const float2 tfz = up2(fma2(pk2(byte_f(fzw[h], b0), byte_f(fzw[h], b1)), sz2, cz2));
        const float tn0 = max3f(tnx.x, tny.x, fmaxf(tnz.x, 0.0f));
        const float tn1 = max3f(tnx.y, tny.y, fmaxf(tnz.y, 0.0f));
        const float tf0 = min3f(tfx.x, tfy.x, fminf(tfz.x, tbest));
        const float tf1 = min3f(tfx.y, tfy.y, fminf(tfz.y, tbest));
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int s = c + e;
            const uint32_t m = (meta[h] >> (8 * (s & 3))) & 0xFFu;
            // internal child: one bit at 24 + (slot ^ octant); leaf: its triangles' bits
            const uint32_t idx = (m & 31u) ^ (((imask >> s) & 1u) ? oct : 0u);
            const bool hit = (e == 0 ? tn0 <= tf0 : tn1 <= tf1);
            if (hit) bits |= (m >> 5) << idx;
        }
    }
    *ng = make_uint2(__float_as_uint(v1.x), (bits & 0xFF000000u) | imask);
    *tg = make_uint2(__float_as_uint(v1.y), bits & 0x00FFFFFFu);
}

// One round: node groups until this lane holds triangles (or ran out) while any active lane
// still walks, then the triangles.  Every step of a walking lane consumes a child bit or a
// stack entry, so the node loop ends.  (Postponing a lane's triangles onto the stack while
// few lanes hold some, as Ylitie et al. do, did not raise lane use in a lockstep CPU
// emulation of this loop: 24-26 % either way on incoherent rays.)  ANY: stop at the first
// triangle accepted on (0, tmax].
template <bool ANY = false, bool PAIRED = true>
__device__ __forceinline__ void trav_round(Traversal& t, const DevBVH& bvh, StackEntry* stack) {
    while (t.tg.y == 0u) {
        if ((t.ng.y >> 24) == 0u) {
            if (t.sp == 0) break;
            t.ng = stack[--t.sp];
        } else {
            const uint32_t b = (uint32_t)__ffs(t.ng.y >> 24) - 1u;
            t.ng.y &= ~(1u << (24u + b));
            const uint32_t slot = b ^ t.oct;
            const uint32_t node = t.ng.x + (uint32_t)__popc(t.ng.y & 0xFFu & ((1u << slot) - 1u));
            if (t.ng.y >> 24) {
                if (t.sp < kStackSize) stack[t.sp++] = t.ng;
                else t.overflow = true;
            }
#if OCC_CHECKS
            if (node >= bvh.n_nodes) {
                t.bad = true;
                trav_clear(t);
                return;
            }
#endif
            count_node(bvh, node);
            visit_cw(bvh, node, t.r, t.tbest, t.oct, &t.ng, &t.tg);
        }
        if (!__any_sync(__activemask(), t.tg.y == 0u && !trav_done(t))) break;
    }
    while (t.tg.y) {
        const uint32_t i = t.tg.x + (uint32_t)__ffs(t.tg.y) - 1u;
        t.tg.y &= t.tg.y - 1u;
#if OCC_CHECKS
        if (i >= bvh.n_tris) {
            t.bad = true;
            trav_clear(t);
            return;
        }
#endif
        count_tri(bvh, i);
        const float4* tr = bvh.tris + 3ull * i;
        triangle_test(t.r, __ldg(tr), __ldg(tr + 1), __ldg(tr + 2), i, t.tbest, t.best_id,
                      t.best_slot);
        if (ANY && t.best_id != kNoHit) {
            trav_clear(t);
            return;
        }
    }
}

#endif  // OCC_BVH_CW8

// Closest hit on (0, tmax] from `start` (see trav_init).  Sets kStatusStackOverflowBit in
// *status if the short stack would overflow (the builder bounds the tree depth so that it
// cannot).
__device__ __forceinline__ Hit closest_hit(const DevBVH& bvh, float3 o, float3 d, float tmax,
                                           unsigned int* status, uint32_t start = 0u) {
    Traversal t;
    StackEntry stack[kStackSize];
    trav_init(t, o, d, tmax, start);
    while (!trav_done(t)) trav_round(t, bvh, stack);
    if (t.overflow && status) atomicOr(status, kStatusStackOverflowBit);
    if (OCC_CHECKS && t.bad && status) atomicOr(status, kStatusBadIndexBit);
    Hit h;
    h.id = t.best_id;
    h.slot = t.best_slot;
    h.t = t.tbest;
    return h;
}

// Whether any triangle is hit on (0, tmax].
__device__ __forceinline__ bool any_hit(const DevBVH& bvh, float3 o, float3 d, float tmax,
                                        unsigned int* status) {
    Traversal t;
    StackEntry stack[kStackSize];
    trav_init(t, o, d, tmax, 0u);
    while (!trav_done(t)) trav_round<true>(t, bvh, stack);
    if (t.overflow && status) atomicOr(status, kStatusStackOverflowBit);
    if (OCC_CHECKS && t.bad && status) atomicOr(status, kStatusBadIndexBit);
    return t.best_id != kNoHit;
}

// Start reference for rays whose segments all lie inside the box [qlo, qhi]: walk down
// from the root while exactly one child box overlaps the query box.  The subtree
// returned holds every triangle that any such ray can meet (the skipped siblings' boxes
// do not reach the query box); kEmptyRef means no triangle can be met.  Uniform across
// the calling threads when the query box is.
__device__ __forceinline__ uint32_t start_node(const DevBVH& bvh, float3 qlo, float3 qhi) {
#if OCC_BVH_CW8
    return 0u;   // compressed nodes: every ray starts at the root
#else
    uint32_t cur = 0;
    for (int level = 0; level < kStackSize; ++level) {
        count_node(bvh, cur);
        const float4* nb = reinterpret_cast<const float4*>(bvh.nodes + cur);
        int count = 0;
        uint32_t only = kEmptyRef;
#pragma unroll
        for (int h = 0; h < kPlaneVecs; ++h) {
            const float4 lox = __ldg(nb + 0 * kPlaneVecs + h), hix = __ldg(nb + 1 * kPlaneVecs + h);
            const float4 loy = __ldg(nb + 2 * kPlaneVecs + h), hiy = __ldg(nb + 3 * kPlaneVecs + h);
            const float4 loz = __ldg(nb + 4 * kPlaneVecs + h), hiz = __ldg(nb + 5 * kPlaneVecs + h);
            const uint4 ch = __ldg(reinterpret_cast<const uint4*>(nb + 6 * kPlaneVecs + h));
            const float lx[4] = {lox.x, lox.y, lox.z, lox.w}, hx[4] = {hix.x, hix.y, hix.z, hix.w};
            const float ly[4] = {loy.x, loy.y, loy.z, loy.w}, hy[4] = {hiy.x, hiy.y, hiy.z, hiy.w};
            const float lz[4] = {loz.x, loz.y, loz.z, loz.w}, hz[4] = {hiz.x, hiz.y, hiz.z, hiz.w};
            const uint32_t cref[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const bool ov = cref[c] != kEmptyRef && lx[c] <= qhi.x && hx[c] >= qlo.x &&
                                ly[c] <= qhi.y && hy[c] >= qlo.y && lz[c] <= qhi.z && hz[c] >= qlo.z;
                if (ov) {
                    ++count;
                    only = cref[c];
                }
            }
        }
        if (count == 0) return kEmptyRef;
        if (count > 1 || is_leaf_ref(only)) return count > 1 ? cur : only;
        cur = only;
    }
    return cur;
#endif
}

// Unit geometric normal of BVH triangle `slot`, turned against direction d.
__device__ __forceinline__ float3 hit_normal(const DevBVH& bvh, uint32_t slot, float3 d) {
    const float4* t = bvh.tris + 3ull * slot;
    const float3 v0 = f3(__ldg(t)), v1 = f3(__ldg(t + 1)), v2 = f3(__ldg(t + 2));
    float3 n = normalize3(cross3(sub3(v1, v0), sub3(v2, v0)));
    if (dot3(n, d) > 0.0f) n = make_float3(-n.x, -n.y, -n.z);
    return n;
}

}  // namespace occ
