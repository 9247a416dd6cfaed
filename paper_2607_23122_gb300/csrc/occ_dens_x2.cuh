// occ_dens_x2.cuh -- the pair densities of two receivers at once on paired FP32
// instructions (occ_f32x2.cuh), shared by the group and window reuse kernels.  Each lane
// follows the operation order of the scalar densities (dens_ao / dens_sh in occ_path.cuh,
// pair_density in kernels_reuse_tile.cu), so each lane equals them bit for bit; the gain is
// half the issue slots for the arithmetic.
#pragma once

#include "occ_device.cuh"
#include "occ_f32x2.cuh"
#include "occ_kernels.h"

namespace occ {

// AO support test: min(n_x.d, -n_z.d, r^2) > 0 as one three-input minimum instead of three
// compares (the same outcome for every finite input; a NaN in d makes all three NaN and
// fails both forms).
#ifndef OCC_DENS_MIN3
#define OCC_DENS_MIN3 0
#endif

// Eq. 15 without Occ and 1/pi for candidate (z, n_z) at members with points (xx, xy, xz) and
// normals (nx, ny, nz) as lane pairs; (mnx, mny, mnz) = -n_z in both lanes.  An invalid
// member carries a zero normal (n_x.d = 0 fails the support test).
__device__ __forceinline__ float2 dens_ao_x2(f32x2 zx, f32x2 zy, f32x2 zz, f32x2 mnx, f32x2 mny,
                                             f32x2 mnz, f32x2 xx, f32x2 xy, f32x2 xz, f32x2 nx,
                                             f32x2 ny, f32x2 nz, float R2s) {
    const f32x2 dx = sub2(zx, xx), dy = sub2(zy, xy), dz = sub2(zz, xz);
    const f32x2 r2 = dot3x2(dx, dy, dz, dx, dy, dz);
    const f32x2 a = dot3x2(nx, ny, nz, dx, dy, dz);
    const f32x2 b = dot3x2(mnx, mny, mnz, dx, dy, dz);   // -(n_z . d), exactly
    const float2 A = up2(a), B = up2(b), R = up2(r2), AB = up2(mul2(a, b)), R4 = up2(mul2(r2, r2));
#if OCC_DENS_MIN3
    const bool ok0 = (min3f(A.x, B.x, R.x) > 0.0f) & (R.x <= R2s);
    const bool ok1 = (min3f(A.y, B.y, R.y) > 0.0f) & (R.y <= R2s);
#else
    const bool ok0 = (A.x > 0.0f) & (B.x > 0.0f) & (R.x > 0.0f) & (R.x <= R2s);
    const bool ok1 = (A.y > 0.0f) & (B.y > 0.0f) & (R.y > 0.0f) & (R.y <= R2s);
#endif
    return make_float2(ok0 ? __fdividef(AB.x, R4.x) : 0.0f, ok1 ? __fdividef(AB.y, R4.y) : 0.0f);
}

// Eqs. 20-21 without Occ and 1/Area: the members' precomputed plane terms
// (n_L.(c - x), (x - c).e_u, (x - c).e_v) come in (h, u, v); an invalid member carries zero
// terms (s_L = 0 fails s_L > 1).  Every term is evaluated for both lanes and the support
// tests are combined at the end.
__device__ __forceinline__ float2 dens_sh_x2(f32x2 zx, f32x2 zy, f32x2 zz, f32x2 mnx, f32x2 mny,
                                             f32x2 mnz, f32x2 xx, f32x2 xy, f32x2 xz, f32x2 h,
                                             f32x2 u, f32x2 v, const RectLight& L) {
    const f32x2 dx = sub2(zx, xx), dy = sub2(zy, xy), dz = sub2(zz, xz);
    const float2 nd = up2(dot3x2(bc2(L.n.x), bc2(L.n.y), bc2(L.n.z), dx, dy, dz));
    const float2 cz = up2(dot3x2(mnx, mny, mnz, dx, dy, dz));   // -(n_z . d), exactly
    const float2 inv = make_float2(__fdividef(1.0f, nd.x), __fdividef(1.0f, nd.y));
    const f32x2 sL = mul2(h, pk2(inv.x, inv.y));
    const f32x2 du = dot3x2(dx, dy, dz, bc2(L.eu.x), bc2(L.eu.y), bc2(L.eu.z));
    const f32x2 dv = dot3x2(dx, dy, dz, bc2(L.ev.x), bc2(L.ev.y), bc2(L.ev.z));
    const float2 A = up2(mul2(fma2(sL, du, u), bc2(L.inv_eu2)));
    const float2 B = up2(mul2(fma2(sL, dv, v), bc2(L.inv_ev2)));
    const float2 J = up2(mul2(mul2(mul2(sL, sL), pk2(cz.x, cz.y)), pk2(-inv.x, -inv.y)));
    const float2 S = up2(sL);
    const bool ok0 = (nd.x < 0.0f) & (cz.x > 0.0f) & (S.x > 1.0f) & !(fabsf(A.x) > L.lim) &
                     !(fabsf(B.x) > L.lim);
    const bool ok1 = (nd.y < 0.0f) & (cz.y > 0.0f) & (S.y > 1.0f) & !(fabsf(A.y) > L.lim) &
                     !(fabsf(B.y) > L.lim);
    return make_float2(ok0 ? J.x : 0.0f, ok1 ? J.y : 0.0f);
}

template <int EFFECT>
__device__ __forceinline__ float2 dens_x2_pairs(f32x2 zx, f32x2 zy, f32x2 zz, f32x2 mnx, f32x2 mny,
                                                f32x2 mnz, f32x2 xx, f32x2 xy, f32x2 xz, f32x2 t0,
                                                f32x2 t1, f32x2 t2, float R2s, const RectLight& L) {
    if (EFFECT == kAO) return dens_ao_x2(zx, zy, zz, mnx, mny, mnz, xx, xy, xz, t0, t1, t2, R2s);
    return dens_sh_x2(zx, zy, zz, mnx, mny, mnz, xx, xy, xz, t0, t1, t2, L);
}

}  // namespace occ
