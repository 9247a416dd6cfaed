// occ_reuse.cuh -- definitions shared by the reuse translation units (kernels_reuse.cu and
// kernels_reuse_group.cu): the kernel arguments, the record and receiver fetches, and the
// group-kernel entry points.
#pragma once

#include <cuda_runtime.h>

#include "occ_device.cuh"
#include "occ_kernels.h"
#include "occ_path.cuh"

namespace occ {

struct ReuseArgs {
    GBufView gb;
    RecView rec;
    PatternParams pat;
    float R2s;          // AO: R^2 (1 + 2^-16)
    LightParams lp;
    DevBVH bvh;         // unbiased only
    float* out;
    unsigned* status;
    // queued first-hit validation of the group kernel (unbiased): query list, its length,
    // and one word per candidate pixel whose bit k marks a validated member k
    uint32_t* vq;
    unsigned* vcount;
    uint32_t* vbits;
    // group kernel: planes prefetched into L2 for the CTA `pf_ahead` launches later (0 none,
    // 3: G-buffer position and normal and record plane 0, 4: also record plane 1)
    int32_t pf_planes;
    int32_t pf_ahead;
};

// Passes of the queued unbiased group reuse (internal estimator codes): collect the
// (candidate, member) pairs that need Eq. 7, then estimate with the validated pairs.
constexpr int kUnbCollect = 100;
constexpr int kUnbFinal = 101;

// Receiver data of pixel q, from either G-buffer format.
template <int EFFECT>
__device__ __forceinline__ Recv fetch_recv(const GBufView& gb, int q, const RectLight& L) {
    float3 x = make_float3(0.0f, 0.0f, 0.0f), n = x;
    const bool v = gb_fetch(gb, q, &x, &n);
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

inline int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n;
}

// GROUP patterns 2x1, 2x2, 4x2, 4x4 in the warp-cooperative kernel (kernels_reuse_group.cu):
// est kBiased, kUnbiased (validation rays traced inline), kUnbCollect or kUnbFinal; false
// (nothing launched) for other shapes or mixed formats.
bool launch_group_reuse(int effect, int est, const ReuseArgs& a, cudaStream_t s);
// Persistent first-hit validation of the queued pairs (a.vq, a.vcount, a.vbits).
cudaError_t launch_validate(const ReuseArgs& a, cudaStream_t s);

}  // namespace occ
