// occ_internal.h -- library-private definitions of the opaque handles of include/occ.h,
// shared by the translation units of the C ABI (occ_api.cu, occ_server.cu).
#pragma once
#include <string>

#include <cuda_runtime.h>

#include "occ.h"
#include "occ_kernels.h"

#define OCC_EXPORT extern "C" __attribute__((visibility("default")))

struct occ_ctx {
    int device = 0;
    unsigned* status = nullptr;          // device status word (kStatus* bits)
    unsigned* counter = nullptr;         // ray counter of the persistent trace kernel
    // queued first-hit validation of unbiased group reuse: query list and validation words
    // (its two counters live in the status allocation, after the ray counter)
    uint32_t* vq = nullptr;
    size_t vq_cap = 0;
    uint32_t* vbits = nullptr;
    size_t vbits_cap = 0;
    std::string last_error;
    // workspace of occ_frame_host: pos4, nrm4, records, output
    void* ws = nullptr;
    size_t ws_bytes = 0;
    occ::Tuning tune;
    // work table of occ_frame_batch: device copy, pinned staging, upload-done event
    void* batch_dev = nullptr;
    void* batch_host = nullptr;
    size_t batch_bytes = 0;
    cudaEvent_t batch_ev = nullptr;
};

struct occ_batch {
    int device = 0;
    occ::BatchView* views = nullptr;     // device
    occ::BatchDyn* dyn = nullptr;        // device
    occ::BatchDyn* dyn_host = nullptr;   // pinned
    cudaEvent_t uploaded = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_views = 0;
};

struct occ_bvh {
    int device = 0;
    occ::BvhNode* nodes = nullptr;
    float4* tris = nullptr;
    occ_bvh_stats stats{};
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};   // scene bounds
    // instrumented build only (OCC_COUNTERS): visit counters and touched-node / triangle
    // bitmaps, one allocation
    unsigned long long* ctr = nullptr;
    size_t ctr_bytes = 0;
};

namespace occ {
// argument checks of the C ABI (occ_api.cu); set ctx->last_error on failure
occ_status check_light(occ_ctx* ctx, const occ_rect_light* l);
occ_status make_pattern(occ_ctx* ctx, const occ_pattern* pat, int32_t K, PatternParams* out);
}  // namespace occ
