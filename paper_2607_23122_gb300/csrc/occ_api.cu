// occ_api.cu -- the C ABI declared in include/occ.h: argument checks, ownership,
// launches on the caller's stream, and error / device-status reporting.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "occ_bvh_host.h"
#include "occ_internal.h"

namespace {

occ_status fail(occ_ctx* ctx, occ_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

occ_status cuda_fail(occ_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? OCC_ERR_OOM : OCC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

occ_status check_ctx(occ_ctx* ctx) {
    if (!ctx) return OCC_ERR_INVALID_ARG;
    const cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return OCC_OK;
}

// float4 entries of each plane of a tiled W x H G-buffer
int64_t tiled_entries(int32_t W, int32_t H) {
    return (int64_t)((W + 7) / 8) * ((H + 7) / 8) * 64;
}

occ_status check_gbuffer(occ_ctx* ctx, const occ_gbuffer* gb) {
    if (!gb) return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer is NULL");
    if (gb->W <= 0 || gb->H <= 0 || (int64_t)gb->W * gb->H > (int64_t)1 << 31)
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer size %dx%d out of range", gb->W, gb->H);
    if (gb->format != OCC_GB_FP32 && gb->format != OCC_GB_PACKED)
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer format %d invalid", gb->format);
    if (!gb->pos4 || (gb->format == OCC_GB_FP32 && !gb->nrm4))
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer pointers are NULL");
    if (!aligned16(gb->pos4) || (gb->format == OCC_GB_FP32 && !aligned16(gb->nrm4)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer pointers must be 16-byte aligned");
    if (gb->layout != OCC_LAYOUT_LINEAR && gb->layout != OCC_LAYOUT_TILED)
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer layout %d invalid", gb->layout);
    if (gb->layout == OCC_LAYOUT_TILED) {
        if (gb->pitch_px != 0)
            return fail(ctx, OCC_ERR_INVALID_ARG, "a tiled gbuffer takes pitch_px 0, not %lld",
                        (long long)gb->pitch_px);
        if (tiled_entries(gb->W, gb->H) > ((int64_t)1 << 31))
            return fail(ctx, OCC_ERR_INVALID_ARG, "tiled gbuffer %dx%d too large", gb->W, gb->H);
        return OCC_OK;
    }
    if (gb->pitch_px != 0 &&
        (gb->pitch_px < gb->W || (int64_t)(gb->H - 1) * gb->pitch_px + gb->W > ((int64_t)1 << 31)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer pitch %lld invalid for width %d",
                    (long long)gb->pitch_px, gb->W);
    return OCC_OK;
}

occ_status check_occluders(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* o) {
    if (!o) return fail(ctx, OCC_ERR_INVALID_ARG, "occluders is NULL");
    if (o->W != gb->W || o->H != gb->H)
        return fail(ctx, OCC_ERR_INVALID_ARG, "occluder size %dx%d != gbuffer size %dx%d", o->W,
                    o->H, gb->W, gb->H);
    if (o->format != OCC_REC_FP32 && o->format != OCC_REC_PACKED)
        return fail(ctx, OCC_ERR_UNSUPPORTED, "occluder format %d not supported", o->format);
    if (!o->data || !aligned16(o->data))
        return fail(ctx, OCC_ERR_INVALID_ARG, "occluder data must be a 16-byte aligned pointer");
    return OCC_OK;
}

}  // namespace

namespace occ {

occ_status check_light(occ_ctx* ctx, const occ_rect_light* l) {
    if (!l) return fail(ctx, OCC_ERR_INVALID_ARG, "light is NULL");
    double eu2 = 0, ev2 = 0, uv = 0;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(l->c[a]) || !std::isfinite(l->eu[a]) || !std::isfinite(l->ev[a]))
            return fail(ctx, OCC_ERR_INVALID_ARG, "light has non-finite values");
        eu2 += (double)l->eu[a] * l->eu[a];
        ev2 += (double)l->ev[a] * l->ev[a];
        uv += (double)l->eu[a] * l->ev[a];
    }
    if (!(eu2 > 0) || !(ev2 > 0)) return fail(ctx, OCC_ERR_INVALID_ARG, "light edges are zero");
    if (std::fabs(uv) > 1e-6 * std::sqrt(eu2 * ev2))
        return fail(ctx, OCC_ERR_INVALID_ARG, "light edges eu and ev must be orthogonal");
    return OCC_OK;
}

occ::LightParams to_params(const occ_rect_light* l) {
    occ::LightParams p{};
    if (l) {
        std::memcpy(p.c, l->c, sizeof(p.c));
        std::memcpy(p.eu, l->eu, sizeof(p.eu));
        std::memcpy(p.ev, l->ev, sizeof(p.ev));
    }
    return p;
}

occ_status make_pattern(occ_ctx* ctx, const occ_pattern* pat, int32_t K, occ::PatternParams* out) {
    if (!pat) return fail(ctx, OCC_ERR_INVALID_ARG, "pattern is NULL");
    std::memset(out, 0, sizeof(*out));
    out->kind = pat->kind;
    out->K = K;
    if (K < 1 || K > occ::kMaxMembers)
        return fail(ctx, OCC_ERR_INVALID_ARG, "K = %d must be in [1, %d]", K, occ::kMaxMembers);
    if (pat->kind == OCC_PAT_GROUP || pat->kind == OCC_PAT_BOX) {
        if (pat->gw < 1 || pat->gh < 1 || pat->gw > 64 || pat->gh > 64)
            return fail(ctx, OCC_ERR_INVALID_ARG, "pattern extent %dx%d invalid", pat->gw, pat->gh);
        if (pat->gw * pat->gh != K)
            return fail(ctx, OCC_ERR_INVALID_ARG, "K = %d != gw*gh = %d", K, pat->gw * pat->gh);
        out->gw = pat->gw;
        out->gh = pat->gh;
        const int hx0 = (pat->gw - 1) / 2, hy0 = (pat->gh - 1) / 2;
        out->halo[0] = hx0;
        out->halo[1] = pat->gw / 2;
        out->halo[2] = hy0;
        out->halo[3] = pat->gh / 2;
    } else if (pat->kind == OCC_PAT_OFFSETS) {
        if (pat->n_offsets != K - 1)
            return fail(ctx, OCC_ERR_INVALID_ARG, "K = %d != n_offsets + 1 = %d", K, pat->n_offsets + 1);
        if (pat->n_offsets > 0 && !pat->offsets_host)
            return fail(ctx, OCC_ERR_INVALID_ARG, "offsets_host is NULL");
        out->gw = out->gh = 1;
        out->n_off = pat->n_offsets;
        for (int a = 0; a < pat->n_offsets; ++a) {
            const int dx = pat->offsets_host[2 * a], dy = pat->offsets_host[2 * a + 1];
            if (dx == 0 && dy == 0)
                return fail(ctx, OCC_ERR_INVALID_ARG, "offset %d is (0, 0)", a);
            if (dx < -256 || dx > 256 || dy < -256 || dy > 256)
                return fail(ctx, OCC_ERR_INVALID_ARG, "offset %d out of [-256, 256]", a);
            for (int b = 0; b < a; ++b)
                if (pat->offsets_host[2 * b] == dx && pat->offsets_host[2 * b + 1] == dy)
                    return fail(ctx, OCC_ERR_INVALID_ARG, "offset %d repeats offset %d", a, b);
            out->off[a] = make_int2(dx, dy);
            out->halo[0] = std::max(out->halo[0], -dx);
            out->halo[1] = std::max(out->halo[1], dx);
            out->halo[2] = std::max(out->halo[2], -dy);
            out->halo[3] = std::max(out->halo[3], dy);
        }
    } else if (pat->kind == OCC_PAT_RANDOM) {
        if (pat->n_offsets != K - 1)
            return fail(ctx, OCC_ERR_INVALID_ARG, "K = %d != n_offsets + 1 = %d", K, pat->n_offsets + 1);
        if (pat->radius_px < 1 || pat->radius_px > 64)
            return fail(ctx, OCC_ERR_INVALID_ARG, "radius_px = %d must be in [1, 64]", pat->radius_px);
        out->gw = out->gh = 1;
        out->n_off = pat->n_offsets;
        out->radius = pat->radius_px;
        out->seed = pat->seed;
        for (int i = 0; i < 4; ++i) out->halo[i] = pat->radius_px;
    } else {
        return fail(ctx, OCC_ERR_INVALID_ARG, "pattern kind %d invalid", pat->kind);
    }
    return OCC_OK;
}

}  // namespace occ

namespace {

using occ::check_light;
using occ::make_pattern;
using occ::to_params;

occ::GBufView view(const occ_gbuffer* gb) {
    return occ::GBufView{gb->W, gb->H, reinterpret_cast<const float4*>(gb->pos4),
                         reinterpret_cast<const float4*>(gb->nrm4), gb->format == OCC_GB_PACKED,
                         gb->pitch_px ? (int32_t)gb->pitch_px : gb->W,
                         gb->layout == OCC_LAYOUT_TILED ? 1 : 0};
}

occ::RecView rec_view(const occ_occluders* o) {
    float4* base = reinterpret_cast<float4*>(o->data);
    if (o->format == OCC_REC_PACKED) return occ::RecView{base, nullptr, 1};
    return occ::RecView{base, base + (size_t)o->W * o->H, 0};
}

occ::DevBVH dev_bvh(const occ_bvh* b) {
    occ::DevBVH d{b->nodes, b->tris, (uint32_t)b->stats.num_nodes, (uint32_t)b->stats.num_tris};
#if OCC_COUNTERS
    if (b->ctr) {
        d.ctr = b->ctr;
        d.node_bits = reinterpret_cast<uint32_t*>(b->ctr + 2);
        d.tri_bits = d.node_bits + (b->stats.num_nodes + 31) / 32;
    }
#endif
    return d;
}

occ_status launched(occ_ctx* ctx, cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return OCC_OK;
}

// 1: unbiased group reuse queues its first-hit validation rays for a persistent trace
// kernel; 0: the group kernel traces them inline.
#ifndef OCC_VALIDATE_QUEUE
#define OCC_VALIDATE_QUEUE 1
#endif

occ_status reuse_common(occ_ctx* ctx, int effect, const occ_gbuffer* gb, const occ_occluders* occ,
                        const occ_pattern* pattern, int32_t K, int32_t estimator,
                        const occ_bvh* bvh, float* out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if ((st = check_occluders(ctx, gb, occ)) != OCC_OK) return st;
    if (occ->effect != effect)
        return fail(ctx, OCC_ERR_INVALID_ARG, "occluder records were traced for effect %d, not %d",
                    occ->effect, effect);
    if (estimator < OCC_EST_NOREUSE || estimator > OCC_EST_LIGHT_UNBIASED)
        return fail(ctx, OCC_ERR_INVALID_ARG, "estimator %d invalid", estimator);
    if (estimator == OCC_EST_LIGHT_UNBIASED && effect != OCC_EFFECT_SHADOW)
        return fail(ctx, OCC_ERR_INVALID_ARG, "light-sample reuse is defined for shadows only");
    const bool traces = estimator == OCC_EST_UNBIASED || estimator == OCC_EST_LIGHT_UNBIASED;
    if (traces && !bvh)
        return fail(ctx, OCC_ERR_INVALID_ARG, "the unbiased estimators need the BVH");
    if (!traces && bvh)
        return fail(ctx, OCC_ERR_INVALID_ARG, "bvh_or_null must be NULL unless the estimator is unbiased");
    if (!out) return fail(ctx, OCC_ERR_INVALID_ARG, "out is NULL");
    if (effect == OCC_EFFECT_SHADOW && (st = check_light(ctx, &occ->light)) != OCC_OK) return st;
    if (effect == OCC_EFFECT_AO && !(occ->radius > 0.0f && std::isfinite(occ->radius)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "AO radius must be positive and finite");
    occ::PatternParams pat;
    if ((st = make_pattern(ctx, pattern, K, &pat)) != OCC_OK) return st;
    pat.sample = occ->sample;
    const occ::DevBVH b = bvh ? dev_bvh(bvh) : occ::DevBVH{nullptr, nullptr};
    const occ::LightParams lp = to_params(&occ->light);
    occ::ValidateWs vws{nullptr, 0, nullptr, 0, nullptr};
    if (OCC_VALIDATE_QUEUE && estimator == OCC_EST_UNBIASED && pat.kind == OCC_PAT_GROUP &&
        pat.K <= 16) {
        // queued validation: (K - 1) query words and one validation word per pixel, grown
        // on demand (a context's calls run in order on the device, so the previous contents
        // are no longer needed once cudaFree returns)
        const size_t P = (size_t)gb->W * gb->H, nq = (size_t)(pat.K - 1) * P;
        if (nq > ctx->vq_cap || P > ctx->vbits_cap) {
            cudaFree(ctx->vq);
            cudaFree(ctx->vbits);
            ctx->vq = nullptr;
            ctx->vbits = nullptr;
            ctx->vq_cap = ctx->vbits_cap = 0;
            cudaError_t e = cudaMalloc(&ctx->vq, (nq > 0 ? nq : 1) * sizeof(uint32_t));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->vbits, P * sizeof(uint32_t));
            if (e != cudaSuccess) {
                cudaFree(ctx->vq);
                ctx->vq = nullptr;
                return cuda_fail(ctx, e, "validation workspace");
            }
            ctx->vq_cap = nq;
            ctx->vbits_cap = P;
        }
        vws = occ::ValidateWs{ctx->vq, ctx->vq_cap, ctx->vbits, ctx->vbits_cap, ctx->counter + 1};
    }
    return launched(ctx,
                    occ::launch_reuse(effect, estimator, view(gb), rec_view(occ), pat, occ->radius,
                                      lp, bvh ? &b : nullptr, out, ctx->status,
                                      (cudaStream_t)stream, ctx->tune, occ->seed, occ->sample,
                                      vws.queue ? &vws : nullptr),
                    "reuse launch");
}

occ_status trace_common(occ_ctx* ctx, int effect, const occ_gbuffer* gb, const occ_bvh* bvh,
                        float radius, const occ_rect_light* light, uint64_t seed, uint32_t sample,
                        occ_occluders* out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if (!bvh) return fail(ctx, OCC_ERR_INVALID_ARG, "bvh is NULL");
    if (bvh->device != ctx->device)
        return fail(ctx, OCC_ERR_INVALID_ARG, "bvh lives on device %d, context on %d", bvh->device,
                    ctx->device);
    if ((st = check_occluders(ctx, gb, out)) != OCC_OK) return st;
    if (effect == OCC_EFFECT_AO && !(radius > 0.0f && std::isfinite(radius)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "AO radius must be positive and finite");
    if (effect == OCC_EFFECT_SHADOW && (st = check_light(ctx, light)) != OCC_OK) return st;
    out->effect = effect;
    out->radius = effect == OCC_EFFECT_AO ? radius : 0.0f;
    if (effect == OCC_EFFECT_SHADOW)
        out->light = *light;
    else
        std::memset(&out->light, 0, sizeof(out->light));
    out->seed = seed;
    out->sample = sample;
    return launched(ctx,
                    occ::launch_trace(effect, view(gb), dev_bvh(bvh), radius, to_params(light), seed,
                                      sample, rec_view(out), ctx->status, (cudaStream_t)stream,
                                      ctx->counter, &ctx->tune),
                    "trace launch");
}

occ_status trace_reuse_common(occ_ctx* ctx, int effect, const occ_gbuffer* gb, const occ_bvh* bvh,
                              float radius, const occ_rect_light* light, uint64_t seed,
                              uint32_t sample, const occ_pattern* pattern, int32_t K,
                              int32_t estimator, occ_occluders* rec, float* out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if (!bvh) return fail(ctx, OCC_ERR_INVALID_ARG, "bvh is NULL");
    if (bvh->device != ctx->device)
        return fail(ctx, OCC_ERR_INVALID_ARG, "bvh lives on device %d, context on %d", bvh->device,
                    ctx->device);
    if (rec && (st = check_occluders(ctx, gb, rec)) != OCC_OK) return st;
    if (!out) return fail(ctx, OCC_ERR_INVALID_ARG, "out is NULL");
    if (effect == OCC_EFFECT_AO && !(radius > 0.0f && std::isfinite(radius)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "AO radius must be positive and finite");
    if (effect == OCC_EFFECT_SHADOW && (st = check_light(ctx, light)) != OCC_OK) return st;
    if (estimator < OCC_EST_NOREUSE || estimator > OCC_EST_BOXMEAN)
        return fail(ctx, OCC_ERR_INVALID_ARG, "estimator %d invalid for the fused pass", estimator);
    occ::PatternParams pat;
    if ((st = make_pattern(ctx, pattern, K, &pat)) != OCC_OK) return st;
    if (pat.kind != OCC_PAT_GROUP || !occ::frame_group_shape(pat.gw, pat.gh))
        return fail(ctx, OCC_ERR_UNSUPPORTED,
                    "the fused pass takes GROUP patterns 2x1, 2x2, 4x2 or 4x4 (got kind %d, %dx%d)",
                    pat.kind, pat.gw, pat.gh);
    occ::RecView rv{nullptr, nullptr, 0};
    if (rec) {
        rec->effect = effect;
        rec->radius = effect == OCC_EFFECT_AO ? radius : 0.0f;
        if (effect == OCC_EFFECT_SHADOW)
            rec->light = *light;
        else
            std::memset(&rec->light, 0, sizeof(rec->light));
        rec->seed = seed;
        rec->sample = sample;
        rv = rec_view(rec);
    }
    return launched(ctx,
                    occ::launch_trace_reuse(effect, estimator, view(gb), dev_bvh(bvh), radius,
                                            to_params(light), seed, sample, pat.gw, pat.gh, rv, out,
                                            ctx->status, (cudaStream_t)stream, ctx->counter,
                                            ctx->tune.fused_ao_path),
                    "fused trace + reuse launch");
}

}  // namespace

OCC_EXPORT const char* occ_version(void) { return "occreuse 0.1 (sm_103a)"; }

OCC_EXPORT occ_status occ_create(int device, occ_ctx** out) {
    if (!out) return OCC_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return OCC_ERR_INVALID_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return OCC_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return OCC_ERR_UNSUPPORTED;
    if (cudaSetDevice(device) != cudaSuccess) return OCC_ERR_CUDA;
    occ_ctx* ctx = new occ_ctx();
    ctx->device = device;
    // status word (word 0), ray counter (word 8), validation counters (words 9, 10)
    cudaError_t e = cudaMalloc(&ctx->status, 64);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, 64);
    ctx->counter = ctx->status + 8;
    if (e != cudaSuccess) {
        cudaFree(ctx->status);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? OCC_ERR_OOM : OCC_ERR_CUDA;
    }
    *out = ctx;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_destroy(occ_ctx* ctx) {
    if (!ctx) return OCC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->status);
    cudaFree(ctx->vq);
    cudaFree(ctx->vbits);
    cudaFree(ctx->ws);
    cudaFree(ctx->batch_dev);
    cudaFreeHost(ctx->batch_host);
    if (ctx->batch_ev) cudaEventDestroy(ctx->batch_ev);
    delete ctx;
    return OCC_OK;
}

OCC_EXPORT const char* occ_last_error(const occ_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : "context is NULL";
}

OCC_EXPORT occ_status occ_sync(occ_ctx* ctx, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream");
    unsigned flags = 0;
    e = cudaMemcpy(&flags, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (flags) {
        cudaMemset(ctx->status, 0, sizeof(unsigned));
        return fail(ctx, OCC_ERR_DEVICE_CHECK, "device check flags 0x%x (%s%s%s)", flags,
                    (flags & occ::kStatusStackOverflowBit) ? "stack overflow " : "",
                    (flags & occ::kStatusWaitTimeoutBit) ? "wait timeout " : "",
                    (flags & occ::kStatusBadIndexBit) ? "bad index" : "");
    }
    return OCC_OK;
}

OCC_EXPORT occ_status occ_trace_reuse_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                                         float radius, uint64_t seed, uint32_t sample,
                                         const occ_pattern* pattern, int32_t K, int32_t estimator,
                                         occ_occluders* occ_or_null, float* out, void* stream) {
    return trace_reuse_common(ctx, OCC_EFFECT_AO, gb, bvh, radius, nullptr, seed, sample, pattern,
                              K, estimator, occ_or_null, out, stream);
}

OCC_EXPORT occ_status occ_trace_reuse_shadow(occ_ctx* ctx, const occ_gbuffer* gb,
                                             const occ_bvh* bvh, const occ_rect_light* light,
                                             uint64_t seed, uint32_t sample,
                                             const occ_pattern* pattern, int32_t K,
                                             int32_t estimator, occ_occluders* occ_or_null,
                                             float* out, void* stream) {
    return trace_reuse_common(ctx, OCC_EFFECT_SHADOW, gb, bvh, 0.0f, light, seed, sample, pattern,
                              K, estimator, occ_or_null, out, stream);
}

OCC_EXPORT occ_status occ_debug_bvh_host(const float* tris_host, int64_t T, float* nodes_out,
                                         int64_t nodes_cap, float* tris_out, int64_t tris_cap,
                                         int64_t* n_nodes, int32_t* depth) {
    if (!tris_host || T <= 0 || !n_nodes || !depth) return OCC_ERR_INVALID_ARG;
    occ::HostBVH hb;
    std::string err;
    if (!occ::build_bvh4(tris_host, T, &hb, &err)) return OCC_ERR_INVALID_ARG;
    *n_nodes = (int64_t)hb.nodes.size();
    *depth = hb.depth;
    if (!nodes_out) return OCC_OK;
    if (nodes_cap < (int64_t)hb.nodes.size() || !tris_out || tris_cap < T ||
        sizeof(occ::BvhNode) != 128)
        return OCC_ERR_INVALID_ARG;
    std::memcpy(nodes_out, hb.nodes.data(), hb.nodes.size() * sizeof(occ::BvhNode));
    std::memcpy(tris_out, hb.tris.data(), hb.tris.size() * sizeof(float4));
    return OCC_OK;
}

OCC_EXPORT occ_status occ_bvh_build(occ_ctx* ctx, const float* tris_host, int64_t T, occ_bvh** out) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!out || !tris_host || T <= 0) return fail(ctx, OCC_ERR_INVALID_ARG, "bad bvh_build arguments");
    *out = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    occ::HostBVH hb;
    std::string err;
    if (!occ::build_bvh4(tris_host, T, &hb, &err)) return fail(ctx, OCC_ERR_INVALID_ARG, "%s", err.c_str());
    occ_bvh* b = new occ_bvh();
    b->device = ctx->device;
    const size_t nb = hb.nodes.size() * sizeof(occ::BvhNode), tb = hb.tris.size() * sizeof(float4);
    cudaError_t e = cudaMalloc(&b->nodes, nb);
    if (e == cudaSuccess) e = cudaMalloc(&b->tris, tb);
    if (e == cudaSuccess) e = cudaMemcpy(b->nodes, hb.nodes.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tris, hb.tris.data(), tb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->nodes);
        cudaFree(b->tris);
        delete b;
        return cuda_fail(ctx, e, "bvh upload");
    }
    for (int a = 0; a < 3; ++a) {
        b->lo[a] = tris_host[a];
        b->hi[a] = tris_host[a];
    }
    for (int64_t i = 0; i < 3 * T; ++i)
        for (int a = 0; a < 3; ++a) {
            b->lo[a] = std::min(b->lo[a], tris_host[3 * i + a]);
            b->hi[a] = std::max(b->hi[a], tris_host[3 * i + a]);
        }
    b->stats.num_tris = T;
    b->stats.num_nodes = (int64_t)hb.nodes.size();
    b->stats.num_leaves = hb.num_leaves;
    b->stats.depth = hb.depth;
    b->stats.max_leaf_tris = hb.max_leaf_tris;
    b->stats.bytes = (int64_t)(nb + tb);
    b->stats.build_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (OCC_COUNTERS) {
        // two 64-bit counters, then one bit per node and one per triangle slot
        b->ctr_bytes = 16 + 4 * (size_t)((b->stats.num_nodes + 31) / 32 + (T + 31) / 32);
        e = cudaMalloc(&b->ctr, b->ctr_bytes);
        if (e == cudaSuccess) e = cudaMemset(b->ctr, 0, b->ctr_bytes);
        if (e != cudaSuccess) {
            cudaFree(b->ctr);
            cudaFree(b->nodes);
            cudaFree(b->tris);
            delete b;
            return cuda_fail(ctx, e, "bvh counters");
        }
    }
    *out = b;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_bvh_free(occ_ctx* ctx, occ_bvh* bvh) {
    if (!ctx || !bvh) return OCC_ERR_INVALID_ARG;
    cudaSetDevice(bvh->device);
    cudaFree(bvh->nodes);
    cudaFree(bvh->tris);
    cudaFree(bvh->ctr);
    delete bvh;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_bvh_info(const occ_bvh* bvh, occ_bvh_stats* out) {
    if (!bvh || !out) return OCC_ERR_INVALID_ARG;
    *out = bvh->stats;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_gbuffer_pinhole(occ_ctx* ctx, const occ_bvh* bvh, const float* cam_host,
                                          float eps, int32_t W, int32_t H, float* pos4,
                                          float* nrm4, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!bvh || !cam_host || !pos4 || W <= 0 || H <= 0 || !std::isfinite(eps))
        return fail(ctx, OCC_ERR_INVALID_ARG, "bad gbuffer_pinhole arguments");
    if (!aligned16(pos4) || (nrm4 && !aligned16(nrm4)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "gbuffer pointers must be 16-byte aligned");
    if (!(cam_host[9] > 0.0f && cam_host[9] < 180.0f))
        return fail(ctx, OCC_ERR_INVALID_ARG, "vertical fov must be in (0, 180) degrees");
    return launched(ctx,
                    occ::launch_gbuffer(dev_bvh(bvh), cam_host, eps, W, H,
                                        reinterpret_cast<float4*>(pos4),
                                        reinterpret_cast<float4*>(nrm4), ctx->status,
                                        (cudaStream_t)stream),
                    "gbuffer launch");
}

OCC_EXPORT occ_status occ_pack_gbuffer(occ_ctx* ctx, const occ_gbuffer* gb, float* packed_out,
                                       void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if (gb->format != OCC_GB_FP32)
        return fail(ctx, OCC_ERR_INVALID_ARG, "occ_pack_gbuffer needs an FP32 G-buffer");
    if (!packed_out || !aligned16(packed_out))
        return fail(ctx, OCC_ERR_INVALID_ARG, "packed_out must be a 16-byte aligned pointer");
    return launched(ctx,
                    occ::launch_pack_gbuffer(view(gb), reinterpret_cast<float4*>(packed_out),
                                             (cudaStream_t)stream),
                    "pack launch");
}

OCC_EXPORT occ_status occ_tile_gbuffer(occ_ctx* ctx, const occ_gbuffer* gb, float* pos_out,
                                       float* nrm_out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    const bool fp32 = gb->format == OCC_GB_FP32;
    if (!pos_out || !aligned16(pos_out) || (fp32 && (!nrm_out || !aligned16(nrm_out))) ||
        (!fp32 && nrm_out))
        return fail(ctx, OCC_ERR_INVALID_ARG,
                    "occ_tile_gbuffer needs 16-byte aligned pos_out (and nrm_out for FP32 only)");
    if (tiled_entries(gb->W, gb->H) > ((int64_t)1 << 31))
        return fail(ctx, OCC_ERR_INVALID_ARG, "tiled gbuffer %dx%d too large", gb->W, gb->H);
    // byte ranges: the input planes and the outputs must not overlap
    const int64_t out_bytes = tiled_entries(gb->W, gb->H) * 16;
    const int64_t in_bytes = 16 * (gb->layout == OCC_LAYOUT_TILED
                                       ? tiled_entries(gb->W, gb->H)
                                       : (int64_t)(gb->H - 1) * (gb->pitch_px ? gb->pitch_px : gb->W) + gb->W);
    auto overlap = [](const void* a, int64_t an, const void* b, int64_t bn) {
        const char *pa = static_cast<const char*>(a), *pb = static_cast<const char*>(b);
        return a && b && pa < pb + bn && pb < pa + an;
    };
    if (overlap(pos_out, out_bytes, gb->pos4, in_bytes) || overlap(pos_out, out_bytes, gb->nrm4, in_bytes) ||
        overlap(nrm_out, out_bytes, gb->pos4, in_bytes) || overlap(nrm_out, out_bytes, gb->nrm4, in_bytes) ||
        overlap(pos_out, out_bytes, nrm_out, out_bytes))
        return fail(ctx, OCC_ERR_INVALID_ARG, "occ_tile_gbuffer outputs overlap its input or each other");
    return launched(ctx,
                    occ::launch_tile_gbuffer(view(gb), reinterpret_cast<float4*>(pos_out),
                                             reinterpret_cast<float4*>(nrm_out), (cudaStream_t)stream),
                    "tile launch");
}

OCC_EXPORT occ_status occ_trace_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                                   float radius, uint64_t seed, uint32_t sample,
                                   occ_occluders* out, void* stream) {
    return trace_common(ctx, OCC_EFFECT_AO, gb, bvh, radius, nullptr, seed, sample, out, stream);
}

OCC_EXPORT occ_status occ_trace_shadow(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                                       const occ_rect_light* light, uint64_t seed, uint32_t sample,
                                       occ_occluders* out, void* stream) {
    return trace_common(ctx, OCC_EFFECT_SHADOW, gb, bvh, 0.0f, light, seed, sample, out, stream);
}

OCC_EXPORT occ_status occ_reuse_ao(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                                   const occ_pattern* pattern, int32_t K, int32_t estimator,
                                   const occ_bvh* bvh_or_null, float* out, void* stream) {
    return reuse_common(ctx, OCC_EFFECT_AO, gb, occ, pattern, K, estimator, bvh_or_null, out, stream);
}

OCC_EXPORT occ_status occ_reuse_shadow(occ_ctx* ctx, const occ_gbuffer* gb,
                                       const occ_occluders* occ, const occ_pattern* pattern,
                                       int32_t K, int32_t estimator, const occ_bvh* bvh_or_null,
                                       float* out, void* stream) {
    return reuse_common(ctx, OCC_EFFECT_SHADOW, gb, occ, pattern, K, estimator, bvh_or_null, out,
                        stream);
}

namespace {

// Copies, trace, reuse and the estimate's download of one host frame, enqueued on `stream`.
occ_status frame_host_enqueue(occ_ctx* ctx, const occ_bvh* bvh, int32_t effect,
                              const float* pos4_host, const float* nrm4_host, int32_t W, int32_t H,
                              float radius, const occ_rect_light* light, uint64_t seed,
                              uint32_t sample, const occ_pattern* pattern, int32_t K,
                              int32_t estimator, float* out_host, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!bvh || !pos4_host || !nrm4_host || !out_host || W <= 0 || H <= 0)
        return fail(ctx, OCC_ERR_INVALID_ARG, "bad frame_host arguments");
    if (effect != OCC_EFFECT_AO && effect != OCC_EFFECT_SHADOW)
        return fail(ctx, OCC_ERR_INVALID_ARG, "effect %d invalid", effect);
    const size_t P = (size_t)W * H;
    const size_t need = P * (16 + 16 + 32 + 4) + 256;
    if (need > ctx->ws_bytes) {
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        const cudaError_t e = cudaMalloc(&ctx->ws, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "frame workspace");
        ctx->ws_bytes = need;
    }
    char* base = reinterpret_cast<char*>(ctx->ws);
    float* pos = reinterpret_cast<float*>(base);
    float* nrm = reinterpret_cast<float*>(base + 16 * P);
    void* recs = base + 32 * P;
    float* out = reinterpret_cast<float*>(base + 64 * P);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(pos, pos4_host, 16 * P, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nrm, nrm4_host, 16 * P, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame upload");
    occ_gbuffer gb{W, H, pos, nrm};
    occ_occluders oc{};
    oc.W = W;
    oc.H = H;
    oc.format = OCC_REC_FP32;
    oc.data = recs;
    st = effect == OCC_EFFECT_AO ? occ_trace_ao(ctx, &gb, bvh, radius, seed, sample, &oc, stream)
                                 : occ_trace_shadow(ctx, &gb, bvh, light, seed, sample, &oc, stream);
    if (st != OCC_OK) return st;
    const occ_bvh* vb =
        estimator == OCC_EST_UNBIASED || estimator == OCC_EST_LIGHT_UNBIASED ? bvh : nullptr;
    st = effect == OCC_EFFECT_AO
             ? occ_reuse_ao(ctx, &gb, &oc, pattern, K, estimator, vb, out, stream)
             : occ_reuse_shadow(ctx, &gb, &oc, pattern, K, estimator, vb, out, stream);
    if (st != OCC_OK) return st;
    e = cudaMemcpyAsync(out_host, out, 4 * P, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "frame download");
    return OCC_OK;
}

}  // namespace

OCC_EXPORT occ_status occ_frame_host(occ_ctx* ctx, const occ_bvh* bvh, int32_t effect,
                                     const float* pos4_host, const float* nrm4_host, int32_t W,
                                     int32_t H, float radius, const occ_rect_light* light,
                                     uint64_t seed, uint32_t sample, const occ_pattern* pattern,
                                     int32_t K, int32_t estimator, float* out_host, void* stream) {
    const occ_status st = frame_host_enqueue(ctx, bvh, effect, pos4_host, nrm4_host, W, H, radius,
                                             light, seed, sample, pattern, K, estimator, out_host,
                                             stream);
    if (st != OCC_OK) return st;
    return occ_sync(ctx, stream);
}

OCC_EXPORT occ_status occ_frame_host_async(occ_ctx* ctx, const occ_bvh* bvh, int32_t effect,
                                           const float* pos4_host, const float* nrm4_host,
                                           int32_t W, int32_t H, float radius,
                                           const occ_rect_light* light, uint64_t seed,
                                           uint32_t sample, const occ_pattern* pattern, int32_t K,
                                           int32_t estimator, float* out_host, void* stream) {
    return frame_host_enqueue(ctx, bvh, effect, pos4_host, nrm4_host, W, H, radius, light, seed,
                              sample, pattern, K, estimator, out_host, stream);
}

OCC_EXPORT occ_status occ_shadow_lights(occ_ctx* ctx, const occ_gbuffer* gb, const occ_bvh* bvh,
                                        const occ_rect_light* lights_host, const float* weights_host,
                                        int32_t n_lights, uint64_t seed, uint32_t sample,
                                        const occ_pattern* pattern, int32_t K, int32_t estimator,
                                        occ_occluders* recs, float* vis, float* out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if (!lights_host || !weights_host || !recs || !vis || !out)
        return fail(ctx, OCC_ERR_INVALID_ARG, "lights, weights, recs, vis and out must be set");
    if (n_lights < 1 || n_lights > occ::kMaxLights)
        return fail(ctx, OCC_ERR_INVALID_ARG, "n_lights must be in [1, %d]", occ::kMaxLights);
    occ::LightWeights w{};
    w.n = n_lights;
    for (int l = 0; l < n_lights; ++l) {
        if (!std::isfinite(weights_host[l]))
            return fail(ctx, OCC_ERR_INVALID_ARG, "weight %d is not finite", l);
        if ((st = check_light(ctx, &lights_host[l])) != OCC_OK) return st;
        w.w[l] = weights_host[l];
    }
    const int64_t P = (int64_t)gb->W * gb->H;
    const bool traces = estimator == OCC_EST_UNBIASED || estimator == OCC_EST_LIGHT_UNBIASED;
    for (int l = 0; l < n_lights; ++l) {
        st = occ_trace_shadow(ctx, gb, bvh, &lights_host[l], seed + (uint64_t)l, sample, &recs[l],
                              stream);
        if (st == OCC_OK)
            st = occ_reuse_shadow(ctx, gb, &recs[l], pattern, K, estimator, traces ? bvh : nullptr,
                                  vis + (size_t)l * P, stream);
        if (st != OCC_OK) return st;
    }
    return launched(ctx, occ::launch_weighted_sum(vis, P, w, out, (cudaStream_t)stream),
                    "weighted sum");
}

OCC_EXPORT occ_status occ_debug_philox(occ_ctx* ctx, const uint32_t* in_dev, int64_t n,
                                       uint32_t* out_dev, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (n < 0 || (n > 0 && (!in_dev || !out_dev))) return fail(ctx, OCC_ERR_INVALID_ARG, "bad arguments");
    return launched(ctx, occ::launch_debug_philox(in_dev, n, out_dev, (cudaStream_t)stream),
                    "philox launch");
}

OCC_EXPORT occ_status occ_debug_closest_hit(occ_ctx* ctx, const occ_bvh* bvh, const float* rays_dev,
                                            int64_t n, int32_t any, int32_t* tri_dev, float* t_dev,
                                            void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!bvh || n < 0 || (n > 0 && (!rays_dev || !tri_dev || !t_dev)) || !aligned16(rays_dev))
        return fail(ctx, OCC_ERR_INVALID_ARG, "bad debug_closest_hit arguments");
    return launched(ctx,
                    occ::launch_debug_closest_hit(dev_bvh(bvh), reinterpret_cast<const float4*>(rays_dev),
                                                  n, any != 0, tri_dev, t_dev, ctx->status,
                                                  (cudaStream_t)stream),
                    "debug_closest_hit launch");
}

OCC_EXPORT occ_status occ_debug_fp32_peak(occ_ctx* ctx, int32_t paired, int32_t iters,
                                          int32_t blocks, float* sink_dev, double* flop_host,
                                          void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((paired != 0 && paired != 1) || iters < 1 || iters > (1 << 24) || blocks < 1 ||
        blocks > (1 << 20) || !sink_dev || !flop_host)
        return fail(ctx, OCC_ERR_INVALID_ARG, "bad fp32_peak arguments");
    return launched(ctx,
                    occ::launch_fp32_peak(paired, iters, blocks, sink_dev, flop_host,
                                          (cudaStream_t)stream),
                    "fp32 probe launch");
}

OCC_EXPORT occ_status occ_debug_stream_ceiling(occ_ctx* ctx, const occ_gbuffer* gb,
                                               const occ_occluders* occ, float* out, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if ((st = check_occluders(ctx, gb, occ)) != OCC_OK) return st;
    if (gb->format != OCC_GB_FP32 || occ->format != OCC_REC_FP32)
        return fail(ctx, OCC_ERR_UNSUPPORTED, "the streaming probe reads FP32 G-buffers and records");
    if (!out) return fail(ctx, OCC_ERR_INVALID_ARG, "out is NULL");
    return launched(ctx, occ::launch_stream_ceiling(view(gb), rec_view(occ), out, (cudaStream_t)stream),
                    "stream probe launch");
}

OCC_EXPORT occ_status occ_debug_bvh_counters(occ_ctx* ctx, const occ_bvh* bvh, int32_t reset,
                                             uint64_t* out_host) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!bvh || !out_host) return fail(ctx, OCC_ERR_INVALID_ARG, "bad bvh_counters arguments");
    if (!OCC_COUNTERS || !bvh->ctr)
        return fail(ctx, OCC_ERR_UNSUPPORTED,
                    "traversal counters need the instrumented library (OCC_COUNTERS=1)");
    cudaError_t e = cudaDeviceSynchronize();
    std::vector<uint32_t> words(bvh->ctr_bytes / 4);
    if (e == cudaSuccess) e = cudaMemcpy(words.data(), bvh->ctr, bvh->ctr_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counter read");
    uint64_t visits[2];
    std::memcpy(visits, words.data(), 16);
    const size_t nw = (size_t)(bvh->stats.num_nodes + 31) / 32;
    uint64_t nodes = 0, tris = 0;
    for (size_t i = 0; i < nw; ++i) nodes += (uint64_t)__builtin_popcount(words[4 + i]);
    for (size_t i = 4 + nw; i < words.size(); ++i) tris += (uint64_t)__builtin_popcount(words[i]);
    out_host[0] = visits[0];
    out_host[1] = visits[1];
    out_host[2] = nodes;
    out_host[3] = tris;
    out_host[4] = nodes * sizeof(occ::BvhNode) + tris * 3 * sizeof(float4);
    if (reset) {
        e = cudaMemset(bvh->ctr, 0, bvh->ctr_bytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "counter reset");
    }
    return OCC_OK;
}

OCC_EXPORT occ_status occ_debug_wait_timeout(occ_ctx* ctx, uint32_t spins, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (spins < 1 || spins > (1u << 24)) return fail(ctx, OCC_ERR_INVALID_ARG, "spins must be in [1, 2^24]");
    return launched(ctx, occ::launch_debug_wait_timeout(spins, ctx->status, (cudaStream_t)stream),
                    "wait-timeout launch");
}

OCC_EXPORT occ_status occ_debug_rays(occ_ctx* ctx, const occ_gbuffer* gb, int32_t effect,
                                     float radius, const occ_rect_light* light, uint64_t seed,
                                     uint32_t sample, float* out_dev, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if (!out_dev || !aligned16(out_dev)) return fail(ctx, OCC_ERR_INVALID_ARG, "bad out_dev");
    if (effect == OCC_EFFECT_SHADOW && (st = check_light(ctx, light)) != OCC_OK) return st;
    return launched(ctx,
                    occ::launch_debug_rays(effect, view(gb), radius, to_params(light), seed, sample,
                                           reinterpret_cast<float4*>(out_dev), (cudaStream_t)stream),
                    "rays launch");
}

OCC_EXPORT occ_status occ_debug_mis(occ_ctx* ctx, const occ_gbuffer* gb, const occ_occluders* occ,
                                    const occ_pattern* pattern, int32_t K, int32_t estimator,
                                    const occ_bvh* bvh_or_null, const int32_t* pix_host, int32_t n,
                                    int32_t* members_host, float* w_host) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if ((st = check_gbuffer(ctx, gb)) != OCC_OK) return st;
    if ((st = check_occluders(ctx, gb, occ)) != OCC_OK) return st;
    if (n < 0 || (n > 0 && (!pix_host || !members_host || !w_host)))
        return fail(ctx, OCC_ERR_INVALID_ARG, "bad debug_mis arguments");
    if (estimator != OCC_EST_BIASED && estimator != OCC_EST_UNBIASED)
        return fail(ctx, OCC_ERR_INVALID_ARG, "debug_mis needs the biased or unbiased estimator");
    if (estimator == OCC_EST_UNBIASED && !bvh_or_null)
        return fail(ctx, OCC_ERR_INVALID_ARG, "the unbiased estimator needs the BVH");
    for (int i = 0; i < n; ++i)
        if (pix_host[i] < 0 || pix_host[i] >= gb->W * gb->H)
            return fail(ctx, OCC_ERR_INVALID_ARG, "pixel %d out of range", pix_host[i]);
    occ::PatternParams pat;
    if ((st = make_pattern(ctx, pattern, K, &pat)) != OCC_OK) return st;
    pat.sample = occ->sample;
    if (n == 0) return OCC_OK;
    const size_t wn = (size_t)n * occ::kMaxMembers * occ::kMaxMembers;
    int32_t *d_pix = nullptr, *d_mem = nullptr;
    float* d_w = nullptr;
    cudaError_t e = cudaMalloc(&d_pix, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_mem, sizeof(int32_t) * n * occ::kMaxMembers);
    if (e == cudaSuccess) e = cudaMalloc(&d_w, sizeof(float) * wn);
    if (e == cudaSuccess) e = cudaMemcpy(d_pix, pix_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    const occ::DevBVH b = bvh_or_null ? dev_bvh(bvh_or_null) : occ::DevBVH{nullptr, nullptr};
    if (e == cudaSuccess)
        e = occ::launch_debug_mis(occ->effect, estimator, view(gb), rec_view(occ), pat, occ->radius,
                                  to_params(&occ->light), bvh_or_null ? &b : nullptr, d_pix, n,
                                  d_mem, d_w, ctx->status, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(members_host, d_mem, sizeof(int32_t) * n * occ::kMaxMembers, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w_host, d_w, sizeof(float) * wn, cudaMemcpyDeviceToHost);
    cudaFree(d_pix);
    cudaFree(d_mem);
    cudaFree(d_w);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "debug_mis");
    return OCC_OK;
}

// ---------------------------------------------------------------------------------------
// Batched frames (occ_frame_batch), captured batches (occ_batch_*) and tuning.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kBatchTileW = 16, kBatchTileH = 8;

// Validates the views and fills the device work table (host side); writes the record
// metadata back into each view as the trace calls do.
occ_status build_batch(occ_ctx* ctx, const occ_bvh* bvh, occ_view* views, int32_t n,
                       std::vector<occ::BatchView>* table, std::vector<occ::BatchDyn>* dyn,
                       int* n_tiles, int* max_k) {
    if (!bvh) return fail(ctx, OCC_ERR_INVALID_ARG, "bvh is NULL");
    if (!views || n < 1 || n > occ::kMaxBatchViews)
        return fail(ctx, OCC_ERR_INVALID_ARG, "n_views must be in [1, %d]", occ::kMaxBatchViews);
    table->resize(n);
    dyn->resize(n);
    int64_t tiles = 0;
    *max_k = 1;
    for (int i = 0; i < n; ++i) {
        occ_view& v = views[i];
        occ_status st;
        if ((st = check_gbuffer(ctx, &v.gb)) != OCC_OK) return st;
        if ((st = check_occluders(ctx, &v.gb, &v.rec)) != OCC_OK) return st;
        if (v.effect == OCC_EFFECT_AO && !(v.radius > 0.0f && std::isfinite(v.radius)))
            return fail(ctx, OCC_ERR_INVALID_ARG, "view %d: AO radius must be positive", i);
        if (v.effect == OCC_EFFECT_SHADOW && (st = check_light(ctx, &v.light)) != OCC_OK) return st;
        if (v.effect != OCC_EFFECT_AO && v.effect != OCC_EFFECT_SHADOW)
            return fail(ctx, OCC_ERR_INVALID_ARG, "view %d: effect %d invalid", i, v.effect);
        if (v.estimator < OCC_EST_NOREUSE || v.estimator > OCC_EST_BOXMEAN)
            return fail(ctx, OCC_ERR_INVALID_ARG, "view %d: estimator invalid", i);
        if (v.K > 16) return fail(ctx, OCC_ERR_UNSUPPORTED, "view %d: batched views need K <= 16", i);
        if (!v.out) return fail(ctx, OCC_ERR_INVALID_ARG, "view %d: out is NULL", i);
        occ::BatchView& b = (*table)[i];
        std::memset(&b, 0, sizeof(b));
        if ((st = make_pattern(ctx, &v.pattern, v.K, &b.pat)) != OCC_OK) return st;
        v.rec.effect = v.effect;
        v.rec.radius = v.effect == OCC_EFFECT_AO ? v.radius : 0.0f;
        if (v.effect == OCC_EFFECT_SHADOW) v.rec.light = v.light;
        else std::memset(&v.rec.light, 0, sizeof(v.rec.light));
        v.rec.seed = v.seed;
        v.rec.sample = v.sample;
        b.gb = view(&v.gb);
        b.rec = rec_view(&v.rec);
        b.effect = v.effect;
        b.estimator = v.estimator;
        b.radius = v.rec.radius;
        b.light = to_params(v.effect == OCC_EFFECT_SHADOW ? &v.light : nullptr);
        b.R2s = (float)((double)v.rec.radius * (double)v.rec.radius * (1.0 + 1.0 / 65536.0));
        b.out = v.out;
        b.tiles_x = (v.gb.W + kBatchTileW - 1) / kBatchTileW;
        b.first_tile = (int32_t)tiles;
        tiles += (int64_t)b.tiles_x * ((v.gb.H + kBatchTileH - 1) / kBatchTileH);
        (*dyn)[i].seed = v.seed;
        (*dyn)[i].sample = v.sample;
        (*dyn)[i].pad = 0;
        *max_k = std::max(*max_k, v.K);
    }
    if (tiles > (int64_t)1 << 30) return fail(ctx, OCC_ERR_INVALID_ARG, "batch too large");
    *n_tiles = (int)tiles;
    return OCC_OK;
}

cudaError_t launch_batch(occ_ctx* ctx, const occ_bvh* bvh, const occ::BatchView* views,
                         const occ::BatchDyn* dyn, int n, int n_tiles, int max_k, cudaStream_t s) {
    const occ::DevBVH b = dev_bvh(bvh);
    cudaError_t e = occ::launch_trace_batch(views, dyn, n, n_tiles, b,
                                            occ::trace_batch_ctas(ctx->tune.batch_per_sm), ctx->status, s);
    if (e == cudaSuccess)
        e = occ::launch_reuse_batch(views, dyn, n, n_tiles, max_k, b, ctx->tune.batch_per_sm,
                                    ctx->status, s);
    return e;
}

}  // namespace

OCC_EXPORT occ_status occ_frame_batch(occ_ctx* ctx, const occ_bvh* bvh, occ_view* views,
                                      int32_t n_views, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    std::vector<occ::BatchView> table;
    std::vector<occ::BatchDyn> dyn;
    int n_tiles = 0, max_k = 1;
    if ((st = build_batch(ctx, bvh, views, n_views, &table, &dyn, &n_tiles, &max_k)) != OCC_OK) return st;
    const size_t tb = table.size() * sizeof(occ::BatchView), db = dyn.size() * sizeof(occ::BatchDyn);
    cudaError_t e = cudaSuccess;
    if (!ctx->batch_ev) e = cudaEventCreateWithFlags(&ctx->batch_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && ctx->batch_bytes < tb + db) {
        // the previous upload must be done before its buffers go away
        if (ctx->batch_bytes) cudaEventSynchronize(ctx->batch_ev);
        cudaFree(ctx->batch_dev);
        cudaFreeHost(ctx->batch_host);
        ctx->batch_dev = ctx->batch_host = nullptr;
        ctx->batch_bytes = 0;
        e = cudaMalloc(&ctx->batch_dev, tb + db);
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->batch_host, tb + db);
        if (e == cudaSuccess) ctx->batch_bytes = tb + db;
    } else if (e == cudaSuccess) {
        e = cudaEventSynchronize(ctx->batch_ev);   // staging is free once the last upload ran
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch table");
    char* host = static_cast<char*>(ctx->batch_host);
    std::memcpy(host, table.data(), tb);
    std::memcpy(host + tb, dyn.data(), db);
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(ctx->batch_dev, host, tb + db, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->batch_ev, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    char* dev = static_cast<char*>(ctx->batch_dev);
    return launched(ctx,
                    launch_batch(ctx, bvh, reinterpret_cast<occ::BatchView*>(dev),
                                 reinterpret_cast<occ::BatchDyn*>(dev + tb), n_views, n_tiles, max_k, s),
                    "batch launch");
}

OCC_EXPORT occ_status occ_batch_capture(occ_ctx* ctx, const occ_bvh* bvh, occ_view* views,
                                        int32_t n_views, occ_batch** out) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!out) return fail(ctx, OCC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::vector<occ::BatchView> table;
    std::vector<occ::BatchDyn> dyn;
    int n_tiles = 0, max_k = 1;
    if ((st = build_batch(ctx, bvh, views, n_views, &table, &dyn, &n_tiles, &max_k)) != OCC_OK) return st;
    occ_batch* b = new occ_batch();
    b->device = ctx->device;
    b->n_views = n_views;
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    const size_t tb = table.size() * sizeof(occ::BatchView), db = dyn.size() * sizeof(occ::BatchDyn);
    cudaError_t e = cudaMalloc(&b->views, tb);
    if (e == cudaSuccess) e = cudaMalloc(&b->dyn, db);
    if (e == cudaSuccess) e = cudaMallocHost(&b->dyn_host, db);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(b->views, table.data(), tb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->dyn, dyn.data(), db, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t le = launch_batch(ctx, bvh, b->views, b->dyn, n_views, n_tiles, max_k, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        occ_batch_free(ctx, b);
        return cuda_fail(ctx, e, "batch capture");
    }
    *out = b;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_batch_launch(occ_ctx* ctx, occ_batch* b, const uint64_t* seeds_host,
                                       const uint32_t* samples_host, void* stream) {
    occ_status st = check_ctx(ctx);
    if (st != OCC_OK) return st;
    if (!b || b->device != ctx->device) return fail(ctx, OCC_ERR_INVALID_ARG, "bad batch");
    if (!seeds_host || !samples_host) return fail(ctx, OCC_ERR_INVALID_ARG, "seeds/samples are NULL");
    cudaError_t e = cudaEventSynchronize(b->uploaded);   // the pinned values are free again
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch staging");
    for (int i = 0; i < b->n_views; ++i) {
        b->dyn_host[i].seed = seeds_host[i];
        b->dyn_host[i].sample = samples_host[i];
        b->dyn_host[i].pad = 0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(b->dyn, b->dyn_host, sizeof(occ::BatchDyn) * b->n_views, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->uploaded, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    return launched(ctx, e, "batch replay");
}

OCC_EXPORT occ_status occ_batch_free(occ_ctx* ctx, occ_batch* b) {
    if (!ctx || !b) return OCC_ERR_INVALID_ARG;
    cudaSetDevice(b->device);
    if (b->uploaded) cudaEventSynchronize(b->uploaded);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->uploaded) cudaEventDestroy(b->uploaded);
    cudaFree(b->views);
    cudaFree(b->dyn);
    cudaFreeHost(b->dyn_host);
    delete b;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_set_tuning(occ_ctx* ctx, const occ_tuning* t) {
    if (!ctx || !t) return OCC_ERR_INVALID_ARG;
    if (t->reuse_tile_rows != 0 && t->reuse_tile_rows != 4 && t->reuse_tile_rows != 8 &&
        t->reuse_tile_rows != 16)
        return fail(ctx, OCC_ERR_INVALID_ARG, "reuse_tile_rows must be 0, 4, 8 or 16");
    if (t->reuse_window_path < 0 || t->reuse_window_path > 3)
        return fail(ctx, OCC_ERR_INVALID_ARG, "reuse_window_path must be 0, 1, 2 or 3");
    if (t->batch_ctas_per_sm < 0 || t->batch_ctas_per_sm > 16)
        return fail(ctx, OCC_ERR_INVALID_ARG, "batch_ctas_per_sm must be in [0, 16]");
    if (t->fused_ao_path < 0 || t->fused_ao_path > 2)
        return fail(ctx, OCC_ERR_INVALID_ARG, "fused_ao_path must be 0, 1 or 2");
    if (t->group_prefetch < 0 || t->group_prefetch > 3)
        return fail(ctx, OCC_ERR_INVALID_ARG, "group_prefetch must be 0, 1, 2 or 3");
    if (t->trace_path < 0 || t->trace_path > 2)
        return fail(ctx, OCC_ERR_INVALID_ARG, "trace_path must be 0, 1 or 2");
    if (t->trace_ctas_per_sm < 0 || t->trace_ctas_per_sm > 16)
        return fail(ctx, OCC_ERR_INVALID_ARG, "trace_ctas_per_sm must be in [0, 16]");
    if (t->trace_refill < 0 || t->trace_refill > 32)
        return fail(ctx, OCC_ERR_INVALID_ARG, "trace_refill must be in [0, 32]");
    if (t->trace_order < 0 || t->trace_order > 2)
        return fail(ctx, OCC_ERR_INVALID_ARG, "trace_order must be 0, 1 or 2");
    ctx->tune.tile_rows = t->reuse_tile_rows;
    ctx->tune.window_path = t->reuse_window_path;
    ctx->tune.batch_per_sm = t->batch_ctas_per_sm;
    ctx->tune.fused_ao_path = t->fused_ao_path;
    ctx->tune.group_prefetch = t->group_prefetch;
    ctx->tune.trace_path = t->trace_path;
    ctx->tune.trace_ctas_per_sm = t->trace_ctas_per_sm;
    ctx->tune.trace_refill = t->trace_refill;
    ctx->tune.trace_order = t->trace_order;
    return OCC_OK;
}

OCC_EXPORT occ_status occ_get_tuning(const occ_ctx* ctx, occ_tuning* t) {
    if (!ctx || !t) return OCC_ERR_INVALID_ARG;
    t->reuse_tile_rows = ctx->tune.tile_rows;
    t->reuse_window_path = ctx->tune.window_path;
    t->batch_ctas_per_sm = ctx->tune.batch_per_sm;
    t->fused_ao_path = ctx->tune.fused_ao_path;
    t->group_prefetch = ctx->tune.group_prefetch;
    t->trace_path = ctx->tune.trace_path;
    t->trace_ctas_per_sm = ctx->tune.trace_ctas_per_sm;
    t->trace_refill = ctx->tune.trace_refill;
    t->trace_order = ctx->tune.trace_order;
    return OCC_OK;
}

// ---------------------------------------------------------------------------------------
// occ_frame_noalloc: one frame (trace + reuse) that allocates no device memory.
//
// Callers such as render-engine plugins that must draw all device memory from the
// host application's own pools, or real-time frame loops that cannot afford the
// device-wide synchronisation cudaMalloc / cudaFree may cause, cannot create an
// occ_ctx (its status word is allocated) nor hand the library a workspace.  This
// entry point keeps its scratch -- the occluder records of the frame and the device
// status word -- in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxPixels = int64_t(1) << 20;   // e.g. 1280x720 or 1024x1024
constexpr int kNoAllocMaxDevices = 64;

// [0, 2 * max) : two float4 record planes; [2 * max] : device status word; [2 * max + 1] :
// work counter of the persistent AO trace (the rest is padding)
static __device__ __align__(256) float4 g_noalloc_scratch[2 * kNoAllocMaxPixels + 16];

std::mutex g_noalloc_mutex;
float4* g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace

OCC_EXPORT occ_status occ_frame_noalloc(const occ_gbuffer* gb, const occ_bvh* bvh, int32_t effect,
                                        float radius, const occ_rect_light* light, uint64_t seed,
                                        uint32_t sample, const occ_pattern* pattern, int32_t K,
                                        int32_t estimator, float* out, uint32_t* flags_host,
                                        char* err_msg, int32_t err_len, void* stream) {
    occ_ctx local;   // carries validation messages only; owns no device memory
    auto finish = [&](occ_status st) {
        if (st != OCC_OK && err_msg && err_len > 0)
            snprintf(err_msg, (size_t)err_len, "%s", local.last_error.c_str());
        return st;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return finish(cuda_fail(&local, e, "cudaGetDevice"));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return finish(fail(&local, OCC_ERR_UNSUPPORTED, "device %d beyond the supported %d", dev,
                           kNoAllocMaxDevices));
    local.device = dev;
    occ_status st = check_gbuffer(&local, gb);
    if (st != OCC_OK) return finish(st);
    const int64_t P = (int64_t)gb->W * gb->H;
    if (P > kNoAllocMaxPixels)
        return finish(fail(&local, OCC_ERR_INVALID_ARG,
                           "frame of %lld pixels exceeds the %lld-pixel maximum of the static "
                           "scratch of occ_frame_noalloc",
                           (long long)P, (long long)kNoAllocMaxPixels));
    if (!bvh) return finish(fail(&local, OCC_ERR_INVALID_ARG, "bvh is NULL"));
    if (bvh->device != dev)
        return finish(fail(&local, OCC_ERR_INVALID_ARG, "bvh lives on device %d, current device is %d",
                           bvh->device, dev));
    if (effect != OCC_EFFECT_AO && effect != OCC_EFFECT_SHADOW)
        return finish(fail(&local, OCC_ERR_INVALID_ARG, "effect %d invalid", effect));
    if (effect == OCC_EFFECT_AO && !(radius > 0.0f && std::isfinite(radius)))
        return finish(fail(&local, OCC_ERR_INVALID_ARG, "AO radius must be positive and finite"));
    if (effect == OCC_EFFECT_SHADOW && (st = check_light(&local, light)) != OCC_OK) return finish(st);
    if (estimator < OCC_EST_NOREUSE || estimator > OCC_EST_BOXMEAN)
        return finish(fail(&local, OCC_ERR_INVALID_ARG, "estimator %d invalid", estimator));
    if (!out) return finish(fail(&local, OCC_ERR_INVALID_ARG, "out is NULL"));
    occ::PatternParams pat;
    if ((st = make_pattern(&local, pattern, K, &pat)) != OCC_OK) return finish(st);
    pat.sample = sample;

    float4* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return finish(cuda_fail(&local, e, "cudaGetSymbolAddress"));
            g_noalloc_ptr[dev] = static_cast<float4*>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    const occ::RecView rec{base, base + P};
    unsigned* status = reinterpret_cast<unsigned*>(base + 2 * kNoAllocMaxPixels);
    unsigned* counter = reinterpret_cast<unsigned*>(base + 2 * kNoAllocMaxPixels + 1);
    cudaStream_t s = (cudaStream_t)stream;
    const occ::LightParams lp = to_params(effect == OCC_EFFECT_SHADOW ? light : nullptr);
    const occ::DevBVH b = dev_bvh(bvh);
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    // the counter selects the same trace kernels as occ_trace_ao / occ_trace_shadow
    if (e == cudaSuccess)
        e = occ::launch_trace(effect, view(gb), b, radius, lp, seed, sample, rec, status, s,
                              counter);
    if (e == cudaSuccess)
        e = occ::launch_reuse(effect, estimator, view(gb), rec, pat, radius, lp,
                              estimator == OCC_EST_UNBIASED ? &b : nullptr, out, status, s);
    if (e != cudaSuccess) return finish(cuda_fail(&local, e, "occ_frame_noalloc launch"));
    if (flags_host) {
        e = cudaMemcpyAsync(flags_host, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return finish(cuda_fail(&local, e, "occ_frame_noalloc status"));
        if (*flags_host)
            return finish(fail(&local, OCC_ERR_DEVICE_CHECK, "device check flags 0x%x", *flags_host));
    }
    return OCC_OK;
}
