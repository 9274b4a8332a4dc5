// pc_api.cu -- host runtime behind the C ABI declared in include/pcurv.h:
// argument checks, the context, staging buffers for host-memory calls, and
// the choice of kernel instantiation.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/pcurv.h"
#include "pc_internal.h"

struct pc_ctx {
    pcurv::Camera cam;
    pcurv::FitConfig cfg;
    pc_params params;
    // device staging buffers of pc_compute_host
    int stage_device = -1;
    size_t stage_px = 0;
    float* d_depth = nullptr;
    float* d_k1 = nullptr;
    float* d_k2 = nullptr;
    float* d_normal = nullptr;
    char last_error[256] = {0};
};

namespace {

pc_status cuda_fail(pc_ctx* ctx, cudaError_t e, const char* where) {
    if (ctx) snprintf(ctx->last_error, sizeof ctx->last_error, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
}

bool finite_f(float x) { return std::isfinite(x); }

bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

// A pointer the kernels may dereference: device or managed memory.
bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pc_status check_params(const pc_params& p) {
    if (!(finite_f(p.k) && p.k > 0.f)) return PC_ERR_INVALID_ARG;
    if (p.reject != 0 && p.reject != 1) return PC_ERR_INVALID_ARG;
    if (!(finite_f(p.reject_ratio) && p.reject_ratio > 0.f)) return PC_ERR_INVALID_ARG;
    if (p.normal_radius < 1 || p.normal_radius > PC_MAX_NORMAL_RADIUS) return PC_ERR_INVALID_ARG;
    if (p.stride < 1 || p.stride > PC_MAX_RADIUS) return PC_ERR_INVALID_ARG;
    if (!(finite_f(p.det_tol) && p.det_tol >= 0.f)) return PC_ERR_INVALID_ARG;
    if (!(finite_f(p.pivot_tol) && p.pivot_tol >= 0.f)) return PC_ERR_INVALID_ARG;
    if (p.min_window < 6) return PC_ERR_INVALID_ARG;  // six parameters need six points
    return PC_OK;
}

pc_status check_image(int H, int W) {
    if (H < 0 || W < 0 || H > PC_MAX_DIM || W > PC_MAX_DIM) return PC_ERR_INVALID_ARG;
    return PC_OK;
}

}  // namespace

namespace pcurv {

cudaError_t launch_fit(const float* depth, int H, int W, const Camera& cam, const FitConfig& cfg,
                       float* k1, float* k2, float* normal, cudaStream_t stream) {
    if (cfg.stride == 1 && cfg.r >= 1 && cfg.r <= 4)
        return launch_fit_r1_4(depth, H, W, cam, cfg, k1, k2, normal, stream);
    if (cfg.stride == 1 && cfg.r >= 5 && cfg.r <= 8)
        return launch_fit_r5_8(depth, H, W, cam, cfg, k1, k2, normal, stream);
    if (cfg.stride == 1 && cfg.r >= 9 && cfg.r <= 12)
        return launch_fit_r9_12(depth, H, W, cam, cfg, k1, k2, normal, stream);
    return launch_fit_generic(depth, H, W, cam, cfg, k1, k2, normal, stream);
}

}  // namespace pcurv

extern "C" {

void pc_params_default(pc_params* p) {
    if (!p) return;
    p->k = 1e-4f;
    p->reject = 0;
    p->reject_ratio = 2.f;
    p->normal_radius = 3;
    p->stride = 1;
    p->det_tol = 1e-6f;
    p->pivot_tol = 1e-5f;
    p->min_window = 6;
}

pc_status pc_create(float fx, float fy, float cx, float cy, int window_radius, int iterations,
                    const pc_params* params, pc_ctx** out) {
    if (!out) return PC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!(finite_f(fx) && finite_f(fy) && finite_f(cx) && finite_f(cy) && fx > 0.f && fy > 0.f))
        return PC_ERR_INVALID_ARG;
    if (window_radius < 1 || window_radius > PC_MAX_RADIUS) return PC_ERR_INVALID_ARG;
    if (iterations < 0 || iterations > PC_MAX_ITERATIONS) return PC_ERR_INVALID_ARG;
    pc_params p;
    pc_params_default(&p);
    if (params) p = *params;
    const pc_status st = check_params(p);
    if (st != PC_OK) return st;
    pc_ctx* c = new (std::nothrow) pc_ctx;
    if (!c) return PC_ERR_OOM;
    c->params = p;
    c->cam = pcurv::Camera{fx, fy, cx, cy, 1.f / fx, 1.f / fy};
    c->cfg = pcurv::FitConfig{window_radius, p.normal_radius, iterations, p.stride, 1.f / p.k,
                              p.reject, p.reject_ratio, p.det_tol, p.pivot_tol, p.min_window};
    *out = c;
    return PC_OK;
}

pc_status pc_compute(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* k1_out,
                     float* k2_out, float* normal_out) {
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!depth || !k1_out || !k2_out) return PC_ERR_INVALID_ARG;
    if (!aligned4(depth) || !aligned4(k1_out) || !aligned4(k2_out) || !aligned4(normal_out))
        return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(depth) || !is_device_ptr(k1_out) || !is_device_ptr(k2_out) ||
        (normal_out && !is_device_ptr(normal_out)))
        return PC_ERR_INVALID_ARG;
    const cudaError_t e = pcurv::launch_fit(depth, H, W, ctx->cam, ctx->cfg, k1_out, k2_out,
                                            normal_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_compute launch");
    return PC_OK;
}

static void free_stage(pc_ctx* ctx) {
    cudaFree(ctx->d_depth);
    cudaFree(ctx->d_k1);
    cudaFree(ctx->d_k2);
    cudaFree(ctx->d_normal);
    ctx->d_depth = ctx->d_k1 = ctx->d_k2 = ctx->d_normal = nullptr;
    ctx->stage_px = 0;
}

pc_status pc_compute_host(pc_ctx* ctx, const float* depth_host, int H, int W, void* stream,
                          float* k1_host, float* k2_host, float* normal_host) {
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!depth_host || !k1_host || !k2_host) return PC_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    const size_t npx = (size_t)H * W;
    if (ctx->stage_device != dev || ctx->stage_px < npx) {
        if (ctx->stage_px) {
            // the old buffers may still be in use by queued work
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceSynchronize");
            free_stage(ctx);
        }
        if ((e = cudaMalloc(&ctx->d_depth, npx * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->d_k1, npx * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->d_k2, npx * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&ctx->d_normal, 3 * npx * sizeof(float))) != cudaSuccess) {
            free_stage(ctx);
            return cuda_fail(ctx, e, "staging cudaMalloc");
        }
        ctx->stage_px = npx;
        ctx->stage_device = dev;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemcpyAsync(ctx->d_depth, depth_host, npx * sizeof(float), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess)
        return cuda_fail(ctx, e, "depth H2D");
    e = pcurv::launch_fit(ctx->d_depth, H, W, ctx->cam, ctx->cfg, ctx->d_k1, ctx->d_k2,
                          normal_host ? ctx->d_normal : nullptr, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host launch");
    if ((e = cudaMemcpyAsync(k1_host, ctx->d_k1, npx * sizeof(float), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(k2_host, ctx->d_k2, npx * sizeof(float), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "curvature D2H");
    if (normal_host &&
        (e = cudaMemcpyAsync(normal_host, ctx->d_normal, 3 * npx * sizeof(float),
                             cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "normal D2H");
    return PC_OK;
}

pc_status pc_destroy(pc_ctx* ctx) {
    if (!ctx) return PC_OK;
    if (ctx->stage_px) {
        cudaDeviceSynchronize();
        free_stage(ctx);
    }
    delete ctx;
    return PC_OK;
}

const char* pc_status_string(pc_status s) {
    switch (s) {
        case PC_OK: return "ok";
        case PC_ERR_INVALID_ARG: return "invalid argument";
        case PC_ERR_CUDA: return "CUDA error";
        case PC_ERR_OOM: return "out of memory";
        case PC_ERR_TIMEOUT: return "device wait timed out";
        case PC_ERR_UNSUPPORTED: return "unsupported parameters";
    }
    return "unknown status";
}

const char* pc_last_error(const pc_ctx* ctx) { return ctx ? ctx->last_error : ""; }

}  // extern "C"
