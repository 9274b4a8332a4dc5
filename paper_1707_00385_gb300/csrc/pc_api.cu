// pc_api.cu -- host runtime behind the C ABI declared in include/pcurv.h:
// argument checks, the context, staging buffers for host-memory calls, the
// batch scratch and its CUDA graphs, and the choice of kernel instantiation.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pcurv.h"
#include "pc_internal.h"

// The fused kernels stage halo rows of at most 96 columns (three warp ballots).
static_assert(pcurv::TILE_W + 2 * PC_MAX_RADIUS <= 96 && PC_MAX_NORMAL_RADIUS <= PC_MAX_RADIUS,
              "staged halo rows exceed the three ballots of the fused kernels");

namespace {

// Host-side NVTX range over one API call, named after it (ncu --nvtx can
// select kernels by it; without a CUDA tool attached the calls do nothing).
struct HostRange {
    explicit HostRange(const char* name) { nvtxRangePushA(name); }
    ~HostRange() { nvtxRangePop(); }
    HostRange(const HostRange&) = delete;
    HostRange& operator=(const HostRange&) = delete;
};

}  // namespace

namespace {

// Device scratch of pc_compute_batch: the frame table and the tile counter,
// two page-locked staging copies of the table (alternating between calls so
// that a call rarely waits), and one graph per staging copy.
struct BatchScratch {
    int device = -1;
    int cap = 0;                              // frames the table holds
    pcurv::BatchTable* d_table = nullptr;     // device
    unsigned* d_counter = nullptr;            // device
    pcurv::BatchTable* h_table[2] = {nullptr, nullptr};  // page-locked host
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool pending[2] = {false, false};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_grid[2] = {0, 0};
    int graph_cap[2] = {0, 0};
    int graph_variant[2] = {-1, -1};
    cudaStream_t capture = nullptr;           // private stream used only for capture
    int grid[pcurv::NUM_TILE_VARIANTS] = {};  // persistent CTAs per tile variant
    const pcurv::KernelOps* packed_ops = nullptr;  // kernels packed_grid was sized for
    int packed_grid = 0;                      // persistent CTAs of the 16-bit storage batch
    int next = 0;                             // staging copy of the next call
};

// Most bands of one pc_compute_host frame (each about a wave of CTAs or more).
constexpr int HOST_BANDS = 8;

// Pipeline of pc_compute_host_batch: two device staging slots (each holds the
// ranges and results of one chunk of frames) and four streams -- copies in,
// two compute streams (chunks alternate between them, each with its own batch
// scratch), copies out -- ordered by events, so that the copies of one chunk
// overlap the computation of its neighbours and consecutive chunks' kernels
// overlap where one ends and the next begins.
struct HostPipe {
    int device = -1;
    cudaStream_t in = nullptr, comp[2] = {nullptr, nullptr}, out = nullptr;
    cudaEvent_t start = nullptr, tail = nullptr;
    cudaEvent_t in_done[2] = {nullptr, nullptr}, comp_done[2] = {nullptr, nullptr};
    cudaEvent_t slot_free[2] = {nullptr, nullptr};
    bool slot_used[2] = {false, false};
    float* buf[2] = {nullptr, nullptr};      // device, px * 6 floats per slot
    size_t cap_px[2] = {0, 0};
    pc_frame* dev_frames = nullptr;          // host: device descriptors of one chunk
    // pc_compute_host: one frame in bands of tile rows on the same streams
    cudaEvent_t band_in[HOST_BANDS] = {}, band_done[HOST_BANDS] = {};
};

// Tile variant chosen by pc_autotune for one image size.
struct Plan {
    int H = 0, W = 0, variant = 0;
    long long stamp = 0;
};

}  // namespace

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
    BatchScratch batch;
    BatchScratch batch_alt;                   // odd chunks of pc_compute_host_batch
    HostPipe pipe;
    Plan plans[16];
    long long plan_clock = 0;
    int sms_device = -1;
    int sms = 0;                              // SMs of that device
    int resident[pcurv::NUM_TILE_VARIANTS] = {};  // CTAs of each tile variant resident there (0: not queried)
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
        cudaGetLastError();  // clear the error of an unknown pointer
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
    if (p.batch_graph != 0 && p.batch_graph != 1) return PC_ERR_INVALID_ARG;
    if (p.kahan != 0 && p.kahan != 1) return PC_ERR_INVALID_ARG;
    if (p.tile_height != 0 && p.tile_height != 8 && p.tile_height != 4) return PC_ERR_INVALID_ARG;
    if (p.lanes_per_pixel != 0 && p.lanes_per_pixel != 1 && pcurv::variant_of_lanes(p.lanes_per_pixel) < 0)
        return PC_ERR_INVALID_ARG;
    // a lane group fixes its own tile (32 x 8/lanes) and runs the plain FP32 form
    if (p.lanes_per_pixel > 1 && (p.tile_height != 0 || p.kahan)) return PC_ERR_INVALID_ARG;
    if (!(finite_f(p.fp64_solve_cond) && p.fp64_solve_cond >= 0.f)) return PC_ERR_INVALID_ARG;
    return PC_OK;
}

pc_status check_image(int H, int W) {
    if (H < 0 || W < 0 || H > PC_MAX_DIM || W > PC_MAX_DIM) return PC_ERR_INVALID_ARG;
    return PC_OK;
}

bool valid_intrinsics(float fx, float fy, float cx, float cy) {
    return finite_f(fx) && finite_f(fy) && finite_f(cx) && finite_f(cy) && fx > 0.f && fy > 0.f;
}

// Device buffers of one frame: present, aligned, on the device.
pc_status check_buffers(const float* depth, const float* k1, const float* k2, const float* normal) {
    if (!depth || !k1 || !k2) return PC_ERR_INVALID_ARG;
    if (!aligned4(depth) || !aligned4(k1) || !aligned4(k2) || !aligned4(normal)) return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(depth) || !is_device_ptr(k1) || !is_device_ptr(k2) ||
        (normal && !is_device_ptr(normal)))
        return PC_ERR_INVALID_ARG;
    return PC_OK;
}

void release_batch(BatchScratch& b) {
    for (int i = 0; i < 2; i++) {
        if (b.pending[i]) cudaEventSynchronize(b.done[i]);
        b.pending[i] = false;
        if (b.graph[i]) cudaGraphExecDestroy(b.graph[i]);
        b.graph[i] = nullptr;
        b.graph_grid[i] = b.graph_cap[i] = 0;
        b.graph_variant[i] = -1;
        if (b.h_table[i]) cudaFreeHost(b.h_table[i]);
        b.h_table[i] = nullptr;
        if (b.done[i]) cudaEventDestroy(b.done[i]);
        b.done[i] = nullptr;
    }
    cudaFree(b.d_table);
    cudaFree(b.d_counter);
    b.d_table = nullptr;
    b.d_counter = nullptr;
    if (b.capture) cudaStreamDestroy(b.capture);
    b.capture = nullptr;
    b.cap = 0;
    for (int& g : b.grid) g = 0;
    b.packed_ops = nullptr;
    b.packed_grid = 0;
    b.device = -1;
}

int round_up_pow2(int n) {
    int c = 1;
    while (c < n) c <<= 1;
    return c;
}

}  // namespace

namespace pcurv {

namespace {

// Index 1..12: the dense window of that radius (unrolled); index 0: run-time
// radius and stride.  Each entry joins the one-lane variants of its
// translation unit with the lane-group variants, which take radius and stride
// at run time for every window (pc_fit_lanes.cu: unrolled copies for each
// radius would multiply the build time for frames that are small anyway).
// Index 13: the sparse 37 x 37 patch (radius 18, stride 3).
struct OpsTable {
    KernelOps ops[14];
    OpsTable() {
        for (int i = 0; i <= 13; i++) {
            const KernelOps* one = i == 0    ? ops_generic()
                                   : i <= 4  ? ops_r1_4(i)
                                   : i <= 8  ? ops_r5_8(i)
                                   : i <= 12 ? ops_r9_12(i)
                                             : ops_sparse(SPARSE_RADIUS, SPARSE_STRIDE);
            const KernelOps* lanes = ops_lanes();
            ops[i] = *one;
            for (int v = 0; v < NUM_TILE_VARIANTS; v++) {
                if (!lanes->fit[v]) continue;
                ops[i].fit[v] = lanes->fit[v];
                ops[i].batch[v] = lanes->batch[v];
                ops[i].occupancy[v] = lanes->occupancy[v];
            }
        }
    }
};

}  // namespace

const KernelOps* select_ops(const FitConfig& cfg) {
    if (cfg.kahan) return ops_precision(1, 0);
    static const OpsTable table;  // built once (thread-safe initialisation)
    const bool dense = cfg.stride == 1 && cfg.r >= 1 && cfg.r <= 12;
    if (cfg.r == SPARSE_RADIUS && cfg.stride == SPARSE_STRIDE) return &table.ops[13];
    return &table.ops[dense ? cfg.r : 0];
}

const KernelOps* select_packed_ops(const FitConfig& cfg, int format) {
    if (!cfg.kahan && cfg.stride == 1) {
        const KernelOps* k = format == 1 ? ops_packed_f16(cfg.r) : format == 2 ? ops_packed_bf16(cfg.r) : nullptr;
        if (k) return k;
    }
    return ops_precision(cfg.kahan, format);
}

const FitConfig& ctx_config(const pc_ctx* ctx) { return ctx->cfg; }

void ctx_set_error(pc_ctx* ctx, const char* msg) {
    if (ctx) snprintf(ctx->last_error, sizeof ctx->last_error, "%s", msg);
}

}  // namespace pcurv

namespace {

// SMs of the current device (cached per device in ctx).
cudaError_t sm_count(pc_ctx* ctx, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (ctx->sms_device != dev) {
        if ((e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        ctx->sms_device = dev;
        for (int& n : ctx->resident) n = 0;
    }
    *sms = ctx->sms;
    return cudaSuccess;
}

// CTAs of tile variant v of ops that the current device holds at once (one wave).
cudaError_t resident_ctas(pc_ctx* ctx, const pcurv::KernelOps* ops, int v, int* n) {
    int sms = 0;
    cudaError_t e = sm_count(ctx, &sms);
    if (e != cudaSuccess) return e;
    if (ctx->resident[v] == 0) {
        int per_sm = 0;
        if ((e = ops->occupancy[v](ctx->cfg, &per_sm)) != cudaSuccess) return e;
        ctx->resident[v] = sms * (per_sm > 0 ? per_sm : 1);
    }
    *n = ctx->resident[v];
    return cudaSuccess;
}

// The variant params fix (a lane group, or a one-lane tile height), else -1.
int forced_variant(const pc_ctx* ctx) {
    if (ctx->params.lanes_per_pixel > 1) return pcurv::variant_of_lanes(ctx->params.lanes_per_pixel);
    return ctx->params.tile_height == 8 ? 0 : ctx->params.tile_height == 4 ? 1 : -1;
}

// Whether the autotuner and the plans may use variant v: lanes_per_pixel = 1
// keeps to one lane per pixel.
bool plan_allows(const pc_ctx* ctx, int v) { return ctx->params.lanes_per_pixel != 1 || pcurv::lanes_of(v) == 1; }

// 32 x 8 tiles when there are at least 1.5 per SM, else 32 x 4 (GB300:
// 32 x 4 is a third faster at 160 x 120, even at 320 x 240).
int heuristic_variant(long long tiles8, int sms) { return 2 * tiles8 >= 3LL * sms ? 0 : 1; }

// Tile variant for one H x W image: forced, tuned, or the heuristic (one lane
// per pixel); always one that ops has.
cudaError_t variant_for(pc_ctx* ctx, const pcurv::KernelOps* ops, int H, int W, int* v) {
    int choice = forced_variant(ctx);
    if (choice < 0) {
        for (const Plan& pl : ctx->plans)
            if (pl.stamp && pl.H == H && pl.W == W && plan_allows(ctx, pl.variant)) choice = pl.variant;
    }
    if (choice < 0) {
        int sms = 0;
        const cudaError_t e = sm_count(ctx, &sms);
        if (e != cudaSuccess) return e;
        choice = heuristic_variant(pcurv::tiles_of(H, W, 8), sms);
    }
    *v = ops->fit[choice] ? choice : 0;
    return cudaSuccess;
}

// Tile rows of an H-row frame in variant v, and one launch over all of them.
int tile_rows(int H, int v) {
    const int th = pcurv::tile_h_of(v);
    return (H + th - 1) / th;
}
cudaError_t fit_frame(const pcurv::KernelOps* ops, int v, const pcurv::FrameArgs& f, const pcurv::FitConfig& cfg,
                      cudaStream_t s) {
    return ops->fit[v](f, cfg, s, 0, tile_rows(f.H, v));
}

void remember_plan(pc_ctx* ctx, int H, int W, int variant) {
    Plan* slot = &ctx->plans[0];
    for (Plan& pl : ctx->plans) {
        if (pl.stamp && pl.H == H && pl.W == W) { slot = &pl; break; }
        if (pl.stamp < slot->stamp) slot = &pl;
    }
    slot->H = H;
    slot->W = W;
    slot->variant = variant;
    slot->stamp = ++ctx->plan_clock;
}

}  // namespace

namespace pcurv {
int ctx_forced_variant(const pc_ctx* ctx) { return forced_variant(ctx); }
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
    p->batch_graph = 1;
    p->kahan = 0;
    p->fp64_solve_cond = 0.f;
    p->tile_height = 0;
    p->lanes_per_pixel = 0;
}

pc_status pc_create(float fx, float fy, float cx, float cy, int window_radius, int iterations,
                    const pc_params* params, pc_ctx** out) {
    if (!out) return PC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_intrinsics(fx, fy, cx, cy)) return PC_ERR_INVALID_ARG;
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
                              p.reject, p.reject_ratio, p.det_tol, p.pivot_tol, p.min_window,
                              p.kahan, p.fp64_solve_cond > 0.f ? 1.f / p.fp64_solve_cond : 0.f};
    *out = c;
    return PC_OK;
}

pc_status pc_compute(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* k1_out,
                     float* k2_out, float* normal_out) {
    const HostRange range("pc_compute");
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if ((st = check_buffers(depth, k1_out, k2_out, normal_out)) != PC_OK) return st;
    const pcurv::FrameArgs f{depth, H, W, ctx->cam, k1_out, k2_out, normal_out, nullptr, nullptr};
    const pcurv::KernelOps* ops = pcurv::select_ops(ctx->cfg);
    int v = 0;
    cudaError_t e = variant_for(ctx, ops, H, W, &v);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_compute plan");
    e = fit_frame(ops, v, f, ctx->cfg, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_compute launch");
    return PC_OK;
}

pc_status pc_autotune(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* k1_out,
                      float* k2_out, float* normal_out) {
    const HostRange range("pc_autotune");
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if ((st = check_buffers(depth, k1_out, k2_out, normal_out)) != PC_OK) return st;
    const pcurv::FrameArgs f{depth, H, W, ctx->cam, k1_out, k2_out, normal_out, nullptr, nullptr};
    const pcurv::KernelOps* ops = pcurv::select_ops(ctx->cfg);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "pc_autotune events");
    }
    int best = 0;
    float best_ms = 3.4e38f;
    for (int v = 0; v < pcurv::NUM_TILE_VARIANTS && e == cudaSuccess; v++) {
        if (!ops->fit[v] || !plan_allows(ctx, v)) continue;
        e = fit_frame(ops, v, f, ctx->cfg, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int i = 0; i < 3 && e == cudaSuccess; i++) e = fit_frame(ops, v, f, ctx->cfg, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_autotune");
    remember_plan(ctx, H, W, best);
    return PC_OK;
}

int pc_plan_tile_height(pc_ctx* ctx, int H, int W) {
    if (!ctx || check_image(H, W) != PC_OK) return 0;
    int v = 0;
    if (variant_for(ctx, pcurv::select_ops(ctx->cfg), H, W, &v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return pcurv::tile_h_of(v);
}

int pc_plans_export(const pc_ctx* ctx, int* H, int* W, int* tile_height, int* lanes_per_pixel, int capacity) {
    if (!ctx || capacity < 0 || (capacity > 0 && (!H || !W || !tile_height || !lanes_per_pixel))) return -1;
    // oldest first, so that importing them in order keeps their age order
    const Plan* order[16];
    int n = 0;
    for (const Plan& pl : ctx->plans)
        if (pl.stamp) order[n++] = &pl;
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && order[j]->stamp < order[j - 1]->stamp; j--) {
            const Plan* t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int i = 0; i < n && i < capacity; i++) {
        H[i] = order[i]->H;
        W[i] = order[i]->W;
        tile_height[i] = pcurv::tile_h_of(order[i]->variant);
        lanes_per_pixel[i] = pcurv::lanes_of(order[i]->variant);
    }
    return n;
}

pc_status pc_plans_import(pc_ctx* ctx, const int* H, const int* W, const int* tile_height,
                          const int* lanes_per_pixel, int n) {
    const HostRange range("pc_plans_import");
    if (!ctx || n < 0 || (n > 0 && (!H || !W || !tile_height || !lanes_per_pixel))) return PC_ERR_INVALID_ARG;
    int v[64];
    if (n > 64) return PC_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        if (check_image(H[i], W[i]) != PC_OK || H[i] == 0 || W[i] == 0) return PC_ERR_INVALID_ARG;
        v[i] = -1;
        for (int k = 0; k < pcurv::NUM_TILE_VARIANTS; k++)
            if (pcurv::tile_h_of(k) == tile_height[i] && pcurv::lanes_of(k) == lanes_per_pixel[i]) v[i] = k;
        // a variant this context's kernels lack (lane groups with compensated sums) is not a plan for it
        if (v[i] < 0 || !pcurv::select_ops(ctx->cfg)->fit[v[i]]) return PC_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; i++) remember_plan(ctx, H[i], W[i], v[i]);
    return PC_OK;
}

int pc_plan_lanes_per_pixel(pc_ctx* ctx, int H, int W) {
    if (!ctx || check_image(H, W) != PC_OK) return 0;
    int v = 0;
    if (variant_for(ctx, pcurv::select_ops(ctx->cfg), H, W, &v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return pcurv::lanes_of(v);
}

static bool aligned2(const void* p) { return ((uintptr_t)p & 1u) == 0; }

pc_status pc_pack_depth(pc_ctx* ctx, const float* depth, int H, int W, int format, void* stream,
                        unsigned short* packed, float* tile_base) {
    if (!ctx || (format != PC_DEPTH_F16 && format != PC_DEPTH_BF16)) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!depth || !packed || !tile_base || !aligned4(depth) || !aligned2(packed) || !aligned4(tile_base))
        return PC_ERR_INVALID_ARG;
    if (!is_device_ptr(depth) || !is_device_ptr(packed) || !is_device_ptr(tile_base))
        return PC_ERR_INVALID_ARG;
    const cudaError_t e = pcurv::launch_pack(depth, H, W, format, packed, tile_base, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_pack_depth launch");
    return PC_OK;
}

pc_status pc_compute_packed(pc_ctx* ctx, const unsigned short* packed, const float* tile_base, int format,
                            int H, int W, void* stream, float* k1_out, float* k2_out, float* normal_out) {
    const HostRange range("pc_compute_packed");
    if (!ctx || (format != PC_DEPTH_F16 && format != PC_DEPTH_BF16)) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!packed || !tile_base || !aligned2(packed) || !aligned4(tile_base) || !is_device_ptr(packed) ||
        !is_device_ptr(tile_base))
        return PC_ERR_INVALID_ARG;
    if (!k1_out || !k2_out || !aligned4(k1_out) || !aligned4(k2_out) || !aligned4(normal_out) ||
        !is_device_ptr(k1_out) || !is_device_ptr(k2_out) || (normal_out && !is_device_ptr(normal_out)))
        return PC_ERR_INVALID_ARG;
    const pcurv::FrameArgs f{nullptr, H, W, ctx->cam, k1_out, k2_out, normal_out, packed, tile_base};
    const cudaError_t e =
        fit_frame(pcurv::select_packed_ops(ctx->cfg, format), 0, f, ctx->cfg, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_packed launch");
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

static pc_status ensure_pipe(pc_ctx* ctx);

pc_status pc_compute_host(pc_ctx* ctx, const float* depth_host, int H, int W, void* stream,
                          float* k1_host, float* k2_host, float* normal_host) {
    const HostRange range("pc_compute_host");
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
    const pcurv::FrameArgs f{ctx->d_depth, H, W, ctx->cam, ctx->d_k1, ctx->d_k2,
                             normal_host ? ctx->d_normal : nullptr, nullptr, nullptr};
    const pcurv::KernelOps* ops = pcurv::select_ops(ctx->cfg);
    int v = 0;
    if ((e = variant_for(ctx, ops, H, W, &v)) != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host plan");
    const int rows = tile_rows(H, v), th = pcurv::tile_h_of(v);
    const long long tiles = (long long)rows * ((W + pcurv::TILE_W - 1) / pcurv::TILE_W);
    // A frame of several waves of CTAs goes in bands of tile rows, each about
    // a wave or more: band b's ranges are copied in (with the halo rows its
    // windows read), its kernel runs, its results are copied out, on the
    // pipeline's streams, so that only the first band's copy in and the last
    // band's copy out are not hidden behind a kernel.  Consecutive bands'
    // kernels alternate between two streams and overlap at their ends.
    int wave = 0;
    if ((e = resident_ctas(ctx, ops, v, &wave)) != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host occupancy");
    long long bands_ll = (2 * tiles + wave) / (2 * wave);  // bands of at least 7/8 of a wave
    if (bands_ll > HOST_BANDS) bands_ll = HOST_BANDS;
    if (bands_ll > rows) bands_ll = rows;
    const int bands = (int)bands_ll;
    if (bands <= 1) {
        if ((e = cudaMemcpyAsync(ctx->d_depth, depth_host, npx * sizeof(float), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return cuda_fail(ctx, e, "depth H2D");
        if ((e = fit_frame(ops, v, f, ctx->cfg, s)) != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host launch");
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
    if ((st = ensure_pipe(ctx)) != PC_OK) return st;
    HostPipe& p = ctx->pipe;
    // start after the caller's earlier work and after every earlier host
    // call's copies out (the staging buffers are reused)
    if ((e = cudaEventRecord(p.start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(p.in, p.start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p.in, p.tail, 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "pc_compute_host start");
    const int halo = pcurv::halo_of(ctx->cfg);
    int copied = 0;  // rows of ranges enqueued so far
    for (int b = 0; b < bands; b++) {
        const int ty0 = (int)((long long)rows * b / bands), ty1 = (int)((long long)rows * (b + 1) / bands);
        const int last = ty1 * th + halo;
        const int need = b + 1 < bands && last < H ? last : H;
        if (need > copied) {
            if ((e = cudaMemcpyAsync(ctx->d_depth + (size_t)copied * W, depth_host + (size_t)copied * W,
                                     (size_t)(need - copied) * W * sizeof(float), cudaMemcpyHostToDevice, p.in)) !=
                cudaSuccess)
                return cuda_fail(ctx, e, "depth H2D");
            copied = need;
        }
        cudaStream_t c = p.comp[b & 1];
        if ((e = cudaEventRecord(p.band_in[b], p.in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c, p.band_in[b], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "pc_compute_host order");
        if ((e = ops->fit[v](f, ctx->cfg, c, ty0, ty1)) != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host launch");
        if ((e = cudaEventRecord(p.band_done[b], c)) != cudaSuccess) return cuda_fail(ctx, e, "pc_compute_host order");
    }
    // copies out after all kernels are enqueued (a copy to pageable memory may block the host)
    for (int b = 0; b < bands; b++) {
        const int v0 = (int)((long long)rows * b / bands) * th;
        const int v1e = (int)((long long)rows * (b + 1) / bands) * th, v1 = v1e < H ? v1e : H;
        const size_t o = (size_t)v0 * W, n = (size_t)(v1 - v0) * W;
        if ((e = cudaStreamWaitEvent(p.out, p.band_done[b], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "pc_compute_host order");
        if ((e = cudaMemcpyAsync(k1_host + o, ctx->d_k1 + o, n * sizeof(float), cudaMemcpyDeviceToHost, p.out)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(k2_host + o, ctx->d_k2 + o, n * sizeof(float), cudaMemcpyDeviceToHost, p.out)) !=
                cudaSuccess)
            return cuda_fail(ctx, e, "curvature D2H");
        if (normal_host &&
            (e = cudaMemcpyAsync(normal_host + 3 * o, ctx->d_normal + 3 * o, 3 * n * sizeof(float),
                                 cudaMemcpyDeviceToHost, p.out)) != cudaSuccess)
            return cuda_fail(ctx, e, "normal D2H");
    }
    // the caller's stream completes when the last results are on the host
    if ((e = cudaEventRecord(p.tail, p.out)) != cudaSuccess || (e = cudaStreamWaitEvent(s, p.tail, 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "pc_compute_host end");
    return PC_OK;
}

// Batch scratch b (of ctx) for at least n frames on the current device.
static pc_status ensure_batch(pc_ctx* ctx, BatchScratch& b, int n) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    if (b.device == dev && b.cap >= n) return PC_OK;
    release_batch(b);
    const int cap = round_up_pow2(n < 16 ? 16 : n);
    const size_t bytes = pcurv::batch_table_bytes(cap);
    const pcurv::KernelOps* ops = pcurv::select_ops(ctx->cfg);
    int sms = 0, bps[pcurv::NUM_TILE_VARIANTS] = {};
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(ctx, e, "batch occupancy");
    for (int v = 0; v < pcurv::NUM_TILE_VARIANTS; v++)
        if (ops->occupancy[v] && (e = ops->occupancy[v](ctx->cfg, &bps[v])) != cudaSuccess)
            return cuda_fail(ctx, e, "batch occupancy");
    if ((e = cudaMalloc(&b.d_table, bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b.d_counter, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaHostAlloc(&b.h_table[0], bytes, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaHostAlloc(&b.h_table[1], bytes, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b.done[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b.done[1], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b.capture, cudaStreamNonBlocking)) != cudaSuccess) {
        release_batch(b);
        return cuda_fail(ctx, e, "batch scratch");
    }
    b.device = dev;
    b.cap = cap;
    for (int v = 0; v < pcurv::NUM_TILE_VARIANTS; v++) b.grid[v] = sms * (bps[v] > 0 ? bps[v] : 1);
    return PC_OK;
}

// Copy of the staged table, queue reset and persistent kernel (tile variant v,
// `grid` CTAs), on `s`.
static cudaError_t enqueue_batch(pc_ctx* ctx, BatchScratch& b, int slot, size_t bytes, int v, int grid,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(b.d_table, b.h_table[slot], bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    return pcurv::select_ops(ctx->cfg)->batch[v](b.d_table, b.d_counter, grid, ctx->cfg, s);
}

// The graph of staging copy `slot` (captured on the private stream once per
// capacity and tile variant).
static pc_status ensure_graph(pc_ctx* ctx, BatchScratch& b, int slot, int v) {
    if (b.graph[slot] && b.graph_cap[slot] == b.cap && b.graph_grid[slot] == b.grid[v] &&
        b.graph_variant[slot] == v)
        return PC_OK;
    if (b.graph[slot]) cudaGraphExecDestroy(b.graph[slot]);
    b.graph[slot] = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b.capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture begin");
    const cudaError_t e1 = enqueue_batch(ctx, b, slot, pcurv::batch_table_bytes(b.cap), v, b.grid[v], b.capture);
    e = cudaStreamEndCapture(b.capture, &g);
    if (e1 != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e1 != cudaSuccess ? e1 : e, "graph capture");
    }
    e = cudaGraphInstantiate(&b.graph[slot], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b.graph[slot] = nullptr;
        return cuda_fail(ctx, e, "graph instantiate");
    }
    b.graph_cap[slot] = b.cap;
    b.graph_grid[slot] = b.grid[v];
    b.graph_variant[slot] = v;
    return PC_OK;
}

// pc_compute_batch on batch scratch b of ctx.
static pc_status batch_on(pc_ctx* ctx, BatchScratch& b, const pc_frame* frames, int n, void* stream) {
    if (!ctx || n < 0 || n > PC_MAX_BATCH || (n > 0 && !frames)) return PC_ERR_INVALID_ARG;
    long long total = 0;  // 32 x 8 tiles
    int live = 0;
    for (int i = 0; i < n; i++) {
        const pc_frame& fr = frames[i];
        pc_status st = check_image(fr.H, fr.W);
        if (st != PC_OK) return st;
        if (fr.H == 0 || fr.W == 0) continue;
        if (!valid_intrinsics(fr.fx, fr.fy, fr.cx, fr.cy)) return PC_ERR_INVALID_ARG;
        if ((st = check_buffers(fr.depth, fr.k1, fr.k2, fr.normal)) != PC_OK) return st;
        total += pcurv::tiles_of(fr.H, fr.W, 8);
        live++;
    }
    if (live == 0) return PC_OK;
    if (2 * total > 0x7fffffffLL) return PC_ERR_INVALID_ARG;
    pc_status st = ensure_batch(ctx, b, live);
    if (st != PC_OK) return st;
    const pcurv::KernelOps* ops = pcurv::select_ops(ctx->cfg);
    int v = forced_variant(ctx);
    if (v < 0) {
        int sms = 0;
        cudaError_t es = sm_count(ctx, &sms);
        if (es != cudaSuccess) return cuda_fail(ctx, es, "batch plan");
        v = heuristic_variant(total, sms);
    }
    if (!ops->batch[v]) v = 0;
    const int th = pcurv::tile_h_of(v);
    const int slot = b.next;
    b.next ^= 1;
    cudaError_t e;
    if (b.pending[slot]) {
        // the batch before last may still be reading this staging copy
        if ((e = cudaEventSynchronize(b.done[slot])) != cudaSuccess) return cuda_fail(ctx, e, "batch wait");
        b.pending[slot] = false;
    }
    pcurv::BatchTable* t = b.h_table[slot];
    int k = 0, begin = 0;
    for (int i = 0; i < n; i++) {
        const pc_frame& fr = frames[i];
        if (fr.H == 0 || fr.W == 0) continue;
        pcurv::BatchFrame& d = t->frames[k++];
        d.f = pcurv::FrameArgs{fr.depth, fr.H, fr.W,
                               pcurv::Camera{fr.fx, fr.fy, fr.cx, fr.cy, 1.f / fr.fx, 1.f / fr.fy},
                               fr.k1, fr.k2, fr.normal, nullptr, nullptr};
        d.tiles_x = (fr.W + pcurv::TILE_W - 1) / pcurv::TILE_W;
        d.tile_begin = begin;
        begin += d.tiles_x * ((fr.H + th - 1) / th);
    }
    t->nframes = live;
    t->total_tiles = begin;
    cudaStream_t s = (cudaStream_t)stream;
    // A queue shorter than the persistent grid gets one CTA per tile: the
    // hardware spreads a small grid over the SMs, while the first CTAs of a
    // full persistent grid may share SMs (GB300: one 160 x 120 frame in 32 x 4
    // tiles, 150 tiles on a 608-CTA grid, took 88 us against 58 us).  Such
    // launches bypass the graph, which holds the full grid.
    const int grid = begin < b.grid[v] ? begin : b.grid[v];
    if (ctx->params.batch_graph && grid == b.grid[v]) {
        if ((st = ensure_graph(ctx, b, slot, v)) != PC_OK) return st;
        if ((e = cudaGraphLaunch(b.graph[slot], s)) != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    } else if ((e = enqueue_batch(ctx, b, slot, pcurv::batch_table_bytes(live), v, grid, s)) != cudaSuccess) {
        return cuda_fail(ctx, e, "batch launch");
    }
    if ((e = cudaEventRecord(b.done[slot], s)) != cudaSuccess) return cuda_fail(ctx, e, "batch event");
    b.pending[slot] = true;
    return PC_OK;
}

pc_status pc_compute_batch(pc_ctx* ctx, const pc_frame* frames, int n, void* stream) {
    const HostRange range("pc_compute_batch");
    return ctx ? batch_on(ctx, ctx->batch, frames, n, stream) : PC_ERR_INVALID_ARG;
}

// Device buffers of one packed frame: present, aligned, on the device.
static pc_status check_packed_frame(const pc_packed_frame& f) {
    if (!f.packed || !f.tile_base || !aligned2(f.packed) || !aligned4(f.tile_base) || !is_device_ptr(f.packed) ||
        !is_device_ptr(f.tile_base))
        return PC_ERR_INVALID_ARG;
    if (!f.k1 || !f.k2 || !aligned4(f.k1) || !aligned4(f.k2) || !aligned4(f.normal) || !is_device_ptr(f.k1) ||
        !is_device_ptr(f.k2) || (f.normal && !is_device_ptr(f.normal)))
        return PC_ERR_INVALID_ARG;
    return PC_OK;
}

pc_status pc_compute_packed_batch(pc_ctx* ctx, const pc_packed_frame* frames, int n, int format, void* stream) {
    const HostRange range("pc_compute_packed_batch");
    if (!ctx || n < 0 || n > PC_MAX_BATCH || (n > 0 && !frames) ||
        (format != PC_DEPTH_F16 && format != PC_DEPTH_BF16))
        return PC_ERR_INVALID_ARG;
    long long total = 0;  // 32 x 8 tiles
    int live = 0;
    for (int i = 0; i < n; i++) {
        const pc_packed_frame& fr = frames[i];
        pc_status st = check_image(fr.H, fr.W);
        if (st != PC_OK) return st;
        if (fr.H == 0 || fr.W == 0) continue;
        if (!valid_intrinsics(fr.fx, fr.fy, fr.cx, fr.cy)) return PC_ERR_INVALID_ARG;
        if ((st = check_packed_frame(fr)) != PC_OK) return st;
        total += pcurv::tiles_of(fr.H, fr.W, 8);
        live++;
    }
    if (live == 0) return PC_OK;
    if (total > 0x7fffffffLL) return PC_ERR_INVALID_ARG;
    BatchScratch& b = ctx->batch;
    pc_status st = ensure_batch(ctx, b, live);
    if (st != PC_OK) return st;
    const pcurv::KernelOps* ops = pcurv::select_packed_ops(ctx->cfg, format);
    cudaError_t e;
    if (b.packed_ops != ops) {  // sized once per kernel and device (ensure_batch resets it)
        int sms = 0, per_sm = 0;
        e = sm_count(ctx, &sms);
        if (e == cudaSuccess) e = ops->occupancy[0](ctx->cfg, &per_sm);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "packed batch occupancy");
        b.packed_grid = sms * (per_sm > 0 ? per_sm : 1);
        b.packed_ops = ops;
    }
    const int slot = b.next;
    b.next ^= 1;
    if (b.pending[slot]) {
        // the batch before last may still be reading this staging copy
        if ((e = cudaEventSynchronize(b.done[slot])) != cudaSuccess) return cuda_fail(ctx, e, "batch wait");
        b.pending[slot] = false;
    }
    pcurv::BatchTable* t = b.h_table[slot];
    int k = 0, begin = 0;
    for (int i = 0; i < n; i++) {
        const pc_packed_frame& fr = frames[i];
        if (fr.H == 0 || fr.W == 0) continue;
        pcurv::BatchFrame& d = t->frames[k++];
        d.f = pcurv::FrameArgs{nullptr, fr.H, fr.W,
                               pcurv::Camera{fr.fx, fr.fy, fr.cx, fr.cy, 1.f / fr.fx, 1.f / fr.fy},
                               fr.k1, fr.k2, fr.normal, fr.packed, fr.tile_base};
        d.tiles_x = (fr.W + pcurv::TILE_W - 1) / pcurv::TILE_W;
        d.tile_begin = begin;
        begin += d.tiles_x * ((fr.H + 7) / 8);
    }
    t->nframes = live;
    t->total_tiles = begin;
    cudaStream_t s = (cudaStream_t)stream;
    const int slots = b.packed_grid;  // one CTA per tile when the queue is shorter
    if ((e = cudaMemcpyAsync(b.d_table, t, pcurv::batch_table_bytes(live), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned), s)) != cudaSuccess ||
        (e = ops->batch[0](b.d_table, b.d_counter, begin < slots ? begin : slots, ctx->cfg, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "packed batch launch");
    if ((e = cudaEventRecord(b.done[slot], s)) != cudaSuccess) return cuda_fail(ctx, e, "batch event");
    b.pending[slot] = true;
    return PC_OK;
}

static void release_pipe(HostPipe& p) {
    if (p.out) cudaStreamSynchronize(p.out);
    for (int i = 0; i < 2; i++) {
        cudaFree(p.buf[i]);
        p.buf[i] = nullptr;
        p.cap_px[i] = 0;
        p.slot_used[i] = false;
        for (cudaEvent_t* ev : {&p.in_done[i], &p.comp_done[i], &p.slot_free[i]}) {
            if (*ev) cudaEventDestroy(*ev);
            *ev = nullptr;
        }
    }
    for (cudaEvent_t* ev : {&p.start, &p.tail}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    for (int b = 0; b < HOST_BANDS; b++)
        for (cudaEvent_t* ev : {&p.band_in[b], &p.band_done[b]}) {
            if (*ev) cudaEventDestroy(*ev);
            *ev = nullptr;
        }
    delete[] p.dev_frames;
    p.dev_frames = nullptr;
    for (cudaStream_t* st : {&p.in, &p.comp[0], &p.comp[1], &p.out}) {
        if (*st) cudaStreamDestroy(*st);
        *st = nullptr;
    }
    p.device = -1;
}

// Streams and events of the host pipeline on the current device.
static pc_status ensure_pipe(pc_ctx* ctx) {
    HostPipe& p = ctx->pipe;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    if (p.device == dev) return PC_OK;
    if (p.device >= 0) release_pipe(p);
    p.device = dev;
    for (cudaStream_t* st : {&p.in, &p.comp[0], &p.comp[1], &p.out})
        if ((e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking)) != cudaSuccess) break;
    for (int i = 0; i < 2 && e == cudaSuccess; i++)
        for (cudaEvent_t* ev : {&p.in_done[i], &p.comp_done[i], &p.slot_free[i]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (cudaEvent_t* ev : {&p.start, &p.tail})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (int b = 0; b < HOST_BANDS; b++)
        for (cudaEvent_t* ev : {&p.band_in[b], &p.band_done[b]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        p.dev_frames = new (std::nothrow) pc_frame[PC_MAX_BATCH];
        if (!p.dev_frames) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        release_pipe(p);
        return cuda_fail(ctx, e, "pipeline streams");
    }
    return PC_OK;
}

pc_status pc_compute_host_batch(pc_ctx* ctx, const pc_frame* frames, int n, void* stream) {
    const HostRange range("pc_compute_host_batch");
    if (!ctx || n < 0 || (n > 0 && !frames)) return PC_ERR_INVALID_ARG;
    size_t total_px = 0;
    for (int i = 0; i < n; i++) {
        const pc_frame& fr = frames[i];
        pc_status st = check_image(fr.H, fr.W);
        if (st != PC_OK) return st;
        if (fr.H == 0 || fr.W == 0) continue;
        if (!valid_intrinsics(fr.fx, fr.fy, fr.cx, fr.cy)) return PC_ERR_INVALID_ARG;
        if (!fr.depth || !fr.k1 || !fr.k2) return PC_ERR_INVALID_ARG;
        total_px += (size_t)fr.H * fr.W;
    }
    if (total_px == 0) return PC_OK;
    pc_status st = ensure_pipe(ctx);
    if (st != PC_OK) return st;
    HostPipe& p = ctx->pipe;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    // start after the work the caller has already enqueued on `stream`
    if ((e = cudaEventRecord(p.start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(p.in, p.start, 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "pipeline start");
    pc_frame* dev = p.dev_frames;
    int i = 0, chunk = 0;
    size_t left = total_px;
    while (i < n) {
        // next chunk: frames up to a pixel limit (at least one frame).  The limit
        // is PC_HOST_CHUNK_PIXELS, smaller at both ends, where copies are not
        // hidden behind computation: the first chunk's copy in and the last
        // one's copy out.  The first chunk takes an eighth; over the last two
        // chunks' worth of pixels each chunk takes half of what is left.
        const size_t full = (size_t)PC_HOST_CHUNK_PIXELS;
        size_t cap = chunk == 0 ? full / 8 : full;
        if (left <= 2 * full) cap = left / 2 > full / 16 ? left / 2 : full / 16;
        int j = i;
        size_t px = 0;
        while (j < n && j - i < PC_MAX_BATCH) {
            const size_t f = (size_t)frames[j].H * frames[j].W;
            if (j > i && px + f > cap) break;
            px += f;
            j++;
        }
        left -= px;
        const int slot = chunk & 1;
        if (px > p.cap_px[slot]) {
            // grow: wait until the chunk that last used the slot has been copied out
            if (p.slot_used[slot] && (e = cudaEventSynchronize(p.slot_free[slot])) != cudaSuccess)
                return cuda_fail(ctx, e, "pipeline wait");
            cudaFree(p.buf[slot]);
            p.buf[slot] = nullptr;
            p.cap_px[slot] = 0;
            if ((e = cudaMalloc(&p.buf[slot], px * 6 * sizeof(float))) != cudaSuccess)
                return cuda_fail(ctx, e, "pipeline cudaMalloc");
            p.cap_px[slot] = px;
        }
        if (p.slot_used[slot] && (e = cudaStreamWaitEvent(p.in, p.slot_free[slot], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "pipeline order");
        // device layout of the slot: ranges, k1, k2 (px each), normals (3 px)
        float* d_depth = p.buf[slot];
        float* d_k1 = d_depth + px;
        float* d_k2 = d_k1 + px;
        float* d_nrm = d_k2 + px;
        size_t off = 0;
        int m = 0;
        for (int q = i; q < j; q++) {
            const pc_frame& fr = frames[q];
            const size_t f = (size_t)fr.H * fr.W;
            if (f == 0) continue;
            if ((e = cudaMemcpyAsync(d_depth + off, fr.depth, f * sizeof(float), cudaMemcpyHostToDevice, p.in)) !=
                cudaSuccess)
                return cuda_fail(ctx, e, "pipeline H2D");
            dev[m++] = pc_frame{d_depth + off, fr.H, fr.W, fr.fx, fr.fy, fr.cx, fr.cy, d_k1 + off, d_k2 + off,
                                fr.normal ? d_nrm + 3 * off : nullptr};
            off += f;
        }
        // chunks alternate between two compute streams, each with its own batch
        // scratch, so that a chunk's kernel can start on the SMs the previous
        // chunk's last tiles leave idle
        if ((e = cudaEventRecord(p.in_done[slot], p.in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p.comp[slot], p.in_done[slot], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "pipeline order");
        if ((st = batch_on(ctx, slot ? ctx->batch_alt : ctx->batch, dev, m, p.comp[slot])) != PC_OK) return st;
        if ((e = cudaEventRecord(p.comp_done[slot], p.comp[slot])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p.out, p.comp_done[slot], 0)) != cudaSuccess)
            return cuda_fail(ctx, e, "pipeline order");
        off = 0;
        for (int q = i; q < j; q++) {
            const pc_frame& fr = frames[q];
            const size_t f = (size_t)fr.H * fr.W;
            if (f == 0) continue;
            if ((e = cudaMemcpyAsync(fr.k1, d_k1 + off, f * sizeof(float), cudaMemcpyDeviceToHost, p.out)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(fr.k2, d_k2 + off, f * sizeof(float), cudaMemcpyDeviceToHost, p.out)) !=
                    cudaSuccess ||
                (fr.normal && (e = cudaMemcpyAsync(fr.normal, d_nrm + 3 * off, 3 * f * sizeof(float),
                                                   cudaMemcpyDeviceToHost, p.out)) != cudaSuccess))
                return cuda_fail(ctx, e, "pipeline D2H");
            off += f;
        }
        if ((e = cudaEventRecord(p.slot_free[slot], p.out)) != cudaSuccess) return cuda_fail(ctx, e, "pipeline order");
        p.slot_used[slot] = true;
        i = j;
        chunk++;
    }
    // the caller's stream completes when the last results are on the host
    if ((e = cudaEventRecord(p.tail, p.out)) != cudaSuccess || (e = cudaStreamWaitEvent(s, p.tail, 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "pipeline end");
    return PC_OK;
}

pc_status pc_backproject(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* xyz) {
    const HostRange range("pc_backproject");
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!depth || !xyz || !aligned4(depth) || !aligned4(xyz) || !is_device_ptr(depth) || !is_device_ptr(xyz))
        return PC_ERR_INVALID_ARG;
    int sms = 0;
    cudaError_t e = sm_count(ctx, &sms);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_backproject");
    e = pcurv::launch_backproject(depth, H, W, ctx->cam, xyz, sms, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_backproject launch");
    return PC_OK;
}

pc_status pc_initial_normals(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* normal) {
    const HostRange range("pc_initial_normals");
    if (!ctx) return PC_ERR_INVALID_ARG;
    pc_status st = check_image(H, W);
    if (st != PC_OK) return st;
    if (H == 0 || W == 0) return PC_OK;
    if (!depth || !normal || !aligned4(depth) || !aligned4(normal) || !is_device_ptr(depth) ||
        !is_device_ptr(normal))
        return PC_ERR_INVALID_ARG;
    int sms = 0;
    cudaError_t e = sm_count(ctx, &sms);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_initial_normals");
    e = pcurv::launch_initial_normals(depth, H, W, ctx->cam, ctx->cfg.rn, ctx->cfg.det_tol, normal, sms,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pc_initial_normals launch");
    return PC_OK;
}

pc_status pc_destroy(pc_ctx* ctx) {
    if (!ctx) return PC_OK;
    if (ctx->stage_px) {
        cudaDeviceSynchronize();
        free_stage(ctx);
    }
    if (ctx->pipe.device >= 0) release_pipe(ctx->pipe);
    if (ctx->batch.device >= 0) release_batch(ctx->batch);
    if (ctx->batch_alt.device >= 0) release_batch(ctx->batch_alt);
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
