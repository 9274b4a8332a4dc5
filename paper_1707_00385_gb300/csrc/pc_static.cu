// pc_static.cu -- pc_compute_batch_static: the batched method with its
// scratch in a fixed array of this library instead of allocated memory, for
// callers that cannot allocate device memory (see include/pcurv.h).
//
// The array holds the tile counter (alone in the first 256 bytes) followed by
// the frame table.  Host code never uses the array's name as an address: in
// host code it only names a host-side stand-in.  The device address comes
// from cudaGetSymbolAddress, looked up once per device, and is passed to the
// same persistent kernel pc_compute_batch launches, in the tile variant
// pc_compute_batch would choose when the context's parameters force one.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/pcurv.h"
#include "pc_internal.h"

namespace {

constexpr int kMaxFrames = PC_STATIC_MAX_FRAMES;
constexpr size_t kCounterBytes = 256;
constexpr size_t kTableBytes =
    (sizeof(pcurv::BatchTable) + (kMaxFrames - 1) * sizeof(pcurv::BatchFrame) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCounterBytes + kTableBytes;
constexpr int kMaxDevices = 64;
constexpr int kSlotCache = 8;  // grid sizes remembered per device

static __device__ __align__(256) unsigned char pc_static_scratch[kScratchBytes];

// CTAs one wave of a kernel variant holds on a device: the persistent grid.
// The kernel is fixed by its instantiation (ops), tile variant and the
// reject flag; its shared memory by the halo.
struct SlotEntry {
    const pcurv::KernelOps* ops;
    int variant, reject, halo, slots;
};

std::mutex g_mu;                              // guards the tables below
unsigned char* g_scratch[kMaxDevices];        // device address of the array, per device
unsigned char g_host_table[kTableBytes];      // host staging of the frame table
SlotEntry g_slots[kMaxDevices][kSlotCache];   // per device, filled in order, then round robin
int g_slot_next[kMaxDevices];

bool ok_intrinsics(const pc_frame& f) {
    return std::isfinite(f.fx) && std::isfinite(f.fy) && std::isfinite(f.cx) && std::isfinite(f.cy) &&
           f.fx > 0.f && f.fy > 0.f;
}

bool device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool ok_buffers(const pc_frame& f) {
    const uintptr_t a = (uintptr_t)f.depth | (uintptr_t)f.k1 | (uintptr_t)f.k2 | (uintptr_t)f.normal;
    if (!f.depth || !f.k1 || !f.k2 || (a & 3u)) return false;
    return device_ptr(f.depth) && device_ptr(f.k1) && device_ptr(f.k2) && (!f.normal || device_ptr(f.normal));
}

// The persistent grid of (ops, variant) under cfg on device dev; g_mu held.
cudaError_t slots_of(int dev, const pcurv::KernelOps* ops, int v, const pcurv::FitConfig& cfg, int* slots) {
    const int halo = pcurv::halo_of(cfg);
    for (const SlotEntry& e : g_slots[dev])
        if (e.ops == ops && e.variant == v && e.reject == cfg.reject && e.halo == halo && e.slots > 0) {
            *slots = e.slots;
            return cudaSuccess;
        }
    int sms = 0, bps = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = ops->occupancy[v](cfg, &bps);
    if (e != cudaSuccess) return e;
    *slots = sms * (bps > 0 ? bps : 1);
    g_slots[dev][g_slot_next[dev]] = SlotEntry{ops, v, cfg.reject, halo, *slots};
    g_slot_next[dev] = (g_slot_next[dev] + 1) % kSlotCache;
    return cudaSuccess;
}

pc_status fail(pc_ctx* ctx, pc_status st, const char* what, cudaError_t e) {
    char msg[200];
    if (e != cudaSuccess)
        snprintf(msg, sizeof msg, "pc_compute_batch_static: %s: %s", what, cudaGetErrorString(e));
    else
        snprintf(msg, sizeof msg, "pc_compute_batch_static: %s", what);
    pcurv::ctx_set_error(ctx, msg);
    return st;
}

}  // namespace

extern "C" pc_status pc_compute_batch_static(pc_ctx* ctx, const pc_frame* frames, int n, void* stream) {
    if (!ctx || n < 0 || (n > 0 && !frames)) return PC_ERR_INVALID_ARG;
    if (n > kMaxFrames) {
        char what[96];
        snprintf(what, sizeof what, "%d frames exceed the fixed scratch of %d frames", n, kMaxFrames);
        return fail(ctx, PC_ERR_INVALID_ARG, what, cudaSuccess);
    }
    const pcurv::FitConfig& cfg = pcurv::ctx_config(ctx);
    const pcurv::KernelOps* ops = pcurv::select_ops(cfg);
    // the variant pc_compute_batch runs: the one the parameters force (a lane
    // group changes the order of the moment sums), else 32 x 8 tiles (the same
    // bits as the 32 x 4 tiles its heuristic may pick instead)
    int v = pcurv::ctx_forced_variant(ctx);
    if (v < 0 || !ops->batch[v]) v = 0;
    const int th = pcurv::tile_h_of(v);
    long long total = 0;
    int live = 0;
    for (int i = 0; i < n; i++) {
        const pc_frame& f = frames[i];
        if (f.H < 0 || f.W < 0 || f.H > PC_MAX_DIM || f.W > PC_MAX_DIM) return PC_ERR_INVALID_ARG;
        if (f.H == 0 || f.W == 0) continue;
        if (!ok_intrinsics(f) || !ok_buffers(f)) return PC_ERR_INVALID_ARG;
        total += pcurv::tiles_of(f.H, f.W, th);
        live++;
    }
    if (live == 0) return PC_OK;
    if (total > 0x7fffffffLL) return PC_ERR_INVALID_ARG;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(ctx, PC_ERR_UNSUPPORTED, "device index", cudaSuccess);

    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        // set-up, once per device, with that device current
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, pc_static_scratch)) != cudaSuccess)
            return fail(ctx, PC_ERR_CUDA, "cudaGetSymbolAddress", e);
        g_scratch[dev] = (unsigned char*)p;
    }
    int slots = 0;
    if ((e = slots_of(dev, ops, v, cfg, &slots)) != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "occupancy", e);
    unsigned* counter = (unsigned*)g_scratch[dev];
    pcurv::BatchTable* table = (pcurv::BatchTable*)(g_scratch[dev] + kCounterBytes);

    pcurv::BatchTable* t = (pcurv::BatchTable*)g_host_table;
    int k = 0, begin = 0;
    for (int i = 0; i < n; i++) {
        const pc_frame& f = frames[i];
        if (f.H == 0 || f.W == 0) continue;
        pcurv::BatchFrame& d = t->frames[k++];
        d.f = pcurv::FrameArgs{f.depth, f.H, f.W,
                               pcurv::Camera{f.fx, f.fy, f.cx, f.cy, 1.f / f.fx, 1.f / f.fy},
                               f.k1, f.k2, f.normal, nullptr, nullptr};
        d.tiles_x = (f.W + pcurv::TILE_W - 1) / pcurv::TILE_W;
        d.tile_begin = begin;
        begin += d.tiles_x * ((f.H + th - 1) / th);
    }
    t->nframes = live;
    t->total_tiles = begin;
    cudaStream_t s = (cudaStream_t)stream;
    // g_host_table is pageable memory, refilled by the next call as soon as
    // this one returns.  That relies on the documented behaviour of
    // cudaMemcpyAsync from pageable host memory to device memory: the call
    // copies the source into a staging buffer before it returns, so the
    // source may be overwritten afterwards even though the transfer itself
    // completes later in stream order.
    const size_t bytes = pcurv::batch_table_bytes(live);
    if ((e = cudaMemcpyAsync(table, t, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(ctx, PC_ERR_CUDA, "frame table copy", e);
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s)) != cudaSuccess)
        return fail(ctx, PC_ERR_CUDA, "counter reset", e);
    // one CTA per tile when the queue is shorter than the persistent grid
    if ((e = ops->batch[v](table, counter, begin < slots ? begin : slots, cfg, s)) != cudaSuccess)
        return fail(ctx, PC_ERR_CUDA, "launch", e);
    return PC_OK;
}
