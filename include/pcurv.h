/*
 * pcurv.h -- C ABI of the GB300 (sm_103a) principal-curvature library.
 *
 * Method: Spek, Li, Drummond, "A Fast Method For Computing Principal
 * Curvatures From Range Images" (arXiv 1707.00385).  For every pixel of a
 * range image the library
 *   - back-projects the window around it through the pinhole intrinsics
 *     (Sec. 3.2, first pipeline item), relative to the pixel's own point
 *     (p'_i = p_i - p, Sec. 3.1.2);
 *   - estimates an initial normal by regressing z on x and y over a
 *     (2*normal_radius+1)^2 patch (Sec. 3.2.1, Eq. initialnormal);
 *   - fits the parabolic patch z = A/2 x^2 + B x y + C/2 y^2 in a frame
 *     rotated by (theta_x, theta_y) and offset by t_z (Sec. 3.1.2, Eq. quad),
 *     by `iterations` re-weighted Gauss-Newton steps with weights
 *     W(eps) = k / (k + eps^2) (Sec. 3.2.3, Eqs. iter_reweighted_update and
 *     weighting_function);
 *   - returns k1 = T1 + T2 >= k2 = T1 - T2, T1 = (A + C)/2,
 *     T2 = sqrt(T1^2 - AC + B^2) (Sec. 3.1.2), and the refined normal, the
 *     local z axis of the final frame (Sec. 3.2.4).
 *
 * Conventions
 *   - Range images are float32, row major, H rows by W columns, in metres;
 *     pixel (u, v) is column u, row v, with its centre at integer (u, v).
 *     A range that is not finite or not > 0 marks "no measurement".
 *   - Curvatures are in 1/metre; a surface convex towards the camera is
 *     positive (a sphere of radius rho gives 1/rho, 1/rho).  Normals are unit
 *     vectors in the camera frame pointing away from the camera, stored as
 *     H*W*3 interleaved floats (n_x, n_y, n_z per pixel).
 *   - A pixel without a result (no range, degenerate normal patch, fewer than
 *     min_window valid window points, or a singular re-weighted system)
 *     gets quiet NaN in k1, k2 and all three normal components.
 *   - Device pointers are caller-owned CUDA device memory (cudaMalloc or
 *     managed), 4-byte aligned, with no overlap between inputs and outputs.
 *     Host pointers are caller-owned host memory; page-locked memory lets the
 *     copies run asynchronously.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute calls only enqueue work: they return once the work is
 *     queued; the caller synchronises the stream before reading results.
 *   - Arguments are checked before anything is enqueued; a call that returns
 *     an error has enqueued nothing, except PC_ERR_CUDA from a failed launch
 *     or copy (pc_last_error() then holds the CUDA message).
 *   - A context is not thread safe: use one per host thread.  No C++
 *     exception crosses this interface.
 */
#ifndef PCURV_H
#define PCURV_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_ctx pc_ctx; /* opaque; owns parameters and staging buffers */

typedef enum pc_status {
    PC_OK = 0,
    PC_ERR_INVALID_ARG = 1, /* NULL/misaligned/host pointer, size or parameter out of range */
    PC_ERR_CUDA = 2,        /* a CUDA call failed; see pc_last_error() */
    PC_ERR_OOM = 3,         /* device or host allocation failed */
    PC_ERR_TIMEOUT = 4,     /* reserved: a bounded device wait gave up */
    PC_ERR_UNSUPPORTED = 5  /* parameter combination the library does not implement */
} pc_status;

/* Limits checked by every call. */
#define PC_MAX_RADIUS 24         /* window radius r: (2r+1)^2 points */
#define PC_MAX_NORMAL_RADIUS 8   /* initial-normal patch radius */
#define PC_MAX_ITERATIONS 64     /* re-weighted iterations */
#define PC_MAX_DIM 16384         /* H and W */
#define PC_MAX_BATCH 4096        /* frames per pc_compute_batch call */

/* Tunable parameters of the method.  Fill with pc_params_default() first. */
typedef struct pc_params {
    float k;             /* constant k of W(eps) = k/(k+eps^2), m^2 (Sec. 3.2.3). Default 1e-4 */
    int reject;          /* 1 = rejection filter: W = 0 unless eps^2 <= reject_ratio * MSE of the
                            window at the same iteration (Sec. 3.2.3). Default 0 */
    float reject_ratio;  /* default 2 ("twice the mean squared error", Sec. 3.2.3) */
    int normal_radius;   /* initial-normal patch radius; 3 gives the 7x7 patch of Sec. 3.2.1 */
    int stride;          /* window sampling stride (1 = dense; >1 samples the (2r+1)^2
                            square sparsely, as the 37x37 patch of Sec. 4.2.1). Default 1 */
    float det_tol;       /* normal patch degenerate when det M <= det_tol * (tr M)^2. Default 1e-6 */
    float pivot_tol;     /* re-weighted system singular when a pivot of the Jacobi-scaled
                            Cholesky factorisation is <= pivot_tol (a scaled condition estimate
                            above 1/pivot_tol).  Default 1e-5: single-precision moment sums
                            carry ~1e-6 relative error, so smaller pivots are not resolved */
    int min_window;      /* fewest valid window points accepted. Default 6 */
    int batch_graph;     /* 1 = pc_compute_batch replays a CUDA graph (copy of the frame table,
                            reset of the tile queue, persistent kernel) captured once per
                            table capacity; 0 = enqueue the three steps directly.  A batch
                            with fewer tiles than the persistent grid is always enqueued
                            directly, with one CTA per tile. Default 1 */
    int kahan;           /* 1 = compensated (Kahan) summation of the window moments in FP32;
                            costs about 2.3x the time of plain sums. Default 0 */
    float fp64_solve_cond; /* > 0: when the scaled condition estimate of the re-weighted system
                            (1 / smallest scaled pivot) exceeds this value, the 6x6 system is
                            factorised again in FP64 and singularity is judged on the FP64
                            pivots. 0 = off (default) */
    int tile_height;     /* pixel rows of the 32-column tile one CTA computes with one thread per
                            pixel: 8 or 4; 0 = choose per image (the size's pc_autotune result
                            when there is one, else 8 when the image has at least 1.5 32x8
                            tiles per SM, else 4).  Results do not depend on it.  Default 0 */
    int lanes_per_pixel; /* threads that share one pixel's window: 2, 4 or 8 lanes of a warp
                            split the window rows and add their moment sums by shuffles before
                            each solve (tiles of 32 x 8/lanes pixels, 256 threads).  For images
                            too small to fill the GPU with one thread per pixel; on large
                            images it costs throughput.  It changes only the order of the
                            moment sums, so results differ from one lane per pixel by single-
                            precision rounding (the lanes' tree of partial sums rounds less:
                            more pixels agree with exact arithmetic).  Needs tile_height = 0 and kahan = 0.  1 = one
                            lane per pixel, even where pc_autotune found a lane group faster;
                            0 = the size's pc_autotune result, else one lane.  Default 0 */
} pc_params;

/* Writes the defaults above into *p (no-op for NULL). */
void pc_params_default(pc_params* p);

/* Creates a context for camera intrinsics fx, fy, cx, cy (pixels; fx, fy > 0,
 * all finite), window radius 1..PC_MAX_RADIUS, iterations 0..PC_MAX_ITERATIONS
 * and params (NULL = defaults).  Host only: touches no GPU.  On success *out
 * receives the context; on error *out is set to NULL. */
pc_status pc_create(float fx, float fy, float cx, float cy, int window_radius, int iterations,
                    const pc_params* params, pc_ctx** out);

/* Principal curvatures of one range image (the whole pipeline of Sec. 3.2).
 *   depth      device, H*W floats (read only)
 *   k1_out     device, H*W floats: larger principal curvature, 1/m
 *   k2_out     device, H*W floats: smaller principal curvature, 1/m
 *   normal_out device, H*W*3 floats, or NULL to skip the refined normals
 * H == 0 or W == 0 is a valid empty image (PC_OK, nothing enqueued). */
pc_status pc_compute(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* k1_out,
                     float* k2_out, float* normal_out);

/* The same from and to HOST buffers: copies depth to device staging buffers
 * owned by ctx, computes, and copies k1, k2 (and normal when not NULL) back,
 * all ordered on `stream` (the work starts after what `stream` already holds,
 * and `stream` completes when the results are on the host).  An image of
 * several waves of thread blocks goes in up to eight bands of tile rows whose
 * copies in, kernels and copies out overlap, on streams owned by ctx; a
 * smaller one runs on `stream` itself.  Results are those of pc_compute, bit
 * for bit.  The host buffers must stay valid until the stream is
 * synchronised; pinned buffers let the copies run asynchronously.  Staging
 * buffers are (re)allocated on the current device when a larger image arrives
 * (PC_ERR_OOM if that fails); successive calls on one ctx must use one
 * stream, or synchronise in between. */
pc_status pc_compute_host(pc_ctx* ctx, const float* depth_host, int H, int W, void* stream,
                          float* k1_host, float* k2_host, float* normal_host);

/* Range storage formats of pc_pack_depth / pc_compute_packed. */
#define PC_DEPTH_F16 1           /* IEEE half offsets from a per-tile FP32 base */
#define PC_DEPTH_BF16 2          /* bfloat16 offsets from a per-tile FP32 base */
#define PC_PACK_TILE_W 32        /* pixels per storage tile: 32 columns x 8 rows */
#define PC_PACK_TILE_H 8

/* Packs a float32 range image into centred 16-bit storage: for each 32x8
 * tile (row-major over ceil(W/32) x ceil(H/8) tiles) one FP32 base, the
 * midpoint of its valid ranges, and per pixel the offset (range - base)
 * rounded to the nearest FP16 or BF16 value (format PC_DEPTH_F16 or
 * PC_DEPTH_BF16).  Pixels without a valid range store NaN.
 *   depth     device, H*W floats
 *   packed    device, H*W 16-bit values (2-byte aligned)
 *   tile_base device, ceil(W/32)*ceil(H/8) floats */
pc_status pc_pack_depth(pc_ctx* ctx, const float* depth, int H, int W, int format, void* stream,
                        unsigned short* packed, float* tile_base);

/* pc_compute reading the packed storage of pc_pack_depth (range = base +
 * offset, in FP32).  The arithmetic after loading is that of pc_compute; the
 * storage rounding is the only difference (its error against the FP64 oracle
 * is measured, not bounded by the FP32 tolerance).  Windows of radius 3, 7
 * and 11 (dense, plain sums) run kernels with unrolled columns, others the
 * run-time-radius kernels; both give the same bits. */
pc_status pc_compute_packed(pc_ctx* ctx, const unsigned short* packed, const float* tile_base,
                            int format, int H, int W, void* stream, float* k1_out, float* k2_out,
                            float* normal_out);

/* One frame of a batch: its own size, intrinsics (pixels) and device buffers,
 * with the layouts of pc_compute. */
typedef struct pc_frame {
    const float* depth;  /* device, H*W floats */
    int H, W;            /* 0 <= H, W <= PC_MAX_DIM; an empty frame is skipped */
    float fx, fy, cx, cy;
    float* k1;           /* device, H*W floats */
    float* k2;           /* device, H*W floats */
    float* normal;       /* device, H*W*3 floats, or NULL */
} pc_frame;

/* One frame of pc_compute_packed_batch: the packed storage of pc_pack_depth
 * (offsets: H*W 16-bit values; bases: one float per 32 x 8 tile, row-major
 * over ceil(H/8) x ceil(W/32) tiles), its size, intrinsics and outputs as in
 * pc_frame. */
typedef struct pc_packed_frame {
    const unsigned short* packed;  /* device, H*W, 2-byte aligned */
    const float* tile_base;        /* device, 4-byte aligned */
    int H, W;                      /* 0 <= H, W <= PC_MAX_DIM; an empty frame is skipped */
    float fx, fy, cx, cy;
    float* k1;                     /* device, H*W floats */
    float* k2;                     /* device, H*W floats */
    float* normal;                 /* device, H*W*3 floats, or NULL */
} pc_packed_frame;

/* The method on n frames of any sizes and intrinsics (0 <= n <= PC_MAX_BATCH)
 * in one persistent launch over a flattened queue of (frame, tile) items,
 * with the window radius, iterations and parameters of ctx.  `frames` is host
 * memory, read during the call.  The frame table is staged through one of two
 * page-locked buffers owned by ctx and copied into device scratch owned by ctx
 * (allocated on the first call, grown to the next power of two of n; the call
 * may wait for the batch before the previous one to finish reading its
 * buffer).  The launch uses one thread per pixel, or the lane group that
 * params.lanes_per_pixel forces (autotune plans do not apply to a batch).
 * Results equal those of pc_compute frame by frame, bit for bit, where
 * pc_compute uses the same lanes per pixel (always, unless a pc_autotune plan
 * chose a lane group for that size).  Successive batch calls on one ctx must use one stream, or synchronise in
 * between, because the device scratch is shared. */
pc_status pc_compute_batch(pc_ctx* ctx, const pc_frame* frames, int n, void* stream);

/* pc_compute_batch for frames held in the 16-bit range storage of
 * pc_pack_depth, all in one format (PC_DEPTH_F16 or PC_DEPTH_BF16): n frames
 * (0 <= n <= PC_MAX_BATCH) of any sizes and intrinsics in one persistent
 * launch over a flattened queue of their 32 x 8 tiles, with the window radius,
 * iterations and parameters of ctx (one thread per pixel; lanes_per_pixel and
 * tile_height do not apply).  Results equal pc_compute_packed frame by frame,
 * bit for bit (Sec. 3.2 per pixel; the storage is ours, see pc_pack_depth).
 * It uses ctx's batch scratch and staging like pc_compute_batch: successive
 * batch calls on one ctx must use one stream, or synchronise in between.
 * Arguments are checked before anything is enqueued (PC_ERR_INVALID_ARG). */
pc_status pc_compute_packed_batch(pc_ctx* ctx, const pc_packed_frame* frames, int n, int format, void* stream);

/* pc_compute_batch for callers that cannot allocate device memory.  Some
 * host programs own every byte of device memory themselves (a framework's
 * pool whose accounting must stay exact, or a fixed budget reserved at
 * start-up), and latency-bound loops cannot afford cudaMalloc, which can wait
 * for the whole device.  This entry point allocates nothing: its scratch (the
 * tile counter and a frame table of at most PC_STATIC_MAX_FRAMES frames) is a
 * fixed array inside the library (about 19 KB, held on every GPU that loads
 * the library until the process exits), and the frame table is staged
 * through a fixed host array.  The paper has no counterpart.  It runs the
 * kernel variant pc_compute_batch runs with the same ctx (the lane group that
 * params.lanes_per_pixel forces, else one thread per pixel), so the results
 * equal pc_compute_batch's bit for bit.
 *   - n > PC_STATIC_MAX_FRAMES is rejected with PC_ERR_INVALID_ARG (message
 *     in pc_last_error); other arguments as for pc_compute_batch.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.  This header makes no statement on capturing later
 *     calls into a CUDA graph.
 *   - The frame table is copied from pageable host memory inside the
 *     library, which the next call overwrites once this one has returned.
 *   - Every call uses the same array (the counter is cleared by each call, the
 *     table overwritten), so calls that overlap on the GPU -- on different
 *     streams or from different threads -- race: keep them on one stream or
 *     synchronise in between. */
#define PC_STATIC_MAX_FRAMES 256
pc_status pc_compute_batch_static(pc_ctx* ctx, const pc_frame* frames, int n, void* stream);

/* The method on n frames held in HOST memory (0 <= n; the pc_frame pointers
 * are host addresses, page-locked for the copies to overlap; normal may be
 * NULL).  Frames are taken in order in chunks of at most
 * PC_HOST_CHUNK_PIXELS pixels or PC_MAX_BATCH frames (a larger frame is a
 * chunk of its own; the first chunk takes at most an eighth of that, and over
 * the last two chunks' worth of pixels each chunk takes half of what is left,
 * so that the copies that nothing overlaps -- the first in, the last out --
 * stay short); each chunk's ranges are copied into one of two device
 * staging slots owned by ctx, computed by one pc_compute_batch launch and its
 * results copied back.  Copies in, computation and copies out run on four
 * streams owned by ctx (two for computation: chunks alternate between them,
 * each with its own batch scratch, so that the next chunk's kernel can start
 * while the last tiles of the previous one finish), ordered by events, so that
 * the copies of one chunk overlap the computation of the chunks beside it.  The work starts after
 * what is already enqueued on `stream`, and `stream` waits for the last copy
 * out: once it is synchronised every result is on the host.  Host buffers
 * must stay valid until then.  Results equal pc_compute_batch's bit for bit.  The
 * ctx's batch scratch is used on the internal compute streams: do not run
 * pc_compute_batch on the same ctx concurrently.  Staging slots grow to the
 * largest chunk seen (24 B per pixel each).  Errors: argument errors are
 * reported before anything is enqueued; a CUDA error in the middle of the
 * call (e.g. PC_ERR_OOM growing a slot) returns at once, while chunks already
 * enqueued still run on the internal streams -- synchronise the device before
 * reusing the host buffers after an error. */
#define PC_HOST_CHUNK_PIXELS 4194304  /* 4 Mi pixels */
pc_status pc_compute_host_batch(pc_ctx* ctx, const pc_frame* frames, int n, void* stream);

/* Organised point cloud of a range image: the back-projection of Sec. 3
 * (first step of the pipeline of Sec. 3.2) written out for downstream use.
 *   depth  device, H*W floats
 *   xyz    device, H*W*3 floats: for pixel (u, v), u the column and v the row,
 *          ((u - cx) Z / fx, (v - cy) Z / fy, Z) in metres, NaN where the range
 *          is not valid (Z <= 0, infinite or NaN).  16-byte aligned buffers and
 *          W a multiple of 4 take the vectorised path; any 4-byte aligned
 *          buffers work.
 * H == 0 or W == 0 is a valid empty image. */
pc_status pc_backproject(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* xyz);

/* Field of initial normals alone (Sec. 3.2.1, Eq. initialnormal): for every
 * pixel with a valid range the least-squares plane z = a x + b y + c through
 * the valid back-projected points of its (2 normal_radius + 1)^2 patch,
 * normal = (-a, -b, 1) / sqrt(1 + a^2 + b^2), camera frame, n_z > 0.  NaN
 * where the range is invalid, fewer than 3 patch points are valid or the
 * 2x2 system is singular (det M <= det_tol (tr M)^2).  These are the normals
 * pc_compute starts its iterations from (same arithmetic).
 *   depth   device, H*W floats
 *   normal  device, H*W*3 floats */
pc_status pc_initial_normals(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* normal);

/* Times the kernel variants on this image -- 32x8 and 32x4 tiles with one
 * thread per pixel, and 2, 4 or 8 lanes per pixel (only the one-lane tiles
 * when params.lanes_per_pixel is 1) -- with one warm-up and three timed runs
 * of each on `stream`, which it synchronises; remembers the fastest for
 * images of this H x W in ctx (up to 16 sizes; the oldest is forgotten
 * first) and leaves the last run's results in the outputs (layouts as
 * pc_compute).  pc_compute and pc_compute_host then use it for that size;
 * pc_compute_batch does not (one lane per pixel unless params force a lane
 * group).  Has no effect on the choice when params.tile_height or
 * params.lanes_per_pixel > 1 fixes it. */
pc_status pc_autotune(pc_ctx* ctx, const float* depth, int H, int W, void* stream, float* k1_out,
                      float* k2_out, float* normal_out);

/* Tile height (8, 4, 2 or 1 pixel rows) pc_compute uses for an H x W image on
 * the current device; 0 for a NULL context or sizes out of range. */
int pc_plan_tile_height(pc_ctx* ctx, int H, int W);

/* Lanes per pixel (1, 2, 4 or 8) pc_compute uses for an H x W image on the
 * current device; 0 for a NULL context or sizes out of range. */
int pc_plan_lanes_per_pixel(pc_ctx* ctx, int H, int W);

/* The plans of ctx -- per image size, the variant pc_autotune found fastest
 * (or pc_plans_import gave) -- to keep them across processes: plans are a
 * property of the GPU model and of the window radius, stride, iterations and
 * precision of ctx, not of the frames.  Writes up to `capacity` plans, oldest
 * first, into H, W, tile_height (8, 4, 2 or 1) and lanes_per_pixel (1, 2, 4
 * or 8), and returns how many plans ctx holds (at most 16; capacity 0 with
 * NULL arrays asks for the count); -1 for a NULL ctx or bad arrays. */
int pc_plans_export(const pc_ctx* ctx, int* H, int* W, int* tile_height, int* lanes_per_pixel, int capacity);

/* Adds n plans (0 <= n <= 64) to ctx as pc_autotune would remember them, in
 * order (with more than 16 sizes the oldest are forgotten first).  An entry
 * with a size out of range or empty, or a (tile_height, lanes_per_pixel) pair
 * that is not a variant of this context, is PC_ERR_INVALID_ARG and nothing is
 * added.  Host only: touches no GPU. */
pc_status pc_plans_import(pc_ctx* ctx, const int* H, const int* W, const int* tile_height,
                          const int* lanes_per_pixel, int n);

/* Frees the context, its staging buffers, batch scratch and graphs
 * (synchronising the device first when it owns any).  NULL is a no-op
 * returning PC_OK. */
pc_status pc_destroy(pc_ctx* ctx);

/* Static description of a status code. */
const char* pc_status_string(pc_status s);

/* Message of the last failing CUDA call seen by ctx ("" if none; ctx may be NULL). */
const char* pc_last_error(const pc_ctx* ctx);

/* Measurement utility, not part of the method (the paper has no counterpart):
 * the single-precision issue ceiling of the current GPU, against which the
 * curvature kernels' counted FLOP/s are reported.  Enqueues on `stream` one
 * launch of `blocks` CTAs of 256 threads; each thread runs `iters` rounds of 32
 * independent fused multiply-adds (packed = 1: as 16 packed FP32x2
 * instructions; packed = 0: as 32 scalar ones), all reusing the same two
 * operand registers, and writes one float to sink[CTA * 256 + thread] so that
 * no work is removed.  sink: caller-owned device memory of sink_len >= blocks
 * * 256 floats, 4-byte aligned.  *flop_out (may be NULL) receives the launch's
 * FP32 FLOP (2 per multiply-add).  PC_ERR_INVALID_ARG for bad sizes or a sink
 * that is not device memory; PC_ERR_CUDA if the launch fails.  Time it with
 * CUDA events on `stream`; it changes no GPU setting. */
pc_status pc_fp32_peak_kernel(int blocks, int iters, int packed, float* sink, long long sink_len, void* stream,
                              double* flop_out);

/* Design measurement, not part of the method (the paper has no counterpart):
 * times the window moments of the re-weighted iterations (Sec. 3.2.3, Eq.
 * iter_reweighted_update: J^T W J and J^T W eps over a 15 x 15 window) on
 * synthetic windows, accumulated either on the FP32 pipe as the curvature
 * kernels do (mode 0) or with tensor cores (mode 1: mma.sync m16n8k8 TF32,
 * three products per block for single-precision accuracy, the features staged
 * in shared memory per warp, J^T W eps on the FP32 pipe).  Both modes share
 * the per-point work of the curvature kernels (coordinates, residual, weight,
 * Jacobian).  Enqueues one launch on `stream` over `pixels` windows (in tiles
 * of 32 x 8) for `iters` iterations; each thread writes one float to
 * sink[CTA * 256 + thread] so that no work is removed.  sink: caller-owned
 * device memory of sink_len floats, at least 512 per SM of the GPU;
 * *blocks_out (may be NULL) receives the CTAs launched.  PC_ERR_INVALID_ARG
 * for bad arguments or a short sink; PC_ERR_CUDA if the launch fails. */
pc_status pc_moments_probe(int mode, int pixels, int iters, float* sink, long long sink_len, void* stream,
                           int* blocks_out);

#ifdef __cplusplus
}
#endif

#endif /* PCURV_H */
