/* stp.h -- C ABI of the GB300 (sm_103a) StopThePop renderer (libstp.so).
 *
 * Hierarchical sorted Gaussian splatting: Radl, Steiner et al., "StopThePop: Sorted Gaussian
 * Splatting for View-Consistent Real-time Rendering", TOG 43(4) 2024, arXiv 2402.00525.
 * The forward pass is the paper's four stages (Sec. 3, Fig. "pipeline"): Preprocess,
 * Duplicate (with exact tile culling and the per-tile t_opt key), a global sort of
 * (tile, depth) keys, and the hierarchical Render with tail / mid / head queues. The backward
 * pass walks the same blend order front to back (Sec. 3.5): the order the forward stored per
 * pixel, or a replay of the queues where it did not fit.
 *
 * Conventions shared by every entry point:
 *   - Every array pointer is a DEVICE pointer owned by the caller unless the comment says
 *     "host". The library never allocates device memory: scratch lives in a caller-owned
 *     workspace sized by stp_workspace_size().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Launches are
 *     asynchronous on it; nothing in stp_render / stp_render_backward synchronises the host.
 *   - Gaussians are float32 structure-of-arrays: means [N,3], log_scales [N,3], quats [N,4]
 *     in (w, x, y, z) order (normalised inside), opacity_logits [N] (opacity = sigmoid),
 *     sh [N, (deg+1)^2, 3] (deg <= 3).
 *   - Cameras map world to camera space as p = R x + t (R row major), OpenCV axes (x right,
 *     y down, z forward), pinhole intrinsics in pixels; pixel (u, v) has its centre at
 *     (u + 0.5, v + 0.5). Tiles are 16 x 16 pixels, row major.
 *   - Images of several views are packed view after view: view v starts at pixel offset
 *     sum_{u<v} W_u H_u; rgb is [pixels, 3] (HWC), depth and T are [pixels].
 *   - Return values are stp_status. Argument errors are detected on the host before any
 *     launch (STP_ERR_ARG, nothing launched). Conditions that only the device can see
 *     (sort-entry capacity exceeded, a bounded wait that gave up) are recorded in the
 *     workspace's status block and read back with stp_read_status() after the stream work.
 *   - stp_last_error() returns a host-side, thread-local message for the last failure.
 */
#ifndef STP_H
#define STP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STP_OK = 0,
    STP_ERR_ARG = 1,            /* invalid argument; nothing was launched                   */
    STP_ERR_CAPACITY = 2,       /* more (Gaussian, tile) entries than the workspace holds    */
    STP_ERR_TIMEOUT = 3,        /* a bounded device wait gave up                             */
    STP_ERR_CUDA = 4,           /* a CUDA runtime call failed (message in stp_last_error)    */
    STP_ERR_NOT_SUPPORTED = 5,  /* parameter combination not compiled in                      */
    STP_ERR_INCONSISTENT = 6    /* a backward's recomputed blend sequence disagreed with the
                                   forward's (status error bit 8): the workspace or the inputs
                                   changed between the two calls                            */
} stp_status;

/* Blend orders (Sec. 3.3, 3.4). HIER: the hierarchical resort (tail / mid / head queues).
 * The others are forward-only comparison orders over the same sorted tile lists: FULL, every
 * Gaussian with alpha >= eps_O in exact per-pixel t_opt order (ties by list position);
 * GLOBAL, tile-list order (the global sort alone); WINDOW, a per-pixel k-buffer of window_k
 * entries (1, 2, 4, 8 or 16) fed in tile-list order.                                      */
enum { STP_MODE_HIER = 0, STP_MODE_FULL = 1, STP_MODE_GLOBAL = 2, STP_MODE_WINDOW = 3 };

/* flag bits of stp_params.flags */
enum {
    STP_FLAG_HEAD_EVICT_FIRST = 1,   /* head queue blends before inserting (alternative reading) */
    STP_FLAG_LEVEL_CENTRE_RAYS = 2,  /* 4x4 / 2x2 depth from the level-centre ray             */
    STP_FLAG_TILE_CENTRE_KEY = 4,    /* tile key from the tile-centre ray                    */
    STP_FLAG_VIEW_DEPTH_KEY = 8,     /* tile key = view-space depth of the mean (3DGS)       */
    STP_FLAG_NO_LOAD_BALANCE = 16,   /* every Gaussian processed by its own thread           */
    STP_FLAG_DEBUG_STATS = 32,       /* workspace also receives per-pixel blend count and hash */
    STP_FLAG_BACKWARD = 64,          /* workspace also holds the backward pass's scratch; the
                                        forward and backward calls must both set it          */
    STP_FLAG_DEBUG_TRACE = 128,      /* workspace also receives, per pixel, the ids of the first
                                        STP_TRACE_LEN blended Gaussians (-1 padded)          */
    STP_FLAG_GLOBAL_SORT = 256,      /* order the entries with one global LSD radix sort of
                                        (tile, depth) keys instead of the default partitioned
                                        per-tile sort (appendix B.3); same result            */
    STP_FLAG_NO_TILE_CULL = 512,     /* Duplicate keeps every tile of a Gaussian's rectangle
                                        (ablation D, Tab. performance_ablation)              */
    STP_FLAG_NO_HIER_CULL = 1024     /* Render does not cull at the 4x4 / 2x2 levels; only the
                                        per-pixel alpha test drops Gaussians (ablation E)     */
};
#define STP_TRACE_LEN 64

typedef struct {
    const float* means;          /* [N,3] */
    const float* log_scales;     /* [N,3] */
    const float* quats;          /* [N,4] (w, x, y, z) */
    const float* opacity_logits; /* [N]   */
    const float* sh;             /* [N, (sh_degree+1)^2, 3] */
    int64_t n;                   /* number of Gaussians, 0 <= n < 2^31                        */
    int32_t sh_degree;           /* 0..3 */
    int32_t reserved;            /* padding to 8 bytes; ignored                              */
} stp_gaussians;

typedef struct {                 /* gradient outputs in the input layout, ACCUMULATED (+=)   */
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_logits;
    float* sh;
} stp_gaussians_grad;

typedef struct {
    float R[9];                  /* world -> camera rotation, row major (host value)          */
    float t[3];
    float fx, fy, cx, cy;        /* pixels */
    int32_t width, height;       /* 1 .. 16384 */
} stp_camera;

typedef struct {
    int32_t tail;                /* tail (4x4) queue size: 32n + 32, n >= 1 (Sec. 3.4)       */
    int32_t mid;                 /* mid (2x2) queue size: 4m + 4, m >= 1                    */
    int32_t head;                /* head (per-pixel) queue size, 1..16                      */
    int32_t lb_threshold;        /* load-balancing threshold in tiles (Sec. 3.4), >= 1      */
    float eps_o;                 /* contribution threshold, 1/255                           */
    float t_min;                 /* transmittance early-out, 1e-4                           */
    float alpha_max;             /* 0.99 */
    float inv_scale_max;         /* bound on entries of S^-1, 1e3 (Sec. 3.2)               */
    float dilation;              /* EWA low-pass added to Sigma2, 0.3                       */
    float frustum_clamp;         /* Jacobian clamp factor, 1.3                              */
    float znear;                 /* near plane, 0.2                                         */
    float bg[3];                 /* background colour                                       */
    int32_t mode;                /* STP_MODE_*                                              */
    int32_t window_k;            /* k of STP_MODE_WINDOW                                    */
    int32_t flags;               /* STP_FLAG_* */
    int32_t blend_cap;           /* 0..4096. With STP_FLAG_BACKWARD in STP_MODE_HIER the forward
                                    Render stores, per pixel, the ids of the first blend_cap
                                    Gaussians it blends, in blend order (workspace regions
                                    blend_ids / blend_count: 1 KB per pixel at 256); the backward
                                    then walks those ids instead of replaying the queues, and
                                    only warps (8x4 pixel strips) with a pixel that blended more
                                    replay the schedule. Same gradients either way (up to the
                                    order of float atomics). 0 = every warp replays.        */
    int64_t max_entries;         /* capacity of (Gaussian, tile) sort entries for one call  */
    int32_t full_max_passes;     /* STP_MODE_FULL: bound on the peeling passes over a tile's list
                                    (each pass blends the next 16 entries of every pixel in
                                    depth order). 0 = list length / 16 + 2, which always
                                    suffices; a smaller bound that runs out stops the tile and
                                    sets status error bit 4 (STP_ERR_TIMEOUT). >= 0        */
    int32_t slice_k;             /* STP_MODE_HIER with the partitioned sort: depth-slice lists.
                                    The per-tile sort orders only the prefix of a tile's list up
                                    to the first boundary of its depth buckets (the sort's own
                                    equal-width buckets over the tile's key range) that holds at
                                    least slice_k entries. A Render warp whose pixels all
                                    terminate within the complete 32-entry batches of that
                                    prefix produced exactly the whole list's result; the others
                                    (counted in stp_run_status.redo_warps) are rendered again
                                    after their tiles' whole lists are sorted. Same images,
                                    hashes, blend orders and gradients as slice_k = 0 (whole
                                    lists). >= 0                                            */
} stp_params;

typedef struct {                 /* device status block, read back by stp_read_status        */
    uint32_t error_bits;         /* 1 capacity exceeded, 2 count mismatch padded, 4 timeout,
                                    8 the backward's blend sequence disagreed with the forward
                                    (recomputed final T or blend count)                      */
    uint32_t mismatched;         /* Gaussians whose Duplicate count differed from Preprocess  */
    uint64_t num_entries;        /* entries the last forward needed (may exceed capacity)    */
    uint64_t capacity;           /* entries the workspace holds                              */
    uint64_t counters[5];        /* with STP_FLAG_DEBUG_STATS, work units of the last forward
                                    Render: [0] (entry, 4x4 subtile) evaluations, [1] 4x4
                                    survivors, [2] (entry, 2x2 quad) evaluations, [3] blends,
                                    [4] (entry, pixel) evaluations                         */
    uint64_t invalid_gaussians;  /* Gaussians the last forward dropped as invalid, summed over
                                    scenes: a non-finite mean, log-scale, quaternion component,
                                    opacity logit or SH coefficient, or a quaternion of squared
                                    length below 1e-20. Such a Gaussian covers no pixel and
                                    receives zero gradient; it is not an error.              */
    uint64_t redo_warps;         /* slice_k > 0: Render warps (8x4 pixel strips) of the last
                                    forward that needed entries past their tile's prefix and
                                    were rendered again over the whole list                  */
} stp_run_status;

typedef struct {                 /* byte offsets of workspace regions (for inspection)       */
    size_t status;               /* stp_run_status                                           */
    size_t views;                /* internal view table                                      */
    size_t scenes;               /* internal scene table                                     */
    size_t geom;                 /* [M] 96-byte render records (layout in stp_common.cuh);
                                    M = sum over views of the N of the view's scene, view
                                    after view, Gaussian id ascending within a view          */
    size_t view_z;               /* [M] float camera-space depth of the projected mean (the tile
                                      key of STP_FLAG_VIEW_DEPTH_KEY)                         */
    size_t rect;                 /* [M] ushort4 tile rectangles [x0, y0, x1, y1)             */
    size_t counts;               /* [M] uint32 entries per (view, Gaussian)                  */
    size_t offsets;              /* [M] uint32 exclusive prefix sum of counts                */
    size_t keep_mask;            /* [M] uint32 kept tiles of rectangles of <= 32 tiles        */
    size_t scan_partials;        /* scan scratch                                             */
    size_t keys, vals;           /* [capacity] uint64 / uint32 radix-sort buffer B           */
    size_t keys_alt, vals_alt;   /* [capacity] radix-sort buffer A (Duplicate output)        */
    size_t sorted_keys;          /* = keys or keys_alt: where the sorted (tile, depth) keys  */
    size_t sorted_vals;          /*   and Gaussian ids end up (the per-tile sort writes the
                                      keys only with STP_FLAG_DEBUG_STATS: Render reads ids) */
    size_t ranges;               /* [total tiles] uint2 [start, end) into the sorted pairs   */
    size_t tfinal;               /* [total pixels] float final transmittance                 */
    size_t pix_state;            /* [total pixels] float4 (colour without background, depth) */
    size_t scratch;              /* sort histogram scratch                                   */
    size_t dbg_nblend;           /* [total pixels] uint32 blends per pixel (flag 32), else 0 */
    size_t dbg_hash;             /* [total pixels] uint64 blend-order hash (flag 32), else 0 */
    size_t dbg_delta;            /* [total pixels] float sort error delta (flag 32): the sum
                                    of t_opt steps backwards along the blend order (Sec. 3.3) */
    size_t grad_geom;            /* [M*24] float backward scratch (flag 64), else 0: M*12 alpha and
                                    colour terms, then M*12 depth-factor terms (used with d_depth) */
    size_t dbg_trace;            /* [total pixels][STP_TRACE_LEN] int32 blend ids (flag 128)  */
    size_t tile_counts;          /* [total tiles] uint32 entries per tile (partitioned sort)  */
    size_t tile_offsets;         /* [total tiles] uint32 first entry of each tile            */
    size_t tile_cursor;          /* [total tiles] uint32 placement cursors                   */
    size_t tile_partials;        /* scan scratch of the tile counts                          */
    size_t blend_ids;            /* [total tiles * 8 warps][blend_cap][32] uint32 stored blend
                                    order (flag 64, HIER, blend_cap > 0), else 0: slot k of the
                                    warp's lane l (pixel of its 8x4 strip) at (w*cap + k)*32 + l */
    size_t blend_count;          /* [total pixels] uint32 blends per pixel (with blend_ids)  */
    size_t replay_warps;         /* [total tiles * 8] uint32 backward work list: tile warps with
                                    a pixel past blend_cap, replayed (with blend_ids)        */
    size_t tile_front;           /* [total tiles] uint32 entries of the sorted prefix (the whole
                                    count when the list is whole); slice_k > 0, else 0, like
                                    the next two regions                                       */
    size_t tile_redo;            /* [total tiles] uint32 1 = the second pass sorts the whole list */
    size_t redo_warps;           /* [total tiles * 8] uint32 tile warps (gtile * 8 + warp) the
                                    second pass renders                                       */
    size_t total;                /* total bytes                                              */
    int64_t capacity;            /* sort-entry capacity                                      */
    int64_t total_tiles, total_pixels;
    int32_t key_bits;            /* bits of the radix-sort key: 32 + bits(total tiles)       */
    int32_t reserved;            /* padding to 8 bytes; written 0                            */
} stp_workspace_layout;

/* Size of the workspace one stp_render call needs for `nviews` cameras of N Gaussians
 * (Sec. 3: per-view records, sort entries, tile ranges, per-pixel T). Host-only, no CUDA
 * call. Returns 0 on invalid arguments (see stp_last_error).                              */
size_t stp_workspace_size(int64_t n, const stp_camera* cams /* host, [nviews] */, int32_t nviews,
                          const stp_params* prm /* host */);

/* Same sizing, with the byte offset of every region (host).                               */
stp_status stp_workspace_layout_get(int64_t n, const stp_camera* cams /* host */, int32_t nviews,
                                    const stp_params* prm /* host */, stp_workspace_layout* out /* host */);

/* Forward pass (Sec. 3): Preprocess -> Duplicate -> per-tile depth sort (appendix B.3;
 * STP_FLAG_GLOBAL_SORT selects one global radix sort instead; with slice_k > 0 it orders only
 * each list's prefix, and a second sort and Render pass over the queued warps follows, whose
 * kernels return at once when nothing was queued) -> hierarchical Render, for
 * `nviews` views of one scene (1 <= nviews <= STP_MAX_VIEWS) in one launch per stage. Writes
 * rgb [pixels,3], depth [pixels] (volumetric depth with phi = t_opt, Sec. 4.1 "Depth
 * Evaluation") and, if not NULL, tfinal [pixels]; pixels are packed view after view, row
 * major within a view. The workspace keeps the state the backward pass needs (sorted lists,
 * records, final T). Asynchronous; call stp_read_status() to learn whether the capacity
 * sufficed (if not, rgb / depth are undefined and num_entries tells the size needed).
 * Launches only kernels and memsets after the first call for a given parameter set (kernel
 * attributes are set once per device), so a call can be recorded under stream capture.  */
stp_status stp_render(const stp_gaussians* g /* host struct of device pointers */,
                      const stp_camera* cams /* host, [nviews] */, int32_t nviews,
                      const stp_params* prm /* host */, void* workspace, size_t ws_bytes,
                      float* rgb, float* depth, float* tfinal, void* stream);

/* Backward pass (Sec. 3.5): walks the forward's blend order front to back using the
 * workspace of the preceding stp_render with the same arguments (which must not have been
 * modified): the per-pixel order stored by the forward (blend_cap > 0), else, and for warps
 * whose pixels blended more than blend_cap Gaussians, a replay of the queues. ACCUMULATES (+=) the gradients of <d_rgb, rgb> + <d_depth, depth> into
 * `grad` (device arrays in the input layout; zero them first for a fresh gradient).
 * d_depth may be NULL. Asynchronous.                                                       */
stp_status stp_render_backward(const stp_gaussians* g, const stp_camera* cams, int32_t nviews,
                               const stp_params* prm, void* workspace, size_t ws_bytes,
                               const float* d_rgb, const float* d_depth,
                               const stp_gaussians_grad* grad /* host struct of device ptrs */,
                               void* stream);

/* Batched rendering of several scenes (each with its own Gaussians and views) in one launch
 * per stage. Scene s (0 <= s < nscenes <= STP_MAX_SCENES) owns views_per_scene[s] consecutive
 * cameras of cams, starting after the views of scenes 0..s-1; the counts sum to nviews
 * (<= STP_MAX_VIEWS). Results are identical to one stp_render call per scene with the same
 * parameters; outputs are packed view after view over all scenes. `n` (host, [nscenes]) is
 * each scene's Gaussian count. The batched backward ACCUMULATES into grads[s] (host array
 * of nscenes structs of device pointers) for scene s.                                     */
#define STP_MAX_SCENES 64
#define STP_MAX_VIEWS 64
size_t     stp_workspace_size_batched(const int64_t* n, const int32_t* views_per_scene, int32_t nscenes,
                                      const stp_camera* cams, int32_t nviews, const stp_params* prm);
stp_status stp_workspace_layout_batched(const int64_t* n, const int32_t* views_per_scene, int32_t nscenes,
                                        const stp_camera* cams, int32_t nviews, const stp_params* prm,
                                        stp_workspace_layout* out);
stp_status stp_render_batched(const stp_gaussians* scenes /* host, [nscenes] */, int32_t nscenes,
                              const int32_t* views_per_scene /* host, [nscenes] */,
                              const stp_camera* cams /* host, [nviews] */, int32_t nviews,
                              const stp_params* prm, void* workspace, size_t ws_bytes,
                              float* rgb, float* depth, float* tfinal, void* stream);
stp_status stp_render_backward_batched(const stp_gaussians* scenes, int32_t nscenes,
                                       const int32_t* views_per_scene, const stp_camera* cams,
                                       int32_t nviews, const stp_params* prm, void* workspace,
                                       size_t ws_bytes, const float* d_rgb, const float* d_depth,
                                       const stp_gaussians_grad* grads /* host, [nscenes] */,
                                       void* stream);

/* Synchronises `stream`, copies the workspace's status block to *out (host) and returns
 * STP_ERR_CAPACITY / STP_ERR_TIMEOUT / STP_ERR_INCONSISTENT if the device recorded that
 * condition (error bits 1 / 4 / 8, in that order of precedence), else STP_OK.              */
stp_status stp_read_status(const void* workspace, stp_run_status* out /* host */, void* stream);

/* Stable LSD radix sort of (uint64 key, uint32 value) pairs on the low `key_bits` bits
 * (1..64), the sort of Sec. 2.1 / 3.4 that orders (tile, depth) keys. keys_in / vals_in are
 * read, keys_out / vals_out receive the sorted pairs; `n` may also be read from the device
 * (n_dev != NULL: the count is min(*n_dev, n)). temp is device scratch of
 * stp_sort_temp_bytes(n) bytes. The four arrays must not overlap. Asynchronous.            */
size_t     stp_sort_temp_bytes(int64_t n);
stp_status stp_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                          uint32_t* vals_out, int64_t n, const uint64_t* n_dev, int32_t key_bits,
                          void* temp, size_t temp_bytes, void* stream);

/* The same sort for callers that cannot allocate device memory: code recording into a CUDA
 * graph under stream capture, plugins whose host framework owns the device memory pool, and
 * loops that must not allocate after start-up. It takes no scratch argument and allocates
 * nothing: its scratch is a fixed device array inside the library, sized for at most
 * STP_SORT_STATIC_MAX_N pairs (12.25 MiB, held by every GPU that loads the library until the
 * process exits). The paper has no counterpart; this is a deployment variant of
 * stp_sort_pairs with the same arguments minus temp and the same results.
 *   - n > STP_SORT_STATIC_MAX_N is rejected with STP_ERR_ARG before any work.
 *   - A call on a stream that is not capturing looks up the array's device address on the
 *     current device (which allocates nothing); a call under stream capture reuses the
 *     address found by the device's last call outside capture. So make one call on each
 *     device before any stream capture, and again after a cudaDeviceReset, which reloads
 *     the library's device code; a capture with no such earlier call fails with
 *     STP_ERR_CUDA.
 *   - All calls share the array: calls whose work overlaps on the GPU (other streams, other
 *     host threads) race and must be serialised by the caller. Nothing in the array needs
 *     to start at zero.                                                                    */
#define STP_SORT_STATIC_MAX_N 1048576
stp_status stp_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, int64_t n, const uint64_t* n_dev, int32_t key_bits,
                                  void* stream);

/* Stage timing with CUDA events (Sec. 4.3 reports per-stage times). After
 * stp_profile_enable(max_calls), each stp_render / stp_render_backward call on this host
 * thread records STP_NUM_STAGE_EVENTS events on its stream into the next of max_calls slots
 * (further calls are not recorded); max_calls = 0 disables and frees the events.
 * stp_profile_read synchronises the recorded events and writes, per recorded call, the
 * milliseconds of each stage (ms[call * STP_NUM_STAGES + stage]); *ncalls receives the number
 * of calls recorded; recording then restarts at slot 0. Stages of a forward call: 0 status and
 * view table, 1 Preprocess, 2 scan, 3 Duplicate, 4 sort, 5 tile ranges, 6 Render; of a
 * backward call: 4 view and scene tables, 5 clearing the gradient scratch, 6 backward Render,
 * 7 backward Preprocess (the others are 0).                                                                     */
#define STP_NUM_STAGES 8
#define STP_NUM_STAGE_EVENTS (STP_NUM_STAGES + 1)
stp_status stp_profile_enable(int32_t max_calls);
stp_status stp_profile_read(float* ms /* host, [max_calls * STP_NUM_STAGES] */, int32_t max_calls,
                            int32_t* ncalls /* host */);

/* Number of kernels the library has enqueued in this process so far (all threads, all
 * devices; memsets and copies are not counted; a replayed CUDA graph is not counted again). */
uint64_t stp_kernel_launches(void);

/* Thread-local message of the last error on this host thread (empty if none).            */
const char* stp_last_error(void);

/* Library version, e.g. 0x000300 for 0.3.0.                                              */
int32_t stp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STP_H */
