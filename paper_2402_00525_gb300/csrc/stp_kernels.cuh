// stp_kernels.cuh -- launch interfaces between the C-ABI host code (stp_api.cu) and the
// kernels of libstp. Internal to the library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "stp_common.cuh"

namespace stp {

struct PipeArgs {
    // inputs: the scene table (device copy in the workspace; pointers caller owned)
    const SceneDesc* scenes;
    int nscenes;
    long long threads;       // per-Gaussian thread count: sum over scenes of n rounded up to kSceneAlign
    long long rec_threads;   // per-record thread count: sum over scenes of n * views, rounded likewise
    long long m;             // render records: sum over views of the view's scene size
    int nviews, lb_threshold, flags, mode, window_k, tail, mid, head;
    float eps_o, t_min, alpha_max, inv_scale_max, dilation, znear;
    float bg[3];
    int total_tiles;
    long long total_pixels;
    // workspace regions
    const ViewDesc* views;
    Status* status;
    float4* geom;            // [m*kRecFloat4]
    float* view_z;           // [V*N] camera-space depth of the mean (ablation B's tile key)
    ushort4* rect;           // [V*N]
    uint32_t* counts;        // [V*N]
    uint32_t* keep_mask;     // [V*N] kept candidate tiles of the per-thread path (bit k = k-th tile)
    uint32_t* offsets;       // [V*N]
    unsigned long long* scan_partials;
    uint64_t* keys;          // sort buffer B
    uint32_t* vals;
    uint64_t* keys_alt;      // sort buffer A (Duplicate writes here)
    uint32_t* vals_alt;
    uint64_t* dup_keys;      // = keys_alt
    uint32_t* dup_vals;
    const uint64_t* skeys;   // sorted pairs (A or B, see pipeline_sorted_in_alt)
    const uint32_t* svals;
    unsigned long long capacity;
    uint2* ranges;           // [total_tiles]
    int partitioned;         // 1: per-tile counting + placement + per-tile sort (appendix B.3)
    uint32_t* tile_counts;   // [total_tiles] entries per tile (partitioned)
    uint32_t* tile_offsets;  // [total_tiles] exclusive prefix sum of tile_counts
    uint32_t* tile_cursor;   // [total_tiles] placement cursors
    unsigned long long* tile_partials;
    float* tfinal_ws;        // [total_pixels]
    float* pix_state;        // [total_pixels] float4 (C without background, depth)
    uint32_t* dbg_nblend;    // [total_pixels] or null
    unsigned long long* dbg_hash;   // [total_pixels] or null
    int* dbg_trace;          // [total_pixels][kTraceLen] or null
    float* dbg_delta;        // [total_pixels] per-pixel sort error or null
    void* sort_temp;
    size_t sort_temp_bytes;
    int key_bits;
    // outputs
    float* rgb;
    float* depth;
    float* tfinal_out;
    // backward
    const float* d_rgb;
    const float* d_depth;
    float* grad_geom;        // [m*kGradStride] per-(view, Gaussian) 2D gradients (alpha and colour terms)
    float* grad_depth;       // [m*kGradStride] the depth-factor terms (written only with d_depth)
    // stored blend order (HIER forward with a backward to follow): per tile warp (8 per tile)
    // blend_cap x 32 ids, slot k of lane l at (warp * blend_cap + k) * 32 + l; null = replay
    uint32_t* blist;
    uint32_t* blist_count;   // [total_pixels] blends of the pixel (may exceed blend_cap)
    uint32_t* replay_warps;  // [total_tiles * 8] tile warps (gtile * 8 + warp) the backward replays
    int blend_cap;
    int full_max_passes;     // FULL order: host bound on peeling passes (0 = always enough)
    // depth slices (HIER, partitioned sort, slice_k > 0): the first pass sorts each tile's list
    // only up to the first bucket boundary holding >= slice_k entries; the second pass sorts the
    // whole lists of the tiles whose Render warps needed more and renders those warps again
    int slice_k;             // 0 = whole lists in one pass
    int slice_pass;          // 0 first pass, 1 second pass (per-tile sort, Render)
    uint32_t* tile_front;    // [total_tiles] sorted prefix length (tile_counts when whole)
    uint32_t* tile_redo;     // [total_tiles] 1 = sorted whole by the second pass
    uint32_t* redo_warps;    // [total_tiles * 8] queued tile warps (gtile * 8 + warp)
};

// Scene of the thread block whose first thread is t0 (largest s with thread_off <= t0).
__device__ __forceinline__ int scene_of(const PipeArgs& a, long long t0)
{
    int lo = 0, hi = a.nscenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.scenes[mid].thread_off <= t0) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Scene of the per-record thread block whose first thread is t0.
__device__ __forceinline__ int scene_of_rec(const PipeArgs& a, long long t0)
{
    int lo = 0, hi = a.nscenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.scenes[mid].rec_thread_off <= t0) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kTraceLen = 64;
// gradient scratch per (view, Gaussian), two regions of kGradStride floats a record:
// grad_geom: sum dGG d (2), dconic (3), sum dGG (1), dcolour (3), pad (3);
// grad_depth: dm (9), dc (3) -- cleared and read only when the loss has a depth term
constexpr int kGradStride = 12;

cudaError_t launch_tables_init(const ViewDesc* host_views, int nviews, ViewDesc* dev_views,
                               const SceneDesc* host_scenes, int nscenes, SceneDesc* dev_scenes,
                               cudaStream_t s);
// count of kernel launches the library has enqueued (stp_kernel_launches)
void note_launches(int n);

cudaError_t launch_preprocess(const PipeArgs& a, cudaStream_t s);
cudaError_t launch_scan_counts(const PipeArgs& a, cudaStream_t s);
cudaError_t launch_scan_tiles(const PipeArgs& a, cudaStream_t s);
cudaError_t launch_tile_sort(const PipeArgs& a, cudaStream_t s);
size_t tile_sort_smem_bytes();
cudaError_t launch_duplicate(const PipeArgs& a, cudaStream_t s);
cudaError_t launch_ranges(const PipeArgs& a, cudaStream_t s);
// forward with a.slice_pass = 1: the second depth-slice pass over the queued tile warps
cudaError_t launch_render(const PipeArgs& a, bool backward, cudaStream_t s);
cudaError_t launch_backward_preprocess(const PipeArgs& a, cudaStream_t s);

size_t scan_partials_count(long long m);
size_t sort_hist_bytes();
bool pipeline_sorted_in_alt(int key_bits);
cudaError_t pipeline_sort(const PipeArgs& a, cudaStream_t s);
size_t render_smem_bytes(int tail, int mid);
bool render_head_supported(int head);
size_t sort_temp_bytes(long long n);
cudaError_t sort_pairs(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                       long long n, const unsigned long long* n_dev, int key_bits, void* temp,
                       size_t temp_bytes, cudaStream_t s);
long long sort_static_max_n();
cudaError_t sort_pairs_static(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                              long long n, const unsigned long long* n_dev, int key_bits, cudaStream_t s);

}  // namespace stp
