// stp_api.cu -- the C ABI of libstp (declared in include/stp.h): argument checks, the
// workspace layout, and the launch sequence of the forward and backward passes.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/stp.h"
#include "stp_common.cuh"
#include "stp_kernels.cuh"

namespace {

thread_local std::string g_err;
std::atomic<unsigned long long> g_launches{0};

// ---- stage timing (stp_profile_enable / stp_profile_read)
struct Profiler {
    std::vector<cudaEvent_t> ev;     // [max_calls][STP_NUM_STAGE_EVENTS]
    std::vector<int> kind;           // 0 forward, 1 backward per recorded call
    int max_calls = 0, next = 0;
};
thread_local Profiler g_prof;

// event index `e` of the current call, or nullptr if not recording
cudaEvent_t prof_event(int e)
{
    if (g_prof.next >= g_prof.max_calls) return nullptr;
    return g_prof.ev[(size_t)g_prof.next * STP_NUM_STAGE_EVENTS + e];
}
void prof_mark(int e, cudaStream_t s)
{
    cudaEvent_t ev = prof_event(e);
    if (ev) cudaEventRecord(ev, s);
}
void prof_finish(int kind)
{
    if (g_prof.next < g_prof.max_calls) {
        g_prof.kind[g_prof.next] = kind;
        g_prof.next++;
    }
}

stp_status fail(stp_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

stp_status cuda_fail(cudaError_t e, const char* where)
{
    return fail(STP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr int kFlagDebug = 32;      // per-pixel blend count / hash written to the workspace
constexpr int kFlagBackward = 64;   // workspace also holds the backward pass's scratch
constexpr int kFlagTrace = 128;     // per-pixel ids of the first kTraceLen blended Gaussians
constexpr int kFlagGlobalSort = 256;  // one global LSD radix sort instead of the per-tile sort

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

int bits_for(long long v)   // bits needed to store the value v (v >= 1)
{
    int b = 0;
    while ((1LL << b) <= v) b++;
    return b;
}

// Checks shared by every entry point: scene sizes, cameras, parameters.
stp_status check(const int64_t* ns, const int32_t* vps, int32_t nscenes, const stp_camera* cams, int32_t nviews,
                 const stp_params* p)
{
    if (!cams || !p || !ns || !vps) return fail(STP_ERR_ARG, "null camera, parameter or scene-size pointer");
    if (nscenes < 1 || nscenes > stp::kMaxScenes)
        return fail(STP_ERR_ARG, "nscenes = %d out of range [1, %d]", nscenes, stp::kMaxScenes);
    if (nviews < 1 || nviews > stp::kMaxViews)
        return fail(STP_ERR_ARG, "nviews = %d out of range [1, %d]", nviews, stp::kMaxViews);
    long long vsum = 0, threads = 0, m = 0;
    for (int s = 0; s < nscenes; s++) {
        if (ns[s] < 0 || ns[s] >= (1LL << 31))
            return fail(STP_ERR_ARG, "scene %d: n = %lld out of range [0, 2^31)", s, (long long)ns[s]);
        if (vps[s] < 0) return fail(STP_ERR_ARG, "scene %d: negative view count", s);
        vsum += vps[s];
        threads += (ns[s] + stp::kSceneAlign - 1) / stp::kSceneAlign * stp::kSceneAlign;
        m += ns[s] * (long long)vps[s];
    }
    if (vsum != nviews) return fail(STP_ERR_ARG, "views per scene sum to %lld, nviews = %d", vsum, nviews);
    if (threads / 256 >= (1LL << 31) || (m + 256LL * nscenes) / 256 >= (1LL << 31))
        return fail(STP_ERR_ARG, "scenes too large for one launch sequence");
    for (int v = 0; v < nviews; v++) {
        const stp_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
            return fail(STP_ERR_ARG, "view %d: image size %dx%d out of range", v, c.width, c.height);
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy))
            return fail(STP_ERR_ARG, "view %d: invalid intrinsics", v);
    }
    if (p->tail < 64 || p->tail > 256 || p->tail % 32)
        return fail(STP_ERR_ARG, "tail = %d: must be 32n+32 in [64, 256]", p->tail);
    if (p->mid < 8 || p->mid > stp::kMaxMid || p->mid % 4)
        return fail(STP_ERR_ARG, "mid = %d: must be 4m+4 in [8, %d]", p->mid, stp::kMaxMid);
    if (!stp::render_head_supported(p->head))
        return fail(STP_ERR_NOT_SUPPORTED, "head = %d: compiled sizes are 1, 2, 4, 8, 16", p->head);
    if (p->lb_threshold < 1) return fail(STP_ERR_ARG, "lb_threshold must be >= 1");
    if (!(p->eps_o > 0.f && p->eps_o < 1.f)) return fail(STP_ERR_ARG, "eps_o must be in (0, 1)");
    if (!(p->t_min >= 0.f && p->t_min < 1.f)) return fail(STP_ERR_ARG, "t_min must be in [0, 1)");
    if (!(p->alpha_max > p->eps_o && p->alpha_max < 1.f)) return fail(STP_ERR_ARG, "alpha_max must be in (eps_o, 1)");
    if (!(p->inv_scale_max > 0.f)) return fail(STP_ERR_ARG, "inv_scale_max must be > 0");
    if (!(p->dilation >= 0.f) || !(p->frustum_clamp > 0.f) || !(p->znear > 0.f))
        return fail(STP_ERR_ARG, "dilation >= 0, frustum_clamp > 0 and znear > 0 required");
    if (p->mode < STP_MODE_HIER || p->mode > STP_MODE_WINDOW)
        return fail(STP_ERR_ARG, "mode %d: must be one of STP_MODE_HIER, FULL, GLOBAL, WINDOW", p->mode);
    if (p->mode == STP_MODE_WINDOW && !stp::render_head_supported(p->window_k))
        return fail(STP_ERR_NOT_SUPPORTED, "window_k = %d: compiled sizes are 1, 2, 4, 8, 16", p->window_k);
    if (p->blend_cap < 0 || p->blend_cap > 4096)
        return fail(STP_ERR_ARG, "blend_cap = %d: must be in [0, 4096]", p->blend_cap);
    if (p->max_entries < 0 || p->max_entries >= 0xFFFFFFFFLL)
        return fail(STP_ERR_ARG, "max_entries must be in [0, 2^32 - 1)");
    if (p->full_max_passes < 0) return fail(STP_ERR_ARG, "full_max_passes must be >= 0");
    if (p->slice_k < 0) return fail(STP_ERR_ARG, "slice_k must be >= 0");
    return STP_OK;
}

struct Plan {
    stp_workspace_layout L;
    long long m;                       // render records: sum over views of the view's scene size
    long long threads;                 // per-Gaussian threads (scenes aligned to kSceneAlign)
    long long rec_threads;             // per-(Gaussian, view) threads (likewise)
    std::vector<stp::ViewDesc> views;
    std::vector<stp::SceneDesc> scenes;   // sizes and view ranges; pointers filled per call
};

// Depth-slice list building applies to the hierarchical Render over the partitioned sort.
bool slicing(const stp_params* p)
{
    return p->slice_k > 0 && p->mode == STP_MODE_HIER && !(p->flags & kFlagGlobalSort);
}

void make_plan(const int64_t* ns, const int32_t* vps, int32_t nscenes, const stp_camera* cams, int32_t nviews,
               const stp_params* p, Plan& P)
{
    std::memset(&P.L, 0, sizeof P.L);
    P.views.resize(nviews);
    P.scenes.resize(nscenes);
    long long tiles = 0, pixels = 0, rec = 0, threads = 0, rec_threads = 0;
    int v = 0;
    for (int sc = 0; sc < nscenes; sc++) {
        stp::SceneDesc& S = P.scenes[sc];
        std::memset(&S, 0, sizeof S);
        S.n = (int)ns[sc];
        S.view_begin = v;
        S.view_end = v + vps[sc];
        S.thread_off = threads;
        S.rec_thread_off = rec_threads;
        threads += (ns[sc] + stp::kSceneAlign - 1) / stp::kSceneAlign * stp::kSceneAlign;
        rec_threads += (ns[sc] * vps[sc] + stp::kSceneAlign - 1) / stp::kSceneAlign * stp::kSceneAlign;
        for (; v < S.view_end; v++) {
            const stp_camera& c = cams[v];
            stp::ViewDesc& d = P.views[v];
            std::memset(&d, 0, sizeof d);
            for (int k = 0; k < 9; k++) d.R[k] = c.R[k];
            for (int k = 0; k < 3; k++) d.t[k] = c.t[k];
            for (int k = 0; k < 3; k++)   // o = -R^T t
                d.o[k] = -(c.R[k] * c.t[0] + c.R[3 + k] * c.t[1] + c.R[6 + k] * c.t[2]);
            d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
            d.ifx = 1.f / c.fx; d.ify = 1.f / c.fy;
            d.limx = p->frustum_clamp * 0.5f * c.width / c.fx;
            d.limy = p->frustum_clamp * 0.5f * c.height / c.fy;
            d.W = c.width; d.H = c.height;
            d.tiles_x = (c.width + 15) / 16;
            d.tiles_y = (c.height + 15) / 16;
            d.tile_off = (int)tiles;
            d.pix_off = pixels;
            d.rec_off = rec;
            tiles += (long long)d.tiles_x * d.tiles_y;
            pixels += (long long)c.width * c.height;
            rec += ns[sc];
        }
    }
    P.m = rec;
    P.threads = threads;
    P.rec_threads = rec_threads;
    long long cap = p->max_entries > 0 ? p->max_entries : std::max<long long>(1LL << 20, 4LL * P.m);
    if (cap > 0xFFFFFFFELL) cap = 0xFFFFFFFELL;
    stp_workspace_layout& L = P.L;
    L.capacity = cap;
    L.total_tiles = tiles;
    L.total_pixels = pixels;
    L.key_bits = 32 + bits_for(tiles);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    L.status = take(sizeof(stp::Status));
    L.views = take(sizeof(stp::ViewDesc) * nviews);
    L.scenes = take(sizeof(stp::SceneDesc) * nscenes);
    L.geom = take((size_t)P.m * 16 * stp::kRecFloat4);
    L.view_z = take((size_t)P.m * 4);
    L.rect = take((size_t)P.m * 8);
    L.counts = take((size_t)P.m * 4);
    L.offsets = take((size_t)P.m * 4);
    L.keep_mask = take((size_t)P.m * 4);
    L.scan_partials = take(stp::scan_partials_count(P.m) * 8);
    L.keys = take((size_t)cap * 8);
    L.vals = take((size_t)cap * 4);
    L.keys_alt = take((size_t)cap * 8);
    L.vals_alt = take((size_t)cap * 4);
    L.ranges = take((size_t)tiles * 8);
    L.tfinal = take((size_t)pixels * 4);
    L.pix_state = take((size_t)pixels * 16);
    L.scratch = take(stp::sort_hist_bytes());
    L.dbg_nblend = L.dbg_hash = L.dbg_delta = 0;
    if (p->flags & kFlagDebug) {
        L.dbg_nblend = take((size_t)pixels * 4);
        L.dbg_hash = take((size_t)pixels * 8);
        L.dbg_delta = take((size_t)pixels * 4);
    }
    const bool in_alt = (p->flags & kFlagGlobalSort) && stp::pipeline_sorted_in_alt(L.key_bits);
    L.sorted_keys = in_alt ? L.keys_alt : L.keys;
    L.sorted_vals = in_alt ? L.vals_alt : L.vals;
    L.tile_counts = take((size_t)tiles * 4);
    L.tile_offsets = take((size_t)tiles * 4);
    L.tile_cursor = take((size_t)tiles * 4);
    L.tile_partials = take(stp::scan_partials_count(tiles) * 8);
    L.grad_geom = 0;
    if (p->flags & kFlagBackward) L.grad_geom = take((size_t)P.m * 2 * stp::kGradStride * 4);   // both regions
    L.blend_ids = L.blend_count = L.replay_warps = 0;
    if ((p->flags & kFlagBackward) && p->mode == STP_MODE_HIER && p->blend_cap > 0) {
        L.blend_ids = take((size_t)tiles * 256 * (size_t)p->blend_cap * 4);
        L.blend_count = take((size_t)pixels * 4);
        L.replay_warps = take((size_t)tiles * 8 * 4);
    }
    L.dbg_trace = 0;
    if (p->flags & kFlagTrace) L.dbg_trace = take((size_t)pixels * stp::kTraceLen * 4);
    L.tile_front = L.tile_redo = L.redo_warps = 0;
    if (slicing(p)) {
        L.tile_front = take((size_t)tiles * 4);
        L.tile_redo = take((size_t)tiles * 4);
        L.redo_warps = take((size_t)tiles * 8 * 4);
    }
    L.total = o;
}

stp::PipeArgs make_args(const stp_params* p, const Plan& P, void* ws)
{
    stp::PipeArgs a;
    std::memset(&a, 0, sizeof a);
    char* b = (char*)ws;
    const stp_workspace_layout& L = P.L;
    a.scenes = (const stp::SceneDesc*)(b + L.scenes);
    a.nscenes = (int)P.scenes.size();
    a.threads = P.threads;
    a.rec_threads = P.rec_threads;
    a.m = P.m;
    a.nviews = (int)P.views.size();
    a.lb_threshold = p->lb_threshold; a.flags = p->flags; a.mode = p->mode; a.window_k = p->window_k;
    a.tail = p->tail; a.mid = p->mid; a.head = p->head;
    a.eps_o = p->eps_o; a.t_min = p->t_min; a.alpha_max = p->alpha_max;
    a.inv_scale_max = p->inv_scale_max; a.dilation = p->dilation; a.znear = p->znear;
    for (int k = 0; k < 3; k++) a.bg[k] = p->bg[k];
    a.total_tiles = (int)L.total_tiles;
    a.total_pixels = L.total_pixels;
    a.views = (const stp::ViewDesc*)(b + L.views);
    a.status = (stp::Status*)(b + L.status);
    a.geom = (float4*)(b + L.geom);
    a.view_z = (float*)(b + L.view_z);
    a.rect = (ushort4*)(b + L.rect);
    a.counts = (uint32_t*)(b + L.counts);
    a.offsets = (uint32_t*)(b + L.offsets);
    a.keep_mask = (uint32_t*)(b + L.keep_mask);
    a.scan_partials = (unsigned long long*)(b + L.scan_partials);
    a.keys = (uint64_t*)(b + L.keys);
    a.vals = (uint32_t*)(b + L.vals);
    a.keys_alt = (uint64_t*)(b + L.keys_alt);
    a.vals_alt = (uint32_t*)(b + L.vals_alt);
    a.dup_keys = a.keys_alt;
    a.dup_vals = a.vals_alt;
    a.skeys = (const uint64_t*)(b + L.sorted_keys);
    a.svals = (const uint32_t*)(b + L.sorted_vals);
    a.capacity = (unsigned long long)L.capacity;
    a.ranges = (uint2*)(b + L.ranges);
    a.tfinal_ws = (float*)(b + L.tfinal);
    a.pix_state = (float*)(b + L.pix_state);
    a.dbg_nblend = L.dbg_nblend ? (uint32_t*)(b + L.dbg_nblend) : nullptr;
    a.dbg_hash = L.dbg_hash ? (unsigned long long*)(b + L.dbg_hash) : nullptr;
    a.dbg_delta = L.dbg_delta ? (float*)(b + L.dbg_delta) : nullptr;
    a.sort_temp = b + L.scratch;
    a.sort_temp_bytes = stp::sort_hist_bytes();
    a.key_bits = L.key_bits;
    a.grad_geom = L.grad_geom ? (float*)(b + L.grad_geom) : nullptr;
    a.grad_depth = L.grad_geom ? a.grad_geom + (size_t)P.m * stp::kGradStride : nullptr;
    a.blist = L.blend_ids ? (uint32_t*)(b + L.blend_ids) : nullptr;
    a.blist_count = L.blend_count ? (uint32_t*)(b + L.blend_count) : nullptr;
    a.replay_warps = L.replay_warps ? (uint32_t*)(b + L.replay_warps) : nullptr;
    a.blend_cap = L.blend_ids ? p->blend_cap : 0;
    a.full_max_passes = p->full_max_passes;
    a.dbg_trace = L.dbg_trace ? (int*)(b + L.dbg_trace) : nullptr;
    a.partitioned = (p->flags & kFlagGlobalSort) ? 0 : 1;
    a.tile_counts = (uint32_t*)(b + L.tile_counts);
    a.tile_offsets = (uint32_t*)(b + L.tile_offsets);
    a.tile_cursor = (uint32_t*)(b + L.tile_cursor);
    a.tile_partials = (unsigned long long*)(b + L.tile_partials);
    a.slice_k = L.tile_front ? p->slice_k : 0;
    a.slice_pass = 0;
    a.tile_front = L.tile_front ? (uint32_t*)(b + L.tile_front) : nullptr;
    a.tile_redo = L.tile_redo ? (uint32_t*)(b + L.tile_redo) : nullptr;
    a.redo_warps = L.redo_warps ? (uint32_t*)(b + L.redo_warps) : nullptr;
    return a;
}

__global__ void k_status_init(stp::Status* st, unsigned long long cap)
{
    st->error_bits = 0;
    st->mismatched = 0;
    st->num_entries = 0;
    st->capacity = cap;
    for (int k = 0; k < 5; k++) st->counters[k] = 0;
    st->invalid = 0;
    st->redo_n = 0;
    st->redo_next = 0;
}

stp_status check_scene(const stp_gaussians& g, int s)
{
    if (g.sh_degree < 0 || g.sh_degree > 3) return fail(STP_ERR_ARG, "scene %d: sh_degree must be 0..3", s);
    if (g.n > 0 && (!g.means || !g.log_scales || !g.quats || !g.opacity_logits || !g.sh))
        return fail(STP_ERR_ARG, "scene %d: null Gaussian parameter array", s);
    return STP_OK;
}

// Validates the scenes, builds the plan and fills the scene table's input pointers.
stp_status prepare(const stp_gaussians* scenes, int32_t nscenes, const int32_t* vps, const stp_camera* cams,
                   int32_t nviews, const stp_params* prm, size_t ws_bytes, const void* workspace, Plan& P)
{
    if (!scenes) return fail(STP_ERR_ARG, "null Gaussian struct");
    if (nscenes < 1 || nscenes > stp::kMaxScenes)
        return fail(STP_ERR_ARG, "nscenes = %d out of range [1, %d]", nscenes, stp::kMaxScenes);
    std::vector<int64_t> ns(nscenes);
    for (int s = 0; s < nscenes; s++) ns[s] = scenes[s].n;
    stp_status st = check(ns.data(), vps, nscenes, cams, nviews, prm);
    if (st != STP_OK) return st;
    for (int s = 0; s < nscenes; s++)
        if ((st = check_scene(scenes[s], s)) != STP_OK) return st;
    make_plan(ns.data(), vps, nscenes, cams, nviews, prm, P);
    if (!workspace || ws_bytes < P.L.total)
        return fail(STP_ERR_ARG, "workspace of %zu bytes, %zu needed", ws_bytes, P.L.total);
    for (int s = 0; s < nscenes; s++) {
        stp::SceneDesc& S = P.scenes[s];
        const stp_gaussians& g = scenes[s];
        S.means = g.means; S.log_scales = g.log_scales; S.quats = g.quats;
        S.logits = g.opacity_logits; S.sh = g.sh;
        S.sh_k = (g.sh_degree + 1) * (g.sh_degree + 1);
    }
    return STP_OK;
}

stp_status render_impl(const stp_gaussians* scenes, int32_t nscenes, const int32_t* vps, const stp_camera* cams,
                       int32_t nviews, const stp_params* prm, void* workspace, size_t ws_bytes, float* rgb,
                       float* depth, float* tfinal, void* stream)
{
    g_err.clear();
    Plan P;
    stp_status st = prepare(scenes, nscenes, vps, cams, nviews, prm, ws_bytes, workspace, P);
    if (st != STP_OK) return st;
    if (!rgb || !depth) return fail(STP_ERR_ARG, "null rgb or depth output");
    cudaStream_t s = (cudaStream_t)stream;
    stp::PipeArgs a = make_args(prm, P, workspace);
    a.rgb = rgb;
    a.depth = depth;
    a.tfinal_out = tfinal;
    cudaError_t e;
    prof_mark(0, s);
    k_status_init<<<1, 1, 0, s>>>(a.status, a.capacity);
    stp::note_launches(1);
    if ((e = stp::launch_tables_init(P.views.data(), nviews, const_cast<stp::ViewDesc*>(a.views), P.scenes.data(),
                                     nscenes, const_cast<stp::SceneDesc*>(a.scenes), s)) != cudaSuccess)
        return cuda_fail(e, "view and scene tables");
    if (a.partitioned) {
        if ((e = cudaMemsetAsync(a.tile_counts, 0, (size_t)a.total_tiles * 4, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(a.tile_cursor, 0, (size_t)a.total_tiles * 4, s)) != cudaSuccess)
            return cuda_fail(e, "clear tile counters");
    }
    prof_mark(1, s);
    if ((e = stp::launch_preprocess(a, s)) != cudaSuccess) return cuda_fail(e, "preprocess");
    prof_mark(2, s);
    if ((e = a.partitioned ? stp::launch_scan_tiles(a, s) : stp::launch_scan_counts(a, s)) != cudaSuccess)
        return cuda_fail(e, "scan");
    prof_mark(3, s);
    if ((e = stp::launch_duplicate(a, s)) != cudaSuccess) return cuda_fail(e, "duplicate");
    prof_mark(4, s);
    if (a.partitioned) {
        if ((e = stp::launch_tile_sort(a, s)) != cudaSuccess) return cuda_fail(e, "tile sort");
        prof_mark(5, s);
    } else {
        if ((e = stp::pipeline_sort(a, s)) != cudaSuccess) return cuda_fail(e, "sort");
        prof_mark(5, s);
        if ((e = stp::launch_ranges(a, s)) != cudaSuccess) return cuda_fail(e, "ranges");
    }
    if (a.dbg_trace && (e = cudaMemsetAsync(a.dbg_trace, 0xFF, (size_t)a.total_pixels * stp::kTraceLen * 4, s)) != cudaSuccess)
        return cuda_fail(e, "clear trace");
    prof_mark(6, s);
    if ((e = stp::launch_render(a, false, s)) != cudaSuccess) return cuda_fail(e, "render");
    prof_mark(7, s);
    if (a.slice_k) {
        // second depth-slice pass: sort the whole lists of the tiles with queued warps (the
        // kernels return at once when the queue is empty) and render those warps again
        stp::PipeArgs b = a;
        b.slice_pass = 1;
        if ((e = stp::launch_tile_sort(b, s)) != cudaSuccess) return cuda_fail(e, "second pass: tile sort");
        if ((e = stp::launch_render(b, false, s)) != cudaSuccess) return cuda_fail(e, "second pass: render");
    }
    prof_mark(8, s);
    prof_finish(0);
    return STP_OK;
}

stp_status backward_impl(const stp_gaussians* scenes, int32_t nscenes, const int32_t* vps, const stp_camera* cams,
                         int32_t nviews, const stp_params* prm, void* workspace, size_t ws_bytes,
                         const float* d_rgb, const float* d_depth, const stp_gaussians_grad* grads, void* stream)
{
    g_err.clear();
    if (prm && !(prm->flags & kFlagBackward))
        return fail(STP_ERR_ARG, "the forward pass must reserve backward scratch (flag 64)");
    if (prm && prm->mode != STP_MODE_HIER)
        return fail(STP_ERR_NOT_SUPPORTED, "the backward pass replays the hierarchical order only (STP_MODE_HIER)");
    Plan P;
    stp_status st = prepare(scenes, nscenes, vps, cams, nviews, prm, ws_bytes, workspace, P);
    if (st != STP_OK) return st;
    if (!d_rgb || !grads) return fail(STP_ERR_ARG, "null gradient input or output");
    for (int sc = 0; sc < nscenes; sc++) {
        const stp_gaussians_grad& gr = grads[sc];
        if (scenes[sc].n > 0 && (!gr.means || !gr.log_scales || !gr.quats || !gr.opacity_logits || !gr.sh))
            return fail(STP_ERR_ARG, "scene %d: null gradient array", sc);
        stp::SceneDesc& S = P.scenes[sc];
        S.g_means = gr.means; S.g_log_scales = gr.log_scales; S.g_quats = gr.quats;
        S.g_logits = gr.opacity_logits; S.g_sh = gr.sh;
    }
    cudaStream_t s = (cudaStream_t)stream;
    stp::PipeArgs a = make_args(prm, P, workspace);
    a.d_rgb = d_rgb;
    a.d_depth = d_depth;
    cudaError_t e;
    for (int k = 0; k <= 4; k++) prof_mark(k, s);
    if ((e = stp::launch_tables_init(P.views.data(), nviews, const_cast<stp::ViewDesc*>(a.views), P.scenes.data(),
                                     nscenes, const_cast<stp::SceneDesc*>(a.scenes), s)) != cudaSuccess)
        return cuda_fail(e, "view and scene tables");
    prof_mark(5, s);
    // the depth-factor region is written (and read) only when the loss has a depth term
    const size_t scratch = (size_t)P.m * stp::kGradStride * 4 * (a.d_depth ? 2 : 1);
    if ((e = cudaMemsetAsync(a.grad_geom, 0, scratch, s)) != cudaSuccess)
        return cuda_fail(e, "clear gradient scratch");
    // empty replay queue (the stored-order kernel fills it)
    if (a.blist && (e = cudaMemsetAsync(&a.status->replay_n, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess)
        return cuda_fail(e, "clear replay queue");
    prof_mark(6, s);
    if ((e = stp::launch_render(a, true, s)) != cudaSuccess) return cuda_fail(e, "backward render");
    prof_mark(7, s);
    if ((e = stp::launch_backward_preprocess(a, s)) != cudaSuccess) return cuda_fail(e, "backward preprocess");
    prof_mark(8, s);
    prof_finish(1);
    return STP_OK;
}

}  // namespace

namespace stp {
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace stp

extern "C" {

uint64_t stp_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* stp_last_error(void) { return g_err.c_str(); }

int32_t stp_version(void) { return 0x000300; }

stp_status stp_workspace_layout_batched(const int64_t* n, const int32_t* views_per_scene, int32_t nscenes,
                                        const stp_camera* cams, int32_t nviews, const stp_params* prm,
                                        stp_workspace_layout* out)
{
    stp_status st = check(n, views_per_scene, nscenes, cams, nviews, prm);
    if (st != STP_OK) return st;
    if (!out) return fail(STP_ERR_ARG, "null layout pointer");
    Plan P;
    make_plan(n, views_per_scene, nscenes, cams, nviews, prm, P);
    *out = P.L;
    return STP_OK;
}

size_t stp_workspace_size_batched(const int64_t* n, const int32_t* views_per_scene, int32_t nscenes,
                                  const stp_camera* cams, int32_t nviews, const stp_params* prm)
{
    stp_workspace_layout L;
    if (stp_workspace_layout_batched(n, views_per_scene, nscenes, cams, nviews, prm, &L) != STP_OK) return 0;
    return L.total;
}

stp_status stp_workspace_layout_get(int64_t n, const stp_camera* cams, int32_t nviews, const stp_params* prm,
                                    stp_workspace_layout* out)
{
    return stp_workspace_layout_batched(&n, &nviews, 1, cams, nviews, prm, out);
}

size_t stp_workspace_size(int64_t n, const stp_camera* cams, int32_t nviews, const stp_params* prm)
{
    return stp_workspace_size_batched(&n, &nviews, 1, cams, nviews, prm);
}

stp_status stp_render(const stp_gaussians* g, const stp_camera* cams, int32_t nviews, const stp_params* prm,
                      void* workspace, size_t ws_bytes, float* rgb, float* depth, float* tfinal, void* stream)
{
    return render_impl(g, 1, &nviews, cams, nviews, prm, workspace, ws_bytes, rgb, depth, tfinal, stream);
}

stp_status stp_render_batched(const stp_gaussians* scenes, int32_t nscenes, const int32_t* views_per_scene,
                              const stp_camera* cams, int32_t nviews, const stp_params* prm, void* workspace,
                              size_t ws_bytes, float* rgb, float* depth, float* tfinal, void* stream)
{
    return render_impl(scenes, nscenes, views_per_scene, cams, nviews, prm, workspace, ws_bytes, rgb, depth,
                       tfinal, stream);
}

stp_status stp_render_backward(const stp_gaussians* g, const stp_camera* cams, int32_t nviews,
                               const stp_params* prm, void* workspace, size_t ws_bytes, const float* d_rgb,
                               const float* d_depth, const stp_gaussians_grad* grad, void* stream)
{
    return backward_impl(g, 1, &nviews, cams, nviews, prm, workspace, ws_bytes, d_rgb, d_depth, grad, stream);
}

stp_status stp_render_backward_batched(const stp_gaussians* scenes, int32_t nscenes, const int32_t* views_per_scene,
                                       const stp_camera* cams, int32_t nviews, const stp_params* prm,
                                       void* workspace, size_t ws_bytes, const float* d_rgb, const float* d_depth,
                                       const stp_gaussians_grad* grads, void* stream)
{
    return backward_impl(scenes, nscenes, views_per_scene, cams, nviews, prm, workspace, ws_bytes, d_rgb, d_depth,
                         grads, stream);
}

stp_status stp_read_status(const void* workspace, stp_run_status* out, void* stream)
{
    if (!workspace || !out) return fail(STP_ERR_ARG, "null workspace or output");
    cudaStream_t s = (cudaStream_t)stream;
    stp::Status h;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "read status");
    std::memset(out, 0, sizeof *out);
    out->error_bits = h.error_bits;
    out->mismatched = h.mismatched;
    out->num_entries = h.num_entries;
    out->capacity = h.capacity;
    for (int k = 0; k < 5; k++) out->counters[k] = h.counters[k];
    out->invalid_gaussians = h.invalid;
    out->redo_warps = h.redo_n;
    if (h.error_bits & 1u)
        return fail(STP_ERR_CAPACITY, "%llu entries needed, capacity %llu", h.num_entries, h.capacity);
    if (h.error_bits & 4u) return fail(STP_ERR_TIMEOUT, "a bounded device wait gave up");
    if (h.error_bits & 8u)
        return fail(STP_ERR_INCONSISTENT, "the backward's blend sequence disagreed with the forward's");
    return STP_OK;
}

stp_status stp_profile_enable(int32_t max_calls)
{
    if (max_calls < 0 || max_calls > 100000) return fail(STP_ERR_ARG, "max_calls out of range");
    for (cudaEvent_t e : g_prof.ev) cudaEventDestroy(e);
    g_prof.ev.clear();
    g_prof.kind.assign(max_calls, 0);
    g_prof.max_calls = 0;
    g_prof.next = 0;
    for (int k = 0; k < max_calls * STP_NUM_STAGE_EVENTS; k++) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return cuda_fail(r, "create timing events");
        g_prof.ev.push_back(e);
    }
    g_prof.max_calls = max_calls;
    return STP_OK;
}

stp_status stp_profile_read(float* ms, int32_t max_calls, int32_t* ncalls)
{
    if (!ms || !ncalls) return fail(STP_ERR_ARG, "null output");
    const int n = std::min(g_prof.next, (int)max_calls);
    for (int c = 0; c < n; c++) {
        cudaEvent_t* ev = &g_prof.ev[(size_t)c * STP_NUM_STAGE_EVENTS];
        cudaError_t r = cudaEventSynchronize(ev[STP_NUM_STAGE_EVENTS - 1]);
        if (r != cudaSuccess) return cuda_fail(r, "synchronise timing events");
        for (int k = 0; k < STP_NUM_STAGES; k++) {
            float t = 0.f;
            r = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (r != cudaSuccess) return cuda_fail(r, "elapsed time");
            ms[c * STP_NUM_STAGES + k] = t;
        }
    }
    *ncalls = n;
    g_prof.next = 0;
    return STP_OK;
}

size_t stp_sort_temp_bytes(int64_t n) { return n < 0 ? 0 : stp::sort_temp_bytes(n); }

stp_status stp_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                          int64_t n, const uint64_t* n_dev, int32_t key_bits, void* temp, size_t temp_bytes,
                          void* stream)
{
    g_err.clear();
    if (n < 0 || n >= 0xFFFFFFFFLL) return fail(STP_ERR_ARG, "n out of range");
    if (key_bits < 1 || key_bits > 64) return fail(STP_ERR_ARG, "key_bits must be in 1..64");
    if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out))
        return fail(STP_ERR_ARG, "null array");
    if (n > 0 && (!temp || temp_bytes < stp::sort_temp_bytes(n)))
        return fail(STP_ERR_ARG, "temp of %zu bytes, %zu needed", temp_bytes, stp::sort_temp_bytes(n));
    cudaError_t e = stp::sort_pairs(keys_in, vals_in, keys_out, vals_out, n,
                                    (const unsigned long long*)n_dev, key_bits, temp, temp_bytes,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sort");
    return STP_OK;
}

stp_status stp_sort_pairs_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out,
                                  uint32_t* vals_out, int64_t n, const uint64_t* n_dev, int32_t key_bits,
                                  void* stream)
{
    g_err.clear();
    if (n < 0 || n > stp::sort_static_max_n())
        return fail(STP_ERR_ARG, "stp_sort_pairs_noalloc: n = %lld exceeds the fixed scratch of %lld pairs",
                    (long long)n, stp::sort_static_max_n());
    if (key_bits < 1 || key_bits > 64) return fail(STP_ERR_ARG, "key_bits must be in 1..64");
    if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return fail(STP_ERR_ARG, "null array");
    cudaError_t e = stp::sort_pairs_static(keys_in, vals_in, keys_out, vals_out, n,
                                           (const unsigned long long*)n_dev, key_bits, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sort (static scratch)");
    return STP_OK;
}

}  // extern "C"
