// stp_render.cu -- hierarchical sorted Render (forward) and the backward over its blend order.
//
// StopThePop (arXiv 2402.00525) Sec. 3.4 "Hierarchically sorted rendering", Fig. "pipeline",
// appendix B.4 "Render"; backward Sec. 3.5.
//
// A 16x16 tile is rendered by eight warps (two 4-warp blocks by default). Warp w of the tile
// owns the two horizontally adjacent 4x4 subtiles 2w and 2w+1 (an 8x4 pixel strip); half-warp
// h owns subtile 2w+h, its 4-lane groups own the subtile's four 2x2 quads, and every lane owns
// one pixel. Each warp walks the tile's sorted list on its own -- the subtiles are independent
// -- so no block-wide barrier is needed and a warp whose 32 pixels are all saturated retires
// early.
//
// Queues (per warp, shared memory; entries are (ordered depth key, Gaussian id)):
//   tail  : per subtile, double-buffered, TAIL = 32n + 32 entries (the paper's 4x4 queue)
//   mid   : per quad, MID = 4m + 4 entries (the paper's 2x2 queue)
//   head  : per pixel, HEAD entries in registers (the paper's per-ray queue / k-buffer)
// Push discipline (the same reading as the CPU oracle):
//   * the list is consumed in batches of 32 (one entry per lane); every lane culls its entry
//     against both subtile boxes with Algorithm 1 and computes t_opt on the ray through the
//     box's x_hat; each subtile's survivors are ranked stably (ties by list position) and
//     merged into its tail by binary search, existing entries first on ties;
//   * while a tail holds more than TAIL-32 entries its front 16 go to the mid level; at the end
//     the tails drain in chunks of at most 16;
//   * a chunk goes to the quads in sub-batches of 4: each quad culls the 4 against its box,
//     computes t_opt through its x_hat, ranks them (three shuffles in the 4-lane group) and
//     merges them into its mid queue; when the mid queue then holds more than MID-4 entries
//     its front 4 go to the quad's pixels; at the end the mid queues flush in groups of 4;
//   * a pixel drops alpha < eps_O, computes t_opt on its own ray and inserts into its head;
//     when the head holds more than HEAD entries the smallest is blended.
// Blending is front to back with the 3DGS early-out (the Gaussian that would take T below
// t_min is not blended and the ray stops).
//
// Depth slices (slice_k > 0): when the per-tile sort ordered only a prefix of a tile's list, a
// warp renders that prefix's complete 32-entry batches (the whole list's first batches); a warp
// still holding an unsaturated pixel when it needs the next batch writes nothing and queues
// itself, and after its tile's list is sorted whole k_render_queue renders it again.
//
// Backward (Sec. 3.5): the gradients of a blend need the suffix colour C - C_i and T_N / T_i,
// so the blends are visited front to back in the forward's order. A forward that a backward
// follows stores each pixel's first blend_cap blended ids (4 bytes a blend), and
// k_render_bwd_list walks them, recomputing alpha with the forward's rounding. A warp with a
// pixel past blend_cap is queued and replayed: k_render_queue runs the forward code with
// BWD = true, which recomputes the identical decisions and forms the same terms at each
// blend. With blend_cap 0, k_render<HEAD, true> replays every warp (the paper's way).
#include <algorithm>

#include <cuda_runtime.h>

#include "stp_common.cuh"
#include "stp_kernels.cuh"

namespace stp {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Block shape of the hierarchical Render: a tile's eight warps (two subtiles each) are
// independent, so a tile is split over 8 / kRenderWarps blocks. The kernel is latency bound at
// low occupancy, so each instantiation is given the resident-block count (register cap) that
// measured fastest on 16 Full-HD views of 3M Gaussians with 4-warp blocks: HEAD <= 4 forward
// 6 blocks (80 registers, 32.8 ms against 37.6 ms at 111 registers and 2 x 8-warp blocks),
// backward replay 5 (96 registers, 54.8 ms against 59.8 ms when it replayed every warp); wider
// heads hold more registers.
// Build-time knobs: -DSTP_RENDER_WARPS=..., -DSTP_RENDER_MIN_BLOCKS_FWD / _BWD=... (HEAD <= 4),
// -DSTP_RENDER_MIN_BLOCKS=... (all instantiations).
#ifndef STP_RENDER_WARPS
#define STP_RENDER_WARPS 4
#endif
constexpr int kRenderWarps = STP_RENDER_WARPS;
constexpr int kBlocksPerTile = 8 / kRenderWarps;
static_assert(kRenderWarps == 1 || kRenderWarps == 2 || kRenderWarps == 4 || kRenderWarps == 8, "warps per block");

#ifndef STP_RENDER_MIN_BLOCKS_FWD
#define STP_RENDER_MIN_BLOCKS_FWD 6
#endif
#ifndef STP_RENDER_MIN_BLOCKS_BWD
#define STP_RENDER_MIN_BLOCKS_BWD 5
#endif
template <int HEAD, bool BWD>
constexpr int render_min_blocks()
{
#ifdef STP_RENDER_MIN_BLOCKS
    return STP_RENDER_MIN_BLOCKS;
#else
    return (HEAD <= 4 ? (BWD ? STP_RENDER_MIN_BLOCKS_BWD : STP_RENDER_MIN_BLOCKS_FWD) : HEAD <= 8 ? 4 : 2) * 4 / kRenderWarps;
#endif
}

// Head-stage FIFO: a quad's mid-queue pops are appended to its FIFO (ids, in pop order) and
// its pixels consume them at the end of each iteration of the list loop (a batch of 32 list
// entries, or one drain step), all quads of the warp together. A pixel sees exactly the
// sequence it would see if it consumed every pop at once, so the results are the same; the
// warp's lanes are busy together instead of only the lanes of the quads that happened to pop.
// One iteration appends at most 32 + MID - 4 entries to a FIFO: a batch makes a tail pop at
// most twice (it adds <= 32 entries to a tail holding <= TAIL - 32), and the quad's mid queue
// holds <= MID - 4 entries between sub-batches.
constexpr int kFifo = 48;
static_assert(kFifo >= 32 + kMaxMid - 4, "head FIFO must hold one iteration's pops");

// The head queue compares depths as floats. A NaN or +inf depth (a degenerate splat) is held
// as FLT_MAX, so +inf marks an empty slot below which every real entry sorts.
constexpr float kEmptyT = __builtin_huge_valf();
__device__ __forceinline__ float head_depth(float t) { return fminf(t, 3.402823466e38f); }

__device__ __forceinline__ uint32_t depth_key(float t)
{
    const uint32_t k = fkey(t);
    return k == kInvalidKey ? kInvalidKey - 1u : k;
}

// cull threshold of the 4x4 / 2x2 levels: eps_O, or -1 (nothing culled, ablation E) since
// opacity * G2 >= 0
__device__ __forceinline__ float level_cull_eps(const PipeArgs& a)
{
    return (a.flags & kFlagNoHierCull) ? -1.f : a.eps_o;
}

// per-warp shared memory in uint2 units: tails (2 subtiles x 2 buffers), the batch staging,
// the eight mid queues and the eight head FIFOs (kFifo ids each)
__host__ __device__ constexpr int render_warp_smem(int tail, int mid) { return 4 * tail + 64 + 8 * mid + 4 * kFifo; }

// Debug state of a pixel (blend-order hash, sort error): held only by the DBG instantiations,
// so the timed path carries none of it in registers and takes no debug branch per blend.
template <bool DBG> struct PxDbg {};
template <> struct PxDbg<true> {
    unsigned long long hash;
    float last_t, delta;         // sort error: sum of the backward steps of the blended t_opt
    unsigned long long nq, npx;  // work counters (entry, 2x2) and (entry, pixel), added at the end
};

template <int HEAD, bool DBG>
struct Px : PxDbg<DBG> {
    float T, C0, C1, C2, Z;
    bool done;
    int nh;                      // entries in the head, at the front of hk / hid / hv
    float hk[HEAD];              // ascending depths t_opt at the pixel, kEmptyT beyond nh
    uint32_t hid[HEAD];
    float hv[HEAD];              // opacity * G2 at the pixel (before the alpha_max clamp)
    uint32_t nbl;
};

struct PixCtx {
    float xc, yc;                // pixel centre
    float u, w, n;               // camera-normalised coordinates of the centre, |(u, w, 1)|
    long long pix;               // packed pixel index, -1 outside the image
    float g0, g1, g2, gz, gbg;   // backward: dL/drgb, dL/ddepth, <dL/drgb, bg>
    float Cf0, Cf1, Cf2, Zf, Tf; // backward: final colour (no background), depth, T
    long long bl;                // stored blend order: slot 0 of this pixel (slot k at bl + 32 k)
    const float4* vrec;          // this view's first record (records of view-local ids follow)
    float* vgrad;                // this view's first gradient-scratch record (backward)
};

// Record `i` of a view from the view's first record: one 32 x 32 -> 64-bit multiply-add for
// the address instead of 64-bit index arithmetic at every load.
__device__ __forceinline__ Rec load_rec_v(const float4* __restrict__ base, uint32_t i)
{
    Rec r;
    const float4* p = base + (unsigned long long)i * kRecFloat4;
    r.r0 = __ldg(p);
    r.r1 = __ldg(p + 1);
    r.r2 = __ldg(p + 2);
    r.r3 = __ldg(p + 3);
    r.r4 = __ldg(p + 4);
    r.r5 = __ldg(p + 5);
    return r;
}

// Gradient terms of one blended Gaussian (Sec. 3.5), given the pixel's state just after the
// blend: T = T_i (transmittance in front of it), C / Z = colour and depth accumulated up to
// and including it. dL/dalpha_i uses the suffix C_final - C_i and T_N / (1 - alpha_i).
// Per-(view, Gaussian) scratch: [0..7] (sum dGG d.xy, dA00, dA01, dA11, sum dGG, dcolour.rg),
// [8] dcolour.b in grad_geom, and the depth factors (dm_k 9, dc_k 3) in grad_depth. The first
// nine are returned in (q0, q1, qc) for the caller to accumulate; the depth factors (only with
// a depth gradient) are accumulated here with vector reductions (red.global.add.v4.f32).
__device__ __forceinline__ void grad_terms(const PipeArgs& a, const PixCtx& c, long long ri, const float4 col,
                                           const float4 r0, float alpha, float val, float t, float T,
                                           float C0, float C1, float C2, float Z,
                                           float4& q0, float4& q1, float& qc)
{
    const float wgt = alpha * T;
    const float inv = __fdividef(1.f, 1.f - alpha);     // 1 - alpha >= 1 - alpha_max > 0
    float da = c.g0 * (col.x * T - (c.Cf0 - C0) * inv) + c.g1 * (col.y * T - (c.Cf1 - C1) * inv) +
               c.g2 * (col.z * T - (c.Cf2 - C2) * inv) - c.gbg * c.Tf * inv;
    da += c.gz * (t * T - (c.Zf - Z) * inv);
    Rec r;
    r.r0 = r0;
    q0 = make_float4(0.f, 0.f, 0.f, 0.f);
    q1 = make_float4(0.f, 0.f, c.g0 * wgt, c.g1 * wgt);
    qc = c.g2 * wgt;
    if (val < a.alpha_max) {
        // val = opacity * G at this pixel, so with dGG = da * val: dL/dopacity gets dGG /
        // opacity, dL/dA gets -dGG d d^T / 2 and dL/dmean2 gets A dGG d (d = x - mean2).
        // The factors A and 1 / opacity are the same for every pixel of this (view,
        // Gaussian), so the scratch sums dGG d and dGG, and the backward Preprocess
        // applies them once.
        const float dx = off_x(r, c.xc), dy = off_y(r, c.yc);
        const float dGG = da * val;
        q0 = make_float4(dGG * dx, dGG * dy, dGG * (-0.5f * dx * dx), dGG * (-dx * dy));
        q1.x = dGG * (-0.5f * dy * dy);
        q1.y = dGG;
    }
    if (c.gz != 0.f) {
        // t = |d| N / D with a_k = m_k . d, N = sum a_k c_k, D = sum a_k^2 (record layout);
        // the depth factors r3..r5 are loaded only here
        float* gd = a.grad_depth + ri * kGradStride;
        const float4* rp = a.geom + kRecFloat4 * ri;
        r.r3 = __ldg(rp + 3);
        r.r4 = __ldg(rp + 4);
        r.r5 = __ldg(rp + 5);
        const float u = c.u, w = c.w;
        const float m[3][3] = {{r.r3.x, r.r3.y, r.r3.z}, {r.r3.w, r.r4.x, r.r4.y}, {r.r4.z, r.r4.w, r.r5.x}};
        const float cc[3] = {r.r5.y, r.r5.z, r.r5.w};
        float ak[3], dak[3];
        for (int k = 0; k < 3; k++) ak[k] = m[k][0] * u + m[k][1] * w + m[k][2];
        const float num = ak[0] * cc[0] + ak[1] * cc[1] + ak[2] * cc[2];
        const float den = ak[0] * ak[0] + ak[1] * ak[1] + ak[2] * ak[2];
        const float n = sqrtf(u * u + w * w + 1.f);
        const float dt = c.gz * wgt;
        const float tq = num / den;
        for (int k = 0; k < 3; k++) dak[k] = dt * n * (cc[k] - 2.f * tq * ak[k]) / den;   // dt/da_k
        const float fc = dt * n / den;                                                   // dt/dc_k = fc a_k
        atomicAdd(reinterpret_cast<float4*>(gd), make_float4(dak[0] * u, dak[0] * w, dak[0], dak[1] * u));
        atomicAdd(reinterpret_cast<float4*>(gd + 4), make_float4(dak[1] * w, dak[1], dak[2] * u, dak[2] * w));
        atomicAdd(reinterpret_cast<float4*>(gd + 8), make_float4(dak[2], fc * ak[0], fc * ak[1], fc * ak[2]));
    }
}

// accumulate the nine terms of grad_terms into the (view, Gaussian) scratch
__device__ __forceinline__ void grad_red(const PipeArgs& a, long long ri, const float4 q0, const float4 q1, float qc)
{
    float* gg = a.grad_geom + ri * kGradStride;
    atomicAdd(reinterpret_cast<float4*>(gg), q0);
    atomicAdd(reinterpret_cast<float4*>(gg + 4), q1);
    atomicAdd(gg + 8, qc);
}

template <int HEAD, bool BWD, bool DBG>
__device__ __forceinline__ void blend(const PipeArgs& a, const ViewDesc& V, Px<HEAD, DBG>& s,
                                      const PixCtx& c, float t, uint32_t id, float val)
{
    const float alpha = fminf(a.alpha_max, val);
    const float Tn = __fmul_rn(s.T, __fsub_rn(1.f, alpha));
    if (!BWD && !DBG) {
        // The timed forward blends without branches: a saturated or saturating pixel adds a
        // zero weight (its record, a valid one, is loaded all the same) and stores nothing, so
        // the warp takes no divergent region per blend.
        const bool go = !s.done && !(Tn < a.t_min);
        s.done = !go;
        const float4 r2 = __ldg(c.vrec + (unsigned long long)id * kRecFloat4 + 2);   // (opacity, colour)
        const float wgt = go ? alpha * s.T : 0.f;
        s.C0 += r2.y * wgt;
        s.C1 += r2.z * wgt;
        s.C2 += r2.w * wgt;
        s.Z += t * wgt;
        if (go && a.blist && s.nbl < (uint32_t)a.blend_cap) __stcs(a.blist + c.bl + 32ll * s.nbl, id);
        s.T = go ? Tn : s.T;
        s.nbl += go ? 1u : 0u;
        return;
    }
    if (s.done) return;
    if (Tn < a.t_min) {
        s.done = true;
        return;
    }
    const long long ri = V.rec_off + id;
    const float4 r2 = __ldg(c.vrec + (unsigned long long)id * kRecFloat4 + 2);       // (opacity, colour)
    const float4 col = make_float4(r2.y, r2.z, r2.w, 0.f);
    const float wgt = alpha * s.T;
    s.C0 += col.x * wgt;
    s.C1 += col.y * wgt;
    s.C2 += col.z * wgt;
    s.Z += t * wgt;
    if (BWD) {
        float4 q0, q1;
        float qc;
        grad_terms(a, c, ri, col, __ldg(c.vrec + (unsigned long long)id * kRecFloat4), alpha, val, t, s.T, s.C0, s.C1, s.C2, s.Z, q0, q1, qc);
        float* gg = c.vgrad + (unsigned long long)id * kGradStride;
        atomicAdd(reinterpret_cast<float4*>(gg), q0);
        atomicAdd(reinterpret_cast<float4*>(gg + 4), q1);
        atomicAdd(gg + 8, qc);
    }
    // the stored blend order (backward without replay): the first blend_cap ids of the pixel,
    // stored and later loaded with the evict-first hint (each id is touched once either way)
    if (!BWD && a.blist && s.nbl < (uint32_t)a.blend_cap) __stcs(a.blist + c.bl + 32ll * s.nbl, id);
    if constexpr (DBG && !BWD) {
        if (a.dbg_trace && s.nbl < (uint32_t)kTraceLen) a.dbg_trace[c.pix * kTraceLen + s.nbl] = (int)id;
        if (a.dbg_hash) {              // debug statistics: order hash and sort error
            s.hash = s.hash * kHashMul + (unsigned long long)(id + 1u);
            if (s.nbl > 0 && s.last_t > t) s.delta += s.last_t - t;
            s.last_t = t;
        }
    }
    s.T = Tn;
    s.nbl++;
}

// head (per-pixel k-buffer, Sec. 3.3) primitives on register arrays with static indices.
// Insert into a head holding nh < HEAD entries, after equal keys (stable).
template <int HEAD, bool DBG>
__device__ __forceinline__ void head_insert(Px<HEAD, DBG>& s, float key, uint32_t id, float val)
{
    float nk[HEAD];
    uint32_t ni[HEAD];
    float nv[HEAD];
    bool prev_le = true;
#pragma unroll
    for (int j = 0; j < HEAD; j++) {
        // slot j keeps its entry if it is <= key; else it takes key (if slot j-1 kept its
        // entry) or slot j-1's entry (shifted back by one)
        const bool le = s.hk[j] <= key;
        const int p = j > 0 ? j - 1 : 0;
        nk[j] = le ? s.hk[j] : (prev_le ? key : s.hk[p]);
        ni[j] = le ? s.hid[j] : (prev_le ? id : s.hid[p]);
        nv[j] = le ? s.hv[j] : (prev_le ? val : s.hv[p]);
        prev_le = le;
    }
#pragma unroll
    for (int j = 0; j < HEAD; j++) {
        s.hk[j] = nk[j];
        s.hid[j] = ni[j];
        s.hv[j] = nv[j];
    }
    s.nh++;
}

// The head is full: insert (key, id, val) after equal keys and take the smallest of the HEAD + 1
// entries out, in one pass. If the new entry is smaller than every held one it leaves at once
// and the head is unchanged; otherwise the front leaves and the new entry is merged into the
// other HEAD - 1. (key, id, val) returns the entry taken out.
template <int HEAD, bool DBG>
__device__ __forceinline__ void head_exchange(Px<HEAD, DBG>& s, float& key, uint32_t& id, float& val)
{
    const bool pass = key < s.hk[0];
    bool le[HEAD];
#pragma unroll
    for (int j = 0; j < HEAD; j++) le[j] = s.hk[j] <= key;
    float nk[HEAD];
    uint32_t ni[HEAD];
    float nv[HEAD];
#pragma unroll
    for (int j = 0; j < HEAD; j++) {
        // slot j takes the next held entry if it is <= key, else the new entry if the entry
        // before it is <= key (slot 0: unless the new entry passes), else keeps its own
        const int n = j + 1 < HEAD ? j + 1 : j;
        const bool nxt = j + 1 < HEAD && le[n];
        const bool nw = j == 0 ? !pass : le[j];
        nk[j] = nxt ? s.hk[n] : (nw ? key : s.hk[j]);
        ni[j] = nxt ? s.hid[n] : (nw ? id : s.hid[j]);
        nv[j] = nxt ? s.hv[n] : (nw ? val : s.hv[j]);
    }
    const float ok = s.hk[0], ov = s.hv[0];
    const uint32_t oi = s.hid[0];
    key = pass ? key : ok;
    id = pass ? id : oi;
    val = pass ? val : ov;
#pragma unroll
    for (int j = 0; j < HEAD; j++) {
        s.hk[j] = nk[j];
        s.hid[j] = ni[j];
        s.hv[j] = nv[j];
    }
}

template <int HEAD, bool DBG>
__device__ __forceinline__ void head_pop(Px<HEAD, DBG>& s, float& key, uint32_t& id, float& val)
{
    key = s.hk[0];
    id = s.hid[0];
    val = s.hv[0];
#pragma unroll
    for (int j = 0; j + 1 < HEAD; j++) {
        s.hk[j] = s.hk[j + 1];
        s.hid[j] = s.hid[j + 1];
        s.hv[j] = s.hv[j + 1];
    }
    s.hk[HEAD - 1] = kEmptyT;
    s.nh--;
}

// Insert (key, id, val); when more than HEAD entries are held blend the smallest (Sec. 3.3
// k-buffer; evict_first = the alternative "blend before insert" reading, where the front of a
// full head is blended first and the new entry then inserted). The blend and the insertion
// each sit at one call site, so that their bodies (the blend is large in the backward replay)
// are inlined once.
template <int HEAD, bool BWD, bool DBG>
__device__ __forceinline__ void head_push(const PipeArgs& a, const ViewDesc& V, Px<HEAD, DBG>& s,
                                          const PixCtx& c, float key, uint32_t id, float val,
                                          bool evict_first)
{
    const bool full = s.nh == HEAD;
    if (full) {
        float k = key, v = val;
        uint32_t i = id;
        if (evict_first) {
            head_pop(s, k, i, v);
        } else if (key >= s.hk[HEAD - 1]) {
            // the common case (entries reach a pixel nearly in depth order): the new entry is
            // behind every held one, so the exchange reduces to a shift -- the front leaves, the
            // rest move up, the new entry goes last (after equal keys, as the network would put it)
            k = s.hk[0];
            i = s.hid[0];
            v = s.hv[0];
#pragma unroll
            for (int j = 0; j + 1 < HEAD; j++) {
                s.hk[j] = s.hk[j + 1];
                s.hid[j] = s.hid[j + 1];
                s.hv[j] = s.hv[j + 1];
            }
            s.hk[HEAD - 1] = key;
            s.hid[HEAD - 1] = id;
            s.hv[HEAD - 1] = val;
        } else {
            head_exchange(s, k, i, v);
        }
        blend<HEAD, BWD, DBG>(a, V, s, c, k, i, v);
    }
    if (!full || (evict_first && !s.done)) head_insert(s, key, id, val);
}

// blend what the head still holds, nearest first
template <int HEAD, bool BWD, bool DBG>
__device__ __forceinline__ void head_flush(const PipeArgs& a, const ViewDesc& V, Px<HEAD, DBG>& s, const PixCtx& c)
{
#pragma unroll 1
    while (s.nh > 0 && !s.done) {
        float k, v;
        uint32_t i;
        head_pop(s, k, i, v);
        blend<HEAD, BWD, DBG>(a, V, s, c, k, i, v);
    }
}

template <int HEAD, bool DBG>
__device__ __forceinline__ void px_init(Px<HEAD, DBG>& s, bool inside)
{
    s.T = 1.f;
    s.C0 = s.C1 = s.C2 = s.Z = 0.f;
    s.done = !inside;
    s.nh = 0;
    s.nbl = 0;
    if constexpr (DBG) {
        s.hash = kHashInit;
        s.last_t = 0.f;
        s.delta = 0.f;
        s.nq = s.npx = 0;
    }
#pragma unroll
    for (int j = 0; j < HEAD; j++) {
        s.hk[j] = kEmptyT;
        s.hid[j] = 0;
        s.hv[j] = 0.f;
    }
}

struct Warp {                    // warp-uniform tail state and per-quad mid state
    int nt[2], ts[2], tb[2];
    int nm, ms;                  // this lane's quad: mid-queue length and front
    int fc;                      // this lane's quad: entries waiting in its head FIFO
};

// The pixels consume their quads' FIFOs (every lane of the warp calls this). Not unrolled:
// one inlined copy of the head step (and of its blend).
template <int HEAD, bool BWD, bool DBG>
__device__ __forceinline__ void head_consume(const PipeArgs& a, const ViewDesc& V, Px<HEAD, DBG>& s,
                                             const PixCtx& c, Warp& wq, const uint32_t* fq)
{
    const bool evict_first = (a.flags & 1) != 0;
    const int n = wq.fc;
#pragma unroll 1
    for (int k = 0; k < n && !s.done; k++) {
        const uint32_t gid = fq[k];
        const Rec r = load_rec_v(c.vrec, gid);
        const float val = splat_value(r, c.xc, c.yc);
        if constexpr (DBG && !BWD) s.npx++;
        // the depth on the pixel's ray for every entry, dropped or not: no divergent region
        // around it (the entries dropped by the opacity test are about a tenth)
        const float t = depth_uvn(r, c.u, c.w, c.n);
        if (fminf(a.alpha_max, val) >= a.eps_o) head_push<HEAD, BWD, DBG>(a, V, s, c, head_depth(t), gid, val, evict_first);
    }
    wq.fc = 0;
    __syncwarp();                                 // the FIFOs are refilled after this
}

// Append the front `cnt` entries of this lane's quad's mid queue to the quad's FIFO (the four
// lanes of the quad copy them). Every lane of the warp calls it.
__device__ __forceinline__ void mid_pop(Warp& wq, const uint2* mq, uint32_t* fq, int cnt, int pq)
{
    for (int k = pq; k < cnt; k += 4) fq[wq.fc + k] = mq[wq.ms + k].y;
    wq.ms += cnt;
    wq.nm -= cnt;
    wq.fc += cnt;
    __syncwarp();
}

template <int HEAD, bool BWD, bool DBG>
__device__ void midstage(const PipeArgs& a, const ViewDesc& V, Px<HEAD, DBG>& s, const PixCtx& c,
                         Warp& wq, const uint2* tailb, uint2* mq, uint32_t* fq, const Box& bQ, bool qval,
                         int c0, int c1, int lane)
{
    const int h = lane >> 4, pq = lane & 3, qbase = lane & ~3;
    const int cnt = h ? c1 : c0;
    const uint2* chunk = tailb + (h * 2 + wq.tb[h]) * a.tail + wq.ts[h];
    const int cmax = max(c0, c1);
    const int MID = a.mid;
    const bool centre = (a.flags & 2) != 0;
    const float cull_eps = level_cull_eps(a);
    // a quad whose four pixels are saturated takes no further part (its results are final)
    const unsigned live = __ballot_sync(kFull, !s.done);
    const bool qlive = qval && ((live >> qbase) & 0xFu) != 0;
    for (int j0 = 0; j0 < cmax; j0 += 4) {
        const int e = j0 + pq;
        uint32_t key = kInvalidKey, gid = 0;
        if (e < cnt) {
            gid = chunk[e].y;
            if (qlive) {
                const Rec r = load_rec_v(c.vrec, gid);
                const Box bq = bQ;
                float t;
                if (box_keep_depth(r, bq, V, cull_eps, centre, &t)) key = depth_key(t);
            }
        }
        // stable rank of the new entry among the quad's (up to) four
        uint32_t rk = 0;
#pragma unroll
        for (int k = 1; k < 4; k++) {
            const int op = (pq + k) & 3;
            const uint32_t o = __shfl_sync(kFull, key, qbase | op);
            rk += (o < key) || (o == key && op < pq);
        }
        const unsigned bal = __ballot_sync(kFull, key != kInvalidKey);
        const int nn = __popc((bal >> qbase) & 0xFu);
        if constexpr (DBG && !BWD) s.nq += (unsigned long long)__popc(__ballot_sync(kFull, e < cnt && qval));
        uint32_t nk[4];
#pragma unroll
        for (int k = 0; k < 4; k++) nk[k] = __shfl_sync(kFull, key, qbase | k);
        // merge: existing entries first on equal keys
        uint2 ex[4];
        int exp[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int i = pq + 4 * r;
            exp[r] = -1;
            if (i < wq.nm) {
                ex[r] = mq[wq.ms + i];
                int cl = 0;
#pragma unroll
                for (int k = 0; k < 4; k++) cl += nk[k] < ex[r].x;
                exp[r] = i + cl;
            }
        }
        int npos = -1;
        if (key != kInvalidKey) {
            int cle = 0;
            for (int i = 0; i < wq.nm; i++) cle += mq[wq.ms + i].x <= key;
            npos = (int)rk + cle;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; r++)
            if (exp[r] >= 0) mq[exp[r]] = ex[r];
        if (npos >= 0) mq[npos] = make_uint2(key, gid);
        __syncwarp();
        wq.nm += nn;
        wq.ms = 0;
        const bool pop = wq.nm > MID - 4;
        if (__any_sync(kFull, pop)) mid_pop(wq, mq, fq, pop ? 4 : 0, pq);
    }
}

__device__ __forceinline__ void merge_tail(const uint2* src, int ne, const uint2* nw, int nn, uint2* dst, int lane)
{
    // warp-uniform common case: the batch's survivors all lie behind the tail (existing entries
    // first on equal keys), so the merge is a copy and an append
    if (nn == 0 || ne == 0 || nw[0].x >= src[ne - 1].x) {
        for (int e = lane; e < ne; e += 32) dst[e] = src[e];
        if (lane < nn) dst[ne + lane] = nw[lane];
        return;
    }
    for (int e = lane; e < ne; e += 32) {
        const uint2 x = src[e];
        int lo = 0, hi = nn;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (nw[m].x < x.x) lo = m + 1; else hi = m;
        }
        dst[e + lo] = x;
    }
    if (lane < nn) {
        const uint2 x = nw[lane];
        int lo = 0, hi = ne;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (src[m].x <= x.x) lo = m + 1; else hi = m;
        }
        dst[lane + lo] = x;
    }
}

// One warp's share of a tile (two 4x4 subtiles) through the whole hierarchical Render: the
// forward, or its replay for the backward. tailb is the warp's shared-memory queue area.
template <int HEAD, bool BWD, bool DBG>
__device__ __forceinline__ void render_warp(const PipeArgs& a, const int gtile, const int warp, const int lane,
                                            uint2* tailb)
{
    const int TAIL = a.tail, MID = a.mid;
    uint2* stage = tailb + 4 * TAIL;
    uint2* midb = stage + 64;
    uint32_t* fifob = reinterpret_cast<uint32_t*>(midb + 8 * MID);
    int lo = 0, hi = a.nviews - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (a.views[m].tile_off <= gtile) lo = m; else hi = m - 1;
    }
    // a local copy: read through a reference, its fields would be reloaded after every store
    const ViewDesc V = a.views[lo];
    const int W = V.W, H = V.H;
    const int tile = gtile - V.tile_off;
    const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
    const int h = lane >> 4, q = (lane & 15) >> 2, pq = lane & 3;

    Box bS[2];
    bool sval[2];
#pragma unroll
    for (int hh = 0; hh < 2; hh++) {
        const int sidx = warp * 2 + hh;
        const int ox = tx * kTile + (sidx & 3) * 4, oy = ty * kTile + (sidx >> 2) * 4;
        sval[hh] = ox < W && oy < H;
        bS[hh] = block_box(ox, oy, 4, W, H);
    }
    const int sme = warp * 2 + h;
    const int qox = tx * kTile + (sme & 3) * 4 + (q & 1) * 2, qoy = ty * kTile + (sme >> 2) * 4 + (q >> 1) * 2;
    const bool qval = qox < W && qoy < H;
    const Box bQ = block_box(qox, qoy, 2, W, H);
    const int pxi = qox + (pq & 1), pyi = qoy + (pq >> 1);
    const bool inside = pxi < W && pyi < H;

    PixCtx c;
    c.xc = pxi + 0.5f;
    c.yc = pyi + 0.5f;
    c.u = to_u(V, c.xc);
    c.w = to_w(V, c.yc);
    c.n = ray_norm(c.u, c.w);
    c.pix = inside ? V.pix_off + (long long)pyi * W + pxi : -1;
    c.bl = ((long long)(gtile * 8 + warp) * a.blend_cap) * 32 + lane;
    c.vrec = a.geom + kRecFloat4 * V.rec_off;
    c.vgrad = a.grad_geom ? a.grad_geom + V.rec_off * kGradStride : nullptr;
    c.g0 = c.g1 = c.g2 = c.gz = c.gbg = 0.f;
    c.Cf0 = c.Cf1 = c.Cf2 = c.Zf = c.Tf = 0.f;
    if (BWD && inside) {
        c.g0 = a.d_rgb[3 * c.pix];
        c.g1 = a.d_rgb[3 * c.pix + 1];
        c.g2 = a.d_rgb[3 * c.pix + 2];
        c.gz = a.d_depth ? a.d_depth[c.pix] : 0.f;
        c.gbg = c.g0 * a.bg[0] + c.g1 * a.bg[1] + c.g2 * a.bg[2];
        const float4 cz = reinterpret_cast<const float4*>(a.pix_state)[c.pix];
        c.Cf0 = cz.x; c.Cf1 = cz.y; c.Cf2 = cz.z; c.Zf = cz.w;
        c.Tf = a.tfinal_ws[c.pix];
    }

    Px<HEAD, DBG> s;
    px_init(s, inside);
    Warp wq;
    wq.nt[0] = wq.nt[1] = wq.ts[0] = wq.ts[1] = wq.tb[0] = wq.tb[1] = 0;
    wq.nm = wq.ms = wq.fc = 0;
    uint2* mq = midb + (h * 4 + q) * MID;
    uint32_t* fq = fifob + (h * 4 + q) * kFifo;

    const uint2 rg = a.ranges[gtile];
    const int lst = (int)rg.x;
    int nL = (int)(rg.y - rg.x);
    // Depth slices: a list that is only a prefix of the tile's sorted entries renders as far as
    // its complete 32-entry batches, which are the whole list's first batches; a warp with a pixel
    // still unsaturated when it needs the next batch is queued for the second pass, which
    // renders it again over the completed list.
    const bool trunc = a.slice_k && a.tile_front[gtile] < a.tile_counts[gtile];
    if (trunc) nL &= ~31;
    bool redo = false;
    const bool centre = (a.flags & 2) != 0;
    const float cull_eps = level_cull_eps(a);
    const bool count = DBG && !BWD && a.dbg_nblend != nullptr;
    unsigned long long n_eval_s = 0, n_surv_s = 0;
    // One loop for the batches and the drain, so that the mid stage (and the head stage and
    // blend inside it) is inlined once. While batches remain, a batch is loaded and merged and
    // the tails pop 16 while they hold more than TAIL-32; afterwards each iteration pops one
    // chunk of at most 16 per subtile until the tails are empty.
    int b0 = 0;
    for (;;) {
        const bool batch = b0 < nL;
        if (__all_sync(kFull, s.done)) break;
        if (trunc && !batch) {
            redo = true;
            break;
        }
        bool last = false;
        if (batch) {
            const int idx = b0 + lane;
            const bool in = idx < nL;
            const uint32_t gid = in ? __ldg(a.svals + lst + idx) : 0u;
            uint32_t k0 = kInvalidKey, k1 = kInvalidKey;
            // a subtile whose sixteen pixels are saturated takes no further part
            const unsigned live = __ballot_sync(kFull, !s.done);
            const bool s0 = sval[0] && (live & 0xFFFFu) != 0, s1 = sval[1] && (live >> 16) != 0;
            if (in && (s0 || s1)) {
                const Rec r = load_rec_v(c.vrec, gid);
                float t;
                if (s0 && box_keep_depth(r, bS[0], V, cull_eps, centre, &t)) k0 = depth_key(t);
                if (s1 && box_keep_depth(r, bS[1], V, cull_eps, centre, &t)) k1 = depth_key(t);
            }
            // stable rank: lanes with a smaller key, plus lanes before this one with an equal key
            uint32_t r0 = __popc(__match_any_sync(kFull, k0) & lanemask_lt());
            uint32_t r1 = __popc(__match_any_sync(kFull, k1) & lanemask_lt());
#pragma unroll 8
            for (int j = 0; j < 32; j++) {
                const uint32_t o0 = __shfl_sync(kFull, k0, j), o1 = __shfl_sync(kFull, k1, j);
                r0 += o0 < k0;
                r1 += o1 < k1;
            }
            const int nn0 = __popc(__ballot_sync(kFull, k0 != kInvalidKey));
            const int nn1 = __popc(__ballot_sync(kFull, k1 != kInvalidKey));
            if (count && lane == 0) {
                const int nin = min(32, nL - b0);
                n_eval_s += (unsigned long long)nin * ((sval[0] ? 1 : 0) + (sval[1] ? 1 : 0));
                n_surv_s += (unsigned long long)(nn0 + nn1);
            }
            if (k0 != kInvalidKey) stage[r0] = make_uint2(k0, gid);
            if (k1 != kInvalidKey) stage[32 + r1] = make_uint2(k1, gid);
            __syncwarp();
            merge_tail(tailb + (0 * 2 + wq.tb[0]) * TAIL + wq.ts[0], wq.nt[0], stage, nn0,
                       tailb + (0 * 2 + (wq.tb[0] ^ 1)) * TAIL, lane);
            merge_tail(tailb + (1 * 2 + wq.tb[1]) * TAIL + wq.ts[1], wq.nt[1], stage + 32, nn1,
                       tailb + (1 * 2 + (wq.tb[1] ^ 1)) * TAIL, lane);
            __syncwarp();
            wq.nt[0] += nn0;
            wq.nt[1] += nn1;
            wq.ts[0] = wq.ts[1] = 0;
            wq.tb[0] ^= 1;
            wq.tb[1] ^= 1;
            b0 += 32;
        } else if (wq.nt[0] == 0 && wq.nt[1] == 0) {
            // tails drained: the mid queues flush into the FIFOs behind their pops, and the
            // pixels take everything in this last iteration
            mid_pop(wq, mq, fq, wq.nm, pq);
            last = true;
        } else {
            const unsigned live = __ballot_sync(kFull, !s.done);
            if ((live & 0xFFFFu) == 0) wq.nt[0] = 0;
            if ((live >> 16) == 0) wq.nt[1] = 0;
        }
        for (; !last;) {
            int c0, c1;
            if (batch) {
                c0 = wq.nt[0] > TAIL - 32 ? 16 : 0;
                c1 = wq.nt[1] > TAIL - 32 ? 16 : 0;
                if (c0 == 0 && c1 == 0) break;
            } else {
                c0 = min(16, wq.nt[0]);
                c1 = min(16, wq.nt[1]);
            }
            midstage<HEAD, BWD, DBG>(a, V, s, c, wq, tailb, mq, fq, bQ, qval, c0, c1, lane);
            wq.ts[0] += c0; wq.nt[0] -= c0;
            wq.ts[1] += c1; wq.nt[1] -= c1;
            if (!batch) break;
        }
        // the pixels take this iteration's pops now (so the saturation test above is current)
        if (__any_sync(kFull, wq.fc > 0)) head_consume<HEAD, BWD, DBG>(a, V, s, c, wq, fq);
        if (last) break;
    }
    if (redo) {
        // the outputs, blend order and counters of this warp come from the second pass (in the
        // backward this cannot happen: the forward ended this warp within the prefix)
        if (lane == 0) {
            if (BWD) {
                atomicOr(&a.status->error_bits, 8u);
            } else if (a.slice_pass) {        // the completed list is still short: cannot happen
                atomicOr(&a.status->error_bits, 2u);
            } else {
                const unsigned slot = atomicAdd(&a.status->redo_n, 1u);
                if (slot < (unsigned)a.total_tiles * 8u) a.redo_warps[slot] = (uint32_t)(gtile * 8 + warp);
                a.tile_redo[gtile] = 1u;
            }
        }
        return;
    }
    head_flush<HEAD, BWD, DBG>(a, V, s, c);
    if constexpr (DBG && !BWD) {
        if (count) {
            if (lane == 0) {
                atomicAdd(&a.status->counters[0], n_eval_s);
                atomicAdd(&a.status->counters[1], n_surv_s);
                atomicAdd(&a.status->counters[2], s.nq);
            }
            atomicAdd(&a.status->counters[3], (unsigned long long)s.nbl);
            atomicAdd(&a.status->counters[4], s.npx);
        }
    }
    if (!inside) return;
    const long long p = c.pix;
    if (!BWD) {
        a.rgb[3 * p] = s.C0 + s.T * a.bg[0];
        a.rgb[3 * p + 1] = s.C1 + s.T * a.bg[1];
        a.rgb[3 * p + 2] = s.C2 + s.T * a.bg[2];
        a.depth[p] = s.Z;
        a.tfinal_ws[p] = s.T;
        if (a.grad_geom) reinterpret_cast<float4*>(a.pix_state)[p] = make_float4(s.C0, s.C1, s.C2, s.Z);
        if (a.blist) a.blist_count[p] = s.nbl;
        if (a.tfinal_out) a.tfinal_out[p] = s.T;
        if constexpr (DBG) {
            if (a.dbg_nblend) a.dbg_nblend[p] = s.nbl;
            if (a.dbg_hash) a.dbg_hash[p] = s.hash;
            if (a.dbg_delta) a.dbg_delta[p] = s.delta;
        }
    } else if constexpr (DBG) {
        if (a.dbg_nblend && a.dbg_nblend[p] != s.nbl) atomicOr(&a.status->error_bits, 8u);
    }
}

template <int HEAD, bool BWD, bool DBG>
__global__ void __launch_bounds__(32 * kRenderWarps, (render_min_blocks<HEAD, BWD>())) k_render(PipeArgs a)
{
    extern __shared__ uint2 sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (a.status->error_bits & 1u) return;
    render_warp<HEAD, BWD, DBG>(a, (int)(blockIdx.x / kBlocksPerTile), (int)(blockIdx.x % kBlocksPerTile) * kRenderWarps + wib,
                           lane, sm + wib * render_warp_smem(a.tail, a.mid));
}

// Work-list kernels: a grid of resident blocks whose warps take queued tile warps one at a
// time, so that a few queued warps cost no launch of a block per tile. BWD: the backward replay
// of the warps the stored-order kernel queued (a pixel past blend_cap). Forward: the second
// depth-slice pass over the warps the first could not finish within their tiles' prefixes
// (their lists are whole now).
template <int HEAD, bool BWD, bool DBG>
__global__ void __launch_bounds__(32 * kRenderWarps, (render_min_blocks<HEAD, BWD>())) k_render_queue(PipeArgs a)
{
    extern __shared__ uint2 sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (a.status->error_bits & 1u) return;
    const unsigned n = BWD ? a.status->replay_n : a.status->redo_n;
    unsigned* next = BWD ? &a.status->replay_next : &a.status->redo_next;
    const uint32_t* list = BWD ? a.replay_warps : a.redo_warps;
    uint2* tailb = sm + wib * render_warp_smem(a.tail, a.mid);
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(next, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n) break;
        const uint32_t w = list[item];
        render_warp<HEAD, BWD, DBG>(a, (int)(w >> 3), (int)(w & 7), lane, tailb);
        __syncwarp();
    }
}

// Backward over the stored blend order (Sec. 3.5). The forward Render recorded, per pixel, the
// ids it blended in blend order, so the gradients need no replay of the queues: each thread
// walks its pixel's ids front to back, recomputes alpha (and, for a depth gradient, t_opt) from
// the record with the forward's own rounding, and forms the same terms as the replay. Warps with
// a pixel past the capacity are queued for the replay (k_render_queue with BWD = true).
// Same block shape and pixel mapping as the forward. The product of the recomputed (1 - alpha)
// must reproduce the forward's final T bit for bit; a pixel where it does not sets error bit 8.
//
// Neighbouring pixels often blend the same Gaussian at the same step (on 16 Full-HD views of 3M
// Gaussians a step of a warp holds about 11 distinct ids over 27 live lanes), so the lanes of a
// step that share an id sum their nine terms in shared memory and one of them issues the
// reductions: 40% of the per-lane reductions, which dominate this kernel's L2 traffic. The
// staging is vectorised (three 16-byte stores per lane, three loads per peer): with nine scalar
// accesses each the shared-memory pipe, not L2, was the limit (ncu: L1 at 97% of peak).
#ifndef STP_BWD_LIST_MIN_BLOCKS
#define STP_BWD_LIST_MIN_BLOCKS 8
#endif
__global__ void __launch_bounds__(32 * kRenderWarps, STP_BWD_LIST_MIN_BLOCKS * 4 / kRenderWarps) k_render_bwd_list(PipeArgs a)
{
    // per lane (q0, q1, qc) as three float4: 16-byte stores at a 48-byte lane stride are
    // conflict-free, and a group leader reads a peer's terms with three loads
    __shared__ __align__(16) float sagg[kRenderWarps][32 * 12];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (int)(blockIdx.x % kBlocksPerTile) * kRenderWarps + wib;   // warp of the tile
    if (a.status->error_bits & 1u) return;
    const int gtile = (int)(blockIdx.x / kBlocksPerTile);
    int lo = 0, hi = a.nviews - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (a.views[m].tile_off <= gtile) lo = m; else hi = m - 1;
    }
    const ViewDesc V = a.views[lo];
    const int tile = gtile - V.tile_off;
    const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
    const int h = lane >> 4, q = (lane & 15) >> 2, pq = lane & 3;
    const int sme = warp * 2 + h;
    const int pxi = tx * kTile + (sme & 3) * 4 + (q & 1) * 2 + (pq & 1);
    const int pyi = ty * kTile + (sme >> 2) * 4 + (q >> 1) * 2 + (pq >> 1);
    const bool inside = pxi < V.W && pyi < V.H;
    PixCtx c;
    c.xc = pxi + 0.5f;
    c.yc = pyi + 0.5f;
    c.u = to_u(V, c.xc);
    c.w = to_w(V, c.yc);
    c.n = ray_norm(c.u, c.w);
    c.pix = inside ? V.pix_off + (long long)pyi * V.W + pxi : -1;
    c.bl = ((long long)(gtile * 8 + warp) * a.blend_cap) * 32 + lane;
    c.vrec = a.geom + kRecFloat4 * V.rec_off;
    c.vgrad = a.grad_geom ? a.grad_geom + V.rec_off * kGradStride : nullptr;
    const uint32_t nb = inside ? a.blist_count[c.pix] : 0u;
    if (__any_sync(kFull, nb > (uint32_t)a.blend_cap)) {           // queued for the replay
        if (lane == 0) a.replay_warps[atomicAdd(&a.status->replay_n, 1u)] = (uint32_t)(gtile * 8 + warp);
        return;
    }
    c.g0 = c.g1 = c.g2 = c.gz = c.gbg = 0.f;
    c.Cf0 = c.Cf1 = c.Cf2 = c.Zf = c.Tf = 0.f;
    if (inside) {
        c.g0 = a.d_rgb[3 * c.pix];
        c.g1 = a.d_rgb[3 * c.pix + 1];
        c.g2 = a.d_rgb[3 * c.pix + 2];
        c.gz = a.d_depth ? a.d_depth[c.pix] : 0.f;
        c.gbg = c.g0 * a.bg[0] + c.g1 * a.bg[1] + c.g2 * a.bg[2];
        const float4 cz = reinterpret_cast<const float4*>(a.pix_state)[c.pix];
        c.Cf0 = cz.x; c.Cf1 = cz.y; c.Cf2 = cz.z; c.Zf = cz.w;
        c.Tf = a.tfinal_ws[c.pix];
    }
    const bool with_depth = a.d_depth != nullptr;
    const uint32_t* ids = a.blist + c.bl;
    float* const vgrad = a.grad_geom + V.rec_off * kGradStride;   // this view's first scratch record
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Z = 0.f;
    const uint32_t nmax = __reduce_max_sync(kFull, nb);
    uint32_t nxt = nb > 0 ? __ldcs(ids) : 0u;
    // every lane runs the warp's longest list so that the steps stay aligned for the sharing
#pragma unroll 1
    for (uint32_t k = 0; k < nmax; k++) {
        const bool valid = k < nb;
        const uint32_t id = valid ? nxt : 0xFFFFFFFFu;
        if (k + 1 < nb) nxt = __ldcs(ids + 32ll * (k + 1));
        const long long ri = V.rec_off + (valid ? id : 0u);
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
        float qc = 0.f;
        if (valid) {
            const float4* rp = c.vrec + (unsigned long long)id * kRecFloat4;
            Rec r;
            r.r0 = __ldg(rp);
            r.r1 = __ldg(rp + 1);
            r.r2 = __ldg(rp + 2);
            const float val = splat_value(r, c.xc, c.yc);
            float t = 0.f;
            if (with_depth) {
                r.r3 = __ldg(rp + 3);
                r.r4 = __ldg(rp + 4);
                r.r5 = __ldg(rp + 5);
                t = depth_uvn(r, c.u, c.w, c.n);
            }
            const float alpha = fminf(a.alpha_max, val);
            const float4 col = make_float4(r.r2.y, r.r2.z, r.r2.w, 0.f);   // r2 holds the colour
            const float wgt = alpha * T;
            C0 += col.x * wgt;
            C1 += col.y * wgt;
            C2 += col.z * wgt;
            Z += t * wgt;
            grad_terms(a, c, ri, col, r.r0, alpha, val, t, T, C0, C1, C2, Z, q0, q1, qc);
            T = __fmul_rn(T, __fsub_rn(1.f, alpha));
        }
        // lanes holding the same id; a lane past its list takes an id of its own (no Gaussian id
        // has the top bit set), so it stages nothing and issues nothing
        const unsigned peers = __match_any_sync(kFull, valid ? id : (0x80000000u | lane));
        const bool solo = peers == (1u << lane);
        const int leader = __ffs(peers) - 1;
        float* sa = &sagg[wib][0];
        if (!solo) {
            float4* me = reinterpret_cast<float4*>(sa + lane * 12);
            me[0] = q0;
            me[1] = q1;
            me[2] = make_float4(qc, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        if (!solo && lane == leader) {
            unsigned rest = peers & (peers - 1u);     // the other lanes of the group
            while (rest) {
                const int p = __ffs(rest) - 1;
                rest &= rest - 1u;
                const float4* o = reinterpret_cast<const float4*>(sa + p * 12);
                const float4 a0 = o[0], a1 = o[1];
                q0.x += a0.x; q0.y += a0.y; q0.z += a0.z; q0.w += a0.w;
                q1.x += a1.x; q1.y += a1.y; q1.z += a1.z; q1.w += a1.w;
                qc += o[2].x;
            }
        }
        __syncwarp();                                 // the next step rewrites the staging
        if (valid && lane == leader) {
            float* gg = vgrad + (unsigned long long)id * kGradStride;
            atomicAdd(reinterpret_cast<float4*>(gg), q0);
            atomicAdd(reinterpret_cast<float4*>(gg + 4), q1);
            atomicAdd(gg + 8, qc);
        }
    }
    if (inside && __float_as_uint(T) != __float_as_uint(c.Tf)) atomicOr(&a.status->error_bits, 8u);
}

template <int HEAD, bool DBG>
cudaError_t launch_head(const PipeArgs& a, bool bwd, size_t smem, cudaStream_t s)
{
    static int set_fwd[64], set_bwd[64];
    cudaError_t e;
    if (bwd) {
        if ((e = ensure_smem_limit(k_render<HEAD, true, DBG>, smem, set_bwd, 64)) != cudaSuccess) return e;
        if (a.blist) {
            static int set_rep[64];
            if ((e = ensure_smem_limit(k_render_queue<HEAD, true, DBG>, smem, set_rep, 64)) != cudaSuccess) return e;
            int dev = 0, nsm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            const long long resident = (long long)nsm * render_min_blocks<HEAD, true>();
            const unsigned grid = (unsigned)std::min<long long>(resident, (long long)a.total_tiles * kBlocksPerTile);
            k_render_bwd_list<<<a.total_tiles * kBlocksPerTile, 32 * kRenderWarps, 0, s>>>(a);
            k_render_queue<HEAD, true, DBG><<<grid, 32 * kRenderWarps, smem, s>>>(a);
            note_launches(2);
        } else {
            k_render<HEAD, true, DBG><<<a.total_tiles * kBlocksPerTile, 32 * kRenderWarps, smem, s>>>(a);
            note_launches(1);
        }
    } else {
        if (a.slice_pass) {      // the second depth-slice pass: resident blocks over the queue
            static int set_redo[64];
            if ((e = ensure_smem_limit(k_render_queue<HEAD, false, DBG>, smem, set_redo, 64)) != cudaSuccess) return e;
            int dev = 0, nsm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            const long long resident = (long long)nsm * render_min_blocks<HEAD, false>();
            const unsigned grid = (unsigned)std::min<long long>(resident, (long long)a.total_tiles * kBlocksPerTile);
            k_render_queue<HEAD, false, DBG><<<grid, 32 * kRenderWarps, smem, s>>>(a);
        } else {
            if ((e = ensure_smem_limit(k_render<HEAD, false, DBG>, smem, set_fwd, 64)) != cudaSuccess) return e;
            k_render<HEAD, false, DBG><<<a.total_tiles * kBlocksPerTile, 32 * kRenderWarps, smem, s>>>(a);
        }
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- flat per-pixel modes
// The comparison orders of Sec. 3.3 / 4.2 over the same sorted tile lists (forward only):
//   GLOBAL   blend every entry with alpha >= eps_O in tile-list order (the global sort alone);
//   WINDOW-k the per-pixel k-buffer alone: insert into a HEAD-entry window in list order and
//            blend the nearest when it overflows (the hierarchy's head queue without the
//            tail and mid levels);
//   FULL     the exact per-ray order: every entry with alpha >= eps_O by (t_opt at the pixel,
//            list position). Computed by peeling: each pass over the list keeps the HEAD
//            smallest (key, position) pairs above the last blended one and blends them.
// One 256-thread block per 16x16 tile, one thread per pixel (row major); the tile's records
// are staged in shared memory 256 at a time and every pixel evaluates them in list order.
constexpr int kFlatBatch = 256;

__device__ __forceinline__ void flat_init(const PipeArgs& a, const ViewDesc& V, int pxi, int pyi, PixCtx& c)
{
    c.xc = pxi + 0.5f;
    c.yc = pyi + 0.5f;
    c.u = to_u(V, c.xc);
    c.w = to_w(V, c.yc);
    c.n = ray_norm(c.u, c.w);
    c.pix = (pxi < V.W && pyi < V.H) ? V.pix_off + (long long)pyi * V.W + pxi : -1;
    c.bl = 0;                    // the flat orders store no blend order
    c.vrec = a.geom + kRecFloat4 * V.rec_off;
    c.vgrad = a.grad_geom ? a.grad_geom + V.rec_off * kGradStride : nullptr;
    c.g0 = c.g1 = c.g2 = c.gz = c.gbg = 0.f;
    c.Cf0 = c.Cf1 = c.Cf2 = c.Zf = c.Tf = 0.f;
}


template <int HEAD>
__global__ void __launch_bounds__(256) k_render_flat(PipeArgs a)
{
    __shared__ float4 srec[kFlatBatch * kRecFloat4];
    __shared__ uint32_t sid[kFlatBatch];
    if (a.status->error_bits & 1u) return;
    const int gtile = blockIdx.x;
    int lo = 0, hi = a.nviews - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (a.views[m].tile_off <= gtile) lo = m; else hi = m - 1;
    }
    // a local copy: read through a reference, its fields would be reloaded after every store
    const ViewDesc V = a.views[lo];
    const int tile = gtile - V.tile_off;
    const int tx = tile % V.tiles_x, ty = tile / V.tiles_x;
    const int pxi = tx * kTile + (threadIdx.x & 15), pyi = ty * kTile + (threadIdx.x >> 4);
    PixCtx c;
    flat_init(a, V, pxi, pyi, c);
    const bool inside = c.pix >= 0;
    Px<HEAD, true> s;                // comparison orders: debug outputs checked at run time
    px_init(s, inside);
    const uint2 rg = a.ranges[gtile];
    const int lst = (int)rg.x, nL = (int)(rg.y - rg.x);
    const int mode = a.mode;
    const bool evict_first = (a.flags & 1) != 0;
    const bool count = a.dbg_nblend != nullptr;
    unsigned long long n_eval = 0;
    // FULL: the (key << 32 | position) of the last blended entry; peeled candidates
    unsigned long long last = 0ull;
    bool has_last = false, more = mode == STP_MODE_FULL_ID && !s.done;
    // every pass that continues blends HEAD entries of some pixel, so nL / HEAD + 1 passes
    // exhaust any list; the bound makes that explicit, and the caller may lower it
    const int max_pass = a.full_max_passes > 0 ? min(a.full_max_passes, nL / HEAD + 2) : nL / HEAD + 2;
    int pass = 0;
    do {
        unsigned long long ck[HEAD];
        uint32_t cid[HEAD];
        float cv[HEAD];
        int nc = 0;
#pragma unroll
        for (int j = 0; j < HEAD; j++) {
            ck[j] = ~0ull;
            cid[j] = 0;
            cv[j] = 0.f;
        }
        for (int b0 = 0; b0 < nL; b0 += kFlatBatch) {
            if (__syncthreads_and(s.done || (mode == STP_MODE_FULL_ID && !more))) break;
            const int idx = b0 + (int)threadIdx.x;
            if (idx < nL) {
                const uint32_t gid = __ldg(a.svals + lst + idx);
                sid[threadIdx.x] = gid;
                const float4* g = a.geom + kRecFloat4 * (V.rec_off + gid);
#pragma unroll
                for (int k = 0; k < kRecFloat4; k++) srec[threadIdx.x * kRecFloat4 + k] = __ldg(g + k);
            }
            __syncthreads();
            const int nb = min(kFlatBatch, nL - b0);
            if (!s.done && (mode != STP_MODE_FULL_ID || more)) {
                for (int j = 0; j < nb; j++) {
                    Rec r;
                    r.r0 = srec[j * kRecFloat4 + 0]; r.r1 = srec[j * kRecFloat4 + 1];
                    r.r2 = srec[j * kRecFloat4 + 2]; r.r3 = srec[j * kRecFloat4 + 3];
                    r.r4 = srec[j * kRecFloat4 + 4]; r.r5 = srec[j * kRecFloat4 + 5];
                    const float val = splat_value(r, c.xc, c.yc);
                    n_eval++;
                    if (!(fminf(a.alpha_max, val) >= a.eps_o)) continue;
                    const float t = depth_uvn(r, c.u, c.w, c.n);
                    const uint32_t gid = sid[j];
                    if (mode == STP_MODE_GLOBAL_ID) {
                        blend<HEAD, false, true>(a, V, s, c, t, gid, val);
                        if (s.done) break;
                    } else if (mode == STP_MODE_WINDOW_ID) {
                        head_push<HEAD, false, true>(a, V, s, c, head_depth(t), gid, val, evict_first);
                        if (s.done) break;
                    } else {
                        const uint32_t key = depth_key(t);
                        const unsigned long long ek = ((unsigned long long)key << 32) | (uint32_t)(b0 + j);
                        if ((has_last && ek <= last) || ek >= ck[HEAD - 1]) continue;
                        // keep the HEAD smallest: insert ek into the ascending ck
#pragma unroll
                        for (int q = HEAD - 1; q >= 0; q--) {
                            const bool shift = q > 0 && ck[q - 1] > ek;
                            const bool here = ck[q] > ek && !shift;
                            if (shift) { ck[q] = ck[q - 1]; cid[q] = cid[q - 1]; cv[q] = cv[q - 1]; }
                            else if (here) { ck[q] = ek; cid[q] = gid; cv[q] = val; }
                        }
                        nc = min(nc + 1, HEAD);
                    }
                }
            }
            __syncthreads();
        }
        if (mode == STP_MODE_FULL_ID) {
            if (more) {
                if (nc > 0) {
#pragma unroll
                    for (int q = 0; q < HEAD; q++)
                        if (q == nc - 1) last = ck[q];
                    has_last = true;
                }
                // blend the peeled entries nearest first (shifting keeps the indices static)
#pragma unroll 1
                for (int j = 0; j < nc && !s.done; j++) {
                    blend<HEAD, false, true>(a, V, s, c, fkey_inv((uint32_t)(ck[0] >> 32)), cid[0], cv[0]);
#pragma unroll
                    for (int q = 0; q + 1 < HEAD; q++) {
                        ck[q] = ck[q + 1];
                        cid[q] = cid[q + 1];
                        cv[q] = cv[q + 1];
                    }
                }
                more = nc == HEAD && !s.done;     // fewer than HEAD found: the list is exhausted
            }
            if (++pass >= max_pass) {
                if (more) atomicOr(&a.status->error_bits, 4u);
                break;
            }
            if (!__syncthreads_or(more)) break;
        }
    } while (mode == STP_MODE_FULL_ID);
    if (mode == STP_MODE_WINDOW_ID) head_flush<HEAD, false, true>(a, V, s, c);
    if (count) {
        atomicAdd(&a.status->counters[4], n_eval);
        atomicAdd(&a.status->counters[3], (unsigned long long)s.nbl);
    }
    if (!inside) return;
    const long long p = c.pix;
    a.rgb[3 * p] = s.C0 + s.T * a.bg[0];
    a.rgb[3 * p + 1] = s.C1 + s.T * a.bg[1];
    a.rgb[3 * p + 2] = s.C2 + s.T * a.bg[2];
    a.depth[p] = s.Z;
    a.tfinal_ws[p] = s.T;
    if (a.tfinal_out) a.tfinal_out[p] = s.T;
    if (a.dbg_nblend) a.dbg_nblend[p] = s.nbl;
    if (a.dbg_hash) a.dbg_hash[p] = s.hash;
    if (a.dbg_delta) a.dbg_delta[p] = s.delta;
}

template <int HEAD>
cudaError_t launch_flat(const PipeArgs& a, cudaStream_t s)
{
    k_render_flat<HEAD><<<a.total_tiles, 256, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

size_t render_smem_bytes(int tail, int mid) { return (size_t)kRenderWarps * render_warp_smem(tail, mid) * sizeof(uint2); }

bool render_head_supported(int head) { return head == 1 || head == 2 || head == 4 || head == 8 || head == 16; }

cudaError_t launch_render(const PipeArgs& a, bool backward, cudaStream_t s)
{
    if (a.total_tiles == 0) return cudaSuccess;
    if (a.mode != STP_MODE_HIER_ID) {
        if (backward) return cudaErrorInvalidValue;
        if (a.mode == STP_MODE_GLOBAL_ID) return launch_flat<1>(a, s);
        if (a.mode == STP_MODE_FULL_ID) return launch_flat<16>(a, s);
        switch (a.window_k) {
            case 1: return launch_flat<1>(a, s);
            case 2: return launch_flat<2>(a, s);
            case 4: return launch_flat<4>(a, s);
            case 8: return launch_flat<8>(a, s);
            case 16: return launch_flat<16>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    const size_t smem = render_smem_bytes(a.tail, a.mid);
    // debug outputs (blend counts, hashes, sort error, traces, work counters) select the
    // instantiations that keep and write them
    const bool dbg = a.dbg_nblend || a.dbg_hash || a.dbg_delta || a.dbg_trace;
    switch (a.head) {
        case 1: return dbg ? launch_head<1, true>(a, backward, smem, s) : launch_head<1, false>(a, backward, smem, s);
        case 2: return dbg ? launch_head<2, true>(a, backward, smem, s) : launch_head<2, false>(a, backward, smem, s);
        case 4: return dbg ? launch_head<4, true>(a, backward, smem, s) : launch_head<4, false>(a, backward, smem, s);
        case 8: return dbg ? launch_head<8, true>(a, backward, smem, s) : launch_head<8, false>(a, backward, smem, s);
        case 16: return dbg ? launch_head<16, true>(a, backward, smem, s) : launch_head<16, false>(a, backward, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace stp
