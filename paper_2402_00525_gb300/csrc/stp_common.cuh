// stp_common.cuh -- device-side types and arithmetic shared by the kernels of libstp.
//
// StopThePop (Radl et al., TOG 43(4) 2024, arXiv 2402.00525). Every decision the pipeline
// takes more than once -- the Algorithm 1 cull test counted in Preprocess and re-taken in
// Duplicate, and the cull / alpha / depth decisions of the forward Render that the backward
// Render replays -- is written with explicit round-to-nearest intrinsics (__fmaf_rn,
// __fmul_rn, ...). The compiler may not contract or reassociate those, so every kernel that
// inlines these functions computes bit-identical values and therefore identical decisions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stp {

constexpr uint32_t kInvalidKey = 0xFFFFFFFFu;   // culled entry / empty queue slot
constexpr int kTile = 16;
constexpr int kMaxViews = 64;                    // views per launch sequence (all scenes)
constexpr int kMaxScenes = 64;
constexpr int STP_MODE_HIER_ID = 0;              // stp_params.mode values (include/stp.h)
constexpr int STP_MODE_FULL_ID = 1;
constexpr int STP_MODE_GLOBAL_ID = 2;
constexpr int STP_MODE_WINDOW_ID = 3;
constexpr int kFlagDebugStats = 32;              // debug outputs (also the per-tile sort's sorted keys)
constexpr int kFlagNoTileCull = 512;             // ablation D: Duplicate keeps every rectangle tile
constexpr int kFlagNoHierCull = 1024;            // ablation E: no culling at the 4x4 / 2x2 levels                   // scenes per launch sequence
constexpr int kSceneAlign = 256;                 // first thread of each scene: multiple of this
constexpr int kMaxMid = 20;                      // largest supported mid-queue size
constexpr uint64_t kHashInit = 1469598103934665603ULL;
constexpr uint64_t kHashMul = 1099511628211ULL;

// ---------------------------------------------------------------- device status block
struct Status {
    unsigned int error_bits;      // 1 capacity, 2 count mismatch padded, 4 timeout
    unsigned int mismatched;
    unsigned long long num_entries;
    unsigned long long capacity;
    unsigned long long counters[5];   // debug counters (see stp_api.cu)
    unsigned int replay_n;        // backward: warps queued for the replay (pixels past blend_cap)
    unsigned int replay_next;     // backward: next queued warp to take
    unsigned long long invalid;   // forward: Gaussians dropped as invalid (counted once per scene)
    unsigned int redo_n;          // forward, depth slices: tile warps queued for the second pass
    unsigned int redo_next;       // forward, depth slices: next queued warp to take
};

// ---------------------------------------------------------------- per-view constants
struct ViewDesc {
    float R[9], t[3];            // world -> camera
    float o[3];                  // camera centre in world space
    float fx, fy, cx, cy;
    float ifx, ify;              // 1 / fx, 1 / fy
    float limx, limy;            // Jacobian clamp limits on x/z and y/z
    int W, H, tiles_x, tiles_y;
    int tile_off;                // first global tile id of this view
    int pad;
    long long pix_off;           // first pixel of this view in the packed image arrays
    long long rec_off;           // first render record of this view (sum of N over earlier views)
};

// ---------------------------------------------------------------- per-scene constants
// The per-Gaussian kernels run one thread per (scene, Gaussian), the per-record kernels one
// thread per (scene, Gaussian, view); each scene starts on a kSceneAlign boundary of either
// thread index space, so a thread block never straddles two scenes.
struct SceneDesc {
    const float* means;          // [n][3]
    const float* log_scales;     // [n][3]
    const float* quats;          // [n][4] (w, x, y, z)
    const float* logits;         // [n]
    const float* sh;             // [n][sh_k][3]
    float* g_means;              // gradients (backward only; null in the forward pass)
    float* g_log_scales;
    float* g_quats;
    float* g_logits;
    float* g_sh;
    int n, sh_k;
    int view_begin, view_end;    // the scene's views [view_begin, view_end)
    long long thread_off;        // per-Gaussian kernels: first thread (multiple of kSceneAlign)
    long long rec_thread_off;    // per-(Gaussian, view) kernels: first thread (multiple of
                                 // kSceneAlign); thread t of the scene takes Gaussian t / nv of
                                 // view view_begin + t % nv (views fastest within a warp)
};

// ---------------------------------------------------------------- render record
// 96-byte per-(view, Gaussian) record written by Preprocess:
//   r0 = (mean2.x hi, mean2.y hi, mean2.x lo, mean2.y lo)   mean2 = hi + lo (projected in FP64)
//   r1 = (e.x, e.y, 1/lambda_max, 1/lambda_min)             conic A = Sigma2^-1 in eigen form
//   r2 = (opacity, colour r, g, b)
//   r3 = (m0.x, m0.y, m0.z, m1.x)
//   r4 = (m1.y, m1.z, m2.x, m2.y)
//   r5 = (m2.z, c0, c1, c2)
// r0..r2 are all a blend needs (alpha and colour), so the backward over a stored blend order
// loads three vectors per blend; r3..r5 are the depth factors. The camera-space depth p.z of
// the mean (the tile key of ablation B only) lives in a separate float per record.
// The conic is kept as its unit major axis e and inverse eigenvalues, so the 2D Mahalanobis
// form q(D) = (e.D)^2 / lambda_max + (e_perp.D)^2 / lambda_min is a sum of non-negative terms,
// and the mean as an unevaluated float pair, so D = x - mean2 keeps its relative accuracy:
// both matter for the cull and alpha decisions of long, thin splats (aspect up to ~2000:1).
// m_k = s_k^-1 (R_c R_q) e_k are the camera-space axes of the Gaussian scaled by the clamped
// inverse scales (Sigma^-1 = R S^-1 S^-1 R^T, appendix A; S^-1 entries <= 1e3, Sec. 3.2) and
// c_k = m_k . p with p the mean in camera space. For the ray through pixel-space point x,
// d = ((x - cx) / fx, (y - cy) / fy, 1), a_k = m_k . d and (Eq. "dopt")
//   t_opt(x) = |d| (sum_k a_k c_k) / (sum_k a_k^2),
// again a sum of per-axis terms without cancellation between eigen-directions.
struct Rec {
    float4 r0, r1, r2, r3, r4, r5;
};
constexpr int kRecFloat4 = 6;

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ geom, long long i)
{
    Rec r;
    const float4* p = geom + kRecFloat4 * i;
    r.r0 = __ldg(p);
    r.r1 = __ldg(p + 1);
    r.r2 = __ldg(p + 2);
    r.r3 = __ldg(p + 3);
    r.r4 = __ldg(p + 4);
    r.r5 = __ldg(p + 5);
    return r;
}

__device__ __forceinline__ float rec_opacity(const Rec& r) { return r.r2.x; }

// order-preserving map float -> uint32 (total order on non-NaN floats)
__device__ __forceinline__ uint32_t fkey(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k)
{
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}

// offset of pixel-space coordinate x from the mean, x - (hi + lo)
__device__ __forceinline__ float off_x(const Rec& r, float x) { return __fsub_rn(__fsub_rn(x, r.r0.x), r.r0.z); }
__device__ __forceinline__ float off_y(const Rec& r, float y) { return __fsub_rn(__fsub_rn(y, r.r0.y), r.r0.w); }

// q(D) = D^T Sigma2^-1 D in the eigen form
__device__ __forceinline__ float quad_form(const Rec& r, float dx, float dy)
{
    const float pe = __fmaf_rn(r.r1.x, dx, __fmul_rn(r.r1.y, dy));
    const float pp = __fmaf_rn(r.r1.x, dy, -__fmul_rn(r.r1.y, dx));
    return __fmaf_rn(r.r1.z, __fmul_rn(pe, pe), __fmul_rn(r.r1.w, __fmul_rn(pp, pp)));
}

// opacity * G2 at offset D (Sec. 2.1: alpha = opacity times the 2D splat)
__device__ __forceinline__ float splat_at(const Rec& r, float dx, float dy)
{
    return __fmul_rn(rec_opacity(r), __expf(__fmul_rn(-0.5f, quad_form(r, dx, dy))));
}
__device__ __forceinline__ float splat_value(const Rec& r, float x, float y)
{
    return splat_at(r, off_x(r, x), off_y(r, y));
}

// ---------------------------------------------------------------- Algorithm 1
// Point of the box [x0,x1] x [y0,y1] where the 2D Gaussian is largest (appendix B.1): the
// mean if inside; otherwise a clamped line search along the edge(s) leaving the corner nearest
// to the mean (exactly one of the two searches can move off the corner for a positive-definite
// conic). Computed in mean-relative coordinates; returns the offset D = x_hat - mean2.
__device__ __forceinline__ float2 box_max_offset(const Rec& r, float x0, float x1, float y0, float y1)
{
    const float bx0 = off_x(r, x0), bx1 = off_x(r, x1), by0 = off_y(r, y0), by1 = off_y(r, y1);
    const bool inx = (bx0 <= 0.f) && (bx1 >= 0.f);
    const bool iny = (by0 <= 0.f) && (by1 >= 0.f);
    const float px = bx0 > 0.f ? bx0 : (bx1 < 0.f ? bx1 : (-bx0 <= bx1 ? bx0 : bx1));
    const float py = by0 > 0.f ? by0 : (by1 < 0.f ? by1 : (-by0 <= by1 ? by0 : by1));
    const float ex = __fsub_rn(px == bx0 ? bx1 : bx0, px);   // edge vector along x
    const float ey = __fsub_rn(py == by0 ? by1 : by0, py);   // edge vector along y
    // A p_hat with A = Sigma2^-1 in eigen form
    const float pe = __fmaf_rn(r.r1.x, px, __fmul_rn(r.r1.y, py));
    const float pp = __fmaf_rn(r.r1.x, py, -__fmul_rn(r.r1.y, px));
    const float se = __fmul_rn(r.r1.z, pe), sp = __fmul_rn(r.r1.w, pp);
    const float Apx = __fmaf_rn(se, r.r1.x, -__fmul_rn(sp, r.r1.y));
    const float Apy = __fmaf_rn(se, r.r1.y, __fmul_rn(sp, r.r1.x));
    // both edge searches, selected (no divergent region; the same values as taking them only
    // off the mean's row / column, and the mean itself when it lies in the box)
    const float Ayy = __fmaf_rn(r.r1.z, __fmul_rn(r.r1.y, r.r1.y), __fmul_rn(r.r1.w, __fmul_rn(r.r1.x, r.r1.x)));
    const float deny = __fmul_rn(ey, Ayy);
    const float tyc = deny != 0.f ? fminf(1.f, fmaxf(0.f, __fdividef(-Apy, deny))) : 0.f;
    const float Axx = __fmaf_rn(r.r1.z, __fmul_rn(r.r1.x, r.r1.x), __fmul_rn(r.r1.w, __fmul_rn(r.r1.y, r.r1.y)));
    const float denx = __fmul_rn(ex, Axx);
    const float txc = denx != 0.f ? fminf(1.f, fmaxf(0.f, __fdividef(-Apx, denx))) : 0.f;
    const float tx = iny ? 0.f : txc, ty = inx ? 0.f : tyc;
    const float2 o = make_float2(__fmaf_rn(tx, ex, px), __fmaf_rn(ty, ey, py));
    return (inx && iny) ? make_float2(0.f, 0.f) : o;
}

// t_opt on the ray through camera-normalised coordinates (u, w) = ((x-cx)/fx, (y-cy)/fy),
// n = |(u, w, 1)| (precomputed for a pixel's own ray)
__device__ __forceinline__ float depth_uvn(const Rec& r, float u, float w, float n)
{
    const float a0 = __fmaf_rn(r.r3.x, u, __fmaf_rn(r.r3.y, w, r.r3.z));
    const float a1 = __fmaf_rn(r.r3.w, u, __fmaf_rn(r.r4.x, w, r.r4.y));
    const float a2 = __fmaf_rn(r.r4.z, u, __fmaf_rn(r.r4.w, w, r.r5.x));
    const float num = __fmaf_rn(a0, r.r5.y, __fmaf_rn(a1, r.r5.z, __fmul_rn(a2, r.r5.w)));
    const float den = __fmaf_rn(a0, a0, __fmaf_rn(a1, a1, __fmul_rn(a2, a2)));
    return __fmul_rn(n, __fdividef(num, den));
}
__device__ __forceinline__ float ray_norm(float u, float w) { return __fsqrt_rn(__fmaf_rn(u, u, __fmaf_rn(w, w, 1.f))); }
__device__ __forceinline__ float depth_uv(const Rec& r, float u, float w) { return depth_uvn(r, u, w, ray_norm(u, w)); }

__device__ __forceinline__ float to_u(const ViewDesc& V, float x) { return __fmul_rn(__fsub_rn(x, V.cx), V.ifx); }
__device__ __forceinline__ float to_w(const ViewDesc& V, float y) { return __fmul_rn(__fsub_rn(y, V.cy), V.ify); }

// Pixel-centre box of the s x s block at pixel origin (ox, oy), clipped to the image.
struct Box { float x0, x1, y0, y1; };
__device__ __forceinline__ Box block_box(int ox, int oy, int s, int W, int H)
{
    const int xe = min(ox + s - 1, W - 1), ye = min(oy + s - 1, H - 1);
    return Box{ox + 0.5f, xe + 0.5f, oy + 0.5f, ye + 0.5f};
}

// Cull test of a box (Sec. 3.4, "Tile-based culling") and, if kept, the key depth on the
// ray through the box's x_hat ("Tile-depth adjustment"); centre_ray selects the box centre.
__device__ __forceinline__ bool box_keep(const Rec& r, const Box& b, float eps_o)
{
    const float2 d = box_max_offset(r, b.x0, b.x1, b.y0, b.y1);
    return splat_at(r, d.x, d.y) >= eps_o;
}
// key depth of a box already known to be kept (the same arithmetic as box_keep_depth)
__device__ __forceinline__ float box_depth(const Rec& r, const Box& b, const ViewDesc& V, bool centre_ray)
{
    const float2 d = box_max_offset(r, b.x0, b.x1, b.y0, b.y1);
    const float x = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.x0, b.x1)) : __fadd_rn(r.r0.x, __fadd_rn(r.r0.z, d.x));
    const float y = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.y0, b.y1)) : __fadd_rn(r.r0.y, __fadd_rn(r.r0.w, d.y));
    return depth_uv(r, to_u(V, x), to_w(V, y));
}
__device__ __forceinline__ bool box_keep_depth(const Rec& r, const Box& b, const ViewDesc& V,
                                               float eps_o, bool centre_ray, float* t)
{
    const float2 d = box_max_offset(r, b.x0, b.x1, b.y0, b.y1);
    const bool keep = splat_at(r, d.x, d.y) >= eps_o;
    // the depth is taken for a culled box too (no divergent region; callers read *t only for a
    // kept box, and a degenerate value there is never used)
    const float x = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.x0, b.x1)) : __fadd_rn(r.r0.x, __fadd_rn(r.r0.z, d.x));
    const float y = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.y0, b.y1)) : __fadd_rn(r.r0.y, __fadd_rn(r.r0.w, d.y));
    *t = depth_uv(r, to_u(V, x), to_w(V, y));
    return keep;
}

// Raise a kernel's dynamic shared-memory limit once per device (host side). Later launches,
// including launches recorded under stream capture, then make no attribute call.
template <typename F>
inline cudaError_t ensure_smem_limit(F* fn, size_t bytes, int* done_per_device, int ndev)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < ndev && done_per_device[dev] >= (int)bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && dev >= 0 && dev < ndev) done_per_device[dev] = (int)bytes;
    return e;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace stp
