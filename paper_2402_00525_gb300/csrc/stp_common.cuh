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
constexpr int kMaxViews = 64;                    // views per launch sequence
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
    long long rec_off;           // view * N: first render record of this view
};

// ---------------------------------------------------------------- render record
// 64-byte per-(view, Gaussian) record written by Preprocess:
//   r0 = (mean2.x, mean2.y, A00, A01)       conic A = Sigma2^-1
//   r1 = (A11, opacity, v.x, v.y)           v = S p (camera space, p = mean in camera space)
//   r2 = (v.z, S00, 2 S01, 2 S02)           S = R_c Sigma^-1 R_c^T (camera space, clamped)
//   r3 = (S11, 2 S12, S22, p.z)
// so that t_opt on the ray through pixel-space point x is
//   t(x) = |d| (v . d) / (d^T S d),  d = ((x - cx) / fx, (y - cy) / fy, 1)   (Eq. "dopt")
struct Rec {
    float4 r0, r1, r2, r3;
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ geom, long long i)
{
    Rec r;
    const float4* p = geom + 4 * i;
    r.r0 = __ldg(p);
    r.r1 = __ldg(p + 1);
    r.r2 = __ldg(p + 2);
    r.r3 = __ldg(p + 3);
    return r;
}

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

// ---------------------------------------------------------------- Algorithm 1
// Point of the box [x0,x1] x [y0,y1] where the 2D Gaussian (mx, my, conic a, b, c) is
// largest: the mean if inside; else a clamped line search along the edge(s) leaving the
// corner nearest to the mean (appendix B.1). Exactly one of the two searches can move off
// the corner for a positive-definite conic.
__device__ __forceinline__ float2 box_max_point(float mx, float my, float a, float b, float c,
                                                float x0, float x1, float y0, float y1)
{
    const bool inx = (mx >= x0) && (mx <= x1);
    const bool iny = (my >= y0) && (my <= y1);
    if (inx && iny) return make_float2(mx, my);
    const float px = mx < x0 ? x0 : (mx > x1 ? x1 : (__fsub_rn(mx, x0) <= __fsub_rn(x1, mx) ? x0 : x1));
    const float py = my < y0 ? y0 : (my > y1 ? y1 : (__fsub_rn(my, y0) <= __fsub_rn(y1, my) ? y0 : y1));
    const float ex = __fsub_rn(px == x0 ? x1 : x0, px);   // edge vector along x
    const float ey = __fsub_rn(py == y0 ? y1 : y0, py);   // edge vector along y
    const float dx = __fsub_rn(mx, px), dy = __fsub_rn(my, py);
    float tx = 0.f, ty = 0.f;
    if (!inx) {     // search along the y-edge x = px
        const float num = __fmul_rn(ey, __fmaf_rn(b, dx, __fmul_rn(c, dy)));
        const float den = __fmul_rn(__fmul_rn(ey, ey), c);
        ty = den > 0.f ? fminf(1.f, fmaxf(0.f, __fdiv_rn(num, den))) : 0.f;
    }
    if (!iny) {     // search along the x-edge y = py
        const float num = __fmul_rn(ex, __fmaf_rn(a, dx, __fmul_rn(b, dy)));
        const float den = __fmul_rn(__fmul_rn(ex, ex), a);
        tx = den > 0.f ? fminf(1.f, fmaxf(0.f, __fdiv_rn(num, den))) : 0.f;
    }
    return make_float2(__fmaf_rn(tx, ex, px), __fmaf_rn(ty, ey, py));
}

// opacity * G2(x) (Sec. 3.1: alpha = opacity times the 2D splat)
__device__ __forceinline__ float splat_value(const Rec& r, float x, float y)
{
    const float dx = __fsub_rn(x, r.r0.x), dy = __fsub_rn(y, r.r0.y);
    const float q = __fmaf_rn(r.r0.z, __fmul_rn(dx, dx),
                              __fmaf_rn(r.r1.x, __fmul_rn(dy, dy),
                                        __fmul_rn(2.f, __fmul_rn(r.r0.w, __fmul_rn(dx, dy)))));
    return __fmul_rn(r.r1.y, expf(__fmul_rn(-0.5f, q)));
}

// t_opt on the ray through camera-normalised coordinates (u, w) = ((x-cx)/fx, (y-cy)/fy)
__device__ __forceinline__ float depth_uv(const Rec& r, float u, float w)
{
    const float L = __fmaf_rn(r.r1.z, u, __fmaf_rn(r.r1.w, w, r.r2.x));
    const float Q = __fmaf_rn(u, __fmaf_rn(r.r2.y, u, __fmaf_rn(r.r2.z, w, r.r2.w)),
                              __fmaf_rn(w, __fmaf_rn(r.r3.x, w, r.r3.y), r.r3.z));
    const float n = __fsqrt_rn(__fmaf_rn(u, u, __fmaf_rn(w, w, 1.f)));
    return __fmul_rn(n, __fdiv_rn(L, Q));
}

__device__ __forceinline__ float to_u(const ViewDesc& V, float x) { return __fmul_rn(__fsub_rn(x, V.cx), V.ifx); }
__device__ __forceinline__ float to_w(const ViewDesc& V, float y) { return __fmul_rn(__fsub_rn(y, V.cy), V.ify); }

// Pixel-centre box of the s x s block at pixel origin (ox, oy), clipped to the image.
struct Box { float x0, x1, y0, y1; };
__device__ __forceinline__ Box block_box(int ox, int oy, int s, int W, int H)
{
    const int xe = min(ox + s - 1, W - 1), ye = min(oy + s - 1, H - 1);
    return Box{ox + 0.5f, xe + 0.5f, oy + 0.5f, ye + 0.5f};
}

// Cull test of a box (Sec. 4.4, "Tile-based culling") and, if kept, the key depth on the
// ray through the box's x_hat ("Tile-depth adjustment"); centre_ray selects the box centre.
__device__ __forceinline__ bool box_keep(const Rec& r, const Box& b, float eps_o)
{
    const float2 xh = box_max_point(r.r0.x, r.r0.y, r.r0.z, r.r0.w, r.r1.x, b.x0, b.x1, b.y0, b.y1);
    return splat_value(r, xh.x, xh.y) >= eps_o;
}
__device__ __forceinline__ bool box_keep_depth(const Rec& r, const Box& b, const ViewDesc& V,
                                               float eps_o, bool centre_ray, float* t)
{
    const float2 xh = box_max_point(r.r0.x, r.r0.y, r.r0.z, r.r0.w, r.r1.x, b.x0, b.x1, b.y0, b.y1);
    if (!(splat_value(r, xh.x, xh.y) >= eps_o)) return false;
    const float x = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.x0, b.x1)) : xh.x;
    const float y = centre_ray ? __fmul_rn(0.5f, __fadd_rn(b.y0, b.y1)) : xh.y;
    *t = depth_uv(r, to_u(V, x), to_w(V, y));
    return true;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace stp
