// stp_preprocess.cu -- Preprocess, the scan of tile counts, and Duplicate.
//
// StopThePop (arXiv 2402.00525) Sec. 3.4 and appendix B: per Gaussian and view, the EWA 2D
// splat, SH colour, Sigma^-1 with the S^-1 clamp in factored form for the depth evaluation,
// the candidate tiles from the opacity-aware extent (appendix B.2; here the axis-aligned box
// of the ellipse o G >= eps_O), and the number of tiles that survive exact culling (Algorithm
// 1), with the kept candidates of small rectangles recorded in a bit mask. Duplicate writes
// one (tile, t_opt) key per kept tile (computing depths only for the masked tiles, or taking
// the same cull decisions again for larger rectangles). Both stages use the paper's two-phase
// load balancing: a record with at most `lb_threshold` candidate tiles is handled by its own
// thread; larger ones by the whole warp (ballot / shuffle / popc offsets).
//
// One thread per (Gaussian, view), the views of a Gaussian in neighbouring lanes, so the
// Gaussian's parameters (236 bytes at SH degree 3) are read from HBM once for all its views.
#include <cuda_runtime.h>

#include "stp_common.cuh"
#include "stp_kernels.cuh"

namespace stp {


namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Real spherical harmonics to degree 3, Condon-Shortley phase, as polynomials of the unit
// view direction; constants sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0).
// Returns false if a channel's sum is not finite (a non-finite coefficient: NaN and +-inf
// propagate through the sum whatever the basis values, 0 included).
__device__ __forceinline__ bool sh_colour(const float* __restrict__ c, int K, float x, float y,
                                          float z, float out[3])
{
    const float k0 = 0.28209479177387814f, k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
    float Y[16];
    Y[0] = k0;
    if (K > 1) {
        Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (2.f * zz - xx - yy);
        Y[7] = -k2a * x * z; Y[8] = k2c * (xx - yy);
        if (K > 9) {
            Y[9] = -k3a * y * (3.f * xx - yy);
            Y[10] = k3b * x * y * z;
            Y[11] = -k3c * y * (4.f * zz - xx - yy);
            Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -k3c * x * (4.f * zz - xx - yy);
            Y[14] = k3e * z * (xx - yy);
            Y[15] = -k3a * x * (xx - 3.f * yy);
        }
    }
    float s0 = 0.5f, s1 = 0.5f, s2 = 0.5f;
    if (K == 16 && (reinterpret_cast<uintptr_t>(c) & 15) == 0) {
        // degree 3 (48 floats): twelve 16-byte loads, summed in the same order as below
        const float4* c4 = reinterpret_cast<const float4*>(c);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float4 v0 = __ldg(c4 + 3 * q), v1 = __ldg(c4 + 3 * q + 1), v2 = __ldg(c4 + 3 * q + 2);
            const float cr[4] = {v0.x, v0.w, v1.z, v2.y}, cg[4] = {v0.y, v1.x, v1.w, v2.z}, cb[4] = {v0.z, v1.y, v2.x, v2.w};
#pragma unroll
            for (int u = 0; u < 4; u++) {
                s0 += Y[4 * q + u] * cr[u];
                s1 += Y[4 * q + u] * cg[u];
                s2 += Y[4 * q + u] * cb[u];
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; j++) {           // static indices: Y stays in registers
            if (j < K) {
                s0 += Y[j] * __ldg(c + 3 * j);
                s1 += Y[j] * __ldg(c + 3 * j + 1);
                s2 += Y[j] * __ldg(c + 3 * j + 2);
            }
        }
    }
    out[0] = fmaxf(s0, 0.f);
    out[1] = fmaxf(s1, 0.f);
    out[2] = fmaxf(s2, 0.f);
    return isfinite(s0) && isfinite(s1) && isfinite(s2);
}

// every SH coefficient of a Gaussian is finite (checked where the colour was not evaluated)
__device__ __noinline__ bool sh_finite(const float* __restrict__ c, int K)
{
    bool ok = true;
    for (int j = 0; j < 3 * K; j++) ok &= isfinite(__ldg(c + j));
    return ok;
}

enum RecKind { kRecInvisible = 0, kRecVisible = 1, kRecInvalid = 2 };

struct GaussIn {             // view-independent quantities of one Gaussian
    float mu[3];
    float s[3];              // scales
    float Rq[9];             // rotation of the normalised quaternion (row major)
    float si[3];             // clamped inverse scales min(1/s, inv_scale_max)
    float opacity;
    const float* sh;         // this Gaussian's SH coefficients [sh_k][3]
    int sh_k;
    bool valid;              // finite parameters and a quaternion of non-zero length
};

__device__ __forceinline__ void load_gauss(const PipeArgs& a, const SceneDesc& S, int i, GaussIn& g)
{
    g.mu[0] = __ldg(S.means + 3 * i);
    g.mu[1] = __ldg(S.means + 3 * i + 1);
    g.mu[2] = __ldg(S.means + 3 * i + 2);
    float qw = __ldg(S.quats + 4 * i), qx = __ldg(S.quats + 4 * i + 1);
    float qy = __ldg(S.quats + 4 * i + 2), qz = __ldg(S.quats + 4 * i + 3);
    const float q[4] = {qw, qx, qy, qz};
    const float q2 = qw * qw + qx * qx + qy * qy + qz * qz;
    const float ql = rsqrtf(q2);
    qw *= ql; qx *= ql; qy *= ql; qz *= ql;
    const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    for (int k = 0; k < 3; k++) {
        const float ls = __ldg(S.log_scales + 3 * i + k);
        g.s[k] = expf(ls);
        g.si[k] = fminf(expf(-ls), a.inv_scale_max);
    }
    for (int k = 0; k < 9; k++) g.Rq[k] = R[k];
    const float logit = __ldg(S.logits + i);
    g.opacity = 1.f / (1.f + expf(-logit));
    g.sh = S.sh + (long long)i * S.sh_k * 3;
    g.sh_k = S.sh_k;
    // Inputs outside the method's domain make the Gaussian invalid: it is dropped before any
    // other step and counted (the SH coefficients are checked through the colour sum). x * 0
    // is NaN exactly when x is NaN or infinite, so one sum tests all eleven scalars.
    float chk = logit * 0.f;
    for (int k = 0; k < 3; k++) chk += g.mu[k] * 0.f + __ldg(S.log_scales + 3 * i + k) * 0.f;
    chk += (q[0] * 0.f + q[1] * 0.f) + (q[2] * 0.f + q[3] * 0.f);
    g.valid = chk == 0.f && q2 >= 1e-20f;
}


// An invalid Gaussian is counted once per scene, by the thread of the scene's first view
// (count = true). Where that view culls the Gaussian before its colour is evaluated, the SH
// coefficients are checked directly.
__device__ __forceinline__ int invisible(const PipeArgs& a, const GaussIn& g, bool count)
{
    if (count && !sh_finite(g.sh, g.sh_k)) {
        atomicAdd(&a.status->invalid, 1ull);
        return kRecInvalid;
    }
    return kRecInvisible;
}
__device__ __forceinline__ int invalid(const PipeArgs& a, bool count)
{
    if (count) atomicAdd(&a.status->invalid, 1ull);
    return kRecInvalid;
}

// ---------------------------------------------------------------- float-float arithmetic
// An unevaluated pair hi + lo of FP32 values (about 44 significant bits) built from the
// error-free transformations of Dekker and Knuth: the product of two floats is exactly
// p + e with p = a*b rounded and e = fma(a, b, -p); the sum is exactly s + e with Knuth's
// six-operation two-sum. The FP64 pipe of this GPU issues at 1/64 of the FP32 rate, so these
// pairs carry the precision the projected mean and the depth factors need.
struct ff { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ ff renorm(float s, float e)      // |e| small against s
{
    const float h = __fadd_rn(s, e);
    return ff{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// c + sum_j a_j b_j over three terms, compensated: accurate to about the pair's precision
__device__ __forceinline__ ff dot3_ff(const float a[3], const float b[3], float c)
{
    float s = c, err = 0.f;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float p = __fmul_rn(a[j], b[j]);
        const float pe = __fmaf_rn(a[j], b[j], -p);
        float e;
        two_sum(s, p, s, e);
        err = __fadd_rn(err, __fadd_rn(e, pe));
    }
    return renorm(s, err);
}
// sum_j a_j x_j with float a_j and pair x_j
__device__ __forceinline__ ff dot3_f_ff(const float a[3], const ff x[3])
{
    float s = 0.f, err = 0.f;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float p = __fmul_rn(a[j], x[j].hi);
        const float pe = __fmaf_rn(a[j], x[j].hi, -p);
        float e;
        two_sum(s, p, s, e);
        err = __fadd_rn(err, __fadd_rn(e, __fmaf_rn(a[j], x[j].lo, pe)));
    }
    return renorm(s, err);
}
__device__ __forceinline__ ff mul_ff(ff x, ff y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.hi, -p);
    return renorm(p, __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e)));
}
__device__ __forceinline__ ff rcp_ff(ff x)                  // 1 / x, one Newton correction
{
    const float y = __frcp_rn(x.hi);
    const float p = __fmul_rn(x.hi, y);
    const float pe = __fmaf_rn(x.hi, y, -p);
    const float r = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(x.lo, y));   // 1 - x y
    return renorm(y, __fmul_rn(y, r));
}
// a x + b with float a, b and pair x
__device__ __forceinline__ ff fma_f_ff(float a, ff x, float b)
{
    const float p = __fmul_rn(a, x.hi);
    const float pe = __fmaf_rn(a, x.hi, -p);
    float s, e;
    two_sum(p, b, s, e);
    return renorm(s, __fadd_rn(e, __fmaf_rn(a, x.lo, pe)));
}

// Per-(view, Gaussian) record (layout in stp_common.cuh). Returns kRecVisible, kRecInvisible
// (near plane, opacity below eps_O, degenerate splat: the colour is not evaluated) or
// kRecInvalid (non-finite inputs); the record stays zero unless visible.
// The camera-space mean and its projection are evaluated in float-float pairs (about 44 bits):
// mean2 is ~1e3 px, where an FP32 rounding of 6e-5 px would move the alpha of a sub-pixel-wide
// splat by ~1e-3 relative; the record keeps mean2 as such a pair. Sigma2 = B B^T + dilation I with B = T M
// (M = R_q diag(s), Sigma = M M^T), so det Sigma2 = |b0 x b1|^2 + dil (|b0|^2 + |b1|^2) + dil^2
// is a sum of non-negative terms instead of the cancelling a c - b^2.
__device__ int make_record(const PipeArgs& a, const ViewDesc& V, const GaussIn& g, int i,
                           Rec& rec, float& vz, ushort4& rect, bool count)
{
    rect = make_ushort4(0, 0, 0, 0);
    rec.r0 = rec.r1 = rec.r2 = rec.r3 = rec.r4 = rec.r5 = make_float4(0.f, 0.f, 0.f, 0.f);
    vz = 0.f;
    if (!g.valid) return invalid(a, count);
    ff pd[3];                                     // camera-space mean R mu + t
    for (int k = 0; k < 3; k++) {
        const float rk[3] = {V.R[3 * k], V.R[3 * k + 1], V.R[3 * k + 2]};
        pd[k] = dot3_ff(rk, g.mu, V.t[k]);
    }
    if (!(pd[2].hi > a.znear)) return invisible(a, g, count);
    if (!(g.opacity >= a.eps_o)) return invisible(a, g, count);
    const ff izd = rcp_ff(pd[2]);
    const ff uxd = mul_ff(pd[0], izd), uyd = mul_ff(pd[1], izd);
    const ff mxd = fma_f_ff(V.fx, uxd, V.cx), myd = fma_f_ff(V.fy, uyd, V.cy);
    const float p[3] = {pd[0].hi, pd[1].hi, pd[2].hi};
    const float iz = 1.f / p[2];
    const float ux = uxd.hi, uy = uyd.hi;
    const float cx = fminf(V.limx, fmaxf(-V.limx, ux)), cy = fminf(V.limy, fmaxf(-V.limy, uy));
    const float J00 = V.fx * iz, J02 = -V.fx * cx * iz, J11 = V.fy * iz, J12 = -V.fy * cy * iz;
    float T[2][3];
    for (int c = 0; c < 3; c++) {
        T[0][c] = J00 * V.R[c] + J02 * V.R[6 + c];
        T[1][c] = J11 * V.R[3 + c] + J12 * V.R[6 + c];
    }
    // B = T R_q diag(s): rows b0, b1
    float B[2][3];
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++)
            B[r][k] = (T[r][0] * g.Rq[k] + T[r][1] * g.Rq[3 + k] + T[r][2] * g.Rq[6 + k]) * g.s[k];
    const float n0 = B[0][0] * B[0][0] + B[0][1] * B[0][1] + B[0][2] * B[0][2];
    const float n1 = B[1][0] * B[1][0] + B[1][1] * B[1][1] + B[1][2] * B[1][2];
    const float cb = B[0][0] * B[1][0] + B[0][1] * B[1][1] + B[0][2] * B[1][2];
    const float x0 = B[0][1] * B[1][2] - B[0][2] * B[1][1];
    const float x1 = B[0][2] * B[1][0] - B[0][0] * B[1][2];
    const float x2 = B[0][0] * B[1][1] - B[0][1] * B[1][0];
    const float dil = a.dilation;
    const float ca = n0 + dil, cc = n1 + dil;
    const float det = (x0 * x0 + x1 * x1 + x2 * x2) + dil * (n0 + n1) + dil * dil;
    if (!(det > 0.f)) return invisible(a, g, count);
    // eigen form of Sigma2: lambda_max = mean + sqrt(half-difference^2 + b^2), lambda_min = det/lambda_max
    const float hd = 0.5f * (ca - cc);
    const float lmax = 0.5f * (ca + cc) + sqrtf(hd * hd + cb * cb);
    const float lmin = det / lmax;
    float ex = cb, ey = lmax - ca;                 // (Sigma2 - lmax I) v = 0
    const float fx2 = lmax - cc, fy2 = cb;
    if (fx2 * fx2 + fy2 * fy2 > ex * ex + ey * ey) { ex = fx2; ey = fy2; }
    const float en = ex * ex + ey * ey;
    if (en > 0.f) {
        const float inv = rsqrtf(en);
        ex *= inv;
        ey *= inv;
    } else {
        ex = 1.f;
        ey = 0.f;
    }
    const float mx_hi = mxd.hi, my_hi = myd.hi;
    const float mx_lo = mxd.lo, my_lo = myd.lo;
    // camera-space axes scaled by the clamped inverse scales, and their projections of p
    float m[3][3], c[3];
    for (int k = 0; k < 3; k++) {
        for (int r = 0; r < 3; r++)
            m[k][r] = g.si[k] * (V.R[3 * r] * g.Rq[k] + V.R[3 * r + 1] * g.Rq[3 + k] + V.R[3 * r + 2] * g.Rq[6 + k]);
        const ff ck = dot3_f_ff(m[k], pd);
        c[k] = __fadd_rn(ck.hi, ck.lo);
    }
    rec.r0 = make_float4(mx_hi, my_hi, mx_lo, my_lo);
    rec.r1 = make_float4(ex, ey, 1.f / lmax, 1.f / lmin);
    rec.r3 = make_float4(m[0][0], m[0][1], m[0][2], m[1][0]);
    rec.r4 = make_float4(m[1][1], m[1][2], m[2][0], m[2][1]);
    rec.r5 = make_float4(m[2][2], c[0], c[1], c[2]);
    vz = p[2];
    // colour: SH with the direction from the camera centre to the mean
    float d[3] = {g.mu[0] - V.o[0], g.mu[1] - V.o[1], g.mu[2] - V.o[2]};
    const float dl = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    float rgb[3];
    if (!sh_colour(g.sh, g.sh_k, d[0] * dl, d[1] * dl, d[2] * dl, rgb)) {
        rec.r0 = rec.r1 = rec.r2 = rec.r3 = rec.r4 = rec.r5 = make_float4(0.f, 0.f, 0.f, 0.f);
        vz = 0.f;
        return invalid(a, count);
    }
    rec.r2 = make_float4(g.opacity, rgb[0], rgb[1], rgb[2]);
    // Candidate tiles. With the opacity-aware radius of appendix B.2, o G >= eps_O holds only on
    // the ellipse (x - mean2)^T A (x - mean2) <= t_O^2, whose axis-aligned half-widths are
    // t_O sqrt(Sigma2_xx) and t_O sqrt(Sigma2_yy) -- never more than the paper's square radius
    // ceil(t_O sqrt(lambda_max)), often far less for anisotropic splats. Every tile this box
    // drops would fail Algorithm 1's test, so the kept entries are the same; only fewer tiles
    // are tested. The box takes the tiles holding a pixel centre within it (small slack for
    // rounding). Without tile-based culling (ablation D) every tile of the paper's square is kept,
    // so that case keeps the square.
    const float tO = sqrtf(2.f * logf(g.opacity / a.eps_o));
    const float rad = ceilf(tO * sqrtf(lmax));
    const bool square = (a.flags & kFlagNoTileCull) != 0;
    const float hx = square ? rad : fminf(rad, fmaf(tO * sqrtf(ca), 1.0001f, 0.01f));
    const float hy = square ? rad : fminf(rad, fmaf(tO * sqrtf(cc), 1.0001f, 0.01f));
    const float mx = mxd.hi, my = myd.hi;
    const float fx0 = ceilf((mx - hx - 15.5f) * (1.f / 16.f)), fx1 = floorf((mx + hx - 0.5f) * (1.f / 16.f));
    const float fy0 = ceilf((my - hy - 15.5f) * (1.f / 16.f)), fy1 = floorf((my + hy - 0.5f) * (1.f / 16.f));
    const int tx0 = (int)fmaxf(0.f, fx0), ty0 = (int)fmaxf(0.f, fy0);
    const int tx1 = (int)fminf((float)(V.tiles_x - 1), fx1), ty1 = (int)fminf((float)(V.tiles_y - 1), fy1);
    if (tx1 >= tx0 && ty1 >= ty0)
        rect = make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)(tx1 + 1),
                            (unsigned short)(ty1 + 1));
    return kRecVisible;
}

__device__ __forceinline__ Rec shfl_rec(const Rec& r, int src)
{
    Rec o;
    o.r0 = make_float4(__shfl_sync(kFull, r.r0.x, src), __shfl_sync(kFull, r.r0.y, src),
                       __shfl_sync(kFull, r.r0.z, src), __shfl_sync(kFull, r.r0.w, src));
    o.r1 = make_float4(__shfl_sync(kFull, r.r1.x, src), __shfl_sync(kFull, r.r1.y, src),
                       __shfl_sync(kFull, r.r1.z, src), __shfl_sync(kFull, r.r1.w, src));
    o.r2 = make_float4(__shfl_sync(kFull, r.r2.x, src), 0.f, 0.f, 0.f);   // opacity (no colour here)
    o.r3 = make_float4(__shfl_sync(kFull, r.r3.x, src), __shfl_sync(kFull, r.r3.y, src),
                       __shfl_sync(kFull, r.r3.z, src), __shfl_sync(kFull, r.r3.w, src));
    o.r4 = make_float4(__shfl_sync(kFull, r.r4.x, src), __shfl_sync(kFull, r.r4.y, src),
                       __shfl_sync(kFull, r.r4.z, src), __shfl_sync(kFull, r.r4.w, src));
    o.r5 = make_float4(__shfl_sync(kFull, r.r5.x, src), __shfl_sync(kFull, r.r5.y, src),
                       __shfl_sync(kFull, r.r5.z, src), __shfl_sync(kFull, r.r5.w, src));
    return o;
}

__device__ __forceinline__ float tile_cull_eps(const PipeArgs& a)
{
    return (a.flags & kFlagNoTileCull) ? -1.f : a.eps_o;
}

// Depth key of one (Gaussian, tile) pair if the tile is kept: ordered bits of t_opt on the ray
// through the tile's x_hat (or the tile centre / the view-space depth, by flag).
__device__ __forceinline__ bool tile_depth_key(const PipeArgs& a, const ViewDesc& V, const Rec& r, float vz,
                                               int tx, int ty, uint32_t* dkey)
{
    const Box b = block_box(tx * kTile, ty * kTile, kTile, V.W, V.H);
    float t = 0.f;
    if (!box_keep_depth(r, b, V, tile_cull_eps(a), (a.flags & 4) != 0, &t)) return false;
    if (a.flags & 8) t = vz;
    *dkey = fkey(t);
    return true;
}

// Tile-based culling decision (Sec. 3.4); flag kFlagNoTileCull keeps every tile of the
// rectangle (ablation D of the paper's performance table) through a threshold of -1.
__device__ __forceinline__ bool tile_keep(const PipeArgs& a, const Rec& r, const Box& b)
{
    return box_keep(r, b, tile_cull_eps(a));
}

// Partitioned sort (appendix B.3): count a kept entry of global tile `gt`. (Aggregating the
// lanes of a warp that hit the same tile measured slower than plain atomics here.)
__device__ __forceinline__ void count_entry(const PipeArgs& a, uint32_t gt)
{
    atomicAdd(&a.tile_counts[gt], 1u);
}

// Partitioned sort: place an entry in its tile's range through the tile's atomic cursor. The
// order inside a range is arbitrary here and fixed by the per-tile sort on (depth, id).
__device__ __forceinline__ void place_entry(const PipeArgs& a, uint32_t gt, uint32_t dkey, uint32_t gid)
{
    const uint32_t slot = atomicAdd(&a.tile_cursor[gt], 1u);
    if (slot >= a.tile_counts[gt]) {   // more entries than Preprocess counted: cannot happen
        atomicOr(&a.status->error_bits, 2u);
        return;
    }
    const unsigned long long pos = (unsigned long long)a.tile_offsets[gt] + slot;
    if (pos < a.capacity) a.dup_keys[pos] = ((unsigned long long)dkey << 32) | gid;
}

// depth key of a tile Preprocess found kept
__device__ __forceinline__ uint32_t kept_depth_key(const PipeArgs& a, const ViewDesc& V, const Rec& r, float vz,
                                                   int tx, int ty)
{
    const Box b = block_box(tx * kTile, ty * kTile, kTile, V.W, V.H);
    float t = box_depth(r, b, V, (a.flags & 4) != 0);
    if (a.flags & 8) t = vz;
    return fkey(t);
}

// Column and row of the k-th tile (row major) of a rectangle w tiles wide, with rw = 1 / w
// rounded to nearest, and no integer division: the quotient (k + 1/2) / w lies at least 1/(2w)
// from an integer, and its float evaluation errs by under 2^-22 of its value, so the floor is
// exact for every k below 2^20 (a rectangle never holds more tiles than a 16384 x 16384
// view's 2^20).
__device__ __forceinline__ int2 rect_cell(int k, int w, float rw)
{
    const int y = (int)(((float)k + 0.5f) * rw);
    return make_int2(k - y * w, y);
}
__device__ __forceinline__ float rect_rcp(int w) { return w > 0 ? 1.f / (float)w : 0.f; }

// Count (EMIT = false) or write (EMIT = true) the kept tiles of this lane's Gaussian, with the
// two-phase warp load balancing. Every lane of the warp must call it. Preprocess records the
// kept candidates of the per-thread phase in a bit mask (rectangles of at most 32 tiles), so
// Duplicate computes depths only for kept tiles and never re-takes a cull decision there.
// With the global radix sort the keys go to the Gaussian's own range [off, off + want) in
// tile order; with the partitioned sort they go to their tiles' ranges.
template <bool EMIT>
__device__ uint32_t tiles_pass(const PipeArgs& a, const ViewDesc& V, int vidx, bool has, const Rec& r, float vz,
                               ushort4 rc, uint32_t off, uint32_t want, uint32_t gid, uint32_t* mask_io)
{
    const int lane = threadIdx.x & 31;
    const int w = (int)rc.z - (int)rc.x, h = (int)rc.w - (int)rc.y;
    const int ncand = has ? w * h : 0;
    const bool big = ncand > a.lb_threshold && !(a.flags & 16);
    const bool part = a.partitioned != 0;
    uint32_t cnt = 0;
    if (!big) {
        if (!EMIT) {
            uint32_t mask = 0;
            int cx = 0, cy = 0;                          // column and row of candidate k
            for (int k = 0; k < ncand; k++, cx = cx + 1 < w ? cx + 1 : 0, cy += cx == 0) {
                const int tx = rc.x + cx, ty = rc.y + cy;
                const Box b = block_box(tx * kTile, ty * kTile, kTile, V.W, V.H);
                if (tile_keep(a, r, b)) {
                    cnt++;
                    if (k < 32) mask |= 1u << k;
                    if (part) count_entry(a, (uint32_t)(V.tile_off + ty * V.tiles_x + tx));
                }
            }
            *mask_io = mask;
        } else if (ncand <= 32) {
            // emit the kept tiles of the mask, four cursor reservations in flight at a time
            uint32_t mask = *mask_io;
            while (mask) {
                uint32_t gts[4], dks[4];
                int np = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int tx = rc.x + k % w, ty = rc.y + k / w;
                        gts[j] = (uint32_t)(V.tile_off + ty * V.tiles_x + tx);
                        dks[j] = kept_depth_key(a, V, r, vz, tx, ty);
                        np = j + 1;
                    }
                }
                if (part) {
                    uint32_t slot[4];
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (j < np) slot[j] = atomicAdd(&a.tile_cursor[gts[j]], 1u);
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (j < np) {
                            if (slot[j] >= a.tile_counts[gts[j]]) {
                                atomicOr(&a.status->error_bits, 2u);
                            } else {
                                const unsigned long long pos = (unsigned long long)a.tile_offsets[gts[j]] + slot[j];
                                if (pos < a.capacity) a.dup_keys[pos] = ((unsigned long long)dks[j] << 32) | gid;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (j < np) {
                            const unsigned long long pos = (unsigned long long)off + cnt;
                            if (cnt < want && pos < a.capacity) {
                                a.dup_keys[pos] = ((unsigned long long)gts[j] << 32) | dks[j];
                                a.dup_vals[pos] = gid;
                            }
                            cnt++;
                        }
                    }
                }
                if (part) cnt += np;
            }
        } else {
            // per-thread path with more than 32 candidates (lb_threshold > 32): evaluate again
            for (int k = 0; k < ncand; k++) {
                const int tx = rc.x + k % w, ty = rc.y + k / w;
                const uint32_t gt = (uint32_t)(V.tile_off + ty * V.tiles_x + tx);
                uint32_t dk;
                if (tile_depth_key(a, V, r, vz, tx, ty, &dk)) {
                    if (part) {
                        place_entry(a, gt, dk, gid);
                    } else {
                        const unsigned long long pos = (unsigned long long)off + cnt;
                        if (cnt < want && pos < a.capacity) {
                            a.dup_keys[pos] = ((unsigned long long)gt << 32) | dk;
                            a.dup_vals[pos] = gid;
                        }
                    }
                    cnt++;
                }
            }
        }
    }
    unsigned bigmask = __ballot_sync(kFull, big);
    while (bigmask) {
        const int src = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        const Rec rs = shfl_rec(r, src);
        const int ws = __shfl_sync(kFull, w, src), nc = __shfl_sync(kFull, ncand, src);
        // the count divides without an integer division; Duplicate keeps k % w, k / w (the float
        // path measured slower there, its spread placement being register bound)
        const float rws = EMIT ? 0.f : __shfl_sync(kFull, rect_rcp(w), src);
        const int x0 = __shfl_sync(kFull, (int)rc.x, src), y0 = __shfl_sync(kFull, (int)rc.y, src);
        const uint32_t offs = __shfl_sync(kFull, off, src), wants = __shfl_sync(kFull, want, src);
        const uint32_t gids = __shfl_sync(kFull, gid, src);
        const ViewDesc& Vs = a.views[__shfl_sync(kFull, vidx, src)];    // the source lane's view
        const float vzs = __shfl_sync(kFull, vz, src);
        uint32_t base = 0;
        for (int k0 = 0; k0 < nc; k0 += 32) {
            const int k = k0 + lane;
            bool keep = false;
            uint32_t dk = 0, gt = 0;
            if (k < nc) {
                const int2 cl = EMIT ? make_int2(k % ws, k / ws) : rect_cell(k, ws, rws);
                const int tx = x0 + cl.x, ty = y0 + cl.y;
                gt = (uint32_t)(Vs.tile_off + ty * Vs.tiles_x + tx);
                if (EMIT) keep = tile_depth_key(a, Vs, rs, vzs, tx, ty, &dk);
                else keep = tile_keep(a, rs, block_box(tx * kTile, ty * kTile, kTile, Vs.W, Vs.H));
            }
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                if (EMIT) {
                    if (part) {
                        place_entry(a, gt, dk, gids);
                    } else {
                        const uint32_t rank = base + __popc(m & lanemask_lt());
                        const unsigned long long pos = (unsigned long long)offs + rank;
                        if (rank < wants && pos < a.capacity) {
                            a.dup_keys[pos] = ((unsigned long long)gt << 32) | dk;
                            a.dup_vals[pos] = gids;
                        }
                    }
                } else if (part) {
                    count_entry(a, gt);
                }
            }
            base += __popc(m);
        }
        if (lane == src) cnt = base;
    }
    return cnt;
}

// One thread per (Gaussian, view), the scene's views fastest within a warp: lanes that share a
// Gaussian see it from different cameras, so their tile counts are alike (little divergence).
// 128-thread blocks (scenes start on 256-thread boundaries, so a block never straddles two),
// ten (Preprocess) and twelve (Duplicate) resident per SM: the register caps spill to L1, but
// the occupancy hides the latency of the loads and tile-counter atomics (chosen by sweeping
// 8..16 blocks on 16 Full-HD views of 3M Gaussians).
#ifndef STP_PRE_MIN_BLOCKS
#define STP_PRE_MIN_BLOCKS 10
#endif
#ifndef STP_DUP_MIN_BLOCKS
#define STP_DUP_MIN_BLOCKS 12
#endif

struct RecThread {
    SceneDesc S;
    int i, v;                    // Gaussian (scene-local) and view (global index)
    bool live;
};

__device__ __forceinline__ RecThread rec_thread(const PipeArgs& a)
{
    RecThread t;
    const long long t0 = (long long)blockIdx.x * blockDim.x;
    t.S = a.scenes[scene_of_rec(a, t0)];
    const int nv = t.S.view_end - t.S.view_begin;
    const long long lt = t0 - t.S.rec_thread_off + threadIdx.x;
    long long q = 0, rm = 0;
    if (nv > 0) {
        if (lt < 0xFFFFFFFFll) {         // 32-bit division when it fits (the common case)
            q = (uint32_t)lt / (uint32_t)nv;
            rm = (uint32_t)lt - (uint32_t)q * (uint32_t)nv;
        } else {
            q = lt / nv;
            rm = lt - q * nv;
        }
    }
    t.i = q < (1LL << 31) ? (int)q : 0x7FFFFFFF;
    t.v = t.S.view_begin + (int)rm;
    t.live = nv > 0 && t.i < t.S.n;
    return t;
}

// Tile-culling count of the records with at most 32 candidate tiles (not above the
// load-balancing threshold), spread over the warp: the warp's (record, candidate tile) pairs are
// numbered by a scan of the lanes' candidate counts and tested 32 at a time, one per lane, with
// the owning record's mean, conic and opacity taken by shuffle. Each owner assembles its kept-
// tile mask (bit k = k-th candidate, row major) from the rounds' ballots and returns its count.
// The decisions are the ones the owner's own loop would take (same arithmetic, same inputs).
__device__ uint32_t count_spread(const PipeArgs& a, int vidx, const Rec& r, ushort4 rc, int n, uint32_t* mask_out)
{
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int first_me = incl - n;
    const int w = (int)rc.z - (int)rc.x;
    const float rw = rect_rcp(w);
    uint32_t mask = 0;
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        int own = 0;                                   // first lane whose inclusive count exceeds p
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(kFull, incl, own + st - 1) <= p) own += st;
        const int src = p < total ? own : 0;
        const int first = __shfl_sync(kFull, first_me, src);
        const int x0 = __shfl_sync(kFull, (int)rc.x, src), y0 = __shfl_sync(kFull, (int)rc.y, src);
        const int ws = __shfl_sync(kFull, w, src);
        const float rws = __shfl_sync(kFull, rw, src);
        const int vs = __shfl_sync(kFull, vidx, src);
        Rec rs;                                        // what the cull test reads: mean, conic, opacity
        rs.r0 = make_float4(__shfl_sync(kFull, r.r0.x, src), __shfl_sync(kFull, r.r0.y, src),
                            __shfl_sync(kFull, r.r0.z, src), __shfl_sync(kFull, r.r0.w, src));
        rs.r1 = make_float4(__shfl_sync(kFull, r.r1.x, src), __shfl_sync(kFull, r.r1.y, src),
                            __shfl_sync(kFull, r.r1.z, src), __shfl_sync(kFull, r.r1.w, src));
        rs.r2 = make_float4(__shfl_sync(kFull, r.r2.x, src), 0.f, 0.f, 0.f);
        rs.r3 = rs.r4 = rs.r5 = make_float4(0.f, 0.f, 0.f, 0.f);
        bool keep = false;
        if (p < total) {
            const int2 cl = rect_cell(p - first, ws, rws);
            const int tx = x0 + cl.x, ty = y0 + cl.y;
            const ViewDesc& Vs = a.views[vs];
            keep = tile_keep(a, rs, block_box(tx * kTile, ty * kTile, kTile, Vs.W, Vs.H));
            if (keep && a.partitioned) count_entry(a, (uint32_t)(Vs.tile_off + ty * Vs.tiles_x + tx));
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        const int lo = max(first_me, base), hi = min(first_me + n, base + 32);
        if (hi > lo) {
            const int wd = hi - lo;
            const unsigned bits = (bal >> (lo - base)) & (wd >= 32 ? 0xFFFFFFFFu : ((1u << wd) - 1u));
            mask |= bits << (lo - first_me);
        }
    }
    *mask_out = mask;
    return (uint32_t)__popc(mask);
}

__global__ void __launch_bounds__(128, STP_PRE_MIN_BLOCKS) k_preprocess(PipeArgs a)
{
    const RecThread th = rec_thread(a);
    const int i = th.i;
    const ViewDesc& V = a.views[th.v];
    Rec r;
    float vz = 0.f;
    ushort4 rc = make_ushort4(0, 0, 0, 0);
    bool vis = false;
    if (th.live) {
        GaussIn g;
        load_gauss(a, th.S, i, g);
        vis = make_record(a, V, g, i, r, vz, rc, th.v == th.S.view_begin) == kRecVisible;
    } else {
        r.r0 = r.r1 = r.r2 = r.r3 = r.r4 = r.r5 = make_float4(0.f, 0.f, 0.f, 0.f);
        vz = 0.f;
    }
    // every lane takes both calls (both hold warp-wide shuffles): the spread count for the
    // records of at most 32 candidates, the two-phase count (its big-rectangle path) for the rest
    uint32_t mask = 0, smask = 0, scnt = 0;
    bool spread = false;
    if (!(a.flags & 16)) {
        const int nc = vis ? ((int)rc.z - (int)rc.x) * ((int)rc.w - (int)rc.y) : 0;
        spread = vis && nc <= 32 && nc <= a.lb_threshold;
        scnt = count_spread(a, th.v, r, rc, spread ? nc : 0, &smask);
    }
    uint32_t cnt = tiles_pass<false>(a, V, th.v, vis && !spread, r, vz, rc, 0, 0, 0, &mask);
    if (spread) {
        cnt = scnt;
        mask = smask;
    }
    if (th.live) {
        const long long o = V.rec_off + i;
        a.keep_mask[o] = mask;
        float4* gp = a.geom + kRecFloat4 * o;
        gp[0] = r.r0; gp[1] = r.r1; gp[2] = r.r2; gp[3] = r.r3; gp[4] = r.r4; gp[5] = r.r5;
        a.view_z[o] = vz;
        a.rect[o] = rc;
        a.counts[o] = cnt;
    }
}

// Position of the n-th (0-based) set bit of m (m has more than n set bits).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n)
{
    int pos = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int c = __popc(m & ((1u << s) - 1u));
        if (c <= n) {
            n -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

// Partitioned placement of the kept tiles recorded in the lanes' masks, spread over the warp:
// the warp's (record, kept tile) pairs are numbered by an exclusive scan of the lanes' counts
// and taken 32 at a time, one pair per lane, so every lane works whatever its own record's
// tile count (a lane's own loop over its tiles leaves the lanes of small records idle). A lane
// reads the owning record again (an L1 hit: the owner just loaded it) and computes the key and
// placement exactly as the owner would; lanes of a round that place into the same tile take
// their slots with one cursor atomic. The order inside a tile's range is fixed later by the
// per-tile sort on (depth, id).
__device__ void place_spread(const PipeArgs& a, int vidx, ushort4 rc, uint32_t gid, float vz, uint32_t mask)
{
    const int lane = threadIdx.x & 31;
    const int n = __popc(mask);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int w = (int)rc.z - (int)rc.x;
    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        int own = 0;                                   // first lane whose inclusive count exceeds p
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(kFull, incl, own + st - 1) <= p) own += st;
        const int src = p < total ? own : 0;
        const int first = __shfl_sync(kFull, incl - n, src);
        const uint32_t ms = __shfl_sync(kFull, mask, src);
        const int x0 = __shfl_sync(kFull, (int)rc.x, src), y0 = __shfl_sync(kFull, (int)rc.y, src);
        const int ws = __shfl_sync(kFull, w, src);
        const uint32_t gs = __shfl_sync(kFull, gid, src);
        const int vs = __shfl_sync(kFull, vidx, src);
        const float zs = __shfl_sync(kFull, vz, src);
        uint32_t gt = 0xFFFFFFFFu - lane, dk = 0;
        if (p < total) {
            const int k = nth_set_bit(ms, p - first);
            const int tx = x0 + k % ws, ty = y0 + k / ws;
            const ViewDesc& Vs = a.views[vs];
            const Rec rs = load_rec(a.geom, Vs.rec_off + gs);
            gt = (uint32_t)(Vs.tile_off + ty * Vs.tiles_x + tx);
            dk = kept_depth_key(a, Vs, rs, zs, tx, ty);
        }
        // lanes placing into the same tile reserve their slots with one cursor atomic
        const unsigned peers = __match_any_sync(kFull, gt);
        const int leader = __ffs(peers) - 1;
        uint32_t sbase = 0;
        if (p < total && lane == leader) sbase = atomicAdd(&a.tile_cursor[gt], (uint32_t)__popc(peers));
        sbase = __shfl_sync(kFull, sbase, leader);
        if (p < total) {
            const uint32_t slot = sbase + __popc(peers & lanemask_lt());
            if (slot >= a.tile_counts[gt]) {
                atomicOr(&a.status->error_bits, 2u);
            } else {
                const unsigned long long pos = (unsigned long long)a.tile_offsets[gt] + slot;
                if (pos < a.capacity) a.dup_keys[pos] = ((unsigned long long)dk << 32) | gs;
            }
        }
    }
}

// Duplicate's mapping: thread t of the scene takes Gaussian t % n of view view_begin + t / n,
// so a warp holds consecutive Gaussians of one view: its record loads are coalesced, and
// neighbouring Gaussians (close in space in a trained or clustered scene) often share tiles,
// whose lanes then reserve their slots together (place_spread). Preprocess keeps the views of a
// Gaussian in neighbouring lanes, which read its SH coefficients once.
__device__ __forceinline__ RecThread rec_thread_view_major(const PipeArgs& a)
{
    RecThread t;
    const long long t0 = (long long)blockIdx.x * blockDim.x;
    t.S = a.scenes[scene_of_rec(a, t0)];
    const int nv = t.S.view_end - t.S.view_begin;
    const long long lt = t0 - t.S.rec_thread_off + threadIdx.x;
    const long long n = t.S.n;
    long long q = 0, rm = 0;
    if (n > 0) {
        if (lt < 0xFFFFFFFFll && n < 0xFFFFFFFFll) {
            q = (uint32_t)lt / (uint32_t)n;
            rm = (uint32_t)lt - (uint32_t)q * (uint32_t)n;
        } else {
            q = lt / n;
            rm = lt - q * n;
        }
    }
    t.i = (int)rm;
    t.v = t.S.view_begin + (int)(q < nv ? q : 0);
    t.live = n > 0 && q < nv;
    return t;
}

__global__ void __launch_bounds__(128, STP_DUP_MIN_BLOCKS) k_duplicate(PipeArgs a)
{
    const RecThread th = rec_thread_view_major(a);
    const int i = th.i;
    const ViewDesc& V = a.views[th.v];
    const long long o = V.rec_off + i;
    Rec r;
    ushort4 rc = make_ushort4(0, 0, 0, 0);
    uint32_t off = 0, want = 0, mask = 0;
    float vz = 0.f;
    if (th.live) {
        r = load_rec(a.geom, o);
        if (a.flags & 8) vz = a.view_z[o];
        rc = a.rect[o];
        off = a.partitioned ? 0u : a.offsets[o];
        want = a.counts[o];
        mask = a.keep_mask[o];
    } else {
        r.r0 = r.r1 = r.r2 = r.r3 = r.r4 = r.r5 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool has = th.live && want > 0;
    if (a.partitioned && !(a.flags & 16)) {
        // the records whose kept tiles Preprocess recorded in a mask (at most 32 candidates,
        // not above the load-balancing threshold) are placed by the whole warp together; the
        // rest keep the two-phase path, which then sees neither their tiles nor their mask
        const int nc = has ? ((int)rc.z - (int)rc.x) * ((int)rc.w - (int)rc.y) : 0;
        const bool spread = has && nc <= 32 && nc <= a.lb_threshold;
        place_spread(a, th.v, rc, (uint32_t)i, vz, spread ? mask : 0u);
        if (spread) {
            has = false;
            mask = 0u;
        }
    }
    const uint32_t got = tiles_pass<true>(a, V, th.v, has, r, vz, rc, off, want, (uint32_t)i, &mask);
    if (th.live && got != want && !a.partitioned) {
        // Preprocess and Duplicate disagree (cannot happen with the shared rounding of the
        // decision arithmetic; kept as the paper's safety net, appendix B.4): pad with
        // dummy keys that sort behind every tile.
        for (uint32_t k = got; k < want; k++) {
            const unsigned long long pos = (unsigned long long)off + k;
            if (pos < a.capacity) { a.dup_keys[pos] = ~0ull; a.dup_vals[pos] = (uint32_t)i; }
        }
        atomicOr(&a.status->error_bits, 2u);
        atomicAdd(&a.status->mismatched, 1u);
    }
}

// ---------------------------------------------------------------- scan of the counts
constexpr int kScanThreads = 256, kScanItems = 16, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x)
{
    const int lane = threadIdx.x & 31;
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// exclusive block scan of one value per thread; returns the prefix, *total the block sum
__device__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long* total)
{
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long wtot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned long long inc = warp_incl_scan(x);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long s = lane < nw ? ws[lane] : 0ull;
        const unsigned long long si = warp_incl_scan(s);
        if (lane < nw) ws[lane] = si - s;
        if (lane == nw - 1) wtot = si;
    }
    __syncthreads();
    const unsigned long long r = ws[warp] + inc - x;
    if (total) *total = wtot;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, long long m,
                                                              unsigned long long* partials)
{
    const long long base = (long long)blockIdx.x * kScanTile;
    unsigned long long s = 0;
    for (int k = 0; k < kScanItems; k++) {
        const long long idx = base + (long long)k * kScanThreads + threadIdx.x;
        if (idx < m) s += in[idx];
    }
    unsigned long long tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* partials, int np, Status* st)
{
    // one block: each thread scans a contiguous run, then a block scan of the run sums
    const int per = (np + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(np, b + per);
    unsigned long long s = 0;
    for (int k = b; k < e; k++) s += partials[k];
    unsigned long long tot;
    unsigned long long run = block_excl_scan(s, &tot);
    for (int k = b; k < e; k++) {
        const unsigned long long v = partials[k];
        partials[k] = run;
        run += v;
    }
    if (threadIdx.x == 0) {
        st->num_entries = tot;
        if (tot > st->capacity) atomicOr(&st->error_bits, 1u);
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ in, long long m,
                                                             const unsigned long long* partials, uint32_t* out)
{
    // blocked arrangement: thread t owns items [t*kScanItems, (t+1)*kScanItems) of the tile
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
    for (int k = 0; k < kScanItems; k++) {
        const long long idx = base + k;
        v[k] = idx < m ? in[idx] : 0u;
        s += v[k];
    }
    unsigned long long run = block_excl_scan(s, nullptr) + partials[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        const long long idx = base + k;
        if (idx < m) out[idx] = run > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)run;
        run += v[k];
    }
}

struct TablePack {
    ViewDesc v[kMaxViews];
    SceneDesc sc[kMaxScenes];
};

__global__ void k_tables_copy(TablePack pack, int nviews, ViewDesc* dv, int nscenes, SceneDesc* ds)
{
    const int k = threadIdx.x;
    if (k < nviews) dv[k] = pack.v[k];
    if (k < nscenes) ds[k] = pack.sc[k];
}

}  // namespace

size_t scan_partials_count(long long m) { return (size_t)((m + kScanTile - 1) / kScanTile) + 1; }

cudaError_t launch_tables_init(const ViewDesc* host_views, int nviews, ViewDesc* dev_views,
                               const SceneDesc* host_scenes, int nscenes, SceneDesc* dev_scenes, cudaStream_t s)
{
    static_assert(sizeof(TablePack) <= 32000, "kernel parameter block too large");
    TablePack pack;
    for (int k = 0; k < nviews && k < kMaxViews; k++) pack.v[k] = host_views[k];
    for (int k = 0; k < nscenes && k < kMaxScenes; k++) pack.sc[k] = host_scenes[k];
    k_tables_copy<<<1, kMaxViews, 0, s>>>(pack, nviews, dev_views, nscenes, dev_scenes);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const PipeArgs& a, cudaStream_t s)
{
    if (a.rec_threads == 0) return cudaSuccess;
    k_preprocess<<<(unsigned)(a.rec_threads / 128), 128, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

static cudaError_t scan_u32(const uint32_t* in, uint32_t* out, unsigned long long* partials, long long m,
                            Status* st, cudaStream_t s)
{
    const int nb = (int)((m + kScanTile - 1) / kScanTile);
    if (nb > 0) k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, m, partials);
    k_scan_partials<<<1, 1024, 0, s>>>(partials, nb, st);
    if (nb > 0) k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, m, partials, out);
    note_launches(nb > 0 ? 3 : 1);
    return cudaGetLastError();
}

cudaError_t launch_scan_counts(const PipeArgs& a, cudaStream_t s)
{
    return scan_u32(a.counts, a.offsets, a.scan_partials, a.m, a.status, s);
}

cudaError_t launch_scan_tiles(const PipeArgs& a, cudaStream_t s)
{
    return scan_u32(a.tile_counts, a.tile_offsets, a.tile_partials, (long long)a.total_tiles, a.status, s);
}

cudaError_t launch_duplicate(const PipeArgs& a, cudaStream_t s)
{
    if (a.rec_threads == 0) return cudaSuccess;
    k_duplicate<<<(unsigned)(a.rec_threads / 128), 128, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace stp
