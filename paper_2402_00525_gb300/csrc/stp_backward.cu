// stp_backward.cu -- adjoint of Preprocess.
//
// StopThePop (arXiv 2402.00525) Sec. 3.5 keeps 3DGS's gradient flow: the backward Render
// (stp_render.cu, BWD = true) accumulates per (view, Gaussian) the gradient of the conic and of
// the colour, the sums dGG (x - mean2) and dGG from which this kernel forms the gradients of
// the 2D mean (A times the first) and of the opacity (the second over the opacity), and --
// when a depth gradient is given -- those of the depth factors (m_k, c_k) of the record; this
// kernel chains them back to the inputs:
//   colour  -> SH coefficients, and through the view direction -> mean
//   opacity -> logit
//   conic   -> Sigma2 -> (Sigma, J) -> (scale, rotation) and the camera-space mean -> mean
//   mean2   -> camera-space mean -> mean
//   m_k,c_k -> rotation, clamped inverse scales (S^-1 clamp respected), camera-space mean
// One thread per Gaussian loops over the views of the launch and adds once into the caller's
// gradient arrays, so gradients of several views of one scene need no atomics.
#include <cuda_runtime.h>

#include "stp_common.cuh"
#include "stp_kernels.cuh"

namespace stp {

namespace {

// real SH basis (same polynomials as Preprocess) and its gradient w.r.t. (x, y, z)
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int K, float Y[16], float dY[16][3])
{
    const float k0 = 0.28209479177387814f, k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
#pragma unroll
    for (int j = 0; j < 16; j++) { Y[j] = 0.f; dY[j][0] = dY[j][1] = dY[j][2] = 0.f; }
    Y[0] = k0;
    if (K > 1) {
        Y[1] = -k1 * y; dY[1][1] = -k1;
        Y[2] = k1 * z;  dY[2][2] = k1;
        Y[3] = -k1 * x; dY[3][0] = -k1;
    }
    if (K > 4) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = k2a * x * y;  dY[4][0] = k2a * y; dY[4][1] = k2a * x;
        Y[5] = -k2a * y * z; dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
        Y[6] = k2b * (2.f * zz - xx - yy); dY[6][0] = -2.f * k2b * x; dY[6][1] = -2.f * k2b * y; dY[6][2] = 4.f * k2b * z;
        Y[7] = -k2a * x * z; dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
        Y[8] = k2c * (xx - yy); dY[8][0] = 2.f * k2c * x; dY[8][1] = -2.f * k2c * y;
        if (K > 9) {
            Y[9] = -k3a * y * (3.f * xx - yy);
            dY[9][0] = -6.f * k3a * x * y; dY[9][1] = -k3a * (3.f * xx - 3.f * yy);
            Y[10] = k3b * x * y * z;
            dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
            Y[11] = -k3c * y * (4.f * zz - xx - yy);
            dY[11][0] = 2.f * k3c * x * y; dY[11][1] = -k3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * k3c * y * z;
            Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            dY[12][0] = -6.f * k3d * x * z; dY[12][1] = -6.f * k3d * y * z; dY[12][2] = k3d * (6.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -k3c * x * (4.f * zz - xx - yy);
            dY[13][0] = -k3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * k3c * x * y; dY[13][2] = -8.f * k3c * x * z;
            Y[14] = k3e * z * (xx - yy);
            dY[14][0] = 2.f * k3e * x * z; dY[14][1] = -2.f * k3e * y * z; dY[14][2] = k3e * (xx - yy);
            Y[15] = -k3a * x * (xx - 3.f * yy);
            dY[15][0] = -k3a * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * k3a * x * y;
        }
    }
}

#ifndef STP_BWDPRE_MIN_BLOCKS
#define STP_BWDPRE_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(128, STP_BWDPRE_MIN_BLOCKS) k_backward_pre(PipeArgs a)
{
    const long long t0 = (long long)blockIdx.x * blockDim.x;
    const SceneDesc& S = a.scenes[scene_of(a, t0)];
    const int i = (int)(t0 - S.thread_off) + threadIdx.x;
    if (i >= S.n) return;
    const int K = S.sh_k;
    float mu[3] = {S.means[3 * i], S.means[3 * i + 1], S.means[3 * i + 2]};
    float q[4] = {S.quats[4 * i], S.quats[4 * i + 1], S.quats[4 * i + 2], S.quats[4 * i + 3]};
    const float ql = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float qw = q[0] / ql, qx = q[1] / ql, qy = q[2] / ql, qz = q[3] / ql;
    const float Rq[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                            {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                            {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    float sc[3], si[3];
    bool unclamped[3];
    for (int k = 0; k < 3; k++) {
        const float ls = S.log_scales[3 * i + k];
        sc[k] = expf(ls);
        const float s_inv = expf(-ls);
        unclamped[k] = s_inv < a.inv_scale_max;
        si[k] = fminf(s_inv, a.inv_scale_max);
    }
    float Sig[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            Sig[r][c] = 0.f;
            for (int k = 0; k < 3; k++) Sig[r][c] += Rq[r][k] * sc[k] * sc[k] * Rq[c][k];
        }
    const float opac = 1.f / (1.f + expf(-S.logits[i]));
    const float* shc = S.sh + (long long)i * K * 3;

    float dmu[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dlogit = 0.f;
    float dRq[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float dSig[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float dsi[3] = {0.f, 0.f, 0.f};
    float dsh[48];
#pragma unroll
    for (int k = 0; k < 48; k++) dsh[k] = 0.f;
    bool any = false;

    for (int v = S.view_begin; v < S.view_end; v++) {
        const ViewDesc& V = a.views[v];
        const long long ri = V.rec_off + i;
        const float4* gg = reinterpret_cast<const float4*>(a.grad_geom + ri * kGradStride);
        const float4* gd = reinterpret_cast<const float4*>(a.grad_depth + ri * kGradStride);
        float g[24];
        bool nz = false;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            // g[12..23], the depth-factor terms, exist only when the loss has a depth term
            const float4 q = k < 3 ? gg[k] : (a.d_depth ? gd[k - 3] : make_float4(0.f, 0.f, 0.f, 0.f));
            g[4 * k] = q.x;
            g[4 * k + 1] = q.y;
            g[4 * k + 2] = q.z;
            g[4 * k + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < 24; k++) nz |= g[k] != 0.f;
        // no pixel blended this (view, Gaussian): nothing to chain (this also skips the views
        // where it is invisible, whose scratch stays zero, without reading their records)
        if (!nz) continue;
        any = true;
        float p[3];
        for (int k = 0; k < 3; k++) p[k] = V.R[3 * k] * mu[0] + V.R[3 * k + 1] * mu[1] + V.R[3 * k + 2] * mu[2] + V.t[k];
        // colour -> SH and view direction
        float d[3] = {mu[0] - V.o[0], mu[1] - V.o[1], mu[2] - V.o[2]};
        const float dl = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float dir[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
        float Y[16], dY[16][3];
        sh_basis_grad(dir[0], dir[1], dir[2], K, Y, dY);
        float ddir[3] = {0.f, 0.f, 0.f};
        // static indices throughout (j < 16 unrolled, K tested inside), so the basis and the
        // accumulators stay in registers instead of local memory
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float raw = 0.5f;
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (j < K) raw += Y[j] * shc[3 * j + ch];
            const float dr = raw > 0.f ? g[6 + ch] : 0.f;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                if (j < K) {
                    dsh[3 * j + ch] += dr * Y[j];
                    const float cf = dr * shc[3 * j + ch];
                    ddir[0] += cf * dY[j][0];
                    ddir[1] += cf * dY[j][1];
                    ddir[2] += cf * dY[j][2];
                }
            }
        }
        const float dd = ddir[0] * dir[0] + ddir[1] * dir[1] + ddir[2] * dir[2];
        for (int k = 0; k < 3; k++) dmu[k] += (ddir[k] - dd * dir[k]) / dl;
        // opacity -> logit (the scratch holds sum dGG = opacity * dL/dopacity)
        dlogit += g[5] * (1.f - opac);
        // projection quantities
        const float iz = 1.f / p[2];
        const float ux = p[0] * iz, uy = p[1] * iz;
        const bool clx = ux < -V.limx || ux > V.limx, cly = uy < -V.limy || uy > V.limy;
        const float cx = fminf(V.limx, fmaxf(-V.limx, ux)), cy = fminf(V.limy, fmaxf(-V.limy, uy));
        const float J[2][3] = {{V.fx * iz, 0.f, -V.fx * cx * iz}, {0.f, V.fy * iz, -V.fy * cy * iz}};
        float T[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) T[r][c] = J[r][0] * V.R[c] + J[r][1] * V.R[3 + c] + J[r][2] * V.R[6 + c];
        float TS[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) TS[r][c] = T[r][0] * Sig[0][c] + T[r][1] * Sig[1][c] + T[r][2] * Sig[2][c];
        // Sigma2 = B B^T + dil I with B = T Rq diag(s); det from |b0 x b1|^2 (no cancellation)
        float B[2][3];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) B[r][k] = (T[r][0] * Rq[0][k] + T[r][1] * Rq[1][k] + T[r][2] * Rq[2][k]) * sc[k];
        const float n0 = B[0][0] * B[0][0] + B[0][1] * B[0][1] + B[0][2] * B[0][2];
        const float n1 = B[1][0] * B[1][0] + B[1][1] * B[1][1] + B[1][2] * B[1][2];
        const float cb = B[0][0] * B[1][0] + B[0][1] * B[1][1] + B[0][2] * B[1][2];
        const float x0 = B[0][1] * B[1][2] - B[0][2] * B[1][1];
        const float x1 = B[0][2] * B[1][0] - B[0][0] * B[1][2];
        const float x2 = B[0][0] * B[1][1] - B[0][1] * B[1][0];
        const float ca = n0 + a.dilation, cc = n1 + a.dilation;
        const float det = (x0 * x0 + x1 * x1 + x2 * x2) + a.dilation * (n0 + n1) + a.dilation * a.dilation;
        const float idet = 1.f / det;
        const float A[2][2] = {{cc * idet, -cb * idet}, {-cb * idet, ca * idet}};
        const float Ab[2][2] = {{g[2], 0.5f * g[3]}, {0.5f * g[3], g[4]}};
        float tmp[2][2], S2b[2][2];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) tmp[r][c] = A[r][0] * Ab[0][c] + A[r][1] * Ab[1][c];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) S2b[r][c] = -(tmp[r][0] * A[0][c] + tmp[r][1] * A[1][c]);
        // Sigma2 = T Sigma T^T + dil I
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++)
                for (int a2 = 0; a2 < 2; a2++)
                    for (int b2 = 0; b2 < 2; b2++) dSig[r][c] += T[a2][r] * S2b[a2][b2] * T[b2][c];
        float Tb[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++)
                Tb[r][c] = 2.f * (S2b[r][0] * TS[0][c] + S2b[r][1] * TS[1][c]);
        float Jb[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) Jb[r][c] = Tb[r][0] * V.R[3 * c] + Tb[r][1] * V.R[3 * c + 1] + Tb[r][2] * V.R[3 * c + 2];
        float dp[3] = {0.f, 0.f, 0.f};
        const float iz2 = iz * iz;
        dp[2] += Jb[0][0] * (-V.fx * iz2) + Jb[1][1] * (-V.fy * iz2);
        if (!clx) { dp[0] += Jb[0][2] * (-V.fx * iz2); dp[2] += Jb[0][2] * (2.f * V.fx * p[0] * iz2 * iz); }
        else dp[2] += Jb[0][2] * (V.fx * cx * iz2);
        if (!cly) { dp[1] += Jb[1][2] * (-V.fy * iz2); dp[2] += Jb[1][2] * (2.f * V.fy * p[1] * iz2 * iz); }
        else dp[2] += Jb[1][2] * (V.fy * cy * iz2);
        // mean2 (the scratch holds sum dGG (x - mean2); dL/dmean2 = A of it)
        const float gm0 = A[0][0] * g[0] + A[0][1] * g[1], gm1 = A[1][0] * g[0] + A[1][1] * g[1];
        dp[0] += gm0 * V.fx * iz;
        dp[1] += gm1 * V.fy * iz;
        dp[2] -= (gm0 * V.fx * p[0] + gm1 * V.fy * p[1]) * iz2;
        // depth factors: m_k = si_k R_c Rq e_k, c_k = m_k . p
        bool depth_nz = false;
        for (int k = 12; k < 24; k++) depth_nz |= g[k] != 0.f;
        if (depth_nz) {
            for (int k = 0; k < 3; k++) {
                float mk[3];   // camera-space axis k (unscaled)
                for (int r = 0; r < 3; r++) mk[r] = V.R[3 * r] * Rq[0][k] + V.R[3 * r + 1] * Rq[1][k] + V.R[3 * r + 2] * Rq[2][k];
                const float dc = g[21 + k];
                float dm[3];
                for (int r = 0; r < 3; r++) {
                    dp[r] += dc * si[k] * mk[r];
                    dm[r] = g[12 + 3 * k + r] + dc * p[r];
                }
                // world-space gradient of the unscaled axis and of the scale factor
                float gw[3];
                for (int r = 0; r < 3; r++) gw[r] = V.R[r] * dm[0] + V.R[3 + r] * dm[1] + V.R[6 + r] * dm[2];
                for (int r = 0; r < 3; r++) dRq[r][k] += si[k] * gw[r];
                dsi[k] += Rq[0][k] * gw[0] + Rq[1][k] * gw[1] + Rq[2][k] * gw[2];
            }
        }
        for (int k = 0; k < 3; k++) dmu[k] += V.R[k] * dp[0] + V.R[3 + k] * dp[1] + V.R[6 + k] * dp[2];
    }
    if (!any) return;
    // Sigma = M M^T with M = Rq diag(s): M bar = 2 Sigma bar M (Sigma bar symmetric)
    for (int r = 0; r < 3; r++)
        for (int k = 0; k < 3; k++) {
            float mb = 0.f;
            for (int j = 0; j < 3; j++) mb += 2.f * dSig[r][j] * Rq[j][k] * sc[k];
            dls[k] += mb * Rq[r][k] * sc[k];
            dRq[r][k] += mb * sc[k];
        }
    // clamped inverse scales si_k = min(exp(-log s_k), inv_scale_max)
    for (int k = 0; k < 3; k++)
        if (unclamped[k]) dls[k] += dsi[k] * (-si[k]);
    // rotation -> normalised quaternion -> raw quaternion
    const float(*R)[3] = dRq;
    float gq[4];
    gq[0] = 2.f * (-qz * R[0][1] + qy * R[0][2] + qz * R[1][0] - qx * R[1][2] - qy * R[2][0] + qx * R[2][1]);
    gq[1] = 2.f * (qy * R[0][1] + qz * R[0][2] + qy * R[1][0] - 2.f * qx * R[1][1] - qw * R[1][2] + qz * R[2][0] +
                   qw * R[2][1] - 2.f * qx * R[2][2]);
    gq[2] = 2.f * (-2.f * qy * R[0][0] + qx * R[0][1] + qw * R[0][2] + qx * R[1][0] + qz * R[1][2] - qw * R[2][0] +
                   qz * R[2][1] - 2.f * qy * R[2][2]);
    gq[3] = 2.f * (-2.f * qz * R[0][0] - qw * R[0][1] + qx * R[0][2] + qw * R[1][0] - 2.f * qz * R[1][1] +
                   qy * R[1][2] + qx * R[2][0] + qy * R[2][1]);
    const float dot = gq[0] * qw + gq[1] * qx + gq[2] * qy + gq[3] * qz;
    const float qn[4] = {qw, qx, qy, qz};
    for (int k = 0; k < 3; k++) {
        S.g_means[3 * i + k] += dmu[k];
        S.g_log_scales[3 * i + k] += dls[k];
    }
    for (int k = 0; k < 4; k++) S.g_quats[4 * i + k] += (gq[k] - dot * qn[k]) / ql;
    S.g_logits[i] += dlogit;
#pragma unroll
    for (int k = 0; k < 48; k++)
        if (k < 3 * K) S.g_sh[(long long)i * K * 3 + k] += dsh[k];
}

}  // namespace

cudaError_t launch_backward_preprocess(const PipeArgs& a, cudaStream_t s)
{
    if (a.threads == 0) return cudaSuccess;
    k_backward_pre<<<(unsigned)(a.threads / 128), 128, 0, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace stp
