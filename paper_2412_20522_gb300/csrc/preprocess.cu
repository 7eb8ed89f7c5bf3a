// Preprocess (forward and backward): mask sampling (Sec. 3.3) fused with the
// splat of every Gaussian (Sec. 3.1) for every view.
//
// One thread per Gaussian; the attributes are read once and reused for all
// views that see the Gaussian.  SH rows (the bulk of the bytes) are read only
// for Gaussians visible in some view, with 128-bit loads.
//
// Decisions (cull, radius, tile rectangle, depth key, mask) use a fixed
// sequence of correctly rounded FP32 operations (__fadd_rn, __fmul_rn, ...),
// never a contracted FMA, so that they reproduce bit for bit.  The 2D
// covariance is formed from its factor P = J W R S: Sigma_bar = P P^T + 0.3 I,
// det by Cauchy-Binet, eigenvalue gap as a sum of squares.  The splat is
// stored in eigen form (major axis u, h_k = -log2(e) / (2 lambda_k)), which
// stays accurate in FP32 for needle-shaped splats whose conic entries cancel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include "internal.cuh"

namespace mg {

constexpr int kPreThreads = 128;

template <int ROW>
struct StageStride { static constexpr int value = (ROW % 2 == 0) ? ROW + 1 : ROW; };

// ---------------------------------------------------------------------------
// Attribute storage: log-scales, quaternions, opacity logits and SH are read
// as FP32, BF16 or FP16 (ST) and unpacked to FP32 exactly; means and mask
// scores are always FP32.  Every computation is FP32 after the load.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

template <typename ST>
__device__ __forceinline__ float ld_attr(const void *base, int64_t i) {
    if constexpr (sizeof(ST) == 4) {
        return __ldg(reinterpret_cast<const float *>(base) + i);
    } else {
        const unsigned short u = __ldg(reinterpret_cast<const unsigned short *>(base) + i);
        ST v;
        memcpy(&v, &u, 2);
        return to_f32(v);
    }
}

template <typename ST>
__device__ __forceinline__ void ld_quat(const void *base, int64_t i, float q[4]) {
    if constexpr (sizeof(ST) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(base) + i);
        q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
    } else {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(base) + i);
        ST e[4];
        memcpy(e, &v, 8);
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = to_f32(e[k]);
    }
}

// Calls f(index, value) for the ROW values of SH row i, with 128-bit loads
// when rows are 16-byte multiples.
template <typename ST, int ROW, typename Fn>
__device__ __forceinline__ void for_sh_row(const void *sh, int64_t i, Fn &&f) {
    constexpr int PER = 16 / (int)sizeof(ST);
    if constexpr ((ROW * sizeof(ST)) % 16 == 0) {
        const uint4 *row = reinterpret_cast<const uint4 *>(sh) + i * (ROW / PER);
#pragma unroll
        for (int q = 0; q < ROW / PER; ++q) {
            const uint4 v = __ldg(row + q);
            ST e[PER];
            memcpy(e, &v, 16);
#pragma unroll
            for (int u = 0; u < PER; ++u) f(q * PER + u, to_f32(e[u]));
        }
    } else {
#pragma unroll
        for (int k = 0; k < ROW; ++k) f(k, ld_attr<ST>(sh, i * ROW + k));
    }
}

struct Splat32 {
    // decision-path quantities
    float tz, px, py, a, b, c, det, mid, disc, rf;
    int x0, x1, y0, y1;
    bool visible;
    // factor and pieces reused by the backward
    float P[2][3], M[3][3], R[3][3], T[2][3], s[3], qn[4], nrm, tzs, txc, tyc, ux, uy;
    bool clampx, clampy;
};

// The FP32 decision path for one Gaussian and one camera (every op rounded).
__device__ __forceinline__ void splat_fp32(const mg_camera &C, float limx, float limy, int tw,
                                           int th, int gx, int gy, float x, float y, float z,
                                           const float ls[3], const float q[4], Splat32 &S) {
    const float *V = C.viewmat;
    const float tx = ad(dot3(V[0], x, V[1], y, V[2], z), V[3]);
    const float ty = ad(dot3(V[4], x, V[5], y, V[6], z), V[7]);
    S.tz = ad(dot3(V[8], x, V[9], y, V[10], z), V[11]);
    const bool in_front = S.tz > C.near_plane;
    S.tzs = in_front ? S.tz : 1.0f;
    S.ux = dv(tx, S.tzs);
    S.uy = dv(ty, S.tzs);
    S.px = ad(ml(C.fx, S.ux), C.cx);
    S.py = ad(ml(C.fy, S.uy), C.cy);

    S.s[0] = exp32(ls[0]);
    S.s[1] = exp32(ls[1]);
    S.s[2] = exp32(ls[2]);
    float w = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float n2 = ad(ad(ad(ml(w, w), ml(qx, qx)), ml(qy, qy)), ml(qz, qz));
    const bool qvalid = n2 > 0.0f;
    S.nrm = __fsqrt_rn(qvalid ? n2 : 1.0f);
    w = dv(w, S.nrm); qx = dv(qx, S.nrm); qy = dv(qy, S.nrm); qz = dv(qz, S.nrm);
    S.qn[0] = w; S.qn[1] = qx; S.qn[2] = qy; S.qn[3] = qz;
    S.R[0][0] = sb(1.0f, ml(2.0f, ad(ml(qy, qy), ml(qz, qz))));
    S.R[0][1] = ml(2.0f, sb(ml(qx, qy), ml(w, qz)));
    S.R[0][2] = ml(2.0f, ad(ml(qx, qz), ml(w, qy)));
    S.R[1][0] = ml(2.0f, ad(ml(qx, qy), ml(w, qz)));
    S.R[1][1] = sb(1.0f, ml(2.0f, ad(ml(qx, qx), ml(qz, qz))));
    S.R[1][2] = ml(2.0f, sb(ml(qy, qz), ml(w, qx)));
    S.R[2][0] = ml(2.0f, sb(ml(qx, qz), ml(w, qy)));
    S.R[2][1] = ml(2.0f, ad(ml(qy, qz), ml(w, qx)));
    S.R[2][2] = sb(1.0f, ml(2.0f, ad(ml(qx, qx), ml(qy, qy))));
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) S.M[j][k] = ml(S.R[j][k], S.s[k]);

    const float cux = fminf(limx, fmaxf(-limx, S.ux));
    const float cuy = fminf(limy, fmaxf(-limy, S.uy));
    S.clampx = cux != S.ux;
    S.clampy = cuy != S.uy;
    S.txc = ml(cux, S.tzs);
    S.tyc = ml(cuy, S.tzs);
    const float tz2 = ml(S.tzs, S.tzs);
    const float j00 = dv(C.fx, S.tzs);
    const float j02 = -dv(ml(C.fx, S.txc), tz2);
    const float j11 = dv(C.fy, S.tzs);
    const float j12 = -dv(ml(C.fy, S.tyc), tz2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S.T[0][k] = ad(ml(j00, V[k]), ml(j02, V[8 + k]));
        S.T[1][k] = ad(ml(j11, V[4 + k]), ml(j12, V[8 + k]));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            S.P[i][k] = dot3(S.T[i][0], S.M[0][k], S.T[i][1], S.M[1][k], S.T[i][2], S.M[2][k]);
    const float n0 = dot3(S.P[0][0], S.P[0][0], S.P[0][1], S.P[0][1], S.P[0][2], S.P[0][2]);
    const float n1 = dot3(S.P[1][0], S.P[1][0], S.P[1][1], S.P[1][1], S.P[1][2], S.P[1][2]);
    S.a = ad(n0, kLowpass);
    S.b = dot3(S.P[0][0], S.P[1][0], S.P[0][1], S.P[1][1], S.P[0][2], S.P[1][2]);
    S.c = ad(n1, kLowpass);
    const float m01 = sb(ml(S.P[0][0], S.P[1][1]), ml(S.P[0][1], S.P[1][0]));
    const float m02 = sb(ml(S.P[0][0], S.P[1][2]), ml(S.P[0][2], S.P[1][0]));
    const float m12 = sb(ml(S.P[0][1], S.P[1][2]), ml(S.P[0][2], S.P[1][1]));
    S.det = ad(ad(dot3(m01, m01, m02, m02, m12, m12), ml(kLowpass, ad(n0, n1))),
               ml(kLowpass, kLowpass));
    S.mid = ml(0.5f, ad(S.a, S.c));
    const float hd = ml(0.5f, sb(S.a, S.c));
    S.disc = ad(ml(hd, hd), ml(S.b, S.b));
    const float lam = ad(S.mid, __fsqrt_rn(fmaxf(0.1f, S.disc)));
    float rf = ceilf(ml(3.0f, __fsqrt_rn(lam)));
    const bool ok = in_front && qvalid && (S.det > 0.0f) && isfinite(S.px) && isfinite(S.py) &&
                    isfinite(rf);
    rf = ok ? fminf(rf, 1e9f) : 0.0f;   // radius capped at 1e9 px (exact in float and int)
    S.rf = rf;
    S.visible = ok && rf > 0.0f &&
                tile_rect(S.px, S.py, rf, tw, th, gx, gy, S.x0, S.x1, S.y0, S.y1);
}

// The pieces of the splat the backward differentiates through (P = J W R S,
// its factors, the normalised quaternion, t_z, and Sigma_bar's a, b, c, det,
// mid, disc), in ordinary contracted FP32 -- the gradient needs no bit-exact
// rounding.  The one decision on this chain, whether the Jacobian's point was
// clamped, is taken exactly as in the forward (the correctly rounded ux, uy
// against the same limits), so both use the same branch.
__device__ __forceinline__ void splat_grad_pieces(const mg_camera &C, float limx, float limy,
                                                  float x, float y, float z, const float ls[3],
                                                  const float q[4], Splat32 &S) {
    const float *V = C.viewmat;
    const float tx = ad(dot3(V[0], x, V[1], y, V[2], z), V[3]);
    const float ty = ad(dot3(V[4], x, V[5], y, V[6], z), V[7]);
    S.tz = ad(dot3(V[8], x, V[9], y, V[10], z), V[11]);
    S.tzs = S.tz > C.near_plane ? S.tz : 1.0f;
    S.ux = dv(tx, S.tzs);
    S.uy = dv(ty, S.tzs);
    const float cux = fminf(limx, fmaxf(-limx, S.ux));
    const float cuy = fminf(limy, fmaxf(-limy, S.uy));
    S.clampx = cux != S.ux;
    S.clampy = cuy != S.uy;

    S.s[0] = __expf(ls[0]);
    S.s[1] = __expf(ls[1]);
    S.s[2] = __expf(ls[2]);
    const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    const float inr = rsqrtf(n2 > 0.0f ? n2 : 1.0f);
    S.nrm = __fdividef(1.0f, inr);
    const float w = q[0] * inr, qx = q[1] * inr, qy = q[2] * inr, qz = q[3] * inr;
    S.qn[0] = w; S.qn[1] = qx; S.qn[2] = qy; S.qn[3] = qz;
    S.R[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    S.R[0][1] = 2.0f * (qx * qy - w * qz);
    S.R[0][2] = 2.0f * (qx * qz + w * qy);
    S.R[1][0] = 2.0f * (qx * qy + w * qz);
    S.R[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
    S.R[1][2] = 2.0f * (qy * qz - w * qx);
    S.R[2][0] = 2.0f * (qx * qz - w * qy);
    S.R[2][1] = 2.0f * (qy * qz + w * qx);
    S.R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) S.M[j][k] = S.R[j][k] * S.s[k];

    S.txc = cux * S.tzs;
    S.tyc = cuy * S.tzs;
    const float itz = __fdividef(1.0f, S.tzs);
    const float j00 = C.fx * itz, j11 = C.fy * itz;
    const float j02 = -C.fx * S.txc * itz * itz, j12 = -C.fy * S.tyc * itz * itz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S.T[0][k] = j00 * V[k] + j02 * V[8 + k];
        S.T[1][k] = j11 * V[4 + k] + j12 * V[8 + k];
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            S.P[i][k] = S.T[i][0] * S.M[0][k] + S.T[i][1] * S.M[1][k] + S.T[i][2] * S.M[2][k];
    const float n0 = S.P[0][0] * S.P[0][0] + S.P[0][1] * S.P[0][1] + S.P[0][2] * S.P[0][2];
    const float n1 = S.P[1][0] * S.P[1][0] + S.P[1][1] * S.P[1][1] + S.P[1][2] * S.P[1][2];
    S.a = n0 + kLowpass;
    S.b = S.P[0][0] * S.P[1][0] + S.P[0][1] * S.P[1][1] + S.P[0][2] * S.P[1][2];
    S.c = n1 + kLowpass;
    const float m01 = S.P[0][0] * S.P[1][1] - S.P[0][1] * S.P[1][0];
    const float m02 = S.P[0][0] * S.P[1][2] - S.P[0][2] * S.P[1][0];
    const float m12 = S.P[0][1] * S.P[1][2] - S.P[0][2] * S.P[1][1];
    S.det = m01 * m01 + m02 * m02 + m12 * m12 + kLowpass * (n0 + n1) + kLowpass * kLowpass;
    S.mid = 0.5f * (S.a + S.c);
    const float hd = 0.5f * (S.a - S.c);
    S.disc = hd * hd + S.b * S.b;
}

// Major axis (cos, sin) and the two eigenvalues of [[a, b], [b, c]] from the
// Cauchy-Binet determinant; continuous, so ordinary fast arithmetic.
__device__ __forceinline__ float sqrt_fast(float x) {   // x >= 0; a few ulp
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

__device__ __forceinline__ void eigen2(const Splat32 &S, float &uxo, float &uyo, float &lam1,
                                       float &lam2) {
    const float sq = sqrt_fast(S.disc);
    lam1 = S.mid + sq;
    lam2 = __fdividef(S.det, lam1);
    if (sq > 0.0f) {
        const float isq = __fdividef(1.0f, sq);
        const float c2 = 0.5f * (S.a - S.c) * isq, s2 = S.b * isq;
        if (c2 >= 0.0f) {
            uxo = sqrt_fast(0.5f * (1.0f + c2));
            uyo = __fdividef(s2, 2.0f * uxo);
        } else {
            uyo = sqrt_fast(0.5f * (1.0f - c2));
            uxo = __fdividef(s2, 2.0f * uyo);
        }
    } else {
        uxo = 1.0f;
        uyo = 0.0f;
    }
}

// sum_k Y_k sh[i][k][ch] for the three channels, streaming the Gaussian's SH
// row from global memory.
template <int DEG, typename ST>
__device__ __forceinline__ void sh_colour(const void *sh, int64_t i, const float *Y,
                                          float acc[3]) {
    constexpr int ROW = 3 * (DEG + 1) * (DEG + 1);
    for_sh_row<ST, ROW>(sh, i, [&](int e, float v) { acc[e % 3] = fmaf(Y[e / 3], v, acc[e % 3]); });
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The SH rows are read only for Gaussians that are visible in a view, one
// row per lane with 128-bit loads (no row of an invisible Gaussian is read).
// Eight CTAs per SM: the 64 registers this leaves hold the kernel without
// spills for FP32 storage (8 bytes spill with 16-bit storage), and the
// memory latency it waits on wants the extra warps.
template <int DEG, typename ST>
__global__ void __launch_bounds__(kPreThreads, 8)
preprocess_kernel(ViewTable vt, mg_gaussians g, mg_raster_cfg cfg, mg_splats out) {
    grid_dependency_wait();
    const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
    const bool active = i < g.n;

    // the Gaussian's attributes first: their loads travel during the mask
    // sample's arithmetic (lanes past the end read Gaussian 0, unused)
    const int64_t ia = active ? i : 0;
    const float *means = reinterpret_cast<const float *>(g.means);
    const float x = __ldg(means + 3 * ia), y = __ldg(means + 3 * ia + 1),
                z = __ldg(means + 3 * ia + 2);
    const float ls[3] = {ld_attr<ST>(g.log_scales, 3 * ia),
                         ld_attr<ST>(g.log_scales, 3 * ia + 1),
                         ld_attr<ST>(g.log_scales, 3 * ia + 2)};
    float q[4];
    ld_quat<ST>(g.quats, ia, q);
    const float ol = ld_attr<ST>(g.opacity_logit, ia);

    // --- mask (Sec. 3.3): Gumbel-max over the two existence scores, or the
    // threshold of the straight-through ablation (Sec. 4.3)
    float Mf = active ? 1.0f : 0.0f;
    if (active) {
        if (cfg.mask_mode == MG_MASK_GUMBEL) {
            const uint64_t it = cfg.iteration + (cfg.iteration_dev ? *cfg.iteration_dev : 0ull);
            const uint4 x = gumbel_counter(i, it, 0u, cfg.seed);
            const float2 l = __ldg(reinterpret_cast<const float2 *>(g.mask_logits) + i);  // FP32
            const float d = gumbel_margin(l, x);
            Mf = d >= 0.0f ? 1.0f : 0.0f;
            out.mask_soft[i] = __fdividef(1.0f, 1.0f + __expf(__fdividef(-d, cfg.tau)));
        } else if (cfg.mask_mode == MG_MASK_STE) {
            const float2 l = __ldg(reinterpret_cast<const float2 *>(g.mask_logits) + i);
            const float d = sb(l.x, l.y);
            Mf = d > cfg.ste_logit ? 1.0f : 0.0f;
            out.mask_soft[i] = __fdividef(1.0f, 1.0f + __expf(-d));
        } else {
            if (cfg.mask_mode == MG_MASK_GIVEN) Mf = cfg.given_mask[i] ? 1.0f : 0.0f;
            out.mask_soft[i] = 1.0f;
        }
        out.mask[i] = Mf != 0.0f;
    }
    // sum of M over each view's range (for L_m, Eq. 7): one atomic per warp
    if (out.mask_count != nullptr) {
        for (int v = 0; v < vt.n_views; ++v) {
            const bool in = active && i >= vt.g_off[v] && i < vt.g_off[v] + vt.g_cnt[v];
            const unsigned b = __ballot_sync(0xffffffffu, in && Mf != 0.0f);
            if ((threadIdx.x & 31) == 0 && b != 0u) atomicAdd(out.mask_count + v, (uint32_t)__popc(b));
        }
    }
    if (!active) return;

    const float op = __fdividef(1.0f, 1.0f + __expf(-ol));

    bool sh_requested = false;
    for (int v = 0; v < vt.n_views; ++v) {
        if (i < vt.g_off[v] || i >= vt.g_off[v] + vt.g_cnt[v]) continue;
        const int64_t r = vt.rec_off[v] + (i - vt.g_off[v]);
        const mg_camera &C = vt.cam[v];
        Splat32 S;
        splat_fp32(C, vt.limx[v], vt.limy[v], vt.tile_w, vt.tile_h, vt.gx[v], vt.gy[v], x, y, z,
                   ls, q, S);
        if (!S.visible) {
            out.tiles_touched[r] = 0u;
            out.radius[r] = 0;
            out.clamp[r] = 0;
            if (out.depth_key != nullptr) out.depth_key[r] = 0xFFFFFFFFu;
            continue;
        }
        if (!sh_requested) {
            // the SH row towards L2 now: the binning and eigen work below
            // runs while it travels
            constexpr int RB = 3 * (DEG + 1) * (DEG + 1) * (int)sizeof(ST);
            const char *sp0 = reinterpret_cast<const char *>(g.sh) + i * RB;
#pragma unroll
            for (int o = 0; o < RB; o += 128) prefetch_l2(sp0 + o);
            prefetch_l2(sp0 + RB - 1);
            sh_requested = true;
        }
        // the binning's candidate tiles: the whole 3-sigma rectangle, or (tile
        // filter) its tiles that the filter can keep
        int x0 = S.x0, x1 = S.x1, y0 = S.y0, y1 = S.y1;
        const float tdet = ml(kBinThreshold, S.det);
        const bool binned = cfg.bin_mode != MG_BIN_FILTERED ||
                            candidate_rect(S.px, S.py, S.a, S.b, S.c, tdet, vt.tile_w,
                                           vt.tile_h, x0, x1, y0, y1);
        out.tiles_touched[r] = binned ? (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1)) : 0u;
        // depth-order key: the float bits of tz > 0 order like the values
        if (out.depth_key != nullptr)
            out.depth_key[r] = binned ? __float_as_uint(S.tz) : 0xFFFFFFFFu;
        // binning record: tile-filter inputs (decision path) and the rectangle
        float4 *br = reinterpret_cast<float4 *>(out.bin_record) + 3 * r;
        br[0] = make_float4(S.px, S.py, S.a, S.b);
        br[1] = make_float4(S.c, tdet, dv(S.b, S.a), dv(S.b, S.c));
        reinterpret_cast<uint4 *>(br)[2] =
            make_uint4((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)(x1 - x0 + 1),
                       (uint32_t)(vt.tile_off[v] + (int64_t)y0 * vt.gx[v] + x0),
                       (uint32_t)vt.gx[v]);
        out.radius[r] = (int32_t)S.rf;
        float ux, uy, l1, l2;
        eigen2(S, ux, uy, l1, l2);
        // view-dependent colour: SH at dir = normalise(p - cam_pos)
        float dx = x - C.cam_pos[0], dy = y - C.cam_pos[1], dz = z - C.cam_pos[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis(DEG, dx, dy, dz, Y);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        sh_colour<DEG, ST>(g.sh, i, Y, rgb);
        uint8_t cl = 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (rgb[ch] < 0.0f) {
                cl |= (uint8_t)(1u << ch);
                rgb[ch] = 0.0f;
            }
        }
        out.clamp[r] = cl;
        float4 *rec = reinterpret_cast<float4 *>(out.record) + 3 * r;
        rec[0] = make_float4(S.px, S.py, ux, uy);
        // mask in the sign of the opacity; e_min just below log2(1/(255 o)) (a
        // splat with o under the floor never reaches it: e_min = 1 > any e)
        // (mask x opacity ablation: the opacity is M o, +0 for a masked splat)
        const bool by_opacity = cfg.mask_apply == MG_APPLY_OPACITY;
        const float o_eff = by_opacity ? Mf * op : op;
        const float e_min = o_eff >= kAlphaMin ? __log2f(__fdividef(kAlphaMin, o_eff)) - 1e-3f
                                               : 1.0f;
        rec[1] = make_float4(__fdividef(-0.5f * kLog2e, l1), __fdividef(-0.5f * kLog2e, l2),
                             (by_opacity || Mf != 0.0f) ? o_eff : -op, e_min);
        rec[2] = make_float4(rgb[0], rgb[1], rgb[2], S.tz);
    }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Backward of the covariance chain: conic Q = Sigma_bar^-1 -> Sigma_bar =
// P P^T + 0.3 I -> P = T M (T = J W, M = R diag(s)) -> s = exp(log s),
// R(q / |q|), J(t).  FP32 throughout except the 2x2 inversion's backward
// dSigma = -Q Ghat Q (Ghat = dL/dQ) for ill-conditioned splats
// (lambda_1 / lambda_2 above kFp64Condition): there Q's two eigenvalues are
// far apart and the FP32 products leave dSigma's major-axis component as
// rounding noise (about eps lambda_1^2 / lambda_2^2 relative), which P then
// carries into the long axis's scale and rotation gradients.  Q and dSigma
// are then formed in FP64 from the FP32 a, b, c and Cauchy-Binet determinant
// (an emulation of this chain on the benchmark view against the FP64 oracle:
// relative L2 1.0e-3 / 2.0e-3 on dL/dlog_scales / dL/dquats in FP32 alone,
// 3.5e-6 / 6.7e-5 with this step in FP64 above the condition 100).
// ---------------------------------------------------------------------------
constexpr float kFp64Condition = 100.0f;

struct CovState {
    float P[2][3], M[3][3], R[3][3], T[2][3], s[3], qn[4], nrm, tzs, txc, tyc;
};

__device__ __forceinline__ void cov_state(const Splat32 &S, CovState &F) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F.P[i][k] = S.P[i][k];
            F.T[i][k] = S.T[i][k];
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        F.s[j] = S.s[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F.M[j][k] = S.M[j][k];
            F.R[j][k] = S.R[j][k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) F.qn[k] = S.qn[k];
    F.nrm = S.nrm;
    F.tzs = S.tzs;
    F.txc = S.txc;
    F.tyc = S.tyc;
}

// dSigma = -Q Ghat Q, Ghat = [[G_a, G_b / 2], [G_b / 2, G_c]] (the conic's
// off-diagonal entry appears once in the quadratic form), in the type F.
template <typename F>
__device__ __forceinline__ void inverse_backward(F Q00, F Q01, F Q11, float dca, float dcb,
                                                 float dcc, float &dS00, float &dS01,
                                                 float &dS11) {
    const F G00 = dca, G01 = F(0.5) * (F)dcb, G11 = dcc;
    const F A00 = Q00 * G00 + Q01 * G01, A01 = Q00 * G01 + Q01 * G11;
    const F A10 = Q01 * G00 + Q11 * G01, A11 = Q01 * G01 + Q11 * G11;
    dS00 = (float)(-(A00 * Q00 + A01 * Q01));
    dS01 = (float)(-(A00 * Q01 + A01 * Q11));
    dS11 = (float)(-(A10 * Q01 + A11 * Q11));
}

// The inversion's backward for one splat: FP32 from the eigen form when it is
// well conditioned, FP64 from (a, b, c, det) when it is not.
__device__ __forceinline__ void conic_backward(const Splat32 &S, float ux, float uy, float l1,
                                               float l2, float dca, float dcb, float dcc,
                                               float &dS00, float &dS01, float &dS11) {
    if (l1 > kFp64Condition * l2) {
        const double id = 1.0 / (double)S.det;
        inverse_backward<double>((double)S.c * id, -(double)S.b * id, (double)S.a * id, dca, dcb,
                                 dcc, dS00, dS01, dS11);
    } else {
        const float w1 = __fdividef(1.0f, l1), w2 = __fdividef(1.0f, l2);
        inverse_backward<float>(w1 * ux * ux + w2 * uy * uy, (w1 - w2) * ux * uy,
                                w1 * uy * uy + w2 * ux * ux, dca, dcb, dcc, dS00, dS01, dS11);
    }
}

__device__ __forceinline__ void cov_backward(const CovState &S, const mg_camera &C, bool clampx,
                                             bool clampy, float dS00, float dS01, float dS11,
                                             float d_ls[3], float d_q[4], float dL_dt[3]) {
    const float *V = C.viewmat;
    // Sigma_bar = P P^T + 0.3 I  =>  dP = 2 dSigma P
    float dP[2][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dP[0][k] = 2.0f * (dS00 * S.P[0][k] + dS01 * S.P[1][k]);
        dP[1][k] = 2.0f * (dS01 * S.P[0][k] + dS11 * S.P[1][k]);
    }
    // P = T M:  dT = dP M^T, dM = T^T dP
    float dT[2][3], dM[3][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dT[r][j] = dP[r][0] * S.M[j][0] + dP[r][1] * S.M[j][1] + dP[r][2] * S.M[j][2];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) dM[j][k] = S.T[0][j] * dP[0][k] + S.T[1][j] * dP[1][k];
    // M = R diag(s), s = exp(log s)
    float dR[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) dR[j][k] = dM[j][k] * S.s[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ds = dM[0][k] * S.R[0][k] + dM[1][k] * S.R[1][k] + dM[2][k] * S.R[2][k];
        d_ls[k] += ds * S.s[k];
    }
    // R(q_hat), then q_hat = q / |q|
    {
        const float w = S.qn[0], qx = S.qn[1], qy = S.qn[2], qz = S.qn[3];
        const float gw = 2.0f * (qz * (dR[1][0] - dR[0][1]) + qy * (dR[0][2] - dR[2][0]) +
                                 qx * (dR[2][1] - dR[1][2]));
        const float gx = 2.0f * (qy * (dR[1][0] + dR[0][1]) + qz * (dR[2][0] + dR[0][2]) +
                                 w * (dR[2][1] - dR[1][2])) - 4.0f * qx * (dR[1][1] + dR[2][2]);
        const float gy = 2.0f * (qx * (dR[1][0] + dR[0][1]) + w * (dR[0][2] - dR[2][0]) +
                                 qz * (dR[1][2] + dR[2][1])) - 4.0f * qy * (dR[0][0] + dR[2][2]);
        const float gz = 2.0f * (w * (dR[1][0] - dR[0][1]) + qx * (dR[2][0] + dR[0][2]) +
                                 qy * (dR[1][2] + dR[2][1])) - 4.0f * qz * (dR[0][0] + dR[1][1]);
        const float dot = gw * w + gx * qx + gy * qy + gz * qz;
        const float in = __fdividef(1.0f, S.nrm);
        d_q[0] += (gw - dot * w) * in;
        d_q[1] += (gx - dot * qx) * in;
        d_q[2] += (gy - dot * qy) * in;
        d_q[3] += (gz - dot * qz) * in;
    }
    // T = J W:  dJ = dT W^T ; J = [[fx/tz, 0, -fx txc/tz^2], [0, fy/tz, -fy tyc/tz^2]]
    float dJ00 = 0.0f, dJ02 = 0.0f, dJ11 = 0.0f, dJ12 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dJ00 += dT[0][k] * V[k];
        dJ02 += dT[0][k] * V[8 + k];
        dJ11 += dT[1][k] * V[4 + k];
        dJ12 += dT[1][k] * V[8 + k];
    }
    const float fx = C.fx, fy = C.fy;
    const float itz = __fdividef(1.0f, S.tzs), itz2 = itz * itz, itz3 = itz2 * itz;
    // d J02 / d tz: 2 fx txc / tz^3 unclamped, fx txc / tz^3 clamped
    dL_dt[2] += -dJ00 * fx * itz2 - dJ11 * fy * itz2 +
                dJ02 * fx * S.txc * itz3 * (clampx ? 1.0f : 2.0f) +
                dJ12 * fy * S.tyc * itz3 * (clampy ? 1.0f : 2.0f);
    if (!clampx) dL_dt[0] += -dJ02 * fx * itz2;
    if (!clampy) dL_dt[1] += -dJ12 * fy * itz2;
}

// dL/dsh accumulates over views in a per-warp shared-memory tile (one row
// per lane, odd row stride) and leaves with coalesced 128-bit stores; SH rows
// are read only for Gaussians visible in some view.  Five CTAs per SM: the
// 96 registers this leaves cost a few bytes of spills, and the latency-bound
// kernel gains more from the fifth CTA's warps.
template <int DEG, typename ST>
__global__ void __launch_bounds__(kPreThreads, 5)
preprocess_backward_kernel(ViewTable vt, mg_gaussians g, mg_raster_cfg cfg, mg_splats sp,
                           const float *__restrict__ grad2d, mg_param_grads out) {
    grid_dependency_wait();
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int ROW = 3 * K;
    constexpr int S_ = StageStride<ROW>::value;
    __shared__ float sm_dsh[kPreThreads / 32][32 * S_];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw0 = ((int64_t)blockIdx.x * kPreThreads) + warp * 32;
    if (gw0 >= g.n) return;
    const int nrows = (int)(g.n - gw0 < 32 ? g.n - gw0 : 32);
    float *dsh = sm_dsh[warp];
    const int64_t i = gw0 + lane;
    float *drow = dsh + lane * S_;
    if (lane < nrows) {
        // the Gaussian's attributes first: their loads travel while the
        // visibility is read and the prefetches go out
        const float *means = reinterpret_cast<const float *>(g.means);
        const float x = __ldg(means + 3 * i), y = __ldg(means + 3 * i + 1),
                    z = __ldg(means + 3 * i + 2);
        const float ls[3] = {ld_attr<ST>(g.log_scales, 3 * i), ld_attr<ST>(g.log_scales, 3 * i + 1),
                             ld_attr<ST>(g.log_scales, 3 * i + 2)};
        float q[4];
        ld_quat<ST>(g.quats, i, q);
        const float op_logit = ld_attr<ST>(g.opacity_logit, i);
        // a Gaussian visible in some view: start its 2D gradients, clamp bits
        // and SH row towards L2 before the dependent work that reads them
        bool vis = false;
        for (int v = 0; v < vt.n_views; ++v) {
            if (i < vt.g_off[v] || i >= vt.g_off[v] + vt.g_cnt[v]) continue;
            const int64_t r = vt.rec_off[v] + (i - vt.g_off[v]);
            if (sp.radius[r] == 0) continue;
            vis = true;
            const char *gp = reinterpret_cast<const char *>(grad2d + 12 * r);
            prefetch_l2(gp);
            prefetch_l2(gp + 47);
            prefetch_l2(sp.clamp + r);
        }
        if (vis) {
            constexpr int RB = ROW * (int)sizeof(ST);
            const char *sp0 = reinterpret_cast<const char *>(g.sh) + i * RB;
#pragma unroll
            for (int o = 0; o < RB; o += 128) prefetch_l2(sp0 + o);
            prefetch_l2(sp0 + RB - 1);
        }
        // the lane's own staging row (bank 17 l + c mod 32: no conflicts)
#pragma unroll
        for (int f = 0; f < ROW; ++f) drow[f] = 0.0f;
        const float op = __fdividef(1.0f, 1.0f + __expf(-op_logit));

        float d_mean[3] = {0, 0, 0}, d_ls[3] = {0, 0, 0}, d_q[4] = {0, 0, 0, 0}, d_op = 0.0f,
              d_M = 0.0f;
        for (int v = 0; v < vt.n_views; ++v) {
            if (i < vt.g_off[v] || i >= vt.g_off[v] + vt.g_cnt[v]) continue;
            const int64_t r = vt.rec_off[v] + (i - vt.g_off[v]);
            if (sp.radius[r] == 0) continue;
            const float4 *G4 = reinterpret_cast<const float4 *>(grad2d) + 3 * r;
            const float4 g0 = G4[0], g1 = G4[1], g2 = G4[2];
            // g0 = (dmx, dmy, dca, dcb), g1 = (dcc, dop, dr, dg), g2 = (db, dM, -, -)
            d_M += g2.y;
            d_op += g1.y;
            const mg_camera &C = vt.cam[v];
            Splat32 S;
            splat_grad_pieces(C, vt.limx[v], vt.limy[v], x, y, z, ls, q, S);
            const float *V = C.viewmat;
            float dL_dt[3] = {0, 0, 0};   // camera-space centre

            // ---- colour: rgb_c = max(0, sum_k Y_k sh_kc + 0.5)
            {
                const float vx = x - C.cam_pos[0], vy = y - C.cam_pos[1], vz = z - C.cam_pos[2];
                const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
                const float dx = vx * inv, dy = vy * inv, dz = vz * inv;
                float Y[16];
                sh_basis(DEG, dx, dy, dz, Y);
                const uint8_t cl = sp.clamp[r];
                const float grgb[3] = {(cl & 1) ? 0.0f : g1.z, (cl & 2) ? 0.0f : g1.w,
                                       (cl & 4) ? 0.0f : g2.x};
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) drow[3 * k + ch] = fmaf(Y[k], grgb[ch], drow[3 * k + ch]);
                if (DEG > 0) {
                    // t_k = sum_c grgb_c sh_kc, streamed from the SH row
                    float t[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) t[k] = 0.0f;
                    for_sh_row<ST, ROW>(g.sh, i, [&](int e, float v) {
                        t[e / 3] = fmaf(grgb[e % 3], v, t[e / 3]);
                    });
                    float Yx[16], Yy[16], Yz[16];
                    sh_basis_grad(DEG, dx, dy, dz, Yx, Yy, Yz);
                    float gd[3] = {0, 0, 0};
#pragma unroll
                    for (int k = 1; k < K; ++k) {
                        gd[0] = fmaf(t[k], Yx[k], gd[0]);
                        gd[1] = fmaf(t[k], Yy[k], gd[1]);
                        gd[2] = fmaf(t[k], Yz[k], gd[2]);
                    }
                    // through dir = v / |v|
                    const float dot = gd[0] * dx + gd[1] * dy + gd[2] * dz;
                    d_mean[0] += (gd[0] - dot * dx) * inv;
                    d_mean[1] += (gd[1] - dot * dy) * inv;
                    d_mean[2] += (gd[2] - dot * dz) * inv;
                }
            }

            // ---- 2D mean: px = fx tx/tz + cx, py = fy ty/tz + cy
            {
                const float itz = __fdividef(1.0f, S.tzs);
                dL_dt[0] += g0.x * C.fx * itz;
                dL_dt[1] += g0.y * C.fy * itz;
                dL_dt[2] -= (g0.x * C.fx * S.ux + g0.y * C.fy * S.uy) * itz;
            }

            // ---- conic -> Sigma_bar -> P = J W R S -> scales, rotation, J
            float ux, uy, l1, l2;
            eigen2(S, ux, uy, l1, l2);
            float dS00, dS01, dS11;
            conic_backward(S, ux, uy, l1, l2, g0.z, g0.w, g1.x, dS00, dS01, dS11);
            CovState F;
            cov_state(S, F);
            cov_backward(F, C, S.clampx, S.clampy, dS00, dS01, dS11, d_ls, d_q, dL_dt);
            // t = W p + t_cam  =>  dp += W^T dt
#pragma unroll
            for (int k = 0; k < 3; ++k)
                d_mean[k] += V[k] * dL_dt[0] + V[4 + k] * dL_dt[1] + V[8 + k] * dL_dt[2];
        }

        out.means[3 * i] = d_mean[0];
        out.means[3 * i + 1] = d_mean[1];
        out.means[3 * i + 2] = d_mean[2];
        out.log_scales[3 * i] = d_ls[0];
        out.log_scales[3 * i + 1] = d_ls[1];
        out.log_scales[3 * i + 2] = d_ls[2];
        reinterpret_cast<float4 *>(out.quats)[i] = make_float4(d_q[0], d_q[1], d_q[2], d_q[3]);
        if (cfg.mask_apply == MG_APPLY_OPACITY) {
            // o' = M o: dL/do = M dL/do', dL/dM = o dL/do'
            const float Mf = sp.mask[i] ? 1.0f : 0.0f;
            d_M = op * d_op;
            d_op *= Mf;
        }
        out.opacity_logit[i] = d_op * op * (1.0f - op);
        // lambda_m dL_m/dM_i of the Gaussian's scene (Eq. 7-8)
        if (cfg.lambda_m != 0.0f && sp.mask_count != nullptr) {
            for (int v = 0; v < vt.n_views; ++v) {
                if (i < vt.g_off[v] || i >= vt.g_off[v] + vt.g_cnt[v]) continue;
                const float iN = __fdividef(1.0f, (float)vt.g_cnt[v]);
                d_M += cfg.mask_loss == MG_MASK_LOSS_L1
                           ? cfg.lambda_m * iN
                           : 2.0f * cfg.lambda_m * ((float)sp.mask_count[v] * iN) * iN;
                break;
            }
        }
        float dl0 = 0.0f;
        if (cfg.mask_mode == MG_MASK_GUMBEL) {
            const float y0 = sp.mask_soft[i];
            dl0 = __fdividef(d_M * y0 * (1.0f - y0), cfg.tau);
        } else if (cfg.mask_mode == MG_MASK_STE) {
            const float p = sp.mask_soft[i];
            dl0 = d_M * p * (1.0f - p);
        }
        reinterpret_cast<float2 *>(out.mask_logits)[i] = make_float2(dl0, -dl0);
    }
    __syncwarp();
    // ---- the warp's dL/dsh rows are contiguous in global memory
    float *dst = out.sh + gw0 * ROW;
    const int total = nrows * ROW;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        const int n4 = total >> 2;
        for (int qq = lane; qq < n4; qq += 32) {
            float e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = 4 * qq + u;
                e[u] = dsh[(f / ROW) * S_ + (f % ROW)];
            }
            d4[qq] = make_float4(e[0], e[1], e[2], e[3]);
        }
        done = n4 << 2;
    }
    for (int f = done + lane; f < total; f += 32) dst[f] = dsh[(f / ROW) * S_ + (f % ROW)];
}

}  // namespace mg

using namespace mg;

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static size_t attr_bytes(int32_t dtype) { return dtype == MG_DTYPE_F32 ? 4 : 2; }

static mg_status check_gaussians(const mg_gaussians *g) {
    if (g == nullptr || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3 ||
        (g->dtype != MG_DTYPE_F32 && g->dtype != MG_DTYPE_BF16 && g->dtype != MG_DTYPE_F16))
        return MG_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logit || !g->sh ||
                     !g->mask_logits))
        return MG_ERR_INVALID_ARG;
    const size_t eb = attr_bytes(g->dtype);
    if (!aligned(g->quats, 4 * eb) || !aligned(g->mask_logits, 8) || !aligned(g->sh, 16) ||
        !aligned(g->means, 4) || !aligned(g->log_scales, eb) || !aligned(g->opacity_logit, eb))
        return MG_ERR_INVALID_ARG;
    if (g->n >= (int64_t(1) << 31)) return MG_ERR_INVALID_ARG;
    return MG_OK;
}

template <int DEG>
static void launch_preprocess(int32_t dtype, dim3 grid, cudaStream_t s, const ViewTable &vt,
                              const mg_gaussians &g, const mg_raster_cfg &cfg,
                              const mg_splats &out) {
    if (dtype == MG_DTYPE_BF16)
        launch_pdl(preprocess_kernel<DEG, __nv_bfloat16>, dim3(grid), dim3(kPreThreads), 0, s, vt,
            g, cfg, out);
    else if (dtype == MG_DTYPE_F16)
        launch_pdl(preprocess_kernel<DEG, __half>, dim3(grid), dim3(kPreThreads), 0, s, vt, g, cfg,
            out);
    else
        launch_pdl(preprocess_kernel<DEG, float>, dim3(grid), dim3(kPreThreads), 0, s, vt, g, cfg,
            out);
}

template <int DEG>
static void launch_preprocess_backward(int32_t dtype, dim3 grid, cudaStream_t s,
                                       const ViewTable &vt, const mg_gaussians &g,
                                       const mg_raster_cfg &cfg, const mg_splats &sp,
                                       const float *grad2d, const mg_param_grads &out) {
    if (dtype == MG_DTYPE_BF16)
        launch_pdl(preprocess_backward_kernel<DEG, __nv_bfloat16>, dim3(grid), dim3(kPreThreads), 0,
            s, vt, g, cfg, sp, grad2d, out);
    else if (dtype == MG_DTYPE_F16)
        launch_pdl(preprocess_backward_kernel<DEG, __half>, dim3(grid), dim3(kPreThreads), 0, s, vt,
            g, cfg, sp, grad2d, out);
    else
        launch_pdl(preprocess_backward_kernel<DEG, float>, dim3(grid), dim3(kPreThreads), 0, s, vt,
            g, cfg, sp, grad2d, out);
}

static mg_status check_views(const mg_gaussians *g, const mg_view *views, int32_t n_views,
                             const mg_raster_cfg *cfg, ViewTable *vt) {
    mg_status st = mg_host::build_view_table(views, n_views, cfg, vt);
    if (st != MG_OK) return st;
    for (int v = 0; v < n_views; ++v)
        if (views[v].gaussian_offset + views[v].gaussian_count > g->n) return MG_ERR_INVALID_ARG;
    if (vt->rec_off[n_views] >= (int64_t(1) << 32)) return MG_ERR_INVALID_ARG;
    return MG_OK;
}

static mg_status check_mask_cfg(const mg_raster_cfg *cfg) {
    if (!(cfg->tau > 0.0f)) return MG_ERR_INVALID_ARG;
    if (cfg->mask_mode < MG_MASK_GUMBEL || cfg->mask_mode > MG_MASK_STE) return MG_ERR_INVALID_ARG;
    if (cfg->mask_mode == MG_MASK_GIVEN && cfg->given_mask == nullptr) return MG_ERR_INVALID_ARG;
    if (cfg->mask_apply != MG_APPLY_RASTER && cfg->mask_apply != MG_APPLY_OPACITY)
        return MG_ERR_INVALID_ARG;
    if (cfg->mask_loss != MG_MASK_LOSS_L2 && cfg->mask_loss != MG_MASK_LOSS_L1)
        return MG_ERR_INVALID_ARG;
    if (!isfinite(cfg->lambda_m) || !isfinite(cfg->ste_logit)) return MG_ERR_INVALID_ARG;
    return MG_OK;
}

extern "C" mg_status mg_preprocess(const mg_gaussians *g, const mg_view *views, int32_t n_views,
                                   const mg_raster_cfg *cfg, const mg_splats *out,
                                   mg_status_word *d_status, mg_stream_t stream) {
    (void)d_status;
    if (check_gaussians(g) != MG_OK || cfg == nullptr || out == nullptr ||
        check_mask_cfg(cfg) != MG_OK)
        return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = check_views(g, views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (out->mask_count != nullptr &&
        cudaMemsetAsync(out->mask_count, 0, sizeof(uint32_t) * n_views, s) != cudaSuccess)
        return MG_ERR_CUDA;
    if (g->n == 0) return MG_OK;
    if (!out->record || !out->tiles_touched || !out->radius || !out->clamp || !out->mask ||
        !out->mask_soft || !out->bin_record || !aligned(out->record, 16) ||
        !aligned(out->bin_record, 16))
        return MG_ERR_INVALID_ARG;
    for (int v = 0; v < n_views; ++v)
        if (vt.gx[v] >= 65536 || vt.gy[v] >= 65536) return MG_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((g->n + kPreThreads - 1) / kPreThreads));
    switch (g->sh_degree) {
        case 0: launch_preprocess<0>(g->dtype, grid, s, vt, *g, *cfg, *out); break;
        case 1: launch_preprocess<1>(g->dtype, grid, s, vt, *g, *cfg, *out); break;
        case 2: launch_preprocess<2>(g->dtype, grid, s, vt, *g, *cfg, *out); break;
        default: launch_preprocess<3>(g->dtype, grid, s, vt, *g, *cfg, *out); break;
    }
    return mg_host::launch_status();
}

extern "C" mg_status mg_preprocess_backward(const mg_gaussians *g, const mg_view *views,
                                            int32_t n_views, const mg_raster_cfg *cfg,
                                            const mg_splats *splats, const float *grad2d,
                                            const mg_param_grads *out, mg_stream_t stream) {
    if (check_gaussians(g) != MG_OK || cfg == nullptr || splats == nullptr || out == nullptr ||
        check_mask_cfg(cfg) != MG_OK)
        return MG_ERR_INVALID_ARG;
    if (cfg->lambda_m != 0.0f && splats->mask_count == nullptr) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = check_views(g, views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    if (g->n == 0) return MG_OK;
    if (!grad2d || !aligned(grad2d, 16) || !out->means || !out->log_scales || !out->quats ||
        !aligned(out->quats, 16) || !out->opacity_logit || !out->sh || !out->mask_logits ||
        !aligned(out->mask_logits, 8) || !splats->radius || !splats->clamp || !splats->mask_soft ||
        !splats->mask)
        return MG_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((g->n + kPreThreads - 1) / kPreThreads));
    cudaStream_t s = (cudaStream_t)stream;
    switch (g->sh_degree) {
        case 0: launch_preprocess_backward<0>(g->dtype, grid, s, vt, *g, *cfg, *splats, grad2d, *out); break;
        case 1: launch_preprocess_backward<1>(g->dtype, grid, s, vt, *g, *cfg, *splats, grad2d, *out); break;
        case 2: launch_preprocess_backward<2>(g->dtype, grid, s, vt, *g, *cfg, *splats, grad2d, *out); break;
        default: launch_preprocess_backward<3>(g->dtype, grid, s, vt, *g, *cfg, *splats, grad2d, *out); break;
    }
    return mg_host::launch_status();
}

// ---------------------------------------------------------------------------
// Mask loss value (Eq. 7-8): lambda_m L_m per scene, a scene being a distinct
// Gaussian range among the views.
// ---------------------------------------------------------------------------
namespace mg {
struct SceneList {
    int32_t n;
    int32_t view[MG_MAX_VIEWS];
    int64_t count[MG_MAX_VIEWS];
};

__global__ void mask_loss_kernel(SceneList sl, const uint32_t *__restrict__ mask_count,
                                 float lambda_m, int32_t kind, float *loss) {
    grid_dependency_wait();
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int k = 0; k < sl.n; ++k) {
        const double frac = (double)mask_count[sl.view[k]] / (double)sl.count[k];
        acc += kind == MG_MASK_LOSS_L1 ? frac : frac * frac;
    }
    *loss += (float)((double)lambda_m * acc);
}
}  // namespace mg

namespace mg {
__global__ void advance_iteration_kernel(uint64_t *it, uint64_t by) {
    grid_dependency_wait();
    *it += by;
}
}  // namespace mg

extern "C" mg_status mg_advance_iteration(uint64_t *iteration_dev, uint64_t by,
                                          mg_stream_t stream) {
    if (iteration_dev == nullptr || (reinterpret_cast<uintptr_t>(iteration_dev) & 7u) != 0)
        return MG_ERR_INVALID_ARG;
    launch_pdl(advance_iteration_kernel, dim3(1), dim3(1), 0, (cudaStream_t)stream,
        iteration_dev, by);
    return mg_host::launch_status();
}

extern "C" mg_status mg_mask_loss(const mg_splats *splats, const mg_view *views, int32_t n_views,
                                  const mg_raster_cfg *cfg, float *loss, mg_stream_t stream) {
    if (splats == nullptr || views == nullptr || cfg == nullptr || loss == nullptr ||
        splats->mask_count == nullptr || n_views < 1 || n_views > MG_MAX_VIEWS ||
        (cfg->mask_loss != MG_MASK_LOSS_L2 && cfg->mask_loss != MG_MASK_LOSS_L1) ||
        !isfinite(cfg->lambda_m))
        return MG_ERR_INVALID_ARG;
    SceneList sl;
    sl.n = 0;
    for (int v = 0; v < n_views; ++v) {
        if (views[v].gaussian_count <= 0) continue;
        bool seen = false;
        for (int u = 0; u < v; ++u)
            seen |= views[u].gaussian_offset == views[v].gaussian_offset &&
                    views[u].gaussian_count == views[v].gaussian_count;
        if (seen) continue;
        sl.view[sl.n] = v;
        sl.count[sl.n] = views[v].gaussian_count;
        ++sl.n;
    }
    if (sl.n == 0 || cfg->lambda_m == 0.0f) return MG_OK;
    launch_pdl(mask_loss_kernel, dim3(1), dim3(32), 0, (cudaStream_t)stream, sl, splats->mask_count,
        cfg->lambda_m, cfg->mask_loss, loss);
    return mg_host::launch_status();
}
