// Masked rasterisation, forward (Eq. 3-4) and backward (Eq. 6, Appendix A),
// and the L1 render loss.
//
// One CTA of 128 threads per tile, two pixels per thread: warp w owns an 8x8
// block of the tile, a lane one column of it at two rows 4 apart.  The
// tile's depth-sorted splats are staged through shared memory in batches
// (each thread gathers 48-byte records and culls each splat against the
// four warp blocks), then every warp walks only the splats that can reach its
// block, applying each to both of a thread's pixels.  The forward skips
// masked splats outright: with M_i = 0 they neither add colour nor attenuate
// T (Eq. 3-4).  The backward walks the same lists back to front from each
// pixel's stop index, recovers T_i = T_{i+1}/(1 - M_i alpha_i), sums each
// splat's ten gradient terms over a thread's two pixels, then over the warp
// with a halving shuffle exchange into the warp's own shared-memory slot,
// adds the warps' slots when the batch is flushed, and issues three vector
// atomics per splat and tile.  Masked splats carry only dL/dM (one scalar
// reduction and atomic).
//
// alpha is evaluated by the same explicitly rounded sequence in both kernels
// so that the forward's and the backward's per-fragment decisions agree.
#include "internal.cuh"

namespace mg {

constexpr int kPix = 2;                          // pixels per thread (one column pair)
constexpr int kRenderThreads = 256 / kPix;       // threads per CTA (one 256-pixel tile)
constexpr int kRenderWarps = kRenderThreads / 32;
constexpr int kBatch = 256;                      // splats staged per batch (default)

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic for the alpha of a thread's two pixels (.x = the
// first pixel, .y = the one kRowStep rows below): one instruction for both,
// per component the correctly rounded scalar operation.
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float sqrt_approx(float x) {   // x >= 0
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha = min(0.99, o 2^e), e = h1 p1^2 + h2 p2^2, p1 = d.u, p2 = d.u_perp,
// d = pixel centre - mean.  A = (mx, my, ux, uy), B = (h1, h2, +-o, e_min):
// the sign of B.z is the mask (negative = masked), and e_min (stored by the
// preprocess, just below log2(1/(255 o))) bounds the ellipse the warp-block
// culling tests; every fragment a warp walks is decided by the alpha test,
// evaluated identically in both kernels.
// A thread's two pixels share a column, kRowStep rows apart: the second
// pixel's offsets follow from the first's (d.y + 4, p1 + 4 uy, p2 + 4 ux).
constexpr float kRowStep = 4.0f;

struct FragPair {
    float dx;            // pixel centre - mean, x (one column: shared by the pair)
    float dy0;           // y offset of the first pixel; the second's is dy0 + kRowStep
    float2 araw, alpha;  // o 2^e and min(0.99, o 2^e) of both pixels
    bool on0, on1;       // alpha reaches the 1/255 floor
};

__device__ __forceinline__ FragPair frag_alpha_pair(const float4 &A, const float4 &B, float fpx,
                                                    float fpy0) {
    FragPair f;
    f.dx = __fsub_rn(fpx, A.x);
    f.dy0 = __fsub_rn(fpy0, A.y);
    const float p10 = __fmaf_rn(f.dy0, A.w, __fmul_rn(f.dx, A.z));
    const float p20 = __fmaf_rn(f.dy0, A.z, -__fmul_rn(f.dx, A.w));
    const float2 p1 = make_float2(p10, __fmaf_rn(kRowStep, A.w, p10));
    const float2 p2 = make_float2(p20, __fmaf_rn(kRowStep, A.z, p20));
    // e = (h1 p1) p1 + (h2 p2) p2, the products rounded, the sum fused
    const float2 e = fma2(mul2(bcast2(B.x), p1), p1, mul2(mul2(bcast2(B.y), p2), p2));
    // straight-line: the exp unit has room, a branch per pixel costs more
    const float2 G = make_float2(ex2_approx(e.x), ex2_approx(e.y));
    f.araw = mul2(bcast2(fabsf(B.z)), G);
    f.alpha = make_float2(fminf(kAlphaMax, f.araw.x), fminf(kAlphaMax, f.araw.y));
    f.on0 = f.alpha.x >= kAlphaMin;
    f.on1 = f.alpha.y >= kAlphaMin;
    return f;
}

// Tile of the CTA and the kPix pixels of this thread.  Each warp owns one
// 8x8 block of the tile (square blocks: fewer splats straddle a block edge
// than with 16x4 strips), block w at (8 (w % nbx), 8 (w / nbx)), nbx =
// tile_w / 8; lane l's pixels are (l % 8, l / 8) and the same column 4 rows
// further down.
constexpr int kBlock = 8;

struct TileInfo {
    int v;
    int x0, y0;          // tile origin (pixels)
    int nbx;             // 8x8 blocks per tile row
    int px[kPix], py[kPix];
    bool inside[kPix];
    int64_t pix[kPix];   // pixel index within the view
};

__device__ __forceinline__ TileInfo tile_info(const ViewTable &vt, int64_t t) {
    TileInfo ti;
    ti.v = view_of_tile(vt, t);
    const int64_t lt = t - vt.tile_off[ti.v];
    const int gx = vt.gx[ti.v];
    ti.x0 = (int)(lt % gx) * vt.tile_w;
    ti.y0 = (int)(lt / gx) * vt.tile_h;
    ti.nbx = vt.tile_w / kBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = ti.x0 + kBlock * (warp % ti.nbx), by = ti.y0 + kBlock * (warp / ti.nbx);
    const mg_camera &C = vt.cam[ti.v];
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        ti.px[k] = bx + (lane & (kBlock - 1));
        ti.py[k] = by + (lane >> 3) + k * (32 / kBlock);
        ti.inside[k] = ti.px[k] < C.width && ti.py[k] < C.height;
        ti.pix[k] = (int64_t)ti.py[k] * C.width + ti.px[k];
    }
    return ti;
}

// ---------------------------------------------------------------------------
// Per-warp culling.  When a batch is staged, the thread that loads splat j
// tests the splat's alpha = 1/255 ellipse, enlarged by a margin, against each
// warp's pixel block with a separating-axis test (tile axes and the ellipse's
// axes; it never separates shapes that overlap).  Every pixel whose FP32
// alpha reaches the floor lies inside the enlarged ellipse, so skipping the
// splat for a block it misses changes no result: both kernels still apply the
// per-pixel alpha test, on the same set of splats.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_mask(const float4 &A, const float4 &B, float x0,
                                               float y0, int nbx) {
    // e_min < 0 is the stored skip threshold (already pushed outwards by
    // 1e-3 in log2 alpha); e_min > 0 marks a splat that never reaches the floor
    const float e_thr = B.w;
    if (!(e_thr < 0.0f)) return 0u;
    // approximate square roots and divisions (relative errors of a few 1e-7)
    // stay far inside the 1e-4 relative and 0.02 px margins
    const float r1 = sqrt_approx(__fdividef(e_thr, B.x)) * 1.0001f + 0.02f;   // along u
    const float r2 = sqrt_approx(__fdividef(e_thr, B.y)) * 1.0001f + 0.02f;   // along u_perp
    const float ux = A.z, uy = A.w;
    const float aux = fabsf(ux), auy = fabsf(uy);
    const float ex = sqrt_approx(r1 * r1 * ux * ux + r2 * r2 * uy * uy) + 0.02f;
    const float ey = sqrt_approx(r1 * r1 * uy * uy + r2 * r2 * ux * ux) + 0.02f;
    // pixel centres of a block span its origin + 0.5 .. + 7.5
    const float hw = 0.5f * (float)(kBlock - 1), hh = hw;
    uint32_t m = 0u;
#pragma unroll
    for (int w = 0; w < kRenderWarps; ++w) {
        const float cx = x0 + (float)(kBlock * (w % nbx)) + 0.5f * (float)kBlock;
        const float cy = y0 + (float)(kBlock * (w / nbx)) + 0.5f * (float)kBlock;
        const float dx = cx - A.x, dy = cy - A.y;
        const bool sep_x = fabsf(dx) > ex + hw;
        const bool sep_y = fabsf(dy) > ey + hh;
        const bool sep_u = fabsf(dx * ux + dy * uy) > r1 + hw * aux + hh * auy + 0.02f;
        const bool sep_v = fabsf(dy * ux - dx * uy) > r2 + hw * auy + hh * aux + 0.02f;
        if (!(sep_x || sep_y || sep_u || sep_v)) m |= 1u << w;
    }
    return m;
}

__device__ __forceinline__ bool all_done(const bool *done) {
    bool a = true;
#pragma unroll
    for (int k = 0; k < kPix; ++k) a = a && done[k];
    return a;
}

__device__ __forceinline__ float l1_sign(float d, float inv) {
    return d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// COUNT = true adds per-fragment counters (an untimed diagnostic variant):
// [0] positions walked (sum of n_contrib), [1] unmasked positions walked,
// [2] unmasked splats blended, [3] masked splats above the alpha floor.
// They count every walked position, culled or not.  AUX = false is the
// inference form: the image only, no final_T / n_contrib for a backward.
// L1 = true also takes the L1 render loss in the epilogue, from the colours
// in registers: dL/dimage = sign(C - target) / (3 W H) and one atomic per CTA
// adding the CTA's sum of |C - target| / (3 W H) to *loss.
// Twelve CTAs per SM (48 warps): the 40 registers this leaves hold the
// kernel without spills, and the extra warps fill the issue slots that the
// staging barriers leave idle (ten CTAs at 48 registers measured 1 % slower).
template <bool COUNT, bool AUX = true, bool L1 = false, int BATCH = kBatch>
__global__ void __launch_bounds__(kRenderThreads, 12)
render_forward_kernel(ViewTable vt, const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, const uint32_t *__restrict__ tile_order,
                      float bg0, float bg1, float bg2,
                      float *__restrict__ image, float *__restrict__ final_T,
                      uint32_t *__restrict__ n_contrib, unsigned long long *frag_count,
                      const float *__restrict__ target = nullptr,
                      float *__restrict__ dL_dimage = nullptr, float *loss = nullptr,
                      float4 *__restrict__ reset4 = nullptr, int64_t reset_n4 = 0) {
    grid_dependency_wait();
    // the training forward also resets the backward's 2D-gradient accumulator:
    // each CTA stores zeros over its share (the kernel's memory path is nearly
    // idle, and the backward starts only once this kernel has completed)
    if (reset4 != nullptr) {
        const int64_t per = (reset_n4 + gridDim.x - 1) / gridDim.x;
        const int64_t q0 = (int64_t)blockIdx.x * per;
        const int64_t q1 = min(q0 + per, reset_n4);
        for (int64_t q = q0 + threadIdx.x; q < q1; q += kRenderThreads)
            reset4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __shared__ float4 sA[BATCH], sB[BATCH], sC[BATCH];
    __shared__ uint8_t sM[BATCH];
    __shared__ unsigned long long s_frags[4];
    const int64_t t = tile_order ? (int64_t)tile_order[blockIdx.x] : (int64_t)blockIdx.x;
    const TileInfo ti = tile_info(vt, t);
    const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float fpx[kPix], fpy[kPix], T[kPix], C0[kPix], C1[kPix], C2[kPix];
    bool done[kPix];
    uint32_t stop[kPix];
    uint32_t c_unmasked = 0, c_blend = 0, c_masked = 0;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        fpx[k] = (float)ti.px[k] + 0.5f;
        fpy[k] = (float)ti.py[k] + 0.5f;
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        done[k] = !ti.inside[k];
        stop[k] = end - start;
    }
    if (threadIdx.x < 4) s_frags[threadIdx.x] = 0ull;

    for (uint32_t b0 = start; b0 < end; b0 += BATCH) {
        if (__syncthreads_count(all_done(done)) == kRenderThreads) break;
#pragma unroll
        for (int h = 0; h < (BATCH + kRenderThreads - 1) / kRenderThreads; ++h) {
            const int i = threadIdx.x + h * kRenderThreads;
            if (b0 + i < end) {
                const uint32_t r = vals[b0 + i];
                const float4 A = rec[3 * (int64_t)r], B = rec[3 * (int64_t)r + 1];
                sA[i] = A;
                sB[i] = B;
                sC[i] = rec[3 * (int64_t)r + 2];
                // masked splats neither colour nor attenuate: out of every forward list
                sM[i] = (uint8_t)((B.z > 0.0f)
                                      ? block_mask(A, B, (float)ti.x0, (float)ti.y0, ti.nbx)
                                      : 0u);
            }
        }
        __syncthreads();
        const int cnt = (int)min(end - b0, (uint32_t)BATCH);
        if (COUNT) {
            // diagnostic counts over every position (culled or not) up to the stop
#pragma unroll
            for (int k = 0; k < kPix; ++k) {
                if (done[k]) continue;
                float Tc = T[k];
                for (int j = 0; j < cnt; ++j) {
                    const float4 B = sB[j];
                    const FragPair f = frag_alpha_pair(sA[j], B, fpx[0], fpy[0]);
                    const bool on = k == 0 ? f.on0 : f.on1;
                    const float alpha = k == 0 ? f.alpha.x : f.alpha.y;
                    if (B.z < 0.0f) {
                        c_masked += on;
                        continue;
                    }
                    ++c_unmasked;
                    if (!on) continue;
                    const float tT = Tc * (1.0f - alpha);
                    if (tT < kTMin) {
                        --c_unmasked;
                        break;
                    }
                    ++c_blend;
                    Tc = tT;
                }
            }
        }
        if (__all_sync(0xffffffffu, all_done(done))) continue;
        const int nchunks = (cnt + 31) >> 5;
        for (int ch = 0; ch < nchunks; ++ch) {
            const int jj = (ch << 5) + lane;
            unsigned word = __ballot_sync(0xffffffffu, jj < cnt && ((sM[jj] >> warp) & 1u));
            while (word) {
                const int j = (ch << 5) + __ffs(word) - 1;
                word &= word - 1;
                const float4 A = sA[j], B = sB[j], c = sC[j];
                const FragPair f = frag_alpha_pair(A, B, fpx[0], fpy[0]);
                const bool on[kPix] = {f.on0, f.on1};
                const float al[kPix] = {f.alpha.x, f.alpha.y};
#pragma unroll
                for (int k = 0; k < kPix; ++k) {
                    if (done[k]) continue;
                    if (!on[k]) continue;
                    const float testT = T[k] * (1.0f - al[k]);
                    if (testT < kTMin) {
                        done[k] = true;
                        stop[k] = (b0 - start) + j;
                        continue;
                    }
                    const float w = al[k] * T[k];
                    C0[k] = fmaf(w, c.x, C0[k]);
                    C1[k] = fmaf(w, c.y, C1[k]);
                    C2[k] = fmaf(w, c.z, C2[k]);
                    T[k] = testT;
                }
            }
            if (__all_sync(0xffffffffu, all_done(done))) break;
        }
    }
    if (COUNT) {
        unsigned long long walked = 0;
#pragma unroll
        for (int k = 0; k < kPix; ++k) walked += ti.inside[k] ? stop[k] : 0u;
        unsigned long long c[4] = {walked, c_unmasked, c_blend, c_masked};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_down_sync(0xffffffffu, c[k], o);
        }
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&s_frags[k], c[k]);
        __syncthreads();
        if (threadIdx.x < 4) atomicAdd(frag_count + threadIdx.x, s_frags[threadIdx.x]);
    }
    const mg_camera &Cm = vt.cam[ti.v];
    const int64_t HW = (int64_t)Cm.width * Cm.height;
    float *img = image + 3 * vt.pix_off[ti.v];
    const float inv = 1.0f / (float)(3 * HW);
    float lsum = 0.0f;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        if (!ti.inside[k]) continue;
        const float c[3] = {C0[k] + T[k] * bg0, C1[k] + T[k] * bg1, C2[k] + T[k] * bg2};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            img[ch * HW + ti.pix[k]] = c[ch];
            if (L1) {
                const int64_t e = 3 * vt.pix_off[ti.v] + ch * HW + ti.pix[k];
                const float d = c[ch] - target[e];
                dL_dimage[e] = l1_sign(d, inv);
                lsum += fabsf(d);
            }
        }
        if (AUX) {
            final_T[vt.pix_off[ti.v] + ti.pix[k]] = T[k];
            n_contrib[vt.pix_off[ti.v] + ti.pix[k]] = stop[k];
        }
    }
    if (L1) {
        __shared__ float s_loss[kRenderThreads / 32];
        lsum = warp_sum(lsum);
        if (lane == 0) s_loss[warp] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
#pragma unroll
            for (int w = 0; w < kRenderThreads / 32; ++w) t += s_loss[w];
            atomicAdd(loss, t * inv);
        }
    }
}

// Warp sums of a splat's ten gradient terms by halving exchanges that split
// the values unevenly where ten does not halve (10 -> 5 -> 3|2 -> 2|1 -> 1):
// 12 shuffles.  On return the lane holds the warp sum of term
// red_term(lane) (see below); every term is held by at least two lanes.
__device__ __forceinline__ float warp_transpose_sum10(const float v[10], int lane) {
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
    // xor 16: keep five (0-4 or 5-9), send the other five
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float send = b16 ? v[i] : v[i + 5];
        const float keep = b16 ? v[i + 5] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    // xor 8: lanes without bit 8 keep a0..a2, lanes with it keep a3, a4
    float b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float send = b8 ? a[i] : (i < 2 ? a[i + 3] : 0.0f);
        const float keep = b8 ? (i < 2 ? a[i + 3] : 0.0f) : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    // xor 4: three values split 2 | 1, two values split 1 | 1
    float c[2];
    {
        // first exchange: (no bit 8) bit 4 clear keeps b0, sends b2; set keeps b2, sends b0
        //                 (bit 8)    bit 4 clear keeps b0, sends b1; set keeps b1, sends b0
        const float send0 = b4 ? b[0] : (b8 ? b[1] : b[2]);
        const float keep0 = b4 ? (b8 ? b[1] : b[2]) : b[0];
        c[0] = keep0 + __shfl_xor_sync(0xffffffffu, send0, 4);
        // second exchange: only the three-value lanes move b1 (kept by bit 4 clear)
        const float send1 = (!b8 && b4) ? b[1] : 0.0f;
        const float keep1 = (!b8 && !b4) ? b[1] : 0.0f;
        c[1] = keep1 + __shfl_xor_sync(0xffffffffu, send1, 4);
    }
    // xor 2: the two-value lanes (no bit 8, no bit 4) split c0 | c1; the others add
    float d;
    {
        const bool two = !b8 && !b4;
        const float send = two ? (b2 ? c[0] : c[1]) : c[0];
        const float keep = two ? (b2 ? c[1] : c[0]) : c[0];
        d = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// The term whose warp sum warp_transpose_sum10 leaves in `lane`, and whether
// the lane is the one that flushes it (one lane per term).
__device__ __forceinline__ int red_term(int lane, bool &writer) {
    const int hi = (lane & 16) ? 5 : 0;
    const bool b8 = lane & 8, b4 = lane & 4, b2 = lane & 2, b1 = lane & 1;
    int term;
    if (!b8 && !b4) {
        term = hi + (b2 ? 1 : 0);
        writer = !b1;
    } else {
        term = hi + (b8 ? (b4 ? 4 : 3) : 2);
        writer = !b1 && !b2;
    }
    return term;
}

// Per splat and tile, the backward accumulates in shared memory
//   S0 = sum dpow, S1 = sum dpow dx, S2 = sum dpow dy,
//   S3 = sum dpow dx^2, S4 = sum dpow dx dy, S5 = sum dpow dy^2,
//   S6..S8 = sum alpha T_i g (colour), S9 = sum dL/dM,
// with dpow = dL/dalpha * alpha (dL/dpower of the unclamped alpha) and
// d = pixel centre - mean; then dL/do = S0 / o, dL/dmean2d = Sigma^-1 (S1, S2),
// dL/dconic = (-S3/2, -S4, -S5/2).
constexpr int kAcc = 10;

// COUNT = true accumulates profiling counters (an untimed variant):
// [0] (warp, splat) list iterations, [1] of which masked, [2] unmasked with a
// contributing pixel, [3] masked with a contributing pixel, [4] contributing
// pixels over [2], [5] staged batches.
// Eight CTAs per SM (32 warps): the register cap this asks for (64) holds
// without spills, and eight copies of the 27.3 KB of shared memory fit (a
// ninth does not).
constexpr int kBatchB = 128;                    // splats staged per backward batch (default)
template <bool COUNT, int BATCHB = kBatchB>
__global__ void __launch_bounds__(kRenderThreads, 1024 / kRenderThreads)
render_backward_kernel(ViewTable vt, const float4 *__restrict__ rec,
                       const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
                       const uint32_t *__restrict__ tile_order,
                       float bg0, float bg1, float bg2, const float *__restrict__ final_T,
                       const uint32_t *__restrict__ n_contrib, const float *__restrict__ dL_dimage,
                       float *__restrict__ grad2d, unsigned long long *counters) {
    grid_dependency_wait();
    unsigned long long cnt_it = 0, cnt_m = 0, cnt_cu = 0, cnt_cm = 0, cnt_pix = 0, cnt_b = 0;
    __shared__ float4 sA[BATCHB], sB[BATCHB], sC[BATCHB];
    __shared__ uint32_t sR[BATCHB];
    __shared__ uint8_t sM[BATCHB];
    __shared__ float sG[kRenderWarps][BATCHB][kAcc];   // per-warp sums: plain stores
    __shared__ uint32_t s_maxstop;
    __shared__ uint32_t s_wstop[kRenderWarps];
    const int64_t t = tile_order ? (int64_t)tile_order[blockIdx.x] : (int64_t)blockIdx.x;
    const TileInfo ti = tile_info(vt, t);
    const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool red_writer;
    const int red_t = red_term(lane, red_writer);   // term this lane flushes

    static_assert(kPix == 2, "the backward's moment sums assume a column pair");
    const float fpx = (float)ti.px[0] + 0.5f, fpy0 = (float)ti.py[0] + 0.5f;
    // gb = g . b, g = dL/dC of the pixel and b the colour behind (Appendix A's
    // b_{i+1} with the background folded in): the backward needs b only in
    // g . (c_i - b), so the scalar replaces the three channels
    float T[kPix], g0[kPix], g1[kPix], g2[kPix], gb[kPix];
    uint32_t stop[kPix];
    const mg_camera &Cm = vt.cam[ti.v];
    const int64_t HW = (int64_t)Cm.width * Cm.height;
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
        T[k] = 1.0f;
        g0[k] = g1[k] = g2[k] = 0.0f;
        stop[k] = 0;
        if (ti.inside[k]) {
            const int64_t p = vt.pix_off[ti.v] + ti.pix[k];
            T[k] = final_T[p];
            stop[k] = n_contrib[p];
            const float *gi = dL_dimage + 3 * vt.pix_off[ti.v];
            g0[k] = gi[ti.pix[k]];
            g1[k] = gi[HW + ti.pix[k]];
            g2[k] = gi[2 * HW + ti.pix[k]];
        }
        gb[k] = fmaf(g2[k], bg2, fmaf(g1[k], bg1, g0[k] * bg0));   // b_{N+1} = background
    }
    // the pixel pair's state as pairs for the paired FP32 arithmetic
    float2 T2 = make_float2(T[0], T[1]), GB = make_float2(gb[0], gb[1]);
    const float2 G0 = make_float2(g0[0], g0[1]), G1 = make_float2(g1[0], g1[1]),
                 G2 = make_float2(g2[0], g2[1]);
    uint32_t tstop = 0;
#pragma unroll
    for (int k = 0; k < kPix; ++k) tstop = max(tstop, stop[k]);
    if (threadIdx.x == 0) s_maxstop = 0;
    __syncthreads();
    atomicMax(&s_maxstop, tstop);
    __syncthreads();
    const uint32_t maxstop = min(s_maxstop, end - start);
    if (maxstop == 0) return;
    const int nb = (int)((maxstop + BATCHB - 1) / BATCHB);
    if (COUNT) cnt_b = nb;
    uint32_t wstop = tstop;                                    // warp's largest stop
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wstop = max(wstop, __shfl_xor_sync(0xffffffffu, wstop, o));
    if (lane == 0) s_wstop[warp] = wstop;

    for (int bi = nb - 1; bi >= 0; --bi) {
        const uint32_t pos0 = (uint32_t)bi * BATCHB;
        const int cnt = (int)min(maxstop - pos0, (uint32_t)BATCHB);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < (BATCHB + kRenderThreads - 1) / kRenderThreads; ++h) {
            const int i = threadIdx.x + h * kRenderThreads;
            if (i < cnt) {
                const uint32_t r = vals[start + pos0 + i];
                const float4 A = rec[3 * (int64_t)r], B = rec[3 * (int64_t)r + 1];
                sR[i] = r;
                sA[i] = A;
                sB[i] = B;
                sC[i] = rec[3 * (int64_t)r + 2];
                sM[i] = (uint8_t)block_mask(A, B, (float)ti.x0, (float)ti.y0, ti.nbx);
            }
        }
        __syncthreads();

        if (pos0 < wstop) {
            const int nchunks = (cnt + 31) >> 5;
            for (int ch = nchunks - 1; ch >= 0; --ch) {
                const int jj = (ch << 5) + lane;
                // the warp's splats of this chunk, up to its largest stop index
                unsigned word = __ballot_sync(0xffffffffu, jj < cnt && pos0 + jj < wstop &&
                                                               ((sM[jj] >> warp) & 1u));
                while (word) {
                    const int hb = 31 - __clz(word);
                    word &= ~(1u << hb);
                    const int j = (ch << 5) + hb;
                    const float4 A = sA[j], B = sB[j];
                    const bool masked = B.z < 0.0f;
                    const FragPair f = frag_alpha_pair(A, B, fpx, fpy0);
                    const bool on[kPix] = {pos0 + j < stop[0] && f.on0,
                                           pos0 + j < stop[1] && f.on1};
                    const float al[kPix] = {f.alpha.x, f.alpha.y};
                    const float ar[kPix] = {f.araw.x, f.araw.y};
                    const int ncontrib = (int)on[0] + (int)on[1];
                    if (!COUNT && !__any_sync(0xffffffffu, ncontrib > 0)) {
                        // every (warp, splat) of the warp's list leaves its sums
                        if (masked ? lane == 0 : red_writer) sG[warp][j][masked ? 9 : red_t] = 0.0f;
                        continue;
                    }
                    const float4 c = sC[j];
                    // the mask is uniform over the warp: two straight-line paths.  A
                    // pixel that is off (under the floor, or at or past its stop)
                    // takes alpha = 0: its T and colour behind then stay exactly as
                    // they are and it adds nothing, so the pixel arithmetic has no
                    // per-lane branches
                    const float2 a = make_float2(on[0] ? al[0] : 0.0f, on[1] ? al[1] : 0.0f);
                    float v[10];
                    if (masked) {
                        // M = 0: T and the colour behind are unchanged; only dL/dM
                        const float gc0 = fmaf(G2.x, c.z, fmaf(G1.x, c.y, G0.x * c.x)) - GB.x;
                        const float gc1 = fmaf(G2.y, c.z, fmaf(G1.y, c.y, G0.y * c.x)) - GB.y;
                        v[9] = fmaf(a.y * T2.y, gc1, (a.x * T2.x) * gc0);   // Eq. 6 + Appendix A
                    } else {
                        // T_i = T_{i+1} / (1 - alpha) = T_{i+1} + T_{i+1} alpha / (1 - alpha)
                        // (exactly T_{i+1} for alpha = 0); b_i = b_{i+1} + alpha (c_i -
                        // b_{i+1}); dL/dM = alpha T_i g.(c_i - b_{i+1}) (Eq. 6 + Appendix
                        // A), dL/dc = alpha T_i g, dL/dalpha alpha = dL/dM unless clamped
                        const bool any0 = __any_sync(0xffffffffu, on[0]);
                        const bool any1 = __any_sync(0xffffffffu, on[1]);
                        float m0 = 0.0f, m1 = 0.0f;
                        if (any0 && any1) {
                            // both pixel rows of the warp: paired FP32, one instruction per pair
                            const float2 om = fma2(a, bcast2(-1.0f), bcast2(1.0f));
                            const float2 r = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                            const float2 Tj = fma2(mul2(T2, a), r, T2);
                            const float2 gc = fma2(G2, bcast2(c.z),
                                                   fma2(G1, bcast2(c.y),
                                                        fma2(G0, bcast2(c.x), neg2(GB))));
                            const float2 wt = mul2(a, Tj);
                            const float2 dm = mul2(wt, gc);
                            v[9] = dm.x + dm.y;
                            v[6] = fmaf(wt.y, G0.y, wt.x * G0.x);
                            v[7] = fmaf(wt.y, G1.y, wt.x * G1.x);
                            v[8] = fmaf(wt.y, G2.y, wt.x * G2.x);
                            GB = fma2(a, gc, GB);
                            T2 = Tj;
                            m0 = ar[0] < kAlphaMax ? dm.x : 0.0f;
                            m1 = ar[1] < kAlphaMax ? dm.y : 0.0f;
                        } else if (any0) {
                            // only the first row: the second pixels all contribute nothing
                            const float Tj = fmaf(T2.x * a.x, rcp_approx(1.0f - a.x), T2.x);
                            const float gc = fmaf(G2.x, c.z, fmaf(G1.x, c.y, G0.x * c.x)) - GB.x;
                            const float wt = a.x * Tj;
                            const float dm = wt * gc;
                            v[9] = dm;
                            v[6] = wt * G0.x;
                            v[7] = wt * G1.x;
                            v[8] = wt * G2.x;
                            GB.x = fmaf(a.x, gc, GB.x);
                            T2.x = Tj;
                            m0 = ar[0] < kAlphaMax ? dm : 0.0f;
                        } else {
                            const float Tj = fmaf(T2.y * a.y, rcp_approx(1.0f - a.y), T2.y);
                            const float gc = fmaf(G2.y, c.z, fmaf(G1.y, c.y, G0.y * c.x)) - GB.y;
                            const float wt = a.y * Tj;
                            const float dm = wt * gc;
                            v[9] = dm;
                            v[6] = wt * G0.y;
                            v[7] = wt * G1.y;
                            v[8] = wt * G2.y;
                            GB.y = fmaf(a.y, gc, GB.y);
                            T2.y = Tj;
                            m1 = ar[1] < kAlphaMax ? dm : 0.0f;
                        }
                        v[0] = m0 + m1;
                        const float s1 = kRowStep * m1;
                        // the pair shares dx and its dy differ by kRowStep: the
                        // moments follow from the sum of m and the second's m
                        v[1] = v[0] * f.dx;                               // sum m dx
                        v[2] = fmaf(f.dy0, v[0], s1);                     // sum m dy
                        v[3] = v[1] * f.dx;                               // sum m dx^2
                        v[4] = v[2] * f.dx;                               // sum m dx dy
                        v[5] = fmaf(v[2], f.dy0, s1 * __fadd_rn(f.dy0, kRowStep));  // sum m dy^2
                    }
                    if (COUNT) {
                        const unsigned cb = __ballot_sync(0xffffffffu, ncontrib > 0);
                        const int tot = __reduce_add_sync(0xffffffffu, (unsigned)ncontrib);
                        ++cnt_it;
                        cnt_m += masked;
                        cnt_cu += (!masked && cb);
                        cnt_cm += (masked && cb);
                        cnt_pix += masked ? 0 : tot;
                    }
                    if (masked) {
                        const float dm = warp_sum(v[9]);
                        if (lane == 0) sG[warp][j][9] = dm;
                    } else {
                        const float r = warp_transpose_sum10(v, lane);
                        if (red_writer) sG[warp][j][red_t] = r;
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < (BATCHB + kRenderThreads - 1) / kRenderThreads; ++h) {
            const int i = threadIdx.x + h * kRenderThreads;
            if (i >= cnt) continue;
            float4 *G4 = reinterpret_cast<float4 *>(grad2d) + 3 * (int64_t)sR[i];
            const float4 B = sB[i];
            // sum the slots of the warps whose list held the splat (a warp
            // skips the splats at or past its pixels' largest stop index)
            uint32_t wm = sM[i];
#pragma unroll
            for (int w = 0; w < kRenderWarps; ++w)
                if (pos0 + (uint32_t)i >= s_wstop[w]) wm &= ~(1u << w);
            float S[kAcc];
#pragma unroll
            for (int q = 0; q < kAcc; ++q) S[q] = 0.0f;
            if (B.z < 0.0f) {
#pragma unroll
                for (int w = 0; w < kRenderWarps; ++w)
                    if ((wm >> w) & 1u) S[9] += sG[w][i][9];
            } else {
#pragma unroll
                for (int w = 0; w < kRenderWarps; ++w)
                    if ((wm >> w) & 1u)
#pragma unroll
                        for (int q = 0; q < kAcc; ++q) S[q] += sG[w][i][q];
            }
            if (B.z < 0.0f) {
                if (S[9] != 0.0f) atomicAdd(&G4[2].y, S[9]);
            } else {
                const float4 A = sA[i];
                // Sigma^-1 in eigen form: w_k = -2 h_k / log2(e)
                const float w1 = (-2.0f / kLog2e) * B.x, w2 = (-2.0f / kLog2e) * B.y;
                const float q00 = w1 * A.z * A.z + w2 * A.w * A.w;
                const float q01 = (w1 - w2) * A.z * A.w;
                const float q11 = w1 * A.w * A.w + w2 * A.z * A.z;
                const float dmx = q00 * S[1] + q01 * S[2];
                const float dmy = q01 * S[1] + q11 * S[2];
                if (dmx != 0.0f || dmy != 0.0f || S[3] != 0.0f || S[4] != 0.0f)
                    atomicAdd(&G4[0], make_float4(dmx, dmy, -0.5f * S[3], -S[4]));
                if (S[5] != 0.0f || S[0] != 0.0f || S[6] != 0.0f || S[7] != 0.0f)
                    atomicAdd(&G4[1], make_float4(-0.5f * S[5], __fdividef(S[0], fabsf(B.z)),
                                                  S[6], S[7]));
                if (S[8] != 0.0f || S[9] != 0.0f)
                    atomicAdd(reinterpret_cast<float2 *>(&G4[2]), make_float2(S[8], S[9]));
            }
        }
    }
    if (COUNT && lane == 0) {   // per-warp counts (iteration counts are warp-uniform)
        atomicAdd(counters + 0, cnt_it);
        atomicAdd(counters + 1, cnt_m);
        atomicAdd(counters + 2, cnt_cu);
        atomicAdd(counters + 3, cnt_cm);
        atomicAdd(counters + 4, cnt_pix);
        if (warp == 0) atomicAdd(counters + 5, cnt_b);
    }
}

// One view per blockIdx.y; 128-bit loads and stores over the view's aligned
// body, scalar over its (at most 3 + 3) unaligned ends.
__global__ void l1_loss_grad_kernel(ViewTable vt, const float *__restrict__ image,
                                    const float *__restrict__ target, float *__restrict__ grad,
                                    float *loss) {
    grid_dependency_wait();
    const int v = blockIdx.y;
    const int64_t n = 3 * (vt.pix_off[v + 1] - vt.pix_off[v]);
    const int64_t o = 3 * vt.pix_off[v];
    const float inv = 1.0f / (float)n;
    float acc = 0.0f;
    const int64_t h0 = (4 - (o & 3)) & 3;                                  // to a 16-byte boundary
    const int64_t head = h0 < n ? h0 : n;
    const int64_t nb = (n - head) >> 2;                                    // float4 body
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const float4 *a4 = reinterpret_cast<const float4 *>(image + o + head);
    const float4 *b4 = reinterpret_cast<const float4 *>(target + o + head);
    float4 *g4 = reinterpret_cast<float4 *>(grad + o + head);
    for (int64_t q = tid; q < nb; q += nthr) {
        const float4 a = a4[q], b = b4[q];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        g4[q] = make_float4(l1_sign(d0, inv), l1_sign(d1, inv), l1_sign(d2, inv), l1_sign(d3, inv));
        acc += (fabsf(d0) + fabsf(d1)) + (fabsf(d2) + fabsf(d3));
    }
    // the unaligned head and tail
    const int64_t tail0 = head + (nb << 2);
    if (tid < head) {
        const float d = image[o + tid] - target[o + tid];
        grad[o + tid] = l1_sign(d, inv);
        acc += fabsf(d);
    }
    if (tid < n - tail0) {
        const int64_t i = o + tail0 + tid;
        const float d = image[i] - target[i];
        grad[i] = l1_sign(d, inv);
        acc += fabsf(d);
    }
    acc = warp_sum(acc);
    __shared__ float s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float a = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0f;
        a = warp_sum(a);
        if (threadIdx.x == 0 && loss != nullptr) atomicAdd(loss, a * inv);
    }
}

}  // namespace mg

using namespace mg;

// Staging depths the kernels are built for (mg_raster_cfg.render_batch and
// render_batch_bwd; 0 = the default).
static bool fwd_batch(const mg_raster_cfg *cfg, int *b) {
    *b = cfg->render_batch == 0 ? kBatch : cfg->render_batch;
    return *b == 128 || *b == 256;
}

static bool bwd_batch(const mg_raster_cfg *cfg, int *b) {
    *b = cfg->render_batch_bwd == 0 ? kBatchB : cfg->render_batch_bwd;
    return *b == 64 || *b == 128;
}

// The render with the L1 loss; grad2d (nullable) is reset on the way.
static mg_status render_l1(const mg_splats *splats, const uint32_t *sorted_vals,
                           const uint32_t *ranges, const uint32_t *tile_order,
                           const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                           float *image, float *final_T, uint32_t *n_contrib, const float *target,
                           float *dL_dimage, float *loss, float *grad2d, mg_stream_t stream) {
    if (!splats || !splats->record || !sorted_vals || !ranges || !image || !final_T ||
        !n_contrib || !target || !dL_dimage || !loss)
        return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->record) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(grad2d) & 15u) != 0)
        return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t tiles = vt.tile_off[n_views];
    if (tiles >= (int64_t(1) << 31)) return MG_ERR_INVALID_ARG;
    int batch;
    if (!fwd_batch(cfg, &batch)) return MG_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(splats->record);
    float4 *reset4 = reinterpret_cast<float4 *>(grad2d);
    const int64_t reset_n4 = grad2d ? vt.rec_off[n_views] * (MG_GRAD2D_FLOATS / 4) : 0;
    if (tiles == 0) {   // no tile to carry the reset
        if (grad2d && reset_n4 > 0 &&
            mg_host::zero_async(grad2d, sizeof(float4) * (size_t)reset_n4, (cudaStream_t)stream) !=
                MG_OK)
            return MG_ERR_CUDA;
        return MG_OK;
    }
    if (batch == 128)
        launch_pdl(render_forward_kernel<false, true, true, 128>, dim3((unsigned)tiles),
            dim3(kRenderThreads), 0, (cudaStream_t)stream, vt, rec, sorted_vals, ranges, tile_order,
            cfg->bg[0], cfg->bg[1], cfg->bg[2], image, final_T, n_contrib, nullptr, target,
            dL_dimage, loss, reset4, reset_n4);
    else
        launch_pdl(render_forward_kernel<false, true, true>, dim3((unsigned)tiles),
            dim3(kRenderThreads), 0, (cudaStream_t)stream, vt, rec, sorted_vals, ranges, tile_order,
            cfg->bg[0], cfg->bg[1], cfg->bg[2], image, final_T, n_contrib, nullptr, target,
            dL_dimage, loss, reset4, reset_n4);
    return mg_host::launch_status();
}

extern "C" mg_status mg_render_l1(const mg_splats *splats, const uint32_t *sorted_vals,
                                  const uint32_t *ranges, const uint32_t *tile_order,
                                  const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                                  float *image, float *final_T, uint32_t *n_contrib,
                                  const float *target, float *dL_dimage, float *loss,
                                  mg_stream_t stream) {
    return render_l1(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image, final_T,
                     n_contrib, target, dL_dimage, loss, nullptr, stream);
}

extern "C" mg_status mg_render_l1_reset2d(const mg_splats *splats, const uint32_t *sorted_vals,
                                          const uint32_t *ranges, const uint32_t *tile_order,
                                          const mg_view *views, int32_t n_views,
                                          const mg_raster_cfg *cfg, float *image, float *final_T,
                                          uint32_t *n_contrib, const float *target,
                                          float *dL_dimage, float *loss, float *grad2d,
                                          mg_stream_t stream) {
    if (grad2d == nullptr) return MG_ERR_INVALID_ARG;
    return render_l1(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, image, final_T,
                     n_contrib, target, dL_dimage, loss, grad2d, stream);
}

extern "C" mg_status mg_render(const mg_splats *splats, const uint32_t *sorted_vals,
                               const uint32_t *ranges, const uint32_t *tile_order,
                               const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                               float *image, float *final_T, uint32_t *n_contrib,
                               uint64_t *frag_count, mg_stream_t stream) {
    if (!splats || !splats->record || !sorted_vals || !ranges || !image || !final_T || !n_contrib)
        return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->record) & 15u) != 0) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t tiles = vt.tile_off[n_views];
    if (tiles >= (int64_t(1) << 31)) return MG_ERR_INVALID_ARG;
    int batch;
    if (!fwd_batch(cfg, &batch)) return MG_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(splats->record);
    if (frag_count != nullptr)      // the counting variant: default staging depth
        launch_pdl(render_forward_kernel<true>, dim3((unsigned)tiles), dim3(kRenderThreads), 0,
            (cudaStream_t)stream, vt, rec, sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1],
            cfg->bg[2], image, final_T, n_contrib,
            reinterpret_cast<unsigned long long *>(frag_count), nullptr, nullptr, nullptr, nullptr,
            (int64_t)0);
    else if (batch == 128)
        launch_pdl(render_forward_kernel<false, true, false, 128>, dim3((unsigned)tiles),
            dim3(kRenderThreads), 0, (cudaStream_t)stream, vt, rec, sorted_vals, ranges, tile_order,
            cfg->bg[0], cfg->bg[1], cfg->bg[2], image, final_T, n_contrib, nullptr, nullptr,
            nullptr, nullptr, nullptr, (int64_t)0);
    else
        launch_pdl(render_forward_kernel<false>, dim3((unsigned)tiles), dim3(kRenderThreads), 0,
            (cudaStream_t)stream, vt, rec, sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1],
            cfg->bg[2], image, final_T, n_contrib, nullptr, nullptr, nullptr, nullptr, nullptr,
            (int64_t)0);
    return mg_host::launch_status();
}

extern "C" mg_status mg_render_inference(const mg_splats *splats, const uint32_t *sorted_vals,
                                         const uint32_t *ranges, const uint32_t *tile_order,
                                         const mg_view *views, int32_t n_views,
                                         const mg_raster_cfg *cfg, float *image,
                                         mg_stream_t stream) {
    if (!splats || !splats->record || !sorted_vals || !ranges || !image)
        return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->record) & 15u) != 0) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t tiles = vt.tile_off[n_views];
    if (tiles >= (int64_t(1) << 31)) return MG_ERR_INVALID_ARG;
    int batch;
    if (!fwd_batch(cfg, &batch)) return MG_ERR_INVALID_ARG;
    if (batch == 128)
        launch_pdl(render_forward_kernel<false, false, false, 128>, dim3((unsigned)tiles),
            dim3(kRenderThreads), 0, (cudaStream_t)stream, vt,
            reinterpret_cast<const float4 *>(splats->record), sorted_vals, ranges, tile_order,
            cfg->bg[0], cfg->bg[1], cfg->bg[2], image, nullptr, nullptr, nullptr, nullptr, nullptr,
            nullptr, nullptr, (int64_t)0);
    else
        launch_pdl(render_forward_kernel<false, false>, dim3((unsigned)tiles), dim3(kRenderThreads),
            0, (cudaStream_t)stream, vt, reinterpret_cast<const float4 *>(splats->record),
            sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1], cfg->bg[2], image, nullptr,
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, (int64_t)0);
    return mg_host::launch_status();
}

// The render backward, resetting grad2d first (zero) or adding into it.
static mg_status render_backward(const mg_splats *splats, const uint32_t *sorted_vals,
                                 const uint32_t *ranges, const uint32_t *tile_order,
                                 const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                                 const float *final_T, const uint32_t *n_contrib,
                                 const float *dL_dimage, float *grad2d, uint64_t *counters,
                                 mg_stream_t stream, bool zero) {
    if (!splats || !splats->record || !sorted_vals || !ranges || !final_T || !n_contrib ||
        !dL_dimage || !grad2d)
        return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->record) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(grad2d) & 15u) != 0)
        return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t tiles = vt.tile_off[n_views];
    const int64_t R = vt.rec_off[n_views];
    int batch;
    if (!bwd_batch(cfg, &batch)) return MG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (zero && R > 0 &&
        mg_host::zero_async(grad2d, sizeof(float) * MG_GRAD2D_FLOATS * (size_t)R, s) != MG_OK)
        return MG_ERR_CUDA;
    const float4 *rec = reinterpret_cast<const float4 *>(splats->record);
    if (counters != nullptr)
        launch_pdl(render_backward_kernel<true>, dim3((unsigned)tiles), dim3(kRenderThreads), 0, s,
            vt, rec, sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1], cfg->bg[2], final_T,
            n_contrib, dL_dimage, grad2d, reinterpret_cast<unsigned long long *>(counters));
    else if (batch == 64)
        launch_pdl(render_backward_kernel<false, 64>, dim3((unsigned)tiles), dim3(kRenderThreads),
            0, s, vt, rec, sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1], cfg->bg[2],
            final_T, n_contrib, dL_dimage, grad2d, nullptr);
    else
        launch_pdl(render_backward_kernel<false>, dim3((unsigned)tiles), dim3(kRenderThreads), 0, s,
            vt, rec, sorted_vals, ranges, tile_order, cfg->bg[0], cfg->bg[1], cfg->bg[2], final_T,
            n_contrib, dL_dimage, grad2d, nullptr);
    return mg_host::launch_status();
}

extern "C" mg_status mg_render_backward(const mg_splats *splats, const uint32_t *sorted_vals,
                                        const uint32_t *ranges, const uint32_t *tile_order,
                                        const mg_view *views, int32_t n_views,
                                        const mg_raster_cfg *cfg,
                                        const float *final_T, const uint32_t *n_contrib,
                                        const float *dL_dimage, float *grad2d,
                                        uint64_t *counters, mg_stream_t stream) {
    return render_backward(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, final_T,
                           n_contrib, dL_dimage, grad2d, counters, stream, true);
}

extern "C" mg_status mg_render_backward_accumulate(
    const mg_splats *splats, const uint32_t *sorted_vals, const uint32_t *ranges,
    const uint32_t *tile_order, const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
    const float *final_T, const uint32_t *n_contrib, const float *dL_dimage, float *grad2d,
    uint64_t *counters, mg_stream_t stream) {
    return render_backward(splats, sorted_vals, ranges, tile_order, views, n_views, cfg, final_T,
                           n_contrib, dL_dimage, grad2d, counters, stream, false);
}

extern "C" mg_status mg_l1_loss_grad(const float *image, const float *target,
                                     const mg_view *views, int32_t n_views, float *dL_dimage,
                                     float *loss, mg_stream_t stream) {
    if (!image || !target || !dL_dimage) return MG_ERR_INVALID_ARG;
    if (((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
          reinterpret_cast<uintptr_t>(dL_dimage)) & 15u) != 0)
        return MG_ERR_INVALID_ARG;
    mg_raster_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tile_w = cfg.tile_h = 16;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, &cfg, &vt);
    if (st != MG_OK) return st;
    int64_t most = 0;
    for (int v = 0; v < n_views; ++v) most = max(most, 3 * (vt.pix_off[v + 1] - vt.pix_off[v]));
    const int64_t bx = (most + 1023) / 1024;
    const dim3 grid((unsigned)(bx < 2048 ? (bx > 0 ? bx : 1) : 2048), (unsigned)n_views);
    launch_pdl(l1_loss_grad_kernel, dim3(grid), dim3(256), 0, (cudaStream_t)stream, vt, image,
        target, dL_dimage, loss);
    return mg_host::launch_status();
}

// ---------------------------------------------------------------------------
// Longest-first tile order.  A tile's render time grows with its list length
// and one CTA renders one tile, so launching the long lists first keeps the
// SMs busy to the end (list scheduling, longest processing time first).  A
// one-block counting sort over quarter-octave buckets of the list length;
// the order inside a bucket is whatever the shared-memory atomics give (it
// changes only which CTA starts first, never a result).
// ---------------------------------------------------------------------------
namespace mg {
constexpr int kOrderBuckets = 128;

__device__ __forceinline__ int length_bucket(uint32_t c) {
    if (c < 4) return (int)c;
    const int msb = 31 - __clz(c);
    return 4 * (msb - 1) + (int)((c >> (msb - 2)) & 3u);      // 4 .. 123
}

__global__ void __launch_bounds__(1024)
tile_order_kernel(const uint32_t *__restrict__ ranges, int64_t n, uint32_t *__restrict__ order) {
    grid_dependency_wait();
    __shared__ uint32_t hist[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint2 r = reinterpret_cast<const uint2 *>(ranges)[t];
        atomicAdd(&hist[length_bucket(r.y - r.x)], 1u);
    }
    __syncthreads();
    static_assert(kOrderBuckets == 4 * 32, "one warp scans the buckets, four per lane");
    if (threadIdx.x < 32) {                       // starts, longest bucket first
        const int l = threadIdx.x;
        uint32_t c[4], own = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = hist[kOrderBuckets - 1 - (4 * l + u)];
            own += c[u];
        }
        uint32_t inc = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (l >= o) inc += y;
        }
        uint32_t run = inc - own;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            hist[kOrderBuckets - 1 - (4 * l + u)] = run;
            run += c[u];
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint2 r = reinterpret_cast<const uint2 *>(ranges)[t];
        order[atomicAdd(&hist[length_bucket(r.y - r.x)], 1u)] = (uint32_t)t;
    }
}
}  // namespace mg

extern "C" mg_status mg_tile_order(const uint32_t *ranges, int64_t n_tiles_total,
                                   uint32_t *tile_order, mg_stream_t stream) {
    if (ranges == nullptr || tile_order == nullptr || n_tiles_total <= 0 ||
        n_tiles_total >= (int64_t(1) << 31) || (reinterpret_cast<uintptr_t>(ranges) & 7u) != 0)
        return MG_ERR_INVALID_ARG;
    launch_pdl(tile_order_kernel, dim3(1), dim3(1024), 0, (cudaStream_t)stream, ranges,
        n_tiles_total, tile_order);
    return mg_host::launch_status();
}
