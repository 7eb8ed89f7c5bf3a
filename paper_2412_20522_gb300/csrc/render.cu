// Masked rasterisation, forward (Eq. 3-4) and backward (Eq. 6, Appendix A),
// and the L1 render loss.
//
// One CTA of 256 threads per tile, one thread per pixel.  The tile's
// depth-sorted splats are staged through shared memory in batches of 256
// (one 48-byte record gathered per thread), then every thread walks the batch.
// The forward skips masked splats outright: with M_i = 0 they neither add
// colour nor attenuate T (Eq. 3-4).  The backward walks the same lists back
// to front from each pixel's stop index, recovers T_i = T_{i+1}/(1 - M_i
// alpha_i), and reduces each splat's gradient over the warp with shuffles,
// over the CTA in shared memory, then issues one vector atomic per splat and
// tile.  Masked splats carry only dL/dM (one scalar reduction and atomic).
//
// alpha is evaluated by the same explicitly rounded sequence in both kernels
// so that the forward's and the backward's per-fragment decisions agree.
#include "internal.cuh"

namespace mg {

constexpr int kRenderThreads = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Frag {
    float dx, dy, p1, p2, G, araw, alpha;
};

// alpha = min(0.99, o 2^(h1 p1^2 + h2 p2^2)), p1 = d.u, p2 = d.u_perp,
// d = pixel centre - mean.  A = (mx, my, ux, uy), B = (h1, h2, o, M).
__device__ __forceinline__ void frag_alpha(const float4 &A, const float4 &B, float fpx, float fpy,
                                           Frag &f) {
    f.dx = __fsub_rn(fpx, A.x);
    f.dy = __fsub_rn(fpy, A.y);
    f.p1 = __fmaf_rn(f.dy, A.w, __fmul_rn(f.dx, A.z));
    f.p2 = __fmaf_rn(f.dy, A.z, -__fmul_rn(f.dx, A.w));
    const float e = __fmaf_rn(__fmul_rn(B.x, f.p1), f.p1, __fmul_rn(__fmul_rn(B.y, f.p2), f.p2));
    f.G = ex2_approx(e);
    f.araw = __fmul_rn(B.z, f.G);
    f.alpha = fminf(kAlphaMax, f.araw);
}

struct TileInfo {
    int v, px, py;
    bool inside;
    int64_t pix;     // pixel index within the view
};

__device__ __forceinline__ TileInfo tile_info(const ViewTable &vt, int64_t t) {
    TileInfo ti;
    ti.v = view_of_tile(vt, t);
    const int64_t lt = t - vt.tile_off[ti.v];
    const int gx = vt.gx[ti.v];
    const int tx = (int)(lt % gx), ty = (int)(lt / gx);
    ti.px = tx * vt.tile_w + (threadIdx.x & (vt.tile_w - 1));
    ti.py = ty * vt.tile_h + (threadIdx.x >> vt.log2_tw);
    const mg_camera &C = vt.cam[ti.v];
    ti.inside = ti.px < C.width && ti.py < C.height;
    ti.pix = (int64_t)ti.py * C.width + ti.px;
    return ti;
}

// COUNT = true adds per-fragment counters (an untimed diagnostic variant):
// [0] positions walked (sum of n_contrib), [1] unmasked positions walked,
// [2] unmasked splats blended, [3] masked splats above the alpha floor.
template <bool COUNT>
__global__ void __launch_bounds__(kRenderThreads)
render_forward_kernel(ViewTable vt, const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ ranges, float bg0, float bg1, float bg2,
                      float *__restrict__ image, float *__restrict__ final_T,
                      uint32_t *__restrict__ n_contrib, unsigned long long *frag_count) {
    __shared__ float4 sA[kRenderThreads], sB[kRenderThreads], sC[kRenderThreads];
    __shared__ unsigned long long s_frags[4];
    const int64_t t = blockIdx.x;
    const TileInfo ti = tile_info(vt, t);
    const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    const float fpx = (float)ti.px + 0.5f, fpy = (float)ti.py + 0.5f;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    bool done = !ti.inside;
    uint32_t stop = end - start;
    uint32_t c_unmasked = 0, c_blend = 0, c_masked = 0;
    if (threadIdx.x < 4) s_frags[threadIdx.x] = 0ull;

    for (uint32_t b0 = start; b0 < end; b0 += kRenderThreads) {
        if (__syncthreads_count(done) == kRenderThreads) break;
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < end) {
            const uint32_t r = vals[idx];
            sA[threadIdx.x] = rec[3 * (int64_t)r];
            sB[threadIdx.x] = rec[3 * (int64_t)r + 1];
            sC[threadIdx.x] = rec[3 * (int64_t)r + 2];
        }
        __syncthreads();
        const int cnt = (int)min(end - b0, (uint32_t)kRenderThreads);
        if (!done) {
            int j = 0;
            for (; j < cnt; ++j) {
                const float4 B = sB[j];
                if (B.w == 0.0f) {                  // masked: no colour, no attenuation
                    if (COUNT) {
                        Frag f;
                        frag_alpha(sA[j], B, fpx, fpy, f);
                        c_masked += f.alpha >= kAlphaMin;
                    }
                    continue;
                }
                if (COUNT) ++c_unmasked;
                Frag f;
                frag_alpha(sA[j], B, fpx, fpy, f);
                if (f.alpha < kAlphaMin) continue;
                const float testT = T * (1.0f - f.alpha);
                if (testT < kTMin) {
                    done = true;
                    stop = (b0 - start) + j;
                    if (COUNT) --c_unmasked;        // the stopping splat is not walked
                    break;
                }
                if (COUNT) ++c_blend;
                const float4 c = sC[j];
                const float w = f.alpha * T;
                C0 = fmaf(w, c.x, C0);
                C1 = fmaf(w, c.y, C1);
                C2 = fmaf(w, c.z, C2);
                T = testT;
            }
        }
    }
    if (COUNT) {
        unsigned long long c[4] = {ti.inside ? stop : 0u, c_unmasked, c_blend, c_masked};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_down_sync(0xffffffffu, c[k], o);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&s_frags[k], c[k]);
        __syncthreads();
        if (threadIdx.x < 4) atomicAdd(frag_count + threadIdx.x, s_frags[threadIdx.x]);
    }
    if (ti.inside) {
        const mg_camera &C = vt.cam[ti.v];
        const int64_t HW = (int64_t)C.width * C.height;
        float *img = image + 3 * vt.pix_off[ti.v];
        img[ti.pix] = C0 + T * bg0;
        img[HW + ti.pix] = C1 + T * bg1;
        img[2 * HW + ti.pix] = C2 + T * bg2;
        final_T[vt.pix_off[ti.v] + ti.pix] = T;
        n_contrib[vt.pix_off[ti.v] + ti.pix] = stop;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kRenderThreads)
render_backward_kernel(ViewTable vt, const float4 *__restrict__ rec,
                       const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
                       float bg0, float bg1, float bg2, const float *__restrict__ final_T,
                       const uint32_t *__restrict__ n_contrib, const float *__restrict__ dL_dimage,
                       float *__restrict__ grad2d) {
    __shared__ float4 sA[kRenderThreads], sB[kRenderThreads], sC[kRenderThreads];
    __shared__ uint32_t sR[kRenderThreads];
    __shared__ float sG[kRenderThreads][10];
    __shared__ uint32_t s_maxstop;
    const int64_t t = blockIdx.x;
    const TileInfo ti = tile_info(vt, t);
    const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
    const float fpx = (float)ti.px + 0.5f, fpy = (float)ti.py + 0.5f;
    const int lane = threadIdx.x & 31;

    float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    uint32_t stop = 0;
    if (ti.inside) {
        const mg_camera &C = vt.cam[ti.v];
        const int64_t HW = (int64_t)C.width * C.height;
        const int64_t p = vt.pix_off[ti.v] + ti.pix;
        T = final_T[p];
        stop = n_contrib[p];
        const float *gi = dL_dimage + 3 * vt.pix_off[ti.v];
        g0 = gi[ti.pix];
        g1 = gi[HW + ti.pix];
        g2 = gi[2 * HW + ti.pix];
    }
    float b0c = bg0, b1c = bg1, b2c = bg2;   // colour behind, background folded in
    if (threadIdx.x == 0) s_maxstop = 0;
    __syncthreads();
    atomicMax(&s_maxstop, stop);
    __syncthreads();
    const uint32_t maxstop = min(s_maxstop, end - start);
    if (maxstop == 0) return;
    const int nb = (int)((maxstop + kRenderThreads - 1) / kRenderThreads);

    for (int bi = nb - 1; bi >= 0; --bi) {
        const uint32_t pos0 = (uint32_t)bi * kRenderThreads;
        const int cnt = (int)min(maxstop - pos0, (uint32_t)kRenderThreads);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const uint32_t r = vals[start + pos0 + threadIdx.x];
            sR[threadIdx.x] = r;
            sA[threadIdx.x] = rec[3 * (int64_t)r];
            sB[threadIdx.x] = rec[3 * (int64_t)r + 1];
            sC[threadIdx.x] = rec[3 * (int64_t)r + 2];
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) sG[threadIdx.x][k] = 0.0f;
        __syncthreads();

        for (int j = cnt - 1; j >= 0; --j) {
            const float4 B = sB[j];
            const bool masked = B.w == 0.0f;
            float dM = 0.0f, dmx = 0.0f, dmy = 0.0f, dca = 0.0f, dcb = 0.0f, dcc = 0.0f,
                  dop = 0.0f, dr = 0.0f, dg = 0.0f, db = 0.0f;
            bool contrib = false;
            if (pos0 + j < stop) {
                const float4 A = sA[j];
                Frag f;
                frag_alpha(A, B, fpx, fpy, f);
                if (f.alpha >= kAlphaMin) {
                    contrib = true;
                    const float4 c = sC[j];
                    const float ma = masked ? 0.0f : f.alpha;
                    const float Tj = T / (1.0f - ma);
                    const float gcb = g0 * (c.x - b0c) + g1 * (c.y - b1c) + g2 * (c.z - b2c);
                    dM = f.alpha * Tj * gcb;                   // Eq. 6 + Appendix A
                    if (!masked) {
                        const float wt = f.alpha * Tj;
                        dr = wt * g0;
                        dg = wt * g1;
                        db = wt * g2;
                        b0c = fmaf(f.alpha, c.x - b0c, b0c);
                        b1c = fmaf(f.alpha, c.y - b1c, b1c);
                        b2c = fmaf(f.alpha, c.z - b2c, b2c);
                        T = Tj;
                        if (f.araw < kAlphaMax) {
                            const float dA = Tj * gcb;       // dL/dalpha (M = 1)
                            dop = dA * f.G;
                            const float dpow = dA * f.alpha;
                            dca = -0.5f * dpow * f.dx * f.dx;
                            dcb = -dpow * f.dx * f.dy;
                            dcc = -0.5f * dpow * f.dy * f.dy;
                            // Sigma^-1 d in eigen form: w_k = -2 h_k / log2(e)
                            const float q1 = (-2.0f / kLog2e) * B.x * f.p1;
                            const float q2 = (-2.0f / kLog2e) * B.y * f.p2;
                            dmx = dpow * (q1 * A.z - q2 * A.w);
                            dmy = dpow * (q1 * A.w + q2 * A.z);
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                if (masked) {
                    dM = warp_sum(dM);
                    if (lane == 0) atomicAdd(&sG[j][9], dM);
                } else {
                    dmx = warp_sum(dmx); dmy = warp_sum(dmy);
                    dca = warp_sum(dca); dcb = warp_sum(dcb); dcc = warp_sum(dcc);
                    dop = warp_sum(dop);
                    dr = warp_sum(dr); dg = warp_sum(dg); db = warp_sum(db);
                    dM = warp_sum(dM);
                    if (lane == 0) {
                        atomicAdd(&sG[j][0], dmx); atomicAdd(&sG[j][1], dmy);
                        atomicAdd(&sG[j][2], dca); atomicAdd(&sG[j][3], dcb);
                        atomicAdd(&sG[j][4], dcc); atomicAdd(&sG[j][5], dop);
                        atomicAdd(&sG[j][6], dr); atomicAdd(&sG[j][7], dg);
                        atomicAdd(&sG[j][8], db); atomicAdd(&sG[j][9], dM);
                    }
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const float *s = sG[threadIdx.x];
            float4 *G4 = reinterpret_cast<float4 *>(grad2d) + 3 * (int64_t)sR[threadIdx.x];
            if (sB[threadIdx.x].w == 0.0f) {
                if (s[9] != 0.0f) atomicAdd(&G4[2].y, s[9]);
            } else {
                if (s[0] != 0.0f || s[1] != 0.0f || s[2] != 0.0f || s[3] != 0.0f)
                    atomicAdd(&G4[0], make_float4(s[0], s[1], s[2], s[3]));
                if (s[4] != 0.0f || s[5] != 0.0f || s[6] != 0.0f || s[7] != 0.0f)
                    atomicAdd(&G4[1], make_float4(s[4], s[5], s[6], s[7]));
                if (s[8] != 0.0f || s[9] != 0.0f)
                    atomicAdd(reinterpret_cast<float2 *>(&G4[2]), make_float2(s[8], s[9]));
            }
        }
    }
}

__global__ void l1_loss_grad_kernel(ViewTable vt, const float *__restrict__ image,
                                    const float *__restrict__ target, float *__restrict__ grad,
                                    float *loss) {
    const int v = blockIdx.y;
    const int64_t n = 3 * (vt.pix_off[v + 1] - vt.pix_off[v]);
    const int64_t o = 3 * vt.pix_off[v];
    const float inv = 1.0f / (float)n;
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = image[o + i] - target[o + i];
        grad[o + i] = d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
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

extern "C" mg_status mg_render(const mg_splats *splats, const uint32_t *sorted_vals,
                               const uint32_t *ranges, const mg_view *views, int32_t n_views,
                               const mg_raster_cfg *cfg, float *image, float *final_T,
                               uint32_t *n_contrib, uint64_t *frag_count, mg_stream_t stream) {
    if (!splats || !splats->record || !sorted_vals || !ranges || !image || !final_T || !n_contrib)
        return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->record) & 15u) != 0) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t tiles = vt.tile_off[n_views];
    if (tiles >= (int64_t(1) << 31)) return MG_ERR_INVALID_ARG;
    const float4 *rec = reinterpret_cast<const float4 *>(splats->record);
    if (frag_count != nullptr)
        render_forward_kernel<true><<<(unsigned)tiles, kRenderThreads, 0, (cudaStream_t)stream>>>(
            vt, rec, sorted_vals, ranges, cfg->bg[0], cfg->bg[1], cfg->bg[2], image, final_T,
            n_contrib, reinterpret_cast<unsigned long long *>(frag_count));
    else
        render_forward_kernel<false><<<(unsigned)tiles, kRenderThreads, 0, (cudaStream_t)stream>>>(
            vt, rec, sorted_vals, ranges, cfg->bg[0], cfg->bg[1], cfg->bg[2], image, final_T,
            n_contrib, nullptr);
    return mg_host::launch_status();
}

extern "C" mg_status mg_render_backward(const mg_splats *splats, const uint32_t *sorted_vals,
                                        const uint32_t *ranges, const mg_view *views,
                                        int32_t n_views, const mg_raster_cfg *cfg,
                                        const float *final_T, const uint32_t *n_contrib,
                                        const float *dL_dimage, float *grad2d,
                                        mg_stream_t stream) {
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
    cudaStream_t s = (cudaStream_t)stream;
    if (R > 0 && cudaMemsetAsync(grad2d, 0, sizeof(float) * MG_GRAD2D_FLOATS * (size_t)R, s) !=
                     cudaSuccess)
        return MG_ERR_CUDA;
    render_backward_kernel<<<(unsigned)tiles, kRenderThreads, 0, s>>>(
        vt, reinterpret_cast<const float4 *>(splats->record), sorted_vals, ranges, cfg->bg[0],
        cfg->bg[1], cfg->bg[2], final_T, n_contrib, dL_dimage, grad2d);
    return mg_host::launch_status();
}

extern "C" mg_status mg_l1_loss_grad(const float *image, const float *target,
                                     const mg_view *views, int32_t n_views, float *dL_dimage,
                                     float *loss, mg_stream_t stream) {
    if (!image || !target || !dL_dimage) return MG_ERR_INVALID_ARG;
    mg_raster_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.tile_w = cfg.tile_h = 16;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, &cfg, &vt);
    if (st != MG_OK) return st;
    const dim3 grid(152, (unsigned)n_views);
    l1_loss_grad_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(vt, image, target, dL_dimage,
                                                               loss);
    return mg_host::launch_status();
}
