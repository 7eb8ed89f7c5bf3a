// Host-side helpers of the C ABI: argument checks, the view table, status.
#include <math.h>
#include <string.h>

#include "internal.cuh"

namespace mg {

// words [0, n) of p set to 0: 128-bit stores over the 16-byte aligned body,
// 32-bit ones at the ends
__global__ void zero_kernel(uint32_t *__restrict__ p, int64_t n) {
    grid_dependency_wait();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int64_t head = (int64_t)(((16u - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) / 4u);
    if (head > n) head = n;
    const int64_t n4 = (n - head) / 4;
    for (int64_t i = t; i < head; i += nt) p[i] = 0u;
    uint4 *q = reinterpret_cast<uint4 *>(p + head);
    for (int64_t i = t; i < n4; i += nt) q[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = head + 4 * n4 + t; i < n; i += nt) p[i] = 0u;
}

}  // namespace mg

namespace mg_host {

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

mg_status build_view_table(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                           mg::ViewTable *vt) {
    if (views == nullptr || cfg == nullptr || vt == nullptr) return MG_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > MG_MAX_VIEWS) return MG_ERR_INVALID_ARG;
    // 256-pixel tiles made of four 8x8 warp blocks: 16x16, 32x8 or 8x32
    if (!pow2(cfg->tile_w) || !pow2(cfg->tile_h) || cfg->tile_w * cfg->tile_h != mg::kTilePixels ||
        cfg->tile_w < 8 || cfg->tile_h < 8)
        return MG_ERR_INVALID_ARG;
    memset(vt, 0, sizeof(*vt));
    vt->n_views = n_views;
    vt->tile_w = cfg->tile_w;
    vt->tile_h = cfg->tile_h;
    int l = 0;
    while ((1 << l) < cfg->tile_w) ++l;
    vt->log2_tw = l;
    for (int v = 0; v < n_views; ++v) {
        const mg_view &w = views[v];
        if (w.cam.width <= 0 || w.cam.height <= 0 || w.gaussian_offset < 0 ||
            w.gaussian_count < 0 || !(w.cam.fx > 0.0f) || !(w.cam.fy > 0.0f))
            return MG_ERR_INVALID_ARG;
        vt->cam[v] = w.cam;
        vt->g_off[v] = w.gaussian_offset;
        vt->g_cnt[v] = w.gaussian_count;
        vt->gx[v] = (w.cam.width + cfg->tile_w - 1) / cfg->tile_w;
        vt->gy[v] = (w.cam.height + cfg->tile_h - 1) / cfg->tile_h;
        // FP32 operations, each correctly rounded (no product is added, so
        // nothing can be contracted): the values the device would compute
        const float tanx = ((float)w.cam.width * 0.5f) / w.cam.fx;
        const float tany = ((float)w.cam.height * 0.5f) / w.cam.fy;
        vt->limx[v] = 1.3f * tanx;
        vt->limy[v] = 1.3f * tany;
        vt->rec_off[v + 1] = vt->rec_off[v] + w.gaussian_count;
        vt->tile_off[v + 1] = vt->tile_off[v] + (int64_t)vt->gx[v] * vt->gy[v];
        vt->pix_off[v + 1] = vt->pix_off[v] + (int64_t)w.cam.width * w.cam.height;
    }
    return MG_OK;
}

mg_status launch_status(void) {
    return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

mg_status zero_async(void *p, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return MG_OK;
    if (p == nullptr || (bytes & 3u) != 0 || (reinterpret_cast<uintptr_t>(p) & 3u) != 0)
        return MG_ERR_INVALID_ARG;
    const int64_t words = (int64_t)(bytes / 4);
    const int64_t blocks = (words / 4 + 255) / 256;
    const int64_t cap = 4 * 152;
    mg::launch_pdl(mg::zero_kernel, dim3((unsigned)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap))),
                   dim3(256), 0, s, static_cast<uint32_t *>(p), words);
    return launch_status();
}

}  // namespace mg_host

extern "C" {

int64_t mg_total_tiles(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg) {
    mg::ViewTable vt;
    if (mg_host::build_view_table(views, n_views, cfg, &vt) != MG_OK) return -1;
    return vt.tile_off[n_views];
}

int32_t mg_tile_bits(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg) {
    const int64_t t = mg_total_tiles(views, n_views, cfg);
    if (t <= 0) return -1;
    int b = 0;
    while ((int64_t(1) << b) < t) ++b;
    return b > 0 ? b : 1;
}

mg_status mg_read_status(const mg_status_word *d_status, mg_status_word *h_out,
                         mg_stream_t stream) {
    if (d_status == nullptr || h_out == nullptr) return MG_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(h_out, d_status, sizeof(mg_status_word), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess)
        return MG_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MG_ERR_CUDA;
    return MG_OK;
}

const char *mg_status_string(int32_t status) {
    switch (status) {
        case MG_OK: return "ok";
        case MG_ERR_INVALID_ARG: return "invalid argument";
        case MG_ERR_CUDA: return "CUDA error";
        case MG_ERR_CAPACITY: return "instance capacity exceeded";
        case MG_ERR_BOUNDS: return "index or range outside its buffer";
        case MG_ERR_TIMEOUT: return "device-side wait timed out";
        case MG_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char *mg_version(void) { return "maskgs 0.1.0 (sm_103a)"; }

}  // extern "C"

// Self-test of the bounded device-side waits: one thread runs the look-back
// every cross-block wait of the library uses, for partition 1 of a status
// array whose partition 0 never publishes; after max_polls polls it gives up
// and raises MG_ERR_TIMEOUT (detail 4) in the status word.
namespace mg {
__global__ void selftest_wait_kernel(int max_polls, mg_status_word *st) {
    __shared__ uint64_t status[2];
    status[0] = 0;                    // partition 0: nothing ever published
    status[1] = 0;
    lookback<uint64_t, 62>(status, 1, 1, st, 4, max_polls);
}

// The same for the warp-wide look-back of the single-pass scans (one warp,
// partition 40 of an array where nothing is published; detail 5).
__global__ void selftest_warp_wait_kernel(int max_polls, mg_status_word *st) {
    __shared__ uint64_t status[41];
    for (int i = threadIdx.x; i < 41; i += 32) status[i] = 0;
    __syncwarp();
    warp_lookback64(status, 40, st, 5, max_polls);
}
}  // namespace mg

extern "C" {

mg_status mg_selftest_wait_timeout(int32_t max_polls, mg_status_word *d_status,
                                   mg_stream_t stream) {
    if (d_status == nullptr || max_polls < 0 || max_polls > (1 << 24)) return MG_ERR_INVALID_ARG;
    mg::selftest_wait_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(max_polls, d_status);
    return mg_host::launch_status();
}

mg_status mg_selftest_warp_wait_timeout(int32_t max_polls, mg_status_word *d_status,
                                        mg_stream_t stream) {
    if (d_status == nullptr || max_polls < 0 || max_polls > (1 << 24)) return MG_ERR_INVALID_ARG;
    mg::selftest_warp_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(max_polls, d_status);
    return mg_host::launch_status();
}

}  // extern "C"
