// Internal device helpers of libmaskgs (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/maskgs.h"

namespace mg {

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLowpass = 0.3f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kTilePixels = 256;
constexpr int kMaxTimeoutSpins = 1 << 22;   // bounded waits: ~4M polls, then give up

// Views in kernel parameter space (captured by value in CUDA graphs).
struct ViewTable {
    int32_t n_views;
    int32_t tile_w, tile_h, log2_tw;
    mg_camera cam[MG_MAX_VIEWS];
    int64_t g_off[MG_MAX_VIEWS];     // first Gaussian of the view
    int64_t g_cnt[MG_MAX_VIEWS];     // Gaussians seen by the view
    int64_t rec_off[MG_MAX_VIEWS + 1];   // first record of the view
    int64_t tile_off[MG_MAX_VIEWS + 1];  // first global tile of the view
    int64_t pix_off[MG_MAX_VIEWS + 1];   // first pixel of the view
    int32_t gx[MG_MAX_VIEWS], gy[MG_MAX_VIEWS];
    // clamp limits of the Jacobian's point, 1.3 tan(fov/2) = 1.3 ((W/2) / fx)
    // (and the same in y), each FP32 operation correctly rounded on the host
    float limx[MG_MAX_VIEWS], limy[MG_MAX_VIEWS];
};

// device status word helpers -------------------------------------------------
__device__ __forceinline__ void raise_status(mg_status_word *w, int32_t st, int32_t detail,
                                             uint64_t required) {
    if (w == nullptr) return;
    atomicCAS(&w->status, 0, st);
    atomicMax((unsigned long long *)&w->required, (unsigned long long)required);
    atomicCAS(&w->detail, 0, detail);
}

// Bounds checks of the debug build (MG_DEBUG_BOUNDS): true when the access
// may go ahead; otherwise MG_ERR_BOUNDS is raised with the offending value
// and the caller skips the access.  In the ordinary build the test is not
// compiled.
#ifdef MG_DEBUG_BOUNDS
#define MG_IN_BOUNDS(cond, st, detail, value)                                                   \
    ((cond) ? true : (::mg::raise_status((st), MG_ERR_BOUNDS, (detail), (uint64_t)(value)), false))
#else
#define MG_IN_BOUNDS(cond, st, detail, value) true
#endif

// Programmatic dependent launch.  The step's kernels are launched with
// launch_pdl, which lets the next kernel on the stream be scheduled while
// the previous one drains; each of them first waits in
// grid_dependency_wait until the previous kernel has completed and its
// writes are visible (for a kernel launched the ordinary way, or after a
// memset or copy, the wait returns at once and stream order holds as usual).
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // every CTA of this kernel has started once all of them get here: the
    // next kernel may then be scheduled onto the SMs this one frees (its
    // own wait still holds it until this kernel has completed)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// single-pass scans (decoupled look-back) ------------------------------------
// A partition's 64-bit status word: flag in the top two bits (1 = aggregate
// only, 2 = inclusive prefix), value below.
constexpr uint64_t kFlagAgg64 = 1ull << 62, kFlagPrefix64 = 2ull << 62,
                   kValMask64 = (1ull << 62) - 1ull;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ uint64_t ld_volatile(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

__device__ __forceinline__ uint64_t block_exclusive_scan_u64(uint64_t v, uint64_t *sm_warp,
                                                             uint64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sm_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (int)(blockDim.x >> 5) ? sm_warp[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)(blockDim.x >> 5)) sm_warp[lane] = wi - w;
        if (lane == 31) sm_warp[32] = wi;
    }
    __syncthreads();
    total = sm_warp[32];
    return sm_warp[warp] + inc - v;
}

// Decoupled look-back: the exclusive prefix of partition `part` from the
// status words of its predecessors (word of partition q at status[q * stride]),
// summing aggregates back to the first inclusive prefix.  kLookbackWindow
// predecessors are read at once, so a walk over published aggregates costs
// one memory round trip per window instead of one per partition.  A word not
// yet published is polled at most kMaxTimeoutSpins times; then MG_ERR_TIMEOUT
// (with `detail`) is raised and the partial sum returned.
constexpr int kLookbackWindow = 8;

template <typename W, int FLAG_SHIFT>
__device__ __forceinline__ W lookback(const W *status, int64_t stride, int64_t part,
                                      mg_status_word *st, int32_t detail,
                                      int max_spins = kMaxTimeoutSpins) {
    constexpr W kMask = (W(1) << FLAG_SHIFT) - W(1);
    W excl = 0;
    int64_t q = part - 1;
    while (q >= 0) {
        W s[kLookbackWindow];
#pragma unroll
        for (int k = 0; k < kLookbackWindow; ++k)
            s[k] = (q - k >= 0) ? ld_volatile(status + (q - k) * stride) : W(0);
#pragma unroll
        for (int k = 0; k < kLookbackWindow; ++k) {
            if (q - k < 0) return excl;
            int spins = 0;
            while ((s[k] >> FLAG_SHIFT) == 0 && spins < max_spins) {
                __nanosleep(20);
                s[k] = ld_volatile(status + (q - k) * stride);
                ++spins;
            }
            if ((s[k] >> FLAG_SHIFT) == 0) {
                raise_status(st, MG_ERR_TIMEOUT, detail, 0);
                return excl;
            }
            excl += s[k] & kMask;
            if ((s[k] >> FLAG_SHIFT) == 2) return excl;
        }
        q -= kLookbackWindow;
    }
    return excl;
}

// Warp-wide decoupled look-back over 64-bit status words (flag in bits
// 62-63, value below): the calling warp reads its 32 nearest predecessors at
// once, waits only for those up to the nearest inclusive prefix, and sums
// them; it moves to the next 32 only while none of them holds an inclusive
// prefix -- a walk over published aggregates costs one round trip per 32
// partitions.  Called by all 32 lanes of one warp; every lane returns the
// exclusive prefix.  Waits are bounded as in lookback().
__device__ __forceinline__ uint64_t warp_lookback64(const uint64_t *status, int64_t part,
                                                    mg_status_word *st, int32_t detail,
                                                    int max_spins = kMaxTimeoutSpins) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    constexpr uint64_t kMask = (1ull << 62) - 1ull;
    uint64_t excl = 0;
    for (int64_t q = part - 1; q >= 0; q -= 32) {
        const int64_t idx = q - lane;
        // before partition 0: an empty inclusive prefix
        uint64_t s = idx >= 0 ? ld_volatile(status + idx) : kFlagPrefix64;
        for (int spins = 0;; ++spins) {
            const unsigned inc = __ballot_sync(FULL, (s >> 62) == 2u);
            // lanes up to the nearest inclusive prefix (lane 0 is the nearest)
            const unsigned need = inc ? (2u << (__ffs(inc) - 1)) - 1u : FULL;
            const unsigned missing = __ballot_sync(FULL, (s >> 62) == 0u) & need;
            if (missing == 0u) {
                uint64_t v = ((need >> lane) & 1u) ? (s & kMask) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                excl += v;
                if (inc) return excl;
                break;
            }
            if (spins >= max_spins) {
                if (lane == 0) raise_status(st, MG_ERR_TIMEOUT, detail, 0);
                return excl;
            }
            __nanosleep(20);
            if ((missing >> lane) & 1u) s = ld_volatile(status + idx);
        }
    }
    return excl;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float uniform24(uint32_t x) {
    return __fmul_rn((float)(((x >> 9) << 1) | 1u), 0x1p-24f);
}

// ---------------------------------------------------------------------------
// Own FP32 log / exp for decisions, each step one correctly rounded op.
// log: x = m 2^e, m in [1/sqrt2, sqrt2), log m = 2 atanh((m-1)/(m+1)) by its
// series to s^11/11, Cody-Waite split of ln 2.
// exp: x = k ln2 + r, Taylor series of exp(r) to r^7/7!, times 2^k.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float log32(float x) {
    const uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
    if (m >= 0x1.6a09e6p+0f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fadd_rn(m, -1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = 0x1.745d18p-4f;
    p = __fadd_rn(__fmul_rn(p, z), 0x1.c71c72p-4f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.24924ap-3f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.99999ap-3f);
    p = __fadd_rn(__fmul_rn(p, z), 0x1.555556p-2f);
    p = __fadd_rn(__fmul_rn(p, z), 1.0f);
    const float lm = __fmul_rn(__fmul_rn(s, 2.0f), p);
    const float ef = (float)e;
    return __fadd_rn(__fmul_rn(ef, 0x1.62e4p-1f), __fadd_rn(__fmul_rn(ef, 0x1.7f7d1cp-20f), lm));
}

__device__ __forceinline__ float exp32(float x) {
    // clamp to [-80, 80] by comparisons: a NaN stays NaN (fminf/fmaxf drop it)
    x = x < -80.0f ? -80.0f : (x > 80.0f ? 80.0f : x);
    const float k = rintf(__fmul_rn(x, 0x1.715476p+0f));
    const float r = __fadd_rn(__fadd_rn(x, -__fmul_rn(k, 0x1.62e4p-1f)), -__fmul_rn(k, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = __fadd_rn(__fmul_rn(p, r), 0x1.6c16c2p-10f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    const float two_k = __uint_as_float((uint32_t)((int)k + 127) << 23);
    return __fmul_rn(p, two_k);
}

// exact-rounding shorthands for the decision path
__device__ __forceinline__ float ad(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sb(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ml(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dv(float a, float b) { return __fdiv_rn(a, b); }
// (a*b + c*d) + e*f with every product and sum rounded
// Mask sample of Sec. 3.3.  Noise block of Gaussian i for one draw: Philox
// counter (i, iteration_lo, iteration_hi, draw), key (seed_lo, seed_hi); the
// training sample is draw 0, the pruning draws of Sec. 3.5 are 1, 2, ...
__device__ __forceinline__ uint4 gumbel_counter(int64_t i, uint64_t iteration, uint32_t draw,
                                                uint64_t seed) {
    return philox4x32_10(
        make_uint4((uint32_t)i, (uint32_t)iteration, (uint32_t)(iteration >> 32), draw),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Gumbel-max margin (l_0 + g_0) - (l_1 + g_1), g_k = -log(-log u_k), every
// operation correctly rounded FP32 (M = 1 iff the margin is >= 0).
__device__ __forceinline__ float gumbel_margin(float2 l, uint4 x) {
    const float g0 = -log32(-log32(uniform24(x.x)));
    const float g1 = -log32(-log32(uniform24(x.y)));
    return sb(ad(l.x, g0), ad(l.y, g1));
}

__device__ __forceinline__ float dot3(float a, float b, float c, float d, float e, float f) {
    return ad(ad(ml(a, b), ml(c, d)), ml(e, f));
}

// 2^-k for v = 2^k (the tile sizes): x / v correctly rounded equals x * 2^-k
// correctly rounded (both round the same real number), so the divisions by a
// tile size below are exact multiplications.
__device__ __forceinline__ float inv_pow2(int v) {
    return __int_as_float((127 - (31 - __clz(v))) << 23);
}

// Rectangle of tiles overlapped by the square [p - r, p + r] (inclusive),
// clamped to the grid; false when empty.
__device__ __forceinline__ bool tile_rect(float px, float py, float rf, int tw, int th, int gx,
                                          int gy, int &x0, int &x1, int &y0, int &y1) {
    const float itw = inv_pow2(tw), ith = inv_pow2(th);
    const float fx0 = fmaxf(floorf(ml(sb(px, rf), itw)), 0.0f);
    const float fx1 = fminf(floorf(ml(ad(px, rf), itw)), (float)(gx - 1));
    const float fy0 = fmaxf(floorf(ml(sb(py, rf), ith)), 0.0f);
    const float fy1 = fminf(floorf(ml(ad(py, rf), ith)), (float)(gy - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return false;
    x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
    return true;
}

// Real SH basis with the Condon-Shortley phase, m = -l..l, degree <= 3.
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f, kSH2b = 0.31539156525252005f,
                kSH2c = 0.5462742152960396f;
constexpr float kSH3a = 0.5900435899266435f, kSH3b = 2.890611442640554f,
                kSH3c = 0.4570457994644658f, kSH3d = 0.3731763325901154f,
                kSH3e = 1.445305721320277f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = kSH0;
    if (deg < 1) return;
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    Y[4] = kSH2a * xy;
    Y[5] = -kSH2a * yz;
    Y[6] = kSH2b * (3.0f * zz - 1.0f);
    Y[7] = -kSH2a * xz;
    Y[8] = kSH2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kSH3a * y * (3.0f * xx - yy);
    Y[10] = kSH3b * xy * z;
    Y[11] = -kSH3c * y * (5.0f * zz - 1.0f);
    Y[12] = kSH3d * z * (5.0f * zz - 3.0f);
    Y[13] = -kSH3c * x * (5.0f * zz - 1.0f);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.0f * yy);
}

// d Y_k / d(x, y, z) for the same basis (direction not yet normalised out).
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float *dx,
                                              float *dy, float *dz) {
    dx[0] = dy[0] = dz[0] = 0.0f;
    if (deg < 1) return;
    dx[1] = 0.0f;  dy[1] = -kSH1;  dz[1] = 0.0f;
    dx[2] = 0.0f;  dy[2] = 0.0f;   dz[2] = kSH1;
    dx[3] = -kSH1; dy[3] = 0.0f;   dz[3] = 0.0f;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dx[4] = kSH2a * y;          dy[4] = kSH2a * x;           dz[4] = 0.0f;
    dx[5] = 0.0f;               dy[5] = -kSH2a * z;          dz[5] = -kSH2a * y;
    dx[6] = 0.0f;               dy[6] = 0.0f;                dz[6] = 6.0f * kSH2b * z;
    dx[7] = -kSH2a * z;         dy[7] = 0.0f;                dz[7] = -kSH2a * x;
    dx[8] = 2.0f * kSH2c * x;   dy[8] = -2.0f * kSH2c * y;   dz[8] = 0.0f;
    if (deg < 3) return;
    dx[9] = -kSH3a * 6.0f * x * y;            dy[9] = -kSH3a * 3.0f * (xx - yy);       dz[9] = 0.0f;
    dx[10] = kSH3b * y * z;                   dy[10] = kSH3b * x * z;                  dz[10] = kSH3b * x * y;
    dx[11] = 0.0f;                            dy[11] = -kSH3c * (5.0f * zz - 1.0f);    dz[11] = -kSH3c * 10.0f * y * z;
    dx[12] = 0.0f;                            dy[12] = 0.0f;                           dz[12] = kSH3d * (15.0f * zz - 3.0f);
    dx[13] = -kSH3c * (5.0f * zz - 1.0f);     dy[13] = 0.0f;                           dz[13] = -kSH3c * 10.0f * x * z;
    dx[14] = kSH3e * 2.0f * x * z;            dy[14] = -kSH3e * 2.0f * y * z;          dz[14] = kSH3e * (xx - yy);
    dx[15] = -kSH3a * 3.0f * (xx - yy);       dy[15] = kSH3a * 6.0f * x * y;           dz[15] = 0.0f;
}

// Tile filter of the binning (Sec. 3.1: only Gaussians whose alpha reaches
// the floor take part): drop a Gaussian from a tile of its rectangle when its
// quadratic form q = d^T Sigma_bar^-1 d exceeds 2 ln 255 at every pixel centre
// of the tile -- there alpha = o exp(-q/2) < 1/255 for any opacity o <= 1,
// so the pair is a no-op and dropping it changes no result.  The minimum of
// N = c dx^2 - 2 b dx dy + a dy^2 = det q over the box of pixel centres is 0
// if the mean is inside, else the least of the four edges' minima at their
// clamped stationary points; the pair is kept if N <= 11.1 det + 1e-4 (sum
// of |terms|) (11.1 > 2 ln 255; the slack covers N's rounding).  Every
// operation is a correctly rounded FP32 one, in a fixed order, so the
// decision is reproducible bit for bit.
constexpr float kBinThreshold = 11.1f;
constexpr float kBinRelSlack = 1e-4f;

__device__ __forceinline__ bool bin_edge_hit(float t1, float t2, float t3, float tdet) {
    const float t22 = ad(t2, t2);
    const float N = ad(sb(t1, t22), t3);
    const float bnd = ad(ad(t1, fabsf(t22)), t3);
    return N <= ad(tdet, ml(kBinRelSlack, bnd));
}

__device__ __forceinline__ bool bin_tile_hit(float px, float py, float a, float b, float c,
                                             float tdet, float rba, float rbc, int tx, int ty,
                                             int tw, int th) {
    const float X0 = ad((float)(tx * tw), 0.5f), Y0 = ad((float)(ty * th), 0.5f);
    const float X1 = ad(X0, (float)(tw - 1)), Y1 = ad(Y0, (float)(th - 1));
    const float dx0 = sb(X0, px), dx1 = sb(X1, px), dy0 = sb(Y0, py), dy1 = sb(Y1, py);
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return true;
    bool hit = false;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dxe = e ? dx1 : dx0;
        const float dyc = fminf(fmaxf(ml(rba, dxe), dy0), dy1);
        hit |= bin_edge_hit(ml(c, ml(dxe, dxe)), ml(ml(b, dxe), dyc), ml(a, ml(dyc, dyc)), tdet);
        const float dye = e ? dy1 : dy0;
        const float dxc = fminf(fmaxf(ml(rbc, dye), dx0), dx1);
        hit |= bin_edge_hit(ml(c, ml(dxc, dxc)), ml(ml(b, dxc), dye), ml(a, ml(dye, dye)), tdet);
    }
    return hit;
}

// Candidate tiles of the filtered binning: the tiles of the 3-sigma
// rectangle [x0, x1] x [y0, y1] that meet the bounding box of
// d^T M' d <= T, M' = [[c sqrt(kappa), -b], [-b, a sqrt(kappa)]],
// T = 11.1 det, an ellipse that holds every point where the filter can keep
// a tile (its test N <= 11.1 det + 1e-4 S, N rounded by at most 4 eps S,
// S <= 2 (c dx^2 + a dy^2), so kappa = 0.9995 <= (1 - 2.005e-4)^2 covers the
// slack).  Box half-widths sqrt(T a / det'), sqrt(T c / det'),
// det' = kappa a c - b^2, in correctly rounded FP32 in a fixed order
// (reproducible bit for bit), only where det' >= 1e-3 a c (its rounding then
// stays below 2e-4 of it), grown by 1e-3 relative and 0.05 px (the rounding
// of det', of the filter's offsets and of px -+ h); elsewhere the rectangle
// stays.  False when no tile remains.
constexpr float kCandKappa = 0.9995f;
constexpr float kCandMinDet = 1e-3f;
constexpr float kCandGrow = 1.001f;
constexpr float kCandMargin = 0.05f;

__device__ __forceinline__ bool candidate_rect(float px, float py, float a, float b, float c,
                                               float tdet, int tw, int th, int &x0, int &x1,
                                               int &y0, int &y1) {
    const float ac = __fmul_rn(a, c);
    const float detk = __fsub_rn(__fmul_rn(kCandKappa, ac), __fmul_rn(b, b));
    if (!(detk > __fmul_rn(kCandMinDet, ac))) return true;
    const float T = __fmul_rn(tdet, kCandGrow);
    const float hx = __fadd_rn(
        __fmul_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(T, a), detk)), kCandGrow), kCandMargin);
    const float hy = __fadd_rn(
        __fmul_rn(__fsqrt_rn(__fdiv_rn(__fmul_rn(T, c), detk)), kCandGrow), kCandMargin);
    const float itw = inv_pow2(tw), ith = inv_pow2(th);
    const float fx0 = fmaxf((float)x0, floorf(__fmul_rn(__fsub_rn(px, hx), itw)));
    const float fx1 = fminf((float)x1, floorf(__fmul_rn(__fadd_rn(px, hx), itw)));
    const float fy0 = fmaxf((float)y0, floorf(__fmul_rn(__fsub_rn(py, hy), ith)));
    const float fy1 = fminf((float)y1, floorf(__fmul_rn(__fadd_rn(py, hy), ith)));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return false;
    x0 = (int)fx0;
    x1 = (int)fx1;
    y0 = (int)fy0;
    y1 = (int)fy1;
    return true;
}

__host__ __device__ __forceinline__ int view_of_tile(const ViewTable &vt, int64_t t) {
    int v = 0;
    while (v + 1 < vt.n_views && vt.tile_off[v + 1] <= t) ++v;
    return v;
}

}  // namespace mg

// host-side helpers shared by the entry points
namespace mg_host {
mg_status build_view_table(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                           mg::ViewTable *vt);
mg_status launch_status(void);
// Zero `bytes` (a multiple of 4, at a 4-byte aligned address) on the stream
// with a kernel launched like the step's kernels (launch_pdl), in place of a
// memset node between two of them.
mg_status zero_async(void *p, size_t bytes, cudaStream_t s);
}
