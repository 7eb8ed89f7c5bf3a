// Pruning (Sec. 3.5): every Gaussian is sampled n times (the paper: 10) and
// the ones never sampled present are removed.
//
//   prune_sample   one thread per Gaussian, the draws of the training sampler
//                  with counter word 3 = 1..n (the training sample is draw 0),
//                  stopping at the first 'present' (the OR is decided then)
//   compact scan   single-pass exclusive scan of the keep flags with decoupled
//                  look-back: new_index[i] = row of i among the survivors, -1
//                  if removed, and the survivor count
//   compact copy   every attribute array, rows of its own width, copied by
//                  the widest aligned word (16, 8, 4 or 2 bytes) that divides
//                  the row: reads and writes stay contiguous, and the sectors
//                  of removed rows are not read
//
// Every cross-block wait is bounded (MG_ERR_TIMEOUT, detail 3).
#include "internal.cuh"

namespace mg {

constexpr int kPruneThreads = 256;
constexpr int kCompactThreads = 256, kCompactItems = 16,
              kCompactPart = kCompactThreads * kCompactItems;
constexpr int kCopyRows = 256;
constexpr int kAttrs = 6;

__global__ void __launch_bounds__(kPruneThreads)
prune_sample_kernel(const float2 *__restrict__ logits, int64_t n, uint64_t seed,
                    uint64_t iteration, int32_t n_draws, uint8_t *__restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * kPruneThreads + threadIdx.x;
    if (i >= n) return;
    const float2 l = __ldg(logits + i);
    uint8_t k = 0;
    for (int d = 1; d <= n_draws && k == 0; ++d)
        k = gumbel_margin(l, gumbel_counter(i, iteration, (uint32_t)d, seed)) >= 0.0f ? 1 : 0;
    keep[i] = k;
}

struct CompactWS {
    uint32_t counter;
    uint32_t pad;
    uint64_t status[1];   // [n_parts]
};

__global__ void __launch_bounds__(kCompactThreads)
compact_scan_kernel(const uint8_t *__restrict__ keep, int64_t n, int32_t *__restrict__ new_index,
                    int64_t *d_n_kept, CompactWS *ws, int64_t n_parts, mg_status_word *st) {
    __shared__ uint64_t sm_warp[33];
    __shared__ uint64_t sm_prefix;
    __shared__ int64_t sm_part;
    if (threadIdx.x == 0) sm_part = atomicAdd(&ws->counter, 1u);
    __syncthreads();
    const int64_t part = sm_part;
    if (part >= n_parts) return;
    const int64_t base = part * kCompactPart + (int64_t)threadIdx.x * kCompactItems;
    uint8_t f[kCompactItems];
    if (base + kCompactItems <= n && (reinterpret_cast<uintptr_t>(keep + base) & 15u) == 0) {
        const uint4 w = *reinterpret_cast<const uint4 *>(keep + base);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k) f[k] = (uint8_t)((words[k >> 2] >> (8 * (k & 3))) & 0xFFu);
    } else {
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k) f[k] = (base + k < n) ? keep[base + k] : 0;
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) cnt += f[k] != 0;
    uint64_t agg;
    const uint64_t excl = block_exclusive_scan_u64(cnt, sm_warp, agg);
    if (threadIdx.x < 32) {   // warp 0 publishes and looks back
        uint64_t prefix = 0;
        if (part == 0) {
            if (threadIdx.x == 0)
                atomicExch((unsigned long long *)&ws->status[0],
                           (unsigned long long)(kFlagPrefix64 | agg));
        } else {
            if (threadIdx.x == 0)
                atomicExch((unsigned long long *)&ws->status[part],
                           (unsigned long long)(kFlagAgg64 | agg));
            prefix = warp_lookback64(ws->status, part, st, 3);
            if (threadIdx.x == 0)
                atomicExch((unsigned long long *)&ws->status[part],
                           (unsigned long long)(kFlagPrefix64 | (prefix + agg)));
        }
        if (threadIdx.x == 0) sm_prefix = prefix;
        if (threadIdx.x == 0 && part == n_parts - 1) *d_n_kept = (int64_t)(prefix + agg);
    }
    __syncthreads();
    int32_t run = (int32_t)(sm_prefix + excl);
    int32_t out[kCompactItems];
#pragma unroll
    for (int k = 0; k < kCompactItems; ++k) {
        out[k] = f[k] ? run : -1;
        run += f[k] != 0;
    }
    if (base + kCompactItems <= n && (reinterpret_cast<uintptr_t>(new_index + base) & 15u) == 0) {
        int4 *o4 = reinterpret_cast<int4 *>(new_index + base);
#pragma unroll
        for (int q = 0; q < kCompactItems / 4; ++q)
            o4[q] = make_int4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k)
            if (base + k < n) new_index[base + k] = out[k];
    }
}

struct AttrCopy {
    const char *src;
    char *dst;
    int32_t row_bytes;
    int32_t word;         // 16, 8, 4 or 2
};

struct CopyArgs {
    AttrCopy a[kAttrs];
};

template <typename W>
__device__ __forceinline__ void copy_rows(const AttrCopy &A, const int32_t *sidx, int64_t r0,
                                          int nrows) {
    const int wpr = A.row_bytes / (int)sizeof(W);
    const W *src = reinterpret_cast<const W *>(A.src) + r0 * wpr;
    W *dst = reinterpret_cast<W *>(A.dst);
    const int total = nrows * wpr;
    for (int f = threadIdx.x; f < total; f += kCopyRows) {
        const int row = f / wpr;
        const int32_t j = sidx[row];
        if (j >= 0) dst[(int64_t)j * wpr + (f - row * wpr)] = src[f];
    }
}

__global__ void __launch_bounds__(kCopyRows)
compact_copy_kernel(CopyArgs args, const int32_t *__restrict__ new_index, int64_t n) {
    __shared__ int32_t sidx[kCopyRows];
    __shared__ int s_any;
    const int64_t r0 = (int64_t)blockIdx.x * kCopyRows;
    const int nrows = (int)(n - r0 < kCopyRows ? n - r0 : kCopyRows);
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    const int32_t j = threadIdx.x < nrows ? new_index[r0 + threadIdx.x] : -1;
    sidx[threadIdx.x] = j;
    if (j >= 0) s_any = 1;
    __syncthreads();
    if (!s_any) return;                       // every row of the block removed
#pragma unroll 1
    for (int a = 0; a < kAttrs; ++a) {
        const AttrCopy &A = args.a[a];
        switch (A.word) {
            case 16: copy_rows<uint4>(A, sidx, r0, nrows); break;
            case 8: copy_rows<uint2>(A, sidx, r0, nrows); break;
            case 4: copy_rows<uint32_t>(A, sidx, r0, nrows); break;
            default: copy_rows<uint16_t>(A, sidx, r0, nrows); break;
        }
    }
}

}  // namespace mg

using namespace mg;

static bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static int64_t compact_parts(int64_t n) { return (n + kCompactPart - 1) / kCompactPart; }

static size_t compact_header_bytes(int64_t n) {
    const size_t h = 8 + 8 * (size_t)(compact_parts(n) > 0 ? compact_parts(n) : 1);
    return (h + 255) & ~(size_t)255;
}

extern "C" size_t mg_compact_workspace_bytes(int64_t n) {
    if (n < 0) return 0;
    return compact_header_bytes(n) + 4 * (size_t)n + 256;
}

extern "C" mg_status mg_prune_sample(const mg_gaussians *g, uint64_t seed, uint64_t iteration,
                                     int32_t n_draws, uint8_t *keep, mg_stream_t stream) {
    if (g == nullptr || g->n < 0 || g->n >= (int64_t(1) << 31) || n_draws < 1 || n_draws > 1024)
        return MG_ERR_INVALID_ARG;
    if (g->n == 0) return MG_OK;
    if (g->mask_logits == nullptr || keep == nullptr || !aligned_to(g->mask_logits, 8))
        return MG_ERR_INVALID_ARG;
    const unsigned blocks = (unsigned)((g->n + kPruneThreads - 1) / kPruneThreads);
    prune_sample_kernel<<<blocks, kPruneThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2 *>(g->mask_logits), g->n, seed, iteration, n_draws, keep);
    return mg_host::launch_status();
}

static int pick_word(const void *s, const void *d, int row_bytes) {
    for (int w = 16; w >= 2; w >>= 1)
        if (row_bytes % w == 0 && aligned_to(s, w) && aligned_to(d, w)) return w;
    return 0;
}

extern "C" mg_status mg_compact(const mg_gaussians *src, const uint8_t *keep,
                                const mg_gaussian_arrays *dst, int32_t *new_index,
                                int64_t *d_n_kept, void *workspace, size_t workspace_bytes,
                                mg_status_word *d_status, mg_stream_t stream) {
    if (src == nullptr || dst == nullptr || d_n_kept == nullptr || src->n < 0 ||
        src->n >= (int64_t(1) << 31) || src->sh_degree < 0 || src->sh_degree > 3 ||
        (src->dtype != MG_DTYPE_F32 && src->dtype != MG_DTYPE_BF16 && src->dtype != MG_DTYPE_F16))
        return MG_ERR_INVALID_ARG;
    const int64_t n = src->n;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0)
        return cudaMemsetAsync(d_n_kept, 0, sizeof(int64_t), s) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
    if (keep == nullptr || workspace == nullptr || workspace_bytes < mg_compact_workspace_bytes(n))
        return MG_ERR_INVALID_ARG;
    const int eb = src->dtype == MG_DTYPE_F32 ? 4 : 2;
    const int K = (src->sh_degree + 1) * (src->sh_degree + 1);
    const void *sp[kAttrs] = {src->means, src->log_scales, src->quats, src->opacity_logit, src->sh,
                              src->mask_logits};
    void *dp[kAttrs] = {dst->means, dst->log_scales, dst->quats, dst->opacity_logit, dst->sh,
                        dst->mask_logits};
    const int rb[kAttrs] = {12, 3 * eb, 4 * eb, eb, 3 * K * eb, 8};
    CopyArgs args;
    for (int a = 0; a < kAttrs; ++a) {
        if (sp[a] == nullptr || dp[a] == nullptr) return MG_ERR_INVALID_ARG;
        const char *s0 = static_cast<const char *>(sp[a]);
        const char *d0 = static_cast<const char *>(dp[a]);
        const size_t bytes = (size_t)rb[a] * (size_t)n;
        if (s0 < d0 + bytes && d0 < s0 + bytes) return MG_ERR_INVALID_ARG;   // overlap
        args.a[a].src = s0;
        args.a[a].dst = static_cast<char *>(dp[a]);
        args.a[a].row_bytes = rb[a];
        args.a[a].word = pick_word(sp[a], dp[a], rb[a]);
        if (args.a[a].word == 0) return MG_ERR_INVALID_ARG;
    }
    char *ws = static_cast<char *>(workspace);
    const uintptr_t a0 = (reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255;
    ws = reinterpret_cast<char *>(a0);
    CompactWS *hdr = reinterpret_cast<CompactWS *>(ws);
    int32_t *idx = new_index != nullptr
                       ? new_index
                       : reinterpret_cast<int32_t *>(ws + compact_header_bytes(n));
    const int64_t parts = compact_parts(n);
    if (cudaMemsetAsync(hdr, 0, 8 + 8 * (size_t)parts, s) != cudaSuccess) return MG_ERR_CUDA;
    compact_scan_kernel<<<(unsigned)parts, kCompactThreads, 0, s>>>(keep, n, idx, d_n_kept, hdr,
                                                                    parts, d_status);
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    compact_copy_kernel<<<(unsigned)((n + kCopyRows - 1) / kCopyRows), kCopyRows, 0, s>>>(args, idx,
                                                                                        n);
    return mg_host::launch_status();
}
