// Tile binning (Sec. 3.1: a Gaussian takes part in a tile's pixels only if it
// intersects the tile) and depth ordering (Sec. 3.1: the blend visits a
// pixel's Gaussians front to back by depth).
//
//   depth order  stable radix sort of the splat records by the float bits of
//                their depth (4 passes over R records)
//   scan         single-pass exclusive scan of tiles_touched, in depth order
//                (decoupled look-back)
//   duplicate    one tile-id key per intersected tile, row-major per splat,
//                splats in depth order
//   sort         stable LSD radix sort of the instances by tile id (2 passes
//                for up to 65536 tiles): as the instances arrive in depth
//                order, every tile's list comes out ordered by (depth, record
//                index) -- the order a full sort of 64-bit (tile, depth) keys
//                of record-ordered instances gives, with a quarter of the
//                traffic
//   ranges       [start, end) of every tile in the sorted list
//
// The radix sort is "onesweep" (Adinets & Merrill, "Onesweep: a faster least
// significant digit radix sort for GPUs", 2022): 8-bit digits, one kernel per
// digit, local ranking by warp multi-split (lanes with equal digits found
// through per-warp mask words in shared memory), global offsets by decoupled
// look-back.
//
// Every cross-block wait is bounded: after kMaxTimeoutSpins polls the kernel
// records MG_ERR_TIMEOUT in the status word and carries on (results are then
// invalid, but the GPU never hangs).  Partition ids come from an atomic
// counter, so a block only ever waits on partitions held by running blocks.
#include <mutex>

#include "internal.cuh"

namespace mg {

constexpr int kScanThreads = 256, kScanItems = 8, kScanPart = kScanThreads * kScanItems;
// instance slots per duplication warp (the scan marks each chunk's owner)
constexpr int kDupChunk = 512;
// 512 threads x 12 keys: with every partition of a small sort running at
// once, a partition's look-back ends at the nearest inclusive prefix, which
// spreads about a window per round trip -- fewer, larger partitions shorten
// that chain (one digit per thread for the first 256 threads).
constexpr int kSortThreads = 512, kSortItems = 10, kSortPart = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 2u << 30, kValMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 8;

// --------------------------------------------------------------------------
// scan of tiles_touched (in the given order)
// --------------------------------------------------------------------------
struct ScanWS {
    uint32_t counter;
    uint32_t pad;
    uint64_t status[1];   // [n_parts]
};

__global__ void __launch_bounds__(kScanThreads)
scan_kernel(const uint32_t *__restrict__ in, const uint32_t *__restrict__ order, int64_t n,
            uint32_t *__restrict__ out, uint64_t *d_total, uint64_t capacity, ScanWS *ws,
            int64_t n_parts, mg_status_word *st, uint32_t *__restrict__ owner_hint) {
    grid_dependency_wait();
    __shared__ uint64_t sm_warp[33];
    __shared__ uint64_t sm_prefix;
    __shared__ int64_t sm_part;
    if (threadIdx.x == 0) sm_part = atomicAdd(&ws->counter, 1u);
    __syncthreads();
    const int64_t part = sm_part;
    if (part >= n_parts) return;
    const int64_t base = part * kScanPart + (int64_t)threadIdx.x * kScanItems;
    // 128-bit loads of the positions' records and stores of their offsets
    // where both arrays are 16-byte aligned (base is a multiple of 8)
    const bool vec =
        ((reinterpret_cast<uintptr_t>(order) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    uint32_t v[kScanItems];
    uint64_t sum = 0;
    if (order == nullptr && base + kScanItems <= n) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 a = *reinterpret_cast<const uint4 *>(in + base + 4 * q);
            v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
        }
    } else if (order != nullptr && vec && base + kScanItems <= n) {
        // the positions' records with 128-bit loads, then the gather
        uint32_t o[kScanItems];
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 a = *reinterpret_cast<const uint4 *>(order + base + 4 * q);
            o[4 * q] = a.x; o[4 * q + 1] = a.y; o[4 * q + 2] = a.z; o[4 * q + 3] = a.w;
        }
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t idx = (int64_t)o[k];
            if (!MG_IN_BOUNDS(idx < n, st, 1, idx)) idx = n;   // skipped
            v[k] = idx < n ? in[idx] : 0u;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            int64_t idx = order ? (int64_t)order[base + k < n ? base + k : 0] : base + k;
            if (base + k < n && !MG_IN_BOUNDS(idx < n, st, 1, idx)) idx = n;   // skipped
            v[k] = (base + k < n && idx < n) ? in[idx] : 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += v[k];
    uint64_t agg;
    const uint64_t excl = block_exclusive_scan_u64(sum, sm_warp, agg);
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
            prefix = warp_lookback64(ws->status, part, st, 1);
            if (threadIdx.x == 0)
                atomicExch((unsigned long long *)&ws->status[part],
                           (unsigned long long)(kFlagPrefix64 | (prefix + agg)));
        }
        if (threadIdx.x == 0) sm_prefix = prefix;
        if (threadIdx.x == 0 && part == n_parts - 1) {
            *d_total = prefix + agg;
            if (prefix + agg > capacity) raise_status(st, MG_ERR_CAPACITY, 1, prefix + agg);
        }
    }
    __syncthreads();
    uint64_t run = sm_prefix + excl;
    const bool whole = vec && base + kScanItems <= n;
    uint32_t ov[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        ov[k] = run > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)run;
        if (!whole && base + k < n) out[base + k] = ov[k];
        // the position owns slots [run, run + v): it marks the duplication
        // chunks that start among them (owner_hint[c C] = position, C =
        // kDupChunk), below the capacity
        if (owner_hint != nullptr) {
            const uint64_t e = run + v[k] < capacity ? run + v[k] : capacity;
            for (uint64_t c = (run + kDupChunk - 1) / kDupChunk; c * kDupChunk < e; ++c)
                owner_hint[c * kDupChunk] = (uint32_t)(base + k);
        }
        run += v[k];
    }
    if (whole) {
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q)
            *reinterpret_cast<uint4 *>(out + base + 4 * q) =
                make_uint4(ov[4 * q], ov[4 * q + 1], ov[4 * q + 2], ov[4 * q + 3]);
    }
}

// --------------------------------------------------------------------------
// key duplication
// --------------------------------------------------------------------------
// Slot-parallel: warp w writes instance slots [w C, (w + 1) C), C = 512,
// whatever splats they belong to.  (A warp per 32 splats would leave the
// nearest splats -- first in depth order, and the largest, thousands of
// tiles each -- to a few warps: the kernel's time was their tail.)  The warp
// reads the position owning its first slot (the last position whose offset
// is <= the slot) from the mark the scan left in that slot's value, then
// walks positions 32 at a time: each lane holds one position's offset, slot
// count (the step to the next offset), record and binning record, and every
// 32 consecutive slots find their owner lane by a binary search over the
// lanes (shuffles) and are written fully coalesced.  Slot m of a rectangle is tile (x0 + m % w,
// y0 + m / w), the quotient through an FP32 reciprocal corrected to the
// exact integer.  A slot whose tile the Gaussian cannot reach above the
// alpha floor (bin_tile_hit) gets the key kDroppedKey, which the tile sort
// drops.
constexpr uint32_t kDroppedKey = 0xFFFFFFFFu;

__global__ void __launch_bounds__(256)
duplicate_kernel(const float4 *__restrict__ bin_record, const uint32_t *__restrict__ order,
                 const uint32_t *__restrict__ offsets, int64_t n_records, const uint64_t *__restrict__ d_num_instances,
                 uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, uint64_t capacity,
                 int tile_w, int tile_h, bool filter, mg_status_word *st) {
    grid_dependency_wait();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t total = *d_num_instances;
    const uint64_t K = total < capacity ? total : capacity;
    const uint64_t s0 = (uint64_t)gw * kDupChunk;
    if (s0 >= K) return;                                  // warp-uniform
    const uint64_t s1 = s0 + kDupChunk < K ? s0 + kDupChunk : K;

    // owner of slot s0 (the last position i with offsets[i] <= s0), marked
    // by the scan in the slot's value
    const int64_t lo = (int64_t)vals[s0];
    if (!MG_IN_BOUNDS(lo < n_records, st, 1, lo)) return;     // warp-uniform
    const uint32_t total32 = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;

    // the offsets and record indices of the next 32 positions are loaded
    // one group ahead, so they travel during the current group's slots
    auto load_group = [&](int64_t ip, uint32_t &off, uint32_t &r, uint32_t &nxt) {
        off = 0xFFFFFFFFu;
        r = 0;
        nxt = total32;
        if (ip < n_records) {
            off = offsets[ip];
            r = order ? order[ip] : (uint32_t)ip;
            if (lane == 31 && ip + 1 < n_records) nxt = offsets[ip + 1];
        }
    };
    uint32_t off_n, r_n, nxt_n;
    load_group(lo + lane, off_n, r_n, nxt_n);
    uint64_t s = s0;
    for (int64_t i = lo; s < s1; i += 32) {
        const int64_t ip = i + lane;
        uint32_t off = off_n, nxt = nxt_n, r = r_n, xy0 = 0, w = 1, first = 0, gx = 1;
        float4 b0 = make_float4(0.f, 0.f, 1.f, 0.f), b1 = make_float4(1.f, 0.f, 0.f, 0.f);
        bool rec_ok = true;
        if (ip < n_records) rec_ok = MG_IN_BOUNDS((int64_t)r < n_records, st, 1, r);
        // a position's slot count is the step to the next offset (the last
        // position ends at the total; offsets below the capacity are exact)
        const uint32_t down = __shfl_down_sync(FULL, off, 1);
        if (lane < 31 && ip + 1 < n_records) nxt = down;
        const uint32_t nt = ip < n_records ? nxt - off : 0u;
        if (nt != 0 && rec_ok) {
            const float4 *br = bin_record + 3 * (int64_t)r;
            b0 = br[0];
            b1 = br[1];
            const uint4 u = reinterpret_cast<const uint4 *>(br)[2];
            xy0 = u.x;
            w = u.y;
            first = u.z;
            gx = u.w;
        }
        const float rw = 1.0f / (float)w;
        // slots of these 32 positions: up to the end of the last valid one
        const uint64_t last = ip < n_records ? (uint64_t)off + nt : K;
        const uint64_t gend_all = __shfl_sync(FULL, last, 31);
        const uint64_t gend = gend_all < s1 ? gend_all : s1;
        if (gend < s1) load_group(ip + 32, off_n, r_n, nxt_n);    // another group follows
        for (uint64_t base = s; base < gend; base += 32) {      // warp-uniform trip count
            const uint64_t p = base + lane;
            const uint32_t pp = (uint32_t)p;
            int L = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t oc = __shfl_sync(FULL, off, L + step);
                if (oc <= pp) L += step;
            }
            const uint32_t m = pp - __shfl_sync(FULL, off, L);
            const uint32_t wl = __shfl_sync(FULL, w, L);
            const float rwl = __shfl_sync(FULL, rw, L);
            uint32_t q = (uint32_t)((float)m * rwl);
            int32_t rem = (int32_t)(m - q * wl);
            if (rem < 0) { --q; rem += (int32_t)wl; }
            else if (rem >= (int32_t)wl) { ++q; rem -= (int32_t)wl; }
            const uint32_t xy = __shfl_sync(FULL, xy0, L);
            const bool hit = !filter || bin_tile_hit(
                __shfl_sync(FULL, b0.x, L), __shfl_sync(FULL, b0.y, L), __shfl_sync(FULL, b0.z, L),
                __shfl_sync(FULL, b0.w, L), __shfl_sync(FULL, b1.x, L), __shfl_sync(FULL, b1.y, L),
                __shfl_sync(FULL, b1.z, L), __shfl_sync(FULL, b1.w, L),
                (int)(xy & 0xFFFFu) + rem, (int)(xy >> 16) + (int)q, tile_w, tile_h);
            const uint32_t fl = __shfl_sync(FULL, first, L);     // every lane shuffles
            const uint32_t gl = __shfl_sync(FULL, gx, L);
            // (debug build: a position whose record index was out of range has
            // its slots dropped, so nothing later reads with it)
            const bool okl = __shfl_sync(FULL, (int)rec_ok, L) != 0;
            const uint32_t key = hit && okl ? fl + q * gl + (uint32_t)rem : kDroppedKey;
            const uint32_t rr = __shfl_sync(FULL, r, L);
            if (p < gend) {
                keys[p] = key;
                vals[p] = rr;
            }
        }
        s = gend;
    }
}

// --------------------------------------------------------------------------
// radix sort (keys of type K, 8-bit digits from begin_bit up)
// --------------------------------------------------------------------------
// Instances to sort: all of them, or none when they overflowed the capacity
// (the buffers then hold an incomplete list; the status word says so).
// Element count of a sort: *d_n (0 if it exceeds capacity), or capacity when
// the count is known on the host (d_n null).
__device__ __forceinline__ int64_t sort_count(const uint64_t *d_n, uint64_t capacity) {
    if (d_n == nullptr) return (int64_t)capacity;
    const uint64_t n = *d_n;
    return n <= capacity ? (int64_t)n : 0;
}

struct SortWS {
    uint64_t n;                        // element count for sorts whose count is host-known
    uint64_t n_kept;                   // elements kept (all but dropped keys), set per sort
    uint32_t hist[kMaxPasses][256];    // digit counts, then exclusive offsets
    uint32_t counter[kMaxPasses];
    uint32_t pad[6];
    uint32_t status[1];                // [2][max_parts][256]
};

// Digit counts of every pass in one read of the keys: a few blocks per SM,
// each with a shared-memory histogram flushed once (the flush contends on the
// same 256 counters per pass, so the grid stays small).
// reset (nullable): reset_n words the caller wants zeroed before the sort's
// later kernels (the tile ranges), cleared here in passing.
template <typename K>
__global__ void sort_histogram_kernel(const K *__restrict__ keys, const uint64_t *d_n,
                                      uint64_t capacity, int begin_bit, int passes, SortWS *ws,
                                      int64_t max_parts, bool drop, uint32_t *__restrict__ reset,
                                      int64_t reset_n) {
    grid_dependency_wait();
    if (reset != nullptr)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < reset_n;
             i += (int64_t)gridDim.x * blockDim.x)
            reset[i] = 0u;
    __shared__ uint32_t h[kMaxPasses][256];
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = sort_count(d_n, capacity);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    if (sizeof(K) == 4) {
        // 4 keys per 128-bit load
        const int64_t n4 = n >> 2;
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
        for (int64_t q = t; q < n4; q += nt) {
            const uint4 v = k4[q];
            const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (drop && e[u] == kDroppedKey) continue;
                const uint64_t k = (uint64_t)e[u] >> begin_bit;
                for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
            }
        }
        for (int64_t i = (n4 << 2) + t; i < n; i += nt) {
            if (drop && (uint32_t)keys[i] == kDroppedKey) continue;
            const uint64_t k = (uint64_t)keys[i] >> begin_bit;
            for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
        }
    } else {
        for (int64_t i = t; i < n; i += nt) {
            const uint64_t k = (uint64_t)keys[i] >> begin_bit;
            for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
        }
    }
    // clear the look-back status of the first pass for the partitions in use
    const int64_t parts = (n + kSortPart - 1) / kSortPart;
    const int64_t lim = min(parts, max_parts) * 256;
    for (int64_t i = t; i < lim; i += nt) ws->status[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&(&ws->hist[0][0])[i], c);
    }
}

__global__ void sort_offsets_kernel(SortWS *ws) {
    grid_dependency_wait();
    // one block per pass, 256 threads: exclusive scan of the digit counts
    __shared__ uint64_t sm_warp[33];
    const int p = blockIdx.x;
    const uint32_t c = ws->hist[p][threadIdx.x];
    uint64_t tot;
    const uint64_t e = block_exclusive_scan_u64(c, sm_warp, tot);
    ws->hist[p][threadIdx.x] = (uint32_t)e;
    if (p == 0 && threadIdx.x == 0) ws->n_kept = tot;      // elements the sort keeps
}

// IDX = true: no value array; the values are the input positions.
template <typename K, bool DROP, bool IDX = false>
__global__ void __launch_bounds__(kSortThreads, 2048 / kSortThreads / 2)
onesweep_kernel(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                K *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint64_t *d_n,
                uint64_t capacity, int pass, int shift, SortWS *ws, int64_t max_parts,
                mg_status_word *st) {
    grid_dependency_wait();
    // staged keys and values of the partition: dynamic shared memory (above
    // the 48 KB a kernel may declare statically)
    extern __shared__ __align__(16) unsigned char sort_stage[];
    K *sk = reinterpret_cast<K *>(sort_stage);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sort_stage + sizeof(K) * kSortPart);
    __shared__ uint32_t whist[kSortWarps][256];
    __shared__ uint32_t wmatch[kSortWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ int64_t gbase[256];
    __shared__ uint64_t sm_warp[33];
    __shared__ int64_t sm_part;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = sort_count(d_n, capacity);
    const int64_t parts = min((n + kSortPart - 1) / kSortPart, max_parts);
    uint32_t *status = ws->status + (int64_t)(pass & 1) * max_parts * 256;
    uint32_t *status_next = ws->status + (int64_t)((pass + 1) & 1) * max_parts * 256;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wmatch[0][0])[i] = 0u;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm_part = atomicAdd(&ws->counter[pass], 1u);
        for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&whist[0][0])[i] = 0;
        __syncthreads();
        const int64_t part = sm_part;
        if (part >= parts) break;
        if (threadIdx.x < 256) status_next[part * 256 + threadIdx.x] = 0u;   // for the next pass

        // ---- load and rank within the warp (stable: slot-major, lane-minor)
        const int64_t wbase = part * kSortPart + (int64_t)warp * (32 * kSortItems);
        K k[kSortItems];
        uint32_t val[kSortItems], rank[kSortItems];
        int dig[kSortItems];
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const int64_t idx = wbase + i * 32 + lane;
            const bool valid = idx < n;
            k[i] = valid ? keys_in[idx] : (K)0;
            val[i] = valid ? (IDX ? (uint32_t)idx : vals_in[idx]) : 0u;
            const bool kept = valid && !(DROP && (uint32_t)k[i] == kDroppedKey);
            dig[i] = kept ? (int)(((uint64_t)k[i] >> shift) & 0xFF) : 256;
        }
        // lanes with equal digits find each other through a per-warp mask
        // word per digit (shared-memory atomicOr, read back, reset by the
        // group's highest lane)
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const bool kept = dig[i] < 256;
            if (kept) atomicOr(&wmatch[warp][dig[i]], 1u << lane);
            __syncwarp();
            const unsigned peers = kept ? wmatch[warp][dig[i]] : 0u;
            __syncwarp();
            const int leader = kept ? 31 - __clz(peers) : lane;
            uint32_t old = 0;
            if (kept && lane == leader) {
                old = whist[warp][dig[i]];
                whist[warp][dig[i]] = old + __popc(peers);
                wmatch[warp][dig[i]] = 0u;
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[i] = old + __popc(peers & lanemask_lt);
            __syncwarp();
        }
        __syncthreads();

        // ---- block digit counts, per-warp offsets, local digit starts
        const int d = threadIdx.x;
        const bool digit_thread = d < 256;
        uint32_t tot = 0;
        if (digit_thread) {
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = whist[w][d];
                whist[w][d] = tot;
                tot += c;
            }
            if (part == 0)
                atomicExch(&status[d], kFlagPrefix | tot);
            else
                atomicExch(&status[part * 256 + d], kFlagAgg | tot);
        }
        uint64_t dummy;
        const uint64_t ds = block_exclusive_scan_u64(tot, sm_warp, dummy);
        if (digit_thread) {
            dstart[d] = (uint32_t)ds;
            // ---- decoupled look-back per digit
            uint32_t excl = 0;
            if (part > 0) {
                excl = lookback<uint32_t, 30>(status + d, 256, part, st, 2);
                atomicExch(&status[part * 256 + d], kFlagPrefix | ((excl + tot) & kValMask));
            }
            gbase[d] = (int64_t)ws->hist[pass][d] + excl - (int64_t)ds;
        }
        __syncthreads();

        // ---- scatter into shared memory in block order, then out
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            if (dig[i] < 256) {
                const uint32_t pos = dstart[dig[i]] + whist[warp][dig[i]] + rank[i];
                sk[pos] = k[i];
                sv[pos] = val[i];
            }
        }
        __syncthreads();
        // kept elements of the partition: the block total of the digit counts
        const int cnt = DROP ? (int)sm_warp[32]
                             : (int)(n - part * kSortPart < kSortPart ? n - part * kSortPart
                                                                      : kSortPart);
        for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
            const K kk = sk[j];
            const int64_t dst = gbase[((uint64_t)kk >> shift) & 0xFF] + j;
            if (!MG_IN_BOUNDS(dst >= 0 && dst < n, st, 2, dst)) continue;
            keys_out[dst] = kk;
            vals_out[dst] = sv[j];
        }
    }
}

// Also copies the sorted count to d_num_sorted (nullable), so no copy node
// sits between the last sort pass and this kernel.
__global__ void ranges_kernel(const uint32_t *__restrict__ keys, const uint64_t *d_n,
                              uint64_t capacity, uint32_t *__restrict__ ranges, int64_t n_tiles,
                              uint64_t *d_num_sorted) {
    grid_dependency_wait();
    if (d_num_sorted != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *d_num_sorted = *d_n;
    const int64_t n = sort_count(d_n, capacity);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i0 < n; i0 += stride) {
        // the thread's four keys (one 128-bit load where aligned), the one
        // before and the one after
        uint32_t k4[5];
        if (vec && i0 + 4 <= n) {
            const uint4 a = *reinterpret_cast<const uint4 *>(keys + i0);
            k4[0] = a.x; k4[1] = a.y; k4[2] = a.z; k4[3] = a.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) k4[u] = i0 + u < n ? keys[i0 + u] : 0xFFFFFFFFu;
        }
        k4[4] = i0 + 4 < n ? keys[i0 + 4] : 0xFFFFFFFFu;
        uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u;
            if (i >= n) break;
            const uint32_t t = k4[u];
            const uint32_t next = i + 1 < n ? k4[u + 1] : 0xFFFFFFFFu;
            if ((int64_t)t < n_tiles) {
                if (i == 0 || prev != t) ranges[2 * (int64_t)t] = (uint32_t)i;
                if (i == n - 1 || next != t) ranges[2 * (int64_t)t + 1] = (uint32_t)(i + 1);
            }
            prev = t;
        }
    }
}

// Depth keys of the records: float bits of the depth (positive, so the bits
// order like the values); records outside every tile go last.
__global__ void depth_keys_kernel(const float *__restrict__ record,
                                  const uint32_t *__restrict__ tiles, int64_t n,
                                  uint32_t *__restrict__ keys, uint32_t *__restrict__ idx,
                                  uint64_t *d_n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        keys[r] = tiles[r] ? __float_as_uint(record[12 * r + 11]) : 0xFFFFFFFFu;
        idx[r] = (uint32_t)r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n = (uint64_t)n;
}

static unsigned dup_blocks(uint64_t capacity) {
    const uint64_t warps = (capacity + kDupChunk - 1) / kDupChunk;
    const uint64_t blocks = (warps + 7) / 8;
    return (unsigned)(blocks > 0 ? blocks : 1);
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static int64_t sort_max_parts(uint64_t capacity) {
    return (int64_t)((capacity + kSortPart - 1) / kSortPart) + 1;
}

static size_t sort_ws_bytes(uint64_t capacity) {
    return sizeof(SortWS) + sizeof(uint32_t) * 2 * 256 * (size_t)sort_max_parts(capacity) + 256;
}

// Enqueue a radix sort of the first *d_n pairs by key bits [begin_bit,
// begin_bit + 8 passes); tells whether the result is in the alt buffers.
// Opt the sort kernels in to their dynamic shared memory, once per device
// (the first call on a device should come before any stream capture).
template <typename K>
static mg_status sort_smem_optin(size_t bytes) {
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(onesweep_kernel<K, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess ||
            cudaFuncSetAttribute(onesweep_kernel<K, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess ||
            cudaFuncSetAttribute(onesweep_kernel<K, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess)
            return MG_ERR_CUDA;
        done[dev] = true;
    }
    return MG_OK;
}

// With `drop`, elements whose key is kDroppedKey leave in the first pass; the
// count kept is ws->n_kept (device), the count the later passes use.
// src_keys (nullable): the first pass reads these keys, with the input
// positions 0, 1, 2, ... as values, instead of (keys, vals).
template <typename K>
static mg_status radix_sort(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt,
                            const uint64_t *d_n, uint64_t capacity, int begin_bit, int passes,
                            bool drop, SortWS *ws, mg_status_word *st, cudaStream_t s,
                            bool *in_alt, const K *src_keys = nullptr,
                            uint32_t *reset = nullptr, int64_t reset_n = 0) {
    *in_alt = (passes & 1) != 0;
    if (mg_host::zero_async(&ws->hist[0][0], sizeof(ws->hist) + sizeof(ws->counter), s) != MG_OK)
        return MG_ERR_CUDA;
    if (capacity == 0 || passes == 0) return MG_OK;
    const int sms = sm_count();
    const int64_t max_parts = sort_max_parts(capacity);
    const int64_t hblocks = (int64_t)((capacity + 4095) / 4096);
    const int64_t hcap = (int64_t)sms * 2;
    const K *k0 = src_keys != nullptr ? src_keys : keys;
    launch_pdl(sort_histogram_kernel<K>,
        dim3((unsigned)(hblocks < hcap ? (hblocks > 0 ? hblocks : 1) : hcap)), dim3(512), 0, s, k0,
        d_n, capacity, begin_bit, passes, ws, max_parts, drop, reset, reset_n);
    launch_pdl(sort_offsets_kernel, dim3(passes), dim3(256), 0, s, ws);
    const size_t stage_bytes = (sizeof(K) + sizeof(uint32_t)) * (size_t)kSortPart;
    if (sort_smem_optin<K>(stage_bytes) != MG_OK) return MG_ERR_CUDA;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel<K, false>, kSortThreads,
                                                  stage_bytes);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = (int64_t)sms * per_sm < max_parts ? (int64_t)sms * per_sm : max_parts;
    K *kin = keys, *kout = keys_alt;
    uint32_t *vin = vals, *vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        // after a dropping first pass the later ones sort the kept elements
        const uint64_t *np_ = (drop && p > 0) ? &ws->n_kept : d_n;
        if (p == 0 && src_keys != nullptr)
            launch_pdl(onesweep_kernel<K, false, true>, dim3((unsigned)grid), dim3(kSortThreads),
                stage_bytes, s, src_keys, nullptr, kout, vout, np_, capacity, p, begin_bit, ws,
                max_parts, st);
        else if (drop && p == 0)
            launch_pdl(onesweep_kernel<K, true>, dim3((unsigned)grid), dim3(kSortThreads),
                stage_bytes, s, kin, vin, kout, vout, np_, capacity, p, begin_bit + 8 * p, ws,
                max_parts, st);
        else
            launch_pdl(onesweep_kernel<K, false>, dim3((unsigned)grid), dim3(kSortThreads),
                stage_bytes, s, kin, vin, kout, vout, np_, capacity, p, begin_bit + 8 * p, ws,
                max_parts, st);
        K *tk = kin; kin = kout; kout = tk;
        uint32_t *tv = vin; vin = vout; vout = tv;
    }
    return MG_OK;
}

// --------------------------------------------------------------------------
// Tile-bucket sort: the instances grouped by tile in one counting pass over
// the whole tile id (a digit as wide as the key), then every tile's list
// ordered by (depth key, record index).  The depth order of the records is
// not needed beforehand, so the instances may come in record order; the lists
// equal those of the depth sort + stable tile sort.
//
//   count    block b counts the kept instances of a contiguous range per tile
//            (shared-memory histogram over the range's tile window) into row
//            b of a B x T matrix H
//   columns  per tile, H's column becomes its exclusive prefix over the
//            blocks (block b's base inside the tile) and the tile's count
//   scan     exclusive scan of the tile counts (the tile starts)
//   scatter  block b places its instances at start[t] + H[b][t] onwards,
//            shared-memory atomics handing out the slots (so the order
//            inside a tile is arbitrary here), as 64-bit (depth_key << 32 |
//            record) keys
//   order    each tile's keys sorted by a bitonic network held in registers
//            (8 keys per thread; warp shuffles for distances up to 128,
//            shared memory only across warps): lists of up to 1024 keys by
//            128-thread CTAs, longer ones by 512-thread CTAs, in 4096-key
//            chunks merged in global scratch past 4096
// No global atomics on contended addresses: the per-tile bases come from
// the column prefixes.  Every loop over instances issues kBucketIlp
// independent loads per thread before using any of them.
// --------------------------------------------------------------------------
constexpr int kBucketThreads = 256;
constexpr int kBucketIlp = 8;
constexpr int kBucketTile = kBucketThreads * kBucketIlp;
constexpr int kBucketWindow = 8192;           // tile ids per block histogram (32 KB)
constexpr int kBucketBlocksMax = 1024;
constexpr int kSortE = 8;                     // keys per thread in the register sort
constexpr int kSortSmallThreads = 128;        // lists of up to 1024 keys
constexpr int kSortLargeThreads = 512;        // lists of up to 4096 keys per chunk

__device__ __forceinline__ void block_range(int64_t n, int64_t &b0, int64_t &b1) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    b0 = (int64_t)blockIdx.x * per;
    b1 = b0 + per < n ? b0 + per : n;
}

// kBucketIlp keys of the block's range starting at i0 (kDroppedKey past b1,
// and for tile ids outside [0, n_tiles)).
__device__ __forceinline__ void load_keys(const uint32_t *__restrict__ keys, int64_t i0, int64_t b1,
                                          int64_t n_tiles, uint32_t k[kBucketIlp]) {
#pragma unroll
    for (int u = 0; u < kBucketIlp; ++u) {
        const int64_t i = i0 + u * kBucketThreads + threadIdx.x;
        const uint32_t x = i < b1 ? __ldg(keys + i) : kDroppedKey;
        k[u] = (int64_t)x < n_tiles ? x : kDroppedKey;
    }
}

// The tile window [lo, hi] of the block's range (lo > hi: nothing kept).
__device__ __forceinline__ uint2 range_window(const uint32_t *__restrict__ keys, int64_t b0,
                                              int64_t b1, int64_t n_tiles, uint32_t *s_lo,
                                              uint32_t *s_hi) {
    const unsigned FULL = 0xffffffffu;
    if (threadIdx.x == 0) {
        *s_lo = 0xFFFFFFFFu;
        *s_hi = 0u;
    }
    __syncthreads();
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int64_t i0 = b0; i0 < b1; i0 += kBucketTile) {
        uint32_t k[kBucketIlp];
        load_keys(keys, i0, b1, n_tiles, k);
#pragma unroll
        for (int u = 0; u < kBucketIlp; ++u)
            if (k[u] != kDroppedKey) {
                lo = min(lo, k[u]);
                hi = max(hi, k[u]);
            }
    }
    lo = __reduce_min_sync(FULL, lo);
    hi = __reduce_max_sync(FULL, hi);
    if ((threadIdx.x & 31) == 0 && lo <= hi) {
        atomicMin(s_lo, lo);
        atomicMax(s_hi, hi);
    }
    __syncthreads();
    return make_uint2(*s_lo, *s_hi);
}

// Row b of H (zeroed beforehand): the block's kept instances per tile.
__global__ void __launch_bounds__(kBucketThreads)
bucket_count_kernel(const uint32_t *__restrict__ keys, const uint64_t *d_n, uint64_t capacity,
                    int64_t n_tiles, uint32_t *__restrict__ H, uint2 *__restrict__ window) {
    __shared__ uint32_t sh[kBucketWindow];
    __shared__ uint32_t s_lo, s_hi;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t n = sort_count(d_n, capacity);
    int64_t b0, b1;
    block_range(n, b0, b1);
    const uint2 win = range_window(keys, b0, b1, n_tiles, &s_lo, &s_hi);
    const uint32_t lo = win.x, hi = win.y;
    if (threadIdx.x == 0) window[blockIdx.x] = win;
    if (lo > hi) return;                                    // nothing kept here
    uint32_t *row = H + (int64_t)blockIdx.x * n_tiles;
    const bool windowed = hi - lo < (uint32_t)kBucketWindow;
    if (windowed) {
        for (uint32_t w = threadIdx.x; w <= hi - lo; w += kBucketThreads) sh[w] = 0u;
        __syncthreads();
    }
    for (int64_t i0 = b0; i0 < b1; i0 += kBucketTile) {      // block-uniform trip count
        uint32_t k[kBucketIlp];
        load_keys(keys, i0, b1, n_tiles, k);
#pragma unroll
        for (int u = 0; u < kBucketIlp; ++u) {
            if (windowed) {
                if (k[u] != kDroppedKey) atomicAdd(&sh[k[u] - lo], 1u);
            } else {
                const unsigned peers = __match_any_sync(FULL, k[u]);
                if (k[u] != kDroppedKey && lane == __ffs(peers) - 1)
                    atomicAdd(&row[k[u]], (uint32_t)__popc(peers));
            }
        }
    }
    if (windowed) {
        __syncthreads();
        for (uint32_t w = threadIdx.x; w <= hi - lo; w += kBucketThreads) row[lo + w] = sh[w];
    }
}

// Per tile: H's column -> its exclusive prefix over the blocks, and the
// tile's count.  A CTA takes 32 tiles (one per lane); its 8 warps split the
// blocks into 8 segments, summed, scanned across warps, then rewritten.
constexpr int kColWarps = 8;
__global__ void __launch_bounds__(32 * kColWarps)
bucket_columns_kernel(uint32_t *__restrict__ H, int64_t n_blocks, int64_t n_tiles,
                      uint32_t *__restrict__ tile_count) {
    __shared__ uint32_t seg[kColWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * 32 + lane;
    const int64_t per = (n_blocks + kColWarps - 1) / kColWarps;
    const int64_t r0 = warp * per, r1 = min(r0 + per, n_blocks);
    // 8 rows per round trip: the loads of a round are independent
    constexpr int U = 8;
    uint32_t sum = 0u;
    if (t < n_tiles)
        for (int64_t r = r0; r < r1; r += U) {
            uint32_t c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) c[u] = r + u < r1 ? H[(r + u) * n_tiles + t] : 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) sum += c[u];
        }
    seg[warp][lane] = sum;
    __syncthreads();
    uint32_t run = 0u;
    for (int w = 0; w < warp; ++w) run += seg[w][lane];
    if (t < n_tiles) {
        for (int64_t r = r0; r < r1; r += U) {
            uint32_t c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) c[u] = r + u < r1 ? H[(r + u) * n_tiles + t] : 0u;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (r + u < r1) {
                    H[(r + u) * n_tiles + t] = run;
                    run += c[u];
                }
        }
        if (warp == kColWarps - 1) tile_count[t] = run;
    }
}

// Block b places its kept instances at start[t] + H[b][t] onwards as
// (depth_key << 32 | record) keys.  The records of a block's range are nearly
// consecutive, so their depth keys are read almost in order.
__global__ void __launch_bounds__(kBucketThreads)
bucket_scatter_kernel(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                      const uint32_t *__restrict__ depth_key, const uint64_t *d_n,
                      uint64_t capacity, int64_t n_tiles, const uint32_t *__restrict__ tile_start,
                      uint32_t *__restrict__ H, const uint2 *__restrict__ window,
                      uint64_t *__restrict__ grouped, mg_status_word *st) {
    __shared__ uint32_t sh[kBucketWindow];
    const int64_t n = sort_count(d_n, capacity);
    int64_t b0, b1;
    block_range(n, b0, b1);
    const uint2 win = window[blockIdx.x];
    const uint32_t lo = win.x, hi = win.y;
    if (lo > hi) return;
    uint32_t *row = H + (int64_t)blockIdx.x * n_tiles;
    const bool windowed = hi - lo < (uint32_t)kBucketWindow;
    if (windowed) {
        for (uint32_t w = threadIdx.x; w <= hi - lo; w += kBucketThreads)
            sh[w] = tile_start[lo + w] + row[lo + w];
        __syncthreads();
    }
    for (int64_t i0 = b0; i0 < b1; i0 += kBucketTile) {
        uint32_t k[kBucketIlp], v[kBucketIlp], d[kBucketIlp];
        load_keys(keys, i0, b1, n_tiles, k);
#pragma unroll
        for (int u = 0; u < kBucketIlp; ++u) {
            const int64_t i = i0 + u * kBucketThreads + threadIdx.x;
            v[u] = k[u] != kDroppedKey ? __ldg(vals + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kBucketIlp; ++u) d[u] = k[u] != kDroppedKey ? __ldg(depth_key + v[u]) : 0u;
#pragma unroll
        for (int u = 0; u < kBucketIlp; ++u) {
            if (k[u] == kDroppedKey) continue;
            const uint32_t pos = windowed ? atomicAdd(&sh[k[u] - lo], 1u)
                                          : tile_start[k[u]] + atomicAdd(&row[k[u]], 1u);
            if (!MG_IN_BOUNDS((uint64_t)pos < (uint64_t)n, st, 3, pos)) continue;
            grouped[pos] = ((uint64_t)d[u] << 32) | v[u];
        }
    }
}

// ---- per-tile merge sort -------------------------------------------------------
// A tile's keys (distinct 64-bit (depth_key << 32 | record)) sorted by one
// CTA: each thread sorts kSortE keys in registers (Batcher's 19-comparator
// network for 8), then runs are merged pairwise in shared memory, every
// thread producing kSortE outputs of its pair after a merge-path binary
// search for where its share starts.  O(n log n) work: a bitonic network's
// O(n log^2 n) cost 4-5x more on these lists.

__device__ __forceinline__ void ce_asc(uint64_t &a, uint64_t &b) {
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

__device__ __forceinline__ void sort8_regs(uint64_t (&v)[kSortE]) {
    ce_asc(v[0], v[1]); ce_asc(v[2], v[3]); ce_asc(v[4], v[5]); ce_asc(v[6], v[7]);
    ce_asc(v[0], v[2]); ce_asc(v[1], v[3]); ce_asc(v[4], v[6]); ce_asc(v[5], v[7]);
    ce_asc(v[1], v[2]); ce_asc(v[5], v[6]);
    ce_asc(v[0], v[4]); ce_asc(v[1], v[5]); ce_asc(v[2], v[6]); ce_asc(v[3], v[7]);
    ce_asc(v[2], v[4]); ce_asc(v[3], v[5]);
    ce_asc(v[1], v[2]); ce_asc(v[3], v[4]); ce_asc(v[5], v[6]);
}

// Shared-memory slot of key e: the low three bits XORed with a hash of the
// thread row (e >> 3), so that the 32 threads of a warp writing their 8-key
// rows hit distinct banks.
__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 3) ^ (e >> 6)) & 7); }

// Sorts keys[0 .. L) (L <= THREADS kSortE) into out (records: the low 32
// bits), using S0 and S1 (THREADS kSortE keys each) in shared memory.
template <int THREADS>
__device__ void merge_sort_tile(const uint64_t *__restrict__ keys, int L,
                                uint32_t *__restrict__ out, uint64_t *S0, uint64_t *S1) {
    const int n8 = (L + kSortE - 1) & ~(kSortE - 1);          // runs of kSortE, padded with ~0
    const int base = threadIdx.x * kSortE;
    const bool mine = base < n8;
    uint64_t v[kSortE];
#pragma unroll
    for (int r = 0; r < kSortE; ++r) v[r] = base + r < L ? keys[base + r] : ~0ull;
    if (mine) {
        sort8_regs(v);
#pragma unroll
        for (int r = 0; r < kSortE; ++r) S0[swz(base + r)] = v[r];
    }
    __syncthreads();
    uint64_t *cur = S0, *nxt = S1;
    for (int w = kSortE; w < n8; w <<= 1) {
        if (mine) {
            const int a0 = (base / (2 * w)) * (2 * w);
            const int la = min(w, n8 - a0);
            const int b0 = a0 + la;
            const int lb = min(w, n8 - b0);
            const int d0 = base - a0;                          // this thread's first output
            int lo = d0 > lb ? d0 - lb : 0, hi = d0 < la ? d0 : la;
            while (lo < hi) {                                  // A's share of the first d0
                const int mid = (lo + hi) >> 1;
                if (cur[swz(a0 + mid)] < cur[swz(b0 + d0 - 1 - mid)]) lo = mid + 1;
                else hi = mid;
            }
            int ia = lo, ib = d0 - lo;
            uint64_t x = ia < la ? cur[swz(a0 + ia)] : ~0ull;
            uint64_t y = ib < lb ? cur[swz(b0 + ib)] : ~0ull;
#pragma unroll
            for (int r = 0; r < kSortE; ++r) {
                const bool take_a = x < y;                     // keys are distinct; ~0 pads last
                v[r] = take_a ? x : y;
                if (take_a) {
                    ++ia;
                    x = ia < la ? cur[swz(a0 + ia)] : ~0ull;
                } else {
                    ++ib;
                    y = ib < lb ? cur[swz(b0 + ib)] : ~0ull;
                }
            }
        }
        __syncthreads();
        if (mine) {
#pragma unroll
            for (int r = 0; r < kSortE; ++r) nxt[swz(base + r)] = v[r];
        }
        __syncthreads();
        uint64_t *t = cur;
        cur = nxt;
        nxt = t;
    }
#pragma unroll
    for (int r = 0; r < kSortE; ++r)
        if (base + r < L) out[base + r] = (uint32_t)v[r];
}

// Merge of the sorted runs a[0 .. la) and b[0 .. lb) into out by the whole
// CTA: each thread takes an equal share of the output and finds where it
// starts on the merge path by a binary search (keys are distinct).
template <int THREADS>
__device__ void merge_runs(const uint64_t *a, int64_t la, const uint64_t *b, int64_t lb,
                           uint64_t *out) {
    const int64_t total = la + lb;
    const int64_t d0 = total * threadIdx.x / THREADS;
    const int64_t d1 = total * (threadIdx.x + 1) / THREADS;
    int64_t lo = d0 > lb ? d0 - lb : 0, hi = d0 < la ? d0 : la;
    while (lo < hi) {                      // elements of a among the first d0 outputs
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < b[d0 - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    int64_t ia = lo, ib = d0 - lo;
    for (int64_t d = d0; d < d1; ++d) {
        const bool take_a = ib >= lb || (ia < la && a[ia] < b[ib]);
        out[d] = take_a ? a[ia++] : b[ib++];
    }
}

// Lists of 2 .. 1024 keys, one 128-thread CTA per tile (other tiles return);
// also writes every tile's range and the one-key lists.
__global__ void __launch_bounds__(kSortSmallThreads)
tile_sort_small_kernel(const uint32_t *__restrict__ tile_start,
                       const uint32_t *__restrict__ tile_count,
                       const uint64_t *__restrict__ grouped, uint32_t *__restrict__ sorted,
                       uint32_t *__restrict__ ranges, uint32_t *__restrict__ long_tiles,
                       uint32_t *long_count) {
    __shared__ uint64_t S0[kSortSmallThreads * kSortE], S1[kSortSmallThreads * kSortE];
    const int64_t t = blockIdx.x;
    const uint32_t s = tile_start[t], L = tile_count[t];
    if (threadIdx.x == 0) {
        ranges[2 * t] = s;
        ranges[2 * t + 1] = s + L;
        if (L == 1u) sorted[s] = (uint32_t)grouped[s];
        // longer lists go to the large sort's work list
        if (L > (uint32_t)(kSortSmallThreads * kSortE)) long_tiles[atomicAdd(long_count, 1u)] = (uint32_t)t;
    }
    if (L < 2u || L > (uint32_t)(kSortSmallThreads * kSortE)) return;
    merge_sort_tile<kSortSmallThreads>(grouped + s, (int)L, sorted + s, S0, S1);
}

// Lists longer than 1024 keys, from the work list the small sort filled: a
// persistent grid of 512-thread CTAs takes them in turn.  Chunks of up to
// 4096 keys are merge-sorted in shared memory; longer lists are merged
// pairwise in global scratch (grouped and tmp, the tile's own range).
__device__ void sort_long_tile(uint32_t s, uint32_t L, uint64_t *__restrict__ grouped,
                               uint32_t *__restrict__ sorted, uint64_t *__restrict__ tmp,
                               uint64_t *S0, uint64_t *S1) {
    constexpr int kCap = kSortLargeThreads * kSortE;
    if (L <= (uint32_t)kCap) {
        merge_sort_tile<kSortLargeThreads>(grouped + s, (int)L, sorted + s, S0, S1);
        __syncthreads();
        return;
    }
    // chunks sorted in shared memory and written back, then merged pairwise
    uint64_t *A = grouped + s, *B = tmp + s;
    for (uint32_t c0 = 0; c0 < L; c0 += kCap) {
        const int m = (int)min(L - c0, (uint32_t)kCap);
        // sort the chunk; its records land in sorted (overwritten later) and
        // its keys are read back from shared memory in order
        merge_sort_tile<kSortLargeThreads>(A + c0, m, sorted + s + c0, S0, S1);
        __syncthreads();
        // the sorted chunk: recover the keys in order (run order after the
        // last pass is in whichever buffer the passes ended on)
        const int n8 = (m + kSortE - 1) & ~(kSortE - 1);
        int passes = 0;
        for (int w = kSortE; w < n8; w <<= 1) ++passes;
        const uint64_t *fin = (passes & 1) ? S1 : S0;
        for (int i = threadIdx.x; i < m; i += kSortLargeThreads) A[c0 + i] = fin[swz(i)];
        __syncthreads();
    }
    for (int64_t w = kCap; w < (int64_t)L; w <<= 1) {
        __syncthreads();
        for (int64_t p0 = 0; p0 < (int64_t)L; p0 += 2 * w) {
            const int64_t la = min(w, (int64_t)L - p0);
            const int64_t lb = min(w, (int64_t)L - p0 - la);
            merge_runs<kSortLargeThreads>(A + p0, la, A + p0 + la, lb, B + p0);
        }
        uint64_t *x = A;
        A = B;
        B = x;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < L; i += kSortLargeThreads) sorted[s + i] = (uint32_t)A[i];
    __syncthreads();
}

__global__ void __launch_bounds__(kSortLargeThreads)
tile_sort_large_kernel(const uint32_t *__restrict__ tile_start,
                       const uint32_t *__restrict__ tile_count,
                       const uint32_t *__restrict__ long_tiles, const uint32_t *long_count,
                       uint64_t *__restrict__ grouped, uint32_t *__restrict__ sorted,
                       uint64_t *__restrict__ tmp) {
    extern __shared__ __align__(16) unsigned char sort_smem[];
    uint64_t *S0 = reinterpret_cast<uint64_t *>(sort_smem), *S1 = S0 + kSortLargeThreads * kSortE;
    const uint32_t n_long = *long_count;
    for (uint32_t i = blockIdx.x; i < n_long; i += gridDim.x) {
        const uint32_t t = long_tiles[i];
        sort_long_tile(tile_start[t], tile_count[t], grouped, sorted, tmp, S0, S1);
    }
}

}  // namespace mg

using namespace mg;

extern "C" size_t mg_depth_order_workspace_bytes(int64_t n_records) {
    return sort_ws_bytes((uint64_t)(n_records > 0 ? n_records : 0));
}

extern "C" mg_status mg_depth_order(const mg_splats *splats, const mg_view *views,
                                    int32_t n_views, const mg_raster_cfg *cfg, uint32_t *order,
                                    uint32_t *order_alt, uint32_t *keys, uint32_t *keys_alt,
                                    void *workspace, size_t workspace_bytes,
                                    mg_status_word *d_status, mg_stream_t stream) {
    if (splats == nullptr || !splats->record || !splats->tiles_touched || !workspace)
        return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t R = vt.rec_off[n_views];
    if (R == 0) return MG_OK;
    if (!order || !order_alt || !keys || !keys_alt) return MG_ERR_INVALID_ARG;
    if (R > (int64_t)kValMask) return MG_ERR_INVALID_ARG;
    if (workspace_bytes < mg_depth_order_workspace_bytes(R)) return MG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    SortWS *ws = reinterpret_cast<SortWS *>(workspace);
    bool in_alt = false;
    // 4 passes (an even number): the result is back in (keys, order)
    if (splats->depth_key != nullptr) {
        // keys written by the preprocess; the first pass takes the record
        // indices as values
        st = radix_sort<uint32_t>(keys, order, keys_alt, order_alt, nullptr, (uint64_t)R, 0, 4,
                                  false, ws, d_status, s, &in_alt, splats->depth_key);
    } else {
        depth_keys_kernel<<<sm_count() * 4, 256, 0, s>>>(splats->record, splats->tiles_touched,
                                                          R, keys, order, &ws->n);
        st = radix_sort<uint32_t>(keys, order, keys_alt, order_alt, &ws->n, (uint64_t)R, 0, 4,
                                  false, ws, d_status, s, &in_alt);
    }
    if (st != MG_OK) return st;
    return mg_host::launch_status();
}

extern "C" size_t mg_bin_workspace_bytes(int64_t n_records) {
    const int64_t parts = (n_records + kScanPart - 1) / kScanPart + 1;
    return sizeof(ScanWS) + sizeof(uint64_t) * (size_t)parts + 256;
}

extern "C" size_t mg_sort_workspace_bytes(uint64_t capacity, int32_t key_bits) {
    (void)key_bits;
    return sort_ws_bytes(capacity);
}

extern "C" mg_status mg_bin(const mg_splats *splats, const mg_view *views, int32_t n_views,
                            const mg_raster_cfg *cfg, const uint32_t *order, uint32_t *offsets,
                            uint32_t *keys, uint32_t *vals, uint64_t capacity,
                            uint64_t *d_num_instances, void *workspace, size_t workspace_bytes,
                            mg_status_word *d_status, mg_stream_t stream) {
    if (splats == nullptr || !splats->bin_record || !splats->tiles_touched || !offsets ||
        !d_num_instances || !workspace)
        return MG_ERR_INVALID_ARG;
    if (capacity > 0 && (!keys || !vals)) return MG_ERR_INVALID_ARG;
    if (cfg == nullptr || (cfg->bin_mode != MG_BIN_FILTERED && cfg->bin_mode != MG_BIN_RECT))
        return MG_ERR_INVALID_ARG;
    if (capacity > (uint64_t)kValMask) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t R = vt.rec_off[n_views];
    if (workspace_bytes < mg_bin_workspace_bytes(R)) return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->tiles_touched) & 15u) != 0) return MG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t parts = (R + kScanPart - 1) / kScanPart;
    ScanWS *ws = reinterpret_cast<ScanWS *>(workspace);
    if (mg_host::zero_async(ws, sizeof(ScanWS) + sizeof(uint64_t) * (size_t)(parts + 1), s) !=
        MG_OK)
        return MG_ERR_CUDA;
    if (R == 0) {
        if (cudaMemsetAsync(d_num_instances, 0, sizeof(uint64_t), s) != cudaSuccess)
            return MG_ERR_CUDA;
        return MG_OK;
    }
    launch_pdl(scan_kernel, dim3((unsigned)parts), dim3(kScanThreads), 0, s, splats->tiles_touched,
        order, R, offsets, d_num_instances, capacity, ws, parts, d_status,
        capacity > 0 ? vals : nullptr);
    if (capacity > 0)
        launch_pdl(duplicate_kernel, dim3(dup_blocks(capacity)), dim3(256), 0, s,
            reinterpret_cast<const float4 *>(splats->bin_record), order, offsets, R,
            d_num_instances, keys, vals, capacity, cfg->tile_w, cfg->tile_h,
            cfg->bin_mode == MG_BIN_FILTERED, d_status);
    return mg_host::launch_status();
}

extern "C" mg_status mg_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                             uint32_t *vals_alt, const uint64_t *d_num_instances,
                             uint64_t capacity, int32_t key_bits, uint32_t *ranges,
                             int64_t n_tiles_total, void *workspace, size_t workspace_bytes,
                             int32_t *result_in_alt, uint64_t *d_num_sorted,
                             mg_status_word *d_status, mg_stream_t stream) {
    if (!keys || !vals || !keys_alt || !vals_alt || !d_num_instances || !ranges || !workspace ||
        !result_in_alt || key_bits < 1 || key_bits > 32 || n_tiles_total <= 0)
        return MG_ERR_INVALID_ARG;
    if (capacity > (uint64_t)kValMask) return MG_ERR_INVALID_ARG;
    if (workspace_bytes < mg_sort_workspace_bytes(capacity, key_bits)) return MG_ERR_INVALID_ARG;
    if ((n_tiles_total >> 32) != 0 || (key_bits < 32 && (n_tiles_total >> key_bits) > 1) ||
        (key_bits < 32 && (n_tiles_total > (int64_t(1) << key_bits))) ||
        n_tiles_total >= (int64_t)kDroppedKey)
        return MG_ERR_INVALID_ARG;
    const int passes = (key_bits + 7) / 8;
    cudaStream_t s = (cudaStream_t)stream;
    SortWS *ws = reinterpret_cast<SortWS *>(workspace);
    bool in_alt = false;
    // filtered instances (key kDroppedKey) leave in the first pass; the
    // histogram kernel also clears the ranges (tiles with no instance keep
    // [0, 0)) -- or a reset kernel does when there is nothing to sort
    if (capacity == 0 &&
        mg_host::zero_async(ranges, sizeof(uint32_t) * 2 * (size_t)n_tiles_total, s) != MG_OK)
        return MG_ERR_CUDA;
    mg_status st = radix_sort<uint32_t>(keys, vals, keys_alt, vals_alt, d_num_instances, capacity,
                                        0, passes, true, ws, d_status, s, &in_alt, nullptr, ranges,
                                        2 * n_tiles_total);
    if (st != MG_OK) return st;
    *result_in_alt = in_alt ? 1 : 0;
    if (capacity == 0) return mg_host::launch_status();
    const int64_t rblocks = (int64_t)((capacity + 1023) / 1024);
    launch_pdl(ranges_kernel, dim3((unsigned)(rblocks < 65535 ? rblocks : 65535)), dim3(256), 0, s,
        in_alt ? keys_alt : keys, &ws->n_kept, capacity, ranges, n_tiles_total, d_num_sorted);
    return mg_host::launch_status();
}

// --------------------------------------------------------------------------
// mg_sort_by_tile: the tile-bucket sort (see the kernels above).
// --------------------------------------------------------------------------
namespace {

struct BucketLayout {
    size_t count, start, window, scan, long_count, n_kept, long_tiles, hist, grouped, tmp, total;
    int64_t scan_parts, blocks;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// three blocks per SM, at least 4096 instances per block
int64_t bucket_blocks(uint64_t capacity) {
    const int64_t by_size = (int64_t)((capacity + 4095) / 4096);
    int64_t blocks = 3 * (int64_t)sm_count();
    if (blocks > by_size) blocks = by_size;
    if (blocks > kBucketBlocksMax) blocks = kBucketBlocksMax;
    return blocks < 1 ? 1 : blocks;
}

constexpr size_t kTileSortLargeSmem = 2 * sizeof(uint64_t) * kSortLargeThreads * kSortE;

// The large tile sort's 64 KB of dynamic shared memory, opted in once per device.
mg_status tile_sort_smem_optin() {
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        if (cudaFuncSetAttribute(tile_sort_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTileSortLargeSmem) != cudaSuccess)
            return MG_ERR_CUDA;
        done[dev] = true;
    }
    return MG_OK;
}

BucketLayout bucket_layout(uint64_t capacity, int64_t n_tiles, int64_t blocks) {
    BucketLayout L;
    L.blocks = blocks;
    size_t o = 0;
    L.count = o;
    o = align256(o + sizeof(uint32_t) * (size_t)n_tiles);
    L.start = o;
    o = align256(o + sizeof(uint32_t) * (size_t)n_tiles);
    L.window = o;
    o = align256(o + sizeof(uint2) * (size_t)kBucketBlocksMax);
    L.scan_parts = (n_tiles + kScanPart - 1) / kScanPart;
    L.scan = o;
    o = align256(o + sizeof(ScanWS) + sizeof(uint64_t) * (size_t)(L.scan_parts + 1));
    L.long_count = o;                     // zeroed with the scan's words
    o = align256(o + sizeof(uint32_t));
    L.n_kept = o;
    o = align256(o + sizeof(uint64_t));
    L.long_tiles = o;
    o = align256(o + sizeof(uint32_t) * (size_t)n_tiles);
    L.hist = o;
    o = align256(o + sizeof(uint32_t) * (size_t)n_tiles * (size_t)blocks);
    L.grouped = o;
    o = align256(o + sizeof(uint64_t) * (size_t)capacity);
    L.tmp = o;
    o = align256(o + sizeof(uint64_t) * (size_t)capacity);
    L.total = o;
    return L;
}

}  // namespace

extern "C" size_t mg_sort_by_tile_workspace_bytes(uint64_t capacity, int64_t n_tiles_total) {
    if (n_tiles_total < 0) n_tiles_total = 0;
    return bucket_layout(capacity, n_tiles_total, bucket_blocks(capacity)).total;
}

extern "C" mg_status mg_sort_by_tile(const uint32_t *keys, const uint32_t *vals,
                                     const uint32_t *depth_key, const uint64_t *d_num_instances,
                                     uint64_t capacity, int64_t n_tiles_total,
                                     uint32_t *sorted_vals, uint32_t *ranges, void *workspace,
                                     size_t workspace_bytes, uint64_t *d_num_sorted,
                                     mg_status_word *d_status, mg_stream_t stream) {
    if (!keys || !vals || !depth_key || !d_num_instances || !sorted_vals || !ranges ||
        !workspace || n_tiles_total <= 0 || n_tiles_total >= (int64_t(1) << 31) ||
        n_tiles_total >= (int64_t)kDroppedKey)
        return MG_ERR_INVALID_ARG;
    if (capacity > (uint64_t)kValMask) return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 15u) != 0) return MG_ERR_INVALID_ARG;
    const int64_t blocks = bucket_blocks(capacity);
    const BucketLayout L = bucket_layout(capacity, n_tiles_total, blocks);
    if (workspace_bytes < L.total) return MG_ERR_INVALID_ARG;
    if (tile_sort_smem_optin() != MG_OK) return MG_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = reinterpret_cast<char *>(workspace);
    uint32_t *count = reinterpret_cast<uint32_t *>(ws + L.count);
    uint32_t *start = reinterpret_cast<uint32_t *>(ws + L.start);
    uint2 *window = reinterpret_cast<uint2 *>(ws + L.window);
    ScanWS *scan_ws = reinterpret_cast<ScanWS *>(ws + L.scan);
    uint64_t *n_kept = reinterpret_cast<uint64_t *>(ws + L.n_kept);
    uint32_t *H = reinterpret_cast<uint32_t *>(ws + L.hist);
    uint64_t *grouped = reinterpret_cast<uint64_t *>(ws + L.grouped);
    // the scan's look-back words and the block-by-tile counts start at 0
    if (cudaMemsetAsync(ws + L.scan, 0, L.n_kept - L.scan, s) != cudaSuccess ||
        cudaMemsetAsync(H, 0, sizeof(uint32_t) * (size_t)n_tiles_total * (size_t)blocks, s) !=
            cudaSuccess)
        return MG_ERR_CUDA;
    bucket_count_kernel<<<(unsigned)blocks, kBucketThreads, 0, s>>>(
        keys, d_num_instances, capacity, n_tiles_total, H, window);
    bucket_columns_kernel<<<(unsigned)((n_tiles_total + 31) / 32), 32 * kColWarps, 0, s>>>(
        H, blocks, n_tiles_total, count);
    scan_kernel<<<(unsigned)L.scan_parts, kScanThreads, 0, s>>>(
        count, nullptr, n_tiles_total, start, d_num_sorted != nullptr ? d_num_sorted : n_kept,
        ~0ull, scan_ws, L.scan_parts, d_status, nullptr);
    bucket_scatter_kernel<<<(unsigned)blocks, kBucketThreads, 0, s>>>(
        keys, vals, depth_key, d_num_instances, capacity, n_tiles_total, start, H, window,
        grouped, d_status);
    uint32_t *long_tiles = reinterpret_cast<uint32_t *>(ws + L.long_tiles);
    uint32_t *long_count = reinterpret_cast<uint32_t *>(ws + L.long_count);
    tile_sort_small_kernel<<<(unsigned)n_tiles_total, kSortSmallThreads, 0, s>>>(
        start, count, grouped, sorted_vals, ranges, long_tiles, long_count);
    const int64_t long_grid = min((int64_t)2 * sm_count(), n_tiles_total);
    tile_sort_large_kernel<<<(unsigned)long_grid, kSortLargeThreads, kTileSortLargeSmem, s>>>(
        start, count, long_tiles, long_count, grouped, sorted_vals,
        reinterpret_cast<uint64_t *>(ws + L.tmp));
    return mg_host::launch_status();
}

// --------------------------------------------------------------------------
// mg_validate_lists: the tile lists checked against their bounds.
// --------------------------------------------------------------------------
namespace mg {

constexpr int kValidateThreads = 1024;

// One block walks the tiles in order: every range ordered and inside
// [0, n), a non-empty range starting at or after the largest end of the
// non-empty ranges before it (a running maximum carried over block-wide
// max-scans), and the lengths summing to n.
__global__ void __launch_bounds__(kValidateThreads)
validate_ranges_kernel(const uint32_t *__restrict__ ranges, int64_t n_tiles,
                       const uint64_t *d_n, uint64_t capacity, mg_status_word *st) {
    __shared__ uint32_t s_warp[kValidateThreads / 32];
    __shared__ uint32_t s_run;
    __shared__ unsigned long long s_total;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t dn = *d_n;
    if (dn > capacity) {
        if (threadIdx.x == 0) raise_status(st, MG_ERR_BOUNDS, 9, dn);
        return;
    }
    if (threadIdx.x == 0) {
        s_run = 0u;
        s_total = 0ull;
    }
    __syncthreads();
    for (int64_t t0 = 0; t0 < n_tiles; t0 += kValidateThreads) {
        const int64_t t = t0 + threadIdx.x;
        uint32_t s = 0u, e = 0u;
        if (t < n_tiles) {
            s = ranges[2 * t];
            e = ranges[2 * t + 1];
            if (e < s || (uint64_t)e > dn) raise_status(st, MG_ERR_BOUNDS, 7, (uint64_t)t);
        }
        const bool nonempty = t < n_tiles && e > s;
        // exclusive max over this chunk's earlier tiles of the non-empty ends
        uint32_t inc = nonempty ? e : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc = max(inc, x);
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        uint32_t before = s_run;
        for (int w = 0; w < warp; ++w) before = max(before, s_warp[w]);
        const uint32_t lane_prev = __shfl_up_sync(FULL, inc, 1);
        if (lane > 0) before = max(before, lane_prev);
        if (nonempty) {
            if (s < before) raise_status(st, MG_ERR_BOUNDS, 7, (uint64_t)t);
            atomicAdd(&s_total, (unsigned long long)(e - s));
        }
        __syncthreads();
        if (threadIdx.x == kValidateThreads - 1) s_run = max(before, inc);
        __syncthreads();
    }
    if (threadIdx.x == 0 && s_total != dn) raise_status(st, MG_ERR_BOUNDS, 9, s_total);
}

__global__ void validate_values_kernel(const uint32_t *__restrict__ vals, const uint64_t *d_n,
                                       uint64_t capacity, int64_t n_records, mg_status_word *st) {
    const uint64_t dn = *d_n;
    const int64_t n = (int64_t)(dn < capacity ? dn : capacity);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if ((int64_t)vals[i] >= n_records) raise_status(st, MG_ERR_BOUNDS, 8, (uint64_t)i);
}

}  // namespace mg

extern "C" mg_status mg_validate_lists(const uint32_t *sorted_vals, const uint32_t *ranges,
                                       int64_t n_tiles_total, const uint64_t *d_num_sorted,
                                       uint64_t capacity, int64_t n_records,
                                       mg_status_word *d_status, mg_stream_t stream) {
    if (!sorted_vals || !ranges || !d_num_sorted || !d_status || n_tiles_total <= 0 ||
        n_records < 0)
        return MG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    validate_ranges_kernel<<<1, kValidateThreads, 0, s>>>(ranges, n_tiles_total, d_num_sorted,
                                                         capacity, d_status);
    const int64_t blocks = (int64_t)((capacity + 1023) / 1024);
    validate_values_kernel<<<(unsigned)(blocks < 2048 ? (blocks > 0 ? blocks : 1) : 2048), 256, 0,
                             s>>>(sorted_vals, d_num_sorted, capacity, n_records, d_status);
    return mg_host::launch_status();
}

// --------------------------------------------------------------------------
// mg_bin_noalloc: mg_bin without a caller-provided workspace.
//
// For callers that cannot allocate device memory themselves, for example a
// plugin whose host application owns every allocation, or code that runs
// where cudaMalloc is not permitted.  The scan's scratch (partition counter
// and look-back words) lives in one file-scope device array instead, sized
// for at most kNoAllocMaxRecords splat records; every GPU that loads the
// library holds it until the process exits.  No allocation happens here.
// --------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxRecords = int64_t(1) << 24;
constexpr int64_t kNoAllocParts = (kNoAllocMaxRecords + mg::kScanPart - 1) / mg::kScanPart + 1;
constexpr size_t kNoAllocScratchBytes = sizeof(mg::ScanWS) + sizeof(uint64_t) * kNoAllocParts;
constexpr int kNoAllocMaxDevices = 256;

static __device__ __align__(256) unsigned char g_bin_scratch[kNoAllocScratchBytes];

std::mutex g_bin_scratch_mutex;
void *g_bin_scratch_addr[kNoAllocMaxDevices] = {};

// Device address of g_bin_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
mg_status bin_scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MG_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return MG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_bin_scratch_mutex);
    if (g_bin_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || p == nullptr) {
            // take the (non-sticky) error off the runtime's last-error slot so
            // that a later, unrelated launch check does not report it
            cudaGetLastError();
            return MG_ERR_CUDA;
        }
        g_bin_scratch_addr[dev] = p;
    }
    *out = g_bin_scratch_addr[dev];
    return MG_OK;
}

}  // namespace

extern "C" mg_status mg_bin_noalloc(const mg_splats *splats, const mg_view *views,
                                    int32_t n_views, const mg_raster_cfg *cfg,
                                    const uint32_t *order, uint32_t *offsets, uint32_t *keys,
                                    uint32_t *vals, uint64_t capacity, uint64_t *d_num_instances,
                                    mg_status_word *d_status, mg_stream_t stream) {
    if (splats == nullptr || !splats->bin_record || !splats->tiles_touched || !offsets ||
        !d_num_instances)
        return MG_ERR_INVALID_ARG;
    if (capacity > 0 && (!keys || !vals)) return MG_ERR_INVALID_ARG;
    if (cfg == nullptr || (cfg->bin_mode != MG_BIN_FILTERED && cfg->bin_mode != MG_BIN_RECT))
        return MG_ERR_INVALID_ARG;
    if (capacity > (uint64_t)kValMask) return MG_ERR_INVALID_ARG;
    ViewTable vt;
    mg_status st = mg_host::build_view_table(views, n_views, cfg, &vt);
    if (st != MG_OK) return st;
    const int64_t R = vt.rec_off[n_views];
    if (R > kNoAllocMaxRecords) return MG_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats->tiles_touched) & 15u) != 0) return MG_ERR_INVALID_ARG;
    void *scratch = nullptr;
    st = bin_scratch_address(&scratch);
    if (st != MG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t parts = (R + kScanPart - 1) / kScanPart;
    ScanWS *ws = reinterpret_cast<ScanWS *>(scratch);
    // the array keeps the previous call's contents: clear the counter and the
    // look-back words this call uses
    if (cudaMemsetAsync(ws, 0, sizeof(ScanWS) + sizeof(uint64_t) * (size_t)(parts + 1), s) !=
        cudaSuccess)
        return MG_ERR_CUDA;
    if (R == 0) {
        if (cudaMemsetAsync(d_num_instances, 0, sizeof(uint64_t), s) != cudaSuccess)
            return MG_ERR_CUDA;
        return MG_OK;
    }
    scan_kernel<<<(unsigned)parts, kScanThreads, 0, s>>>(splats->tiles_touched, order, R, offsets,
                                                         d_num_instances, capacity, ws, parts,
                                                         d_status, capacity > 0 ? vals : nullptr);
    if (capacity > 0)
        duplicate_kernel<<<dup_blocks(capacity), 256, 0, s>>>(
            reinterpret_cast<const float4 *>(splats->bin_record), order,
            offsets, R, d_num_instances, keys, vals, capacity, cfg->tile_w, cfg->tile_h,
            cfg->bin_mode == MG_BIN_FILTERED, d_status);
    return mg_host::launch_status();
}
