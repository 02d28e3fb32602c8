// sm_103a kernels of the batched scan and their launcher: many reads of uneven length,
// each against its own resident table, in one persistent launch (plus the pack, plan and
// tail kernels around it). The walk itself is the one of the scan kernels
// (pfac_device.cuh), bounded by each read's end.
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "../../include/pfac.h"
#include "pfac_internal.h"
#include "pfac_device.cuh"

namespace pfac {

// ---------------------------------------------------------------------------
// Batched scan: many reads of uneven length, each against its own table, in one
// persistent launch (plus the pack, plan and tail kernels around it).
//   pack_bits_kernel    ASCII reads -> 2-bit words + one invalid bit per base
//   plan_kernel         reads -> first work item of each read (512 or 1024 offsets per
//                       item), and the read of every work item
//   batched_scan_kernel each warp takes every W-th item (W warps in the grid), with the
//                       next item's read and bounds loaded while it scans the current
//                       one; each item runs the same per-warp filter test and skip walks
//                       as kernel 2, with its read's table and every walk bounded by its
//                       read's end
//   batched_tail_kernel deferred long walks, with the table recorded in each item
// ---------------------------------------------------------------------------

// A work item is 32 lanes x LW offsets (LW = 16 or 32): 512 or 1024 offsets.

struct BatchParams {
    const DeviceTable *sets;
    int32_t n_sets;
    const uint32_t *packed;
    const uint32_t *invalid;
    int64_t n;
    const int64_t *read_off;
    const int32_t *read_set;
    int32_t n_reads;
    const int64_t *item_start;
    const int32_t *item_read;    // read of each work item, for the first item_cap items
    int64_t item_cap;
    int32_t item;                // offsets per work item (32 x LW)
    int32_t *out;
    DeferItem *defer;
    int64_t defer_cap;
    unsigned long long *defer_count;
    int32_t walk_loads;
};

__global__ void pack_bits_kernel(const uint8_t *__restrict__ text, int64_t len, uint32_t *__restrict__ packed,
                                 uint32_t *__restrict__ invalid)
{
    const int64_t n_bw = (len + 31) >> 5;
    const int64_t n_words = (len + 15) >> 4;
    const bool aligned = ((uintptr_t)text & 15u) == 0;
    for (int64_t bw = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; bw < n_bw; bw += (int64_t)gridDim.x * blockDim.x) {
        uint32_t inv = 0;
        for (int h = 0; h < 2; h++) {
            const int64_t b0 = (bw << 5) + 16 * h;
            uint32_t word = 0, badm = 0;
            if (aligned && b0 + 16 <= len) {
                word = pack16(__ldg(reinterpret_cast<const uint4 *>(text + b0)), &badm);
            } else {
                for (int i = 0; i < 16; i++) {
                    const int c = b0 + i < len ? base_code_or_neg(text[b0 + i]) : -1;
                    if (c < 0) badm |= 1u << i;
                    else word |= (uint32_t)c << (2 * i);
                }
            }
            if (2 * bw + h < n_words) packed[2 * bw + h] = word;
            inv |= badm << (16 * h);
        }
        invalid[bw] = inv;
    }
}

__device__ __forceinline__ void read_bounds(const int64_t *read_off, int32_t r, int64_t n, int64_t *rs, int64_t *re)
{
    const int64_t a = min(max(read_off[r], (int64_t)0), n);
    const int64_t b = min(max(read_off[r + 1], a), n);
    *rs = a;
    *re = b;
}

// One CTA: exclusive prefix of the number of work items per read. The reads' bounds are
// loaded kPlanRounds rounds of 1,024 reads at a time, all loads in flight together, before
// the rounds' block scans run one after another.
constexpr int kPlanRounds = 8;

__global__ void __launch_bounds__(1024) plan_kernel(const int64_t *__restrict__ read_off, int32_t n_reads, int64_t n,
                                                    int32_t item, int64_t *__restrict__ item_start,
                                                    int32_t *__restrict__ item_read, int64_t item_cap)
{
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base0 = 0; base0 < n_reads; base0 += (int64_t)kPlanRounds * blockDim.x) {
        int64_t items[kPlanRounds];
#pragma unroll
        for (int q = 0; q < kPlanRounds; q++) {
            const int64_t r = base0 + (int64_t)q * blockDim.x + tid;
            items[q] = 0;
            if (r < n_reads) {
                int64_t rs, re;
                read_bounds(read_off, (int32_t)r, n, &rs, &re);
                items[q] = (re - rs + item - 1) / item;
            }
        }
#pragma unroll
        for (int q = 0; q < kPlanRounds; q++) {
            const int64_t base = base0 + (int64_t)q * blockDim.x;
            if (base >= n_reads) break;
            const int64_t r = base + tid;
            const int64_t v = items[q];
            int64_t incl = v;
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
                if (lane >= d) incl += o;
            }
            if (lane == 31) warp_sum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                int64_t ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
                for (int d = 1; d < 32; d <<= 1) {
                    const int64_t o = __shfl_up_sync(0xFFFFFFFFu, ws, d);
                    if (lane >= d) ws += o;
                }
                warp_sum[lane] = ws;   // inclusive over warps
            }
            __syncthreads();
            const int64_t before = (warp ? warp_sum[warp - 1] : 0) + incl - v;
            if (r < n_reads) {
                const int64_t k0 = carry + before;
                item_start[r] = k0;
                // the read of each of this read's work items (items past item_cap are found
                // by search instead)
                const int64_t k1 = min(k0 + v, item_cap);
                for (int64_t k = k0; k < k1; k++) item_read[k] = (int32_t)r;
            }
            __syncthreads();
            if (tid == 0) carry += warp_sum[(blockDim.x >> 5) - 1];
            __syncthreads();
        }
    }
    if (tid == 0) item_start[n_reads] = carry;
}

// Where a work item lies: its read, the read's bounds and table, the item's first offset.
struct ItemMeta {
    int64_t rs, re, base;
    int32_t set;
};

// The metadata of work item `it` (the read from the plan's map, or by search past its
// capacity: the last r with item_start[r] <= it).
template <int LW>
__device__ __forceinline__ ItemMeta item_meta(const BatchParams &P, int64_t it)
{
    int32_t r = 0;
    if (it < P.item_cap) {
        r = P.item_read[it];
    } else {
        int32_t hi = P.n_reads - 1;
        while (r < hi) {
            const int32_t mid = (int32_t)(((int64_t)r + hi + 1) >> 1);
            if (P.item_start[mid] <= it) r = mid;
            else hi = mid - 1;
        }
    }
    ItemMeta m;
    read_bounds(P.read_off, r, P.n, &m.rs, &m.re);
    m.set = P.read_set[r];
    m.base = m.rs + (it - P.item_start[r]) * (32 * LW);
    return m;
}

// Warp w takes work items w, w + W, w + 2W, ... (W warps in the grid); the metadata of
// its next item is loaded before the current one is scanned, so those dependent loads
// overlap the scan instead of preceding it.
template <int LW>
__global__ void __launch_bounds__(256, 4) batched_scan_kernel(const BatchParams P)
{
    constexpr int kItem = 32 * LW;
    constexpr uint32_t kAll = LW == 32 ? 0xFFFFFFFFu : ((1u << LW) - 1u);
    const int lane = threadIdx.x & 31;
    const int64_t total = P.item_start[P.n_reads];
    const uint64_t pol = policy_evict_first();
    Sink K{};
    K.out = P.out;
    K.defer = P.defer;
    K.defer_cap = P.defer_cap;
    K.defer_count = P.defer_count;
    const int64_t n_words = (P.n + 15) >> 4;
    const int64_t n_bw = (P.n + 31) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    ItemMeta m{};
    if (it < total) m = item_meta<LW>(P, it);
    while (it < total) {
        const int64_t nxt = it + stride;
        ItemMeta mn{};
        if (nxt < total) mn = item_meta<LW>(P, nxt);
        const int32_t set = m.set;
        if (set < 0 || set >= P.n_sets) {
            if (lane == 0) record_error(P.sets[0].status, PFAC_ERR_INVALID_ARG);
        } else {
            const DeviceTable T = P.sets[set];
            const int64_t base = m.base, re = m.re;
            const int64_t item_end = min(base + kItem, re);
            // this lane's LW offsets and the 64 bases from its first one
            const int64_t p0 = base + LW * lane;
            const int64_t wi = p0 >> 4;
            const uint32_t sh = (uint32_t)(p0 & 15) * 2;
            uint32_t w[5];
#pragma unroll
            for (int k = 0; k < 5; k++) w[k] = (wi + k < n_words) ? __ldg(P.packed + wi + k) : 0u;
            const uint32_t x0 = __funnelshift_r(w[0], w[1], sh), x1 = __funnelshift_r(w[1], w[2], sh);
            const uint32_t x2 = __funnelshift_r(w[2], w[3], sh), x3 = __funnelshift_r(w[3], w[4], sh);
            const int64_t bi = p0 >> 5;
            const uint32_t sb = (uint32_t)(p0 & 31);
            uint32_t iv[3];
#pragma unroll
            for (int k = 0; k < 3; k++) iv[k] = (bi + k < n_bw) ? __ldg(P.invalid + bi + k) : 0xFFFFFFFFu;
            uint64_t bad = ((uint64_t)__funnelshift_r(iv[1], iv[2], sb) << 32) | __funnelshift_r(iv[0], iv[1], sb);
            const int64_t rem_read = re - p0;   // walks stop at the read's end
            if (rem_read < 64) bad |= rem_read > 0 ? (~0ull << rem_read) : ~0ull;
            const int64_t rem_item = item_end - p0;
            const uint32_t valid = rem_item >= LW ? kAll : (rem_item > 0 ? ((1u << rem_item) - 1u) : 0u);
            const bool vec_ok = (((uintptr_t)(P.out + base)) & 15u) == 0;
            scan_lane_batch<true, false, false, true, LW>(T, K, nullptr, nullptr, P.walk_loads, (uint32_t)set,
                                                          P.packed, P.invalid, re, base, lane, x0, x1, x2, x3, bad,
                                                          valid, vec_ok, pol);
        }
        it = nxt;
        m = mn;
    }
}

__global__ void __launch_bounds__(256) batched_tail_kernel(const BatchParams P)
{
    const unsigned long long cnt = *P.defer_count;
    const int64_t m = min((int64_t)cnt, P.defer_cap);
    Sink K{};
    K.out = P.out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const DeferItem it = P.defer[i];
        const DeviceTable T = P.sets[it.q_set >> 16];
        emit_match<false>(K, it.gp, walk_global<true>(T, P.packed, P.invalid, it.gp + it.span, it.gp, it.s,
                                                      (int)(it.q_set & 0xFFFFu), it.best));
    }
}

// ---------------------------------------------------------------------------
// Fused batched pass (batches of up to kFusedMaxReads reads): ONE launch, one CTA per
// SM, no packed copy of the text, no planning or tail launch.
//   1. Every CTA plans the whole batch in shared memory, and every CTA gets the same
//      plan: the reads are ordered by table bucket (table index mod kFusedBuckets) by a
//      counting sort whose ranks come from per-(bucket, warp) counts, so the order does
//      not depend on timing; the work items are numbered in that order. A work item is
//      one aligned 32*LW-base chunk of the concatenated text intersected with one read.
//   2. The items are dealt to the CTAs in runs of kDealRun (run k to CTA k mod G), and
//      a CTA's warps claim its items in order from a counter in shared memory, each claim
//      issued one item ahead. An SM's warps thus work on one or two runs at a time, mostly
//      of one table, whose filter words stay in its L1, and every CTA gets a sample of
//      every table's items, so that the CTAs' loads even out. A warp copies the
//      next item's bytes (and the 64 after them) and its table's descriptor into shared
//      memory with cp.async while it scans the current one; each lane packs its own 16
//      bytes and takes the rest of its 64-base window by shuffles, as kernel 2 does for
//      ASCII text.
//   3. After a block barrier the CTA finishes the long walks its items deferred, kept in
//      its own slice of the deferred-walk list.
// ---------------------------------------------------------------------------

constexpr int kFusedBuckets = 128;
constexpr int kDealRun = 16;
constexpr int kGuide = 1024;   // guide entries: the sorted place of every (I / kGuide)-th item

struct FusedParams {
    const DeviceTable *sets;
    int32_t n_sets;
    const uint8_t *text;
    int64_t n;
    const int64_t *read_off;
    const int32_t *read_set;
    int32_t n_reads;
    int32_t *out;
    DeferItem *defer;                // defer_per_cta items for each CTA
    int64_t defer_per_cta;
    int32_t walk_loads;
};

// Reads one fused launch plans in shared memory.
constexpr int32_t kFusedMaxReads = 8192;

// Bytes of one warp's text buffer: a work item and the 64 bases after it.
template <int LW>
__host__ __device__ constexpr int fused_buf_bytes() { return 32 * LW + 64; }

// Bytes of one warp buffer slot: the text buffer, then a copy of the item's table
// descriptor (16-byte aligned, copied with cp.async ahead of its use).
constexpr int kTableCopy = (int)sizeof(DeviceTable);
static_assert(kTableCopy % 16 == 0, "table descriptors are copied in whole 16-byte pieces");
template <int LW>
__host__ __device__ constexpr int fused_slot_bytes() { return fused_buf_bytes<LW>() + kTableCopy; }

// Shared memory of the fused kernel for `warps` warps per CTA, n_reads reads and LW
// offsets per lane. Kept throughout: the deferred-walk and claim counts, the guide to the
// sorted places, and per read its sorted place, first item and first chunk. Then one
// region that first holds what only the plan uses (per-(bucket, warp) read counts and
// item sums, the scan's warp totals, per read its item count and bucket) and then the
// two buffer slots (text and table descriptor) of every warp.
static size_t fused_plan_bytes(int warps, size_t r16)
{
    return (size_t)(warps + 1) * kFusedBuckets * 4 * 2 + 32 * 8 + r16 * 4 + r16;
}
static size_t fused_smem_bytes(int warps, int32_t n_reads, int lw)
{
    const size_t r16 = ((size_t)n_reads + 4) / 4 * 4;   // n_reads + 1 entries, rounded to 16 bytes
    return 16 + (kGuide + 4) * 4 + r16 * 4 * 3 +
           std::max(fused_plan_bytes(warps, r16), (size_t)warps * 2 * (32 * lw + 64 + kTableCopy));
}

// Sixteen ASCII bytes from position p of the text (bases at or past n are bad).
__device__ __forceinline__ uint32_t ascii16(const uint8_t *__restrict__ text, int64_t n, int64_t p, bool aligned,
                                            uint32_t *bad16)
{
    if (aligned && p + 16 <= n) return pack16(__ldg(reinterpret_cast<const uint4 *>(text + p)), bad16);
    uint32_t w = 0, b = 0;
    for (int i = 0; i < 16; i++) {
        const int c = p + i < n ? base_code_or_neg(__ldg(text + p + i)) : -1;
        if (c < 0) b |= 1u << i;
        else w |= (uint32_t)c << (2 * i);
    }
    *bad16 = b;
    return w;
}

// Asynchronous 16-byte copy global -> shared that bypasses L1; the bytes past `valid`
// (0 .. 16) are zero-filled (a zero byte is not a base).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t fused_bucket(int32_t set) { return (uint32_t)set % (uint32_t)kFusedBuckets; }

// Work items of the read [rs, re): the aligned item-size chunks it touches.
__device__ __forceinline__ int32_t fused_items(int64_t rs, int64_t re, int shift)
{
    return re > rs ? (int32_t)(((re - 1) >> shift) - (rs >> shift) + 1) : 0;
}

// A claimed work item: its first offset (chunk-aligned), and its read's raw bounds and
// table as loaded (clamped only when the item is scanned, so that nothing waits on
// these loads while the previous item is still being scanned).
struct FusedItem {
    int64_t base, lo, hi;
    int32_t set;
};

template <int LW>
__global__ void __launch_bounds__(1024, 1) fused_batched_kernel(const FusedParams P)
{
    constexpr int kItem = 32 * LW;
    constexpr int kShift = LW == 32 ? 10 : 9;
    constexpr int kBuf = fused_buf_bytes<LW>();
    constexpr int kSlot = fused_slot_bytes<LW>();
    constexpr uint32_t kFull = 0xFFFFFFFFu;
    extern __shared__ __align__(16) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = blockDim.x >> 5;
    const int R = P.n_reads;
    const int R16 = (R + 4) / 4 * 4;
    // per-(bucket, warp) counts at bucket * (W + 1) + warp: the lanes of a warp, each
    // adding to its own bucket, meet different banks
    const int WP = W + 1;
    unsigned long long *dcount = reinterpret_cast<unsigned long long *>(smem);       // deferred walks
    unsigned int *claimed = reinterpret_cast<unsigned int *>(dcount + 1);             // items claimed
    int32_t *guide = reinterpret_cast<int32_t *>(dcount + 2);                         // [kGuide + 4]
    int32_t *sorted_read = guide + kGuide + 4;                                        // [R]
    int32_t *item_start = sorted_read + R16;                                          // [R + 1]
    int32_t *read_chunk = item_start + R16;                                           // [R]
    uint8_t *region = reinterpret_cast<uint8_t *>(read_chunk + R16);
    // the plan's scratch ...
    uint32_t *cnt_reads = reinterpret_cast<uint32_t *>(region);                       // [bucket][W + 1]
    uint32_t *cnt_items = cnt_reads + WP * kFusedBuckets;                             // [bucket][W + 1]
    unsigned long long *wsum = reinterpret_cast<unsigned long long *>(cnt_items + WP * kFusedBuckets);   // [32]
    int32_t *read_items = reinterpret_cast<int32_t *>(wsum + 32);                     // [R]
    uint8_t *read_bucket = reinterpret_cast<uint8_t *>(read_items + R16);             // [R]
    // ... and then the text buffers, once the plan is done
    uint8_t *tbuf = region;                                                           // [warp][2][kSlot]

    // ---- 1. the plan ----
    for (int i = tid; i < 2 * WP * kFusedBuckets; i += blockDim.x) cnt_reads[i] = 0;
    if (tid == 0) {
        *dcount = 0;
        *claimed = 0;
    }
    __syncthreads();
    const int seg = ((R + W - 1) / W + 31) & ~31;   // reads per warp, whole rounds of 32
    const int r0 = min(R, warp * seg), r1 = min(R, r0 + seg);
    // the reads' bounds and tables, kPlanRounds rounds of 32 reads in flight at once
    for (int cb = r0; cb < r1; cb += 32 * kPlanRounds) {
        int64_t lo_[kPlanRounds], hi_[kPlanRounds];
        int32_t set_[kPlanRounds];
#pragma unroll
        for (int q = 0; q < kPlanRounds; q++) {
            const int r = cb + 32 * q + lane;
            lo_[q] = hi_[q] = 0;
            set_[q] = 0;
            if (r < r1) {
                lo_[q] = P.read_off[r];
                hi_[q] = P.read_off[r + 1];
                set_[q] = P.read_set[r];
            }
        }
#pragma unroll
        for (int q = 0; q < kPlanRounds; q++) {
            const int r = cb + 32 * q + lane;
            if (r < r1) {
                const int64_t rs = min(max(lo_[q], (int64_t)0), P.n), re = min(max(hi_[q], rs), P.n);
                const int32_t items = fused_items(rs, re, kShift);
                const uint32_t bk = fused_bucket(set_[q]);
                read_items[r] = items;
                read_chunk[r] = (int32_t)(rs >> kShift);
                read_bucket[r] = (uint8_t)bk;
                atomicAdd(&cnt_reads[bk * WP + warp], 1u);
                atomicAdd(&cnt_items[bk * WP + warp], (uint32_t)items);
            }
        }
    }
    __syncthreads();
    // exclusive scan of the (reads << 32 | items) counts in (bucket, warp) order; the
    // item total stays below 2^31, so the low half never carries into the high one
    {
        constexpr int kPer = kFusedBuckets / 32;   // W * kFusedBuckets entries over 32 * W threads
        const int lg_w = __ffs(W) - 1;              // W is 8, 16 or 32
        unsigned long long v[kPer], sum = 0;
        int at[kPer];
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const int i = kPer * tid + q;                 // place in (bucket, warp) order
            at[q] = (i >> lg_w) * WP + (i & (W - 1));
            v[q] = ((unsigned long long)cnt_reads[at[q]] << 32) | cnt_items[at[q]];
            sum += v[q];
        }
        unsigned long long incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long o = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long x = lane < W ? wsum[lane] : 0ull;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long o = __shfl_up_sync(kFull, x, d);
                if (lane >= d) x += o;
            }
            wsum[lane] = x;   // inclusive over warps
        }
        __syncthreads();
        unsigned long long run = (warp ? wsum[warp - 1] : 0ull) + incl - sum;
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            cnt_reads[at[q]] = (uint32_t)(run >> 32);
            cnt_items[at[q]] = (uint32_t)run;
            run += v[q];
        }
        if (tid == 0) item_start[R] = (int32_t)(uint32_t)wsum[W - 1];
    }
    __syncthreads();
    // each read's place: its (bucket, warp) base, moved on past the reads of the same
    // bucket in this warp's earlier rounds, plus those in lower lanes of this round
    for (int cb = r0; cb < r1; cb += 32) {
        const int r = cb + lane;
        const bool act = r < r1;
        const int32_t items = act ? read_items[r] : 0;
        const uint32_t bk = act ? (uint32_t)read_bucket[r] : 0xFFFFFFFFu;
        // the lanes with this lane's bucket: eight ballots, one per bit of the bucket
        uint32_t grp = kFull;
#pragma unroll
        for (int bit = 0; bit < 8; bit++) {
            const uint32_t set_b = __ballot_sync(kFull, (bk >> bit) & 1u);
            grp &= ((bk >> bit) & 1u) ? set_b : ~set_b;
        }
        uint32_t base_r = 0, base_i = 0;
        if (act) {
            base_r = cnt_reads[bk * WP + warp];
            base_i = cnt_items[bk * WP + warp];
        }
        __syncwarp();
        if (act) {
            const uint32_t lower = grp & ((1u << lane) - 1u);
            uint32_t pre = 0;
            for (uint32_t m = lower; m; m &= m - 1u) pre += (uint32_t)read_items[cb + __ffs(m) - 1];
            const uint32_t pos = base_r + (uint32_t)__popc(lower);
            sorted_read[pos] = r;
            item_start[pos] = (int32_t)(base_i + pre);
            if ((grp >> lane) == 1u) {   // the group's last lane moves the running base on
                cnt_reads[bk * WP + warp] = base_r + (uint32_t)__popc(grp);
                cnt_items[bk * WP + warp] = base_i + pre + (uint32_t)items;
            }
        }
        __syncwarp();
    }
    __syncthreads();

    // the guide: the sorted place holding item g * gstep, for every g (each item lies in
    // exactly one place's range, so each entry has one writer)
    const int64_t I = item_start[R];
    int lg_g = 4;
    while (((int64_t)kGuide << lg_g) < I) lg_g++;
    for (int a = tid; a < R; a += blockDim.x) {
        const int64_t s0 = item_start[a], s1 = item_start[a + 1];
        for (int64_t g = (s0 + (1 << lg_g) - 1) >> lg_g; (g << lg_g) < s1; g++) guide[g] = a;
    }
    __syncthreads();

    // ---- 2. work items, claimed in plan order ----
    const bool aligned = ((uintptr_t)P.text & 15u) == 0;
    const bool out_aligned = ((uintptr_t)P.out & 15u) == 0;
    const uint64_t pol = policy_evict_first();
    Sink K{};
    K.out = P.out;
    K.defer = P.defer + (int64_t)blockIdx.x * P.defer_per_cta;
    K.defer_cap = P.defer_per_cta;
    K.defer_count = dcount;
    uint8_t *mybuf = tbuf + (size_t)warp * 2 * kSlot;
    // work item `it`: the last sorted place whose first item is <= it (a read with no
    // items shares its first item with the next place), its chunk from shared memory,
    // and its read's bounds and table loaded for later
    auto locate = [&](int64_t it) {
        const int64_t g = it >> lg_g;
        int a = guide[g], b = ((g + 1) << lg_g) < I ? guide[g + 1] : R - 1;
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if ((int64_t)item_start[mid] <= it) a = mid;
            else b = mid - 1;
        }
        const int32_t r = sorted_read[a];
        FusedItem f;
        f.base = ((int64_t)read_chunk[r] + (it - item_start[a])) << kShift;
        f.lo = P.read_off[r];
        f.hi = P.read_off[r + 1];
        f.set = P.read_set[r];
        return f;
    };
    // start copying the bytes of the item at `cbase`, and the 64 after it, into buffer b
    auto fetch = [&](int64_t cbase, int b) {
        const uint32_t dst = smem_addr(mybuf + b * kSlot);
        for (int c = lane; c < kBuf / 16; c += 32) {
            const int64_t p = cbase + 16 * c;
            const int64_t left = P.n - p;
            const uint32_t nb = left >= 16 ? 16u : (left > 0 ? (uint32_t)left : 0u);
            cp_async16(dst + 16 * c, P.text + (nb ? p : 0), nb);
        }
        cp_async_commit();
    };
    // the CTA's t-th item: run t / kDealRun of this CTA's runs, item t mod kDealRun of it
    // (increasing in t, so the first one past the end ends the claims)
    auto item_of = [&](uint32_t t) -> int64_t {
        return ((int64_t)(t / kDealRun) * gridDim.x + blockIdx.x) * kDealRun + (t % kDealRun);
    };
    // claims: lane 0 holds the answer of the claim after the next
    uint32_t pending = 0;
    if (lane == 0) pending = atomicAdd(claimed, 1u);
    int64_t it = item_of(__shfl_sync(kFull, pending, 0));
    if (lane == 0) pending = atomicAdd(claimed, 1u);
    FusedItem cur{};
    // start copying the table descriptor of an item into slot b (one group; empty for a
    // table index outside the set list)
    auto fetch_table = [&](int32_t set, int b) {
        if (set >= 0 && set < P.n_sets && lane < kTableCopy / 16)
            cp_async16(smem_addr(mybuf + b * kSlot + kBuf) + 16 * lane,
                       reinterpret_cast<const uint8_t *>(P.sets + set) + 16 * lane, 16);
        cp_async_commit();
    };
    if (it < I) {
        cur = locate(it);
        if (aligned) fetch(cur.base, 0);
        fetch_table(cur.set, 0);
    }
    for (int k = 0; it < I; k ^= 1) {
        const int64_t nxt = item_of(__shfl_sync(kFull, pending, 0));
        const bool more = nxt < I;
        FusedItem nx{};
        if (more) {
            if (lane == 0) pending = atomicAdd(claimed, 1u);
            nx = locate(nxt);
            if (aligned) fetch(nx.base, k ^ 1);
        }
        // everything but the next item's text: this item's text and table descriptor
        if (aligned && more) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncwarp();
        if (cur.set < 0 || cur.set >= P.n_sets) {
            if (lane == 0) record_error(P.sets[0].status, PFAC_ERR_INVALID_ARG);
        } else {
            const DeviceTable &T = *reinterpret_cast<const DeviceTable *>(mybuf + k * kSlot + kBuf);
            const int64_t cbase = cur.base;
            const int64_t rs = min(max(cur.lo, (int64_t)0), P.n), re = min(max(cur.hi, rs), P.n);
            const int64_t p0 = cbase + (int64_t)LW * lane;
            const uint8_t *buf = mybuf + k * kSlot;
            // 16 bytes from byte `o` of the item: from the warp's buffer, or from the text
            auto word = [&](int o, uint32_t *bad16) -> uint32_t {
                if (aligned) return pack16_scan(lds_v4(buf + o), bad16);
                return ascii16(P.text, P.n, cbase + o, false, bad16);
            };
            uint32_t x0, x1, x2, x3, b0, b1, b2, b3;
            if constexpr (LW == 16) {
                uint32_t h = 0, hb = 0xFFFFu;
                x0 = word(16 * lane, &b0);
                // the bases after the item, unless the read ends within it
                if (cbase + kItem < re && lane < 3) h = word(kItem + 16 * lane, &hb);
                const uint32_t d1 = __shfl_down_sync(kFull, x0, 1), e1 = __shfl_down_sync(kFull, b0, 1);
                const uint32_t d2 = __shfl_down_sync(kFull, x0, 2), e2 = __shfl_down_sync(kFull, b0, 2);
                const uint32_t d3 = __shfl_down_sync(kFull, x0, 3), e3 = __shfl_down_sync(kFull, b0, 3);
                const uint32_t g1 = __shfl_sync(kFull, h, (lane + 1) & 31), f1 = __shfl_sync(kFull, hb, (lane + 1) & 31);
                const uint32_t g2 = __shfl_sync(kFull, h, (lane + 2) & 31), f2 = __shfl_sync(kFull, hb, (lane + 2) & 31);
                const uint32_t g3 = __shfl_sync(kFull, h, (lane + 3) & 31), f3 = __shfl_sync(kFull, hb, (lane + 3) & 31);
                x1 = lane < 31 ? d1 : g1;
                b1 = lane < 31 ? e1 : f1;
                x2 = lane < 30 ? d2 : g2;
                b2 = lane < 30 ? e2 : f2;
                x3 = lane < 29 ? d3 : g3;
                b3 = lane < 29 ? e3 : f3;
            } else {
                uint32_t h0 = 0, h1 = 0, hb0 = 0xFFFFu, hb1 = 0xFFFFu;
                x0 = word(32 * lane, &b0);
                x1 = word(32 * lane + 16, &b1);
                if (cbase + kItem < re && lane == 0) {
                    h0 = word(kItem, &hb0);
                    h1 = word(kItem + 16, &hb1);
                }
                const uint32_t d2 = __shfl_down_sync(kFull, x0, 1), e2 = __shfl_down_sync(kFull, b0, 1);
                const uint32_t d3 = __shfl_down_sync(kFull, x1, 1), e3 = __shfl_down_sync(kFull, b1, 1);
                const uint32_t g2 = __shfl_sync(kFull, h0, 0), f2 = __shfl_sync(kFull, hb0, 0);
                const uint32_t g3 = __shfl_sync(kFull, h1, 0), f3 = __shfl_sync(kFull, hb1, 0);
                x2 = lane < 31 ? d2 : g2;
                b2 = lane < 31 ? e2 : f2;
                x3 = lane < 31 ? d3 : g3;
                b3 = lane < 31 ? e3 : f3;
            }
            uint64_t bad = (uint64_t)b0 | ((uint64_t)b1 << 16) | ((uint64_t)b2 << 32) | ((uint64_t)b3 << 48);
            const int64_t rem_read = re - p0;   // walks stop at the read's end
            if (rem_read < 64) bad |= rem_read > 0 ? (~0ull << rem_read) : ~0ull;
            // this lane's offsets inside the read
            const int64_t va = max(rs, p0) - p0, vb = min(re, p0 + LW) - p0;
            uint32_t valid = 0;
            if (vb > va) {
                const uint32_t span = (uint32_t)(vb - va);
                valid = (span >= 32 ? 0xFFFFFFFFu : ((1u << span) - 1u)) << (uint32_t)va;
            }
            scan_lane_batch<false, false, false, true, LW>(T, K, nullptr, nullptr, P.walk_loads, (uint32_t)cur.set,
                                                           P.text, nullptr, re, cbase, lane, x0, x1, x2, x3, bad,
                                                           valid, out_aligned, pol);
        }
        // the slot just read is the one the next fetches fill; the next item's table
        // descriptor is fetched now, its table index long loaded
        __syncwarp();
        if (more) fetch_table(nx.set, k ^ 1);
        it = nxt;
        cur = nx;
    }

    // ---- 3. the long walks this CTA's items deferred ----
    __syncthreads();
    const int64_t nd = min((int64_t)*dcount, P.defer_per_cta);
    for (int64_t i = tid; i < nd; i += blockDim.x) {
        const DeferItem d = K.defer[i];
        const DeviceTable T = P.sets[d.q_set >> 16];
        emit_match<false>(K, d.gp, walk_global<false>(T, P.text, nullptr, d.gp + d.span, d.gp, d.s,
                                                       (int)(d.q_set & 0xFFFFu), d.best));
    }
}

// Work items of reads that do not overlap: at most one partial item per read plus one
// per 512 bases.
static int64_t item_capacity(int64_t n, int32_t n_reads) { return n / 512 + (int64_t)n_reads + 1; }

int64_t batch_scratch_bytes(int64_t n, int32_t n_reads, int64_t defer_cap)
{
    const int64_t words = (n + 15) / 16, bw = (n + 31) / 32;
    return 256 + ((words * 4 + 255) & ~255LL) + (((bw + 1) * 4 + 255) & ~255LL) +
           ((((int64_t)n_reads + 1) * 8 + 255) & ~255LL) + ((item_capacity(n, n_reads) * 4 + 255) & ~255LL) +
           defer_cap * (int64_t)sizeof(DeferItem);
}

int launch_batched(const DeviceTable *d_sets, int32_t n_sets, const uint8_t *texts, int64_t n, const int64_t *read_off,
                   const int32_t *read_set, int32_t n_reads, int32_t *out, void *scratch, int64_t defer_cap,
                   const BatchConfig &bc, cudaStream_t st, const DeviceProps &dp)
{
    const int lw = bc.lane_offsets == 32 ? 32 : 16;
    const int blocks_per_sm = std::min(8, std::max(1, bc.blocks_per_sm));
    if (n == 0 || n_reads == 0) return PFAC_OK;
    uint8_t *p = (uint8_t *)scratch;
    unsigned long long *counters = (unsigned long long *)p;       // [1]: deferred walks
    p += 256;
    const int64_t words = (n + 15) / 16, bw = (n + 31) / 32;
    uint32_t *packed = (uint32_t *)p;
    p += (words * 4 + 255) & ~255LL;
    uint32_t *invalid = (uint32_t *)p;
    p += ((bw + 1) * 4 + 255) & ~255LL;
    int64_t *item_start = (int64_t *)p;
    p += ((((int64_t)n_reads + 1) * 8) + 255) & ~255LL;
    const int64_t item_cap = item_capacity(n, n_reads);
    int32_t *item_read = (int32_t *)p;
    p += (item_cap * 4 + 255) & ~255LL;
    DeferItem *defer = (DeferItem *)p;
    const int64_t fused_items_max = n / (32 * lw) + (int64_t)n_reads + 1;
    const int fused_threads = 256 * std::min(4, blocks_per_sm);
    if (n_reads <= kFusedMaxReads && fused_items_max < (1LL << 30) &&
        fused_smem_bytes(fused_threads / 32, n_reads, lw) <= (size_t)dp.smem_optin) {
        // one launch: every CTA plans the batch, scans the items dealt to it and finishes
        // the walks its items deferred
        const size_t smem = fused_smem_bytes(fused_threads / 32, n_reads, lw);
        {
            // the most any batch can need, set once per kernel and device (so that a call
            // being captured into a graph never sets it)
            static std::mutex mu;
            static bool done[2][64];
            std::lock_guard<std::mutex> lk(mu);
            bool &d = done[lw == 32][dp.device & 63];
            if (!d) {
                const void *kern =
                    lw == 32 ? (const void *)fused_batched_kernel<32> : (const void *)fused_batched_kernel<16>;
                const size_t most = std::min<size_t>(fused_smem_bytes(32, kFusedMaxReads, lw), dp.smem_optin);
                if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) != cudaSuccess)
                    return PFAC_ERR_CUDA;
                d = true;
            }
        }
        FusedParams F{};
        F.sets = d_sets;
        F.n_sets = n_sets;
        F.text = texts;
        F.n = n;
        F.read_off = read_off;
        F.read_set = read_set;
        F.n_reads = n_reads;
        F.out = out;
        F.defer = defer;
        F.defer_per_cta = std::max<int64_t>(1, defer_cap / dp.num_sms);
        F.walk_loads = bc.walk_loads > 0 ? bc.walk_loads : 4;   // measured best on the batched workload
        if (lw == 32) fused_batched_kernel<32><<<dp.num_sms, fused_threads, smem, st>>>(F);
        else fused_batched_kernel<16><<<dp.num_sms, fused_threads, smem, st>>>(F);
        return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
    }
    if (cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    const int pack_blocks = (int)std::min<int64_t>((bw + 255) / 256, (int64_t)dp.num_sms * 16);
    pack_bits_kernel<<<std::max(1, pack_blocks), 256, 0, st>>>(texts, n, packed, invalid);
    plan_kernel<<<1, 1024, 0, st>>>(read_off, n_reads, n, 32 * lw, item_start, item_read, item_cap);
    BatchParams P{};
    P.sets = d_sets;
    P.n_sets = n_sets;
    P.packed = packed;
    P.invalid = invalid;
    P.n = n;
    P.read_off = read_off;
    P.read_set = read_set;
    P.n_reads = n_reads;
    P.item_start = item_start;
    P.item_read = item_read;
    P.item_cap = item_cap;
    P.out = out;
    P.defer = defer;
    P.defer_cap = defer_cap;
    P.defer_count = counters + 1;
    P.item = 32 * lw;
    P.walk_loads = bc.walk_loads > 0 ? bc.walk_loads : 2;
    if (lw == 32) batched_scan_kernel<32><<<dp.num_sms * blocks_per_sm, 256, 0, st>>>(P);
    else batched_scan_kernel<16><<<dp.num_sms * blocks_per_sm, 256, 0, st>>>(P);
    batched_tail_kernel<<<dp.num_sms * 4, 256, 0, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}
}  // namespace pfac
