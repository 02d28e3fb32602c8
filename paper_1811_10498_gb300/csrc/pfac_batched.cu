// sm_103a kernels of the batched scan and their launcher: many reads of uneven length,
// each against its own resident table, in one persistent launch (plus the pack, plan and
// tail kernels around it). The walk itself is the one of the scan kernels
// (pfac_device.cuh), bounded by each read's end.
#include <stdint.h>

#include <algorithm>

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
