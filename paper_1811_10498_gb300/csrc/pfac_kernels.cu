// sm_103a kernels of the PFAC scan and their launchers.
//
// The scan (Section IV): every text offset walks the failure-less goto trie from the
// root, one edge per base, until no edge exists, and reports the longest pattern that
// ended on the way. The paper's kernel (Section V-B) runs one thread per character
// over a 4-column table in global memory; kernel 1 below keeps that structure (one
// thread per offset, 16-byte rows), kernel 2 is the Blackwell design:
//   * the text of a tile plus a halo of max_len bases is staged into shared memory by
//     a TMA bulk copy (double-buffered, mbarrier-tracked, bounded waits);
//   * phase 1 resolves every offset of the tile with one lookup in a k-mer jump table
//     (the first k steps of the walk, an exact shortcut through the same trie) and one
//     ALU step through the compact node word it returns; offsets whose walk goes on are
//     pushed to a shared-memory queue with one atomic per warp;
//   * phase 2 walks the queued offsets over 4-byte compact nodes: a window of the
//     breadth-first levels right below the jump depth sits in shared memory, deeper
//     states come from L2/HBM;
//   * results are staged in shared memory and leave by a TMA bulk store with an
//     evict-first L2 hint (or are compacted into (offset, id) pairs with one atomic per
//     warp).
#include <stdint.h>
#include <stdio.h>

#include <algorithm>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace pfac {

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the given phase of an mbarrier, giving up after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((int64_t)(global_timer_ns() - t0) > limit_ns) return false;
    }
}

// Bulk (TMA) copy global -> shared, completion counted on an mbarrier. Source and
// destination 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Bulk (TMA) copy shared -> global with an L2 eviction-priority hint.
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes, uint64_t policy)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(src), "r"(bytes), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void record_error(int32_t *status, int32_t code)
{
    if (status) atomicCAS(status, PFAC_OK, code);
}

// ---------------------------------------------------------------------------
// Base codes. A=0x41, C=0x43, G=0x47, T=0x54: ((b >> 1) & 3) ^ ((b >> 2) & 1)
// maps them to 0, 1, 2, 3.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int base_code_or_neg(uint32_t b)
{
    const bool ok = (b == 0x41u) | (b == 0x43u) | (b == 0x47u) | (b == 0x54u);
    const int c = (int)(((b >> 1) & 3u) ^ ((b >> 2) & 1u));
    return ok ? c : -1;
}

// Four ASCII bytes -> four 2-bit codes in the low 8 bits, plus a 4-bit mask of bytes
// that are not A, C, G or T.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t *bad4)
{
    const uint32_t okA = __vcmpeq4(x, 0x41414141u), okC = __vcmpeq4(x, 0x43434343u);
    const uint32_t okG = __vcmpeq4(x, 0x47474747u), okT = __vcmpeq4(x, 0x54545454u);
    const uint32_t ok = okA | okC | okG | okT;           // 0xFF per valid byte
    const uint32_t t = (((x >> 1) & 0x03030303u) ^ ((x >> 2) & 0x01010101u)) & ok;
    const uint32_t codes = (t & 0x3u) | ((t >> 6) & 0xCu) | ((t >> 12) & 0x30u) | ((t >> 18) & 0xC0u);
    const uint32_t bad = ~ok;
    *bad4 = (bad & 1u) | ((bad >> 7) & 2u) | ((bad >> 14) & 4u) | ((bad >> 21) & 8u);
    return codes;
}

// Sixteen ASCII bytes -> one packed word, plus a 16-bit mask of invalid bytes.
__device__ __forceinline__ uint32_t pack16(uint4 v, uint32_t *bad16)
{
    uint32_t b0, b1, b2, b3;
    const uint32_t c0 = pack4(v.x, &b0), c1 = pack4(v.y, &b1), c2 = pack4(v.z, &b2), c3 = pack4(v.w, &b3);
    *bad16 = b0 | (b1 << 4) | (b2 << 8) | (b3 << 12);
    return c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
}

// ---------------------------------------------------------------------------
// Packing (ASCII -> 2 bits per base)
// ---------------------------------------------------------------------------

__global__ void pack_kernel(const uint8_t *__restrict__ text, int64_t len, uint32_t *__restrict__ packed,
                            int32_t *status, unsigned long long *bad)
{
    const int64_t n_words = (len + 15) >> 4;
    const bool aligned = ((uintptr_t)text & 15u) == 0;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b0 = w << 4;
        uint32_t word, badm;
        if (aligned && b0 + 16 <= len) {
            word = pack16(__ldg(reinterpret_cast<const uint4 *>(text + b0)), &badm);
        } else {
            word = 0;
            badm = 0;
            for (int i = 0; i < 16 && b0 + i < len; i++) {
                const int c = base_code_or_neg(text[b0 + i]);
                if (c < 0) badm |= 1u << i;
                else word |= (uint32_t)c << (2 * i);
            }
        }
        packed[w] = word;
        if (badm) {
            if (status) *status = PFAC_ERR_BAD_SYMBOL;
            if (bad) atomicMin(bad, (unsigned long long)(b0 + __ffs(badm) - 1));
        }
    }
}

int launch_pack(const uint8_t *text, int64_t len, uint32_t *packed, int32_t *status, int64_t *bad,
                cudaStream_t st, const DeviceProps &dp)
{
    if (status && cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (bad && cudaMemsetAsync(bad, 0xFF, sizeof(int64_t), st) != cudaSuccess) return PFAC_ERR_CUDA;
    const int64_t n_words = (len + 15) >> 4;
    if (n_words == 0) return PFAC_OK;
    const int threads = 256;
    const int64_t want = (n_words + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)dp.num_sms * 16);
    pack_kernel<<<blocks, threads, 0, st>>>(text, len, packed, status, (unsigned long long *)bad);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Kernel 1: one thread per offset over 16-byte rows in global memory (the paper's
// kernel structure, Section V-B). Also the fallback for tables without compact nodes
// and for unaligned buffers.
// ---------------------------------------------------------------------------

template <bool PACKED, bool COMPACT>
__global__ void __launch_bounds__(256) walk_rows_kernel(DeviceTable t, const void *__restrict__ text,
                                                        int64_t n, int32_t *__restrict__ out,
                                                        int64_t *__restrict__ c_off,
                                                        int32_t *__restrict__ c_ids, int64_t cap,
                                                        unsigned long long *count)
{
    const int32_t *__restrict__ rows = t.rows;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // Uniform trip count across the grid so that warp-wide ballots see every lane.
    const int64_t base_lo = (int64_t)blockIdx.x * blockDim.x;
    for (int64_t i0 = base_lo; i0 < n; i0 += stride) {
        const int64_t i = i0 + (first - base_lo);
        int32_t res = 0;
        if (i < n) {
            int32_t s = 0, best = 0;
            const int64_t end = min(n, i + (int64_t)t.max_len);
            for (int64_t k = i; k < end; k++) {
                int c;
                if (PACKED) {
                    c = (int)((__ldg((const uint32_t *)text + (k >> 4)) >> ((k & 15) * 2)) & 3u);
                } else {
                    c = base_code_or_neg(__ldg((const uint8_t *)text + k));
                    if (c < 0) break;
                }
                const int32_t e = __ldg(rows + 4 * (int64_t)s + c);
                if (e == 0) break;
                s = e & 0x7FFFFFFF;
                if (e < 0) best = s;
            }
            res = best ? __ldg(t.out_id + best) : 0;
            if (!COMPACT) out[i] = res;
        }
        if (COMPACT) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, res != 0);
            if (m) {
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                unsigned long long b = 0;
                if (lane == leader) b = atomicAdd(count, (unsigned long long)__popc(m));
                b = __shfl_sync(0xFFFFFFFFu, b, leader);
                if (res) {
                    const int64_t k = (int64_t)b + __popc(m & ((1u << lane) - 1));
                    if (k < cap) { c_off[k] = i; c_ids[k] = res; }
                }
            }
        }
    }
}

int launch_walk_rows_any(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out,
                         int64_t *c_off, int32_t *c_ids, int64_t cap, unsigned long long *count,
                         cudaStream_t st, const DeviceProps &dp)
{
    if (count && cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (n == 0) return PFAC_OK;
    const int threads = 256;
    const int64_t want = (n + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)dp.num_sms * 8);
    const bool compact = c_off != nullptr;
    if (packed) {
        if (compact) walk_rows_kernel<true, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
        else walk_rows_kernel<true, false><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
    } else {
        if (compact) walk_rows_kernel<false, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
        else walk_rows_kernel<false, false><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
    }
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

int launch_walk_rows(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out,
                     cudaStream_t st, const DeviceProps &dp)
{
    return launch_walk_rows_any(t, text, packed, n, out, nullptr, nullptr, 0, nullptr, st, dp);
}

// ---------------------------------------------------------------------------
// Kernel 2: tiled, TMA-staged, jump table + compact nodes.
// ---------------------------------------------------------------------------

struct TiledParams {
    DeviceTable t;
    const void *text;
    int64_t n;              // bases
    int64_t n_units;        // packed: words, ASCII: bytes (what the text buffer holds)
    int32_t *out;
    int64_t *c_off;
    int32_t *c_ids;
    int64_t cap;
    unsigned long long *count;
    int64_t n_tiles;
    int32_t tile;           // bases per tile, multiple of 64
    int32_t jump_smem;      // jump table copied into shared memory
    uint32_t win_lo;        // node window [win_lo, win_lo + win_len) in shared memory
    uint32_t win_len;
    int32_t buf_units;      // packed words (or ASCII bytes) per text buffer
    int32_t conv_words;     // ASCII: packed words converted per tile
    uint32_t off_jump, off_win, off_text0, off_text1, off_conv, off_inv, off_out, off_queue;
    int64_t timeout_ns;
};

struct TiledLayout {
    uint32_t off_jump, off_win, off_text0, off_text1, off_conv, off_inv, off_out, off_queue, total;
    int32_t buf_units, conv_words;
};

static inline uint32_t align16(uint64_t x) { return (uint32_t)((x + 15) & ~(uint64_t)15); }

// Shared memory without the node window. Layout: [mbarriers, queue count][jump]
// [window][text 0][text 1][converted text][invalid mask][staged results][queue].
static TiledLayout tiled_layout(int32_t tile, int32_t max_len, int32_t jump_k, bool jump_smem, bool packed,
                                uint32_t win_len)
{
    TiledLayout L{};
    // packed words a tile's walks can touch: tile, halo of max_len bases, one word of
    // look-ahead for the 16-base register window.
    const int32_t words = tile / 16 + (max_len + 31) / 16 + 1;
    uint64_t off = 32;
    L.off_jump = (uint32_t)off;
    if (jump_smem) off += align16((uint64_t)4 << (2 * jump_k));
    L.off_win = (uint32_t)off;
    off += align16((uint64_t)win_len * 4);
    if (packed) {
        L.buf_units = words;
        L.conv_words = 0;
        L.off_text0 = (uint32_t)off; off += align16((uint64_t)words * 4);
        L.off_text1 = (uint32_t)off; off += align16((uint64_t)words * 4);
        L.off_conv = L.off_inv = 0;
    } else {
        L.buf_units = words * 16;   // bytes
        L.conv_words = words;
        L.off_text0 = (uint32_t)off; off += align16((uint64_t)words * 16);
        L.off_text1 = (uint32_t)off; off += align16((uint64_t)words * 16);
        L.off_conv = (uint32_t)off; off += align16((uint64_t)words * 4);
        // one bit per base: (words + 1) / 2 words, plus two sentinel words (four
        // 16-bit halves set to "invalid" past the converted bases)
        L.off_inv = (uint32_t)off; off += align16((((uint64_t)words + 1) / 2 + 2) * 4);
    }
    L.off_out = (uint32_t)off; off += align16((uint64_t)tile * 4);
    L.off_queue = (uint32_t)off; off += align16((uint64_t)tile * 8);
    L.total = (uint32_t)off;
    return L;
}

// Consecutive valid bases from p (at most maxrun), from the invalid-byte mask.
__device__ __forceinline__ int valid_run(const uint32_t *inv, int p, int maxrun)
{
    int w = p >> 5;
    uint32_t bits = inv[w] >> (p & 31);
    int run = 32 - (p & 31);
    if (bits) return min(__ffs(bits) - 1, maxrun);
    while (run < maxrun) {
        bits = inv[++w];
        if (bits) return min(run + __ffs(bits) - 1, maxrun);
        run += 32;
    }
    return maxrun;
}

__device__ __forceinline__ uint32_t window16(const uint32_t *tw, int pos)
{
    return __funnelshift_r(tw[pos >> 4], tw[(pos >> 4) + 1], (pos & 15) * 2);
}

__device__ __forceinline__ uint32_t node_at(uint32_t s, const uint32_t *sw, uint32_t win_lo, uint32_t win_len,
                                            const uint32_t *__restrict__ nodes)
{
    const uint32_t rel = s - win_lo;
    return rel < win_len ? sw[rel] : __ldg(nodes + s);
}

template <bool PACKED, bool COMPACT>
__global__ void __launch_bounds__(1024, 1) tiled_kernel(const TiledParams P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    uint32_t *qcount = reinterpret_cast<uint32_t *>(smem + 16);
    uint32_t *sj = reinterpret_cast<uint32_t *>(smem + P.off_jump);
    uint32_t *sw = reinterpret_cast<uint32_t *>(smem + P.off_win);
    int32_t *out_s = reinterpret_cast<int32_t *>(smem + P.off_out);
    uint2 *queue = reinterpret_cast<uint2 *>(smem + P.off_queue);
    uint32_t *conv = reinterpret_cast<uint32_t *>(smem + P.off_conv);
    uint32_t *inv = reinterpret_cast<uint32_t *>(smem + P.off_inv);

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
    const DeviceTable &T = P.t;
    const int K = T.jump_k;
    const uint32_t kmask = (K >= 16) ? 0xFFFFFFFFu : ((1u << (2 * K)) - 1u);
    const int max_len = T.max_len;
    const int64_t n = P.n;
    const uint32_t bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);
    const uint32_t text_off[2] = {P.off_text0, P.off_text1};

    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        fence_mbar_init();
    }
    // Table parts kept in shared memory for the whole (persistent) kernel.
    if (P.jump_smem) {
        const int64_t E = (int64_t)1 << (2 * K);
        for (int64_t i = tid; i < E; i += nthr) sj[i] = __ldg(T.jump + i);
    }
    for (uint32_t i = tid; i < P.win_len; i += nthr) sw[i] = __ldg(T.nodes + P.win_lo + i);
    __syncthreads();

    const int unit_bytes = PACKED ? 4 : 1;
    const int64_t tile_units = PACKED ? (P.tile >> 4) : P.tile;  // units per tile step
    uint64_t policy = 0;
    if (tid == 0) policy = policy_evict_first();

    // Issue the staging copy of tile `tt` into buffer `b`; returns the units that the
    // threads must still load by hand (the ragged < 16-byte tail).
    auto issue = [&](int64_t tt, int b) {
        const int64_t u0 = tt * tile_units;
        const int64_t cnt = min((int64_t)P.buf_units, P.n_units - u0);
        const uint32_t bytes = (uint32_t)((cnt * unit_bytes) & ~(int64_t)15);
        const uint32_t bar = b ? bar1 : bar0;
        fence_proxy_async();
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes) bulk_load(smem_addr(smem + text_off[b]), (const uint8_t *)P.text + u0 * unit_bytes, bytes, bar);
    };

    int64_t t = blockIdx.x;
    if (tid == 0 && t < P.n_tiles) issue(t, 0);

    for (int it = 0; t < P.n_tiles; t += gridDim.x, it++) {
        const int b = it & 1;
        const uint32_t parity = (uint32_t)((it >> 1) & 1);
        const int64_t b0 = t * (int64_t)P.tile;
        const int tile_len = (int)min((int64_t)P.tile, n - b0);
        const int64_t tn = t + gridDim.x;
        if (tid == 0 && tn < P.n_tiles) issue(tn, b ^ 1);

        const bool ok = mbar_wait_bounded(b ? bar1 : bar0, parity, P.timeout_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                record_error(T.status, PFAC_ERR_TIMEOUT);
                // Let this CTA's own copies finish (again with a limit) before leaving.
                mbar_wait_bounded(b ? bar1 : bar0, parity, P.timeout_ns);
                if (tn < P.n_tiles) mbar_wait_bounded(b ? bar0 : bar1, (uint32_t)(((it + 1) >> 1) & 1), P.timeout_ns);
                bulk_wait_all();
            }
            return;
        }
        // Ragged tail of the staged text (the bulk copy moves whole 16-byte chunks).
        {
            const int64_t u0 = t * tile_units;
            const int64_t cnt = min((int64_t)P.buf_units, P.n_units - u0);
            const int64_t bulk_units = ((cnt * unit_bytes) & ~(int64_t)15) / unit_bytes;
            uint8_t *buf = smem + text_off[b];
            if (PACKED) {
                if (tid < cnt - bulk_units)
                    reinterpret_cast<uint32_t *>(buf)[bulk_units + tid] =
                        __ldg((const uint32_t *)P.text + u0 + bulk_units + tid);
            } else {
                if (tid < cnt - bulk_units) buf[bulk_units + tid] = __ldg((const uint8_t *)P.text + u0 + bulk_units + tid);
            }
            if (!PACKED) {
                __syncthreads();
                // ASCII -> packed words + invalid mask; bytes past the loaded ones are invalid.
                const uint4 *raw = reinterpret_cast<const uint4 *>(buf);
                uint16_t *inv16 = reinterpret_cast<uint16_t *>(inv);
                for (int w = tid; w < P.conv_words; w += nthr) {
                    uint32_t badm;
                    const uint32_t word = pack16(raw[w], &badm);
                    const int64_t have = cnt - (int64_t)w * 16;
                    if (have < 16) badm |= have <= 0 ? 0xFFFFu : (0xFFFFu << have) & 0xFFFFu;
                    conv[w] = word;
                    inv16[w] = (uint16_t)badm;
                }
                if (tid < 4) inv16[P.conv_words + tid] = 0xFFFFu;
            }
        }
        if (tid == 0) {
            if (!COMPACT) bulk_wait_read_all();   // previous tile's result store has read out_s
            *qcount = 0;
        }
        __syncthreads();

        const uint32_t *tw = PACKED ? reinterpret_cast<const uint32_t *>(smem + text_off[b]) : conv;

        // ---- phase 1: jump lookup + one step for every offset -------------------
        for (int r0 = 0; r0 < tile_len; r0 += nthr) {
            const int p = r0 + tid;
            bool pend = false;
            uint32_t item_s = 0, item_f = 0;
            if (p < tile_len) {
                const int64_t gp = b0 + p;
                const int maxrun = (int)min(n - gp, (int64_t)max_len);
                const int lim = PACKED ? maxrun : valid_run(inv, p, maxrun);
                int32_t res = 0;
                if (K > 0 && lim >= K) {
                    const uint32_t win = window16(tw, p);
                    const uint32_t kmer = win & kmask;
                    const uint32_t e = P.jump_smem ? sj[kmer] : __ldg(T.jump + kmer);
                    if ((e & 0x1Fu) == 0) {
                        res = (int32_t)(e >> kNodeFirstShift);
                    } else {
                        const bool pf = (e & kNodeTermBit) != 0;
                        if (lim > K) {
                            const uint32_t c = (win >> (2 * K)) & 3u;
                            if ((e >> c) & 1u) {
                                pend = true;
                                item_s = (e >> kNodeFirstShift) + __popc(e & ((1u << c) - 1u));
                                item_f = pf;
                            }
                        }
                        if (!pend && pf) {
                            const int32_t bs = __ldg(T.jump_best + kmer);
                            res = bs ? __ldg(T.out_id + bs) : 0;
                        }
                    }
                } else if (lim > 0) {
                    pend = true;      // too close to the end (or no jump table): walk from the root
                }
                if (!pend) out_s[p] = res;
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, pend);
            if (m) {
                const int leader = __ffs(m) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(qcount, (uint32_t)__popc(m));
                base = __shfl_sync(0xFFFFFFFFu, base, leader);
                if (pend) queue[base + __popc(m & ((1u << lane) - 1u))] = make_uint2(item_s, (uint32_t)p | (item_f << 31));
            }
        }
        __syncthreads();

        // ---- phase 2: walk the queued offsets ----------------------------------
        const int nq = (int)*qcount;
        for (int i = tid; i < nq; i += nthr) {
            const uint2 item = queue[i];
            const int p = (int)(item.y & 0x7FFFFFFFu);
            uint32_t s = item.x;
            const int64_t gp = b0 + p;
            const int maxrun = (int)min(n - gp, (int64_t)max_len);
            const int lim = PACKED ? maxrun : valid_run(inv, p, maxrun);
            int q;
            uint32_t best = 0, nd;
            if (s == 0) {
                q = 0;
                nd = node_at(0, sw, P.win_lo, P.win_len, T.nodes);
            } else {
                q = K + 1;
                if (item.y >> 31) best = (uint32_t)__ldg(T.jump_best + (window16(tw, p) & kmask));
                nd = node_at(s, sw, P.win_lo, P.win_len, T.nodes);
                if (nd & kNodeTermBit) best = s;
            }
            uint32_t win = 0;
            int avail = 0;
            while (q < lim) {
                if (avail == 0) { win = window16(tw, p + q); avail = 16; }
                const uint32_t c = win & 3u;
                win >>= 2;
                avail--;
                if (!((nd >> c) & 1u)) break;
                s = (nd >> kNodeFirstShift) + __popc(nd & ((1u << c) - 1u));
                nd = node_at(s, sw, P.win_lo, P.win_len, T.nodes);
                if (nd & kNodeTermBit) best = s;
                q++;
            }
            out_s[p] = best ? __ldg(T.out_id + best) : 0;
        }

        // ---- results ------------------------------------------------------------
        if (!COMPACT) {
            fence_proxy_async();
            __syncthreads();
            const int bulk_n = tile_len & ~3;
            if (tid == 0 && bulk_n) {
                bulk_store(P.out + b0, smem_addr(out_s), (uint32_t)bulk_n * 4u, policy);
                bulk_commit();
            }
            if (tid < tile_len - bulk_n) P.out[b0 + bulk_n + tid] = out_s[bulk_n + tid];
        } else {
            __syncthreads();
            for (int r0 = (tid & ~31); r0 < tile_len; r0 += nthr) {
                const int p = r0 + lane;
                const int32_t v = p < tile_len ? out_s[p] : 0;
                const unsigned m = __ballot_sync(0xFFFFFFFFu, v != 0);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    unsigned long long base = 0;
                    if (lane == leader) base = atomicAdd(P.count, (unsigned long long)__popc(m));
                    base = __shfl_sync(0xFFFFFFFFu, base, leader);
                    if (v) {
                        const int64_t k = (int64_t)base + __popc(m & ((1u << lane) - 1u));
                        if (k < P.cap) { P.c_off[k] = b0 + p; P.c_ids[k] = v; }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0 && !COMPACT) bulk_wait_all();
}

int64_t tiled_smem_bytes(const DeviceTable &t, const TiledConfig &cfg, bool packed, int32_t *win_len_out,
                         int32_t *jump_smem_out, const DeviceProps &dp)
{
    const bool jump_smem = t.jump_k > 0 && t.jump_k <= 7;
    const TiledLayout base = tiled_layout(cfg.tile, t.max_len, t.jump_k, jump_smem, packed, 0);
    int64_t room = (int64_t)dp.smem_optin - base.total;
    if (room < 0) return -1;
    int64_t win = 0;
    if (t.nodes && cfg.smem_table_bytes >= 0) {
        int64_t budget = cfg.smem_table_bytes > 0 ? std::min<int64_t>(cfg.smem_table_bytes, room) : room;
        win = std::min<int64_t>(budget / 4, t.n_states - t.win_lo);
        if (win < 0) win = 0;
    }
    if (win_len_out) *win_len_out = (int32_t)win;
    if (jump_smem_out) *jump_smem_out = jump_smem;
    return tiled_layout(cfg.tile, t.max_len, t.jump_k, jump_smem, packed, (uint32_t)win).total;
}

template <bool PACKED, bool COMPACT>
static int launch_tiled_t(const TiledParams &P, int grid, int threads, uint32_t smem, cudaStream_t st)
{
    auto kern = tiled_kernel<PACKED, COMPACT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PFAC_ERR_CUDA;
    kern<<<grid, threads, smem, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

int launch_tiled(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out, int64_t *c_off,
                 int32_t *c_ids, int64_t cap, unsigned long long *count, const TiledConfig &cfg, cudaStream_t st,
                 const DeviceProps &dp)
{
    const bool compact = c_off != nullptr;
    if (compact && cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (n == 0) return PFAC_OK;
    if (!t.nodes || cfg.tile <= 0 || (cfg.tile & 63) || cfg.threads <= 0 || (cfg.threads & 31) ||
        cfg.threads > 1024 || cfg.tile > 32768)
        return PFAC_ERR_INVALID_ARG;
    int32_t win_len = 0, jump_smem = 0;
    const int64_t smem = tiled_smem_bytes(t, cfg, packed, &win_len, &jump_smem, dp);
    if (smem < 0 || smem > dp.smem_optin) return PFAC_ERR_UNSUPPORTED;
    const bool jsm = jump_smem != 0;
    const TiledLayout L = tiled_layout(cfg.tile, t.max_len, t.jump_k, jsm, packed, (uint32_t)win_len);
    TiledParams P{};
    P.t = t;
    P.text = text;
    P.n = n;
    P.n_units = packed ? (n + 15) / 16 : n;
    P.out = out;
    P.c_off = c_off;
    P.c_ids = c_ids;
    P.cap = cap;
    P.count = count;
    P.tile = cfg.tile;
    P.n_tiles = (n + cfg.tile - 1) / cfg.tile;
    P.jump_smem = jsm;
    P.win_lo = (uint32_t)t.win_lo;
    P.win_len = (uint32_t)win_len;
    P.buf_units = L.buf_units;
    P.conv_words = L.conv_words;
    P.off_jump = L.off_jump;
    P.off_win = L.off_win;
    P.off_text0 = L.off_text0;
    P.off_text1 = L.off_text1;
    P.off_conv = L.off_conv;
    P.off_inv = L.off_inv;
    P.off_out = L.off_out;
    P.off_queue = L.off_queue;
    P.timeout_ns = cfg.timeout_ns > 0 ? cfg.timeout_ns : 2000000000LL;
    const int64_t grid64 = std::min<int64_t>(P.n_tiles, (int64_t)dp.num_sms * std::max(1, cfg.ctas_per_sm));
    const int grid = (int)std::max<int64_t>(1, grid64);
    if (packed) {
        return compact ? launch_tiled_t<true, true>(P, grid, cfg.threads, L.total, st)
                       : launch_tiled_t<true, false>(P, grid, cfg.threads, L.total, st);
    }
    return compact ? launch_tiled_t<false, true>(P, grid, cfg.threads, L.total, st)
                   : launch_tiled_t<false, false>(P, grid, cfg.threads, L.total, st);
}

// ---------------------------------------------------------------------------
// Timeout probe (exercises the bounded wait without any fault or hang).
// ---------------------------------------------------------------------------

__global__ void timeout_probe_kernel(int32_t *status, int64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Nothing ever arrives on this barrier, so the wait must give up after limit_ns.
    const bool ok = mbar_wait_bounded(b, 0, limit_ns);
    if (!ok && threadIdx.x == 0) record_error(status, PFAC_ERR_TIMEOUT);
}

int launch_timeout_probe(int32_t *status, int64_t limit_ns, cudaStream_t st)
{
    timeout_probe_kernel<<<1, 32, 0, st>>>(status, limit_ns);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

int get_device_props(DeviceProps *p)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PFAC_ERR_CUDA;
    p->device = dev;
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->l2_bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->persist_l2_max, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess)
        return PFAC_ERR_CUDA;
    return PFAC_OK;
}

}  // namespace pfac
