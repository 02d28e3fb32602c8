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
#include <mutex>
#include <type_traits>

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

// Four ASCII bytes -> four 2-bit codes in the low 8 bits (a byte outside ACGT codes as
// A), plus a 4-bit mask of bytes that are not A, C, G or T. Byte-parallel arithmetic:
//   t      the code each byte would have if it were a base (see base_code_or_neg);
//   c8     t's four codes gathered into one byte by one multiply (the products of
//          different bytes land below bit 24 or above bit 31, without carries);
//   sel    the codes spread to one nibble each, a byte-permute selector that picks the
//          byte each code stands for out of "ACGT";
//   diff   zero exactly in the bytes that equal that byte, i.e. are bases;
//   nz     bit 7 of each nonzero byte of diff (the zero-byte test), gathered into 4 bits
//          by a second multiply.
// Checked against the per-byte definition for all 2^32 inputs.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t *bad4)
{
    const uint32_t t = ((x >> 1) & 0x03030303u) ^ ((x >> 2) & 0x01010101u);
    const uint32_t c8 = (t * 0x01041040u) >> 24;
    const uint32_t y = (c8 | (c8 << 4)) & 0x0F0Fu;
    const uint32_t sel = (y | (y << 2)) & 0x3333u;
    const uint32_t diff = x ^ __byte_perm(0x54474341u, 0u, sel);
    const uint32_t nz = (((diff & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | diff) & 0x80808080u;
    *bad4 = (nz * 0x00204081u) >> 28;
    return ((t & ~((nz >> 7) * 0xFFu)) * 0x01041040u) >> 24;
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
    // Each thread packs four consecutive words (64 bases): four independent 16-byte
    // loads in flight, one 16-byte store.
    const int64_t n_words = (len + 15) >> 4;
    const int64_t n_quads = (n_words + 3) >> 2;
    const bool aligned = (((uintptr_t)text | (uintptr_t)packed) & 15u) == 0;
    for (int64_t qd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qd < n_quads;
         qd += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w0 = qd << 2;
        const int64_t b0 = w0 << 4;
        uint32_t word[4], badm[4];
        if (aligned && b0 + 64 <= len) {
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = __ldg(reinterpret_cast<const uint4 *>(text + b0) + k);
#pragma unroll
            for (int k = 0; k < 4; k++) word[k] = pack16(v[k], &badm[k]);
            *reinterpret_cast<uint4 *>(packed + w0) = make_uint4(word[0], word[1], word[2], word[3]);
        } else {
            for (int k = 0; k < 4; k++) {
                word[k] = 0;
                badm[k] = 0;
                const int64_t bk = b0 + 16 * k;
                for (int i = 0; i < 16 && bk + i < len; i++) {
                    const int c = base_code_or_neg(text[bk + i]);
                    if (c < 0) badm[k] |= 1u << i;
                    else word[k] |= (uint32_t)c << (2 * i);
                }
                if (w0 + k < n_words) packed[w0 + k] = word[k];
            }
        }
        if (badm[0] | badm[1] | badm[2] | badm[3]) {
            if (status) *status = PFAC_ERR_BAD_SYMBOL;
            if (bad) {
                for (int k = 0; k < 4; k++)
                    if (badm[k]) {
                        atomicMin(bad, (unsigned long long)(b0 + 16 * k + __ffs(badm[k]) - 1));
                        break;
                    }
            }
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
    const int64_t want = ((n_words + 3) / 4 + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)dp.num_sms * 16);
    pack_kernel<<<blocks, threads, 0, st>>>(text, len, packed, status, (unsigned long long *)bad);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Kernel 1: one thread per offset over 16-byte rows in global memory (the paper's
// kernel structure, Section V-B). Also the fallback for tables without compact nodes
// and for unaligned buffers.
// ---------------------------------------------------------------------------

// ALL: list every pattern that ends on the walk (each terminal state passed), not only
// the longest, in the match list.
template <bool PACKED, bool COMPACT, bool ALL = false>
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
                if (e < 0) {
                    if (ALL) {
                        const unsigned long long kk = atomicAdd(count, 1ull);
                        if ((int64_t)kk < cap) {
                            c_off[kk] = i;
                            c_ids[kk] = __ldg(t.out_id + s);
                        }
                    } else {
                        best = s;
                    }
                }
            }
            res = best ? __ldg(t.out_id + best) : 0;
            if (!COMPACT) out[i] = res;
        }
        if (COMPACT && !ALL) {
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
                         cudaStream_t st, const DeviceProps &dp, bool all_matches)
{
    if (count && cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (n == 0) return PFAC_OK;
    const int threads = 256;
    const int64_t want = (n + threads - 1) / threads;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)dp.num_sms * 8);
    const bool compact = c_off != nullptr;
    if (all_matches) {
        if (packed) walk_rows_kernel<true, true, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
        else walk_rows_kernel<false, true, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
    } else if (packed) {
        if (compact) walk_rows_kernel<true, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
        else walk_rows_kernel<true, false><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
    } else {
        if (compact) walk_rows_kernel<false, true><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
        else walk_rows_kernel<false, false><<<blocks, threads, 0, st>>>(t, text, n, out, c_off, c_ids, cap, count);
    }
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}


// ---------------------------------------------------------------------------
// Kernel 2: warp-specialised pipeline.
//
//   * one producer warp stages the text of each tile (32 x 16 or 32 x 32 bases per
//     consumer warp)
//     into an S-stage shared-memory ring with TMA bulk copies; full/empty mbarriers
//     hand stages to the consumer warps and back, with bounded waits;
//   * each consumer lane owns 16 (or 32) consecutive offsets and reads one 64-base
//     window (four packed words) from the stage. A fully unrolled, branch-free block tests
//     the prefix filter for every offset (one shared-memory load): a clear bit means
//     the walk ends before depth b with no pattern on the way, answer 0;
//   * the offsets whose bit is set (a few percent) are spread over the warp by a
//     shuffle scan; each takes its filter bit's rank (shared-memory rank index) to a
//     dense skip entry, the state of depth b, and walks on through skip entries
//     (chains of single-child edges compared up to 16 bases at a time) inside the
//     register window;
//   * a walk that needs more than a couple of dependent table loads, or reaches the end
//     of the window while the text goes on, is appended to a deferred list in global
//     scratch memory and finished by a tail kernel, so rounds are never held up by the
//     few long walks (true hits along long patterns).
// Results: zeros go out as 128-bit stores (evict-first), matches as single stores.
// ---------------------------------------------------------------------------

struct DeferItem {
    long long gp;      // text offset of the walk
    uint32_t s;        // state reached
    uint32_t best;     // deepest terminal state passed (0 = none)
    uint32_t q_set;    // bases consumed (low 16 bits) | table index in a batch (high 16 bits)
    int32_t span;      // bases from gp to the end of the walk's text (or read), capped at 2^31-1
};

struct ScanParams {
    DeviceTable t;
    const void *text;
    int64_t n;                   // bases
    int64_t n_units;             // packed words or ASCII bytes in the text buffer
    int32_t *out;
    int64_t *c_off;
    int32_t *c_ids;
    int64_t cap;
    unsigned long long *count;
    DeferItem *defer;
    int64_t defer_cap;
    unsigned long long *defer_count;
    int64_t n_tiles;
    int32_t tile;                // bases per tile = 512 * consumers
    int32_t consumers;           // consumer warps (the producer is warp `consumers`)
    int32_t stages;
    int32_t stage_units;         // packed words or ASCII bytes per stage
    int32_t rank_smem;           // rank index copied into shared memory
    int32_t walk_loads;          // dependent table loads a walk may take before it is deferred
    uint32_t off_filter, off_rank, off_bar, off_queue, off_stage, stage_bytes;
    int64_t timeout_ns;
};

constexpr int kMaxStages = 8;
constexpr uint32_t kBarBytes = 256;   // full[8], empty[8], abort flag
// Packed text: offsets that pass the filter wait in a per-warp ring of kQueue entries
// until a full warp of them can be walked together. An entry is the offset coded as
// (tile round of the CTA) << kRelBits | (offset within the tile).
constexpr uint32_t kQueue = 64;
constexpr int kRelBits = 15;

// Wait for an mbarrier phase, giving up after limit_ns or when another warp of the
// CTA has raised the abort flag. Returns false if it gave up.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, int64_t limit_ns,
                                              volatile uint32_t *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(global_timer_ns() - t0) > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory loads the compiler keeps in program order with the other asm
// statements (the stage words, read before the stage is released).
__device__ __forceinline__ uint32_t lds_u32(const void *p)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ uint4 lds_v4(const void *p)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_addr(p))
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_global_v4_hint(int32_t *p, int4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// Mask of the first L 2-bit bases (L = 1..16).
__device__ __forceinline__ uint32_t base_mask(uint32_t L)
{
    return L >= 16 ? 0xFFFFFFFFu : ((1u << (2 * L)) - 1u);
}

// Sixteen bases of the text from position pos (packed or ASCII) read from global
// memory, with a mask of the bases that cannot be read (at or past `end`, ASCII bytes
// outside ACGT, or bases marked in the optional invalid-base bitmap of packed text).
template <bool PACKED>
__device__ __forceinline__ uint32_t text16(const void *__restrict__ text, const uint32_t *__restrict__ invalid,
                                           int64_t end, int64_t pos, uint32_t *bad)
{
    const int64_t rem = end - pos;
    uint32_t b = rem >= 16 ? 0u : (rem > 0 ? (0xFFFFu << rem) & 0xFFFFu : 0xFFFFu);
    uint32_t w = 0;
    if (PACKED) {
        const int64_t wi = pos >> 4;
        const int64_t n_words = (end + 15) >> 4;
        const uint32_t lo = wi < n_words ? __ldg((const uint32_t *)text + wi) : 0u;
        const uint32_t hi = wi + 1 < n_words ? __ldg((const uint32_t *)text + wi + 1) : 0u;
        w = __funnelshift_r(lo, hi, (uint32_t)(pos & 15) * 2);
        if (invalid) {
            const int64_t bi = pos >> 5;
            const int64_t n_bw = (end + 31) >> 5;
            const uint32_t blo = bi < n_bw ? __ldg(invalid + bi) : 0xFFFFFFFFu;
            const uint32_t bhi = bi + 1 < n_bw ? __ldg(invalid + bi + 1) : 0xFFFFFFFFu;
            b |= __funnelshift_r(blo, bhi, (uint32_t)(pos & 31)) & 0xFFFFu;
        }
    } else {
        for (int i = 0; i < 16 && pos + i < end; i++) {
            const int c = base_code_or_neg(__ldg((const uint8_t *)text + pos + i));
            if (c < 0) b |= 1u << i;
            else w |= (uint32_t)c << (2 * i);
        }
    }
    *bad = b;
    return w;
}

// Where results go: the dense output array (whose slots already hold 0) or the match
// list, plus the deferred-walk list.
struct Sink {
    int32_t *out;
    int64_t *c_off;
    int32_t *c_ids;
    int64_t cap;
    unsigned long long *count;
    DeferItem *defer;
    int64_t defer_cap;
    unsigned long long *defer_count;
};

// Record a non-zero result.
template <bool COMPACT>
__device__ __forceinline__ void emit_match(const Sink &K, int64_t gp, int32_t v)
{
    if (!v) return;
    if (COMPACT) {
        const unsigned long long k = atomicAdd(K.count, 1ull);
        if ((int64_t)k < K.cap) {
            K.c_off[k] = gp;
            K.c_ids[k] = v;
        }
    } else {
        K.out[gp] = v;
    }
}

// Continue a walk from state s with `q` bases consumed, reading the text from global
// memory up to `end` (deferred walks, and walks the deferred list had no room for).
// Returns the pattern id (0 if none). ALL: every terminal state reached from here goes
// to the match list *K instead (each is met once, at the top of the loop) and 0 is
// returned.
template <bool PACKED, bool ALL = false>
__device__ int32_t walk_global(const DeviceTable &T, const void *__restrict__ text,
                               const uint32_t *__restrict__ invalid, int64_t end, int64_t gp, uint32_t s, int q,
                               uint32_t best, const Sink *K = nullptr)
{
    uint4 e = __ldg(T.skip + s);
    for (;;) {
        if (e.y & kSkipSelfTerm) {
            if (ALL) emit_match<true>(*K, gp, __ldg(T.out_id + s));
            else best = s;
        }
        const uint32_t L = e.y & kSkipLenMask;
        uint32_t bad;
        const uint32_t win = text16<PACKED>(text, invalid, end, gp + q, &bad);
        const uint32_t need = L ? L : 1u;
        if (bad & ((need >= 16) ? 0xFFFFu : ((1u << need) - 1u))) break;   // cannot read the next step
        if (L) {
            if ((win ^ e.x) & base_mask(L)) break;
            q += (int)L;
            s = e.z;
            if (!ALL && (e.y & kSkipTargetTerm)) best = s;
        } else {
            const uint32_t c = win & 3u;
            if (!((e.w >> c) & 1u)) break;
            s = (e.w >> kNodeFirstShift) + __popc(e.w & ((1u << c) - 1u));
            q++;
        }
        e = __ldg(T.skip + s);
    }
    return (!ALL && best) ? __ldg(T.out_id + best) : 0;
}

// Mask of positions j < 32 (bit j) such that bits j .. j+w-1 of `bad` are all clear.
__device__ __forceinline__ uint32_t clear_runs(uint64_t bad, int w)
{
    uint64_t t = bad;
    int have = 1;
    while (have * 2 <= w) {
        t |= t >> have;
        have *= 2;
    }
    if (have < w) t |= t >> (w - have);
    return (uint32_t)(~t);
}

// Sixteen bases of a lane's 64-base window from position p (0 <= p < 64); bases past
// the window read as 0.
__device__ __forceinline__ uint32_t window_at(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, int p)
{
    const int w = p >> 4;
    const uint32_t lo = w == 0 ? x0 : (w == 1 ? x1 : (w == 2 ? x2 : x3));
    const uint32_t hi = w == 0 ? x1 : (w == 1 ? x2 : (w == 2 ? x3 : 0u));
    return __funnelshift_r(lo, hi, (uint32_t)(p & 15) * 2);
}

// Prefix-filter bits of a lane's LW offsets: bit j is the filter bit of the b bases
// from offset j (window bases j .. j+b-1; x0, x1, x2 hold window bases 0 .. 47). A
// clear bit means the walk from offset j ends before depth b with no pattern on the
// way. The shared-memory copy of the filter (sf) holds each word bit-reversed: the bit of
// b-mer w is bit 31 - (w mod 32) of word w / 32. With that copy at shared-memory offset 0
// and b >= 3, the byte address of a filter word is the window shifted and masked, a
// left rotate by the window (whose low five bits are w mod 32, taken as they are) brings
// the bit to the top, and a funnel shift moves it into the result: two shifts per
// offset after the load.
template <bool FSMEM, int LW>
__device__ __forceinline__ uint32_t filter_bits(const DeviceTable &T, const uint32_t *sf, uint32_t x0, uint32_t x1,
                                                uint32_t x2, uint32_t bmask)
{
    uint32_t pend = 0;
    if (FSMEM && bmask >= 31u) {
        const uint32_t amask = (bmask >> 3) & ~3u;
        const uint8_t *fb = reinterpret_cast<const uint8_t *>(sf);
#pragma unroll
        for (int j = LW - 1; j >= 0; j--) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t word = *reinterpret_cast<const uint32_t *>(fb + ((win >> 3) & amask));
            pend = __funnelshift_l(__funnelshift_l(word, word, win), pend, 1);
        }
    } else {
#pragma unroll
        for (int j = 0; j < LW; j++) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t kmer = win & bmask;
            const uint32_t word = FSMEM ? __brev(sf[kmer >> 5]) : __ldg(T.filter + (kmer >> 5));
            pend |= ((word >> (kmer & 31u)) & 1u) << j;
        }
    }
    return pend;
}

// Zeros for a warp-batch's valid offsets. Any lane may store any of the warp's zeros.
// When the whole batch is valid its 32*LW outputs are contiguous from warp_base, and
// each 16-byte store instruction covers 512 contiguous bytes (lane l at warp_base +
// 4l + 128v): full sectors, where a lane writing its own offsets would leave every
// sector half-written by two instructions.
template <int LW>
__device__ __forceinline__ void zero_batch(const Sink &K, int64_t warp_base, int lane, uint32_t valid, bool vec_ok,
                                           uint64_t pol)
{
    const uint32_t all = LW == 32 ? 0xFFFFFFFFu : ((1u << LW) - 1u);
    const int64_t gp0 = warp_base + (int64_t)lane * LW;
    const int4 z = make_int4(0, 0, 0, 0);
    if (__all_sync(0xFFFFFFFFu, vec_ok && valid == all)) {
        int32_t *o = K.out + warp_base + 4 * lane;
#pragma unroll
        for (int v = 0; v < LW / 4; v++) st_global_v4_hint(o + 128 * v, z, pol);
    } else if (vec_ok && valid == all) {
        int32_t *o = K.out + gp0;
#pragma unroll
        for (int v = 0; v < LW / 4; v++) st_global_v4_hint(o + 4 * v, z, pol);
    } else if (valid) {
        for (int j = 0; j < LW; j++)
            if ((valid >> j) & 1u) K.out[gp0 + j] = 0;
    }
}

// The walk from one offset gp that passed the filter (or could not be tested). The
// text from gp is window bases j, j+1, ... of x0..x3 (64 bases), of which wlim can be
// read; `ends` when the text (or the run of readable bases) really stops there rather
// than the window. `fast`: the b bases from gp are readable, so the walk starts at the
// dense entry of their b-mer (unless that entry is marked special) at depth b; else at
// the root. It goes on through skip entries inside the window with at most walk_loads
// dependent table loads; a longer walk is deferred to the tail kernel.
template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, bool ALL = false>
__device__ __forceinline__ void walk_item(const DeviceTable &T, const Sink &K, const uint32_t *sf, const void *srank,
                                          int walk_loads, uint32_t set_index, const void *text,
                                          const uint32_t *invalid, int64_t end, int64_t gp, uint32_t x0, uint32_t x1,
                                          uint32_t x2, uint32_t x3, int j, int wlim, bool ends, bool fast)
{
    using RankT = typename std::conditional<RANK16, uint16_t, uint32_t>::type;
    const int B = T.filter_b;
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    uint32_t s = 0, best = 0;
    int q = 0;
    uint4 e;
    bool from_root = true;
    if (fast) {
        const uint32_t kmer = window_at(x0, x1, x2, x3, j) & bmask;
        const uint32_t widx = kmer >> 5;
        const uint32_t word = FSMEM ? __brev(sf[widx]) : __ldg(T.filter + widx);
        uint32_t base_rank;
        if (srank) base_rank = (uint32_t)reinterpret_cast<const RankT *>(srank)[widx];
        else if (T.rank_wide) base_rank = __ldg(reinterpret_cast<const uint32_t *>(T.rank) + widx);
        else base_rank = (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(T.rank) + widx);
        const uint32_t rk = base_rank + __popc(word & ((1u << (kmer & 31u)) - 1u));
        e = __ldg(T.dense + rk);
        if (!(e.y & kSkipSpecial)) {
            from_root = false;
            q = B;
        }
    }
    if (from_root) e = __ldg(T.skip);
    bool defer = false;
    for (int loads = 1;; loads++) {
        // every state the walk enters is met here once (ALL lists each terminal one)
        if (e.y & kSkipSelfTerm) {
            if (ALL) emit_match<true>(K, gp, __ldg(T.out_id + s));
            else best = s;
        }
        const uint32_t L = e.y & kSkipLenMask;
        const int need = L ? (int)L : 1;
        if (q + need > wlim) {
            defer = !ends;     // the window ran out before the text did
            break;
        }
        const uint32_t win = window_at(x0, x1, x2, x3, j + q);
        if (L) {
            if ((win ^ e.x) & base_mask(L)) break;
            q += (int)L;
            s = e.z;
            if (!ALL && (e.y & kSkipTargetTerm)) best = s;
        } else {
            const uint32_t c = win & 3u;
            if (!((e.w >> c) & 1u)) break;
            s = (e.w >> kNodeFirstShift) + __popc(e.w & ((1u << c) - 1u));
            q++;
        }
        if (loads >= walk_loads) {
            defer = true;      // the tail kernel takes it from state s
            break;
        }
        e = __ldg(T.skip + s);
    }
    if (defer) {
        // long walk: finish it in the tail kernel (or here if the list is full)
        const unsigned long long di = atomicAdd(K.defer_count, 1ull);
        if ((int64_t)di < K.defer_cap) {
            DeferItem it;
            it.gp = gp;
            it.s = s;
            it.best = ALL ? 0u : best;
            it.q_set = (uint32_t)q | (set_index << 16);
            it.span = (int32_t)min(end - gp, (int64_t)0x7FFFFFFF);
            K.defer[di] = it;
        } else {
            emit_match<COMPACT>(K, gp, walk_global<PACKED, ALL>(T, text, invalid, end, gp, s, q, best, &K));
        }
    } else if (!ALL && best) {
        emit_match<COMPACT>(K, gp, __ldg(T.out_id + best));
    }
}

// One warp-batch: lane `lane` owns the LW offsets gp0 = warp_base + lane*LW .. +LW-1
// and holds the 64 bases from gp0 in x0..x3 with `bad` marking the bases that cannot
// be read (past the end of its text or read, or not A/C/G/T); `valid` marks the
// offsets this call must answer. Every offset's prefix-filter bit is tested; the
// offsets that pass are spread over the warp (item r of the warp, in lane order then
// offset order, goes to lane r mod 32 in round r / 32, with the owner's window by
// shuffle) and walked at once. Used for ASCII text and for batched reads.
// sf / srank: filter and rank index in shared memory, or nullptr for global memory.
template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, int LW, bool ALL = false>
__device__ __forceinline__ void scan_lane_batch(const DeviceTable &T, const Sink &K, const uint32_t *sf,
                                                const void *srank, int walk_loads, uint32_t set_index,
                                                const void *text, const uint32_t *invalid, int64_t end,
                                                int64_t warp_base, int lane, uint32_t x0, uint32_t x1, uint32_t x2,
                                                uint32_t x3, uint64_t bad, uint32_t valid, bool vec_ok, uint64_t pol)
{
    const int B = T.filter_b;
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    const uint32_t fast = clear_runs(bad, B) & valid;   // the b-mer is readable
    uint32_t pend = filter_bits<FSMEM, LW>(T, sf, x0, x1, x2, bmask) & fast;
    // Offsets whose b bases cannot all be read (a byte outside ACGT, or the end of the
    // text or read, within b bases) walk from the root, unless fewer bases than the
    // shortest pattern can be read: then no pattern starts there.
    if (T.min_len < B) pend |= valid & ~fast & clear_runs(bad, T.min_len);

    if (!COMPACT) zero_batch<LW>(K, warp_base, lane, valid, vec_ok, pol);
    // The zeros above were stored by one lane and a match found below is stored by
    // whichever lane walks it, often another. The warp barrier orders the first before
    // the second.
    __syncwarp();

    const uint32_t cnt = __popc(pend);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += o;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
        const uint32_t r = r0 + lane;
        // owner = the last lane whose first item is <= r
        int owner = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, owner + step);
            if (e <= r) owner += step;
        }
        const uint32_t om = __shfl_sync(0xFFFFFFFFu, pend, owner);
        const uint32_t oe = __shfl_sync(0xFFFFFFFFu, excl, owner);
        const uint32_t ofast = __shfl_sync(0xFFFFFFFFu, fast, owner);
        const uint32_t ox0 = __shfl_sync(0xFFFFFFFFu, x0, owner);
        const uint32_t ox1 = __shfl_sync(0xFFFFFFFFu, x1, owner);
        const uint32_t ox2 = __shfl_sync(0xFFFFFFFFu, x2, owner);
        const uint32_t ox3 = __shfl_sync(0xFFFFFFFFu, x3, owner);
        const uint32_t obad_lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)bad, owner);
        const uint32_t obad_hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(bad >> 32), owner);
        if (r >= total) continue;
        // the (r - oe)-th set bit of the owner's mask (r - oe < popcount by construction)
        uint32_t m = om;
        for (uint32_t i = r - oe; i > 0; i--) m &= m - 1u;
        const int j = (__ffs(m) - 1) & (LW - 1);
        const int64_t gp = warp_base + (int64_t)owner * LW + j;
        const uint64_t badj = (((uint64_t)obad_hi << 32) | obad_lo) >> j;
        // bases readable from the window; `ends` when the text (or the run of ACGT
        // bytes) really stops there rather than the window
        const int wlim = badj ? __ffsll((long long)badj) - 1 : 64 - j;
        walk_item<PACKED, COMPACT, FSMEM, RANK16, ALL>(T, K, sf, srank, walk_loads, set_index, text, invalid, end, gp,
                                                  ox0, ox1, ox2, ox3, j, wlim, badj != 0, (ofast >> j) & 1u);
    }
}

// Walk `count` (<= 32) queued offsets of packed text, one per lane. Each lane reads the
// 64 bases from its offset straight from the packed text (an L2 hit: the tile was
// staged moments ago), so nothing moves between lanes.
template <bool COMPACT, bool FSMEM, bool RANK16, bool ALL = false>
__device__ __forceinline__ void queue_round(const ScanParams &P, const Sink &K, const uint32_t *sf,
                                            const void *srank, const volatile uint32_t *queue, uint32_t head, uint32_t count,
                                            int lane)
{
    if ((uint32_t)lane >= count) return;
    const uint32_t code = queue[(head + (uint32_t)lane) & (kQueue - 1)];
    const int64_t t = (int64_t)blockIdx.x + (int64_t)(code >> kRelBits) * gridDim.x;
    const int64_t gp = t * P.tile + (code & ((1u << kRelBits) - 1u));
    const int64_t rem = P.n - gp;
    const uint32_t *words = reinterpret_cast<const uint32_t *>(P.text);
    const int64_t wi = gp >> 4;
    const uint32_t sh = (uint32_t)(gp & 15) * 2;
    uint32_t w[5];
#pragma unroll
    for (int k = 0; k < 5; k++) w[k] = wi + k < P.n_units ? __ldg(words + wi + k) : 0u;
    const uint32_t x0 = __funnelshift_r(w[0], w[1], sh), x1 = __funnelshift_r(w[1], w[2], sh);
    const uint32_t x2 = __funnelshift_r(w[2], w[3], sh), x3 = __funnelshift_r(w[3], w[4], sh);
    const int wlim = rem < 64 ? (int)rem : 64;
    walk_item<true, COMPACT, FSMEM, RANK16, ALL>(P.t, K, sf, srank, P.walk_loads, 0u, P.text, nullptr, P.n, gp, x0, x1,
                                            x2, x3, 0, wlim, rem <= 64, wlim >= P.t.filter_b);
}

template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, int LW, bool ALL = false>
__global__ void __launch_bounds__(1024, 1) scan_kernel(const ScanParams P)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + P.off_bar);
    uint64_t *empty = reinterpret_cast<uint64_t *>(smem + P.off_bar + 64);
    volatile uint32_t *abort_flag = reinterpret_cast<volatile uint32_t *>(smem + P.off_bar + 128);
    // the filter sits at offset 0 when it is in shared memory
    const uint32_t *sf = reinterpret_cast<const uint32_t *>(smem);
    uint8_t *stage0 = smem + P.off_stage;
    using RankT = typename std::conditional<RANK16, uint16_t, uint32_t>::type;
    const RankT *srank = reinterpret_cast<const RankT *>(smem + P.off_rank);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const DeviceTable &T = P.t;
    const int B = T.filter_b;
    const int S = P.stages;
    const int64_t n = P.n;

    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(smem_addr(&full[i]), 1);
            mbar_init(smem_addr(&empty[i]), (uint32_t)P.consumers);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    {
        // filter and rank index, resident for the whole persistent kernel
        auto copy_in = [&](uint32_t off, const void *src_v, int64_t bytes) {
            uint8_t *dst = smem + off;
            const uint8_t *src = (const uint8_t *)src_v;
            for (int64_t i = 16 * (int64_t)tid; i + 16 <= bytes; i += 16 * (int64_t)blockDim.x)
                *reinterpret_cast<uint4 *>(dst + i) = __ldg(reinterpret_cast<const uint4 *>(src + i));
            for (int64_t i = (bytes & ~(int64_t)15) + tid; i < bytes; i += blockDim.x) dst[i] = src[i];
        };
        const int64_t words = B >= 3 ? ((int64_t)1 << (2 * B)) / 32 : 1;
        if (FSMEM) {
            // the filter's words go in bit-reversed (see filter_bits)
            uint32_t *dst = reinterpret_cast<uint32_t *>(smem + P.off_filter);
            for (int64_t i = 4 * (int64_t)tid; i + 4 <= words; i += 4 * (int64_t)blockDim.x) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(T.filter + i));
                *reinterpret_cast<uint4 *>(dst + i) = make_uint4(__brev(v.x), __brev(v.y), __brev(v.z), __brev(v.w));
            }
            for (int64_t i = (words & ~(int64_t)3) + tid; i < words; i += blockDim.x) dst[i] = __brev(__ldg(T.filter + i));
        }
        if (P.rank_smem) copy_in(P.off_rank, T.rank, words * (int64_t)sizeof(RankT));
    }
    __syncthreads();

    const int unit = PACKED ? 4 : 1;
    const int64_t tile_units = PACKED ? (P.tile >> 4) : P.tile;

    if (warp == P.consumers) {
        // ---------------- producer warp ----------------
        if (lane == 0) {
            int k = 0;
            for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, k++) {
                const int st = k % S;
                if (k >= S && !wait_or_abort(smem_addr(&empty[st]), (uint32_t)(((k / S) - 1) & 1), P.timeout_ns,
                                             abort_flag))
                    break;
                const int64_t u0 = t * tile_units;
                const int64_t cnt = min((int64_t)P.stage_units, P.n_units - u0);
                const uint32_t bytes = (uint32_t)((cnt * unit) & ~(int64_t)15);
                uint8_t *dst = stage0 + (size_t)st * P.stage_bytes;
                // the ragged (< 16-byte) tail by plain loads, published by the arrive below
                for (int64_t b = bytes; b < cnt * unit; b++) dst[b] = __ldg((const uint8_t *)P.text + u0 * unit + b);
                mbar_arrive_expect_tx(smem_addr(&full[st]), bytes);
                if (bytes) bulk_load(smem_addr(dst), (const uint8_t *)P.text + u0 * unit, bytes, smem_addr(&full[st]));
            }
            // Let every copy this CTA issued land before the CTA can exit (bounded).
            for (int i = 0; i < S && i < k; i++) {
                const int kk = k - 1 - i;
                mbar_wait_bounded(smem_addr(&full[kk % S]), (uint32_t)((kk / S) & 1), P.timeout_ns);
            }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const uint64_t pol = policy_evict_first();
    Sink K;
    K.out = P.out;
    K.c_off = P.c_off;
    K.c_ids = P.c_ids;
    K.cap = P.cap;
    K.count = P.count;
    K.defer = P.defer;
    K.defer_cap = P.defer_cap;
    K.defer_count = P.defer_count;
    const void *rank_ptr = P.rank_smem ? (const void *)srank : nullptr;
    const uint32_t all = LW == 32 ? 0xFFFFFFFFu : ((1u << LW) - 1u);
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    volatile uint32_t *queue = reinterpret_cast<volatile uint32_t *>(smem + P.off_queue) + warp * kQueue;
    uint32_t qhead = 0, qcount = 0;   // warp-uniform
    int k = 0;
    for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, k++) {
        const int st = k % S;
        if (!wait_or_abort(smem_addr(&full[st]), (uint32_t)((k / S) & 1), P.timeout_ns, abort_flag)) {
            if (lane == 0) record_error(T.status, PFAC_ERR_TIMEOUT);
            return;
        }
        const uint8_t *stage = stage0 + (size_t)st * P.stage_bytes;
        const int p_rel = warp * (32 * LW) + lane * LW;
        const int64_t warp_base = t * (int64_t)P.tile + warp * (32 * LW);
        const int64_t gp0 = t * (int64_t)P.tile + p_rel;
        const int64_t rem = n - gp0;
        uint64_t bad = rem < 64 ? (rem > 0 ? (~0ull << rem) : ~0ull) : 0ull;
        const uint32_t valid = rem >= LW ? all : (rem > 0 ? ((1u << rem) - 1u) : 0u);
        if constexpr (PACKED) {
            // The filter reads window bases 0 .. LW+b-2 (three words at most); the walks
            // of the offsets that pass read their text again when their round comes.
            uint32_t x0 = 0, x1 = 0, x2 = 0;
            if (rem > 0) {
                const uint32_t *w = reinterpret_cast<const uint32_t *>(stage) + (p_rel >> 4);
                x0 = lds_u32(w);
                x1 = lds_u32(w + 1);
                if (LW == 32) x2 = lds_u32(w + 2);
            }
            const uint32_t fast = bad ? clear_runs(bad, B) & valid : valid;   // the b-mer is readable
            uint32_t pend = filter_bits<FSMEM, LW>(T, sf, x0, x1, x2, bmask) & fast;
            // near the text end: offsets with fewer than b readable bases walk from the
            // root when a pattern shorter than b could still fit
            if (T.min_len < B) pend |= valid & ~fast & clear_runs(bad, T.min_len);
            // Release the stage only once every lane has used its words: the producer
            // refills it as soon as all consumer warps have arrived, and a word read
            // after that would come from the next fill.
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
            if (!COMPACT) zero_batch<LW>(K, warp_base, lane, valid, true, pol);
            // Zeros stored above by one lane are ordered before matches stored by another
            // lane in a later round by the warp barriers between them (this one first).
            __syncwarp();

            // Queue the offsets that pass: lane l's items take the places after those of
            // lanes 0 .. l-1 (exclusive prefix of the counts, by ballots).
            const uint32_t c = __popc(pend);
            const uint32_t lt = (1u << lane) - 1u;
            uint32_t idx = 0, total = 0;
            for (uint32_t b = 0; b < (uint32_t)LW; b++) {
                const uint32_t vb = __ballot_sync(0xFFFFFFFFu, c > b);
                if (!vb) break;
                idx += __popc(vb & lt);
                total += __popc(vb);
            }
            const uint32_t code0 = ((uint32_t)k << kRelBits) | (uint32_t)p_rel;
            uint32_t mine = pend;
            while (total) {   // warp-uniform
                const uint32_t take = min(kQueue - qcount, total);
                while (mine && idx < take) {
                    const int j = __ffs(mine) - 1;
                    mine &= mine - 1u;
                    queue[(qhead + qcount + idx) & (kQueue - 1)] = code0 + (uint32_t)j;
                    idx++;
                }
                idx -= min(idx, take);
                qcount += take;
                total -= take;
                __syncwarp();
                while (qcount >= 32) {
                    queue_round<COMPACT, FSMEM, RANK16, ALL>(P, K, sf, rank_ptr, queue, qhead, 32, lane);
                    qhead = (qhead + 32) & (kQueue - 1);
                    qcount -= 32;
                    __syncwarp();   // the entries just read may be written again
                }
            }
        } else {
            // ASCII: the lane packs its 64-base window from the stage and walks what
            // passes at once, through scan_lane_batch.
            uint32_t x0 = 0, x1 = 0, x2 = 0, x3 = 0;
            if (rem > 0) {
                const uint8_t *r = stage + p_rel;
                uint32_t b0, b1, b2, b3;
                x0 = pack16(lds_v4(r), &b0);
                x1 = pack16(lds_v4(r + 16), &b1);
                x2 = pack16(lds_v4(r + 32), &b2);
                x3 = pack16(lds_v4(r + 48), &b3);
                bad |= (uint64_t)b0 | ((uint64_t)b1 << 16) | ((uint64_t)b2 << 32) | ((uint64_t)b3 << 48);
            }
            // release the stage once every lane has used its bytes (see the packed path)
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
            scan_lane_batch<PACKED, COMPACT, FSMEM, RANK16, LW, ALL>(T, K, sf, rank_ptr, P.walk_loads, 0u, P.text,
                                                                nullptr, n, warp_base, lane, x0, x1, x2, x3, bad,
                                                                valid, true, pol);
        }
    }
    if (PACKED && qcount) queue_round<COMPACT, FSMEM, RANK16, ALL>(P, K, sf, rank_ptr, queue, qhead, qcount, lane);
}

// Deferred walks: one thread per item.
template <bool PACKED, bool COMPACT, bool ALL = false>
__global__ void __launch_bounds__(256) tail_kernel(const ScanParams P)
{
    const unsigned long long cnt = *P.defer_count;
    const int64_t m = min((int64_t)cnt, P.defer_cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const DeferItem it = P.defer[i];
        Sink K;
        K.out = P.out;
        K.c_off = P.c_off;
        K.c_ids = P.c_ids;
        K.cap = P.cap;
        K.count = P.count;
        emit_match<COMPACT>(K, it.gp, walk_global<PACKED, ALL>(P.t, P.text, nullptr, it.gp + it.span, it.gp, it.s,
                                                               (int)(it.q_set & 0xFFFFu), it.best, &K));
    }
}

struct ScanLayout {
    uint32_t off_filter, off_rank, off_bar, off_queue, off_stage, stage_bytes, total;
    int32_t stage_units;
};

static inline uint32_t align128(uint64_t x) { return (uint32_t)((x + 127) & ~(uint64_t)127); }

static ScanLayout scan_layout(int consumers, int lw, int stages, int64_t filter_smem_bytes, int64_t rank_smem_bytes,
                              bool packed)
{
    ScanLayout L{};
    const int64_t tile = 32LL * lw * consumers;
    // The filter comes first, at offset 0, so that its lookups need no base address.
    uint64_t off = 0;
    L.off_filter = (uint32_t)off;
    off += align128((uint64_t)filter_smem_bytes);
    L.off_rank = (uint32_t)off;
    off += align128((uint64_t)rank_smem_bytes);
    L.off_bar = (uint32_t)off;
    off += kBarBytes;
    L.off_queue = (uint32_t)off;
    if (packed) off += align128((uint64_t)consumers * kQueue * 4);
    // a lane reads 64 bases from its first offset: 2 words (32 bytes) past the tile
    L.stage_units = packed ? (int32_t)(tile / 16 + 4) : (int32_t)(tile + 64);
    L.stage_bytes = align128((uint64_t)L.stage_units * (packed ? 4 : 1));
    L.off_stage = (uint32_t)off;
    off += (uint64_t)L.stage_bytes * stages;
    L.total = (uint32_t)off;
    return L;
}

static int consumers_of(const TiledConfig &cfg) { return cfg.threads / 32 - 1; }
static int lane_width_of(const TiledConfig &cfg) { return cfg.lane_offsets == 32 ? 32 : 16; }
static int stages_of(const TiledConfig &cfg, bool packed) { return cfg.stages > 0 ? cfg.stages : (packed ? 3 : 2); }

// Shared memory per CTA, by priority: the text stages, the prefix filter (read for
// every offset), then the rank index (read for every walk the filter passes).
struct SmemPlan {
    int64_t filter_bytes, rank_bytes;   // bytes copied into shared memory (0 = global)
    int64_t total;
};

static SmemPlan plan_smem(const DeviceTable &t, const TiledConfig &cfg, bool packed, const DeviceProps &dp)
{
    SmemPlan pl{};
    const int C = consumers_of(cfg);
    const int LW = lane_width_of(cfg);
    const int S = stages_of(cfg, packed);
    const int64_t per_cta = (int64_t)dp.smem_per_sm / std::max(1, cfg.ctas_per_sm) - 1024;
    const int64_t limit = std::min<int64_t>(dp.smem_optin, per_cta);
    const int64_t words = t.filter_b >= 3 ? ((int64_t)1 << (2 * t.filter_b)) / 32 : 1;
    const int64_t fbytes = words * 4;
    const int64_t rbytes = words * (t.rank_wide ? 4 : 2);
    auto total = [&](int64_t f, int64_t r) { return (int64_t)scan_layout(C, LW, S, f, r, packed).total; };
    if (total(0, 0) > limit) {
        pl.total = -1;
        return pl;
    }
    pl.filter_bytes = total(fbytes, 0) <= limit ? fbytes : 0;
    pl.rank_bytes = (cfg.smem_table_bytes >= 0 && total(pl.filter_bytes, rbytes) <= limit) ? rbytes : 0;
    pl.total = total(pl.filter_bytes, pl.rank_bytes);
    return pl;
}

int64_t tiled_smem_bytes(const DeviceTable &t, const TiledConfig &cfg, bool packed, const DeviceProps &dp)
{
    return plan_smem(t, cfg, packed, dp).total;
}

// Access-policy window that keeps the skip entries in L2 (persisting) while the
// output streams through it. The set-aside for persisting lines is a limit of the whole
// context: it is set by the first launch that asks for the window and given back
// (limit 0, persisting lines reset to normal) by the next launch that does not, so the
// other launches of the process keep the whole L2.
static std::mutex g_persist_mu;
static bool g_persist_set[64];

static cudaError_t release_persisting_l2(int dev)
{
    std::lock_guard<std::mutex> lk(g_persist_mu);
    if (dev < 0 || dev >= 64 || !g_persist_set[dev]) return cudaSuccess;
    cudaError_t e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    if (e == cudaSuccess) e = cudaCtxResetPersistingL2Cache();
    if (e == cudaSuccess) g_persist_set[dev] = false;
    return e;
}

template <typename Kern>
static cudaError_t launch_with_policy(Kern kern, const ScanParams &P, int grid, int threads, uint32_t smem,
                                      cudaStream_t st, const TiledConfig &cfg, const DeviceProps &dp)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    lc.attrs = attr;
    lc.numAttrs = 0;
    const int64_t skip_bytes = P.t.n_states * 16;
    if (cfg.l2_persist > 0 && dp.persist_l2_max > 0 && skip_bytes > 0) {
        const int dev = dp.device;
        {
            std::lock_guard<std::mutex> lk(g_persist_mu);
            if (dev >= 0 && dev < 64 && !g_persist_set[dev]) {
                if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)dp.persist_l2_max) != cudaSuccess)
                    return cudaGetLastError();
                g_persist_set[dev] = true;
            }
        }
        int max_win = 0;
        cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        const int64_t win = std::min<int64_t>(skip_bytes, max_win);
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = (void *)P.t.skip;
        attr[0].val.accessPolicyWindow.num_bytes = (size_t)win;
        attr[0].val.accessPolicyWindow.hitRatio =
            (float)std::min<double>(1.0, (double)dp.persist_l2_max / (double)std::max<int64_t>(win, 1));
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        lc.numAttrs = 1;
    } else {
        const cudaError_t e = release_persisting_l2(dp.device);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernelEx(&lc, kern, P);
}

template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, bool ALL>
static int launch_scan_t(const ScanParams &P, int grid, int threads, uint32_t smem, int tail_grid, cudaStream_t st,
                         const TiledConfig &cfg, const DeviceProps &dp)
{
    auto kern = lane_width_of(cfg) == 32 ? scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL>
                                         : scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 16, ALL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PFAC_ERR_CUDA;
    if (launch_with_policy(kern, P, grid, threads, smem, st, cfg, dp) != cudaSuccess) return PFAC_ERR_CUDA;
    tail_kernel<PACKED, COMPACT, ALL><<<tail_grid, 256, 0, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

template <bool PACKED, bool COMPACT, bool ALL = false>
static int launch_scan_w(const ScanParams &P, bool fsmem, bool rank16, int grid, int threads, uint32_t smem,
                         int tail_grid, cudaStream_t st, const TiledConfig &cfg, const DeviceProps &dp)
{
    if (fsmem)
        return rank16 ? launch_scan_t<PACKED, COMPACT, true, true, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp)
                      : launch_scan_t<PACKED, COMPACT, true, false, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp);
    return rank16 ? launch_scan_t<PACKED, COMPACT, false, true, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp)
                  : launch_scan_t<PACKED, COMPACT, false, false, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp);
}

int launch_tiled(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out, int64_t *c_off,
                 int32_t *c_ids, int64_t cap, unsigned long long *count, const TiledConfig &cfg,
                 const DeferScratch &scratch, cudaStream_t st, const DeviceProps &dp, bool all_matches)
{
    const bool compact = c_off != nullptr;
    if (compact && cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (n == 0) return PFAC_OK;
    const int C = consumers_of(cfg);
    const int LW = lane_width_of(cfg);
    const int S = stages_of(cfg, packed);
    if (!t.skip || !t.filter || !t.rank || !t.dense || t.filter_b < 1 || t.filter_b > kMaxFilterB || C < 1 ||
        (cfg.threads & 31) || cfg.threads > 1024 || S < 2 || S > kMaxStages || !scratch.items || !scratch.count)
        return PFAC_ERR_INVALID_ARG;
    const SmemPlan pl = plan_smem(t, cfg, packed, dp);
    if (pl.total < 0 || pl.total > dp.smem_optin) return PFAC_ERR_UNSUPPORTED;
    const ScanLayout L = scan_layout(C, LW, S, pl.filter_bytes, pl.rank_bytes, packed);
    if (cudaMemsetAsync(scratch.count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    ScanParams P{};
    P.t = t;
    P.text = text;
    P.n = n;
    P.n_units = packed ? (n + 15) / 16 : n;
    P.out = out;
    P.c_off = c_off;
    P.c_ids = c_ids;
    P.cap = cap;
    P.count = count;
    P.defer = (DeferItem *)scratch.items;
    P.defer_cap = scratch.cap;
    P.defer_count = scratch.count;
    P.tile = 32 * LW * C;
    P.n_tiles = (n + P.tile - 1) / P.tile;
    if (P.tile > (1 << kRelBits)) return PFAC_ERR_INVALID_ARG;
    P.consumers = C;
    P.stages = S;
    P.stage_units = L.stage_units;
    P.rank_smem = pl.rank_bytes > 0;
    P.walk_loads = cfg.walk_loads > 0 ? cfg.walk_loads : 2;
    P.off_filter = L.off_filter;
    P.off_rank = L.off_rank;
    P.off_bar = L.off_bar;
    P.off_queue = L.off_queue;
    P.off_stage = L.off_stage;
    P.stage_bytes = L.stage_bytes;
    P.timeout_ns = cfg.timeout_ns > 0 ? cfg.timeout_ns : 2000000000LL;
    const int64_t grid64 = std::min<int64_t>(P.n_tiles, (int64_t)dp.num_sms * std::max(1, cfg.ctas_per_sm));
    const int grid = (int)std::max<int64_t>(1, grid64);
    // a queued offset codes its tile round in 32 - kRelBits bits
    if (packed && (P.n_tiles + grid - 1) / grid > ((int64_t)1 << (32 - kRelBits))) return PFAC_ERR_UNSUPPORTED;
    const int tail_grid = dp.num_sms * 4;
    const bool fsmem = pl.filter_bytes > 0;
    const bool rank16 = !t.rank_wide;
    if (all_matches) {   // the match list of every pattern on every walk (packed text only)
        if (!packed || !compact) return PFAC_ERR_INVALID_ARG;
        return launch_scan_w<true, true, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp);
    }
    if (packed)
        return compact ? launch_scan_w<true, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp)
                       : launch_scan_w<true, false>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp);
    return compact ? launch_scan_w<false, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp)
                   : launch_scan_w<false, false>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp);
}

size_t defer_item_bytes() { return sizeof(DeferItem); }

// ---------------------------------------------------------------------------
// Batched scan: many reads of uneven length, each against its own table, in one
// persistent launch (plus the pack, plan and tail kernels around it).
//   pack_bits_kernel    ASCII reads -> 2-bit words + one invalid bit per base
//   plan_kernel         reads -> first work item of each read (512 or 1024 offsets per
//                       item), and the read of every work item
//   batched_scan_kernel warps take items from a counter; each item runs the same
//                       per-warp filter test and skip walks as kernel 2, with its
//                       read's table and every walk bounded by its read's end
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
    unsigned long long *item_next;
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

// One CTA: exclusive prefix of the number of work items per read.
__global__ void __launch_bounds__(1024) plan_kernel(const int64_t *__restrict__ read_off, int32_t n_reads, int64_t n,
                                                    int32_t item, int64_t *__restrict__ item_start,
                                                    int32_t *__restrict__ item_read, int64_t item_cap)
{
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n_reads; base += blockDim.x) {
        const int64_t r = base + tid;
        int64_t v = 0;
        if (r < n_reads) {
            int64_t rs, re;
            read_bounds(read_off, (int32_t)r, n, &rs, &re);
            v = (re - rs + item - 1) / item;
        }
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
        if (r < n_reads) item_start[r] = carry + before;
        __syncthreads();
        if (tid == 0) carry += warp_sum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (tid == 0) item_start[n_reads] = carry;
    __syncthreads();
    // the read of each work item (items past item_cap are found by search instead)
    for (int64_t r = tid; r < n_reads; r += blockDim.x) {
        const int64_t k1 = min(item_start[r + 1], item_cap);
        for (int64_t k = item_start[r]; k < k1; k++) item_read[k] = (int32_t)r;
    }
}

template <int LW>
__global__ void __launch_bounds__(256) batched_scan_kernel(const BatchParams P)
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
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(P.item_next, 1ull);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if ((int64_t)it >= total) break;
        // the read holding item `it`: the last r with item_start[r] <= it, from the plan's
        // map, or by search past its capacity (reads that overlap one another)
        int32_t lo = 0;
        if ((int64_t)it < P.item_cap) {
            lo = P.item_read[it];
        } else {
            int32_t hi = P.n_reads - 1;
            while (lo < hi) {
                const int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
                if (P.item_start[mid] <= (int64_t)it) lo = mid;
                else hi = mid - 1;
            }
        }
        int64_t rs, re;
        read_bounds(P.read_off, lo, P.n, &rs, &re);
        const int64_t base = rs + ((int64_t)it - P.item_start[lo]) * kItem;
        const int64_t item_end = min(base + kItem, re);
        const int32_t set = P.read_set[lo];
        if (set < 0 || set >= P.n_sets) {
            if (lane == 0) record_error(P.sets[0].status, PFAC_ERR_INVALID_ARG);
            continue;
        }
        const DeviceTable T = P.sets[set];
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
        scan_lane_batch<true, false, false, true, LW>(T, K, nullptr, nullptr, P.walk_loads, (uint32_t)set, P.packed,
                                                      P.invalid, re, base, lane, x0, x1, x2, x3, bad, valid, vec_ok,
                                                      pol);
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
    unsigned long long *counters = (unsigned long long *)p;       // [0] next item, [1] deferred walks
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
    P.item_next = counters;
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
static_assert(sizeof(DeferItem) == kDeferItemBytes, "deferred-walk record size");

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
        cudaDeviceGetAttribute(&p->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->l2_bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->persist_l2_max, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess)
        return PFAC_ERR_CUDA;
    return PFAC_OK;
}

}  // namespace pfac
