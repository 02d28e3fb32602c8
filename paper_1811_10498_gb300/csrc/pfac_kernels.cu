// sm_103a kernels of the PFAC scan and their launchers.
//
// The scan (Section IV): every text offset walks the failure-less goto trie from the
// root, one edge per base, until no edge exists, and reports the longest pattern that
// ended on the way. The paper's kernel (Section V-B) runs one thread per character over
// a 4-column table in global memory; kernel 1 below keeps that structure (one thread per
// offset, 16-byte rows). Kernel 2 is the Blackwell design:
//   * a producer warp stages each tile of text (2-bit packed or ASCII) plus a 64-base
//     halo into a shared-memory ring with TMA bulk copies, tracked by mbarriers whose
//     waits are bounded;
//   * consumer lanes test every offset against the prefix filter in shared memory (one
//     bit per b-mer: a clear bit settles the offset, answer 0);
//   * the few offsets that pass are queued per warp and walked 32 at a time from the
//     dense entry of their b-mer over path-compressed skip entries; the few long walks
//     go to a deferred list finished by the tail kernel;
//   * zeros leave as 512-byte-contiguous 16-byte stores with an evict-first L2 hint,
//     matches as single stores (or as (offset, id) pairs in a match list).
// The device-side pieces shared with the batched kernels are in pfac_device.cuh.
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <type_traits>
#include <utility>

#include "../../include/pfac.h"
#include "pfac_internal.h"
#include "pfac_device.cuh"

namespace pfac {
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
                        const unsigned long long kk = warp_aggregated_slot(count);
                        if ((int64_t)kk < cap) {
                            c_off[kk] = i;
                            c_ids[kk] = __ldg(t.out_id + s);
                        } else {
                            record_error(t.status, PFAC_ERR_OVERFLOW);
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
                    else record_error(t.status, PFAC_ERR_OVERFLOW);
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
// The paper's memory-placement experiments (Section V-C; Section VII, Figs. 6-8) on the
// one-thread-per-offset kernel: the transition table as two arrays (nextState and
// matchedPatternId, a pitch of four) or merged into one array of pairs; table loads
// through the read-only (texture) path, the default L1-cached path, or with L1 bypassed
// (the paper's L1-off configuration); text read from global memory or first staged per
// block in shared memory. Dense ids, the longest pattern per offset as everywhere else.
// ---------------------------------------------------------------------------

template <int LOADS>
__device__ __forceinline__ int32_t ld_table(const int32_t *p)
{
    if (LOADS == 0) return __ldg(p);
    if (LOADS == 1) return __ldca(p);
    return __ldcg(p);
}

template <int LOADS>
__device__ __forceinline__ int2 ld_table(const int2 *p)
{
    if (LOADS == 0) return __ldg(p);
    if (LOADS == 1) return __ldca(p);
    return __ldcg(p);
}

constexpr int kPaperBlock = 256;          // threads per block, as in the paper's kernel

template <bool PACKED, int LAYOUT, int LOADS, bool TSMEM>
__global__ void __launch_bounds__(kPaperBlock) paper_walk_kernel(DeviceTable t, PaperTables pt,
                                                                 const void *__restrict__ text, int64_t n,
                                                                 int32_t *__restrict__ out)
{
    extern __shared__ __align__(16) uint8_t tile[];
    const int64_t stride = (int64_t)gridDim.x * kPaperBlock;
    const int max_len = t.max_len;
    for (int64_t i0 = (int64_t)blockIdx.x * kPaperBlock; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        // the block's text: its offsets plus the longest walk's reach past the last one
        const int64_t tile_end = min(n, i0 + kPaperBlock + max_len - 1);
        if (TSMEM) {
            __syncthreads();                 // the previous tile's readers are done
            if (PACKED) {
                const uint32_t *src = (const uint32_t *)text + (i0 >> 4);
                uint32_t *dst = reinterpret_cast<uint32_t *>(tile);
                const int64_t words = ((tile_end + 15) >> 4) - (i0 >> 4);
                for (int64_t k = threadIdx.x; k < words; k += kPaperBlock) dst[k] = __ldg(src + k);
            } else {
                const uint8_t *src = (const uint8_t *)text + i0;
                for (int64_t k = threadIdx.x; k < tile_end - i0; k += kPaperBlock) tile[k] = __ldg(src + k);
            }
            __syncthreads();
        }
        if (i < n) {
            int32_t s = 0, best = 0;
            const int64_t end = min(n, i + (int64_t)max_len);
            for (int64_t k = i; k < end; k++) {
                int c;
                if (PACKED) {
                    const uint32_t w = TSMEM ? reinterpret_cast<const uint32_t *>(tile)[(k - i0) >> 4]
                                             : __ldg((const uint32_t *)text + (k >> 4));
                    c = (int)((w >> ((k & 15) * 2)) & 3u);
                } else {
                    c = base_code_or_neg(TSMEM ? tile[k - i0] : __ldg((const uint8_t *)text + k));
                    if (c < 0) break;
                }
                const int64_t cell = 4 * (int64_t)s + c;
                if (LAYOUT == 0) {
                    const int32_t e = ld_table<LOADS>(t.rows + cell);
                    if (e == 0) break;
                    s = e & 0x7FFFFFFF;
                    if (e < 0) best = s;
                } else if (LAYOUT == 1) {
                    const int32_t nx = ld_table<LOADS>(pt.next + cell);
                    const int32_t id = ld_table<LOADS>(pt.pid + cell);
                    if (nx == 0) break;
                    if (id) best = id;
                    s = nx;
                } else {
                    const int2 e = ld_table<LOADS>(pt.pair + cell);
                    if (e.x == 0) break;
                    if (e.y) best = e.y;
                    s = e.x;
                }
            }
            if (LAYOUT == 0) best = best ? __ldg(t.out_id + best) : 0;
            out[i] = best;
        }
    }
}

template <bool PACKED, int LAYOUT, int LOADS>
static void launch_paper_t(bool tsmem, int blocks, size_t smem, cudaStream_t st, const DeviceTable &t,
                           const PaperTables &pt, const void *text, int64_t n, int32_t *out)
{
    if (tsmem) paper_walk_kernel<PACKED, LAYOUT, LOADS, true><<<blocks, kPaperBlock, smem, st>>>(t, pt, text, n, out);
    else paper_walk_kernel<PACKED, LAYOUT, LOADS, false><<<blocks, kPaperBlock, 0, st>>>(t, pt, text, n, out);
}

template <bool PACKED, int LAYOUT>
static void launch_paper_l(int loads, bool tsmem, int blocks, size_t smem, cudaStream_t st, const DeviceTable &t,
                           const PaperTables &pt, const void *text, int64_t n, int32_t *out)
{
    if (loads == 1) launch_paper_t<PACKED, LAYOUT, 1>(tsmem, blocks, smem, st, t, pt, text, n, out);
    else if (loads == 2) launch_paper_t<PACKED, LAYOUT, 2>(tsmem, blocks, smem, st, t, pt, text, n, out);
    else launch_paper_t<PACKED, LAYOUT, 0>(tsmem, blocks, smem, st, t, pt, text, n, out);
}

template <bool PACKED>
static void launch_paper_p(const PaperConfig &pc, int blocks, size_t smem, cudaStream_t st, const DeviceTable &t,
                           const PaperTables &pt, const void *text, int64_t n, int32_t *out)
{
    const bool ts = pc.text_smem != 0;
    if (pc.layout == 1) launch_paper_l<PACKED, 1>(pc.loads, ts, blocks, smem, st, t, pt, text, n, out);
    else if (pc.layout == 2) launch_paper_l<PACKED, 2>(pc.loads, ts, blocks, smem, st, t, pt, text, n, out);
    else launch_paper_l<PACKED, 0>(pc.loads, ts, blocks, smem, st, t, pt, text, n, out);
}

int launch_paper_walk(const DeviceTable &t, const PaperTables &pt, const PaperConfig &pc, const void *text,
                      bool packed, int64_t n, int32_t *out, cudaStream_t st, const DeviceProps &dp)
{
    if (n == 0) return PFAC_OK;
    if (pc.layout < 0 || pc.layout > 2 || pc.loads < 0 || pc.loads > 2) return PFAC_ERR_INVALID_ARG;
    if ((pc.layout == 1 && (!pt.next || !pt.pid)) || (pc.layout == 2 && !pt.pair)) return PFAC_ERR_UNSUPPORTED;
    // shared-memory tile: 256 offsets plus max_len - 1 bases (packed: whole words, one
    // more for a tile that starts mid-word)
    const int64_t tile_bases = kPaperBlock + (int64_t)t.max_len - 1;
    const int64_t smem = packed ? 4 * ((tile_bases + 15) / 16 + 1) : tile_bases;
    if (pc.text_smem && smem > 48 * 1024) return PFAC_ERR_UNSUPPORTED;
    const int64_t want = (n + kPaperBlock - 1) / kPaperBlock;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)dp.num_sms * 8);
    if (packed) launch_paper_p<true>(pc, blocks, (size_t)smem, st, t, pt, text, n, out);
    else launch_paper_p<false>(pc, blocks, (size_t)smem, st, t, pt, text, n, out);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

__global__ void derive_paper_kernel(const int32_t *__restrict__ rows, const int32_t *__restrict__ out_id, int64_t cells,
                                    int32_t *next, int32_t *pid, int2 *pair)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < cells; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = rows[k];
        const int32_t nx = e & 0x7FFFFFFF;
        const int32_t id = e < 0 ? out_id[nx] : 0;    // bit 31: the state reached is terminal
        if (next) {
            next[k] = nx;
            pid[k] = id;
        }
        if (pair) pair[k] = make_int2(nx, id);
    }
}

int derive_paper_tables(const DeviceTable &t, int32_t *next, int32_t *pid, int2 *pair, cudaStream_t st)
{
    if ((next == nullptr) != (pid == nullptr)) return PFAC_ERR_INVALID_ARG;
    const int64_t cells = 4 * t.n_states;
    const int blocks = (int)std::min<int64_t>((cells + 255) / 256, 4096);
    derive_paper_kernel<<<std::max(1, blocks), 256, 0, st>>>(t.rows, t.out_id, cells, next, pid, pair);
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
    uint32_t off_zero, zero_chunk;   // zero tile of the bulk-store writer (ZW = 2)
    int64_t timeout_ns;
};

constexpr int kMaxStages = 8;
constexpr uint32_t kBarBytes = 256;   // full[8], empty[8], abort flag, zero-writer progress
constexpr uint32_t kAbortAt = 128, kZeroDoneAt = 192;

__device__ __forceinline__ void st_release_cta(volatile uint32_t *p, uint32_t v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr((const void *)p)), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_cta(const volatile uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr((const void *)p)) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_2() { asm volatile("cp.async.bulk.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_1() { asm volatile("cp.async.bulk.wait_group 1;" ::: "memory"); }

// The zero writer of dense packed scans (a warp of its own, so that the consumer warps
// only test, walk and store matches). For each tile round k of the CTA it writes the
// tile's zeros and then publishes in *zdone how many rounds are complete, with release
// semantics; a consumer stores a match of round k only after reading *zdone > k with
// acquire semantics, so the match lands after the zero it replaces.
//   ZW = 1: all 32 lanes, 16-byte stores (512 contiguous bytes per instruction);
//   ZW = 2: one lane, TMA bulk stores of a zero tile in shared memory, two rounds in
//           flight; a round counts as done once its bulk group has completed and a
//           proxy fence orders those writes before the consumers' ordinary stores.
template <int ZW>
__device__ void zero_writer(const ScanParams &P, uint8_t *smem, volatile uint32_t *zdone, int lane)
{
    const uint64_t pol = policy_evict_first();
    uint32_t k = 0;
    if (ZW == 1) {
        const int4 z = make_int4(0, 0, 0, 0);
        for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, k++) {
            const int64_t lo = t * P.tile, cnt = min((int64_t)P.tile, P.n - lo);
            int32_t *o = P.out + lo;
            const int64_t nv = cnt >> 2;
            for (int64_t v = lane; v < nv; v += 32) st_global_v4_hint(o + 4 * v, z, pol);
            for (int64_t i = 4 * nv + lane; i < cnt; i += 32) o[i] = 0;
            __syncwarp();
            if (lane == 0) st_release_cta(zdone, k + 1);
        }
    } else if (lane == 0) {
        const uint32_t zb = smem_addr(smem + P.off_zero);
        for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, k++) {
            const int64_t lo = t * P.tile, cnt = min((int64_t)P.tile, P.n - lo);
            uint8_t *dst = reinterpret_cast<uint8_t *>(P.out + lo);
            const int64_t full = (cnt * 4) & ~(int64_t)15;
            for (int64_t b = 0; b < full; b += P.zero_chunk)
                bulk_store(dst + b, zb, (uint32_t)min((int64_t)P.zero_chunk, full - b), pol);
            for (int64_t i = full / 4; i < cnt; i++) P.out[lo + i] = 0;    // the last < 4 ids
            bulk_commit();
            bulk_wait_2();                       // the groups of rounds <= k - 2 are complete
            if (k >= 2) {
                fence_proxy_async_global();
                st_release_cta(zdone, k - 1);
            }
        }
        bulk_wait_all();
        fence_proxy_async_global();
        st_release_cta(zdone, k);
    }
}

// A consumer's wait until the zeros of its rounds < need are written (bounded; gives up
// when the CTA aborts).
__device__ __forceinline__ bool wait_zeros(const volatile uint32_t *zdone, uint32_t need, int64_t limit_ns,
                                           volatile uint32_t *abort_flag)
{
    if (ld_acquire_cta(zdone) >= need) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (ld_acquire_cta(zdone) >= need) return true;
        if (*abort_flag) return false;
        if ((int64_t)(global_timer_ns() - t0) > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}
// Packed text: offsets that pass the filter wait in a per-warp ring of kQueue entries
// until a full warp of them can be walked together. An entry is the offset coded as
// (tile round of the CTA) << kRelBits | (offset within the tile).
constexpr uint32_t kQueue = 64;
constexpr int kRelBits = 15;

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

// Main-filter bits (global memory) of the lane's offsets whose bit is set in `screen`
// (the first-level filter's verdict); the loads of the other offsets are skipped.
template <int LW>
__device__ __forceinline__ uint32_t filter_bits_screened(const DeviceTable &T, uint32_t x0, uint32_t x1, uint32_t x2,
                                                         uint32_t bmask, uint32_t screen)
{
    uint32_t pend = 0;
#pragma unroll
    for (int j = 0; j < LW; j++) {
        if ((screen >> j) & 1u) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t kmer = win & bmask;
            const uint32_t word = __ldg(T.filter + (kmer >> 5));
            pend |= ((word >> (kmer & 31u)) & 1u) << j;
        }
    }
    return pend;
}

// One probe of the sampled screen: the bit of the q-gram that starts the window `win`.
// SCR 2: 13-grams in global memory; SCR 3: 10-grams in shared memory at offset 0, each
// word bit-reversed as the prefix filter's copy is (see filter_bits).
template <int SCR>
__device__ __forceinline__ uint32_t probe_bit(const DeviceTable &T, const uint8_t *fb, uint32_t win)
{
    if constexpr (SCR == 2) {
        const uint32_t g = win & ((1u << (2 * kSampleQ)) - 1u);
        return (__ldg(T.sample + (g >> 5)) >> (g & 31u)) & 1u;
    } else {
        constexpr uint32_t amask = ((((1u << (2 * kSampleQSmem)) - 1u) >> 3) & ~3u);
        const uint32_t word = *reinterpret_cast<const uint32_t *>(fb + ((win >> 3) & amask));
        return __funnelshift_l(word, word, win) >> 31;
    }
}

// The sampled screen of a lane's 32 offsets (packed text, window bases 0 .. 47 in x0, x1,
// x2): probe m reads the q-gram at window offset 4m (m = 0 .. 8; the ninth is the next
// lane's first, taken by shuffle, and probed directly by the warp's last lane). Offset r
// can start a match only if the probe at 4 * ceil(r / 4) is set (every pattern's q-gram
// at position (-i) mod 4 is in the set), so the result marks offset 0 with probe 0,
// offsets 4m-3 .. 4m with probe m, and 29 .. 31 with probe 8. Probes past the text end
// read bases that are not the text's: they can only add offsets, which the exact prefix
// filter then rejects.
template <int SCR>
__device__ __forceinline__ uint32_t sampled_candidates(const DeviceTable &T, const uint8_t *fb, uint32_t x0,
                                                       uint32_t x1, uint32_t x2, int lane)
{
    static_assert(kSampleS == 4, "probes every 4th offset of a lane's 32");
    uint32_t cand = 0, p0 = 0;
#pragma unroll
    for (int m = 0; m < 8; m++) {
        const int j = 4 * m;
        const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
        const uint32_t bit = probe_bit<SCR>(T, fb, win);
        if (m == 0) p0 = bit;
        cand |= (0u - bit) & (m == 0 ? 1u : (0xFu << (4 * m - 3)));
    }
    uint32_t p8 = __shfl_down_sync(0xFFFFFFFFu, p0, 1);
    if (lane == 31) p8 = probe_bit<SCR>(T, fb, x2);
    return cand | ((0u - p8) & 0xE0000000u);
}

// Main-filter bits (global memory) of the offsets in `m`, one at a time (a lane's few
// candidates: the warp runs as many rounds as its busiest lane has candidates).
__device__ __forceinline__ uint32_t filter_bits_of(const DeviceTable &T, uint32_t x0, uint32_t x1, uint32_t x2,
                                                   uint32_t bmask, uint32_t m)
{
    uint32_t pend = 0;
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
        const uint32_t kmer = win & bmask;
        pend |= ((__ldg(T.filter + (kmer >> 5)) >> (kmer & 31u)) & 1u) << j;
    }
    return pend;
}

// SCR (packed text): 1 = the main filter is in global memory and the first-level filter
// of order kFilter1B sits in shared memory at offset 0 and screens every offset first;
// 2 = the main filter is in global memory and the sampled 13-gram screen (global memory)
// picks the offsets whose main-filter bit is read; 3 = the sampled 10-gram screen sits in
// shared memory at offset 0 in place of the order-10 filter, which is read from global
// memory for the offsets the screen lets through.
// ZW (dense packed scans): 0 = each consumer warp stores its own zeros; 1 or 2 = a zero
// writer warp (warp consumers + 1) stores them (see zero_writer); 3 = each consumer warp
// stores its own zeros with TMA bulk copies of a zero tile, and stores the matches of a
// tile only once that tile's bulk group has completed.
template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, int LW, bool ALL = false, int SCR = 0, int ZW = 0>
__global__ void __launch_bounds__(1024, 1) scan_kernel(const ScanParams P)
{
    static_assert(ZW == 0 || (PACKED && !COMPACT && !ALL), "a zero writer serves dense packed scans");
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + P.off_bar);
    uint64_t *empty = reinterpret_cast<uint64_t *>(smem + P.off_bar + 64);
    volatile uint32_t *abort_flag = reinterpret_cast<volatile uint32_t *>(smem + P.off_bar + kAbortAt);
    volatile uint32_t *zdone = reinterpret_cast<volatile uint32_t *>(smem + P.off_bar + kZeroDoneAt);
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
        *zdone = 0;
        fence_mbar_init();
    }
    if ((ZW == 2 || ZW == 3) && tid < 32) {
        // the zero tile the writer's bulk stores read; made visible to the async proxy
        for (uint32_t i = 16 * (uint32_t)tid; i < P.zero_chunk; i += 16 * 32)
            *reinterpret_cast<int4 *>(smem + P.off_zero + i) = make_int4(0, 0, 0, 0);
        fence_proxy_async();
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
        if (FSMEM || SCR == 1 || SCR == 3) {
            // the filter's words go in bit-reversed (see filter_bits): the main filter, or
            // the first-level one
            const uint32_t *src = SCR == 1 ? T.filter1 : (SCR == 3 ? T.sample : T.filter);
            const int64_t fwords = SCR == 1 ? ((int64_t)1 << (2 * kFilter1B)) / 32
                                            : (SCR == 3 ? ((int64_t)1 << (2 * kSampleQSmem)) / 32 : words);
            uint32_t *dst = reinterpret_cast<uint32_t *>(smem + P.off_filter);
            for (int64_t i = 4 * (int64_t)tid; i + 4 <= fwords; i += 4 * (int64_t)blockDim.x) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + i));
                *reinterpret_cast<uint4 *>(dst + i) = make_uint4(__brev(v.x), __brev(v.y), __brev(v.z), __brev(v.w));
            }
            for (int64_t i = (fwords & ~(int64_t)3) + tid; i < fwords; i += blockDim.x) dst[i] = __brev(__ldg(src + i));
        }
        if (P.rank_smem) copy_in(P.off_rank, T.rank, words * (int64_t)sizeof(RankT));
    }
    __syncthreads();

    const int unit = PACKED ? 4 : 1;
    const int64_t tile_units = PACKED ? (P.tile >> 4) : P.tile;

    if ((ZW == 1 || ZW == 2) && warp == P.consumers + 1) {
        zero_writer<ZW>(P, smem, zdone, lane);
        return;
    }
    if (warp == P.consumers) {
        // ---------------- producer warp ----------------
        if (lane == 0) {
            // tile k goes to stage st = k mod S in the phase ph = (k / S) mod 2 of that
            // stage, both kept by counting (no division per tile)
            int k = 0, st = 0;
            uint32_t ph = 0;
            for (int64_t t = blockIdx.x; t < P.n_tiles;
                 t += gridDim.x, k++, ph ^= (st + 1 == S) ? 1u : 0u, st = (st + 1 == S) ? 0 : st + 1) {
                if (k >= S && !wait_or_abort(smem_addr(&empty[st]), ph ^ 1u, P.timeout_ns, abort_flag))
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
    K.status = T.status;
    const void *rank_ptr = P.rank_smem ? (const void *)srank : nullptr;
    const uint32_t all = LW == 32 ? 0xFFFFFFFFu : ((1u << LW) - 1u);
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    volatile uint32_t *queue = reinterpret_cast<volatile uint32_t *>(smem + P.off_queue) + warp * kQueue;
    uint32_t qhead = 0, qcount = 0;   // warp-uniform
    int k = 0, st = 0;
    uint32_t ph = 0;   // stage k mod S and its phase (k / S) mod 2, kept by counting
    for (int64_t t = blockIdx.x; t < P.n_tiles;
         t += gridDim.x, k++, ph ^= (st + 1 == S) ? 1u : 0u, st = (st + 1 == S) ? 0 : st + 1) {
        if (!wait_or_abort(smem_addr(&full[st]), ph, P.timeout_ns, abort_flag)) {
            if (lane == 0) {
                record_error(T.status, PFAC_ERR_TIMEOUT);
                if (ZW == 3) bulk_wait_all();
            }
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
            uint32_t pend;
            if constexpr (SCR == 1) {
                const uint32_t bmask1 = (1u << (2 * kFilter1B)) - 1u;
                pend = filter_bits<true, LW>(T, sf, x0, x1, x2, bmask1) & fast;
                pend = filter_bits_screened<LW>(T, x0, x1, x2, bmask, pend);
            } else if constexpr (SCR == 2) {
                static_assert(LW == 32, "the sampled screen covers a lane's 32 offsets");
                pend = filter_bits_screened<LW>(T, x0, x1, x2, bmask,
                                                sampled_candidates<2>(T, nullptr, x0, x1, x2, lane) & fast);
            } else if constexpr (SCR == 3) {
                static_assert(LW == 32, "the sampled screen covers a lane's 32 offsets");
                const uint8_t *fb = reinterpret_cast<const uint8_t *>(sf);
                pend = filter_bits_of(T, x0, x1, x2, bmask, sampled_candidates<3>(T, fb, x0, x1, x2, lane) & fast);
            } else {
                pend = filter_bits<FSMEM, LW>(T, sf, x0, x1, x2, bmask) & fast;
            }
            // near the text end: offsets with fewer than b readable bases walk from the
            // root when a pattern shorter than b could still fit
            if (T.min_len < B) pend |= valid & ~fast & clear_runs(bad, T.min_len);
            // Release the stage only once every lane has used its words: the producer
            // refills it as soon as all consumer warps have arrived, and a word read
            // after that would come from the next fill.
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
            if (!COMPACT && !ZW) zero_batch<LW>(K, warp_base, lane, valid, true, pol);
            if constexpr (ZW == 3) {
                // the warp's zeros as bulk copies, one bulk group per tile (empty past the
                // text's end), the last < 4 ids by plain stores
                const int64_t cnt = min((int64_t)(32 * LW), n - warp_base);
                if (lane == 0) {
                    if (cnt > 0) {
                        uint8_t *dst = reinterpret_cast<uint8_t *>(P.out + warp_base);
                        const int64_t full = (cnt * 4) & ~(int64_t)15;
                        const uint32_t zb = smem_addr(smem + P.off_zero);
                        for (int64_t bb = 0; bb < full; bb += P.zero_chunk)
                            bulk_store(dst + bb, zb, (uint32_t)min((int64_t)P.zero_chunk, full - bb), pol);
                        for (int64_t i = full / 4; i < cnt; i++) P.out[warp_base + i] = 0;
                    }
                    bulk_commit();
                }
            }
            // Zeros stored above by one lane are ordered before matches stored by another
            // lane in a later round by the warp barriers between them (this one first).
            __syncwarp();
            uint32_t qold = qcount;          // queued offsets of earlier tiles

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
                if ((ZW == 1 || ZW == 2) && qcount >= 32 &&
                    !wait_zeros(zdone, (uint32_t)k + 1, P.timeout_ns, abort_flag)) {
                    if (lane == 0) record_error(T.status, PFAC_ERR_TIMEOUT);
                    return;
                }
                if (ZW == 3 && qcount >= 32) {
                    // rounds of earlier tiles need their bulk groups complete (all but this
                    // tile's); a round with this tile's offsets needs this tile's too
                    const uint32_t taken = qcount & ~31u;
                    if (lane == 0) {
                        if (taken <= qold) bulk_wait_1();
                        else bulk_wait_all();
                        fence_proxy_async_global();
                    }
                    __syncwarp();
                    qold -= min(qold, taken);
                }
                while (qcount >= 32) {
                    queue_round<COMPACT, FSMEM, RANK16, ALL>(P, K, sf, rank_ptr, queue, qhead, 32, lane);
                    qhead = (qhead + 32) & (kQueue - 1);
                    qcount -= 32;
                    __syncwarp();   // the entries just read may be written again
                }
            }
        } else {
            // ASCII: each lane packs only its own LW bytes from the stage; the rest of its
            // 64-base window comes from the next lanes by shuffles, and the window of the
            // last lanes from the bytes right after the warp's span (the next warp's
            // first bytes or the stage's halo), which the first lanes pack. Then the lane
            // walks what passes at once, through scan_lane_batch.
            constexpr uint32_t kFull = 0xFFFFFFFFu;
            const uint8_t *r = stage + p_rel;
            uint32_t x0 = 0, x1 = 0, x2 = 0, x3 = 0;
            uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;
            if constexpr (LW == 16) {
                uint32_t h = 0, hb = 0;
                if (rem > 0) x0 = pack16(lds_v4(r), &b0);
                if (lane < 3) h = pack16(lds_v4(r + 512), &hb);          // words 32..34 of the warp
                // window word k of this lane: word lane + k of the warp
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
                uint32_t h0 = 0, h1 = 0, hb0 = 0, hb1 = 0;
                if (rem > 0) {
                    x0 = pack16(lds_v4(r), &b0);
                    x1 = pack16(lds_v4(r + 16), &b1);
                }
                if (lane == 0) {                                          // words 64, 65 of the warp
                    h0 = pack16(lds_v4(r + 1024), &hb0);
                    h1 = pack16(lds_v4(r + 1040), &hb1);
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
            // bytes past the text are already marked in `bad` from `rem`
            bad |= (uint64_t)b0 | ((uint64_t)b1 << 16) | ((uint64_t)b2 << 32) | ((uint64_t)b3 << 48);
            // release the stage once every lane has used its bytes (see the packed path)
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty[st]));
            scan_lane_batch<PACKED, COMPACT, FSMEM, RANK16, LW, ALL>(T, K, sf, rank_ptr, P.walk_loads, 0u, P.text,
                                                                nullptr, n, warp_base, lane, x0, x1, x2, x3, bad,
                                                                valid, true, pol);
        }
    }
    if (ZW == 3 && lane == 0) {
        bulk_wait_all();                 // every bulk copy of the warp has read its source
        fence_proxy_async_global();
    }
    __syncwarp();
    if (PACKED && qcount) {
        if ((ZW == 1 || ZW == 2) && !wait_zeros(zdone, (uint32_t)k, P.timeout_ns, abort_flag)) {
            if (lane == 0) record_error(T.status, PFAC_ERR_TIMEOUT);
            return;
        }
        queue_round<COMPACT, FSMEM, RANK16, ALL>(P, K, sf, rank_ptr, queue, qhead, qcount, lane);
    }
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
        K.status = P.t.status;
        emit_match<COMPACT>(K, it.gp, walk_global<PACKED, ALL>(P.t, P.text, nullptr, it.gp + it.span, it.gp, it.s,
                                                               (int)(it.q_set & 0xFFFFu), it.best, &K));
    }
}

struct ScanLayout {
    uint32_t off_filter, off_rank, off_bar, off_queue, off_stage, stage_bytes, off_zero, total;
    int32_t stage_units;
};

static inline uint32_t align128(uint64_t x) { return (uint32_t)((x + 127) & ~(uint64_t)127); }

static ScanLayout scan_layout(int consumers, int lw, int stages, int64_t filter_smem_bytes, int64_t rank_smem_bytes,
                              bool packed, int64_t zero_bytes = 0)
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
    L.off_zero = (uint32_t)off;
    off += align128((uint64_t)zero_bytes);
    L.total = (uint32_t)off;
    return L;
}

// The zero writer a launch uses: only dense scans of packed text with 32 offsets per
// lane have one (other launches store zeros from the consumer warps).
static int zero_writer_of(const TiledConfig &cfg, bool packed, bool compact, bool all)
{
    if (!packed || compact || all || cfg.lane_offsets != 32) return 0;
    return cfg.zero_writer >= 1 && cfg.zero_writer <= 3 ? cfg.zero_writer : 0;
}

static int consumers_of(const TiledConfig &cfg, int zw = 0)
{
    return cfg.threads / 32 - 1 - ((zw == 1 || zw == 2) ? 1 : 0);
}
static int lane_width_of(const TiledConfig &cfg) { return cfg.lane_offsets == 32 ? 32 : 16; }
static int stages_of(const TiledConfig &cfg, bool packed) { return cfg.stages > 0 ? cfg.stages : (packed ? 3 : 2); }

// Shared memory per CTA, by priority: the text stages, the prefix filter (read for
// every offset), then the rank index (read for every walk the filter passes).
struct SmemPlan {
    int64_t filter_bytes, rank_bytes;   // bytes copied into shared memory (0 = global)
    int64_t total;
    int scr;                            // 1: filter_bytes hold the first-level filter;
                                        // 2: the sampled screen (global memory) is used
    int zw;                             // zero writer (0 = the consumer warps)
    int64_t zero_chunk;                 // bytes of the bulk-store zero tile (zw == 2 or 3)
};

// With a bulk-store zero writer (zw == 2) the zero tile comes after the filter and before
// the rank index: 2 KB at least (else the writer uses 16-byte stores, zw = 1), then up to
// 16 KB from what the rank index leaves.
static SmemPlan plan_smem(const DeviceTable &t, const TiledConfig &cfg, bool packed, const DeviceProps &dp,
                          int zw = 0)
{
    SmemPlan pl{};
    const int C = consumers_of(cfg, zw);
    const int LW = lane_width_of(cfg);
    const int S = stages_of(cfg, packed);
    const int64_t per_cta = (int64_t)dp.smem_per_sm / std::max(1, cfg.ctas_per_sm) - 1024;
    const int64_t limit = std::min<int64_t>(dp.smem_optin, per_cta);
    const int64_t words = t.filter_b >= 3 ? ((int64_t)1 << (2 * t.filter_b)) / 32 : 1;
    const int64_t fbytes = words * 4;
    const int64_t rbytes = words * (t.rank_wide ? 4 : 2);
    int64_t zb = (zw == 2 || zw == 3) ? 2048 : 0;
    auto total = [&](int64_t f, int64_t r) { return (int64_t)scan_layout(C, LW, S, f, r, packed, zb).total; };
    if (total(0, 0) > limit) {
        pl.total = -1;
        return pl;
    }
    pl.zw = zw;
    pl.filter_bytes = total(fbytes, 0) <= limit ? fbytes : 0;
    const bool sampled = t.sample && t.sample_q == kSampleQ && t.sample_s == kSampleS && LW == 32;
    const int64_t g10 = ((int64_t)1 << (2 * kSampleQSmem)) / 8;
    const bool sampled10 = t.sample && t.sample_q == kSampleQSmem && t.sample_s == kSampleS && LW == 32 && packed &&
                           total(g10, 0) <= limit;
    if (sampled10 && cfg.screen == 2) {
        pl.filter_bytes = g10;           // the 10-gram screen in place of the filter
        pl.scr = 3;
    } else if (!pl.filter_bytes && packed && sampled && cfg.screen != 1) {
        pl.scr = 2;
    } else if (!pl.filter_bytes && packed && t.filter1_b == kFilter1B && t.filter1 && cfg.screen != 2) {
        const int64_t f1 = ((int64_t)1 << (2 * kFilter1B)) / 8;
        if (total(f1, 0) <= limit) {
            pl.filter_bytes = f1;
            pl.scr = 1;
        }
    }
    if ((zw == 2 || zw == 3) && total(pl.filter_bytes, 0) > limit) {
        zw = pl.zw = zw == 2 ? 1 : 0;    // no room for a zero tile: 16-byte stores instead
        zb = 0;
    }
    pl.rank_bytes = ((pl.scr == 0 || pl.scr == 3) && cfg.smem_table_bytes >= 0 &&
                     total(pl.filter_bytes, rbytes) <= limit) ? rbytes : 0;
    if (zw == 3) pl.zero_chunk = zb;
    if (zw == 2) {
        for (int64_t c = 16384; c > 2048; c >>= 1) {
            zb = c;
            if (total(pl.filter_bytes, pl.rank_bytes) <= limit) break;
            zb = 2048;
        }
        pl.zero_chunk = zb;
    }
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
    // the window: the skip entries (l2_persist 1), or the prefix filter and the sampled
    // screen, adjacent in the table's allocation (l2_persist 2, tables with a screen)
    const int64_t skip_bytes = P.t.n_states * 16;
    const void *win_base = P.t.skip;
    int64_t win_bytes = skip_bytes;
    if (cfg.l2_persist == 2) {
        win_base = P.t.filter;
        win_bytes = P.t.sample && P.t.filter
                        ? (int64_t)((const uint8_t *)P.t.sample - (const uint8_t *)P.t.filter) +
                              ((int64_t)1 << (2 * P.t.sample_q)) / 8
                        : 0;
    }
    if (cfg.l2_persist > 0 && dp.persist_l2_max > 0 && win_bytes > 0) {
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
        const int64_t win = std::min<int64_t>(win_bytes, max_win);
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = (void *)win_base;
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

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per
// (kernel, device): later launches, including those captured into a CUDA graph, make
// no attribute call.
static cudaError_t allow_max_smem(const void *kern, const DeviceProps &dp)
{
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({kern, dp.device})) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dp.smem_optin);
    if (e == cudaSuccess) done.insert({kern, dp.device});
    return e;
}

template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, bool ALL, int SCR>
static void (*scan_kernel_for(bool lw32, int zw))(const ScanParams)
{
    if constexpr (PACKED && !COMPACT && !ALL) {
        if (zw == 1) return scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL, SCR, 1>;
        if (zw == 2) return scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL, SCR, 2>;
        if (zw == 3) return scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL, SCR, 3>;
    }
    if constexpr (SCR >= 2) {
        return scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL, SCR>;
    } else {
        return lw32 ? scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 32, ALL, SCR>
                    : scan_kernel<PACKED, COMPACT, FSMEM, RANK16, 16, ALL, SCR>;
    }
}

template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, bool ALL, int SCR = 0>
static int launch_scan_t(const ScanParams &P, int grid, int threads, uint32_t smem, int tail_grid, cudaStream_t st,
                         const TiledConfig &cfg, const DeviceProps &dp, int zw)
{
    const bool lw32 = lane_width_of(cfg) == 32;
    auto kern = scan_kernel_for<PACKED, COMPACT, FSMEM, RANK16, ALL, SCR>(lw32, zw);
    if ((int64_t)smem > (int64_t)dp.smem_optin) return PFAC_ERR_UNSUPPORTED;
    if (allow_max_smem((const void *)kern, dp) != cudaSuccess) return PFAC_ERR_CUDA;
    if (launch_with_policy(kern, P, grid, threads, smem, st, cfg, dp) != cudaSuccess) return PFAC_ERR_CUDA;
    tail_kernel<PACKED, COMPACT, ALL><<<tail_grid, 256, 0, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? PFAC_OK : PFAC_ERR_CUDA;
}

template <bool PACKED, bool COMPACT, bool ALL = false>
static int launch_scan_w(const ScanParams &P, bool fsmem, bool rank16, int grid, int threads, uint32_t smem,
                         int tail_grid, cudaStream_t st, const TiledConfig &cfg, const DeviceProps &dp,
                         int scr = 0, int zw = 0)
{
    if constexpr (PACKED) {
        if (scr == 1)
            return rank16 ? launch_scan_t<PACKED, COMPACT, false, true, ALL, 1>(P, grid, threads, smem, tail_grid,
                                                                              st, cfg, dp, zw)
                          : launch_scan_t<PACKED, COMPACT, false, false, ALL, 1>(P, grid, threads, smem, tail_grid,
                                                                               st, cfg, dp, zw);
        if (scr == 2)
            return rank16 ? launch_scan_t<PACKED, COMPACT, false, true, ALL, 2>(P, grid, threads, smem, tail_grid,
                                                                              st, cfg, dp, zw)
                          : launch_scan_t<PACKED, COMPACT, false, false, ALL, 2>(P, grid, threads, smem, tail_grid,
                                                                               st, cfg, dp, zw);
        if (scr == 3)
            return rank16 ? launch_scan_t<PACKED, COMPACT, false, true, ALL, 3>(P, grid, threads, smem, tail_grid,
                                                                              st, cfg, dp, zw)
                          : launch_scan_t<PACKED, COMPACT, false, false, ALL, 3>(P, grid, threads, smem, tail_grid,
                                                                               st, cfg, dp, zw);
    }
    if (fsmem)
        return rank16 ? launch_scan_t<PACKED, COMPACT, true, true, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp, zw)
                      : launch_scan_t<PACKED, COMPACT, true, false, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp,
                                                                         zw);
    return rank16 ? launch_scan_t<PACKED, COMPACT, false, true, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp, zw)
                  : launch_scan_t<PACKED, COMPACT, false, false, ALL>(P, grid, threads, smem, tail_grid, st, cfg, dp, zw);
}

int launch_tiled(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out, int64_t *c_off,
                 int32_t *c_ids, int64_t cap, unsigned long long *count, const TiledConfig &cfg,
                 const DeferScratch &scratch, cudaStream_t st, const DeviceProps &dp, bool all_matches)
{
    const bool compact = c_off != nullptr;
    if (compact && cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return PFAC_ERR_CUDA;
    if (n == 0) return PFAC_OK;
    const int zw_asked = zero_writer_of(cfg, packed, compact, all_matches);
    const int LW = lane_width_of(cfg);
    const int S = stages_of(cfg, packed);
    if (!t.skip || !t.filter || !t.rank || !t.dense || t.filter_b < 1 || t.filter_b > kMaxFilterB ||
        consumers_of(cfg, zw_asked) < 1 || (cfg.threads & 31) || cfg.threads > 1024 || S < 2 || S > kMaxStages ||
        !scratch.items || !scratch.count)
        return PFAC_ERR_INVALID_ARG;
    const SmemPlan pl = plan_smem(t, cfg, packed, dp, zw_asked);
    if (pl.total < 0 || pl.total > dp.smem_optin) return PFAC_ERR_UNSUPPORTED;
    const int zw = pl.zw;
    const int C = consumers_of(cfg, zw);
    const ScanLayout L = scan_layout(C, LW, S, pl.filter_bytes, pl.rank_bytes, packed, pl.zero_chunk);
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
    P.off_zero = L.off_zero;
    P.zero_chunk = (uint32_t)pl.zero_chunk;
    P.timeout_ns = cfg.timeout_ns > 0 ? cfg.timeout_ns : 2000000000LL;
    const int64_t grid64 = std::min<int64_t>(P.n_tiles, (int64_t)dp.num_sms * std::max(1, cfg.ctas_per_sm));
    const int grid = (int)std::max<int64_t>(1, grid64);
    // a queued offset codes its tile round in 32 - kRelBits bits
    if (packed && (P.n_tiles + grid - 1) / grid > ((int64_t)1 << (32 - kRelBits))) return PFAC_ERR_UNSUPPORTED;
    const int tail_grid = dp.num_sms * 4;
    const bool fsmem = pl.filter_bytes > 0 && pl.scr == 0;
    const int scr = pl.scr;
    const bool rank16 = !t.rank_wide;
    if (all_matches) {   // the match list of every pattern on every walk (packed text only)
        if (!packed || !compact) return PFAC_ERR_INVALID_ARG;
        return launch_scan_w<true, true, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp,
                                               scr);
    }
    if (packed)
        return compact ? launch_scan_w<true, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp,
                                                   scr)
                       : launch_scan_w<true, false>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp,
                                                    scr, zw);
    return compact ? launch_scan_w<false, true>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp)
                   : launch_scan_w<false, false>(P, fsmem, rank16, grid, cfg.threads, L.total, tail_grid, st, cfg, dp);
}

size_t defer_item_bytes() { return sizeof(DeferItem); }

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
