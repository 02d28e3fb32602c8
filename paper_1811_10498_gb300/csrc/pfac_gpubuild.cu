// Table construction on the GPU (pfac_build_device in pfac.h): the same tables as the
// host builder (trie_build.cpp), bit for bit, for dictionaries whose patterns are
// already in device memory.
//
// The trie is built one depth at a time. The states of depth d are the ids
// [level[d], level[d+1]) in breadth-first order, and every pattern longer than d sits at
// one of them. Each such pattern marks the pair (its state, its base at position d); an
// exclusive prefix sum over the marks, laid out state by state and base by base (A, C,
// G, T), numbers the distinct pairs, and pair k becomes state level[d+1] + k. This is
// the breadth-first order with children in A, C, G, T order, i.e. the numbering of the
// insertion procedure of Section V-A followed by the breadth-first rearrangement cited in
// Section II. A pattern that ends at depth d + 1 gives its 1-based id to the state it
// reaches; the lowest id wins, as in the host builder.
//
// Then, from the rows: node words and skip entries (each state follows its chain of
// single-child edges, at most 16 bases); the prefix filter of order b (every b-mer walked
// from the root: set when the walk reaches depth b, or when a pattern ends on the way,
// which makes the entry special), its rank index (an exclusive prefix sum of the words'
// popcounts) and dense entries; the first-level filter of order 10 and the sampled
// screen, under the host builder's conditions.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace pfac {
namespace {

constexpr uint32_t kNoId = 0xFFFFFFFFu;
constexpr uint32_t kValNone = 0xFFFFFFFFu, kValSpecial = 0xFFFFFFFEu;
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int dev_base_code(uint32_t b)
{
    return b == 'A' ? 0 : b == 'C' ? 1 : b == 'G' ? 2 : b == 'T' ? 3 : -1;
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of uint32 values (device-wide, in place), by tiles of 4096.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kScanThreads) scan_tiles(uint32_t *data, int64_t n, uint32_t *tile_sums,
                                                          unsigned long long *total)
{
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = base + i < n ? data[base + i] : 0u;
        sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t ws = warp_sums[lane];
        uint32_t wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, wi, d);
            if (lane >= d) wi += o;
        }
        warp_sums[lane] = wi - ws;     // exclusive over warps
        if (lane == 31) {
            if (tile_sums) tile_sums[blockIdx.x] = wi;
            if (total) *total = wi;
        }
    }
    __syncthreads();
    uint32_t run = warp_sums[warp] + incl - sum;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

__global__ void add_tile_offsets(uint32_t *data, int64_t n, const uint32_t *tile_offsets)
{
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const uint32_t add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t j = i + (int64_t)k * kScanThreads;
        if (j < n) data[j] += add;
    }
}

// Scratch for the tile sums of every level of the recursion.
static int64_t scan_scratch_words(int64_t n)
{
    int64_t words = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        words += n + 64;
    }
    return words + 64;
}

static void scan_exclusive(uint32_t *data, int64_t n, unsigned long long *total, uint32_t *scratch, cudaStream_t st)
{
    if (n <= kScanTile) {
        scan_tiles<<<1, kScanThreads, 0, st>>>(data, n, nullptr, total);
        return;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(data, n, scratch, nullptr);
    scan_exclusive(scratch, tiles, total, scratch + tiles + 64, st);
    add_tile_offsets<<<(unsigned)tiles, kScanThreads, 0, st>>>(data, n, scratch);
}

// ---------------------------------------------------------------------------
// Kernels of the construction.
// ---------------------------------------------------------------------------

struct BuildStats {
    unsigned long long total;      // bases over all patterns
    int32_t max_len, min_len;
    uint32_t errors;               // bit 0: empty pattern, 1: bad offsets, 2: byte outside ACGT
    uint32_t terminals;            // states where a pattern ends
};

__global__ void validate_kernel(const uint8_t *__restrict__ blob, const int64_t *__restrict__ off, int32_t n,
                                BuildStats *stats)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[j], len = off[j + 1] - a;
        if (a < 0 || len < 0) {
            atomicOr(&stats->errors, 2u);
            continue;
        }
        if (len == 0) {
            atomicOr(&stats->errors, 1u);
            continue;
        }
        bool bad = false;
        for (int64_t k = 0; k < len; k++) bad |= dev_base_code(blob[a + k]) < 0;
        if (bad) atomicOr(&stats->errors, 4u);
        atomicAdd(&stats->total, (unsigned long long)len);
        atomicMax(&stats->max_len, (int32_t)min(len, (int64_t)0x7FFFFFFF));
        atomicMin(&stats->min_len, (int32_t)min(len, (int64_t)0x7FFFFFFF));
    }
}

// Each pattern longer than d marks (its state at depth d, its base d).
__global__ void mark_kernel(const uint8_t *__restrict__ blob, const int64_t *__restrict__ off, int32_t n, int32_t d,
                            int64_t lvl_d, const uint32_t *__restrict__ cur, uint32_t *flag)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[j];
        if (off[j + 1] - a <= d) continue;
        const int c = dev_base_code(blob[a + d]);
        flag[((int64_t)cur[j] - lvl_d) * 4 + c] = 1u;
    }
}

// ... then moves to the state its pair was numbered, writes the edge, and gives its id to
// the state when it ends there (lowest id wins).
__global__ void assign_kernel(const uint8_t *__restrict__ blob, const int64_t *__restrict__ off, int32_t n, int32_t d,
                              int64_t lvl_d, int64_t lvl_d1, uint32_t *cur, const uint32_t *__restrict__ pos,
                              int32_t *rows, uint32_t *out_id)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[j], len = off[j + 1] - a;
        if (len <= d) continue;
        const int c = dev_base_code(blob[a + d]);
        const uint32_t s = cur[j];
        const uint32_t child = (uint32_t)(lvl_d1 + pos[((int64_t)s - lvl_d) * 4 + c]);
        rows[4 * (int64_t)s + c] = (int32_t)child;
        cur[j] = child;
        if (len == d + 1) atomicMin(&out_id[child], (uint32_t)(j + 1));
    }
}

// No id -> 0; count the terminal states; set bit 31 of every edge into one.
__global__ void finish_ids_kernel(uint32_t *out_id, int64_t S, BuildStats *stats)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = out_id[s];
        if (v == kNoId) out_id[s] = 0;
        else atomicAdd(&stats->terminals, 1u);
    }
}

__global__ void terminal_flags_kernel(int32_t *rows, const uint32_t *__restrict__ out_id, int64_t cells)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < cells; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = (uint32_t)rows[k];
        if (e && out_id[e]) rows[k] = (int32_t)(e | 0x80000000u);
    }
}

// Node word: child mask, terminal bit, first child.
__global__ void node_kernel(const int32_t *__restrict__ rows, const uint32_t *__restrict__ out_id, int64_t S,
                            uint32_t *node)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t mask = 0, first = 0;
        for (int c = 3; c >= 0; c--) {
            const uint32_t e = (uint32_t)rows[4 * s + c];
            if (e) {
                mask |= 1u << c;
                first = e & 0x7FFFFFFFu;
            }
        }
        node[s] = mask | (first << kNodeFirstShift) | (out_id[s] ? kNodeTermBit : 0u);
    }
}

// Skip entry of s: follow the single-child edges below s, at most kSkipMaxLen of them,
// stopping right after entering a terminal state or a state without exactly one child.
__global__ void skip_kernel(const uint32_t *__restrict__ node, int64_t S, uint32_t *skip)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t nd = node[s];
        uint32_t label = 0, len = 0, target = 0, target_term = 0;
        uint32_t cur = nd;
        while (len < (uint32_t)kSkipMaxLen && __popc(cur & kNodeMaskBits) == 1) {
            const uint32_t c = (uint32_t)(__ffs(cur & kNodeMaskBits) - 1);
            const uint32_t ch = cur >> kNodeFirstShift;
            label |= c << (2 * len);
            len++;
            target = ch;
            cur = node[ch];
            if (cur & kNodeTermBit) {
                target_term = kSkipTargetTerm;
                break;
            }
            if (__popc(cur & kNodeMaskBits) != 1) break;
        }
        uint32_t *e = skip + 4 * s;
        e[0] = label;
        e[1] = len | target_term | ((nd & kNodeTermBit) ? kSkipSelfTerm : 0u);
        e[2] = target;
        e[3] = nd;
    }
}

// The walk over the b-mer w from the root: the state reached at depth b, kValSpecial
// when a pattern ends on the way (even if the walk then stops), kValNone when the walk
// stops first with no pattern on the way.
__device__ __forceinline__ uint32_t bmer_value(const int32_t *__restrict__ rows, uint32_t w, int b)
{
    uint32_t s = 0;
    bool seen = false;
    for (int j = 0; j < b; j++) {
        const uint32_t e = (uint32_t)__ldg(rows + 4 * (int64_t)s + ((w >> (2 * j)) & 3u));
        if (!e) return seen ? kValSpecial : kValNone;
        s = e & 0x7FFFFFFFu;
        seen |= (e >> 31) != 0;
    }
    return seen ? kValSpecial : s;
}

// One warp per filter word: 32 walks and a ballot. Also the popcount of each word (for
// the rank index).
__global__ void filter_kernel(const int32_t *__restrict__ rows, int b, int64_t E, int64_t words, uint32_t *filter,
                              uint32_t *popc)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words; w += warps) {
        const int64_t k = w * 32 + lane;
        const bool on = k < E && bmer_value(rows, (uint32_t)k, b) != kValNone;
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, on);
        if (lane == 0) {
            filter[w] = word;
            popc[w] = (uint32_t)__popc(word);
        }
    }
}

// Dense entries (the skip entry of the depth-b state, or the special entry) in b-mer
// order; the rank index (16- or 32-bit); the first-level filter's bits.
__global__ void dense_kernel(const int32_t *__restrict__ rows, const uint32_t *__restrict__ skip, int b, int64_t E,
                             int64_t words, const uint32_t *__restrict__ filter, const uint32_t *__restrict__ rank,
                             uint32_t *dense, uint16_t *rank16, uint32_t *rank32, uint32_t *filter1)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words; w += warps) {
        const uint32_t word = filter[w];
        const uint32_t r0 = rank[w];
        if (lane == 0) {
            if (rank16) rank16[w] = (uint16_t)r0;
            if (rank32) rank32[w] = r0;
        }
        if (!((word >> lane) & 1u)) continue;
        const int64_t k = w * 32 + lane;
        const uint32_t v = bmer_value(rows, (uint32_t)k, b);
        const uint32_t r = r0 + (uint32_t)__popc(word & ((1u << lane) - 1u));
        uint4 d;
        if (v == kValSpecial) d = make_uint4(0u, kSkipSpecial, 0u, 0u);
        else d = *reinterpret_cast<const uint4 *>(skip + 4 * (int64_t)v);
        *reinterpret_cast<uint4 *>(dense + 4 * (int64_t)r) = d;
        if (filter1) {
            const uint32_t w1 = (uint32_t)(k & ((1LL << (2 * kFilter1B)) - 1));
            atomicOr(filter1 + (w1 >> 5), 1u << (w1 & 31u));
        }
    }
    (void)E;
}

// Sampled screen: the q-grams at positions 0 .. s-1 of every pattern.
__global__ void sample_kernel(const uint8_t *__restrict__ blob, const int64_t *__restrict__ off, int32_t n, int q,
                              uint32_t *sample)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t *p = blob + off[j];
        for (int d = 0; d < kSampleS; d++) {
            uint32_t g = 0;
            for (int k = 0; k < q; k++) g |= (uint32_t)dev_base_code(p[d + k]) << (2 * k);
            atomicOr(sample + (g >> 5), 1u << (g & 31u));
        }
    }
}

// Device allocations of one construction, freed together.
struct Allocs {
    std::vector<void *> ptrs;
    ~Allocs()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t get(T **out, size_t bytes)
    {
        void *p = nullptr;
        const cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) ptrs.push_back(p);
        *out = (T *)p;
        return e;
    }
};

int grid_for(int64_t items, int threads, const DeviceProps &dp)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads, (int64_t)dp.num_sms * 32));
}

}  // namespace

int build_device_tables(const uint8_t *d_blob, const int64_t *d_off, int32_t n, int32_t filter_b_opt,
                        int32_t sample_mode, cudaStream_t st, const DeviceProps &dp, DeviceBuild *out)
{
    if (n <= 0 || !d_blob || !d_off || !out || filter_b_opt > kMaxFilterB) return PFAC_ERR_INVALID_ARG;
#define PFAC_CK(x)                                                                      \
    do {                                                                                \
        const cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                        \
            cudaGetLastError();                                                         \
            return e_ == cudaErrorMemoryAllocation ? PFAC_ERR_OOM : PFAC_ERR_CUDA;     \
        }                                                                               \
    } while (0)
    Allocs tmp;
    // ---- validate ----------------------------------------------------------------
    BuildStats *d_stats = nullptr;
    PFAC_CK(tmp.get(&d_stats, sizeof(BuildStats)));
    BuildStats hs{};
    hs.max_len = 0;
    hs.min_len = 0x7FFFFFFF;
    PFAC_CK(cudaMemcpyAsync(d_stats, &hs, sizeof hs, cudaMemcpyHostToDevice, st));
    validate_kernel<<<grid_for(n, 256, dp), 256, 0, st>>>(d_blob, d_off, n, d_stats);
    PFAC_CK(cudaGetLastError());
    PFAC_CK(cudaMemcpyAsync(&hs, d_stats, sizeof hs, cudaMemcpyDeviceToHost, st));
    PFAC_CK(cudaStreamSynchronize(st));
    if (hs.errors & 2u) return PFAC_ERR_INVALID_ARG;
    if (hs.errors & 1u) return PFAC_ERR_EMPTY_PATTERN;
    if (hs.errors & 4u) return PFAC_ERR_BAD_SYMBOL;
    const int32_t max_len = hs.max_len, min_len = hs.min_len;
    const int64_t cap_states = (int64_t)hs.total + 1;         // every base a new state at most

    // ---- the trie, one depth at a time ---------------------------------------------
    int32_t *rows = nullptr;
    uint32_t *out_id = nullptr, *cur = nullptr, *flag = nullptr, *scratch = nullptr;
    unsigned long long *d_count = nullptr;
    const int64_t max_flags = 4 * (int64_t)n + 4;
    PFAC_CK(tmp.get(&rows, (size_t)cap_states * 16));
    PFAC_CK(tmp.get(&out_id, (size_t)cap_states * 4));
    PFAC_CK(tmp.get(&cur, (size_t)n * 4));
    PFAC_CK(tmp.get(&flag, (size_t)max_flags * 4));
    PFAC_CK(tmp.get(&scratch, (size_t)scan_scratch_words(max_flags) * 4));
    PFAC_CK(tmp.get(&d_count, sizeof(unsigned long long)));
    PFAC_CK(cudaMemsetAsync(rows, 0, (size_t)cap_states * 16, st));
    PFAC_CK(cudaMemsetAsync(out_id, 0xFF, (size_t)cap_states * 4, st));
    PFAC_CK(cudaMemsetAsync(cur, 0, (size_t)n * 4, st));
    std::vector<int64_t> level((size_t)max_len + 2, 0);
    level[1] = 1;
    const int g = grid_for(n, 256, dp);
    for (int32_t d = 0; d < max_len; d++) {
        const int64_t width = level[(size_t)d + 1] - level[(size_t)d];
        const int64_t flags = 4 * width;
        PFAC_CK(cudaMemsetAsync(flag, 0, (size_t)flags * 4, st));
        mark_kernel<<<g, 256, 0, st>>>(d_blob, d_off, n, d, level[(size_t)d], cur, flag);
        scan_exclusive(flag, flags, d_count, scratch, st);
        assign_kernel<<<g, 256, 0, st>>>(d_blob, d_off, n, d, level[(size_t)d], level[(size_t)d + 1], cur, flag, rows,
                                         out_id);
        PFAC_CK(cudaGetLastError());
        unsigned long long added = 0;
        PFAC_CK(cudaMemcpyAsync(&added, d_count, sizeof added, cudaMemcpyDeviceToHost, st));
        PFAC_CK(cudaStreamSynchronize(st));
        level[(size_t)d + 2] = level[(size_t)d + 1] + (int64_t)added;
        if (level[(size_t)d + 2] > 0x7FFFFFFF) return PFAC_ERR_TOO_MANY_STATES;
    }
    const int64_t S = level[(size_t)max_len + 1];
    finish_ids_kernel<<<grid_for(S, 256, dp), 256, 0, st>>>(out_id, S, d_stats);
    terminal_flags_kernel<<<grid_for(4 * S, 256, dp), 256, 0, st>>>(rows, out_id, 4 * S);
    PFAC_CK(cudaGetLastError());

    // ---- skip entries -----------------------------------------------------------------
    const bool with_skip = S < kMaxNodeStates;
    uint32_t *node = nullptr, *skip = nullptr;
    if (with_skip) {
        PFAC_CK(tmp.get(&node, (size_t)S * 4));
        PFAC_CK(tmp.get(&skip, (size_t)S * 16));
        node_kernel<<<grid_for(S, 256, dp), 256, 0, st>>>(rows, out_id, S, node);
        skip_kernel<<<grid_for(S, 256, dp), 256, 0, st>>>(node, S, skip);
        PFAC_CK(cudaGetLastError());
    }

    // ---- prefix filter, rank index, dense entries, first-level filter --------------
    const double auto_b = std::ceil(std::log((double)n) / std::log(4.0) + 2.2);
    int32_t b = filter_b_opt == 0 ? (int32_t)std::min(12.0, std::max(6.0, auto_b))
                                  : (filter_b_opt < 0 ? 0 : filter_b_opt);
    if (filter_b_opt == 0 && n >= kDeepFilterMinPatterns && min_len >= kDeepFilterB) b = kDeepFilterB;
    int64_t words = 0, count = 0;
    int32_t rank_wide = 0, filter_b = 0, filter1_b = 0;
    uint32_t *filter = nullptr, *rank = nullptr, *dense = nullptr, *filter1 = nullptr, *rank32 = nullptr;
    uint16_t *rank16 = nullptr;
    if (b > 0 && with_skip) {
        filter_b = b;
        const int64_t E = (int64_t)1 << (2 * b);
        words = E >= 32 ? E / 32 : 1;
        PFAC_CK(tmp.get(&filter, (size_t)words * 4));
        PFAC_CK(tmp.get(&rank, (size_t)words * 4));
        uint32_t *fscratch = nullptr;
        PFAC_CK(tmp.get(&fscratch, (size_t)scan_scratch_words(words) * 4));
        const int fg = grid_for(words * 32, 256, dp);
        filter_kernel<<<fg, 256, 0, st>>>(rows, b, E, words, filter, rank);
        scan_exclusive(rank, words, d_count, fscratch, st);
        unsigned long long c = 0;
        PFAC_CK(cudaMemcpyAsync(&c, d_count, sizeof c, cudaMemcpyDeviceToHost, st));
        PFAC_CK(cudaStreamSynchronize(st));
        count = (int64_t)c;
        rank_wide = count > 65535;
        PFAC_CK(tmp.get(&dense, (size_t)count * 16));
        if (rank_wide) PFAC_CK(tmp.get(&rank32, (size_t)words * 4));
        else PFAC_CK(tmp.get(&rank16, (size_t)words * 2));
        if (b > kFilter1B) {
            filter1_b = kFilter1B;
            PFAC_CK(tmp.get(&filter1, ((size_t)1 << (2 * kFilter1B)) / 8));
            PFAC_CK(cudaMemsetAsync(filter1, 0, ((size_t)1 << (2 * kFilter1B)) / 8, st));
        }
        dense_kernel<<<fg, 256, 0, st>>>(rows, skip, b, E, words, filter, rank, dense, rank16, rank32, filter1);
        PFAC_CK(cudaGetLastError());
    }

    // ---- sampled screen -------------------------------------------------------------
    uint32_t *sample = nullptr;
    const int32_t q = sample_q_for(filter_b, min_len, sample_mode);
    const bool sampled = q > 0;
    const size_t sample_bytes = sampled ? ((size_t)1 << (2 * q)) / 8 : 0;
    if (sampled) {
        PFAC_CK(tmp.get(&sample, sample_bytes));
        PFAC_CK(cudaMemsetAsync(sample, 0, sample_bytes, st));
        sample_kernel<<<g, 256, 0, st>>>(d_blob, d_off, n, q, sample);
        PFAC_CK(cudaGetLastError());
    }
    PFAC_CK(cudaMemcpyAsync(&hs, d_stats, sizeof hs, cudaMemcpyDeviceToHost, st));
    PFAC_CK(cudaStreamSynchronize(st));

    // ---- one allocation in the layout of pfac_build_ex ---------------------------------
    auto r256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t rank_bytes = (size_t)words * (rank_wide ? 4 : 2);
    struct Part {
        const void *src;
        size_t bytes;
    } parts[] = {{rows, (size_t)S * 16},
                 {out_id, (size_t)S * 4},
                 {skip, with_skip ? (size_t)S * 16 : 0},
                 {filter, (size_t)words * 4},
                 {sample, sample_bytes},
                 {rank_wide ? (const void *)rank32 : (const void *)rank16, filter_b ? rank_bytes : 0},
                 {dense, (size_t)count * 16},
                 {filter1, filter1 ? ((size_t)1 << (2 * kFilter1B)) / 8 : 0}};
    size_t total = 256;
    for (auto &p : parts) total += r256(p.bytes);
    void *mem = nullptr;
    PFAC_CK(cudaMalloc(&mem, total));
    uint8_t *base = (uint8_t *)mem;
    const void **dst[] = {(const void **)&out->dt.rows, (const void **)&out->dt.out_id, (const void **)&out->dt.skip,
                          (const void **)&out->dt.filter, (const void **)&out->dt.sample, (const void **)&out->dt.rank,
                          (const void **)&out->dt.dense, (const void **)&out->dt.filter1};
    cudaError_t e = cudaMemsetAsync(base, 0, 256, st);
    size_t o = 256;
    for (size_t i = 0; i < sizeof(parts) / sizeof(parts[0]); i++) {
        *dst[i] = parts[i].bytes ? (const void *)(base + o) : nullptr;
        if (e == cudaSuccess && parts[i].bytes)
            e = cudaMemcpyAsync(base + o, parts[i].src, parts[i].bytes, cudaMemcpyDeviceToDevice, st);
        o += r256(parts[i].bytes);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(mem);
        cudaGetLastError();
        return PFAC_ERR_CUDA;
    }
    out->mem = mem;
    out->bytes = total;
    out->dt.status = (int32_t *)base;
    out->dt.n_states = S;
    out->dt.max_len = max_len;
    out->dt.min_len = min_len;
    out->dt.filter_b = filter_b;
    out->dt.filter1_b = filter1_b;
    out->dt.rank_wide = rank_wide;
    out->dt.sample_q = q;
    out->dt.sample_s = sampled ? kSampleS : 0;
    out->level = std::move(level);
    out->n_duplicates = (int64_t)n - (int64_t)hs.terminals;
    out->filter_set = count;
    out->skip_bytes = with_skip ? S * 16 : 0;
    return PFAC_OK;
#undef PFAC_CK
}

}  // namespace pfac
