// Internal declarations shared by the host trie builder, the runtime and the kernels.
#pragma once

#include <stdint.h>

#include <memory>
#include <new>
#include <utility>
#include <vector>

namespace pfac {

// Compact node word (4 bytes per state, breadth-first numbering):
//   bits 0..3  : child mask, bit c set if the state has an edge for base c (A,C,G,T)
//   bit  4     : terminal flag (a pattern ends at this state)
//   bits 5..31 : breadth-first id of the first child. Children of one state are
//                consecutive in breadth-first order, so the child for base c is
//                first + popcount(mask & ((1 << c) - 1)).
// Available when the trie has fewer than 2^27 states.
constexpr uint32_t kNodeMaskBits = 0xFu;
constexpr uint32_t kNodeTermBit = 0x10u;
constexpr int kNodeFirstShift = 5;
constexpr int64_t kMaxNodeStates = int64_t(1) << 27;

// Skip entry of a state s (16 bytes, one per state): the chain of single-child edges
// below s, compressed into one comparison (path compression of the same trie).
//   x : label, the bases of the chain (base i in bits 2i..2i+1), i < len
//   y : bits 0..4  len, 0..16 (0 when s has no child or two or more children)
//       bit  8     s itself is terminal
//       bit  9     special (dense entries only, see below): walk from the root
//       bit 10     the chain's last state is terminal
//   z : the chain's last state (the state len bases below s), when len > 0
//   w : the node word of s (to step from s when len == 0)
// A chain stops after 16 bases, at a state with no child or with two or more
// children, and right after entering a terminal state, so no state strictly inside a
// chain is terminal.
constexpr uint32_t kSkipLenMask = 31u;
constexpr uint32_t kSkipSelfTerm = 1u << 8;
constexpr uint32_t kSkipSpecial = 1u << 9;
constexpr uint32_t kSkipTargetTerm = 1u << 10;
constexpr int kSkipMaxLen = 16;

// Prefix filter of order b: one bit per b-mer w (base j of w in bits 2j..2j+1). The bit
// is 0 when the walk over w ends before depth b and no pattern ends on the way, so the
// answer at any offset where w starts is 0 whatever follows; it is 1 otherwise (the
// walk is still going at depth b, or a pattern ends within w). Bit w is bit w mod 32
// of word w / 32.
//
// Rank index of the filter: rank[i] = number of set bits in words 0 .. i-1 (16-bit
// when the filter has fewer than 65536 set bits, else 32-bit). The set bit of b-mer w
// has rank r = rank[w / 32] + popcount(word & ((1 << (w mod 32)) - 1)) and its entry
// is dense[r]: the skip entry of the state the walk over w reaches at depth b, or an
// entry with the special bit when a pattern ends within w (the answer then needs the
// walk from the root).
constexpr int kMaxFilterB = 14;
constexpr int kFilter1B = 10;      // order of the shared-memory first-level filter
// Automatic order for large dictionaries without short patterns (see the builder).
constexpr int kDeepFilterB = 14;
constexpr int32_t kDeepFilterMinPatterns = 1 << 19;

// Sampled screen: the q-grams (q = kSampleQ) at positions 0 .. kSampleS - 1 of every
// pattern, one bit per q-gram (bit g = bit g mod 32 of word g / 32, base j of g in bits
// 2j..2j+1). Built for tables whose filter lives in global memory and whose patterns
// all have at least kSampleQ + kSampleS - 1 bases: a scan probes it at every
// kSampleS-th offset, and an offset i can start a match only if the probe at the next
// multiple of kSampleS at or after i finds its bit set.
constexpr int kSampleQ = 13;
constexpr int kSampleS = 4;
// A table whose filter (order kFilter1B) fits in shared memory gets a sampled screen of
// 10-grams instead, kept in shared memory in its place (the filter is then read from
// global memory, for the offsets the screen lets through).
constexpr int kSampleQSmem = kFilter1B;

// q-gram length of the sampled screen a table gets (0 = none). sample_mode: -1 never,
// 0 the 13-gram screen of filters in global memory, 1 also the 10-gram screen of order-10
// filters (slower on the genome-like workload than the filter it replaces; kept as an
// option for the measurement).
inline int32_t sample_q_for(int32_t filter_b, int32_t min_len, int32_t sample_mode)
{
    if (sample_mode < 0) return 0;
    if (filter_b > kFilter1B && min_len >= kSampleQ + kSampleS - 1) return kSampleQ;
    if (sample_mode > 0 && filter_b == kFilter1B && min_len >= kSampleQSmem + kSampleS - 1) return kSampleQSmem;
    return 0;
}

// Allocator whose construction without a value leaves the element uninitialised: the
// builder sizes its largest arrays with resize() and then writes every element from
// several threads, instead of zero-filling gigabytes on one thread first.
template <typename T>
struct NoInitAllocator : std::allocator<T> {
    template <typename U> struct rebind { using other = NoInitAllocator<U>; };
    NoInitAllocator() = default;
    template <typename U> NoInitAllocator(const NoInitAllocator<U> &) noexcept {}
    template <typename U> void construct(U *p) noexcept { ::new ((void *)p) U; }
    template <typename U, typename... A> void construct(U *p, A &&...a) { ::new ((void *)p) U(std::forward<A>(a)...); }
};
template <typename T> using TableVector = std::vector<T, NoInitAllocator<T>>;

struct HostTables {
    int64_t n_states = 0;
    int32_t n_patterns = 0;
    int32_t max_len = 0;
    int32_t min_len = 0;
    int64_t n_duplicates = 0;
    TableVector<int32_t> rows;       // 4 * n_states: child | (terminal(child) << 31), 0 = none
    TableVector<int32_t> out_id;     // n_states: pattern id ending at the state, 0 = none
    std::vector<int64_t> level;      // max_len + 2: states of depth d in [level[d], level[d+1])
    TableVector<uint32_t> skip;      // 4 * n_states (empty when the trie has 2^27 states or more)
    int32_t filter_b = 0;            // 0 = no prefix filter
    std::vector<uint32_t> filter;    // 4^b bits
    int32_t rank_wide = 0;           // 32-bit rank entries
    std::vector<uint16_t> rank16;    // one per filter word
    std::vector<uint32_t> rank32;
    std::vector<uint32_t> dense;     // 4 per set filter bit
    // Filter of order kFilter1B derived from the main one when that is of a higher
    // order (too large for shared memory): bit w10 is the OR of the main bits of every
    // b-mer whose first kFilter1B bases are w10, i.e. the order-kFilter1B filter itself.
    int32_t filter1_b = 0;
    std::vector<uint32_t> filter1;
    int32_t sample_q = 0, sample_s = 0;   // 0 = no sampled screen
    std::vector<uint32_t> sample;         // 4^sample_q bits
};

// Status codes match pfac.h.
int build_host_tables(const char *const *patterns, const int32_t *lengths, int32_t n,
                      int32_t filter_b_opt, HostTables *out, int32_t sample_mode = 0);

}  // namespace pfac

// ---------------------------------------------------------------------------
// Device-side view of a table and the launchers (pfac_kernels.cu).
// ---------------------------------------------------------------------------
#include <cuda_runtime.h>

struct pfac_table;

namespace pfac {

struct DeviceTable {
    const int32_t *rows;       // 4 * n_states
    const int32_t *out_id;     // n_states
    const uint4 *skip;         // n_states skip entries, or nullptr
    const uint32_t *filter;    // 4^filter_b bits, or nullptr
    const uint32_t *filter1;   // first-level filter of order filter1_b, or nullptr
    const void *rank;          // one entry per filter word (uint16 or uint32)
    const uint4 *dense;        // one skip entry per set filter bit
    int64_t n_states;
    int32_t max_len;
    int32_t min_len;           // shortest pattern
    int32_t filter_b;          // 0 = no prefix filter
    int32_t filter1_b;         // 0 = no first-level filter
    int32_t rank_wide;
    int32_t *status;           // device status word (PFAC_OK or the first error)
    const uint32_t *sample;    // sampled screen (4^sample_q bits), or nullptr
    int32_t sample_q, sample_s;
};

struct TiledConfig {
    int32_t threads;           // threads per CTA: one producer warp + consumer warps
    int32_t ctas_per_sm;
    int32_t stages;            // text stages in the shared-memory ring (0 = default)
    int32_t walk_loads;        // dependent table loads a walk may take in kernel 2 (0 = default 2)
    int32_t lane_offsets;      // offsets per consumer lane: 16 (default) or 32
    int32_t smem_table_bytes;  // < 0: keep the rank index in global memory
    int32_t l2_persist;        // > 0: access-policy window over the skip entries
    int32_t screen;            // main filter in global memory, packed text: 0 = automatic
                               // (the sampled screen when the table has one, else the
                               // first-level filter), 1 = first-level filter, 2 = sampled
                               // screen (when available)
    int32_t zero_writer;       // dense packed scans, 32 offsets per lane: 0 = consumer warps
                               // store their zeros, 1 = a writer warp with 16-byte stores,
                               // 2 = a writer warp with TMA bulk stores of a zero tile,
                               // 3 = consumer warps with TMA bulk stores of a zero tile
    int64_t timeout_ns;        // limit of every bounded wait
};

// Global scratch for walks deferred to the tail kernel.
struct DeferScratch {
    void *items;                 // cap items of defer_item_bytes() each
    int64_t cap;
    unsigned long long *count;   // reset by every launch
};

size_t defer_item_bytes();
constexpr size_t kDeferItemBytes = 24;   // sizeof the kernel's deferred-walk record

struct DeviceProps {
    int device;
    int num_sms;
    int smem_optin;            // max dynamic shared memory per block
    int smem_per_sm;
    int l2_bytes;
    int persist_l2_max;
};

int get_device_props(DeviceProps *p);

int launch_pack(const uint8_t *text, int64_t len, uint32_t *packed, int32_t *status,
                int64_t *bad, cudaStream_t st, const DeviceProps &dp);

// Kernel 1 with either a dense output (c_off == nullptr) or a compacted match list;
// all_matches: the list holds every pattern that ends on each walk, not only the longest.
int launch_walk_rows_any(const DeviceTable &t, const void *text, bool packed, int64_t n,
                         int32_t *out, int64_t *c_off, int32_t *c_ids, int64_t cap,
                         unsigned long long *count, cudaStream_t st, const DeviceProps &dp,
                         bool all_matches = false);

// The paper's transition-table layouts (Section V-B: the kernel reads the arrays
// nextState and matchedPatternId with a pitch of four; Section VII: "array merge"
// interleaves them), derived on the device from the 16-byte rows:
//   next[4s + c] = the state reached from s on base c (0 = no edge)
//   pid[4s + c]  = the id of the pattern that ends on that state (0 = none)
//   pair[4s + c] = (next[4s + c], pid[4s + c]) in one 8-byte element
struct PaperTables {
    const int32_t *next;
    const int32_t *pid;
    const int2 *pair;
};

// Launch options of the one-thread-per-offset kernel (the paper's kernel structure):
//   layout    0 = 16-byte rows with the terminal flag, ids by state; 1 = two arrays;
//             2 = merged pairs
//   loads     0 = read-only data path (ld.global.nc, the texture path); 1 = default
//             global loads (ld.global.ca, cached in L1); 2 = L1 bypassed (ld.global.cg)
//   text_smem 1 = each block stages its text (its 256 offsets plus max_len - 1 bases)
//             in shared memory and walks from there
struct PaperConfig {
    int32_t layout;
    int32_t loads;
    int32_t text_smem;
};

// Dense ids with the kernel above. PFAC_ERR_UNSUPPORTED when the layout's arrays are
// missing or the shared-memory tile would exceed 48 KB.
int launch_paper_walk(const DeviceTable &t, const PaperTables &pt, const PaperConfig &pc, const void *text,
                      bool packed, int64_t n, int32_t *out, cudaStream_t st, const DeviceProps &dp);

// Fill the two-array layout (next, pid: 4 * n_states each) and/or the merged layout
// (pair: 4 * n_states) from the rows and ids of `t`; either output may be null.
int derive_paper_tables(const DeviceTable &t, int32_t *next, int32_t *pid, int2 *pair, cudaStream_t st);

// Kernel 2 (and its tail kernel). Dense output when c_off == nullptr, otherwise the
// compacted match list.
int launch_tiled(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out,
                 int64_t *c_off, int32_t *c_ids, int64_t cap, unsigned long long *count,
                 const TiledConfig &cfg, const DeferScratch &scratch, cudaStream_t st,
                 const DeviceProps &dp, bool all_matches = false);

// Launch shape of the batched scan: offsets per lane (16 or 32; a work item is 32 x that),
// 256-thread blocks per SM of the persistent scan kernel (1..8), dependent table loads a
// walk may take before it is deferred (0 = 2).
struct BatchConfig {
    int32_t lane_offsets;
    int32_t blocks_per_sm;
    int32_t walk_loads;
};

// Batched scan: scratch bytes for n bases, n_reads reads and defer_cap deferred walks,
// and the launch (pack, plan, scan and tail kernels on `st`). d_sets: device array of
// n_sets table descriptors.
int64_t batch_scratch_bytes(int64_t n, int32_t n_reads, int64_t defer_cap);
int launch_batched(const DeviceTable *d_sets, int32_t n_sets, const uint8_t *texts, int64_t n,
                   const int64_t *read_off, const int32_t *read_set, int32_t n_reads, int32_t *out,
                   void *scratch, int64_t defer_cap, const BatchConfig &bc, cudaStream_t st,
                   const DeviceProps &dp);

// Shared memory kernel 2 would use for a configuration (bytes), -1 if it cannot run.
int64_t tiled_smem_bytes(const DeviceTable &t, const TiledConfig &cfg, bool packed, const DeviceProps &dp);

// A kernel whose only job is a bounded wait on an mbarrier that nothing completes:
// it must give up after limit_ns and record PFAC_ERR_TIMEOUT in *status.
int launch_timeout_probe(int32_t *status, int64_t limit_ns, cudaStream_t st);

// pfac_match_packed with caller-provided deferred-walk scratch (used by the
// allocation-free entry point in pfac_noalloc.cu). Returns a PFAC_* status.
int scan_packed_with_scratch(struct ::pfac_table *h, const uint32_t *d_packed, int64_t n_bases,
                             int32_t *d_out_ids, const DeferScratch &scratch, cudaStream_t st);

// Table construction on the device (pfac_gpubuild.cu): the tables of build_host_tables
// for the same patterns, in one device allocation laid out as pfac_build_ex lays out its
// upload. Synchronous on `st`.
struct DeviceBuild {
    DeviceTable dt{};
    void *mem = nullptr;
    size_t bytes = 0;
    std::vector<int64_t> level;
    int64_t n_duplicates = 0, filter_set = 0, skip_bytes = 0;
};
int build_device_tables(const uint8_t *d_blob, const int64_t *d_off, int32_t n, int32_t filter_b_opt,
                        int32_t sample_mode, cudaStream_t st, const DeviceProps &dp, DeviceBuild *out);

// Record a status (or a CUDA error) as this thread's last error; returns the status.
int set_last_error(int code);
int set_last_cuda_error(cudaError_t e);

}  // namespace pfac
