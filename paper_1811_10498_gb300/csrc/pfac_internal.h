// Internal declarations shared by the host trie builder, the runtime and the kernels.
#pragma once

#include <stdint.h>

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

// Jump table of order k: one entry per k-mer w (base j of w in bits 2j..2j+1), the
// index of the state the first k bases lead to inside the "level-k window", an array
// of node words that starts with two sentinels and continues with every state of
// depth k, in breadth-first order:
//   0             the walk over w ends before depth k and no pattern ends on the way
//                 (answer 0); window slot 0 is a node with no edges;
//   1             special: a pattern ends within the first k bases (the answer, or a
//                 prefix of it, comes from the prefix), so the walk is redone from the
//                 root; window slot 1 is a node with all four edges, so the next step
//                 always "continues" and sends the offset to that slower path;
//   2 + i         the i-th state of depth k (breadth-first id level[k] + i); no pattern
//                 ends within the first k bases.
// Entries are 16-bit when depth k has at most 65533 states, else 32-bit.
//
// Prefix filter of order b: one bit per b-mer w. The bit is 0 when the walk over w ends
// before depth b and no pattern ends on the way, so that the answer at any offset
// where w starts is 0 whatever follows; it is 1 otherwise (the walk is still going at
// depth b, or a pattern ends within w). Bit w is bit (w mod 32) of word w / 32.
constexpr int kMaxJumpK = 12;
constexpr int kMaxFilterB = 12;
constexpr uint32_t kJumpDead = 0;
constexpr uint32_t kJumpSpecial = 1;
constexpr uint32_t kJumpFirst = 2;
constexpr int64_t kJump16MaxLevel = 65533;

struct HostTables {
    int64_t n_states = 0;
    int32_t n_patterns = 0;
    int32_t max_len = 0;
    int32_t min_len = 0;
    int64_t n_duplicates = 0;
    std::vector<int32_t> rows;       // 4 * n_states: child | (terminal(child) << 31), 0 = none
    std::vector<int32_t> out_id;     // n_states: pattern id ending at the state, 0 = none
    std::vector<uint32_t> nodes;     // n_states compact node words (empty if too many states)
    std::vector<int64_t> level;      // max_len + 2: states of depth d in [level[d], level[d+1])
    int32_t jump_k = 0;              // 0 = no jump table
    int32_t jump_wide = 0;           // 1: 32-bit entries (jump32), 0: 16-bit (jump16)
    std::vector<uint16_t> jump16;    // 4^k entries
    std::vector<uint32_t> jump32;    // 4^k entries
    int32_t filter_b = 0;            // 0 = no prefix filter
    std::vector<uint32_t> filter;    // 4^b bits
};

// Status codes match pfac.h.
int build_host_tables(const char *const *patterns, const int32_t *lengths, int32_t n,
                      int32_t jump_k_opt, int32_t filter_b_opt, HostTables *out);

// Order of the jump table chosen when the caller leaves it to the library, from the
// number of states per depth level.
int32_t auto_jump_k(const std::vector<int64_t> &level, int32_t max_len);

}  // namespace pfac

// ---------------------------------------------------------------------------
// Device-side view of a table and the launchers (pfac_kernels.cu).
// ---------------------------------------------------------------------------
#include <cuda_runtime.h>

namespace pfac {

struct DeviceTable {
    const int32_t *rows;       // 4 * n_states
    const uint32_t *nodes;     // n_states compact node words, or nullptr
    const int32_t *out_id;     // n_states
    const void *jump;          // 4^jump_k entries (uint16 or uint32), or nullptr
    int64_t n_states;
    int32_t max_len;
    int32_t jump_k;            // 0 = no jump table
    int32_t jump_wide;         // 32-bit jump entries
    const uint32_t *filter;    // 4^filter_b bits, or nullptr
    int32_t filter_b;          // 0 = no prefix filter
    int64_t level_k;           // first state of depth jump_k (window slot kJumpFirst)
    int64_t level_k1;          // first state of depth jump_k + 1
    int32_t *status;           // device status word (PFAC_OK or the first error)
};

struct TiledConfig {
    int32_t threads;           // threads per CTA: one producer warp + consumer warps
    int32_t ctas_per_sm;
    int32_t stages;            // text stages in the shared-memory ring (0 = default)
    int32_t step_cap;          // steps past the jump depth before a walk is deferred (0 = default)
    int32_t smem_table_bytes;  // shared-memory budget for the node window (< 0: none, 0: all)
    int32_t l2_persist;        // > 0: access-policy window over the nodes after the smem window
    int64_t timeout_ns;        // limit of every bounded wait
};

// Global scratch for walks deferred to the tail kernel.
struct DeferScratch {
    void *items;                 // cap items of defer_item_bytes() each
    int64_t cap;
    unsigned long long *count;   // reset by every launch
};

size_t defer_item_bytes();

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

int launch_walk_rows(const DeviceTable &t, const void *text, bool packed, int64_t n,
                     int32_t *out, cudaStream_t st, const DeviceProps &dp);

// Kernel 1 with either a dense output (c_off == nullptr) or a compacted match list.
int launch_walk_rows_any(const DeviceTable &t, const void *text, bool packed, int64_t n,
                         int32_t *out, int64_t *c_off, int32_t *c_ids, int64_t cap,
                         unsigned long long *count, cudaStream_t st, const DeviceProps &dp);

// Dense output when c_off == nullptr, otherwise the compacted match list.
int launch_tiled(const DeviceTable &t, const void *text, bool packed, int64_t n, int32_t *out,
                 int64_t *c_off, int32_t *c_ids, int64_t cap, unsigned long long *count,
                 const TiledConfig &cfg, const DeferScratch &scratch, cudaStream_t st,
                 const DeviceProps &dp);

// Shared memory the tiled kernel needs for a configuration (bytes), and the window
// of nodes it would hold.
int64_t tiled_smem_bytes(const DeviceTable &t, const TiledConfig &cfg, bool packed,
                         int32_t *win_len, int32_t *jump_smem, const DeviceProps &dp);

// A kernel whose only job is a bounded wait on an mbarrier that nothing completes:
// it must give up after limit_ns and record PFAC_ERR_TIMEOUT in *status.
int launch_timeout_probe(int32_t *status, int64_t limit_ns, cudaStream_t st);

}  // namespace pfac
