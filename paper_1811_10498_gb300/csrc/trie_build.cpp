// Host-side construction of the PFAC goto table.
//
// Step 1 (Section V-A, the insertion procedure after Table I): patterns are inserted
// one by one into a 4-column table; from state 0, each symbol either follows the
// existing edge or creates the next free state. The state of a pattern's last symbol
// is terminal and carries the pattern's id (the paper writes it into the cell; here
// it is kept per state, and the first id given for a string is kept).
//
// Step 2 (the breadth-first state rearrangement cited in Section II): states are
// renumbered breadth-first, children visited in A, C, G, T order, so each depth level
// is a contiguous range of ids and the children of one state are consecutive. The
// shallow levels that every walk visits become a short prefix of the table.
//
// Step 3: the table is encoded for the device (see pfac_internal.h): 16-byte rows
// (4 x int32, one per base, bit 31 = target is terminal, the paper's 4-column layout),
// per-state skip entries that compress chains of single-child edges (up to 16 bases
// compared at once), and a prefix filter over b-mers with a rank index into skip
// entries for the states of depth b. All of them describe the same trie exactly.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace pfac {

namespace {

inline int base_code(unsigned char b)
{
    switch (b) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

constexpr int64_t kMaxStates = int64_t(0x7FFFFFFF);

// A skip label is kSkipMaxLen two-bit symbols, low symbol first, in one 32-bit word.
static_assert(kSkipMaxLen == 16, "skip labels fill exactly one 32-bit word");

}  // namespace

int build_host_tables(const char *const *patterns, const int32_t *lengths, int32_t n,
                      int32_t filter_b_opt, HostTables *out)
{
    if (n <= 0 || !patterns || !lengths || !out) return PFAC_ERR_INVALID_ARG;
    if (filter_b_opt > kMaxFilterB) return PFAC_ERR_INVALID_ARG;
    try {
        // ---- validate ----------------------------------------------------------
        int64_t total = 0;
        int32_t max_len = 0, min_len = INT32_MAX;
        for (int32_t j = 0; j < n; j++) {
            if (lengths[j] <= 0) return lengths[j] == 0 ? PFAC_ERR_EMPTY_PATTERN : PFAC_ERR_INVALID_ARG;
            if (!patterns[j]) return PFAC_ERR_INVALID_ARG;
            const unsigned char *p = (const unsigned char *)patterns[j];
            for (int32_t k = 0; k < lengths[j]; k++)
                if (base_code(p[k]) < 0) return PFAC_ERR_BAD_SYMBOL;
            total += lengths[j];
            max_len = std::max(max_len, lengths[j]);
            min_len = std::min(min_len, lengths[j]);
        }

        // ---- step 1: insertion-order trie --------------------------------------
        std::vector<int32_t> go;      // 4 per state, 0 = no edge
        std::vector<int32_t> term;    // pattern id per state
        int64_t cap = std::min<int64_t>(total + 1, kMaxStates);
        go.reserve((size_t)std::min<int64_t>(cap, 1 << 24) * 4);
        go.assign(4, 0);
        term.assign(1, 0);
        int64_t n_states = 1;
        int64_t dups = 0;
        for (int32_t j = 0; j < n; j++) {
            const unsigned char *p = (const unsigned char *)patterns[j];
            int64_t s = 0;
            for (int32_t k = 0; k < lengths[j]; k++) {
                int c = base_code(p[k]);
                int32_t nxt = go[(size_t)(4 * s + c)];
                if (nxt == 0) {
                    if (n_states >= kMaxStates) return PFAC_ERR_TOO_MANY_STATES;
                    nxt = (int32_t)n_states++;
                    go[(size_t)(4 * s + c)] = nxt;
                    go.insert(go.end(), 4, 0);
                    term.push_back(0);
                }
                s = nxt;
            }
            if (term[(size_t)s] == 0) term[(size_t)s] = j + 1;
            else dups++;
        }

        // ---- steps 2 and 3a: breadth-first renumbering, rows and pattern ids -----
        // The queue holds old ids in their new order; the children of the state at
        // `head` take the next new ids, so its row is written as soon as it is visited.
        HostTables &T = *out;
        T = HostTables();
        T.n_states = n_states;
        T.n_patterns = n;
        T.max_len = max_len;
        T.min_len = min_len;
        T.n_duplicates = dups;
        T.rows.assign((size_t)n_states * 4, 0);
        T.out_id.assign((size_t)n_states, 0);
        T.level.assign((size_t)max_len + 2, n_states);
        std::vector<int32_t> order((size_t)n_states);    // new id -> old id
        std::vector<int32_t> parent((size_t)n_states);   // new id -> new id of its parent
        {
            int64_t head = 0, tail = 1, depth_end = 1;
            int32_t depth = 0;
            order[0] = 0;
            parent[0] = 0;
            T.out_id[0] = term[0];
            T.level[0] = 0;
            constexpr int64_t kAhead = 16;   // queue entries whose rows are fetched early
            while (head < tail) {
                if (head == depth_end) {     // every state of `depth` has been visited
                    T.level[(size_t)++depth] = head;
                    depth_end = tail;
                }
                if (head + kAhead < tail) __builtin_prefetch(&go[(size_t)(4 * (int64_t)order[(size_t)(head + kAhead)])]);
                const int32_t *g = &go[(size_t)(4 * (int64_t)order[(size_t)head])];
                for (int c = 0; c < 4; c++) {
                    const int32_t ch = g[c];
                    if (!ch) continue;
                    uint32_t e = (uint32_t)tail;
                    if (term[(size_t)ch]) e |= 0x80000000u;
                    T.rows[(size_t)(4 * head + c)] = (int32_t)e;
                    T.out_id[(size_t)tail] = term[(size_t)ch];
                    parent[(size_t)tail] = (int32_t)head;
                    order[(size_t)tail++] = ch;
                }
                head++;
            }
        }
        for (int d = max_len; d >= 0; d--) T.level[(size_t)d] = std::min(T.level[(size_t)d], T.level[(size_t)d + 1]);
        std::vector<int32_t>().swap(go);
        std::vector<int32_t>().swap(term);
        std::vector<int32_t>().swap(order);

        // ---- step 3b: skip entries ----------------------------------------------
        // From the deepest state up, so a child's entry is final before its parent's.
        // A single-child state s with child ch (edge symbol c) stops at ch when ch is
        // terminal or has other than one child; otherwise its chain is c followed by
        // ch's chain, cut at kSkipMaxLen symbols: a chain of ch that already has
        // kSkipMaxLen symbols loses its last one, so s stops at the parent of ch's
        // target, which lies strictly inside ch's chain and so is not terminal.
        if (n_states < kMaxNodeStates) {
            T.skip.assign((size_t)n_states * 4, 0u);
            for (int64_t s = n_states - 1; s >= 0; s--) {
                uint32_t mask = 0, first = 0;
                int onlyc = 0;
                for (int c = 3; c >= 0; c--) {
                    const uint32_t e = (uint32_t)T.rows[(size_t)(4 * s + c)];
                    if (e) { mask |= 1u << c; first = e & 0x7FFFFFFFu; onlyc = c; }
                }
                uint32_t node = mask | (first << kNodeFirstShift);
                if (T.out_id[(size_t)s]) node |= kNodeTermBit;
                uint32_t label = 0, len = 0, target = 0, target_term = 0;
                if (__builtin_popcount(mask) == 1) {
                    const uint32_t *ce = &T.skip[(size_t)(4 * (int64_t)first)];
                    const uint32_t child_node = ce[3];
                    if ((child_node & kNodeTermBit) || __builtin_popcount(child_node & kNodeMaskBits) != 1) {
                        label = (uint32_t)onlyc;
                        len = 1;
                        target = first;
                        target_term = child_node & kNodeTermBit ? kSkipTargetTerm : 0u;
                    } else {
                        const uint32_t child_len = ce[1] & kSkipLenMask;
                        label = (uint32_t)onlyc | (ce[0] << 2);   // a 17th symbol falls off the top
                        if (child_len < (uint32_t)kSkipMaxLen) {
                            len = child_len + 1;
                            target = ce[2];
                            target_term = ce[1] & kSkipTargetTerm;
                        } else {
                            len = kSkipMaxLen;
                            target = (uint32_t)parent[(size_t)ce[2]];
                        }
                    }
                }
                uint32_t *e = &T.skip[(size_t)(4 * s)];
                e[0] = label;
                e[1] = len | target_term | (T.out_id[(size_t)s] ? kSkipSelfTerm : 0u);
                e[2] = target;
                e[3] = node;
            }
        }
        std::vector<int32_t>().swap(parent);

        // ---- step 3c: prefix filter, rank index, dense entries ------------------------
        // Depth-first over the trie down to depth b. A b-mer's bit is set when its walk
        // is still going at depth b (its dense entry is that state's skip entry), or when
        // a pattern ends on the walk before it stops (special entry). A prefix of d
        // symbols whose walk stops at symbol d fixes every b-mer that starts with it: the
        // indices congruent to the prefix code modulo 4^(d+1).
        // Automatic order: about log4(patterns) + 2.2, so that a few percent of the
        // b-mers of a random text pass (a b-mer passes when it is a path of the trie,
        // about min(1, patterns / 4^b) of them), between 6 and 12.
        const double auto_b = std::ceil(std::log((double)n) / std::log(4.0) + 2.2);
        const int32_t b = filter_b_opt == 0 ? (int32_t)std::min(12.0, std::max(6.0, auto_b))
                                            : (filter_b_opt < 0 ? 0 : filter_b_opt);
        if (b > 0 && !T.skip.empty()) {
            T.filter_b = b;
            const size_t E = (size_t)1 << (2 * b);
            const uint32_t kNone = 0xFFFFFFFFu, kSpecialVal = 0xFFFFFFFEu;
            std::vector<uint32_t> val(E, kNone);      // state reached at depth b, or special
            struct Frame { int32_t s; int32_t d; uint32_t code; bool term; };
            std::vector<Frame> stack;
            stack.push_back({0, 0, 0u, false});
            while (!stack.empty()) {
                Frame f = stack.back();
                stack.pop_back();
                if (f.d == b) {
                    val[f.code] = f.term ? kSpecialVal : (uint32_t)f.s;
                    continue;
                }
                for (int c = 0; c < 4; c++) {
                    const uint32_t code = f.code | ((uint32_t)c << (2 * f.d));
                    const uint32_t e = (uint32_t)T.rows[(size_t)(4 * (int64_t)f.s + c)];
                    if (e) {
                        stack.push_back({(int32_t)(e & 0x7FFFFFFFu), f.d + 1, code, f.term || (e & 0x80000000u)});
                    } else if (f.term) {
                        const size_t stride = (size_t)1 << (2 * (f.d + 1));
                        for (size_t idx = code; idx < E; idx += stride) val[idx] = kSpecialVal;
                    }
                }
            }
            const size_t words = E >= 32 ? E / 32 : 1;
            T.filter.assign(words, 0u);
            std::vector<uint32_t> rank(words, 0u);
            uint64_t count = 0;
            for (size_t w = 0; w < words; w++) {
                rank[w] = (uint32_t)count;
                for (size_t i = 0; i < 32 && w * 32 + i < E; i++) {
                    const uint32_t v = val[w * 32 + i];
                    if (v == kNone) continue;
                    T.filter[w] |= 1u << i;
                    count++;
                    if (v == kSpecialVal) {
                        T.dense.insert(T.dense.end(), {0u, kSkipSpecial, 0u, 0u});
                    } else {
                        const uint32_t *e = &T.skip[(size_t)(4 * (int64_t)v)];
                        T.dense.insert(T.dense.end(), {e[0], e[1], e[2], e[3]});
                    }
                }
            }
            T.rank_wide = count > 65535;
            if (T.rank_wide) T.rank32.swap(rank);
            else T.rank16.assign(rank.begin(), rank.end());
            // A main filter above order kFilter1B gets a first-level filter of that order:
            // a b-mer whose first kFilter1B bases have a clear bit there has a clear bit
            // in the main filter too, so the first level screens offsets in shared memory
            // before the main filter is read from global memory.
            if (b > kFilter1B) {
                const size_t E1 = (size_t)1 << (2 * kFilter1B);
                T.filter1_b = kFilter1B;
                T.filter1.assign(E1 / 32, 0u);
                for (size_t w = 0; w < E; w++)
                    if ((T.filter[w >> 5] >> (w & 31)) & 1u) {
                        const size_t w1 = w & (E1 - 1);   // the first kFilter1B bases
                        T.filter1[w1 >> 5] |= 1u << (w1 & 31);
                    }
            }
        }
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return PFAC_ERR_OOM;
    }
}

}  // namespace pfac
