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
// Steps 1 and 2 run on several host threads. The patterns are split by their first
// three bases; below each such prefix, a sub-trie is built by the insertion procedure
// (patterns in input order) and numbered by its own breadth-first order. Breadth-first
// order lists each depth's states by their strings in lexicographic order, so the ids
// of one depth are the sub-tries' states of that depth, sub-trie after sub-trie in
// prefix order: per-depth counts give every sub-trie's id ranges. The trie and its
// numbering are the ones the single insertion-order trie gives; only the work is split.
//
// Step 3: the table is encoded for the device (see pfac_internal.h): 16-byte rows
// (4 x int32, one per base, bit 31 = target is terminal, the paper's 4-column layout),
// per-state skip entries that compress chains of single-child edges (up to 16 bases
// compared at once), and a prefix filter over b-mers with a rank index into skip
// entries for the states of depth b. All of them describe the same trie exactly.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <system_error>
#include <thread>
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

// Patterns are split by their first kTopDepth bases: the states of depth kTopDepth and
// more below one such prefix form a sub-trie, and the sub-tries are built side by side.
constexpr int kTopDepth = 3;
constexpr int kSubTries = 1 << (2 * kTopDepth);
constexpr int kMaxThreads = 16;
constexpr int64_t kBasesPerThread = int64_t(1) << 20;   // below this, one thread
constexpr int64_t kAhead = 16;                          // queue entries whose rows are fetched early

// The states of depth >= kTopDepth under one prefix of kTopDepth bases, numbered by
// their own breadth-first order (position 0 = the state of the prefix itself).
struct SubTrie {
    std::vector<int32_t> pats;     // pattern indices, in input order
    std::vector<int32_t> rows;     // 4 per position: child position | terminal bit, 0 = none
    std::vector<int32_t> out;      // pattern id per position (0 = not terminal)
    std::vector<int32_t> parent;   // parent position per position
    std::vector<int64_t> start;    // first position of each depth below the prefix, then the size
    std::vector<int64_t> base;     // global id of the first state of each of those depths
    int64_t dups = 0;
};

// Steps 1 and 2 inside one sub-trie: insertion in input order, then breadth-first
// positions. The queue holds insertion ids in breadth-first order; the children of the
// state at `head` take the next positions, so its row is written when it is visited.
int build_subtrie(SubTrie &B, const char *const *patterns, const int32_t *lengths)
{
    std::vector<int32_t> go(4, 0);     // 4 per state in insertion order, 0 = no edge
    std::vector<int32_t> term(1, 0);   // pattern id per state
    int64_t ns = 1;
    for (const int32_t j : B.pats) {
        const unsigned char *p = (const unsigned char *)patterns[j];
        int64_t s = 0;
        for (int32_t k = kTopDepth; k < lengths[j]; k++) {
            const int c = base_code(p[k]);
            int32_t nxt = go[(size_t)(4 * s + c)];
            if (nxt == 0) {
                if (ns >= kMaxStates) return PFAC_ERR_TOO_MANY_STATES;
                nxt = (int32_t)ns++;
                go[(size_t)(4 * s + c)] = nxt;
                go.insert(go.end(), 4, 0);
                term.push_back(0);
            }
            s = nxt;
        }
        if (term[(size_t)s] == 0) term[(size_t)s] = j + 1;
        else B.dups++;
    }
    B.rows.assign((size_t)ns * 4, 0);
    B.out.assign((size_t)ns, 0);
    B.parent.assign((size_t)ns, 0);
    std::vector<int32_t> order((size_t)ns);
    order[0] = 0;
    B.out[0] = term[0];
    B.start.assign(1, 0);
    int64_t head = 0, tail = 1, depth_end = 1;
    while (head < tail) {
        if (head == depth_end) {       // every state of the depth above has been visited
            B.start.push_back(head);
            depth_end = tail;
        }
        if (head + kAhead < tail) __builtin_prefetch(&go[(size_t)(4 * (int64_t)order[(size_t)(head + kAhead)])]);
        const int32_t *g = &go[(size_t)(4 * (int64_t)order[(size_t)head])];
        for (int c = 0; c < 4; c++) {
            const int32_t ch = g[c];
            if (!ch) continue;
            uint32_t e = (uint32_t)tail;
            if (term[(size_t)ch]) e |= 0x80000000u;
            B.rows[(size_t)(4 * head + c)] = (int32_t)e;
            B.out[(size_t)tail] = term[(size_t)ch];
            B.parent[(size_t)tail] = (int32_t)head;
            order[(size_t)tail++] = ch;
        }
        head++;
    }
    B.start.push_back(ns);
    return PFAC_OK;
}

// Runs fn(i) for every i in [0, count) on up to `threads` threads, the caller's one
// included, and returns the first status other than PFAC_OK that a call gave (the
// remaining calls are then skipped).
template <typename Fn>
int run_parallel(size_t count, int threads, Fn fn)
{
    std::atomic<size_t> next{0};
    std::atomic<int> status{PFAC_OK};
    auto work = [&]() {
        for (;;) {
            if (status.load() != PFAC_OK) return;
            const size_t i = next.fetch_add(1);
            if (i >= count) return;
            int st;
            try {
                st = fn(i);
            } catch (const std::bad_alloc &) {
                st = PFAC_ERR_OOM;
            }
            if (st != PFAC_OK) {
                int ok = PFAC_OK;
                status.compare_exchange_strong(ok, st);
            }
        }
    };
    std::vector<std::thread> pool;
    pool.reserve((size_t)std::max(threads, 1));
    for (int t = 1; t < threads && (size_t)t < count; t++) {
        try {
            pool.emplace_back(work);
        } catch (const std::system_error &) {
            break;                      // fewer threads: the others take the work
        }
    }
    work();
    for (auto &th : pool) th.join();
    return status.load();
}

}  // namespace

int build_host_tables(const char *const *patterns, const int32_t *lengths, int32_t n,
                      int32_t filter_b_opt, HostTables *out, int32_t sample_mode)
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

        // ---- step 1: the shallow states, then the sub-tries side by side -------------
        // A prefix of d < kTopDepth bases is a state when some pattern starts with it;
        // prefix codes put the first base in the most significant bits.
        std::vector<std::vector<uint8_t>> top_on(kTopDepth);
        std::vector<std::vector<int32_t>> top_term(kTopDepth), top_id(kTopDepth);
        for (int d = 0; d < kTopDepth; d++) {
            top_on[d].assign((size_t)1 << (2 * d), 0);
            top_term[d].assign((size_t)1 << (2 * d), 0);
        }
        top_on[0][0] = 1;
        std::vector<SubTrie> sub(kSubTries);
        int64_t dups = 0;
        for (int32_t j = 0; j < n; j++) {
            const unsigned char *p = (const unsigned char *)patterns[j];
            const int dmax = std::min(lengths[j], (int32_t)kTopDepth);
            uint32_t code = 0;
            for (int d = 1; d <= dmax; d++) {
                code = code * 4 + (uint32_t)base_code(p[d - 1]);
                if (d < kTopDepth) top_on[(size_t)d][code] = 1;
            }
            if (lengths[j] >= kTopDepth) sub[code].pats.push_back(j);
            else if (top_term[(size_t)lengths[j]][code] == 0) top_term[(size_t)lengths[j]][code] = j + 1;
            else dups++;
        }
        std::vector<int32_t> used;        // sub-tries that have patterns, most patterns first
        for (int t = 0; t < kSubTries; t++)
            if (!sub[(size_t)t].pats.empty()) used.push_back(t);
        std::stable_sort(used.begin(), used.end(),
                         [&](int32_t x, int32_t y) { return sub[(size_t)x].pats.size() > sub[(size_t)y].pats.size(); });
        const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
        const int threads = (int)std::max<int64_t>(
            1, std::min({hw, (int64_t)kMaxThreads, (int64_t)used.size(), total / kBasesPerThread}));
        int st = run_parallel(used.size(), threads, [&](size_t i) {
            return build_subtrie(sub[(size_t)used[i]], patterns, lengths);
        });
        if (st != PFAC_OK) return st;
        for (int32_t t : used) dups += sub[(size_t)t].dups;

        // ---- step 2: breadth-first numbering ---------------------------------------
        // Breadth-first order with children in A, C, G, T order lists the states of one
        // depth by their strings in lexicographic order. So a depth below kTopDepth is
        // its prefixes in code order, and a deeper one is the sub-tries in prefix-code
        // order, each with its own states of that depth in its own breadth-first order.
        const int depths = std::max((int)max_len, kTopDepth) + 2;
        std::vector<int64_t> level((size_t)depths + 1, 0);
        for (int d = 0; d < kTopDepth; d++)
            for (uint8_t on : top_on[(size_t)d]) level[(size_t)d + 1] += on;
        for (int32_t t : used) {
            const SubTrie &B = sub[(size_t)t];
            for (size_t e = 0; e + 1 < B.start.size(); e++)
                level[(size_t)kTopDepth + e + 1] += B.start[e + 1] - B.start[e];
        }
        for (int d = 0; d < depths; d++) level[(size_t)d + 1] += level[(size_t)d];
        const int64_t n_states = level[(size_t)depths];
        if (n_states > kMaxStates) return PFAC_ERR_TOO_MANY_STATES;
        for (int d = 0; d < kTopDepth; d++) {
            top_id[(size_t)d].assign(top_on[(size_t)d].size(), 0);
            int64_t next = level[(size_t)d];
            for (size_t code = 0; code < top_on[(size_t)d].size(); code++)
                if (top_on[(size_t)d][code]) top_id[(size_t)d][code] = (int32_t)next++;
        }
        {
            std::vector<int64_t> next(level.begin() + kTopDepth, level.end());
            for (int t = 0; t < kSubTries; t++) {
                SubTrie &B = sub[(size_t)t];
                if (B.pats.empty()) continue;
                B.base.resize(B.start.size() - 1);
                for (size_t e = 0; e < B.base.size(); e++) {
                    B.base[e] = next[e];
                    next[e] += B.start[e + 1] - B.start[e];
                }
            }
        }

        HostTables &T = *out;
        T = HostTables();
        T.n_states = n_states;
        T.n_patterns = n;
        T.max_len = max_len;
        T.min_len = min_len;
        T.n_duplicates = dups;
        T.level.assign(level.begin(), level.begin() + max_len + 2);
        // Sized without a fill: the passes below write every element of these arrays.
        T.rows.resize((size_t)n_states * 4);
        T.out_id.resize((size_t)n_states);
        TableVector<int32_t> parent((size_t)n_states);      // id -> id of its parent
        const bool with_skip = n_states < kMaxNodeStates;
        if (with_skip) T.skip.resize((size_t)n_states * 4);

        // ---- step 3a: rows and pattern ids -------------------------------------------
        // Row entries: the child's id, bit 31 set when the child is terminal.
        for (int d = 0; d < kTopDepth; d++)
            for (size_t code = 0; code < top_on[(size_t)d].size(); code++) {
                if (!top_on[(size_t)d][code]) continue;
                const int64_t g = top_id[(size_t)d][code];
                T.out_id[(size_t)g] = top_term[(size_t)d][code];
                parent[(size_t)g] = d ? top_id[(size_t)d - 1][code >> 2] : 0;
                for (int c = 0; c < 4; c++) {
                    const size_t cc = code * 4 + (size_t)c;
                    uint32_t e = 0;
                    if (d + 1 < kTopDepth) {
                        if (top_on[(size_t)d + 1][cc])
                            e = (uint32_t)top_id[(size_t)d + 1][cc] | (top_term[(size_t)d + 1][cc] ? 0x80000000u : 0u);
                    } else if (!sub[cc].pats.empty()) {
                        e = (uint32_t)sub[cc].base[0] | (sub[cc].out[0] ? 0x80000000u : 0u);
                    }
                    T.rows[(size_t)(4 * g + c)] = (int32_t)e;
                }
            }

        // ---- step 3b: skip entries ----------------------------------------------
        // A single-child state s with child ch (edge symbol c) stops at ch when ch is
        // terminal or has other than one child; otherwise its chain is c followed by
        // ch's chain, cut at kSkipMaxLen symbols: a chain of ch that already has
        // kSkipMaxLen symbols loses its last one, so s stops at the parent of ch's
        // target, which lies strictly inside ch's chain and so is not terminal. A
        // child's entry is therefore made before its parent's.
        auto skip_entry = [&](int64_t s) {
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
        };

        // Steps 3a and 3b for the sub-tries, side by side: each one's positions map to
        // contiguous id ranges per depth, and its skip entries need only its own states.
        st = run_parallel(used.size(), threads, [&](size_t i) {
            SubTrie &B = sub[(size_t)used[i]];
            const size_t E = B.base.size();
            const int32_t up = top_id[kTopDepth - 1][(size_t)used[i] >> 2];   // parent of position 0
            for (size_t e = 0; e < E; e++)
                for (int64_t q = B.start[e]; q < B.start[e + 1]; q++) {
                    const int64_t g = B.base[e] + (q - B.start[e]);
                    T.out_id[(size_t)g] = B.out[(size_t)q];
                    parent[(size_t)g] = e ? (int32_t)(B.base[e - 1] + (B.parent[(size_t)q] - B.start[e - 1])) : up;
                    for (int c = 0; c < 4; c++) {
                        const uint32_t v = (uint32_t)B.rows[(size_t)(4 * q + c)];
                        uint32_t w = 0;
                        if (v) {
                            const int64_t child = B.base[e + 1] + ((int64_t)(v & 0x7FFFFFFFu) - B.start[e + 1]);
                            w = (uint32_t)child | (v & 0x80000000u);
                        }
                        T.rows[(size_t)(4 * g + c)] = (int32_t)w;
                    }
                }
            std::vector<int32_t>().swap(B.rows);
            std::vector<int32_t>().swap(B.out);
            std::vector<int32_t>().swap(B.parent);
            if (with_skip)
                for (size_t e = E; e-- > 0;)
                    for (int64_t g = B.base[e] + (B.start[e + 1] - B.start[e]) - 1; g >= B.base[e]; g--) skip_entry(g);
            return PFAC_OK;
        });
        if (st != PFAC_OK) return st;
        if (with_skip)
            for (int64_t s = level[kTopDepth] - 1; s >= 0; s--) skip_entry(s);
        std::vector<SubTrie>().swap(sub);
        TableVector<int32_t>().swap(parent);

        // ---- step 3c: prefix filter, rank index, dense entries ------------------------
        // Depth-first over the trie down to depth b. A b-mer's bit is set when its walk
        // is still going at depth b (its dense entry is that state's skip entry), or when
        // a pattern ends on the walk before it stops (special entry). A prefix of d
        // symbols whose walk stops at symbol d fixes every b-mer that starts with it: the
        // indices congruent to the prefix code modulo 4^(d+1).
        // Automatic order: about log4(patterns) + 2.2, so that a few percent of the
        // b-mers of a random text pass (a b-mer passes when it is a path of the trie,
        // about min(1, patterns / 4^b) of them), between 6 and 12.
        // Dictionaries of kDeepFilterMinPatterns patterns or more, none shorter than
        // kDeepFilterB, get the order-kDeepFilterB filter: too large for shared memory
        // either way, and the deeper the order, the fewer offsets start a walk.
        const double auto_b = std::ceil(std::log((double)n) / std::log(4.0) + 2.2);
        int32_t b = filter_b_opt == 0 ? (int32_t)std::min(12.0, std::max(6.0, auto_b))
                                      : (filter_b_opt < 0 ? 0 : filter_b_opt);
        if (filter_b_opt == 0 && n >= kDeepFilterMinPatterns && min_len >= kDeepFilterB) b = kDeepFilterB;
        if (b > 0 && !T.skip.empty() && min_len >= b) {
            // No pattern ends before depth b, so no bit stands for a range of b-mers: the
            // set bits are the codes of the states of depth b, one dense entry each (the
            // special entry for a state where a pattern ends).
            T.filter_b = b;
            const size_t E = (size_t)1 << (2 * b);
            const int64_t lo = T.level[(size_t)b], hi = T.level[(size_t)b + 1];
            std::vector<uint64_t> code((size_t)hi, 0);      // b-mer code << 32 | state
            for (int32_t d = 0; d < b; d++)
                for (int64_t st = T.level[(size_t)d]; st < T.level[(size_t)d + 1]; st++)
                    for (int c = 0; c < 4; c++) {
                        const uint32_t e = (uint32_t)T.rows[(size_t)(4 * st + c)];
                        if (e) code[e & 0x7FFFFFFFu] = code[(size_t)st] | ((uint64_t)c << (32 + 2 * d));
                    }
            std::vector<uint64_t> at_b((size_t)(hi - lo));
            for (int64_t st = lo; st < hi; st++) at_b[(size_t)(st - lo)] = code[(size_t)st] | (uint64_t)st;
            std::vector<uint64_t>().swap(code);
            std::sort(at_b.begin(), at_b.end());
            const size_t words = E >= 32 ? E / 32 : 1;
            T.filter.assign(words, 0u);
            T.dense.resize(4 * at_b.size());
            for (size_t r = 0; r < at_b.size(); r++) {
                const uint32_t w = (uint32_t)(at_b[r] >> 32), st = (uint32_t)at_b[r];
                T.filter[w >> 5] |= 1u << (w & 31);
                if (T.out_id[st]) {
                    const uint32_t special[4] = {0u, kSkipSpecial, 0u, 0u};
                    memcpy(&T.dense[4 * r], special, 16);
                } else {
                    memcpy(&T.dense[4 * r], &T.skip[(size_t)(4 * (int64_t)st)], 16);
                }
            }
            std::vector<uint32_t> rank(words, 0u);
            uint64_t count = 0;
            for (size_t w = 0; w < words; w++) {
                rank[w] = (uint32_t)count;
                count += (uint64_t)__builtin_popcount(T.filter[w]);
            }
            T.rank_wide = count > 65535;
            if (T.rank_wide) T.rank32.swap(rank);
            else T.rank16.assign(rank.begin(), rank.end());
            if (b > kFilter1B) {
                const size_t E1 = (size_t)1 << (2 * kFilter1B);
                T.filter1_b = kFilter1B;
                T.filter1.assign(E1 / 32, 0u);
                for (const uint64_t v : at_b) {
                    const size_t w1 = (size_t)(v >> 32) & (E1 - 1);   // the first kFilter1B bases
                    T.filter1[w1 >> 5] |= 1u << (w1 & 31);
                }
            }
        } else if (b > 0 && !T.skip.empty()) {
            T.filter_b = b;
            const size_t E = (size_t)1 << (2 * b);
            const uint32_t kNone = 0xFFFFFFFFu, kSpecialVal = 0xFFFFFFFEu;
            std::vector<uint32_t> val(E, kNone);      // state reached at depth b, or special
            // One pass over the states of depth <= b in id order (a parent's id is below
            // its children's): each state carries the code of its string (first base in
            // the low bits) and whether a pattern ends on its path, and hands both to
            // its children. Every entry of val is written by one state or one missing
            // edge, so the order of the writes does not matter.
            const int32_t top = std::min(b, max_len);
            const int64_t upto = T.level[(size_t)top + 1];
            std::vector<uint32_t> code((size_t)upto, 0u);
            std::vector<uint8_t> seen((size_t)upto, 0);
            for (int32_t d = 0; d <= top; d++) {
                for (int64_t s = T.level[(size_t)d]; s < T.level[(size_t)d + 1]; s++) {
                    if (d == b) {
                        val[code[(size_t)s]] = seen[(size_t)s] ? kSpecialVal : (uint32_t)s;
                        continue;
                    }
                    for (int c = 0; c < 4; c++) {
                        const uint32_t k = code[(size_t)s] | ((uint32_t)c << (2 * d));
                        const uint32_t e = (uint32_t)T.rows[(size_t)(4 * s + c)];
                        if (e) {
                            const size_t child = e & 0x7FFFFFFFu;
                            code[child] = k;
                            seen[child] = (uint8_t)(seen[(size_t)s] | (e >> 31));
                        } else if (seen[(size_t)s]) {
                            const size_t stride = (size_t)1 << (2 * (d + 1));
                            for (size_t idx = k; idx < E; idx += stride) val[idx] = kSpecialVal;
                        }
                    }
                }
            }
            std::vector<uint32_t>().swap(code);
            std::vector<uint8_t>().swap(seen);
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

        // ---- step 3d: sampled screen -----------------------------------------------
        // When every pattern has at least q + s - 1 bases, a match at offset i puts the
        // pattern's q-gram at position d = (-i) mod s at the offset i + d, a multiple of
        // s. So a bit set of the q-grams at positions 0 .. s-1 of every pattern, probed at
        // every s-th offset, lists a superset of the offsets where a pattern can start
        // (the s offsets up to each probe whose q-gram is set). q = 13 for filters in
        // global memory, 10 for an order-10 filter (see sample_q_for).
        const int32_t q = sample_q_for(T.filter_b, min_len, sample_mode);
        if (q) {
            T.sample_q = q;
            T.sample_s = kSampleS;
            T.sample.assign(((size_t)1 << (2 * q)) / 32, 0u);
            for (int32_t j = 0; j < n; j++) {
                const unsigned char *p = (const unsigned char *)patterns[j];
                for (int d = 0; d < kSampleS; d++) {
                    uint32_t g = 0;
                    for (int k = 0; k < q; k++) g |= (uint32_t)base_code(p[d + k]) << (2 * k);
                    T.sample[g >> 5] |= 1u << (g & 31);
                }
            }
        }
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return PFAC_ERR_OOM;
    }
}

}  // namespace pfac
