/*
 * CPU oracle for the PFAC match scan — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. The product path (the CUDA library) never calls it, and this file
 * includes nothing from the CUDA library's sources.
 *
 * It is deliberately plain and slow:
 *   - an insertion-order goto trie built exactly as the paper inserts patterns
 *     (Section V-A, the insertion procedure after Table I; Section III, goto
 *     function and Fig. 1 numbering), with no breadth-first renumbering, no flag
 *     bits, no packing and no tiling;
 *   - the failure-less scan of Section IV: every text offset starts its own walk
 *     at the root, follows goto edges until none exists, and keeps the longest
 *     pattern that ended on the way (Section IV: PFAC reports only the longest
 *     pattern at each start, not its sub-patterns);
 *   - an independent classic Aho-Corasick machine with failure links and output
 *     sets (Section III; Fig. 2), used only to cross-check the scan.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - pattern ids are 1-based in input order, 0 means "no match" (Table I uses
 *     ids 1..3 and 0 for empty cells);
 *   - when the same string is given twice, the lowest id is kept;
 *   - a text byte outside {A,C,G,T} has no goto edge, so it ends a walk;
 *   - a walk never reads at or past the end of the text (no wrap-around);
 *   - every node of the goto graph is a state, terminal ones included, so the
 *     states of Fig. 1 are numbered 0..9 and AC, ACG, CTGT, TG end at 2, 3, 7, 9.
 *
 * Build: gcc -O2 -shared -fPIC pfac_oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Symbol code of a text or pattern byte: A=0, C=1, G=2, T=3, anything else -1.
 * (The paper orders its table columns A,T,C,G; the order is not observable in
 * any result.) */
static int sym(uint8_t b)
{
    switch (b) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

enum { OR_OK = 0, OR_BAD_ARG = 1, OR_EMPTY = 2, OR_BAD_SYMBOL = 3, OR_OOM = 4 };

/* ------------------------------------------------------------------------ */
/* Goto trie in insertion order (Section V-A; Section III goto function).    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;        /* states in use; state 0 is the root */
    int64_t cap;
    int32_t *go;      /* go[4*s + c] = next state, 0 = no edge (root is never a target) */
    int32_t *term;    /* term[s] = id of the pattern that ends at s, 0 if none */
} otrie;

static int trie_grow(otrie *t)
{
    int64_t cap = t->cap ? 2 * t->cap : 1024;
    int32_t *go = realloc(t->go, (size_t)cap * 4 * sizeof(int32_t));
    if (!go) return OR_OOM;
    t->go = go;
    int32_t *term = realloc(t->term, (size_t)cap * sizeof(int32_t));
    if (!term) return OR_OOM;
    t->term = term;
    memset(t->go + 4 * t->cap, 0, (size_t)(cap - t->cap) * 4 * sizeof(int32_t));
    memset(t->term + t->cap, 0, (size_t)(cap - t->cap) * sizeof(int32_t));
    t->cap = cap;
    return OR_OK;
}

void oracle_trie_free(otrie *t)
{
    if (!t) return;
    free(t->go);
    free(t->term);
    free(t);
}

/* Insert patterns one by one: from the root, follow the edge for each symbol if
 * it exists, otherwise create the next free state and the edge to it; the state
 * reached by the last symbol is terminal with the pattern's id (first writer
 * keeps it, so the lowest id wins for a duplicated string).
 * Pattern j is blob[offsets[j] .. offsets[j+1]) and has id j+1. */
otrie *oracle_trie_build(const uint8_t *blob, const int64_t *offsets, int32_t n, int32_t *err)
{
    *err = OR_OK;
    if (n <= 0 || !blob || !offsets) { *err = OR_BAD_ARG; return NULL; }
    otrie *t = calloc(1, sizeof(otrie));
    if (!t || trie_grow(t) != OR_OK) { free(t); *err = OR_OOM; return NULL; }
    t->n = 1;
    for (int32_t j = 0; j < n; j++) {
        int64_t lo = offsets[j], hi = offsets[j + 1];
        if (hi <= lo) { *err = OR_EMPTY; oracle_trie_free(t); return NULL; }
        int64_t s = 0;
        for (int64_t k = lo; k < hi; k++) {
            int c = sym(blob[k]);
            if (c < 0) { *err = OR_BAD_SYMBOL; oracle_trie_free(t); return NULL; }
            if (t->go[4 * s + c] == 0) {
                if (t->n == t->cap && trie_grow(t) != OR_OK) {
                    *err = OR_OOM; oracle_trie_free(t); return NULL;
                }
                t->go[4 * s + c] = (int32_t)t->n;
                t->n++;
            }
            s = t->go[4 * s + c];
        }
        if (t->term[s] == 0) t->term[s] = j + 1;
    }
    return t;
}

int64_t oracle_trie_states(const otrie *t) { return t->n; }

/* Copy the table out: go[4*S] (columns A,C,G,T) and term[S]. */
void oracle_trie_export(const otrie *t, int32_t *go, int32_t *term)
{
    memcpy(go, t->go, (size_t)t->n * 4 * sizeof(int32_t));
    memcpy(term, t->term, (size_t)t->n * sizeof(int32_t));
}

/* ------------------------------------------------------------------------ */
/* The failure-less scan (Section IV).                                       */
/* ------------------------------------------------------------------------ */

/* For every offset i in [begin, end): start at the root, read text[i], text[i+1],
 * ... while i+k < len, the byte is in {A,C,G,T} and a goto edge exists; remember
 * the last terminal state passed; out[i] = its pattern id, or 0.
 * Since every pattern that matches at i is a path from the root along
 * text[i..], the last terminal passed is the longest such pattern. */
void oracle_pfac_scan(const otrie *t, const uint8_t *text, int64_t len,
                      int64_t begin, int64_t end, int32_t *out)
{
    for (int64_t i = begin; i < end; i++) {
        int64_t s = 0;
        int32_t best = 0;
        for (int64_t k = i; k < len; k++) {
            int c = sym(text[k]);
            if (c < 0) break;
            int64_t nxt = t->go[4 * s + c];
            if (nxt == 0) break;
            s = nxt;
            if (t->term[s] != 0) best = t->term[s];
        }
        out[i] = best;
    }
}

/* ------------------------------------------------------------------------ */
/* Classic Aho-Corasick (Section III, Fig. 2): goto g, failure f, output.     */
/* ------------------------------------------------------------------------ */

typedef struct {
    otrie *g;          /* the same insertion-order goto graph, built independently */
    int32_t *fail;     /* f(s) */
    int32_t *depth;    /* depth[s] = length of the string spelled from the root to s */
    int32_t *onext;    /* nearest state down the failure chain of s whose own output
                          is non-empty, 0 if none */
    int64_t *id_start; /* own output of s = ids[id_start[s] .. id_start[s+1]), ascending */
    int32_t *ids;
} oac;

void oracle_ac_free(oac *m)
{
    if (!m) return;
    oracle_trie_free(m->g);
    free(m->fail);
    free(m->depth);
    free(m->onext);
    free(m->id_start);
    free(m->ids);
    free(m);
}

static int64_t end_state(const otrie *g, const uint8_t *blob, int64_t lo, int64_t hi)
{
    int64_t s = 0;
    for (int64_t k = lo; k < hi; k++) s = g->go[4 * s + sym(blob[k])];
    return s;
}

/* Goto graph as above. Own output of a state = every pattern id whose string ends
 * there (several ids when a string is repeated). Failure function by a
 * breadth-first pass: f = 0 at depth 1; for r = g(s, c), follow t = f(s), f(f(s)),
 * ... until g(t, c) exists (the root loops to itself on a symbol with no edge), and
 * set f(r) = g(t, c). The full output is own(r) ∪ output(f(r)); it is kept as a
 * link to the nearest failure ancestor whose own output is non-empty. */
oac *oracle_ac_build(const uint8_t *blob, const int64_t *offsets, int32_t n, int32_t *err)
{
    otrie *g = oracle_trie_build(blob, offsets, n, err);
    if (!g) return NULL;
    int64_t S = g->n;
    oac *m = calloc(1, sizeof(oac));
    int32_t *queue = malloc((size_t)S * sizeof(int32_t));
    int64_t *endst = malloc((size_t)n * sizeof(int64_t));
    if (m) {
        m->g = g;
        m->fail = calloc((size_t)S, sizeof(int32_t));
        m->depth = calloc((size_t)S, sizeof(int32_t));
        m->onext = calloc((size_t)S, sizeof(int32_t));
        m->id_start = calloc((size_t)S + 1, sizeof(int64_t));
        m->ids = malloc((size_t)n * sizeof(int32_t));
    }
    if (!m || !queue || !endst || !m->fail || !m->depth || !m->onext || !m->id_start || !m->ids) {
        if (m) oracle_ac_free(m); else oracle_trie_free(g);
        free(queue); free(endst);
        *err = OR_OOM;
        return NULL;
    }
    /* Own outputs as a bucket list, ids ascending within a state. */
    for (int32_t j = 0; j < n; j++) {
        endst[j] = end_state(g, blob, offsets[j], offsets[j + 1]);
        m->id_start[endst[j] + 1]++;
    }
    for (int64_t s = 0; s < S; s++) m->id_start[s + 1] += m->id_start[s];
    {
        int64_t *fill = calloc((size_t)S, sizeof(int64_t));
        if (!fill) { oracle_ac_free(m); free(queue); free(endst); *err = OR_OOM; return NULL; }
        for (int32_t j = 0; j < n; j++) {
            int64_t s = endst[j];
            m->ids[m->id_start[s] + fill[s]++] = j + 1;
        }
        free(fill);
    }
    free(endst);
    /* Breadth-first pass: depth, failure, output link. */
    int64_t qh = 0, qt = 0;
    queue[qt++] = 0;
    while (qh < qt) {
        int32_t s = queue[qh++];
        for (int c = 0; c < 4; c++) {
            int32_t r = g->go[4 * s + c];
            if (!r) continue;
            queue[qt++] = r;
            m->depth[r] = m->depth[s] + 1;
            if (s == 0) {
                m->fail[r] = 0;
            } else {
                int32_t t = m->fail[s];
                while (t != 0 && g->go[4 * t + c] == 0) t = m->fail[t];
                m->fail[r] = g->go[4 * t + c];    /* 0 when the root has no edge c */
            }
            int32_t f = m->fail[r];
            m->onext[r] = (m->id_start[f + 1] > m->id_start[f]) ? f : m->onext[f];
        }
    }
    free(queue);
    return m;
}

int64_t oracle_ac_states(const oac *m) { return m->g->n; }

/* Copy out f (to check it against failure links derived by hand). */
void oracle_ac_export_fail(const oac *m, int32_t *fail)
{
    memcpy(fail, m->fail, (size_t)m->g->n * sizeof(int32_t));
}

/* Copy out the full output set of state s (own ids, then those of the failure
 * chain); returns its size (at most cap ids written). */
int64_t oracle_ac_output(const oac *m, int32_t s, int32_t *ids, int64_t cap)
{
    int64_t k = 0;
    int32_t o = (m->id_start[s + 1] > m->id_start[s]) ? s : m->onext[s];
    for (; o != 0; o = m->onext[o])
        for (int64_t q = m->id_start[o]; q < m->id_start[o + 1]; q++, k++)
            if (k < cap) ids[k] = m->ids[q];
    return k;
}

/* Run the sequential machine over the text (Section III): on each symbol follow
 * failure links until a goto edge exists (the root loops to itself), move, and
 * emit every pattern of output(state). A byte outside {A,C,G,T} has no edge
 * anywhere, so the machine falls back to the root.
 *
 * Each occurrence (end position e, pattern id p) goes to up to two sinks:
 *  - longest[start], start = e - |p| + 1, keeps the longest pattern that starts
 *    there, and the lowest id among equal strings (0 where none starts);
 *  - occ_end/occ_id (if non-NULL) store the first `cap` occurrences in order.
 * Returns the total number of occurrences. */
int64_t oracle_ac_scan(const oac *m, const uint8_t *text, int64_t len, int32_t *longest,
                       int64_t *occ_end, int32_t *occ_id, int64_t cap)
{
    const otrie *g = m->g;
    int32_t *best_len = NULL;
    if (longest) {
        best_len = calloc((size_t)(len > 0 ? len : 1), sizeof(int32_t));
        if (!best_len) return -1;
        memset(longest, 0, (size_t)len * sizeof(int32_t));
    }
    int64_t total = 0;
    int32_t s = 0;
    for (int64_t i = 0; i < len; i++) {
        int c = sym(text[i]);
        if (c < 0) { s = 0; continue; }
        while (s != 0 && g->go[4 * s + c] == 0) s = m->fail[s];
        s = g->go[4 * s + c];
        int32_t o = (m->id_start[s + 1] > m->id_start[s]) ? s : m->onext[s];
        for (; o != 0; o = m->onext[o]) {
            int32_t L = m->depth[o];
            int64_t start = i - L + 1;
            for (int64_t q = m->id_start[o]; q < m->id_start[o + 1]; q++) {
                int32_t id = m->ids[q];
                if (longest && (L > best_len[start] ||
                                (L == best_len[start] && id < longest[start]))) {
                    best_len[start] = L;
                    longest[start] = id;
                }
                if (occ_end && total < cap) { occ_end[total] = i; occ_id[total] = id; }
                total++;
            }
        }
    }
    free(best_len);
    return total;
}
