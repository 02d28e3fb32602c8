/* The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer (test
 * infrastructure checking test infrastructure): random tries, failure-link machines and
 * scans over texts with bytes outside ACGT; the failure-less scan and the classic
 * machine must agree. Exit status 0 = agreement and no sanitizer report. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct otrie otrie;
typedef struct oac oac;
otrie *oracle_trie_build(const uint8_t *blob, const int64_t *offsets, int32_t n, int32_t *err);
void oracle_trie_free(otrie *t);
void oracle_pfac_scan(const otrie *t, const uint8_t *text, int64_t len, int64_t begin, int64_t end, int32_t *out);
oac *oracle_ac_build(const uint8_t *blob, const int64_t *offsets, int32_t n, int32_t *err);
void oracle_ac_free(oac *m);
int64_t oracle_ac_scan(const oac *m, const uint8_t *text, int64_t len, int32_t *longest, int64_t *occ_end,
                       int32_t *occ_id, int64_t cap);

static uint64_t state = 88172645463325252ull;
static uint64_t next(void)
{
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return state;
}

int main(void)
{
    const char alpha[6] = {'A', 'C', 'G', 'T', 'N', '\n'};
    for (int iter = 0; iter < 400; iter++) {
        const int n = 1 + (int)(next() % 20);
        uint8_t blob[20 * 12];
        int64_t offs[21];
        offs[0] = 0;
        for (int j = 0; j < n; j++) {
            const int len = 1 + (int)(next() % 12);
            for (int k = 0; k < len; k++) blob[offs[j] + k] = (uint8_t)alpha[next() % 4];
            offs[j + 1] = offs[j] + len;
        }
        const int64_t tl = (int64_t)(next() % 300);
        uint8_t *text = malloc((size_t)(tl > 0 ? tl : 1));
        for (int64_t i = 0; i < tl; i++) text[i] = (uint8_t)alpha[next() % 6];
        int32_t err = 0;
        otrie *t = oracle_trie_build(blob, offs, n, &err);
        oac *m = oracle_ac_build(blob, offs, n, &err);
        if (!t || !m) { fprintf(stderr, "oracle_fuzz: build failed\n"); return 1; }
        int32_t *a = calloc((size_t)(tl > 0 ? tl : 1), sizeof(int32_t));
        int32_t *b = calloc((size_t)(tl > 0 ? tl : 1), sizeof(int32_t));
        int64_t ends[4096];
        int32_t ids[4096];
        oracle_pfac_scan(t, text, tl, 0, tl, a);
        oracle_ac_scan(m, text, tl, b, ends, ids, 4096);
        if (tl && memcmp(a, b, (size_t)tl * sizeof(int32_t)) != 0) {
            fprintf(stderr, "oracle_fuzz: scans disagree (case %d)\n", iter);
            return 1;
        }
        free(a);
        free(b);
        free(text);
        oracle_trie_free(t);
        oracle_ac_free(m);
    }
    printf("oracle_fuzz: ok\n");
    return 0;
}
