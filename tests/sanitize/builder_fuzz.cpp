// Host table builder under AddressSanitizer and UndefinedBehaviorSanitizer, or under
// ThreadSanitizer: random pattern sets (duplicates, nested prefixes, one-base patterns,
// every filter order) are built and the encodings checked against their definitions'
// simplest consequences. The last sets are large enough for the builder to spread its
// sub-tries over several threads; the argument "threaded" runs only those.
// Exit status 0 = every check passed and no sanitizer report.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <random>
#include <string>
#include <vector>

#include "../../paper_1811_10498_gb300/csrc/pfac_internal.h"

static int fail(const char *what, int iter)
{
    fprintf(stderr, "builder_fuzz: %s (case %d)\n", what, iter);
    return 1;
}

static std::vector<std::string> random_set(std::mt19937_64 &rng, int n, int max_len)
{
    const char acgt[4] = {'A', 'C', 'G', 'T'};
    std::vector<std::string> pats;
    for (int j = 0; j < n; j++) {
        if (j > 0 && rng() % 5 == 0) {             // a prefix or a copy of an earlier pattern
            const std::string &p = pats[rng() % pats.size()];
            pats.push_back(p.substr(0, 1 + rng() % p.size()));
            continue;
        }
        const int len = 1 + (int)(rng() % max_len);
        std::string p;
        for (int k = 0; k < len; k++) p += acgt[rng() % 4];
        pats.push_back(p);
    }
    return pats;
}

static int build_and_check(const std::vector<std::string> &pats, int32_t fb, int iter)
{
    const int n = (int)pats.size();
    std::vector<const char *> ptrs;
    std::vector<int32_t> lens;
    for (auto &p : pats) {
        ptrs.push_back(p.data());
        lens.push_back((int32_t)p.size());
    }
    pfac::HostTables T;
    if (pfac::build_host_tables(ptrs.data(), lens.data(), n, fb, &T) != 0) return fail("build failed", iter);
    if ((int64_t)T.rows.size() != 4 * T.n_states || (int64_t)T.out_id.size() != T.n_states)
        return fail("row / id sizes", iter);
    int64_t terminals = 0;
    for (int64_t s = 0; s < T.n_states; s++) {
        if (T.out_id[(size_t)s]) terminals++;
        for (int c = 0; c < 4; c++) {
            const uint32_t e = (uint32_t)T.rows[(size_t)(4 * s + c)];
            const int64_t t = e & 0x7FFFFFFFu;
            if (e && (t <= s || t >= T.n_states)) return fail("edge not breadth-first", iter);
            if (e && ((e >> 31) != 0) != (T.out_id[(size_t)t] != 0)) return fail("terminal flag", iter);
        }
    }
    if (terminals + T.n_duplicates != n) return fail("terminals + duplicates != patterns", iter);
    if (T.filter_b > 0) {
        int64_t set = 0;
        for (uint32_t w : T.filter) set += __builtin_popcount(w);
        if ((int64_t)T.dense.size() != 4 * set) return fail("dense entries != set filter bits", iter);
    }
    return 0;
}

int main(int argc, char **argv)
{
    const bool threaded_only = argc > 1 && strcmp(argv[1], "threaded") == 0;
    std::mt19937_64 rng(1234);
    for (int iter = 0; iter < 300 && !threaded_only; iter++) {
        const int n = 1 + (int)(rng() % 60);
        const std::vector<std::string> pats = random_set(rng, n, iter % 3 == 0 ? 6 : 40);
        // -1 (none), 0 (automatic), 1..9, and the largest order, 12, once
        const int32_t fb = iter == 299 ? 12 : (int32_t)(iter % 11) - 1;
        if (build_and_check(pats, fb, iter)) return 1;
    }
    // about 3M bases: several threads
    for (int iter = 300; iter < 302; iter++)
        if (build_and_check(random_set(rng, 100000, 60), iter == 300 ? 0 : 8, iter)) return 1;
    if (!threaded_only) {
        // every error path
        const char *bad[] = {"ACGT", "ACNT"};
        const int32_t bl[] = {4, 4};
        pfac::HostTables T;
        if (pfac::build_host_tables(bad, bl, 2, 0, &T) == 0) return fail("bad symbol accepted", -1);
        const int32_t zl[] = {4, 0};
        if (pfac::build_host_tables(bad, zl, 2, 0, &T) == 0) return fail("empty pattern accepted", -1);
        if (pfac::build_host_tables(bad, bl, 0, 0, &T) == 0) return fail("no pattern accepted", -1);
    }
    printf("builder_fuzz: ok\n");
    return 0;
}
