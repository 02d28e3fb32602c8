/* A plain C99 client of libpfac.so: the boundary used from C with no Python. It builds
 * host-only tables through the C ABI (no device call) and checks what it reads back.
 * Exit status 0 = every check passed; the last line printed is "c_client: ok". */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pfac.h"

static int fail(const char *what)
{
    fprintf(stderr, "c_client: %s\n", what);
    return 1;
}

int main(void)
{
    /* Fig. 1 patterns: AC, ACG, CTGT, TG -> 10 states, longest pattern 4 */
    const char *pats[] = {"AC", "ACG", "CTGT", "TG"};
    const int32_t lens[] = {2, 3, 4, 2};
    pfac_build_opts o;
    memset(&o, 0, sizeof o);
    o.host_only = 1;
    pfac_handle h = pfac_build_ex(pats, lens, 4, &o);
    if (!h) return fail(pfac_error_string(pfac_last_error()));
    int64_t n_states = 0, bytes = -1;
    int32_t max_len = 0;
    if (pfac_info(h, &n_states, &max_len, &bytes) != PFAC_OK) return fail("pfac_info");
    if (n_states != 10 || max_len != 4 || bytes != 0) return fail("table size");
    int32_t rows[40], out_id[10];
    int64_t level[6];
    if (pfac_export(h, rows, out_id, level) != PFAC_OK) return fail("pfac_export");
    /* breadth-first: root, A, C, T, then AC, CT, TG, then ACG, CTG, then CTGT */
    const int64_t want_level[6] = {0, 1, 4, 7, 9, 10};
    if (memcmp(level, want_level, sizeof level) != 0) return fail("levels");
    int terminals = 0;
    for (int s = 0; s < 10; s++) terminals += out_id[s] != 0;
    if (terminals != 4) return fail("terminal states");
    if (pfac_destroy(h) != PFAC_OK) return fail("pfac_destroy");

    /* errors come back as status codes and through pfac_last_error */
    const char *bad[] = {"ACNT"};
    const int32_t bad_len[] = {4};
    if (pfac_build_ex(bad, bad_len, 1, &o) != NULL || pfac_last_error() != PFAC_ERR_BAD_SYMBOL)
        return fail("bad symbol");
    if (pfac_build_ex(pats, lens, 0, &o) != NULL || pfac_last_error() != PFAC_ERR_INVALID_ARG)
        return fail("no patterns");
    if (pfac_info(NULL, NULL, NULL, NULL) != PFAC_ERR_INVALID_ARG) return fail("NULL handle");
    if (strcmp(pfac_error_string(PFAC_ERR_OOM), "out of memory") != 0) return fail("error strings");
    printf("c_client: ok\n");
    return 0;
}
