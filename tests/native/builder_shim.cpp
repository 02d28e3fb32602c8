// A C entry point around the table builder alone (csrc/trie_build.cpp), for tests that
// compile the builder with the host compiler, with no CUDA: build, size and export the
// host tables the library would upload.
#include <stdint.h>
#include <string.h>

#include <new>

#include "pfac.h"
#include "pfac_internal.h"

extern "C" {

void *shim_build(const char *const *patterns, const int32_t *lengths, int32_t n, int32_t filter_b, int32_t sample,
                 int32_t *status)
{
    pfac::HostTables *T = new (std::nothrow) pfac::HostTables();
    if (!T) {
        *status = PFAC_ERR_OOM;
        return nullptr;
    }
    *status = pfac::build_host_tables(patterns, lengths, n, filter_b, T, sample);
    if (*status != PFAC_OK) {
        delete T;
        return nullptr;
    }
    return T;
}

void shim_destroy(void *h) { delete (pfac::HostTables *)h; }

// n_states, n_patterns, max_len, min_len, n_duplicates, filter_b, filter bits set, has skip
void shim_info(void *h, int64_t *out)
{
    const pfac::HostTables &T = *(const pfac::HostTables *)h;
    out[0] = T.n_states;
    out[1] = T.n_patterns;
    out[2] = T.max_len;
    out[3] = T.min_len;
    out[4] = T.n_duplicates;
    out[5] = T.filter_b;
    out[6] = (int64_t)(T.dense.size() / 4);
    out[7] = T.skip.empty() ? 0 : 1;
}

void shim_export(void *h, int32_t *rows, int32_t *out_id, int64_t *level)
{
    const pfac::HostTables &T = *(const pfac::HostTables *)h;
    memcpy(rows, T.rows.data(), T.rows.size() * 4);
    memcpy(out_id, T.out_id.data(), T.out_id.size() * 4);
    memcpy(level, T.level.data(), T.level.size() * 8);
}

// sample_q, sample_s, and the sampled screen's words (when `sample` is not NULL)
void shim_export_sample(void *h, int32_t *qs, uint32_t *sample)
{
    const pfac::HostTables &T = *(const pfac::HostTables *)h;
    qs[0] = T.sample_q;
    qs[1] = T.sample_s;
    if (sample && !T.sample.empty()) memcpy(sample, T.sample.data(), T.sample.size() * 4);
}

void shim_export_shortcuts(void *h, uint32_t *skip, uint32_t *filter, uint32_t *dense)
{
    const pfac::HostTables &T = *(const pfac::HostTables *)h;
    if (!T.skip.empty()) memcpy(skip, T.skip.data(), T.skip.size() * 4);
    if (!T.filter.empty()) memcpy(filter, T.filter.data(), T.filter.size() * 4);
    if (!T.dense.empty()) memcpy(dense, T.dense.data(), T.dense.size() * 4);
}

}  // extern "C"
