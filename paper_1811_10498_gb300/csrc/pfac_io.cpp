// File front end: patterns and texts read from files, as the paper's host program does
// before it builds the table and launches the scan (Section V-B, Figs. 4 and 5).
//
// Pattern files hold one pattern per line (a trailing '\r' is dropped, empty lines are
// skipped). A file whose first non-empty line starts with '>' is read as FASTA: each
// record's sequence lines, joined, make one pattern, and header lines are skipped.
//
// Text files are read as they are, newlines included (a newline has no edge in the trie,
// so no walk crosses from one line into the next), or as FASTA: header lines dropped,
// the sequence lines of a record joined, one '\n' between records.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace {

// The whole file, or false if it cannot be opened or read.
bool slurp(const char *path, std::vector<uint8_t> *out)
{
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    bool ok = true;
    if (fseek(f, 0, SEEK_END) != 0) ok = false;
    long size = ok ? ftell(f) : -1;
    if (size < 0 || fseek(f, 0, SEEK_SET) != 0) ok = false;
    if (ok) {
        out->resize((size_t)size);
        if (size > 0 && fread(out->data(), 1, (size_t)size, f) != (size_t)size) ok = false;
    }
    fclose(f);
    return ok;
}

// Calls fn(begin, end) for every line of [p, e) without its '\n' and trailing '\r'.
template <typename Fn>
void for_each_line(const uint8_t *p, const uint8_t *e, Fn fn)
{
    while (p < e) {
        const uint8_t *nl = (const uint8_t *)memchr(p, '\n', (size_t)(e - p));
        const uint8_t *end = nl ? nl : e;
        const uint8_t *le = end;
        if (le > p && le[-1] == '\r') le--;
        fn(p, le);
        p = nl ? nl + 1 : e;
    }
}

bool is_fasta(const std::vector<uint8_t> &data)
{
    for (uint8_t c : data) {
        if (c == '\n' || c == '\r' || c == ' ' || c == '\t') continue;
        return c == '>';
    }
    return false;
}

// FASTA records joined in place: each record's sequence lines are moved together
// (header lines dropped), with one '\n' between records when `newline_between` is set.
// Returns each record's (offset, length) in `data`, which is cut to the joined bytes.
// A record opens at a header line, or at a sequence line before the first header.
// Writes never pass the line being read: a sequence line moves left onto itself or
// earlier, and the one separator byte a record adds replaces its header's '>'.
std::vector<std::pair<size_t, size_t>> fasta_join_in_place(std::vector<uint8_t> &data, bool newline_between)
{
    std::vector<std::pair<size_t, size_t>> recs;
    uint8_t *base = data.data();
    size_t w = 0;
    for_each_line(base, base + data.size(), [&](const uint8_t *b, const uint8_t *e) {
        if (b == e) return;
        const bool header = *b == '>';
        if (header || recs.empty()) {
            if (newline_between && !recs.empty()) base[w++] = '\n';
            recs.emplace_back(w, 0);
            if (header) return;
        }
        const size_t len = (size_t)(e - b);
        memmove(base + w, b, len);
        w += len;
        recs.back().second += len;
    });
    data.resize(w);
    return recs;
}

}  // namespace

extern "C" pfac_handle pfac_build_file(const char *path, const pfac_build_opts *opts)
{
    if (!path) {
        pfac::set_last_error(PFAC_ERR_INVALID_ARG);
        return nullptr;
    }
    try {
        std::vector<uint8_t> data;
        if (!slurp(path, &data)) {
            pfac::set_last_error(PFAC_ERR_IO);
            return nullptr;
        }
        // Patterns point into the file's bytes: lines as they are, FASTA records
        // joined in place.
        std::vector<std::pair<size_t, size_t>> pats;
        if (is_fasta(data)) {
            pats = fasta_join_in_place(data, false);
        } else {
            for_each_line(data.data(), data.data() + data.size(), [&](const uint8_t *b, const uint8_t *e) {
                if (b < e) pats.emplace_back((size_t)(b - data.data()), (size_t)(e - b));
            });
        }
        if (pats.empty() || pats.size() > (size_t)INT32_MAX) {
            pfac::set_last_error(PFAC_ERR_INVALID_ARG);
            return nullptr;
        }
        std::vector<const char *> ptrs(pats.size());
        std::vector<int32_t> lens(pats.size());
        for (size_t j = 0; j < pats.size(); j++) {
            if (pats[j].second > (size_t)INT32_MAX) {
                pfac::set_last_error(PFAC_ERR_INVALID_ARG);
                return nullptr;
            }
            ptrs[j] = (const char *)data.data() + pats[j].first;
            lens[j] = (int32_t)pats[j].second;
        }
        return pfac_build_ex(ptrs.data(), lens.data(), (int32_t)pats.size(), opts);
    } catch (const std::bad_alloc &) {
        pfac::set_last_error(PFAC_ERR_OOM);
        return nullptr;
    }
}

extern "C" int pfac_read_text_file(const char *path, int32_t fasta, uint8_t *buf, int64_t cap, int64_t *len)
{
    if (!path || !len || cap < 0 || (cap > 0 && !buf)) return pfac::set_last_error(PFAC_ERR_INVALID_ARG);
    try {
        std::vector<uint8_t> data;
        if (!slurp(path, &data)) return pfac::set_last_error(PFAC_ERR_IO);
        if (fasta) fasta_join_in_place(data, true);
        *len = (int64_t)data.size();
        if (buf && cap > 0) memcpy(buf, data.data(), (size_t)std::min<int64_t>(cap, (int64_t)data.size()));
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return pfac::set_last_error(PFAC_ERR_OOM);
    }
}
