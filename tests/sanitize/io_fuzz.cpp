// The file front end (csrc/pfac_io.cpp) under AddressSanitizer and
// UndefinedBehaviorSanitizer: random files (FASTA headers, sequence lines, blank lines,
// CRLF endings, bytes of every value) are read as texts and as pattern files. The table
// build behind pfac_build_file is replaced here by a stand-in that reads every byte of
// every pattern it is given, so a pattern pointer outside the file's buffer is reported.
// Exit status 0 = no sanitizer report and every check passed.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <random>
#include <string>
#include <vector>

#include "pfac.h"

namespace pfac {
int set_last_error(int code) { return code; }
}  // namespace pfac

static uint64_t g_checksum = 0;
static int g_dummy_table = 0;

extern "C" pfac_handle pfac_build_ex(const char *const *patterns, const int32_t *lengths, int32_t n,
                                     const pfac_build_opts *)
{
    for (int32_t j = 0; j < n; j++)
        for (int32_t k = 0; k < lengths[j]; k++) g_checksum += (unsigned char)patterns[j][k];
    return (pfac_handle)&g_dummy_table;
}

int main(int argc, char **argv)
{
    const char *path = argc > 1 ? argv[1] : "io_fuzz.tmp";
    std::mt19937_64 rng(99);
    for (int iter = 0; iter < 2000; iter++) {
        std::string raw;
        const int lines = (int)(rng() % 30);
        for (int i = 0; i < lines; i++) {
            const int kind = (int)(rng() % 10);
            if (kind < 3) raw += ">h" + std::to_string(rng() % 100);
            else if (kind < 4) raw += "";
            else if (kind < 5)
                for (int k = (int)(rng() % 8); k > 0; k--) raw += (char)(rng() % 256);
            else
                for (int k = 1 + (int)(rng() % 40); k > 0; k--) raw += "ACGT"[rng() % 4];
            if (i + 1 < lines || rng() % 2) raw += rng() % 3 ? "\n" : "\r\n";
        }
        FILE *f = fopen(path, "wb");
        if (!f) return 1;
        if (!raw.empty() && fwrite(raw.data(), 1, raw.size(), f) != raw.size()) return 1;
        fclose(f);
        for (int fasta = 0; fasta < 2; fasta++) {
            int64_t len = -1;
            if (pfac_read_text_file(path, fasta, nullptr, 0, &len) != PFAC_OK) return 1;
            if (len < 0 || len > (int64_t)raw.size()) return 1;
            std::vector<uint8_t> buf((size_t)len + 1);
            int64_t got = -1;
            if (pfac_read_text_file(path, fasta, buf.data(), len, &got) != PFAC_OK || got != len) return 1;
            if (!fasta && memcmp(buf.data(), raw.data(), (size_t)len) != 0) return 1;
        }
        pfac_build_opts o{};
        o.host_only = 1;
        (void)pfac_build_file(path, &o);
    }
    remove(path);
    printf("io_fuzz: ok (%llu)\n", (unsigned long long)g_checksum);
    return 0;
}
