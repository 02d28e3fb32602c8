// C ABI of the PFAC scan (include/pfac.h): table handles, upload, argument checks,
// launch configuration and dispatch to the kernels in pfac_kernels.cu.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pfac.h"
#include "pfac_internal.h"

struct pfac_table {
    pfac::HostTables host;
    int device = -1;
    void *dmem = nullptr;
    size_t dbytes = 0;
    int64_t rows_bytes = 0, skip_bytes = 0, filter_set = 0;
    pfac::DeviceTable dt{};
    std::mutex mu;
    bool cfg_set = false;
    pfac_config cfg{};
    // the paper's table layouts, derived on the device when a configuration asks for
    // them: two arrays (next, pid) and merged pairs
    void *paper_two = nullptr;
    void *paper_pair = nullptr;
    pfac::PaperTables paper{};
};

namespace {

thread_local int g_last_error = PFAC_OK;
thread_local std::string g_last_cuda;

int fail(int code)
{
    g_last_error = code;
    return code;
}

int cuda_fail(cudaError_t e)
{
    g_last_cuda = cudaGetErrorString(e);
    cudaGetLastError();   // clear a non-sticky error so later calls start clean
    return fail(PFAC_ERR_CUDA);
}

std::mutex g_props_mu;
std::map<int, pfac::DeviceProps> g_props;

int device_props(pfac::DeviceProps *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> lk(g_props_mu);
    auto it = g_props.find(dev);
    if (it == g_props.end()) {
        pfac::DeviceProps p{};
        int rc = pfac::get_device_props(&p);
        if (rc != PFAC_OK) return cuda_fail(cudaGetLastError());
        it = g_props.emplace(dev, p).first;
    }
    *out = it->second;
    return PFAC_OK;
}

// A d_* argument must be device (or managed) memory.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_handle_for_launch(pfac_handle h, pfac::DeviceProps *dp)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    if (h->device < 0 || !h->dmem) return fail(PFAC_ERR_HOST_ONLY);
    int rc = device_props(dp);
    if (rc != PFAC_OK) return rc;
    if (dp->device != h->device) return fail(PFAC_ERR_INVALID_ARG);
    return PFAC_OK;
}

bool has_kernel2(const pfac_table *h) { return h->dt.skip && h->dt.filter && h->dt.dense; }

pfac_config default_config(const pfac_table *h, bool packed)
{
    pfac_config c{};
    c.kernel = has_kernel2(h) ? 2 : 1;
    c.threads = 1024;
    c.ctas_per_sm = 1;
    // measured on the genome-scale scan: 32 offsets per lane and 3 stages beat 16 and 4
    // on packed text by 6 %; ASCII tiles are four times larger in shared memory
    c.stages = packed ? 3 : 2;
    c.lane_offsets = packed ? 32 : 16;
    c.rank_in_smem = 0;
    c.l2_persist = 0;
    return c;
}

pfac_config effective_config(pfac_table *h, bool packed)
{
    pfac_config d = default_config(h, packed);
    std::lock_guard<std::mutex> lk(h->mu);
    if (!h->cfg_set) return d;
    pfac_config c = h->cfg;
    if (c.kernel == 0) c.kernel = d.kernel;
    if (c.threads == 0) c.threads = d.threads;
    if (c.ctas_per_sm == 0) c.ctas_per_sm = d.ctas_per_sm;
    if (c.stages == 0) c.stages = d.stages;
    if (c.lane_offsets == 0) c.lane_offsets = d.lane_offsets;
    return c;
}

pfac::TiledConfig tiled_config(const pfac_config &c)
{
    pfac::TiledConfig t{};
    t.threads = c.threads;
    t.ctas_per_sm = c.ctas_per_sm;
    t.stages = c.stages;
    t.smem_table_bytes = c.rank_in_smem < 0 ? -1 : 0;
    t.walk_loads = c.walk_loads;
    t.lane_offsets = c.lane_offsets;
    t.l2_persist = c.l2_persist;
    t.zero_writer = c.zero_writer > 0 ? c.zero_writer - 1 : 0;
    t.screen = c.screen;
    t.timeout_ns = 2000000000LL;
    return t;
}

// Deferred-walk scratch, one buffer per (device, stream): launches on one stream are
// ordered, launches on different streams never share a buffer. Allocated on first use
// and grown when a longer text needs more room.
struct Scratch {
    void *mem = nullptr;
    int64_t cap = 0;
};
std::mutex g_scratch_mu;
std::map<std::pair<int, cudaStream_t>, Scratch> g_scratch;

// Items of deferred-walk scratch for a text of n bases. PFAC_DEFER_CAP overrides it
// (tests use a tiny list to exercise walks that find the list full).
int64_t defer_capacity(int64_t n)
{
    if (const char *env = getenv("PFAC_DEFER_CAP")) {
        long long v = atoll(env);
        if (v >= 1) return v;
    }
    return std::min<int64_t>(std::max<int64_t>(n / 256, 65536), 1LL << 24);
}

int get_scratch(int dev, cudaStream_t st, int64_t n, pfac::DeferScratch *out)
{
    const int64_t want = defer_capacity(n);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    Scratch &sc = g_scratch[{dev, st}];
    if (sc.cap < want) {
        if (sc.mem) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaFree(sc.mem);
            if (e != cudaSuccess) return cuda_fail(e);
            sc.mem = nullptr;
            sc.cap = 0;
        }
        void *m = nullptr;
        cudaError_t e = cudaMalloc(&m, 256 + (size_t)want * pfac::defer_item_bytes());
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? PFAC_ERR_OOM : PFAC_ERR_CUDA);
        }
        sc.mem = m;
        sc.cap = want;
    }
    out->count = (unsigned long long *)sc.mem;
    out->items = (uint8_t *)sc.mem + 256;
    out->cap = sc.cap;
    return PFAC_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Batched scans: a device array of table descriptors per distinct list of handles
// (uploaded once, dropped when one of its handles is destroyed), and scratch per
// (device, stream) grown on demand.
std::mutex g_sets_mu;
std::map<std::pair<int, std::vector<pfac_handle>>, void *> g_sets;

int set_descriptors(const pfac_handle *sets, int32_t n_sets, int dev, const pfac::DeviceTable **out)
{
    std::vector<pfac_handle> key(sets, sets + n_sets);
    std::lock_guard<std::mutex> lk(g_sets_mu);
    auto it = g_sets.find({dev, key});
    if (it == g_sets.end()) {
        std::vector<pfac::DeviceTable> host((size_t)n_sets);
        for (int32_t i = 0; i < n_sets; i++) host[(size_t)i] = sets[i]->dt;
        void *d = nullptr;
        cudaError_t e = cudaMalloc(&d, host.size() * sizeof(pfac::DeviceTable));
        if (e == cudaSuccess) e = cudaMemcpy(d, host.data(), host.size() * sizeof(pfac::DeviceTable), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            return cuda_fail(e);
        }
        it = g_sets.emplace(std::make_pair(dev, key), d).first;
    }
    *out = (const pfac::DeviceTable *)it->second;
    return PFAC_OK;
}

void forget_handle(pfac_handle h)
{
    std::lock_guard<std::mutex> lk(g_sets_mu);
    for (auto it = g_sets.begin(); it != g_sets.end();) {
        const auto &v = it->first.second;
        if (std::find(v.begin(), v.end(), h) != v.end()) {
            cudaFree(it->second);
            it = g_sets.erase(it);
        } else {
            ++it;
        }
    }
}

std::mutex g_bscratch_mu;
std::map<std::pair<int, cudaStream_t>, Scratch> g_bscratch;

int batch_scratch(int dev, cudaStream_t st, int64_t bytes, void **out)
{
    std::lock_guard<std::mutex> lk(g_bscratch_mu);
    Scratch &sc = g_bscratch[{dev, st}];
    if (sc.cap < bytes) {
        if (sc.mem) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = cudaFree(sc.mem);
            if (e != cudaSuccess) return cuda_fail(e);
            sc.mem = nullptr;
            sc.cap = 0;
        }
        cudaError_t e = cudaMalloc(&sc.mem, (size_t)bytes);
        if (e != cudaSuccess) {
            sc.mem = nullptr;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? PFAC_ERR_OOM : PFAC_ERR_CUDA);
        }
        sc.cap = bytes;
    }
    *out = sc.mem;
    return PFAC_OK;
}

// Run the scan with the handle's configuration. Kernel 2 needs 16-byte aligned text
// and output, the filter and the skip entries; otherwise kernel 1 runs.
int run_scan(pfac_handle h, const void *text, bool packed, int64_t n, int32_t *out, int64_t *c_off,
             int32_t *c_ids, int64_t cap, int64_t *count, cudaStream_t st, const pfac::DeviceProps &dp,
             bool all_matches = false)
{
    pfac_config c = effective_config(h, packed);
    const bool compact = c_off != nullptr;
    bool tiled = c.kernel == 2 && has_kernel2(h) && aligned16(text) && (compact || aligned16(out));
    int rc = PFAC_OK;
    if (tiled) {
        pfac::TiledConfig tc = tiled_config(c);
        pfac::DeferScratch scratch{};
        rc = get_scratch(dp.device, st, n, &scratch);
        if (rc != PFAC_OK) return rc;
        rc = pfac::launch_tiled(h->dt, text, packed, n, out, c_off, c_ids, cap, (unsigned long long *)count, tc,
                                scratch, st, dp, all_matches);
        if (rc == PFAC_ERR_UNSUPPORTED) tiled = false;   // the configuration does not fit shared memory
        else if (rc != PFAC_OK) return rc == PFAC_ERR_CUDA ? cuda_fail(cudaGetLastError()) : fail(rc);
    }
    if (!tiled) {
        if (!compact) {
            // dense ids: the one-thread-per-offset kernel with the handle's placement
            pfac::PaperConfig pc{c.table_layout, c.row_loads, c.text_smem};
            pfac::PaperTables pt{};
            {
                std::lock_guard<std::mutex> lk(h->mu);
                pt = h->paper;
            }
            rc = pfac::launch_paper_walk(h->dt, pt, pc, text, packed, n, out, st, dp);
            if (rc == PFAC_ERR_UNSUPPORTED && pc.text_smem) {   // tile above 48 KB: text from global memory
                pc.text_smem = 0;
                rc = pfac::launch_paper_walk(h->dt, pt, pc, text, packed, n, out, st, dp);
            }
        } else {
            rc = pfac::launch_walk_rows_any(h->dt, text, packed, n, out, c_off, c_ids, cap,
                                            (unsigned long long *)count, st, dp, all_matches);
        }
        if (rc != PFAC_OK) return rc == PFAC_ERR_CUDA ? cuda_fail(cudaGetLastError()) : fail(rc);
    }
    return PFAC_OK;
}

// Derive the paper's layout `layout` (1 = two arrays, 2 = merged pairs) on the handle's
// device, once; synchronous.
int ensure_paper_layout(pfac_handle h, int layout)
{
    if (layout == 0 || h->device < 0) return PFAC_OK;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if ((layout == 1 && h->paper_two) || (layout == 2 && h->paper_pair)) return PFAC_OK;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    const size_t bytes = (size_t)h->dt.n_states * 32;    // 4 cells x 8 bytes
    void *m = nullptr;
    cudaError_t e = cudaMalloc(&m, bytes);
    int rc = PFAC_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(e == cudaErrorMemoryAllocation ? PFAC_ERR_OOM : PFAC_ERR_CUDA);
    } else {
        int32_t *next = layout == 1 ? (int32_t *)m : nullptr;
        int32_t *pid = layout == 1 ? (int32_t *)m + 4 * h->dt.n_states : nullptr;
        int2 *pair = layout == 2 ? (int2 *)m : nullptr;
        rc = pfac::derive_paper_tables(h->dt, next, pid, pair, nullptr);
        if (rc == PFAC_OK) {
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) rc = cuda_fail(e);
        } else {
            rc = cuda_fail(cudaGetLastError());
        }
        if (rc != PFAC_OK) {
            cudaFree(m);
        } else {
            std::lock_guard<std::mutex> lk(h->mu);
            void *&slot = layout == 1 ? h->paper_two : h->paper_pair;
            if (slot) {
                cudaFree(m);                       // another thread got there first
            } else {
                slot = m;
                if (layout == 1) {
                    h->paper.next = next;
                    h->paper.pid = pid;
                } else {
                    h->paper.pair = pair;
                }
            }
        }
    }
    if (cur != h->device) cudaSetDevice(cur);
    return rc;
}

}  // namespace

namespace pfac {

// The packed scan with deferred-walk scratch supplied by the caller instead of the
// per-stream scratch of run_scan. Same checks and the same kernels.
int scan_packed_with_scratch(pfac_table *h, const uint32_t *d_packed, int64_t n_bases, int32_t *d_out_ids,
                             const DeferScratch &scratch, cudaStream_t st)
{
    DeviceProps dp{};
    int rc = check_handle_for_launch(h, &dp);
    if (rc != PFAC_OK) return rc;
    if (n_bases < 0) return fail(PFAC_ERR_INVALID_ARG);
    if (n_bases == 0) return PFAC_OK;
    if (!is_device_ptr(d_packed) || !is_device_ptr(d_out_ids)) return fail(PFAC_ERR_INVALID_ARG);
    const pfac_config c = effective_config(h, true);
    bool tiled = c.kernel == 2 && has_kernel2(h) && aligned16(d_packed) && aligned16(d_out_ids);
    if (tiled) {
        rc = launch_tiled(h->dt, d_packed, true, n_bases, d_out_ids, nullptr, nullptr, 0, nullptr, tiled_config(c),
                          scratch, st, dp);
        if (rc == PFAC_ERR_UNSUPPORTED) tiled = false;
        else if (rc != PFAC_OK) return rc == PFAC_ERR_CUDA ? cuda_fail(cudaGetLastError()) : fail(rc);
    }
    if (!tiled) {
        // kernel 1 keeps no scratch
        rc = launch_walk_rows_any(h->dt, d_packed, true, n_bases, d_out_ids, nullptr, nullptr, 0, nullptr, st, dp);
        if (rc != PFAC_OK) return rc == PFAC_ERR_CUDA ? cuda_fail(cudaGetLastError()) : fail(rc);
    }
    return PFAC_OK;
}

int set_last_error(int code) { return fail(code); }
int set_last_cuda_error(cudaError_t e) { return cuda_fail(e); }

}  // namespace pfac

extern "C" {

int pfac_last_error(void) { return g_last_error; }

const char *pfac_last_cuda_error(void) { return g_last_cuda.c_str(); }

const char *pfac_error_string(int status)
{
    switch (status) {
    case PFAC_OK: return "ok";
    case PFAC_ERR_INVALID_ARG: return "invalid argument";
    case PFAC_ERR_EMPTY_PATTERN: return "empty pattern";
    case PFAC_ERR_BAD_SYMBOL: return "byte outside A, C, G, T";
    case PFAC_ERR_TOO_MANY_STATES: return "too many trie states (2^31 or more)";
    case PFAC_ERR_OOM: return "out of memory";
    case PFAC_ERR_CUDA: return "CUDA runtime error";
    case PFAC_ERR_OVERFLOW: return "more matches than capacity";
    case PFAC_ERR_TIMEOUT: return "bounded device wait ran out";
    case PFAC_ERR_HOST_ONLY: return "handle has no device copy";
    case PFAC_ERR_UNSUPPORTED: return "option not supported for this table";
    case PFAC_ERR_SCRATCH_LIMIT: return "text longer than the allocation-free scan's fixed scratch allows";
    case PFAC_ERR_IO: return "file cannot be opened or read";
    default: return "unknown status";
    }
}

pfac_handle pfac_build_ex(const char *const *patterns, const int32_t *lengths, int32_t n,
                          const pfac_build_opts *opts)
{
    g_last_error = PFAC_OK;
    pfac_build_opts o{};
    if (opts) o = *opts;
    pfac_table *h = new (std::nothrow) pfac_table();
    if (!h) { fail(PFAC_ERR_OOM); return nullptr; }
    if (o.sample < -1 || o.sample > 1) { delete h; fail(PFAC_ERR_INVALID_ARG); return nullptr; }
    int rc = pfac::build_host_tables(patterns, lengths, n, o.filter_b, &h->host, o.sample);
    if (rc != PFAC_OK) { delete h; fail(rc); return nullptr; }
    const pfac::HostTables &T = h->host;
    h->rows_bytes = T.n_states * 16;
    h->skip_bytes = (int64_t)T.skip.size() * 4;
    h->filter_set = (int64_t)T.dense.size() / 4;
    if (!o.host_only) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) { delete h; cuda_fail(e); return nullptr; }
        const size_t rank_bytes = T.rank16.size() * 2 + T.rank32.size() * 4;
        struct Part { const void **dst; const void *src; size_t bytes; } parts[] = {
            {(const void **)&h->dt.rows, T.rows.data(), T.rows.size() * 4},
            {(const void **)&h->dt.out_id, T.out_id.data(), T.out_id.size() * 4},
            {(const void **)&h->dt.skip, T.skip.data(), T.skip.size() * 4},
            // the filter and the sampled screen side by side: one L2 window can cover both
            {(const void **)&h->dt.filter, T.filter.data(), T.filter.size() * 4},
            {(const void **)&h->dt.sample, T.sample.data(), T.sample.size() * 4},
            {(const void **)&h->dt.rank, T.rank_wide ? (const void *)T.rank32.data() : (const void *)T.rank16.data(),
             rank_bytes},
            {(const void **)&h->dt.dense, T.dense.data(), T.dense.size() * 4},
            {(const void **)&h->dt.filter1, T.filter1.data(), T.filter1.size() * 4},
        };
        size_t total = 256;   // status word
        for (auto &p : parts) total += round256(p.bytes);
        h->dbytes = total;
        e = cudaMalloc(&h->dmem, h->dbytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            fail(e == cudaErrorMemoryAllocation ? PFAC_ERR_OOM : PFAC_ERR_CUDA);
            return nullptr;
        }
        uint8_t *base = (uint8_t *)h->dmem;
        h->dt.status = (int32_t *)base;
        e = cudaMemset(h->dt.status, 0, 256);
        size_t off = 256;
        for (auto &p : parts) {
            *p.dst = p.bytes ? (const void *)(base + off) : nullptr;
            if (e == cudaSuccess && p.bytes) e = cudaMemcpy(base + off, p.src, p.bytes, cudaMemcpyHostToDevice);
            off += round256(p.bytes);
        }
        if (e != cudaSuccess) {
            cudaFree(h->dmem);
            delete h;
            cuda_fail(e);
            return nullptr;
        }
        h->device = dev;
        h->dt.n_states = T.n_states;
        h->dt.max_len = T.max_len;
        h->dt.min_len = T.min_len;
        h->dt.filter_b = T.filter_b;
        h->dt.filter1_b = T.filter1_b;
        h->dt.rank_wide = T.rank_wide;
        h->dt.sample_q = T.sample_q;
        h->dt.sample_s = T.sample_s;
        // The device copy is complete; the host keeps rows, ids and levels for export.
        pfac::TableVector<uint32_t>().swap(h->host.skip);
        std::vector<uint32_t>().swap(h->host.filter);
        std::vector<uint16_t>().swap(h->host.rank16);
        std::vector<uint32_t>().swap(h->host.rank32);
        std::vector<uint32_t>().swap(h->host.dense);
        std::vector<uint32_t>().swap(h->host.filter1);
        std::vector<uint32_t>().swap(h->host.sample);
    }
    return h;
}

pfac_handle pfac_build(const char *const *patterns, const int32_t *lengths, int32_t n)
{
    return pfac_build_ex(patterns, lengths, n, nullptr);
}

pfac_handle pfac_build_device(const uint8_t *d_blob, const int64_t *d_offsets, int32_t n,
                              const pfac_build_opts *opts, void *stream)
{
    g_last_error = PFAC_OK;
    pfac_build_opts o{};
    if (opts) o = *opts;
    if (n <= 0 || o.host_only || o.filter_b > 14 || o.sample < -1 || o.sample > 1 || !is_device_ptr(d_blob) ||
        !is_device_ptr(d_offsets)) {
        fail(PFAC_ERR_INVALID_ARG);
        return nullptr;
    }
    pfac::DeviceProps dp{};
    if (device_props(&dp) != PFAC_OK) return nullptr;
    pfac_table *h = new (std::nothrow) pfac_table();
    if (!h) { fail(PFAC_ERR_OOM); return nullptr; }
    pfac::DeviceBuild B;
    int rc = PFAC_OK;
    try {
        rc = pfac::build_device_tables(d_blob, d_offsets, n, o.filter_b, o.sample, (cudaStream_t)stream, dp, &B);
    } catch (const std::bad_alloc &) {
        rc = PFAC_ERR_OOM;
    }
    if (rc != PFAC_OK) {
        delete h;
        if (rc == PFAC_ERR_CUDA) cuda_fail(cudaGetLastError());
        else fail(rc);
        return nullptr;
    }
    h->device = dp.device;
    h->dmem = B.mem;
    h->dbytes = B.bytes;
    h->dt = B.dt;
    pfac::HostTables &T = h->host;
    T.n_states = B.dt.n_states;
    T.n_patterns = n;
    T.max_len = B.dt.max_len;
    T.min_len = B.dt.min_len;
    T.n_duplicates = B.n_duplicates;
    T.level = std::move(B.level);
    T.filter_b = B.dt.filter_b;
    T.filter1_b = B.dt.filter1_b;
    T.rank_wide = B.dt.rank_wide;
    T.sample_q = B.dt.sample_q;
    T.sample_s = B.dt.sample_s;
    h->rows_bytes = B.dt.n_states * 16;
    h->skip_bytes = B.skip_bytes;
    h->filter_set = B.filter_set;
    return h;
}

int pfac_destroy(pfac_handle h)
{
    if (!h) return PFAC_OK;
    forget_handle(h);
    int rc = PFAC_OK;
    if (h->dmem) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != h->device) cudaSetDevice(h->device);
        if (h->paper_two) cudaFree(h->paper_two);
        if (h->paper_pair) cudaFree(h->paper_pair);
        cudaError_t e = cudaFree(h->dmem);
        if (cur != h->device) cudaSetDevice(cur);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    delete h;
    return rc;
}

int pfac_info(pfac_handle h, int64_t *n_states, int32_t *max_len, int64_t *table_bytes)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    if (n_states) *n_states = h->host.n_states;
    if (max_len) *max_len = h->host.max_len;
    if (table_bytes) *table_bytes = (int64_t)h->dbytes;
    return PFAC_OK;
}

int pfac_info_ex(pfac_handle h, pfac_table_info *info)
{
    if (!h || !info) return fail(PFAC_ERR_INVALID_ARG);
    pfac_table_info i{};
    i.n_states = h->host.n_states;
    i.n_patterns = h->host.n_patterns;
    i.max_len = h->host.max_len;
    i.min_len = h->host.min_len;
    i.filter_b = h->host.filter_b;
    i.n_duplicates = h->host.n_duplicates;
    i.table_bytes = (int64_t)h->dbytes;
    i.rows_bytes = h->rows_bytes;
    i.skip_bytes = h->skip_bytes;
    i.filter_set = h->filter_set;
    i.has_skip = h->skip_bytes > 0;
    i.rank_wide = h->host.rank_wide;
    i.device = h->device;
    i.sample_q = h->host.sample_q;
    i.sample_s = h->host.sample_s;
    *info = i;
    return PFAC_OK;
}

int pfac_export(pfac_handle h, int32_t *rows, int32_t *out_id, int64_t *level)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    const pfac::HostTables &T = h->host;
    if (level) memcpy(level, T.level.data(), T.level.size() * 8);
    if (T.rows.empty() && T.n_states > 0) {
        // built on the device: the rows and ids live there only
        cudaError_t e = cudaSuccess;
        if (rows) e = cudaMemcpy(rows, h->dt.rows, (size_t)T.n_states * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && out_id) e = cudaMemcpy(out_id, h->dt.out_id, (size_t)T.n_states * 4, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? PFAC_OK : cuda_fail(e);
    }
    if (rows) memcpy(rows, T.rows.data(), T.rows.size() * 4);
    if (out_id) memcpy(out_id, T.out_id.data(), T.out_id.size() * 4);
    return PFAC_OK;
}

int pfac_export_shortcuts(pfac_handle h, uint32_t *skip, int64_t skip_words, uint32_t *filter, int64_t filter_words,
                          uint32_t *dense, int64_t dense_words)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    const pfac::HostTables &T = h->host;
    const bool on_device = h->device >= 0;       // the host copies were dropped after the upload
    const size_t fwords = T.filter_b ? std::max<size_t>(1, ((size_t)1 << (2 * T.filter_b)) / 32) : 0;
    struct Out { uint32_t *dst; int64_t cap; const void *src; size_t words; } outs[] = {
        {skip, skip_words, on_device ? (const void *)h->dt.skip : T.skip.data(),
         on_device ? (size_t)h->skip_bytes / 4 : T.skip.size()},
        {filter, filter_words, on_device ? (const void *)h->dt.filter : T.filter.data(),
         on_device ? fwords : T.filter.size()},
        {dense, dense_words, on_device ? (const void *)h->dt.dense : T.dense.data(),
         on_device ? (size_t)h->filter_set * 4 : T.dense.size()}};
    for (auto &o : outs)
        if (o.dst && o.cap < (int64_t)o.words) return fail(PFAC_ERR_INVALID_ARG);
    for (auto &o : outs) {
        if (!o.dst || !o.words || !o.src) continue;
        if (on_device) {
            const cudaError_t e = cudaMemcpy(o.dst, o.src, o.words * 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e);
        } else {
            memcpy(o.dst, o.src, o.words * 4);
        }
    }
    return PFAC_OK;
}

int pfac_export_sample(pfac_handle h, uint32_t *sample, int64_t words)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    const int32_t q = h->host.sample_q;
    const size_t have = q ? ((size_t)1 << (2 * q)) / 32 : 0;
    if (sample && words < (int64_t)have) return fail(PFAC_ERR_INVALID_ARG);
    if (!sample || !have) return PFAC_OK;
    if (h->device >= 0) {
        const cudaError_t e = cudaMemcpy(sample, h->dt.sample, have * 4, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? PFAC_OK : cuda_fail(e);
    }
    memcpy(sample, h->host.sample.data(), have * 4);
    return PFAC_OK;
}

int pfac_set_config(pfac_handle h, const pfac_config *cfg)
{
    if (!h) return fail(PFAC_ERR_INVALID_ARG);
    if (cfg) {
        if (cfg->kernel < 0 || cfg->kernel > 2 || cfg->threads < 0 || (cfg->threads & 31) || cfg->threads > 1024 ||
            (cfg->threads > 0 && cfg->threads < 64) || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32 ||
            cfg->stages < 0 || cfg->stages == 1 || cfg->stages > 8 || cfg->walk_loads < 0 ||
            (cfg->lane_offsets != 0 && cfg->lane_offsets != 16 && cfg->lane_offsets != 32) ||
            cfg->table_layout < 0 || cfg->table_layout > 2 || cfg->row_loads < 0 || cfg->row_loads > 2 ||
            cfg->text_smem < 0 || cfg->text_smem > 1 || cfg->zero_writer < 0 || cfg->zero_writer > 4 ||
            cfg->screen < 0 || cfg->screen > 2 || cfg->reserved != 0 || cfg->l2_persist < -1 || cfg->l2_persist > 2)
            return fail(PFAC_ERR_INVALID_ARG);
        if (cfg->kernel == 2 && !(h->skip_bytes > 0 && h->host.filter_b > 0)) return fail(PFAC_ERR_UNSUPPORTED);
        const int rc = ensure_paper_layout(h, cfg->table_layout);
        if (rc != PFAC_OK) return rc;
    }
    std::lock_guard<std::mutex> lk(h->mu);
    h->cfg_set = cfg != nullptr;
    if (cfg) h->cfg = *cfg;
    return PFAC_OK;
}

int pfac_get_config(pfac_handle h, int64_t n_bases, pfac_config *cfg)
{
    (void)n_bases;
    if (!h || !cfg) return fail(PFAC_ERR_INVALID_ARG);
    *cfg = effective_config(h, true);
    return PFAC_OK;
}

int pfac_pack(const uint8_t *d_text, int64_t len, uint32_t *d_packed, int32_t *d_status, int64_t *d_bad,
              void *stream)
{
    if (len < 0) return fail(PFAC_ERR_INVALID_ARG);
    if (len > 0 && (!is_device_ptr(d_text) || !is_device_ptr(d_packed))) return fail(PFAC_ERR_INVALID_ARG);
    if ((d_status && !is_device_ptr(d_status)) || (d_bad && !is_device_ptr(d_bad))) return fail(PFAC_ERR_INVALID_ARG);
    pfac::DeviceProps dp{};
    int rc = device_props(&dp);
    if (rc != PFAC_OK) return rc;
    rc = pfac::launch_pack(d_text, len, d_packed, d_status, d_bad, (cudaStream_t)stream, dp);
    return rc == PFAC_OK ? PFAC_OK : cuda_fail(cudaGetLastError());
}

int pfac_match(pfac_handle h, const uint8_t *d_text, int64_t len, int32_t *d_out_ids, void *stream)
{
    pfac::DeviceProps dp{};
    int rc = check_handle_for_launch(h, &dp);
    if (rc != PFAC_OK) return rc;
    if (len < 0) return fail(PFAC_ERR_INVALID_ARG);
    if (len == 0) return PFAC_OK;
    if (!is_device_ptr(d_text) || !is_device_ptr(d_out_ids)) return fail(PFAC_ERR_INVALID_ARG);
    return run_scan(h, d_text, false, len, d_out_ids, nullptr, nullptr, 0, nullptr, (cudaStream_t)stream, dp);
}

int pfac_match_packed(pfac_handle h, const uint32_t *d_packed, int64_t n_bases, int32_t *d_out_ids, void *stream)
{
    pfac::DeviceProps dp{};
    int rc = check_handle_for_launch(h, &dp);
    if (rc != PFAC_OK) return rc;
    if (n_bases < 0) return fail(PFAC_ERR_INVALID_ARG);
    if (n_bases == 0) return PFAC_OK;
    if (!is_device_ptr(d_packed) || !is_device_ptr(d_out_ids)) return fail(PFAC_ERR_INVALID_ARG);
    return run_scan(h, d_packed, true, n_bases, d_out_ids, nullptr, nullptr, 0, nullptr, (cudaStream_t)stream, dp);
}

static int match_list(pfac_handle h, const uint32_t *d_packed, int64_t n_bases, int64_t *d_offsets, int32_t *d_ids,
                      int64_t capacity, int64_t *d_count, void *stream, bool all_matches)
{
    pfac::DeviceProps dp{};
    int rc = check_handle_for_launch(h, &dp);
    if (rc != PFAC_OK) return rc;
    if (n_bases < 0 || capacity < 0 || !is_device_ptr(d_count)) return fail(PFAC_ERR_INVALID_ARG);
    if (capacity > 0 && (!is_device_ptr(d_offsets) || !is_device_ptr(d_ids))) return fail(PFAC_ERR_INVALID_ARG);
    if (n_bases > 0 && !is_device_ptr(d_packed)) return fail(PFAC_ERR_INVALID_ARG);
    if (n_bases == 0) {
        cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), (cudaStream_t)stream);
        return e == cudaSuccess ? PFAC_OK : cuda_fail(e);
    }
    int64_t *offs = d_offsets ? d_offsets : (int64_t *)d_count;   // never written when capacity == 0
    int32_t *ids = d_ids ? d_ids : (int32_t *)d_count;
    return run_scan(h, d_packed, true, n_bases, nullptr, offs, ids, capacity, d_count, (cudaStream_t)stream, dp,
                    all_matches);
}

int pfac_match_compact(pfac_handle h, const uint32_t *d_packed, int64_t n_bases, int64_t *d_offsets, int32_t *d_ids,
                       int64_t capacity, int64_t *d_count, void *stream)
{
    return match_list(h, d_packed, n_bases, d_offsets, d_ids, capacity, d_count, stream, false);
}

int pfac_match_all(pfac_handle h, const uint32_t *d_packed, int64_t n_bases, int64_t *d_offsets, int32_t *d_ids,
                   int64_t capacity, int64_t *d_count, void *stream)
{
    return match_list(h, d_packed, n_bases, d_offsets, d_ids, capacity, d_count, stream, true);
}

int pfac_device_status(pfac_handle h, int32_t *status, void *stream)
{
    if (!h || !status) return fail(PFAC_ERR_INVALID_ARG);
    if (h->device < 0) return fail(PFAC_ERR_HOST_ONLY);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->dt.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dt.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    *status = v;
    return PFAC_OK;
}

int pfac_match_batched(const pfac_handle *sets, int32_t n_sets, const uint8_t *d_texts, int64_t text_len,
                       const int64_t *d_read_offsets, const int32_t *d_read_set, int32_t n_reads, int32_t *d_out_ids,
                       void *stream)
{
    if (!sets || n_sets < 1 || n_sets > 65535 || text_len < 0 || n_reads < 0) return fail(PFAC_ERR_INVALID_ARG);
    pfac::DeviceProps dp{};
    for (int32_t i = 0; i < n_sets; i++) {
        int rc = check_handle_for_launch(sets[i], &dp);
        if (rc != PFAC_OK) return rc;
        if (!has_kernel2(sets[i])) return fail(PFAC_ERR_UNSUPPORTED);
    }
    if (text_len == 0 || n_reads == 0) return PFAC_OK;
    if (!is_device_ptr(d_texts) || !is_device_ptr(d_read_offsets) || !is_device_ptr(d_read_set) ||
        !is_device_ptr(d_out_ids))
        return fail(PFAC_ERR_INVALID_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    const pfac::DeviceTable *d_sets = nullptr;
    int rc = set_descriptors(sets, n_sets, dp.device, &d_sets);
    if (rc != PFAC_OK) return rc;
    const int64_t defer_cap = defer_capacity(text_len);
    void *scratch = nullptr;
    rc = batch_scratch(dp.device, st, pfac::batch_scratch_bytes(text_len, n_reads, defer_cap), &scratch);
    if (rc != PFAC_OK) return rc;
    // The pass takes its launch shape from the configuration of sets[0]: offsets per
    // lane, walk_loads, and threads x ctas_per_sm threads per SM in 256-thread blocks.
    const pfac_config c = effective_config(sets[0], false);
    pfac::BatchConfig bc{};
    bc.lane_offsets = c.lane_offsets;
    bc.blocks_per_sm = (int32_t)std::max<int64_t>(1, (int64_t)c.threads * c.ctas_per_sm / 256);
    bc.walk_loads = c.walk_loads;
    rc = pfac::launch_batched(d_sets, n_sets, d_texts, text_len, d_read_offsets, d_read_set, n_reads, d_out_ids,
                              scratch, defer_cap, bc, st, dp);
    return rc == PFAC_OK ? PFAC_OK : cuda_fail(cudaGetLastError());
}

int pfac_debug_timeout_probe(int32_t *d_status, int64_t limit_ns, void *stream)
{
    if (!is_device_ptr(d_status) || limit_ns <= 0) return fail(PFAC_ERR_INVALID_ARG);
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = pfac::launch_timeout_probe(d_status, limit_ns, (cudaStream_t)stream);
    return rc == PFAC_OK ? PFAC_OK : cuda_fail(cudaGetLastError());
}

}  // extern "C"
