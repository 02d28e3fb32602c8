// Device-side building blocks shared by the scan kernels (pfac_kernels.cu) and the
// batched kernels (pfac_batched.cu): PTX wrappers (mbarriers, bulk copies, cache
// policies), base codes and byte-parallel packing, the deferred-walk record, result
// sinks, the skip-entry walk, the prefix-filter test and the warp-level lane batch.
#pragma once

#include <stdint.h>

#include <type_traits>

#include <cooperative_groups.h>

#include "../../include/pfac.h"
#include "pfac_internal.h"

namespace pfac {


// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the given phase of an mbarrier, giving up after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((int64_t)(global_timer_ns() - t0) > limit_ns) return false;
    }
}

// Bulk (TMA) copy global -> shared, completion counted on an mbarrier. Source and
// destination 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Bulk (TMA) copy shared -> global with an L2 eviction-priority hint.
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes, uint64_t policy)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(src), "r"(bytes), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void record_error(int32_t *status, int32_t code)
{
    if (status) atomicCAS(status, PFAC_OK, code);
}

// ---------------------------------------------------------------------------
// Base codes. A=0x41, C=0x43, G=0x47, T=0x54: ((b >> 1) & 3) ^ ((b >> 2) & 1)
// maps them to 0, 1, 2, 3.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int base_code_or_neg(uint32_t b)
{
    const bool ok = (b == 0x41u) | (b == 0x43u) | (b == 0x47u) | (b == 0x54u);
    const int c = (int)(((b >> 1) & 3u) ^ ((b >> 2) & 1u));
    return ok ? c : -1;
}

// Four ASCII bytes -> four 2-bit codes in the low 8 bits (a byte outside ACGT codes as
// A), plus a 4-bit mask of bytes that are not A, C, G or T. Byte-parallel arithmetic:
//   t      the code each byte would have if it were a base (see base_code_or_neg);
//   c8     t's four codes gathered into one byte by one multiply (the products of
//          different bytes land below bit 24 or above bit 31, without carries);
//   sel    the codes spread to one nibble each, a byte-permute selector that picks the
//          byte each code stands for out of "ACGT";
//   diff   zero exactly in the bytes that equal that byte, i.e. are bases;
//   nz     bit 7 of each nonzero byte of diff (the zero-byte test), gathered into 4 bits
//          by a second multiply.
// Checked against the per-byte definition for all 2^32 inputs.
__device__ __forceinline__ uint32_t pack4(uint32_t x, uint32_t *bad4)
{
    const uint32_t t = ((x >> 1) & 0x03030303u) ^ ((x >> 2) & 0x01010101u);
    const uint32_t c8 = (t * 0x01041040u) >> 24;
    const uint32_t y = (c8 | (c8 << 4)) & 0x0F0Fu;
    const uint32_t sel = (y | (y << 2)) & 0x3333u;
    const uint32_t diff = x ^ __byte_perm(0x54474341u, 0u, sel);
    const uint32_t nz = (((diff & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | diff) & 0x80808080u;
    *bad4 = (nz * 0x00204081u) >> 28;
    return ((t & ~((nz >> 7) * 0xFFu)) * 0x01041040u) >> 24;
}

// Four bytes' codes (c8, as in pack4) and the XOR of the bytes with the bases those
// codes stand for: zero exactly in the bytes that are A, C, G or T. Unlike pack4, the
// code of a byte outside ACGT is left as the arithmetic gives it: scans never read a
// code at a position their mask marks (walks stop before it, and the filter bits of
// windows that contain it are masked off).
__device__ __forceinline__ uint32_t codes4(uint32_t x, uint32_t *diff)
{
    const uint32_t t = ((x >> 1) & 0x03030303u) ^ ((x >> 2) & 0x01010101u);
    const uint32_t c8 = (t * 0x01041040u) >> 24;
    const uint32_t y = (c8 | (c8 << 4)) & 0x0F0Fu;
    const uint32_t sel = (y | (y << 2)) & 0x3333u;
    *diff = x ^ __byte_perm(0x54474341u, 0u, sel);
    return c8;
}

// The 4-bit mask of the nonzero bytes of d.
__device__ __forceinline__ uint32_t nonzero_bytes4(uint32_t d)
{
    const uint32_t nz = (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & 0x80808080u;
    return (nz * 0x00204081u) >> 28;
}

// pack16 for scans (codes as codes4 leaves them); the per-byte mask is worked out only
// when some byte of the sixteen is not a base.
__device__ __forceinline__ uint32_t pack16_scan(uint4 v, uint32_t *bad16)
{
    uint32_t d0, d1, d2, d3;
    const uint32_t c0 = codes4(v.x, &d0), c1 = codes4(v.y, &d1), c2 = codes4(v.z, &d2), c3 = codes4(v.w, &d3);
    uint32_t b = 0;
    if (d0 | d1 | d2 | d3)
        b = nonzero_bytes4(d0) | (nonzero_bytes4(d1) << 4) | (nonzero_bytes4(d2) << 8) | (nonzero_bytes4(d3) << 12);
    *bad16 = b;
    return c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
}

// Sixteen ASCII bytes -> one packed word, plus a 16-bit mask of invalid bytes.
__device__ __forceinline__ uint32_t pack16(uint4 v, uint32_t *bad16)
{
    uint32_t b0, b1, b2, b3;
    const uint32_t c0 = pack4(v.x, &b0), c1 = pack4(v.y, &b1), c2 = pack4(v.z, &b2), c3 = pack4(v.w, &b3);
    *bad16 = b0 | (b1 << 4) | (b2 << 8) | (b3 << 12);
    return c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
}

struct DeferItem {
    long long gp;      // text offset of the walk
    uint32_t s;        // state reached
    uint32_t best;     // deepest terminal state passed (0 = none)
    uint32_t q_set;    // bases consumed (low 16 bits) | table index in a batch (high 16 bits)
    int32_t span;      // bases from gp to the end of the walk's text (or read), capped at 2^31-1
};

// Wait for an mbarrier phase, giving up after limit_ns or when another warp of the
// CTA has raised the abort flag. Returns false if it gave up.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, int64_t limit_ns,
                                              volatile uint32_t *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(global_timer_ns() - t0) > limit_ns) {
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory loads the compiler keeps in program order with the other asm
// statements (the stage words, read before the stage is released).
__device__ __forceinline__ uint32_t lds_u32(const void *p)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}

__device__ __forceinline__ uint4 lds_v4(const void *p)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_addr(p))
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_global_v4_hint(int32_t *p, int4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// Mask of the first L 2-bit bases (L = 1..16).
__device__ __forceinline__ uint32_t base_mask(uint32_t L)
{
    return L >= 16 ? 0xFFFFFFFFu : ((1u << (2 * L)) - 1u);
}

// Sixteen bases of the text from position pos (packed or ASCII) read from global
// memory, with a mask of the bases that cannot be read (at or past `end`, ASCII bytes
// outside ACGT, or bases marked in the optional invalid-base bitmap of packed text).
template <bool PACKED>
__device__ __forceinline__ uint32_t text16(const void *__restrict__ text, const uint32_t *__restrict__ invalid,
                                           int64_t end, int64_t pos, uint32_t *bad)
{
    const int64_t rem = end - pos;
    uint32_t b = rem >= 16 ? 0u : (rem > 0 ? (0xFFFFu << rem) & 0xFFFFu : 0xFFFFu);
    uint32_t w = 0;
    if (PACKED) {
        const int64_t wi = pos >> 4;
        const int64_t n_words = (end + 15) >> 4;
        const uint32_t lo = wi < n_words ? __ldg((const uint32_t *)text + wi) : 0u;
        const uint32_t hi = wi + 1 < n_words ? __ldg((const uint32_t *)text + wi + 1) : 0u;
        w = __funnelshift_r(lo, hi, (uint32_t)(pos & 15) * 2);
        if (invalid) {
            const int64_t bi = pos >> 5;
            const int64_t n_bw = (end + 31) >> 5;
            const uint32_t blo = bi < n_bw ? __ldg(invalid + bi) : 0xFFFFFFFFu;
            const uint32_t bhi = bi + 1 < n_bw ? __ldg(invalid + bi + 1) : 0xFFFFFFFFu;
            b |= __funnelshift_r(blo, bhi, (uint32_t)(pos & 31)) & 0xFFFFu;
        }
    } else {
        for (int i = 0; i < 16 && pos + i < end; i++) {
            const int c = base_code_or_neg(__ldg((const uint8_t *)text + pos + i));
            if (c < 0) b |= 1u << i;
            else w |= (uint32_t)c << (2 * i);
        }
    }
    *bad = b;
    return w;
}

// Where results go: the dense output array (whose slots already hold 0) or the match
// list, plus the deferred-walk list.
struct Sink {
    int32_t *out;
    int64_t *c_off;
    int32_t *c_ids;
    int64_t cap;
    unsigned long long *count;
    DeferItem *defer;
    int64_t defer_cap;
    unsigned long long *defer_count;
    int32_t *status;           // device status word: PFAC_ERR_OVERFLOW when the list is full
};

// Places for the lanes that reach this call together (any subset of the warp): one
// atomicAdd on *counter for all of them (ballot of the active lanes, popcount, the
// leader's add, a shuffle of the base), then the lanes' ranks among them. Returns this
// lane's place.
__device__ __forceinline__ unsigned long long warp_aggregated_slot(unsigned long long *counter)
{
    namespace cg = cooperative_groups;
    const cg::coalesced_group g = cg::coalesced_threads();
    unsigned long long base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned long long)g.size());
    return g.shfl(base, 0) + g.thread_rank();
}

// Record a non-zero result. In the match list the lanes that find matches together take
// their places with one atomic; a match past the capacity is counted but not written,
// and PFAC_ERR_OVERFLOW goes to the status word.
template <bool COMPACT>
__device__ __forceinline__ void emit_match(const Sink &K, int64_t gp, int32_t v)
{
    if (!v) return;
    if (COMPACT) {
        const unsigned long long k = warp_aggregated_slot(K.count);
        if ((int64_t)k < K.cap) {
            K.c_off[k] = gp;
            K.c_ids[k] = v;
        } else {
            record_error(K.status, PFAC_ERR_OVERFLOW);
        }
    } else {
        K.out[gp] = v;
    }
}

// Continue a walk from state s with `q` bases consumed, reading the text from global
// memory up to `end` (deferred walks, and walks the deferred list had no room for).
// Returns the pattern id (0 if none). ALL: every terminal state reached from here goes
// to the match list *K instead (each is met once, at the top of the loop) and 0 is
// returned.
template <bool PACKED, bool ALL = false>
__device__ int32_t walk_global(const DeviceTable &T, const void *__restrict__ text,
                               const uint32_t *__restrict__ invalid, int64_t end, int64_t gp, uint32_t s, int q,
                               uint32_t best, const Sink *K = nullptr)
{
    uint4 e = __ldg(T.skip + s);
    for (;;) {
        if (e.y & kSkipSelfTerm) {
            if (ALL) emit_match<true>(*K, gp, __ldg(T.out_id + s));
            else best = s;
        }
        const uint32_t L = e.y & kSkipLenMask;
        uint32_t bad;
        const uint32_t win = text16<PACKED>(text, invalid, end, gp + q, &bad);
        const uint32_t need = L ? L : 1u;
        if (bad & ((need >= 16) ? 0xFFFFu : ((1u << need) - 1u))) break;   // cannot read the next step
        if (L) {
            if ((win ^ e.x) & base_mask(L)) break;
            q += (int)L;
            s = e.z;
            if (!ALL && (e.y & kSkipTargetTerm)) best = s;
        } else {
            const uint32_t c = win & 3u;
            if (!((e.w >> c) & 1u)) break;
            s = (e.w >> kNodeFirstShift) + __popc(e.w & ((1u << c) - 1u));
            q++;
        }
        e = __ldg(T.skip + s);
    }
    return (!ALL && best) ? __ldg(T.out_id + best) : 0;
}

// Mask of positions j < 32 (bit j) such that bits j .. j+w-1 of `bad` are all clear.
__device__ __forceinline__ uint32_t clear_runs(uint64_t bad, int w)
{
    uint64_t t = bad;
    int have = 1;
    while (have * 2 <= w) {
        t |= t >> have;
        have *= 2;
    }
    if (have < w) t |= t >> (w - have);
    return (uint32_t)(~t);
}

// Sixteen bases of a lane's 64-base window from position p (0 <= p < 64); bases past
// the window read as 0.
__device__ __forceinline__ uint32_t window_at(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, int p)
{
    const int w = p >> 4;
    const uint32_t lo = w == 0 ? x0 : (w == 1 ? x1 : (w == 2 ? x2 : x3));
    const uint32_t hi = w == 0 ? x1 : (w == 1 ? x2 : (w == 2 ? x3 : 0u));
    return __funnelshift_r(lo, hi, (uint32_t)(p & 15) * 2);
}

// Prefix-filter bits of a lane's LW offsets: bit j is the filter bit of the b bases
// from offset j (window bases j .. j+b-1; x0, x1, x2 hold window bases 0 .. 47). A
// clear bit means the walk from offset j ends before depth b with no pattern on the
// way. The shared-memory copy of the filter (sf) holds each word bit-reversed: the bit of
// b-mer w is bit 31 - (w mod 32) of word w / 32. With that copy at shared-memory offset 0
// and b >= 3, the byte address of a filter word is the window shifted and masked, a
// left rotate by the window (whose low five bits are w mod 32, taken as they are) brings
// the bit to the top, and a funnel shift moves it into the result: two shifts per
// offset after the load.
template <bool FSMEM, int LW>
__device__ __forceinline__ uint32_t filter_bits(const DeviceTable &T, const uint32_t *sf, uint32_t x0, uint32_t x1,
                                                uint32_t x2, uint32_t bmask)
{
    uint32_t pend = 0;
    if (FSMEM && bmask >= 31u) {
        const uint32_t amask = (bmask >> 3) & ~3u;
        const uint8_t *fb = reinterpret_cast<const uint8_t *>(sf);
#pragma unroll
        for (int j = LW - 1; j >= 0; j--) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t word = *reinterpret_cast<const uint32_t *>(fb + ((win >> 3) & amask));
            pend = __funnelshift_l(__funnelshift_l(word, word, win), pend, 1);
        }
    } else if (!FSMEM && bmask >= 31u) {
        // global memory, words as stored: a left rotate by 31 - (w mod 32), the window's
        // complement taken as it is, brings the bit of b-mer w to the top
#pragma unroll
        for (int j = LW - 1; j >= 0; j--) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t word = __ldg(T.filter + ((win & bmask) >> 5));
            pend = __funnelshift_l(__funnelshift_l(word, word, ~win), pend, 1);
        }
    } else {
#pragma unroll
        for (int j = 0; j < LW; j++) {
            const uint32_t win = j < 16 ? __funnelshift_r(x0, x1, 2 * j) : __funnelshift_r(x1, x2, 2 * (j - 16));
            const uint32_t kmer = win & bmask;
            const uint32_t word = FSMEM ? __brev(sf[kmer >> 5]) : __ldg(T.filter + (kmer >> 5));
            pend |= ((word >> (kmer & 31u)) & 1u) << j;
        }
    }
    return pend;
}

// Zeros for a warp-batch's valid offsets. Any lane may store any of the warp's zeros.
// When the whole batch is valid its 32*LW outputs are contiguous from warp_base, and
// each 16-byte store instruction covers 512 contiguous bytes (lane l at warp_base +
// 4l + 128v): full sectors, where a lane writing its own offsets would leave every
// sector half-written by two instructions.
template <int LW>
__device__ __forceinline__ void zero_batch(const Sink &K, int64_t warp_base, int lane, uint32_t valid, bool vec_ok,
                                           uint64_t pol)
{
    const uint32_t all = LW == 32 ? 0xFFFFFFFFu : ((1u << LW) - 1u);
    const int64_t gp0 = warp_base + (int64_t)lane * LW;
    const int4 z = make_int4(0, 0, 0, 0);
    if (__all_sync(0xFFFFFFFFu, vec_ok && valid == all)) {
        int32_t *o = K.out + warp_base + 4 * lane;
#pragma unroll
        for (int v = 0; v < LW / 4; v++) st_global_v4_hint(o + 128 * v, z, pol);
    } else if (vec_ok && valid == all) {
        int32_t *o = K.out + gp0;
#pragma unroll
        for (int v = 0; v < LW / 4; v++) st_global_v4_hint(o + 4 * v, z, pol);
    } else if (valid) {
        for (int j = 0; j < LW; j++)
            if ((valid >> j) & 1u) K.out[gp0 + j] = 0;
    }
}

// The walk from one offset gp that passed the filter (or could not be tested). The
// text from gp is window bases j, j+1, ... of x0..x3 (64 bases), of which wlim can be
// read; `ends` when the text (or the run of readable bases) really stops there rather
// than the window. `fast`: the b bases from gp are readable, so the walk starts at the
// dense entry of their b-mer (unless that entry is marked special) at depth b; else at
// the root. It goes on through skip entries inside the window with at most walk_loads
// dependent table loads; a longer walk is deferred to the tail kernel.
template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, bool ALL = false>
__device__ __forceinline__ void walk_item(const DeviceTable &T, const Sink &K, const uint32_t *sf, const void *srank,
                                          int walk_loads, uint32_t set_index, const void *text,
                                          const uint32_t *invalid, int64_t end, int64_t gp, uint32_t x0, uint32_t x1,
                                          uint32_t x2, uint32_t x3, int j, int wlim, bool ends, bool fast)
{
    using RankT = typename std::conditional<RANK16, uint16_t, uint32_t>::type;
    const int B = T.filter_b;
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    uint32_t s = 0, best = 0;
    int q = 0;
    uint4 e;
    bool from_root = true;
    if (fast) {
        const uint32_t kmer = window_at(x0, x1, x2, x3, j) & bmask;
        const uint32_t widx = kmer >> 5;
        const uint32_t word = FSMEM ? __brev(sf[widx]) : __ldg(T.filter + widx);
        uint32_t base_rank;
        if (srank) base_rank = (uint32_t)reinterpret_cast<const RankT *>(srank)[widx];
        else if (T.rank_wide) base_rank = __ldg(reinterpret_cast<const uint32_t *>(T.rank) + widx);
        else base_rank = (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(T.rank) + widx);
        const uint32_t rk = base_rank + __popc(word & ((1u << (kmer & 31u)) - 1u));
        e = __ldg(T.dense + rk);
        if (!(e.y & kSkipSpecial)) {
            from_root = false;
            q = B;
        }
    }
    if (from_root) e = __ldg(T.skip);
    bool defer = false;
    for (int loads = 1;; loads++) {
        // every state the walk enters is met here once (ALL lists each terminal one)
        if (e.y & kSkipSelfTerm) {
            if (ALL) emit_match<true>(K, gp, __ldg(T.out_id + s));
            else best = s;
        }
        const uint32_t L = e.y & kSkipLenMask;
        const int need = L ? (int)L : 1;
        if (q + need > wlim) {
            defer = !ends;     // the window ran out before the text did
            break;
        }
        const uint32_t win = window_at(x0, x1, x2, x3, j + q);
        if (L) {
            if ((win ^ e.x) & base_mask(L)) break;
            q += (int)L;
            s = e.z;
            if (!ALL && (e.y & kSkipTargetTerm)) best = s;
        } else {
            const uint32_t c = win & 3u;
            if (!((e.w >> c) & 1u)) break;
            s = (e.w >> kNodeFirstShift) + __popc(e.w & ((1u << c) - 1u));
            q++;
        }
        if (loads >= walk_loads) {
            defer = true;      // the tail kernel takes it from state s
            break;
        }
        e = __ldg(T.skip + s);
    }
    if (defer) {
        // long walk: finish it in the tail kernel (or here if the list is full)
        const unsigned long long di = warp_aggregated_slot(K.defer_count);
        if ((int64_t)di < K.defer_cap) {
            DeferItem it;
            it.gp = gp;
            it.s = s;
            it.best = ALL ? 0u : best;
            it.q_set = (uint32_t)q | (set_index << 16);
            it.span = (int32_t)min(end - gp, (int64_t)0x7FFFFFFF);
            K.defer[di] = it;
        } else {
            emit_match<COMPACT>(K, gp, walk_global<PACKED, ALL>(T, text, invalid, end, gp, s, q, best, &K));
        }
    } else if (!ALL && best) {
        emit_match<COMPACT>(K, gp, __ldg(T.out_id + best));
    }
}

// One warp-batch: lane `lane` owns the LW offsets gp0 = warp_base + lane*LW .. +LW-1
// and holds the 64 bases from gp0 in x0..x3 with `bad` marking the bases that cannot
// be read (past the end of its text or read, or not A/C/G/T); `valid` marks the
// offsets this call must answer. Every offset's prefix-filter bit is tested; the
// offsets that pass are spread over the warp (item r of the warp, in lane order then
// offset order, goes to lane r mod 32 in round r / 32, with the owner's window by
// shuffle) and walked at once. Used for ASCII text and for batched reads.
// sf / srank: filter and rank index in shared memory, or nullptr for global memory.
template <bool PACKED, bool COMPACT, bool FSMEM, bool RANK16, int LW, bool ALL = false>
__device__ __forceinline__ void scan_lane_batch(const DeviceTable &T, const Sink &K, const uint32_t *sf,
                                                const void *srank, int walk_loads, uint32_t set_index,
                                                const void *text, const uint32_t *invalid, int64_t end,
                                                int64_t warp_base, int lane, uint32_t x0, uint32_t x1, uint32_t x2,
                                                uint32_t x3, uint64_t bad, uint32_t valid, bool vec_ok, uint64_t pol)
{
    const int B = T.filter_b;
    const uint32_t bmask = (uint32_t)((1ull << (2 * B)) - 1ull);
    const uint32_t fast = clear_runs(bad, B) & valid;   // the b-mer is readable
    uint32_t pend = filter_bits<FSMEM, LW>(T, sf, x0, x1, x2, bmask) & fast;
    // Offsets whose b bases cannot all be read (a byte outside ACGT, or the end of the
    // text or read, within b bases) walk from the root, unless fewer bases than the
    // shortest pattern can be read: then no pattern starts there.
    if (T.min_len < B) pend |= valid & ~fast & clear_runs(bad, T.min_len);

    if (!COMPACT) zero_batch<LW>(K, warp_base, lane, valid, vec_ok, pol);
    // The zeros above were stored by one lane and a match found below is stored by
    // whichever lane walks it, often another. The warp barrier orders the first before
    // the second.
    __syncwarp();

    const uint32_t cnt = __popc(pend);
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += o;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (uint32_t r0 = 0; r0 < total; r0 += 32) {
        const uint32_t r = r0 + lane;
        // owner = the last lane whose first item is <= r
        int owner = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, owner + step);
            if (e <= r) owner += step;
        }
        const uint32_t om = __shfl_sync(0xFFFFFFFFu, pend, owner);
        const uint32_t oe = __shfl_sync(0xFFFFFFFFu, excl, owner);
        const uint32_t ofast = __shfl_sync(0xFFFFFFFFu, fast, owner);
        const uint32_t ox0 = __shfl_sync(0xFFFFFFFFu, x0, owner);
        const uint32_t ox1 = __shfl_sync(0xFFFFFFFFu, x1, owner);
        const uint32_t ox2 = __shfl_sync(0xFFFFFFFFu, x2, owner);
        const uint32_t ox3 = __shfl_sync(0xFFFFFFFFu, x3, owner);
        const uint32_t obad_lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)bad, owner);
        const uint32_t obad_hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(bad >> 32), owner);
        if (r >= total) continue;
        // the (r - oe)-th set bit of the owner's mask (r - oe < popcount by construction)
        uint32_t m = om;
        for (uint32_t i = r - oe; i > 0; i--) m &= m - 1u;
        const int j = (__ffs(m) - 1) & (LW - 1);
        const int64_t gp = warp_base + (int64_t)owner * LW + j;
        const uint64_t badj = (((uint64_t)obad_hi << 32) | obad_lo) >> j;
        // bases readable from the window; `ends` when the text (or the run of ACGT
        // bytes) really stops there rather than the window
        const int wlim = badj ? __ffsll((long long)badj) - 1 : 64 - j;
        walk_item<PACKED, COMPACT, FSMEM, RANK16, ALL>(T, K, sf, srank, walk_loads, set_index, text, invalid, end, gp,
                                                  ox0, ox1, ox2, ox3, j, wlim, badj != 0, (ofast >> j) & 1u);
    }
}

}  // namespace pfac
