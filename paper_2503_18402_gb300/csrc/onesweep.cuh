// onesweep.cuh -- single-pass radix passes and a single-pass exclusive scan,
// both built on decoupled look-back (Merrill & Garland, "Single-pass Parallel
// Prefix Scan with Decoupled Look-back", 2016; the radix form follows
// Adinets & Merrill, "Onesweep: A Faster Least Significant Digit Radix Sort
// for GPUs", 2022).  Used by the binning stages, where the classic
// histogram -> scan -> scatter passes spent most of their time in launch
// gaps.
//
// A pass is one kernel.  Each CTA takes a tile number from a counter when it
// starts, ranks its RS_TILE keys by digit (warp match_any within warp-owned
// segments, so the pass is stable), publishes its per-digit totals, and sums
// the totals of the tiles before it by walking back over their published
// words until one holds an inclusive prefix.  A CTA only waits on tiles taken
// by CTAs that started before it and that never wait on a later tile, so every
// wait ends; each is bounded all the same, and a wait that gives up records
// DG_ERR_TIMEOUT and carries on with what it has.
//
// The global start of each digit comes from the histograms of all passes,
// counted in one read of the keys before the first pass (a one-CTA kernel
// scans them).  Look-back words are cleared one pass ahead: the
// histogram kernel clears the first pass's words, pass p clears the words of
// pass p + 1 (the two alternate between two regions), so no pass needs a
// separate clearing launch.
#pragma once

#include "radix.cuh"

namespace dg {
namespace {

constexpr int OS_MAXPASS = 6;
constexpr uint64_t kLbAgg = 1ull << 62;   // word holds the tile's own total
constexpr uint64_t kLbInc = 2ull << 62;   // word holds the inclusive prefix
constexpr uint64_t kLbCount = (1ull << 62) - 1;
constexpr int kLbPolls = 1 << 20;         // polls of one word before giving up

// Per-call control block, zeroed by the caller before the histogram kernel.
// The histogram CTAs add their counts into one of OS_HCOPIES copies (by CTA
// index) so that thousands of CTAs do not queue on the same 256 words.
constexpr int OS_HCOPIES = 16;
struct OsCtl {
    uint32_t ctr[OS_MAXPASS];              // tile counters of the passes (and of the scan)
    int32_t err;                           // DG_ERR_TIMEOUT once a wait gave up
    uint32_t hist[OS_MAXPASS][OS_HCOPIES][1 << RS_MAXBITS];
    uint32_t base[OS_MAXPASS][1 << RS_MAXBITS];  // exclusive scan of the summed counts
};

// This CTA's copy of pass p's counts.
__device__ __forceinline__ uint32_t* os_hist(OsCtl* ctl, int p)
{
    return ctl->hist[p][blockIdx.x % OS_HCOPIES];
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum of the counts the tiles before tile t published in column d of a
// [tiles][stride] word array, up to and including the nearest inclusive
// word.  The words of OS_WINDOW predecessors are read at once: when every
// tile publishes at about the same time, the walk back to an inclusive word
// takes about sqrt(2 t / OS_WINDOW) round trips instead of sqrt(2 t).
constexpr int OS_WINDOW = 16;
__device__ inline uint64_t os_lookback(const uint64_t* look, long long t, int stride, int d, int* err,
                                       int max_polls = kLbPolls)
{
    uint64_t sum = 0;
    long long j = t;  // the window covers tiles j - OS_WINDOW .. j - 1
    int polls = 0;
    while (j > 0) {
        uint64_t w[OS_WINDOW];
#pragma unroll
        for (int q = 0; q < OS_WINDOW; ++q)
            w[q] = j - 1 - q >= 0 ? ld_relaxed(look + (j - 1 - q) * stride + d) : kLbInc;
        int used = OS_WINDOW;
#pragma unroll
        for (int q = 0; q < OS_WINDOW; ++q) {
            if (used < OS_WINDOW) break;
            const uint64_t st = w[q] >> 62;
            if (st == 0) {
                used = q;  // tile j - 1 - q has not published yet: read again from there
            } else {
                sum += w[q] & kLbCount;
                if (st == 2) return sum;
            }
        }
        j -= used;
        if (used < OS_WINDOW) {
            if (++polls > max_polls) {
                atomicExch(err, DG_ERR_TIMEOUT);
                return sum;
            }
            __nanosleep(32);
        }
    }
    return sum;
}

// One CTA of 256 threads, launched after the histogram kernel: sums the
// copies and writes the exclusive scan of each pass's counts to ctl->base.
// (A separate launch instead of a last-CTA step: that step needs a fence
// that makes every histogram CTA wait for its own output writes.)
__global__ void __launch_bounds__(256) k_os_base(OsCtl* ctl, int npass)
{
    __shared__ uint32_t sm[33];
    for (int p = 0; p < npass; ++p) {
        uint32_t c = 0;
#pragma unroll
        for (int q = 0; q < OS_HCOPIES; ++q) c += ctl->hist[p][q][threadIdx.x];
        uint32_t tot;
        const uint32_t ex = block_excl_scan<uint32_t>(c, sm, &tot);
        ctl->base[p][threadIdx.x] = ex;
    }
}

struct OsPass {
    uint64_t* look;        // [tiles][mask + 1] look-back words of this pass
    uint64_t* look_next;   // the next pass's words, cleared here (null after the last pass)
    int next_nbins;        // digits of the next pass
    uint32_t* ctr;         // this pass's tile counter (zero before the launch)
    const uint32_t* base;  // global start of each digit
    int* err;
    int shift;
    uint32_t mask;
};

// Key sources of a pass: item i of the input gives (key, value).
struct SrcKV {
    const uint32_t* k;
    const uint32_t* v;
    __device__ void operator()(long long i, uint32_t& key, uint32_t& val) const { key = k[i]; val = v[i]; }
};

// One stable pass on digit (key >> shift) & mask; kout may be null (values only).
template <class Src>
__global__ void __launch_bounds__(RS_THREADS, 4)
k_os_pass(Src src, uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const long long* n_dev,
          long long n_cap, OsPass ps)
{
    __shared__ uint32_t cnt[RS_WARPS][1 << RS_MAXBITS];
    __shared__ uint32_t dstart[1 << RS_MAXBITS];
    __shared__ uint32_t gstart[1 << RS_MAXBITS];
    __shared__ uint32_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ uint32_t scan_sm[33];
    __shared__ uint32_t s_t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long n = eff_count(n_dev, n_cap);
    if (threadIdx.x == 0) s_t = atomicAdd(ps.ctr, 1u);
    __syncthreads();
    const long long t = s_t;
    const long long base = t * RS_TILE;
    if (base >= n) return;
    const int nbins = (int)ps.mask + 1;
    if (ps.look_next)
        for (int d = threadIdx.x; d < ps.next_nbins; d += RS_THREADS) ps.look_next[t * ps.next_nbins + d] = 0;
    const long long seg = base + (long long)warp * (32 * RS_IPT);
    for (int d = lane; d < nbins; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    uint32_t key[RS_IPT], val[RS_IPT], rank[RS_IPT];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = seg + (long long)k * 32 + lane;
        key[k] = 0u;
        val[k] = 0u;
        if (i < n) src(i, key[k], val[k]);
    }
    warp_rank(key, rank, seg, n, ps.shift, ps.mask, false, cnt[warp], lane, lt);
    __syncthreads();
    // per digit: exclusive prefix over warps (tile-local) and the tile total;
    // the aggregate is published at once so that later tiles can pass it
    uint32_t total = 0;
    if ((int)threadIdx.x < nbins) {
        const int d = threadIdx.x;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = total;
            total += c;
        }
        st_relaxed(ps.look + t * nbins + d, (t == 0 ? kLbInc : kLbAgg) | total);
    }
    uint32_t all;
    const uint32_t ex = block_excl_scan<uint32_t>(total, scan_sm, &all);
    if ((int)threadIdx.x < nbins) dstart[threadIdx.x] = ex;
    __syncthreads();
    // stage the tile in digit order (the keys' registers are free after this)
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = seg + (long long)k * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[k] >> ps.shift) & ps.mask;
            const uint32_t p = dstart[d] + cnt[warp][d] + rank[k];
            sk[p] = key[k];
            sv[p] = val[k];
        }
    }
    // global start of each digit: counts of all earlier tiles
    if ((int)threadIdx.x < nbins) {
        const int d = threadIdx.x;
        uint32_t before = 0;
        if (t > 0) {
            before = (uint32_t)os_lookback(ps.look, t, nbins, d, ps.err);
            st_relaxed(ps.look + t * nbins + d, kLbInc | (uint64_t)(before + total));
        }
        gstart[d] = ps.base[d] + before;
    }
    __syncthreads();
    const int nvalid = (int)((n - base) < RS_TILE ? (n - base) : RS_TILE);
    for (int j = threadIdx.x; j < nvalid; j += RS_THREADS) {
        const uint32_t kk = sk[j];
        const uint32_t d = (kk >> ps.shift) & ps.mask;
        const uint32_t pos = gstart[d] + (uint32_t)j - dstart[d];
        if (kout) kout[pos] = kk;
        vout[pos] = sv[j];
    }
}

// Exclusive scan of ld(0..n) into out in one pass over SCAN_TILE-item tiles;
// *total receives the sum.  look: one word per tile, zero before the launch;
// ctr: zero before the launch.
template <typename Load>
__global__ void __launch_bounds__(SCAN_THREADS)
k_os_scan(Load ld, long long n, uint64_t* __restrict__ out, uint64_t* look, uint32_t* ctr, long long* total,
          int* err)
{
    // one pad word per 16 keeps both the coalesced and the per-thread accesses
    // free of bank conflicts
    __shared__ uint64_t s_buf[SCAN_TILE + SCAN_TILE / 16];
    auto at = [](int i) { return i + (i >> 4); };
    __shared__ uint64_t sm[33];
    __shared__ uint32_t s_t;
    __shared__ uint64_t s_ex;
    if (threadIdx.x == 0) s_t = atomicAdd(ctr, 1u);
    __syncthreads();
    const long long t = s_t;
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (t >= ntiles) return;
    const long long tb = t * SCAN_TILE;
    // coalesced load, then each thread takes SCAN_IPT consecutive items
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const long long i = tb + (long long)k * SCAN_THREADS + threadIdx.x;
        s_buf[at(k * SCAN_THREADS + threadIdx.x)] = i < n ? ld(i) : 0;
    }
    __syncthreads();
    uint64_t v[SCAN_IPT];
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        v[k] = s_buf[at(threadIdx.x * SCAN_IPT + k)];
        acc += v[k];
    }
    uint64_t tot;
    uint64_t run = block_excl_scan<uint64_t>(acc, sm, &tot);  // ends with a barrier
    // in-tile exclusive prefixes first (frees v before the look-back)
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        s_buf[at(threadIdx.x * SCAN_IPT + k)] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) {
        uint64_t ex = 0;
        if (t == 0) {
            st_relaxed(look, kLbInc | tot);
        } else {
            st_relaxed(look + t, kLbAgg | tot);
            ex = os_lookback(look, t, 1, 0, err);
            st_relaxed(look + t, kLbInc | ((ex + tot) & kLbCount));
        }
        s_ex = ex;
        if (t == ntiles - 1) *total = (long long)(ex + tot);
    }
    __syncthreads();
    const uint64_t ex = s_ex;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const long long i = tb + (long long)k * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = ex + s_buf[at(k * SCAN_THREADS + threadIdx.x)];
    }
}

}  // namespace
}  // namespace dg
