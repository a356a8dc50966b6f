// radix.cuh -- device-wide exclusive scan and stable LSD radix sort of
// (uint32 key, uint32 value) pairs, shared by the binning and densification
// kernels.  Kernels live in an anonymous namespace: each including
// translation unit gets its own copy.
//
// Radix pass = per-block digit histogram, exclusive scan of the digit-major
// histogram, stable scatter.  Each warp owns a contiguous segment of a block's
// tile and finds the lanes with equal digits by one ballot per digit bit;
// per-warp digit counts give the block-local offsets, so the scatter is
// stable without a block-wide sort.
#pragma once

#include "common.cuh"

namespace dg {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_MAXBITS = 8;

// Lanes of the warp holding the same `nbits`-bit digit as this lane, among the
// lanes with ok set (the mask __match_any_sync would give over those lanes),
// from one ballot per digit bit: the cost does not grow with the number of
// distinct digits in the warp.  A lane without ok gets its own bit only.
__device__ __forceinline__ uint32_t warp_peers(uint32_t d, int nbits, bool ok, int lane)
{
    uint32_t m = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < RS_MAXBITS; ++b) {
        if (b < nbits) {
            const bool bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            m &= bit ? bal : ~bal;
        }
    }
    return ok ? m : (1u << lane);
}

// Stable rank of a warp's RS_IPT x 32 keys (item k of lane l at position
// seg + 32 k + l, valid below n) among the equal digits of the warp's
// segment, in position order; wcnt: the warp's running count of each digit
// (zero on entry, the digit totals on return).  Peer masks by ballots
// (`ballot`: fixed cost, for digits that are nearly all distinct within a
// warp) or by __match_any_sync (fast when a warp holds few distinct digits).
__device__ __forceinline__ void warp_rank(const uint32_t (&key)[RS_IPT], uint32_t (&rank)[RS_IPT], long long seg,
                                          long long n, int shift, uint32_t mask, bool ballot, uint32_t* wcnt,
                                          int lane, uint32_t lt)
{
    const int nbits = __popc(mask);
    uint32_t peers[RS_IPT];
    if (ballot) {
#pragma unroll
        for (int k = 0; k < RS_IPT; ++k)
            peers[k] = warp_peers((key[k] >> shift) & mask, nbits, seg + (long long)k * 32 + lane < n, lane);
    } else {
#pragma unroll
        for (int k = 0; k < RS_IPT; ++k) {
            // out-of-range lanes get a digit no valid lane can have
            const bool ok = seg + (long long)k * 32 + lane < n;
            peers[k] = __match_any_sync(0xffffffffu, ok ? ((key[k] >> shift) & mask) : (0x10000u + (uint32_t)lane));
        }
    }
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const bool ok = seg + (long long)k * 32 + lane < n;
        const uint32_t d = (key[k] >> shift) & mask;
        uint32_t before = 0;
        if (ok) before = wcnt[d];
        __syncwarp();
        rank[k] = before + __popc(peers[k] & lt);
        if (ok && (peers[k] & lt) == 0) wcnt[d] = before + __popc(peers[k]);
        __syncwarp();
    }
}

template <typename T>
__device__ inline T warp_incl_scan(T x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread; *total receives the sum.
// smem: at least 33 elements.  Ends with a barrier so smem can be reused.
template <typename T>
__device__ inline T block_excl_scan(T v, T* smem, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const T inc = warp_incl_scan(v, lane);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? smem[lane] : T(0);
        w = warp_incl_scan(w, lane);
        smem[lane] = w;
    }
    __syncthreads();
    const T pre = warp > 0 ? smem[warp - 1] : T(0);
    *total = smem[nw - 1];
    __syncthreads();
    return pre + inc - v;
}

// --------------------------------------------------------------- scan
struct LoadU32 {
    const uint32_t* a;
    __device__ uint64_t operator()(long long i) const { return a[i]; }
};
struct LoadTilesInOrder {  // tiles touched by the Gaussian at sorted position s
    const int* tiles;
    const uint32_t* order;
    __device__ uint64_t operator()(long long s) const { return (uint64_t)tiles[order[s]]; }
};

template <typename Load>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(Load ld, long long n, uint64_t* bsum)
{
    __shared__ uint64_t sm[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const long long i = base + (long long)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += ld(i);
    }
    uint64_t tot;
    block_excl_scan<uint64_t>(acc, sm, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint64_t* bsum, int nb, long long* total_out)
{
    __shared__ uint64_t sm[33];
    uint64_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan<uint64_t>(v, sm, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = (long long)carry;
}

template <typename Load, typename TOut>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(Load ld, long long n, const uint64_t* bsum, TOut* out)
{
    __shared__ uint64_t sm[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
    uint64_t v[SCAN_IPT];
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const long long i = base + k;
        v[k] = i < n ? ld(i) : 0;
        acc += v[k];
    }
    uint64_t tot;
    uint64_t run = block_excl_scan<uint64_t>(acc, sm, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const long long i = base + k;
        if (i < n) out[i] = (TOut)run;
        run += v[k];
    }
}

template <typename Load, typename TOut>
static void exclusive_scan(Load ld, long long n, TOut* out, uint64_t* bsum, long long* total, cudaStream_t s)
{
    const int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (nb == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(long long), s);
        return;
    }
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(ld, n, bsum);
    dg_note_launch();
    k_scan_top<<<1, 1024, 0, s>>>(bsum, nb, total);
    dg_note_launch();
    k_scan_down<<<nb, SCAN_THREADS, 0, s>>>(ld, n, bsum, out);
    dg_note_launch();
}

// --------------------------------------------------------------- radix sort
// n_dev: when non-null, the element count is read on the device as
// (*n_dev <= n_cap ? *n_dev : 0); grids are sized by n_cap.
__device__ inline long long eff_count(const long long* n_dev, long long n_cap)
{
    if (!n_dev) return n_cap;
    const long long n = *n_dev;
    return n <= n_cap ? n : 0;
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const uint32_t* __restrict__ keys, const long long* n_dev, long long n_cap, int shift,
          uint32_t mask, uint32_t* __restrict__ hist, int nblk)
{
    __shared__ uint32_t h[1 << RS_MAXBITS];
    for (int d = threadIdx.x; d < (1 << RS_MAXBITS); d += RS_THREADS) h[d] = 0;
    __syncthreads();
    const long long n = eff_count(n_dev, n_cap);
    const long long base = (long long)blockIdx.x * RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = base + (long long)k * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask; d += RS_THREADS) hist[(long long)d * nblk + blockIdx.x] = h[d];
}

// Stable scatter of one radix pass.  Ranks are computed per warp-owned
// segment (ballot peer masks within each 32-item round, running per-warp digit
// counts), the block's items are first placed in shared memory in digit order,
// then written out so that consecutive threads write consecutive addresses of
// each digit's run.  kout may be null (values only).
__global__ void __launch_bounds__(RS_THREADS, 4)
k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const long long* n_dev,
             long long n_cap, int shift, uint32_t mask, bool ballot, const uint32_t* __restrict__ offs, int nblk)
{
    __shared__ uint32_t cnt[RS_WARPS][1 << RS_MAXBITS];
    __shared__ uint32_t dstart[1 << RS_MAXBITS];
    __shared__ uint32_t gstart[1 << RS_MAXBITS];
    __shared__ uint32_t sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    __shared__ uint32_t scan_sm[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long n = eff_count(n_dev, n_cap);
    const long long base = (long long)blockIdx.x * RS_TILE;
    if (base >= n) return;
    const long long seg = base + (long long)warp * (32 * RS_IPT);
    const int nbins = (int)mask + 1;
    for (int d = lane; d < nbins; d += 32) cnt[warp][d] = 0;
    __syncwarp();
    uint32_t key[RS_IPT], val[RS_IPT], rank[RS_IPT];
    const uint32_t lt = (1u << lane) - 1u;
    // all loads first, then the peer masks, then the running per-warp counts
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = seg + (long long)k * 32 + lane;
        key[k] = i < n ? kin[i] : 0u;
        val[k] = i < n ? vin[i] : 0u;
    }
    warp_rank(key, rank, seg, n, shift, mask, ballot, cnt[warp], lane, lt);
    __syncthreads();
    // per digit: exclusive prefix over warps (block-local), digit total, global start
    uint32_t total = 0;
    if ((int)threadIdx.x < nbins) {
        const int d = threadIdx.x;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = total;
            total += c;
        }
        gstart[d] = offs[(long long)d * nblk + blockIdx.x];
    }
    uint32_t all;
    const uint32_t ex = block_excl_scan<uint32_t>(total, scan_sm, &all);
    if ((int)threadIdx.x < nbins) dstart[threadIdx.x] = ex;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = seg + (long long)k * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[k] >> shift) & mask;
            const uint32_t p = dstart[d] + cnt[warp][d] + rank[k];
            sk[p] = key[k];
            sv[p] = val[k];
        }
    }
    __syncthreads();
    const int nvalid = (int)((n - base) < RS_TILE ? (n - base) : RS_TILE);
    for (int j = threadIdx.x; j < nvalid; j += RS_THREADS) {
        const uint32_t kk = sk[j];
        const uint32_t d = (kk >> shift) & mask;
        const uint32_t pos = gstart[d] + (uint32_t)j - dstart[d];
        if (kout) kout[pos] = kk;
        vout[pos] = sv[j];
    }
}

struct SortBufs {
    uint32_t* hist;   // (1 << RS_MAXBITS) * nblk
    uint64_t* bsum;   // scan block sums
};

// Stable LSD sort of (key, val) over the low `bits` key bits.  Input in
// (k0, v0); (k1, v1) is ping-pong space.  The last pass writes to
// (kfin, vfin) when vfin is given (kfin may then be null: values only; they
// must not alias k0/k1, v0/v1), else to the ping-pong buffer whose turn it
// is.  When hist0_ready, the caller already wrote pass 0's per-block
// histogram into sb.hist.  Returns where the result lies.
struct KV { uint32_t* k; uint32_t* v; };

static KV radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t* kfin,
                     uint32_t* vfin, const long long* n_dev, long long n_cap, int bits,
                     const SortBufs& sb, cudaStream_t s, bool hist0_ready = false, uint32_t ballot_passes = 0)
{
    const int nblk = (int)((n_cap + RS_TILE - 1) / RS_TILE);
    if (nblk == 0) return KV{k0, v0};
    if (bits == 0) {
        if (kfin) cudaMemcpyAsync(kfin, k0, sizeof(uint32_t) * n_cap, cudaMemcpyDeviceToDevice, s);
        if (vfin) cudaMemcpyAsync(vfin, v0, sizeof(uint32_t) * n_cap, cudaMemcpyDeviceToDevice, s);
        return KV{kfin ? kfin : k0, vfin ? vfin : v0};
    }
    const int npass = (bits + RS_MAXBITS - 1) / RS_MAXBITS;
    const int per = (bits + npass - 1) / npass;
    uint32_t *ks = k0, *vs = v0;
    for (int p = 0; p < npass; ++p) {
        const int shift = p * per;
        const int b = (bits - shift) < per ? (bits - shift) : per;
        const uint32_t mask = (1u << b) - 1u;
        const bool last = p == npass - 1;
        uint32_t* kd = (last && vfin) ? kfin : (ks == k0 ? k1 : k0);
        uint32_t* vd = (last && vfin) ? vfin : (vs == v0 ? v1 : v0);
        if (!(p == 0 && hist0_ready)) {
            k_rs_hist<<<nblk, RS_THREADS, 0, s>>>(ks, n_dev, n_cap, shift, mask, sb.hist, nblk);
            dg_note_launch();
        }
        const long long nh = (long long)(mask + 1) * nblk;
        exclusive_scan(LoadU32{sb.hist}, nh, sb.hist, sb.bsum, (long long*)nullptr, s);
        k_rs_scatter<<<nblk, RS_THREADS, 0, s>>>(ks, vs, kd, vd, n_dev, n_cap, shift, mask, (ballot_passes >> p) & 1u,
                                                 sb.hist, nblk);
        dg_note_launch();
        ks = kd;
        vs = vd;
    }
    return KV{ks, vs};
}

// Digit width of the first pass of radix_sort over `bits` bits.
static int first_pass_bits(int bits)
{
    if (bits == 0) return 0;
    const int npass = (bits + RS_MAXBITS - 1) / RS_MAXBITS;
    const int per = (bits + npass - 1) / npass;
    return bits < per ? bits : per;
}

}  // namespace
}  // namespace dg
