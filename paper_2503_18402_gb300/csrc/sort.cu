// sort.cu -- tile binning: depth order, pair emission, stable tile sort, ranges.
//
// The per-tile lists must come out ordered by (tile, depth bits, Gaussian
// index).  Instead of one radix sort over 64-bit (tile | depth) keys of all
// M pairs (6 passes of 8 bits), the order is built in two cheaper stages:
//   1. a stable 32-bit LSD radix sort of the P visible depths (ties keep the
//      index order), then an exclusive scan of the tile counts in that order;
//   2. pairs are emitted in depth order, then stably sorted by tile id alone
//      (ceil(log2(tiles)) bits: 2 passes at 1237x822 / 16^2 = 4056 tiles).
// Stability of stage 2 preserves the depth order inside each tile, so the
// result equals the lexicographic (tile, depth bits, index) order.
//
// Radix pass = per-block digit histogram, exclusive scan of the
// digit-major histogram, stable scatter.  Each warp owns a contiguous
// segment of a block's tile and ranks equal digits with __match_any_sync;
// per-warp digit counts give the block-local offsets, so the scatter is
// stable without a block-wide sort.
#include "common.cuh"

namespace dg {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_MAXBITS = 8;

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
// segment (match_any within each 32-item round, running per-warp digit
// counts), the block's items are first placed in shared memory in digit order,
// then written out so that consecutive threads write consecutive addresses of
// each digit's run.  kout may be null (values only).
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const long long* n_dev,
             long long n_cap, int shift, uint32_t mask, const uint32_t* __restrict__ offs, int nblk)
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
#pragma unroll
    for (int k = 0; k < RS_IPT; ++k) {
        const long long i = seg + (long long)k * 32 + lane;
        const bool ok = i < n;
        key[k] = ok ? kin[i] : 0u;
        val[k] = ok ? vin[i] : 0u;
        // out-of-range lanes get a digit no valid lane can have
        const uint32_t d = ok ? ((key[k] >> shift) & mask) : (0x10000u + (uint32_t)lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (ok) before = cnt[warp][d];
        __syncwarp();
        rank[k] = before + __popc(peers & lt);
        if (ok && (peers & lt) == 0) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
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
                     const SortBufs& sb, cudaStream_t s, bool hist0_ready = false)
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
        k_rs_scatter<<<nblk, RS_THREADS, 0, s>>>(ks, vs, kd, vd, n_dev, n_cap, shift, mask, sb.hist, nblk);
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

// --------------------------------------------------------------- binning
__global__ void k_depth_keys(const float* __restrict__ depth, const int* __restrict__ tiles, int P,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    keys[i] = tiles[i] > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
    idx[i] = (uint32_t)i;
}

// First sorted position whose pair range holds each RS_TILE block's first pair.
__global__ void k_block_starts(const uint64_t* __restrict__ poff, int P, const long long* M_dev, long long M_cap,
                               int* __restrict__ bstart)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const long long M = *M_dev;
    if (s >= P || M > M_cap) return;
    const long long a = (long long)poff[s];
    const long long e = s + 1 < P ? (long long)poff[s + 1] : M;
    if (e <= a) return;
    for (long long b = (a + RS_TILE - 1) / RS_TILE; b * RS_TILE < e; ++b) bstart[b] = s;
}

// Pair emission, one RS_TILE block of consecutive pairs per CTA.  The block's
// Gaussians (at most RS_TILE, all with >= 1 pair) are staged in shared memory
// with their rects; each pair finds its Gaussian by binary search over the
// staged starts.  Writes key = tile id and value = Gaussian index, coalesced,
// and the per-block histogram of the first radix digit.
__global__ void __launch_bounds__(RS_THREADS)
k_emit(const float4* __restrict__ feat, const int* __restrict__ radius, const uint32_t* __restrict__ order,
       const uint64_t* __restrict__ poff, const int* __restrict__ bstart, int P, const long long* M_dev,
       long long M_cap, int B, int TX, int TY, uint32_t mask0, uint32_t* __restrict__ pkey,
       uint32_t* __restrict__ pval, uint32_t* __restrict__ hist0, int nblk, int* status)
{
    __shared__ int w_start[RS_TILE];      // pair offset of each staged Gaussian, relative to the block
    __shared__ uint32_t w_xy[RS_TILE];    // rect x0 | y0 << 16
    __shared__ int w_wx[RS_TILE];         // rect width in tiles
    __shared__ uint32_t w_g[RS_TILE];     // Gaussian index
    __shared__ uint32_t h[1 << RS_MAXBITS];
    const long long M = *M_dev;
    if (M > M_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *status = DG_ERR_CAPACITY;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = DG_OK;
    __shared__ int s_nw;
    for (int d = threadIdx.x; d < (1 << RS_MAXBITS); d += RS_THREADS) h[d] = 0;
    if (threadIdx.x == 0) s_nw = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
    if (base < M) {  // block-uniform
        const long long end = (base + RS_TILE) < M ? (base + RS_TILE) : M;
        const int s_lo = bstart[blockIdx.x];
        // stage the Gaussians whose pair range starts before `end` (a prefix of s_lo, s_lo+1, ...)
        int top = 0;
        for (int w = threadIdx.x; w < RS_TILE; w += RS_THREADS) {
            const int s = s_lo + w;
            if (s >= P) break;
            const long long st = (long long)poff[s];
            if (st >= end) break;
            const uint32_t g = order[s];
            const float4 f0 = feat[3 * (size_t)g];
            const Rect q = tile_rect(f0.x, f0.y, radius[g], B, TX, TY);
            w_start[w] = (int)(st - base);
            w_xy[w] = (uint32_t)q.x0 | ((uint32_t)q.y0 << 16);
            w_wx[w] = q.x1 - q.x0;
            w_g[w] = g;
            top = w + 1;
        }
        if (top > 0) atomicMax(&s_nw, top);
        __syncthreads();
        const int nw = s_nw;
#pragma unroll 2
        for (int k = 0; k < RS_IPT; ++k) {
            const long long i = base + (long long)k * RS_THREADS + threadIdx.x;
            if (i >= end) break;
            const int rel = (int)(i - base);
            int lo = 0, hi = nw - 1;  // w_start[0] <= 0 <= rel
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (w_start[mid] <= rel) lo = mid; else hi = mid - 1;
            }
            const int j = rel - w_start[lo];
            const int wx = w_wx[lo];
            const uint32_t xy = w_xy[lo];
            const int ty = (int)(xy >> 16) + j / wx;
            const int tx = (int)(xy & 0xffffu) + j % wx;
            const uint32_t key = (uint32_t)(ty * TX + tx);
            pkey[i] = key;
            pval[i] = w_g[lo];
            atomicAdd(&h[key & mask0], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask0; d += RS_THREADS) hist0[(long long)d * nblk + blockIdx.x] = h[d];
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const long long* M_dev, long long M_cap,
                         uint2* __restrict__ ranges)
{
    const long long M = eff_count(M_dev, M_cap);
    const long long nq = (M + 3) / 4;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 3 < M) {
            const uint4 v = *(const uint4*)(keys + i0);
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
            for (int c = 0; c < 4; ++c) k[c] = i0 + c < M ? keys[i0 + c] : 0xffffffffu;
        }
        uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
        const uint32_t next = i0 + 4 < M ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long i = i0 + c;
            if (i >= M) break;
            const uint32_t nx = c < 3 ? k[c + 1] : next;
            if (i == 0 || prev != k[c]) ranges[k[c]].x = (uint32_t)i;
            if (i == M - 1 || nx != k[c]) ranges[k[c]].y = (uint32_t)(i + 1);
            prev = k[c];
        }
    }
}

// Workspace layout (offsets 256-byte aligned).  The pair count and the
// P-sized buffers come first so that their offsets do not depend on M_cap:
// phase 1 and phase 2 may be called with workspaces laid out for different
// capacities as long as the P part was carried over.
struct BinWs {
    long long* M;                       // total pair count
    uint32_t *dk0, *dv0, *dk1, *dv1;   // depth sort, P each
    uint64_t* poff;                     // P pair offsets
    uint32_t *pk0, *pv0, *pk1, *pv1;   // pair sort, M_cap each
    uint32_t* pkfin;                    // sorted pair keys, M_cap
    int* bstart;                        // first sorted position of each pair block
    uint32_t* hist;
    uint64_t* bsum;
    size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static BinWs bin_layout(char* base, long long P, long long M_cap)
{
    BinWs w;
    size_t o = 0;
    auto take = [&](size_t bytes) { char* p = base + o; o += align256(bytes); return p; };
    w.M = (long long*)take(8);
    w.dk0 = (uint32_t*)take(4 * P); w.dv0 = (uint32_t*)take(4 * P);
    w.dk1 = (uint32_t*)take(4 * P); w.dv1 = (uint32_t*)take(4 * P);
    w.poff = (uint64_t*)take(8 * P);
    w.pk0 = (uint32_t*)take(4 * M_cap); w.pv0 = (uint32_t*)take(4 * M_cap);
    w.pk1 = (uint32_t*)take(4 * M_cap); w.pv1 = (uint32_t*)take(4 * M_cap);
    w.pkfin = (uint32_t*)take(4 * M_cap);
    w.bstart = (int*)take(4 * ((M_cap + RS_TILE - 1) / RS_TILE + 1));
    const long long n = P > M_cap ? P : M_cap;
    const long long nblk = (n + RS_TILE - 1) / RS_TILE;
    const long long nh = (long long)(1 << RS_MAXBITS) * nblk;
    w.hist = (uint32_t*)take(4 * nh);
    const long long nscan = (nh > n ? nh : n);
    w.bsum = (uint64_t*)take(8 * ((nscan + SCAN_TILE - 1) / SCAN_TILE + 1));
    w.bytes = o;
    return w;
}

}  // namespace dg

extern "C" size_t dg_bin_workspace_size(int64_t P, int64_t M_cap, int32_t n_tiles)
{
    (void)n_tiles;
    if (P < 0 || M_cap < 0) return 0;
    return dg::bin_layout(nullptr, P, M_cap).bytes;
}

extern "C" dg_status dg_bin_count(const float* depth, const int32_t* tiles, int64_t P, void* ws,
                                  size_t ws_bytes, int64_t M_cap, int32_t n_tiles, int64_t* M_out,
                                  dg_stream stream)
{
    if (P < 0 || P > INT32_MAX || M_cap < 0 || M_cap > (int64_t)UINT32_MAX || n_tiles < 1) {
        dg_set_error("bad sizes P=%lld M_cap=%lld n_tiles=%d", (long long)P, (long long)M_cap, n_tiles);
        return DG_ERR_ARG;
    }
    if (!ws || !M_out || (P > 0 && (!depth || !tiles))) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const dg::BinWs w = dg::bin_layout((char*)ws, P, M_cap);
    if (ws_bytes < w.bytes) { dg_set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return DG_ERR_CAPACITY; }
    cudaStream_t s = (cudaStream_t)stream;
    if (P == 0) {
        cudaMemsetAsync(w.M, 0, sizeof(long long), s);
        cudaMemsetAsync(M_out, 0, sizeof(long long), s);
        return dg_check_launch("bin_count");
    }
    dg::k_depth_keys<<<(int)((P + 255) / 256), 256, 0, s>>>(depth, tiles, (int)P, w.dk0, w.dv0);
    dg_note_launch();
    dg::SortBufs sb{w.hist, w.bsum};
    // 32 key bits = 4 passes ping-ponging dk0 -> dk1 -> dk0 -> dk1 -> dk0: the
    // depth order ends in dv0 (checked below so a change of pass count cannot
    // silently move it).
    const dg::KV r = dg::radix_sort(w.dk0, w.dv0, w.dk1, w.dv1, nullptr, nullptr, nullptr, P, 32, sb, s);
    if (r.v != w.dv0) { dg_set_error("internal: depth order buffer"); return DG_ERR_CUDA; }
    dg::exclusive_scan(dg::LoadTilesInOrder{tiles, w.dv0}, P, w.poff, w.bsum, w.M, s);
    cudaMemcpyAsync(M_out, w.M, sizeof(long long), cudaMemcpyDeviceToDevice, s);
    return dg_check_launch("bin_count");
}

extern "C" dg_status dg_bin_sort(const float* feat, const int32_t* radius, int64_t P, const dg_camera* cam,
                                 int32_t tile, void* ws, size_t ws_bytes, int64_t M_cap, uint32_t* gid,
                                 uint32_t* ranges, int32_t* status, dg_stream stream)
{
    if (!cam || tile < 1 || cam->width <= 0 || cam->height <= 0) { dg_set_error("bad camera or tile"); return DG_ERR_ARG; }
    if (P < 0 || P > INT32_MAX || M_cap < 0 || M_cap > (int64_t)UINT32_MAX) { dg_set_error("bad sizes"); return DG_ERR_ARG; }
    if (!ws || !ranges || !status || (P > 0 && (!feat || !radius)) || (M_cap > 0 && !gid)) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const dg::BinWs w = dg::bin_layout((char*)ws, P, M_cap);
    if (ws_bytes < w.bytes) { dg_set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return DG_ERR_CAPACITY; }
    const int TX = (cam->width + tile - 1) / tile, TY = (cam->height + tile - 1) / tile;
    const long long n_tiles = (long long)TX * TY;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * n_tiles, s);
    cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    int bits = 0;
    while ((1ll << bits) < n_tiles) ++bits;
    const int b0 = dg::first_pass_bits(bits);
    const uint32_t mask0 = b0 > 0 ? (1u << b0) - 1u : 0u;
    const int nblk = (int)((M_cap + dg::RS_TILE - 1) / dg::RS_TILE);
    const int pb = (int)((P + 255) / 256);
    if (P > 0 && nblk > 0) {
        dg::k_block_starts<<<pb, 256, 0, s>>>(w.poff, (int)P, w.M, M_cap, w.bstart);
        dg_note_launch();
    }
    // emit pairs in depth order (slots from phase 1) with pass-0 histogram, or flag overflow
    dg::k_emit<<<nblk > 0 ? nblk : 1, dg::RS_THREADS, 0, s>>>((const float4*)feat, radius, w.dv0, w.poff, w.bstart,
                                                            (int)P, w.M, M_cap, tile, TX, TY, mask0, w.pk0, w.pv0,
                                                            w.hist, nblk > 0 ? nblk : 1, status);
    dg_note_launch();
    if (M_cap == 0) return dg_check_launch("bin_sort");
    dg::SortBufs sb{w.hist, w.bsum};
    dg::radix_sort(w.pk0, w.pv0, w.pk1, w.pv1, w.pkfin, gid, w.M, M_cap, bits, sb, s, /*hist0_ready=*/bits > 0);
    const long long nq = (M_cap + 3) / 4;
    long long rb = (nq + 255) / 256;
    if (rb > 152 * 32) rb = 152 * 32;
    dg::k_ranges<<<(int)(rb > 0 ? rb : 1), 256, 0, s>>>(w.pkfin, w.M, M_cap, (uint2*)ranges);
    dg_note_launch();
    return dg_check_launch("bin_sort");
}
