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
// Several views: records are r = v * P + i; stage 1 adds one stable pass on
// the view index after the depth passes (order (view, depth, index)) and the
// tile ids are global, view_offset[v] + ty * TX_v + tx, so each view's tiles
// form one contiguous block of the range table.  The pair payload is the
// record index r.
//
// Stage 1 runs each radix pass as one kernel with decoupled look-back
// (onesweep.cuh), the digit counts of all passes counted in one read before
// the first pass, and the tile-count scan likewise in one kernel.  Stage 2
// keeps the classic pass (per-block digit histogram, scan of the
// digit-major histogram, stable scatter; the first histogram comes out of
// the emission kernel): measured on 8.2M pairs, the emission kernel's extra
// work for all-pass counts cost more than the launches it saved.
// Both rank equal digits within warp-owned segments (__match_any_sync, or
// per-bit ballots on the low tile digit), so every pass is stable.
#include "onesweep.cuh"

namespace dg {

// Tile-sort passes that rank by per-bit ballots instead of __match_any_sync
// (bit p: pass p).  The low tile digit (neighbouring tiles of one Gaussian's
// rectangle) is nearly all distinct within a warp; measured at 2M Gaussians,
// ballots there took the pair sort from 0.266 to 0.244 ms, ballots on the high
// digit too 0.256 ms.  The depth passes stay on __match_any_sync: ballots made
// them slower on every digit (0.201 ms with none, 0.229 on the two low digits,
// 0.255 on all four).
constexpr uint32_t kTileBallotPasses = 0x1;

// --------------------------------------------------------------- binning
// Depth-order key of record i: its depth bits when it touches a tile, else
// all ones (culled records sort last); the value is the record index.
struct SrcDepth {
    const float* depth;
    const int* tiles;
    __device__ void operator()(long long i, uint32_t& key, uint32_t& val) const
    {
        key = tiles[i] > 0 ? __float_as_uint(depth[i]) : 0xffffffffu;
        val = (uint32_t)i;
    }
};

// View key of the record r = v * P + i at a sorted position: its view v, or
// n_views for a culled record, so that every culled record (no pairs) ends up
// behind all visible records of all views.  (Left between two views, runs of
// culled records would fill k_emit's window of staged Gaussians.)
struct SrcView {
    const uint32_t* order;
    const int* tiles;
    uint32_t P, n_views;
    __device__ void operator()(long long i, uint32_t& key, uint32_t& val) const
    {
        val = order[i];
        key = tiles[val] > 0 ? val / P : n_views;
    }
};

// Digit counts of the four depth passes (and of the view pass when vbits >
// 0) in one read of the depths; clears the first pass's look-back words.
__global__ void __launch_bounds__(RS_THREADS)
k_os_hist_depth(const float* __restrict__ depth, const int* __restrict__ tiles, long long N, uint32_t P,
                uint32_t n_views, int vbits, OsCtl* ctl, uint64_t* __restrict__ look0)
{
    __shared__ uint32_t h[5][1 << RS_MAXBITS];
    const int npass = vbits > 0 ? 5 : 4;
    for (int i = threadIdx.x; i < 5 * (1 << RS_MAXBITS); i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * RS_THREADS;
    for (long long i = (long long)blockIdx.x * RS_THREADS + threadIdx.x; i < N; i += stride) {
        const bool vis = tiles[i] > 0;
        const uint32_t k = vis ? __float_as_uint(depth[i]) : 0xffffffffu;
        atomicAdd(&h[0][k & 255u], 1u);
        atomicAdd(&h[1][(k >> 8) & 255u], 1u);
        atomicAdd(&h[2][(k >> 16) & 255u], 1u);
        atomicAdd(&h[3][k >> 24], 1u);
        if (vbits > 0) atomicAdd(&h[4][vis ? (uint32_t)i / P : n_views], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * (1 << RS_MAXBITS); i += RS_THREADS) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&os_hist(ctl, i >> RS_MAXBITS)[i & ((1 << RS_MAXBITS) - 1)], c);
    }
    const long long nw = (N + RS_TILE - 1) / RS_TILE * (1 << RS_MAXBITS);
    for (long long i = (long long)blockIdx.x * RS_THREADS + threadIdx.x; i < nw; i += stride) look0[i] = 0;
}

struct TileGrid {
    int n;
    int TX[DG_MAX_VIEWS], TY[DG_MAX_VIEWS];
    int off[DG_MAX_VIEWS + 1];  // first global tile id of each view
};

// First sorted position whose pair range holds each RS_TILE block's first pair.
__global__ void k_block_starts(const uint64_t* __restrict__ poff, long long P, const long long* M_dev, long long M_cap,
                               int* __restrict__ bstart)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long M = *M_dev;
    if (s >= P || M > M_cap) return;
    const long long a = (long long)poff[s];
    const long long e = s + 1 < P ? (long long)poff[s + 1] : M;
    if (e <= a) return;
    for (long long b = (a + RS_TILE - 1) / RS_TILE; b * RS_TILE < e; ++b) bstart[b] = (int)s;
}

// Pair emission, one RS_TILE block of consecutive pairs per CTA.  The block's
// Gaussians (at most RS_TILE, all with >= 1 pair) are staged in shared memory
// with their rects; each pair finds its Gaussian by binary search over the
// staged starts.  Writes key = tile id and value = Gaussian index, coalesced,
// and the per-block histogram of the first radix digit.
__global__ void __launch_bounds__(RS_THREADS)
k_emit(const float4* __restrict__ feat, const int* __restrict__ radius, const uint32_t* __restrict__ order,
       const uint64_t* __restrict__ poff, const int* __restrict__ bstart, long long P, uint32_t Pv,
       const long long* M_dev, long long M_cap, int B, TileGrid tg, uint32_t mask0, uint32_t* __restrict__ pkey,
       uint32_t* __restrict__ pval, uint32_t* __restrict__ hist0, int nblk, const int* __restrict__ err1,
       int* status)
{
    const uint32_t n_tiles = (uint32_t)tg.off[tg.n];
    // staged Gaussians: pair offset relative to the block (the first one's,
    // <= 0, in s_first; the others' lie in 1 .. RS_TILE - 1), rect corner,
    // rect width and view, record index, tile mask (0: every tile of the rect)
    __shared__ uint16_t w_start[RS_TILE];
    __shared__ uint32_t w_xy[RS_TILE];    // rect x0 | y0 << 16
    __shared__ uint32_t w_wv[RS_TILE];    // rect width in tiles | view << 16
    __shared__ uint32_t w_g[RS_TILE];     // record index
    __shared__ unsigned long long w_m[RS_TILE];
    __shared__ int s_first;
    __shared__ int s_off[DG_MAX_VIEWS];   // global tile id of each view's tile (0, 0)
    __shared__ int s_tx[DG_MAX_VIEWS];    // tiles per row of each view
    __shared__ uint32_t h[1 << RS_MAXBITS];
    const long long M = *M_dev;
    // a failed wait of the depth order (phase 1) is reported here
    if (blockIdx.x == 0 && threadIdx.x == 0 && *err1 != 0) *status = *err1;
    if (M > M_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *status = DG_ERR_CAPACITY;
        return;
    }
    // (status was cleared by the host before this launch; blocks only set errors)
    __shared__ int s_nw;
    for (int d = threadIdx.x; d < (1 << RS_MAXBITS); d += RS_THREADS) h[d] = 0;
    for (int v = threadIdx.x; v < tg.n; v += RS_THREADS) {
        s_off[v] = tg.off[v];
        s_tx[v] = tg.TX[v];
    }
    if (threadIdx.x == 0) s_nw = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RS_TILE;
    if (base < M) {  // block-uniform
        const long long end = (base + RS_TILE) < M ? (base + RS_TILE) : M;
        const int s_lo = bstart[blockIdx.x];
        // stage the Gaussians whose pair range starts before `end` (a prefix of
        // s_lo, s_lo + 1, ...).  A candidate's pair offset and record index are
        // loaded together (both follow from its sorted position), then its
        // record; each link is issued for all of a thread's candidates at once,
        // the second half of the candidates only when the block holds more
        // than RS_TILE / 2 Gaussians (fewer than 4 pairs each).
        constexpr int HALF = RS_IPT / 2;
        long long st[RS_IPT];
        uint32_t gk[RS_IPT];
#pragma unroll
        for (int k = 0; k < HALF; ++k) {
            const long long s = (long long)s_lo + threadIdx.x + k * RS_THREADS;
            st[k] = s < P ? (long long)poff[s] : LLONG_MAX;
            gk[k] = s < P ? order[s] : 0u;
        }
        const bool more = __syncthreads_or(st[HALF - 1] < end) != 0;
#pragma unroll
        for (int k = HALF; k < RS_IPT; ++k) {
            const long long s = (long long)s_lo + threadIdx.x + k * RS_THREADS;
            st[k] = more && s < P ? (long long)poff[s] : LLONG_MAX;
            gk[k] = more && s < P ? order[s] : 0u;
        }
        int top = 0;
#pragma unroll
        for (int k = 0; k < RS_IPT; ++k) {
            if (st[k] < end) {
                const int w = (int)threadIdx.x + k * RS_THREADS;
                const uint32_t g = gk[k];
                const int v = (int)(g / Pv);
                const float4 f0 = feat[3 * (size_t)g];
                const float4 f2 = feat[3 * (size_t)g + 2];
                const Rect q = tile_rect(f0.x, f0.y, radius[g], B, tg.TX[v], tg.TY[v]);
                if (w == 0) s_first = (int)(st[k] - base);
                else w_start[w] = (uint16_t)(st[k] - base);
                w_xy[w] = (uint32_t)q.x0 | ((uint32_t)q.y0 << 16);
                w_wv[w] = (uint32_t)(q.x1 - q.x0) | ((uint32_t)v << 16);
                w_g[w] = g;
                w_m[w] = (unsigned long long)__float_as_uint(f2.y) |
                         ((unsigned long long)__float_as_uint(f2.z) << 32);
                top = w + 1;
            }
        }
        if (top > 0) atomicMax(&s_nw, top);
        __syncthreads();
        const int nw = s_nw;
        // each thread emits RS_IPT consecutive pairs: one search, then an incremental tile walk
        static_assert(RS_IPT == 8, "the vector stores below write 8 pairs per thread");
        const int rel0 = (int)threadIdx.x * RS_IPT;
        const int nblock = (int)(end - base);
        if (rel0 < nblock) {
            int lo = 0, hi = nw - 1;  // the first staged Gaussian starts at or before 0 <= rel0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;  // >= 1
                if ((int)w_start[mid] <= rel0) lo = mid; else hi = mid - 1;
            }
            const int j = rel0 - (lo > 0 ? (int)w_start[lo] : s_first);
            uint32_t wv = w_wv[lo];
            int wx = (int)(wv & 0xffffu);
            uint32_t xy = w_xy[lo];
            uint32_t g = w_g[lo];
            // with a tile mask, pair j is the j-th set bit (row-major, 8 bits per row)
            unsigned long long mk = w_m[lo];
            int tb = s_off[wv >> 16], TXv = s_tx[wv >> 16];
            int next = lo + 1 < nw ? (int)w_start[lo + 1] : nblock;
            int rx, ry;
            if (mk) {
                for (int c = 0; c < j; ++c) mk &= mk - 1;
                const int b = __ffsll((long long)mk) - 1;
                rx = b & 7; ry = b >> 3;
            } else {
                ry = j / wx; rx = j - ry * wx;
            }
            uint32_t kk[RS_IPT], vv[RS_IPT];
            const int cnt = nblock - rel0 < RS_IPT ? nblock - rel0 : RS_IPT;
#pragma unroll
            for (int e = 0; e < RS_IPT; ++e) {
                if (e < cnt) {
                    if (rel0 + e >= next) {  // next Gaussian of the window
                        ++lo;
                        wv = w_wv[lo];
                        wx = (int)(wv & 0xffffu); xy = w_xy[lo]; g = w_g[lo];
                        mk = w_m[lo];
                        tb = s_off[wv >> 16]; TXv = s_tx[wv >> 16];
                        next = lo + 1 < nw ? (int)w_start[lo + 1] : nblock;
                        if (mk) {
                            const int b = __ffsll((long long)mk) - 1;
                            rx = b & 7; ry = b >> 3;
                        } else {
                            rx = 0; ry = 0;
                        }
                    }
                    uint32_t key = (uint32_t)(tb + ((int)(xy >> 16) + ry) * TXv + (int)(xy & 0xffffu) + rx);
                    if (key >= n_tiles) {  // cannot happen for consistent inputs; never index past the grid
                        *status = DG_ERR_CUDA;
                        key = 0;
                    }
                    kk[e] = key;
                    vv[e] = g;
                    atomicAdd(&h[key & mask0], 1u);
                    if (mk) {
                        mk &= mk - 1;  // the next kept tile (none left when the Gaussian's pairs end)
                        const int b = __ffsll((long long)mk) - 1;
                        rx = b & 7; ry = b >> 3;
                    } else if (++rx == wx) {
                        rx = 0; ++ry;
                    }
                }
            }
            const long long i0 = base + rel0;
            if (cnt == RS_IPT) {
                uint4* kp = (uint4*)(pkey + i0);
                uint4* vp = (uint4*)(pval + i0);
                kp[0] = make_uint4(kk[0], kk[1], kk[2], kk[3]);
                kp[1] = make_uint4(kk[4], kk[5], kk[6], kk[7]);
                vp[0] = make_uint4(vv[0], vv[1], vv[2], vv[3]);
                vp[1] = make_uint4(vv[4], vv[5], vv[6], vv[7]);
            } else {
                for (int e = 0; e < cnt; ++e) {
                    pkey[i0 + e] = kk[e];
                    pval[i0 + e] = vv[e];
                }
            }
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
    OsCtl* ctl1;                        // phase 1 control block, then the scan's look-back words
    uint64_t* slook;
    size_t ctl1_bytes;                  // bytes phase 1 clears from ctl1 on
    uint64_t* look[2];                  // phase 1 radix look-back words, alternating between passes
    uint32_t *pk0, *pv0, *pk1, *pv1;   // pair sort, M_cap each
    uint32_t* pkfin;                    // sorted pair keys, M_cap
    int* bstart;                        // first sorted position of each pair block
    uint32_t* hist;                     // phase 2 per-block digit counts
    uint64_t* bsum;                     // phase 2 scan block sums
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
    const size_t c0 = o;
    w.ctl1 = (OsCtl*)take(sizeof(OsCtl));
    w.slook = (uint64_t*)take(8 * ((P + SCAN_TILE - 1) / SCAN_TILE + 1));
    w.ctl1_bytes = o - c0;
    const long long nlook = (P + RS_TILE - 1) / RS_TILE * (1 << RS_MAXBITS);
    w.look[0] = (uint64_t*)take(8 * nlook);
    w.look[1] = (uint64_t*)take(8 * nlook);
    w.pk0 = (uint32_t*)take(4 * M_cap); w.pv0 = (uint32_t*)take(4 * M_cap);
    w.pk1 = (uint32_t*)take(4 * M_cap); w.pv1 = (uint32_t*)take(4 * M_cap);
    w.pkfin = (uint32_t*)take(4 * M_cap);
    w.bstart = (int*)take(4 * ((M_cap + RS_TILE - 1) / RS_TILE + 1));
    const long long nblk = (M_cap + RS_TILE - 1) / RS_TILE;
    const long long nh = (long long)(1 << RS_MAXBITS) * nblk;
    w.hist = (uint32_t*)take(4 * nh);
    const long long nscan = (nh > M_cap ? nh : M_cap);
    w.bsum = (uint64_t*)take(8 * ((nscan + SCAN_TILE - 1) / SCAN_TILE + 1));
    w.bytes = o;
    return w;
}

// Where phase 1 leaves the (view, depth, index) order of the records.
static uint32_t* order_buffer(const BinWs& w, int n_views) { return n_views > 1 ? w.dv1 : w.dv0; }

static int view_bits(int n_views)
{
    int b = 0;
    while ((1 << b) < n_views) ++b;
    return b;
}

}  // namespace dg

extern "C" size_t dg_bin_workspace_size(int64_t P, int32_t n_views, int64_t M_cap)
{
    if (P < 0 || M_cap < 0 || n_views < 1 || n_views > DG_MAX_VIEWS) return 0;
    return dg::bin_layout(nullptr, P * n_views, M_cap).bytes;
}

extern "C" dg_status dg_bin_count(const float* depth, const int32_t* tiles, int64_t P, int32_t n_views, void* ws,
                                  size_t ws_bytes, int64_t M_cap, int64_t* M_out, dg_stream stream)
{
    if (P < 0 || n_views < 1 || n_views > DG_MAX_VIEWS || P * n_views > (int64_t)UINT32_MAX || M_cap < 0 ||
        M_cap > (int64_t)UINT32_MAX) {
        dg_set_error("bad sizes P=%lld n_views=%d M_cap=%lld", (long long)P, n_views, (long long)M_cap);
        return DG_ERR_ARG;
    }
    if (!ws || !M_out || (P > 0 && (!depth || !tiles))) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    const long long N = P * n_views;
    const dg::BinWs w = dg::bin_layout((char*)ws, N, M_cap);
    if (ws_bytes < w.bytes) { dg_set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return DG_ERR_CAPACITY; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(w.ctl1, 0, w.ctl1_bytes, s);  // counters, error word, scan look-back
    if (N == 0) {
        cudaMemsetAsync(w.M, 0, sizeof(long long), s);
        cudaMemsetAsync(M_out, 0, sizeof(long long), s);
        return dg_check_launch("bin_count");
    }
    using namespace dg;
    const int vb = n_views > 1 ? view_bits(n_views + 1) : 0;
    const int npass = vb > 0 ? 5 : 4;
    const long long ntile = (N + RS_TILE - 1) / RS_TILE;
    const int hb = (int)(ntile < 152 * 4 ? ntile : 152 * 4);
    k_os_hist_depth<<<hb, RS_THREADS, 0, s>>>(depth, tiles, N, (uint32_t)P, (uint32_t)n_views, vb, w.ctl1,
                                              w.look[0]);
    k_os_base<<<1, 256, 0, s>>>(w.ctl1, npass);
    dg_note_launch(2);
    // 4 depth passes: (depth, index) -> 1 -> 0 -> 1 -> values only in dv0;
    // then the view pass dv0 -> dv1 (order_buffer tells which holds the result)
    auto pass = [&](int p, int bits) {
        OsPass ps;
        ps.look = w.look[p & 1];
        ps.look_next = p + 1 < npass ? w.look[(p + 1) & 1] : nullptr;
        ps.next_nbins = p + 1 < npass ? (p + 1 < 4 ? 256 : 1 << vb) : 0;
        ps.ctr = &w.ctl1->ctr[p];
        ps.base = w.ctl1->base[p];
        ps.err = &w.ctl1->err;
        ps.shift = p < 4 ? 8 * p : 0;
        ps.mask = (1u << bits) - 1u;
        return ps;
    };
    const int nblk = (int)ntile;
    k_os_pass<<<nblk, RS_THREADS, 0, s>>>(SrcDepth{depth, tiles}, w.dk1, w.dv1, nullptr, N, pass(0, 8));
    k_os_pass<<<nblk, RS_THREADS, 0, s>>>(SrcKV{w.dk1, w.dv1}, w.dk0, w.dv0, nullptr, N, pass(1, 8));
    k_os_pass<<<nblk, RS_THREADS, 0, s>>>(SrcKV{w.dk0, w.dv0}, w.dk1, w.dv1, nullptr, N, pass(2, 8));
    k_os_pass<<<nblk, RS_THREADS, 0, s>>>(SrcKV{w.dk1, w.dv1}, nullptr, w.dv0, nullptr, N, pass(3, 8));
    dg_note_launch(4);
    if (vb > 0) {
        k_os_pass<<<nblk, RS_THREADS, 0, s>>>(SrcView{w.dv0, tiles, (uint32_t)P, (uint32_t)n_views}, nullptr,
                                              w.dv1, nullptr, N, pass(4, vb));
        dg_note_launch();
    }
    const int sb = (int)((N + SCAN_TILE - 1) / SCAN_TILE);
    k_os_scan<<<sb, SCAN_THREADS, 0, s>>>(LoadTilesInOrder{tiles, order_buffer(w, n_views)}, N, w.poff, w.slook,
                                          &w.ctl1->ctr[OS_MAXPASS - 1], w.M, &w.ctl1->err);
    dg_note_launch();
    cudaMemcpyAsync(M_out, w.M, sizeof(long long), cudaMemcpyDeviceToDevice, s);
    return dg_check_launch("bin_count");
}

bool dg_check_cameras(const dg_camera* cams, int n_views);

extern "C" dg_status dg_bin_sort(const float* feat, const int32_t* radius, int64_t P, const dg_camera* cams,
                                 int32_t n_views, int32_t tile, void* ws, size_t ws_bytes, int64_t M_cap,
                                 uint32_t* gid, uint32_t* ranges, int32_t* status, dg_stream stream)
{
    if (!dg_check_cameras(cams, n_views)) return DG_ERR_ARG;
    if (tile < 1 || tile > 64) { dg_set_error("bad tile %d", tile); return DG_ERR_ARG; }
    if (P < 0 || P * n_views > (int64_t)UINT32_MAX || M_cap < 0 || M_cap > (int64_t)UINT32_MAX) {
        dg_set_error("bad sizes");
        return DG_ERR_ARG;
    }
    if (!ws || !ranges || !status || (P > 0 && (!feat || !radius)) || (M_cap > 0 && !gid)) {
        dg_set_error("null buffer");
        return DG_ERR_ARG;
    }
    const long long N = P * n_views;
    const dg::BinWs w = dg::bin_layout((char*)ws, N, M_cap);
    if (ws_bytes < w.bytes) { dg_set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return DG_ERR_CAPACITY; }
    dg::TileGrid tg;
    tg.n = n_views;
    long long n_tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        tg.TX[v] = (cams[v].width + tile - 1) / tile;
        tg.TY[v] = (cams[v].height + tile - 1) / tile;
        tg.off[v] = (int)n_tiles;
        n_tiles += (long long)tg.TX[v] * tg.TY[v];
    }
    tg.off[n_views] = (int)n_tiles;
    if (n_tiles > (1ll << 30)) { dg_set_error("too many tiles"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * n_tiles, s);
    cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    int bits = 0;
    while ((1ll << bits) < n_tiles) ++bits;
    const int b0 = dg::first_pass_bits(bits);
    const uint32_t mask0 = b0 > 0 ? (1u << b0) - 1u : 0u;
    const int nblk = (int)((M_cap + dg::RS_TILE - 1) / dg::RS_TILE);
    const int pb = (int)((N + 255) / 256);
    uint32_t* order = dg::order_buffer(w, n_views);
    if (N > 0 && nblk > 0) {
        dg::k_block_starts<<<pb, 256, 0, s>>>(w.poff, N, w.M, M_cap, w.bstart);
        dg_note_launch();
    }
    // emit pairs in (view, depth) order (slots from phase 1) with pass-0 histogram, or flag overflow
    dg::k_emit<<<nblk > 0 ? nblk : 1, dg::RS_THREADS, 0, s>>>((const float4*)feat, radius, order, w.poff, w.bstart,
                                                            N, (uint32_t)(P > 0 ? P : 1), w.M, M_cap, tile, tg, mask0,
                                                            w.pk0, w.pv0, w.hist, nblk > 0 ? nblk : 1, &w.ctl1->err,
                                                            status);
    dg_note_launch();
    if (M_cap == 0) return dg_check_launch("bin_sort");
    dg::SortBufs sb{w.hist, w.bsum};
    dg::radix_sort(w.pk0, w.pv0, w.pk1, w.pv1, w.pkfin, gid, w.M, M_cap, bits, sb, s, /*hist0_ready=*/bits > 0,
                   dg::kTileBallotPasses);
    const long long nq = (M_cap + 3) / 4;
    long long rb = (nq + 255) / 256;
    if (rb > 152 * 32) rb = 152 * 32;
    dg::k_ranges<<<(int)(rb > 0 ? rb : 1), 256, 0, s>>>(w.pkfin, w.M, M_cap, (uint2*)ranges);
    dg_note_launch();
    return dg_check_launch("bin_sort");
}

// ------------------------------------------------------------ look-back probe
namespace dg {
__global__ void k_lookback_probe(const uint64_t* look, long long t, int stride, int d, int max_polls,
                                 uint64_t* sum, int* err)
{
    *err = 0;
    __threadfence();
    *sum = os_lookback(look, t, stride, d, err, max_polls);
}
}  // namespace dg

extern "C" dg_status dg_lookback_probe(const uint64_t* look, int64_t tile, int32_t stride, int32_t digit,
                                       int32_t max_polls, uint64_t* sum, int32_t* err, dg_stream stream)
{
    if (!sum || !err || (tile > 0 && !look)) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (tile < 0 || stride < 1 || digit < 0 || digit >= stride) {
        dg_set_error("bad look-back probe: tile=%lld stride=%d digit=%d", (long long)tile, stride, digit);
        return DG_ERR_ARG;
    }
    if (max_polls < 0 || max_polls > dg::kLbPolls) {
        dg_set_error("max_polls %d outside 0..%d", max_polls, dg::kLbPolls);
        return DG_ERR_ARG;
    }
    dg::k_lookback_probe<<<1, 1, 0, (cudaStream_t)stream>>>(look, tile, stride, digit, max_polls, sum, err);
    dg_note_launch();
    return dg_check_launch("lookback_probe");
}
