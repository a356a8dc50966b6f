// render.cu -- Eq. 1 compositing per tile (forward) and its adjoint (backward).
//
// Persistent launches over all views: one CTA per resident slot, each taking
// work items from an atomic counter until none are left, so items of very
// different cost balance across the SMs and all views of a batch share one
// launch.  Each warp owns an 8-pixel-wide block of 4*PPT rows of a B x B
// tile, each lane PPT vertically adjacent pixels of one column.  A work item's
// list entries are streamed through shared memory in batches of B*B/PPT
// records (one coalesced 48-byte gather per thread per batch); every staged
// record is then evaluated for the thread's PPT pixels.
//
// Work items.  Without splitting, an item is a whole tile.  A tile's list is
// walked in order, so a tile with a long list is a serial chain that no other
// SM can help with; at low resolution (few tiles, thousands of entries each)
// those chains set the time of the launch.  With splitting, a tile whose list
// is longer than L entries becomes ceil(n/L) chunks of L entries, each its own
// work item.  Eq. 1 composes over chunks: the transmittance in front of
// chunk c is the product of the (1 - alpha) factors of chunks 0..c-1, and the
// colour is the sum of the chunks' contributions.  Three passes keep the
// result that of the sequential rule, early stop included:
//   1. product pass: each chunk but the last computes, per pixel, the product
//      of its (1 - alpha) factors starting from 1, stopping as soon as the
//      product drops below the stop threshold (from then on the pixel has
//      stopped whatever the transmittance in front of the chunk);
//   2. compositing pass: each chunk starts from T_in = product of the earlier
//      chunks' products and applies Eq. 1 with the stop rule exactly; a pixel
//      whose T_in is already below the threshold stopped in an earlier chunk;
//   3. combine: per pixel, the colour sum over chunks, T_final from the chunk
//      where compositing stopped (else the last chunk), last = the largest
//      last of any chunk; and, for the backward, the colour behind each chunk.
// The backward takes the same items: a chunk starts from its own end
// transmittance and the colour behind it instead of T_final and T_final * bg.
// By default lists are split only when the batch has fewer than two tiles per
// resident CTA, with L = max(64, M / resident CTAs); L is raised where needed
// to keep the chunk count within the workspace.
//
//   Forward: front to back; an item stops once every pixel has terminated
//   (__syncthreads_count).
//   Backward: back to front from each pixel's last contributor; the
//   transmittance in front of entry j is recovered as T_j = T_{j+1} / (1 - a_j).
//   A thread first sums its PPT pixels' partial gradients, the warp then sums
//   the nine values by recursive halving (12 shuffles) and nine lanes add the
//   totals with one atomic instruction; warps with no contributing pixel skip
//   the reduction.
// Tile-level skip: while a batch is staged, each entry is tested once against
// the whole tile: the minimum of its quadratic form over the rectangle of the
// tile's pixel centres (closed form on the four edges when the mean lies
// outside).  If even that maximum alpha is below 1/255 (with a margin that
// absorbs float32 rounding of the per-pixel evaluation), every pixel would
// skip the entry, so it is dropped from the batch (stable compaction; the
// original list position is kept for `last`).  Results are unchanged.
#include <climits>
#include <stdlib.h>
#include <string.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "radix.cuh"

namespace dg {


// Pixel layout of a work item: warp w owns an 8-pixel-wide block of 4*PPT
// rows (blocks tile the B x B tile row-major); lane l owns column l % 8 and the
// PPT adjacent rows (l / 8) * PPT + k.
template <int B, int PPT>
__device__ inline void pix_of(int tid, int* lx, int* ly0)
{
    constexpr int NBX = B / 8;
    const int w = tid >> 5, l = tid & 31;
    *lx = (w % NBX) * 8 + (l & 7);
    *ly0 = (w / NBX) * (4 * PPT) + (l >> 3) * PPT;
}

// 2^x on the MUFU unit (ex2.approx, flush-to-zero).
__device__ inline float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Forward: list entries evaluated per loop iteration (a launch-shape constant;
// the result does not depend on it).
#ifndef DG_FWD_UNROLL
#define DG_FWD_UNROLL 2
#endif
constexpr int kFwdUnroll = DG_FWD_UNROLL;
// Backward: list entries whose quadratic forms are formed per loop iteration.
#ifndef DG_BWD_UNROLL
#define DG_BWD_UNROLL 1
#endif
constexpr int kBwdUnroll = DG_BWD_UNROLL;

constexpr float kLog2e = 1.4426950408889634f;
// log2(1/255): the alpha >= 1/255 test is taken in the log2 domain, before the
// exponential, identically in the forward and the backward
constexpr float kLog2AlphaMin = -7.994353436858858f;

// Backward: a warp whose contributing lanes number at most this many adds their
// partial gradients with per-lane vector atomics instead of reducing first
// (0: always reduce; 16 measured fastest on the 2M-Gaussian full-resolution
// step).  A launch-shape constant: results differ only in the
// order of the float additions.
#ifndef DG_BWD_DIRECT_LANES
#define DG_BWD_DIRECT_LANES 16
#endif
constexpr int kBwdDirectLanes = DG_BWD_DIRECT_LANES;

// Stable block-wide compaction index of `keep`; *total = number kept.  Ends with a barrier.
template <int NT>
__device__ inline int compact_index(bool keep, int* s_w, int* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_w[w] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const int c = s_w[i];
        pre += i < w ? c : 0;
        tot += c;
    }
    *total = tot;
    __syncthreads();
    return pre + __popc(bal & ((1u << lane) - 1u));
}

// One projected record as (u, v, A, B), (C, o, r, g), b.  REC 0: the FP32
// record of dg_project (three float4).  REC 1: the mixed-precision record of
// dg_pack_records (24 bytes: u, v float32 | A, B float16 | C, o float16 |
// r, g bfloat16 | b bfloat16, pad), widened to float32 here; all arithmetic
// after the load is float32.
template <int REC>
__device__ inline void load_record(const void* __restrict__ feat, uint32_t g, float4& a, float4& b, float& c)
{
    if (REC == 0) {
        const float4* f = (const float4*)feat + 3 * (size_t)g;
        a = f[0];
        b = f[1];
        c = f[2].x;
    } else {
        const uint2* f = (const uint2*)feat + 3 * (size_t)g;
        const uint2 w0 = f[0], w1 = f[1], w2 = f[2];
        __half2 ab, co;
        __nv_bfloat162 rg;
        memcpy(&ab, &w1.x, 4);
        memcpy(&co, &w1.y, 4);
        memcpy(&rg, &w2.x, 4);
        const float2 fab = __half22float2(ab), fco = __half22float2(co), frg = __bfloat1622float2(rg);
        a = make_float4(__uint_as_float(w0.x), __uint_as_float(w0.y), fab.x, fab.y);
        b = make_float4(fco.x, fco.y, frg.x, frg.y);
        c = __uint_as_float(w2.y << 16);  // bfloat16 in the low half: its float32 is the bits shifted up
    }
}

// Views of one launch: image sizes, tile grids and where each view's tiles and
// pixels start in the global tile range table and the concatenated images.
struct RViews {
    int n;
    int total;                      // tiles of all views
    int W[DG_MAX_VIEWS], H[DG_MAX_VIEWS], TX[DG_MAX_VIEWS];
    int toff[DG_MAX_VIEWS + 1];
    long long poff[DG_MAX_VIEWS];   // first pixel of each view
    float bg0, bg1, bg2;
};

// Head of the render workspace.  The forward writes the split plan here and
// in the arrays after it; the backward of the same batch reads it.
struct RHdr {
    int cnt_prod, cnt_fwd, cnt_bwd, cnt_pad;  // work counters of the three persistent launches
    int planned;                              // 1: items/sitems hold a split plan
    int L;                                    // chunk length of that plan
    int n_items, n_slots;                     // items (all chunks), chunks of split tiles
    long long M;                              // entries in the range table
    long long totals;                         // scan total: items (low 32 bits), split chunks (high 32)
};
static_assert(sizeof(RHdr) <= 256, "render header");

// Per-pixel state of split chunks: planes [cap][B*B], chunk slot s = slot0 + c.
struct Slots {
    float* prod;   // product of the chunk's (1 - alpha), pass 1
    float* tout;   // transmittance at the chunk's end (or where compositing stopped)
    float* c0;     // colour added by the chunk; after the combine, the colour behind it
    float* c1;
    float* c2;
    int* last;     // 1-based list position of the chunk's last blend | kStopFlag if it stopped there
    int* nbl;      // entries blended in the chunk
    int* stop;     // list position where compositing stopped (-1 if not in this chunk)
};
constexpr int kStopFlag = 1 << 30;

struct SplitCfg {
    int Lreq;  // > 0: requested chunk length; 0: automatic
    int R;     // resident CTAs of the compositing launch
    int cap;   // chunk slots in the workspace
};

// Shortest automatic chunk (entries): shorter chunks fill more CTAs but give
// the combine pass more chunks to walk per pixel.
#ifndef DG_SPLIT_MIN_LEN
#define DG_SPLIT_MIN_LEN 64
#endif

// Chunk length for M entries: requested or max(DG_SPLIT_MIN_LEN, M/R), raised
// to 2M/cap so that the chunks of split tiles (each tile has n > L, so
// ceil(n/L) < 2n/L) never exceed the slots.
__host__ __device__ inline int split_len(long long M, SplitCfg s)
{
    long long L = s.Lreq > 0 ? s.Lreq : (M + s.R - 1) / s.R;
    if (s.Lreq <= 0 && L < DG_SPLIT_MIN_LEN) L = DG_SPLIT_MIN_LEN;
    const long long Lcap = (2 * M + s.cap - 1) / s.cap;
    if (L < Lcap) L = Lcap;
    if (L < 1) L = 1;
    if (L > (INT_MAX >> 2)) L = INT_MAX >> 2;
    return (int)L;
}

struct LoadLen {
    const uint2* ranges;
    __device__ uint64_t operator()(long long t) const { const uint2 r = ranges[t]; return (uint64_t)(r.y - r.x); }
};
// Items (low 32 bits) and split chunks (high 32 bits) of tile t.
struct LoadChunks {
    const uint2* ranges;
    const RHdr* hdr;
    SplitCfg cfg;
    __device__ uint64_t operator()(long long t) const
    {
        const long long L = split_len(hdr->M, cfg);
        const uint2 r = ranges[t];
        const long long n = (long long)(r.y - r.x);
        if (n <= L) return 1;
        const uint64_t k = (uint64_t)((n + L - 1) / L);
        return (k << 32) | k;
    }
};

__global__ void k_plan_items(const uint2* __restrict__ ranges, int n_tiles, RHdr* hdr, SplitCfg cfg,
                             const uint64_t* __restrict__ toff, int4* __restrict__ items, int4* __restrict__ sitems)
{
    const long long M = hdr->M;
    const int L = split_len(M, cfg);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long tot = (unsigned long long)hdr->totals;
        hdr->L = L;
        hdr->n_items = (int)(tot & 0xffffffffull);
        hdr->n_slots = (int)(tot >> 32);
        hdr->planned = 1;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        const long long n = (long long)(r.y - r.x);  // as counted by LoadChunks
        const uint64_t off = toff[t];
        const int io = (int)(off & 0xffffffffull), so = (int)(off >> 32);
        if (n <= L) {
            items[io] = make_int4(t, 0, 1, -1);
            continue;
        }
        const int k = (int)((n + L - 1) / L);
        for (int c = 0; c < k; ++c) {
            const int4 w = make_int4(t, c, k, so);
            items[io + c] = w;
            sitems[so + c] = w;
        }
    }
}

// A work item: tile (global over views), chunk c of nch, first chunk slot
// (-1: the tile is not split), and the tile's place in its view.
struct Item { int tile, c, nch, slot0, v, tx, ty, W, H; long long poff; };

// Next work item of this CTA from `list` (or tile `index` when list is null);
// item.tile < 0: none left.  Ends with a barrier.
__device__ inline Item next_item(int* counter, int count, const int4* list, const RViews& rv, int4* s_item)
{
    if (threadIdx.x == 0) {
        const int i = atomicAdd(counter, 1);
        int4 w = make_int4(-1, 0, 1, -1);
        if (i < count) w = list ? list[i] : make_int4(i, 0, 1, -1);
        *s_item = w;
    }
    __syncthreads();
    const int4 w = *s_item;
    __syncthreads();
    Item it;
    it.tile = w.x; it.c = w.y; it.nch = w.z; it.slot0 = w.w;
    if (it.tile < 0) return it;
    int v = 0;
    while (v + 1 < rv.n && it.tile >= rv.toff[v + 1]) ++v;
    const int t = it.tile - rv.toff[v];
    it.v = v;
    it.tx = t % rv.TX[v];
    it.ty = t / rv.TX[v];
    it.W = rv.W[v];
    it.H = rv.H[v];
    it.poff = rv.poff[v];
    return it;
}

// Per-pair blend flag written by the forward: 0 when no pixel of the item
// blended the entry; otherwise bit w set when a pixel of warp w's block did.
// With 8x8 tiles and one pixel per thread (two warps of 8x4 pixels, the
// layout of k_render_bwd_ep) bit 7 marks that the low bits are per-warp bits
// of that layout; other layouts set bit 0 only.
constexpr uint8_t kFlagWarpBits = 0x80;
template <int B, int PPT, int NW, int NS>
__device__ inline uint8_t blend_flag(const uint8_t (&s_bl)[NW][NS], int slot)
{
    uint8_t f = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) f |= s_bl[w][slot] ? 1 : 0;
    if (B == 8 && PPT == 1 && f) {
        f = kFlagWarpBits;
#pragma unroll
        for (int w = 0; w < NW; ++w) f |= s_bl[w][slot] ? (uint8_t)(1u << w) : 0;
    }
    return f;
}

// Compositing of one work item.  PROD: pass 1 of a split tile (product of
// the chunk's (1 - alpha) factors from 1, no colour).  Otherwise Eq. 1 over
// the item's entries from T_in, writing the final pixels (whole tile) or the
// chunk's slot (split tile).
template <int B, int PPT, bool PROD, int REC>
__global__ void __launch_bounds__(B * B / PPT)
k_render_fwd(const void* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, RViews rv, RHdr* hdr, const int4* __restrict__ items,
             const int4* __restrict__ sitems, Slots sl, uint8_t* __restrict__ flags, long long flags_cap,
             float* __restrict__ img, float* __restrict__ Tout, int* __restrict__ lastout,
             int* __restrict__ exout, int* __restrict__ blout)
{
    constexpr int NT = B * B / PPT;
    constexpr int NPIX = B * B;
    __shared__ float4 s_a[NT];    // u, v, a', b'  (prescaled conic, see below)
    __shared__ float2 s_q[NT];    // c', log2 o
    __shared__ float4 s_col[NT];  // r, g, b, list position (int bits)
    // staged entry blended by some pixel of warp w's block (one row per warp, no
    // two warps write the same byte)
    constexpr int NW = NT / 32;
    __shared__ uint8_t s_bl[NW][NT];
    __shared__ int s_w[NT / 32];
    __shared__ int4 s_item;
    const bool planned = hdr->planned != 0 && items != nullptr;
    const int L = planned ? hdr->L : INT_MAX;
    const int count = PROD ? hdr->n_slots : (planned ? hdr->n_items : rv.total);
    const int4* list = PROD ? sitems : (planned ? items : nullptr);
    int* counter = PROD ? &hdr->cnt_prod : &hdr->cnt_fwd;
    for (;;) {
    const Item it = next_item(counter, count, list, rv, &s_item);
    if (it.tile < 0) break;
    if (PROD && it.c == it.nch - 1) continue;  // the last chunk's product is never needed
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
    int lx, ly0;
    pix_of<B, PPT>(threadIdx.x, &lx, &ly0);
    const int x = tx * B + lx;
    const int y0 = ty * B + ly0;
    const float pxc = (float)x + 0.5f;
    const float tpx0 = (float)(tx * B) + 0.5f, tpx1 = tpx0 + (float)(B - 1);
    const float tpy0 = (float)(ty * B) + 0.5f, tpy1 = tpy0 + (float)(B - 1);
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const bool split = it.slot0 >= 0;
    const int lo = split ? it.c * L : 0;
    const int hi = split ? (int)min((long long)n, (long long)lo + L) : n;
    float pyc[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT];
    int last[PPT], stop[PPT], nbl[PPT];
    bool done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k;
        pyc[k] = (float)y + 0.5f;
        T[k] = 1.f; c0[k] = c1[k] = c2[k] = 0.f;
        last[k] = 0; stop[k] = -1; nbl[k] = 0;
        done[k] = !(x < W && y < H);
        if (!PROD && split && it.c > 0) {
            // transmittance in front of the chunk: product of the earlier chunks' products
            const int p = (ly0 + k) * B + lx;
            for (int c = 0; c < it.c; ++c) T[k] *= sl.prod[(size_t)(it.slot0 + c) * NPIX + p];
            if (T[k] < kTMin) done[k] = true;  // stopped in an earlier chunk
        }
    }
    bool alldone = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) alldone = alldone && done[k];
    // flag bytes of the previous batch, written once the next barrier has
    // passed (every lane's blends of that batch are then in s_bl, and the next
    // staging writes s_bl only after compact_index's barriers)
    int pj = -1, pslot = 0;
    bool pkeep = false;
    auto write_flags = [&]() {
        if (PROD || !flags || pj < 0) return;
        const long long gj = (long long)rg.x + pj;
        if (pj < hi && gj < flags_cap) flags[gj] = pkeep ? blend_flag<B, PPT>(s_bl, pslot) : 0;
    };
    for (int base = lo; base < hi; base += NT) {
        if (__syncthreads_count(alldone) == NT) break;
        write_flags();
        const int j = base + (int)threadIdx.x;
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        if (j < hi) {
            const uint32_t g = gid[rg.x + j];
            load_record<REC>(feat, g, ga, gb, gc);
            keep = !tile_skip(ga, gb, tpx0, tpx1, tpy0, tpy1);
        }
        int cnt;
        const int slot = compact_index<NT>(keep, s_w, &cnt);
        if (keep) {
            // prescaled: p = log2(e) * power = dx (a' dx + b' dy) + c' dy^2, alpha = 2^(p + log2 o)
            s_a[slot] = make_float4(ga.x, ga.y, -0.5f * kLog2e * ga.z, -kLog2e * ga.w);
            s_q[slot] = make_float2(-0.5f * kLog2e * gb.x, __log2f(gb.y));
            s_col[slot] = make_float4(gb.z, gb.w, gc, __int_as_float(j));
#pragma unroll
            for (int w = 0; w < NW; ++w) s_bl[w][slot] = 0;
        }
        __syncthreads();
        // Eq. 1 for entry kk at the thread's pixel k, given the entry's power p
        // (log2 scale) and e = p + log2 o
        auto blend = [&](int k, int kk, float p, float e) {
            if (done[k] || !(p <= 0.f && e >= kLog2AlphaMin)) return;
            const float alpha = fminf(kAlphaMax, ex2_approx(e));
            const float Tn = fmaf(-alpha, T[k], T[k]);
            const float4 col = s_col[kk];
            const int pos = __float_as_int(col.w);
            if (Tn < kTMin) {
                done[k] = true;
                stop[k] = pos;
                if (PROD) T[k] = Tn;  // below the threshold: every later chunk is stopped
            } else {
                if (!PROD) {
                    const float w = alpha * T[k];
                    c0[k] += w * col.x;
                    c1[k] += w * col.y;
                    c2[k] += w * col.z;
                    last[k] = pos + 1;
                    ++nbl[k];
                    s_bl[threadIdx.x >> 5][kk] = 1;
                }
                T[k] = Tn;
            }
        };
        // DG_FWD_UNROLL entries per iteration: their quadratic forms do not depend
        // on the transmittance chain, so all are evaluated before any is blended
        for (int kk = 0; kk < cnt && !alldone; kk += kFwdUnroll) {
            float pu[kFwdUnroll][PPT], eu[kFwdUnroll][PPT];
#pragma unroll
            for (int u = 0; u < kFwdUnroll; ++u) {
                const int ku = kk + u < cnt ? kk + u : cnt - 1;
                const float4 a = s_a[ku];
                const float2 q = s_q[ku];
                const float dx = a.x - pxc;
                const float adx = a.z * dx;
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float dy = a.y - pyc[k];
                    pu[u][k] = fmaf(dx, fmaf(a.w, dy, adx), q.x * dy * dy);
                    eu[u][k] = pu[u][k] + q.y;
                }
            }
#pragma unroll
            for (int u = 0; u < kFwdUnroll; ++u) {
                if (kk + u < cnt) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) blend(k, kk + u, pu[u][k], eu[u][k]);
                }
            }
            alldone = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) alldone = alldone && done[k];
        }
        // per list entry: blended by some pixel of this item (the backward
        // stages only those); every entry of the batch gets its byte
        pj = j;
        pkeep = keep;
        pslot = slot;
    }
    if (!PROD && flags) {
        __syncthreads();
        write_flags();
    }
    if (split) {
        const size_t s0 = (size_t)(it.slot0 + it.c) * NPIX;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const size_t s = s0 + (size_t)((ly0 + k) * B + lx);
            if (PROD) {
                sl.prod[s] = T[k];
            } else {
                sl.tout[s] = T[k];
                sl.c0[s] = c0[k]; sl.c1[s] = c1[k]; sl.c2[s] = c2[k];
                sl.last[s] = last[k] | (stop[k] >= 0 ? kStopFlag : 0);
                sl.nbl[s] = nbl[k];
                sl.stop[s] = stop[k];
            }
        }
        continue;
    }
    const size_t HW = (size_t)W * H;
    float* im = img + 3 * it.poff;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k;
        if (x < W && y < H) {
            const size_t pix = (size_t)y * W + x;
            im[pix] = c0[k] + T[k] * rv.bg0;
            im[HW + pix] = c1[k] + T[k] * rv.bg1;
            im[2 * HW + pix] = c2[k] + T[k] * rv.bg2;
            Tout[it.poff + pix] = T[k];
            lastout[it.poff + pix] = last[k];
            // entries visited: up to and including the one that stopped compositing
            if (exout) exout[it.poff + pix] = stop[k] >= 0 ? stop[k] + 1 : n;
            if (blout) blout[it.poff + pix] = nbl[k];
        }
    }
    }  // work items
}

// Pass 3 of split tiles: one CTA per split tile, one thread per pixel.
template <int B>
__global__ void __launch_bounds__(B * B)
k_render_combine(const uint2* __restrict__ ranges, RViews rv, const RHdr* hdr, const int4* __restrict__ sitems,
                 Slots sl, float* __restrict__ img, float* __restrict__ Tout, int* __restrict__ lastout,
                 int* __restrict__ exout, int* __restrict__ blout)
{
    constexpr int NPIX = B * B;
    if (!hdr->planned) return;
    const int count = hdr->n_slots;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int4 w = sitems[i];
        if (w.y != 0) continue;
        int v = 0;
        while (v + 1 < rv.n && w.x >= rv.toff[v + 1]) ++v;
        const int t = w.x - rv.toff[v];
        const int W = rv.W[v], H = rv.H[v];
        const int lx = (int)(threadIdx.x % B), ly = (int)(threadIdx.x / B);
        const int x = (t % rv.TX[v]) * B + lx, y = (t / rv.TX[v]) * B + ly;
        if (!(x < W && y < H)) continue;
        const uint2 rg = ranges[w.x];
        const int n = (int)(rg.y - rg.x);
        const int nch = w.z;
        const size_t p = (size_t)threadIdx.x;
        // A few tiles hold dozens of chunks each and only their blocks work, so
        // each walk loads CB chunks' fields before using any (chunk order, and
        // so every sum's rounding, unchanged).
        constexpr int CB = 8;
        float C0 = 0.f, C1 = 0.f, C2 = 0.f;
        int lastv = 0, nb = 0, cstop = -1;
        for (int cb = 0; cb < nch; cb += CB) {
            int lt[CB], nbv[CB];
            float a0[CB], a1[CB], a2[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                if (cb + j < nch) {
                    const size_t s = (size_t)(w.w + cb + j) * NPIX + p;
                    lt[j] = sl.last[s]; nbv[j] = sl.nbl[s];
                    a0[j] = sl.c0[s]; a1[j] = sl.c1[s]; a2[j] = sl.c2[s];
                }
            }
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                if (cb + j < nch) {
                    C0 += a0[j]; C1 += a1[j]; C2 += a2[j];
                    lastv = max(lastv, lt[j] & (kStopFlag - 1));
                    nb += nbv[j];
                    if ((lt[j] & kStopFlag) && cstop < 0) cstop = cb + j;
                }
            }
        }
        // T at the end: from the chunk where the pixel stopped, else the last chunk
        const size_t sf = (size_t)(w.w + (cstop >= 0 ? cstop : nch - 1)) * NPIX + p;
        const float Tf = sl.tout[sf];
        const int ex = cstop >= 0 ? sl.stop[sf] + 1 : n;
        // colour behind each chunk (the backward's starting S), back to front
        float S0 = Tf * rv.bg0, S1 = Tf * rv.bg1, S2 = Tf * rv.bg2;
        for (int cb = nch - 1; cb >= 0; cb -= CB) {
            float a0[CB], a1[CB], a2[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                if (cb - j >= 0) {
                    const size_t s = (size_t)(w.w + cb - j) * NPIX + p;
                    a0[j] = sl.c0[s]; a1[j] = sl.c1[s]; a2[j] = sl.c2[s];
                }
            }
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                if (cb - j >= 0) {
                    const size_t s = (size_t)(w.w + cb - j) * NPIX + p;
                    sl.c0[s] = S0; sl.c1[s] = S1; sl.c2[s] = S2;
                    S0 += a0[j]; S1 += a1[j]; S2 += a2[j];
                }
            }
        }
        const size_t HW = (size_t)W * H;
        const size_t pix = (size_t)y * W + x;
        float* im = img + 3 * rv.poff[v];
        im[pix] = C0 + Tf * rv.bg0;
        im[HW + pix] = C1 + Tf * rv.bg1;
        im[2 * HW + pix] = C2 + Tf * rv.bg2;
        Tout[rv.poff[v] + pix] = Tf;
        lastout[rv.poff[v] + pix] = lastv;
        if (exout) exout[rv.poff[v] + pix] = ex;
        if (blout) blout[rv.poff[v] + pix] = nb;
    }
}

// Sum of 9 per-lane values over the warp by recursive halving: at each step a
// lane keeps half of its values and receives its partner's partial sums of
// that half (12 shuffles instead of 45).  Returns the total of value `*idx`
// (0..8) on the lanes where *idx is valid (*idx = -1 elsewhere); both lanes of
// each final pair hold it, only the even one reports it.
__device__ inline float warp_sum9(const float v[9], int lane, int* idx)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a1[6];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float lo = v[i], hi = i + 5 < 9 ? v[i + 5] : 0.f;
        const float keep = b4 ? hi : lo, send = b4 ? lo : hi;
        a1[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    a1[5] = 0.f;
    float a2[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float keep = b3 ? a1[i + 3] : a1[i], send = b3 ? a1[i] : a1[i + 3];
        a2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    a2[3] = 0.f;
    float a3[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float keep = b2 ? a2[i + 2] : a2[i], send = b2 ? a2[i] : a2[i + 2];
        a3[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float a4;
    {
        const float keep = b1 ? a3[1] : a3[0], send = b1 ? a3[0] : a3[1];
        a4 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    a4 += __shfl_xor_sync(0xffffffffu, a4, 1);
    const int i2 = (b2 ? 2 : 0) + (b1 ? 1 : 0);        // index into a2 (3 = padding)
    const int i1 = (b3 ? 3 : 0) + i2;                   // index into a1 (5 = padding)
    const int i0 = (b4 ? 5 : 0) + i1;                   // original index (9 = padding)
    *idx = ((lane & 1) == 0 && i2 < 3 && i1 < 5 && i0 < 9) ? i0 : -1;
    return a4;
}

template <int B, int PPT, int REC>
__global__ void __launch_bounds__(B * B / PPT)
k_render_bwd(const void* __restrict__ feat, const uint32_t* __restrict__ gid,
             const uint2* __restrict__ ranges, RViews rv, RHdr* hdr, const int4* __restrict__ items, Slots sl,
             const uint8_t* __restrict__ flags, long long flags_cap,
             const float* __restrict__ Tfin, const int* __restrict__ lastin,
             const float* __restrict__ dLdimg, float4* __restrict__ grad2d)
{
    constexpr int NT = B * B / PPT;
    constexpr int NPIX = B * B;
    __shared__ float4 s_a[NT];    // u, v, a', b'  (the forward's prescaled conic)
    __shared__ float2 s_q[NT];    // c', log2 o
    __shared__ float4 s_k[NT];    // A, B, C, 1/o
    __shared__ float4 s_col[NT];  // r, g, b, list position (int bits)
    __shared__ uint32_t s_g[NT];
    __shared__ int s_w[NT / 32];
    __shared__ int s_n;
    __shared__ int4 s_item;
    const float bg0 = rv.bg0, bg1 = rv.bg1, bg2 = rv.bg2;
    // (a whole-tile walk is exact whatever the forward did; items is null when
    // the workspace was laid out without splitting)
    const bool planned = hdr->planned != 0 && items != nullptr;
    const int L = planned ? hdr->L : INT_MAX;
    const int count = planned ? hdr->n_items : rv.total;
    for (;;) {
    const Item it = next_item(&hdr->cnt_bwd, count, planned ? items : nullptr, rv, &s_item);
    if (it.tile < 0) break;
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
    int lx, ly0;
    pix_of<B, PPT>(threadIdx.x, &lx, &ly0);
    const int x = tx * B + lx;
    const int y0 = ty * B + ly0;
    const float pxc = (float)x + 0.5f;
    const float tpx0 = (float)(tx * B) + 0.5f, tpx1 = tpx0 + (float)(B - 1);
    const float tpy0 = (float)(ty * B) + 0.5f, tpy1 = tpy0 + (float)(B - 1);
    const uint2 rg = ranges[tile];
    const int nlist = (int)(rg.y - rg.x);
    const bool split = it.slot0 >= 0;
    const int lo = split ? it.c * L : 0;
    const int hi = split ? (int)min((long long)nlist, (long long)lo + L) : nlist;
    const size_t HW = (size_t)W * H;
    // per pixel: transmittance, dL/dC, and gS = dL/dC . S where S is the
    // colour composited behind the current entry (the only way S enters the
    // gradient: dL/dalpha_j = T_j (g . c_j) - (g . S_j) / (1 - alpha_j))
    float pyc[PPT], T[PPT], g0[PPT], g1[PPT], g2[PPT], gS[PPT];
    int lastp[PPT];
    int mylast = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int y = y0 + k;
        pyc[k] = (float)y + 0.5f;
        T[k] = 1.f; g0[k] = g1[k] = g2[k] = 0.f; lastp[k] = 0;
        gS[k] = 0.f;
        if (x < W && y < H) {
            const size_t pix = (size_t)y * W + x;
            const float* dl = dLdimg + 3 * it.poff;
            lastp[k] = lastin[it.poff + pix];
            g0[k] = dl[pix];
            g1[k] = dl[HW + pix];
            g2[k] = dl[2 * HW + pix];
            if (split) {
                // the chunk's end transmittance and the colour behind the chunk
                const size_t s = (size_t)(it.slot0 + it.c) * NPIX + (size_t)((ly0 + k) * B + lx);
                T[k] = sl.tout[s];
                gS[k] = g0[k] * sl.c0[s] + g1[k] * sl.c1[s] + g2[k] * sl.c2[s];
            } else {
                T[k] = Tfin[it.poff + pix];
                gS[k] = T[k] * (g0[k] * bg0 + g1[k] * bg1 + g2[k] * bg2);  // behind the last entry: T bg
            }
        }
        mylast = max(mylast, lastp[k]);
    }
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(&s_n, mylast);
    __syncthreads();
    // never walk past the item's own entries, whatever `last` holds
    const int top = min(s_n, hi);
    const int lane = threadIdx.x & 31;
    // this lane's partial gradient of the current entry: du, dv, dA, dB, dC,
    // d opacity, d r, d g, d b.  With one pixel per thread each blending lane
    // assigns all nine (no per-entry zeroing; lanes that did not blend are
    // masked at the reduction); with several pixels they accumulate from zero.
    float vd[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) vd[i] = 0.f;
    for (int base = top > lo ? lo + ((top - lo - 1) / NT) * NT : lo - 1; base >= lo; base -= NT) {
        const int j = base + (int)threadIdx.x;
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        uint32_t g = 0;
        if (j < top) {
            const long long gj = (long long)rg.x + j;
            if (flags && gj < flags_cap) {
                // the forward's record of this entry: blended by some pixel of the
                // tile or not (an entry no pixel blended has no gradient)
                keep = flags[gj] != 0;
                if (keep) {
                    g = gid[gj];
                    load_record<REC>(feat, g, ga, gb, gc);
                }
            } else {
                g = gid[gj];
                load_record<REC>(feat, g, ga, gb, gc);
                keep = !tile_skip(ga, gb, tpx0, tpx1, tpy0, tpy1);
            }
        }
        int cnt;
        const int slot = compact_index<NT>(keep, s_w, &cnt);
        if (keep) {
            s_g[slot] = g;
            s_a[slot] = make_float4(ga.x, ga.y, -0.5f * kLog2e * ga.z, -kLog2e * ga.w);
            s_q[slot] = make_float2(-0.5f * kLog2e * gb.x, __log2f(gb.y));
            s_k[slot] = make_float4(ga.z, ga.w, gb.x, __frcp_rn(gb.y));
            s_col[slot] = make_float4(gb.z, gb.w, gc, __int_as_float(j));
        }
        __syncthreads();
        // one list entry, given its quadratic forms at this thread's pixels
        auto entry = [&](int kk, const float4& col, float dx, const float* dyv, const float* pv) {
            const int pos = __float_as_int(col.w);
            if (!__any_sync(0xffffffffu, pos < mylast)) return;
            const float cr = col.x, cg = col.y, cb = col.z;
            const float qy = s_q[kk].y;
            if (PPT > 1) {
#pragma unroll
                for (int i = 0; i < 9; ++i) vd[i] = 0.f;
            }
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (pos < lastp[k]) {
                    // the forward's blend test and alpha, bit for bit
                    const float dy = dyv[k];
                    const float p = pv[k];
                    const float e = p + qy;
                    if (p <= 0.f && e >= kLog2AlphaMin) {
                        const float raw = ex2_approx(e);
                        const float alpha = fminf(kAlphaMax, raw);
                        const float4 kc = s_k[kk];  // A, B, C, 1/o
                        any = true;
                        // hardware reciprocal (about 1 ulp; 1 - alpha is in [0.01, 1]): the
                        // exactly rounded one costs a measured 6% of the kernel
                        const float inv = __fdividef(1.f, 1.f - alpha);
                        T[k] *= inv;  // transmittance in front of this entry
                        const float wT = alpha * T[k];
                        const float gcol = fmaf(g0[k], cr, fmaf(g1[k], cg, g2[k] * cb));
                        const float dLda = fmaf(T[k], gcol, -gS[k] * inv);
                        gS[k] = fmaf(wT, gcol, gS[k]);
                        // below the clamp: d alpha / d o = exp(power), d alpha / d power = alpha
                        const float dp = raw <= kAlphaMax ? dLda * alpha : 0.f;
                        const float dopa = raw <= kAlphaMax ? dLda * raw * kc.w : 0.f;
                        const float qx = dp * dx, qdy = dp * dy;
                        const float v[9] = {-fmaf(kc.x, qx, kc.y * qdy), -fmaf(kc.y, qx, kc.z * qdy),
                                            -0.5f * qx * dx, -qx * dy, -0.5f * qdy * dy, dopa,
                                            wT * g0[k], wT * g1[k], wT * g2[k]};
#pragma unroll
                        for (int i = 0; i < 9; ++i) vd[i] = PPT == 1 ? v[i] : vd[i] + v[i];
                    }
                }
            }
            const unsigned anym = __ballot_sync(0xffffffffu, any);
            if (!anym) return;
            if (kBwdDirectLanes > 0 && __popc(anym) <= kBwdDirectLanes) {
                // few contributing lanes: each adds its own partial sums (three
                // vector atomics) instead of the 12-shuffle warp reduction
                if (any) {
                    float4* gp = grad2d + 3 * (size_t)s_g[kk];
                    atomicAdd(gp, make_float4(vd[0], vd[1], vd[2], vd[3]));
                    atomicAdd(gp + 1, make_float4(vd[4], vd[5], vd[6], vd[7]));
                    atomicAdd((float*)(gp + 2), vd[8]);
                }
                return;
            }
            float vals[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) vals[i] = any ? vd[i] : 0.f;
            int idx;
            const float tot = warp_sum9(vals, lane, &idx);
            if (idx >= 0) atomicAdd((float*)(grad2d + 3 * (size_t)s_g[kk]) + idx, tot);
        };
        // kBwdUnroll entries per iteration, back to front: their quadratic forms
        // are formed first (independent of the transmittance chain)
        for (int kk = cnt - 1; kk >= 0; kk -= kBwdUnroll) {
            float4 colu[kBwdUnroll];
            float dxu[kBwdUnroll], dyu[kBwdUnroll][PPT], pu[kBwdUnroll][PPT];
#pragma unroll
            for (int u = 0; u < kBwdUnroll; ++u) {
                const int ku = kk - u >= 0 ? kk - u : kk;
                colu[u] = s_col[ku];
                const float4 a = s_a[ku];
                const float2 q = s_q[ku];
                dxu[u] = a.x - pxc;
                const float adx = a.z * dxu[u];
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    dyu[u][k] = a.y - pyc[k];
                    pu[u][k] = fmaf(dxu[u], fmaf(a.w, dyu[u][k], adx), q.x * dyu[u][k] * dyu[u][k]);
                }
            }
#pragma unroll
            for (int u = 0; u < kBwdUnroll; ++u)
                if (kk - u >= 0) entry(kk - u, colu[u], dxu[u], dyu[u], pu[u]);
        }
        __syncthreads();
    }
    }  // work items
}

constexpr int kEpG = 16;
constexpr int kEpPitch = 33;  // float2 per entry row of the (entry, pixel) matrix: 32 pixels + 1

// Next work item of this warp: item index w covers tile (or chunk) w / 2 and
// the 8x4 pixel block w % 2 of it; *blk receives the block.  Warp-uniform.
__device__ inline Item next_item_warp(int* counter, int count, const int4* list, const RViews& rv, int* blk)
{
    int w = 0;
    if ((threadIdx.x & 31) == 0) w = atomicAdd(counter, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    Item it;
    it.tile = -1;
    if (w >= 2 * count) return it;
    const int i = w >> 1;
    *blk = w & 1;
    const int4 q = list ? list[i] : make_int4(i, 0, 1, -1);
    it.tile = q.x; it.c = q.y; it.nch = q.z; it.slot0 = q.w;
    int v = 0;
    while (v + 1 < rv.n && it.tile >= rv.toff[v + 1]) ++v;
    const int t = it.tile - rv.toff[v];
    it.v = v;
    it.tx = t % rv.TX[v];
    it.ty = t / rv.TX[v];
    it.W = rv.W[v];
    it.H = rv.H[v];
    it.poff = rv.poff[v];
    return it;
}

// Backward of 8x8 tiles with one pixel per thread, entry-parallel gradient
// sums, each warp on its own.  A work item is one 8x4 block of a tile (or of a
// chunk of a split tile), taken by the warp from the shared counter; no
// CTA-wide barrier, so the two blocks of a tile, whose lists and walks
// differ, do not wait for each other.  The warp walks back from the largest
// `last` of its own 32 pixels and stages, in batches of 32 candidates, only
// the entries some pixel of its block blended (the forward's per-block bit,
// or every flagged entry when the forward ran at another launch shape; the
// block-rectangle alpha test when there are no flags).  Per group of 16
// staged entries:
//   A. pixel-parallel (lane = pixel): walks the group's entries back to front
//      exactly as k_render_bwd (the forward's blend test bit for bit, T
//      recovered through 1/(1 - alpha), dL/dalpha from the running g . S) and
//      stores per (entry, pixel) the two scalars the gradient needs,
//      dp = dL/dpower and wT = alpha T (0, 0 where the pixel does not blend).
//      Four entries at a time: their tests, alphas and reciprocals do not
//      depend on the transmittance chain and are formed first;
//   B. entry-parallel (lane = entry of the group, one of two 8x2 halves of the
//      block): the sums over the half's pixels of dp dx, dp dy, dp dx^2,
//      dp dx dy, dp dy^2 (dx, dy: Gaussian centre minus pixel centre) follow
//      from moments of dp about the half's centre, whose pixel offsets are
//      compile-time constants (per row sum dp and sum dp ox, and sum dp ox^2;
//      ox in -3.5 .. 3.5, oy = -0.5 / +0.5; expanding about the half's own
//      centre keeps cancellation small), plus the colour sums sum wT dL/dC;
//      one shuffle adds the halves and three vector atomics per entry go out.
// The opacity term uses d alpha / d o = alpha / o below the clamp: sum(dp) / o.
template <int REC>
__global__ void __launch_bounds__(64, 14)
k_render_bwd_ep(const void* __restrict__ feat, const uint32_t* __restrict__ gid,
                const uint2* __restrict__ ranges, RViews rv, RHdr* hdr, const int4* __restrict__ items, Slots sl,
                const uint8_t* __restrict__ flags, long long flags_cap,
                const float* __restrict__ Tfin, const int* __restrict__ lastin,
                const float* __restrict__ dLdimg, float4* __restrict__ grad2d)
{
    constexpr int B = 8, NPIX = 64;
    __shared__ float4 s_a[2][32];    // u, v, a', b'  (the forward's prescaled conic)
    __shared__ float2 s_q[2][32];    // c', log2 o
    __shared__ float4 s_k[2][32];    // A, B, C, 1/o
    __shared__ float4 s_col[2][32];  // r, g, b, list position (int bits)
    __shared__ uint32_t s_g[2][32];
    __shared__ float2 s_m[2][kEpG * kEpPitch];  // per warp: [entry][pixel] (dp, wT)
    __shared__ float4 s_gp[2][32];               // per warp: dL/dC of its pixels
    const float bg0 = rv.bg0, bg1 = rv.bg1, bg2 = rv.bg2;
    const bool planned = hdr->planned != 0 && items != nullptr;
    const int L = planned ? hdr->L : INT_MAX;
    const int count = planned ? hdr->n_items : rv.total;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float2* sm = s_m[wp];
    float4* wa = s_a[wp];
    float2* wq = s_q[wp];
    float4* wk = s_k[wp];
    float4* wc = s_col[wp];
    uint32_t* wg = s_g[wp];
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
    int blk = 0;
    const Item it = next_item_warp(&hdr->cnt_bwd, count, planned ? items : nullptr, rv, &blk);
    if (it.tile < 0) break;
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
    const int lx = lane & 7, ly0 = 4 * blk + (lane >> 3);
    const int x = tx * B + lx;
    const int y = ty * B + ly0;
    const float pxc = (float)x + 0.5f, pyc = (float)y + 0.5f;
    // this block's pixel centres: [bx0, bx1] x [by0, by1]
    const float bx0 = (float)(tx * B) + 0.5f, bx1 = bx0 + 7.f;
    const float by0 = (float)(ty * B + 4 * blk) + 0.5f, by1 = by0 + 3.f;
    const uint2 rg = ranges[tile];
    const int nlist = (int)(rg.y - rg.x);
    const bool split = it.slot0 >= 0;
    const int lo = split ? it.c * L : 0;
    const int hi = split ? (int)min((long long)nlist, (long long)lo + L) : nlist;
    const size_t HW = (size_t)W * H;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, gS = 0.f;
    int lastp = 0;
    if (x < W && y < H) {
        const size_t pix = (size_t)y * W + x;
        const float* dl = dLdimg + 3 * it.poff;
        lastp = lastin[it.poff + pix];
        g0 = dl[pix];
        g1 = dl[HW + pix];
        g2 = dl[2 * HW + pix];
        if (split) {
            const size_t sidx = (size_t)(it.slot0 + it.c) * NPIX + (size_t)(ly0 * B + lx);
            T = sl.tout[sidx];
            gS = g0 * sl.c0[sidx] + g1 * sl.c1[sidx] + g2 * sl.c2[sidx];
        } else {
            T = Tfin[it.poff + pix];
            gS = T * (g0 * bg0 + g1 * bg1 + g2 * bg2);
        }
    }
    s_gp[wp][lane] = make_float4(g0, g1, g2, 0.f);
    const int top = min(__reduce_max_sync(0xffffffffu, lastp), hi);
    // phase B: this lane's entry of the group and half of the block's pixels
    // (pixels 16 h .. 16 h + 15 = rows 2h, 2h + 1 of the block)
    const int be = lane & (kEpG - 1), bh = lane >> 4;
    const float bpx0 = bx0, bpy0 = by0 + (float)(2 * bh);
    __syncwarp();
    // the flag byte and Gaussian index of a batch are loaded one batch ahead,
    // so a batch waits only for its records (kNoFlag: no flag for the entry);
    // 14 blocks per SM (72 registers) leave room for them (16 blocks at 64
    // registers spilled: 0.466 -> 0.478 ms; 14 blocks without them 0.450,
    // with them 0.435 ms, 12 blocks 0.444 ms)
    constexpr uint32_t kNoFlag = 0x100u;
    const int base0 = top > lo ? lo + ((top - lo - 1) / 32) * 32 : lo - 1;
    uint32_t fn = kNoFlag, gn = 0;
    auto fetch = [&](int b) {
        const int jj = b + lane;
        fn = kNoFlag;
        gn = 0;
        if (b >= lo && jj < top) {
            const long long gj = (long long)rg.x + jj;
            if (flags && gj < flags_cap) fn = flags[gj];
            gn = gid[gj];
        }
    };
    fetch(base0);
    for (int base = base0; base >= lo; base -= 32) {
        const int j = base + lane;
        const uint32_t fcur = fn, g = gn;
        fetch(base - 32);
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        if (j < top) {
            if (fcur != kNoFlag) {
                keep = (fcur & kFlagWarpBits) ? ((fcur >> blk) & 1u) != 0 : fcur != 0;
                if (keep) load_record<REC>(feat, g, ga, gb, gc);
            } else {
                load_record<REC>(feat, g, ga, gb, gc);
                keep = !tile_skip(ga, gb, bx0, bx1, by0, by1);
            }
        }
        const uint32_t km = __ballot_sync(0xffffffffu, keep);
        const int cnt = __popc(km);
        if (keep) {
            const int slot = __popc(km & lt);
            wg[slot] = g;
            wa[slot] = make_float4(ga.x, ga.y, -0.5f * kLog2e * ga.z, -kLog2e * ga.w);
            wq[slot] = make_float2(-0.5f * kLog2e * gb.x, __log2f(gb.y));
            wk[slot] = make_float4(ga.z, ga.w, gb.x, __frcp_rn(gb.y));
            wc[slot] = make_float4(gb.z, gb.w, gc, __int_as_float(j));
        }
        __syncwarp();
        for (int kb = ((cnt - 1) / kEpG) * kEpG; kb >= 0 && cnt > 0; kb -= kEpG) {
            const int ke = min(cnt, kb + kEpG);
            // A: this lane's pixel over the group's entries, back to front, four at a time
            uint32_t mine = 0;
            for (int k0 = ke - 1; k0 >= kb; k0 -= 4) {
                float al[4], iv[4], gcl[4];
                bool bl[4], un[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int kk = k0 - u >= kb ? k0 - u : kb;
                    const float4 col = wc[kk];
                    const float4 a = wa[kk];
                    const float2 q = wq[kk];
                    const float dx = a.x - pxc, dy = a.y - pyc;
                    const float p = fmaf(dx, fmaf(a.w, dy, a.z * dx), q.x * dy * dy);
                    const float e = p + q.y;
                    bl[u] = k0 - u >= kb && __float_as_int(col.w) < lastp && p <= 0.f && e >= kLog2AlphaMin;
                    const float raw = ex2_approx(e);
                    al[u] = fminf(kAlphaMax, raw);
                    un[u] = raw <= kAlphaMax;
                    iv[u] = __fdividef(1.f, 1.f - al[u]);
                    gcl[u] = fmaf(g0, col.x, fmaf(g1, col.y, g2 * col.z));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (k0 - u < kb) break;
                    float dpv = 0.f, wTv = 0.f;
                    if (bl[u]) {
                        T *= iv[u];
                        wTv = al[u] * T;
                        const float dLda = fmaf(T, gcl[u], -gS * iv[u]);
                        gS = fmaf(wTv, gcl[u], gS);
                        dpv = un[u] ? dLda * al[u] : 0.f;
                        mine |= 1u << (k0 - u - kb);
                    }
                    sm[(k0 - u - kb) * kEpPitch + lane] = make_float2(dpv, wTv);
                }
            }
            const uint32_t used = __reduce_or_sync(0xffffffffu, mine);
            __syncwarp();
            if (used) {
                const int ek = kb + be;
                const bool act = ek < ke && ((used >> be) & 1u);
                float4 kc = make_float4(0.f, 0.f, 0.f, 0.f);
                float dx0 = 0.f, dy0 = 0.f;
                if (act) {
                    kc = wk[ek];
                    const float4 a = wa[ek];
                    dx0 = a.x - (bpx0 + 3.5f);
                    dy0 = a.y - (bpy0 + 0.5f);
                }
                float s0a = 0.f, s0b = 0.f, sxa = 0.f, sxb = 0.f, sxx = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
                const float2* row = sm + be * kEpPitch + 16 * bh;
                const float4* gpx = s_gp[wp] + 16 * bh;
#pragma unroll 1
                for (int r = 0; r < 2; ++r) {
                    float s0 = 0.f, sx = 0.f;
#pragma unroll
                    for (int px = 0; px < 8; ++px) {
                        const float2 m = row[8 * r + px];
                        const float4 gp = gpx[8 * r + px];
                        const float ox = (float)px - 3.5f;
                        s0 += m.x;
                        sx = fmaf(m.x, ox, sx);
                        sxx = fmaf(m.x, ox * ox, sxx);
                        c0 = fmaf(m.y, gp.x, c0);
                        c1 = fmaf(m.y, gp.y, c1);
                        c2 = fmaf(m.y, gp.z, c2);
                    }
                    if (r == 0) { s0a = s0; sxa = sx; } else { s0b = s0; sxb = sx; }
                }
                const float S0 = s0a + s0b, Sx = sxa + sxb, Sy = 0.5f * (s0b - s0a), Sxy = 0.5f * (sxb - sxa);
                const float Syy = 0.25f * S0;
                const float qx = fmaf(dx0, S0, -Sx), qy = fmaf(dy0, S0, -Sy);
                float acc[9];
                acc[0] = fmaf(kc.x, qx, kc.y * qy);
                acc[1] = fmaf(kc.y, qx, kc.z * qy);
                acc[2] = fmaf(dx0, fmaf(dx0, S0, -2.f * Sx), sxx);
                acc[3] = fmaf(dx0, fmaf(dy0, S0, -Sy), fmaf(-dy0, Sx, Sxy));
                acc[4] = fmaf(dy0, fmaf(dy0, S0, -2.f * Sy), Syy);
                acc[5] = S0;
                acc[6] = c0;
                acc[7] = c1;
                acc[8] = c2;
#pragma unroll
                for (int i = 0; i < 9; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 16);
                if (act && bh == 0) {
                    float4* gq = grad2d + 3 * (size_t)wg[ek];
                    atomicAdd(gq, make_float4(-acc[0], -acc[1], -0.5f * acc[2], -acc[3]));
                    atomicAdd(gq + 1, make_float4(-0.5f * acc[4], acc[5] * kc.w, acc[6], acc[7]));
                    atomicAdd((float*)(gq + 2), acc[8]);
                }
            }
            __syncwarp();
        }
    }
    __syncwarp();
    }  // work items
}

// Forward of 8x8 tiles with one pixel per thread, each warp on its own: a work
// item is one 8x4 block of a tile (or of a chunk of a split tile), taken per
// warp from the counter (the same compositing as k_render_fwd, pixel for
// pixel and bit for bit).  The warp stages its block's candidates in batches
// of 32 with the alpha test over the block's rectangle of pixel centres
// (tighter than the tile's), stops as soon as its own 32 pixels are done, and
// needs no CTA barrier.  Blend flags: the flag bytes are cleared before the
// launch, and each entry some pixel of the block blended gets bit 7 and the
// block's bit OR-ed into its byte (one 32-bit atomic OR per entry and block).
template <bool PROD, int REC>
// (16 blocks of 64 threads per SM, 64 registers: 0.366 -> 0.353 ms against the
// compiler's 56-register choice of 18 blocks)
__global__ void __launch_bounds__(64, 16)
k_render_fwd_w(const void* __restrict__ feat, const uint32_t* __restrict__ gid,
               const uint2* __restrict__ ranges, RViews rv, RHdr* hdr, const int4* __restrict__ items,
               const int4* __restrict__ sitems, Slots sl, uint8_t* __restrict__ flags, long long flags_cap,
               float* __restrict__ img, float* __restrict__ Tout, int* __restrict__ lastout,
               int* __restrict__ exout, int* __restrict__ blout)
{
    constexpr int B = 8, NPIX = 64;
    __shared__ float4 s_uv[2][16];   // entry pairs: (u, u', v, v')
    __shared__ float4 s_ab[2][16];   // (a, a', b, b') prescaled conic
    __shared__ float4 s_cl[2][16];   // (c, c', log2 o, log2 o')
    __shared__ float4 s_col[2][32];  // r, g, b, list position (int bits)
    const bool planned = hdr->planned != 0 && items != nullptr;
    const int L = planned ? hdr->L : INT_MAX;
    const int count = PROD ? hdr->n_slots : (planned ? hdr->n_items : rv.total);
    const int4* list = PROD ? sitems : (planned ? items : nullptr);
    int* counter = PROD ? &hdr->cnt_prod : &hdr->cnt_fwd;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float4* wuv = s_uv[wp];
    float4* wab = s_ab[wp];
    float4* wcl = s_cl[wp];
    float4* wc = s_col[wp];
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
    int blk = 0;
    const Item it = next_item_warp(counter, count, list, rv, &blk);
    if (it.tile < 0) break;
    if (PROD && it.c == it.nch - 1) continue;  // the last chunk's product is never needed
    const int tile = it.tile, tx = it.tx, ty = it.ty, W = it.W, H = it.H;
    const int lx = lane & 7, ly0 = 4 * blk + (lane >> 3);
    const int x = tx * B + lx;
    const int y = ty * B + ly0;
    const float pxc = (float)x + 0.5f, pyc = (float)y + 0.5f;
    const float bx0 = (float)(tx * B) + 0.5f, bx1 = bx0 + 7.f;
    const float by0 = (float)(ty * B + 4 * blk) + 0.5f, by1 = by0 + 3.f;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const bool split = it.slot0 >= 0;
    const int lo = split ? it.c * L : 0;
    const int hi = split ? (int)min((long long)n, (long long)lo + L) : n;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    int last = 0, stop = -1, nbl = 0;
    bool done = !(x < W && y < H);
    const int p = ly0 * B + lx;  // pixel within the tile
    if (!PROD && split && it.c > 0) {
        for (int c = 0; c < it.c; ++c) T *= sl.prod[(size_t)(it.slot0 + c) * NPIX + p];
        if (T < kTMin) done = true;
    }
    bool alldone = __all_sync(0xffffffffu, done);
    // the Gaussian indices of a batch are loaded one batch ahead, so a batch
    // waits only for its records
    uint32_t gn = lo + lane < hi ? gid[rg.x + lo + lane] : 0u;
    for (int base = lo; base < hi && !alldone; base += 32) {
        const int j = base + lane;
        const uint32_t g = gn;
        gn = j + 32 < hi ? gid[rg.x + j + 32] : 0u;
        bool keep = false;
        float4 ga, gb;
        float gc = 0.f;
        if (j < hi) {
            load_record<REC>(feat, g, ga, gb, gc);
            keep = !tile_skip(ga, gb, bx0, bx1, by0, by1);
        }
        const uint32_t km = __ballot_sync(0xffffffffu, keep);
        const int cnt = __popc(km);
        if (keep) {
            const int slot = __popc(km & lt);
            const int pm = slot >> 1, ph = slot & 1;
            float* fuv = (float*)&wuv[pm];
            float* fab = (float*)&wab[pm];
            float* fcl = (float*)&wcl[pm];
            fuv[ph] = ga.x; fuv[2 + ph] = ga.y;
            fab[ph] = -0.5f * kLog2e * ga.z; fab[2 + ph] = -kLog2e * ga.w;
            fcl[ph] = -0.5f * kLog2e * gb.x; fcl[2 + ph] = __log2f(gb.y);
            wc[slot] = make_float4(gb.z, gb.w, gc, __int_as_float(j));
        }
        __syncwarp();
        uint32_t mine = 0;  // staged entries this pixel blended
        auto blend = [&](int kk, float pw, float e) {
            if (done || !(pw <= 0.f && e >= kLog2AlphaMin)) return;
            const float alpha = fminf(kAlphaMax, ex2_approx(e));
            const float Tn = fmaf(-alpha, T, T);
            const float4 col = wc[kk];
            const int pos = __float_as_int(col.w);
            if (Tn < kTMin) {
                done = true;
                stop = pos;
                if (PROD) T = Tn;
            } else {
                if (!PROD) {
                    const float w = alpha * T;
                    c0 += w * col.x;
                    c1 += w * col.y;
                    c2 += w * col.z;
                    last = pos + 1;
                    ++nbl;
                    mine |= 1u << kk;
                }
                T = Tn;
            }
        };
        // two entries per iteration, their offsets, quadratic forms and log2
        // alphas as packed float32 pairs (the staging keeps an entry pair's
        // fields side by side): the same roundings as the scalar form, so the
        // backward's test agrees bit for bit (render_fwd 0.43 -> 0.38 ms at
        // 2M Gaussians); with an odd count the last pair's second half is
        // stale and not used
        const f32x2 npx = f2_pack(-pxc, -pxc), npy = f2_pack(-pyc, -pyc);
        for (int kk = 0; kk < cnt && !done; kk += 2) {
            const int pm = kk >> 1;
            const f32x2 dx = f2_add(f2_ld(wuv[pm].x), npx), dy = f2_add(f2_ld(wuv[pm].z), npy);
            const f32x2 pu = f2_fma(dx, f2_fma(f2_ld(wab[pm].z), dy, f2_mul(f2_ld(wab[pm].x), dx)),
                                    f2_mul(f2_mul(f2_ld(wcl[pm].x), dy), dy));
            const f32x2 eu = f2_add(pu, f2_ld(wcl[pm].z));
            float p0, p1, e0, e1;
            f2_unpack(pu, p0, p1);
            f2_unpack(eu, e0, e1);
            blend(kk, p0, e0);
            if (kk + 1 < cnt) blend(kk + 1, p1, e1);
        }
        if (!PROD && flags) {
            const uint32_t bm = __reduce_or_sync(0xffffffffu, mine);
            if (lane < cnt && ((bm >> lane) & 1u)) {
                const long long gj = (long long)rg.x + __float_as_int(wc[lane].w);
                if ((gj | 3) < flags_cap)
                    atomicOr((unsigned int*)(flags + (gj & ~3ll)),
                             (unsigned int)(kFlagWarpBits | (1u << blk)) << (8 * (int)(gj & 3)));
            }
        }
        alldone = __all_sync(0xffffffffu, done);
        __syncwarp();
    }
    if (split) {
        const size_t s0 = (size_t)(it.slot0 + it.c) * NPIX + (size_t)p;
        if (PROD) {
            sl.prod[s0] = T;
        } else {
            sl.tout[s0] = T;
            sl.c0[s0] = c0; sl.c1[s0] = c1; sl.c2[s0] = c2;
            sl.last[s0] = last | (stop >= 0 ? kStopFlag : 0);
            sl.nbl[s0] = nbl;
            sl.stop[s0] = stop;
        }
        continue;
    }
    if (x < W && y < H) {
        const size_t HW = (size_t)W * H;
        float* im = img + 3 * it.poff;
        const size_t pix = (size_t)y * W + x;
        im[pix] = c0 + T * rv.bg0;
        im[HW + pix] = c1 + T * rv.bg1;
        im[2 * HW + pix] = c2 + T * rv.bg2;
        Tout[it.poff + pix] = T;
        lastout[it.poff + pix] = last;
        if (exout) exout[it.poff + pix] = stop >= 0 ? stop + 1 : n;
        if (blout) blout[it.poff + pix] = nbl;
    }
    }  // work items
}

}  // namespace dg

static dg::RViews make_rviews(const dg_camera* cams, int n, int B, const dg_raster_opts* o)
{
    dg::RViews rv;
    rv.n = n;
    int tiles = 0;
    long long pix = 0;
    for (int v = 0; v < n; ++v) {
        rv.W[v] = cams[v].width;
        rv.H[v] = cams[v].height;
        rv.TX[v] = (cams[v].width + B - 1) / B;
        rv.toff[v] = tiles;
        rv.poff[v] = pix;
        tiles += rv.TX[v] * ((cams[v].height + B - 1) / B);
        pix += (long long)cams[v].width * cams[v].height;
    }
    rv.toff[n] = tiles;
    rv.total = tiles;
    rv.bg0 = o->bg[0]; rv.bg1 = o->bg[1]; rv.bg2 = o->bg[2];
    return rv;
}

// Resident CTAs of a kernel on this device.
template <typename Kern>
static int resident_ctas(Kern kern, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    const long long g = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    return (int)(g < (1 << 20) ? g : (1 << 20));
}

// Layout of the render workspace for n_tiles tiles of edge B.
struct RenderWs {
    dg::RHdr* hdr;
    uint8_t* flags;       // per pair: blended by some pixel of its tile (written by the forward)
    long long flags_cap;  // pairs the flag array holds
    int4* items;
    int4* sitems;
    uint64_t* toff;
    uint64_t* bsum;
    dg::Slots sl;
    int cap;
    size_t bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Chunk slots: 2^20 pixels' worth (32 MiB of per-pixel chunk state).
static int slot_cap(int B) { return (1 << 20) / (B * B); }

// Layout of the render workspace; the per-pair flag array takes whatever
// follows the fixed part (ws_bytes - fixed bytes).
static RenderWs render_ws_fixed(void* base, long long n_tiles, int B, bool split);
static RenderWs render_ws(void* base, long long n_tiles, int B, bool split, size_t ws_bytes = 0)
{
    RenderWs w = render_ws_fixed(base, n_tiles, B, split);
    w.flags = (uint8_t*)base + w.bytes;
    w.flags_cap = ws_bytes > w.bytes ? (long long)(ws_bytes - w.bytes) : 0;
    if (!base) w.flags = nullptr;
    return w;
}

static RenderWs render_ws_fixed(void* base, long long n_tiles, int B, bool split)
{
    RenderWs w{};
    char* p = (char*)base;
    size_t off = 256;
    w.hdr = (dg::RHdr*)p;
    if (!split) { w.bytes = off; return w; }
    const int cap = slot_cap(B);
    const long long nb = (n_tiles + dg::SCAN_TILE - 1) / dg::SCAN_TILE;
    const size_t npix = (size_t)cap * B * B;
    w.cap = cap;
    w.items = (int4*)(p + off);  off = align256(off + sizeof(int4) * (size_t)(n_tiles + cap));
    w.sitems = (int4*)(p + off); off = align256(off + sizeof(int4) * (size_t)cap);
    w.toff = (uint64_t*)(p + off); off = align256(off + sizeof(uint64_t) * (size_t)(n_tiles > 0 ? n_tiles : 1));
    w.bsum = (uint64_t*)(p + off); off = align256(off + sizeof(uint64_t) * (size_t)(nb > 0 ? nb : 1));
    float** fp[5] = {&w.sl.prod, &w.sl.tout, &w.sl.c0, &w.sl.c1, &w.sl.c2};
    for (int i = 0; i < 5; ++i) { *fp[i] = (float*)(p + off); off = align256(off + sizeof(float) * npix); }
    int** ip[3] = {&w.sl.last, &w.sl.nbl, &w.sl.stop};
    for (int i = 0; i < 3; ++i) { *ip[i] = (int*)(p + off); off = align256(off + sizeof(int) * npix); }
    w.bytes = off;
    return w;
}

// Tile 8, one pixel per thread: the warp-per-block forward (k_render_fwd_w).
template <int REC>
static dg_status launch_fwd_w(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg::RViews& rv,
                              const RenderWs& w, int split_req, float* img, float* T, int* last, int* ex, int* bl,
                              cudaStream_t s)
{
    const uint2* rg = (const uint2*)ranges;
    auto kern = dg::k_render_fwd_w<false, REC>;
    const int R = resident_ctas(kern, 64);
    cudaMemsetAsync(w.hdr, 0, 256, s);
    if (w.flags && w.flags_cap > 0) cudaMemsetAsync(w.flags, 0, (size_t)w.flags_cap, s);
    const bool split = rv.total > 0 && (split_req > 0 || (split_req == 0 && rv.total < 2LL * R));
    if (split) {
        const dg::SplitCfg cfg{split_req, R, w.cap};
        const long long n = rv.total;
        const int nb = (int)((n + dg::SCAN_TILE - 1) / dg::SCAN_TILE);
        dg::k_scan_reduce<<<nb, dg::SCAN_THREADS, 0, s>>>(dg::LoadLen{rg}, n, w.bsum);
        dg::k_scan_top<<<1, 1024, 0, s>>>(w.bsum, nb, &w.hdr->M);
        dg_note_launch(2);
        dg::exclusive_scan(dg::LoadChunks{rg, w.hdr, cfg}, n, w.toff, w.bsum, &w.hdr->totals, s);
        const int pg = (int)((n + 255) / 256);
        dg::k_plan_items<<<pg < 1024 ? pg : 1024, 256, 0, s>>>(rg, (int)n, w.hdr, cfg, w.toff, w.items, w.sitems);
        auto kprod = dg::k_render_fwd_w<true, REC>;
        kprod<<<resident_ctas(kprod, 64), 64, 0, s>>>((const void*)feat, gid, rg, rv, w.hdr, w.items, w.sitems, w.sl,
                                                      nullptr, 0, img, T, last, ex, bl);
        dg_note_launch(2);
    }
    const int grid = split ? R : (R < rv.total ? R : (rv.total > 0 ? rv.total : 1));
    kern<<<grid, 64, 0, s>>>((const void*)feat, gid, rg, rv, w.hdr, w.items, w.sitems, w.sl, w.flags, w.flags_cap,
                             img, T, last, ex, bl);
    dg_note_launch();
    if (split) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dg::k_render_combine<8><<<4 * (sms > 0 ? sms : 1), 64, 0, s>>>(rg, rv, w.hdr, w.sitems, w.sl, img, T, last,
                                                                      ex, bl);
        dg_note_launch();
    }
    return DG_OK;
}

template <int B, int PPT, int REC>
static dg_status launch_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg::RViews& rv,
                            const RenderWs& w, int split_req, float* img, float* T, int* last, int* ex, int* bl,
                            cudaStream_t s)
{
    const uint2* rg = (const uint2*)ranges;
    if (B == 8 && PPT == 1) return launch_fwd_w<REC>(feat, gid, ranges, rv, w, split_req, img, T, last, ex, bl, s);
    auto kern = dg::k_render_fwd<B, PPT, false, REC>;
    const int R = resident_ctas(kern, B * B / PPT);
    cudaMemsetAsync(w.hdr, 0, 256, s);
    // automatic: split only when the tiles alone leave resident CTAs idle
    // (with at least two tiles per CTA the persistent launch balances itself,
    // and splitting costs the product pass)
    const bool split = rv.total > 0 && (split_req > 0 || (split_req == 0 && rv.total < 2LL * R));
    if (split) {
        const dg::SplitCfg cfg{split_req, R, w.cap};
        const long long n = rv.total;
        const int nb = (int)((n + dg::SCAN_TILE - 1) / dg::SCAN_TILE);
        dg::k_scan_reduce<<<nb, dg::SCAN_THREADS, 0, s>>>(dg::LoadLen{rg}, n, w.bsum);
        dg::k_scan_top<<<1, 1024, 0, s>>>(w.bsum, nb, &w.hdr->M);
        dg_note_launch(2);
        dg::exclusive_scan(dg::LoadChunks{rg, w.hdr, cfg}, n, w.toff, w.bsum, &w.hdr->totals, s);
        const int pg = (int)((n + 255) / 256);
        dg::k_plan_items<<<pg < 1024 ? pg : 1024, 256, 0, s>>>(rg, (int)n, w.hdr, cfg, w.toff, w.items, w.sitems);
        auto kprod = dg::k_render_fwd<B, PPT, true, REC>;
        kprod<<<resident_ctas(kprod, B * B / PPT), B * B / PPT, 0, s>>>(
            (const void*)feat, gid, rg, rv, w.hdr, w.items, w.sitems, w.sl, nullptr, 0, img, T, last, ex, bl);
        dg_note_launch(2);
    }
    const int grid = split ? R : (R < rv.total ? R : (rv.total > 0 ? rv.total : 1));
    kern<<<grid, B * B / PPT, 0, s>>>((const void*)feat, gid, rg, rv, w.hdr, w.items, w.sitems, w.sl, w.flags,
                                      w.flags_cap, img, T, last, ex, bl);
    dg_note_launch();
    if (split) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dg::k_render_combine<B><<<4 * (sms > 0 ? sms : 1), B * B, 0, s>>>(rg, rv, w.hdr, w.sitems, w.sl, img, T,
                                                                         last, ex, bl);
        dg_note_launch();
    }
    return DG_OK;
}

// Backward of 8x8 tiles, one pixel per thread: entry-parallel gradient sums
// (k_render_bwd_ep) unless DG_BWD_EP is defined to 0.
#ifndef DG_BWD_EP
#define DG_BWD_EP 1
#endif

template <int B, int PPT, int REC>
static void launch_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges, const dg::RViews& rv,
                       const RenderWs& w, const float* T, const int* last, const float* dL, float* g2, cudaStream_t s)
{
    if (DG_BWD_EP && B == 8 && PPT == 1) {
        auto kew = dg::k_render_bwd_ep<REC>;
        const int grid = resident_ctas(kew, 64);
        cudaMemsetAsync(&w.hdr->cnt_bwd, 0, sizeof(int), s);
        kew<<<grid, 64, 0, s>>>((const void*)feat, gid, (const uint2*)ranges, rv, w.hdr, w.items, w.sl, w.flags,
                                w.flags_cap, T, last, dL, (float4*)g2);
        dg_note_launch();
        return;
    }
    auto kern = dg::k_render_bwd<B, PPT, REC>;
    const int grid = resident_ctas(kern, B * B / PPT);
    cudaMemsetAsync(&w.hdr->cnt_bwd, 0, sizeof(int), s);
    kern<<<grid, B * B / PPT, 0, s>>>((const void*)feat, gid, (const uint2*)ranges, rv, w.hdr, w.items, w.sl,
                                      w.flags, w.flags_cap, T, last, dL, (float4*)g2);
    dg_note_launch();
}

template <int REC>
static void fwd_dispatch(int B, int ppt, const float* feat, const uint32_t* gid, const uint32_t* ranges,
                         const dg::RViews& rv, const RenderWs& w, int sp, float* img, float* T, int* last, int* ex,
                         int* bl, cudaStream_t s)
{
    if (B == 8 && ppt == 2) launch_fwd<8, 2, REC>(feat, gid, ranges, rv, w, sp, img, T, last, ex, bl, s);
    else if (B == 8) launch_fwd<8, 1, REC>(feat, gid, ranges, rv, w, sp, img, T, last, ex, bl, s);
    else if (ppt == 1) launch_fwd<16, 1, REC>(feat, gid, ranges, rv, w, sp, img, T, last, ex, bl, s);
    else if (ppt == 2) launch_fwd<16, 2, REC>(feat, gid, ranges, rv, w, sp, img, T, last, ex, bl, s);
    else launch_fwd<16, 4, REC>(feat, gid, ranges, rv, w, sp, img, T, last, ex, bl, s);
}

template <int REC>
static void bwd_dispatch(int B, int ppt, const float* feat, const uint32_t* gid, const uint32_t* ranges,
                         const dg::RViews& rv, const RenderWs& w, const float* T, const int* last, const float* dL,
                         float* g2, cudaStream_t s)
{
    if (B == 8 && ppt == 2) launch_bwd<8, 2, REC>(feat, gid, ranges, rv, w, T, last, dL, g2, s);
    else if (B == 8) launch_bwd<8, 1, REC>(feat, gid, ranges, rv, w, T, last, dL, g2, s);
    else if (ppt == 1) launch_bwd<16, 1, REC>(feat, gid, ranges, rv, w, T, last, dL, g2, s);
    else if (ppt == 2) launch_bwd<16, 2, REC>(feat, gid, ranges, rv, w, T, last, dL, g2, s);
    else launch_bwd<16, 4, REC>(feat, gid, ranges, rv, w, T, last, dL, g2, s);
}

// Pixels per thread used for (tile, request): tile 16 -> 1, 2 or 4 (0 selects
// the default of each pass), tile 8 -> 1 or 2 (default 1).
static int resolve_ppt(const dg_raster_opts* o, bool backward)
{
    const int req = o->pixels_per_thread;
    if (o->tile == 8) return req == 2 ? 2 : 1;
    if (req == 1 || req == 2 || req == 4) return req;
    return backward ? 4 : 2;
}

bool dg_check_cameras(const dg_camera* cams, int n_views);

static long long total_tiles(const dg_camera* cams, int n_views, int B)
{
    long long t = 0;
    for (int v = 0; v < n_views; ++v)
        t += (long long)((cams[v].width + B - 1) / B) * ((cams[v].height + B - 1) / B);
    return t;
}

static bool render_args(const dg_camera* cams, int n_views, const dg_raster_opts* opts, void* ws, size_t ws_bytes)
{
    if (!dg_check_cameras(cams, n_views)) return false;
    if (!opts) { dg_set_error("opts null"); return false; }
    if (opts->tile != 8 && opts->tile != 16) { dg_set_error("render supports tile 8 or 16, got %d", opts->tile); return false; }
    const int p = opts->pixels_per_thread;
    if (p != 0 && p != 1 && p != 2 && p != 4) { dg_set_error("pixels_per_thread must be 0, 1, 2 or 4, got %d", p); return false; }
    if (total_tiles(cams, n_views, opts->tile) >= (1LL << 30)) { dg_set_error("too many tiles"); return false; }
    if (opts->record != 0 && opts->record != 1) { dg_set_error("record must be 0 (float32) or 1 (mixed), got %d", opts->record); return false; }
    const size_t need = dg_render_workspace_size(cams, n_views, opts, 0);  // the fixed part; flags use the rest
    if (!ws || ws_bytes < need) { dg_set_error("render workspace missing or too small (%zu < %zu bytes)", ws_bytes, need); return false; }
    if (((uintptr_t)ws) & 255u) { dg_set_error("render workspace must be 256-byte aligned"); return false; }
    return true;
}

extern "C" size_t dg_render_workspace_size(const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts,
                                           int64_t M_cap)
{
    if (!cams || !opts || n_views < 1 || n_views > DG_MAX_VIEWS || (opts->tile != 8 && opts->tile != 16)) return 0;
    if (M_cap < 0) return 0;
    for (int v = 0; v < n_views; ++v)
        if (cams[v].width <= 0 || cams[v].height <= 0) return 0;
    const size_t fixed = render_ws_fixed(nullptr, total_tiles(cams, n_views, opts->tile), opts->tile,
                                         opts->split_len >= 0).bytes;
    return fixed + (((size_t)M_cap + 255) & ~(size_t)255);
}

extern "C" dg_status dg_render_fwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts, float* img,
                                   float* T_final, int32_t* last, int32_t* examined, int32_t* blended, void* ws,
                                   size_t ws_bytes, dg_stream stream)
{
    if (!render_args(cams, n_views, opts, ws, ws_bytes)) return DG_ERR_ARG;
    if (!ranges || !img || !T_final || !last) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (feat && (((uintptr_t)feat) & 15u)) { dg_set_error("feat must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int B = opts->tile;
    const dg::RViews rv = make_rviews(cams, n_views, B, opts);
    const RenderWs w = render_ws(ws, rv.total, B, opts->split_len >= 0, ws_bytes);
    const int sp = opts->split_len;
    const int ppt = resolve_ppt(opts, false);
    if (opts->record == 1) fwd_dispatch<1>(B, ppt, feat, gid, ranges, rv, w, sp, img, T_final, last, examined, blended, s);
    else fwd_dispatch<0>(B, ppt, feat, gid, ranges, rv, w, sp, img, T_final, last, examined, blended, s);
    return dg_check_launch("render_fwd");
}

extern "C" dg_status dg_render_bwd(const float* feat, const uint32_t* gid, const uint32_t* ranges,
                                   const dg_camera* cams, int32_t n_views, const dg_raster_opts* opts,
                                   const float* T_final, const int32_t* last, const float* dL_dimg, int64_t n_records,
                                   float* grad2d, void* ws, size_t ws_bytes, dg_stream stream)
{
    if (!render_args(cams, n_views, opts, ws, ws_bytes)) return DG_ERR_ARG;
    if (n_records < 0) { dg_set_error("n_records < 0"); return DG_ERR_ARG; }
    if (!ranges || !T_final || !last || !dL_dimg || (n_records > 0 && !grad2d)) { dg_set_error("null buffer"); return DG_ERR_ARG; }
    if (grad2d && (((uintptr_t)grad2d) & 15u)) { dg_set_error("grad2d must be 16-byte aligned"); return DG_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_records > 0) cudaMemsetAsync(grad2d, 0, sizeof(float) * DG_FEAT_FLOATS * (size_t)n_records, s);
    const int B = opts->tile;
    const dg::RViews rv = make_rviews(cams, n_views, B, opts);
    const RenderWs w = render_ws(ws, rv.total, B, opts->split_len >= 0, ws_bytes);
    const int ppt = resolve_ppt(opts, true);
    if (opts->record == 1) bwd_dispatch<1>(B, ppt, feat, gid, ranges, rv, w, T_final, last, dL_dimg, grad2d, s);
    else bwd_dispatch<0>(B, ppt, feat, gid, ranges, rv, w, T_final, last, dL_dimg, grad2d, s);
    return dg_check_launch("render_bwd");
}
