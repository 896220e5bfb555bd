// blend.cu -- combined sort and accumulate stage and its adjoint (TRIPS Sec. 3.2, 3.6).
//
// One CTA owns one screen tile of one pyramid layer, one thread per pixel.
// It reads the tile's list of (point, tile) entries written by the splat
// pass in chunks.  For each chunk it
//   1. counts the chunk's fragments per pixel (the point's taps inside the
//      tile, Eq. 3-5),
//   2. turns the counts into offsets with a block scan,
//   3. scatters the chunk's fragment keys (z, i) into per-pixel runs in
//      shared memory,
//   4. lets each thread merge its own pixel's run into that pixel's sorted
//      list of the K smallest keys, held in the thread's registers (a
//      branch-free compare-exchange insertion, no atomics, no shared memory).
// After the last chunk every pixel holds exactly the K front-most fragments
// of its full list in (depth, index) order -- the list the paper sorts per
// pixel and clamps to 16 elements (Sec. 3.2) -- without ever storing the full
// list, and the cost of a tile is linear in its fragments whatever their
// arrival order.  The pixel then blends its list front to back (Eq. 6-7).
//
// With coarse-layer inclusion (Sec. 3.6, Implementation Details) the list of
// pixel (L, j, k) also holds the fragments of every coarser pixel that
// contains it.  That list is the pixel's own fragments plus the inclusive list
// of its parent (L+1, j/2, k/2), and the K front-most of a union are among
// the K front-most of each part, so the tiles run layer by layer, coarsest
// first: each coarse pixel stores its kept list (keys and opacities) in the
// workspace, and each child starts its own list from its parent's.
//
// The backward kernels run the adjoint of the blend per pixel back to front
// over the kept list (division-free recurrence) and scatter the point
// gradients with float atomics (one vector atomic per descriptor row).
#include "common.cuh"

namespace tpk {

struct TileGeom {
    int L, x0, y0;
};

__device__ __forceinline__ TileGeom tile_geom(const Frame &F, int tile)
{
    TileGeom g;
    g.L = tile_layer(F, tile);
    const int local = tile - F.tile_base[g.L];
    g.x0 = (local % F.tiles_x[g.L]) * F.tile_w;
    g.y0 = (local / F.tiles_x[g.L]) * F.tile_h;
    return g;
}

// Shared-memory layout of a tile CTA: the current chunk's fragment keys
// grouped by pixel and the per-pixel counters.  Every piece starts on a
// 16-byte boundary whatever the chunk size.
struct TileSmem {
    unsigned long long *ck;      // [4 chunk] chunk fragment keys, grouped by pixel
    unsigned *cnt, *off, *cur;   // [tile_threads]
    unsigned *wsum;              // [32]
    unsigned long long *thr;     // [blockDim] a pixel's current K-th key (forward only)
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Bytes of the blend's fragment region (one chunk: an 8-byte key for at most
// four fragments per entry).
__host__ __device__ inline size_t tile_region_bytes(const Frame &F) { return align16((size_t)32 * F.chunk); }

// The counters are sized by the launch's block (the largest tile CTA of the
// batch), which may exceed this view's own tile_threads.
__device__ __forceinline__ TileSmem carve(const Frame &F, unsigned char *base)
{
    TileSmem m;
    const size_t NT = blockDim.x;
    m.ck = reinterpret_cast<unsigned long long *>(base);
    m.cnt = reinterpret_cast<unsigned *>(base + tile_region_bytes(F));
    m.off = m.cnt + NT;
    m.cur = m.off + NT;
    m.wsum = m.cur + NT;
    m.thr = reinterpret_cast<unsigned long long *>(m.wsum + 32);
    return m;
}

// The backward keeps K slots per pixel (key, entry, T_m: 16 bytes a slot)
// in its region, then the same counters.
__host__ __device__ inline size_t backward_region_bytes(size_t NT, int K) { return align16((size_t)16 * K * NT); }

__device__ __forceinline__ TileSmem carve_backward(int K, unsigned char *base)
{
    TileSmem m;
    const size_t NT = blockDim.x;
    m.ck = reinterpret_cast<unsigned long long *>(base);
    m.cnt = reinterpret_cast<unsigned *>(base + backward_region_bytes(NT, K));
    m.off = m.cnt + NT;
    m.cur = m.off + NT;
    m.wsum = m.cur + NT;
    return m;
}

size_t tile_smem_bytes(const Frame &F, bool backward)
{
    const size_t region = backward ? backward_region_bytes((size_t)F.tile_threads, F.K) : tile_region_bytes(F);
    return region + (3 * (size_t)F.tile_threads + 32) * sizeof(unsigned) + (backward ? 0 : 8 * (size_t)F.tile_threads);
}

// Exclusive scan of v over the CTA (blockDim.x <= 1024, a multiple of 32).
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    return x - v + (warp > 0 ? wsum[warp - 1] : 0u);
}

// The taps of workspace entry e that fall inside the tile; calls fn(px) per tap.
template <class Fn>
__device__ __forceinline__ void entry_taps(const Frame &F, const TileGeom &g, const float4 &pay, Fn &&fn)
{
    const int L = g.L;
    float iota, diota;
    if (!layer_weight(pay.z, L, F.n_layers, F.eps, iota, diota)) return;
    const AxisTaps ax = axis_taps(pay.x, L, F.lw[L]);
    const AxisTaps ay = axis_taps(pay.y, L, F.lh[L]);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if (!(b ? ay.t1 : ay.t0)) continue;
        const int k = ay.j0 + b - g.y0;
        if (k < 0 || k >= F.tile_h) continue;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (!(a ? ax.t1 : ax.t0)) continue;
            const int j = ax.j0 + a - g.x0;
            if (j < 0 || j >= F.tile_w) continue;
            fn(k * F.tile_w + j);
        }
    }
}

// Like entry_taps, also passing each tap's fragment opacity
// gamma = beta * iota * alpha (Eq. 3), multiplied in the order of frag_weights.
template <class Fn>
__device__ __forceinline__ void entry_taps_w(const Frame &F, const TileGeom &g, const float4 &pay, Fn &&fn)
{
    const int L = g.L;
    float iota, diota;
    if (!layer_weight(pay.z, L, F.n_layers, F.eps, iota, diota)) return;
    const AxisTaps ax = axis_taps(pay.x, L, F.lw[L]);
    const AxisTaps ay = axis_taps(pay.y, L, F.lh[L]);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if (!(b ? ay.t1 : ay.t0)) continue;
        const int k = ay.j0 + b - g.y0;
        if (k < 0 || k >= F.tile_h) continue;
        const float wy = b ? ay.a : __fsub_rn(1.0f, ay.a);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (!(a ? ax.t1 : ax.t0)) continue;
            const int j = ax.j0 + a - g.x0;
            if (j < 0 || j >= F.tile_w) continue;
            const float wx = a ? ax.a : __fsub_rn(1.0f, ax.a);
            fn(k * F.tile_w + j, wx * wy * iota * pay.w);
        }
    }
}

// A pixel's kept list: the K smallest fragment keys seen so far, ascending;
// empty slots hold kEmptyKey.  Only the keys travel through the insertion
// chain (the fragment opacities are evaluated again for the kept ones), so a
// chain step is two compares and four selects on 32-bit halves.
template <int K>
struct TopK {
    static_assert(K % 4 == 0, "K must be a multiple of 4");
    unsigned long long key[K];
    int n;  // valid slots

    __device__ __forceinline__ void clear()
    {
        n = 0;
#pragma unroll
        for (int m = 0; m < K; ++m) key[m] = kEmptyKey;
    }

    // Compare-exchange chain over slots [0, L): after slot m, slots 0..m
    // hold the m+1 smallest of (old slots 0..m, new key) in order.  Exact
    // while n < L: slots from n on are empty and the chain only moves empty
    // keys past slot n.
    template <int L>
    __device__ __forceinline__ void insert_first(unsigned long long k)
    {
#pragma unroll
        for (int m = 0; m < L; ++m) {
            const unsigned long long tk = key[m];
            const bool lt = k < tk;
            key[m] = lt ? k : tk;
            k = lt ? tk : k;
        }
        n = n < K ? n + 1 : K;
    }

    // Insertion with a chain of lim slots rounded up to a multiple of K/4;
    // lim is the same for the whole warp (one uniform branch, no divergence)
    // and above every lane's n.  Most pixels hold far fewer than K
    // candidates, so their warps run short chains.
    __device__ __forceinline__ void insert_bounded(unsigned long long k, int lim)
    {
        if (k >= key[K - 1]) return;
        if (lim <= K / 4) insert_first<K / 4>(k);
        else if (lim <= K / 2) insert_first<K / 2>(k);
        else if (lim <= 3 * K / 4) insert_first<3 * K / 4>(k);
        else insert_first<K>(k);
    }
};

// Light tiles: up to kDirectEntries tile-list entries per thread go straight
// into per-pixel buckets of up to kDirectCap keys.
constexpr int kDirectEntries = 1;
constexpr int kDirectCap = 16;

// Builds the kept list of the thread's pixel (thread t owns pixel t of the
// tile, t < tile_px); returns the kept count.  With count_all, *nfrag gets
// the pixel's number of candidate fragments in the tile's own list.  A
// parent row prow >= 0 (coarse-layer inclusion) starts the list from the
// parent pixel's kept list, which is sorted already.
//
// A tile whose list spans several chunks keeps, per pixel, the current K-th
// key after each chunk: a later fragment at or behind it cannot enter the
// list, so the count and scatter passes of the next chunks drop it (fewer
// shared-memory atomics, writes and merge steps on dense tiles).  The kept
// list is the same either way.  Single-chunk tiles, and frames whose
// candidate counts are asked for, skip the thresholds.
template <int K>
__device__ int build_topk(const Frame &F, const Workspace &W, int tile, const TileGeom &g, const TileSmem &S,
                          TopK<K> &top, bool count_all, unsigned *nfrag, long long prow)
{
    const int TP = F.tile_px, tid = threadIdx.x, NT = blockDim.x;
    const bool owner = tid < TP;
    top.clear();
    if (prow >= 0 && TP_IN_RANGE(W.status, prow < W.crows)) {
#pragma unroll
        for (int m = 0; m < K; ++m) {
            top.key[m] = W.ckey[(long long)m * W.crows + prow];
            top.n += top.key[m] != kEmptyKey ? 1 : 0;
        }
    }
    S.cnt[tid] = 0u;
    S.cur[tid] = 0u;
    S.thr[tid] = top.key[K - 1];
    unsigned end = W.tile_off[tile + 1];
    if (end > W.capacity) end = W.capacity;
    unsigned beg = W.tile_off[tile];
    if (beg > end) beg = end;
    unsigned nfr = 0;
    const bool multi = !count_all && end - beg > (unsigned)F.chunk;
    __syncthreads();
    // A light tile (at most kDirectEntries entries per thread) skips the count and scan:
    // each pixel gets a fixed bucket of dcap slots and the entries append to
    // it directly; if any pixel overflows its bucket the tile takes the
    // general path below.
    const int dcap = min(kDirectCap, 4 * F.chunk / NT);
    if (end - beg <= (unsigned)(kDirectEntries * NT) && dcap > 0) {
        for (unsigned e = beg + tid; e < end; e += NT) {
            const unsigned long long key = W.bucket_key[e];
            entry_taps(F, g, W.bucket_pay[e], [&](int px) {
                if (!TP_IN_RANGE(W.status, px >= 0 && px < TP)) return;
                const unsigned q = atomicAdd(S.cnt + px, 1u);
                if (q < (unsigned)dcap) S.ck[px * dcap + q] = key;
            });
        }
        __syncthreads();
        const unsigned my = S.cnt[tid];
        if (!__syncthreads_or(my > (unsigned)dcap)) {
            const int lim = min(K, __reduce_max_sync(0xffffffffu, owner ? top.n : 0) +
                                       (int)__reduce_max_sync(0xffffffffu, owner ? my : 0u));
            if (owner)
                for (unsigned q = 0; q < my; ++q) top.insert_bounded(S.ck[tid * dcap + q], lim);
            *nfrag = my;
            __syncthreads();  // the caller's epilogue reuses the shared memory
            return top.n;
        }
        S.cnt[tid] = 0u;  // a bucket overflowed: the general path
        __syncthreads();
    }
    // A multi-chunk tile's chunks are made of 32-entry blocks of its list taken
    // round-robin (chunk k: blocks k, k + nch, ...), so that every chunk samples
    // the whole list: the fill writes the points of one warp as one run, and
    // contiguous chunks would give a pixel most of its fragments in one chunk,
    // before any threshold of it exists.  Each chunk holds at most
    // floor(chunk / 32) blocks, so at most F.chunk entries.
    const unsigned nb = (end - beg + 31u) / 32u;
    const unsigned bpc = (unsigned)F.chunk / 32u;
    const unsigned nch = multi ? (nb + bpc - 1u) / bpc : (end - beg + (unsigned)F.chunk - 1u) / (unsigned)F.chunk;
    for (unsigned ch = 0; ch < nch; ++ch) {
        const unsigned c0 = beg + ch * (unsigned)F.chunk, c1 = min(end, c0 + (unsigned)F.chunk);
        auto each_entry = [&](auto &&fn) {
            if (multi) {
                for (unsigned bb = ch + nch * (unsigned)(tid >> 5); bb < nb; bb += nch * (unsigned)(NT >> 5)) {
                    const unsigned e = beg + bb * 32u + (unsigned)(tid & 31);
                    if (e < end) fn(e);
                }
            } else {
                for (unsigned e = c0 + tid; e < c1; e += NT) fn(e);
            }
        };
        if (multi) {
            each_entry([&](unsigned e) {
                const unsigned long long key = W.bucket_key[e];
                entry_taps(F, g, W.bucket_pay[e], [&](int px) {
                    if (TP_IN_RANGE(W.status, px >= 0 && px < TP) && key < S.thr[px]) atomicAdd(S.cnt + px, 1u);
                });
            });
        } else {
            each_entry([&](unsigned e) {
                entry_taps(F, g, W.bucket_pay[e], [&](int px) {
                    if (TP_IN_RANGE(W.status, px >= 0 && px < TP)) atomicAdd(S.cnt + px, 1u);
                });
            });
        }
        __syncthreads();
        const unsigned my = S.cnt[tid];
        S.off[tid] = block_exclusive_scan(my, S.wsum);
        __syncthreads();
        each_entry([&](unsigned e) {
            const unsigned long long key = W.bucket_key[e];
            entry_taps(F, g, W.bucket_pay[e], [&](int px) {
                if (!TP_IN_RANGE(W.status, px >= 0 && px < TP)) return;
                if (!multi || key < S.thr[px]) {
                    const unsigned q = S.off[px] + atomicAdd(S.cur + px, 1u);
                    if (TP_IN_RANGE(W.status, q < 4u * (unsigned)F.chunk)) S.ck[q] = key;
                }
            });
        });
        __syncthreads();
        // every list of the warp stays below lim slots during this chunk's merge
        const int lim = min(K, __reduce_max_sync(0xffffffffu, owner ? top.n : 0) +
                                   (int)__reduce_max_sync(0xffffffffu, owner ? my : 0u));
        if (owner) {
            const unsigned a = S.off[tid];
            for (unsigned q = a; q < a + my; ++q) top.insert_bounded(S.ck[q], lim);
            if (multi) S.thr[tid] = top.key[K - 1];
            nfr += my;
        }
        S.cnt[tid] = 0u;
        S.cur[tid] = 0u;
        __syncthreads();
    }
    *nfrag = nfr;
    return top.n;
}

// beta * iota of a point with payload (x, y, s, alpha) at layer-L pixel (j, k),
// with the pieces the adjoint needs.
struct FragW {
    float wx, wy, dwx, dwy, iota, diota;
};

__device__ __forceinline__ FragW frag_weights(const Frame &F, float x, float y, float s, int L, int j, int k)
{
    FragW w;
    layer_weight(s, L, F.n_layers, F.eps, w.iota, w.diota);
    const AxisTaps ax = axis_taps(x, L, F.lw[L]);
    const AxisTaps ay = axis_taps(y, L, F.lh[L]);
    tap_weight(ax, j, L, w.wx, w.dwx);
    tap_weight(ay, k, L, w.wy, w.dwy);
    return w;
}

// A group of descriptor channels [d0, d0 + G) of point i, read with one
// 16-byte load when the rows allow it (G = 4 float32 or 8 bfloat16 channels);
// channels past D read as zero.
template <typename DescT>
struct DescGroup {
    static constexpr int G = sizeof(DescT) == 2 ? 8 : 4;
    float v[G];
};

template <typename DescT>
__device__ __forceinline__ DescGroup<DescT> load_group(const DescT *__restrict__ desc, unsigned i, int D, int d0,
                                                       int vec)
{
    DescGroup<DescT> r;
    const DescT *p = desc + (long long)i * D + d0;
    if (vec) {
        if constexpr (sizeof(DescT) == 4) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
            r.v[0] = a.x;
            r.v[1] = a.y;
            r.v[2] = a.z;
            r.v[3] = a.w;
        } else {
            const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(p));
            const unsigned w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[c]));
                r.v[2 * c] = f.x;
                r.v[2 * c + 1] = f.y;
            }
        }
        return r;
    }
#pragma unroll
    for (int c = 0; c < DescGroup<DescT>::G; ++c) r.v[c] = d0 + c < D ? load_desc(p + c) : 0.0f;
    return r;
}

// STATS: the frame's candidate counts are asked for (n_frag); a separate
// instantiation, so the plain blend carries none of that state.  Registers
// are capped at 80 for K <= 16 so that six 128-thread CTAs fit on an SM
// (the keys-only list and its bounded chains fit without spilling; uncapped
// builds of some instantiations take 104 and fit four, which made the 4K bf16
// blend 14% slower); K = 32 needs its registers for the list.
// layer < 0: every tile of the batch; else the tiles of that layer (the
// coarse-to-fine launches of coarse-layer inclusion).
template <int K, typename DescT, int MaxV, bool STATS>
__global__ void __maxnreg__(K <= 16 ? 80 : 168) k_tile_blend(const __grid_constant__ Batch<MaxV> B, Workspace W,
                                             const DescT *__restrict__ desc,
                             float *__restrict__ pyramid, unsigned *__restrict__ kept,
                             unsigned char *__restrict__ n_kept, float *__restrict__ t_final,
                             unsigned *__restrict__ n_frag, int layer)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    wait_previous_grid();
    allow_dependent_launch();
    if (*((volatile unsigned *)W.status) & TP_FLAG_CAPACITY) return;  // the lists were cut short: outputs invalid
    const int tile = block_tile(B, layer);  // global over the batch
    if (tile < 0) return;
    const int v = view_of_tile(B, tile);
    const Frame &F = B.view[v];
    const TileSmem S = carve(F, smem_raw);
    const TileGeom g = tile_geom(F, tile - B.tile_base[v]);
    const int TP = F.tile_px, tid = threadIdx.x, L = g.L;
    const int j = g.x0 + tid % F.tile_w, k = g.y0 + tid / F.tile_w;
    const bool active = tid < TP && j < F.lw[L] && k < F.lh[L];
    const bool parent = F.coarse && active && L + 1 < F.n_layers;
    TopK<K> top;
    unsigned nfr;
    int nk = build_topk<K>(F, W, tile, g, S, top, STATS, &nfr,
                           parent ? coarse_row(B, v, L + 1, j >> 1, k >> 1) : -1ll);
    if (!active) nk = 0;
    const int nk_warp = __reduce_max_sync(0xffffffffu, nk);
    const long long pix = B.pix_base[v] + F.pix_base[L] + (long long)k * F.lw[L] + j;
    const bool out_ok = active && TP_IN_RANGE(W.status, pix >= 0 && pix < B.n_pix);
    if (out_ok) {
        // the largest kept key: the backward's rebuild keeps exactly the keys <= it
        unsigned long long kmax = 0ull;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            if (m >= nk_warp) break;
            kmax = m < nk ? top.key[m] : kmax;
        }
        W.kmax[pix] = kmax;
        if (F.coarse && L > 0) {  // the children of the next launch start from this list
            const long long row = coarse_row(B, v, L, j, k);
            if (TP_IN_RANGE(W.status, row >= 0 && row < W.crows)) {
#pragma unroll
                for (int m = 0; m < K; ++m) W.ckey[(long long)m * W.crows + row] = top.key[m];
            }
        }
    }
    // The kept fragments' low key words (point index, layer); empty slots 0.
    unsigned lo[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        lo[m] = m < nk ? (unsigned)(top.key[m] & 0xFFFFFFFFull) : 0u;
        if (!TP_IN_RANGE(W.status, (lo[m] >> 4) < (unsigned long long)W.n_points)) lo[m] = 0u;
    }
    // Each kept fragment's opacity gamma = beta iota alpha (Eq. 3) from its
    // point's record, at its own layer and pixel, in the order of the list
    // build's float32 operations; the loads go out four slots at a time
    // (unused slots read point 0, a valid address whose value is ignored).
    constexpr int NB = 4;
    const float4 *__restrict__ rec = W.rec + (long long)v * W.n_points;
    float wgt[K];
#pragma unroll
    for (int m0 = 0; m0 < K; m0 += NB) {
#pragma unroll
        for (int u = 0; u < NB; ++u) wgt[m0 + u] = 0.0f;
        if (m0 >= nk_warp) continue;
        float4 r[NB];
        float al[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            r[u] = rec[lo[m0 + u] >> 4];
            al[u] = __ldg(W.opacity + (lo[m0 + u] >> 4));
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            if (m0 + u < nk) {
                const int Lf = (int)(lo[m0 + u] & 15u), d = Lf - L;
                const FragW w = frag_weights(F, r[u].x, r[u].y, r[u].w, Lf, j >> d, k >> d);
                wgt[m0 + u] = w.wx * w.wy * w.iota * al[u];
            }
        }
    }
    if (out_ok && F.coarse && L > 0) {  // the backward of coarse-layer inclusion reads the parents' opacities
        const long long row = coarse_row(B, v, L, j, k);
        if (TP_IN_RANGE(W.status, row >= 0 && row < W.crows)) {
#pragma unroll
            for (int m = 0; m < K; ++m) W.cgam[(long long)m * W.crows + row] = __float_as_uint(wgt[m]);
        }
    }
    // front to back: weights T_m gamma_m (Eq. 6-7), in place of the opacities
    float T = 1.0f;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        if (m >= nk_warp) break;
        if (m < nk) {
            const float gam = wgt[m];
            wgt[m] = T * gam;
            T = T * (1.0f - gam);
        }
    }
    // descriptor rows of the kept points (empty slots: row 0)
    unsigned row[K];
#pragma unroll
    for (int m = 0; m < K; ++m) row[m] = lo[m] >> 4;
    const int D = F.D;
    constexpr int G = DescGroup<DescT>::G;
    for (int d0 = 0; d0 < D; d0 += G) {
        float c[G];
#pragma unroll
        for (int q = 0; q < G; ++q) c[q] = 0.0f;
#pragma unroll
        for (int m0 = 0; m0 < K; m0 += NB) {
            if (m0 >= nk_warp) break;
            DescGroup<DescT> t[NB];
#pragma unroll
            for (int u = 0; u < NB; ++u)
                t[u] = load_group(desc, row[m0 + u], D, d0, F.desc_vec);
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                if (m0 + u < nk) {
#pragma unroll
                    for (int q = 0; q < G; ++q) c[q] += wgt[m0 + u] * t[u].v[q];
                }
            }
        }
        if (out_ok) {
            float *out = pyramid + pix * D + d0;
            if (F.desc_vec) {
#pragma unroll
                for (int q = 0; q < G; q += 4)
                    *reinterpret_cast<float4 *>(out + q) = make_float4(c[q], c[q + 1], c[q + 2], c[q + 3]);
            } else {
                for (int q = 0; q < G && d0 + q < D; ++q) out[q] = c[q];
            }
        }
    }
    if (!out_ok) return;
    if (kept) {
#pragma unroll
        for (int m = 0; m < K; ++m)
            kept[pix * K + m] = m < nk ? row[m] : kNoPoint;
    }
    if (n_kept) n_kept[pix] = (unsigned char)nk;
    if (t_final) t_final[pix] = T;
    if (STATS) {
        // the parent's count, from the previous launch, covers every coarser layer
        const long long ppix = B.pix_base[v] + F.pix_base[L + 1] + (long long)(k >> 1) * F.lw[L + 1] + (j >> 1);
        if (parent && TP_IN_RANGE(W.status, ppix < B.n_pix)) nfr += n_frag[ppix];
        n_frag[pix] = nfr;
    }
}

constexpr int kMaxGradD = 64;

// Adds v to four consecutive floats (16-byte aligned) with one vector atomic.
__device__ __forceinline__ void atomic_add4(float *p, float4 v)
{
    atomicAdd(reinterpret_cast<float4 *>(p), v);
}

// Adjoint of one kept fragment, given its forward quantities; scatters the
// point gradients.  G is the pixel's dL/dC; R the running back-to-front term.
// t0 holds the first channel group of the point's descriptor, loaded by the caller.
// DC > 0: the descriptor width known at compile time (G stays in registers).
// Camera adjoint of a fragment (Sec. 3.5), accumulated per thread in a
// shared-memory column cam[q * stride]: dL/d(fx, fy, cx, cy, R[9], t[3]) from
// the fragment's screen-space gradient (gx, gy, gs), its camera-space one dXc
// and the point's world position.
struct CamCol {
    float *p;        // null: no camera gradient
    int stride;
    const float *pos;
};

template <typename DescT, int DC, bool CAM = false>
__device__ __forceinline__ void adjoint_fragment(const Frame &F, int L, int j, int k, unsigned i, float x, float y,
                                                 float z, float s, float al, float Tm, const float *G, float &R,
                                                 const DescGroup<DescT> &t0, const DescT *__restrict__ desc,
                                                 float *__restrict__ gpos, float *__restrict__ gsw,
                                                 float *__restrict__ gop, float *__restrict__ gdesc,
                                                 const CamCol &cam = CamCol{nullptr, 0, nullptr})
{
    const int D = DC > 0 ? DC : F.D;
    constexpr int NG = DescGroup<DescT>::G;
    const FragW w = frag_weights(F, x, y, s, L, j, k);
    const float beta = w.wx * w.wy;
    const float gam = beta * w.iota * al;
    float gdot = 0.0f;
#pragma unroll
    for (int d0 = 0; d0 < D; d0 += NG) {
        const DescGroup<DescT> t = d0 == 0 ? t0 : load_group(desc, i, D, d0, F.desc_vec);
#pragma unroll
        for (int q = 0; q < NG; ++q)
            if (d0 + q < D) gdot += G[d0 + q] * t.v[q];
    }
    const float dg = Tm * (gdot - R);
    R = gam * gdot + (1.0f - gam) * R;
    const float tg = Tm * gam;
    float *gd = gdesc + (long long)i * D;
    if (F.grad_vec) {
#pragma unroll
        for (int d0 = 0; d0 < D; d0 += 4)
            atomic_add4(gd + d0, make_float4(tg * G[d0], tg * G[d0 + 1], tg * G[d0 + 2], tg * G[d0 + 3]));
    } else {
        for (int d = 0; d < D; ++d) atomicAdd(gd + d, tg * G[d]);
    }
    atomicAdd(gop + i, dg * beta * w.iota);
    const float dw = dg * al;
    const float gx = dw * w.wy * w.iota * w.dwx;
    const float gy = dw * w.wx * w.iota * w.dwy;
    const float gs = dw * beta * w.diota;
    const float iz = 1.0f / z;
    const float dXc = gx * F.fx * iz;
    const float dYc = gy * F.fy * iz;
    const float dZc = -(gx * (x - F.cx) + gy * (y - F.cy) + gs * s) * iz;
    const float gX = F.R[0] * dXc + F.R[3] * dYc + F.R[6] * dZc;
    const float gY = F.R[1] * dXc + F.R[4] * dYc + F.R[7] * dZc;
    const float gZ = F.R[2] * dXc + F.R[5] * dYc + F.R[8] * dZc;
    if (F.pos4) {  // packed rows (X, Y, Z, s_w): one vector atomic instead of four scalar ones
        atomic_add4(gpos + 4 * (long long)i, make_float4(gX, gY, gZ, gs * F.fx * iz));
    } else {
        atomicAdd(gsw + i, gs * F.fx * iz);
        atomicAdd(gpos + 3 * (long long)i + 0, gX);
        atomicAdd(gpos + 3 * (long long)i + 1, gY);
        atomicAdd(gpos + 3 * (long long)i + 2, gZ);
    }
    if constexpr (CAM) {
        // x = fx Xc/Zc + cx, y = fy Yc/Zc + cy, s = fx sw/Zc: dx/dfx = (x - cx)/fx, ds/dfx = s/fx
        float *c = cam.p;
        const int st = cam.stride;
        const float ifx = 1.0f / F.fx, ify = 1.0f / F.fy;
        c[0] += (gx * (x - F.cx) + gs * s) * ifx;
        c[st] += gy * (y - F.cy) * ify;
        c[2 * st] += gx;
        c[3 * st] += gy;
        const float d[3] = {dXc, dYc, dZc};
        const float Xw[3] = {__ldg(cam.pos + 3 * (long long)i), __ldg(cam.pos + 3 * (long long)i + 1),
                             __ldg(cam.pos + 3 * (long long)i + 2)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) c[(4 + 3 * a + b) * st] += d[a] * Xw[b];  // dL/dR_ab = dL/dXc_a Xw_b
            c[(13 + a) * st] += d[a];                                             // dL/dt = dL/dXc
        }
    }
}

// Backward with the lists rebuilt from the workspace's tile lists.  The blend
// left each pixel's largest kept key; a fragment is kept exactly when its key
// is not larger, so one pass over the tile's entries drops every kept
// fragment into one of its pixel's K slots (no selection work), each pixel's
// thread sorts its at most K slots, and runs the adjoint of its blend back to
// front in a rolled loop.  With coarse-layer inclusion the pixel's other kept
// fragments are the entries of its parent's stored list up to the same key;
// their payload comes from the point records, and their gradients from their
// own layer's pixel (each key carries its layer).
// Registers are capped at 80 for K <= 16 (six 128-thread CTAs per SM, with
// the 34 KB slot region); the kept slots are sorted in shared memory, so no
// register list is live (measured against 96 registers: 1080p backward -2%,
// 4K bf16 -3.4%).
// CAM: also the camera gradient of every view, [n_views][16] doubles in gcam
// (summed over the views' tiles: per-thread shared-memory columns, one
// reduction and 16 double atomics per CTA).
template <int K, typename DescT, int MaxV, int DC, bool CAM>
__global__ void __maxnreg__(K <= 16 ? 80 : 168) k_tile_backward(const __grid_constant__ Batch<MaxV> B, Workspace W,
                                                          const DescT *__restrict__ desc,
                                const float *__restrict__ grad_pyr, float *__restrict__ gpos, float *__restrict__ gsw,
                                float *__restrict__ gop, float *__restrict__ gdesc, long long n,
                                const float4 *__restrict__ rec_all, const float *__restrict__ opacity,
                                const float *__restrict__ pos, double *__restrict__ gcam)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    wait_previous_grid();
    allow_dependent_launch();
    if (*((volatile unsigned *)W.status) & TP_FLAG_CAPACITY) return;  // the lists were cut short: outputs invalid
    const int tile = blockIdx.x;  // global over the batch
    const int v = view_of_tile(B, tile);
    const Frame &F = B.view[v];
    const TileSmem S = carve_backward(K, smem_raw);
    const TileGeom g = tile_geom(F, tile - B.tile_base[v]);
    const int TP = F.tile_px, tid = threadIdx.x, NT = blockDim.x, L = g.L, D = DC > 0 ? DC : F.D;
    const int j = g.x0 + tid % F.tile_w, k = g.y0 + tid / F.tile_w;
    const long long pix = B.pix_base[v] + F.pix_base[L] + (long long)k * F.lw[L] + j;
    const bool active =
        tid < TP && j < F.lw[L] && k < F.lh[L] && TP_IN_RANGE(W.status, pix >= 0 && pix < B.n_pix);
    // slot-major private slots in the backward's region: key [K][TP], entry [K][TP], T_m [K][TP]
    unsigned long long *kk = S.ck;
    unsigned *ke = reinterpret_cast<unsigned *>(S.ck + (size_t)K * TP);
    float *kt = reinterpret_cast<float *>(ke + (size_t)K * TP);
    unsigned long long *thr = reinterpret_cast<unsigned long long *>(S.off);  // [TP] (off, cur are 8-aligned pairs)
    S.cnt[tid] = 0u;
    if (tid < TP) thr[tid] = active ? W.kmax[pix] : 0ull;
    __syncthreads();
    unsigned end = W.tile_off[tile + 1];
    if (end > W.capacity) end = W.capacity;
    unsigned beg = W.tile_off[tile];
    if (beg > end) beg = end;
    for (unsigned e = beg + tid; e < end; e += NT) {
        const unsigned long long key = W.bucket_key[e];
        entry_taps_w(F, g, W.bucket_pay[e], [&](int px, float gam) {
            if (!TP_IN_RANGE(W.status, px >= 0 && px < TP)) return;
            if (key <= thr[px]) {
                const unsigned q = atomicAdd(S.cnt + px, 1u);
                if (q < (unsigned)K) {
                    kk[q * TP + px] = key;
                    ke[q * TP + px] = e;
                    kt[q * TP + px] = gam;
                }
            }
        });
    }
    __syncthreads();
    float *camc = reinterpret_cast<float *>(S.wsum + 32);  // [16][NT] camera-gradient columns (CAM only)
    if constexpr (CAM) {
#pragma unroll
        for (int q = 0; q < 16; ++q) camc[q * NT + tid] = 0.0f;
    }
    auto per_pixel = [&]() {
    if (!active) return;
    int nk = (int)S.cnt[tid];
    const long long prow = F.coarse && L + 1 < F.n_layers ? coarse_row(B, v, L + 1, j >> 1, k >> 1) : -1ll;
    if (prow >= 0 && TP_IN_RANGE(W.status, prow < W.crows)) {
        const unsigned long long km = thr[tid];
        // the stored list is sorted and empty slots hold the largest key: read it four
        // slots at a time (the loads of a group in flight together) until a key passes km
        bool more = true;
        for (int m0 = 0; m0 < K && more; m0 += 4) {
            unsigned long long key[4];
            unsigned gam[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                key[u] = W.ckey[(long long)(m0 + u) * W.crows + prow];
                gam[u] = W.cgam[(long long)(m0 + u) * W.crows + prow];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!more || key[u] > km) {
                    more = false;
                    continue;
                }
                if (nk < K) {
                    kk[nk * TP + tid] = key[u];
                    ke[nk * TP + tid] = kNoPoint;
                    kt[nk * TP + tid] = __uint_as_float(gam[u]);
                }
                ++nk;
            }
        }
    }
    if (nk > K) nk = K;
    if (nk == 0) return;
    const float4 *__restrict__ rec = rec_all + (long long)v * n;
    // insertion sort of the pixel's slots (at most K) by key, in its own
    // shared-memory column (no registers held for the list)
    for (int a = 1; a < nk; ++a) {
        const unsigned long long key = kk[a * TP + tid];
        const unsigned ent = ke[a * TP + tid];
        const float gam = kt[a * TP + tid];
        int b = a - 1;
        while (b >= 0 && kk[b * TP + tid] > key) {
            kk[(b + 1) * TP + tid] = kk[b * TP + tid];
            ke[(b + 1) * TP + tid] = ke[b * TP + tid];
            kt[(b + 1) * TP + tid] = kt[b * TP + tid];
            --b;
        }
        kk[(b + 1) * TP + tid] = key;
        ke[(b + 1) * TP + tid] = ent;
        kt[(b + 1) * TP + tid] = gam;
    }
    // front to back: T_m in place of each kept fragment's opacity, which the
    // rebuild left in its slot (no global loads)
    {
        float T = 1.0f;
        for (int m = 0; m < nk; ++m) {
            const float gam = kt[m * TP + tid];
            kt[m * TP + tid] = T;
            T = T * (1.0f - gam);
        }
    }
    float G[DC > 0 ? DC : kMaxGradD];
#pragma unroll
    for (int d = 0; d < (DC > 0 ? DC : D); ++d) G[d] = __ldg(grad_pyr + pix * D + d);
    // back to front, four slots at a time: the loads of a batch go out first
    float R = 0.0f;
    constexpr int NB = sizeof(DescT) == 2 ? 2 : 4;  // bf16 groups hold 8 channels: fewer in flight
    for (int m1 = nk - 1; m1 >= 0; m1 -= NB) {
        unsigned long long key[NB];
        float4 pay[NB];
        DescGroup<DescT> t0[NB];
        unsigned pi[NB];
        bool ok[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int m = m1 - u >= 0 ? m1 - u : 0;
            key[u] = kk[m * TP + tid];
            pi[u] = key_point(key[u]);
            const unsigned ent = ke[m * TP + tid];
            ok[u] = TP_IN_RANGE(W.status, pi[u] < (unsigned long long)W.n_points &&
                                              (ent == kNoPoint || ent < W.capacity));
            if (!ok[u]) pi[u] = 0u;
            if (ent != kNoPoint) {
                pay[u] = W.bucket_pay[ok[u] ? ent : 0u];
            } else {  // a coarser layer's fragment
                const float4 r = rec[pi[u]];
                pay[u] = make_float4(r.x, r.y, r.w, __ldg(opacity + pi[u]));
            }
            t0[u] = load_group(desc, pi[u], D, 0, F.desc_vec);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int m = m1 - u;
            if (m < 0) break;
            if (!ok[u]) continue;
            const int Lf = key_layer(key[u]), d = Lf - L;  // the fragment's own layer and pixel
            adjoint_fragment<DescT, DC, CAM>(F, Lf, j >> d, k >> d, pi[u], pay[u].x, pay[u].y,
                                    __uint_as_float((unsigned)(key[u] >> 32)), pay[u].z, pay[u].w, kt[m * TP + tid],
                                    G, R, t0[u], desc, gpos, gsw, gop, gdesc, CamCol{camc + tid, NT, pos});
        }
    }
    };
    per_pixel();
    if constexpr (CAM) {
        __syncthreads();
        if (tid < 16) {
            float acc = 0.0f;
            for (int t = 0; t < NT; ++t) acc += camc[tid * NT + t];
            if (acc != 0.0f) atomicAdd(gcam + 16 * v + tid, (double)acc);
        }
    }
}

// Backward with the lists stored by the blend kernel.
template <int K, typename DescT, int MaxV>
__global__ void __launch_bounds__(kBlock) k_stored_backward(const __grid_constant__ Batch<MaxV> B, long long n,
                                                            const float4 *__restrict__ rec_all,
                                                            const float *__restrict__ opacity,
                                                            const DescT *__restrict__ desc,
                                                            const unsigned *__restrict__ kept,
                                                            const unsigned char *__restrict__ n_kept,
                                                            const float *__restrict__ grad_pyr,
                                                            float *__restrict__ gpos, float *__restrict__ gsw,
                                                            float *__restrict__ gop, float *__restrict__ gdesc,
                                                            unsigned *status)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < B.n_pix; pix += stride) {
        int nk = n_kept[pix];
        if (nk == 0) continue;
        if (nk > K) nk = K;
        const int v = view_of_pixel(B, pix);
        const Frame &F = B.view[v];
        const float4 *__restrict__ rec = rec_all + (long long)v * n;
        const long long vpix = pix - B.pix_base[v];
        int L = 0;
        while (L + 1 < F.n_layers && vpix >= F.pix_base[L + 1]) ++L;
        const long long local = vpix - F.pix_base[L];
        const int j = (int)(local % F.lw[L]), k = (int)(local / F.lw[L]);
        float Tm[K];
        float T = 1.0f;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            Tm[m] = 0.0f;
            if (m < nk) {
                const unsigned i = kept[pix * K + m];
                if (!TP_IN_RANGE(status, (long long)i < n)) continue;
                const float4 r = rec[i];
                const FragW w = frag_weights(F, r.x, r.y, r.w, L, j, k);
                Tm[m] = T;
                T = T * (1.0f - w.wx * w.wy * w.iota * __ldg(opacity + i));
            }
        }
        float G[kMaxGradD];
        const int D = F.D;
        for (int d = 0; d < D; ++d) G[d] = __ldg(grad_pyr + pix * D + d);
        float R = 0.0f;
#pragma unroll
        for (int m = K - 1; m >= 0; --m) {
            if (m >= nk) continue;
            const unsigned i = kept[pix * K + m];
            if (!TP_IN_RANGE(status, (long long)i < n)) continue;
            const float4 r = rec[i];
            adjoint_fragment<DescT, 0>(F, L, j, k, i, r.x, r.y, r.z, r.w, __ldg(opacity + i), Tm[m], G, R,
                                    load_group(desc, i, F.D, 0, F.desc_vec), desc, gpos, gsw, gop, gdesc);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

// Raises the kernel's dynamic shared memory limit when needed and checks that
// a CTA of `threads` threads fits the kernel's register use.
template <class KernelT>
static cudaError_t prepare_tile_kernel(KernelT kernel, size_t smem_bytes, int threads)
{
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kernel);
    if (e != cudaSuccess) return e;
    if (threads > attr.maxThreadsPerBlock) return cudaErrorInvalidConfiguration;
    if (smem_bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

// Shared memory of a tile launch: the largest fragment region over the views
// plus counters for the launch's block.
template <int MaxV>
static size_t batch_smem(const Batch<MaxV> &B)
{
    size_t region = 0;
    for (int v = 0; v < B.n_views; ++v) region = region > tile_region_bytes(B.view[v]) ? region : tile_region_bytes(B.view[v]);
    return region + (3 * (size_t)B.max_threads + 32) * sizeof(unsigned) + 8 * (size_t)B.max_threads;
}

// One launch over every tile, or with coarse-layer inclusion one launch per
// layer, coarsest first (each layer reads the lists its parent layer stored).
template <int K, typename DescT, int MaxV, bool STATS>
static cudaError_t blend_launches(const Batch<MaxV> &B, const Workspace &W, const DescT *desc, float *pyramid,
                                  unsigned *kept, unsigned char *n_kept, float *t_final, unsigned *n_frag,
                                  cudaStream_t stream)
{
    const size_t smem = batch_smem(B);
    cudaError_t e = prepare_tile_kernel(k_tile_blend<K, DescT, MaxV, STATS>, smem, B.max_threads);
    if (e != cudaSuccess) return e;
    if (!B.view[0].coarse) {
        return launch_dependent(k_tile_blend<K, DescT, MaxV, STATS>, dim3(B.n_tiles), dim3(B.max_threads), smem,
                                stream, B, W, desc, pyramid, kept, n_kept, t_final, n_frag, -1);
    }
    for (int L = B.view[0].n_layers - 1; L >= 0; --L) {
        int tiles = 0;
        for (int v = 0; v < B.n_views; ++v) tiles += B.view[v].tile_base[L + 1] - B.view[v].tile_base[L];
        if (tiles == 0) continue;
        e = launch_dependent(k_tile_blend<K, DescT, MaxV, STATS>, dim3(tiles), dim3(B.max_threads), smem, stream, B,
                             W, desc, pyramid, kept, n_kept, t_final, n_frag, L);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int K, typename DescT, int MaxV>
static cudaError_t blend_impl(const Batch<MaxV> &B, const Workspace &W, const void *desc, float *pyramid,
                              unsigned *kept, unsigned char *n_kept, float *t_final, unsigned *n_frag,
                              cudaStream_t stream)
{
    const DescT *d = static_cast<const DescT *>(desc);
    if (n_frag) return blend_launches<K, DescT, MaxV, true>(B, W, d, pyramid, kept, n_kept, t_final, n_frag, stream);
    return blend_launches<K, DescT, MaxV, false>(B, W, d, pyramid, kept, n_kept, t_final, n_frag, stream);
}

// Point and camera gradients of the recompute backward (BwdArgs bundles the launch's pointers).
struct BwdArgs {
    const float *grad_pyr;
    float *gpos, *gsw, *gop, *gdesc;
    long long n;
    const float4 *rec;
    const float *opacity;
    const float *pos;  // camera gradients only
    double *gcam;      // [n_views][16] or null
};

template <int K, typename DescT, int MaxV, int DC, bool CAM>
static cudaError_t backward_launch(const Batch<MaxV> &B, const Workspace &W, const DescT *d, const BwdArgs &a,
                                   size_t smem, cudaStream_t stream)
{
    if (CAM) smem += 16 * sizeof(float) * (size_t)B.max_threads;
    cudaError_t e = prepare_tile_kernel(k_tile_backward<K, DescT, MaxV, DC, CAM>, smem, B.max_threads);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_tile_backward<K, DescT, MaxV, DC, CAM>, dim3(B.n_tiles), dim3(B.max_threads), smem,
                            stream, B, W, d, a.grad_pyr, a.gpos, a.gsw, a.gop, a.gdesc, a.n, a.rec, a.opacity, a.pos,
                            a.gcam);
}

template <int K, typename DescT, int MaxV>
static cudaError_t backward_impl(const Batch<MaxV> &B, const Workspace &W, const void *desc, const unsigned *kept,
                                 const unsigned char *n_kept, const BwdArgs &a, cudaStream_t stream)
{
    const DescT *d = static_cast<const DescT *>(desc);
    if (kept) {
        if (a.gcam) return cudaErrorInvalidValue;  // camera gradients come with the recompute backward only
        long long blocks = (B.n_pix + kBlock - 1) / kBlock;
        if (blocks > 152 * 32) blocks = 152 * 32;
        if (blocks < 1) blocks = 1;
        k_stored_backward<K, DescT, MaxV><<<(int)blocks, kBlock, 0, stream>>>(
            B, a.n, a.rec, a.opacity, d, kept, n_kept, a.grad_pyr, a.gpos, a.gsw, a.gop, a.gdesc, W.status);
        return cudaGetLastError();
    }
    const size_t smem = backward_region_bytes((size_t)B.max_threads, K) + (3 * (size_t)B.max_threads + 32) * 4;
    if (a.gcam) {  // batches only: one generic instantiation per K and descriptor type
        if constexpr (MaxV > 1) return backward_launch<K, DescT, MaxV, 0, true>(B, W, d, a, smem, stream);
        return cudaErrorInvalidValue;
    }
    // the common descriptor widths get compile-time instantiations (K = 16)
    if constexpr (K == 16) {
        const int D = B.view[0].D;
        if (D == 4) return backward_launch<K, DescT, MaxV, 4, false>(B, W, d, a, smem, stream);
        if (D == 16) return backward_launch<K, DescT, MaxV, 16, false>(B, W, d, a, smem, stream);
    }
    return backward_launch<K, DescT, MaxV, 0, false>(B, W, d, a, smem, stream);
}

#define TPK_DISPATCH_K(KVAL, ...)                                   \
    switch (KVAL) {                                                 \
    case 4: { constexpr int KC = 4; __VA_ARGS__; } break;           \
    case 8: { constexpr int KC = 8; __VA_ARGS__; } break;           \
    case 16: { constexpr int KC = 16; __VA_ARGS__; } break;         \
    case 32: { constexpr int KC = 32; __VA_ARGS__; } break;         \
    default: return cudaErrorInvalidValue;                          \
    }

template <int MaxV>
cudaError_t launch_blend(const Batch<MaxV> &B, const Workspace &W, const void *desc, int desc_dtype,
                         float *pyramid, unsigned *kept, unsigned char *n_kept, float *t_final, unsigned *n_frag,
                         cudaStream_t stream)
{
    const int K = B.view[0].K;
    if (desc_dtype == TP_BF16) {
        TPK_DISPATCH_K(K, return (blend_impl<KC, __nv_bfloat16, MaxV>(B, W, desc, pyramid, kept, n_kept, t_final,
                                                                     n_frag, stream)));
    } else {
        TPK_DISPATCH_K(K, return (blend_impl<KC, float, MaxV>(B, W, desc, pyramid, kept, n_kept, t_final, n_frag,
                                                             stream)));
    }
    return cudaErrorInvalidValue;
}

template <int MaxV>
cudaError_t launch_backward(const Batch<MaxV> &B, const Workspace &W, long long n, const float4 *rec,
                            const float *opacity, const void *desc, int desc_dtype, const unsigned *kept,
                            const unsigned char *n_kept, const float *grad_pyramid, float *grad_pos,
                            float *grad_sw, float *grad_opacity, float *grad_desc, const float *pos,
                            double *grad_cameras, cudaStream_t stream)
{
    cudaError_t e;
    if (grad_cameras &&
        (e = cudaMemsetAsync(grad_cameras, 0, sizeof(double) * 16 * (size_t)B.n_views, stream)) != cudaSuccess)
        return e;
    if (n == 0) return cudaSuccess;
    const int K = B.view[0].K, D = B.view[0].D;
    const bool pos4 = B.view[0].pos4 != 0;
    if (!B.view[0].grads_zeroed) {
        if ((e = cudaMemsetAsync(grad_pos, 0, sizeof(float) * (pos4 ? 4 : 3) * (size_t)n, stream)) != cudaSuccess)
            return e;
        if (!pos4 && (e = cudaMemsetAsync(grad_sw, 0, sizeof(float) * (size_t)n, stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(grad_opacity, 0, sizeof(float) * (size_t)n, stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(grad_desc, 0, sizeof(float) * (size_t)D * (size_t)n, stream)) != cudaSuccess)
            return e;
    }
    const BwdArgs a{grad_pyramid, grad_pos, grad_sw, grad_opacity, grad_desc, n, rec, opacity, pos, grad_cameras};
    if (desc_dtype == TP_BF16) {
        TPK_DISPATCH_K(K, return (backward_impl<KC, __nv_bfloat16, MaxV>(B, W, desc, kept, n_kept, a, stream)));
    } else {
        TPK_DISPATCH_K(K, return (backward_impl<KC, float, MaxV>(B, W, desc, kept, n_kept, a, stream)));
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_blend<1>(const Batch<1> &, const Workspace &, const void *, int, float *, unsigned *,
                                     unsigned char *, float *, unsigned *, cudaStream_t);
template cudaError_t launch_blend<kMaxViews>(const Batch<kMaxViews> &, const Workspace &, const void *, int,
                                             float *, unsigned *, unsigned char *, float *, unsigned *,
                                             cudaStream_t);
template cudaError_t launch_backward<1>(const Batch<1> &, const Workspace &, long long, const float4 *,
                                        const float *, const void *, int, const unsigned *, const unsigned char *,
                                        const float *, float *, float *, float *, float *, const float *, double *,
                                        cudaStream_t);
template cudaError_t launch_backward<kMaxViews>(const Batch<kMaxViews> &, const Workspace &, long long,
                                                const float4 *, const float *, const void *, int,
                                                const unsigned *, const unsigned char *, const float *, float *,
                                                float *, float *, float *, const float *, double *, cudaStream_t);

}  // namespace tpk
