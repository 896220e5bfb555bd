// bin.cu -- collect, offset-scan and splat stages (TRIPS Sec. 3.6).
//
// The paper's collect pass projects every point and counts the elements of
// every pixel list; an offset scan turns the counts into positions in one
// continuous array; the splatting pass then writes (z, i) pairs into those
// lists.  Here the lists are per screen tile instead of per pixel: a point's
// 2x2x2 splat touches at most 2x2 tiles in each of its two layers, so the
// count and fill passes make 1-2 global atomics per point instead of 4-8,
// and the per-pixel lists are formed later in shared memory by the blend
// kernel (blend.cu), which reads each tile's points with coalesced loads.
// Each tile counter is split into kCopies copies (the points of warp w use
// copy w % kCopies) so that the thousands of points of a dense tile do not
// queue on one address; k_tile_totals folds the copies back together.  The
// lanes of a warp that touch the same tile together make one atomic for the
// group, so a group's entries are consecutive in the tile's list and its
// stores coalesce.
#include "common.cuh"

namespace tpk {

// Calls fn(tile, L) for every screen tile the point's taps touch, at each of
// its layers L.  The taps and layers are exactly those of the blend kernels.
template <class Fn>
__device__ __forceinline__ void for_each_tile(const Frame &F, const float4 &r, Fn &&fn)
{
    const LayerPair lp = layer_pair(r.w, F.n_layers, F.eps);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q >= lp.n) break;
        const int L = lp.L[q];
        const AxisTaps tx = axis_taps(r.x, L, F.lw[L]);
        const AxisTaps ty = axis_taps(r.y, L, F.lh[L]);
        int x0, x1, y0, y1;
        if (!tap_tile_range(tx, F.tile_w, x0, x1) || !tap_tile_range(ty, F.tile_h, y0, y1)) continue;
        const int base = F.tile_base[L];
        const int tpr = F.tiles_x[L];
        for (int b = y0; b <= y1; ++b)
            for (int a = x0; a <= x1; ++a) fn(base + b * tpr + a, L);
    }
}

// The lanes of the calling warp that are here together and hold the same
// tile t: one group, whose lowest lane makes the group's atomic.
__device__ __forceinline__ unsigned tile_group(int t) { return __match_any_sync(__activemask(), t); }

// Copy of the counters point i uses: the same for every lane of its warp (the
// grid's threads are whole warps of consecutive i), so a group's atomic goes
// to the copy each of its points would use.
__device__ __forceinline__ unsigned point_copy(long long i) { return (unsigned)((i >> 5) & (kCopies - 1)); }

// Collect: project, cull, write the record and count (point, tile) pairs.
// blockIdx.y is the view; view v writes records rec[v n + i] and counts into
// its own range of global tiles.
template <int MaxV>
__global__ void __launch_bounds__(kBlock) k_project_count(const __grid_constant__ Batch<MaxV> B, Workspace W,
                                                          long long n, const float *__restrict__ pos,
                                                          const float *__restrict__ size_w, float4 *__restrict__ rec_all)
{
    allow_dependent_launch();
    const int v = MaxV > 1 ? (int)blockIdx.y : 0;
    const Frame &F = B.view[v];
    float4 *__restrict__ rec = rec_all + (long long)v * n;
    unsigned *__restrict__ count = W.tile_count + (size_t)B.tile_base[v] * kCopies;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float X = __ldg(pos + 3 * i), Y = __ldg(pos + 3 * i + 1), Z = __ldg(pos + 3 * i + 2);
        float4 r;
        bool bad;
        const bool vis = project_point(F, X, Y, Z, __ldg(size_w + i), r, bad);
        if (bad) raise_flag(W.status, TP_FLAG_NONFINITE);
        if (!vis) {
            rec[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            continue;
        }
        rec[i] = r;
        const unsigned c = point_copy(i);
        const int lane = threadIdx.x & 31;
        for_each_tile(F, r, [&](int t, int) {
            if (!TP_IN_RANGE(W.status, t >= 0 && t < F.n_tiles)) return;
            const unsigned grp = tile_group(t);
            if (lane == __ffs(grp) - 1) atomicAdd(count + (size_t)t * kCopies + c, (unsigned)__popc(grp));
        });
    }
}

// One warp per tile: the copies' exclusive prefix becomes each copy's fill
// cursor, and the tile's total goes to tile_off[t] for the offset scan.
__global__ void __launch_bounds__(kBlock) k_tile_totals(int n_tiles, Workspace W)
{
    wait_previous_grid();
    allow_dependent_launch();
    const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= n_tiles) return;
    const unsigned v = W.tile_count[(size_t)t * kCopies + lane];
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    W.tile_cursor[(size_t)t * kCopies + lane] = x - v;
    if (lane == 31) W.tile_off[t] = x;
}

// Exclusive scan of the tile totals in tile_off (in place) by one CTA of
// 1024 threads, in chunks of kScanPer x 1024 tiles: each chunk is staged in
// shared memory with coalesced loads (padded one word per kScanPer so that
// each thread's run of kScanPer consecutive values is read without bank
// conflicts), scanned as per-thread runs plus a block scan of the run sums,
// and written back coalesced; a carry links the chunks.
constexpr int kScanPer = 8;
constexpr int kScanTile = 1024 * kScanPer;

__device__ __forceinline__ int scan_slot(int q) { return q + q / kScanPer; }

__global__ void __launch_bounds__(1024) k_scan_tiles(int n_tiles, Workspace W)
{
    __shared__ unsigned sv[kScanTile + kScanTile / kScanPer];
    __shared__ unsigned warp_tot[32];
    wait_previous_grid();
    allow_dependent_launch();
    const int T = n_tiles, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    unsigned carry = 0;
    for (int c0 = 0; c0 < T; c0 += kScanTile) {
        const int n = min(kScanTile, T - c0);
        for (int q = tid; q < kScanTile; q += 1024) sv[scan_slot(q)] = q < n ? W.tile_off[c0 + q] : 0u;
        __syncthreads();
        unsigned run[kScanPer], sum = 0;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            run[i] = sv[scan_slot(tid * kScanPer + i)];
            sum += run[i];
        }
        unsigned v = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) warp_tot[warp] = v;
        __syncthreads();
        if (warp == 0) {
            unsigned w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        unsigned off = carry + v - sum + (warp > 0 ? warp_tot[warp - 1] : 0u);
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            sv[scan_slot(tid * kScanPer + i)] = off;
            off += run[i];
        }
        carry += warp_tot[31];
        __syncthreads();
        for (int q = tid; q < n; q += 1024) W.tile_off[c0 + q] = sv[scan_slot(q)];
        __syncthreads();
    }
    if (tid == 0) {
        W.tile_off[T] = carry;
        if (carry > W.capacity) raise_flag(W.status, TP_FLAG_CAPACITY);
    }
}

// Splat: every point appends its fragment key (z, i, L) and its blend payload
// (x, y, s, alpha) to the list of each tile it touches.
template <int MaxV>
__global__ void __launch_bounds__(kBlock) k_fill(const __grid_constant__ Batch<MaxV> B, Workspace W, long long n,
                                                 const float4 *__restrict__ rec_all, const float *__restrict__ opacity)
{
    const int v = MaxV > 1 ? (int)blockIdx.y : 0;
    const Frame &F = B.view[v];
    const float4 *__restrict__ rec = rec_all + (long long)v * n;
    const unsigned *__restrict__ tile_off = W.tile_off + B.tile_base[v];
    unsigned *__restrict__ cursor = W.tile_cursor + (size_t)B.tile_base[v] * kCopies;
    wait_previous_grid();
    allow_dependent_launch();
    if (*((volatile unsigned *)W.status) & TP_FLAG_CAPACITY) return;  // the lists do not fit: outputs invalid
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 r = rec[i];
        if (!(r.z > 0.0f)) continue;  // culled
        const float4 pay = make_float4(r.x, r.y, r.w, __ldg(opacity + i));
        const unsigned c = point_copy(i);
        const int lane = threadIdx.x & 31;
        for_each_tile(F, r, [&](int t, int L) {
            if (!TP_IN_RANGE(W.status, t >= 0 && t < F.n_tiles)) return;
            const unsigned long long key = frag_key(r.z, (unsigned)i, L);
            // the group takes consecutive slots of its copy, in lane order
            const unsigned grp = tile_group(t);
            const int lead = __ffs(grp) - 1;
            unsigned base = 0u;
            if (lane == lead) base = atomicAdd(cursor + (size_t)t * kCopies + c, (unsigned)__popc(grp));
            const unsigned e =
                tile_off[t] + __shfl_sync(grp, base, lead) + (unsigned)__popc(grp & ((1u << lane) - 1u));
            if (e < W.capacity) {
                W.bucket_key[e] = key;
                W.bucket_pay[e] = pay;
            }
        });
    }
}

static int grid_for(long long n)
{
    long long b = (n + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

template <int MaxV>
cudaError_t launch_project_count(const Batch<MaxV> &B, const Workspace &W, long long n, const float *pos,
                                 const float *size_w, float4 *rec, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(W.status, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(W.tile_count, 0, sizeof(unsigned) * kCopies * (size_t)B.n_tiles, stream);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    const dim3 grid(grid_for(n), B.n_views);
    k_project_count<MaxV><<<grid, kBlock, 0, stream>>>(B, W, n, pos, size_w, rec);
    return cudaGetLastError();
}

template <int MaxV>
cudaError_t launch_scan_fill(const Batch<MaxV> &B, const Workspace &W, long long n, const float4 *rec,
                             const float *opacity, cudaStream_t stream)
{
    const long long threads = (long long)B.n_tiles * 32;
    cudaError_t e = launch_dependent(k_tile_totals, dim3((unsigned)((threads + kBlock - 1) / kBlock)), dim3(kBlock),
                                     0, stream, B.n_tiles, W);
    if (e != cudaSuccess) return e;
    e = launch_dependent(k_scan_tiles, dim3(1), dim3(1024), 0, stream, B.n_tiles, W);
    if (e != cudaSuccess || n == 0) return e;
    const dim3 grid(grid_for(n), B.n_views);
    return launch_dependent(k_fill<MaxV>, grid, dim3(kBlock), 0, stream, B, W, n, rec, opacity);
}

template cudaError_t launch_project_count<1>(const Batch<1> &, const Workspace &, long long, const float *,
                                             const float *, float4 *, cudaStream_t);
template cudaError_t launch_project_count<kMaxViews>(const Batch<kMaxViews> &, const Workspace &, long long,
                                                     const float *, const float *, float4 *, cudaStream_t);
template cudaError_t launch_scan_fill<1>(const Batch<1> &, const Workspace &, long long, const float4 *,
                                         const float *, cudaStream_t);
template cudaError_t launch_scan_fill<kMaxViews>(const Batch<kMaxViews> &, const Workspace &, long long,
                                                 const float4 *, const float *, cudaStream_t);

}  // namespace tpk
