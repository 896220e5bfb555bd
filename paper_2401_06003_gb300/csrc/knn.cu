// knn.cu -- point-size initialisation (TRIPS Sec. 3.6): each point's initial
// world size is the mean distance to its four nearest other points.
//
// Exact k-nearest-neighbour search on hashed uniform grids, all on the device
// (no host round trip):
//   1. bounding box of the finite points and the finest cell size
//      c0 = extent / (8 max(64, 4 n^(1/3)));
//   2. per level m (cell c_m = c0 8^m): counting sort of the points by the
//      hash of their cell -- its Morton code modulo the table size, so that
//      neighbouring cells sit in neighbouring table entries -- (count,
//      three-phase scan, fill), the sorted copy holding (x, y, z, index);
//   3. a ring search per point (level 0: one thread per point; later levels,
//      whose few points meet the densest cells, one warp per point): rings
//      r = 0, 1, 2, ... of cells around the point's cell; every unvisited
//      point is farther than r c_m, so the
//      search stops once it holds k neighbours within r c_m.  A point not
//      settled within kRingsPerLevel rings moves to the next, coarser level
//      (dense regions settle on fine grids, sparse ones climb); the last
//      level is coarse enough to settle every point.
// Candidates are filtered by their own cell, so hash collisions never visit
// a point twice.  Distances are float32; a point's own index is never its
// neighbour, duplicates at distance 0 are; non-finite points are nobody's
// neighbour and get size 0.
#include <algorithm>

#include "common.cuh"

namespace tpk {

namespace {

constexpr int kKnnK = 4;
constexpr int kKnnBlock = 256;
constexpr int kKnnLevels = 6;
constexpr int kRingsPerLevel = 3;
constexpr int kScanChunk = 1024;  // elements per block of the scan's first phase
constexpr int kKnnGrid = 152 * 8;

// Header of the workspace (256 bytes).
struct KnnHdr {
    unsigned bmin[3], bmax[3];  // bounding box, floats in an order-preserving integer encoding
    unsigned n_finite;
    unsigned n_open[2];         // unsettled points handed to the next level (ping-pong)
    unsigned pad;
    float lo[3];                // decoded box minimum
    float c0;                   // finest cell
    float extent;               // largest box side
};

struct KnnWs {
    KnnHdr *hdr;
    unsigned *count;   // [T]
    unsigned *start;   // [T + 1]
    unsigned *bsum;    // [T / kScanChunk]
    float4 *spos;      // [n] points sorted by cell hash: x, y, z, index bits
    unsigned *open[2]; // [n] unsettled point indices
    float *bound[2];   // [n] their best 4th squared distance so far (INFINITY: fewer than 4 seen)
    unsigned T;        // hash table size (power of two)
};

__device__ __forceinline__ unsigned f2ord(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ bool finite3(float x, float y, float z) { return isfinite(x) && isfinite(y) && isfinite(z); }

// Spreads the low 10 bits of v to every third bit.
__device__ __forceinline__ unsigned spread3(unsigned v)
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Table slot of a cell: the Morton code of its low 10 coordinate bits (30
// bits) mixed with a hash of the higher bits, modulo the table size.  Cells
// that are close share high bits, so their slots are close in the table.
__device__ __forceinline__ unsigned cell_hash(int ix, int iy, int iz, unsigned T)
{
    const unsigned ux = (unsigned)ix, uy = (unsigned)iy, uz = (unsigned)iz;
    const unsigned morton = spread3(ux) | (spread3(uy) << 1) | (spread3(uz) << 2);
    const unsigned high = ((ux >> 10) * 73856093u) ^ ((uy >> 10) * 19349663u) ^ ((uz >> 10) * 83492791u);
    return (morton ^ (high << 12)) & (T - 1u);
}

__device__ __forceinline__ int cell_of(float v, float lo, float inv_c) { return (int)floorf((v - lo) * inv_c); }

__global__ void k_knn_bbox(long long n, const float *__restrict__ pos, KnnHdr *hdr)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    unsigned cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!finite3(x, y, z)) continue;
        ++cnt;
        mn[0] = fminf(mn[0], x); mn[1] = fminf(mn[1], y); mn[2] = fminf(mn[2], z);
        mx[0] = fmaxf(mx[0], x); mx[1] = fmaxf(mx[1], y); mx[2] = fmaxf(mx[2], z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0) {
        atomicAdd(&hdr->n_finite, cnt);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&hdr->bmin[a], f2ord(mn[a]));
            atomicMax(&hdr->bmax[a], f2ord(mx[a]));
        }
    }
}

__global__ void k_knn_setup(KnnHdr *hdr)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float lo = hdr->n_finite ? ord2f(hdr->bmin[a]) : 0.0f;
        const float hi = hdr->n_finite ? ord2f(hdr->bmax[a]) : 0.0f;
        hdr->lo[a] = lo;
        ext = fmaxf(ext, hi - lo);
    }
    const float cr = cbrtf((float)(hdr->n_finite > 0 ? hdr->n_finite : 1));
    float c0 = ext / (8.0f * fmaxf(64.0f, 4.0f * cr));
    if (!(c0 > 0.0f)) c0 = 1.0f;  // all points in one place
    hdr->c0 = c0;
    hdr->extent = ext;
    hdr->n_open[0] = hdr->n_open[1] = 0u;
}

__device__ __forceinline__ float level_cell(const KnnHdr *hdr, int level)
{
    float c = hdr->c0;
    for (int m = 0; m < level; ++m) c *= 8.0f;
    return c;
}

__global__ void k_knn_count(long long n, const float *__restrict__ pos, KnnWs W, int level)
{
    const KnnHdr *hdr = W.hdr;
    if (level > 0 && hdr->n_open[(level - 1) & 1] == 0) return;  // every point is settled
    const float inv_c = 1.0f / level_cell(hdr, level);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!finite3(x, y, z)) continue;
        const unsigned h = cell_hash(cell_of(x, hdr->lo[0], inv_c), cell_of(y, hdr->lo[1], inv_c),
                                     cell_of(z, hdr->lo[2], inv_c), W.T);
        atomicAdd(W.count + h, 1u);
    }
}

// Scan phase 1: exclusive scan of each kScanChunk-element block of count into
// start, block totals into bsum (256 threads, 4 consecutive elements each).
__global__ void __launch_bounds__(256) k_scan_blocks(const unsigned *__restrict__ count, unsigned *__restrict__ start,
                                                     unsigned *__restrict__ bsum, unsigned T)
{
    __shared__ unsigned ws[8];
    const unsigned base = blockIdx.x * kScanChunk + threadIdx.x * 4;
    unsigned v[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = base + q < T ? count[base + q] : 0u;
        s += v[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < 8 ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) ws[lane] = w;
    }
    __syncthreads();
    unsigned run = x - s + (warp > 0 ? ws[warp - 1] : 0u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < T) start[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 255) bsum[blockIdx.x] = run;
}

// Scan phase 2: exclusive scan of the block totals in place (one CTA of 1024
// threads, each a contiguous run); start[T] gets the grand total.
__global__ void __launch_bounds__(1024) k_scan_sums(unsigned *__restrict__ bsum, unsigned nb, unsigned *start_end)
{
    __shared__ unsigned ws[32];
    const unsigned per = (nb + 1023) / 1024;
    const unsigned b0 = threadIdx.x * per;
    unsigned s = 0;
    for (unsigned q = 0; q < per; ++q)
        if (b0 + q < nb) s += bsum[b0 + q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    unsigned run = x - s + (warp > 0 ? ws[warp - 1] : 0u);
    for (unsigned q = 0; q < per; ++q) {
        if (b0 + q < nb) {
            const unsigned v = bsum[b0 + q];
            bsum[b0 + q] = run;
            run += v;
        }
    }
    if (threadIdx.x == 1023) *start_end = run;
}

// Scan phase 3: add each block's offset.
__global__ void k_scan_add(unsigned *__restrict__ start, const unsigned *__restrict__ bsum, unsigned T)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T) start[i] += bsum[i / kScanChunk];
}

__global__ void k_knn_fill(long long n, const float *__restrict__ pos, KnnWs W, int level)
{
    const KnnHdr *hdr = W.hdr;
    if (level > 0 && hdr->n_open[(level - 1) & 1] == 0) return;
    const float inv_c = 1.0f / level_cell(hdr, level);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!finite3(x, y, z)) continue;
        const unsigned h = cell_hash(cell_of(x, hdr->lo[0], inv_c), cell_of(y, hdr->lo[1], inv_c),
                                     cell_of(z, hdr->lo[2], inv_c), W.T);
        const unsigned q = W.start[h] + atomicAdd(W.count + h, 1u);
        W.spos[q] = make_float4(x, y, z, __uint_as_float((unsigned)i));
    }
}

// k smallest squared distances, ascending.
struct Best {
    float d[kKnnK];
    int n;
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int q = 0; q < kKnnK; ++q) d[q] = INFINITY;
        n = 0;
    }
    __device__ __forceinline__ void insert(float v)
    {
        if (v >= d[kKnnK - 1]) return;
#pragma unroll
        for (int q = 0; q < kKnnK; ++q) {
            const float t = d[q];
            const bool lt = v < t;
            d[q] = lt ? v : t;
            v = lt ? t : v;
        }
        n = n < kKnnK ? n + 1 : kKnnK;
    }
};

// Squared distance from (x, y, z) to cell (ix, iy, iz) widened by 1% of a
// cell on every side (a binned point may sit that far outside its cell).
__device__ __forceinline__ float cell_dist2(const KnnHdr *hdr, float c, int ix, int iy, int iz, float x, float y,
                                            float z)
{
    const float m = 0.01f * c;
    float d2 = 0.0f;
    const float v[3] = {x, y, z};
    const int id[3] = {ix, iy, iz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = hdr->lo[a] + (float)id[a] * c - m, hi = lo + c + 2.0f * m;
        const float e = v[a] < lo ? lo - v[a] : (v[a] > hi ? v[a] - hi : 0.0f);
        d2 += e * e;
    }
    return d2;
}

// Ring search of one point at one level; true when settled (size written).
// `bound` is an upper bound of the point's 4th squared distance from an
// earlier level (INFINITY if none): cells farther than it are skipped.  On
// return it holds the best bound found here.
__device__ bool search_point(const KnnWs &W, int level, bool last, unsigned self, float x, float y, float z,
                             float &bound, float *__restrict__ size_w)
{
    const KnnHdr *hdr = W.hdr;
    const float c = level_cell(hdr, level), inv_c = 1.0f / c;
    const int cx = cell_of(x, hdr->lo[0], inv_c), cy = cell_of(y, hdr->lo[1], inv_c), cz = cell_of(z, hdr->lo[2], inv_c);
    const unsigned nf = hdr->n_finite;
    const int want = (int)min((unsigned)kKnnK, nf > 0 ? nf - 1 : 0u);
    // rings beyond r_all cover the whole box: every finite point has been seen
    const int r_all = (int)(hdr->extent * inv_c) + 2;
    const int r_max = last ? r_all : min(kRingsPerLevel, r_all);
    Best b;
    b.clear();
    for (int r = 0; r <= r_max; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = dz == -r || dz == r || dy == -r || dy == r;
                for (int dx = -r; dx <= r; dx += face ? 1 : 2 * r) {
                    const int ix = cx + dx, iy = cy + dy, iz = cz + dz;
                    const float prune = fminf(bound, b.n >= kKnnK ? b.d[kKnnK - 1] : INFINITY);
                    if (r > 0 && cell_dist2(hdr, c, ix, iy, iz, x, y, z) > prune)
                        continue;  // every point of the cell is farther than 4 known ones
                    const unsigned h = cell_hash(ix, iy, iz, W.T);
                    const unsigned e1 = W.start[h + 1];
                    for (unsigned q = W.start[h]; q < e1; ++q) {
                        const float4 p = W.spos[q];
                        if (__float_as_uint(p.w) == self) continue;
                        if (cell_of(p.x, hdr->lo[0], inv_c) != ix || cell_of(p.y, hdr->lo[1], inv_c) != iy ||
                            cell_of(p.z, hdr->lo[2], inv_c) != iz)
                            continue;  // another cell with the same hash
                        const float ex = p.x - x, ey = p.y - y, ez = p.z - z;
                        b.insert(ex * ex + ey * ey + ez * ez);
                    }
                    if (r == 0) break;
                }
            }
        }
        // every point outside rings 0..r is at least r c away, less twice the
        // float32 rounding of a cell coordinate (< 0.006 cells below 2^16 cells
        // per axis): a 2% margin covers it
        const float reach = (float)r * c * 0.98f;
        const bool done = r >= r_all || (b.n >= want && (want == 0 || b.d[want - 1] <= reach * reach));
        if (done) {
            float s = 0.0f;
            for (int q = 0; q < want; ++q) s += sqrtf(b.d[q]);
            size_w[self] = want > 0 ? s / (float)want : 0.0f;
            return true;
        }
    }
    if (b.n >= kKnnK) bound = fminf(bound, b.d[kKnnK - 1]);
    return false;
}

// The k smallest of the union of the lanes' lists (each ascending), the same
// in every lane: k rounds of a warp minimum, the lane that held it moving on.
// Squared distances are >= +0, so their bits order like their values.
__device__ __forceinline__ void warp_best(const Best &b, float out[kKnnK], int &cnt)
{
    const int lane = threadIdx.x & 31;
    int p = 0;
    cnt = 0;
#pragma unroll
    for (int r = 0; r < kKnnK; ++r) {
        float mine = INFINITY;
#pragma unroll
        for (int q = 0; q < kKnnK; ++q) mine = p == q ? b.d[q] : mine;
        const unsigned mu = __float_as_uint(mine);
        const unsigned m = __reduce_min_sync(0xffffffffu, mu);
        out[r] = __uint_as_float(m);
        cnt += m != __float_as_uint(INFINITY) ? 1 : 0;
        const unsigned who = __ballot_sync(0xffffffffu, mu == m);
        if (lane == __ffs(who) - 1 && m != __float_as_uint(INFINITY)) ++p;
    }
}

// search_point for one point by a whole warp: the rings and cells are the
// same for every lane, each lane takes every 32nd point of a cell, and the
// lanes' lists are merged at the end of every ring (for the stop test and
// the pruning bound).  For the few points left to the coarser levels, whose
// cells can hold thousands of points.  Same result as search_point.
__device__ bool search_point_warp(const KnnWs &W, int level, bool last, unsigned self, float x, float y, float z,
                                  float &bound, float *__restrict__ size_w)
{
    const KnnHdr *hdr = W.hdr;
    const int lane = threadIdx.x & 31;
    const float c = level_cell(hdr, level), inv_c = 1.0f / c;
    const int cx = cell_of(x, hdr->lo[0], inv_c), cy = cell_of(y, hdr->lo[1], inv_c), cz = cell_of(z, hdr->lo[2], inv_c);
    const unsigned nf = hdr->n_finite;
    const int want = (int)min((unsigned)kKnnK, nf > 0 ? nf - 1 : 0u);
    const int r_all = (int)(hdr->extent * inv_c) + 2;
    const int r_max = last ? r_all : min(kRingsPerLevel, r_all);
    Best b;
    b.clear();
    float merged[kKnnK];
    int n_merged = 0;
    float prune = bound;  // uniform: the carried bound, then the merged 4th distance
    for (int r = 0; r <= r_max; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = dz == -r || dz == r || dy == -r || dy == r;
                for (int dx = -r; dx <= r; dx += face ? 1 : 2 * r) {
                    const int ix = cx + dx, iy = cy + dy, iz = cz + dz;
                    if (r > 0 && cell_dist2(hdr, c, ix, iy, iz, x, y, z) > prune) continue;
                    const unsigned h = cell_hash(ix, iy, iz, W.T);
                    const unsigned e0 = W.start[h], e1 = W.start[h + 1];
                    for (unsigned q = e0 + lane; q < e1; q += 32) {
                        const float4 p = W.spos[q];
                        if (__float_as_uint(p.w) == self) continue;
                        if (cell_of(p.x, hdr->lo[0], inv_c) != ix || cell_of(p.y, hdr->lo[1], inv_c) != iy ||
                            cell_of(p.z, hdr->lo[2], inv_c) != iz)
                            continue;  // another cell with the same hash
                        const float ex = p.x - x, ey = p.y - y, ez = p.z - z;
                        b.insert(ex * ex + ey * ey + ez * ez);
                    }
                    if (r == 0) break;
                }
            }
        }
        warp_best(b, merged, n_merged);
        if (n_merged >= kKnnK) prune = fminf(bound, merged[kKnnK - 1]);
        const float reach = (float)r * c * 0.98f;  // as in search_point
        const bool done = r >= r_all || (n_merged >= want && (want == 0 || merged[want - 1] <= reach * reach));
        if (done) {
            if (lane == 0) {
                float s = 0.0f;
                for (int q = 0; q < want; ++q) s += sqrtf(merged[q]);
                size_w[self] = want > 0 ? s / (float)want : 0.0f;
            }
            return true;
        }
    }
    if (n_merged >= kKnnK) bound = fminf(bound, merged[kKnnK - 1]);
    return false;
}

// Levels >= 1: one warp per point left unsettled.
__global__ void __launch_bounds__(kKnnBlock) k_knn_query_warp(const float *__restrict__ pos, KnnWs W, int level,
                                                              int last, float *__restrict__ size_w)
{
    KnnHdr *hdr = W.hdr;
    const unsigned todo = hdr->n_open[(level - 1) & 1];
    const unsigned *in = W.open[(level - 1) & 1];
    const float *in_bound = W.bound[(level - 1) & 1];
    unsigned *out = W.open[level & 1];
    float *out_bound = W.bound[level & 1];
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < todo; t += warps) {
        const unsigned i = in[t];
        float bound = in_bound[t];
        const float x = pos[3 * (long long)i], y = pos[3 * (long long)i + 1], z = pos[3 * (long long)i + 2];
        if (!search_point_warp(W, level, last != 0, i, x, y, z, bound, size_w) && (threadIdx.x & 31) == 0) {
            const unsigned slot = atomicAdd(&hdr->n_open[level & 1], 1u);
            out[slot] = i;
            out_bound[slot] = bound;
        }
    }
}

// Level 0 visits the points in their sorted order (neighbouring threads search
// neighbouring cells); later levels take the list of points left unsettled.
__global__ void __launch_bounds__(kKnnBlock) k_knn_query(const float *__restrict__ pos, KnnWs W, int level, int last,
                                                         float *__restrict__ size_w)
{
    KnnHdr *hdr = W.hdr;
    const unsigned todo = level == 0 ? hdr->n_finite : hdr->n_open[(level - 1) & 1];
    const unsigned *in = W.open[(level - 1) & 1];
    const float *in_bound = W.bound[(level - 1) & 1];
    unsigned *out = W.open[level & 1];
    float *out_bound = W.bound[level & 1];
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < todo; t += gridDim.x * blockDim.x) {
        float x, y, z, bound = INFINITY;
        unsigned i;
        if (level == 0) {
            const float4 p = W.spos[t];
            x = p.x; y = p.y; z = p.z;
            i = __float_as_uint(p.w);
        } else {
            i = in[t];
            bound = in_bound[t];
            x = pos[3 * (long long)i]; y = pos[3 * (long long)i + 1]; z = pos[3 * (long long)i + 2];
        }
        if (!search_point(W, level, last != 0, i, x, y, z, bound, size_w)) {
            const unsigned slot = atomicAdd(&hdr->n_open[level & 1], 1u);
            out[slot] = i;
            out_bound[slot] = bound;
        }
    }
}

__global__ void k_knn_clear_sizes(long long n, const float *__restrict__ pos, float *__restrict__ size_w)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (!finite3(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2])) size_w[i] = 0.0f;
}

__global__ void k_knn_reset_open(KnnHdr *hdr, int slot) { hdr->n_open[slot] = 0u; }

struct KnnLayout {
    unsigned T;
    int64_t count, start, bsum, spos, open0, open1, bound0, bound1, end;
};

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

KnnLayout knn_layout(int64_t n)
{
    KnnLayout L;
    unsigned T = 1024;
    while ((int64_t)T < 2 * n && T < (1u << 30)) T <<= 1;
    L.T = T;
    L.count = 256;
    L.start = align256(L.count + 4 * (int64_t)T);
    L.bsum = align256(L.start + 4 * ((int64_t)T + 1));
    L.spos = align256(L.bsum + 4 * (int64_t)(T / kScanChunk + 1));
    L.open0 = align256(L.spos + 16 * n);
    L.open1 = align256(L.open0 + 4 * n);
    L.bound0 = align256(L.open1 + 4 * n);
    L.bound1 = align256(L.bound0 + 4 * n);
    L.end = align256(L.bound1 + 4 * n);
    return L;
}

}  // namespace

}  // namespace tpk

extern "C" {

int64_t tp_init_sizes_workspace_bytes(int64_t n_points)
{
    if (n_points < 0 || n_points >= ((int64_t)1 << 31)) return -1;
    return tpk::knn_layout(n_points).end;
}

tp_status tp_init_point_sizes(int64_t n, const float *pos, float *size_w, void *ws, int64_t ws_bytes,
                              tp_stream_t stream)
{
    using namespace tpk;
    if (n < 0 || n >= ((int64_t)1 << 31)) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!pos || !size_w || !ws || ((uintptr_t)ws & 255u) != 0) return TP_ERR_INVALID_ARG;
    const KnnLayout L = knn_layout(n);
    if (ws_bytes < L.end) return TP_ERR_INVALID_ARG;
    char *base = static_cast<char *>(ws);
    KnnWs W;
    W.hdr = reinterpret_cast<KnnHdr *>(base);
    W.count = reinterpret_cast<unsigned *>(base + L.count);
    W.start = reinterpret_cast<unsigned *>(base + L.start);
    W.bsum = reinterpret_cast<unsigned *>(base + L.bsum);
    W.spos = reinterpret_cast<float4 *>(base + L.spos);
    W.open[0] = reinterpret_cast<unsigned *>(base + L.open0);
    W.open[1] = reinterpret_cast<unsigned *>(base + L.open1);
    W.bound[0] = reinterpret_cast<float *>(base + L.bound0);
    W.bound[1] = reinterpret_cast<float *>(base + L.bound1);
    W.T = L.T;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nb = L.T / kScanChunk;
    const int grid_pts = (int)std::min<long long>((n + kKnnBlock - 1) / kKnnBlock, kKnnGrid);
    cudaError_t e = cudaMemsetAsync(W.hdr, 0, sizeof(KnnHdr), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.hdr->bmin, 0xFF, sizeof(W.hdr->bmin), s);
    if (e != cudaSuccess) return TP_ERR_CUDA;
    k_knn_bbox<<<grid_pts, kKnnBlock, 0, s>>>(n, pos, W.hdr);
    k_knn_setup<<<1, 32, 0, s>>>(W.hdr);
    k_knn_clear_sizes<<<grid_pts, kKnnBlock, 0, s>>>(n, pos, size_w);
    for (int level = 0; level < kKnnLevels; ++level) {
        if (level >= 1) k_knn_reset_open<<<1, 1, 0, s>>>(W.hdr, level & 1);
        if (cudaMemsetAsync(W.count, 0, 4 * (size_t)L.T, s) != cudaSuccess) return TP_ERR_CUDA;
        k_knn_count<<<grid_pts, kKnnBlock, 0, s>>>(n, pos, W, level);
        k_scan_blocks<<<nb, 256, 0, s>>>(W.count, W.start, W.bsum, L.T);
        k_scan_sums<<<1, 1024, 0, s>>>(W.bsum, nb, W.start + L.T);
        k_scan_add<<<(L.T + 255) / 256, 256, 0, s>>>(W.start, W.bsum, L.T);
        if (cudaMemsetAsync(W.count, 0, 4 * (size_t)L.T, s) != cudaSuccess) return TP_ERR_CUDA;
        k_knn_fill<<<grid_pts, kKnnBlock, 0, s>>>(n, pos, W, level);
        if (level == 0)
            k_knn_query<<<kKnnGrid, kKnnBlock, 0, s>>>(pos, W, level, 0, size_w);
        else
            k_knn_query_warp<<<kKnnGrid, kKnnBlock, 0, s>>>(pos, W, level, level == kKnnLevels - 1, size_w);
        if (cudaGetLastError() != cudaSuccess) return TP_ERR_CUDA;
    }
    return TP_OK;
}

}  // extern "C"
