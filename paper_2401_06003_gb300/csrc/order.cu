// order.cu -- spatial order of a point cloud (a one-time relabeling of the
// points, outside the render path).
//
// The splatting kernels touch a point's data at every stage -- its tile
// counters and tile-list appends in the collect and splat passes, its
// descriptor row in the blend, its gradient rows in the backward pass -- and
// the points that meet in one screen tile are neighbours in space.  Stored in
// the order of a space-filling curve, neighbours sit next to each other in
// memory, so those accesses share cache lines and DRAM pages instead of
// landing at random.  tp_spatial_order computes that order (the Morton code
// of each point's cell in a 1024^3 grid over the cloud's bounding box, sorted
// stably) and tp_permute_rows applies it to any per-point array.  Rendering a
// relabeled cloud gives the same pixels; only the point indices (and so the
// tie order of fragments at exactly equal depth) follow the new labels.
//
// The sort is a stable least-significant-digit radix sort written for this
// library: four passes of 8 bits over the 32-bit codes, each a per-tile digit
// histogram, an exclusive scan of the histograms (digit-major, tile-minor) and
// a scatter in which each tile places its elements in their original order
// (warp match for the ranks within a warp, per-warp digit counts for the
// ranks across warps).
#include <cstdint>

#include "common.cuh"

namespace tpk {

namespace {

constexpr int kOrdBlock = 256;
constexpr int kOrdWarps = kOrdBlock / 32;
constexpr int kBuckets = 256;
constexpr int kTileChunks = 16;                          // chunks of kOrdBlock elements per sort tile
constexpr int kTileElems = kOrdBlock * kTileChunks;      // 4096
constexpr int kMortonBits = 10;                          // grid cells per axis: 2^10

struct OrdHdr {
    unsigned bmin[3], bmax[3];  // bounding box of the finite points, floats in an order-preserving encoding
    float lo[3];
    float scale;                // (2^10 - 1) / largest box side (0 for a single position)
};

__device__ __forceinline__ unsigned f2ord(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float ord2f(unsigned o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

__global__ void k_ord_init(OrdHdr *hdr)
{
    for (int a = 0; a < 3; ++a) {
        hdr->bmin[a] = 0xFFFFFFFFu;
        hdr->bmax[a] = 0u;
    }
}

__global__ void __launch_bounds__(kOrdBlock) k_ord_bbox(long long n, const float *__restrict__ pos, OrdHdr *hdr)
{
    __shared__ unsigned smin[3], smax[3];
    if (threadIdx.x < 3) {
        smin[threadIdx.x] = 0xFFFFFFFFu;
        smax[threadIdx.x] = 0u;
    }
    __syncthreads();
    unsigned mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0u, 0u, 0u};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
        const unsigned o[3] = {f2ord(x), f2ord(y), f2ord(z)};
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], o[a]);
            mx[a] = max(mx[a], o[a]);
        }
    }
    for (int a = 0; a < 3; ++a) {
        atomicMin(&smin[a], mn[a]);
        atomicMax(&smax[a], mx[a]);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&hdr->bmin[threadIdx.x], smin[threadIdx.x]);
        atomicMax(&hdr->bmax[threadIdx.x], smax[threadIdx.x]);
    }
}

__global__ void k_ord_setup(OrdHdr *hdr)
{
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        if (hdr->bmin[a] > hdr->bmax[a]) {  // no finite point
            hdr->lo[a] = 0.0f;
            continue;
        }
        hdr->lo[a] = ord2f(hdr->bmin[a]);
        ext = fmaxf(ext, __fsub_rn(ord2f(hdr->bmax[a]), hdr->lo[a]));
    }
    hdr->scale = ext > 0.0f ? __fdiv_rn((float)((1 << kMortonBits) - 1), ext) : 0.0f;
}

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

// Morton code of the point's cell (x in the lowest bit of each triple); a
// point with a non-finite coordinate gets the largest code (last).
__global__ void __launch_bounds__(kOrdBlock) k_ord_codes(long long n, const float *__restrict__ pos,
                                                         const OrdHdr *__restrict__ hdr, unsigned *__restrict__ code,
                                                         unsigned *__restrict__ idx)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const float s = hdr->scale;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        unsigned c = 0xFFFFFFFFu;
        if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
            c = 0u;
            for (int a = 0; a < 3; ++a) {
                int q = __float2int_rz(__fmul_rn(__fsub_rn(p[a], hdr->lo[a]), s));
                q = min(max(q, 0), (1 << kMortonBits) - 1);
                c |= spread3((unsigned)q) << a;
            }
        }
        code[i] = c;
        idx[i] = (unsigned)i;
    }
}

// Digit histogram of each sort tile: hist[digit * n_tiles + tile].
__global__ void __launch_bounds__(kOrdBlock) k_ord_hist(long long n, const unsigned *__restrict__ key, int shift,
                                                        unsigned *__restrict__ hist, unsigned n_tiles)
{
    __shared__ unsigned h[kBuckets];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * kTileElems;
    for (int q = 0; q < kTileChunks; ++q) {
        const long long i = t0 + (long long)q * kOrdBlock + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m values in place, one CTA of 1024 threads, in chunks of
// 1024 x 4 values with a running carry.
__global__ void __launch_bounds__(1024) k_ord_scan(unsigned *__restrict__ v, long long m)
{
    __shared__ unsigned wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned carry = 0u;
    for (long long c0 = 0; c0 < m; c0 += 4096) {
        unsigned x[4], sum = 0u;
        for (int k = 0; k < 4; ++k) {
            const long long i = c0 + 4LL * tid + k;
            x[k] = i < m ? v[i] : 0u;
            sum += x[k];
        }
        unsigned incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned w = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        unsigned run = carry + incl - sum + (warp > 0 ? wsum[warp - 1] : 0u);
        for (int k = 0; k < 4; ++k) {
            const long long i = c0 + 4LL * tid + k;
            if (i < m) v[i] = run;
            run += x[k];
        }
        carry += wsum[31];
        __syncthreads();
    }
}

// Stable scatter of one radix pass: each CTA places its tile's elements, in
// their order, after everything of a smaller digit and after the same digit
// of earlier tiles.
__global__ void __launch_bounds__(kOrdBlock) k_ord_scatter(long long n, const unsigned *__restrict__ key_in,
                                                           const unsigned *__restrict__ val_in, int shift,
                                                           const unsigned *__restrict__ hist, unsigned n_tiles,
                                                           unsigned *__restrict__ key_out,
                                                           unsigned *__restrict__ val_out)
{
    __shared__ unsigned base[kBuckets];
    __shared__ unsigned wcnt[kOrdWarps][kBuckets];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = hist[(size_t)tid * n_tiles + blockIdx.x];
    for (int w = 0; w < kOrdWarps; ++w) wcnt[w][tid] = 0u;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * kTileElems;
    for (int q = 0; q < kTileChunks; ++q) {
        const long long i = t0 + (long long)q * kOrdBlock + tid;
        const bool valid = i < n;
        const unsigned k = valid ? key_in[i] : 0u;
        const unsigned v = valid ? val_in[i] : 0u;
        const unsigned d = valid ? ((k >> shift) & 0xFFu) : (unsigned)kBuckets + lane;  // invalid lanes: unique
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // thread tid = digit: offsets of the warps' runs of this digit within the chunk
        unsigned run = 0u;
        for (int w = 0; w < kOrdWarps; ++w) {
            const unsigned c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const unsigned dst = base[d] + wcnt[warp][d] + rank;
            key_out[dst] = k;
            val_out[dst] = v;
        }
        __syncthreads();
        base[tid] += run;
        for (int w = 0; w < kOrdWarps; ++w) wcnt[w][tid] = 0u;
        __syncthreads();
    }
}

__global__ void k_ord_copy(long long n, const unsigned *__restrict__ src, unsigned *__restrict__ dst)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// dst row k = src row perm[k]; rows of `words` 32-bit words.
__global__ void k_permute_rows(long long n, int words, const unsigned *__restrict__ src,
                               const unsigned *__restrict__ perm, unsigned *__restrict__ dst)
{
    const long long total = n * words;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const long long k = q / words;
        const int w = (int)(q - k * words);
        dst[q] = src[(long long)perm[k] * words + w];
    }
}

struct OrdLayout {
    int64_t hdr, code0, idx0, code1, idx1, hist, end;
};

OrdLayout ord_layout(int64_t n)
{
    auto up = [](int64_t v) { return (v + 255) / 256 * 256; };
    const int64_t tiles = (n + kTileElems - 1) / kTileElems;
    OrdLayout L;
    L.hdr = 0;
    L.code0 = up((int64_t)sizeof(OrdHdr));
    L.idx0 = up(L.code0 + 4 * n);
    L.code1 = up(L.idx0 + 4 * n);
    L.idx1 = up(L.code1 + 4 * n);
    L.hist = up(L.idx1 + 4 * n);
    L.end = L.hist + 4 * (int64_t)kBuckets * (tiles > 0 ? tiles : 1);
    return L;
}

int grid_pts(int64_t n)
{
    int64_t b = (n + kOrdBlock - 1) / kOrdBlock;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

}  // namespace tpk

extern "C" {

int64_t tp_spatial_order_workspace_bytes(int64_t n_points)
{
    if (n_points < 0 || n_points >= ((int64_t)1 << 31)) return -1;
    return tpk::ord_layout(n_points).end;
}

tp_status tp_spatial_order(int64_t n, const float *pos, uint32_t *perm, void *ws, int64_t ws_bytes,
                           tp_stream_t stream)
{
    using namespace tpk;
    if (n < 0 || n >= ((int64_t)1 << 31)) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!pos || !perm || !ws || ((uintptr_t)ws % 256) != 0) return TP_ERR_INVALID_ARG;
    const OrdLayout L = ord_layout(n);
    if (ws_bytes < L.end) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char *base = static_cast<char *>(ws);
    OrdHdr *hdr = reinterpret_cast<OrdHdr *>(base + L.hdr);
    unsigned *code[2] = {reinterpret_cast<unsigned *>(base + L.code0), reinterpret_cast<unsigned *>(base + L.code1)};
    unsigned *idx[2] = {reinterpret_cast<unsigned *>(base + L.idx0), reinterpret_cast<unsigned *>(base + L.idx1)};
    unsigned *hist = reinterpret_cast<unsigned *>(base + L.hist);
    const unsigned tiles = (unsigned)((n + kTileElems - 1) / kTileElems);
    k_ord_init<<<1, 1, 0, s>>>(hdr);
    k_ord_bbox<<<grid_pts(n), kOrdBlock, 0, s>>>(n, pos, hdr);
    k_ord_setup<<<1, 1, 0, s>>>(hdr);
    k_ord_codes<<<grid_pts(n), kOrdBlock, 0, s>>>(n, pos, hdr, code[0], idx[0]);
    for (int pass = 0; pass < 4; ++pass) {
        const int a = pass & 1, b = a ^ 1, shift = 8 * pass;
        k_ord_hist<<<tiles, kOrdBlock, 0, s>>>(n, code[a], shift, hist, tiles);
        k_ord_scan<<<1, 1024, 0, s>>>(hist, (long long)kBuckets * tiles);
        k_ord_scatter<<<tiles, kOrdBlock, 0, s>>>(n, code[a], idx[a], shift, hist, tiles, code[b], idx[b]);
    }
    k_ord_copy<<<grid_pts(n), kOrdBlock, 0, s>>>(n, idx[0], perm);
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

tp_status tp_permute_rows(int64_t n, int32_t row_bytes, const void *src, const uint32_t *perm, void *dst,
                          tp_stream_t stream)
{
    using namespace tpk;
    if (n < 0 || row_bytes < 4 || (row_bytes % 4) != 0) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!src || !perm || !dst || src == dst || ((uintptr_t)src % 4) != 0 || ((uintptr_t)dst % 4) != 0)
        return TP_ERR_INVALID_ARG;
    const int words = row_bytes / 4;
    k_permute_rows<<<grid_pts(n * words), kOrdBlock, 0, (cudaStream_t)stream>>>(
        n, words, static_cast<const unsigned *>(src), perm, static_cast<unsigned *>(dst));
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

}  // extern "C"
