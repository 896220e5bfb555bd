// blend.cu -- combined sort and accumulate stage and its adjoint (TRIPS Sec. 3.2, 3.6).
//
// One CTA owns one screen tile of one pyramid layer.  It streams the tile's
// (point, tile) entries written by the splat pass, computes each point's
// taps inside the tile (Eq. 3-5) and inserts the fragment key (z, i) into a
// per-pixel sorted buffer of K slots in shared memory.  The insertion is a
// cascade of atomicMin on 64-bit keys: each slot keeps the smaller of its
// value and the incoming key and passes the larger one on.  Whatever the
// interleaving, slot m ends with the m-th smallest key of all fragments of
// the pixel, so the buffer holds exactly the K front-most fragments in
// (depth, index) order -- the list the paper sorts per pixel and clamps to
// 16 elements (Sec. 3.2), without materialising the full list.  The pixel
// then blends its kept fragments front to back (Eq. 6-7) in registers.
//
// The backward kernels run the adjoint of the blend per pixel back to front
// over the kept list (division-free recurrence) and scatter the point
// gradients with float atomics.
#include "common.cuh"

namespace tpk {

__device__ __forceinline__ unsigned long long ld_relaxed_shared(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.cta.shared.b64 %0, [%1];"
                 : "=l"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}

// Insert a key into a pixel's K sorted slots.  Slots only ever decrease, and
// at every instant they are sorted; a slot that is already smaller than the
// key stays smaller, so the search may skip it.
template <int K>
__device__ __forceinline__ void kbuf_insert(unsigned long long *slots, unsigned long long key)
{
    if (key >= ld_relaxed_shared(slots + K - 1)) return;
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ld_relaxed_shared(slots + mid) > key) hi = mid;
        else lo = mid + 1;
    }
    for (int j = lo; j < K; ++j) {
        const unsigned long long old = atomicMin(slots + j, key);
        if (old == kEmptyKey) return;
        key = old > key ? old : key;
    }
}

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

// Build the K-slot buffers and candidate counts of every pixel of the tile.
template <int K>
__device__ void build_kbuffer(const Frame &F, const Workspace &W, int tile, const TileGeom &g,
                              unsigned long long *kb, unsigned *nf)
{
    const int TW = F.tile_w, TH = F.tile_h, TP = TW * TH;
    for (int q = threadIdx.x; q < TP * K; q += blockDim.x) kb[q] = kEmptyKey;
    for (int q = threadIdx.x; q < TP; q += blockDim.x) nf[q] = 0u;
    __syncthreads();
    unsigned end = W.tile_off[tile + 1];
    if (end > W.capacity) end = W.capacity;
    unsigned beg = W.tile_off[tile];
    if (beg > end) beg = end;
    const int L = g.L;
    for (unsigned e = beg + threadIdx.x; e < end; e += blockDim.x) {
        const float4 r = W.bucket_rec[e];
        const unsigned i = W.bucket_idx[e];
        float iota, diota;
        if (!layer_weight(r.w, L, F.n_layers, F.eps, iota, diota)) continue;
        const AxisTaps ax = axis_taps(r.x, L, F.lw[L]);
        const AxisTaps ay = axis_taps(r.y, L, F.lh[L]);
        const unsigned long long key = frag_key(r.z, i);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!(b ? ay.t1 : ay.t0)) continue;
            const int k = ay.j0 + b - g.y0;
            if (k < 0 || k >= TH) continue;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (!(a ? ax.t1 : ax.t0)) continue;
                const int j = ax.j0 + a - g.x0;
                if (j < 0 || j >= TW) continue;
                const int px = k * TW + j;
                atomicAdd(nf + px, 1u);
                kbuf_insert<K>(kb + px * K, key);
            }
        }
    }
    __syncthreads();
}

// Tap weight beta * iota of point record r at layer-L pixel (j, k), with the
// pieces the adjoint needs.
struct FragW {
    float wx, wy, dwx, dwy, iota, diota;
};

__device__ __forceinline__ FragW frag_weights(const Frame &F, const float4 &r, int L, int j, int k)
{
    FragW w;
    layer_weight(r.w, L, F.n_layers, F.eps, w.iota, w.diota);
    const AxisTaps ax = axis_taps(r.x, L, F.lw[L]);
    const AxisTaps ay = axis_taps(r.y, L, F.lh[L]);
    tap_weight(ax, j, L, w.wx, w.dwx);
    tap_weight(ay, k, L, w.wy, w.dwy);
    return w;
}

// Blend one pixel's kept fragments (ids[0..nk)) and write its outputs.
template <int K, typename DescT>
__device__ __forceinline__ void blend_pixel(const Frame &F, int L, int j, int k, long long pix, const unsigned *ids,
                                            int nk, unsigned nfrag, const float4 *__restrict__ rec,
                                            const float *__restrict__ opacity, const DescT *__restrict__ desc,
                                            float *__restrict__ pyramid, unsigned *__restrict__ kept,
                                            unsigned char *__restrict__ n_kept, float *__restrict__ t_final,
                                            unsigned *__restrict__ n_frag)
{
    float wgt[K];
    float T = 1.0f;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        wgt[m] = 0.0f;
        if (m < nk) {
            const unsigned i = ids[m];
            const float4 r = rec[i];
            const FragW w = frag_weights(F, r, L, j, k);
            const float g = w.wx * w.wy * w.iota * __ldg(opacity + i);
            wgt[m] = T * g;
            T = T * (1.0f - g);
        }
    }
    const int D = F.D;
    float *out = pyramid + pix * D;
    for (int d = 0; d < D; ++d) {
        float c = 0.0f;
#pragma unroll
        for (int m = 0; m < K; ++m)
            if (m < nk) c += wgt[m] * load_desc(desc + (long long)ids[m] * D + d);
        out[d] = c;
    }
    if (kept) {
#pragma unroll
        for (int m = 0; m < K; ++m) kept[pix * K + m] = m < nk ? ids[m] : kNoPoint;
    }
    if (n_kept) n_kept[pix] = (unsigned char)nk;
    if (t_final) t_final[pix] = T;
    if (n_frag) n_frag[pix] = nfrag;
}

template <int K, typename DescT>
__global__ void __launch_bounds__(kBlock) k_tile_blend(Frame F, Workspace W, const float4 *__restrict__ rec,
                                                       const float *__restrict__ opacity,
                                                       const DescT *__restrict__ desc, float *__restrict__ pyramid,
                                                       unsigned *__restrict__ kept, unsigned char *__restrict__ n_kept,
                                                       float *__restrict__ t_final, unsigned *__restrict__ n_frag)
{
    extern __shared__ unsigned long long smem[];
    const int TW = F.tile_w, TP = F.tile_w * F.tile_h;
    unsigned long long *kb = smem;
    unsigned *nf = reinterpret_cast<unsigned *>(smem + TP * K);
    const int tile = blockIdx.x;
    const TileGeom g = tile_geom(F, tile);
    build_kbuffer<K>(F, W, tile, g, kb, nf);
    const int L = g.L;
    for (int px = threadIdx.x; px < TP; px += blockDim.x) {
        const int j = g.x0 + px % TW, k = g.y0 + px / TW;
        if (j >= F.lw[L] || k >= F.lh[L]) continue;
        const long long pix = F.pix_base[L] + (long long)k * F.lw[L] + j;
        const unsigned nfr = nf[px];
        const int nk = nfr < (unsigned)K ? (int)nfr : K;
        unsigned ids[K];
#pragma unroll
        for (int m = 0; m < K; ++m) ids[m] = m < nk ? (unsigned)(kb[px * K + m] & 0xFFFFFFFFull) : kNoPoint;
        blend_pixel<K, DescT>(F, L, j, k, pix, ids, nk, nfr, rec, opacity, desc, pyramid, kept, n_kept, t_final,
                              n_frag);
    }
}

// Adjoint of one pixel's blend, scattered into the point gradients.
template <int K, typename DescT>
__device__ __forceinline__ void adjoint_pixel(const Frame &F, int L, int j, int k, long long pix, const unsigned *ids,
                                              int nk, const float4 *__restrict__ rec,
                                              const float *__restrict__ opacity, const DescT *__restrict__ desc,
                                              const float *__restrict__ grad_pyr, float *__restrict__ gpos,
                                              float *__restrict__ gsw, float *__restrict__ gop,
                                              float *__restrict__ gdesc)
{
    const int D = F.D;
    const float *G = grad_pyr + pix * D;
    float gam[K], Tm[K];
    float T = 1.0f;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        gam[m] = 0.0f;
        Tm[m] = 0.0f;
        if (m < nk) {
            const unsigned i = ids[m];
            const FragW w = frag_weights(F, rec[i], L, j, k);
            const float g = w.wx * w.wy * w.iota * __ldg(opacity + i);
            gam[m] = g;
            Tm[m] = T;
            T = T * (1.0f - g);
        }
    }
    float R = 0.0f;
#pragma unroll
    for (int m = K - 1; m >= 0; --m) {
        if (m >= nk) continue;
        const unsigned i = ids[m];
        const float4 r = rec[i];
        const float al = __ldg(opacity + i);
        const FragW w = frag_weights(F, r, L, j, k);
        const DescT *c = desc + (long long)i * D;
        float gdot = 0.0f;
        for (int d = 0; d < D; ++d) gdot += __ldg(G + d) * load_desc(c + d);
        const float dg = Tm[m] * (gdot - R);
        R = gam[m] * gdot + (1.0f - gam[m]) * R;
        const float tg = Tm[m] * gam[m];
        float *gd = gdesc + (long long)i * D;
        for (int d = 0; d < D; ++d) atomicAdd(gd + d, tg * __ldg(G + d));
        const float beta = w.wx * w.wy;
        atomicAdd(gop + i, dg * beta * w.iota);
        const float dw = dg * al;
        const float gx = dw * w.wy * w.iota * w.dwx;
        const float gy = dw * w.wx * w.iota * w.dwy;
        const float gs = dw * beta * w.diota;
        const float iz = 1.0f / r.z;
        const float dXc = gx * F.fx * iz;
        const float dYc = gy * F.fy * iz;
        const float dZc = -(gx * (r.x - F.cx) + gy * (r.y - F.cy) + gs * r.w) * iz;
        atomicAdd(gsw + i, gs * F.fx * iz);
        atomicAdd(gpos + 3 * (long long)i + 0, F.R[0] * dXc + F.R[3] * dYc + F.R[6] * dZc);
        atomicAdd(gpos + 3 * (long long)i + 1, F.R[1] * dXc + F.R[4] * dYc + F.R[7] * dZc);
        atomicAdd(gpos + 3 * (long long)i + 2, F.R[2] * dXc + F.R[5] * dYc + F.R[8] * dZc);
    }
}

// Backward with the lists recomputed from the tile entries.
template <int K, typename DescT>
__global__ void __launch_bounds__(kBlock) k_tile_backward(Frame F, Workspace W, const float4 *__restrict__ rec,
                                                          const float *__restrict__ opacity,
                                                          const DescT *__restrict__ desc,
                                                          const float *__restrict__ grad_pyr, float *__restrict__ gpos,
                                                          float *__restrict__ gsw, float *__restrict__ gop,
                                                          float *__restrict__ gdesc)
{
    extern __shared__ unsigned long long smem[];
    const int TW = F.tile_w, TP = F.tile_w * F.tile_h;
    unsigned long long *kb = smem;
    unsigned *nf = reinterpret_cast<unsigned *>(smem + TP * K);
    const int tile = blockIdx.x;
    const TileGeom g = tile_geom(F, tile);
    build_kbuffer<K>(F, W, tile, g, kb, nf);
    const int L = g.L;
    for (int px = threadIdx.x; px < TP; px += blockDim.x) {
        const int j = g.x0 + px % TW, k = g.y0 + px / TW;
        if (j >= F.lw[L] || k >= F.lh[L]) continue;
        const unsigned nfr = nf[px];
        const int nk = nfr < (unsigned)K ? (int)nfr : K;
        if (nk == 0) continue;
        const long long pix = F.pix_base[L] + (long long)k * F.lw[L] + j;
        unsigned ids[K];
#pragma unroll
        for (int m = 0; m < K; ++m) ids[m] = m < nk ? (unsigned)(kb[px * K + m] & 0xFFFFFFFFull) : kNoPoint;
        adjoint_pixel<K, DescT>(F, L, j, k, pix, ids, nk, rec, opacity, desc, grad_pyr, gpos, gsw, gop, gdesc);
    }
}

// Backward with the lists stored by the blend kernel.
template <int K, typename DescT>
__global__ void __launch_bounds__(kBlock) k_stored_backward(Frame F, long long P, const float4 *__restrict__ rec,
                                                            const float *__restrict__ opacity,
                                                            const DescT *__restrict__ desc,
                                                            const unsigned *__restrict__ kept,
                                                            const unsigned char *__restrict__ n_kept,
                                                            const float *__restrict__ grad_pyr,
                                                            float *__restrict__ gpos, float *__restrict__ gsw,
                                                            float *__restrict__ gop, float *__restrict__ gdesc)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x; pix < P; pix += stride) {
        int nk = n_kept[pix];
        if (nk == 0) continue;
        if (nk > K) nk = K;
        int L = 0;
        while (L + 1 < F.n_layers && pix >= F.pix_base[L + 1]) ++L;
        const long long local = pix - F.pix_base[L];
        const int j = (int)(local % F.lw[L]), k = (int)(local / F.lw[L]);
        unsigned ids[K];
#pragma unroll
        for (int m = 0; m < K; ++m) ids[m] = m < nk ? kept[pix * K + m] : kNoPoint;
        adjoint_pixel<K, DescT>(F, L, j, k, pix, ids, nk, rec, opacity, desc, grad_pyr, gpos, gsw, gop, gdesc);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <class KernelT>
static cudaError_t allow_smem(KernelT kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static size_t tile_smem(const Frame &F, int K)
{
    const size_t TP = (size_t)F.tile_w * F.tile_h;
    return TP * K * sizeof(unsigned long long) + TP * sizeof(unsigned);
}

template <int K, typename DescT>
static cudaError_t blend_impl(const Frame &F, const Workspace &W, const float4 *rec, const float *opacity,
                              const void *desc, float *pyramid, unsigned *kept, unsigned char *n_kept,
                              float *t_final, unsigned *n_frag, cudaStream_t stream)
{
    const size_t smem = tile_smem(F, K);
    cudaError_t e = allow_smem(k_tile_blend<K, DescT>, smem);
    if (e != cudaSuccess) return e;
    k_tile_blend<K, DescT><<<F.n_tiles, kBlock, smem, stream>>>(
        F, W, rec, opacity, static_cast<const DescT *>(desc), pyramid, kept, n_kept, t_final, n_frag);
    return cudaGetLastError();
}

template <int K, typename DescT>
static cudaError_t backward_impl(const Frame &F, const Workspace &W, const float4 *rec, const float *opacity,
                                 const void *desc, const unsigned *kept, const unsigned char *n_kept,
                                 const float *grad_pyr, float *gpos, float *gsw, float *gop, float *gdesc,
                                 cudaStream_t stream)
{
    const DescT *d = static_cast<const DescT *>(desc);
    if (kept) {
        const long long P = F.pix_base[F.n_layers];
        long long blocks = (P + kBlock - 1) / kBlock;
        if (blocks > 152 * 32) blocks = 152 * 32;
        if (blocks < 1) blocks = 1;
        k_stored_backward<K, DescT><<<(int)blocks, kBlock, 0, stream>>>(F, P, rec, opacity, d, kept, n_kept,
                                                                        grad_pyr, gpos, gsw, gop, gdesc);
        return cudaGetLastError();
    }
    const size_t smem = tile_smem(F, K);
    cudaError_t e = allow_smem(k_tile_backward<K, DescT>, smem);
    if (e != cudaSuccess) return e;
    k_tile_backward<K, DescT><<<F.n_tiles, kBlock, smem, stream>>>(F, W, rec, opacity, d, grad_pyr, gpos, gsw,
                                                                   gop, gdesc);
    return cudaGetLastError();
}

#define TPK_DISPATCH_K(KVAL, ...)                                   \
    switch (KVAL) {                                                 \
    case 4: { constexpr int KC = 4; __VA_ARGS__; } break;           \
    case 8: { constexpr int KC = 8; __VA_ARGS__; } break;           \
    case 16: { constexpr int KC = 16; __VA_ARGS__; } break;         \
    case 32: { constexpr int KC = 32; __VA_ARGS__; } break;         \
    default: return cudaErrorInvalidValue;                          \
    }

cudaError_t launch_blend(const Frame &F, const Workspace &W, const float4 *rec, const float *opacity,
                         const void *desc, int desc_dtype, float *pyramid, unsigned *kept, unsigned char *n_kept,
                         float *t_final, unsigned *n_frag, cudaStream_t stream)
{
    if (desc_dtype == TP_BF16) {
        TPK_DISPATCH_K(F.K, return (blend_impl<KC, __nv_bfloat16>(F, W, rec, opacity, desc, pyramid, kept,
                                                                 n_kept, t_final, n_frag, stream)));
    } else {
        TPK_DISPATCH_K(F.K, return (blend_impl<KC, float>(F, W, rec, opacity, desc, pyramid, kept, n_kept,
                                                         t_final, n_frag, stream)));
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_backward(const Frame &F, const Workspace &W, long long n, const float4 *rec,
                            const float *opacity, const void *desc, int desc_dtype, const unsigned *kept,
                            const unsigned char *n_kept, const float *grad_pyramid, float *grad_pos,
                            float *grad_sw, float *grad_opacity, float *grad_desc, cudaStream_t stream)
{
    cudaError_t e;
    if (n == 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(grad_pos, 0, sizeof(float) * 3 * (size_t)n, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad_sw, 0, sizeof(float) * (size_t)n, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad_opacity, 0, sizeof(float) * (size_t)n, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad_desc, 0, sizeof(float) * (size_t)F.D * (size_t)n, stream)) != cudaSuccess)
        return e;
    if (desc_dtype == TP_BF16) {
        TPK_DISPATCH_K(F.K, return (backward_impl<KC, __nv_bfloat16>(F, W, rec, opacity, desc, kept, n_kept,
                                                                    grad_pyramid, grad_pos, grad_sw, grad_opacity,
                                                                    grad_desc, stream)));
    } else {
        TPK_DISPATCH_K(F.K, return (backward_impl<KC, float>(F, W, rec, opacity, desc, kept, n_kept, grad_pyramid,
                                                            grad_pos, grad_sw, grad_opacity, grad_desc, stream)));
    }
    return cudaErrorInvalidValue;
}

}  // namespace tpk
