// common.cuh -- device-side data and arithmetic shared by the splatting kernels.
//
// The arithmetic here is the float32 evaluation of TRIPS' trilinear point
// splat (Franke et al. 2024): projection and screen size (Sec. 3.1, Eq. 2),
// layer pair and layer weight iota (Sec. 3.1, Eq. 5), bilinear taps beta
// (Eq. 4).  Every operation that decides an integer (culling, layers, taps,
// depth order) is written with explicit round-to-nearest intrinsics so the
// compiler cannot fuse or reorder it; the order is the one documented in
// include/trips.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "trips.h"

namespace tpk {

constexpr int kMaxLayers = 16;
constexpr int kBlock = 256;  // threads per CTA of every kernel
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr unsigned kNoPoint = 0xFFFFFFFFu;

// Everything a kernel needs to know about one frame (passed by value).
struct Frame {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float znear, eps;
    int n_layers, K, D;
    int tile_w, tile_h;
    int n_tiles;
    int tile_px;           // pixels per tile, tile_w * tile_h
    int tile_threads;      // threads per tile CTA: tile_px rounded up to a warp
    int chunk;             // tile-list entries merged per chunk by the tile kernels
    int desc_vec;          // 1 if descriptors can be read 4 channels at a time
    int grad_vec;          // 1 if descriptor gradients can take 4-channel vector atomics
    int pos4;              // 1: position gradients are [n][4] rows (X, Y, Z, s_w), one vector atomic each
    int grads_zeroed;      // 1: the caller cleared the gradient buffers (no memsets in the backward)
    int coarse;            // 1: coarse-layer inclusion (a pixel's list also holds the fragments of
                           //    the coarser-layer pixels that contain it, Sec. 3.6)
    int lw[kMaxLayers], lh[kMaxLayers];            // layer sizes W_L, H_L
    int tiles_x[kMaxLayers], tiles_y[kMaxLayers];  // tiles per layer row / column
    int tile_base[kMaxLayers + 1];                 // first tile id of each layer
    long long pix_base[kMaxLayers + 1];            // first pyramid pixel of each layer
};

// A batch of views rendered by the same launches: view v owns global tiles
// [tile_base[v], tile_base[v+1]) and global pyramid pixels
// [pix_base[v], pix_base[v+1]); its point records are rows [v n, (v+1) n).
// Passed to the kernels by value (MaxV = 1 for a single view, kMaxViews for
// batches; 16 views take about 10 KB of kernel parameters).
constexpr int kMaxViews = 16;

template <int MaxV>
struct Batch {
    int n_views;
    int n_tiles;          // tiles over all views
    long long n_pix;      // pyramid pixels over all views
    int max_threads;      // largest tile CTA over the views
    int tile_base[MaxV + 1];
    long long pix_base[MaxV + 1];
    long long cpix_base[MaxV + 1];  // first coarse-list row of each view (pixels of layers >= 1)
    Frame view[MaxV];
};

// Row of the coarse-list arrays of pixel (j, k) of layer L >= 1 of view v.
template <int MaxV>
__device__ __forceinline__ long long coarse_row(const Batch<MaxV> &B, int v, int L, int j, int k)
{
    const Frame &F = B.view[v];
    return B.cpix_base[v] + (F.pix_base[L] - F.pix_base[1]) + (long long)k * F.lw[L] + j;
}

// The tile of CTA blockIdx.x: every tile of the batch in order (layer < 0), or
// the tiles of one layer, view after view.
template <int MaxV>
__device__ __forceinline__ int block_tile(const Batch<MaxV> &B, int layer)
{
    int c = (int)blockIdx.x;
    if (layer < 0) return c;
    for (int v = 0; v < B.n_views; ++v) {
        const Frame &F = B.view[v];
        const int nt = F.tile_base[layer + 1] - F.tile_base[layer];
        if (c < nt) return B.tile_base[v] + F.tile_base[layer] + c;
        c -= nt;
    }
    return -1;
}

template <int MaxV>
__device__ __forceinline__ int view_of_tile(const Batch<MaxV> &B, int tile)
{
    int v = 0;
    if constexpr (MaxV > 1)
        while (v + 1 < B.n_views && tile >= B.tile_base[v + 1]) ++v;
    return v;
}

template <int MaxV>
__device__ __forceinline__ int view_of_pixel(const Batch<MaxV> &B, long long pix)
{
    int v = 0;
    if constexpr (MaxV > 1)
        while (v + 1 < B.n_views && pix >= B.pix_base[v + 1]) ++v;
    return v;
}

// Device pointers into the caller's workspace.
// Every tile counter exists in kCopies copies; point i uses copy
// (i / 32) % kCopies, the same for the 32 points of a warp.  Hot tiles
// (thousands of points near the horizon) would otherwise serialise their
// atomics on one address.
constexpr int kCopies = 32;

struct Workspace {
    unsigned *status;       // [1] TP_FLAG_* bits
    unsigned *tile_count;   // [n_tiles][kCopies] (point, tile) pairs per tile and copy
    unsigned *tile_off;     // [n_tiles + 1] first entry of each tile's list
    unsigned *tile_cursor;  // [n_tiles][kCopies] fill cursor of each copy (relative to tile_off)
    unsigned long long *bucket_key;  // [capacity] fragment key (z bits, point index) of each entry
    float4 *bucket_pay;     // [capacity] (x, y, s, alpha) of the entry's point
    unsigned long long *kmax;  // [P] largest kept key of each pixel (0: none), written by the blend
    // coarse-layer inclusion only: the kept list of every pixel of layers >= 1
    // (keys, then fragment opacities gamma as float bits), slot-major:
    // slot m of coarse row c at [m * crows + c]; empty slots hold kEmptyKey
    unsigned long long *ckey;
    unsigned *cgam;
    long long crows;
    long long n_points;     // points of the frame (index checks of the checking build)
    unsigned capacity;
    // the frame's point records [views][n] (x, y, z, s) and opacities [n]
    // (caller buffers, read by the blend: it recomputes each kept fragment's
    // opacity gamma from its point)
    const float4 *rec;
    const float *opacity;
};

// ---------------------------------------------------------------------------
// Projection (Eq. 2), float32 in the documented order, no contraction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool project_point(const Frame &F, float X, float Y, float Z, float sw, float4 &rec,
                                              bool &bad)
{
    bad = false;
    if (!(isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(sw)) || sw < 0.0f) {
        bad = true;
        return false;
    }
    float xc = __fmul_rn(F.R[0], X);
    xc = __fadd_rn(xc, __fmul_rn(F.R[1], Y));
    xc = __fadd_rn(xc, __fmul_rn(F.R[2], Z));
    xc = __fadd_rn(xc, F.t[0]);
    float yc = __fmul_rn(F.R[3], X);
    yc = __fadd_rn(yc, __fmul_rn(F.R[4], Y));
    yc = __fadd_rn(yc, __fmul_rn(F.R[5], Z));
    yc = __fadd_rn(yc, F.t[1]);
    float zc = __fmul_rn(F.R[6], X);
    zc = __fadd_rn(zc, __fmul_rn(F.R[7], Y));
    zc = __fadd_rn(zc, __fmul_rn(F.R[8], Z));
    zc = __fadd_rn(zc, F.t[2]);
    if (!(zc > F.znear)) return false;
    float x = __fadd_rn(__fdiv_rn(__fmul_rn(F.fx, xc), zc), F.cx);
    float y = __fadd_rn(__fdiv_rn(__fmul_rn(F.fy, yc), zc), F.cy);
    float s = __fdiv_rn(__fmul_rn(F.fx, sw), zc);
    if (!(isfinite(x) && isfinite(y) && isfinite(s))) {
        bad = true;
        return false;
    }
    rec = make_float4(x, y, zc, s);
    return true;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // exact 2^e

// ---------------------------------------------------------------------------
// Layer pair and layer weights iota (Sec. 3.1, Eq. 5).
// ---------------------------------------------------------------------------
struct LayerPair {
    int n;            // 1 or 2 layers
    int L[2];
    float iota[2];
    float diota[2];   // d iota / d s
};

__device__ __forceinline__ LayerPair layer_pair(float s, int n_layers, float eps)
{
    LayerPair p;
    if (s < 1.0f) {  // sub-pixel point: finest layer, iota >= eps
        p.n = 1;
        p.L[0] = 0;
        p.iota[0] = __fadd_rn(eps, __fmul_rn(__fsub_rn(1.0f, eps), s));
        p.diota[0] = __fsub_rn(1.0f, eps);
        return p;
    }
    const unsigned b = __float_as_uint(s);
    const int Ll = int(b >> 23) - 127;  // floor(log2 s), exact for normal s >= 1
    if (Ll >= n_layers - 1) {           // beyond the coarsest layer: clamp
        p.n = 1;
        p.L[0] = n_layers - 1;
        p.iota[0] = 1.0f;
        p.diota[0] = 0.0f;
        return p;
    }
    const float pl = pow2f(Ll), inv = pow2f(-Ll);
    p.L[0] = Ll;
    p.iota[0] = __fmul_rn(__fsub_rn(__fmul_rn(2.0f, pl), s), inv);  // (2^Lu - s) / 2^Ll, exact
    p.diota[0] = -inv;
    if ((b & 0x7FFFFFu) == 0u) {  // s = 2^Ll: the upper weight is exactly zero
        p.n = 1;
    } else {
        p.n = 2;
        p.L[1] = Ll + 1;
        p.iota[1] = __fmul_rn(__fsub_rn(s, pl), inv);  // (s - 2^Ll) / 2^Ll, exact
        p.diota[1] = inv;
    }
    return p;
}

// iota of layer L for a point of screen size s; false if the point is not in layer L.
__device__ __forceinline__ bool layer_weight(float s, int L, int n_layers, float eps, float &iota, float &diota)
{
    LayerPair p = layer_pair(s, n_layers, eps);
    if (p.L[0] == L) {
        iota = p.iota[0];
        diota = p.diota[0];
        return true;
    }
    if (p.n == 2 && p.L[1] == L) {
        iota = p.iota[1];
        diota = p.diota[1];
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Bilinear taps along one axis at layer L (Eq. 4): pixel centres at j + 0.5.
// ---------------------------------------------------------------------------
struct AxisTaps {
    int j0;     // first tap index floor(u)
    float a;    // u - j0: weight of tap j0 + 1; tap j0 has 1 - a
    bool t0;    // tap j0 exists and is inside the layer
    bool t1;    // tap j0 + 1 exists (a != 0) and is inside the layer
};

__device__ __forceinline__ AxisTaps axis_taps(float pos, int L, int extent)
{
    AxisTaps t;
    t.j0 = 0;
    t.a = 0.0f;
    t.t0 = t.t1 = false;
    const float u = __fsub_rn(__fmul_rn(pos, pow2f(-L)), 0.5f);
    if (!(u > -2.0f && u < __int2float_rn(extent) + 1.0f)) return t;
    const float fl = floorf(u);
    t.j0 = __float2int_rz(fl);
    t.a = __fsub_rn(u, fl);
    t.t0 = t.j0 >= 0 && t.j0 < extent;
    t.t1 = t.a != 0.0f && t.j0 + 1 >= 0 && t.j0 + 1 < extent;
    return t;
}

// Weight and derivative (w.r.t. the full-resolution coordinate) of tap j.
__device__ __forceinline__ void tap_weight(const AxisTaps &t, int j, int L, float &w, float &dw)
{
    const float scale = pow2f(-L);
    if (j == t.j0) {
        w = __fsub_rn(1.0f, t.a);
        dw = -scale;
    } else {
        w = t.a;
        dw = scale;
    }
}

// Inclusive range of tiles along one axis touched by the taps; false if none.
__device__ __forceinline__ bool tap_tile_range(const AxisTaps &t, int tile, int &lo, int &hi)
{
    if (!t.t0 && !t.t1) return false;
    const int jmin = t.t0 ? t.j0 : t.j0 + 1;
    const int jmax = t.t1 ? t.j0 + 1 : t.j0;
    lo = jmin / tile;
    hi = jmax / tile;
    return true;
}

// Sort key of a fragment: depth bits (z > 0, so the bits order like the
// values) above the point index, which breaks ties, above the fragment's own
// pyramid layer (4 bits), which orders a point's two layers in a list that
// holds both (coarse-layer inclusion), the finer first.  Point indices stay
// below 2^27, so the low word holds index and layer.
__device__ __forceinline__ unsigned long long frag_key(float z, unsigned i, int L)
{
    return ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)((i << 4) | (unsigned)L);
}
__device__ __forceinline__ unsigned key_point(unsigned long long key) { return (unsigned)(key & 0xFFFFFFFFull) >> 4; }
__device__ __forceinline__ int key_layer(unsigned long long key) { return (int)(key & 15ull); }

__device__ __forceinline__ int tile_layer(const Frame &F, int tile)
{
    int L = 0;
    while (L + 1 < F.n_layers && tile >= F.tile_base[L + 1]) ++L;
    return L;
}

__device__ __forceinline__ void raise_flag(unsigned *status, unsigned bit)
{
    if ((*((volatile unsigned *)status) & bit) == 0u) atomicOr(status, bit);
}

// Index checks of the checking build (TP_DEBUG): TP_IN_RANGE(status, cond)
// is cond, and a false cond also sets TP_FLAG_BOUNDS; the caller then skips
// the access.  In the release build the macro is the constant true and
// compiles away.
#ifdef TP_DEBUG
__device__ __forceinline__ bool in_range_checked(unsigned *status, bool ok)
{
    if (!ok) raise_flag(status, TP_FLAG_BOUNDS);
    return ok;
}
#define TP_IN_RANGE(status, cond) ::tpk::in_range_checked((status), (cond))
#else
#define TP_IN_RANGE(status, cond) true
#endif

template <typename T>
__device__ __forceinline__ float load_desc(const T *p);
template <>
__device__ __forceinline__ float load_desc<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_desc<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(*p);
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched by launch_dependent may be
// scheduled while the previous kernel of its stream is still finishing; it
// calls wait_previous_grid() before it touches anything that kernel wrote,
// and allow_dependent_launch() to let the next kernel be scheduled early.
// Both are no-ops for a kernel launched the ordinary way.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                    Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in bin.cu and blend.cu, for MaxV = 1 and kMaxViews).
// ---------------------------------------------------------------------------
template <int MaxV>
cudaError_t launch_project_count(const Batch<MaxV> &B, const Workspace &W, long long n, const float *pos,
                                 const float *size_w, float4 *rec, cudaStream_t stream);
template <int MaxV>
cudaError_t launch_scan_fill(const Batch<MaxV> &B, const Workspace &W, long long n, const float4 *rec,
                             const float *opacity, cudaStream_t stream);
template <int MaxV>
cudaError_t launch_blend(const Batch<MaxV> &B, const Workspace &W, const void *desc, int desc_dtype,
                         float *pyramid, unsigned *kept, unsigned char *n_kept, float *t_final, unsigned *n_frag,
                         cudaStream_t stream);
template <int MaxV>
cudaError_t launch_backward(const Batch<MaxV> &B, const Workspace &W, long long n, const float4 *rec,
                            const float *opacity, const void *desc, int desc_dtype, const unsigned *kept,
                            const unsigned char *n_kept, const float *grad_pyramid, float *grad_pos,
                            float *grad_sw, float *grad_opacity, float *grad_desc, const float *pos,
                            double *grad_cameras, cudaStream_t stream);
size_t tile_smem_bytes(const Frame &F, bool backward);

}  // namespace tpk
