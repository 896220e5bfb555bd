// merge.cu -- the pyramid merge of the decoder, without weights (TRIPS Sec. 3.3).
//
// The paper's network upsamples every layer but the finest bilinearly and
// merges it with the next finer layer, down to one full-resolution image.
// Without trained weights the merge is a sum:
//   M_{n-1} = P_{n-1},   M_L = P_L + up2(M_{L+1}),
// where up2 samples layer L+1 at the centres of layer L's pixels: pixel j of
// layer L sits at (j + 0.5) 2^L, at r = (j + 0.5)/2 - 0.5 >= 0 (clamped) in
// layer L+1 units, with taps floor(r) and min(floor(r) + 1, W_{L+1} - 1).
// All weights are multiples of 1/4, exact in float32.  Out of place the merge
// is one launch (k_merge_fused); in place one launch per layer, coarse to
// fine.  The adjoint runs fine to coarse, one launch per layer:
//   dL/dP_L = dL/dM_L,   dL/dM_{L+1} = up2^T dL/dM_L,
// gathering for each coarse pixel the at most 4 x 4 fine pixels that sample it.
#include "common.cuh"

namespace tpk {

namespace {

constexpr int kMergeBlock = 256;
constexpr int kMaxMergeD = 64;  // descriptor width limit of the library

struct Tap {
    int x0, x1;
    float lam;  // weight of x1; x0 has 1 - lam
};

__device__ __forceinline__ Tap up_tap(int j, int n_coarse)
{
    float r = (float)j * 0.5f - 0.25f;  // (j + 0.5)/2 - 0.5, exact
    r = r > 0.0f ? r : 0.0f;
    Tap t;
    t.x0 = (int)r;  // r >= 0: truncation is floor
    t.x1 = min(t.x0 + 1, n_coarse - 1);
    t.lam = r - (float)t.x0;
    return t;
}

// Weight with which fine pixel j samples coarse pixel c.
__device__ __forceinline__ float up_weight(int j, int c, int n_coarse)
{
    const Tap t = up_tap(j, n_coarse);
    return (t.x0 == c ? 1.0f - t.lam : 0.0f) + (t.x1 == c ? t.lam : 0.0f);
}

// Channel groups of DV = 4 floats (one 16-byte access) when D is a multiple
// of 4 and the rows are 16-byte aligned; DV = 1 otherwise.
template <int DV>
struct Vec;
template <>
struct Vec<4> {
    using T = float4;
    static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ float4 fma(float w, float4 a, float4 acc)
    {
        return make_float4(__fmaf_rn(w, a.x, acc.x), __fmaf_rn(w, a.y, acc.y), __fmaf_rn(w, a.z, acc.z),
                           __fmaf_rn(w, a.w, acc.w));
    }
    static __device__ __forceinline__ float4 add(float4 a, float4 b)
    {
        return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
    }
};
template <>
struct Vec<1> {
    using T = float;
    static __device__ __forceinline__ float zero() { return 0.f; }
    static __device__ __forceinline__ float fma(float w, float a, float acc) { return __fmaf_rn(w, a, acc); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
};

// M = P + up2(coarse) at one pixel from its four coarse taps, in a fixed
// order of explicitly rounded operations, so that the per-layer and the fused
// merge give the same bits.
template <int DV>
__device__ __forceinline__ typename Vec<DV>::T up_combine(typename Vec<DV>::T v, typename Vec<DV>::T c00,
                                                          typename Vec<DV>::T c01, typename Vec<DV>::T c10,
                                                          typename Vec<DV>::T c11, const Tap &tx, const Tap &ty)
{
    using V = Vec<DV>;
    const auto top = V::fma(tx.lam, c01, V::fma(1.0f - tx.lam, c00, V::zero()));
    const auto bot = V::fma(tx.lam, c11, V::fma(1.0f - tx.lam, c10, V::zero()));
    return V::add(v, V::fma(ty.lam, bot, V::fma(1.0f - ty.lam, top, V::zero())));
}

// M_L = P_L (+ up2(M_{L+1}) when coarse != null), one thread per (pixel,
// channel group); G = D / DV groups per pixel.  P and M may be the same array.
template <int DV>
__global__ void __launch_bounds__(kMergeBlock) k_merge_layer(int Wf, int Hf, int Wc, int Hc, int G,
                                                             const float *P, const float *__restrict__ coarse,
                                                             float *M)
{
    using V = Vec<DV>;
    using T = typename V::T;
    const long long n = (long long)Wf * Hf * G;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long p = q / G;
    const int gch = (int)(q - p * G);
    const T *Pv = reinterpret_cast<const T *>(P);
    T *Mv = reinterpret_cast<T *>(M);
    T v = Pv[q];
    if (coarse) {
        const int j = (int)(p % Wf), k = (int)(p / Wf);
        const Tap tx = up_tap(j, Wc), ty = up_tap(k, Hc);
        const T *C = reinterpret_cast<const T *>(coarse);
        const T c00 = C[((long long)ty.x0 * Wc + tx.x0) * G + gch], c01 = C[((long long)ty.x0 * Wc + tx.x1) * G + gch];
        const T c10 = C[((long long)ty.x1 * Wc + tx.x0) * G + gch], c11 = C[((long long)ty.x1 * Wc + tx.x1) * G + gch];
        v = up_combine<DV>(v, c00, c01, c10, c11, tx, ty);
    }
    Mv[q] = v;
}

// dL/dM_{L+1} = up2^T dL/dM_L: coarse pixel (jc, kc) gathers the fine pixels
// j in [2 jc - 1, 2 jc + 2], k in [2 kc - 1, 2 kc + 2] that sample it (the
// only ones whose taps can reach it, edge clamping included).
template <int DV>
__global__ void __launch_bounds__(kMergeBlock) k_merge_adjoint_layer(int Wf, int Hf, int Wc, int Hc, int G,
                                                                     const float *__restrict__ gfine,
                                                                     float *__restrict__ gcoarse)
{
    using V = Vec<DV>;
    using T = typename V::T;
    const long long n = (long long)Wc * Hc * G;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long p = q / G;
    const int gch = (int)(q - p * G);
    const int jc = (int)(p % Wc), kc = (int)(p / Wc);
    const T *F = reinterpret_cast<const T *>(gfine);
    T acc = V::zero();
    for (int k = max(2 * kc - 1, 0); k <= min(2 * kc + 2, Hf - 1); ++k) {
        const float wy = up_weight(k, kc, Hc);
        if (wy == 0.0f) continue;
        for (int j = max(2 * jc - 1, 0); j <= min(2 * jc + 2, Wf - 1); ++j) {
            const float w = wy * up_weight(j, jc, Wc);
            if (w != 0.0f) acc = V::fma(w, F[((long long)k * Wf + j) * G + gch], acc);
        }
    }
    reinterpret_cast<T *>(gcoarse)[q] = acc;
}

struct Layers {
    int n;
    int w[kMaxLayers], h[kMaxLayers];
    long long off[kMaxLayers + 1];
};

bool layers_of(const tp_camera *cam, int n_layers, Layers &ly)
{
    if (!cam || cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768) return false;
    if (n_layers < 1 || n_layers > kMaxLayers) return false;
    ly.n = n_layers;
    ly.off[0] = 0;
    for (int L = 0; L < n_layers; ++L) {
        ly.w[L] = (cam->width + (1 << L) - 1) >> L;
        ly.h[L] = (cam->height + (1 << L) - 1) >> L;
        ly.off[L + 1] = ly.off[L] + (long long)ly.w[L] * ly.h[L];
    }
    return true;
}

int blocks_for(long long n) { return (int)((n + kMergeBlock - 1) / kMergeBlock); }

// The whole merge in one launch (out of place).  A CTA owns a kFuseTile^2
// tile of layer 0 and, at every coarser layer L, the pixels c whose corner
// c 2^L lies in that tile (each pixel of the pyramid has exactly one owner).
// Going coarse to fine it evaluates M_L on the pixels its finer layer samples
// (its own pixels plus a halo of about one pixel, recomputed by the
// neighbouring CTAs as well) into shared memory, and writes the pixels it
// owns; layer 0 goes straight to global memory.  Every value is the same
// expression as in k_merge_layer (up_combine), so both give the same bits.
constexpr int kFuseTile = 32;
constexpr int kFuseThreads = 256;
// Shared-memory pixels over layers 1..n-1: at most 18^2 + 10^2 + 6^2 + 4^2
// + 4^2 per further layer (the halo of each layer's range stays within one
// pixel of its owned range, which halves from layer to layer) <= 652 for 16 layers.
constexpr int kFuseSmem = 672;
// channel groups merged per pass (kFuseSmem x groups x 16 bytes <= 43 KB)
constexpr int kFuseGroups4 = 4, kFuseGroups1 = 16;

__device__ __forceinline__ int tap0(int j) { return j == 0 ? 0 : (j - 1) >> 1; }  // = up_tap(j).x0

template <int DV>
__global__ void __launch_bounds__(kFuseThreads) k_merge_fused(Layers ly, int G, const float *__restrict__ P,
                                                              float *__restrict__ M)
{
    using V = Vec<DV>;
    using T = typename V::T;
    constexpr int GC = DV == 4 ? kFuseGroups4 : kFuseGroups1;
    __shared__ T buf[kFuseSmem * GC];
    __shared__ int rx0[kMaxLayers], rx1[kMaxLayers], ry0[kMaxLayers], ry1[kMaxLayers], base[kMaxLayers + 1];
    __shared__ int fits;
    const int X0 = blockIdx.x * kFuseTile, Y0 = blockIdx.y * kFuseTile, n = ly.n;
    if (threadIdx.x == 0) {
        // needed ranges (inclusive), finest first: layer 0 is the owned tile; layer L
        // covers its owned pixels and the taps of layer L-1's range
        rx0[0] = X0;
        rx1[0] = min(X0 + kFuseTile, ly.w[0]) - 1;
        ry0[0] = Y0;
        ry1[0] = min(Y0 + kFuseTile, ly.h[0]) - 1;
        int total = 0;
        base[1] = 0;
        for (int L = 1; L < n; ++L) {
            const int s = 1 << L;
            // owned: c with c s in [X0, X0 + T)
            const int ox0 = (X0 + s - 1) / s, ox1 = min((X0 + kFuseTile - 1) / s, ly.w[L] - 1);
            const int oy0 = (Y0 + s - 1) / s, oy1 = min((Y0 + kFuseTile - 1) / s, ly.h[L] - 1);
            int x0 = ox0, x1 = ox1, y0 = oy0, y1 = oy1;
            if (rx0[L - 1] <= rx1[L - 1] && ry0[L - 1] <= ry1[L - 1]) {
                x0 = min(x0, tap0(rx0[L - 1]));
                x1 = max(x1, min(tap0(rx1[L - 1]) + 1, ly.w[L] - 1));
                y0 = min(y0, tap0(ry0[L - 1]));
                y1 = max(y1, min(tap0(ry1[L - 1]) + 1, ly.h[L] - 1));
            }
            rx0[L] = x0; rx1[L] = x1; ry0[L] = y0; ry1[L] = y1;
            const int area = (x1 >= x0 && y1 >= y0) ? (x1 - x0 + 1) * (y1 - y0 + 1) : 0;
            total += area;
            base[L + 1] = total;
        }
        fits = total <= kFuseSmem;
    }
    __syncthreads();
    if (!fits) return;  // cannot happen for tiles of 32 (see kFuseSmem); never index past buf
    for (int g0 = 0; g0 < G; g0 += GC) {
        const int gc = min(GC, G - g0);  // channel groups of this pass, consecutive in memory
        for (int L = n - 1; L >= 0; --L) {
            const int w = rx1[L] - rx0[L] + 1, h = ry1[L] - ry0[L] + 1;
            if (w > 0 && h > 0) {
                const int s = 1 << L;
                const long long off = ly.off[L];
                for (int q = threadIdx.x; q < w * h * gc; q += blockDim.x) {
                    const int pq = q / gc, gg = q - pq * gc;
                    const int x = rx0[L] + pq % w, y = ry0[L] + pq / w;
                    const long long idx = (off + (long long)y * ly.w[L] + x) * G + g0 + gg;
                    T v = reinterpret_cast<const T *>(P)[idx];
                    if (L + 1 < n) {
                        const int Wc = ly.w[L + 1], Hc = ly.h[L + 1];
                        const Tap tx = up_tap(x, Wc), ty = up_tap(y, Hc);
                        const int cw = rx1[L + 1] - rx0[L + 1] + 1;
                        const T *C = buf + base[L + 1] * gc + gg;
                        const int ax0 = tx.x0 - rx0[L + 1], ax1 = tx.x1 - rx0[L + 1];
                        const int ay0 = ty.x0 - ry0[L + 1], ay1 = ty.x1 - ry0[L + 1];
                        v = up_combine<DV>(v, C[(ay0 * cw + ax0) * gc], C[(ay0 * cw + ax1) * gc],
                                           C[(ay1 * cw + ax0) * gc], C[(ay1 * cw + ax1) * gc], tx, ty);
                    }
                    if (L > 0) buf[base[L] * gc + q] = v;
                    const bool own = x * s >= X0 && x * s < X0 + kFuseTile && y * s >= Y0 && y * s < Y0 + kFuseTile;
                    if (own) reinterpret_cast<T *>(M)[idx] = v;
                }
            }
            __syncthreads();
        }
    }
}

bool vec4_ok(int D, const void *a, const void *b)
{
    return D % 4 == 0 && ((uintptr_t)a & 15u) == 0 && ((uintptr_t)b & 15u) == 0;
}

}  // namespace

}  // namespace tpk

extern "C" {

tp_status tp_merge(const tp_camera *cam, int32_t n_layers, int32_t D, const float *pyramid, float *merged,
                   tp_stream_t stream)
{
    tpk::Layers ly;
    if (!tpk::layers_of(cam, n_layers, ly) || D < 1 || D > tpk::kMaxMergeD || !pyramid || !merged)
        return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool v4 = tpk::vec4_ok(D, pyramid, merged);
    const int G = v4 ? D / 4 : D;
    // Out of place and up to 2^23 pyramid values in layer 0 (about 1080p at D = 4), one launch:
    // there the per-layer launches are launch-bound on the coarse layers.  Larger frames run the
    // per-layer kernels, which stream them better (measured: 1080p D = 4 0.037 vs 0.046 ms;
    // 4K D = 16 0.35 vs 0.30 ms).  Both give the same bits.  In place, the halos of other
    // CTAs could already be merged, so the per-layer kernels run.
    if (merged != pyramid && (long long)ly.w[0] * ly.h[0] * D <= (1ll << 23)) {
        const dim3 grid((unsigned)((ly.w[0] + tpk::kFuseTile - 1) / tpk::kFuseTile),
                        (unsigned)((ly.h[0] + tpk::kFuseTile - 1) / tpk::kFuseTile));
        if (v4)
            tpk::k_merge_fused<4><<<grid, tpk::kFuseThreads, 0, s>>>(ly, G, pyramid, merged);
        else
            tpk::k_merge_fused<1><<<grid, tpk::kFuseThreads, 0, s>>>(ly, G, pyramid, merged);
        return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
    }
    for (int L = n_layers - 1; L >= 0; --L) {
        const long long o = ly.off[L];
        const float *coarse = L + 1 < n_layers ? merged + ly.off[L + 1] * D : nullptr;
        const int Wc = L + 1 < n_layers ? ly.w[L + 1] : 1, Hc = L + 1 < n_layers ? ly.h[L + 1] : 1;
        const long long work = (long long)ly.w[L] * ly.h[L] * G;
        if (v4)
            tpk::k_merge_layer<4><<<tpk::blocks_for(work), tpk::kMergeBlock, 0, s>>>(
                ly.w[L], ly.h[L], Wc, Hc, G, pyramid + o * D, coarse, merged + o * D);
        else
            tpk::k_merge_layer<1><<<tpk::blocks_for(work), tpk::kMergeBlock, 0, s>>>(
                ly.w[L], ly.h[L], Wc, Hc, G, pyramid + o * D, coarse, merged + o * D);
        if (cudaGetLastError() != cudaSuccess) return TP_ERR_CUDA;
    }
    return TP_OK;
}

tp_status tp_merge_backward(const tp_camera *cam, int32_t n_layers, int32_t D, const float *grad_image,
                            float *grad_pyramid, tp_stream_t stream)
{
    tpk::Layers ly;
    if (!tpk::layers_of(cam, n_layers, ly) || D < 1 || D > tpk::kMaxMergeD || !grad_image || !grad_pyramid)
        return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (grad_image != grad_pyramid &&
        cudaMemcpyAsync(grad_pyramid, grad_image, (size_t)ly.off[1] * D * sizeof(float), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return TP_ERR_CUDA;
    const bool v4 = tpk::vec4_ok(D, grad_image, grad_pyramid);
    const int G = v4 ? D / 4 : D;
    for (int L = 1; L < n_layers; ++L) {
        const long long work = (long long)ly.w[L] * ly.h[L] * G;
        if (v4)
            tpk::k_merge_adjoint_layer<4><<<tpk::blocks_for(work), tpk::kMergeBlock, 0, s>>>(
                ly.w[L - 1], ly.h[L - 1], ly.w[L], ly.h[L], G, grad_pyramid + ly.off[L - 1] * D,
                grad_pyramid + ly.off[L] * D);
        else
            tpk::k_merge_adjoint_layer<1><<<tpk::blocks_for(work), tpk::kMergeBlock, 0, s>>>(
                ly.w[L - 1], ly.h[L - 1], ly.w[L], ly.h[L], G, grad_pyramid + ly.off[L - 1] * D,
                grad_pyramid + ly.off[L] * D);
        if (cudaGetLastError() != cudaSuccess) return TP_ERR_CUDA;
    }
    return TP_OK;
}

}  // extern "C"
