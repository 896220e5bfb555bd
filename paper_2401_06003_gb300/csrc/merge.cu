// merge.cu -- the pyramid merge of the decoder, without weights (TRIPS Sec. 3.3).
//
// The paper's network upsamples every layer but the finest bilinearly and
// merges it with the next finer layer, down to one full-resolution image.
// Without trained weights the merge is a sum:
//   M_{n-1} = P_{n-1},   M_L = P_L + up2(M_{L+1}),
// where up2 samples layer L+1 at the centres of layer L's pixels: pixel j of
// layer L sits at (j + 0.5) 2^L, at r = (j + 0.5)/2 - 0.5 >= 0 (clamped) in
// layer L+1 units, with taps floor(r) and min(floor(r) + 1, W_{L+1} - 1).
// All weights are multiples of 1/4, exact in float32.  One launch per layer,
// coarse to fine; the adjoint runs fine to coarse:
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
        return make_float4(acc.x + w * a.x, acc.y + w * a.y, acc.z + w * a.z, acc.w + w * a.w);
    }
    static __device__ __forceinline__ float4 add(float4 a, float4 b)
    {
        return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
};
template <>
struct Vec<1> {
    using T = float;
    static __device__ __forceinline__ float zero() { return 0.f; }
    static __device__ __forceinline__ float fma(float w, float a, float acc) { return acc + w * a; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
};

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
        T top = V::fma(tx.lam, c01, V::fma(1.0f - tx.lam, c00, V::zero()));
        T bot = V::fma(tx.lam, c11, V::fma(1.0f - tx.lam, c10, V::zero()));
        v = V::add(v, V::fma(ty.lam, bot, V::fma(1.0f - ty.lam, top, V::zero())));
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
