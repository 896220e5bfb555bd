// camera.cu -- adjoint of the camera: intrinsics and pose (TRIPS Sec. 3.5).
//
// The paper optimises the cameras along with the points.  The camera enters
// the render only through each point's screen position and size (Eq. 2):
//   X_c = R X_w + t,  x = fx X_c/Z_c + cx,  y = fy Y_c/Z_c + cy,  s = fx s_w/Z_c.
// The backward kernels already reduce every fragment's screen-space gradient
// into the point gradients
//   dL/dX_w = R^T dL/dX_c,   dL/ds_w = (fx/Z_c) sum_frag dL/ds,
// with dL/dX_c = (fx/Z_c Gx, fy/Z_c Gy, -((x-cx) Gx + (y-cy) Gy + s Gs)/Z_c)
// and Gx, Gy, Gs the per-point sums of dL/dx, dL/dy, dL/ds.  So one pass over
// the points recovers dL/dX_c = (R^T)^-1 dL/dX_w, Gx, Gy and Gs, and sums
//   dL/dfx = Gx (x-cx)/fx + Gs s/fx,   dL/dfy = Gy (y-cy)/fy,
//   dL/dcx = Gx,   dL/dcy = Gy,   dL/dt = dL/dX_c,   dL/dR = dL/dX_c X_w^T
// over the visible points, without touching the per-fragment kernels.
#include "common.cuh"

namespace tpk {

namespace {

struct CamArgs {
    float cx, cy, ifx, ify;  // principal point, 1/fx, 1/fy
    float M[9];              // (R^T)^-1, row-major: dL/dX_c = M dL/dX_w
};

constexpr int kCamBlock = 256;
constexpr int kCamOut = 16;  // fx, fy, cx, cy, R[9], t[3]

// gpos rows are ps floats apart (3, or 4 for packed rows whose fourth float
// is dL/ds_w); gsw entries are ss floats apart.
__global__ void __launch_bounds__(kCamBlock) k_camera_grad(CamArgs A, long long n, const float *__restrict__ pos,
                                                           const float4 *__restrict__ rec,
                                                           const float *__restrict__ gpos,
                                                           const float *__restrict__ gsw, int ps, int ss,
                                                           double *__restrict__ out)
{
    float acc[kCamOut];
#pragma unroll
    for (int q = 0; q < kCamOut; ++q) acc[q] = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
#pragma unroll 2
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 r = rec[i];
        if (!(r.z > 0.0f)) continue;  // culled: the record is all zero
        const float g0 = gpos[ps * i], g1 = gpos[ps * i + 1], g2 = gpos[ps * i + 2];
        float dXc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dXc[a] = A.M[3 * a] * g0 + A.M[3 * a + 1] * g1 + A.M[3 * a + 2] * g2;
        const float Z = r.z;
        const float Gx = dXc[0] * Z * A.ifx, Gy = dXc[1] * Z * A.ify, Gs = gsw[ss * i] * Z * A.ifx;
        acc[0] += (Gx * (r.x - A.cx) + Gs * r.w) * A.ifx;
        acc[1] += Gy * (r.y - A.cy) * A.ify;
        acc[2] += Gx;
        acc[3] += Gy;
        const float X[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[4 + 3 * a + c] += dXc[a] * X[c];
            acc[13 + a] += dXc[a];
        }
    }
    __shared__ float part[kCamBlock / 32][kCamOut];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kCamOut; ++q) {
        float v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kCamOut) {
        double v = 0.0;
        for (int w = 0; w < kCamBlock / 32; ++w) v += (double)part[w][threadIdx.x];
        atomicAdd(out + threadIdx.x, v);
    }
}

}  // namespace

}  // namespace tpk

extern "C" {

tp_status tp_camera_backward(const tp_camera *cam, int64_t n, const float *pos, const float *records,
                             const float *grad_pos, const float *grad_size_w, double *grad_camera, tp_stream_t stream)
{
    if (!cam || !grad_camera || n < 0) return TP_ERR_INVALID_ARG;
    if (n > 0 && (!pos || !records || !grad_pos || ((uintptr_t)records & 15u) != 0)) return TP_ERR_INVALID_ARG;
    const bool pos4 = grad_size_w == nullptr;  // packed [n][4] rows (X, Y, Z, s_w)
    if (!(cam->fx != 0.0f) || !(cam->fy != 0.0f)) return TP_ERR_INVALID_ARG;
    // (R^T)^-1 = (R^-1)^T: the transposed cofactor matrix of R^T over det R
    const float *R = cam->R;
    double a[9];
    for (int q = 0; q < 9; ++q) a[q] = R[q];
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (!(det > 1e-12 || det < -1e-12)) return TP_ERR_INVALID_ARG;
    // cofactors of R; (R^-1)^T = cof(R) / det
    const double cof[9] = {c00,
                           c01,
                           c02,
                           a[2] * a[7] - a[1] * a[8],
                           a[0] * a[8] - a[2] * a[6],
                           a[1] * a[6] - a[0] * a[7],
                           a[1] * a[5] - a[2] * a[4],
                           a[2] * a[3] - a[0] * a[5],
                           a[0] * a[4] - a[1] * a[3]};
    tpk::CamArgs A;
    A.ifx = (float)(1.0 / (double)cam->fx);
    A.ify = (float)(1.0 / (double)cam->fy);
    A.cx = cam->cx;
    A.cy = cam->cy;
    for (int q = 0; q < 9; ++q) A.M[q] = (float)(cof[q] / det);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad_camera, 0, tpk::kCamOut * sizeof(double), s) != cudaSuccess) return TP_ERR_CUDA;
    if (n == 0) return TP_OK;
    long long blocks = (n + tpk::kCamBlock - 1) / tpk::kCamBlock;
    if (blocks > 152 * 16) blocks = 152 * 16;
    tpk::k_camera_grad<<<(int)blocks, tpk::kCamBlock, 0, s>>>(A, n, pos, reinterpret_cast<const float4 *>(records),
                                                              grad_pos, pos4 ? grad_pos + 3 : grad_size_w,
                                                              pos4 ? 4 : 3, pos4 ? 4 : 1, grad_camera);
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

}  // extern "C"
