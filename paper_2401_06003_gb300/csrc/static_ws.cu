// static_ws.cu -- a forward render whose workspace lives in a fixed device array.
//
// Some callers may not allocate device memory at run time: a plug-in inside a
// host application that owns every CUDA allocation through its own pool, or a
// real-time frame loop that must not call cudaMalloc (which can synchronise the
// whole device) once it runs.  tp_render_forward_static serves them: it
// enqueues the same kernels as tp_project + tp_splat_forward + tp_blend, but
// the frame's workspace is the array below instead of a caller buffer.
//
// The array belongs to the library's device image: every GPU that loads the
// library's module holds TP_STATIC_WORKSPACE_BYTES of it until the process
// exits.  With lazy module loading (the CUDA default) the module, and with it
// the array, is loaded and reserved by the first call on each device, which
// can therefore fail for lack of device memory (TP_ERR_CUDA): make that first
// call at start-up.  In host code the array's name only stands for the
// device symbol; the device address is looked up with cudaGetSymbolAddress
// once per device, by the first call made with that device current, and
// cached; a cudaDeviceReset of that device voids the cached address, and a
// later call looks it up again only if the lookup itself fails.  All calls on a device share the array, so calls
// that overlap on the GPU race; ordered calls do not, because each call resets
// what must start at zero and overwrites everything else it reads.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_workspace[TP_STATIC_WORKSPACE_BYTES];

std::mutex g_lock;
void *g_address[kMaxDevices];

// Device address of the array on the current device (looked up once per device).
tp_status static_workspace(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TP_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_address[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess || !p) return TP_ERR_CUDA;
        g_address[dev] = p;
    }
    *out = g_address[dev];
    return TP_OK;
}

}  // namespace

extern "C" {

tp_status tp_render_forward_static(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *pos,
                                   const float *size_w, const float *opacity, const void *desc, float *records,
                                   float *pyramid, uint32_t *device_flags, tp_stream_t stream)
{
    const int64_t need = tp_workspace_bytes(cfg, cam, n, 0);
    if (need < 0) return TP_ERR_INVALID_ARG;
    if (need > TP_STATIC_WORKSPACE_BYTES) return TP_ERR_CAPACITY;  // frame too large for the fixed array
    void *ws = nullptr;
    tp_status s = static_workspace(&ws);
    if (s != TP_OK) return s;
    // tp_project zeroes the status word and the tile counters; the scan, fill
    // and blend kernels write every other word they later read.
    s = tp_project(cfg, cam, n, pos, size_w, records, ws, need, stream);
    if (s != TP_OK) return s;
    s = tp_splat_forward(cfg, cam, n, records, opacity, ws, need, stream);
    if (s != TP_OK) return s;
    s = tp_blend(cfg, cam, n, records, opacity, desc, pyramid, nullptr, nullptr, nullptr, nullptr, ws, need, stream);
    if (s != TP_OK || !device_flags) return s;
    // The status word is the workspace's first 4 bytes.
    if (cudaMemcpyAsync(device_flags, ws, sizeof(uint32_t), cudaMemcpyDeviceToDevice, (cudaStream_t)stream) !=
        cudaSuccess)
        return TP_ERR_CUDA;
    return TP_OK;
}

}  // extern "C"
