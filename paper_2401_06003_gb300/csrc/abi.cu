// abi.cu -- the extern "C" entry points declared in include/trips.h.
//
// Host-side argument checks, the frame description of every view (pyramid
// layout and screen-tile table), the workspace layout, and the kernel
// launches.  A single view is a batch of one.  No call allocates, frees or
// synchronises, except tp_get_status.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace {

using tpk::Batch;
using tpk::Frame;
using tpk::kMaxViews;
using tpk::Workspace;

constexpr int64_t kAlign = 256;
constexpr int64_t kMaxPoints = (int64_t)1 << 27;
constexpr size_t kMaxTileSmem = 200 * 1024;

int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool valid_camera(const tp_camera *cam)
{
    if (!cam) return false;
    if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768) return false;
    const float *f = &cam->fx;
    for (int q = 0; q < 17; ++q)
        if (!std::isfinite(f[q])) return false;
    if (!(cam->znear > 0.0f)) return false;
    if (cam->fx == 0.0f || cam->fy == 0.0f) return false;
    return true;
}

void fill_layers(const tp_camera *cam, int n_layers, Frame &F)
{
    F.pix_base[0] = 0;
    for (int L = 0; L < n_layers; ++L) {
        const int64_t s = (int64_t)1 << L;
        F.lw[L] = (int)((cam->width + s - 1) / s);
        F.lh[L] = (int)((cam->height + s - 1) / s);
        F.pix_base[L + 1] = F.pix_base[L] + (long long)F.lw[L] * F.lh[L];
    }
}

tp_status check_config(const tp_config *cfg)
{
    if (!cfg) return TP_ERR_INVALID_ARG;
    if (cfg->n_layers < 1 || cfg->n_layers > tpk::kMaxLayers) return TP_ERR_INVALID_ARG;
    if (cfg->desc_dim < 1 || cfg->desc_dim > 64) return TP_ERR_INVALID_ARG;
    if (!(cfg->eps >= 0.0f && cfg->eps <= 1.0f)) return TP_ERR_INVALID_ARG;
    if (cfg->desc_dtype != TP_F32 && cfg->desc_dtype != TP_BF16) return TP_ERR_INVALID_ARG;
    if (cfg->mode != TP_STORE_LISTS && cfg->mode != TP_RECOMPUTE) return TP_ERR_INVALID_ARG;
    if (cfg->K < 1 || cfg->K > 255) return TP_ERR_INVALID_ARG;
    if (cfg->K != 4 && cfg->K != 8 && cfg->K != 16 && cfg->K != 32) return TP_ERR_UNSUPPORTED;
    if (cfg->tile_w < 0 || cfg->tile_h < 0) return TP_ERR_INVALID_ARG;
    if ((cfg->flags & ~(TP_COARSE_LAYERS | TP_GRADS_ZEROED)) != 0) return TP_ERR_INVALID_ARG;
    return TP_OK;
}

// The frame description of one view with screen tiles of tw x th pixels
// (0 = the default 16 x 8).
tp_status make_frame(const tp_config *cfg, const tp_camera *cam, int tw, int th, Frame &F)
{
    tp_status st = check_config(cfg);
    if (st != TP_OK) return st;
    if (!valid_camera(cam)) return TP_ERR_INVALID_ARG;
    if (tw == 0) tw = 16;
    if (th == 0) th = 8;
    if (tw < 0 || th < 0 || tw > 64 || th > 64) return TP_ERR_INVALID_ARG;
    if (tw * th > 1024) return TP_ERR_UNSUPPORTED;  // one thread per tile pixel
    std::memset(&F, 0, sizeof(F));
    F.fx = cam->fx; F.fy = cam->fy; F.cx = cam->cx; F.cy = cam->cy;
    std::memcpy(F.R, cam->R, sizeof(F.R));
    std::memcpy(F.t, cam->t, sizeof(F.t));
    F.znear = cam->znear;
    F.eps = cfg->eps;
    F.n_layers = cfg->n_layers;
    F.K = cfg->K;
    F.D = cfg->desc_dim;
    F.tile_w = tw;
    F.tile_h = th;
    F.coarse = (cfg->flags & TP_COARSE_LAYERS) ? 1 : 0;
    F.grads_zeroed = (cfg->flags & TP_GRADS_ZEROED) ? 1 : 0;
    fill_layers(cam, cfg->n_layers, F);
    int tiles = 0;
    for (int L = 0; L < F.n_layers; ++L) {
        F.tile_base[L] = tiles;
        F.tiles_x[L] = (F.lw[L] + tw - 1) / tw;
        F.tiles_y[L] = (F.lh[L] + th - 1) / th;
        const int64_t t = (int64_t)tiles + (int64_t)F.tiles_x[L] * F.tiles_y[L];
        if (t > (1 << 28)) return TP_ERR_INVALID_ARG;
        tiles = (int)t;
    }
    F.tile_base[F.n_layers] = tiles;
    F.n_tiles = tiles;
    // Tile CTAs: one thread per pixel, kept lists in registers; shared memory
    // holds one chunk of tile-list entries' fragment keys (8 bytes each, at
    // most four per entry: 32 bytes per chunk entry), sized to about 34 KB per
    // CTA (six 128-thread CTAs per SM), or 28 KB for wide descriptors, whose
    // gathers gain more from the L1 that the smaller carve-out leaves.
    F.tile_px = tw * th;
    F.tile_threads = (F.tile_px + 31) / 32 * 32;
    const int64_t budget = (cfg->desc_dim > 8 ? 28 : 34) * 1024;
    const int64_t avail = budget - (3 * F.tile_threads + 32) * 4;
    int64_t chunk = avail / 32;
    if (chunk < 128) chunk = 128;
    if (chunk > 2048) chunk = 2048;
    F.chunk = (int)((chunk + 15) / 16 * 16);
    if (tpk::tile_smem_bytes(F, true) > kMaxTileSmem) return TP_ERR_UNSUPPORTED;
    return TP_OK;
}

// The batch description of n_views views; tiles is [n_views][2] tile shapes
// or NULL (the config's tile shape for every view).
template <int MaxV>
tp_status make_batch(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, Batch<MaxV> &B)
{
    if (!cfg || !cams || n_views < 1 || n_views > MaxV) return TP_ERR_INVALID_ARG;
    std::memset(&B, 0, sizeof(B));
    B.n_views = n_views;
    for (int v = 0; v < n_views; ++v) {
        const int tw = tiles ? tiles[2 * v] : cfg->tile_w;
        const int th = tiles ? tiles[2 * v + 1] : cfg->tile_h;
        tp_status st = make_frame(cfg, cams + v, tw, th, B.view[v]);
        if (st != TP_OK) return st;
        const Frame &F = B.view[v];
        B.tile_base[v + 1] = B.tile_base[v] + F.n_tiles;
        B.pix_base[v + 1] = B.pix_base[v] + F.pix_base[F.n_layers];
        B.cpix_base[v + 1] = B.cpix_base[v] + (F.pix_base[F.n_layers] - F.pix_base[1]);
        if (F.tile_threads > B.max_threads) B.max_threads = F.tile_threads;
        if ((int64_t)B.tile_base[v + 1] > ((int64_t)1 << 28)) return TP_ERR_INVALID_ARG;
    }
    B.n_tiles = B.tile_base[n_views];
    B.n_pix = B.pix_base[n_views];
    // the launch's block is the largest tile CTA; every view's region must fit with it
    for (int v = 0; v < n_views; ++v) {
        Frame G = B.view[v];
        G.tile_threads = B.max_threads;
        if (tpk::tile_smem_bytes(G, true) > kMaxTileSmem) return TP_ERR_UNSUPPORTED;
    }
    return TP_OK;
}

// Workspace: status word, tile counts [T][copies], tile offsets [T + 1],
// fill cursors [T][copies], the per-pixel largest kept keys [P], with
// coarse-layer inclusion the kept lists of the coarse pixels ([K][rows] keys,
// then [K][rows] opacities), then the tile lists as two arrays: 8-byte
// fragment keys and 16-byte payloads.
constexpr int64_t kEntryBytes = 24;

struct WsLayout {
    int64_t count, off, cursor, kmax, ckey, cgam, key, pay, end;
};

// cslots: K x coarse pixels with coarse-layer inclusion, else 0.
WsLayout layout_for(int64_t n_tiles, int64_t n_pix, int64_t cslots, int64_t capacity)
{
    WsLayout w;
    w.count = kAlign;
    w.off = align_up(w.count + 4 * n_tiles * tpk::kCopies);
    w.cursor = align_up(w.off + 4 * (n_tiles + 1));
    w.kmax = align_up(w.cursor + 4 * n_tiles * tpk::kCopies);
    w.ckey = align_up(w.kmax + 8 * n_pix);
    w.cgam = align_up(w.ckey + 8 * cslots);
    w.key = align_up(w.cgam + 4 * cslots);
    w.pay = align_up(w.key + 8 * capacity);
    w.end = w.pay + 16 * capacity;
    return w;
}

// Entry capacity that fits in ws_bytes (largest c with layout_for(c).end <= ws_bytes).
int64_t capacity_for(int64_t n_tiles, int64_t n_pix, int64_t cslots, int64_t ws_bytes)
{
    const WsLayout w0 = layout_for(n_tiles, n_pix, cslots, 0);
    if (ws_bytes < w0.end) return -1;
    // align_up only adds bytes, so (ws_bytes - key) / 24 is an upper bound;
    // alignment costs < 256 bytes, so the loop runs at most ~11 times.
    int64_t c = (ws_bytes - w0.key) / kEntryBytes;
    if (c < 0) c = 0;
    while (c > 0 && layout_for(n_tiles, n_pix, cslots, c).end > ws_bytes) --c;
    if (c > 0x7FFFFFFF) c = 0x7FFFFFFF;
    return c;
}

// K x coarse pixels of the batch with coarse-layer inclusion, else 0.
template <int MaxV>
int64_t coarse_slots(const tp_config *cfg, const Batch<MaxV> &B)
{
    return (cfg->flags & TP_COARSE_LAYERS) ? (int64_t)cfg->K * B.cpix_base[B.n_views] : 0;
}

template <int MaxV>
tp_status bind_workspace(const tp_config *cfg, const Batch<MaxV> &B, void *ws, int64_t ws_bytes, Workspace &W)
{
    if (!ws || ((uintptr_t)ws % kAlign) != 0) return TP_ERR_INVALID_ARG;
    const int64_t cslots = coarse_slots(cfg, B);
    const int64_t cap = capacity_for(B.n_tiles, B.n_pix, cslots, ws_bytes);
    if (cap < 1) return TP_ERR_INVALID_ARG;
    const WsLayout w = layout_for(B.n_tiles, B.n_pix, cslots, cap);
    char *base = static_cast<char *>(ws);
    W.status = reinterpret_cast<unsigned *>(base);
    W.tile_count = reinterpret_cast<unsigned *>(base + w.count);
    W.tile_off = reinterpret_cast<unsigned *>(base + w.off);
    W.tile_cursor = reinterpret_cast<unsigned *>(base + w.cursor);
    W.kmax = reinterpret_cast<unsigned long long *>(base + w.kmax);
    W.ckey = cslots ? reinterpret_cast<unsigned long long *>(base + w.ckey) : nullptr;
    W.cgam = cslots ? reinterpret_cast<unsigned *>(base + w.cgam) : nullptr;
    W.crows = B.cpix_base[B.n_views];
    W.bucket_key = reinterpret_cast<unsigned long long *>(base + w.key);
    W.bucket_pay = reinterpret_cast<float4 *>(base + w.pay);
    W.capacity = (unsigned)cap;
    return TP_OK;
}

template <int MaxV>
tp_status batch_checks(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, int64_t n,
                       void *ws, int64_t ws_bytes, Batch<MaxV> &B, Workspace &W)
{
    if (n < 0 || n >= kMaxPoints) return TP_ERR_INVALID_ARG;
    // a point makes at most 8 (point, tile) entries per view; the tile offsets are 32-bit
    if (n * (int64_t)(n_views > 0 ? n_views : 1) * 8 >= ((int64_t)1 << 32)) return TP_ERR_INVALID_ARG;
    tp_status s = make_batch(cfg, cams, tiles, n_views, B);
    if (s != TP_OK) return s;
    s = bind_workspace(cfg, B, ws, ws_bytes, W);
    W.n_points = n;
    return s;
}

tp_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return TP_OK;
    if (e == cudaErrorInvalidConfiguration) return TP_ERR_UNSUPPORTED;  // tile too large for the kernel
    return TP_ERR_CUDA;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Descriptors can be read 16 bytes at a time (4 float32 or 8 bfloat16
// channels) when D is a multiple of that group and the rows are 16-byte aligned.
int desc_vector_ok(const tp_config *cfg, const void *desc)
{
    const int group = cfg->desc_dtype == TP_BF16 ? 8 : 4;
    return (cfg->desc_dim % group) == 0 && ((uintptr_t)desc % 16) == 0;
}

template <int MaxV>
void set_vec_flags(Batch<MaxV> &B, int desc_vec, int grad_vec)
{
    for (int v = 0; v < B.n_views; ++v) {
        B.view[v].desc_vec = desc_vec;
        B.view[v].grad_vec = grad_vec;
    }
}

// ---------------------------------------------------------------------------
// The four stages over a batch of views.
// ---------------------------------------------------------------------------

template <int MaxV>
tp_status do_project(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, int64_t n,
                     const float *pos, const float *size_w, float *records, void *ws, int64_t ws_bytes,
                     tp_stream_t stream)
{
    Batch<MaxV> B;
    Workspace W;
    tp_status s = batch_checks(cfg, cams, tiles, n_views, n, ws, ws_bytes, B, W);
    if (s != TP_OK) return s;
    if (n > 0 && (!pos || !size_w || !records || !aligned16(records))) return TP_ERR_INVALID_ARG;
    return from_cuda(tpk::launch_project_count(B, W, n, pos, size_w, reinterpret_cast<float4 *>(records),
                                               (cudaStream_t)stream));
}

template <int MaxV>
tp_status do_splat_forward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, int64_t n,
                           const float *records, const float *opacity, void *ws, int64_t ws_bytes,
                           tp_stream_t stream)
{
    Batch<MaxV> B;
    Workspace W;
    tp_status s = batch_checks(cfg, cams, tiles, n_views, n, ws, ws_bytes, B, W);
    if (s != TP_OK) return s;
    if (n > 0 && (!records || !opacity || !aligned16(records))) return TP_ERR_INVALID_ARG;
    return from_cuda(tpk::launch_scan_fill(B, W, n, reinterpret_cast<const float4 *>(records), opacity,
                                           (cudaStream_t)stream));
}

template <int MaxV>
tp_status do_blend(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, int64_t n,
                   const float *records, const float *opacity, const void *desc, float *pyramid, uint32_t *kept,
                   uint8_t *n_kept, float *t_final, uint32_t *n_frag, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    Batch<MaxV> B;
    Workspace W;
    tp_status s = batch_checks(cfg, cams, tiles, n_views, n, ws, ws_bytes, B, W);
    if (s != TP_OK) return s;
    if (!pyramid) return TP_ERR_INVALID_ARG;
    if (n > 0 && (!desc || !records || !opacity || !aligned16(records))) return TP_ERR_INVALID_ARG;
    W.rec = reinterpret_cast<const float4 *>(records);
    W.opacity = opacity;
    set_vec_flags(B, desc_vector_ok(cfg, desc) && aligned16(pyramid), 0);
    return from_cuda(tpk::launch_blend(B, W, desc, cfg->desc_dtype, pyramid, kept, n_kept, t_final, n_frag,
                                       (cudaStream_t)stream));
}

template <int MaxV>
tp_status do_backward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views, int64_t n,
                      const float *records, const float *opacity, const void *desc, const uint32_t *kept,
                      const uint8_t *n_kept, const float *grad_pyramid, float *grad_pos, float *grad_size_w,
                      float *grad_opacity, float *grad_desc, void *ws, int64_t ws_bytes, tp_stream_t stream,
                      const float *pos = nullptr, double *grad_cameras = nullptr)
{
    Batch<MaxV> B;
    Workspace W;
    tp_status s = batch_checks(cfg, cams, tiles, n_views, n, ws, ws_bytes, B, W);
    if (s != TP_OK) return s;
    if ((kept == nullptr) != (n_kept == nullptr)) return TP_ERR_INVALID_ARG;
    if (grad_cameras && (kept || (n > 0 && !pos))) return TP_ERR_INVALID_ARG;
    if (kept && (cfg->flags & TP_COARSE_LAYERS)) return TP_ERR_UNSUPPORTED;
    if (!grad_pyramid) return TP_ERR_INVALID_ARG;
    // grad_size_w NULL: grad_pos holds packed [n][4] rows (X, Y, Z, s_w), 16-byte aligned
    const bool pos4 = grad_size_w == nullptr;
    if (n > 0 && (!records || !opacity || !desc || !grad_pos || !grad_opacity || !grad_desc ||
                  !aligned16(records) || (pos4 && !aligned16(grad_pos))))
        return TP_ERR_INVALID_ARG;
    set_vec_flags(B, desc_vector_ok(cfg, desc), (cfg->desc_dim % 4) == 0 && aligned16(grad_desc));
    for (int v = 0; v < B.n_views; ++v) B.view[v].pos4 = pos4 ? 1 : 0;
    return from_cuda(tpk::launch_backward(B, W, n, reinterpret_cast<const float4 *>(records), opacity, desc,
                                          cfg->desc_dtype, kept, n_kept, grad_pyramid, grad_pos, grad_size_w,
                                          grad_opacity, grad_desc, pos, grad_cameras, (cudaStream_t)stream));
}

template <int MaxV>
int64_t batch_workspace_bytes(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int n_views,
                              int64_t n_points, int64_t entry_capacity)
{
    Batch<MaxV> B;
    if (n_points < 0 || n_points >= kMaxPoints) return -1;
    if (n_points * (int64_t)(n_views > 0 ? n_views : 1) * 8 >= ((int64_t)1 << 32)) return -1;
    if (make_batch(cfg, cams, tiles, n_views, B) != TP_OK) return -1;
    int64_t cap = entry_capacity > 0 ? entry_capacity : 8 * n_points * n_views;
    if (cap < 1) cap = 1;
    if (cap > 0x7FFFFFFF) cap = 0x7FFFFFFF;
    return layout_for(B.n_tiles, B.n_pix, coarse_slots(cfg, B), cap).end;
}

}  // namespace

extern "C" {

int64_t tp_pyramid_pixels(const tp_camera *cam, int32_t n_layers, int64_t *layer_offsets)
{
    if (!valid_camera(cam) || n_layers < 1 || n_layers > tpk::kMaxLayers) return -1;
    Frame F;
    std::memset(&F, 0, sizeof(F));
    fill_layers(cam, n_layers, F);
    if (layer_offsets)
        for (int L = 0; L <= n_layers; ++L) layer_offsets[L] = F.pix_base[L];
    return F.pix_base[n_layers];
}

int64_t tp_workspace_bytes(const tp_config *cfg, const tp_camera *cam, int64_t n_points, int64_t entry_capacity)
{
    return batch_workspace_bytes<1>(cfg, cam, nullptr, 1, n_points, entry_capacity);
}

tp_status tp_project(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *pos, const float *size_w,
                     float *records, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    return do_project<1>(cfg, cam, nullptr, 1, n, pos, size_w, records, ws, ws_bytes, stream);
}

tp_status tp_splat_forward(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records,
                           const float *opacity, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    return do_splat_forward<1>(cfg, cam, nullptr, 1, n, records, opacity, ws, ws_bytes, stream);
}

tp_status tp_blend(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records, const float *opacity,
                   const void *desc, float *pyramid, uint32_t *kept, uint8_t *n_kept, float *t_final,
                   uint32_t *n_frag, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    return do_blend<1>(cfg, cam, nullptr, 1, n, records, opacity, desc, pyramid, kept, n_kept, t_final, n_frag, ws,
                       ws_bytes, stream);
}

tp_status tp_splat_backward(const tp_config *cfg, const tp_camera *cam, int64_t n, const float *records,
                            const float *opacity, const void *desc, const uint32_t *kept, const uint8_t *n_kept,
                            const float *grad_pyramid, float *grad_pos, float *grad_size_w, float *grad_opacity,
                            float *grad_desc, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    return do_backward<1>(cfg, cam, nullptr, 1, n, records, opacity, desc, kept, n_kept, grad_pyramid, grad_pos,
                          grad_size_w, grad_opacity, grad_desc, ws, ws_bytes, stream);
}

int64_t tp_batch_pixels(const tp_camera *cams, int32_t n_views, int32_t n_layers, int64_t *view_offsets)
{
    if (!cams || n_views < 1 || n_views > kMaxViews) return -1;
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        const int64_t p = tp_pyramid_pixels(cams + v, n_layers, nullptr);
        if (p < 0) return -1;
        if (view_offsets) view_offsets[v] = total;
        total += p;
    }
    if (view_offsets) view_offsets[n_views] = total;
    return total;
}

int64_t tp_batch_workspace_bytes(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                                 int64_t n_points, int64_t entry_capacity)
{
    return batch_workspace_bytes<kMaxViews>(cfg, cams, tiles, n_views, n_points, entry_capacity);
}

tp_status tp_batch_project(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                           int64_t n, const float *pos, const float *size_w, float *records, void *ws,
                           int64_t ws_bytes, tp_stream_t stream)
{
    return do_project<kMaxViews>(cfg, cams, tiles, n_views, n, pos, size_w, records, ws, ws_bytes, stream);
}

tp_status tp_batch_splat_forward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                                 int64_t n, const float *records, const float *opacity, void *ws, int64_t ws_bytes,
                                 tp_stream_t stream)
{
    return do_splat_forward<kMaxViews>(cfg, cams, tiles, n_views, n, records, opacity, ws, ws_bytes, stream);
}

tp_status tp_batch_blend(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles, int32_t n_views,
                         int64_t n, const float *records, const float *opacity, const void *desc, float *pyramid,
                         uint32_t *kept, uint8_t *n_kept, float *t_final, uint32_t *n_frag, void *ws,
                         int64_t ws_bytes, tp_stream_t stream)
{
    return do_blend<kMaxViews>(cfg, cams, tiles, n_views, n, records, opacity, desc, pyramid, kept, n_kept, t_final,
                               n_frag, ws, ws_bytes, stream);
}

tp_status tp_batch_splat_backward(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                  int32_t n_views, int64_t n, const float *records, const float *opacity,
                                  const void *desc, const uint32_t *kept, const uint8_t *n_kept,
                                  const float *grad_pyramid, float *grad_pos, float *grad_size_w,
                                  float *grad_opacity, float *grad_desc, void *ws, int64_t ws_bytes,
                                  tp_stream_t stream)
{
    return do_backward<kMaxViews>(cfg, cams, tiles, n_views, n, records, opacity, desc, kept, n_kept, grad_pyramid,
                                  grad_pos, grad_size_w, grad_opacity, grad_desc, ws, ws_bytes, stream);
}

tp_status tp_batch_splat_backward_cameras(const tp_config *cfg, const tp_camera *cams, const int32_t *tiles,
                                          int32_t n_views, int64_t n, const float *pos, const float *records,
                                          const float *opacity, const void *desc, const float *grad_pyramid,
                                          float *grad_pos, float *grad_size_w, float *grad_opacity, float *grad_desc,
                                          double *grad_cameras, void *ws, int64_t ws_bytes, tp_stream_t stream)
{
    if (!grad_cameras) return TP_ERR_INVALID_ARG;
    return do_backward<kMaxViews>(cfg, cams, tiles, n_views, n, records, opacity, desc, nullptr, nullptr,
                                  grad_pyramid, grad_pos, grad_size_w, grad_opacity, grad_desc, ws, ws_bytes, stream,
                                  pos, grad_cameras);
}

tp_status tp_zero_gradients(const tp_config *cfg, int64_t n, float *grad_pos, float *grad_size_w,
                            float *grad_opacity, float *grad_desc, tp_stream_t stream)
{
    if (check_config(cfg) != TP_OK || n < 0 || n >= kMaxPoints) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!grad_pos || !grad_opacity || !grad_desc) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool pos4 = grad_size_w == nullptr;
    const size_t N = (size_t)n;
    if (cudaMemsetAsync(grad_pos, 0, sizeof(float) * (pos4 ? 4 : 3) * N, s) != cudaSuccess) return TP_ERR_CUDA;
    if (!pos4 && cudaMemsetAsync(grad_size_w, 0, sizeof(float) * N, s) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaMemsetAsync(grad_opacity, 0, sizeof(float) * N, s) != cudaSuccess) return TP_ERR_CUDA;
    if (cudaMemsetAsync(grad_desc, 0, sizeof(float) * (size_t)cfg->desc_dim * N, s) != cudaSuccess)
        return TP_ERR_CUDA;
    return TP_OK;
}

tp_status tp_get_status(const void *ws, tp_stream_t stream, int32_t *device_flags)
{
    if (!ws || !device_flags) return TP_ERR_INVALID_ARG;
    unsigned flags = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&flags, ws, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return TP_ERR_CUDA;
    *device_flags = (int32_t)flags;
    if (flags & TP_FLAG_CAPACITY) return TP_ERR_CAPACITY;
    if (flags & TP_FLAG_BOUNDS) return TP_ERR_BOUNDS;
    if (flags & TP_FLAG_TIMEOUT) return TP_ERR_TIMEOUT;
    if (flags & TP_FLAG_NONFINITE) return TP_ERR_NONFINITE;
    return TP_OK;
}

const char *tp_status_string(tp_status status)
{
    switch (status) {
    case TP_OK: return "ok";
    case TP_ERR_INVALID_ARG: return "invalid argument";
    case TP_ERR_CAPACITY: return "workspace entry capacity exceeded";
    case TP_ERR_NONFINITE: return "non-finite point input (point culled)";
    case TP_ERR_TIMEOUT: return "bounded device wait timed out";
    case TP_ERR_CUDA: return "CUDA error";
    case TP_ERR_UNSUPPORTED: return "unsupported configuration";
    case TP_ERR_BOUNDS: return "out-of-range index caught by the checking build";
    }
    return "unknown status";
}

int32_t tp_version(void) { return 130; }

}  // extern "C"
