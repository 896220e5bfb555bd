/*
 * trips_oracle.c -- plain, slow CPU oracle for differentiable trilinear point
 * splatting (TRIPS: Franke, Rueckert, Fink, Stamminger, Eurographics 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header or table with the CUDA
 * kernels: it is written from the paper's equations, in the paper's order.
 *
 * What it computes (paper references are sections / equations):
 *   - projection of each point to continuous screen coordinates (x, y, z) and
 *     screen size s = f * s_w / z                              (Sec. 3.1, Eq. 2)
 *   - the two pyramid layers floor(log2 s), floor(log2 s)+1    (Sec. 3.1)
 *   - the 2x2x2 trilinear weights gamma = beta * iota * alpha  (Eq. 3-5)
 *   - per (layer, pixel) fragment lists sorted by depth, clamped to K
 *                                                              (Sec. 3.2, Sec. 3.6)
 *   - front-to-back alpha blending C = sum_m T_m alpha_m c_m   (Eq. 6-7)
 *   - the adjoint of all of the above with respect to positions, world
 *     sizes, opacities and descriptors (the paper optimises all of them,
 *     Sec. 3.5 and Sec. 3.6 "the sorted per-pixel lists are stored"), and
 *     with respect to the camera intrinsics and pose (Sec. 3.5).
 *
 * The oracle is the plain definition: enumerate every fragment of every
 * point, sort the complete list of every pixel by (depth, point index), keep
 * the first K and blend.  No tiling, no top-K buffers, no fusion.
 *
 * Readings of the paper that the code fixes (each one is listed in the
 * design notes of the repository):
 *   R1  log is log2 (s_i = 2^L), and floor(log2 s) is read off the binary
 *       exponent of s, which is exact.
 *   R2  pinhole camera, +z forward: x = fx*Xc/Zc + cx, y = fy*Yc/Zc + cy,
 *       s = fx*s_w/Zc, depth key z = Zc.
 *   R3  layer-L pixel j has its centre at x = (j + 0.5) * 2^L; with
 *       u = x/2^L - 0.5, j0 = floor(u), a = u - j0 the taps are j0 (weight
 *       1-a) and j0+1 (weight a); same along y.
 *   R4  for 1 <= s < 2^(n-1): Ll = floor(log2 s), Lu = Ll + 1,
 *       iota_lo = (2^Lu - s)/2^Ll, iota_hi = (s - 2^Ll)/2^Ll  (Eq. 5 with
 *       s_i = 2^L); at s = 2^Ll exactly only the lower layer is written.
 *   R5  s < 1: layer 0 only, iota = eps + (1-eps) s, eps = 0.25.
 *   R6  s >= 2^(n-1): layer n-1 only, iota = 1.
 *   R7  a tap whose bilinear or layer weight is exactly zero is not a
 *       fragment; taps outside the layer are dropped, not renormalised.
 *   R8  W_L = ceil(W / 2^L), H_L = ceil(H / 2^L).
 *   R9  points with Zc <= znear, non-finite inputs or s_w < 0 are culled.
 *   R10 lists are ordered by ascending (z, point index); the first K are kept.
 *   R11 alpha_m of Eq. 6 is the fragment opacity gamma_m; c_m is the point's
 *       descriptor; no background term; T_final = prod (1 - gamma_m) is
 *       returned as well.
 *   R24 coarse-layer inclusion (optional, Sec. 3.6 "Implementation
 *       Details"): the list of pixel (L, j, k) also holds, for every coarser
 *       layer L' > L, the fragments of the layer-L' pixel that contains it,
 *       (j >> (L'-L), k >> (L'-L)), each with its own weight gamma (Eq. 3-5 at
 *       its own layer); lists are ordered by (z, point index, layer), so a
 *       point's two layers follow each other, the finer first.
 *   R12 precision of the decisions: everything that decides an integer
 *       (culling, layer pair, tap indices, zero weights, depth order) is
 *       taken from the projection evaluated either in IEEE float32 with the
 *       fixed operation order below (prec32 = 1, the precision of the GPU
 *       kernels) or in float64 (prec32 = 0, the exact-arithmetic reading used
 *       for finite differences).  Every value after that (weights, blending,
 *       adjoint) is float64.
 *         Xc = ((R0*X + R1*Y) + R2*Z) + t0   (likewise Yc, Zc; no fused ops)
 *         x  = (fx*Xc)/Zc + cx,  y = (fy*Yc)/Zc + cy,  s = (fx*s_w)/Zc
 *         u  = x * 2^-L - 0.5,   j0 = floor(u)
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared.
 * The float32 stage relies on FLT_EVAL_METHOD == 0 and no contraction.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the float32 projection stage needs FLT_EVAL_METHOD == 0"
#endif
#if defined(__FAST_MATH__)
#error "build the oracle without -ffast-math"
#endif

#define ORC_MAX_LAYERS 24

/* ------------------------------------------------------------------------ */
/* Camera and pyramid layout                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    float f[17]; /* fx, fy, cx, cy, R[9] row-major (world->camera), t[3], znear */
    int width, height;
} ocam;

typedef struct {
    int n_layers;
    int w[ORC_MAX_LAYERS], h[ORC_MAX_LAYERS];
    int64_t off[ORC_MAX_LAYERS + 1]; /* first pyramid pixel of each layer */
} olayout;

/* R8: layer L has ceil(W/2^L) x ceil(H/2^L) pixels; layers are concatenated. */
static void make_layout(int W, int H, int n_layers, olayout *ly)
{
    ly->n_layers = n_layers;
    ly->off[0] = 0;
    for (int L = 0; L < n_layers; ++L) {
        int64_t s = (int64_t)1 << L;
        ly->w[L] = (int)((W + s - 1) / s);
        ly->h[L] = (int)((H + s - 1) / s);
        ly->off[L + 1] = ly->off[L] + (int64_t)ly->w[L] * ly->h[L];
    }
}

int64_t orc_pyramid_layout(int W, int H, int n_layers, int64_t *offsets, int32_t *widths, int32_t *heights)
{
    olayout ly;
    if (n_layers < 1 || n_layers > ORC_MAX_LAYERS) return -1;
    make_layout(W, H, n_layers, &ly);
    for (int L = 0; L < n_layers; ++L) {
        if (offsets) offsets[L] = ly.off[L];
        if (widths) widths[L] = ly.w[L];
        if (heights) heights[L] = ly.h[L];
    }
    if (offsets) offsets[n_layers] = ly.off[n_layers];
    return ly.off[n_layers];
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 3.1, Eq. 2)                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int vis;           /* 1 if the point is in front of the near plane (R9) */
    int bad;           /* 1 if an input was non-finite or s_w < 0 */
    double x, y, z, s; /* screen position (full-res pixels), depth Zc, screen size */
    float x32, y32, z32, s32; /* the same in float32 when prec32 */
} oproj;

static int finite3(const float *p) { return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]); }

static void project_point(const ocam *c, const float *p, float sw, int prec32, oproj *o)
{
    const float *f = c->f;
    memset(o, 0, sizeof(*o));
    if (!finite3(p) || !isfinite(sw) || sw < 0.0f) {
        o->bad = 1;
        return;
    }
    if (prec32) {
        /* R12: IEEE float32, one rounding per operation, fixed order. */
        float X = p[0], Y = p[1], Z = p[2];
        float xc, yc, zc, m;
        xc = f[4] * X; m = f[5] * Y; xc = xc + m; m = f[6] * Z; xc = xc + m; xc = xc + f[13];
        yc = f[7] * X; m = f[8] * Y; yc = yc + m; m = f[9] * Z; yc = yc + m; yc = yc + f[14];
        zc = f[10] * X; m = f[11] * Y; zc = zc + m; m = f[12] * Z; zc = zc + m; zc = zc + f[15];
        if (!(zc > f[16])) return;
        float x = f[0] * xc; x = x / zc; x = x + f[2];
        float y = f[1] * yc; y = y / zc; y = y + f[3];
        float s = f[0] * sw; s = s / zc;
        if (!isfinite(x) || !isfinite(y) || !isfinite(s)) {
            o->bad = 1;
            return;
        }
        o->vis = 1;
        o->x32 = x; o->y32 = y; o->z32 = zc; o->s32 = s;
        o->x = x; o->y = y; o->z = zc; o->s = s;
    } else {
        double X = p[0], Y = p[1], Z = p[2];
        double xc = (double)f[4] * X + (double)f[5] * Y + (double)f[6] * Z + (double)f[13];
        double yc = (double)f[7] * X + (double)f[8] * Y + (double)f[9] * Z + (double)f[14];
        double zc = (double)f[10] * X + (double)f[11] * Y + (double)f[12] * Z + (double)f[15];
        if (!(zc > (double)f[16])) return;
        o->vis = 1;
        o->x = (double)f[0] * xc / zc + (double)f[2];
        o->y = (double)f[1] * yc / zc + (double)f[3];
        o->z = zc;
        o->s = (double)f[0] * (double)sw / zc;
    }
}

/* ------------------------------------------------------------------------ */
/* Fragments of one point: layer pair, bilinear taps, weights (Eq. 3-5)       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int layer, j, k;     /* layer and pixel (column j, row k) in that layer */
    double wx, wy;       /* bilinear factors: beta = wx * wy (Eq. 4) */
    double dwx, dwy;     /* d wx / d x and d wy / d y, x, y in full-res pixels */
    double iota, diota;  /* layer weight (Eq. 5) and d iota / d s */
} ofrag;

typedef struct {
    int n;
    int L[2];
    double iota[2], diota[2];
} olayers;

/* R1, R4, R5, R6: which layers the point is written to, with weights. */
static void choose_layers(const oproj *o, int prec32, int n_layers, double eps, olayers *out)
{
    int e;
    double s = o->s;
    out->n = 0;
    if (prec32 ? (o->s32 < 1.0f) : (s < 1.0)) {
        out->n = 1;
        out->L[0] = 0;
        out->iota[0] = eps + (1.0 - eps) * s;
        out->diota[0] = 1.0 - eps;
        return;
    }
    int Ll;
    int exact_pow2;
    if (prec32) {
        float m = frexpf(o->s32, &e); /* s32 = m * 2^e, m in [0.5, 1) */
        Ll = e - 1;
        exact_pow2 = (m == 0.5f);
    } else {
        double m = frexp(s, &e);
        Ll = e - 1;
        exact_pow2 = (m == 0.5);
    }
    if (Ll >= n_layers - 1) {
        out->n = 1;
        out->L[0] = n_layers - 1;
        out->iota[0] = 1.0;
        out->diota[0] = 0.0;
        return;
    }
    double pl = ldexp(1.0, Ll), pu = ldexp(1.0, Ll + 1);
    out->n = 1;
    out->L[0] = Ll;
    out->iota[0] = (pu - s) / pl;
    out->diota[0] = -1.0 / pl;
    if (!exact_pow2) {
        out->n = 2;
        out->L[1] = Ll + 1;
        out->iota[1] = (s - pl) / pl;
        out->diota[1] = 1.0 / pl;
    }
}

/* R3: the one or two taps along one axis at layer L.  Returns the count. */
static int axis_taps(double pos, float pos32, int L, int extent, int prec32,
                     int idx[2], double w[2], double dw[2])
{
    double u, fl;
    double scale = ldexp(1.0, -L);
    if (prec32) {
        float u32 = pos32 * ldexpf(1.0f, -L);
        u32 = u32 - 0.5f;
        if (!(u32 > -2.0f && u32 < (float)extent + 1.0f)) return 0;
        float fl32 = floorf(u32);
        u = u32;
        fl = fl32;
    } else {
        u = pos * scale - 0.5;
        if (!(u > -2.0 && u < (double)extent + 1.0)) return 0;
        fl = floor(u);
    }
    int j0 = (int)fl;
    double a = u - fl; /* exact: u and fl are close and both representable */
    int n = 0;
    if (j0 >= 0 && j0 < extent) {
        idx[n] = j0; w[n] = 1.0 - a; dw[n] = -scale; ++n;
    }
    if (a != 0.0 && j0 + 1 >= 0 && j0 + 1 < extent) {
        idx[n] = j0 + 1; w[n] = a; dw[n] = scale; ++n;
    }
    return n;
}

/* All fragments of one visible point (at most 8).  Returns the count. */
static int point_fragments(const oproj *o, const olayout *ly, int prec32, double eps, ofrag out[8])
{
    olayers lys;
    int n = 0;
    if (!o->vis) return 0;
    choose_layers(o, prec32, ly->n_layers, eps, &lys);
    for (int q = 0; q < lys.n; ++q) {
        int L = lys.L[q];
        int jx[2], ky[2];
        double wx[2], wy[2], dwx[2], dwy[2];
        int nx = axis_taps(o->x, o->x32, L, ly->w[L], prec32, jx, wx, dwx);
        int ny = axis_taps(o->y, o->y32, L, ly->h[L], prec32, ky, wy, dwy);
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                ofrag *fr = &out[n++];
                fr->layer = L; fr->j = jx[a]; fr->k = ky[b];
                fr->wx = wx[a]; fr->wy = wy[b];
                fr->dwx = dwx[a]; fr->dwy = dwy[b];
                fr->iota = lys.iota[q]; fr->diota = lys.diota[q];
            }
    }
    return n;
}

static int64_t frag_pixel(const olayout *ly, const ofrag *fr)
{
    return ly->off[fr->layer] + (int64_t)fr->k * ly->w[fr->layer] + fr->j;
}

/* ------------------------------------------------------------------------ */
/* Frames: all fragment lists of a set of pixels                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t pix;
    double z;
    int32_t i;
    int32_t f;   /* index into frags */
    int32_t lay; /* the fragment's own layer (R24 tie-break) */
} okey;

typedef struct {
    ocam cam;
    olayout ly;
    int K, D, prec32;
    int coarse;        /* R24: lists include the fragments of the containing coarser pixels */
    double eps;
    int64_t n;
    const float *pos, *sw, *alpha, *desc; /* borrowed; must outlive the frame */
    oproj *proj;                          /* [n] */
    int64_t n_pix;
    int64_t *pixels;  /* [n_pix] sorted pyramid pixel ids covered by the frame */
    int full;         /* 1 if pixels == 0..P-1 */
    int64_t n_frag;   /* list entries (with coarse inclusion a fragment can be in many lists) */
    ofrag *frags;     /* the fragments the lists refer to */
    okey *keys;       /* [n_frag] sorted by (pix, z, i, layer) */
    int64_t *pix_start; /* [n_pix + 1] range of keys of each frame pixel */
    int64_t n_bad;
} oframe;

static int cmp_key(const void *pa, const void *pb)
{
    const okey *a = (const okey *)pa, *b = (const okey *)pb;
    if (a->pix != b->pix) return a->pix < b->pix ? -1 : 1;
    if (a->z != b->z) return a->z < b->z ? -1 : 1;
    if (a->i != b->i) return a->i < b->i ? -1 : 1;
    if (a->lay != b->lay) return a->lay < b->lay ? -1 : 1;
    return 0;
}

static int cmp_i64(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return (a > b) - (a < b);
}

/* Index of pyramid pixel `pix` in the frame, or -1. */
static int64_t frame_slot(const oframe *fr, int64_t pix)
{
    if (fr->full) return (pix >= 0 && pix < fr->n_pix) ? pix : -1;
    int64_t lo = 0, hi = fr->n_pix;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (fr->pixels[mid] < pix) lo = mid + 1; else hi = mid;
    }
    return (lo < fr->n_pix && fr->pixels[lo] == pix) ? lo : -1;
}

void orc_frame_free(oframe *fr)
{
    if (!fr) return;
    free(fr->proj);
    free(fr->pixels);
    free(fr->frags);
    free(fr->keys);
    free(fr->pix_start);
    free(fr);
}

/*
 * Build the fragment lists.  The frame covers the pixels in `pix_sel` plus
 * every pixel touched by a point in `pt_sel`; with both empty it covers the
 * whole pyramid.
 */
/* Calls emit(pix) for the pixel of fragment fr and, with coarse inclusion
 * (R24), for every pixel of the finer layers that the fragment's pixel
 * contains. */
#define FOR_EACH_LIST_PIXEL(ly, fr, coarse, BODY)                                          \
    do {                                                                                   \
        const int Lf_ = (fr)->layer;                                                       \
        const int Lmin_ = (coarse) ? 0 : Lf_;                                              \
        for (int L_ = Lf_; L_ >= Lmin_; --L_) {                                            \
            const int d_ = Lf_ - L_;                                                       \
            const int j0_ = (fr)->j << d_, k0_ = (fr)->k << d_;                           \
            const int j1_ = ((fr)->j + 1) << d_ < (ly)->w[L_] ? ((fr)->j + 1) << d_ : (ly)->w[L_]; \
            const int k1_ = ((fr)->k + 1) << d_ < (ly)->h[L_] ? ((fr)->k + 1) << d_ : (ly)->h[L_]; \
            for (int kk_ = k0_; kk_ < k1_; ++kk_)                                          \
                for (int jj_ = j0_; jj_ < j1_; ++jj_) {                                    \
                    const int64_t pix = (ly)->off[L_] + (int64_t)kk_ * (ly)->w[L_] + jj_;  \
                    BODY;                                                                  \
                }                                                                          \
        }                                                                                  \
    } while (0)

oframe *orc_frame_build(const float *cam17, int W, int H, int n_layers, int K, double eps, int D,
                        int64_t n, const float *pos, const float *sw, const float *alpha, const float *desc,
                        int prec32, int64_t n_pix_sel, const int64_t *pix_sel, int64_t n_pt_sel,
                        const int64_t *pt_sel, int coarse)
{
    if (n_layers < 1 || n_layers > ORC_MAX_LAYERS || K < 1 || D < 1 || n < 0) return NULL;
    oframe *fr = (oframe *)calloc(1, sizeof(oframe));
    if (!fr) return NULL;
    memcpy(fr->cam.f, cam17, sizeof(fr->cam.f));
    fr->cam.width = W;
    fr->cam.height = H;
    make_layout(W, H, n_layers, &fr->ly);
    fr->K = K; fr->D = D; fr->eps = eps; fr->prec32 = prec32; fr->coarse = coarse != 0;
    fr->n = n; fr->pos = pos; fr->sw = sw; fr->alpha = alpha; fr->desc = desc;
    int64_t P = fr->ly.off[n_layers];

    fr->proj = (oproj *)calloc((size_t)(n > 0 ? n : 1), sizeof(oproj));
    if (!fr->proj) goto fail;
    for (int64_t i = 0; i < n; ++i) {
        project_point(&fr->cam, pos + 3 * i, sw[i], prec32, &fr->proj[i]);
        fr->n_bad += fr->proj[i].bad;
    }

    /* Pixel set of the frame. */
    if (n_pix_sel <= 0 && n_pt_sel <= 0) {
        fr->full = 1;
        fr->n_pix = P;
    } else {
        /* a selected point's pixels: every list that holds one of its
           fragments (with coarse inclusion, also the finer pixels below) */
        int64_t cap = n_pix_sel > 0 ? n_pix_sel : 0;
        for (int64_t q = 0; q < n_pt_sel; ++q) {
            int64_t i = pt_sel[q];
            if (i < 0 || i >= n) continue;
            ofrag tmp[8];
            int nf = point_fragments(&fr->proj[i], &fr->ly, prec32, eps, tmp);
            for (int t = 0; t < nf; ++t) FOR_EACH_LIST_PIXEL(&fr->ly, &tmp[t], fr->coarse, { (void)pix; ++cap; });
        }
        fr->pixels = (int64_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int64_t));
        if (!fr->pixels) goto fail;
        int64_t m = 0;
        for (int64_t q = 0; q < n_pix_sel; ++q)
            if (pix_sel[q] >= 0 && pix_sel[q] < P) fr->pixels[m++] = pix_sel[q];
        for (int64_t q = 0; q < n_pt_sel; ++q) {
            int64_t i = pt_sel[q];
            if (i < 0 || i >= n) continue;
            ofrag tmp[8];
            int nf = point_fragments(&fr->proj[i], &fr->ly, prec32, eps, tmp);
            for (int t = 0; t < nf; ++t) FOR_EACH_LIST_PIXEL(&fr->ly, &tmp[t], fr->coarse, { fr->pixels[m++] = pix; });
        }
        qsort(fr->pixels, (size_t)m, sizeof(int64_t), cmp_i64);
        int64_t u = 0;
        for (int64_t q = 0; q < m; ++q)
            if (u == 0 || fr->pixels[u - 1] != fr->pixels[q]) fr->pixels[u++] = fr->pixels[q];
        fr->n_pix = u;
    }

    /* Enumerate every fragment of every point that lands in the frame. */
    {
        uint8_t *mask = NULL;
        if (!fr->full) {
            mask = (uint8_t *)calloc((size_t)(P > 0 ? P : 1), 1);
            if (!mask) goto fail;
            for (int64_t q = 0; q < fr->n_pix; ++q) mask[fr->pixels[q]] = 1;
        }
        /* every fragment, and one list entry per pixel whose list holds it */
        int64_t cap_f = 0, cap_k = 0;
        for (int64_t i = 0; i < n; ++i) {
            ofrag tmp[8];
            int nf = point_fragments(&fr->proj[i], &fr->ly, prec32, eps, tmp);
            for (int t = 0; t < nf; ++t) {
                int used = 0;
                FOR_EACH_LIST_PIXEL(&fr->ly, &tmp[t], fr->coarse, if (!mask || mask[pix]) { ++cap_k; used = 1; });
                cap_f += used;
            }
        }
        fr->frags = (ofrag *)malloc((size_t)(cap_f > 0 ? cap_f : 1) * sizeof(ofrag));
        fr->keys = (okey *)malloc((size_t)(cap_k > 0 ? cap_k : 1) * sizeof(okey));
        if (!fr->frags || !fr->keys) { free(mask); goto fail; }
        int64_t mf = 0, mk = 0;
        for (int64_t i = 0; i < n; ++i) {
            ofrag tmp[8];
            int nf = point_fragments(&fr->proj[i], &fr->ly, prec32, eps, tmp);
            for (int t = 0; t < nf; ++t) {
                int used = 0;
                FOR_EACH_LIST_PIXEL(&fr->ly, &tmp[t], fr->coarse, if (!mask || mask[pix]) {
                    fr->keys[mk].pix = pix;
                    fr->keys[mk].z = fr->proj[i].z;
                    fr->keys[mk].i = (int32_t)i;
                    fr->keys[mk].f = (int32_t)mf;
                    fr->keys[mk].lay = tmp[t].layer;
                    ++mk;
                    used = 1;
                });
                if (used) fr->frags[mf++] = tmp[t];
            }
        }
        free(mask);
        fr->n_frag = mk;
    }
    /* R10: each pixel's list in ascending (z, i). */
    qsort(fr->keys, (size_t)fr->n_frag, sizeof(okey), cmp_key);

    fr->pix_start = (int64_t *)malloc((size_t)(fr->n_pix + 1) * sizeof(int64_t));
    if (!fr->pix_start) goto fail;
    {
        int64_t q = 0;
        for (int64_t s = 0; s < fr->n_pix; ++s) {
            int64_t pix = fr->full ? s : fr->pixels[s];
            while (q < fr->n_frag && fr->keys[q].pix < pix) ++q;
            fr->pix_start[s] = q;
        }
        fr->pix_start[fr->n_pix] = fr->n_frag;
    }
    return fr;
fail:
    orc_frame_free(fr);
    return NULL;
}

int64_t orc_frame_num_pixels(const oframe *fr) { return fr->n_pix; }
int64_t orc_frame_num_fragments(const oframe *fr) { return fr->n_frag; }
int64_t orc_frame_num_bad(const oframe *fr) { return fr->n_bad; }

void orc_frame_pixels(const oframe *fr, int64_t *out)
{
    for (int64_t s = 0; s < fr->n_pix; ++s) out[s] = fr->full ? s : fr->pixels[s];
}

/* Projected records: xyzs [n,4] (float64 values; float32 values upcast when prec32) and visibility. */
void orc_frame_records(const oframe *fr, double *xyzs, int8_t *vis)
{
    for (int64_t i = 0; i < fr->n; ++i) {
        const oproj *o = &fr->proj[i];
        xyzs[4 * i + 0] = o->vis ? o->x : 0.0;
        xyzs[4 * i + 1] = o->vis ? o->y : 0.0;
        xyzs[4 * i + 2] = o->vis ? o->z : 0.0;
        xyzs[4 * i + 3] = o->vis ? o->s : 0.0;
        vis[i] = (int8_t)o->vis;
    }
}

/* Every fragment in the frame, in sorted order: pixel, depth, point, weight beta*iota. */
void orc_frame_fragments(const oframe *fr, int64_t *pix, double *z, int32_t *idx, double *w)
{
    for (int64_t q = 0; q < fr->n_frag; ++q) {
        const okey *k = &fr->keys[q];
        const ofrag *f = &fr->frags[k->f];
        if (pix) pix[q] = k->pix;
        if (z) z[q] = k->z;
        if (idx) idx[q] = k->i;
        if (w) w[q] = f->wx * f->wy * f->iota;
    }
}

/* ------------------------------------------------------------------------ */
/* Blending (Eq. 6-7) and its adjoint                                        */
/* ------------------------------------------------------------------------ */

static double frag_gamma(const oframe *fr, const okey *k)
{
    const ofrag *f = &fr->frags[k->f];
    return f->wx * f->wy * f->iota * (double)fr->alpha[k->i];
}

/* Blend one pixel's sorted list: first min(n, K) fragments front to back. */
static void blend_list(const oframe *fr, const okey *list, int64_t n, double *C, double *t_final, int *n_kept)
{
    int D = fr->D;
    int m_end = (int)(n < fr->K ? n : fr->K);
    double T = 1.0;
    for (int d = 0; d < D; ++d) C[d] = 0.0;
    for (int m = 0; m < m_end; ++m) {
        double g = frag_gamma(fr, &list[m]);
        const float *c = fr->desc + (int64_t)D * list[m].i;
        for (int d = 0; d < D; ++d) C[d] += T * g * (double)c[d];
        T *= (1.0 - g);
    }
    if (t_final) *t_final = T;
    if (n_kept) *n_kept = m_end;
}

/* Outputs over the frame's pixels: pyramid [n_pix, D], kept [n_pix, K] (-1 padded),
 * n_kept, t_final, n_frag (the full candidate count of each pixel). */
void orc_frame_render(const oframe *fr, double *pyramid, int32_t *kept, int32_t *n_kept, double *t_final,
                      int32_t *n_frag)
{
    double C[1024];
    int D = fr->D, K = fr->K;
    for (int64_t s = 0; s < fr->n_pix; ++s) {
        const okey *list = fr->keys + fr->pix_start[s];
        int64_t n = fr->pix_start[s + 1] - fr->pix_start[s];
        double T;
        int nk;
        blend_list(fr, list, n, C, &T, &nk);
        if (pyramid)
            for (int d = 0; d < D; ++d) pyramid[s * D + d] = C[d];
        if (kept)
            for (int m = 0; m < K; ++m) kept[s * K + m] = m < nk ? list[m].i : -1;
        if (n_kept) n_kept[s] = nk;
        if (t_final) t_final[s] = T;
        if (n_frag) n_frag[s] = (int32_t)n;
    }
}

/*
 * Adjoint of the blend of one pixel.  With L = G . C and the division-free
 * back-to-front recurrence R_M = 0, R_{m-1} = gamma_m g_m + (1-gamma_m) R_m,
 * where g_m = G . c_m:
 *   dL/dgamma_m = T_m (g_m - R_m),   dL/dc_m = T_m gamma_m G.
 * gamma = wx wy iota alpha chains to alpha, x (through wx), y (through wy)
 * and s (through iota).  Screen-space gradients go to gx, gy, gs.
 */
static void pixel_adjoint(const oframe *fr, const okey *list, int64_t n, const double *G,
                          double *g_alpha, double *g_desc, double *gx, double *gy, double *gs)
{
    int D = fr->D;
    int M = (int)(n < fr->K ? n : fr->K);
    double Tm[1024];
    double T = 1.0;
    for (int m = 0; m < M; ++m) {
        Tm[m] = T;
        T *= 1.0 - frag_gamma(fr, &list[m]);
    }
    double R = 0.0;
    for (int m = M - 1; m >= 0; --m) {
        const okey *k = &list[m];
        const ofrag *f = &fr->frags[k->f];
        const float *c = fr->desc + (int64_t)D * k->i;
        double alpha = (double)fr->alpha[k->i];
        double beta = f->wx * f->wy;
        double gam = beta * f->iota * alpha;
        double g = 0.0;
        for (int d = 0; d < D; ++d) g += G[d] * (double)c[d];
        double dgam = Tm[m] * (g - R);
        R = gam * g + (1.0 - gam) * R;
        if (g_desc)
            for (int d = 0; d < D; ++d) g_desc[(int64_t)D * k->i + d] += Tm[m] * gam * G[d];
        if (g_alpha) g_alpha[k->i] += dgam * beta * f->iota;
        double dw = dgam * alpha; /* d L / d (wx wy iota) */
        if (gx) gx[k->i] += dw * f->wy * f->iota * f->dwx;
        if (gy) gy[k->i] += dw * f->wx * f->iota * f->dwy;
        if (gs) gs[k->i] += dw * beta * f->diota;
    }
}

/* Screen-space gradient (gx, gy, gs) of point i -> world position and world size. */
static void chain_to_world(const oframe *fr, int64_t i, double gx, double gy, double gs, double *gpos, double *gsw)
{
    const float *c = fr->cam.f;
    const oproj *o = &fr->proj[i];
    double fx = c[0], fy = c[1], cx = c[2], cy = c[3];
    double Zc = o->z;
    /* x = fx Xc/Zc + cx, y = fy Yc/Zc + cy, s = fx s_w / Zc */
    double dXc = gx * fx / Zc;
    double dYc = gy * fy / Zc;
    double dZc = -(gx * (o->x - cx) + gy * (o->y - cy) + gs * o->s) / Zc;
    *gsw = gs * fx / Zc;
    /* X_c = R X_w + t  ->  dL/dX_w = R^T dL/dX_c */
    for (int a = 0; a < 3; ++a)
        gpos[a] = (double)c[4 + a] * dXc + (double)c[7 + a] * dYc + (double)c[10 + a] * dZc;
}

/*
 * Gradients of L = sum over the frame's pixels of G . C with respect to
 * every point's position [n,3], world size [n], opacity [n] and descriptor
 * [n,D].  G is [n_pix, D] over the frame's pixels.  Outputs are overwritten.
 * grad_screen (nullable) receives dL/dx, dL/dy, dL/ds per point [n,3].
 */
void orc_frame_backward(const oframe *fr, const double *G, double *grad_pos, double *grad_sw, double *grad_alpha,
                        double *grad_desc, double *grad_screen)
{
    int64_t n = fr->n;
    int D = fr->D;
    double *gx = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *gy = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *gs = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (grad_alpha) memset(grad_alpha, 0, (size_t)n * sizeof(double));
    if (grad_desc) memset(grad_desc, 0, (size_t)n * D * sizeof(double));
    for (int64_t s = 0; s < fr->n_pix; ++s) {
        const okey *list = fr->keys + fr->pix_start[s];
        int64_t cnt = fr->pix_start[s + 1] - fr->pix_start[s];
        if (cnt == 0) continue;
        pixel_adjoint(fr, list, cnt, G + s * D, grad_alpha, grad_desc, gx, gy, gs);
    }
    for (int64_t i = 0; i < n; ++i) {
        double gp[3] = {0, 0, 0}, gw = 0.0;
        if (fr->proj[i].vis) chain_to_world(fr, i, gx[i], gy[i], gs[i], gp, &gw);
        if (grad_pos) { grad_pos[3 * i] = gp[0]; grad_pos[3 * i + 1] = gp[1]; grad_pos[3 * i + 2] = gp[2]; }
        if (grad_sw) grad_sw[i] = gw;
        if (grad_screen) { grad_screen[3 * i] = gx[i]; grad_screen[3 * i + 1] = gy[i]; grad_screen[3 * i + 2] = gs[i]; }
    }
    free(gx); free(gy); free(gs);
}

/*
 * Gradient of L = sum over the frame's pixels of G . C with respect to the
 * camera (the paper optimises camera poses and intrinsics along with the
 * points: Sec. 3 pipeline figure, Sec. 3.5).  The camera enters only through
 * each point's screen position and size (Eq. 2):
 *   X_c = R X_w + t,  x = fx X_c/Z_c + cx,  y = fy Y_c/Z_c + cy,  s = fx s_w/Z_c,
 * so with the point's screen-space gradient (gx, gy, gs) from the pixel
 * adjoints, by the chain rule:
 *   dL/dfx = gx X_c/Z_c + gs s_w/Z_c,   dL/dfy = gy Y_c/Z_c,
 *   dL/dcx = gx,   dL/dcy = gy,
 *   dL/dX_c = (gx fx/Z_c, gy fy/Z_c, -(gx fx X_c + gy fy Y_c + gs fx s_w)/Z_c^2),
 *   dL/dt = dL/dX_c,   dL/dR[r][c] = dL/dX_c[r] X_w[c],
 * summed over the visible points.  X_c/Z_c, Y_c/Z_c and s_w/Z_c are read off
 * the frame's screen state: (x - cx)/fx, (y - cy)/fy, s/fx.  Depth order and
 * layer choice are piecewise constant and carry no gradient.
 * out16 = dL/d(fx, fy, cx, cy, R[0..8] row-major, t[0..2]); overwritten.
 */
void orc_frame_camera_backward(const oframe *fr, const double *G, double *out16)
{
    int64_t n = fr->n;
    int D = fr->D;
    const float *c = fr->cam.f;
    double fx = c[0], fy = c[1], cx = c[2], cy = c[3];
    double *gx = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *gy = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *gs = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int q = 0; q < 16; ++q) out16[q] = 0.0;
    for (int64_t s = 0; s < fr->n_pix; ++s) {
        const okey *list = fr->keys + fr->pix_start[s];
        int64_t cnt = fr->pix_start[s + 1] - fr->pix_start[s];
        if (cnt == 0) continue;
        pixel_adjoint(fr, list, cnt, G + s * D, NULL, NULL, gx, gy, gs);
    }
    for (int64_t i = 0; i < n; ++i) {
        const oproj *o = &fr->proj[i];
        if (!o->vis) continue;
        double Zc = o->z;
        double xn = (o->x - cx) / fx; /* X_c / Z_c */
        double yn = (o->y - cy) / fy; /* Y_c / Z_c */
        double sn = o->s / fx;        /* s_w / Z_c */
        out16[0] += gx[i] * xn + gs[i] * sn;
        out16[1] += gy[i] * yn;
        out16[2] += gx[i];
        out16[3] += gy[i];
        double dXc[3];
        dXc[0] = gx[i] * fx / Zc;
        dXc[1] = gy[i] * fy / Zc;
        dXc[2] = -(gx[i] * fx * xn + gy[i] * fy * yn + gs[i] * fx * sn) / Zc;
        const float *Xw = fr->pos + 3 * i;
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col) out16[4 + 3 * r + col] += dXc[r] * (double)Xw[col];
            out16[13 + r] += dXc[r];
        }
    }
    free(gx); free(gy); free(gs);
}

/* ------------------------------------------------------------------------ */
/* Local central finite differences (float64 frames only)                    */
/* ------------------------------------------------------------------------ */

/* float64 projection of one point from float64 inputs (same formulas as
 * project_point with prec32 = 0). */
static void project_point64(const ocam *c, const double *p, double sw, oproj *o)
{
    const float *f = c->f;
    memset(o, 0, sizeof(*o));
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2]) || !isfinite(sw) || sw < 0.0) {
        o->bad = 1;
        return;
    }
    double xc = (double)f[4] * p[0] + (double)f[5] * p[1] + (double)f[6] * p[2] + (double)f[13];
    double yc = (double)f[7] * p[0] + (double)f[8] * p[1] + (double)f[9] * p[2] + (double)f[14];
    double zc = (double)f[10] * p[0] + (double)f[11] * p[1] + (double)f[12] * p[2] + (double)f[15];
    if (!(zc > (double)f[16])) return;
    o->vis = 1;
    o->x = (double)f[0] * xc / zc + (double)f[2];
    o->y = (double)f[1] * yc / zc + (double)f[3];
    o->z = zc;
    o->s = (double)f[0] * sw / zc;
}

/*
 * Loss restricted to the pixels where point p has fragments, with point p's
 * inputs replaced by (pos3, sw, alpha, desc) in float64.  Also records the
 * pixel set and the kept order, so the caller can check that the discrete
 * state (taps, layers, kept lists) did not change.  Returns 0 on success.
 */
#define ORC_FD_MAXK 64
typedef struct {
    int n;
    int64_t pix[8];
    int nk[8];
    int32_t kept[8][ORC_FD_MAXK];
    double loss;
} olocal;

/* Screen-space state of point p for perturbed inputs.  A float64 frame
 * projects them in float64.  A float32 frame keeps its float32 screen-space
 * state and adds the float64 change of the projection, so the differences
 * are taken around exactly the state the frame's decisions were made at. */
static void eval_proj(const oframe *fr, int64_t p, const double *pos3, double sw, oproj *o)
{
    if (!fr->prec32) {
        project_point64(&fr->cam, pos3, sw, o);
        return;
    }
    const double base3[3] = {fr->pos[3 * p], fr->pos[3 * p + 1], fr->pos[3 * p + 2]};
    oproj b64, q64;
    project_point64(&fr->cam, base3, (double)fr->sw[p], &b64);
    project_point64(&fr->cam, pos3, sw, &q64);
    *o = fr->proj[p];
    if (!o->vis || !b64.vis || !q64.vis) {
        o->vis = 0;
        return;
    }
    o->x += q64.x - b64.x;
    o->y += q64.y - b64.y;
    o->z += q64.z - b64.z;
    o->s += q64.s - b64.s;
}

static int same_taps(const ofrag *a, int na, const ofrag *b, int nb)
{
    if (na != nb) return 0;
    for (int t = 0; t < na; ++t)
        if (a[t].layer != b[t].layer || a[t].j != b[t].j || a[t].k != b[t].k) return 0;
    return 1;
}

static int local_eval(const oframe *fr, int64_t p, const double *pos3, double sw, double alpha,
                      const double *desc, const double *G, olocal *out)
{
    oproj o;
    ofrag frs[8];
    int D = fr->D, K = fr->K;
    if (K > ORC_FD_MAXK) return -1;
    eval_proj(fr, p, pos3, sw, &o);
    int nf = point_fragments(&o, &fr->ly, 0, fr->eps, frs);
    out->n = nf;
    out->loss = 0.0;
    for (int t = 0; t < nf; ++t) {
        int64_t pix = frag_pixel(&fr->ly, &frs[t]);
        int64_t s = frame_slot(fr, pix);
        if (s < 0) return -2; /* pixel outside the frame */
        const okey *base = fr->keys + fr->pix_start[s];
        int64_t cnt = fr->pix_start[s + 1] - fr->pix_start[s];
        /* The pixel's full list with point p's fragment replaced, re-sorted. */
        okey *list = (okey *)malloc((size_t)(cnt + 1) * sizeof(okey));
        if (!list) return -3;
        int64_t m = 0;
        for (int64_t q = 0; q < cnt; ++q)
            if (base[q].i != p) list[m++] = base[q];
        list[m].pix = pix; list[m].z = o.z; list[m].i = (int32_t)p; list[m].f = -1;
        ++m;
        qsort(list, (size_t)m, sizeof(okey), cmp_key);
        int M = (int)(m < K ? m : K);
        double T = 1.0, loss = 0.0;
        out->pix[t] = pix;
        out->nk[t] = M;
        for (int q = 0; q < M; ++q) {
            double g, cd;
            if (list[q].i == p) g = frs[t].wx * frs[t].wy * frs[t].iota * alpha;
            else g = frag_gamma(fr, &list[q]);
            for (int d = 0; d < D; ++d) {
                cd = list[q].i == p ? desc[d] : (double)fr->desc[(int64_t)D * list[q].i + d];
                loss += G[s * D + d] * T * g * cd;
            }
            T *= 1.0 - g;
            out->kept[t][q] = list[q].i;
        }
        out->loss += loss;
        free(list);
    }
    return 0;
}

static int same_state(const olocal *a, const olocal *b)
{
    if (a->n != b->n) return 0;
    for (int t = 0; t < a->n; ++t) {
        if (a->pix[t] != b->pix[t] || a->nk[t] != b->nk[t]) return 0;
        for (int q = 0; q < a->nk[t]; ++q)
            if (a->kept[t][q] != b->kept[t][q]) return 0;
    }
    return 1;
}

/*
 * Central differences of L = sum over the frame's pixels of G . C for the
 * selected points.  Parameters per point, in order: X, Y, Z (step h_pos),
 * s_w (step h_sw_rel * s_w), alpha (step h_alpha), desc[0..D) (step
 * h_desc).  fd is [n_sel, 5 + D]; valid is 1 where the discrete state is
 * identical at -h, 0 and +h (else the entry is 0 and not a derivative).
 * The frame must cover every pixel of the selected points.  In a float32
 * frame the differences are taken around the frame's float32 screen-space
 * state (see eval_proj).  Returns 0, or -1 on bad arguments (also for a
 * frame with coarse-layer inclusion, whose lists this local evaluation does
 * not rebuild).
 */
int orc_frame_fd(const oframe *fr, const double *G, int64_t n_sel, const int64_t *sel, double h_pos,
                 double h_sw_rel, double h_alpha, double h_desc, double *fd, int8_t *valid)
{
    if (fr->coarse) return -1;
    int D = fr->D;
    int np = 5 + D;
    double *d0 = (double *)malloc((size_t)D * sizeof(double));
    double *dv = (double *)malloc((size_t)D * sizeof(double));
    if (!d0 || !dv) { free(d0); free(dv); return -1; }
    for (int64_t q = 0; q < n_sel; ++q) {
        int64_t p = sel[q];
        for (int k = 0; k < np; ++k) { fd[q * np + k] = 0.0; valid[q * np + k] = 0; }
        if (p < 0 || p >= fr->n) continue;
        double pos0[3] = {fr->pos[3 * p], fr->pos[3 * p + 1], fr->pos[3 * p + 2]};
        double sw0 = fr->sw[p], a0 = fr->alpha[p];
        for (int d = 0; d < D; ++d) d0[d] = fr->desc[(int64_t)D * p + d];
        olocal base, plus, minus;
        if (local_eval(fr, p, pos0, sw0, a0, d0, G, &base) != 0) continue;
        {
            /* the unperturbed local state must be the frame's own state */
            ofrag mine[8], here[8];
            oproj o;
            int nm = point_fragments(&fr->proj[p], &fr->ly, fr->prec32, fr->eps, mine);
            eval_proj(fr, p, pos0, sw0, &o);
            int nh = point_fragments(&o, &fr->ly, 0, fr->eps, here);
            if (!same_taps(mine, nm, here, nh)) continue;
        }
        for (int k = 0; k < np; ++k) {
            double h = k < 3 ? h_pos : k == 3 ? h_sw_rel * sw0 : k == 4 ? h_alpha : h_desc;
            double lp = 0.0, lm = 0.0;
            int ok = 1;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double pos[3] = {pos0[0], pos0[1], pos0[2]};
                double sw = sw0, a = a0;
                memcpy(dv, d0, (size_t)D * sizeof(double));
                if (k < 3) pos[k] += sgn * h;
                else if (k == 3) sw += sgn * h;
                else if (k == 4) a += sgn * h;
                else dv[k - 5] += sgn * h;
                olocal *out = sgn > 0 ? &plus : &minus;
                if (local_eval(fr, p, pos, sw, a, dv, G, out) != 0 || !same_state(&base, out)) ok = 0;
            }
            if (!ok) continue;
            lp = plus.loss;
            lm = minus.loss;
            fd[q * np + k] = (lp - lm) / (2.0 * h);
            valid[q * np + k] = 1;
        }
    }
    free(d0);
    free(dv);
    return 0;
}
