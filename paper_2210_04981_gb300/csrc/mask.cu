// adaptive ray mask (Ray Trace section): the G-buffer is smoothed by a
// Gaussian before a Sobel gradient of its normal and depth marks geometry
// edges (the smoothing suppresses noise and staircase edges, as in Canny's
// detector); a luminance variance accumulated over previous frames adds rays
// where the traced result is still noisy or has just appeared.
//
// k_mask_edge: one 16x16 pixel block per CUDA block; the block's (16+6)^2
//   nd halo is staged in shared memory once, the separable 5-tap Gaussian
//   runs as a row pass and a column pass in shared memory, then the 1/8
//   scaled 3x3 Sobel; writes edge bits and marks the mask tiles that hold
//   an edge.
// k_mask_spp: per pixel, dilated tile flag and the variance term -> spp.
#include <cmath>
#include <mutex>

#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

constexpr int B = 16;            // pixel block edge
constexpr int HALO = 3;          // 2 (Gaussian) + 1 (Sobel)
constexpr int SRC = B + 2 * HALO;  // 22
constexpr int FIL = B + 2;         // 18: filtered values needed by the Sobel

struct GaussW {
    float w[5];
};

template <class ND>
struct EdgeArgs {
    const ND* nd;
    int W, H;
    GaussW g;
    float tau;
    int tile, ntx;
    uint8_t* edge;
    uint8_t* tiles;
    Coc coc;        // CoC-scaled mask: the lens's CoC in pixels
    float rmax;     // CoC radius cap (the post-filter's r_max)
    float* tile_r;  // largest CoC radius per mask tile (atomic max of float bits); NULL: fixed dilation
};

template <class ND>
__device__ __forceinline__ void mask_edge_body(const EdgeArgs<ND>& ar, int bx, int by) {
    __shared__ float4 src[SRC][SRC];
    __shared__ float4 row[SRC][FIL];
    __shared__ float4 fil[FIL][FIL];
    const ND* __restrict__ nd = ar.nd;
    const int W = ar.W, H = ar.H, tile = ar.tile, ntx = ar.ntx;
    const GaussW g = ar.g;
    const float tau = ar.tau;
    uint8_t* __restrict__ edge = ar.edge;
    uint8_t* __restrict__ tiles = ar.tiles;
    const int x0 = bx * B, y0 = by * B;
    const int tid = threadIdx.x;
    // stage nd with clamp-to-edge (the Gaussian's border rule)
    for (int k = tid; k < SRC * SRC; k += 256) {
        int r = k / SRC, c = k % SRC;
        int x = min(max(x0 - HALO + c, 0), W - 1), y = min(max(y0 - HALO + r, 0), H - 1);
        src[r][c] = ld4(nd + (size_t)y * W + x);
    }
    __syncthreads();
    if (ar.tile_r) {
        // largest CoC radius min(|c(z)| / 2, r_max) of each mask tile's pixels:
        // a shared-memory maximum per tile this block touches, then one global
        // atomic maximum per tile (non-negative floats order as their bits)
        __shared__ unsigned s_r[B][B];
        const int tx0 = x0 / tile, ty0 = y0 / tile;
        s_r[tid >> 4][tid & 15] = 0u;
        __syncthreads();
        const int i = x0 + (tid & 15), j = y0 + (tid >> 4);
        if (i < W && j < H) {
            const float r = fminf(fabsf(ar.coc(src[(tid >> 4) + HALO][(tid & 15) + HALO].w)) * 0.5f, ar.rmax);
            atomicMax(&s_r[j / tile - ty0][i / tile - tx0], __float_as_uint(r));
        }
        __syncthreads();
        const int nbx = min(x0 + B - 1, W - 1) / tile - tx0 + 1, nby = min(y0 + B - 1, H - 1) / tile - ty0 + 1;
        if (tid < nbx * nby) {
            const int a = tid % nbx, b = tid / nbx;
            const unsigned v = s_r[b][a];
            if (v) atomicMax(reinterpret_cast<unsigned*>(ar.tile_r) + (ty0 + b) * ntx + tx0 + a, v);
        }
    }
    // row pass: filtered columns x0-1 .. x0+16 for all 22 staged rows
    for (int k = tid; k < SRC * FIL; k += 256) {
        int r = k / FIL, c = k % FIL;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            float4 v = src[r][c + t];
            a.x = fmaf(g.w[t], v.x, a.x);
            a.y = fmaf(g.w[t], v.y, a.y);
            a.z = fmaf(g.w[t], v.z, a.z);
            a.w = fmaf(g.w[t], v.w, a.w);
        }
        row[r][c] = a;
    }
    __syncthreads();
    // column pass: filtered rows y0-1 .. y0+16
    for (int k = tid; k < FIL * FIL; k += 256) {
        int r = k / FIL, c = k % FIL;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            float4 v = row[r + t][c];
            a.x = fmaf(g.w[t], v.x, a.x);
            a.y = fmaf(g.w[t], v.y, a.y);
            a.z = fmaf(g.w[t], v.z, a.z);
            a.w = fmaf(g.w[t], v.w, a.w);
        }
        fil[r][c] = a;
    }
    __syncthreads();
    const int lx = tid & 15, ly = tid >> 4;
    const int i = x0 + lx, j = y0 + ly;
    if (i >= W || j >= H) return;
    // Sobel on the filtered image with clamp-to-edge (the Sobel's border rule):
    // an out-of-image neighbour reads the filtered value of the border pixel.
    // fil holds filtered rows y0-1 .. y0+16 and columns x0-1 .. x0+16.
    const int cl = max(i - 1, 0) - (x0 - 1), cc = lx + 1, cr = min(i + 1, W - 1) - (x0 - 1);
    const int ru = max(j - 1, 0) - (y0 - 1), rc = ly + 1, rd = min(j + 1, H - 1) - (y0 - 1);
    const float4 f_ul = fil[ru][cl], f_uc = fil[ru][cc], f_ur = fil[ru][cr];
    const float4 f_cl = fil[rc][cl], f_cr = fil[rc][cr];
    const float4 f_dl = fil[rd][cl], f_dc = fil[rd][cc], f_dr = fil[rd][cr];
    float gx[4], gy[4];
    // gx: right column minus left column, rows weighted 1 2 1; gy: down row minus up row
    gx[0] = (f_ur.x - f_ul.x) + 2.f * (f_cr.x - f_cl.x) + (f_dr.x - f_dl.x);
    gx[1] = (f_ur.y - f_ul.y) + 2.f * (f_cr.y - f_cl.y) + (f_dr.y - f_dl.y);
    gx[2] = (f_ur.z - f_ul.z) + 2.f * (f_cr.z - f_cl.z) + (f_dr.z - f_dl.z);
    gx[3] = (f_ur.w - f_ul.w) + 2.f * (f_cr.w - f_cl.w) + (f_dr.w - f_dl.w);
    gy[0] = (f_dl.x - f_ul.x) + 2.f * (f_dc.x - f_uc.x) + (f_dr.x - f_ur.x);
    gy[1] = (f_dl.y - f_ul.y) + 2.f * (f_dc.y - f_uc.y) + (f_dr.y - f_ur.y);
    gy[2] = (f_dl.z - f_ul.z) + 2.f * (f_dc.z - f_uc.z) + (f_dr.z - f_ur.z);
    gy[3] = (f_dl.w - f_ul.w) + 2.f * (f_dc.w - f_uc.w) + (f_dr.w - f_ur.w);
    for (int c = 0; c < 4; ++c) {
        gx[c] *= 0.125f;
        gy[c] *= 0.125f;
    }
    float en = sqrtf(gx[0] * gx[0] + gy[0] * gy[0] + gx[1] * gx[1] + gy[1] * gy[1] + gx[2] * gx[2] + gy[2] * gy[2]);
    float ez = sqrtf(gx[3] * gx[3] + gy[3] * gy[3]) / fil[ly + 1][lx + 1].w;
    float e = fmaxf(en, ez);
    uint8_t bit = e > tau ? 1 : 0;
    edge[(size_t)j * W + i] = bit;
    if (bit) tiles[(j / tile) * ntx + i / tile] = 1;
}

template <class ND>
__global__ void __launch_bounds__(256) k_mask_edge(EdgeArgs<ND> a) {
    mask_edge_body(a, blockIdx.x, blockIdx.y);
}

struct SppArgs {
    int W, H, tile, ntx, nty, dil;
    const uint8_t* tiles;
    int variance_on;
    const float2* mv;
    const float2* hmom;
    const uint8_t* hhlen;
    int spp_max;
    float var_tau, var_scale;
    int hlen_young;
    uint8_t* spp;
    const float* tile_r;  // CoC-scaled mask: largest CoC radius per tile; NULL: fixed dilation
};

__device__ __forceinline__ void mask_spp_body(const SppArgs& ar, int bx, int by) {
    const int W = ar.W, H = ar.H, tile = ar.tile, ntx = ar.ntx, nty = ar.nty, dil = ar.dil;
    const uint8_t* __restrict__ tiles = ar.tiles;
    const int variance_on = ar.variance_on, spp_max = ar.spp_max, hlen_young = ar.hlen_young;
    const float2* __restrict__ mv = ar.mv;
    const float2* __restrict__ hmom = ar.hmom;
    const uint8_t* __restrict__ hhlen = ar.hhlen;
    const float var_tau = ar.var_tau, var_scale = ar.var_scale;
    uint8_t* __restrict__ spp = ar.spp;
    // the dilated flag of every mask tile this 32x8 block touches, once, in
    // shared memory (at most 32 x 8 tiles, for tile = 1)
    __shared__ unsigned char s_on[8][32];
    const int x0 = bx * 32, y0 = by * 8;
    const int tx0 = x0 / tile, ty0 = y0 / tile;
    const int ntx_b = min(x0 + 31, W - 1) / tile - tx0 + 1, nty_b = min(y0 + 7, H - 1) / tile - ty0 + 1;
    {
        const int e = threadIdx.x, ey = e >> 5, ex = e & 31;
        if (ey < nty_b && ex < ntx_b) {
            const int tx = tx0 + ex, ty = ty0 + ey;
            bool any = false;
            if (!ar.tile_r) {
                for (int b = max(ty - dil, 0); b <= min(ty + dil, nty - 1) && !any; ++b)
                    for (int a = max(tx - dil, 0); a <= min(tx + dil, ntx - 1); ++a)
                        if (__ldg(&tiles[b * ntx + a])) {
                            any = true;
                            break;
                        }
            } else {
                // an edge tile reaches max(dil, ceil(r / tile)) tiles (at most 8),
                // r its pixels' largest CoC radius
                const float inv_tile = 1.f / (float)tile;
                for (int b = max(ty - 8, 0); b <= min(ty + 8, nty - 1) && !any; ++b)
                    for (int a = max(tx - 8, 0); a <= min(tx + 8, ntx - 1); ++a) {
                        if (!__ldg(&tiles[b * ntx + a])) continue;
                        const int reach =
                            min(8, max(dil, (int)ceilf(__ldg(&ar.tile_r[b * ntx + a]) * inv_tile)));
                        if (max(abs(a - tx), abs(b - ty)) <= reach) {
                            any = true;
                            break;
                        }
                    }
            }
            s_on[ey][ex] = any ? 1 : 0;
        }
    }
    __syncthreads();
    int i = x0 + (threadIdx.x & 31), j = y0 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    const bool on = s_on[j / tile - ty0][i / tile - tx0] != 0;
    int s = on ? spp_max : 0;
    if (!on && variance_on) {
        float2 m = __ldg(&mv[q]);
        float fx = floorf((float)i - m.x + 0.5f), fy = floorf((float)j - m.y + 0.5f);
        int hl = 0;
        float m1 = 0.f, m2 = 0.f;
        if (fx >= 0.f && fy >= 0.f && fx < (float)W && fy < (float)H) {
            size_t t = (size_t)fy * W + (size_t)fx;
            hl = __ldg(&hhlen[t]);
            float2 mm = __ldg(&hmom[t]);
            m1 = mm.x;
            m2 = mm.y;
        }
        float sig = sqrtf(fmaxf(0.f, m2 - m1 * m1));
        bool young = hl < hlen_young;
        if (hl >= 1 && (young || sig > var_tau)) {
            if (young) s = spp_max;
            else s = (int)fminf(fmaxf(ceilf((float)spp_max * sig / var_scale), 1.f), (float)spp_max);
        }
    }
    spp[q] = (uint8_t)s;
}

__global__ void __launch_bounds__(256) k_mask_spp(SppArgs a) { mask_spp_body(a, blockIdx.x, blockIdx.y); }

GaussW gauss_weights(float sigma) {
    GaussW g;
    double w[5], sum = 0.0;
    for (int k = -2; k <= 2; ++k) {
        w[k + 2] = std::exp(-(double)(k * k) / (2.0 * (double)sigma * (double)sigma));
        sum += w[k + 2];
    }
    for (int k = 0; k < 5; ++k) g.w[k] = (float)(w[k] / sum);
    return g;
}

template <class ND>
EdgeArgs<ND> edge_args(const hdof_gbuf* in, const hdof_params* p, uint8_t* edge, uint8_t* tiles,
                       const Coc* coc = nullptr, float* tile_r = nullptr) {
    EdgeArgs<ND> a;
    a.nd = static_cast<const ND*>(in->nd);
    a.W = in->width;
    a.H = in->height;
    a.g = gauss_weights(p->gauss_sigma);
    a.tau = p->edge_tau;
    a.tile = p->tile;
    a.ntx = (in->width + p->tile - 1) / p->tile;
    a.edge = edge;
    a.tiles = tiles;
    a.coc = coc ? *coc : Coc{0.f, 0.f};
    a.rmax = p->r_max;
    a.tile_r = coc ? tile_r : nullptr;
    return a;
}

SppArgs spp_args(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p, const uint8_t* tiles,
                 uint8_t* spp, const float* tile_r = nullptr) {
    bool var = p->variance_on && prev_hist;
    SppArgs a;
    a.W = in->width;
    a.H = in->height;
    a.tile = p->tile;
    a.ntx = (in->width + p->tile - 1) / p->tile;
    a.nty = (in->height + p->tile - 1) / p->tile;
    a.dil = p->dilate;
    a.tiles = tiles;
    a.variance_on = var ? 1 : 0;
    a.mv = reinterpret_cast<const float2*>(in->mv);
    a.hmom = var ? reinterpret_cast<const float2*>(prev_hist->mom) : nullptr;
    a.hhlen = var ? prev_hist->hlen : nullptr;
    a.spp_max = p->spp_max;
    a.var_tau = p->var_tau;
    a.var_scale = p->var_scale;
    a.hlen_young = p->hlen_young;
    a.spp = spp;
    a.tile_r = tile_r;
    return a;
}

// launches of both kernels for one view (tiles already cleared)
// coc, tile_r: the CoC-scaled mask (both set) or the fixed dilation (both NULL)
int launch_mask(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p, uint8_t* edge, uint8_t* spp,
                uint8_t* tiles, cudaStream_t s, const Coc* coc = nullptr, float* tile_r = nullptr) {
    const int W = in->width, H = in->height;
    dim3 grid((W + B - 1) / B, (H + B - 1) / B);
    ProfScope ps_("mask", s);
    if (in->dtype_nd == HDOF_F32)
        k_mask_edge<float4><<<grid, 256, 0, s>>>(edge_args<float4>(in, p, edge, tiles, coc, tile_r));
    else
        k_mask_edge<half4s><<<grid, 256, 0, s>>>(edge_args<half4s>(in, p, edge, tiles, coc, tile_r));
    HDOF_LAUNCHED("mask: edge");
    dim3 g2((W + 31) / 32, (H + 7) / 8);
    k_mask_spp<<<g2, 256, 0, s>>>(spp_args(in, prev_hist, p, tiles, spp, coc ? tile_r : nullptr));
    HDOF_LAUNCHED("mask: spp");
    return HDOF_OK;
}

__global__ void __launch_bounds__(256) k_mask_edge_batch(const EdgeArgs<float4>* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    mask_edge_body(batch_record(a, v), bx, by);
}
__global__ void __launch_bounds__(256) k_mask_spp_batch(const SppArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    mask_spp_body(batch_record(a, v), bx, by);
}

}  // namespace
}  // namespace hdof

using namespace hdof;

extern "C" int hdof_mask(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p, uint8_t* edge,
                         uint8_t* spp, void* workspace, size_t workspace_bytes, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_params(p, "hdof_mask")) || (rc = check_gbuf(in, "hdof_mask", false))) return rc;
    HDOF_CHECK_ARG(!p->mask_coc, "hdof_mask: the CoC-scaled mask (mask_coc) needs the lens: call hdof_mask_coc");
    HDOF_CHECK_ARG(edge && spp, "hdof_mask: edge and spp outputs are required");
    const int W = in->width, H = in->height;
    bool var = p->variance_on && prev_hist;
    HDOF_CHECK_ARG(!var || (prev_hist->mom && prev_hist->hlen && in->mv),
                   "hdof_mask: the variance term needs mv and the history mom/hlen planes");
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.mask_tiles, "hdof_mask: workspace of %zu bytes < %zu",
                   workspace_bytes, L.mask_tiles);
    cudaStream_t s = as_stream(stream);
    const int T = p->tile, ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    uint8_t* tiles = static_cast<uint8_t*>(workspace);
    HDOF_CUDA(cudaMemsetAsync(tiles, 0, (size_t)ntx * nty, s), "hdof_mask: clear tiles");
    return launch_mask(in, prev_hist, p, edge, spp, tiles, s);
}

extern "C" int hdof_mask_coc(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_camera* cam,
                             const hdof_lens* lens, const hdof_params* p, uint8_t* edge, uint8_t* spp,
                             void* workspace, size_t workspace_bytes, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_params(p, "hdof_mask_coc")) || (rc = check_gbuf(in, "hdof_mask_coc", false)) ||
        (rc = check_camera(cam, "hdof_mask_coc")) || (rc = check_lens(lens, "hdof_mask_coc")))
        return rc;
    HDOF_CHECK_ARG(edge && spp, "hdof_mask_coc: edge and spp outputs are required");
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height, "hdof_mask_coc: gbuf/camera size mismatch");
    const int W = in->width, H = in->height;
    bool var = p->variance_on && prev_hist;
    HDOF_CHECK_ARG(!var || (prev_hist->mom && prev_hist->hlen && in->mv),
                   "hdof_mask_coc: the variance term needs mv and the history mom/hlen planes");
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.mask_tiles + L.mask_tile_r,
                   "hdof_mask_coc: workspace of %zu bytes < %zu", workspace_bytes, L.mask_tiles + L.mask_tile_r);
    cudaStream_t s = as_stream(stream);
    const int T = p->tile, ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    uint8_t* tiles = static_cast<uint8_t*>(workspace);
    float* tile_r = reinterpret_cast<float*>(static_cast<char*>(workspace) + L.mask_tiles);
    HDOF_CUDA(cudaMemsetAsync(tiles, 0, p->mask_coc ? L.mask_tiles + (size_t)ntx * nty * sizeof(float)
                                                    : (size_t)ntx * nty, s),
              "hdof_mask_coc: clear tiles");
    if (!p->mask_coc) return launch_mask(in, prev_hist, p, edge, spp, tiles, s);
    const Coc coc = make_coc(*lens, cam->height, cam->tan_half_fovy);
    return launch_mask(in, prev_hist, p, edge, spp, tiles, s, &coc, tile_r);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of hdof_mask.
//
// Some callers cannot hand this library any scratch memory: a real-time
// render thread that must never call cudaMalloc/cudaFree (they can
// synchronise the whole device and stall the frame), or a host application
// that owns all device memory through its own arena and gives plug-ins no
// allocator.  For them the mask's only scratch -- one flag byte per mask
// tile -- lives in a fixed file-scope device array instead of the caller's
// workspace.  The array is sized for HDOF_MASK_NOALLOC_MAX_TILES tiles and
// stays resident on every device that loads the library until the process
// exits.  Host code cannot use the array's name as a device address, so its
// address is looked up once per device with cudaGetSymbolAddress.
namespace hdof {
namespace {

static __device__ __align__(256) uint8_t g_mask_tiles_noalloc[HDOF_MASK_NOALLOC_MAX_TILES];

std::mutex g_noalloc_mu;
uint8_t* g_noalloc_ptr[64] = {nullptr};

// device address of g_mask_tiles_noalloc on the current device (looked up once)
int noalloc_tiles(uint8_t** out) {
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "hdof_mask_noalloc: device");
    if (dev < 0 || dev >= 64) {
        set_error("hdof_mask_noalloc: device index %d unsupported", dev);
        return HDOF_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        HDOF_CUDA(cudaGetSymbolAddress(&p, g_mask_tiles_noalloc), "hdof_mask_noalloc: symbol address");
        g_noalloc_ptr[dev] = static_cast<uint8_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return HDOF_OK;
}

}  // namespace
}  // namespace hdof

extern "C" int hdof_mask_noalloc(const hdof_gbuf* in, const hdof_history* prev_hist, const hdof_params* p,
                                 uint8_t* edge, uint8_t* spp, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_params(p, "hdof_mask_noalloc")) || (rc = check_gbuf(in, "hdof_mask_noalloc", false))) return rc;
    HDOF_CHECK_ARG(!p->mask_coc, "hdof_mask_noalloc: the CoC-scaled mask (mask_coc) is not available here");
    HDOF_CHECK_ARG(edge && spp, "hdof_mask_noalloc: edge and spp outputs are required");
    const int W = in->width, H = in->height;
    bool var = p->variance_on && prev_hist;
    HDOF_CHECK_ARG(!var || (prev_hist->mom && prev_hist->hlen && in->mv),
                   "hdof_mask_noalloc: the variance term needs mv and the history mom/hlen planes");
    const int T = p->tile, ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    HDOF_CHECK_ARG((long long)ntx * nty <= HDOF_MASK_NOALLOC_MAX_TILES,
                   "hdof_mask_noalloc: %d x %d mask tiles exceed the fixed capacity of %d tiles", ntx, nty,
                   HDOF_MASK_NOALLOC_MAX_TILES);
    uint8_t* tiles = nullptr;
    if ((rc = noalloc_tiles(&tiles))) return rc;
    cudaStream_t s = as_stream(stream);
    // the array keeps the previous call's flags: clear the tiles this call uses
    HDOF_CUDA(cudaMemsetAsync(tiles, 0, (size_t)ntx * nty, s), "hdof_mask_noalloc: clear tiles");
    return launch_mask(in, prev_hist, p, edge, spp, tiles, s);
}

namespace hdof {

size_t mask_edge_args_size() { return sizeof(EdgeArgs<float4>); }
void mask_edge_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const Coc coc = make_coc(v.lens, v.cam.height, v.cam.tan_half_fovy);
    *reinterpret_cast<EdgeArgs<float4>*>(dst) =
        edge_args<float4>(&v.g, &v.params, v.edge, w.tiles, v.params.mask_coc ? &coc : nullptr, w.tile_r);
    *gx = (v.g.width + B - 1) / B;
    *gy = (v.g.height + B - 1) / B;
}
void mask_edge_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_mask_edge", s);
    k_mask_edge_batch<<<blocks, 256, 0, s>>>(static_cast<const EdgeArgs<float4>*>(args), g);
}

size_t mask_spp_args_size() { return sizeof(SppArgs); }
void mask_spp_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    *reinterpret_cast<SppArgs*>(dst) =
        spp_args(&v.g, &v.hist_in, &v.params, w.tiles, v.spp, v.params.mask_coc ? w.tile_r : nullptr);
    *gx = (v.g.width + 31) / 32;
    *gy = (v.g.height + 7) / 8;
}
void mask_spp_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_mask_spp", s);
    k_mask_spp_batch<<<blocks, 256, 0, s>>>(static_cast<const SppArgs*>(args), g);
}

}  // namespace hdof
