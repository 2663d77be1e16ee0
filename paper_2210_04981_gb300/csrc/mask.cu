// adaptive ray mask (Ray Trace section): the G-buffer is smoothed by a
// Gaussian before a Sobel gradient of its normal and depth marks geometry
// edges (the smoothing suppresses noise and staircase edges, as in Canny's
// detector); a luminance variance accumulated over previous frames adds rays
// where the traced result is still noisy or has just appeared.
//
// k_mask_sweep: a warp walks down a strip of 32 columns (26 output columns
//   plus the 3-pixel halos), one column per lane, keeping the separable 5-tap
//   Gaussian and the 1/8-scaled 3x3 Sobel in registers (neighbour columns by
//   warp shuffles, neighbour rows by register rings): no shared memory, each
//   input pixel loaded once per strip.  Writes edge bits, marks the mask tiles
//   that hold an edge and (CoC-scaled mask) their pixels' largest CoC radius.
// k_mask_spp: per pixel, dilated tile flag and the variance term -> spp.
#include <cmath>
#include <mutex>

#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {


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

// ---- register sweep form of the edge pass ----------------------------------
// A warp owns a strip of 32 input columns (x0 - 3 .. x0 + 28) and SW_ROWS
// output rows; it walks down the strip one input row at a time, lane = column:
//   horizontal Gaussian of the new row from its +-1, +-2 neighbours (shuffles),
//   vertical Gaussian from a ring of the last five horizontally filtered rows,
//   per filtered row its horizontal Sobel difference f(x+1) - f(x-1) and
//   smoothing f(x-1) + 2 f(x) + f(x+1) (+-1 shuffles, clamp-to-edge of the
//   filtered image at the image border), and per output row the Sobel
//   gradients from the last three of those.  Lanes 3..28 hold the 26 output
//   columns.  Nothing goes through shared memory; each input pixel is loaded
//   once per strip (plus the 3-pixel halos).  Edge flags and CoC radii are
//   reduced per mask tile in registers and written once per tile row.
constexpr int SW_OUT = 26;   // output columns per warp
constexpr int SW_ROWS = 32;  // output rows per warp
constexpr int SW_WARPS = 4;  // warps per block (side by side)

// float4 arithmetic as two packed two-lane FP32 operations (Blackwell's
// f32x2 forms: one instruction for two lanes, each rounded as its scalar form)
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\tfma.rn.f32x2 pr, pa, pb, pc;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
struct V4 {
    float2 a, b;  // (x, y), (z, w)
};
__device__ __forceinline__ V4 v4(float4 v) { return V4{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ V4 fma4(float w, V4 v, V4 c) {
    const float2 ww = make_float2(w, w);
    return V4{pk_fma(ww, v.a, c.a), pk_fma(ww, v.b, c.b)};
}
__device__ __forceinline__ V4 mul4(float w, V4 v) { return fma4(w, v, V4{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}); }
__device__ __forceinline__ V4 add4(V4 x, V4 y) { return V4{pk_add(x.a, y.a), pk_add(x.b, y.b)}; }
__device__ __forceinline__ V4 sub4(V4 x, V4 y) { return V4{pk_sub(x.a, y.a), pk_sub(x.b, y.b)}; }

// flush a lane's per-tile edge flag and radius for tile row ty: lanes with the
// same tile column combine, one lane per tile writes
template <class ND>
__device__ __forceinline__ void sw_flush(const EdgeArgs<ND>& ar, int ty, int tx, bool valid, bool& any_edge,
                                         float& rmax) {
    const unsigned grp = __match_any_sync(0xffffffffu, valid ? tx : -1);
    const unsigned e = __ballot_sync(0xffffffffu, any_edge) & grp;
    unsigned rb = __reduce_max_sync(grp, __float_as_uint(rmax));
    const int lane = threadIdx.x & 31;
    if (valid && lane == __ffs(grp) - 1) {
        if (e) ar.tiles[ty * ar.ntx + tx] = 1;
        if (ar.tile_r && rb) atomicMax(reinterpret_cast<unsigned*>(ar.tile_r) + ty * ar.ntx + tx, rb);
    }
    any_edge = false;
    rmax = 0.f;
}

template <class ND>
__device__ __forceinline__ void mask_sweep_body(const EdgeArgs<ND>& ar, int bx, int by) {
    const int W = ar.W, H = ar.H, tile = ar.tile;
    const GaussW g = ar.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = (bx * SW_WARPS + warp) * SW_OUT;  // first output column of the strip
    if (x0 >= W) return;                                // a whole warp leaves together
    const int y0 = by * SW_ROWS, y1 = min(y0 + SW_ROWS, H);
    const int x = x0 - 3 + lane;                      // this lane's column (may lie outside the image)
    const int xc = min(max(x, 0), W - 1);
    const bool out_lane = lane >= 3 && lane < 3 + SW_OUT && x < W;
    // neighbour columns through the warp's own shared row (one 128-bit store,
    // 128-bit loads): Gaussian taps at lane -2..+2 (clamped to the warp; only
    // lanes 2..29 need complete sums), Sobel taps at lane -1, +1 with the
    // filtered image's clamp-to-edge at the image border
    __shared__ float4 s_row[SW_WARPS][32];
    float4* srow = s_row[warp];
    const int lm2 = max(lane - 2, 0), lm1 = max(lane - 1, 0), lp1 = min(lane + 1, 31), lp2 = min(lane + 2, 31);
    const int sl = x == 0 ? lane : lm1, sr = x == W - 1 ? lane : lp1;
    const int tx = out_lane ? x / tile : -1;
    const float tau64 = 64.f * ar.tau * ar.tau;
    const V4 zero4{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    // vertical Gaussian as running sums: A0..A3 hold the partial sums of the
    // filtered rows yi-2 .. yi+1 (their taps from the rows read so far)
    V4 A0 = zero4, A1 = zero4, A2 = zero4, A3 = zero4;
    // Sobel as running sums over the filtered rows: P = D(j-1) + 2 D(j),
    // Q = D(j), Sm = S(j-1), S0 = S(j) (D: horizontal difference, S: horizontal
    // smoothing of a filtered row)
    V4 P = zero4, Q = zero4, Sm = zero4, S0 = zero4;
    float zj = 1.f;  // filtered depth of row j at this column
    bool any_edge = false;
    float rmax = 0.f;
    int cur_ty = y0 / tile, next_row = (cur_ty + 1) * tile;
    // three rows in flight ahead of the one being filtered (loads of rows past
    // the strip's end read clamped, valid rows and are not used)
    auto row = [&](int y) { return ld4(ar.nd + (size_t)min(max(y, 0), H - 1) * W + xc); };
    float4 va = row(y0 - 3), vb = row(y0 - 2), vc = row(y0 - 1);
    for (int yi = y0 - 3; yi <= y1 + 2; ++yi) {
        const float4 v = va;
        va = vb;
        vb = vc;
        vc = row(yi + 3);
        // horizontal Gaussian of input row yi (lanes 2..29 complete)
        __syncwarp();
        srow[lane] = v;
        __syncwarp();
        V4 h = mul4(g.w[0], v4(srow[lm2]));
        h = fma4(g.w[1], v4(srow[lm1]), h);
        h = fma4(g.w[2], v4(v), h);
        h = fma4(g.w[3], v4(srow[lp1]), h);
        h = fma4(g.w[4], v4(srow[lp2]), h);
        // its taps into the running vertical sums; filtered row yi - 2 completes
        const V4 f = fma4(g.w[4], h, A0);
        A0 = fma4(g.w[3], h, A1);
        A1 = fma4(g.w[2], h, A2);
        A2 = fma4(g.w[1], h, A3);
        A3 = mul4(g.w[0], h);
        if (yi < y0 + 1) continue;  // the first filtered row the Sobel needs is y0 - 1 = yi - 2
        // Sobel row terms of filtered row fy = yi - 2
        __syncwarp();
        srow[lane] = make_float4(f.a.x, f.a.y, f.b.x, f.b.y);
        __syncwarp();
        const V4 fl = v4(srow[sl]), fr = v4(srow[sr]);
        const V4 Dn = sub4(fr, fl);
        const V4 Sn = fma4(2.f, f, add4(fl, fr));
        if (yi < y0 + 3) {  // filtered rows y0 - 1 and y0: prime the running sums
            P = fma4(2.f, Dn, Q);
            Q = Dn;
            Sm = S0;
            S0 = Sn;
            zj = f.b.y;
            continue;
        }
        // output row j = yi - 3 from filtered rows j - 1 (in P, Sm), j (Q, S0) and j + 1 (new);
        // rows j - 1 and j + 1 clamped to the image (the Sobel's border rule)
        const int j = yi - 3;
        V4 gx, gy;
        if (j == 0 && j == H - 1) {  // a one-row image: both neighbours are the row itself
            gx = mul4(4.f, Q);
            gy = zero4;
        } else if (j == 0) {
            gx = add4(fma4(2.f, Q, Q), Dn);
            gy = sub4(Sn, S0);
        } else if (j == H - 1) {
            gx = add4(P, Q);
            gy = sub4(S0, Sm);
        } else {
            gx = add4(P, Dn);
            gy = sub4(Sn, Sm);
        }
        const float zc = zj;
        P = fma4(2.f, Dn, Q);
        Q = Dn;
        Sm = S0;
        S0 = Sn;
        zj = f.b.y;
        if (j >= next_row) {
            sw_flush(ar, cur_ty, tx, out_lane, any_edge, rmax);
            cur_ty = j / tile;
            next_row = (cur_ty + 1) * tile;
        }
        // e = max(|grad n|, |grad z| / z~) > tau with the Sobel's 1/8 scale folded
        // into the threshold and both sides squared (no square root, no divide):
        // |8 grad n|^2 > 64 tau^2  or  |8 grad z|^2 > 64 tau^2 z~^2
        const float en2 = fmaf(gx.a.x, gx.a.x, fmaf(gy.a.x, gy.a.x, fmaf(gx.a.y, gx.a.y, fmaf(gy.a.y, gy.a.y,
                          fmaf(gx.b.x, gx.b.x, gy.b.x * gy.b.x)))));
        const float ez2 = fmaf(gx.b.y, gx.b.y, gy.b.y * gy.b.y);
        const bool bit = en2 > tau64 || ez2 > tau64 * zc * zc;
        if (out_lane) {
            ar.edge[(size_t)j * W + x] = bit ? 1 : 0;
            any_edge |= bit;
            if (ar.tile_r) rmax = fmaxf(rmax, fminf(fabsf(ar.coc(ldz(ar.nd + (size_t)j * W + x))) * 0.5f, ar.rmax));
        }
    }
    sw_flush(ar, cur_ty, tx, out_lane, any_edge, rmax);
}

template <class ND>
__global__ void __launch_bounds__(SW_WARPS * 32, 6) k_mask_sweep(EdgeArgs<ND> a) {
    mask_sweep_body(a, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(SW_WARPS * 32, 6) k_mask_sweep_batch(const EdgeArgs<float4>* __restrict__ a,
                                                                     BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    mask_sweep_body(batch_record(a, v), bx, by);
}
// grid of the sweep for a W x H frame
inline dim3 sweep_grid(int W, int H) {
    return dim3((W + SW_OUT * SW_WARPS - 1) / (SW_OUT * SW_WARPS), (H + SW_ROWS - 1) / SW_ROWS);
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

// rays of pixel (i, j) that is not in a traced tile: the variance term
__device__ __forceinline__ int variance_spp(const SppArgs& ar, int i, int j, float2 m) {
    const int W = ar.W, H = ar.H;
    float fx = floorf((float)i - m.x + 0.5f), fy = floorf((float)j - m.y + 0.5f);
    int hl = 0;
    float m1 = 0.f, m2 = 0.f;
    if (fx >= 0.f && fy >= 0.f && fx < (float)W && fy < (float)H) {
        size_t t = (size_t)fy * W + (size_t)fx;
        hl = __ldg(&ar.hhlen[t]);
        float2 mm = __ldg(&ar.hmom[t]);
        m1 = mm.x;
        m2 = mm.y;
    }
    float sig = sqrtf(fmaxf(0.f, m2 - m1 * m1));
    bool young = hl < ar.hlen_young;
    int s = 0;
    if (hl >= 1 && (young || sig > ar.var_tau)) {
        if (young) s = ar.spp_max;
        else s = (int)fminf(fmaxf(ceilf((float)ar.spp_max * sig / ar.var_scale), 1.f), (float)ar.spp_max);
    }
    return s;
}

// block = 128 x 8 pixels, 4 consecutive pixels per thread (vector loads of
// the motion vectors, one 4-byte store of the rays; the history reads of
// the variance term are independent, so four are in flight per thread)
constexpr int SPP_BX = 128, SPP_BY = 8;
__device__ __forceinline__ void mask_spp_body(const SppArgs& ar, int bx, int by) {
    const int W = ar.W, H = ar.H, tile = ar.tile, ntx = ar.ntx, nty = ar.nty, dil = ar.dil;
    const uint8_t* __restrict__ tiles = ar.tiles;
    // the dilated flag of every mask tile this block touches, once, in shared
    // memory (at most 128 x 8 tiles, for tile = 1)
    __shared__ unsigned char s_on[SPP_BY][SPP_BX];
    const int x0 = bx * SPP_BX, y0 = by * SPP_BY;
    const int tx0 = x0 / tile, ty0 = y0 / tile;
    const int ntx_b = min(x0 + SPP_BX - 1, W - 1) / tile - tx0 + 1, nty_b = min(y0 + SPP_BY - 1, H - 1) / tile - ty0 + 1;
    // this thread's pixels and their motion vectors first: the loads are in
    // flight while the block builds its tile flags
    const int i0 = x0 + 4 * (threadIdx.x & 31), j = y0 + (threadIdx.x >> 5);
    const bool live = i0 < W && j < H;
    const size_t q = live ? (size_t)j * W + i0 : 0;
    const bool full = live && i0 + 3 < W && (q & 3) == 0;  // four pixels, 4-byte aligned row position
    float2 m[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (live && ar.variance_on) {
        if (full) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(ar.mv + q));
            const float4 b = __ldg(reinterpret_cast<const float4*>(ar.mv + q + 2));
            m[0] = make_float2(a.x, a.y);
            m[1] = make_float2(a.z, a.w);
            m[2] = make_float2(b.x, b.y);
            m[3] = make_float2(b.z, b.w);
        } else {
            for (int k = 0; k < 4; ++k)
                if (i0 + k < W) m[k] = __ldg(&ar.mv[q + k]);
        }
    }
    for (int e = threadIdx.x; e < ntx_b * nty_b; e += 256) {
        const int ey = e / ntx_b, ex = e % ntx_b;
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
                    const int reach = min(8, max(dil, (int)ceilf(__ldg(&ar.tile_r[b * ntx + a]) * inv_tile)));
                    if (max(abs(a - tx), abs(b - ty)) <= reach) {
                        any = true;
                        break;
                    }
                }
        }
        s_on[ey][ex] = any ? 1 : 0;
    }
    __syncthreads();
    if (i0 >= W || j >= H) return;
    uint8_t out[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = i0 + k;
        int sp = 0;
        if (i < W) {
            const bool on = s_on[j / tile - ty0][i / tile - tx0] != 0;
            sp = on ? ar.spp_max : (ar.variance_on ? variance_spp(ar, i, j, m[k]) : 0);
        }
        out[k] = (uint8_t)sp;
    }
    if (full) {
        *reinterpret_cast<uchar4*>(ar.spp + q) = make_uchar4(out[0], out[1], out[2], out[3]);
    } else {
        for (int k = 0; k < 4; ++k)
            if (i0 + k < W) ar.spp[q + k] = out[k];
    }
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
    const dim3 grid = sweep_grid(W, H);
    ProfScope ps_("mask", s);
    if (in->dtype_nd == HDOF_F32)
        k_mask_sweep<float4><<<grid, SW_WARPS * 32, 0, s>>>(edge_args<float4>(in, p, edge, tiles, coc, tile_r));
    else
        k_mask_sweep<half4s><<<grid, SW_WARPS * 32, 0, s>>>(edge_args<half4s>(in, p, edge, tiles, coc, tile_r));
    HDOF_LAUNCHED("mask: edge");
    dim3 g2((W + SPP_BX - 1) / SPP_BX, (H + SPP_BY - 1) / SPP_BY);
    k_mask_spp<<<g2, 256, 0, s>>>(spp_args(in, prev_hist, p, tiles, spp, coc ? tile_r : nullptr));
    HDOF_LAUNCHED("mask: spp");
    return HDOF_OK;
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
    const dim3 sg = sweep_grid(v.g.width, v.g.height);
    *gx = (int)sg.x;
    *gy = (int)sg.y;
}
void mask_edge_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_mask_edge", s);
    k_mask_sweep_batch<<<blocks, SW_WARPS * 32, 0, s>>>(static_cast<const EdgeArgs<float4>*>(args), g);
}

size_t mask_spp_args_size() { return sizeof(SppArgs); }
void mask_spp_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    *reinterpret_cast<SppArgs*>(dst) =
        spp_args(&v.g, &v.hist_in, &v.params, w.tiles, v.spp, v.params.mask_coc ? w.tile_r : nullptr);
    *gx = (v.g.width + SPP_BX - 1) / SPP_BX;
    *gy = (v.g.height + SPP_BY - 1) / SPP_BY;
}
void mask_spp_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_mask_spp", s);
    k_mask_spp_batch<<<blocks, 256, 0, s>>>(static_cast<const SppArgs*>(args), g);
}

}  // namespace hdof
