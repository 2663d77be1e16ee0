// spatio-temporal reconstruction of the ray-traced layers
// (Reconstruction section).
//
// Temporal (k_temporal, one thread per pixel): near and far colours are
// accumulated separately with an exponential moving average, each weighted
// by its share of the hit ratio.  Near terms are reprojected with the
// screen-space motion vector; far terms with the previous-frame projection
// of the average far world position of the pixel's far hits (or of its
// neighbours' when it has none, or of its G-buffer surface).  The composed
// colour uses this frame's hit ratio when the camera moved and the
// accumulated one otherwise; each layer is normalised by its accumulated
// hit-ratio weight.  The reconstructed CoC blends this frame's near and far
// CoC by the accumulated hit ratio.
//
// Spatial (k_spatial, one thread per traced pixel): a circular gather scaled
// by the pixel's CoC that rejects samples whose CoC radius is smaller than
// their distance, blended by the clamped luminance variance so converged
// regions are not over-blurred.
#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

struct TemporalArgs {
    Cam cam, prev;
    int W, H;
    float alpha, alpha_k;  // EMA weight; per-pixel blend factor threshold (0 = fixed weight)
    int moved;
    const float4* rt;  // 3 per pixel
    const uint8_t* spp;
    const float2* mv;
    const float4* hn;  // previous history
    const float4* hf;
    const float2* hm;
    const uint8_t* hl;
    float4* on;  // new history
    float4* of;
    float2* om;
    uint8_t* ol;
    float4* crt;
    float* hacc;
};

__device__ __forceinline__ void acc(float4& o, float w, float4 v) {
    o.x = fmaf(w, v.x, o.x);
    o.y = fmaf(w, v.y, o.y);
    o.z = fmaf(w, v.z, o.z);
    o.w = fmaf(w, v.w, o.w);
}
__device__ __forceinline__ void acc(float2& o, float w, float2 v) {
    o.x = fmaf(w, v.x, o.x);
    o.y = fmaf(w, v.y, o.y);
}
__device__ __forceinline__ void scale(float4& o, float s) {
    o.x *= s;
    o.y *= s;
    o.z *= s;
    o.w *= s;
}
__device__ __forceinline__ void scale(float2& o, float s) {
    o.x *= s;
    o.y *= s;
}
__device__ __forceinline__ void zero(float4& o) { o = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero(float2& o) { o = make_float2(0.f, 0.f); }

// bilinear history sample over taps that hold history (hlen > 0), renormalised;
// invalid below a total tap weight of 1e-3.  hmax: largest hlen among taps
// with non-zero weight.
template <class T>
__device__ __forceinline__ bool hist_sample(const TemporalArgs& a, float ux, float uy, const T* plane, T& out,
                                            int* hmax) {
    float x0 = floorf(ux), y0 = floorf(uy), fx = ux - x0, fy = uy - y0;
    float ws = 0.f;
    zero(out);
    if (hmax) *hmax = 0;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float x = x0 + c, y = y0 + b;
            if (x < 0.f || y < 0.f || x >= (float)a.W || y >= (float)a.H) continue;
            size_t q = (size_t)y * a.W + (size_t)x;
            int hl = __ldg(&a.hl[q]);
            if (hl == 0) continue;
            float w = (c ? fx : 1.f - fx) * (b ? fy : 1.f - fy);
            ws += w;
            acc(out, w, __ldg(&plane[q]));
            if (hmax && w > 0.f && hl > *hmax) *hmax = hl;
        }
    if (!(ws >= HDOF_HIST_MIN_W)) return false;
    scale(out, 1.f / ws);
    return true;
}

template <class ND>
__device__ __forceinline__ void temporal_body(const TemporalArgs& a, const ND* __restrict__ nd, int bx, int by) {
    int i = bx * 32 + (threadIdx.x & 31), j = by * 8 + (threadIdx.x >> 5);
    if (i >= a.W || j >= a.H) return;
    size_t q = (size_t)j * a.W + i;
    if (a.spp[q] == 0) {
        a.ol[q] = 0;
        a.crt[q] = make_float4(0.f, 0.f, 0.f, -1.f);
        return;
    }
    const float4 r0 = __ldg(&a.rt[3 * q]), r1 = __ldg(&a.rt[3 * q + 1]), r2 = __ldg(&a.rt[3 * q + 2]);
    const float h = r0.w, cn = r1.w, cf = r2.w;
    const bool nok = cn >= 0.f, fok = cf >= 0.f;
    float3 Cn = f3(r0.x, r0.y, r0.z), Cf = f3(r1.x, r1.y, r1.z);
    float3 Ccur = nok ? (fok ? h * Cn + (1.f - h) * Cf : Cn) : Cf;
    float Y = luminance(Ccur);
    // near reprojection
    float2 m = __ldg(&a.mv[q]);
    float un = (float)i - m.x, vn = (float)j - m.y;
    float4 hn;
    float2 hm = make_float2(0.f, 0.f);
    int hl = 0;
    bool vn_ok = hist_sample(a, un, vn, a.hn, hn, &hl);
    if (vn_ok) hist_sample(a, un, vn, a.hm, hm, (int*)nullptr);
    // far world position
    float3 P;
    if (fok) {
        P = f3(r2.x, r2.y, r2.z);
    } else {
        float3 s = f3(0.f, 0.f, 0.f);
        int cnt = 0;
        for (int b = -1; b <= 1; ++b)
            for (int c = -1; c <= 1; ++c) {
                if (!b && !c) continue;
                int x = i + c, y = j + b;
                if (x < 0 || y < 0 || x >= a.W || y >= a.H) continue;
                size_t qq = (size_t)y * a.W + x;
                if (a.spp[qq] == 0) continue;
                float4 p2 = __ldg(&a.rt[3 * qq + 2]);
                if (p2.w < 0.f) continue;
                s = s + f3(p2.x, p2.y, p2.z);
                ++cnt;
            }
        if (cnt > 0) {
            P = (1.f / (float)cnt) * s;
        } else {
            float3 d = pinhole_dir(a.cam, i + 0.5f + a.cam.jx, j + 0.5f + a.cam.jy);
            P = a.cam.pos + ldz(nd + q) * d;
        }
    }
    float uf, vf;
    float4 hf;
    bool vf_ok = project(a.prev, P, uf, vf) && hist_sample(a, uf, vf, a.hf, hf, (int*)nullptr);
    // EMA weight: fixed, or per pixel from the temporal gradient (the paper's
    // per-pixel blend factors against ghosting): the larger of this frame's
    // luminance change against the reprojected history beyond alpha_k of its
    // per-frame spread (relative to the larger luminance) and the hit ratio's
    // change beyond alpha_k binomial standard errors; alpha rises towards 1
    float al = a.alpha;
    if (a.alpha_k > 0.f && vn_ok) {
        const float sg = sqrtf(fmaxf(0.f, hm.y - hm.x * hm.x));
        const float den = fmaxf(fmaxf(Y, hm.x), 1e-3f);
        float lam = fminf(fmaxf((fabsf(Y - hm.x) - a.alpha_k * sg) / den, 0.f), 1.f);
        const float hb = hn.w, se = sqrtf(fmaxf(hb * (1.f - hb), 0.f) / (float)a.spp[q]);
        const float lh = fminf(fmaxf(fabsf(h - hb) - a.alpha_k * se, 0.f), 1.f);
        lam = fmaxf(lam, lh);
        al = fmaf(1.f - al, lam, al);
    }
    float4 cur_n = make_float4(h * Cn.x, h * Cn.y, h * Cn.z, h);
    float4 cur_f = make_float4((1.f - h) * Cf.x, (1.f - h) * Cf.y, (1.f - h) * Cf.z, 1.f - h);
    float4 on = vn_ok ? make_float4(fmaf(al, cur_n.x - hn.x, hn.x), fmaf(al, cur_n.y - hn.y, hn.y),
                                    fmaf(al, cur_n.z - hn.z, hn.z), fmaf(al, cur_n.w - hn.w, hn.w))
                      : cur_n;
    float4 of = vf_ok ? make_float4(fmaf(al, cur_f.x - hf.x, hf.x), fmaf(al, cur_f.y - hf.y, hf.y),
                                    fmaf(al, cur_f.z - hf.z, hf.z), fmaf(al, cur_f.w - hf.w, hf.w))
                      : cur_f;
    float2 om = vn_ok ? make_float2(fmaf(al, Y - hm.x, hm.x), fmaf(al, Y * Y - hm.y, hm.y)) : make_float2(Y, Y * Y);
    int nh = vn_ok ? hl + 1 : 1;
    a.on[q] = on;
    a.of[q] = of;
    a.om[q] = om;
    a.ol[q] = (uint8_t)(nh > 255 ? 255 : nh);
    // accumulated hit ratio and composition
    float Bn = on.w, Bf = of.w;
    float Hacc = (Bn + Bf >= HDOF_EMPTY_W) ? Bn / (Bn + Bf) : h;
    bool an = Bn >= HDOF_EMPTY_W, af = Bf >= HDOF_EMPTY_W;
    float hw = a.moved ? h : Hacc;
    float3 CnA = an ? (1.f / Bn) * f3(on.x, on.y, on.z) : f3(0, 0, 0);
    float3 CfA = af ? (1.f / Bf) * f3(of.x, of.y, of.z) : f3(0, 0, 0);
    float3 C = !an ? CfA : (!af ? CnA : hw * CnA + (1.f - hw) * CfA);
    float crt_c = !nok ? cf : (!fok ? cn : Hacc * cn + (1.f - Hacc) * cf);
    a.crt[q] = make_float4(C.x, C.y, C.z, crt_c);
    a.hacc[q] = Hacc;
}

template <class ND>
__global__ void __launch_bounds__(256) k_temporal(TemporalArgs a, const ND* __restrict__ nd) {
    temporal_body(a, nd, blockIdx.x, blockIdx.y);
}

struct TemporalBatch {
    TemporalArgs t;
    const float4* nd;
};
__global__ void __launch_bounds__(256) k_temporal_batch(const TemporalBatch* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    const TemporalBatch& r = batch_record(a, v);
    temporal_body(r.t, r.nd, bx, by);
}

#ifndef HDOF_SP_UNROLL
#define HDOF_SP_UNROLL 4  // unroll of the spatial gather's tap loop
#endif
constexpr int SP_UNROLL = HDOF_SP_UNROLL;

struct SpatialArgs {
    const float4* crt;
    const float2* mom;
    const uint8_t* hlen;
    int W, H;
    float r_s, var_ref;
    float4* crec;
    float4* aux;
};

// a traced pixel's reconstructed colour from its gathered sums: blended with
// its own by beta = clamp(sigma_L / var_ref, 0, 1) (1 while its history is young)
__device__ __forceinline__ void spatial_finish(const SpatialArgs& a, size_t q, const float4& cp, const float3& S,
                                               float Ws) {
    float2 m = __ldg(&a.mom[q]);
    float sig = sqrtf(fmaxf(0.f, m.y - m.x * m.x));
    float beta = __ldg(&a.hlen[q]) < 2 ? 1.f : clamp01(sig / a.var_ref);
    float3 Csp = (1.f / Ws) * S;
    if (a.aux) a.aux[q] = make_float4(Csp.x, Csp.y, Csp.z, Ws);  // kept for the adjoint
    a.crec[q] = make_float4(cp.x + beta * (Csp.x - cp.x), cp.y + beta * (Csp.y - cp.y), cp.z + beta * (Csp.z - cp.z),
                            0.f);
}

// the spatial gather of one traced pixel (i, j)
__device__ __forceinline__ void spatial_pixel(const SpatialArgs& a, int i, int j) {
    const float4* __restrict__ crt = a.crt;
    const int W = a.W, H = a.H;
    const float r_s = a.r_s;
    const size_t q = (size_t)j * W + i;
    const float4 cp = __ldg(&crt[q]);
    const float rp = fminf(cp.w * 0.5f, r_s);
    // a tap weighs only if d < R = rp + 1/2: per row, the columns of that
    // disk (the bounds lean outwards by 1e-3 pixel; the taps they add weigh 0)
    const float R = rp + 0.5f, R2 = R * R;
    const int K = (int)floorf(R + 1e-3f);
    // s(r - d) = clamp(r + 1/2 - d, 0, 1): the half folded into the radii
    // (R here; for the neighbour min(c/2 + 1/2, r_s + 1/2))
    const float Rq = r_s + 0.5f;
    float3 S = f3(0, 0, 0);
    float Ws = 0.f;
    const int y0 = max(j - K, 0), y1 = min(j + K, H - 1);
    for (int y = y0; y <= y1; ++y) {
        const float dy = (float)(y - j), dy2 = dy * dy;
        const int wr = (int)floorf(sqrtf(fmaxf(R2 - dy2, 0.f)) + 1e-3f);
        const int x0 = max(i - wr, 0), x1 = min(i + wr, W - 1);
        const float4* row = crt + (size_t)y * W;
        float dx = (float)(x0 - i);
#pragma unroll SP_UNROLL
        for (int x = x0; x <= x1; ++x, dx += 1.f) {
            const float4 c = __ldg(&row[x]);
            const float d = sqrt_approx(fmaf(dx, dx, dy2));
            // an untraced neighbour (written as (0, 0, 0, -1)) weighs
            // clamp(-d, 0, 1) = 0 times colour 0: it adds nothing
            const float wq = clamp01(R - d) * clamp01(fminf(fmaf(c.w, 0.5f, 0.5f), Rq) - d);
            S.x = fmaf(wq, c.x, S.x);
            S.y = fmaf(wq, c.y, S.y);
            S.z = fmaf(wq, c.z, S.z);
            Ws += wq;
        }
    }
    spatial_finish(a, q, cp, S, Ws);
}

// One thread gathers the horizontally adjacent pixels (i, j) and (i + 1, j)
// (tl, tr: which of them is traced) over the union of their windows: each
// tap is loaded once, and the right pixel's distance to a tap is the left
// pixel's distance to the previous tap (the same float operations), so both
// sums equal spatial_pixel's bit for bit (the union only adds taps of weight
// exactly 0).  An untraced pixel of the pair gets reach 0 and is not written.
__device__ __forceinline__ void spatial_pair(const SpatialArgs& a, int i, int j, bool tl, bool tr) {
    const float4* __restrict__ crt = a.crt;
    const int W = a.W, H = a.H;
    const float r_s = a.r_s, Rq = r_s + 0.5f;
    const size_t q = (size_t)j * W + i;
    const float4 cl = tl ? __ldg(&crt[q]) : make_float4(0.f, 0.f, 0.f, -1.f);
    const float4 cr = tr ? __ldg(&crt[q + 1]) : make_float4(0.f, 0.f, 0.f, -1.f);
    const float Rl = tl ? fminf(cl.w * 0.5f, r_s) + 0.5f : 0.f;
    const float Rr = tr ? fminf(cr.w * 0.5f, r_s) + 0.5f : 0.f;
    const float Rl2 = Rl * Rl, Rr2 = Rr * Rr;
    const int K = (int)floorf(fmaxf(Rl, Rr) + 1e-3f);
    float3 Sl = f3(0, 0, 0), Sr = f3(0, 0, 0);
    float Wl = 0.f, Wr = 0.f;
    const int y0 = max(j - K, 0), y1 = min(j + K, H - 1);
    for (int y = y0; y <= y1; ++y) {
        const float dy = (float)(y - j), dy2 = dy * dy;
        const int wl = (int)floorf(sqrtf(fmaxf(Rl2 - dy2, 0.f)) + 1e-3f);
        const int wr = (int)floorf(sqrtf(fmaxf(Rr2 - dy2, 0.f)) + 1e-3f);
        const int x0 = max(min(i - wl, i + 1 - wr), 0), x1 = min(max(i + wl, i + 1 + wr), W - 1);
        const float4* row = crt + (size_t)y * W;
        float dx = (float)(x0 - i);
        float dprev = sqrt_approx(fmaf(dx - 1.f, dx - 1.f, dy2));  // the right pixel's distance to x0
#pragma unroll SP_UNROLL
        for (int x = x0; x <= x1; ++x, dx += 1.f) {
            const float4 c = __ldg(&row[x]);
            const float dl = sqrt_approx(fmaf(dx, dx, dy2)), dr = dprev;
            const float rq = fminf(fmaf(c.w, 0.5f, 0.5f), Rq);
            const float ql = clamp01(Rl - dl) * clamp01(rq - dl);
            const float qr = clamp01(Rr - dr) * clamp01(rq - dr);
            Sl.x = fmaf(ql, c.x, Sl.x);
            Sl.y = fmaf(ql, c.y, Sl.y);
            Sl.z = fmaf(ql, c.z, Sl.z);
            Wl += ql;
            Sr.x = fmaf(qr, c.x, Sr.x);
            Sr.y = fmaf(qr, c.y, Sr.y);
            Sr.z = fmaf(qr, c.z, Sr.z);
            Wr += qr;
            dprev = dl;
        }
    }
    if (tl) spatial_finish(a, q, cl, Sl, Wl);
    if (tr) spatial_finish(a, q + 1, cr, Sr, Wr);
}

// block = one T x T tile (T = 8 or 16), one thread per pixel: the tile's
// traced pixels are compacted (row-major) so the threads that run all gather
// for traced pixels, in one round; small blocks keep many tiles resident
// where few of their pixels are traced
constexpr int SP_TILE = 8, SP_THREADS = SP_TILE * SP_TILE;
template <int T>
__device__ __forceinline__ void spatial_body(const SpatialArgs& a, int bx, int by) {
    constexpr int NT = T * T;
    __shared__ unsigned char s_list[NT];
    __shared__ int s_cnt[NT / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int i0 = bx * T + (t % T), j0 = by * T + (t / T);
    const bool traced = i0 < a.W && j0 < a.H && __ldg(&a.crt[(size_t)j0 * a.W + i0].w) >= 0.f;
    const unsigned tm = __ballot_sync(0xffffffffu, traced);
    if (lane == 0) s_cnt[w] = __popc(tm);
    __syncthreads();
    int off = 0, n = 0;
#pragma unroll
    for (int c = 0; c < NT / 32; ++c) {
        off += c < w ? s_cnt[c] : 0;
        n += s_cnt[c];
    }
    if (traced) s_list[off + __popc(tm & ((1u << lane) - 1u))] = (unsigned char)t;
    __syncthreads();
    if (t < n) {
        const int li = s_list[t];
        spatial_pixel(a, bx * T + (li % T), by * T + (li / T));
    }
}

// block = one 16x8 tile as 8x8 horizontal pixel pairs, one thread per pair:
// the pairs holding a traced pixel are compacted so the threads that run
// all gather, in one round
constexpr int SPP_TW = 16, SPP_TH = 8, SPP_THREADS = SPP_TW * SPP_TH / 2;
__global__ void __launch_bounds__(SPP_THREADS) k_spatial(SpatialArgs a) {
    constexpr int NP = SPP_THREADS, PW = SPP_TW / 2;
    __shared__ unsigned char s_list[NP];
    __shared__ int s_cnt[NP / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int i0 = blockIdx.x * SPP_TW + 2 * (t % PW), j0 = blockIdx.y * SPP_TH + t / PW;
    const bool row_in = j0 < a.H;
    const bool tl = row_in && i0 < a.W && __ldg(&a.crt[(size_t)j0 * a.W + i0].w) >= 0.f;
    const bool tr = row_in && i0 + 1 < a.W && __ldg(&a.crt[(size_t)j0 * a.W + i0 + 1].w) >= 0.f;
    const bool act = tl || tr;
    const unsigned tm = __ballot_sync(0xffffffffu, act);
    if (lane == 0) s_cnt[w] = __popc(tm);
    __syncthreads();
    int off = 0, n = 0;
#pragma unroll
    for (int c = 0; c < NP / 32; ++c) {
        off += c < w ? s_cnt[c] : 0;
        n += s_cnt[c];
    }
    // the pair's slot and which of its pixels are traced
    if (act) s_list[off + __popc(tm & ((1u << lane) - 1u))] = (unsigned char)(t | (tl ? 0x80 : 0) | (tr ? 0x40 : 0));
    __syncthreads();
    if (t < n) {
        const int e = s_list[t], p = e & 0x3f;
        spatial_pair(a, blockIdx.x * SPP_TW + 2 * (p % PW), blockIdx.y * SPP_TH + p / PW, (e & 0x80) != 0,
                     (e & 0x40) != 0);
    }
}
template <int T>
__global__ void __launch_bounds__(T * T) k_spatial_batch(const SpatialArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    spatial_body<T>(batch_record(a, v), bx, by);
}

TemporalArgs temporal_args(const float* rt, const hdof_gbuf* in, const uint8_t* spp, const hdof_camera* cam,
                           const hdof_camera* prev, const hdof_params* p, const hdof_history* hist_in,
                           const hdof_history* hist_out, float* crt, float* hacc) {
    TemporalArgs a;
    a.cam = make_cam(*cam);
    a.prev = make_cam(*prev);
    a.W = cam->width;
    a.H = cam->height;
    a.alpha = p->ema_alpha;
    a.alpha_k = p->alpha_k;
    a.moved = p->camera_moved;
    a.rt = reinterpret_cast<const float4*>(rt);
    a.spp = spp;
    a.mv = reinterpret_cast<const float2*>(in->mv);
    a.hn = reinterpret_cast<const float4*>(hist_in->near_acc);
    a.hf = reinterpret_cast<const float4*>(hist_in->far_acc);
    a.hm = reinterpret_cast<const float2*>(hist_in->mom);
    a.hl = hist_in->hlen;
    a.on = reinterpret_cast<float4*>(hist_out->near_acc);
    a.of = reinterpret_cast<float4*>(hist_out->far_acc);
    a.om = reinterpret_cast<float2*>(hist_out->mom);
    a.ol = hist_out->hlen;
    a.crt = reinterpret_cast<float4*>(crt);
    a.hacc = hacc;
    return a;
}

}  // namespace

int launch_spatial(const float4* crt, const float2* mom, const uint8_t* hlen, int W, int H, float r_s, float var_ref,
                   float4* crec, float4* aux, cudaStream_t s) {
    dim3 g2((W + SPP_TW - 1) / SPP_TW, (H + SPP_TH - 1) / SPP_TH);
    ProfScope ps_("spatial", s);
    k_spatial<<<g2, SPP_THREADS, 0, s>>>(SpatialArgs{crt, mom, hlen, W, H, r_s, var_ref, crec, aux});
    HDOF_LAUNCHED("spatial reconstruction");
    return HDOF_OK;
}

}  // namespace hdof

using namespace hdof;

static bool hist_ok(const hdof_history* h) { return h && h->near_acc && h->far_acc && h->mom && h->hlen; }

extern "C" int hdof_reconstruct(const float* rt, const hdof_gbuf* in, const uint8_t* spp, const hdof_camera* cam,
                                const hdof_camera* prev, const hdof_lens* lens, const hdof_params* p,
                                const hdof_history* hist_in, const hdof_history* hist_out, float* crt, float* hacc,
                                float* crec, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_camera(cam, "hdof_reconstruct")) || (rc = check_camera(prev, "hdof_reconstruct: prev")) ||
        (rc = check_lens(lens, "hdof_reconstruct")) || (rc = check_params(p, "hdof_reconstruct")) ||
        (rc = check_gbuf(in, "hdof_reconstruct", true)))
        return rc;
    HDOF_CHECK_ARG(rt && spp && crt && hacc && crec, "hdof_reconstruct: NULL buffer");
    HDOF_CHECK_ARG(hist_ok(hist_in) && hist_ok(hist_out), "hdof_reconstruct: history planes are required");
    HDOF_CHECK_ARG(hist_in->near_acc != hist_out->near_acc && hist_in->far_acc != hist_out->far_acc &&
                       hist_in->mom != hist_out->mom && hist_in->hlen != hist_out->hlen,
                   "hdof_reconstruct: hist_in and hist_out must be distinct buffers");
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height && prev->width == cam->width &&
                       prev->height == cam->height,
                   "hdof_reconstruct: size mismatch");
    cudaStream_t s = as_stream(stream);
    const int W = cam->width, H = cam->height;
    TemporalArgs a = temporal_args(rt, in, spp, cam, prev, p, hist_in, hist_out, crt, hacc);
    dim3 g1((W + 31) / 32, (H + 7) / 8);
    {
        ProfScope ps_("temporal", s);
        if (in->dtype_nd == HDOF_F32)
            k_temporal<float4><<<g1, 256, 0, s>>>(a, static_cast<const float4*>(in->nd));
        else
            k_temporal<half4s><<<g1, 256, 0, s>>>(a, static_cast<const half4s*>(in->nd));
        HDOF_LAUNCHED("hdof_reconstruct: temporal");
    }
    return launch_spatial(reinterpret_cast<const float4*>(crt), reinterpret_cast<const float2*>(hist_out->mom),
                          hist_out->hlen, W, H, p->r_s, p->var_ref, reinterpret_cast<float4*>(crec), nullptr, s);
}

namespace hdof {

size_t temporal_args_size() { return sizeof(TemporalBatch); }
void temporal_fill(const hdof_view& v, const ViewWs&, unsigned*, void* dst, int* gx, int* gy) {
    TemporalBatch* b = reinterpret_cast<TemporalBatch*>(dst);
    b->t = temporal_args(v.rt, &v.g, v.spp, &v.cam, &v.prev, &v.params, &v.hist_in, &v.hist_out, v.crt, v.hacc);
    b->nd = static_cast<const float4*>(v.g.nd);
    *gx = (v.cam.width + 31) / 32;
    *gy = (v.cam.height + 7) / 8;
}
void temporal_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_temporal", s);
    k_temporal_batch<<<blocks, 256, 0, s>>>(static_cast<const TemporalBatch*>(args), g);
}

size_t spatial_args_size() { return sizeof(SpatialArgs); }
void spatial_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    *reinterpret_cast<SpatialArgs*>(dst) =
        SpatialArgs{reinterpret_cast<const float4*>(v.crt), reinterpret_cast<const float2*>(v.hist_out.mom),
                    v.hist_out.hlen, v.cam.width, v.cam.height, v.params.r_s, v.params.var_ref,
                    reinterpret_cast<float4*>(v.crec), nullptr};
    const int T = w.spatial_tile == 16 ? 16 : SP_TILE;
    *gx = (v.cam.width + T - 1) / T;
    *gy = (v.cam.height + T - 1) / T;
}
void spatial_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    spatial_launch_batch_tile(args, g, blocks, SP_TILE, s);
}
void spatial_launch_batch_tile(const void* args, BatchGrid g, int blocks, int tile, cudaStream_t s) {
    ProfScope ps_("batch_spatial", s);
    if (tile == 16) k_spatial_batch<16><<<blocks, 256, 0, s>>>(static_cast<const SpatialArgs*>(args), g);
    else k_spatial_batch<SP_TILE><<<blocks, SP_THREADS, 0, s>>>(static_cast<const SpatialArgs*>(args), g);
}

}  // namespace hdof
