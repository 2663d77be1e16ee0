// Differentiable post-path: the frame's reconstruction, post-filter and
// composite as a function of the sharp colour image and of the lens (focus
// distance, aperture), with the ray-traced visibility held fixed, and its
// hand-written adjoint.  The paper has no gradient; this makes the method's
// post-path usable inside an optimisation loop (e.g. fitting the lens to a
// reference image).
//
// Frozen inputs: per-ray hit records (radiance, view depth) from hdof_trace,
// the mask (spp), the depth plane, and the history already sampled at its
// reprojected positions.  Forward: replay of the trace accumulation at the
// new lens (each hit's CoC, split weight and CoC magnitude change, the hits
// do not) -> temporal EMA over the frozen history samples -> spatial gather
// -> post-filter -> composite; the same kernels as the frame path where the
// definitions coincide.  Backward: composite -> spatial (transposed gather)
// -> temporal and replay (per pixel, recomputed) -> post-filter (transposed
// gather over each source pixel's own disk, gather weights recomputed, not
// stored).  The lens gradient is reduced per block in double precision and
// summed in a fixed order: the result is deterministic.
#include <cmath>

#include "internal.h"

namespace hdof {
namespace {

constexpr float RS2 = 0.35355339059327373f;  // 1 / (2 sqrt2): slope of w_near inside the focus zone

struct LensD {
    float K;           // A H / t
    float izf;         // 1 / zf
    float Ht;          // H / t
    float t;           // tan(fovy / 2)
    const float* dev;  // optional (zf, A) on the device: K and izf are read from it when a kernel starts
};

// K and izf of a lens on the device, by make_lensd's arithmetic
__device__ __forceinline__ LensD lens_at(LensD L, int H) {
    if (L.dev) {
        L.K = __ldg(&L.dev[1]) * (float)H / L.t;
        L.izf = 1.f / __ldg(&L.dev[0]);
    }
    return L;
}

__device__ __forceinline__ float coc_z(float z, const LensD& L) {
    return isinf(z) ? -L.K * L.izf : L.K * (1.f / z - L.izf);
}
// (dc/dzf, dc/dA) of the CoC of a point at depth z (z = inf: the miss CoC)
__device__ __forceinline__ float2 dcoc(float z, const LensD& L) {
    float u = isinf(z) ? -L.izf : 1.f / z - L.izf;
    return make_float2(L.K * L.izf * L.izf, L.Ht * u);
}
__device__ __forceinline__ float wn_slope(float c) { return (c > -HDOF_SQRT2 && c < HDOF_SQRT2) ? RS2 : 0.f; }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 ldf3(const float4& v) { return f3(v.x, v.y, v.z); }

// block sum of a per-thread (float, float) in double, fixed order; lane 0 of
// warp 0 writes the block's partial
__device__ __forceinline__ void block_partial(float2 v, double2* partial) {
    __shared__ double red[2][32];
    double a = v.x, b = v.y;
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (l == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int k = 0; k < nw; ++k) {
            sa += red[0][k];
            sb += red[1][k];
        }
        partial[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(sa, sb);
    }
}

// ------------------------------------------------------------ forward ----

struct ReplaySums {
    float3 SwL, SfL;
    float Sw, Sf, Swc, Sfc;
};

__device__ __forceinline__ ReplaySums replay_sums(const float4* rec, unsigned first, int n, const LensD& L) {
    ReplaySums s;
    s.SwL = s.SfL = f3(0.f, 0.f, 0.f);
    s.Sw = s.Sf = s.Swc = s.Sfc = 0.f;
    for (int k = 0; k < n; ++k) {
        float4 r = __ldg(&rec[first + k]);
        float c = coc_z(r.w, L);
        float w = w_near(c), wf = 1.f - w, ac = fabsf(c);
        s.SwL = s.SwL + w * ldf3(r);
        s.SfL = s.SfL + wf * ldf3(r);
        s.Sw += w;
        s.Sf += wf;
        s.Swc += w * ac;
        s.Sfc += wf * ac;
    }
    return s;
}

__global__ void __launch_bounds__(256) k_replay(const float4* __restrict__ rec, const unsigned* __restrict__ ray_off,
                                                const uint8_t* __restrict__ spp, int W, int H, LensD L,
                                                float4* __restrict__ rt) {
    L = lens_at(L, H);
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    int n = spp[q];
    if (!n) return;
    ReplaySums s = replay_sums(rec, ray_off[q], n, L);
    bool nok = s.Sw >= HDOF_EMPTY_W, fok = s.Sf >= HDOF_EMPTY_W;
    float in = nok ? 1.f / s.Sw : 0.f, inf_ = fok ? 1.f / s.Sf : 0.f;
    rt[3 * q] = make_float4(s.SwL.x * in, s.SwL.y * in, s.SwL.z * in, s.Sw / (float)n);
    rt[3 * q + 1] = make_float4(s.SfL.x * inf_, s.SfL.y * inf_, s.SfL.z * inf_, nok ? s.Swc * in : -1.f);
    rt[3 * q + 2] = make_float4(0.f, 0.f, 0.f, fok ? s.Sfc * inf_ : -1.f);
}

// history sampled at the reprojected positions: (near rgb, B) (far rgb, B) (mu1, mu2, flags, hlen)
struct HistS {
    float4 hn, hf;
    float m1, m2;
    bool vn, vf;
    int hl;
};
__device__ __forceinline__ HistS load_hs(const float4* hs, size_t q) {
    HistS h;
    if (!hs) {
        h.hn = h.hf = make_float4(0.f, 0.f, 0.f, 0.f);
        h.m1 = h.m2 = 0.f;
        h.vn = h.vf = false;
        h.hl = 0;
        return h;
    }
    h.hn = __ldg(&hs[3 * q]);
    h.hf = __ldg(&hs[3 * q + 1]);
    float4 t = __ldg(&hs[3 * q + 2]);
    h.m1 = t.x;
    h.m2 = t.y;
    int fl = (int)t.z;
    h.vn = fl & 1;
    h.vf = (fl >> 1) & 1;
    h.hl = (int)t.w;
    return h;
}

// the temporal step with frozen history samples (forward values used by the adjoint)
struct TempF {
    float h, cn, cf;
    bool nok, fok;
    float3 Cn, Cf, Ccur;
    float Y;
    float4 on, of;
    float2 om;
    float Bn, Bf, Hacc, hw;
    bool an, af, hsum;
    float3 CnA, CfA, C;
    float crt_c;
};

__device__ __forceinline__ TempF temporal_fwd(float4 r0, float4 r1, float4 r2, const HistS& hs, float al, int moved) {
    TempF t;
    t.h = r0.w;
    t.cn = r1.w;
    t.cf = r2.w;
    t.nok = t.cn >= 0.f;
    t.fok = t.cf >= 0.f;
    t.Cn = ldf3(r0);
    t.Cf = ldf3(r1);
    t.Ccur = t.nok ? (t.fok ? t.h * t.Cn + (1.f - t.h) * t.Cf : t.Cn) : t.Cf;
    t.Y = luminance(t.Ccur);
    float4 cur_n = make_float4(t.h * t.Cn.x, t.h * t.Cn.y, t.h * t.Cn.z, t.h);
    float4 cur_f = make_float4((1.f - t.h) * t.Cf.x, (1.f - t.h) * t.Cf.y, (1.f - t.h) * t.Cf.z, 1.f - t.h);
    const float4 hn = hs.hn, hf = hs.hf;
    t.on = hs.vn ? make_float4(fmaf(al, cur_n.x - hn.x, hn.x), fmaf(al, cur_n.y - hn.y, hn.y),
                               fmaf(al, cur_n.z - hn.z, hn.z), fmaf(al, cur_n.w - hn.w, hn.w))
                 : cur_n;
    t.of = hs.vf ? make_float4(fmaf(al, cur_f.x - hf.x, hf.x), fmaf(al, cur_f.y - hf.y, hf.y),
                               fmaf(al, cur_f.z - hf.z, hf.z), fmaf(al, cur_f.w - hf.w, hf.w))
                 : cur_f;
    t.om = hs.vn ? make_float2(fmaf(al, t.Y - hs.m1, hs.m1), fmaf(al, t.Y * t.Y - hs.m2, hs.m2))
                 : make_float2(t.Y, t.Y * t.Y);
    t.Bn = t.on.w;
    t.Bf = t.of.w;
    t.hsum = t.Bn + t.Bf >= HDOF_EMPTY_W;
    t.Hacc = t.hsum ? t.Bn / (t.Bn + t.Bf) : t.h;
    t.an = t.Bn >= HDOF_EMPTY_W;
    t.af = t.Bf >= HDOF_EMPTY_W;
    t.hw = moved ? t.h : t.Hacc;
    t.CnA = t.an ? (1.f / t.Bn) * ldf3(t.on) : f3(0, 0, 0);
    t.CfA = t.af ? (1.f / t.Bf) * ldf3(t.of) : f3(0, 0, 0);
    t.C = !t.an ? t.CfA : (!t.af ? t.CnA : t.hw * t.CnA + (1.f - t.hw) * t.CfA);
    t.crt_c = !t.nok ? t.cf : (!t.fok ? t.cn : t.Hacc * t.cn + (1.f - t.Hacc) * t.cf);
    return t;
}

__global__ void __launch_bounds__(256) k_temporal_frozen(const float4* __restrict__ rt, const uint8_t* __restrict__ spp,
                                                         const float4* __restrict__ hs, int W, int H, float al,
                                                         int moved, float4* __restrict__ crt, float* __restrict__ hacc,
                                                         float2* __restrict__ mom, uint8_t* __restrict__ hlen) {
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    if (!spp[q]) {
        crt[q] = make_float4(0.f, 0.f, 0.f, -1.f);
        hlen[q] = 0;
        return;
    }
    HistS h = load_hs(hs, q);
    TempF t = temporal_fwd(rt[3 * q], rt[3 * q + 1], rt[3 * q + 2], h, al, moved);
    crt[q] = make_float4(t.C.x, t.C.y, t.C.z, t.crt_c);
    hacc[q] = t.Hacc;
    mom[q] = t.om;
    int nh = h.vn ? h.hl + 1 : 1;
    hlen[q] = (uint8_t)(nh > 255 ? 255 : nh);
}

// ----------------------------------------------------------- backward ----

// composite adjoint: per pixel; grad_col <- f g (the sharp term), gradients of
// pp, crec, crt.w, hacc, and this pixel's share of the lens gradient
__global__ void __launch_bounds__(256) k_composite_bwd(const float4* __restrict__ nd, const float4* __restrict__ col,
                                                       const uint8_t* __restrict__ spp, const float4* __restrict__ pp,
                                                       const float4* __restrict__ crt, const float4* __restrict__ crec,
                                                       const float* __restrict__ hacc, const float4* __restrict__ gout,
                                                       int W, int H, LensD L, float h_tau, float4* __restrict__ gcol,
                                                       float4* __restrict__ gpp, float4* __restrict__ gcrec,
                                                       float4* __restrict__ gcrt, float* __restrict__ ghacc,
                                                       double2* partial) {
    L = lens_at(L, H);
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    float2 dth = make_float2(0.f, 0.f);
    if (i < W && j < H) {
        size_t q = (size_t)j * W + i;
        float z = __ldg(&nd[q].w);
        float c = coc_z(z, L);
        bool traced = spp[q] > 0;
        float3 C = ldf3(__ldg(&col[q])), P = ldf3(__ldg(&pp[q])), g = ldf3(__ldg(&gout[q]));
        float ce = traced ? __ldg(&crt[q].w) : fabsf(c);
        float fu = HDOF_SQRT2 + 0.5f - ce, f = clamp01(fu);
        float wn = w_near(c);
        float3 nearc = P, farc = P, R = f3(0, 0, 0);
        float b = 0.f, bu = 0.f;
        if (traced) {
            R = ldf3(__ldg(&crec[q]));
            bu = __ldg(&hacc[q]) / h_tau;
            b = clamp01(bu);
            nearc = R;
            farc = R + b * (P - R);
        }
        float3 blur = wn * nearc + (1.f - wn) * farc;
        float3 gb = (1.f - f) * g;
        float gf = dot3f(g, C - blur);
        float gwn = dot3f(gb, nearc - farc);
        float3 gnear = wn * gb, gfar = (1.f - wn) * gb;
        float gc = wn_slope(c) * gwn;
        float gfu = (fu > 0.f && fu < 1.f) ? gf : 0.f;
        gcol[q] = make_float4(f * g.x, f * g.y, f * g.z, 0.f);
        if (traced) {
            float3 gr = gnear + (1.f - b) * gfar;
            float3 gp = b * gfar;
            float gbb = dot3f(gfar, P - R);
            gpp[q] = make_float4(gp.x, gp.y, gp.z, 0.f);
            gcrec[q] = make_float4(gr.x, gr.y, gr.z, 0.f);
            gcrt[q] = make_float4(0.f, 0.f, 0.f, -gfu);
            ghacc[q] = (bu > 0.f && bu < 1.f) ? gbb / h_tau : 0.f;
        } else {
            float3 gp = gnear + gfar;
            gpp[q] = make_float4(gp.x, gp.y, gp.z, 0.f);
            gc += -gfu * (c > 0.f ? 1.f : (c < 0.f ? -1.f : 0.f));
        }
        float2 dc = dcoc(z, L);
        dth = make_float2(gc * dc.x, gc * dc.y);
    }
    block_partial(dth, partial);
}

// spatial adjoint, part 1 (per traced pixel): direct term, the variance blend,
// and the per-gatherer factors a = beta g / W, b = a . C_sp of the gather
__global__ void __launch_bounds__(256) k_spatial_bwd_prep(const float4* __restrict__ crt, const float2* __restrict__ mom,
                                                          const uint8_t* __restrict__ hlen, const float4* __restrict__ aux,
                                                          const float4* __restrict__ gcrec, int W, int H, float var_ref,
                                                          float4* __restrict__ spb, float4* __restrict__ gcrt,
                                                          float2* __restrict__ gmom) {
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    float4 cp = crt[q];
    if (cp.w < 0.f) return;
    float2 m = mom[q];
    float v = m.y - m.x * m.x;
    float sig = sqrtf(fmaxf(0.f, v));
    bool young = hlen[q] < 2;
    float bu = sig / var_ref;
    float beta = young ? 1.f : clamp01(bu);
    float4 ax = aux[q];
    float3 Csp = ldf3(ax), Crt = ldf3(cp), g = ldf3(gcrec[q]);
    float gbeta = dot3f(g, Csp - Crt);
    float2 gm = make_float2(0.f, 0.f);
    if (!young && bu > 0.f && bu < 1.f && v > 0.f) {
        float gs = gbeta / var_ref;
        gm = make_float2(gs * (-m.x / sig), gs * (0.5f / sig));
    }
    gmom[q] = gm;
    float3 a = (beta / ax.w) * g;
    spb[q] = make_float4(a.x, a.y, a.z, dot3f(a, Csp));
    float4 gc = gcrt[q];
    float3 gd = (1.f - beta) * g;
    gcrt[q] = make_float4(gc.x + gd.x, gc.y + gd.y, gc.z + gd.z, gc.w);
}

// spatial adjoint, part 2 (per traced pixel x over its own window): x as a
// gathered sample of its neighbours and x as a gatherer
__global__ void __launch_bounds__(256) k_spatial_bwd(const float4* __restrict__ crt, const float4* __restrict__ spb,
                                                     int W, int H, float r_s, float4* __restrict__ gcrt) {
    // block = one 16x16 tile; its traced pixels are compacted (row-major) so
    // that every warp which runs works on traced pixels only
    __shared__ unsigned char s_list[256];
    __shared__ int s_wcnt[8];
    const int t = threadIdx.x, lane = t & 31;
    bool traced = false;
    {
        const int i0 = blockIdx.x * 16 + (t & 15), j0 = blockIdx.y * 16 + (t >> 4);
        if (i0 < W && j0 < H) traced = __ldg(&crt[(size_t)j0 * W + i0].w) >= 0.f;
    }
    const unsigned tm = __ballot_sync(0xffffffffu, traced);
    if (lane == 0) s_wcnt[t >> 5] = __popc(tm);
    __syncthreads();
    int off = 0, n = 0;
    for (int k = 0; k < 8; ++k) {
        off += k < (t >> 5) ? s_wcnt[k] : 0;
        n += s_wcnt[k];
    }
    if (traced) s_list[off + __popc(tm & ((1u << lane) - 1u))] = (unsigned char)t;
    __syncthreads();
    if (t >= n) return;
    const int li = s_list[t];
    const int i = blockIdx.x * 16 + (li & 15), j = blockIdx.y * 16 + (li >> 4);
    const size_t q = (size_t)j * W + i;
    const float4 cx = crt[q];
    const float rx = fminf(cx.w * 0.5f, r_s);
    const float rpx = cx.w * 0.5f < r_s ? 0.5f : 0.f;
    const float4 bx = spb[q];
    const float3 Cx = ldf3(cx), ax = ldf3(bx);
    // a neighbour takes part only if d < R = rx + 1/2: per row, the columns
    // of that disk (bounds lean outwards by 1e-3 pixel; taps they add weigh 0)
    const float R = rx + 0.5f, R2 = R * R;
    const int K = (int)floorf(R + 1e-3f);
    float3 gC = f3(0, 0, 0);
    float gcx = 0.f;
    const int y0 = max(j - K, 0), y1 = min(j + K, H - 1);
    for (int y = y0; y <= y1; ++y) {
        const float dy = (float)(y - j), dy2 = dy * dy;
        const int wr = (int)floorf(sqrtf(fmaxf(R2 - dy2, 0.f)) + 1e-3f);
        const int x0 = max(i - wr, 0), x1 = min(i + wr, W - 1);
        for (int x = x0; x <= x1; ++x) {
            float dx = (float)(x - i);
            size_t qq = (size_t)y * W + x;
            // branch-free: untraced neighbours (and their unwritten spb) are
            // selected away, out-of-disk pairs weigh exactly zero
            const float4 cy = __ldg(&crt[qq]), by = __ldg(&spb[qq]);
            const bool ty = cy.w >= 0.f;
            float d = sqrt_approx(fmaf(dx, dx, dy2));
            float ux = R - d, uy = fminf(fmaf(cy.w, 0.5f, 0.5f), r_s + 0.5f) - d;
            float sx = clamp01(ux), sy = ty ? clamp01(uy) : 0.f;
            float spx = (ux > 0.f && ux < 1.f) ? 1.f : 0.f;
            const float3 ay = ty ? ldf3(by) : f3(0.f, 0.f, 0.f);
            const float byw = ty ? by.w : 0.f;
            gC = gC + (sy * sx) * ay;
            gcx += sy * spx * (dot3f(ay, Cx) - byw);               // x gathered by y
            gcx += spx * sy * (dot3f(ax, ldf3(cy)) - bx.w);        // x gathering y
        }
    }
    float4 g = gcrt[q];
    gcrt[q] = make_float4(g.x + gC.x, g.y + gC.y, g.z + gC.z, g.w + gcx * rpx);
}

// temporal + replay adjoint (per traced pixel, forward recomputed): the
// gradient of crt, hacc and the moments back to each hit's CoC
__global__ void __launch_bounds__(256) k_temporal_replay_bwd(const float4* __restrict__ rec,
                                                             const unsigned* __restrict__ ray_off,
                                                             const uint8_t* __restrict__ spp,
                                                             const float4* __restrict__ hs, const float4* __restrict__ gcrt,
                                                             const float* __restrict__ ghacc,
                                                             const float2* __restrict__ gmom, int W, int H, LensD L,
                                                             float al, int moved, double2* partial) {
    L = lens_at(L, H);
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    float2 dth = make_float2(0.f, 0.f);
    size_t q = (size_t)j * W + i;
    int n = (i < W && j < H) ? spp[q] : 0;
    if (n) {
        const unsigned first = ray_off[q];
        ReplaySums s = replay_sums(rec, first, n, L);
        bool nok = s.Sw >= HDOF_EMPTY_W, fok = s.Sf >= HDOF_EMPTY_W;
        float in = nok ? 1.f / s.Sw : 0.f, inf_ = fok ? 1.f / s.Sf : 0.f;
        float4 r0 = make_float4(s.SwL.x * in, s.SwL.y * in, s.SwL.z * in, s.Sw / (float)n);
        float4 r1 = make_float4(s.SfL.x * inf_, s.SfL.y * inf_, s.SfL.z * inf_, nok ? s.Swc * in : -1.f);
        float4 r2 = make_float4(0.f, 0.f, 0.f, fok ? s.Sfc * inf_ : -1.f);
        HistS hsv = load_hs(hs, q);
        TempF t = temporal_fwd(r0, r1, r2, hsv, al, moved);
        // ---- temporal adjoint ----
        float4 g4 = gcrt[q];
        float3 gC = ldf3(g4);
        float gcc = g4.w, gH = ghacc[q];
        float2 gom = gmom[q];
        float3 gCnA = f3(0, 0, 0), gCfA = f3(0, 0, 0);
        float gh = 0.f, ghw = 0.f, gcn = 0.f, gcf = 0.f;
        if (!t.an) gCfA = gC;
        else if (!t.af) gCnA = gC;
        else {
            gCnA = t.hw * gC;
            gCfA = (1.f - t.hw) * gC;
            ghw = dot3f(gC, t.CnA - t.CfA);
        }
        if (moved) gh += ghw;
        else gH += ghw;
        if (!t.nok) gcf += gcc;
        else if (!t.fok) gcn += gcc;
        else {
            gH += gcc * (t.cn - t.cf);
            gcn += t.Hacc * gcc;
            gcf += (1.f - t.Hacc) * gcc;
        }
        float gBn = 0.f, gBf = 0.f;
        if (t.hsum) {
            float S = t.Bn + t.Bf, iS2 = 1.f / (S * S);
            gBn += gH * t.Bf * iS2;
            gBf -= gH * t.Bn * iS2;
        } else {
            gh += gH;
        }
        float3 gon = f3(0, 0, 0), gof = f3(0, 0, 0);
        if (t.an) {
            gon = (1.f / t.Bn) * gCnA;
            gBn -= dot3f(gCnA, ldf3(t.on)) / (t.Bn * t.Bn);
        }
        if (t.af) {
            gof = (1.f / t.Bf) * gCfA;
            gBf -= dot3f(gCfA, ldf3(t.of)) / (t.Bf * t.Bf);
        }
        const float kn = hsv.vn ? al : 1.f, kf = hsv.vf ? al : 1.f;
        float3 gcurn = kn * gon, gcurf = kf * gof;
        float gcurnw = kn * gBn, gcurfw = kf * gBf;
        float gY = kn * (gom.x + 2.f * t.Y * gom.y);
        float3 gCn = t.h * gcurn, gCf = (1.f - t.h) * gcurf;
        gh += dot3f(gcurn, t.Cn) + gcurnw - dot3f(gcurf, t.Cf) - gcurfw;
        float3 gCcur = gY * f3(0.2126f, 0.7152f, 0.0722f);
        if (t.nok && t.fok) {
            gh += dot3f(gCcur, t.Cn - t.Cf);
            gCn = gCn + t.h * gCcur;
            gCf = gCf + (1.f - t.h) * gCcur;
        } else if (t.nok) {
            gCn = gCn + gCcur;
        } else {
            gCf = gCf + gCcur;
        }
        // ---- replay adjoint ----
        float gSw = gh / (float)n, gSf = 0.f, gSwc = 0.f, gSfc = 0.f;
        float3 gSwL = f3(0, 0, 0), gSfL = f3(0, 0, 0);
        if (nok) {
            gSwL = in * gCn;
            gSw -= dot3f(gCn, s.SwL) * in * in;
            gSwc = gcn * in;
            gSw -= gcn * s.Swc * in * in;
        }
        if (fok) {
            gSfL = inf_ * gCf;
            gSf -= dot3f(gCf, s.SfL) * inf_ * inf_;
            gSfc = gcf * inf_;
            gSf -= gcf * s.Sfc * inf_ * inf_;
        }
        for (int k = 0; k < n; ++k) {
            float4 r = __ldg(&rec[first + k]);
            float c = coc_z(r.w, L);
            float w = w_near(c), ac = fabsf(c);
            float gw = gSw - gSf + dot3f(gSwL - gSfL, ldf3(r)) + (gSwc - gSfc) * ac;
            float gac = gSwc * w + gSfc * (1.f - w);
            float gc = gw * wn_slope(c) + gac * (c > 0.f ? 1.f : (c < 0.f ? -1.f : 0.f));
            float2 dc = dcoc(r.w, L);
            dth.x += gc * dc.x;
            dth.y += gc * dc.y;
        }
    }
    block_partial(dth, partial);
}

__device__ __forceinline__ float2 area_and_slope(const float4* tab, int n, float r) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&tab[mid].x) <= r) lo = mid;
        else hi = mid - 1;
    }
    float4 e = __ldg(&tab[lo]);
    return make_float2(fmaf(e.z, r - e.x, e.y), e.z);
}

// post-filter adjoint, part 1 (per pixel p): factors of dL/d(near weight) =
// A . C_q - E and dL/d(far weight) = Af . C_q - Ef, and the sharp-colour
// fallback of an empty far layer
// Written per pixel q: (A, E) and (Af, Ef) in two planes, each split by
// pixel-index parity (even pixels, then odd), and kb_q = 1 / (kz_rel z_q) of
// the forward's depth test, row-major.
__global__ void __launch_bounds__(256) k_pf_bwd_prep(const float4* __restrict__ aux, const float4* __restrict__ gpp,
                                                     const float4* __restrict__ nd, float kz_rel, int W, int H,
                                                     float4* __restrict__ pfb, float* __restrict__ kbp,
                                                     float4* __restrict__ gcol) {
    int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    const size_t px = (size_t)W * H, qs = (q >> 1) + (q & 1) * ((px + 1) >> 1);
    kbp[q] = 1.f / (kz_rel * __ldg(&nd[q].w));
    float4 an = aux[2 * q], af = aux[2 * q + 1];
    float3 g = ldf3(gpp[q]), N = ldf3(an), F = ldf3(af);
    float Wn = an.w, Wf = af.w;
    float alpha = clamp01(Wn);
    float adash = (Wn > 0.f && Wn < 1.f) ? 1.f : 0.f;
    float3 A = Wn > HDOF_PP_MIN_W ? (alpha / Wn) * g : f3(0, 0, 0);
    float E = dot3f(A, N) - adash * dot3f(g, N - F);
    float3 Af = f3(0, 0, 0);
    float Ef = 0.f;
    if (Wf > HDOF_PP_MIN_W) {
        Af = ((1.f - alpha) / Wf) * g;
        Ef = dot3f(Af, F);
    } else {
        float4 gc = gcol[q];  // F is this pixel's sharp colour
        gcol[q] = make_float4(gc.x + (1.f - alpha) * g.x, gc.y + (1.f - alpha) * g.y, gc.z + (1.f - alpha) * g.z, 0.f);
    }
    pfb[qs] = make_float4(A.x, A.y, A.z, E);
    pfb[px + qs] = make_float4(Af.x, Af.y, Af.z, Ef);
}

// per source pixel: the radius and the layer weights of the forward map and
// their slopes with respect to the source's CoC
struct PfSrc {
    float R, rp;         // r + 1/2; dr/dc (0 when clipped at r_max)
    float wnia, fia;     // w/a, (1-w)/a
    float dwnia, dfia;   // their derivatives with respect to c
};
__device__ __forceinline__ PfSrc pf_src(float zq, const LensD& L, float rmax, const float4* tab, int ntab) {
    PfSrc o;
    const float c = coc_z(zq, L);
    const bool clip = fabsf(c) * 0.5f >= rmax;
    const float r = clip ? rmax : fabsf(c) * 0.5f;
    o.R = r + 0.5f;
    o.rp = clip ? 0.f : (c > 0.f ? 0.5f : (c < 0.f ? -0.5f : 0.f));
    const float2 as = area_and_slope(tab, ntab, r);
    const float ia = 1.f / as.x, iap = -as.y * ia * ia * o.rp;
    const float wn = w_near(c), wnp = wn_slope(c);
    o.wnia = wn * ia;
    o.fia = (1.f - wn) * ia;
    o.dwnia = wnp * ia + wn * iap;
    o.dfia = -wnp * ia + (1.f - wn) * iap;
    return o;
}

struct PfBwdAcc {
    float3 gC;
    float S1, S2, S3, S4;
};

// the four sources of a thread against one target: sources (i, j) and
// (i, j + 1) get fresh distances, sources (i + 1, j) and (i + 1, j + 1) the
// previous target's (the same offsets, so the same floats), carried in c
struct PfBwdSrc {
    float zq[4], R[4], wnia[4], fia[4];
    float3 Cq[4];
};
__device__ __forceinline__ void pf_bwd_tap(PfBwdAcc (&acc)[4], float (&c)[2], const PfBwdSrc& src, float dx,
                                           float dy0, float dy1, float ka, float kb, const float4& bn,
                                           const float4& bf) {
    const float3 An = ldf3(bn), Af = ldf3(bf);
    const float dx2 = dx * dx;
    const float e0 = sqrt_approx(dx2 + dy0), e2 = sqrt_approx(dx2 + dy1);
    const float d[4] = {e0, c[0], e2, c[1]};
    c[0] = e0;
    c[1] = e2;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float u = src.R[k] - d[k];
        const float sw = __saturatef(u), sp = (u > 0.f && u < 1.f) ? 1.f : 0.f;
        const float kz = __saturatef(fmaf(-src.zq[k], kb, ka));
        const float an = sw * src.wnia[k], af = sw * src.fia[k] * kz;
        acc[k].gC.x = fmaf(an, An.x, fmaf(af, Af.x, acc[k].gC.x));
        acc[k].gC.y = fmaf(an, An.y, fmaf(af, Af.y, acc[k].gC.y));
        acc[k].gC.z = fmaf(an, An.z, fmaf(af, Af.z, acc[k].gC.z));
        const float tn = dot3f(An, src.Cq[k]) - bn.w, tf = (dot3f(Af, src.Cq[k]) - bf.w) * kz;
        acc[k].S1 = fmaf(tn, sw, acc[k].S1);
        acc[k].S2 = fmaf(tn, sp, acc[k].S2);
        acc[k].S3 = fmaf(tf, sw, acc[k].S3);
        acc[k].S4 = fmaf(tf, sp, acc[k].S4);
    }
}

// post-filter adjoint, part 2: per source pixel q over the target pixels its
// soft disk reaches, the colour gradient and the gradient of q's CoC.  One
// block per 16x16 tile of sources, 64 threads; thread t takes the 2x2 source
// block at (2 (t & 7), 2 (t >> 3)), so every target it loads serves four
// sources.  The loop covers, per target row, the columns closer than the
// tile's largest radius to one of the four (other pairs have zero weight) and
// is branch-free; the depth test is the forward's clamp(ka - z_q kb_p).
#ifndef HDOF_PFB_MINB
#define HDOF_PFB_MINB 8  // resident blocks per SM the post-filter adjoint's register budget targets (128 registers)
#endif
__global__ void __launch_bounds__(64, HDOF_PFB_MINB) k_pf_bwd(const float4* __restrict__ nd, const float4* __restrict__ col,
                                               const float4* __restrict__ pfb, const float* __restrict__ kbp,
                                               const float4* __restrict__ tab, int ntab, int W, int H, LensD L,
                                               float rmax, float kz_rel, float4* __restrict__ gcol,
                                               double2* partial) {
    L = lens_at(L, H);
    __shared__ int s_win;
    if (threadIdx.x == 0) s_win = 0;
    __syncthreads();
    const int i = blockIdx.x * 16 + 2 * (threadIdx.x & 7), j = blockIdx.y * 16 + 2 * (threadIdx.x >> 3);
    const bool in0 = i < W && j < H;
    const bool ok[4] = {in0, in0 && i + 1 < W, in0 && j + 1 < H, in0 && i + 1 < W && j + 1 < H};
    const int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
    PfBwdSrc src;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        src.zq[k] = 1.f;
        src.R[k] = 0.f;  // an absent source weighs nothing
        src.wnia[k] = src.fia[k] = 0.f;
        src.Cq[k] = f3(0, 0, 0);
        if (ok[k]) {
            const size_t q = (size_t)(j + oy[k]) * W + (i + ox[k]);
            src.zq[k] = __ldg(&nd[q].w);
            const PfSrc sr = pf_src(src.zq[k], L, rmax, tab, ntab);
            src.R[k] = sr.R;
            src.wnia[k] = sr.wnia;
            src.fia[k] = sr.fia;
            src.Cq[k] = ldf3(__ldg(&col[q]));
            atomicMax(&s_win, __float_as_int(sr.R));  // positive floats order as their bits
        }
    }
    __syncthreads();
    float2 dth = make_float2(0.f, 0.f);
    if (in0) {
        // the block's reach R = max(r) + 1/2: a pair weighs (and its rim term
        // counts) only closer than that; bounds lean outwards by 1e-3 pixel
        const float Rw = __int_as_float(s_win), R2w = Rw * Rw;
        const int G = (int)floorf(Rw + 1e-3f);
        const float ka = 1.f + 1.f / kz_rel;
        const size_t px = (size_t)W * H, half = (px + 1) >> 1;
        const float4* __restrict__ pn_e = pfb;
        const float4* __restrict__ pn_o = pfb + half;
        const float4* __restrict__ pf_e = pfb + px;
        const float4* __restrict__ pf_o = pfb + px + half;
        const float2* __restrict__ kb2 = reinterpret_cast<const float2*>(kbp);
        PfBwdAcc acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k].gC = f3(0, 0, 0);
            acc[k].S1 = acc[k].S2 = acc[k].S3 = acc[k].S4 = 0.f;
        }
        const int y0 = max(j - G, 0), y1 = min(j + 1 + G, H - 1);
        for (int y = y0; y <= y1; ++y) {
            const float dy = (float)(y - j);
            const float dy0 = dy * dy, dy1 = (dy - 1.f) * (dy - 1.f);
            const float dmin = dy >= 0.f && dy <= 1.f ? 0.f : fminf(dy0, dy1);
            const int w = (int)floorf(sqrtf(fmaxf(R2w - dmin, 0.f)) + 1e-3f);
            const int x0 = max(i - w, 0), x1 = min(i + 1 + w, W - 1);
            float dx = (float)(x0 - i);
            float c[2];
            {
                const float dm = (dx - 1.f) * (dx - 1.f);
                c[0] = sqrt_approx(dm + dy0);
                c[1] = sqrt_approx(dm + dy1);
            }
            // targets in (even, odd) index pairs; a lone odd first and even last on their own
            size_t g = (size_t)y * W + x0;
            const size_t gend = (size_t)y * W + x1 + 1;
            if (g & 1) {
                pf_bwd_tap(acc, c, src, dx, dy0, dy1, ka, __ldg(&kbp[g]), __ldg(&pn_o[g >> 1]), __ldg(&pf_o[g >> 1]));
                ++g;
                dx += 1.f;
            }
            const size_t mend = gend >> 1;
#pragma unroll 1
            for (size_t m = g >> 1; m < mend; ++m, dx += 2.f) {
                const float2 kb = __ldg(&kb2[m]);
                pf_bwd_tap(acc, c, src, dx, dy0, dy1, ka, kb.x, __ldg(&pn_e[m]), __ldg(&pf_e[m]));
                pf_bwd_tap(acc, c, src, dx + 1.f, dy0, dy1, ka, kb.y, __ldg(&pn_o[m]), __ldg(&pf_o[m]));
            }
            if (gend & 1) {
                const size_t gl = gend - 1;
                pf_bwd_tap(acc, c, src, dx, dy0, dy1, ka, __ldg(&kbp[gl]), __ldg(&pn_e[gl >> 1]),
                           __ldg(&pf_e[gl >> 1]));
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!ok[k]) continue;
            const size_t q = (size_t)(j + oy[k]) * W + (i + ox[k]);
            const float4 g0 = gcol[q];
            gcol[q] = make_float4(g0.x + acc[k].gC.x, g0.y + acc[k].gC.y, g0.z + acc[k].gC.z, 0.f);
            const PfSrc sr = pf_src(src.zq[k], L, rmax, tab, ntab);
            const float gc = acc[k].S1 * sr.dwnia + acc[k].S2 * sr.wnia * sr.rp + acc[k].S3 * sr.dfia +
                             acc[k].S4 * sr.fia * sr.rp;
            const float2 dc = dcoc(src.zq[k], L);
            dth.x = fmaf(gc, dc.x, dth.x);
            dth.y = fmaf(gc, dc.y, dth.y);
        }
    }
    block_partial(dth, partial);
}

__global__ void __launch_bounds__(1024) k_reduce(const double2* __restrict__ partial, int n, float* out) {
    __shared__ double red[2][1024];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        a += partial[k].x;
        b += partial[k].y;
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = (float)red[0][0];
        out[1] = (float)red[1][0];
    }
}

LensD make_lensd(const hdof_lens& l, int H, float t) {
    LensD L;
    L.K = l.aperture_radius * (float)H / t;
    L.izf = 1.f / l.focus_dist;
    L.Ht = (float)H / t;
    L.t = t;
    L.dev = nullptr;
    return L;
}
LensD make_lensd_dev(const float* lens_dev, int H, float t) {
    LensD L{};
    L.Ht = (float)H / t;
    L.t = t;
    L.dev = lens_dev;
    return L;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct BwdWs {
    float4 *gpp, *gcrec, *gcrt, *spb, *pfb;
    float *ghacc, *kbp;
    float2* gmom;
    double2* partial;
    int n_partial;
    size_t bytes;
};

BwdWs bwd_layout(int W, int H, char* base) {
    BwdWs b{};
    size_t px = (size_t)W * H, o = 0;
    auto take = [&](size_t n) {
        size_t at = o;
        o += up256(n);
        return base ? base + at : nullptr;
    };
    b.gpp = reinterpret_cast<float4*>(take(16 * px));
    b.gcrec = reinterpret_cast<float4*>(take(16 * px));
    b.gcrt = reinterpret_cast<float4*>(take(16 * px));
    b.spb = reinterpret_cast<float4*>(take(16 * px));
    b.pfb = reinterpret_cast<float4*>(take(32 * px));
    b.kbp = reinterpret_cast<float*>(take(4 * px));
    b.ghacc = reinterpret_cast<float*>(take(4 * px));
    b.gmom = reinterpret_cast<float2*>(take(8 * px));
    int n1 = ((W + 31) / 32) * ((H + 7) / 8), n2 = ((W + 15) / 16) * ((H + 15) / 16);
    b.n_partial = 2 * n1 + n2;
    b.partial = reinterpret_cast<double2*>(take(16 * (size_t)b.n_partial));
    b.bytes = o;
    return b;
}

int check_post(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
               const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p, const hdof_post_state* st,
               const char* who) {
    int rc;
    if ((rc = check_camera(cam, who)) || (lens && (rc = check_lens(lens, who))) || (rc = check_params(p, who)) ||
        (rc = check_gbuf(in, who, false)))
        return rc;
    HDOF_CHECK_ARG(in->dtype_nd == HDOF_F32 && in->dtype_col == HDOF_F32, "%s: the differentiable path is FP32", who);
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height, "%s: gbuf/camera size mismatch", who);
    HDOF_CHECK_ARG(spp && rec && ray_off && st, "%s: spp, rec, ray_off and state are required", who);
    HDOF_CHECK_ARG(st->rt && st->crt && st->hacc && st->mom && st->hlen && st->crec && st->sp_aux && st->pp &&
                       st->pp_aux && st->out,
                   "%s: every state buffer is required", who);
    HDOF_CHECK_ARG(!lens || lens->aperture_radius > 0.f, "%s: the lens gradient needs an aperture > 0", who);
    if (p->alpha_k != 0.f || p->blades != 0 || p->aberration != 0.f || p->spec_pref != 0.f) {
        set_error("%s: the differentiable path takes the fixed EMA weight, the uniform circular lens and no "
                  "specular preference (alpha_k, blades, aberration and spec_pref must be 0)", who);
        return HDOF_EUNSUPPORTED;
    }
    return HDOF_OK;
}

}  // namespace
}  // namespace hdof

using namespace hdof;

extern "C" size_t hdof_post_workspace_bytes(int32_t width, int32_t height, const hdof_params* p) {
    if (width <= 0 || height <= 0) return 0;
    size_t pf = ws_layout(width, height, p).pf;
    size_t bw = bwd_layout(width, height, nullptr).bytes;
    return pf > bw ? pf : bw;
}

namespace hdof {
namespace {

// the forward with the lens as a host record (lens) or on the device (lens_dev)
int post_forward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                 const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens, const float* lens_dev,
                 const hdof_params* p, const hdof_post_state* st, void* workspace, size_t workspace_bytes,
                 void* stream, const char* who) {
    clear_error();
    int rc;
    if ((rc = check_post(in, spp, rec, ray_off, cam, lens, p, st, who))) return rc;
    const int W = in->width, H = in->height;
    HDOF_CHECK_ARG(workspace && workspace_bytes >= hdof_post_workspace_bytes(W, H, p), "%s: workspace of %zu bytes < %zu",
                   who, workspace_bytes, hdof_post_workspace_bytes(W, H, p));
    cudaStream_t s = as_stream(stream);
    const float t = cam->tan_half_fovy;
    LensD L = lens ? make_lensd(*lens, H, t) : make_lensd_dev(lens_dev, H, t);
    dim3 g1((W + 31) / 32, (H + 7) / 8);
    k_replay<<<g1, 256, 0, s>>>(reinterpret_cast<const float4*>(rec), ray_off, spp, W, H, L,
                                reinterpret_cast<float4*>(st->rt));
    k_temporal_frozen<<<g1, 256, 0, s>>>(reinterpret_cast<const float4*>(st->rt), spp,
                                         reinterpret_cast<const float4*>(hist_samples), W, H, p->ema_alpha,
                                         p->camera_moved, reinterpret_cast<float4*>(st->crt), st->hacc,
                                         reinterpret_cast<float2*>(st->mom), st->hlen);
    HDOF_LAUNCHED("post-path forward: replay/temporal");
    if ((rc = launch_spatial(reinterpret_cast<const float4*>(st->crt), reinterpret_cast<const float2*>(st->mom),
                             st->hlen, W, H, p->r_s, p->var_ref, reinterpret_cast<float4*>(st->crec),
                             reinterpret_cast<float4*>(st->sp_aux), s)))
        return rc;
    // with lens_dev the kernels replace coc's lens by the device one
    const hdof_lens unit = {1.f, 1.f, 1.f};
    const Coc coc = make_coc(lens ? *lens : unit, H, t);
    if ((rc = launch_postfilter(in, coc, p, st->pp, reinterpret_cast<float4*>(st->pp_aux), workspace, s, lens_dev, t)))
        return rc;
    return launch_composite(in, spp, st->pp, nullptr, st->crt, st->crec, st->hacc, coc, p->h_tau, 0.f, st->out, s,
                            lens_dev, t);
}

// the backward with the lens as a host record (lens) or on the device (lens_dev)
int post_backward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                  const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens, const float* lens_dev,
                  const hdof_params* p, const hdof_post_state* st, const float* grad_out, float* grad_col,
                  float* grad_lens, void* workspace, size_t workspace_bytes, void* stream, const char* who) {
    clear_error();
    int rc;
    if ((rc = check_post(in, spp, rec, ray_off, cam, lens, p, st, who))) return rc;
    HDOF_CHECK_ARG(grad_out && grad_col && grad_lens, "%s: grad_out, grad_col, grad_lens required", who);
    const int W = in->width, H = in->height;
    HDOF_CHECK_ARG(workspace && workspace_bytes >= hdof_post_workspace_bytes(W, H, p), "%s: workspace of %zu bytes < %zu",
                   who, workspace_bytes, hdof_post_workspace_bytes(W, H, p));
    cudaStream_t s = as_stream(stream);
    if ((rc = ensure_area_table(s))) return rc;
    const float4* tab = nullptr;
    int ntab = 0;
    if ((rc = area_table(&tab, &ntab))) return rc;
    BwdWs b = bwd_layout(W, H, static_cast<char*>(workspace));
    LensD L = lens ? make_lensd(*lens, H, cam->tan_half_fovy) : make_lensd_dev(lens_dev, H, cam->tan_half_fovy);
    const float4* nd = static_cast<const float4*>(in->nd);
    const float4* col = static_cast<const float4*>(in->col);
    float4* gcol = reinterpret_cast<float4*>(grad_col);
    dim3 g1((W + 31) / 32, (H + 7) / 8), g2((W + 15) / 16, (H + 15) / 16);
    const int n1 = g1.x * g1.y;
    HDOF_CUDA(cudaMemsetAsync(b.gcrt, 0, 16 * (size_t)W * H, s), "post-path backward: clear");
    HDOF_CUDA(cudaMemsetAsync(b.gmom, 0, 8 * (size_t)W * H, s), "post-path backward: clear");
    k_composite_bwd<<<g1, 256, 0, s>>>(nd, col, spp, reinterpret_cast<const float4*>(st->pp),
                                       reinterpret_cast<const float4*>(st->crt), reinterpret_cast<const float4*>(st->crec),
                                       st->hacc, reinterpret_cast<const float4*>(grad_out), W, H, L, p->h_tau, gcol, b.gpp,
                                       b.gcrec, b.gcrt, b.ghacc, b.partial);
    k_spatial_bwd_prep<<<g1, 256, 0, s>>>(reinterpret_cast<const float4*>(st->crt),
                                          reinterpret_cast<const float2*>(st->mom), st->hlen,
                                          reinterpret_cast<const float4*>(st->sp_aux), b.gcrec, W, H, p->var_ref, b.spb,
                                          b.gcrt, b.gmom);
    k_spatial_bwd<<<g2, 256, 0, s>>>(reinterpret_cast<const float4*>(st->crt), b.spb, W, H, p->r_s, b.gcrt);
    k_temporal_replay_bwd<<<g1, 256, 0, s>>>(reinterpret_cast<const float4*>(rec), ray_off, spp,
                                             reinterpret_cast<const float4*>(hist_samples), b.gcrt, b.ghacc, b.gmom, W,
                                             H, L, p->ema_alpha, p->camera_moved, b.partial + n1);
    k_pf_bwd_prep<<<g1, 256, 0, s>>>(reinterpret_cast<const float4*>(st->pp_aux), b.gpp, nd, p->kz_rel, W, H, b.pfb,
                                     b.kbp, gcol);
    k_pf_bwd<<<g2, 64, 0, s>>>(nd, col, b.pfb, b.kbp, tab, ntab, W, H, L, p->r_max, p->kz_rel, gcol,
                               b.partial + 2 * n1);
    k_reduce<<<1, 1024, 0, s>>>(b.partial, b.n_partial, grad_lens);
    HDOF_LAUNCHED("post-path backward");
    return HDOF_OK;
}

}  // namespace
}  // namespace hdof

extern "C" int hdof_post_forward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                                 const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens,
                                 const hdof_params* p, const hdof_post_state* st, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    if (!lens) {
        clear_error();
        set_error("hdof_post_forward: lens is required");
        return HDOF_EINVAL;
    }
    return post_forward(in, spp, rec, ray_off, hist_samples, cam, lens, nullptr, p, st, workspace, workspace_bytes,
                        stream, "hdof_post_forward");
}

extern "C" int hdof_post_forward_dlens(const hdof_gbuf* in, const uint8_t* spp, const float* rec,
                                       const uint32_t* ray_off, const float* hist_samples, const hdof_camera* cam,
                                       const float* lens_dev, const hdof_params* p, const hdof_post_state* st,
                                       void* workspace, size_t workspace_bytes, void* stream) {
    if (!lens_dev) {
        clear_error();
        set_error("hdof_post_forward_dlens: lens_dev is required");
        return HDOF_EINVAL;
    }
    return post_forward(in, spp, rec, ray_off, hist_samples, cam, nullptr, lens_dev, p, st, workspace,
                        workspace_bytes, stream, "hdof_post_forward_dlens");
}

extern "C" int hdof_post_backward(const hdof_gbuf* in, const uint8_t* spp, const float* rec, const uint32_t* ray_off,
                                  const float* hist_samples, const hdof_camera* cam, const hdof_lens* lens,
                                  const hdof_params* p, const hdof_post_state* st, const float* grad_out,
                                  float* grad_col, float* grad_lens, void* workspace, size_t workspace_bytes,
                                  void* stream) {
    if (!lens) {
        clear_error();
        set_error("hdof_post_backward: lens is required");
        return HDOF_EINVAL;
    }
    return post_backward(in, spp, rec, ray_off, hist_samples, cam, lens, nullptr, p, st, grad_out, grad_col,
                         grad_lens, workspace, workspace_bytes, stream, "hdof_post_backward");
}

extern "C" int hdof_post_backward_dlens(const hdof_gbuf* in, const uint8_t* spp, const float* rec,
                                        const uint32_t* ray_off, const float* hist_samples, const hdof_camera* cam,
                                        const float* lens_dev, const hdof_params* p, const hdof_post_state* st,
                                        const float* grad_out, float* grad_col, float* grad_lens, void* workspace,
                                        size_t workspace_bytes, void* stream) {
    if (!lens_dev) {
        clear_error();
        set_error("hdof_post_backward_dlens: lens_dev is required");
        return HDOF_EINVAL;
    }
    return post_backward(in, spp, rec, ray_off, hist_samples, cam, nullptr, lens_dev, p, st, grad_out, grad_col,
                         grad_lens, workspace, workspace_bytes, stream, "hdof_post_backward_dlens");
}
