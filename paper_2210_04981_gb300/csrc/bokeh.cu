// Shaped bokeh for the post-filter (the paper's Discussion: bokeh shapes
// other than the uniform circle, by the shape of the sampling kernel and the
// relative weight of its samples).  Used by hdof_postfilter when
// p->blades >= 3 or p->aberration != 0; the circular path stays as it is.
//
// The thin lens images the aperture point O of a source at CoC c onto the
// screen offset (c / 2A)(-O_right, O_up) (screen y grows downwards): a near
// source's bokeh is the aperture scaled to radius |c|/2 and mirrored
// left-right, a far source's mirrored top-bottom.  With the aperture norm
// D(v) = |v| cos(m - pi/N) / cos(pi/N), m = (atan2(v) - rot) mod 2pi/N (the
// N-gon is {D <= A}; the disk: D = |v|), a source q = p + (dx, dy) weighs at
// receiver p
//   near: s(r_q - D(dx, -dy)) w,   far: s(r_q - D(-dx, dy)) w,
//   w = 1 + aberration (2 min(d / r_q, 1)^2 - 1) (1 while r_q < 1), d = |(dx, dy)|,
// normalised by the weighted lattice area a(r) = sum_o s(r - D(o)) w(|o|, r)
// (mirrors map the lattice onto itself, so one area serves both layers).
//
// k_bokeh_norm: D over the window's offsets (a table, built per call).
// k_bokeh_area: a(r) on r = k / 256 (a table); the prep evaluates a(r)
//   exactly for r < 8 and interpolates the table above, where the table's
//   relative error is below 1e-6.
// k_bokeh_prep: per pixel r + 1/2, z and the premultiplied near and far
//   records; per 16x16 tile the largest radius.
// k_bokeh_gather: one thread per pixel over the disk of the largest radius
//   that reaches its tile (D >= d, so taps outside it weigh 0).
#include <cmath>

#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

constexpr int BT = 16;                  // pixel tile of the prep and the gather
constexpr float AREA_STEP = 1.f / 256.f;
constexpr float EXACT_R = 8.f;          // below: the area summed per pixel

struct Shape {
    int K;           // norm table covers offsets [-K, K]^2
    const float* D;  // (2K + 1)^2 aperture norms, row-major in (dy, dx)
    float ab;        // aberration
};

__device__ __forceinline__ float norm_at(const Shape& s, int dx, int dy) {
    return __ldg(&s.D[(dy + s.K) * (2 * s.K + 1) + dx + s.K]);
}
__device__ __forceinline__ float radial_w(const Shape& s, float r, float d) {
    if (r < 1.f) return 1.f;
    const float t = fminf(d / r, 1.f);
    return 1.f + s.ab * (2.f * t * t - 1.f);
}
__device__ __forceinline__ float soft(float x) { return fminf(fmaxf(x + 0.5f, 0.f), 1.f); }

// a(r) by its definition over the lattice
__device__ float area_exact(const Shape& s, float r) {
    const int k = (int)ceilf(r + 0.5f);
    float a = 0.f;
    for (int dy = -k; dy <= k; ++dy)
        for (int dx = -k; dx <= k; ++dx) {
            const float w = soft(r - norm_at(s, dx, dy));
            if (w > 0.f) a += w * radial_w(s, r, sqrtf((float)(dx * dx + dy * dy)));
        }
    return a;
}

__global__ void __launch_bounds__(256) k_bokeh_norm(int K, int blades, float rot, float* __restrict__ D) {
    const int n = 2 * K + 1;
    for (int e = blockIdx.x * 256 + threadIdx.x; e < n * n; e += gridDim.x * 256) {
        const int dx = e % n - K, dy = e / n - K;
        const float d = sqrtf((float)(dx * dx + dy * dy));
        float v = d;
        if (blades >= 3 && d > 0.f) {
            const float sect = 6.28318530717958648f / blades;
            float m = fmodf(atan2f((float)dy, (float)dx) - rot, sect);
            if (m < 0.f) m += sect;
            v = d * cosf(m - 0.5f * sect) / cosf(0.5f * sect);
        }
        D[e] = v;
    }
}

// one block per table entry r = k / 256: block sum over the lattice in a fixed order
__global__ void __launch_bounds__(256) k_bokeh_area(Shape s, int n_r, float* __restrict__ area) {
    const int k = blockIdx.x;
    if (k >= n_r) return;
    const float r = k * AREA_STEP;
    const int kk = (int)ceilf(r + 0.5f), n = 2 * kk + 1;
    float a = 0.f;
    for (int e = threadIdx.x; e < n * n; e += 256) {
        const int dx = e % n - kk, dy = e / n - kk;
        const float w = soft(r - norm_at(s, dx, dy));
        if (w > 0.f) a += w * radial_w(s, r, sqrtf((float)(dx * dx + dy * dy)));
    }
    __shared__ float red[256];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) area[k] = red[0];
}

template <class ND, class COL>
struct BokehPrep {
    const ND* nd;
    const COL* col;
    int W, H, ntx;
    Coc coc;
    float rmax;
    Shape s;
    const float* area;  // a(k / 256)
    int n_r;
    float* rh;
    float* zq;
    float4* nrec;
    float4* frec;
    float* tmax;
};

template <class ND, class COL>
__global__ void __launch_bounds__(256) k_bokeh_prep(BokehPrep<ND, COL> a) {
    const int i = blockIdx.x * BT + (threadIdx.x & 15), j = blockIdx.y * BT + (threadIdx.x >> 4);
    float rt = -1.f;
    if (i < a.W && j < a.H) {
        const size_t q = (size_t)j * a.W + i;
        const float z = ldz(a.nd + q), c = a.coc(z);
        const float r = fminf(fabsf(c) * 0.5f, a.rmax);
        float ar;
        if (r < EXACT_R) {
            ar = area_exact(a.s, r);
        } else {
            const float u = r / AREA_STEP;
            const int k = min((int)u, a.n_r - 2);
            const float f = u - (float)k;
            ar = fmaf(f, __ldg(&a.area[k + 1]) - __ldg(&a.area[k]), __ldg(&a.area[k]));
        }
        const float ia = 1.f / ar, wn = w_near(c), an = wn * ia, af = (1.f - wn) * ia;
        const float4 col = ld4(a.col + q);
        a.rh[q] = r + 0.5f;
        a.zq[q] = z;
        a.nrec[q] = make_float4(col.x * an, col.y * an, col.z * an, an);
        a.frec[q] = make_float4(col.x * af, col.y * af, col.z * af, af);
        rt = r;
    }
    for (int o = 16; o; o >>= 1) rt = fmaxf(rt, __shfl_xor_sync(0xffffffffu, rt, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rt;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = red[0];
        for (int k = 1; k < 8; ++k) m = fmaxf(m, red[k]);
        a.tmax[blockIdx.y * a.ntx + blockIdx.x] = m;
    }
}

template <class COL>
struct BokehGather {
    const float* rh;
    const float* zq;
    const float4* nrec;
    const float4* frec;
    const COL* col;
    const float* tmax;
    int W, H, ntx, nty, kt;
    float kz_rel;
    Shape s;
    float4* out;
};

template <class COL>
__global__ void __launch_bounds__(256) k_bokeh_gather(BokehGather<COL> a) {
    // reach of this tile: the largest radius + 1/2 among tiles that can reach it
    __shared__ float s_reach;
    if (threadIdx.x == 0) s_reach = 0.f;
    __syncthreads();
    {
        const int n = 2 * a.kt + 1;
        for (int e = threadIdx.x; e < n * n; e += 256) {
            const int tx = (int)blockIdx.x + e % n - a.kt, ty = (int)blockIdx.y + e / n - a.kt;
            if (tx < 0 || ty < 0 || tx >= a.ntx || ty >= a.nty) continue;
            const float r = __ldg(&a.tmax[ty * a.ntx + tx]);
            if (r < 0.f) continue;
            const int gx = max(abs(tx - (int)blockIdx.x) - 1, 0) * BT, gy = max(abs(ty - (int)blockIdx.y) - 1, 0) * BT;
            const float gap = sqrtf((float)(gx * gx + gy * gy));
            if (gap < r + 0.5f) atomicMax(reinterpret_cast<unsigned*>(&s_reach), __float_as_uint(r + 0.5f));
        }
    }
    __syncthreads();
    const int i = blockIdx.x * BT + (threadIdx.x & 15), j = blockIdx.y * BT + (threadIdx.x >> 4);
    if (i >= a.W || j >= a.H) return;
    const float R = s_reach;
    const int G = (int)ceilf(R);
    const float zp = __ldg(&a.zq[(size_t)j * a.W + i]);
    const float ka = 1.f / (a.kz_rel * zp);
    float4 Sn = make_float4(0.f, 0.f, 0.f, 0.f), Sf = Sn;
    for (int dy = max(-G, -j); dy <= min(G, a.H - 1 - j); ++dy) {
        const int w = (int)floorf(sqrtf(fmaxf(R * R - (float)(dy * dy), 0.f)));
        for (int dx = max(-w, -i); dx <= min(w, a.W - 1 - i); ++dx) {
            const size_t q = (size_t)(j + dy) * a.W + (i + dx);
            const float rh = __ldg(&a.rh[q]);
            const float d = sqrtf((float)(dx * dx + dy * dy));
            if (d >= rh) continue;  // D >= d: zero weight in both layers
            const float r = rh - 0.5f, rw = radial_w(a.s, r, d);
            const float wn = soft(r - norm_at(a.s, dx, -dy)) * rw;
            const float kz = fminf(fmaxf(1.f - (__ldg(&a.zq[q]) - zp) * ka, 0.f), 1.f);
            const float wf = soft(r - norm_at(a.s, -dx, dy)) * rw * kz;
            const float4 n4 = __ldg(&a.nrec[q]), f4 = __ldg(&a.frec[q]);
            Sn = make_float4(fmaf(wn, n4.x, Sn.x), fmaf(wn, n4.y, Sn.y), fmaf(wn, n4.z, Sn.z), fmaf(wn, n4.w, Sn.w));
            Sf = make_float4(fmaf(wf, f4.x, Sf.x), fmaf(wf, f4.y, Sf.y), fmaf(wf, f4.z, Sf.z), fmaf(wf, f4.w, Sf.w));
        }
    }
    const size_t p = (size_t)j * a.W + i;
    const float4 cp = ld4(a.col + p);
    const float alpha = fminf(fmaxf(Sn.w, 0.f), 1.f);
    const float in = Sn.w > HDOF_PP_MIN_W ? 1.f / Sn.w : 0.f;
    const bool fok = Sf.w > HDOF_PP_MIN_W;
    const float inf_ = fok ? 1.f / Sf.w : 0.f;
    const float3 N = f3(Sn.x * in, Sn.y * in, Sn.z * in);
    const float3 F = fok ? f3(Sf.x * inf_, Sf.y * inf_, Sf.z * inf_) : f3(cp.x, cp.y, cp.z);
    a.out[p] = make_float4(alpha * N.x + (1.f - alpha) * F.x, alpha * N.y + (1.f - alpha) * F.y,
                           alpha * N.z + (1.f - alpha) * F.z, alpha);
}

}  // namespace

bool bokeh_shaped(const hdof_params* p) { return p->blades >= 3 || p->aberration != 0.f; }

size_t bokeh_scratch_bytes(const hdof_params* p) {
    const int K = (int)std::ceil((p ? p->r_max : 100.f) + 0.5f) + 1;
    const size_t n_r = (size_t)((p ? p->r_max : 100.f) / AREA_STEP) + 2;
    return (((size_t)(2 * K + 1) * (2 * K + 1) * sizeof(float) + 255) & ~size_t(255)) +
           ((n_r * sizeof(float) + 255) & ~size_t(255));
}

// the shaped post-filter (scratch: the post-filter regions, then bokeh_scratch_bytes)
int launch_bokeh(const hdof_gbuf* in, const Coc& coc, const hdof_params* p, float* pp, void* scratch,
                 cudaStream_t s) {
    const int W = in->width, H = in->height;
    const WsLayout L = ws_layout(W, H, p);
    ViewWs w = {};
    pf_regions(w, static_cast<char*>(scratch), L);
    char* extra = static_cast<char*>(scratch) + L.pf - L.pf_bokeh;
    const int K = (int)std::ceil(p->r_max + 0.5f) + 1;
    const int n_r = (int)(p->r_max / AREA_STEP) + 2;
    float* D = reinterpret_cast<float*>(extra);
    float* area = reinterpret_cast<float*>(extra + (((size_t)(2 * K + 1) * (2 * K + 1) * sizeof(float) + 255) &
                                                    ~size_t(255)));
    Shape sh{K, D, p->aberration};
    ProfScope ps_("pf_bokeh", s);
    k_bokeh_norm<<<(unsigned)std::min((2 * K + 1) * (2 * K + 1) / 256 + 1, 1024), 256, 0, s>>>(K, p->blades,
                                                                                                p->blade_rot, D);
    HDOF_LAUNCHED("post-filter bokeh: norm table");
    k_bokeh_area<<<n_r, 256, 0, s>>>(sh, n_r, area);
    HDOF_LAUNCHED("post-filter bokeh: area table");
    const int ntx = (W + BT - 1) / BT, nty = (H + BT - 1) / BT;
    dim3 grid(ntx, nty);
    float* tmax = reinterpret_cast<float*>(w.tmax);  // one float per tile suffices here
    const bool f32n = in->dtype_nd == HDOF_F32, f32c = in->dtype_col == HDOF_F32;
    const float4* nd4 = static_cast<const float4*>(in->nd);
    const half4s* ndh = static_cast<const half4s*>(in->nd);
    const float4* col4 = static_cast<const float4*>(in->col);
    const bf164s* colb = static_cast<const bf164s*>(in->col);
    if (f32n && f32c)
        k_bokeh_prep<<<grid, 256, 0, s>>>(BokehPrep<float4, float4>{nd4, col4, W, H, ntx, coc, p->r_max, sh, area, n_r,
                                                                    w.rh, w.zq, w.nrec, w.frec, tmax});
    else if (f32n)
        k_bokeh_prep<<<grid, 256, 0, s>>>(BokehPrep<float4, bf164s>{nd4, colb, W, H, ntx, coc, p->r_max, sh, area,
                                                                    n_r, w.rh, w.zq, w.nrec, w.frec, tmax});
    else if (f32c)
        k_bokeh_prep<<<grid, 256, 0, s>>>(BokehPrep<half4s, float4>{ndh, col4, W, H, ntx, coc, p->r_max, sh, area,
                                                                    n_r, w.rh, w.zq, w.nrec, w.frec, tmax});
    else
        k_bokeh_prep<<<grid, 256, 0, s>>>(BokehPrep<half4s, bf164s>{ndh, colb, W, H, ntx, coc, p->r_max, sh, area,
                                                                    n_r, w.rh, w.zq, w.nrec, w.frec, tmax});
    HDOF_LAUNCHED("post-filter bokeh: prep");
    const int kt = (int)std::ceil((p->r_max + 0.5f) / BT) + 1;
    float4* out = reinterpret_cast<float4*>(pp);
    if (f32c)
        k_bokeh_gather<<<grid, 256, 0, s>>>(BokehGather<float4>{w.rh, w.zq, w.nrec, w.frec, col4, tmax, W, H, ntx, nty,
                                                                kt, p->kz_rel, sh, out});
    else
        k_bokeh_gather<<<grid, 256, 0, s>>>(BokehGather<bf164s>{w.rh, w.zq, w.nrec, w.frec, colb, tmax, W, H, ntx,
                                                                nty, kt, p->kz_rel, sh, out});
    HDOF_LAUNCHED("post-filter bokeh: gather");
    return HDOF_OK;
}

}  // namespace hdof
