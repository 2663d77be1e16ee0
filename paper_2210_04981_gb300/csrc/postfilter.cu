// post-process CoC filter of the sharp image (Design section: the sharp
// rasterised image is blurred by a post-process filter; the Reconstruction
// section gives the gather's rejection rule: a sample counts only if its CoC
// radius reaches the pixel).
//
// Scatter-as-gather with soft disks.  Pixel q scatters its colour over
// s(r_q - d), s(x) = clamp(x + 1/2, 0, 1), r_q = min(|c(z_q)|/2, r_max),
// normalised by the disk's lattice area a(r) = sum_o s(r - |o|) so that each
// pixel scatters unit weight.  a(r) is piecewise linear in r with breaks at
// |o| +- 1/2; a table of its breakpoints is built once per device and
// evaluated by binary search, which is exact up to float rounding.
//
// k_pf_prep: per pixel r + 1/2, z and the premultiplied near and far layer
//   records (c w/a, w/a), row-major; per 16x16
//   tile the largest r feeding each layer and the smallest r feeding the near
//   layer.
// k_pf_rowscan: the row prefix of the near records (row-major).
// k_pf_gather: near and far are gathered in two loops, each bounded per tile
//   by the largest radius among the tiles whose pixels feed that layer and
//   can reach it, and per source row to the columns of that disk; every tap
//   outside has zero weight, so the bounded gathers equal the full ones.
//   Where every near source close to the tile has a large radius, the near
//   taps of weight exactly 1 (the interior) are summed as differences of the
//   row prefix and only the ring around them is tapped.  Each thread gathers
//   a 2x2 pixel block so every tap it loads serves four pixels; the per-tap
//   arithmetic is branch-free (saturating adds).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

constexpr int TP = HDOF_TILE_PF;
#ifndef HDOF_PF_RY
#define HDOF_PF_RY 2  // pixel rows per gather thread (each thread gathers 2 x RY pixels)
#endif
constexpr int PF_RY = HDOF_PF_RY;
constexpr int PF_NPX = 2 * PF_RY;
constexpr int GATHER_THREADS = 8 * (16 / PF_RY);
#ifndef HDOF_PF_MINB
#define HDOF_PF_MINB 16  // resident gather blocks per SM the register budget targets
#endif
#ifndef HDOF_PF_UNROLL
#define HDOF_PF_UNROLL 1  // unroll of the gather's tap-pair loop (1, 2, 4, 8 swept: 1 fastest)
#endif
constexpr int PF_UNROLL = HDOF_PF_UNROLL;
// Shared-memory carve-out (percent of the maximum) for the gather: the taps
// are served from L1, so keep L1 large, but every resident block also holds
// ~1 KB of driver-reserved shared memory; 8% (a 16 KB configuration) admits
// about 14-15 blocks, where the minimum configuration (8 KB) admits only 7
// and a 32 KB one leaves too little L1 for the taps.
#ifndef HDOF_PF_CARVEOUT
#define HDOF_PF_CARVEOUT 8
#endif
constexpr int GATHER_CARVEOUT = HDOF_PF_CARVEOUT;
constexpr int AREA_MAX = 16384;  // breakpoints for radii up to 127.5

// (x_m, a(x_m), slope on [x_m, x_{m+1}], 0)
__device__ float4 g_area[AREA_MAX];
__device__ int g_area_n;

__device__ __forceinline__ float disk_area(float r) {
    int lo = 0, hi = g_area_n - 1;  // largest m with x_m <= r
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&g_area[mid].x) <= r) lo = mid;
        else hi = mid - 1;
    }
    float4 e = __ldg(&g_area[lo]);
    return fmaf(e.z, r - e.x, e.y);
}

// Per source pixel q the gather reads r_q + 1/2, z_q and two premultiplied
// layer records (c_q w/a, w/a) with w = w_near(q) for the near layer and
// 1 - w_near(q) for the far layer; per 16x16 tile, the largest r among its
// pixels that feed each layer (-1: none).  Outside the thin focus zone a
// pixel feeds one layer only, so near and far are gathered in separate loops
// with their own windows (in the workloads here the far field's blur is
// small and the near field's large).
// Layer records in the colour's precision: FP32 colour, float4 records; BF16
// colour (the mixed form), BF16 records (8 bytes: a pair of taps in one
// 128-bit load), accumulated in FP32 like the FP32 ones.
template <class COL>
struct RecOf {
    using T = float4;
};
template <>
struct RecOf<bf164s> {
    using T = bf164s;
};

template <class ND, class COL>
struct PrepArgs {
    const ND* nd;
    const COL* col;
    int W, H;
    Coc coc;
    float rmax;
    int ntx;
    float* rh;      // r + 1/2
    float* zq;      // view depth
    typename RecOf<COL>::T* nrec;  // (c w/a, w/a), near layer
    typename RecOf<COL>::T* frec;  // (c (1-w)/a, (1-w)/a), far layer
    float4* tmax;   // per tile: (max r feeding near, max r feeding far, min r feeding near (+inf: none), 0)
    const float* lens;  // optional (focus distance, aperture radius) on the device, replacing coc's lens
    float t;            // tan(fovy / 2), with lens
};

template <class ND, class COL>
__device__ __forceinline__ void pf_prep_body(const PrepArgs<ND, COL>& a, int bx, int by) {
    const int W = a.W, H = a.H;
    int i = bx * TP + (threadIdx.x & 15), j = by * TP + (threadIdx.x >> 4);
    const float INF = __int_as_float(0x7f800000);
    float rn = -1.f, rf = -1.f, rnmin = INF;
    if (i < W && j < H) {
        size_t q = (size_t)j * W + i;
        float z = ldz(a.nd + q);
        float c = lens_coc(a.coc, a.lens, H, a.t)(z);
        float r = fminf(fabsf(c) * 0.5f, a.rmax);
        float ia = 1.f / disk_area(r);
        float wn = w_near(c), an = wn * ia, af = (1.f - wn) * ia;
        float4 col = ld4(a.col + q);
        a.rh[q] = r + 0.5f;
        a.zq[q] = z;
        st4(a.nrec + q, make_float4(col.x * an, col.y * an, col.z * an, an));
        st4(a.frec + q, make_float4(col.x * af, col.y * af, col.z * af, af));
        rn = wn > 0.f ? r : -1.f;
        rf = wn < 1.f ? r : -1.f;
        rnmin = wn > 0.f ? r : INF;
    }
    for (int o = 16; o; o >>= 1) {
        rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, o));
        rf = fmaxf(rf, __shfl_xor_sync(0xffffffffu, rf, o));
        rnmin = fminf(rnmin, __shfl_xor_sync(0xffffffffu, rnmin, o));
    }
    __shared__ float4 red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float4(rn, rf, rnmin, 0.f);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 m = red[0];
        for (int k = 1; k < 8; ++k)
            m = make_float4(fmaxf(m.x, red[k].x), fmaxf(m.y, red[k].y), fminf(m.z, red[k].z), 0.f);
        a.tmax[by * a.ntx + bx] = m;
    }
}

template <class ND, class COL>
__global__ void __launch_bounds__(256) k_pf_prep(PrepArgs<ND, COL> a) { pf_prep_body(a, blockIdx.x, blockIdx.y); }

// Row prefix of the near records: pre[y][x] = sum over x' <= x of the near
// record of pixel (x', y), row-major.  The gather sums a pixel's interior
// taps (all of weight exactly 1) as differences of it.  One block per row,
// in rounds of 256 consecutive pixels (a block scan per round plus the
// running total): the summation order is fixed.
template <class REC>
struct RowScanArgsT {
    const REC* nrec;  // row-major
    int W, H;
    float4* pre;
};
using RowScanArgs = RowScanArgsT<float4>;

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

template <class REC>
__device__ __forceinline__ void pf_rowscan_body(const RowScanArgsT<REC>& a, int y) {
    const int W = a.W, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const size_t row = (size_t)y * W;
    __shared__ float4 s_warp[8];
    float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int x0 = 0; x0 < W; x0 += 256) {
        const int x = x0 + t;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < W) {
            v = ld4(a.nrec + row + x);
        }
        // inclusive warp scan, then the warps' totals
        for (int o = 1; o < 32; o <<= 1) {
            const float4 u = make_float4(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o),
                                         __shfl_up_sync(0xffffffffu, v.z, o), __shfl_up_sync(0xffffffffu, v.w, o));
            if (lane >= o) v = add4(v, u);
        }
        if (lane == 31) s_warp[w] = v;
        __syncthreads();
        float4 before = carry;
        for (int k = 0; k < w; ++k) before = add4(before, s_warp[k]);
        if (x < W) a.pre[row + x] = add4(before, v);
        float4 total = carry;
        for (int k = 0; k < 8; ++k) total = add4(total, s_warp[k]);
        carry = total;
        __syncthreads();
    }
}

template <class REC>
__global__ void __launch_bounds__(256) k_pf_rowscan(RowScanArgsT<REC> a) { pf_rowscan_body(a, blockIdx.x); }

// Per target pixel: a layer's sums (S.x, S.y) and (S.z, W) as register
// pairs so one packed FMA updates two of them; the far layer also holds its
// depth test's constants ka, kb.
struct NearAcc {
    float2 xy, zw;
};
struct FarAcc {
    float2 xy, zw;
    float ka, kb;
};

// (c.x, c.y) + s (e.x, e.y), each lane rounded once as fmaf would
__device__ __forceinline__ float2 fma2(float s, float ex, float ey, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 ps, pe, pc, pr;\n\t"
        "mov.b64 ps, {%2, %2};\n\t"
        "mov.b64 pe, {%3, %4};\n\t"
        "mov.b64 pc, {%5, %6};\n\t"
        "fma.rn.f32x2 pr, ps, pe, pc;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(s), "f"(ex), "f"(ey), "f"(c.x), "f"(c.y));
    return r;
}

// far = (S.x, S.y, S.z, W) of the far layer
template <class COL>
__device__ __forceinline__ float4 pf_finish(const NearAcc& a, const float4& far, const COL* col, size_t pq,
                                            float4* aux) {
    const float3 Sn = f3(a.xy.x, a.xy.y, a.zw.x), Sf = f3(far.x, far.y, far.z);
    const float Wn = a.zw.y, Wf = far.w;
    float alpha = clamp01(Wn);
    float3 N = Wn > HDOF_PP_MIN_W ? (1.f / Wn) * Sn : f3(0, 0, 0);
    float3 F;
    if (Wf > HDOF_PP_MIN_W) F = (1.f / Wf) * Sf;
    else {
        float4 c = ld4(col + pq);
        F = f3(c.x, c.y, c.z);
    }
    if (aux) {  // layer colours and weights, kept for the adjoint
        aux[2 * pq] = make_float4(N.x, N.y, N.z, Wn);
        aux[2 * pq + 1] = make_float4(F.x, F.y, F.z, Wf);
    }
    float3 o = alpha * N + (1.f - alpha) * F;
    return make_float4(o.x, o.y, o.z, alpha);
}

template <class COL>
struct GatherArgs {
    const float* rh;
    const float* zq;
    const typename RecOf<COL>::T* nrec;
    const typename RecOf<COL>::T* frec;
    const COL* col;  // sharp colour (empty far layer)
    const float4* tmax;
    const float4* pre;  // row prefix of the near records
    int W, H, ntx, nty, kt;
    float kz_rel;
    float4* pp;
    float4* aux;
};

// one source into one target pixel, branch-free: s = clamp(r_q + 1/2 - d, 0, 1)
// (zero outside the disk, and zero layer records, add exact zeros); `in`
// false: the tap lies in the pixel's interior, already summed (weight 0 here)
__device__ __forceinline__ void acc(NearAcc& a, float d, float rh, float, const float4& n, bool in) {
    const float s = in ? __saturatef(rh - d) : 0.f;
    a.xy = fma2(s, n.x, n.y, a.xy);
    a.zw = fma2(s, n.z, n.w, a.zw);
}
__device__ __forceinline__ void acc(FarAcc& a, float d, float rh, float zq, const float4& f, bool) {
    const float t = __saturatef(rh - d) * __saturatef(fmaf(-zq, a.kb, a.ka));
    a.xy = fma2(t, f.x, f.y, a.xy);
    a.zw = fma2(t, f.z, f.w, a.zw);
}

// One (source, thread) tap: the thread's left pixels get fresh distances,
// its right pixels the left pixels' distances of the previous tap (the same
// offsets, so the same floats), carried in c (and the squared column offset
// in pdx2).  MASK: a pixel takes the tap only if its column offset exceeds
// its interior half-width for that row (squared: win2).
template <bool MASK, class A>
__device__ __forceinline__ void pf_tap(A (&a)[PF_NPX], float (&c)[PF_RY], float& pdx2, const float (&dyk)[PF_RY],
                                       const float (&win2)[PF_RY], float dx, float r, float z, const float4& e) {
    const float dx2 = dx * dx;
#pragma unroll
    for (int k = 0; k < PF_RY; ++k) {
        const float d0 = sqrt_approx(dx2 + dyk[k]);
        acc(a[2 * k], d0, r, z, e, !MASK || dx2 > win2[k]);
        acc(a[2 * k + 1], c[k], r, z, e, !MASK || pdx2 > win2[k]);
        c[k] = d0;
    }
    pdx2 = dx2;
}

// two consecutive records (32 bytes, 32-byte aligned) in one 256-bit load
__device__ __forceinline__ void ld_rec_pair(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
// two consecutive BF16 records (16 bytes, 16-byte aligned) in one 128-bit
// load; a BF16 value is the high half of its FP32 bits
__device__ __forceinline__ void ld_rec_pair(const bf164s* p, float4& a, float4& b) {
    unsigned u0, u1, u2, u3;
    asm("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(u0), "=r"(u1), "=r"(u2), "=r"(u3) : "l"(p));
    a = make_float4(__uint_as_float(u0 << 16), __uint_as_float(u0 & 0xffff0000u), __uint_as_float(u1 << 16),
                    __uint_as_float(u1 & 0xffff0000u));
    b = make_float4(__uint_as_float(u2 << 16), __uint_as_float(u2 & 0xffff0000u), __uint_as_float(u3 << 16),
                    __uint_as_float(u3 & 0xffff0000u));
}

// The taps of source row y from column xs to xe (inclusive) for the 2 x RY
// block at (i, j).  Taps go in pairs (even, odd pixel index): one 256-bit
// load of the two records and one float2 load of r + 1/2 (and z) per pair;
// the threads of a row, two columns apart, read consecutive pairs.
template <bool NEAR, bool MASK, class A, class REC>
__device__ __forceinline__ void pf_segment(A (&a)[PF_NPX], const float (&dyk)[PF_RY], const float (&win2)[PF_RY],
                                           int xs, int xe, int i, int y, int W,
                                           const float* __restrict__ rh, const float* __restrict__ zq,
                                           const REC* __restrict__ rec) {
    const float2* __restrict__ rh2 = reinterpret_cast<const float2*>(rh);
    const float2* __restrict__ zq2 = reinterpret_cast<const float2*>(zq);
    float dx = (float)(xs - i);
    float c[PF_RY], pdx2 = (dx - 1.f) * (dx - 1.f);
#pragma unroll
    for (int k = 0; k < PF_RY; ++k) c[k] = sqrt_approx(pdx2 + dyk[k]);
    size_t g = (size_t)y * W + xs;  // pixel index of the next tap
    const size_t gend = (size_t)y * W + xe + 1;
    if (g & 1) {  // an odd first tap on its own
        const float z = NEAR ? 0.f : __ldg(&zq[g]);
        pf_tap<MASK>(a, c, pdx2, dyk, win2, dx, __ldg(&rh[g]), z, ld4(rec + g));
        ++g;
        dx += 1.f;
    }
    size_t m = g >> 1;
    const size_t mend = gend >> 1;  // pairs (2m, 2m + 1) with 2m + 1 < gend
#pragma unroll PF_UNROLL
    for (; m < mend; ++m, dx += 2.f) {
        const float2 r2 = __ldg(&rh2[m]);
        float4 e0, e1;
        ld_rec_pair(rec + 2 * m, e0, e1);
        const float2 z2 = NEAR ? make_float2(0.f, 0.f) : __ldg(&zq2[m]);
        pf_tap<MASK>(a, c, pdx2, dyk, win2, dx, r2.x, z2.x, e0);
        pf_tap<MASK>(a, c, pdx2, dyk, win2, dx + 1.f, r2.y, z2.y, e1);
    }
    if (gend & 1) {  // an even last tap on its own
        const size_t gl = gend - 1;
        const float z = NEAR ? 0.f : __ldg(&zq[gl]);
        pf_tap<MASK>(a, c, pdx2, dyk, win2, dx, __ldg(&rh[gl]), z, ld4(rec + gl));
    }
}

// One layer's loop over a disk-shaped window of radius R around the 2x2
// block at (i, j): every source feeding the layer within reach has
// r + 1/2 <= R, so only taps closer than R to one of the four pixels can
// weigh; per source row, the columns of that disk (squared distances are
// exact integers in float).
// Near layer with Rin >= 0: every source that feeds the near layer and lies
// within Rin of the block has r - 1/2 >= Rin, so a tap closer than Rin
// weighs exactly 1.  Per row, a pixel's taps within its interior half-width
// floor(sqrt(Rin^2 - dy^2)) are summed from the row prefix `pre` (two
// loads); the columns inside every pixel's interior are skipped, the rest
// are tapped with that interior masked out.
template <bool NEAR, class A, class REC>
__device__ __forceinline__ void pf_layer(A (&a)[PF_NPX], float R, float Rin, int i, int j, int W, int H,
                                         const float* __restrict__ rh, const float* __restrict__ zq,
                                         const REC* __restrict__ rec, const float4* __restrict__ pre) {
    if (R < 0.f) return;  // nothing within reach feeds this layer
    // bounds lean outwards by 1e-3 pixel (float rounding); taps they add weigh 0
    const int G = (int)floorf(R + 1e-3f);
    const int y0 = max(j - G, 0), y1 = min(j + PF_RY - 1 + G, H - 1);
    const float R2 = R * R, Rin2 = Rin * Rin;
    for (int y = y0; y <= y1; ++y) {
        const float dy = (float)(y - j);
        float dyk[PF_RY], win2[PF_RY];
#pragma unroll
        for (int k = 0; k < PF_RY; ++k) dyk[k] = (dy - (float)k) * (dy - (float)k);
        // nearest of the thread's rows to this source row
        const float dmin = dy >= 0.f && dy <= (float)(PF_RY - 1) ? 0.f : fminf(dyk[0], dyk[PF_RY - 1]);
        const int w = (int)floorf(sqrtf(fmaxf(R2 - dmin, 0.f)) + 1e-3f);
        const int x0 = max(i - w, 0), x1 = min(i + 1 + w, W - 1);
#pragma unroll
        for (int k = 0; k < PF_RY; ++k) win2[k] = -1.f;
        int wmin = -1;        // interior half-width common to the thread's rows (-1: none)
        bool masked = false;  // some row of the thread has an interior
        if (NEAR && Rin >= 0.f) {
            const float4* prow = pre + (size_t)y * W;
            wmin = 1 << 30;
#pragma unroll
            for (int k = 0; k < PF_RY; ++k) {
                // inward: no outward lean here (Rin already has its margin)
                const int wi = dyk[k] <= Rin2 ? (int)floorf(sqrtf(Rin2 - dyk[k])) : -1;
                win2[k] = wi >= 0 ? (float)(wi * wi) : -1.f;
                wmin = min(wmin, wi);
                if (wi >= 0) {
                    masked = true;
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int xa = i + b;
                        if (xa < W) {
                            const int lo = max(xa - wi, 0), hi = min(xa + wi, W - 1);
                            float4 sum = __ldg(&prow[hi]);
                            if (lo > 0) {
                                const float4 l = __ldg(&prow[lo - 1]);
                                sum = make_float4(sum.x - l.x, sum.y - l.y, sum.z - l.z, sum.w - l.w);
                            }
                            A& t = a[2 * k + b];
                            t.xy = make_float2(t.xy.x + sum.x, t.xy.y + sum.y);
                            t.zw = make_float2(t.zw.x + sum.z, t.zw.y + sum.w);
                        }
                    }
                }
            }
        }
        if (wmin >= 1) {
            // columns [i + 1 - wmin, i + wmin] lie in every pixel's interior
            const int ls = min(x1, i - wmin), rs = max(x0, i + wmin + 1);
            if (x0 <= ls) pf_segment<NEAR, true>(a, dyk, win2, x0, ls, i, y, W, rh, zq, rec);
            if (rs <= x1) pf_segment<NEAR, true>(a, dyk, win2, rs, x1, i, y, W, rh, zq, rec);
        } else if (masked) {
            pf_segment<NEAR, true>(a, dyk, win2, x0, x1, i, y, W, rh, zq, rec);
        } else {
            pf_segment<NEAR, false>(a, dyk, win2, x0, x1, i, y, W, rh, zq, rec);
        }
    }
}

// 8 x (16 / RY) threads per 16x16 tile; thread t gathers the 2 x RY pixel
// block at (2 (t & 7), RY (t >> 3)), so each loaded tap serves 2 RY pixels.
template <class COL>
__device__ __forceinline__ void pf_gather_body(const GatherArgs<COL>& ar, int tx, int ty) {
    const COL* __restrict__ col = ar.col;
    const float4* __restrict__ tmax = ar.tmax;
    const int W = ar.W, H = ar.H, ntx = ar.ntx, nty = ar.nty, kt = ar.kt;
    const int nk = (2 * kt + 1) * (2 * kt + 1);
    float4* __restrict__ pp = ar.pp;
    float4* __restrict__ aux = ar.aux;
    __shared__ int s_win[3];
    if (threadIdx.x < 2) s_win[threadIdx.x] = -1;
    if (threadIdx.x == 2) s_win[2] = 0x7f800000;  // +inf
    __syncthreads();
    // per layer: largest r + 1/2 over tiles whose feeding pixels can reach this tile
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        int ox = k % (2 * kt + 1) - kt, oy = k / (2 * kt + 1) - kt;
        int x = tx + ox, y = ty + oy;
        if (x < 0 || y < 0 || x >= ntx || y >= nty) continue;
        const float4 r = __ldg(&tmax[y * ntx + x]);
        // pixel gap between the two tiles along each axis
        const float gx = ox == 0 ? 0.f : (float)((abs(ox) - 1) * TP + 1);
        const float gy = oy == 0 ? 0.f : (float)((abs(oy) - 1) * TP + 1);
        const float g2 = gx * gx + gy * gy;
        // positive floats order as their bit patterns
        if (r.x >= 0.f && g2 < (r.x + 0.5f) * (r.x + 0.5f)) atomicMax(&s_win[0], __float_as_int(r.x + 0.5f));
        if (r.y >= 0.f && g2 < (r.y + 0.5f) * (r.y + 0.5f)) atomicMax(&s_win[1], __float_as_int(r.y + 0.5f));
    }
    __syncthreads();
    // the layer's reach R (-1: none); a source weighs only closer than R
    const float Gn = s_win[0] < 0 ? -1.f : __int_as_float(s_win[0]);
    const float Gf = s_win[1] < 0 ? -1.f : __int_as_float(s_win[1]);
    // Near interior radius of the tile: a near source q at distance d weighs
    // exactly 1 if d <= r_q - 1/2, so Rin may grow while every tile T that
    // feeds the near layer and lies closer than Rin to this one has
    // r_min(T) - 1/2 >= Rin: Rin = min over T of max(r_min(T) - 1/2, gap(T)),
    // less a margin, at most Gn.  The interior path (two prefix loads per
    // pixel and row, masked taps around it) pays only when the interior is
    // most of the window: below Rin = Gn / 2 the plain loop runs.
    if (Gn >= 0.f) {
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            int ox = k % (2 * kt + 1) - kt, oy = k / (2 * kt + 1) - kt;
            int x = tx + ox, y = ty + oy;
            if (x < 0 || y < 0 || x >= ntx || y >= nty) continue;
            const float4 r = __ldg(&tmax[y * ntx + x]);
            if (r.x < 0.f) continue;  // feeds no near layer
            const float gx = ox == 0 ? 0.f : (float)((abs(ox) - 1) * TP + 1);
            const float gy = oy == 0 ? 0.f : (float)((abs(oy) - 1) * TP + 1);
            const float lim = fmaxf(fmaxf(r.z - 0.5f, sqrtf(gx * gx + gy * gy) - 1e-3f), 0.f);
            atomicMin(&s_win[2], __float_as_int(lim));  // non-negative floats order as their bits
        }
        __syncthreads();
    }
    float Rin = Gn >= 0.f ? fminf(__int_as_float(s_win[2]), Gn) - 1e-3f : -1.f;
    if (Rin < 0.5f * Gn) Rin = -1.f;
    const int i = tx * TP + 2 * (threadIdx.x & 7), j = ty * TP + PF_RY * (threadIdx.x >> 3);
    if (i >= W || j >= H) return;
    // far layer first; its sums wait in the pixels' own pp slots (each pixel
    // is this thread's alone) so they hold no registers during the near loop
    if (Gf >= 0.f) {
        FarAcc f[PF_NPX];  // pixel (i + (k & 1), j + (k >> 1))
        const float ka = 1.f + 1.f / ar.kz_rel;  // k_z = clamp(ka - z_q kb), kb = 1 / (kz_rel z_p)
        const float z00 = __ldg(&ar.zq[(size_t)j * W + i]);
#pragma unroll
        for (int k = 0; k < PF_NPX; ++k) {
            const int x = i + (k & 1), y = j + (k >> 1);
            const float zp = x < W && y < H ? __ldg(&ar.zq[(size_t)y * W + x]) : z00;
            f[k].ka = ka;
            f[k].kb = 1.f / (ar.kz_rel * zp);
            f[k].xy = f[k].zw = make_float2(0.f, 0.f);
        }
        pf_layer<false>(f, Gf, -1.f, i, j, W, H, ar.rh, ar.zq, ar.frec, nullptr);
#pragma unroll
        for (int k = 0; k < PF_NPX; ++k) {
            const int x = i + (k & 1), y = j + (k >> 1);
            if (x < W && y < H) pp[(size_t)y * W + x] = make_float4(f[k].xy.x, f[k].xy.y, f[k].zw.x, f[k].zw.y);
        }
    }
    NearAcc a[PF_NPX];
#pragma unroll
    for (int k = 0; k < PF_NPX; ++k) a[k].xy = a[k].zw = make_float2(0.f, 0.f);
    pf_layer<true>(a, Gn, Rin, i, j, W, H, ar.rh, ar.zq, ar.nrec, ar.pre);
#pragma unroll
    for (int k = 0; k < PF_NPX; ++k) {
        const int x = i + (k & 1), y = j + (k >> 1);
        if (x < W && y < H) {
            const size_t q = (size_t)y * W + x;
            const float4 far = Gf >= 0.f ? pp[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            pp[q] = pf_finish(a[k], far, col, q, aux);
        }
    }
}

template <class COL>
__global__ void __launch_bounds__(GATHER_THREADS, HDOF_PF_MINB) k_pf_gather(GatherArgs<COL> a) {
    pf_gather_body(a, blockIdx.x, blockIdx.y);
}

using PrepF32 = PrepArgs<float4, float4>;
__global__ void __launch_bounds__(256) k_pf_rowscan_batch(const RowScanArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    pf_rowscan_body(batch_record(a, v), by);
}
__global__ void __launch_bounds__(256) k_pf_prep_batch(const PrepF32* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    pf_prep_body(batch_record(a, v), bx, by);
}
__global__ void __launch_bounds__(GATHER_THREADS, HDOF_PF_MINB)
    k_pf_gather_batch(const GatherArgs<float4>* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    pf_gather_body(batch_record(a, v), bx, by);
}

// tiles of reach around a tile: radii up to r_max (+1/2 soft edge) span this many
int gather_tiles(float r_max) { return (int)std::ceil((r_max + 0.5f) / TP) + 1; }

std::mutex g_area_mu;
bool g_area_ready[64] = {false};
int g_area_count[64] = {0};

}  // namespace

int area_table_size() { return AREA_MAX; }

int ensure_area_table(cudaStream_t s) {
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "area table: device");
    if (dev < 0 || dev >= 64) {
        set_error("area table: device index %d unsupported", dev);
        return HDOF_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_area_mu);
    if (g_area_ready[dev]) return HDOF_OK;
    // lattice distances sqrt(k) with multiplicity n(k), |o| < 128.5
    const int R = 129;
    std::vector<int> mult(R * R + 1, 0);
    for (int b = -R; b <= R; ++b)
        for (int a = -R; a <= R; ++a) {
            int k = a * a + b * b;
            if (k <= R * R) mult[k]++;
        }
    std::vector<double> rad, pre_n, pre_nr;  // sorted sqrt(k), prefix sums of n and n*sqrt(k)
    double cn = 0, cnr = 0;
    for (int k = 0; k <= R * R; ++k)
        if (mult[k]) {
            double r = std::sqrt((double)k);
            rad.push_back(r);
            cn += mult[k];
            cnr += mult[k] * r;
            pre_n.push_back(cn);
            pre_nr.push_back(cnr);
        }
    // a(x) = #{|o| <= x - 1/2} + sum_{x-1/2 < |o| < x+1/2} (x + 1/2 - |o|)
    auto area = [&](double x) {
        auto cnt_le = [&](double v, bool strict) -> int {  // number of radii (<= v) or (< v)
            return (int)(strict ? std::lower_bound(rad.begin(), rad.end(), v) - rad.begin()
                                : std::upper_bound(rad.begin(), rad.end(), v) - rad.begin());
        };
        int full = cnt_le(x - 0.5, false);
        int part_end = cnt_le(x + 0.5, true);
        double nf = full ? pre_n[full - 1] : 0.0;
        double np = (part_end ? pre_n[part_end - 1] : 0.0) - nf;
        double nrp = (part_end ? pre_nr[part_end - 1] : 0.0) - (full ? pre_nr[full - 1] : 0.0);
        return nf + (x + 0.5) * np - nrp;
    };
    std::vector<double> bp;
    for (double r : rad) {
        if (r - 0.5 <= 128.0) bp.push_back(r - 0.5);
        if (r + 0.5 <= 128.0) bp.push_back(r + 0.5);
    }
    std::sort(bp.begin(), bp.end());
    bp.erase(std::unique(bp.begin(), bp.end()), bp.end());
    if ((int)bp.size() > AREA_MAX) {
        set_error("area table: %zu breakpoints exceed %d", bp.size(), AREA_MAX);
        return HDOF_EUNSUPPORTED;
    }
    std::vector<float4> tab(bp.size());
    for (size_t m = 0; m < bp.size(); ++m) {
        double a0 = area(bp[m]);
        double slope = 0.0;
        if (m + 1 < bp.size()) slope = (area(bp[m + 1]) - a0) / (bp[m + 1] - bp[m]);
        tab[m] = make_float4((float)bp[m], (float)a0, (float)slope, 0.f);
    }
    int n = (int)tab.size();
    HDOF_CUDA(cudaMemcpyToSymbolAsync(g_area, tab.data(), sizeof(float4) * tab.size(), 0, cudaMemcpyHostToDevice, s),
              "area table: upload");
    HDOF_CUDA(cudaMemcpyToSymbolAsync(g_area_n, &n, sizeof n, 0, cudaMemcpyHostToDevice, s), "area table: upload");
    HDOF_CUDA(cudaStreamSynchronize(s), "area table: upload");
    g_area_ready[dev] = true;
    g_area_count[dev] = n;
    return HDOF_OK;
}

int area_table(const float4** tab, int* n) {
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "area table: device");
    void* p = nullptr;
    HDOF_CUDA(cudaGetSymbolAddress(&p, g_area), "area table: symbol");
    *tab = static_cast<const float4*>(p);
    *n = (dev >= 0 && dev < 64) ? g_area_count[dev] : 0;
    return HDOF_OK;
}

}  // namespace hdof

using namespace hdof;

namespace hdof {

int launch_postfilter(const hdof_gbuf* in, const Coc& coc, const hdof_params* p, float* pp, float4* aux,
                      void* scratch, cudaStream_t s, const float* lens_dev, float t) {
    if (bokeh_shaped(p)) {
        if (aux || lens_dev) {
            set_error("post-filter: shaped bokeh has no adjoint records");
            return HDOF_EUNSUPPORTED;
        }
        return launch_bokeh(in, coc, p, pp, scratch, s);
    }
    int rc;
    if ((rc = ensure_area_table(s))) return rc;
    const int W = in->width, H = in->height;
    ViewWs w = {};
    pf_regions(w, static_cast<char*>(scratch), ws_layout(W, H, p));
    const int ntx = (W + TP - 1) / TP, nty = (H + TP - 1) / TP;
    dim3 grid(ntx, nty);
    const bool f32n = in->dtype_nd == HDOF_F32, f32c = in->dtype_col == HDOF_F32;
    const float4* nd4 = static_cast<const float4*>(in->nd);
    const half4s* ndh = static_cast<const half4s*>(in->nd);
    const float4* col4 = static_cast<const float4*>(in->col);
    const bf164s* colb = static_cast<const bf164s*>(in->col);
    const float rm = p->r_max;
    {
        ProfScope ps_("pf_prep", s);
        if (f32n && f32c)
            k_pf_prep<<<grid, 256, 0, s>>>(
                PrepArgs<float4, float4>{nd4, col4, W, H, coc, rm, ntx, w.rh, w.zq, w.nrec, w.frec, w.tmax, lens_dev, t});
        else if (f32n)
            k_pf_prep<<<grid, 256, 0, s>>>(
                PrepArgs<float4, bf164s>{nd4, colb, W, H, coc, rm, ntx, w.rh, w.zq, reinterpret_cast<bf164s*>(w.nrec),
                                              reinterpret_cast<bf164s*>(w.frec), w.tmax, lens_dev, t});
        else if (f32c)
            k_pf_prep<<<grid, 256, 0, s>>>(
                PrepArgs<half4s, float4>{ndh, col4, W, H, coc, rm, ntx, w.rh, w.zq, w.nrec, w.frec, w.tmax, lens_dev, t});
        else
            k_pf_prep<<<grid, 256, 0, s>>>(
                PrepArgs<half4s, bf164s>{ndh, colb, W, H, coc, rm, ntx, w.rh, w.zq, reinterpret_cast<bf164s*>(w.nrec),
                                              reinterpret_cast<bf164s*>(w.frec), w.tmax, lens_dev, t});
        HDOF_LAUNCHED("post-filter prep");
    }
    {
        ProfScope ps_("pf_rowscan", s);
        if (f32c)
            k_pf_rowscan<float4><<<H, 256, 0, s>>>(RowScanArgsT<float4>{w.nrec, W, H, w.pre});
        else
            k_pf_rowscan<bf164s><<<H, 256, 0, s>>>(
                RowScanArgsT<bf164s>{reinterpret_cast<const bf164s*>(w.nrec), W, H, w.pre});
        HDOF_LAUNCHED("post-filter row prefix");
    }
    const int kt = gather_tiles(p->r_max);
    float4* out = reinterpret_cast<float4*>(pp);
    // the taps are served from L1: a small shared-memory carve-out
    ProfScope ps_("pf_gather", s);
    if (f32c) {
        cudaFuncSetAttribute(k_pf_gather<float4>, cudaFuncAttributePreferredSharedMemoryCarveout, GATHER_CARVEOUT);
        k_pf_gather<float4><<<grid, GATHER_THREADS, 0, s>>>(
            GatherArgs<float4>{w.rh, w.zq, w.nrec, w.frec, col4, w.tmax, w.pre, W, H, ntx, nty, kt, p->kz_rel, out,
                               aux});
    } else {
        cudaFuncSetAttribute(k_pf_gather<bf164s>, cudaFuncAttributePreferredSharedMemoryCarveout, GATHER_CARVEOUT);
        k_pf_gather<bf164s><<<grid, GATHER_THREADS, 0, s>>>(
            GatherArgs<bf164s>{w.rh, w.zq, reinterpret_cast<const bf164s*>(w.nrec),
                               reinterpret_cast<const bf164s*>(w.frec), colb, w.tmax, w.pre, W, H, ntx, nty, kt,
                               p->kz_rel, out,
                               aux});
    }
    HDOF_LAUNCHED("post-filter gather");
    return HDOF_OK;
}

}  // namespace hdof

extern "C" int hdof_postfilter(const hdof_gbuf* in, const hdof_camera* cam, const hdof_lens* lens,
                               const hdof_params* p, float* pp, void* workspace, size_t workspace_bytes,
                               void* stream) {
    clear_error();
    int rc;
    if ((rc = check_camera(cam, "hdof_postfilter")) || (rc = check_lens(lens, "hdof_postfilter")) ||
        (rc = check_params(p, "hdof_postfilter")) || (rc = check_gbuf(in, "hdof_postfilter", false)))
        return rc;
    HDOF_CHECK_ARG(pp, "hdof_postfilter: pp output is required");
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height, "hdof_postfilter: gbuf/camera size mismatch");
    WsLayout L = ws_layout(in->width, in->height, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.total, "hdof_postfilter: workspace of %zu bytes < %zu",
                   workspace_bytes, L.total);
    return launch_postfilter(in, make_coc(*lens, in->height, cam->tan_half_fovy), p, pp, nullptr,
                             static_cast<char*>(workspace) + L.pf_off, as_stream(stream));
}

namespace hdof {
namespace {

// The specular luminance (col.w) of every pixel as an opaque grey colour.
template <class COL>
__global__ void __launch_bounds__(256) k_spec_plane(const COL* __restrict__ col, size_t n, float4* __restrict__ out) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float s = ld4(col + q).w;
    out[q] = make_float4(s, s, s, s);
}

}  // namespace
}  // namespace hdof

extern "C" int hdof_postfilter_spec(const hdof_gbuf* in, const hdof_camera* cam, const hdof_lens* lens,
                                    const hdof_params* p, float* pp_spec, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    clear_error();
    int rc;
    if ((rc = check_camera(cam, "hdof_postfilter_spec")) || (rc = check_lens(lens, "hdof_postfilter_spec")) ||
        (rc = check_params(p, "hdof_postfilter_spec")) || (rc = check_gbuf(in, "hdof_postfilter_spec", false)))
        return rc;
    HDOF_CHECK_ARG(pp_spec, "hdof_postfilter_spec: pp_spec output is required");
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height,
                   "hdof_postfilter_spec: gbuf/camera size mismatch");
    WsLayout L = ws_layout(in->width, in->height, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.total, "hdof_postfilter_spec: workspace of %zu bytes < %zu",
                   workspace_bytes, L.total);
    // the grey plane sits below the post-filter's region (the mask and trace
    // scratch, at least 16 bytes per pixel since spp_max >= 1)
    const size_t n = (size_t)in->width * in->height;
    HDOF_CHECK_ARG(n * sizeof(float4) <= L.pf_off, "hdof_postfilter_spec: no room for the specular plane");
    float4* plane = static_cast<float4*>(workspace);
    cudaStream_t s = as_stream(stream);
    {
        ProfScope ps_("pf_spec_plane", s);
        const unsigned blocks = (unsigned)((n + 255) / 256);
        if (in->dtype_col == HDOF_F32)
            k_spec_plane<<<blocks, 256, 0, s>>>(static_cast<const float4*>(in->col), n, plane);
        else
            k_spec_plane<<<blocks, 256, 0, s>>>(static_cast<const bf164s*>(in->col), n, plane);
    }
    HDOF_LAUNCHED("specular plane");
    hdof_gbuf g = *in;
    g.dtype_col = HDOF_F32;
    g.col = plane;
    return launch_postfilter(&g, make_coc(*lens, in->height, cam->tan_half_fovy), p, pp_spec, nullptr,
                             static_cast<char*>(workspace) + L.pf_off, s);
}

namespace hdof {

size_t pf_prep_args_size() { return sizeof(PrepF32); }
void pf_prep_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TP - 1) / TP;
    *reinterpret_cast<PrepF32*>(dst) =
        PrepF32{static_cast<const float4*>(v.g.nd), static_cast<const float4*>(v.g.col), W, H,
                make_coc(v.lens, H, v.cam.tan_half_fovy), v.params.r_max, ntx, w.rh, w.zq, w.nrec, w.frec, w.tmax};
    *gx = ntx;
    *gy = (H + TP - 1) / TP;
}
void pf_prep_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_pf_prep", s);
    k_pf_prep_batch<<<blocks, 256, 0, s>>>(static_cast<const PrepF32*>(args), g);
}

size_t pf_rowscan_args_size() { return sizeof(RowScanArgs); }
void pf_rowscan_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    *reinterpret_cast<RowScanArgs*>(dst) = RowScanArgs{w.nrec, v.cam.width, v.cam.height, w.pre};
    *gx = 1;  // one block per row
    *gy = v.cam.height;
}
void pf_rowscan_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_pf_rowscan", s);
    k_pf_rowscan_batch<<<blocks, 256, 0, s>>>(static_cast<const RowScanArgs*>(args), g);
}

size_t pf_gather_args_size() { return sizeof(GatherArgs<float4>); }
void pf_gather_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TP - 1) / TP, nty = (H + TP - 1) / TP;
    *reinterpret_cast<GatherArgs<float4>*>(dst) =
        GatherArgs<float4>{w.rh, w.zq, w.nrec, w.frec, static_cast<const float4*>(v.g.col), w.tmax, w.pre, W, H, ntx,
                           nty, gather_tiles(v.params.r_max), v.params.kz_rel, reinterpret_cast<float4*>(v.pp),
                           nullptr};
    *gx = ntx;
    *gy = nty;
    cudaFuncSetAttribute(k_pf_gather_batch, cudaFuncAttributePreferredSharedMemoryCarveout, GATHER_CARVEOUT);
}
void pf_gather_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_pf_gather", s);
    k_pf_gather_batch<<<blocks, GATHER_THREADS, 0, s>>>(static_cast<const GatherArgs<float4>*>(args), g);
}

}  // namespace hdof
