// Device-side building blocks shared by the hdof kernels: small vector math,
// the thin-lens camera, the Philox4x32-10 counter-based generator, G-buffer
// storage conversions, BVH layout and the watertight ray/triangle test.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hdof.h"

#define HDOF_SQRT2 1.41421356237309505f
#define HDOF_EMPTY_W 1e-6f      // layer weight below which a layer is empty
#define HDOF_HIST_MIN_W 1e-3f   // bilinear history weight below which history is invalid
#define HDOF_PP_MIN_W 1e-8f     // post-filter layer weight below which a layer is empty
#define HDOF_MV_OFFSCREEN 1e6f  // motion written when the previous camera cannot see a point
#define HDOF_STACK 64           // traversal stack entries (> tree depth)
#ifndef HDOF_LEAF_MAX
#define HDOF_LEAF_MAX 1         // triangles per leaf of the LBVH builder (<= 8)
#endif
#ifndef HDOF_BIG_MAX
#define HDOF_BIG_MAX 0          // scene-sized triangles kept out of the tree (0: all in the tree)
#endif
#define HDOF_TILE_PF 16         // post-filter bounding tile edge
#define HDOF_STATUS_TIMEOUT 1u

namespace hdof {


// ------------------------------------------------------------------ math --
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }
__device__ __forceinline__ float luminance(float3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }
__device__ __forceinline__ float3 ld3(const float* p) { return f3(p[0], p[1], p[2]); }


// --------------------------------------------------------------- camera --
struct Cam {
    float3 pos, right, up, fwd;
    float t, aspect;
    int W, H;
    float jx, jy;
};

__host__ __device__ inline Cam make_cam(const hdof_camera& c) {
    Cam o;
    o.pos = make_float3(c.pos[0], c.pos[1], c.pos[2]);
    o.right = make_float3(c.right[0], c.right[1], c.right[2]);
    o.up = make_float3(c.up[0], c.up[1], c.up[2]);
    o.fwd = make_float3(c.fwd[0], c.fwd[1], c.fwd[2]);
    o.t = c.tan_half_fovy;
    o.aspect = (float)c.width / (float)c.height;
    o.W = c.width;
    o.H = c.height;
    o.jx = c.jitter[0];
    o.jy = c.jitter[1];
    return o;
}

// Pinhole direction through screen point (sx, sy); its fwd component is 1,
// so the point at view depth z along it is pos + z * d.
__device__ __forceinline__ float3 pinhole_dir(const Cam& c, float sx, float sy) {
    float X = (2.f * sx / c.W - 1.f) * c.aspect * c.t;
    float Y = (1.f - 2.f * sy / c.H) * c.t;
    return X * c.right + Y * c.up + c.fwd;
}

// Index-space projection (u = (i, j) is exactly pixel (i, j)'s sample point).
__device__ __forceinline__ bool project(const Cam& c, float3 P, float& ux, float& uy) {
    float3 v = P - c.pos;
    float zc = dot(v, c.fwd);
    if (!(zc > 0.f)) return false;
    float X = dot(v, c.right) / zc, Y = dot(v, c.up) / zc;
    float sx = (X / (c.aspect * c.t) + 1.f) * 0.5f * c.W;
    float sy = (1.f - Y / c.t) * 0.5f * c.H;
    ux = sx - 0.5f - c.jx;
    uy = sy - 0.5f - c.jy;
    return true;
}

// Signed CoC diameter in pixels (thin lens): c(z) = A H (zf - z) / (z zf t).
struct Coc {
    float k;   // A H / t
    float izf; // 1 / zf
    __device__ __forceinline__ float operator()(float z) const { return k * (1.f / z - izf); }
    __device__ __forceinline__ float at_infinity() const { return -k * izf; }
};
__host__ __device__ inline Coc make_coc(const hdof_lens& l, int H, float t) {
    Coc c;
    c.k = l.aperture_radius * (float)H / t;
    c.izf = 1.f / l.focus_dist;
    return c;
}
// The same constants for a lens read on the device, lens = (focus distance,
// aperture radius), by make_coc's arithmetic; lens NULL: c as given.
__device__ __forceinline__ Coc lens_coc(const Coc& c, const float* lens, int H, float t) {
    if (!lens) return c;
    Coc o;
    o.k = __ldg(&lens[1]) * (float)H / t;
    o.izf = 1.f / __ldg(&lens[0]);
    return o;
}

// Near-layer split weight, linear across the focus zone |c| < sqrt2.
__device__ __forceinline__ float w_near(float c) {
    return clamp01((c + HDOF_SQRT2) * (0.5f / HDOF_SQRT2));
}

// ---------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products on a four-word counter, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
// uniform in [0, 1) with 24 bits: exact in float
__device__ __forceinline__ float u01(unsigned x) { return (float)(x >> 8) * (1.f / 16777216.f); }

// ------------------------------------------------------- G-buffer storage --
struct alignas(8) half4s { __half2 a, b; };
struct alignas(8) bf164s { __nv_bfloat162 a, b; };

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ float4 ld4(const half4s* p) {
    uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    half4s h = *reinterpret_cast<half4s*>(&r);
    float2 a = __half22float2(h.a), b = __half22float2(h.b);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ld4(const bf164s* p) {
    uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    bf164s h = *reinterpret_cast<bf164s*>(&r);
    float2 a = __bfloat1622float2(h.a), b = __bfloat1622float2(h.b);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st4(half4s* p, float4 v) {
    half4s h;
    h.a = __floats2half2_rn(v.x, v.y);
    h.b = __floats2half2_rn(v.z, v.w);
    *p = h;
}
__device__ __forceinline__ void st4(bf164s* p, float4 v) {
    bf164s h;
    h.a = __floats2bfloat162_rn(v.x, v.y);
    h.b = __floats2bfloat162_rn(v.z, v.w);
    *p = h;
}
// depth channel only
__device__ __forceinline__ float ldz(const float4* p) { return __ldg(&p->w); }
__device__ __forceinline__ float ldz(const half4s* p) { return __high2float(__ldg(&p->b)); }

// ------------------------------------------------------------------- BVH --
// Binary BVH node: the boxes of both children in one 64-byte record, so one
// fetch tests both.  Child reference >= 0: internal node; < 0: a leaf of
// 1..8 consecutive sorted triangles, ~(first << 3 | (count - 1)).  Node
// arrays start at an allocation's base, so every record is 64-byte aligned
// (the traversal fetches it with two 256-bit loads).
struct __align__(64) Node {
    float4 xy0;  // c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y
    float4 xy1;  // c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y
    float4 z01;  // c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z
    int4 child;  // c0, c1, parent, unused
};
__host__ __device__ inline int leaf_ref(int first, int count) { return ~((first << 3) | (count - 1)); }

// triangle in leaf order: (v0, original id), (v1, 0), (v2, 0)
struct __align__(16) Tri {
    float4 v0, v1, v2;
};

struct BvhView {
    const Node* nodes;
    const Tri* tris;
    const float4* mat;  // sorted order: [2] per triangle (albedo_a rgb + checker_n, albedo_b rgb + k_s)
    const float2* uv;   // sorted order: [3] per triangle
    int n_tris;
    int root;           // root reference (node 0, or a leaf)
    int big_first;      // sorted slots [big_first, big_first + big_count) hold scene-sized
    int big_count;      //   triangles tested by every ray after the traversal
    const float4* big_box;  // [2] per scene-sized triangle: (lo xyz, 0), (hi xyz, 0)
    const int* slot_of;     // sorted slot of each original triangle id
    int specular;           // some material has k_s > 0 (else every material is Lambertian)
};

// Two floats in one 64-bit register pair, the operand form of the f32x2
// instructions (each lane rounds as the scalar instruction).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
// (a.x b.x + c.x, a.y b.y + c.y), each rounded once
__device__ __forceinline__ float2 fma_x2(f32x2 a, f32x2 b, f32x2 c) {
    float2 r;
    asm("{\n\t.reg .b64 t;\n\tfma.rn.f32x2 t, %2, %3, %4;\n\tmov.b64 {%0, %1}, t;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "l"(a), "l"(b), "l"(c));
    return r;
}

// A ray with its box-test constants in f32x2 form: per axis (1/d, 1/d) and
// (-cl, -ch), cl and ch being o/d shifted so that the distances to a box's
// l- and h-plane err outwards; one fma.rn.f32x2 of a box's (l, h) pair on an
// axis gives both plane distances.
struct Ray {
    float3 o, d;
    f32x2 id2[3];
    f32x2 off2[3];
};

// Plane distances are fma(l, id, -o id): (l - o) id (1 + d1) - (o id) d2 with
// |d1|, |d2| of a few units of 2^-24.  The relative part is covered by
// widening the exit distance relatively; the absolute part, below
// 2^-23 |o id| on that axis, by shifting each axis's offset by
// e = 2^-22 |o id| so that its entry plane reads early and its exit plane
// late (which plane is which follows the sign of d).  A ray nearly parallel
// to an axis has huge distances on it and a large e there: they stay huge,
// so the shift costs no culling.
__device__ __forceinline__ Ray make_ray(float3 o, float3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    const float tiny = 1e-20f;
    const float3 id = f3(1.f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                         1.f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                         1.f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    const float3 ood = f3(o.x * id.x, o.y * id.y, o.z * id.z);
    const float3 e = f3(ldexpf(fabsf(ood.x), -22), ldexpf(fabsf(ood.y), -22), ldexpf(fabsf(ood.z), -22));
    // id > 0: l is the entry plane (distance lowered: offset raised), h the exit
    const float3 cl = f3(id.x > 0.f ? ood.x + e.x : ood.x - e.x, id.y > 0.f ? ood.y + e.y : ood.y - e.y,
                         id.z > 0.f ? ood.z + e.z : ood.z - e.z);
    const float3 ch = f3(id.x > 0.f ? ood.x - e.x : ood.x + e.x, id.y > 0.f ? ood.y - e.y : ood.y + e.y,
                         id.z > 0.f ? ood.z - e.z : ood.z + e.z);
    r.id2[0] = pk2(id.x, id.x);
    r.id2[1] = pk2(id.y, id.y);
    r.id2[2] = pk2(id.z, id.z);
    r.off2[0] = pk2(-cl.x, -ch.x);
    r.off2[1] = pk2(-cl.y, -ch.y);
    r.off2[2] = pk2(-cl.z, -ch.z);
    return r;
}

// hardware approximate square root (relative error ~2^-22): for tap
// distances that only enter soft weights clamp(r + 1/2 - d, 0, 1)
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Slab test of one box; returns entry distance (or +inf on a miss).  With
// the outward plane offsets of make_ray and the exit distance widened by
// 2^-19 (relative rounding of the planes and of a triangle's hit distance,
// which tmax may be), a box that holds a point of the ray at a distance
// <= tmax is not culled: the closest hit, the minimum of (t, id) over the
// triangles the ray hits, does not depend on the order boxes are visited.
// Direction octant: bit k set when component k is negative (its sign bit,
// which is the sign of 1/d as make_ray forms it, -0 included).
__device__ __forceinline__ int ray_octant(const Ray& r) {
    return (int)(__float_as_uint(r.d.x) >> 31) | (int)(__float_as_uint(r.d.y) >> 31) << 1 |
           (int)(__float_as_uint(r.d.z) >> 31) << 2;
}

// The box is given by its (l, h) pair on each axis.
__device__ __forceinline__ bool slab_hit(const Ray& r, f32x2 x, f32x2 y, f32x2 z, float tmax, float& tn) {
    const float2 tx = fma_x2(x, r.id2[0], r.off2[0]);
    const float2 ty = fma_x2(y, r.id2[1], r.off2[1]);
    const float2 tz = fma_x2(z, r.id2[2], r.off2[2]);
    tn = fmaxf(fmaxf(fminf(tx.x, tx.y), fminf(ty.x, ty.y)), fmaxf(fminf(tz.x, tz.y), 0.f));
    const float tf = fminf(fminf(fmaxf(tx.x, tx.y), fmaxf(ty.x, ty.y)), fminf(fmaxf(tz.x, tz.y), tmax));
    return tn <= tf * 1.0000019f;
}
// the same test of a box given by its corners, returning the entry distance
// (or +inf on a miss)
__device__ __forceinline__ float slab(const Ray& r, float lx, float hx, float ly, float hy, float lz,
                                      float hz, float tmax) {
    float tn;
    return slab_hit(r, pk2(lx, hx), pk2(ly, hy), pk2(lz, hz), tmax, tn) ? tn : __int_as_float(0x7f800000);
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013).  Edge
// functions are evaluated without contraction so a shared edge gives exactly
// negated values in its two triangles; exact zeros are re-evaluated in double.
// Returns true for a hit with 0 < t; writes t and barycentrics (b0 at v0).
struct Shear {
    int kx, ky, kz;
    float Sx, Sy, Sz;
};
__device__ __forceinline__ Shear make_shear(float3 d) {
    Shear s;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    s.kz = 0;
    if (ay > ax && ay >= az) s.kz = 1;
    else if (az > ax && az > ay) s.kz = 2;
    s.kx = s.kz == 2 ? 0 : s.kz + 1;
    s.ky = s.kx == 2 ? 0 : s.kx + 1;
    float dk[3] = {d.x, d.y, d.z};
    if (dk[s.kz] < 0.f) {
        int t = s.kx;
        s.kx = s.ky;
        s.ky = t;
    }
    s.Sx = dk[s.kx] / dk[s.kz];
    s.Sy = dk[s.ky] / dk[s.kz];
    s.Sz = 1.f / dk[s.kz];
    return s;
}
__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ bool intersect_tri(float3 o, const Shear& s, float3 v0, float3 v1, float3 v2,
                                              float& t, float& b0, float& b1, float& b2) {
    float3 A = v0 - o, B = v1 - o, C = v2 - o;
    float Akz = comp(A, s.kz), Bkz = comp(B, s.kz), Ckz = comp(C, s.kz);
    float Ax = __fsub_rn(comp(A, s.kx), __fmul_rn(s.Sx, Akz));
    float Ay = __fsub_rn(comp(A, s.ky), __fmul_rn(s.Sy, Akz));
    float Bx = __fsub_rn(comp(B, s.kx), __fmul_rn(s.Sx, Bkz));
    float By = __fsub_rn(comp(B, s.ky), __fmul_rn(s.Sy, Bkz));
    float Cx = __fsub_rn(comp(C, s.kx), __fmul_rn(s.Sx, Ckz));
    float Cy = __fsub_rn(comp(C, s.ky), __fmul_rn(s.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.f || V == 0.f || W == 0.f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return false;
    const float T = __fadd_rn(__fadd_rn(__fmul_rn(U, __fmul_rn(s.Sz, Akz)), __fmul_rn(V, __fmul_rn(s.Sz, Bkz))),
                              __fmul_rn(W, __fmul_rn(s.Sz, Ckz)));
    if (det > 0.f ? !(T > 0.f) : !(T < 0.f)) return false;
    const float inv = __frcp_rn(det);
    t = __fmul_rn(T, inv);
    b0 = __fmul_rn(U, inv);
    b1 = __fmul_rn(V, inv);
    b2 = __fmul_rn(W, inv);
    return true;
}

// Barycentrics of a known hit, recomputed with the arithmetic of
// intersect_tri (same inputs give the same values) but without its rejection
// tests, so a hit found by the traversal is always reproduced.
__device__ __forceinline__ void tri_bary(float3 o, const Shear& s, float3 v0, float3 v1, float3 v2, float& b0,
                                         float& b1, float& b2) {
    float3 A = v0 - o, B = v1 - o, C = v2 - o;
    float Akz = comp(A, s.kz), Bkz = comp(B, s.kz), Ckz = comp(C, s.kz);
    float Ax = __fsub_rn(comp(A, s.kx), __fmul_rn(s.Sx, Akz));
    float Ay = __fsub_rn(comp(A, s.ky), __fmul_rn(s.Sy, Akz));
    float Bx = __fsub_rn(comp(B, s.kx), __fmul_rn(s.Sx, Bkz));
    float By = __fsub_rn(comp(B, s.ky), __fmul_rn(s.Sy, Bkz));
    float Cx = __fsub_rn(comp(C, s.kx), __fmul_rn(s.Sx, Ckz));
    float Cy = __fsub_rn(comp(C, s.ky), __fmul_rn(s.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.f || V == 0.f || W == 0.f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    const float inv = det != 0.f ? __frcp_rn(det) : 0.f;
    b0 = __fmul_rn(U, inv);
    b1 = __fmul_rn(V, inv);
    b2 = __fmul_rn(W, inv);
}

struct Hit {
    float t, b0, b1, b2;
    int slot;  // sorted triangle slot, -1 = miss
    int id;    // original triangle id
};

__device__ __forceinline__ void hit_tri(const BvhView& bvh, int slot, float3 o, const Shear& sh, Hit& h) {
    const Tri* tr = bvh.tris + slot;
    float4 p0 = __ldg(&tr->v0), p1 = __ldg(&tr->v1), p2 = __ldg(&tr->v2);
    float t, b0, b1, b2;
    if (intersect_tri(o, sh, f3(p0.x, p0.y, p0.z), f3(p1.x, p1.y, p1.z), f3(p2.x, p2.y, p2.z), t, b0, b1, b2)) {
        int id = __float_as_int(p0.w);
        if (t < h.t || (t == h.t && id < h.id)) {
            h.t = t;
            h.b0 = b0;
            h.b1 = b1;
            h.b2 = b2;
            h.slot = slot;
            h.id = id;
        }
    }
}

#ifndef HDOF_TRAV_STATS
#define HDOF_TRAV_STATS 0  // count node visits and triangle tests (analysis builds only)
#endif
#if HDOF_TRAV_STATS
// the counters (rays, node visits, triangle tests) sit in the status block
// after the status word, whose address every traversal already has
__device__ __forceinline__ void trav_stat(unsigned* status, int k, unsigned long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(status + 2) + k, v);
}
#endif

// three-input minimum and maximum (one instruction each on sm_100 and later;
// exact, like the nested two-input forms)
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Box test for rays of a known octant (OCT bit k set: direction component k
// negative), so the entry and exit plane of each axis are known and need no
// per-axis min/max; OCT < 0: any direction (slab_hit).  With the outward
// offsets of make_ray an axis's entry distance never exceeds its exit
// distance (rounding is monotone), so the decisions and tn equal slab_hit's.
template <int OCT>
__device__ __forceinline__ bool slab_hit_oct(const Ray& r, f32x2 x, f32x2 y, f32x2 z, float tmax, float& tn) {
    if (OCT < 0) return slab_hit(r, x, y, z, tmax, tn);
    const bool nx = OCT & 1, ny = OCT & 2, nz = OCT & 4;
    const float2 tx = fma_x2(x, r.id2[0], r.off2[0]);  // (l-plane, h-plane) distances
    const float2 ty = fma_x2(y, r.id2[1], r.off2[1]);
    const float2 tz = fma_x2(z, r.id2[2], r.off2[2]);
    tn = max3f(nx ? tx.y : tx.x, ny ? ty.y : ty.x, fmaxf(nz ? tz.y : tz.x, 0.f));
    const float tf = min3f(nx ? tx.x : tx.y, ny ? ty.x : ty.y, fminf(nz ? tz.x : tz.y, tmax));
    return tn <= tf * 1.0000019f;
}

// A node's two child boxes as (l, h) pairs per axis.
struct NodeBoxes {
    f32x2 x0, y0, z0, x1, y1, z1;
    int4 ch;
};
// two 256-bit loads (the node is 64 bytes, 64-byte aligned): the boxes'
// (l, h) pairs arrive as the 64-bit words the f32x2 box test takes
__device__ __forceinline__ NodeBoxes load_node(const Node* n) {
    unsigned long long a0, a1, a2, a3, b0, b1, b2, b3;
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a0), "=l"(a1), "=l"(a2), "=l"(a3) : "l"(n));
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4+32];" : "=l"(b0), "=l"(b1), "=l"(b2), "=l"(b3) : "l"(n));
    NodeBoxes nb;
    nb.x0 = a0;  // xy0 = (c0.lo.x, c0.hi.x), (c0.lo.y, c0.hi.y)
    nb.y0 = a1;
    nb.x1 = a2;  // xy1
    nb.y1 = a3;
    nb.z0 = b0;  // z01 = (c0.lo.z, c0.hi.z), (c1.lo.z, c1.hi.z)
    nb.z1 = b1;
    nb.ch = make_int4((int)(unsigned)b2, (int)(unsigned)(b2 >> 32), (int)(unsigned)b3, (int)(unsigned)(b3 >> 32));
    return nb;
}

// Closest hit: smallest t, equal t -> lower original id.  Stack traversal
// (descend the nearer hit child, push the farther); scene-sized triangles
// (when kept out of the tree) are tested last behind a slab test of their
// box.  cap bounds the node and leaf steps (watchdog).
// hint_slot >= 0: that triangle is tested first (a likely hit tightens the
// traversal; the closest hit, the minimum of (t, id) over all hits, is
// unchanged).
template <int OCT>
__device__ __forceinline__ Hit closest_hit_oct(const BvhView& bvh, float3 o, float3 d, int cap, unsigned* status,
                                               int hint_slot) {
    const float INF = __int_as_float(0x7f800000);
    Ray r = make_ray(o, d);
    Shear sh = make_shear(d);
    Hit h;
    h.t = INF;
    h.slot = -1;
    h.id = 0x7fffffff;
    h.b0 = h.b1 = h.b2 = 0.f;
    if (hint_slot >= 0) hit_tri(bvh, hint_slot, o, sh, h);
    int stack[HDOF_STACK];
    int sp = 0;
    int cur = bvh.root;
    int steps = 0;
#if HDOF_TRAV_STATS
    unsigned nv = 0, nt = 0;
#endif
    while (true) {
        if (cur >= 0) {
#if HDOF_TRAV_STATS
            ++nv;
#endif
            const NodeBoxes nb = load_node(bvh.nodes + cur);
            const int4 ch = nb.ch;
            float t0, t1;
            const bool h0 = slab_hit_oct<OCT>(r, nb.x0, nb.y0, nb.z0, h.t, t0);
            const bool h1 = slab_hit_oct<OCT>(r, nb.x1, nb.y1, nb.z1, h.t, t1);
            if (h0 && h1) {
                int nearc = t0 <= t1 ? ch.x : ch.y, farc = t0 <= t1 ? ch.y : ch.x;
                if (sp < HDOF_STACK) stack[sp++] = farc;
                else atomicOr(status, HDOF_STATUS_TIMEOUT);
                cur = nearc;
            } else if (h0) {
                cur = ch.x;
            } else if (h1) {
                cur = ch.y;
            } else {
                if (sp == 0) break;
                cur = stack[--sp];
            }
        } else {
            int e = ~cur, first = e >> 3, count = (e & 7) + 1;
            for (int k = 0; k < count; ++k) hit_tri(bvh, first + k, o, sh, h);
#if HDOF_TRAV_STATS
            nt += count;
#endif
            if (sp == 0) break;
            cur = stack[--sp];
        }
        if (++steps > cap) {
            atomicOr(status, HDOF_STATUS_TIMEOUT);
            break;
        }
    }
    for (int k = 0; k < bvh.big_count; ++k) {
        float4 lo = __ldg(&bvh.big_box[2 * k]), hi = __ldg(&bvh.big_box[2 * k + 1]);
        if (slab(r, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, h.t) < INF) hit_tri(bvh, bvh.big_first + k, o, sh, h);
    }
#if HDOF_TRAV_STATS
    trav_stat(status, 0, 1ull);
    trav_stat(status, 1, nv);
    trav_stat(status, 2, nt);
#endif
    if (h.slot < 0) h.id = -1;
    return h;
}


// Closest hit of each calling lane's own ray; when the lanes that call
// together share a direction octant (primary rays of a pixel block) the
// traversal specialised to it runs (same results, fewer box-test steps).
__device__ __forceinline__ Hit closest_hit(const BvhView& bvh, float3 o, float3 d, int cap, unsigned* status,
                                           int hint_slot = -1) {
    const unsigned m = __activemask();
    // the signs of 1/d as make_ray forms it (a -0 component gives -1e20)
    const int oct = (signbit(d.x) ? 1 : 0) | (signbit(d.y) ? 2 : 0) | (signbit(d.z) ? 4 : 0);
    const int o0 = __shfl_sync(m, oct, __ffs(m) - 1);
    const int u = __all_sync(m, oct == o0) ? o0 : -1;
    switch (u) {
        case 0: return closest_hit_oct<0>(bvh, o, d, cap, status, hint_slot);
        case 1: return closest_hit_oct<1>(bvh, o, d, cap, status, hint_slot);
        case 2: return closest_hit_oct<2>(bvh, o, d, cap, status, hint_slot);
        case 3: return closest_hit_oct<3>(bvh, o, d, cap, status, hint_slot);
        case 4: return closest_hit_oct<4>(bvh, o, d, cap, status, hint_slot);
        case 5: return closest_hit_oct<5>(bvh, o, d, cap, status, hint_slot);
        case 6: return closest_hit_oct<6>(bvh, o, d, cap, status, hint_slot);
        case 7: return closest_hit_oct<7>(bvh, o, d, cap, status, hint_slot);
        default: return closest_hit_oct<-1>(bvh, o, d, cap, status, hint_slot);
    }
}

// Warp-wide closest hits: all 32 lanes call this together; the active lanes'
// rays share one traversal (node references and the stack are warp-uniform;
// the stack lives in registers, entry k in lane k mod 32, pushed by one lane's
// move and popped by a shuffle, with no shared memory or warp barrier).  A node is
// entered when any active lane's ray enters one of its children before that
// lane's own closest hit so far; each lane tests the triangles of every leaf
// the warp reaches.  A lane's own closest hit lies in a leaf whose every
// ancestor box that lane enters, so the warp reaches it: every lane gets the
// same (t, id) minimum as closest_hit.  Coherent rays (the lens samples of
// neighbouring pixels, the primary rays of a pixel block) visit nearly the
// same nodes, so one broadcast node fetch and one box test per lane serve
// the warp without divergence.  h holds each lane's hit so far (a hint hit
// or a miss); scene-sized triangles are left to the caller.  Returns false
// when the step cap was reached (the warp stops; status is flagged).
template <int OCT>
__device__ __forceinline__ bool closest_hit_warp_oct(const BvhView& bvh, bool act, const Ray& r, float3 o,
                                                     const Shear& sh, Hit& h, int cap, unsigned* status) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int cur = bvh.root, sp = 0, steps = 0;
    // the warp's stack in registers: entry k in lane k & 31 of slo (k < 32) or shi
    static_assert(HDOF_STACK <= 64, "the register stack holds 64 entries");
    int slo = 0, shi = 0;
#if HDOF_TRAV_STATS
    unsigned nv = 0, nt = 0;
#endif
    while (true) {
        bool pop = true;
        if (cur >= 0) {
#if HDOF_TRAV_STATS
            ++nv;
#endif
            const NodeBoxes nb = load_node(bvh.nodes + cur);
            const int4 ch = nb.ch;
            float t0, t1;
            // branch-free: an idle lane tests its placeholder ray and is masked out
            const bool h0 = slab_hit_oct<OCT>(r, nb.x0, nb.y0, nb.z0, h.t, t0) & act;
            const bool h1 = slab_hit_oct<OCT>(r, nb.x1, nb.y1, nb.z1, h.t, t1) & act;
            const unsigned b0 = __ballot_sync(FULL, h0), b1 = __ballot_sync(FULL, h1);
            if (b0 && b1) {
                // first the child nearer for most of the lanes that enter both
                // (or entered by more lanes): only the culling depends on it
                const unsigned both = b0 & b1, nx = __ballot_sync(FULL, h0 && h1 && t0 <= t1);
                const bool x_first = both ? 2 * __popc(nx) >= __popc(both) : __popc(b0) >= __popc(b1);
                const int far = x_first ? ch.y : ch.x;
                if (sp < 32) {
                    if (lane == sp) slo = far;
                    ++sp;
                } else if (sp < HDOF_STACK) {
                    if (lane == sp - 32) shi = far;
                    ++sp;
                } else if (lane == 0) {
                    atomicOr(status, HDOF_STATUS_TIMEOUT);
                }
                cur = x_first ? ch.x : ch.y;
                pop = false;
            } else if (b0 | b1) {
                cur = b0 ? ch.x : ch.y;
                pop = false;
            }
        } else {
            const int e = ~cur, first = e >> 3, count = (e & 7) + 1;
            if (act)
                for (int k = 0; k < count; ++k) hit_tri(bvh, first + k, o, sh, h);
#if HDOF_TRAV_STATS
            nt += count;
#endif
        }
        if (pop) {
            // the cap counts pops: between two, a descent is at most the tree's depth
            if (++steps > cap) {
                if (lane == 0) atomicOr(status, HDOF_STATUS_TIMEOUT);
                return false;
            }
            if (sp == 0) break;
            --sp;
            cur = __shfl_sync(FULL, sp < 32 ? slo : shi, sp & 31);
        }
    }
#if HDOF_TRAV_STATS
    if (lane == 0) {
        trav_stat(status, 1, nv);
        trav_stat(status, 2, nt);
    }
    if (act) trav_stat(status, 0, 1ull);
#endif
    return true;
}

// the traversal specialised to the packet's octant when all its active rays
// share one (the usual case for coherent rays), the general one otherwise
__device__ __forceinline__ bool closest_hit_warp(const BvhView& bvh, bool act, const Ray& r, float3 o,
                                                 const Shear& sh, Hit& h, int cap, unsigned* status) {
    const unsigned FULL = 0xffffffffu;
    const int oct = ray_octant(r);
    const unsigned am = __ballot_sync(FULL, act);
    const int o0 = __shfl_sync(FULL, oct, am ? __ffs(am) - 1 : 0);
    const int u = __all_sync(FULL, !act || oct == o0) ? o0 : -1;
    switch (u) {
        case 0: return closest_hit_warp_oct<0>(bvh, act, r, o, sh, h, cap, status);
        case 1: return closest_hit_warp_oct<1>(bvh, act, r, o, sh, h, cap, status);
        case 2: return closest_hit_warp_oct<2>(bvh, act, r, o, sh, h, cap, status);
        case 3: return closest_hit_warp_oct<3>(bvh, act, r, o, sh, h, cap, status);
        case 4: return closest_hit_warp_oct<4>(bvh, act, r, o, sh, h, cap, status);
        case 5: return closest_hit_warp_oct<5>(bvh, act, r, o, sh, h, cap, status);
        case 6: return closest_hit_warp_oct<6>(bvh, act, r, o, sh, h, cap, status);
        case 7: return closest_hit_warp_oct<7>(bvh, act, r, o, sh, h, cap, status);
        default: return closest_hit_warp_oct<-1>(bvh, act, r, o, sh, h, cap, status);
    }
}

// Lambert shading at a hit: face normal turned towards the ray, albedo from
// the material (checkerboard over the triangle's (u, v) when checker_n > 0).
struct Lights {
    int n;
    float3 dir[4];
    float E[4];
    float ka;
};
__host__ __device__ inline Lights make_lights(const hdof_params& p) {
    Lights l;
    l.n = p.n_lights;
    for (int k = 0; k < 4; ++k) {
        l.dir[k] = make_float3(p.light_dir[k][0], p.light_dir[k][1], p.light_dir[k][2]);
        l.E[k] = p.light_E[k];
    }
    l.ka = p.k_ambient;
    return l;
}

// Shading of a hit seen along the unit direction d: Lambert diffuse under
// directional lights, plus a white Blinn-Phong highlight (exponent 32) for
// materials with k_s > 0, whose luminance is returned in spec.
__device__ __forceinline__ void shade(const BvhView& bvh, const Lights& L, const Hit& h, float3 d, float3& n,
                                      float3& rad, float& spec) {
    const Tri* tr = bvh.tris + h.slot;
    float4 p0 = __ldg(&tr->v0), p1 = __ldg(&tr->v1), p2 = __ldg(&tr->v2);
    float3 v0 = f3(p0.x, p0.y, p0.z);
    n = normalize(cross(f3(p1.x, p1.y, p1.z) - v0, f3(p2.x, p2.y, p2.z) - v0));
    if (dot(n, d) > 0.f) n = -1.f * n;
    float4 ma = __ldg(&bvh.mat[2 * h.slot]);
    float3 alb = f3(ma.x, ma.y, ma.z);
    if (ma.w > 0.f) {
        float2 u0 = __ldg(&bvh.uv[3 * h.slot]), u1 = __ldg(&bvh.uv[3 * h.slot + 1]),
               u2 = __ldg(&bvh.uv[3 * h.slot + 2]);
        float uu = h.b0 * u0.x + h.b1 * u1.x + h.b2 * u2.x;
        float vv = h.b0 * u0.y + h.b1 * u1.y + h.b2 * u2.y;
        int cell = (int)floorf(ma.w * uu) + (int)floorf(ma.w * vv);
        if (cell & 1) {
            float4 mb = __ldg(&bvh.mat[2 * h.slot + 1]);
            alb = f3(mb.x, mb.y, mb.z);
        }
    }
    float irr = L.ka;
    for (int k = 0; k < L.n; ++k) irr += L.E[k] * fmaxf(0.f, dot(n, L.dir[k]));
    rad = irr * alb;
    spec = 0.f;
    if (bvh.specular) {
        const float ks = __ldg(&bvh.mat[2 * h.slot + 1].w);
        if (ks > 0.f) {
            float s = 0.f;
            for (int k = 0; k < L.n; ++k) {
                if (dot(n, L.dir[k]) <= 0.f) continue;
                float c = fmaxf(0.f, dot(n, normalize(L.dir[k] - d)));  // half vector of light and viewer
                c *= c;
                c *= c;
                c *= c;
                c *= c;
                c *= c;
                s += L.E[k] * c;
            }
            spec = ks * s;
            rad = rad + f3(spec, spec, spec);
        }
    }
}

}  // namespace hdof
