// Acceleration structure standing in for the paper's hardware ray-tracing
// acceleration (Abstract), plus the closest-hit query used to check it.
//
// Common steps: scene and centroid bounds -> 63-bit Morton codes -> radix
// sort of (code, triangle) pairs -> triangles, materials and UVs stored in
// sorted order.  The hierarchy over the sorted triangles is then built by
// PLOC (parallel locally-ordered clustering, Meister and Bittner 2018; the
// default, HDOF_BUILDER=1) or by the linear BVH of Karras ("Maximizing
// parallelism in the construction of BVHs, octrees and k-d trees", HPG 2012;
// HDOF_BUILDER=0): one thread per internal node finds its key range and
// split, one thread per leaf refits child boxes bottom-up.  On the 1080p room
// the clustered tree needs 64 node visits per thin-lens ray against 100 for
// the linear one (2.5 ms against 3.3 ms for the frame's 3.4M rays).
#include <cub/cub.cuh>

#include <cstring>

#include "internal.h"

namespace hdof {
namespace {

__device__ __forceinline__ unsigned f2ord(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bounds[0..5]: ordered-float vertex bounds of the scene (lo xyz, hi xyz);
// [6]: bad-index flag; [7]: number of scene-sized triangles;
// [8..13]: centroid bounds of the other triangles; [14..19]: centroid bounds of all
constexpr int NB = 20;

__global__ void k_scene_bounds(const float* __restrict__ v, int nv, const int* __restrict__ idx, int n,
                               unsigned* bounds) {
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    bool bad = false;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int a = idx[3 * t], b = idx[3 * t + 1], c = idx[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
            bad = true;
            continue;
        }
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], fminf(v[3 * a + k], fminf(v[3 * b + k], v[3 * c + k])));
            hi[k] = fmaxf(hi[k], fmaxf(v[3 * a + k], fmaxf(v[3 * b + k], v[3 * c + k])));
        }
    }
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], f2ord(lo[k]));
            atomicMax(&bounds[3 + k], f2ord(hi[k]));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&bounds[6], 1u);
}

__device__ __forceinline__ float box_area(const float lo[3], const float hi[3]) {
    float x = hi[0] - lo[0], y = hi[1] - lo[1], z = hi[2] - lo[2];
    return 2.f * (x * y + y * z + z * x);
}

// A triangle whose box covers more than big_frac of the scene box's surface
// area is "scene-sized" (room walls): kept out of the tree, where its box
// would widen every ancestor, and tested by every ray instead.
__global__ void k_classify(const float* __restrict__ v, const int* __restrict__ idx, int n, float big_frac,
                           unsigned* bounds, uint8_t* big) {
    float slo[3], shi[3];
    for (int k = 0; k < 3; ++k) {
        slo[k] = ord2f(bounds[k]);
        shi[k] = ord2f(bounds[3 + k]);
    }
    const float thr = big_frac * box_area(slo, shi);
    float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    float alo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, ahi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
    unsigned nbig = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int a = idx[3 * t], b = idx[3 * t + 1], c = idx[3 * t + 2];
        float tlo[3], thi[3], cen[3];
        for (int k = 0; k < 3; ++k) {
            float x = v[3 * a + k], y = v[3 * b + k], z = v[3 * c + k];
            tlo[k] = fminf(x, fminf(y, z));
            thi[k] = fmaxf(x, fmaxf(y, z));
            cen[k] = (x + y + z) * (1.f / 3.f);
        }
        bool is_big = box_area(tlo, thi) > thr;
        big[t] = is_big ? 1 : 0;
        nbig += is_big ? 1u : 0u;
        for (int k = 0; k < 3; ++k) {
            alo[k] = fminf(alo[k], cen[k]);
            ahi[k] = fmaxf(ahi[k], cen[k]);
            if (!is_big) {
                lo[k] = fminf(lo[k], cen[k]);
                hi[k] = fmaxf(hi[k], cen[k]);
            }
        }
    }
    for (int k = 0; k < 3; ++k)
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            alo[k] = fminf(alo[k], __shfl_xor_sync(0xffffffffu, alo[k], o));
            ahi[k] = fmaxf(ahi[k], __shfl_xor_sync(0xffffffffu, ahi[k], o));
        }
    for (int o = 16; o; o >>= 1) nbig += __shfl_xor_sync(0xffffffffu, nbig, o);
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[8 + k], f2ord(lo[k]));
            atomicMax(&bounds[11 + k], f2ord(hi[k]));
            atomicMin(&bounds[14 + k], f2ord(alo[k]));
            atomicMax(&bounds[17 + k], f2ord(ahi[k]));
        }
        atomicAdd(&bounds[7], nbig);
    }
}

// spread the low 21 bits of v to every third bit
__device__ __forceinline__ unsigned long long expand21(unsigned v) {
    unsigned long long x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// 63-bit Morton code (21 bits per axis) of the centroid in the given centroid
// bounds: cells of ~1e-6 of the scene extent, so triangles of small objects
// in a large room still get distinct codes.  Scene-sized triangles (when
// separated) get the largest key and sort to the end.
__global__ void k_morton(const float* __restrict__ v, const int* __restrict__ idx, int n,
                         const unsigned* __restrict__ bounds, const uint8_t* __restrict__ big,
                         unsigned long long* keys, int* ids) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    ids[t] = t;
    if (big && big[t]) {
        keys[t] = ~0ull;
        return;
    }
    int a = idx[3 * t], b = idx[3 * t + 1], c = idx[3 * t + 2];
    unsigned q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bounds[k]), hi = ord2f(bounds[3 + k]);
        float cen = (v[3 * a + k] + v[3 * b + k] + v[3 * c + k]) * (1.f / 3.f);
        float ext = hi - lo;
        float u = ext > 0.f ? (cen - lo) / ext : 0.5f;
        q[k] = (unsigned)fminf(fmaxf(u * 2097152.f, 0.f), 2097151.f);
    }
    keys[t] = (expand21(q[0]) << 2) | (expand21(q[1]) << 1) | expand21(q[2]);
}

// common-prefix length of sorted keys i and j (extended key = code, position)
__device__ __forceinline__ int delta(const unsigned long long* __restrict__ keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long a = keys[i], b = keys[j];
    if (a != b) return __clzll(a ^ b);
    return 64 + __clz((unsigned)i ^ (unsigned)j);
}

__global__ void k_hierarchy(const unsigned long long* __restrict__ keys, int n, Node* nodes, int* leaf_parent, int2* rng) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + (d < 0 ? -1 : 0);
    int lo = i < j ? i : j, hi = i < j ? j : i;
    rng[i] = make_int2(lo, hi);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    // separate 4-byte stores: .z (this node's parent) is written by the parent's thread
    nodes[i].child.x = left;
    nodes[i].child.y = right;
    if (left >= 0) nodes[left].child.z = i;
    else leaf_parent[gamma] = i;
    if (right >= 0) nodes[right].child.z = i;
    else leaf_parent[gamma + 1] = i;
}

__device__ __forceinline__ void tri_box(const float* __restrict__ v, const int* __restrict__ idx, int id,
                                        float lo[3], float hi[3]) {
    int a = idx[3 * id], b = idx[3 * id + 1], c = idx[3 * id + 2];
    for (int k = 0; k < 3; ++k) {
        float x = v[3 * a + k], y = v[3 * b + k], z = v[3 * c + k];
        lo[k] = fminf(x, fminf(y, z));
        hi[k] = fmaxf(x, fmaxf(y, z));
    }
}

__device__ __forceinline__ void write_child_box(Node* nd, int which, const float lo[3], const float hi[3]) {
    if (which == 0) {
        nd->xy0 = make_float4(lo[0], hi[0], lo[1], hi[1]);
        nd->z01.x = lo[2];
        nd->z01.y = hi[2];
    } else {
        nd->xy1 = make_float4(lo[0], hi[0], lo[1], hi[1]);
        nd->z01.z = lo[2];
        nd->z01.w = hi[2];
    }
}

__global__ void k_refit(const float* __restrict__ v, const int* __restrict__ idx, const int* __restrict__ ids,
                        int n, const int* __restrict__ leaf_parent, Node* nodes, unsigned* flags) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float lo[3], hi[3];
    tri_box(v, idx, ids[k], lo, hi);
    int me = ~k;
    int p = leaf_parent[k];
    for (int level = 0; p >= 0 && level < 4096; ++level) {  // bounded walk to the root
        Node* nd = nodes + p;
        int4 ch = __ldcg(&nd->child);
        write_child_box(nd, ch.x == me ? 0 : 1, lo, hi);
        __threadfence();
        if (atomicAdd(&flags[p], 1u) == 0) return;  // the sibling finishes this node
        __threadfence();
        float4 a = __ldcg(&nd->xy0), b = __ldcg(&nd->xy1), z = __ldcg(&nd->z01);
        lo[0] = fminf(a.x, b.x);
        hi[0] = fmaxf(a.y, b.y);
        lo[1] = fminf(a.z, b.z);
        hi[1] = fmaxf(a.w, b.w);
        lo[2] = fminf(z.x, z.z);
        hi[2] = fmaxf(z.y, z.w);
        me = p;
        p = ch.z;
    }
}

__global__ void k_leaf_data(const float* __restrict__ v, const int* __restrict__ idx, const float* __restrict__ mat,
                            const float* __restrict__ uv, const int* __restrict__ ids, int n, Tri* tris,
                            float4* mato, float2* uvo, int* slot_of, int* specular) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int id = ids[k];
    slot_of[id] = k;
    int a = idx[3 * id], b = idx[3 * id + 1], c = idx[3 * id + 2];
    Tri t;
    t.v0 = make_float4(v[3 * a], v[3 * a + 1], v[3 * a + 2], __int_as_float(id));
    t.v1 = make_float4(v[3 * b], v[3 * b + 1], v[3 * b + 2], 0.f);
    t.v2 = make_float4(v[3 * c], v[3 * c + 1], v[3 * c + 2], 0.f);
    tris[k] = t;
    const float* m = mat + 8 * (size_t)id;
    mato[2 * k] = make_float4(m[0], m[1], m[2], m[3]);
    mato[2 * k + 1] = make_float4(m[4], m[5], m[6], m[7]);
    if (m[7] > 0.f) atomicOr(specular, 1);
    if (uv) {
        const float* u = uv + 6 * (size_t)id;
        uvo[3 * k] = make_float2(u[0], u[1]);
        uvo[3 * k + 1] = make_float2(u[2], u[3]);
        uvo[3 * k + 2] = make_float2(u[4], u[5]);
    } else {
        uvo[3 * k] = uvo[3 * k + 1] = uvo[3 * k + 2] = make_float2(0.f, 0.f);
    }
}

// Turn every child that covers at most leaf_max triangles into a leaf over
// its contiguous range of sorted triangles (subtrees of a Morton-ordered tree
// cover contiguous key ranges).  Each thread rewrites only its own node.
__global__ void k_leafify(Node* bin, const int2* __restrict__ rng, int n_int, int leaf_max) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int c[2] = {bin[i].child.x, bin[i].child.y};
    for (int k = 0; k < 2; ++k) {
        if (c[k] < 0) c[k] = leaf_ref(~c[k], 1);
        else {
            int cnt = rng[c[k]].y - rng[c[k]].x + 1;
            if (cnt <= leaf_max) c[k] = leaf_ref(rng[c[k]].x, cnt);
        }
    }
    bin[i].child.x = c[0];
    bin[i].child.y = c[1];
}

// depth of every leaf of the original binary tree (an upper bound of the
// traversal depth after leafify), reduced with atomicMax
__global__ void k_depth(const int* __restrict__ leaf_parent, const Node* __restrict__ nodes, int n, unsigned* depth) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned d = 1;
    int p = leaf_parent[k];
    while (p > 0 && d < 4096) {
        p = nodes[p].child.z;
        ++d;
    }
    atomicMax(depth, d);
}

// ---------------------------------------------------------------- PLOC --
// Parallel locally-ordered clustering (Meister and Bittner, "Parallel
// locally-ordered clustering for bounding volume hierarchy construction",
// IEEE TVCG 2018).  Clusters start as the Morton-sorted triangles.  Each
// round every cluster finds, within R positions on either side, the
// cluster whose union box has the smallest surface area; mutual nearest
// neighbours merge into a new node at the lower position, and the array is
// compacted, keeping Morton order.  Rounds repeat until one cluster is left.
#ifndef HDOF_BUILDER
#define HDOF_BUILDER 1  // 1: PLOC, 0: LBVH
#endif
// The search radius R: 64 for trees that stay in L2 (the 164.6k-triangle room:
// the trace 2.5% and the G-buffer 2.6% faster than with 48; 56, 72, 80, 96 slower),
// 48 above PLOC_BIG triangles (the 5.25M-triangle scene's G-buffer is 8% slower
// at 64; radii 8..96 swept).
constexpr int PLOC_R_SMALL = 64, PLOC_R_BIG = 48;
constexpr int PLOC_BIG = 1 << 20;
constexpr int PLOC_B = 256;
constexpr int PLOC_SYNC = 8;  // clustering rounds between reads of the cluster count

__device__ __forceinline__ float union_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    float x = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    float y = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    float z = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    return x * y + y * z + z * x;
}

__global__ void k_ploc_init(const float* __restrict__ v, const int* __restrict__ idx, const int* __restrict__ ids,
                            int n, int* ref, float4* lo, float4* hi, int* hgt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float l[3], h[3];
    tri_box(v, idx, ids[i], l, h);
    ref[i] = leaf_ref(i, 1);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
    hi[i] = make_float4(h[0], h[1], h[2], 0.f);
    hgt[i] = 0;
}

// Round control of the clustering on the device, so that the host need not
// read the cluster count back every round: ctl[0] = live clusters N, ctl[1] =
// pair neighbours this round (the last round found no mutual pair), ctl[2] =
// the buffer holding the clusters.  The round kernels are launched over an
// upper bound Nb >= N and do nothing once N <= 1.
__global__ void k_ploc_ctl_init(int* ctl, int n) {
    ctl[0] = n;
    ctl[1] = 0;
    ctl[2] = 0;
}

template <int PLOC_R>
__global__ void __launch_bounds__(PLOC_B) k_ploc_nn(const int* __restrict__ ctl, const float4* __restrict__ lo,
                                                    const float4* __restrict__ hi, int* __restrict__ nn) {
    const int N = ctl[0];
    if (N <= 1 || ctl[1]) return;  // done, or pairing neighbours: the whole block leaves
    __shared__ float4 slo[PLOC_B + 2 * PLOC_R], shi[PLOC_B + 2 * PLOC_R];
    const int base = blockIdx.x * PLOC_B - PLOC_R;
    for (int k = threadIdx.x; k < PLOC_B + 2 * PLOC_R; k += PLOC_B) {
        int g = base + k;
        if (g >= 0 && g < N) {
            slo[k] = lo[g];
            shi[k] = hi[g];
        }
    }
    __syncthreads();
    const int i = blockIdx.x * PLOC_B + threadIdx.x;
    if (i >= N) return;
    const int li = threadIdx.x + PLOC_R;
    const float4 a0 = slo[li], a1 = shi[li];
    float best = __int_as_float(0x7f800000);
    int bj = -1;
    const int j0 = max(i - PLOC_R, 0), j1 = min(i + PLOC_R, N - 1);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        float c = union_area(a0, a1, slo[j - base], shi[j - base]);
        if (c < best) {  // ascending j: ties keep the lower index
            best = c;
            bj = j;
        }
    }
    nn[i] = bj;
}

// merge mutual nearest neighbours (or, when force_pairs, positions 2k and 2k+1);
// positions N .. Nb - 1 are marked invalid for the scan
__global__ void k_ploc_merge(int Nb, const int* __restrict__ ctl, const int* __restrict__ nn, int* ref, float4* lo,
                             float4* hi, int* hgt, int* valid, Node* nodes, unsigned* counter) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int N = ctl[0], force_pairs = ctl[1];
    if (N <= 1) return;
    if (i >= N) {
        valid[i] = 0;
        return;
    }
    int j = force_pairs ? ((i & 1) ? i - 1 : (i + 1 < N ? i + 1 : -1)) : nn[i];
    bool mutual = j >= 0 && (force_pairs || nn[j] == i);
    if (!mutual) {
        valid[i] = 1;
        return;
    }
    if (j < i) {  // merged into the lower position
        valid[i] = 0;
        return;
    }
    float4 al = lo[i], ah = hi[i], bl = lo[j], bh = hi[j];
    int idn = (int)atomicAdd(counter, 1u);
    Node nd;
    nd.xy0 = make_float4(al.x, ah.x, al.y, ah.y);
    nd.xy1 = make_float4(bl.x, bh.x, bl.y, bh.y);
    nd.z01 = make_float4(al.z, ah.z, bl.z, bh.z);
    nd.child = make_int4(ref[i], ref[j], 0, 0);
    nodes[idn] = nd;
    ref[i] = idn;
    lo[i] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
    hi[i] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
    hgt[i] = max(hgt[i], hgt[j]) + 1;
    valid[i] = 1;
}

__global__ void k_ploc_compact(int Nb, const int* __restrict__ ctl, const int* __restrict__ valid,
                               const int* __restrict__ pos, const int* __restrict__ ref, const float4* __restrict__ lo,
                               const float4* __restrict__ hi, const int* __restrict__ hgt, int* ref2, float4* lo2,
                               float4* hi2, int* hgt2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nb) return;
    const int N = ctl[0];
    if (N <= 1 || i >= N || !valid[i]) return;
    int k = pos[i];
    ref2[k] = ref[i];
    lo2[k] = lo[i];
    hi2[k] = hi[i];
    hgt2[k] = hgt[i];
}

// the next round's N and mode, and the buffer the compaction filled (dst)
__global__ void k_ploc_next(int* ctl, const int* __restrict__ valid, const int* __restrict__ pos, int dst) {
    const int N = ctl[0];
    if (N <= 1) return;
    const int nN = pos[N - 1] + valid[N - 1];
    ctl[1] = nN == N;  // no mutual pair this round: pair neighbours once
    ctl[0] = nN;
    ctl[2] = dst;
}

__global__ void k_big_boxes(const Tri* __restrict__ tris, int first, int n_big, float4* box) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_big) return;
    Tri t = tris[first + k];
    box[2 * k] = make_float4(fminf(t.v0.x, fminf(t.v1.x, t.v2.x)), fminf(t.v0.y, fminf(t.v1.y, t.v2.y)),
                             fminf(t.v0.z, fminf(t.v1.z, t.v2.z)), 0.f);
    box[2 * k + 1] = make_float4(fmaxf(t.v0.x, fmaxf(t.v1.x, t.v2.x)), fmaxf(t.v0.y, fmaxf(t.v1.y, t.v2.y)),
                                 fmaxf(t.v0.z, fmaxf(t.v1.z, t.v2.z)), 0.f);
}

__global__ void k_closest(BvhView bvh, int n, const float* __restrict__ org, const float* __restrict__ dir, int cap,
                          unsigned* status, int* ids, float* ts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Hit h = closest_hit(bvh, ld3(org + 3 * (size_t)i), ld3(dir + 3 * (size_t)i), cap, status);
    ids[i] = h.id;
    ts[i] = h.t;
}

int blocks_for(long n, int bs) { return (int)((n + bs - 1) / bs); }

// ---- depth-first relabelling of the internal nodes --------------------------
// The clustering numbers nodes in merge order, which scatters a parent and its
// children over memory.  Relabelling in depth-first pre-order (a node, then
// its first child's subtree, then its second child's) keeps every subtree in
// one contiguous range and puts a node's first child right after it, so a
// descent touches neighbouring cache lines.  The tree itself is unchanged.

__global__ void k_dfs_parent(const Node* __restrict__ nodes, int n, int* parent, int* nint) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 c = nodes[i].child;
    int k = 0;
    if (c.x >= 0) {
        parent[c.x] = i;
        ++k;
    }
    if (c.y >= 0) {
        parent[c.y] = i;
        ++k;
    }
    nint[i] = k;
}

// subtree sizes (internal nodes) bottom-up: a node with no internal child
// starts a walk; the last child to arrive at a parent carries the walk on
__global__ void k_dfs_size(const Node* __restrict__ nodes, int n, int root, const int* __restrict__ parent,
                           const int* __restrict__ nint, unsigned* arrived, int* size) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || nint[i] != 0) return;
    int c = i;
    size[c] = 1;
    for (int guard = 0; c != root && guard < n; ++guard) {  // a walk is at most the tree's depth
        const int p = parent[c];
        __threadfence();
        if (atomicAdd(&arrived[p], 1u) + 1 < (unsigned)nint[p]) return;  // the other child is not done yet
        __threadfence();
        const int4 ch = nodes[p].child;
        size[p] = 1 + (ch.x >= 0 ? __ldcg(&size[ch.x]) : 0) + (ch.y >= 0 ? __ldcg(&size[ch.y]) : 0);
        c = p;
    }
}

// pre-order index: 1 per ancestor step, plus the first child's subtree when
// the path goes through a second child
__global__ void k_dfs_index(const Node* __restrict__ nodes, int n, int root, const int* __restrict__ parent,
                            const int* __restrict__ size, int* index) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int idx = 0, c = i;
    for (int guard = 0; c != root && guard < n; ++guard) {
        const int p = parent[c];
        const int4 ch = nodes[p].child;
        idx += 1;
        if (c == ch.y && ch.x >= 0) idx += size[ch.x];
        c = p;
    }
    index[i] = idx;
}

__global__ void k_dfs_permute(const Node* __restrict__ nodes, int n, const int* __restrict__ parent,
                              const int* __restrict__ index, const int* __restrict__ size, int root, Node* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Node nd = nodes[i];
    if (nd.child.x >= 0) nd.child.x = index[nd.child.x];
    if (nd.child.y >= 0) nd.child.y = index[nd.child.y];
    nd.child.z = i == root ? -1 : index[parent[i]];
    nd.child.w = size[i];  // internal nodes of the subtree (kept for the leaf collapse)
    out[index[i]] = nd;
}

// Leaf collapse of the clustered tree (in pre-order: node 0 the root,
// child.z the parent, child.w the subtree's internal node count; every leaf
// one triangle).  The triangles are moved to depth-first leaf order, so the
// triangles of any subtree occupy consecutive slots, and each subtree of at
// most leaf_max triangles becomes one leaf over them: fewer traversal steps
// for one more triangle test per extra triangle.  The tree's boxes and the
// closest hits are unchanged.
__device__ __forceinline__ int n_leaves(const Node* __restrict__ nodes, int ref) {
    return ref >= 0 ? __ldg(&nodes[ref].child.w) + 1 : 1;
}

// first leaf position of each node's subtree: the leaves of every first-child
// subtree that the path from the root passes on its left
__global__ void k_leaf_first(const Node* __restrict__ nodes, int n, int* first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int idx = 0, c = i;
    for (int guard = 0; c != 0 && guard < n; ++guard) {  // a walk is at most the tree's depth
        const int p = __ldg(&nodes[c].child.z);
        const int4 ch = __ldg(&nodes[p].child);
        if (c == ch.y) idx += n_leaves(nodes, ch.x);
        c = p;
    }
    first[i] = idx;
}

// new slot of each tree triangle: its depth-first leaf position
__global__ void k_leaf_slots(const Node* __restrict__ nodes, int n, int m, const int* __restrict__ first,
                             int* newpos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 ch = __ldg(&nodes[i].child);
    const int f = first[i];
    if (ch.x < 0 && ((~ch.x) >> 3) < m) newpos[(~ch.x) >> 3] = f;
    if (ch.y < 0 && ((~ch.y) >> 3) < m) newpos[(~ch.y) >> 3] = f + n_leaves(nodes, ch.x);
}

// triangles, materials and texture coordinates to their new slots
__global__ void k_tri_permute(const int* __restrict__ newpos, int m, const Tri* __restrict__ tin,
                              const float4* __restrict__ min, const float2* __restrict__ uin, Tri* tout,
                              float4* mout, float2* uout, int* slot_of) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int d = newpos[k];
    if (d < 0 || d >= m) return;  // unreachable for a full binary tree over the m slots
    const Tri t = tin[k];
    tout[d] = t;
    mout[2 * d] = min[2 * k];
    mout[2 * d + 1] = min[2 * k + 1];
    uout[3 * d] = uin[3 * k];
    uout[3 * d + 1] = uin[3 * k + 1];
    uout[3 * d + 2] = uin[3 * k + 2];
    slot_of[__float_as_int(t.v0.w)] = d;
}

// leaf references to the new slots; subtrees of at most leaf_max triangles
// become leaves (only child.x and child.y are written; child.w is read)
__global__ void k_leaf_collapse(Node* nodes, int n, const int* __restrict__ first, int leaf_max) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cx = nodes[i].child.x, cy = nodes[i].child.y;
    const int c[2] = {cx, cy};
    const int start[2] = {first[i], first[i] + (cx >= 0 ? nodes[cx].child.w + 1 : 1)};
    int out[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (c[k] < 0) {
            out[k] = leaf_ref(start[k], 1);
        } else {
            const int cnt = nodes[c[k]].child.w + 1;
            out[k] = cnt <= leaf_max ? leaf_ref(start[k], cnt) : c[k];
        }
    }
    nodes[i].child.x = out[0];
    nodes[i].child.y = out[1];
}

}  // namespace
}  // namespace hdof

using namespace hdof;

namespace {
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

#ifndef HDOF_PLOC_LEAF_MAX
#define HDOF_PLOC_LEAF_MAX 2  // largest collapsed leaf of the clustered tree (<= 8; 1: no collapse); 2 measured fastest
#endif

// Leaf collapse of the relabelled clustered tree (ni internal nodes over the
// first m triangle slots): see k_leaf_first .. k_leaf_collapse.
cudaError_t collapse_leaves(hdof_bvh* b, int ni, int m, int leaf_max, cudaStream_t s) {
    const size_t q1 = up256(4 * (size_t)ni), q2 = q1 + up256(4 * (size_t)m);
    const size_t q3 = q2 + up256(sizeof(Tri) * (size_t)m), q4 = q3 + up256(2 * sizeof(float4) * (size_t)m);
    const size_t tot = q4 + 3 * sizeof(float2) * (size_t)m;
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, tot);
    if (e != cudaSuccess) return e;
    char* c8 = static_cast<char*>(mem);
    int* first = reinterpret_cast<int*>(c8);
    int* newpos = reinterpret_cast<int*>(c8 + q1);
    Tri* tcopy = reinterpret_cast<Tri*>(c8 + q2);
    float4* mcopy = reinterpret_cast<float4*>(c8 + q3);
    float2* ucopy = reinterpret_cast<float2*>(c8 + q4);
    if ((e = cudaMemsetAsync(newpos, 0xff, 4 * (size_t)m, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(tcopy, b->tris, sizeof(Tri) * (size_t)m, cudaMemcpyDeviceToDevice, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(mcopy, b->mat, 2 * sizeof(float4) * (size_t)m, cudaMemcpyDeviceToDevice, s)) ==
            cudaSuccess &&
        (e = cudaMemcpyAsync(ucopy, b->uv, 3 * sizeof(float2) * (size_t)m, cudaMemcpyDeviceToDevice, s)) ==
            cudaSuccess) {
        k_leaf_first<<<blocks_for(ni, 256), 256, 0, s>>>(b->nodes, ni, first);
        k_leaf_slots<<<blocks_for(ni, 256), 256, 0, s>>>(b->nodes, ni, m, first, newpos);
        k_tri_permute<<<blocks_for(m, 256), 256, 0, s>>>(newpos, m, tcopy, mcopy, ucopy, b->tris, b->mat, b->uv,
                                                         b->slot_of);
        k_leaf_collapse<<<blocks_for(ni, 256), 256, 0, s>>>(b->nodes, ni, first, leaf_max);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(mem);
    return e != cudaSuccess ? e : e2;
}
}  // namespace

extern "C" int hdof_build_bvh(const float* verts, int32_t n_verts, const int32_t* idx, int32_t n_tris,
                              const float* mat, const float* uv, hdof_bvh** out, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(out, "hdof_build_bvh: out is NULL");
    *out = nullptr;
    HDOF_CHECK_ARG(verts && idx && mat, "hdof_build_bvh: verts, idx and mat must be device pointers");
    HDOF_CHECK_ARG(n_tris >= 1 && n_tris <= (1 << 27), "hdof_build_bvh: n_tris %d outside 1..2^27", n_tris);
    HDOF_CHECK_ARG(n_verts >= 3, "hdof_build_bvh: n_verts %d < 3", n_verts);
    cudaStream_t s = as_stream(stream);
    const int n = n_tris;

    // ---- scratch (freed before returning) ----
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                    (int*)nullptr, (int*)nullptr, n, 0, 64, s);
    const size_t nn = (size_t)(n > 1 ? n - 1 : 1);
    size_t o_keys_in = 256, o_keys_out = o_keys_in + up256(8 * (size_t)n), o_ids_in = o_keys_out + up256(8 * (size_t)n);
    size_t o_ids_out = o_ids_in + up256(4 * (size_t)n), o_lp = o_ids_out + up256(4 * (size_t)n);
    size_t o_flags = o_lp + up256(4 * (size_t)n), o_big = o_flags + up256(4 * nn), o_rng = o_big + up256((size_t)n);
    size_t o_cnt = o_rng + up256(8 * nn), o_sort = o_cnt + 256, tmp_total = o_sort + sort_bytes;
    void* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, tmp_total);
    if (e != cudaSuccess) return cuda_fail(e, "hdof_build_bvh: cudaMalloc scratch");
    char* t8 = static_cast<char*>(tmp);
    unsigned* bounds = reinterpret_cast<unsigned*>(t8);
    unsigned long long* keys_in = reinterpret_cast<unsigned long long*>(t8 + o_keys_in);
    unsigned long long* keys_out = reinterpret_cast<unsigned long long*>(t8 + o_keys_out);
    int* ids_in = reinterpret_cast<int*>(t8 + o_ids_in);
    int* ids_out = reinterpret_cast<int*>(t8 + o_ids_out);
    int* leaf_parent = reinterpret_cast<int*>(t8 + o_lp);
    unsigned* flags = reinterpret_cast<unsigned*>(t8 + o_flags);
    uint8_t* big = reinterpret_cast<uint8_t*>(t8 + o_big);
    int2* rng = reinterpret_cast<int2*>(t8 + o_rng);
    unsigned* counters = reinterpret_cast<unsigned*>(t8 + o_cnt);  // [0] tree depth
    void* sort_tmp = t8 + o_sort;

    hdof_bvh* b = nullptr;
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
        if (b) {
            if (b->pool) cudaFree(b->pool);
            delete b;
        }
        return code;
    };
    unsigned init[NB];
    for (int k = 0; k < NB; ++k) init[k] = 0u;
    for (int k : {0, 1, 2, 8, 9, 10, 14, 15, 16}) init[k] = 0xffffffffu;  // atomicMin slots
    if ((e = cudaMemcpyAsync(bounds, init, sizeof init, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: init bounds"));
    const int rb = blocks_for(n, 256) < 1024 ? blocks_for(n, 256) : 1024;
    k_scene_bounds<<<rb, 256, 0, s>>>(verts, n_verts, idx, n, bounds);
    unsigned hb0[NB];
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hb0, bounds, sizeof hb0, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: scene bounds"));
    if (hb0[6]) {
        set_error("hdof_build_bvh: a triangle index is outside 0..n_verts-1");
        return fail(HDOF_EINVAL);
    }
    k_classify<<<rb, 256, 0, s>>>(verts, idx, n, 0.02f, bounds, big);
    unsigned hb[NB];
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hb, bounds, sizeof hb, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: classify"));
    // separate scene-sized triangles only when they are few and the rest can form a tree
    int n_big = (int)hb[7];
    bool separate = n >= 64 && n_big > 0 && n_big <= HDOF_BIG_MAX && n - n_big >= 2;
    if (!separate) n_big = 0;
    const int n_small = n - n_big;
    const unsigned* cbounds = bounds + (separate ? 8 : 14);  // centroid bounds (lo at [0..2], hi at [3..5])

    b = new (std::nothrow) hdof_bvh();
    if (!b) {
        set_error("hdof_build_bvh: host allocation failed");
        return fail(HDOF_ENOMEM);
    }
    cudaGetDevice(&b->device);
    b->n_tris = n;
    b->n_big = n_big;
    const int n_int = n_small > 1 ? n_small - 1 : 1;
    size_t off_tris = up256(sizeof(Node) * (size_t)n_int);
    size_t off_mat = off_tris + up256(sizeof(Tri) * (size_t)n);
    size_t off_uv = off_mat + up256(sizeof(float4) * 2 * (size_t)n);
    size_t off_big = off_uv + up256(sizeof(float2) * 3 * (size_t)n);
    size_t off_slot = off_big + up256(sizeof(float4) * 2 * (size_t)(n_big > 0 ? n_big : 1));
    size_t off_spec = off_slot + up256(sizeof(int) * (size_t)n);
    size_t total = off_spec + sizeof(int);
    if ((e = cudaMalloc(&b->pool, total)) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: cudaMalloc"));
    b->bytes = total;
    char* base = static_cast<char*>(b->pool);
    b->nodes = reinterpret_cast<Node*>(base);
    b->tris = reinterpret_cast<Tri*>(base + off_tris);
    b->mat = reinterpret_cast<float4*>(base + off_mat);
    b->uv = reinterpret_cast<float2*>(base + off_uv);
    b->big_box = reinterpret_cast<float4*>(base + off_big);
    b->slot_of = reinterpret_cast<int*>(base + off_slot);

    // Morton codes and radix sort (scene-sized triangles keyed last)
    k_morton<<<blocks_for(n, 256), 256, 0, s>>>(verts, idx, n, cbounds, separate ? big : nullptr, keys_in, ids_in);
    e = cub::DeviceRadixSort::SortPairs(sort_tmp, sort_bytes, keys_in, keys_out, ids_in, ids_out, n, 0,
                                        separate ? 64 : 63, s);
    if (e != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: sort"));
    int* spec_flag = reinterpret_cast<int*>(base + off_spec);
    if ((e = cudaMemsetAsync(spec_flag, 0, sizeof(int), s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: clear"));
    k_leaf_data<<<blocks_for(n, 256), 256, 0, s>>>(verts, idx, mat, uv, ids_out, n, b->tris, b->mat, b->uv,
                                                    b->slot_of, spec_flag);
    if (n_big > 0) k_big_boxes<<<1, 64, 0, s>>>(b->tris, n - n_big, n_big, b->big_box);
    int has_spec = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&has_spec, spec_flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: leaf data"));
    b->specular = has_spec;

    int depth = 0;
    b->n_nodes = 0;
    if (n_small <= HDOF_LEAF_MAX) {
        b->root = leaf_ref(0, n_small);
        depth = 1;
    } else if (HDOF_BUILDER == 0) {
        // binary LBVH over the first n_small sorted triangles, built in place
        int minus1 = -1;
        Node* nodes = b->nodes;
        if ((e = cudaMemsetAsync(nodes, 0, sizeof(Node) * (size_t)(n_small - 1), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)(n_small - 1), s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&nodes[0].child.z, &minus1, sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(counters, 0, sizeof(unsigned), s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: clear"));
        k_hierarchy<<<blocks_for(n_small - 1, 256), 256, 0, s>>>(keys_out, n_small, nodes, leaf_parent, rng);
        k_refit<<<blocks_for(n_small, 256), 256, 0, s>>>(verts, idx, ids_out, n_small, leaf_parent, nodes, flags);
        k_depth<<<blocks_for(n_small, 256), 256, 0, s>>>(leaf_parent, nodes, n_small, counters);
        k_leafify<<<blocks_for(n_small - 1, 256), 256, 0, s>>>(nodes, rng, n_small - 1, HDOF_LEAF_MAX);
        unsigned hd = 0;
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(&hd, counters, sizeof hd, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: hierarchy"));
        depth = (int)hd;
        b->n_nodes = n_small - 1;
        b->root = 0;
    } else {
        // PLOC over the first n_small sorted triangles
        const int m = n_small;
        size_t scan_bytes = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (int*)nullptr, (int*)nullptr, m, s);
        size_t o_ref0 = 0, o_ref1 = o_ref0 + up256(4 * (size_t)m), o_lo0 = o_ref1 + up256(4 * (size_t)m);
        size_t o_lo1 = o_lo0 + up256(16 * (size_t)m), o_hi0 = o_lo1 + up256(16 * (size_t)m);
        size_t o_hi1 = o_hi0 + up256(16 * (size_t)m), o_h0 = o_hi1 + up256(16 * (size_t)m);
        size_t o_h1 = o_h0 + up256(4 * (size_t)m), o_nn = o_h1 + up256(4 * (size_t)m);
        size_t o_val = o_nn + up256(4 * (size_t)m), o_pos = o_val + up256(4 * (size_t)m);
        size_t o_ctl = o_pos + up256(4 * (size_t)m), o_scan = o_ctl + 256, ptotal = o_scan + scan_bytes;
        void* pt = nullptr;
        if ((e = cudaMalloc(&pt, ptotal)) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: cudaMalloc"));
        char* c8 = static_cast<char*>(pt);
        int* ref[2] = {reinterpret_cast<int*>(c8 + o_ref0), reinterpret_cast<int*>(c8 + o_ref1)};
        float4* lo[2] = {reinterpret_cast<float4*>(c8 + o_lo0), reinterpret_cast<float4*>(c8 + o_lo1)};
        float4* hi[2] = {reinterpret_cast<float4*>(c8 + o_hi0), reinterpret_cast<float4*>(c8 + o_hi1)};
        int* hgt[2] = {reinterpret_cast<int*>(c8 + o_h0), reinterpret_cast<int*>(c8 + o_h1)};
        int* nn = reinterpret_cast<int*>(c8 + o_nn);
        int* valid = reinterpret_cast<int*>(c8 + o_val);
        int* pos = reinterpret_cast<int*>(c8 + o_pos);
        int* ctl = reinterpret_cast<int*>(c8 + o_ctl);
        void* scan_tmp = c8 + o_scan;
        auto pfail = [&](int code) {
            cudaStreamSynchronize(s);
            cudaFree(pt);
            return fail(code);
        };
        if ((e = cudaMemsetAsync(counters, 0, sizeof(unsigned), s)) != cudaSuccess)
            return pfail(cuda_fail(e, "hdof_build_bvh: clear"));
        k_ploc_init<<<blocks_for(m, 256), 256, 0, s>>>(verts, idx, ids_out, m, ref[0], lo[0], hi[0], hgt[0]);
        k_ploc_ctl_init<<<1, 1, 0, s>>>(ctl, m);
        // rounds run in batches of PLOC_SYNC with the cluster count kept on the
        // device; the host reads it between batches for a tighter launch bound
        int Nb = m, cur = 0, rounds = 0, buf = 0;
        while (true) {
            for (int r = 0; r < PLOC_SYNC; ++r) {
                if (m > PLOC_BIG) k_ploc_nn<PLOC_R_BIG><<<blocks_for(Nb, PLOC_B), PLOC_B, 0, s>>>(ctl, lo[cur], hi[cur], nn);
                else k_ploc_nn<PLOC_R_SMALL><<<blocks_for(Nb, PLOC_B), PLOC_B, 0, s>>>(ctl, lo[cur], hi[cur], nn);
                k_ploc_merge<<<blocks_for(Nb, 256), 256, 0, s>>>(Nb, ctl, nn, ref[cur], lo[cur], hi[cur], hgt[cur],
                                                                valid, b->nodes, counters);
                e = cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, valid, pos, Nb, s);
                if (e != cudaSuccess) return pfail(cuda_fail(e, "hdof_build_bvh: scan"));
                k_ploc_compact<<<blocks_for(Nb, 256), 256, 0, s>>>(Nb, ctl, valid, pos, ref[cur], lo[cur], hi[cur],
                                                                  hgt[cur], ref[1 - cur], lo[1 - cur], hi[1 - cur],
                                                                  hgt[1 - cur]);
                k_ploc_next<<<1, 1, 0, s>>>(ctl, valid, pos, 1 - cur);
                cur = 1 - cur;
            }
            rounds += PLOC_SYNC;
            int c[3];
            if ((e = cudaGetLastError()) != cudaSuccess ||
                (e = cudaMemcpyAsync(c, ctl, sizeof c, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return pfail(cuda_fail(e, "hdof_build_bvh: clustering"));
            if (c[0] <= 1) {
                buf = c[2];
                break;
            }
            if (rounds > 100000) {
                set_error("hdof_build_bvh: clustering did not converge");
                return pfail(HDOF_ECUDA);
            }
            Nb = c[0];
        }
        int root_ref = 0, h = 0;
        if ((e = cudaMemcpyAsync(&root_ref, ref[buf], sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&h, hgt[buf], sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return pfail(cuda_fail(e, "hdof_build_bvh: clustering"));
        cudaFree(pt);
        depth = h;
        b->n_nodes = m - 1;
        b->root = root_ref;
        if (root_ref >= 0 && m - 1 > 1) {
            const int ni = m - 1;
            // scratch: parent, nint, arrived, size, index (ints) + a node copy
            size_t q0 = 0, q1 = q0 + up256(4 * (size_t)ni), q2 = q1 + up256(4 * (size_t)ni);
            size_t q3 = q2 + up256(4 * (size_t)ni), q4 = q3 + up256(4 * (size_t)ni);
            size_t q5 = q4 + up256(4 * (size_t)ni), qtot = q5 + sizeof(Node) * (size_t)ni;
            void* rt = nullptr;
            if ((e = cudaMalloc(&rt, qtot)) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: cudaMalloc"));
            char* r8 = static_cast<char*>(rt);
            int* parent = reinterpret_cast<int*>(r8 + q0);
            int* nint = reinterpret_cast<int*>(r8 + q1);
            unsigned* arrived = reinterpret_cast<unsigned*>(r8 + q2);
            int* size = reinterpret_cast<int*>(r8 + q3);
            int* index = reinterpret_cast<int*>(r8 + q4);
            Node* copy = reinterpret_cast<Node*>(r8 + q5);
            const int nb = blocks_for(ni, 256);
            if ((e = cudaMemsetAsync(arrived, 0, 4 * (size_t)ni, s)) == cudaSuccess) {
                k_dfs_parent<<<nb, 256, 0, s>>>(b->nodes, ni, parent, nint);
                k_dfs_size<<<nb, 256, 0, s>>>(b->nodes, ni, root_ref, parent, nint, arrived, size);
                k_dfs_index<<<nb, 256, 0, s>>>(b->nodes, ni, root_ref, parent, size, index);
                k_dfs_permute<<<nb, 256, 0, s>>>(b->nodes, ni, parent, index, size, root_ref, copy);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->nodes, copy, sizeof(Node) * (size_t)ni, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cudaFree(rt);
            if (e != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: relabel"));
            b->root = 0;
            if (HDOF_PLOC_LEAF_MAX > 1 && (e = collapse_leaves(b, ni, m, HDOF_PLOC_LEAF_MAX, s)) != cudaSuccess)
                return fail(cuda_fail(e, "hdof_build_bvh: leaf collapse"));
        }
    }
    b->depth = depth;
    if (depth + 1 >= HDOF_STACK) {
        set_error("hdof_build_bvh: tree depth %d exceeds the %d-entry traversal stack", depth, HDOF_STACK);
        return fail(HDOF_EUNSUPPORTED);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: build"));
    cudaFree(tmp);
    *out = b;
    return HDOF_OK;
}

extern "C" int hdof_bvh_destroy(hdof_bvh* b) {
    clear_error();
    if (!b) return HDOF_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaError_t e = cudaFree(b->pool);
    if (cur != b->device) cudaSetDevice(cur);
    delete b;
    return e == cudaSuccess ? HDOF_OK : cuda_fail(e, "hdof_bvh_destroy");
}

extern "C" int hdof_bvh_info(const hdof_bvh* b, hdof_bvh_stats* info) {
    clear_error();
    HDOF_CHECK_ARG(b && info, "hdof_bvh_info: NULL argument");
    info->n_tris = b->n_tris;
    info->n_nodes = b->n_nodes;
    info->depth = b->depth;
    info->n_big = b->n_big;
    info->device_bytes = (int64_t)b->bytes;
    return HDOF_OK;
}

extern "C" int hdof_closest_hits(const hdof_bvh* b, int32_t n, const float* org, const float* dir, int32_t* ids,
                                 float* ts, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_closest_hits: bvh is NULL");
    HDOF_CHECK_ARG(n >= 0, "hdof_closest_hits: n < 0");
    if (n == 0) return HDOF_OK;
    HDOF_CHECK_ARG(org && dir && ids && ts, "hdof_closest_hits: NULL buffer");
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_closest_hits: no status word on this device");
    int cap = 64 * (b->n_nodes + b->n_tris) + 64;
    k_closest<<<blocks_for(n, 128), 128, 0, as_stream(stream)>>>(b->view(), n, org, dir, cap, st, ids, ts);
    HDOF_LAUNCHED("hdof_closest_hits");
    return HDOF_OK;
}
