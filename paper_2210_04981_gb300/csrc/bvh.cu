// linear BVH build (Karras, "Maximizing parallelism in the construction
// of BVHs, octrees and k-d trees", HPG 2012) standing in for the paper's
// hardware ray-tracing acceleration structure (Abstract), plus the
// closest-hit query used to check it.
//
// Steps: centroid bounds -> 30-bit Morton codes -> radix sort of
// (code, triangle) pairs -> one thread per internal node finds its key range
// and split (ties between equal codes broken by sorted position) -> one
// thread per leaf walks up refitting child boxes (the second child to
// arrive at a node computes the union) -> triangles, materials and UVs are
// stored in leaf order.
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

struct BuildScratch {
    unsigned* bounds;  // 6 ordered floats: centroid lo xyz, hi xyz; [6] = bad-index flag; [7] = depth
    unsigned* keys_in;
    unsigned* keys_out;
    int* ids_in;
    int* ids_out;
    int* leaf_parent;
    unsigned* flags;
    void* sort_tmp;
    size_t sort_bytes;
};

__global__ void k_bounds(const float* __restrict__ v, int nv, const int* __restrict__ idx, int n,
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
            float cen = (v[3 * a + k] + v[3 * b + k] + v[3 * c + k]) * (1.f / 3.f);
            lo[k] = fminf(lo[k], cen);
            hi[k] = fmaxf(hi[k], cen);
        }
    }
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], f2ord(lo[k]));
            atomicMax(&bounds[3 + k], f2ord(hi[k]));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&bounds[6], 1u);
}

__device__ __forceinline__ unsigned expand10(unsigned x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(const float* __restrict__ v, const int* __restrict__ idx, int n,
                         const unsigned* __restrict__ bounds, unsigned* keys, int* ids) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    unsigned code = 0;
    int a = idx[3 * t], b = idx[3 * t + 1], c = idx[3 * t + 2];
    unsigned q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bounds[k]), hi = ord2f(bounds[3 + k]);
        float cen = (v[3 * a + k] + v[3 * b + k] + v[3 * c + k]) * (1.f / 3.f);
        float ext = hi - lo;
        float u = ext > 0.f ? (cen - lo) / ext : 0.5f;
        q[k] = (unsigned)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
    }
    code = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    keys[t] = code;
    ids[t] = t;
}

// common-prefix length of sorted keys i and j (64-bit key = code, position)
__device__ __forceinline__ int delta(const unsigned* __restrict__ keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned a = keys[i], b = keys[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((unsigned)i ^ (unsigned)j);
}

__global__ void k_hierarchy(const unsigned* __restrict__ keys, int n, Node* nodes, int* leaf_parent) {
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
                            float4* mato, float2* uvo) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int id = ids[k];
    int a = idx[3 * id], b = idx[3 * id + 1], c = idx[3 * id + 2];
    Tri t;
    t.v0 = make_float4(v[3 * a], v[3 * a + 1], v[3 * a + 2], __int_as_float(id));
    t.v1 = make_float4(v[3 * b], v[3 * b + 1], v[3 * b + 2], 0.f);
    t.v2 = make_float4(v[3 * c], v[3 * c + 1], v[3 * c + 2], 0.f);
    tris[k] = t;
    const float* m = mat + 8 * (size_t)id;
    mato[2 * k] = make_float4(m[0], m[1], m[2], m[3]);
    mato[2 * k + 1] = make_float4(m[4], m[5], m[6], m[7]);
    if (uv) {
        const float* u = uv + 6 * (size_t)id;
        uvo[3 * k] = make_float2(u[0], u[1]);
        uvo[3 * k + 1] = make_float2(u[2], u[3]);
        uvo[3 * k + 2] = make_float2(u[4], u[5]);
    } else {
        uvo[3 * k] = uvo[3 * k + 1] = uvo[3 * k + 2] = make_float2(0.f, 0.f);
    }
}

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

__global__ void k_single(const float* __restrict__ v, const int* __restrict__ idx, Node* nodes) {
    float lo[3], hi[3];
    tri_box(v, idx, 0, lo, hi);
    Node nd;
    nd.child = make_int4(~0, ~0, -1, 0);
    write_child_box(&nd, 0, lo, hi);
    write_child_box(&nd, 1, lo, hi);
    nodes[0] = nd;
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

}  // namespace
}  // namespace hdof

using namespace hdof;

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
    const int n_nodes = n > 1 ? n - 1 : 1;

    hdof_bvh* b = new (std::nothrow) hdof_bvh();
    if (!b) {
        set_error("hdof_build_bvh: host allocation failed");
        return HDOF_ENOMEM;
    }
    cudaGetDevice(&b->device);
    b->n_tris = n;
    b->n_nodes = n_nodes;
    size_t off_nodes = 0;
    size_t off_tris = (off_nodes + sizeof(Node) * (size_t)n_nodes + 255) & ~size_t(255);
    size_t off_mat = (off_tris + sizeof(Tri) * (size_t)n + 255) & ~size_t(255);
    size_t off_uv = (off_mat + sizeof(float4) * 2 * (size_t)n + 255) & ~size_t(255);
    size_t total = off_uv + sizeof(float2) * 3 * (size_t)n;
    b->bytes = total;
    cudaError_t e = cudaMalloc(&b->pool, total);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "hdof_build_bvh: cudaMalloc");
    }
    char* base = static_cast<char*>(b->pool);
    b->nodes = reinterpret_cast<Node*>(base + off_nodes);
    b->tris = reinterpret_cast<Tri*>(base + off_tris);
    b->mat = reinterpret_cast<float4*>(base + off_mat);
    b->uv = reinterpret_cast<float2*>(base + off_uv);

    // scratch
    BuildScratch sc{};
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (unsigned*)nullptr, (unsigned*)nullptr, (int*)nullptr,
                                    (int*)nullptr, n, 0, 30, s);
    size_t o_b = 0, o_ki = 256, o_ko = o_ki + ((sizeof(unsigned) * n + 255) & ~size_t(255));
    size_t o_ii = o_ko + ((sizeof(unsigned) * n + 255) & ~size_t(255));
    size_t o_io = o_ii + ((sizeof(int) * n + 255) & ~size_t(255));
    size_t o_lp = o_io + ((sizeof(int) * n + 255) & ~size_t(255));
    size_t o_fl = o_lp + ((sizeof(int) * n + 255) & ~size_t(255));
    size_t o_st = o_fl + ((sizeof(unsigned) * n_nodes + 255) & ~size_t(255));
    size_t tmp_total = o_st + sort_bytes;
    void* tmp = nullptr;
    e = cudaMalloc(&tmp, tmp_total);
    if (e != cudaSuccess) {
        cudaFree(b->pool);
        delete b;
        return cuda_fail(e, "hdof_build_bvh: cudaMalloc scratch");
    }
    char* t8 = static_cast<char*>(tmp);
    sc.bounds = reinterpret_cast<unsigned*>(t8 + o_b);
    sc.keys_in = reinterpret_cast<unsigned*>(t8 + o_ki);
    sc.keys_out = reinterpret_cast<unsigned*>(t8 + o_ko);
    sc.ids_in = reinterpret_cast<int*>(t8 + o_ii);
    sc.ids_out = reinterpret_cast<int*>(t8 + o_io);
    sc.leaf_parent = reinterpret_cast<int*>(t8 + o_lp);
    sc.flags = reinterpret_cast<unsigned*>(t8 + o_fl);
    sc.sort_tmp = t8 + o_st;
    sc.sort_bytes = sort_bytes;

    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
        cudaFree(b->pool);
        delete b;
        return code;
    };
    unsigned init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
    if ((e = cudaMemcpyAsync(sc.bounds, init, sizeof init, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: init bounds"));
    k_bounds<<<blocks_for(n, 256) < 1024 ? blocks_for(n, 256) : 1024, 256, 0, s>>>(verts, n_verts, idx, n,
                                                                                    sc.bounds);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: bounds"));
    unsigned hb[8];
    if ((e = cudaMemcpyAsync(hb, sc.bounds, sizeof hb, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "hdof_build_bvh: read bounds"));
    if (hb[6]) {
        set_error("hdof_build_bvh: a triangle index is outside 0..n_verts-1");
        return fail(HDOF_EINVAL);
    }
    if (n == 1) {
        k_single<<<1, 1, 0, s>>>(verts, idx, b->nodes);
        int* zero_id = sc.ids_out;
        if ((e = cudaMemsetAsync(zero_id, 0, sizeof(int), s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: single"));
        k_leaf_data<<<1, 32, 0, s>>>(verts, idx, mat, uv, zero_id, 1, b->tris, b->mat, b->uv);
        b->depth = 1;
    } else {
        k_morton<<<blocks_for(n, 256), 256, 0, s>>>(verts, idx, n, sc.bounds, sc.keys_in, sc.ids_in);
        e = cub::DeviceRadixSort::SortPairs(sc.sort_tmp, sc.sort_bytes, sc.keys_in, sc.keys_out, sc.ids_in,
                                            sc.ids_out, n, 0, 30, s);
        if (e != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: sort"));
        if ((e = cudaMemsetAsync(b->nodes, 0, sizeof(Node) * (size_t)n_nodes, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(sc.flags, 0, sizeof(unsigned) * (size_t)n_nodes, s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: clear"));
        // the root has no parent
        int minus1 = -1;
        if ((e = cudaMemcpyAsync(&b->nodes[0].child.z, &minus1, sizeof(int), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: root"));
        k_hierarchy<<<blocks_for(n - 1, 256), 256, 0, s>>>(sc.keys_out, n, b->nodes, sc.leaf_parent);
        k_refit<<<blocks_for(n, 256), 256, 0, s>>>(verts, idx, sc.ids_out, n, sc.leaf_parent, b->nodes, sc.flags);
        k_leaf_data<<<blocks_for(n, 256), 256, 0, s>>>(verts, idx, mat, uv, sc.ids_out, n, b->tris, b->mat, b->uv);
        if ((e = cudaMemsetAsync(sc.bounds + 7, 0, sizeof(unsigned), s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: depth"));
        k_depth<<<blocks_for(n, 256), 256, 0, s>>>(sc.leaf_parent, b->nodes, n, sc.bounds + 7);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "hdof_build_bvh: kernels"));
        unsigned depth = 0;
        if ((e = cudaMemcpyAsync(&depth, sc.bounds + 7, sizeof depth, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(cuda_fail(e, "hdof_build_bvh: build"));
        b->depth = (int)depth;
        if (depth >= HDOF_STACK) {
            set_error("hdof_build_bvh: tree depth %u exceeds the traversal stack (%d)", depth, HDOF_STACK);
            return fail(HDOF_EUNSUPPORTED);
        }
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
    info->reserved = 0;
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
