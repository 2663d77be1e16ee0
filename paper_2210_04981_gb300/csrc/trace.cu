// compaction of the masked pixels and thin-lens distributed ray
// tracing (Ray Trace section).  Rays originate at random points of the lens
// disk and aim at the pixel's point on the focus plane; each hit is split
// between the near and far layers by its CoC (linear across the focus zone)
// and a hit ratio is kept.
//
// Compaction (deterministic, tile order): k_count counts traced pixels and
// rays per 16x16 tile, k_scan turns the counts into queue offsets, k_scatter
// writes pixel indices in row-major order within each tile.  The persistent
// kernel k_trace then pulls 32-pixel chunks from the queue with one atomic
// per warp; each thread traces all samples of its pixel in sample order and
// writes the normalised per-pixel result once, so the output does not depend
// on scheduling.
#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

constexpr int TB = 16;  // compaction tile edge

struct CountArgs {
    const uint8_t* spp;
    int W, H, ntx;
    unsigned* counts;
};

__device__ __forceinline__ void count_body(const CountArgs& a, int bx, int by) {
    const uint8_t* __restrict__ spp = a.spp;
    const int W = a.W, H = a.H, ntx = a.ntx;
    unsigned* __restrict__ counts = a.counts;
    int i = bx * TB + (threadIdx.x & 15), j = by * TB + (threadIdx.x >> 4);
    unsigned s = (i < W && j < H) ? spp[(size_t)j * W + i] : 0u;
    unsigned px = __syncthreads_count(s > 0);
    __shared__ unsigned red[8];
    unsigned r = s;
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int k = 0; k < 8; ++k) t += red[k];
        int tile = by * ntx + bx;
        counts[2 * tile] = px;
        counts[2 * tile + 1] = t;
    }
}

__global__ void __launch_bounds__(256) k_count(CountArgs a) { count_body(a, blockIdx.x, blockIdx.y); }

// one block: exclusive scans of the per-tile pixel and ray counts -> queue
// and ray offsets; totals -> stats
struct ScanArgs {
    const unsigned* counts;
    int ntiles;
    unsigned* offsets;
    unsigned* roffsets;
    unsigned* totals;
    unsigned* stats;
};

__device__ __forceinline__ void scan_body(const ScanArgs& a) {
    const unsigned* __restrict__ counts = a.counts;
    const int ntiles = a.ntiles;
    unsigned* __restrict__ offsets = a.offsets;
    unsigned* __restrict__ roffsets = a.roffsets;
    unsigned* __restrict__ totals = a.totals;
    unsigned* __restrict__ stats = a.stats;
    __shared__ unsigned wsum[2][32];
    __shared__ unsigned carry[2];
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += 1024) {
        int t = base + threadIdx.x;
        unsigned v[2] = {t < ntiles ? counts[2 * t] : 0u, t < ntiles ? counts[2 * t + 1] : 0u};
        unsigned x[2] = {v[0], v[1]};
        for (int c = 0; c < 2; ++c)
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, x[c], o);
                if (lane >= o) x[c] += y;
            }
        if (lane == 31) {
            wsum[0][w] = x[0];
            wsum[1][w] = x[1];
        }
        __syncthreads();
        if (w < 2) {
            unsigned sv = wsum[w][lane];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += y;
            }
            wsum[w][lane] = sv;
        }
        __syncthreads();
        unsigned e0 = carry[0] + (w ? wsum[0][w - 1] : 0u) + x[0] - v[0];
        unsigned e1 = carry[1] + (w ? wsum[1][w - 1] : 0u) + x[1] - v[1];
        if (t < ntiles) {
            offsets[t] = e0;
            roffsets[t] = e1;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry[0] = e0 + v[0];
            carry[1] = e1 + v[1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = carry[0];  // queue length
        totals[1] = 0;         // queue head
        if (stats) {
            stats[0] = carry[0];
            stats[1] = carry[1];
        }
    }
}

__global__ void __launch_bounds__(1024) k_scan(ScanArgs a) { scan_body(a); }

// queue entries in row-major order within each tile; optionally the first
// ray of every traced pixel (tile ray offset + prefix of spp in queue order)
struct ScatterArgs {
    const uint8_t* spp;
    int W, H, ntx;
    const unsigned* offsets;
    const unsigned* roffsets;
    unsigned* queue;
    unsigned* ray_off;
};

__device__ __forceinline__ void scatter_body(const ScatterArgs& a, int bx, int by) {
    const uint8_t* __restrict__ spp = a.spp;
    const int W = a.W, H = a.H, ntx = a.ntx;
    const unsigned* __restrict__ offsets = a.offsets;
    const unsigned* __restrict__ roffsets = a.roffsets;
    unsigned* __restrict__ queue = a.queue;
    unsigned* __restrict__ ray_off = a.ray_off;
    int i = bx * TB + (threadIdx.x & 15), j = by * TB + (threadIdx.x >> 4);
    unsigned n = (i < W && j < H) ? spp[(size_t)j * W + i] : 0u;
    bool on = n > 0;
    unsigned m = __ballot_sync(0xffffffffu, on);
    __shared__ unsigned wcnt[8], wray[8];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned r = n;  // inclusive warp prefix of spp
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, r, o);
        if (lane >= o) r += y;
    }
    if (lane == 0) wcnt[w] = __popc(m);
    if (lane == 31) wray[w] = r;
    __syncthreads();
    const int tile = by * ntx + bx;
    unsigned base = offsets[tile], rbase = roffsets[tile];
    for (int k = 0; k < w; ++k) {
        base += wcnt[k];
        rbase += wray[k];
    }
    if (on) {
        queue[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)(j * W + i);
        if (ray_off) ray_off[(size_t)j * W + i] = rbase + r - n;
    }
}

__global__ void __launch_bounds__(256) k_scatter(ScatterArgs a) { scatter_body(a, blockIdx.x, blockIdx.y); }

struct TraceArgs {
    BvhView bvh;
    Cam cam;
    Coc coc;
    Lights L;
    float A, zf, miss_dist;
    uint2 key;
    int cap;
    unsigned* status;
    const uint8_t* spp;
    const unsigned* queue;
    unsigned* totals;  // [0] queue length, [1] head
    float4* rt;        // 3 float4 per pixel
    float4* rec;       // optional per-ray (L rgb, z) records, z = +inf for a miss
    const unsigned* ray_off;
};

__device__ __forceinline__ void trace_pixel(const TraceArgs& a, unsigned q) {
    const int W = a.cam.W;
    const int i = (int)(q % (unsigned)W), j = (int)(q / (unsigned)W);
    const int n = a.spp[q];
    const float3 d = pinhole_dir(a.cam, i + 0.5f + a.cam.jx, j + 0.5f + a.cam.jy);
    const float3 Pf = a.cam.pos + a.zf * d;
    float3 SwL = f3(0, 0, 0), SfL = f3(0, 0, 0), SfP = f3(0, 0, 0);
    float Sw = 0.f, Sf = 0.f, Swc = 0.f, Sfc = 0.f;
    for (int smp = 0; smp < n; ++smp) {
        uint4 x = philox4x32_10(make_uint4(q, (unsigned)smp, 0u, 0u), a.key);
        float rho = a.A * sqrtf(u01(x.x));
        float sn, cs;
        sincospif(2.f * u01(x.y), &sn, &cs);
        float3 O = a.cam.pos + (rho * cs) * a.cam.right + (rho * sn) * a.cam.up;
        float3 dir = normalize(Pf - O);
        Hit h = closest_hit(a.bvh, O, dir, a.cap, a.status);
        float3 L, P, nrm;
        float c;
        if (h.slot >= 0) {
            P = O + h.t * dir;
            c = a.coc(dot(P - a.cam.pos, a.cam.fwd));
            shade(a.bvh, a.L, h, dir, nrm, L);
        } else {
            P = O + a.miss_dist * dir;
            c = a.coc.at_infinity();
            L = f3(0.f, 0.f, 0.f);
        }
        if (a.rec) a.rec[a.ray_off[q] + smp] = make_float4(L.x, L.y, L.z, h.slot >= 0 ? dot(P - a.cam.pos, a.cam.fwd)
                                                                                   : __int_as_float(0x7f800000));
        float w = w_near(c), wf = 1.f - w, ac = fabsf(c);
        SwL = SwL + w * L;
        SfL = SfL + wf * L;
        SfP = SfP + wf * P;
        Sw += w;
        Sf += wf;
        Swc += w * ac;
        Sfc += wf * ac;
    }
    bool nok = Sw >= HDOF_EMPTY_W, fok = Sf >= HDOF_EMPTY_W;
    float in = nok ? 1.f / Sw : 0.f, inf_ = fok ? 1.f / Sf : 0.f;
    float4* o = a.rt + 3 * (size_t)q;
    o[0] = make_float4(SwL.x * in, SwL.y * in, SwL.z * in, Sw / (float)n);
    o[1] = make_float4(SfL.x * inf_, SfL.y * inf_, SfL.z * inf_, nok ? Swc * in : -1.f);
    o[2] = make_float4(SfP.x * inf_, SfP.y * inf_, SfP.z * inf_, fok ? Sfc * inf_ : -1.f);
}

#ifndef HDOF_TRACE_MINB
#define HDOF_TRACE_MINB 1
#endif
__global__ void __launch_bounds__(128, HDOF_TRACE_MINB) k_trace(TraceArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned n = __ldcg(&a.totals[0]);
    while (true) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&a.totals[1], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        unsigned k = base + lane;
        if (k < n) trace_pixel(a, __ldg(&a.queue[k]));
    }
}

TraceArgs trace_args(const hdof_bvh* b, const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p,
                     unsigned* st, const uint8_t* spp, const unsigned* queue, unsigned* totals, float* rt, float* rec,
                     const unsigned* ray_off) {
    TraceArgs a;
    a.bvh = b->view();
    a.cam = make_cam(*cam);
    a.coc = make_coc(*lens, cam->height, cam->tan_half_fovy);
    a.L = make_lights(*p);
    a.A = lens->aperture_radius;
    a.zf = lens->focus_dist;
    a.miss_dist = p->miss_dist;
    a.key = make_uint2(p->seed, (unsigned)p->view * 65536u + (unsigned)p->frame);
    a.cap = p->trav_cap > 0 ? p->trav_cap : 64 * (b->n_nodes + b->n_tris) + 64;
    a.status = st;
    a.spp = spp;
    a.queue = queue;
    a.totals = totals;
    a.rt = reinterpret_cast<float4*>(rt);
    a.rec = reinterpret_cast<float4*>(rec);
    a.ray_off = ray_off;
    return a;
}

// ---- multi-view forms -------------------------------------------------------

__global__ void __launch_bounds__(256) k_count_batch(const CountArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    count_body(a[v], bx, by);
}
__global__ void __launch_bounds__(1024) k_scan_batch(const ScanArgs* __restrict__ a) { scan_body(a[blockIdx.x]); }
__global__ void __launch_bounds__(256) k_scatter_batch(const ScatterArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    scatter_body(a[v], bx, by);
}

// exclusive prefix of the views' queue lengths: gq[v] is the first entry of
// view v in the concatenated queue, gq[n] the total; gq[n + 1] (the shared
// queue head) is reset.  One block.
__global__ void __launch_bounds__(1024) k_queue_prefix(const ScanArgs* __restrict__ a, int n,
                                                       unsigned* __restrict__ gq) {
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        int v = base + threadIdx.x;
        unsigned c = v < n ? __ldcg(&a[v].totals[0]) : 0u, x = c;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned sv = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += y;
            }
            wsum[lane] = sv;
        }
        __syncthreads();
        unsigned e = carry + (w ? wsum[w - 1] : 0u) + x - c;
        if (v < n) gq[v] = e;
        __syncthreads();
        if (threadIdx.x == 1023) carry = e + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        gq[n] = carry;
        gq[n + 1] = 0;
    }
}

// persistent trace over the concatenated queues of all views: a warp takes
// 32 * chunk entries per atomic; each entry finds its view by binary search
// of gq and is traced exactly as the single-view kernel traces it
template <int BS>
__global__ void __launch_bounds__(BS) k_trace_batch(const TraceArgs* __restrict__ a, const unsigned* __restrict__ gq,
                                                    int n, unsigned* head, int chunk) {
    const int lane = threadIdx.x & 31;
    const unsigned total = __ldcg(&gq[n]);
    const unsigned step = 32u * (unsigned)chunk;
    while (true) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(head, step);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        for (int c = 0; c < chunk; ++c) {
            unsigned k = base + 32u * (unsigned)c + (unsigned)lane;
            if (k >= total) break;
            int lo = 0, hi = n - 1;  // last view with gq[v] <= k
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (__ldg(&gq[mid]) <= k) lo = mid;
                else hi = mid - 1;
            }
            const TraceArgs& av = a[lo];
            trace_pixel(av, __ldg(&av.queue[k - __ldg(&gq[lo])]));
        }
    }
}

template <int BS>
int trace_batch_occupancy(int* nb) {
    HDOF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_trace_batch<BS>, BS, 0), "batched trace: occupancy");
    if (*nb < 1) *nb = 1;
    return HDOF_OK;
}

}  // namespace

size_t count_args_size() { return sizeof(CountArgs); }
void count_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TB - 1) / TB;
    *reinterpret_cast<CountArgs*>(dst) = CountArgs{v.spp, W, H, ntx, w.counts};
    *gx = ntx;
    *gy = (H + TB - 1) / TB;
}
void count_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    k_count_batch<<<blocks, 256, 0, s>>>(static_cast<const CountArgs*>(args), g);
}

size_t scan_args_size() { return sizeof(ScanArgs); }
void scan_fill(const hdof_view& v, const ViewWs& w, void* dst) {
    const int ntiles = ((v.cam.width + TB - 1) / TB) * ((v.cam.height + TB - 1) / TB);
    *reinterpret_cast<ScanArgs*>(dst) = ScanArgs{w.counts, ntiles, w.offsets, w.roffsets, w.totals, v.stats};
}
void scan_launch_batch(const void* args, int n, cudaStream_t s) {
    k_scan_batch<<<n, 1024, 0, s>>>(static_cast<const ScanArgs*>(args));
}

size_t scatter_args_size() { return sizeof(ScatterArgs); }
void scatter_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TB - 1) / TB;
    *reinterpret_cast<ScatterArgs*>(dst) = ScatterArgs{v.spp, W, H, ntx, w.offsets, w.roffsets, w.queue, nullptr};
    *gx = ntx;
    *gy = (H + TB - 1) / TB;
}
void scatter_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    k_scatter_batch<<<blocks, 256, 0, s>>>(static_cast<const ScatterArgs*>(args), g);
}

size_t trace_args_size() { return sizeof(TraceArgs); }
void trace_fill(const hdof_view& v, const ViewWs& w, unsigned* st, void* dst) {
    *reinterpret_cast<TraceArgs*>(dst) =
        trace_args(v.bvh, &v.cam, &v.lens, &v.params, st, v.spp, w.queue, w.totals, v.rt, nullptr, nullptr);
}
int trace_batch_grid(int block, int* blocks) {
    int nb = 1, rc;
    if (block == 64) rc = trace_batch_occupancy<64>(&nb);
    else if (block == 256) rc = trace_batch_occupancy<256>(&nb);
    else rc = trace_batch_occupancy<128>(&nb);
    if (rc) return rc;
    *blocks = sm_count() * nb;
    return HDOF_OK;
}

int trace_launch_batch(const void* scan_args, const void* trace_args, int n, unsigned* gq, int block, int chunk,
                       int blocks, cudaStream_t s) {
    k_queue_prefix<<<1, 1024, 0, s>>>(static_cast<const ScanArgs*>(scan_args), n, gq);
    HDOF_LAUNCHED("batched trace: queue prefix");
    const TraceArgs* a = static_cast<const TraceArgs*>(trace_args);
    if (block == 64) k_trace_batch<64><<<blocks, 64, 0, s>>>(a, gq, n, gq + n + 1, chunk);
    else if (block == 256) k_trace_batch<256><<<blocks, 256, 0, s>>>(a, gq, n, gq + n + 1, chunk);
    else k_trace_batch<128><<<blocks, 128, 0, s>>>(a, gq, n, gq + n + 1, chunk);
    HDOF_LAUNCHED("batched trace");
    return HDOF_OK;
}

}  // namespace hdof

using namespace hdof;

extern "C" int hdof_trace(const hdof_bvh* b, const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p,
                          const uint8_t* spp, float* rt, uint32_t* stats, float* rec, uint32_t* ray_off,
                          void* workspace, size_t workspace_bytes, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_trace: bvh is NULL");
    int rc;
    if ((rc = check_camera(cam, "hdof_trace")) || (rc = check_lens(lens, "hdof_trace")) ||
        (rc = check_params(p, "hdof_trace")))
        return rc;
    HDOF_CHECK_ARG(spp && rt, "hdof_trace: spp and rt are required");
    HDOF_CHECK_ARG(!rec == !ray_off, "hdof_trace: rec and ray_off go together");
    const int W = cam->width, H = cam->height;
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.trace_counts + L.trace_queue,
                   "hdof_trace: workspace of %zu bytes < %zu", workspace_bytes, L.trace_counts + L.trace_queue);
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_trace: no status word on this device");
    cudaStream_t s = as_stream(stream);
    const int ntx = (W + TB - 1) / TB, nty = (H + TB - 1) / TB, ntiles = ntx * nty;
    unsigned* counts = static_cast<unsigned*>(workspace);            // [2 * ntiles]
    unsigned* offsets = counts + 2 * ntiles;                        // [ntiles]
    unsigned* roffsets = offsets + ntiles;                          // [ntiles]
    unsigned* totals = roffsets + ntiles;                           // [4]
    unsigned* queue = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) + L.trace_counts);
    dim3 tg(ntx, nty);
    k_count<<<tg, 256, 0, s>>>(CountArgs{spp, W, H, ntx, counts});
    k_scan<<<1, 1024, 0, s>>>(ScanArgs{counts, ntiles, offsets, roffsets, totals, stats});
    k_scatter<<<tg, 256, 0, s>>>(ScatterArgs{spp, W, H, ntx, offsets, roffsets, queue, ray_off});
    HDOF_LAUNCHED("hdof_trace: compaction");

    TraceArgs a = trace_args(b, cam, lens, p, st, spp, queue, totals, rt, rec, ray_off);
    static int occ[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !occ[dev]) {
        int nb = 0;
        HDOF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trace, 128, 0), "hdof_trace: occupancy");
        occ[dev] = nb > 0 ? nb : 1;
    }
    int blocks = sm_count() * ((dev >= 0 && dev < 64) ? occ[dev] : 4);
    k_trace<<<blocks, 128, 0, s>>>(a);
    HDOF_LAUNCHED("hdof_trace: trace");
    return HDOF_OK;
}
