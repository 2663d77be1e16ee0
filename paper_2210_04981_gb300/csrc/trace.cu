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
#include "internal.h"

namespace hdof {
namespace {

constexpr int TB = 16;  // compaction tile edge

__global__ void __launch_bounds__(256) k_count(const uint8_t* __restrict__ spp, int W, int H, int ntx,
                                               unsigned* __restrict__ counts) {
    int i = blockIdx.x * TB + (threadIdx.x & 15), j = blockIdx.y * TB + (threadIdx.x >> 4);
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
        int tile = blockIdx.y * ntx + blockIdx.x;
        counts[2 * tile] = px;
        counts[2 * tile + 1] = t;
    }
}

// one block: exclusive scans of the per-tile pixel and ray counts -> queue
// and ray offsets; totals -> stats
__global__ void __launch_bounds__(1024) k_scan(const unsigned* __restrict__ counts, int ntiles,
                                               unsigned* __restrict__ offsets, unsigned* __restrict__ roffsets,
                                               unsigned* __restrict__ totals, unsigned* __restrict__ stats) {
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

// queue entries in row-major order within each tile; optionally the first
// ray of every traced pixel (tile ray offset + prefix of spp in queue order)
__global__ void __launch_bounds__(256) k_scatter(const uint8_t* __restrict__ spp, int W, int H, int ntx,
                                                 const unsigned* __restrict__ offsets,
                                                 const unsigned* __restrict__ roffsets, unsigned* __restrict__ queue,
                                                 unsigned* __restrict__ ray_off) {
    int i = blockIdx.x * TB + (threadIdx.x & 15), j = blockIdx.y * TB + (threadIdx.x >> 4);
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
    const int tile = blockIdx.y * ntx + blockIdx.x;
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

}  // namespace
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
    k_count<<<tg, 256, 0, s>>>(spp, W, H, ntx, counts);
    k_scan<<<1, 1024, 0, s>>>(counts, ntiles, offsets, roffsets, totals, stats);
    k_scatter<<<tg, 256, 0, s>>>(spp, W, H, ntx, offsets, roffsets, queue, ray_off);
    HDOF_LAUNCHED("hdof_trace: compaction");

    TraceArgs a;
    a.bvh = b->view();
    a.cam = make_cam(*cam);
    a.coc = make_coc(*lens, H, cam->tan_half_fovy);
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
