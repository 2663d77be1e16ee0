// Multi-view launches: one grid over the blocks of every view of a batch.
// prefix[v] is the first block of view v (prefix[n] = total); gx[v] is the
// view's grid width in blocks.  A block finds its view by binary search and
// runs the same per-block body as a single-view launch, so every pixel is
// computed by the same code either way.
//
// Each stage file exports three host hooks for the batched frame:
//   <stage>_args_size()              bytes of one view's launch record
//   <stage>_fill(view, ws, st, dst, &gx, &gy)
//                                    writes the view's record at dst and
//                                    its grid (gx x gy blocks)
//   <stage>_launch_batch(args, grid, blocks, stream)
//                                    one launch over all views' blocks
#pragma once

#include "internal.h"

namespace hdof {

struct BatchGrid {
    const int* prefix;
    const int* gx;
    int n;
    __device__ __forceinline__ void locate(int b, int& v, int& bx, int& by) const {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(&prefix[mid]) <= b) lo = mid;
            else hi = mid - 1;
        }
        v = lo;
        int local = b - __ldg(&prefix[lo]), w = __ldg(&gx[lo]);
        bx = local % w;
        by = local / w;
    }
};

// A block's launch record, copied once from the table into shared memory:
// the body then reads it like kernel parameters instead of through a global
// pointer (which, under a tight register bound, the compiler re-loads
// inside hot loops).  Every thread of the block must call it.
template <class T>
__device__ __forceinline__ const T& batch_record(const T* __restrict__ tab, int v) {
    static_assert(sizeof(T) % 4 == 0, "launch records are word-sized");
    __shared__ __align__(16) unsigned s_rec[sizeof(T) / 4];
    const unsigned* src = reinterpret_cast<const unsigned*>(tab + v);
    for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += blockDim.x) s_rec[k] = __ldg(src + k);
    __syncthreads();
    return *reinterpret_cast<const T*>(s_rec);
}

// one view's workspace carved as the single-view calls carve it (the stages
// run one after another, so their regions overlap as they do there)
struct ViewWs {
    uint8_t* tiles;      // mask tile flags
    float* tile_r;       // largest CoC radius per mask tile (CoC-scaled mask)
    int spatial_tile;    // the batch's spatial gather tile (hdof_tuning.spatial_tile), 0 = default
    unsigned* counts;    // [2 * ntiles] traced pixels, rays per 16x16 tile
    unsigned* offsets;   // [ntiles]
    unsigned* roffsets;  // [ntiles]
    unsigned* totals;    // [4] queue length, -, ray count, ray head
    unsigned* queue;     // [W * H] traced pixels
    unsigned* qoff;      // [W * H] first ray of each queue entry
    unsigned* ray_pix;   // [W * H * spp_max] pixel of each ray
    uint8_t* ray_s;      // [W * H * spp_max] sample index of each ray
    float2* rec;         // [W * H * spp_max] (hit distance, triangle) of each ray
    float4* nrec;        // post-filter near-layer record per pixel
    float4* frec;        // post-filter far-layer record per pixel
    float* rh;           // post-filter r + 1/2 per pixel
    float* zq;           // post-filter view depth per pixel
    float4* tmax;        // post-filter per-tile radii (largest near, largest far, smallest near)
    float4* pre;         // post-filter row prefix of the near records (row-major)
};

// the post-filter regions, laid out from `pf` (ws_layout(...).pf bytes)
inline void pf_regions(ViewWs& w, char* pf, const WsLayout& L) {
    size_t f = 0;
    w.nrec = reinterpret_cast<float4*>(pf + f);
    w.frec = reinterpret_cast<float4*>(pf + (f += L.pf_nrec));
    w.rh = reinterpret_cast<float*>(pf + (f += L.pf_frec));
    w.zq = reinterpret_cast<float*>(pf + (f += L.pf_rh));
    w.tmax = reinterpret_cast<float4*>(pf + (f += L.pf_zq));
    w.pre = reinterpret_cast<float4*>(pf + (f += L.pf_tiles));
}

inline ViewWs view_ws(const hdof_view& v) {
    WsLayout L = ws_layout(v.cam.width, v.cam.height, &v.params);
    const int ntx = (v.cam.width + 15) / 16, nty = (v.cam.height + 15) / 16, ntiles = ntx * nty;
    char* base = static_cast<char*>(v.workspace);
    ViewWs w;
    w.tiles = reinterpret_cast<uint8_t*>(base);
    w.tile_r = reinterpret_cast<float*>(base + L.mask_tiles);
    w.spatial_tile = 0;
    w.counts = reinterpret_cast<unsigned*>(base);
    w.offsets = w.counts + 2 * ntiles;
    w.roffsets = w.offsets + ntiles;
    w.totals = w.roffsets + ntiles;
    size_t o = L.trace_counts;
    w.queue = reinterpret_cast<unsigned*>(base + o);
    w.qoff = reinterpret_cast<unsigned*>(base + (o += L.trace_queue));
    w.ray_pix = reinterpret_cast<unsigned*>(base + (o += L.trace_qoff));
    w.ray_s = reinterpret_cast<uint8_t*>(base + (o += L.trace_ray_pix));
    w.rec = reinterpret_cast<float2*>(base + (o += L.trace_ray_s));
    pf_regions(w, base + L.pf_off, L);
    return w;
}

#define HDOF_BATCH_STAGE(name)                                                                             \
    size_t name##_args_size();                                                                             \
    void name##_fill(const hdof_view& v, const ViewWs& w, unsigned* st, void* dst, int* gx, int* gy);      \
    void name##_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s);

HDOF_BATCH_STAGE(gbuffer)
HDOF_BATCH_STAGE(mask_edge)
HDOF_BATCH_STAGE(mask_spp)
HDOF_BATCH_STAGE(count)
HDOF_BATCH_STAGE(scatter)
HDOF_BATCH_STAGE(pf_prep)
HDOF_BATCH_STAGE(pf_rowscan)
HDOF_BATCH_STAGE(pf_gather)
HDOF_BATCH_STAGE(temporal)
HDOF_BATCH_STAGE(spatial)
HDOF_BATCH_STAGE(composite)
#undef HDOF_BATCH_STAGE

// stages that are not one block grid per view
size_t scan_args_size();
void scan_fill(const hdof_view& v, const ViewWs& w, void* dst);
void scan_launch_batch(const void* args, int n, cudaStream_t s);  // one block per view
size_t trace_args_size();
void trace_fill(const hdof_view& v, const ViewWs& w, unsigned* st, void* dst, int* gx, int* gy);
// resident grid of the persistent batched trace for a block size
int trace_batch_grid(int block, int refill, int* blocks);
// ray-count prefix over the views (gq[0..n], gq[n + 1] = head), the
// persistent trace over the concatenated ray lists, and the per-pixel
// resolve (grid of the trace records' gx x gy blocks per view)
int trace_launch_batch(const void* scan_args, const void* trace_args, BatchGrid resolve, int resolve_blocks, int n,
                       unsigned* gq, int block, int refill, int chunk, int blocks, cudaStream_t s);
// the batched spatial gather with a pixel tile of 8 or 16
void spatial_launch_batch_tile(const void* args, BatchGrid g, int blocks, int tile, cudaStream_t s);

}  // namespace hdof
