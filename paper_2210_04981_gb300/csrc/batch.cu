// Batched multi-view frame: every stage of the per-frame path runs as one
// launch over the blocks of all views, so a batch of small views fills the
// GPU the way one large view does and the whole frame is a fixed sequence
// of 15 launches that a CUDA graph can capture.
//
// hdof_batch_create writes each stage's per-view launch records (the same
// records the single-view calls pass by value), the per-view block prefix
// and grid widths, into one device allocation owned by the handle.
// hdof_batch_render only launches kernels: no allocation, no host
// synchronisation, no memcpy.
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

struct ZeroRec {
    uint8_t* ptr;
    unsigned long long bytes;
};

// clears each view's mask tile flags (one block per view)
__global__ void __launch_bounds__(256) k_zero_batch(const ZeroRec* __restrict__ r) {
    const ZeroRec z = r[blockIdx.x];
    for (unsigned long long k = threadIdx.x; k < z.bytes; k += blockDim.x) z.ptr[k] = 0;
}

using FillFn = void (*)(const hdof_view&, const ViewWs&, unsigned*, void*, int*, int*);
using LaunchFn = void (*)(const void*, BatchGrid, int, cudaStream_t);
using SizeFn = size_t (*)();

struct StageDef {
    const char* name;
    SizeFn size;
    FillFn fill;
    LaunchFn launch;
};

// per-view records in launch order (the tile clear, the scan and the
// persistent trace are launched between the grid stages by hand)
enum { S_GBUF, S_MASK_EDGE, S_MASK_SPP, S_COUNT, S_SCATTER, S_TRACE, S_PF_PREP, S_PF_ROWSCAN, S_PF_GATHER, S_TEMPORAL,
       S_SPATIAL, S_COMPOSITE, N_STAGES };

const StageDef kStages[N_STAGES] = {
    {"gbuffer", gbuffer_args_size, gbuffer_fill, gbuffer_launch_batch},
    {"mask edge", mask_edge_args_size, mask_edge_fill, mask_edge_launch_batch},
    {"mask spp", mask_spp_args_size, mask_spp_fill, mask_spp_launch_batch},
    {"count", count_args_size, count_fill, count_launch_batch},
    {"scatter", scatter_args_size, scatter_fill, scatter_launch_batch},
    {"trace", trace_args_size, trace_fill, nullptr},  // its grid is the per-pixel resolve
    {"post-filter prep", pf_prep_args_size, pf_prep_fill, pf_prep_launch_batch},
    {"post-filter row prefix", pf_rowscan_args_size, pf_rowscan_fill, pf_rowscan_launch_batch},
    {"post-filter gather", pf_gather_args_size, pf_gather_fill, pf_gather_launch_batch},
    {"temporal", temporal_args_size, temporal_fill, temporal_launch_batch},
    {"spatial", spatial_args_size, spatial_fill, spatial_launch_batch},
    {"composite", composite_args_size, composite_fill, composite_launch_batch},
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool hist_ok(const hdof_history& h) { return h.near_acc && h.far_acc && h.mom && h.hlen; }

int check_view(const hdof_view& v, int k, int dev) {
    char who[64];
    std::snprintf(who, sizeof who, "hdof_batch_create: view %d", k);
    int rc;
    HDOF_CHECK_ARG(v.bvh, "%s: bvh is NULL", who);
    HDOF_CHECK_ARG(v.bvh->device == dev, "%s: bvh lives on device %d, batch on %d", who, v.bvh->device, dev);
    if ((rc = check_camera(&v.cam, who)) || (rc = check_camera(&v.prev, who)) || (rc = check_lens(&v.lens, who)) ||
        (rc = check_params(&v.params, who)) || (rc = check_gbuf(&v.g, who, true)))
        return rc;
    HDOF_CHECK_ARG(v.g.dtype_nd == HDOF_F32 && v.g.dtype_col == HDOF_F32, "%s: batched views use FP32 G-buffers",
                   who);
    if (bokeh_shaped(&v.params)) {
        set_error("%s: shaped bokeh (blades, aberration) is not batched; render such views with the single-view calls",
                  who);
        return HDOF_EUNSUPPORTED;
    }
    if (v.params.spec_pref != 0.f) {
        set_error("%s: the specular-bokeh preference (spec_pref) is not batched; render such views with the "
                  "single-view calls", who);
        return HDOF_EUNSUPPORTED;
    }
    HDOF_CHECK_ARG(v.g.width == v.cam.width && v.g.height == v.cam.height && v.prev.width == v.cam.width &&
                       v.prev.height == v.cam.height,
                   "%s: size mismatch between gbuf and cameras", who);
    HDOF_CHECK_ARG(v.edge && v.spp && v.rt && v.pp && v.crt && v.hacc && v.crec && v.out, "%s: NULL output buffer",
                   who);
    HDOF_CHECK_ARG(hist_ok(v.hist_in) && hist_ok(v.hist_out), "%s: history planes are required", who);
    HDOF_CHECK_ARG(v.hist_in.near_acc != v.hist_out.near_acc && v.hist_in.far_acc != v.hist_out.far_acc &&
                       v.hist_in.mom != v.hist_out.mom && v.hist_in.hlen != v.hist_out.hlen,
                   "%s: hist_in and hist_out must be distinct buffers", who);
    size_t need = ws_layout(v.cam.width, v.cam.height, &v.params).total;
    HDOF_CHECK_ARG(v.workspace && v.workspace_bytes >= need, "%s: workspace of %zu bytes < %zu", who,
                   v.workspace_bytes, need);
    return HDOF_OK;
}

// offsets of the handle's device block: per stage [records][prefix][gx],
// then scan records, tile-clear records, ray prefix
struct Layout {
    size_t args[N_STAGES], prefix[N_STAGES], gx[N_STAGES];
    size_t scan, zero, gq, bytes;
};

Layout layout(int n) {
    Layout L;
    size_t b = 0;
    for (int k = 0; k < N_STAGES; ++k) {
        L.args[k] = b;
        b = align256(b + (size_t)n * kStages[k].size());
        L.prefix[k] = b;
        b = align256(b + (size_t)(n + 1) * sizeof(int));
        L.gx[k] = b;
        b = align256(b + (size_t)n * sizeof(int));
    }
    L.scan = b;
    b = align256(b + (size_t)n * scan_args_size());
    L.zero = b;
    b = align256(b + (size_t)n * sizeof(ZeroRec));
    L.gq = b;
    L.bytes = align256(b + (size_t)(2 * n + 4) * sizeof(unsigned));
    return L;
}

// writes the host image of the device block; blocks[k] = stage k's grid
int fill_image(const hdof_view* views, int n, unsigned* st, const Layout& L, char* img, int* blocks,
               const hdof_tuning& tune) {
    std::memset(img, 0, L.bytes);
    for (int k = 0; k < N_STAGES; ++k) {
        const size_t sz = kStages[k].size();
        int* prefix = reinterpret_cast<int*>(img + L.prefix[k]);
        int* gxs = reinterpret_cast<int*>(img + L.gx[k]);
        long long total = 0;
        for (int v = 0; v < n; ++v) {
            int gx = 0, gy = 0;
            ViewWs w = view_ws(views[v]);
            w.spatial_tile = tune.spatial_tile;
            kStages[k].fill(views[v], w, st, img + L.args[k] + (size_t)v * sz, &gx, &gy);
            prefix[v] = (int)total;
            gxs[v] = gx;
            total += (long long)gx * gy;
        }
        HDOF_CHECK_ARG(total < (1ll << 31), "hdof_batch: %s grid of %lld blocks too large", kStages[k].name, total);
        prefix[n] = (int)total;
        blocks[k] = (int)total;
    }
    for (int v = 0; v < n; ++v) {
        ViewWs w = view_ws(views[v]);
        scan_fill(views[v], w, img + L.scan + (size_t)v * scan_args_size());
        const hdof_params& p = views[v].params;
        ZeroRec z;
        z.ptr = w.tiles;
        z.bytes = (unsigned long long)((views[v].cam.width + p.tile - 1) / p.tile) *
                  (unsigned long long)((views[v].cam.height + p.tile - 1) / p.tile);
        if (p.mask_coc) {  // the per-tile radii follow the flags (and their padding)
            const WsLayout Lv = ws_layout(views[v].cam.width, views[v].cam.height, &p);
            z.bytes = Lv.mask_tiles + z.bytes * sizeof(float);
        }
        std::memcpy(img + L.zero + (size_t)v * sizeof(ZeroRec), &z, sizeof z);
    }
    return HDOF_OK;
}

}  // namespace
}  // namespace hdof

struct hdof_batch {
    int device;
    int n;
    hdof_tuning tuning;
    int trace_blocks;
    void* dmem;
    struct Stage {
        const void* args;
        hdof::BatchGrid grid;
        int blocks;
    } stage[hdof::N_STAGES];
    const void* scan_args;
    const hdof::ZeroRec* zero;
    unsigned* gq;  // [2 n + 4] ray prefix, total, head; with per-view forms a second one for the ray-level views
    hdof::Layout L;
    char* host;              // pinned host image of the records (hdof_batch_update)
    cudaEvent_t uploaded;    // last upload of the host image
    std::vector<int> sizes;  // width, height, mask tile per view (fixed for the handle's life)
    cudaStream_t crit;       // hdof_batch_render's critical path (highest priority)
    cudaStream_t side;       // its post-filter (lowest priority)
    cudaEvent_t start, fork, join, done;  // caller -> crit, crit -> side, side -> crit, crit -> caller
};

using namespace hdof;

extern "C" int hdof_batch_create(const hdof_view* views, int32_t n_views, const hdof_tuning* tuning,
                                 hdof_batch** out, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(out, "hdof_batch_create: out is NULL");
    *out = nullptr;
    HDOF_CHECK_ARG(views && n_views >= 1 && n_views <= 65536, "hdof_batch_create: need 1..65536 views, got %d",
                   (int)n_views);
    hdof_tuning t = {128, -1, 0, 0};  // each view's trace in its default form
    if (tuning) t = *tuning;
    HDOF_CHECK_ARG(t.trace_block == 64 || t.trace_block == 128 || t.trace_block == 256,
                   "hdof_batch_create: trace_block %d not in {64, 128, 256}", (int)t.trace_block);
    HDOF_CHECK_ARG(t.trace_refill >= -1 && t.trace_refill <= 32, "hdof_batch_create: trace_refill %d not in -1..32",
                   (int)t.trace_refill);
    HDOF_CHECK_ARG(t.trace_chunk >= 0 && t.trace_chunk <= 16, "hdof_batch_create: trace_chunk %d not in 0..16",
                   (int)t.trace_chunk);
    HDOF_CHECK_ARG(t.spatial_tile == 0 || t.spatial_tile == 8 || t.spatial_tile == 16,
                   "hdof_batch_create: spatial_tile %d not in {0, 8, 16}", (int)t.spatial_tile);
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "hdof_batch_create: device");
    const int n = n_views;
    for (int k = 0; k < n; ++k) {
        int rc = check_view(views[k], k, dev);
        if (rc) return rc;
    }
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_batch_create: no status word on this device");
    cudaStream_t s = as_stream(stream);
    int rc;
    if ((rc = ensure_area_table(s))) return rc;
    int trace_blocks = 0;
    if ((rc = trace_batch_grid(t.trace_block, t.trace_refill, &trace_blocks))) return rc;

    Layout L = layout(n);
    char* host = nullptr;
    HDOF_CUDA(cudaMallocHost(&host, L.bytes), "hdof_batch_create: host image");
    int blocks[N_STAGES] = {0};
    if ((rc = fill_image(views, n, st, L, host, blocks, t))) {
        cudaFreeHost(host);
        return rc;
    }
    void* dmem = nullptr;
    cudaEvent_t ev = nullptr, evs[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t crit = nullptr, side = nullptr;
    int least = 0, greatest = 0;
    cudaError_t e = cudaMalloc(&dmem, L.bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&evs[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&crit, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmem, host, L.bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        if (dmem) cudaFree(dmem);
        if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t x : evs)
            if (x) cudaEventDestroy(x);
        if (crit) cudaStreamDestroy(crit);
        if (side) cudaStreamDestroy(side);
        cudaFreeHost(host);
        return cuda_fail(e, "hdof_batch_create: upload");
    }
    hdof_batch* b = new hdof_batch;
    b->device = dev;
    b->n = n;
    b->tuning = t;
    b->trace_blocks = trace_blocks;
    b->dmem = dmem;
    char* base = static_cast<char*>(dmem);
    for (int k = 0; k < N_STAGES; ++k) {
        b->stage[k].args = base + L.args[k];
        b->stage[k].grid.prefix = reinterpret_cast<const int*>(base + L.prefix[k]);
        b->stage[k].grid.gx = reinterpret_cast<const int*>(base + L.gx[k]);
        b->stage[k].grid.n = n;
        b->stage[k].blocks = blocks[k];
    }
    b->scan_args = base + L.scan;
    b->zero = reinterpret_cast<const ZeroRec*>(base + L.zero);
    b->gq = reinterpret_cast<unsigned*>(base + L.gq);
    b->L = L;
    b->host = host;
    b->uploaded = ev;
    b->crit = crit;
    b->side = side;
    b->start = evs[0];
    b->fork = evs[1];
    b->join = evs[2];
    b->done = evs[3];
    for (int v = 0; v < n; ++v) {
        b->sizes.push_back(views[v].cam.width);
        b->sizes.push_back(views[v].cam.height);
        b->sizes.push_back(views[v].params.tile);
    }
    *out = b;
    return HDOF_OK;
}

extern "C" int hdof_batch_destroy(hdof_batch* b) {
    clear_error();
    if (!b) return HDOF_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaError_t e = cudaEventSynchronize(b->uploaded);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->crit);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->side);
    cudaEventDestroy(b->uploaded);
    for (cudaEvent_t x : {b->start, b->fork, b->join, b->done}) cudaEventDestroy(x);
    cudaStreamDestroy(b->crit);
    cudaStreamDestroy(b->side);
    cudaError_t e2 = cudaFree(b->dmem);
    if (e == cudaSuccess) e = e2;
    cudaFreeHost(b->host);
    if (cur != b->device) cudaSetDevice(cur);
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "hdof_batch_destroy");
    return HDOF_OK;
}

extern "C" size_t hdof_batch_bytes(const hdof_batch* b) { return b ? b->L.bytes : 0; }

extern "C" int hdof_batch_update(hdof_batch* b, const hdof_view* views, int32_t n_views, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b && views, "hdof_batch_update: NULL argument");
    HDOF_CHECK_ARG(n_views == b->n, "hdof_batch_update: %d views, the batch was created with %d", (int)n_views, b->n);
    int dev = 0, rc;
    HDOF_CUDA(cudaGetDevice(&dev), "hdof_batch_update: device");
    HDOF_CHECK_ARG(dev == b->device, "hdof_batch_update: batch belongs to device %d, current is %d", b->device, dev);
    for (int v = 0; v < b->n; ++v) {
        if ((rc = check_view(views[v], v, dev))) return rc;
        HDOF_CHECK_ARG(views[v].cam.width == b->sizes[3 * v] && views[v].cam.height == b->sizes[3 * v + 1] &&
                           views[v].params.tile == b->sizes[3 * v + 2],
                       "hdof_batch_update: view %d changed its size or mask tile", v);
    }
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_batch_update: no status word on this device");
    // the previous upload may still read the host image
    HDOF_CUDA(cudaEventSynchronize(b->uploaded), "hdof_batch_update: previous upload");
    int blocks[N_STAGES];
    if ((rc = fill_image(views, b->n, st, b->L, b->host, blocks, b->tuning))) return rc;
    cudaStream_t s = as_stream(stream);
    HDOF_CUDA(cudaMemcpyAsync(b->dmem, b->host, b->L.bytes, cudaMemcpyHostToDevice, s), "hdof_batch_update: upload");
    HDOF_CUDA(cudaEventRecord(b->uploaded, s), "hdof_batch_update: event");
    return HDOF_OK;
}

extern "C" int hdof_batch_render_range(const hdof_batch* b, int32_t first, int32_t last, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_batch_render: batch is NULL");
    HDOF_CHECK_ARG(0 <= first && first <= last && last < HDOF_BATCH_STAGES,
                   "hdof_batch_render_range: stages [%d, %d] outside [0, %d]", (int)first, (int)last,
                   HDOF_BATCH_STAGES - 1);
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "hdof_batch_render: device");
    HDOF_CHECK_ARG(dev == b->device, "hdof_batch_render: batch belongs to device %d, current is %d", b->device, dev);
    cudaStream_t s = as_stream(stream);
    auto run = [&](int k) {
        const hdof_batch::Stage& g = b->stage[k];
        kStages[k].launch(g.args, g.grid, g.blocks, s);
    };
    for (int stage = first; stage <= last; ++stage) {
        switch (stage) {
            case HDOF_STAGE_GBUFFER: run(S_GBUF); break;
            case HDOF_STAGE_MASK:
                k_zero_batch<<<b->n, 256, 0, s>>>(b->zero);
                run(S_MASK_EDGE);
                run(S_MASK_SPP);
                break;
            case HDOF_STAGE_COMPACT:
                run(S_COUNT);
                scan_launch_batch(b->scan_args, b->n, s);
                run(S_SCATTER);
                break;
            case HDOF_STAGE_TRACE: {
                const hdof_batch::Stage& t = b->stage[S_TRACE];
                int rc = trace_launch_batch(b->scan_args, t.args, t.grid, t.blocks, b->n, b->gq,
                                            b->tuning.trace_block, b->tuning.trace_refill, b->tuning.trace_chunk,
                                            b->trace_blocks, s);
                if (rc) return rc;
                break;
            }
            case HDOF_STAGE_POSTFILTER:
                run(S_PF_PREP);
                run(S_PF_ROWSCAN);
                run(S_PF_GATHER);
                break;
            case HDOF_STAGE_RECONSTRUCT: {
                run(S_TEMPORAL);
                const hdof_batch::Stage& g = b->stage[S_SPATIAL];
                spatial_launch_batch_tile(g.args, g.grid, g.blocks, b->tuning.spatial_tile, s);
                break;
            }
            default: run(S_COMPOSITE); break;
        }
        HDOF_LAUNCHED("hdof_batch_render");
    }
    return HDOF_OK;
}

// The frame is forked from the caller's stream onto the batch's critical
// path stream (highest priority: its kernels get the SMs first); the
// post-filter needs only the G-buffer and uses its own workspace regions,
// so it runs on the batch's side stream (lowest priority), forked after
// the G-buffer and joined before the composite, concurrently with the mask,
// compaction, trace and reconstruction; the frame is joined back to the
// caller's stream at its end (forks and joins in a captured graph).
extern "C" int hdof_batch_render(const hdof_batch* b, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_batch_render: batch is NULL");
    cudaStream_t s = as_stream(stream), c = b->crit;
    void* cv = static_cast<void*>(c);
    int rc;
    HDOF_CUDA(cudaEventRecord(b->start, s), "hdof_batch_render: fork");
    HDOF_CUDA(cudaStreamWaitEvent(c, b->start, 0), "hdof_batch_render: fork");
    if ((rc = hdof_batch_render_range(b, HDOF_STAGE_GBUFFER, HDOF_STAGE_GBUFFER, cv))) return rc;
    HDOF_CUDA(cudaEventRecord(b->fork, c), "hdof_batch_render: fork");
    HDOF_CUDA(cudaStreamWaitEvent(b->side, b->fork, 0), "hdof_batch_render: fork");
    if ((rc = hdof_batch_render_range(b, HDOF_STAGE_POSTFILTER, HDOF_STAGE_POSTFILTER, b->side))) return rc;
    HDOF_CUDA(cudaEventRecord(b->join, b->side), "hdof_batch_render: join");
    if ((rc = hdof_batch_render_range(b, HDOF_STAGE_MASK, HDOF_STAGE_TRACE, cv))) return rc;
    if ((rc = hdof_batch_render_range(b, HDOF_STAGE_RECONSTRUCT, HDOF_STAGE_RECONSTRUCT, cv))) return rc;
    HDOF_CUDA(cudaStreamWaitEvent(c, b->join, 0), "hdof_batch_render: join");
    if ((rc = hdof_batch_render_range(b, HDOF_STAGE_COMPOSITE, HDOF_STAGE_COMPOSITE, cv))) return rc;
    HDOF_CUDA(cudaEventRecord(b->done, c), "hdof_batch_render: join");
    HDOF_CUDA(cudaStreamWaitEvent(s, b->done, 0), "hdof_batch_render: join");
    return HDOF_OK;
}
