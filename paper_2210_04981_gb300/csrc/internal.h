// Host-side helpers shared by the C-ABI entry points: thread-local error
// message, CUDA error mapping, argument checks and the BVH handle layout.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/hdof.h"
#include "common.cuh"

namespace hdof {

void set_error(const char* fmt, ...);
void clear_error();

// returns HDOF_ECUDA with a message when err != cudaSuccess
int cuda_fail(cudaError_t err, const char* where);

#define HDOF_CHECK_ARG(cond, ...)        \
    do {                                 \
        if (!(cond)) {                   \
            ::hdof::set_error(__VA_ARGS__); \
            return HDOF_EINVAL;          \
        }                                \
    } while (0)

#define HDOF_CUDA(call, where)                                  \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::hdof::cuda_fail(e_, where); \
    } while (0)

#define HDOF_LAUNCHED(where)                                         \
    do {                                                             \
        cudaError_t e_ = cudaGetLastError();                         \
        if (e_ != cudaSuccess) return ::hdof::cuda_fail(e_, where);  \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int check_camera(const hdof_camera* c, const char* who);
int check_lens(const hdof_lens* l, const char* who);
int check_params(const hdof_params* p, const char* who);
int check_gbuf(const hdof_gbuf* g, const char* who, bool need_mv);

// Kernel timing (hdof_profile): a scope records CUDA events on its stream
// around the launches inside it while profiling is on; nothing otherwise.
bool prof_enabled();
struct ProfScope {
    int idx = -1;
    unsigned gen = 0;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t s_);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;
};

// number of SMs of the current device (cached per device)
int sm_count();

// Device address of the status word (kernels OR in HDOF_STATUS_* bits;
// hdof_sync reads and clears it), for the current device.  NULL on error.
unsigned* status_ptr();

// workspace layout (bytes) for a width x height frame
struct WsLayout {
    size_t mask_tiles;      // uint8 per mask tile
    size_t mask_tile_r;     // float per mask tile: largest CoC radius of its pixels (CoC-scaled mask)
    size_t trace_counts;    // uint32 per 16x16 tile: traced pixels, rays; + scan output
    size_t trace_queue;     // uint32 per pixel: traced pixels in queue order
    size_t trace_qoff;      // uint32 per pixel: first ray of each queue entry
    size_t trace_ray_pix;   // uint32 per possible ray (pixels x spp_max): its pixel
    size_t trace_ray_s;     // uint8 per possible ray: its sample index
    size_t trace_rec;       // float2 per possible ray: hit distance, triangle
    size_t trace;           // sum of the trace regions (laid out in this order)
    size_t pf_nrec;         // float4 per pixel: near-layer record
    size_t pf_frec;         // float4 per pixel: far-layer record
    size_t pf_rh;           // float per pixel: r + 1/2
    size_t pf_zq;           // float per pixel: view depth
    size_t pf_tiles;        // float4 per 16x16 tile: largest r near, far; smallest r near
    size_t pf_pre;          // float4 per pixel: row-major inclusive row prefix of the near records
    size_t pf_bokeh;        // shaped bokeh: aperture-norm and lattice-area tables (at the end of the region)
    size_t pf;              // sum of the post-filter regions (laid out in this order)
    size_t pf_off;          // where the post-filter regions start: after the mask and trace regions, so
                            // the post-filter can run concurrently with them
    size_t total;
};
WsLayout ws_layout(int W, int H, const hdof_params* p);

// Lattice-area table of the soft disk (post-filter normalisation), uploaded
// once per device.  Returns HDOF_OK or an error.
int ensure_area_table(cudaStream_t s);
int area_table_size();
// device address of the table ((x, a(x), slope, 0) per breakpoint) and its length
int area_table(const float4** tab, int* n);

// shaped bokeh (blades >= 3 or aberration != 0): the post-filter's own path
bool bokeh_shaped(const hdof_params* p);
size_t bokeh_scratch_bytes(const hdof_params* p);
int launch_bokeh(const hdof_gbuf* in, const Coc& coc, const hdof_params* p, float* pp, void* scratch, cudaStream_t s);

// launches shared by the frame calls and the differentiable post-path (arguments already checked)
int launch_spatial(const float4* crt, const float2* mom, const uint8_t* hlen, int W, int H, float r_s, float var_ref,
                   float4* crec, float4* aux, cudaStream_t s);
// scratch: ws_layout(W, H, p).pf bytes (the post-filter regions)
int launch_postfilter(const hdof_gbuf* in, const Coc& coc, const hdof_params* p, float* pp, float4* aux,
                      void* scratch, cudaStream_t s, const float* lens_dev = nullptr, float t = 0.f);
int launch_composite(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* pp_spec,
                     const float* crt, const float* crec, const float* hacc, const Coc& coc, float h_tau,
                     float spec_pref, float* out, cudaStream_t s, const float* lens_dev = nullptr, float t = 0.f);

}  // namespace hdof

struct hdof_bvh {
    int device;
    int n_tris;
    int n_nodes;  // binary internal nodes
    int n_big;    // scene-sized triangles kept out of the tree (sorted slots at the end)
    int depth;    // deepest leaf of the binary tree
    int root;
    size_t bytes;
    hdof::Node* nodes;
    hdof::Tri* tris;
    float4* mat;
    float2* uv;
    float4* big_box;  // [2 * n_big]
    int* slot_of;     // [n_tris] sorted slot of each original triangle id
    int specular;     // some material has a specular coefficient k_s > 0
    void* pool;  // single allocation holding all of the above
    hdof::BvhView view() const {
        hdof::BvhView v;
        v.nodes = nodes;
        v.tris = tris;
        v.mat = mat;
        v.uv = uv;
        v.n_tris = n_tris;
        v.root = root;
        v.big_first = n_tris - n_big;
        v.big_count = n_big;
        v.big_box = big_box;
        v.slot_of = slot_of;
        v.specular = specular;
        return v;
    }
};
