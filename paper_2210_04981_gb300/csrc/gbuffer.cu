// G-buffer and sharp image (Design section: deferred shading yields the
// G-buffer and the sharp rasterised image).  Rasterisation is restated as
// the closest hit of the pinhole ray through each pixel's screen point; the
// primary rays of a warp cover an 8x4 pixel block so they stay coherent.
#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

template <class ND, class COL>
struct GbufArgs {
    BvhView bvh;
    Cam cam, prev;
    Lights L;
    float miss_dist;
    int cap;
    unsigned* status;
    ND* nd;
    COL* col;
    float2* mv;
    int* tri;
    const int* hint;  // optional previous primary-hit ids (may alias tri: read before written)
};

// 16x8-pixel blocks; warp w covers the 8x4 sub-block ((w & 1) * 8, (w >> 1) * 4)
// and traces its 32 primary rays as one packet (they are coherent: one node
// fetch serves the warp).  stack: the warp's traversal stack.
template <class ND, class COL>
__device__ __forceinline__ void gbuffer_body(const GbufArgs<ND, COL>& a, int bx, int by) {
    const float INF = __int_as_float(0x7f800000);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int i = bx * 16 + (w & 1) * 8 + (l & 7), j = by * 8 + (w >> 1) * 4 + (l >> 3);
    const Cam& cam = a.cam;
    const bool act = i < cam.W && j < cam.H;
    const size_t q = act ? (size_t)j * cam.W + i : 0;
    float3 d = pinhole_dir(cam, i + 0.5f + cam.jx, j + 0.5f + cam.jy);
    float3 dn = normalize(d);
    const Ray ray = make_ray(cam.pos, dn);
    const Shear sh = make_shear(dn);
    Hit h;
    h.t = INF;
    h.slot = -1;
    h.id = 0x7fffffff;
    h.b0 = h.b1 = h.b2 = 0.f;
    if (act && a.hint) {  // the previous frame's primary hit bounds the search
        const int id = a.hint[q];
        if (id >= 0 && id < a.bvh.n_tris) hit_tri(a.bvh, __ldg(&a.bvh.slot_of[id]), cam.pos, sh, h);
    }
    closest_hit_warp(a.bvh, act, ray, cam.pos, sh, h, a.cap, a.status);
    if (!act) return;
    for (int k = 0; k < a.bvh.big_count; ++k) {
        const float4 lo = __ldg(&a.bvh.big_box[2 * k]), hi = __ldg(&a.bvh.big_box[2 * k + 1]);
        if (slab(ray, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, h.t) < INF)
            hit_tri(a.bvh, a.bvh.big_first + k, cam.pos, sh, h);
    }
    if (h.slot < 0) h.id = -1;
    float3 n, rad, P;
    float z, spec = 0.f;
    if (h.slot >= 0) {
        P = cam.pos + h.t * dn;
        z = dot(P - cam.pos, cam.fwd);
        shade(a.bvh, a.L, h, dn, n, rad, spec);
    } else {
        z = a.miss_dist;
        P = cam.pos + z * d;
        n = -1.f * cam.fwd;
        rad = f3(0.f, 0.f, 0.f);
    }
    st4(a.nd + q, make_float4(n.x, n.y, n.z, z));
    st4(a.col + q, make_float4(rad.x, rad.y, rad.z, spec));
    if (a.tri) a.tri[q] = h.id;
    if (a.mv) {
        float ux, uy;
        a.mv[q] = project(a.prev, P, ux, uy) ? make_float2(i - ux, j - uy)
                                             : make_float2(HDOF_MV_OFFSCREEN, HDOF_MV_OFFSCREEN);
    }
}

// register budget for 10 resident blocks per SM (measured faster than 8 at 64 registers)
template <class ND, class COL>
__global__ void __launch_bounds__(128, 10) k_gbuffer(GbufArgs<ND, COL> a) {
    gbuffer_body(a, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(128) k_gbuffer_batch(const GbufArgs<float4, float4>* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    gbuffer_body(batch_record(a, v), bx, by);
}

template <class ND, class COL>
GbufArgs<ND, COL> gbuf_args(const hdof_bvh* b, const hdof_camera* cam, const hdof_camera* prev, const hdof_params* p,
                            const hdof_gbuf* g, const int* hint, unsigned* st) {
    GbufArgs<ND, COL> a;
    a.bvh = b->view();
    a.cam = make_cam(*cam);
    a.prev = make_cam(*prev);
    a.L = make_lights(*p);
    a.miss_dist = p->miss_dist;
    a.cap = p->trav_cap > 0 ? p->trav_cap : 64 * (b->n_nodes + b->n_tris) + 64;
    a.status = st;
    a.nd = static_cast<ND*>(g->nd);
    a.col = static_cast<COL*>(g->col);
    a.mv = reinterpret_cast<float2*>(g->mv);
    a.tri = g->tri;
    a.hint = hint;
    return a;
}

template <class ND, class COL>
void launch(const hdof_bvh* b, const hdof_camera* cam, const hdof_camera* prev, const hdof_params* p,
            const hdof_gbuf* g, const int* hint, unsigned* st, cudaStream_t s) {
    dim3 grid((cam->width + 15) / 16, (cam->height + 7) / 8);
    ProfScope ps_("gbuffer", s);
    k_gbuffer<ND, COL><<<grid, 128, 0, s>>>(gbuf_args<ND, COL>(b, cam, prev, p, g, hint, st));
}

}  // namespace
}  // namespace hdof

using namespace hdof;

extern "C" int hdof_gbuffer(const hdof_bvh* b, const hdof_camera* cam, const hdof_camera* prev,
                            const hdof_params* p, const int32_t* hint_tri, const hdof_gbuf* out, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_gbuffer: bvh is NULL");
    int rc;
    if ((rc = check_camera(cam, "hdof_gbuffer")) || (rc = check_camera(prev, "hdof_gbuffer: prev")) ||
        (rc = check_params(p, "hdof_gbuffer")) || (rc = check_gbuf(out, "hdof_gbuffer", false)))
        return rc;
    HDOF_CHECK_ARG(out->width == cam->width && out->height == cam->height,
                   "hdof_gbuffer: gbuf %dx%d does not match camera %dx%d", out->width, out->height, cam->width,
                   cam->height);
    HDOF_CHECK_ARG(prev->width == cam->width && prev->height == cam->height,
                   "hdof_gbuffer: previous camera resolution differs");
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_gbuffer: no status word on this device");
    cudaStream_t s = as_stream(stream);
    if (out->dtype_nd == HDOF_F32 && out->dtype_col == HDOF_F32)
        launch<float4, float4>(b, cam, prev, p, out, hint_tri, st, s);
    else if (out->dtype_nd == HDOF_F16 && out->dtype_col == HDOF_BF16)
        launch<half4s, bf164s>(b, cam, prev, p, out, hint_tri, st, s);
    else if (out->dtype_nd == HDOF_F16 && out->dtype_col == HDOF_F32)
        launch<half4s, float4>(b, cam, prev, p, out, hint_tri, st, s);
    else
        launch<float4, bf164s>(b, cam, prev, p, out, hint_tri, st, s);
    HDOF_LAUNCHED("hdof_gbuffer");
    return HDOF_OK;
}

namespace hdof {

size_t gbuffer_args_size() { return sizeof(GbufArgs<float4, float4>); }

void gbuffer_fill(const hdof_view& v, const ViewWs&, unsigned* st, void* dst, int* gx, int* gy) {
    *reinterpret_cast<GbufArgs<float4, float4>*>(dst) =
        gbuf_args<float4, float4>(v.bvh, &v.cam, &v.prev, &v.params, &v.g, v.g.tri, st);
    *gx = (v.cam.width + 15) / 16;
    *gy = (v.cam.height + 7) / 8;
}

void gbuffer_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_gbuffer", s);
    k_gbuffer_batch<<<blocks, 128, 0, s>>>(static_cast<const GbufArgs<float4, float4>*>(args), g);
}

}  // namespace hdof
