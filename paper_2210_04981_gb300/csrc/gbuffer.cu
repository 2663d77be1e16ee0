// G-buffer and sharp image (Design section: deferred shading yields the
// G-buffer and the sharp rasterised image).  Rasterisation is restated as
// the closest hit of the pinhole ray through each pixel's screen point; the
// primary rays of a warp cover an 8x4 pixel block so they stay coherent.
#include "internal.h"

namespace hdof {
namespace {

// 16x8-pixel blocks; warp w covers the 8x4 sub-block ((w & 1) * 8, (w >> 1) * 4)
__device__ __forceinline__ void pixel_of(int& i, int& j) {
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    i = blockIdx.x * 16 + (w & 1) * 8 + (l & 7);
    j = blockIdx.y * 8 + (w >> 1) * 4 + (l >> 3);
}

template <class ND, class COL>
__global__ void __launch_bounds__(128) k_gbuffer(BvhView bvh, Cam cam, Cam prev, Lights L, float miss_dist, int cap,
                                                 unsigned* status, ND* nd, COL* col, float2* mv, int* tri) {
    int i, j;
    pixel_of(i, j);
    if (i >= cam.W || j >= cam.H) return;
    size_t q = (size_t)j * cam.W + i;
    float3 d = pinhole_dir(cam, i + 0.5f + cam.jx, j + 0.5f + cam.jy);
    float3 dn = normalize(d);
    Hit h = closest_hit(bvh, cam.pos, dn, cap, status);
    float3 n, rad, P;
    float z;
    if (h.slot >= 0) {
        P = cam.pos + h.t * dn;
        z = dot(P - cam.pos, cam.fwd);
        shade(bvh, L, h, dn, n, rad);
    } else {
        z = miss_dist;
        P = cam.pos + z * d;
        n = -1.f * cam.fwd;
        rad = f3(0.f, 0.f, 0.f);
    }
    st4(nd + q, make_float4(n.x, n.y, n.z, z));
    st4(col + q, make_float4(rad.x, rad.y, rad.z, luminance(rad)));
    if (tri) tri[q] = h.id;
    if (mv) {
        float ux, uy;
        mv[q] = project(prev, P, ux, uy) ? make_float2(i - ux, j - uy)
                                         : make_float2(HDOF_MV_OFFSCREEN, HDOF_MV_OFFSCREEN);
    }
}

template <class ND, class COL>
void launch(const hdof_bvh* b, const Cam& cam, const Cam& prev, const Lights& L, float miss, int cap, unsigned* st,
            const hdof_gbuf* g, cudaStream_t s) {
    dim3 grid((cam.W + 15) / 16, (cam.H + 7) / 8);
    k_gbuffer<ND, COL><<<grid, 128, 0, s>>>(b->view(), cam, prev, L, miss, cap, st, static_cast<ND*>(g->nd),
                                            static_cast<COL*>(g->col), reinterpret_cast<float2*>(g->mv), g->tri);
}

}  // namespace
}  // namespace hdof

using namespace hdof;

extern "C" int hdof_gbuffer(const hdof_bvh* b, const hdof_camera* cam, const hdof_camera* prev,
                            const hdof_params* p, const hdof_gbuf* out, void* stream) {
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
    Cam c = make_cam(*cam), pc = make_cam(*prev);
    Lights L = make_lights(*p);
    int cap = p->trav_cap > 0 ? p->trav_cap : 64 * (b->n_nodes + b->n_tris) + 64;
    cudaStream_t s = as_stream(stream);
    if (out->dtype_nd == HDOF_F32 && out->dtype_col == HDOF_F32)
        launch<float4, float4>(b, c, pc, L, p->miss_dist, cap, st, out, s);
    else if (out->dtype_nd == HDOF_F16 && out->dtype_col == HDOF_BF16)
        launch<half4s, bf164s>(b, c, pc, L, p->miss_dist, cap, st, out, s);
    else if (out->dtype_nd == HDOF_F16 && out->dtype_col == HDOF_F32)
        launch<half4s, float4>(b, c, pc, L, p->miss_dist, cap, st, out, s);
    else
        launch<float4, bf164s>(b, c, pc, L, p->miss_dist, cap, st, out, s);
    HDOF_LAUNCHED("hdof_gbuffer");
    return HDOF_OK;
}
