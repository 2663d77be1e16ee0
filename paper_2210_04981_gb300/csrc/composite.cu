// composite (Composite section).  Pixels in the focus zone (CoC below
// sqrt2) take the sharp rasterised colour; outside it, near geometry takes
// the ray-traced colour and far geometry blends ray-traced and post-process
// colour by the hit ratio, only below a threshold hit ratio so the edges of
// the ray mask do not show.  Near geometry whose post-process colour carries
// a bright specular component leans toward the post-process colour instead
// (its highlight bokeh is smooth there and noisy in the ray trace), by
// clamp(spec_pref S_pp, 0, 1) with S_pp the post-filtered specular
// luminance.  One thread per pixel, float4 planes.
#include "batch.cuh"
#include "internal.h"

namespace hdof {
namespace {

template <class ND, class COL>
struct CompositeArgs {
    const ND* nd;
    const COL* col;
    const uint8_t* spp;
    const float4* pp;
    const float4* pp_spec;  // post-filtered specular luminance in x; NULL: no preference
    const float4* crt;
    const float4* crec;
    const float* hacc;
    int W, H;
    Coc coc;
    float h_tau;
    float spec_pref;
    float4* out;
    const float* lens;  // optional (focus distance, aperture radius) on the device, replacing coc's lens
    float t;            // tan(fovy / 2), with lens
};

template <class ND, class COL>
__device__ __forceinline__ void composite_body(const CompositeArgs<ND, COL>& a, int bx, int by) {
    const ND* __restrict__ nd = a.nd;
    const COL* __restrict__ col = a.col;
    const uint8_t* __restrict__ spp = a.spp;
    const float4* __restrict__ pp = a.pp;
    const float4* __restrict__ crt = a.crt;
    const float4* __restrict__ crec = a.crec;
    const float* __restrict__ hacc = a.hacc;
    const int W = a.W, H = a.H;
    const Coc coc = lens_coc(a.coc, a.lens, H, a.t);
    const float h_tau = a.h_tau;
    float4* __restrict__ out = a.out;
    int i = bx * 32 + (threadIdx.x & 31), j = by * 8 + (threadIdx.x >> 5);
    if (i >= W || j >= H) return;
    size_t q = (size_t)j * W + i;
    float c = coc(ldz(nd + q));
    bool traced = __ldg(&spp[q]) > 0;
    float4 s4 = ld4(col + q);
    float4 p4 = __ldg(&pp[q]);
    float3 sharp = f3(s4.x, s4.y, s4.z), cpp = f3(p4.x, p4.y, p4.z);
    float ce = fabsf(c);
    float3 nearc = cpp, farc = cpp;
    if (traced) {
        ce = __ldg(&crt[q].w);
        float4 r4 = __ldg(&crec[q]);
        float3 rec = f3(r4.x, r4.y, r4.z);
        float b = clamp01(__ldg(&hacc[q]) / h_tau);
        nearc = rec;
        if (a.pp_spec) nearc = rec + clamp01(a.spec_pref * __ldg(&a.pp_spec[q].x)) * (cpp - rec);
        farc = rec + b * (cpp - rec);
    }
    float f = clamp01(HDOF_SQRT2 + 0.5f - ce);
    float wn = w_near(c);
    float3 blur = wn * nearc + (1.f - wn) * farc;
    float3 o = blur + f * (sharp - blur);
    out[q] = make_float4(o.x, o.y, o.z, 0.f);
}

template <class ND, class COL>
__global__ void __launch_bounds__(256) k_composite(CompositeArgs<ND, COL> a) {
    composite_body(a, blockIdx.x, blockIdx.y);
}

using CompositeF32 = CompositeArgs<float4, float4>;
__global__ void __launch_bounds__(256) k_composite_batch(const CompositeF32* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    composite_body(batch_record(a, v), bx, by);
}

template <class ND, class COL>
void launch(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* pp_spec, const float* crt,
            const float* crec, const float* hacc, Coc coc, float h_tau, float spec_pref, float* out, cudaStream_t s,
            const float* lens_dev, float t) {
    dim3 g((in->width + 31) / 32, (in->height + 7) / 8);
    ProfScope ps_("composite", s);
    k_composite<ND, COL><<<g, 256, 0, s>>>(CompositeArgs<ND, COL>{
        static_cast<const ND*>(in->nd), static_cast<const COL*>(in->col), spp, reinterpret_cast<const float4*>(pp),
        reinterpret_cast<const float4*>(pp_spec), reinterpret_cast<const float4*>(crt),
        reinterpret_cast<const float4*>(crec), hacc, in->width, in->height, coc, h_tau, spec_pref,
        reinterpret_cast<float4*>(out), lens_dev, t});
}

}  // namespace

int launch_composite(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* pp_spec,
                     const float* crt, const float* crec, const float* hacc, const Coc& coc, float h_tau,
                     float spec_pref, float* out, cudaStream_t s, const float* lens_dev, float t) {
    if (in->dtype_nd == HDOF_F32 && in->dtype_col == HDOF_F32)
        launch<float4, float4>(in, spp, pp, pp_spec, crt, crec, hacc, coc, h_tau, spec_pref, out, s, lens_dev, t);
    else if (in->dtype_nd == HDOF_F16 && in->dtype_col == HDOF_BF16)
        launch<half4s, bf164s>(in, spp, pp, pp_spec, crt, crec, hacc, coc, h_tau, spec_pref, out, s, lens_dev, t);
    else if (in->dtype_nd == HDOF_F16)
        launch<half4s, float4>(in, spp, pp, pp_spec, crt, crec, hacc, coc, h_tau, spec_pref, out, s, lens_dev, t);
    else
        launch<float4, bf164s>(in, spp, pp, pp_spec, crt, crec, hacc, coc, h_tau, spec_pref, out, s, lens_dev, t);
    HDOF_LAUNCHED("composite");
    return HDOF_OK;
}

}  // namespace hdof

using namespace hdof;

extern "C" int hdof_composite_spec(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* pp_spec,
                                   const float* crt, const float* crec, const float* hacc, const hdof_camera* cam,
                                   const hdof_lens* lens, const hdof_params* p, float* out, void* stream) {
    clear_error();
    int rc;
    if ((rc = check_camera(cam, "hdof_composite")) || (rc = check_lens(lens, "hdof_composite")) ||
        (rc = check_params(p, "hdof_composite")) || (rc = check_gbuf(in, "hdof_composite", false)))
        return rc;
    HDOF_CHECK_ARG(spp && pp && crt && crec && hacc && out, "hdof_composite: NULL buffer");
    HDOF_CHECK_ARG(in->width == cam->width && in->height == cam->height, "hdof_composite: gbuf/camera size mismatch");
    return launch_composite(in, spp, pp, p->spec_pref > 0.f ? pp_spec : nullptr, crt, crec, hacc,
                            make_coc(*lens, cam->height, cam->tan_half_fovy), p->h_tau, p->spec_pref, out,
                            as_stream(stream));
}

extern "C" int hdof_composite(const hdof_gbuf* in, const uint8_t* spp, const float* pp, const float* crt,
                              const float* crec, const float* hacc, const hdof_camera* cam, const hdof_lens* lens,
                              const hdof_params* p, float* out, void* stream) {
    return hdof_composite_spec(in, spp, pp, nullptr, crt, crec, hacc, cam, lens, p, out, stream);
}

namespace hdof {

size_t composite_args_size() { return sizeof(CompositeF32); }
void composite_fill(const hdof_view& v, const ViewWs&, unsigned*, void* dst, int* gx, int* gy) {
    *reinterpret_cast<CompositeF32*>(dst) = CompositeF32{static_cast<const float4*>(v.g.nd),
                                                         static_cast<const float4*>(v.g.col),
                                                         v.spp,
                                                         reinterpret_cast<const float4*>(v.pp),
                                                         nullptr,
                                                         reinterpret_cast<const float4*>(v.crt),
                                                         reinterpret_cast<const float4*>(v.crec),
                                                         v.hacc,
                                                         v.cam.width,
                                                         v.cam.height,
                                                         make_coc(v.lens, v.cam.height, v.cam.tan_half_fovy),
                                                         v.params.h_tau,
                                                         0.f,
                                                         reinterpret_cast<float4*>(v.out)};
    *gx = (v.cam.width + 31) / 32;
    *gy = (v.cam.height + 7) / 8;
}
void composite_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_composite", s);
    k_composite_batch<<<blocks, 256, 0, s>>>(static_cast<const CompositeF32*>(args), g);
}

}  // namespace hdof
