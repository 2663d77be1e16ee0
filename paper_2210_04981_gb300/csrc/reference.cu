// Full ray-traced depth of field (the quality reference the paper's Fig. 1
// sets beside the hybrid frame) and per-pixel error maps between frames.
//
// hdof_reference_rt traces every pixel with spp_max lens samples per pass
// through the hybrid frame's own trace (compaction, persistent trace,
// resolve); pass k keys its samples with frame + k, so passes are
// independent.  The trace's per-pixel layers give the pass's mean radiance:
// sum_s L_s / n = h C_near + (1 - h) C_far, with h = sum w / n and the layer
// colours their w- and (1 - w)-weighted means.  The passes' means are
// averaged in pass order.  The per-pass trace output and the all-pixels ray
// count plane live in the post-filter region of the workspace, which the
// trace does not use.
//
// hdof_error_map writes |a - b| averaged over rgb per pixel and reduces, in a
// fixed order (fixed grid, per-block partial sums in double precision, one
// final block), the pixel count, sum of |d|, sum of d^2 (per channel) and
// max |d| over all pixels and over a region.
#include "internal.h"

namespace hdof {
namespace {

constexpr int ERR_BLOCKS = 1024;
constexpr int ERR_THREADS = 256;

__global__ void __launch_bounds__(256) k_fill_u8(uint8_t* __restrict__ a, size_t n, uint8_t v) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        a[k] = v;
}

// out[p] (+)= mean radiance of this pass (h C_near + (1 - h) C_far); the
// last pass divides the sum by the number of passes
__global__ void __launch_bounds__(256) k_rt_accum(const float4* __restrict__ rt, int n_px, float4* __restrict__ out,
                                                  int first, int last, float inv_passes) {
    const int q = blockIdx.x * 256 + threadIdx.x;
    if (q >= n_px) return;
    const float4 a = rt[3 * (size_t)q], b = rt[3 * (size_t)q + 1];
    const float h = a.w;
    float3 m = make_float3(h * a.x + (1.f - h) * b.x, h * a.y + (1.f - h) * b.y, h * a.z + (1.f - h) * b.z);
    float4 o = first ? make_float4(0.f, 0.f, 0.f, 0.f) : out[q];
    o.x += m.x;
    o.y += m.y;
    o.z += m.z;
    if (last) {
        o.x *= inv_passes;
        o.y *= inv_passes;
        o.z *= inv_passes;
        o.w = 0.f;
    }
    out[q] = o;
}

// per pixel: err = mean over rgb of |a - b|; per block: [count, sum |d|,
// sum d^2, max |d|] over all pixels, then the same over the region
__global__ void __launch_bounds__(ERR_THREADS) k_err(const float4* __restrict__ a, const float4* __restrict__ b,
                                                     const uint8_t* __restrict__ region, int n_px,
                                                     float* __restrict__ err, double* __restrict__ part) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = blockIdx.x * ERR_THREADS + threadIdx.x; q < n_px; q += ERR_BLOCKS * ERR_THREADS) {
        const float4 x = a[q], y = b[q];
        const float dx = fabsf(x.x - y.x), dy = fabsf(x.y - y.y), dz = fabsf(x.z - y.z);
        const float e = (dx + dy + dz) * (1.f / 3.f);
        if (err) err[q] = e;
        const double s1 = (double)dx + dy + dz, s2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
        const double mx = fmax(fmax((double)dx, (double)dy), (double)dz);
        acc[0] += 1.0;
        acc[1] += s1;
        acc[2] += s2;
        acc[3] = fmax(acc[3], mx);
        if (region && region[q]) {
            acc[4] += 1.0;
            acc[5] += s1;
            acc[6] += s2;
            acc[7] = fmax(acc[7], mx);
        }
    }
    __shared__ double sh[8][ERR_THREADS];
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = ERR_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 8; ++k) {
                const double o = sh[k][threadIdx.x + w];
                sh[k][threadIdx.x] = (k & 3) == 3 ? fmax(sh[k][threadIdx.x], o) : sh[k][threadIdx.x] + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < 8) part[(size_t)blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// one block: the blocks' partials in block order
__global__ void __launch_bounds__(32) k_err_final(const double* __restrict__ part, double* __restrict__ stats) {
    if (threadIdx.x >= 8) return;
    const int k = threadIdx.x;
    double v = 0.0;
    for (int b = 0; b < ERR_BLOCKS; ++b) {
        const double o = part[(size_t)b * 8 + k];
        v = (k & 3) == 3 ? fmax(v, o) : v + o;
    }
    stats[k] = v;
}

}  // namespace
}  // namespace hdof

using namespace hdof;

extern "C" int hdof_reference_rt(const hdof_bvh* b, const hdof_camera* cam, const hdof_lens* lens,
                                 const hdof_params* p, int32_t passes, const int32_t* hint_tri, float* out,
                                 void* workspace, size_t workspace_bytes, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_reference_rt: bvh is NULL");
    int rc;
    if ((rc = check_camera(cam, "hdof_reference_rt")) || (rc = check_lens(lens, "hdof_reference_rt")) ||
        (rc = check_params(p, "hdof_reference_rt")))
        return rc;
    HDOF_CHECK_ARG(out, "hdof_reference_rt: out is NULL");
    HDOF_CHECK_ARG(passes >= 1 && passes <= 65536, "hdof_reference_rt: passes must be 1..65536");
    const int W = cam->width, H = cam->height;
    const size_t npx = (size_t)W * H;
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.total, "hdof_reference_rt: workspace of %zu bytes < %zu",
                   workspace_bytes, L.total);
    // the post-filter region holds the pass's trace output and the ray-count plane
    char* pf = static_cast<char*>(workspace) + L.pf_off;
    float* rt = reinterpret_cast<float*>(pf);
    uint8_t* spp = reinterpret_cast<uint8_t*>(pf + ((npx * 48 + 255) & ~size_t(255)));
    HDOF_CHECK_ARG(((npx * 48 + 255) & ~size_t(255)) + npx <= L.pf, "hdof_reference_rt: workspace layout");
    cudaStream_t s = as_stream(stream);
    {
        ProfScope ps_("reference_fill", s);
        k_fill_u8<<<sm_count() * 4, 256, 0, s>>>(spp, npx, (uint8_t)p->spp_max);
        HDOF_LAUNCHED("hdof_reference_rt: fill");
    }
    for (int k = 0; k < passes; ++k) {
        hdof_params q = *p;
        q.frame = (int32_t)(((unsigned)p->frame + (unsigned)k) & 0xFFFFu);
        if ((rc = hdof_trace(b, cam, lens, &q, spp, hint_tri, rt, nullptr, nullptr, nullptr, workspace,
                             workspace_bytes, nullptr, stream)))
            return rc;
        ProfScope ps_("reference_accum", s);
        k_rt_accum<<<(unsigned)((npx + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(rt), (int)npx,
                                                                reinterpret_cast<float4*>(out), k == 0,
                                                                k == passes - 1, 1.f / (float)passes);
        HDOF_LAUNCHED("hdof_reference_rt: accumulate");
    }
    return HDOF_OK;
}

extern "C" int hdof_error_map(const float* a, const float* b, const uint8_t* region, int32_t width, int32_t height,
                              float* err, double* stats, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(a && b && stats, "hdof_error_map: a, b and stats are required");
    HDOF_CHECK_ARG(width > 0 && height > 0 && (int64_t)width * height < (1ll << 31),
                   "hdof_error_map: bad size %dx%d", width, height);
    cudaStream_t s = as_stream(stream);
    ProfScope ps_("error_map", s);
    k_err<<<ERR_BLOCKS, ERR_THREADS, 0, s>>>(reinterpret_cast<const float4*>(a), reinterpret_cast<const float4*>(b),
                                            region, width * height, err, stats + HDOF_ERR_STATS);
    HDOF_LAUNCHED("hdof_error_map");
    k_err_final<<<1, 32, 0, s>>>(stats + HDOF_ERR_STATS, stats);
    HDOF_LAUNCHED("hdof_error_map: reduce");
    return HDOF_OK;
}
