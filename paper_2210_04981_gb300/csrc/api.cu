// C-ABI plumbing: error reporting, status word, argument validation,
// default parameters and workspace sizing.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace hdof {

// device status word: kernels OR in HDOF_STATUS_* bits, hdof_sync reads and clears it;
// words 2..7 hold the traversal counters of analysis builds (HDOF_TRAV_STATS)
__device__ __align__(8) unsigned int g_status[8] = {0, 0, 0, 0, 0, 0, 0, 0};

unsigned* status_ptr() {
    static unsigned* cached[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!cached[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
        cached[dev] = static_cast<unsigned*>(p);
    }
    return cached[dev];
}

static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}
void clear_error() { t_err.clear(); }

int cuda_fail(cudaError_t err, const char* where) {
    set_error("%s: CUDA error %d (%s)", where, (int)err, cudaGetErrorString(err));
    return err == cudaErrorMemoryAllocation ? HDOF_ENOMEM : HDOF_ECUDA;
}

static bool finite3(const float* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_camera(const hdof_camera* c, const char* who) {
    HDOF_CHECK_ARG(c, "%s: camera is NULL", who);
    HDOF_CHECK_ARG(c->width > 0 && c->height > 0 && c->width <= 16384 && c->height <= 16384,
                   "%s: image size %dx%d outside 1..16384", who, c->width, c->height);
    HDOF_CHECK_ARG(finite3(c->pos) && finite3(c->right) && finite3(c->up) && finite3(c->fwd),
                   "%s: camera pose is not finite", who);
    HDOF_CHECK_ARG(std::isfinite(c->tan_half_fovy) && c->tan_half_fovy > 0.f,
                   "%s: tan_half_fovy must be finite and > 0", who);
    HDOF_CHECK_ARG(std::isfinite(c->jitter[0]) && std::isfinite(c->jitter[1]) && std::fabs(c->jitter[0]) <= 1.f &&
                       std::fabs(c->jitter[1]) <= 1.f,
                   "%s: jitter must be finite and within one pixel", who);
    return HDOF_OK;
}

int check_lens(const hdof_lens* l, const char* who) {
    HDOF_CHECK_ARG(l, "%s: lens is NULL", who);
    HDOF_CHECK_ARG(std::isfinite(l->focus_dist) && l->focus_dist > 0.f, "%s: focus_dist must be > 0", who);
    HDOF_CHECK_ARG(std::isfinite(l->aperture_radius) && l->aperture_radius >= 0.f,
                   "%s: aperture_radius must be >= 0", who);
    return HDOF_OK;
}

int check_params(const hdof_params* p, const char* who) {
    HDOF_CHECK_ARG(p, "%s: params is NULL", who);
    HDOF_CHECK_ARG(p->tile >= 1 && p->tile <= 256, "%s: tile must be 1..256", who);
    HDOF_CHECK_ARG(p->dilate >= 0 && p->dilate <= 8, "%s: dilate must be 0..8", who);
    HDOF_CHECK_ARG(p->spp_max >= 1 && p->spp_max <= 255, "%s: spp_max must be 1..255", who);
    HDOF_CHECK_ARG(p->n_lights >= 0 && p->n_lights <= 4, "%s: n_lights must be 0..4", who);
    HDOF_CHECK_ARG(p->gauss_sigma > 0.f && std::isfinite(p->gauss_sigma), "%s: gauss_sigma must be > 0", who);
    HDOF_CHECK_ARG(p->r_max >= 0.f && p->r_max <= 100.f, "%s: r_max must be 0..100", who);
    HDOF_CHECK_ARG(p->r_s >= 0.f && p->r_s <= 64.f, "%s: r_s must be 0..64", who);
    HDOF_CHECK_ARG(p->ema_alpha > 0.f && p->ema_alpha <= 1.f, "%s: ema_alpha must be in (0, 1]", who);
    HDOF_CHECK_ARG(p->kz_rel > 0.f && p->h_tau > 0.f && p->var_ref > 0.f && p->var_scale > 0.f,
                   "%s: kz_rel, h_tau, var_ref and var_scale must be > 0", who);
    HDOF_CHECK_ARG(p->trav_cap >= 0, "%s: trav_cap must be >= 0", who);
    HDOF_CHECK_ARG(p->frame >= 0 && p->frame < 65536 && p->view >= 0 && p->view < 65536,
                   "%s: frame and view must be 0..65535", who);
    HDOF_CHECK_ARG(std::isfinite(p->alpha_k) && p->alpha_k >= 0.f, "%s: alpha_k must be >= 0", who);
    HDOF_CHECK_ARG(p->mask_coc == 0 || p->mask_coc == 1, "%s: mask_coc must be 0 or 1", who);
    HDOF_CHECK_ARG(p->blades == 0 || (p->blades >= 3 && p->blades <= 16), "%s: blades must be 0 or 3..16", who);
    HDOF_CHECK_ARG(std::isfinite(p->blade_rot) && std::isfinite(p->aberration) && p->aberration >= -1.f &&
                       p->aberration <= 1.f,
                   "%s: blade_rot must be finite and aberration in [-1, 1]", who);
    HDOF_CHECK_ARG(std::isfinite(p->spec_pref) && p->spec_pref >= 0.f, "%s: spec_pref must be >= 0", who);
    return HDOF_OK;
}

int check_gbuf(const hdof_gbuf* g, const char* who, bool need_mv) {
    HDOF_CHECK_ARG(g, "%s: gbuf is NULL", who);
    HDOF_CHECK_ARG(g->width > 0 && g->height > 0 && g->width <= 16384 && g->height <= 16384,
                   "%s: gbuf size %dx%d outside 1..16384", who, g->width, g->height);
    HDOF_CHECK_ARG(g->nd && g->col, "%s: gbuf nd/col planes are NULL", who);
    HDOF_CHECK_ARG(g->dtype_nd == HDOF_F32 || g->dtype_nd == HDOF_F16, "%s: dtype_nd must be F32 or F16", who);
    HDOF_CHECK_ARG(g->dtype_col == HDOF_F32 || g->dtype_col == HDOF_BF16, "%s: dtype_col must be F32 or BF16",
                   who);
    HDOF_CHECK_ARG(!need_mv || g->mv, "%s: gbuf mv plane is NULL", who);
    return HDOF_OK;
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

WsLayout ws_layout(int W, int H, const hdof_params* p) {
    WsLayout l;
    size_t npx = (size_t)W * H;
    int T = p ? p->tile : 16;
    size_t mtiles = (size_t)((W + T - 1) / T) * ((H + T - 1) / T);
    size_t ptiles = (size_t)((W + HDOF_TILE_PF - 1) / HDOF_TILE_PF) * ((H + HDOF_TILE_PF - 1) / HDOF_TILE_PF);
    l.mask_tiles = align256(mtiles);
    l.mask_tile_r = align256(mtiles * sizeof(float));
    size_t nray = npx * (size_t)(p ? p->spp_max : 16);
    l.trace_counts = align256(ptiles * 4 * sizeof(unsigned) + 4 * sizeof(unsigned));
    l.trace_queue = align256(npx * sizeof(unsigned));
    l.trace_qoff = align256(npx * sizeof(unsigned));
    l.trace_ray_pix = align256(nray * sizeof(unsigned));
    l.trace_ray_s = align256(nray);
    l.trace_rec = align256(nray * sizeof(float2));
    l.trace = l.trace_counts + l.trace_queue + l.trace_qoff + l.trace_ray_pix + l.trace_ray_s + l.trace_rec;
    l.pf_nrec = align256(npx * sizeof(float4));
    l.pf_frec = align256(npx * sizeof(float4));
    l.pf_rh = align256(npx * sizeof(float));
    l.pf_zq = align256(npx * sizeof(float));
    l.pf_tiles = align256(ptiles * sizeof(float4));
    l.pf_pre = align256(npx * sizeof(float4));
    l.pf_bokeh = bokeh_scratch_bytes(p);
    l.pf = l.pf_nrec + l.pf_frec + l.pf_rh + l.pf_zq + l.pf_tiles + l.pf_pre + l.pf_bokeh;
    const size_t mask = l.mask_tiles + l.mask_tile_r;
    l.pf_off = align256(mask > l.trace ? mask : l.trace);
    l.total = l.pf_off + l.pf;
    return l;
}


}  // namespace hdof

using namespace hdof;

#if HDOF_TRAV_STATS
// analysis builds only: read and clear (rays, node visits, triangle tests)
extern "C" int hdof_debug_trav_stats(unsigned long long* out) {
    unsigned long long z[3] = {0, 0, 0};
    cudaDeviceSynchronize();
    out[3] = 0;
    cudaMemcpyFromSymbol(out, g_status, sizeof z, 8);
    cudaMemcpyToSymbol(g_status, z, sizeof z, 8);
    return 0;
}
#endif

extern "C" {

const char* hdof_version(void) { return "hdof 0.1 (sm_103a)"; }

int hdof_last_error(char* buf, size_t n) {
    if (buf && n) {
        size_t k = t_err.size() < n - 1 ? t_err.size() : n - 1;
        memcpy(buf, t_err.data(), k);
        buf[k] = 0;
    }
    return (int)t_err.size();
}

int hdof_sync(void* stream) {
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "hdof_sync");
    unsigned st = 0, zero = 0;
    HDOF_CUDA(cudaMemcpyFromSymbol(&st, g_status, sizeof st), "hdof_sync: read status");
    if (st) {
        HDOF_CUDA(cudaMemcpyToSymbol(g_status, &zero, sizeof zero), "hdof_sync: clear status");
        set_error("hdof_sync: a kernel watchdog fired (status 0x%x)", st);
        return HDOF_ETIMEOUT;
    }
    return HDOF_OK;
}

void hdof_default_params(hdof_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->gauss_sigma = 1.f;
    p->edge_tau = 0.1f;
    p->tile = 16;
    p->dilate = 1;
    p->spp_max = 16;
    p->variance_on = 0;
    p->var_tau = 0.02f;
    p->var_scale = 0.1f;
    p->hlen_young = 4;
    p->seed = 0;
    p->k_ambient = 0.05f;
    p->n_lights = 1;
    float l[3] = {0.3f, 0.5f, -1.f};
    float n = std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (int k = 0; k < 3; ++k) p->light_dir[0][k] = l[k] / n;
    p->light_E[0] = 1.f;
    p->miss_dist = 1e4f;
    p->trav_cap = 0;
    p->ema_alpha = 0.2f;
    p->camera_moved = 0;
    p->r_s = 16.f;
    p->var_ref = 0.05f;
    p->r_max = 16.f;
    p->kz_rel = 0.05f;
    p->h_tau = 0.25f;
}

size_t hdof_workspace_bytes(int32_t width, int32_t height, const hdof_params* p) {
    if (width <= 0 || height <= 0) return 0;
    return ws_layout(width, height, p).total;
}

}  // extern "C"
