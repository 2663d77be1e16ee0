// Kernel timing and a measured FP32 arithmetic peak.
//
// Profiling: when switched on (hdof_profile(1)), the stage calls record a
// pair of CUDA events on their stream around each of their kernels; the
// pairs queue up until hdof_profile_read() waits for them and returns the
// per-kernel launch counts and summed device times.  Off by default; when
// off, a launch site costs one flag test.  Events are taken from a pool and
// recycled, so steady-state profiling creates none.
//
// Probe: an FMA-throughput kernel (eight independent chains per thread,
// full occupancy) whose lane-instruction count is known exactly, timed by
// the caller, gives the measured peak rate of FP32 instructions that the
// ALU-bound kernels (traversal, gathers) are compared against.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace hdof {

namespace {

struct Pending {
    const char* name;
    cudaEvent_t a, b;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
unsigned g_gen = 0;  // bumped by every read: scopes opened before it record nothing more
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

bool prof_enabled() { return g_prof_on; }

ProfScope::ProfScope(const char* name, cudaStream_t s_) : s(s_) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t a = take_event();
    if (!a) return;
    if (cudaEventRecord(a, s) != cudaSuccess) {
        g_pool.push_back(a);
        return;
    }
    idx = (int)g_pending.size();
    gen = g_gen;
    g_pending.push_back({name, a, nullptr});
}

ProfScope::~ProfScope() {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (gen != g_gen || idx >= (int)g_pending.size()) return;
    cudaEvent_t b = take_event();
    if (b && cudaEventRecord(b, s) == cudaSuccess) g_pending[idx].b = b;
    else if (b) g_pool.push_back(b);
}

namespace {

// x <- x a + b on eight independent chains, 16 times per loop trip
__global__ void __launch_bounds__(256) k_probe_fma(float a, float b, int iters, float* sink) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
    float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
#pragma unroll 1
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fmaf(x0, a, b);
            x1 = fmaf(x1, a, b);
            x2 = fmaf(x2, a, b);
            x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b);
            x5 = fmaf(x5, a, b);
            x6 = fmaf(x6, a, b);
            x7 = fmaf(x7, a, b);
        }
    }
    const float s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == -1.f) sink[threadIdx.x] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

}  // namespace hdof

using namespace hdof;

extern "C" int hdof_profile(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    // events for the next stretch of launches made up front, so that
    // recording needs no event creation while the stream is being fed
    while (on && g_pool.size() < 2048) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        g_pool.push_back(e);
    }
    return HDOF_OK;
}

extern "C" int hdof_profile_read(hdof_kernel_time* out, int32_t max_out) {
    clear_error();
    std::vector<Pending> done;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        done.swap(g_pending);
        ++g_gen;
    }
    std::vector<hdof_kernel_time> acc;
    int rc = HDOF_OK;
    for (const Pending& p : done) {
        if (p.b) {
            float ms = 0.f;
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "hdof_profile_read");
            } else {
                size_t k = 0;
                while (k < acc.size() && strncmp(acc[k].name, p.name, sizeof acc[k].name) != 0) ++k;
                if (k == acc.size()) {
                    hdof_kernel_time t = {};
                    strncpy(t.name, p.name, sizeof t.name - 1);
                    acc.push_back(t);
                }
                acc[k].launches += 1;
                acc[k].total_ms += ms;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (const Pending& p : done) {
            if (p.a) g_pool.push_back(p.a);
            if (p.b) g_pool.push_back(p.b);
        }
    }
    if (rc) return rc;
    const int n = (int)acc.size();
    if (out)
        for (int k = 0; k < n && k < max_out; ++k) out[k] = acc[k];
    return n;
}

extern "C" int hdof_probe_fma(int32_t blocks_per_sm, int32_t iters, float* sink, double* lane_ops, void* stream) {
    clear_error();
    HDOF_CHECK_ARG(blocks_per_sm >= 1 && blocks_per_sm <= 32, "hdof_probe_fma: blocks_per_sm must be 1..32");
    HDOF_CHECK_ARG(iters >= 1, "hdof_probe_fma: iters must be >= 1");
    HDOF_CHECK_ARG(sink, "hdof_probe_fma: sink is NULL");
    const int blocks = sm_count() * blocks_per_sm;
    k_probe_fma<<<blocks, 256, 0, as_stream(stream)>>>(0.999999f, 1e-7f, iters, sink);
    HDOF_LAUNCHED("hdof_probe_fma");
    if (lane_ops) *lane_ops = (double)blocks * 256.0 * (double)iters * 128.0;
    return HDOF_OK;
}
