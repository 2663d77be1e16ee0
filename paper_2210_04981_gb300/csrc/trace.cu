// compaction of the masked pixels and thin-lens distributed ray
// tracing (Ray Trace section).  Rays originate at random points of the lens
// disk and aim at the pixel's point on the focus plane; each hit is split
// between the near and far layers by its CoC (linear across the focus zone)
// and a hit ratio is kept.
//
// Compaction (deterministic, tile order): k_count counts traced pixels and
// rays per 16x16 tile, k_scan turns the counts into queue and ray offsets,
// k_scatter writes the traced pixels in Z order within each tile and lists
// every ray as (pixel, sample).
//
// Trace: two persistent forms over the ray list, each writing a (hit
// distance, triangle slot) record per ray.  k_trace_packets: a warp takes 32
// consecutive rays and finds their closest hits in one shared traversal
// (narrow lenses: the rays stay close).  k_trace_rays: each lane holds one
// ray and, once fewer than `refill` lanes of the warp are still busy, the
// idle lanes take the next rays with one atomic per warp (dynamic fetch), so
// warps stay full whatever the per-pixel ray counts and traversal lengths.
// k_resolve then shades each pixel's hits and sums them in sample order, so
// the output does not depend on scheduling.
#include "batch.cuh"
#include "internal.h"

namespace hdof {

// default form of a view's trace: warp packets below this CoC scale K =
// A H / (zf tan(fovy/2)) (pixels of CoC per unit of zf/z - 1), ray level with
// refill 4 above
constexpr float PACKET_K_MAX = 20.f;
static bool packet_view(const hdof_lens& l, const hdof_camera& c) {
    const float K = l.aperture_radius * (float)c.height / (l.focus_dist * c.tan_half_fovy);
    return K < PACKET_K_MAX;
}

namespace {

constexpr int TB = 16;  // compaction tile edge

// a pixel traces min(spp, spp_max) rays (the ray lists are sized for spp_max)
struct CountArgs {
    const uint8_t* spp;
    int W, H, ntx, smax;
    unsigned* counts;
};

__device__ __forceinline__ void count_body(const CountArgs& a, int bx, int by) {
    const uint8_t* __restrict__ spp = a.spp;
    const int W = a.W, H = a.H, ntx = a.ntx;
    unsigned* __restrict__ counts = a.counts;
    int i = bx * TB + (threadIdx.x & 15), j = by * TB + (threadIdx.x >> 4);
    unsigned s = (i < W && j < H) ? min((unsigned)spp[(size_t)j * W + i], (unsigned)a.smax) : 0u;
    unsigned px = __syncthreads_count(s > 0);
    __shared__ unsigned red[8];
    unsigned r = s;
    for (int o = 16; o; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int k = 0; k < 8; ++k) t += red[k];
        int tile = by * ntx + bx;
        counts[2 * tile] = px;
        counts[2 * tile + 1] = t;
    }
}

__global__ void __launch_bounds__(256) k_count(CountArgs a) { count_body(a, blockIdx.x, blockIdx.y); }

// one block: exclusive scans of the per-tile pixel and ray counts -> queue
// and ray offsets; totals -> stats.  Each thread takes SCAN_TPT consecutive
// tiles per round (their count pairs in vector loads, a serial prefix), the
// block scans the threads' sums: one round covers 1024 x SCAN_TPT tiles.
struct ScanArgs {
    const unsigned* counts;
    int ntiles;
    unsigned* offsets;
    unsigned* roffsets;
    unsigned* totals;
    unsigned* stats;
};

constexpr int SCAN_TPT = 8;

__device__ __forceinline__ void scan_body(const ScanArgs& a) {
    const unsigned* __restrict__ counts = a.counts;
    const int ntiles = a.ntiles;
    unsigned* __restrict__ offsets = a.offsets;
    unsigned* __restrict__ roffsets = a.roffsets;
    unsigned* __restrict__ totals = a.totals;
    unsigned* __restrict__ stats = a.stats;
    __shared__ unsigned wsum[2][32];
    __shared__ unsigned carry[2];
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // 16-byte vectors when every array allows them (workspace regions do)
    const bool vec = ((reinterpret_cast<uintptr_t>(counts) | reinterpret_cast<uintptr_t>(offsets) |
                       reinterpret_cast<uintptr_t>(roffsets)) & 15) == 0;
    for (int base = 0; base < ntiles; base += 1024 * SCAN_TPT) {
        const int t0 = base + threadIdx.x * SCAN_TPT;
        const bool whole = vec && t0 + SCAN_TPT <= ntiles;
        unsigned c[2 * SCAN_TPT];  // (pixels, rays) of tiles t0 ...
        if (whole) {
            const uint4* p = reinterpret_cast<const uint4*>(counts + 2 * t0);
#pragma unroll
            for (int k = 0; k < SCAN_TPT / 2; ++k) {
                const uint4 u = p[k];
                c[4 * k] = u.x;
                c[4 * k + 1] = u.y;
                c[4 * k + 2] = u.z;
                c[4 * k + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_TPT; ++k) {
                c[2 * k] = t0 + k < ntiles ? counts[2 * (t0 + k)] : 0u;
                c[2 * k + 1] = t0 + k < ntiles ? counts[2 * (t0 + k) + 1] : 0u;
            }
        }
        unsigned v[2] = {0u, 0u};
#pragma unroll
        for (int k = 0; k < SCAN_TPT; ++k) {
            v[0] += c[2 * k];
            v[1] += c[2 * k + 1];
        }
        unsigned x[2] = {v[0], v[1]};
        for (int cc = 0; cc < 2; ++cc)
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, x[cc], o);
                if (lane >= o) x[cc] += y;
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
        unsigned o0[SCAN_TPT], o1[SCAN_TPT];
#pragma unroll
        for (int k = 0; k < SCAN_TPT; ++k) {
            o0[k] = e0;
            o1[k] = e1;
            e0 += c[2 * k];
            e1 += c[2 * k + 1];
        }
        if (whole) {
            uint4* q0 = reinterpret_cast<uint4*>(offsets + t0);
            uint4* q1 = reinterpret_cast<uint4*>(roffsets + t0);
#pragma unroll
            for (int k = 0; k < SCAN_TPT / 4; ++k) {
                q0[k] = make_uint4(o0[4 * k], o0[4 * k + 1], o0[4 * k + 2], o0[4 * k + 3]);
                q1[k] = make_uint4(o1[4 * k], o1[4 * k + 1], o1[4 * k + 2], o1[4 * k + 3]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < SCAN_TPT; ++k)
                if (t0 + k < ntiles) {
                    offsets[t0 + k] = o0[k];
                    roffsets[t0 + k] = o1[k];
                }
        }
        __syncthreads();
        if (threadIdx.x == 1023) {  // its running sums end at the round's totals
            carry[0] = e0;
            carry[1] = e1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = carry[0];  // queue length
        totals[1] = 0;
        totals[2] = carry[1];  // ray count
        totals[3] = 0;         // ray head
        if (stats) {
            stats[0] = carry[0];
            stats[1] = carry[1];
        }
    }
}

__global__ void __launch_bounds__(1024) k_scan(ScanArgs a) { scan_body(a); }

// queue entries in Z (Morton) order within each tile, so four consecutive
// pixels form a 2x2 square and a warp's 32 an 8x4 block (the rays that one
// packet or one warp traces together stay close); optionally the first ray
// of every traced pixel (tile ray offset + prefix of spp in queue order)
struct ScatterArgs {
    const uint8_t* spp;
    int W, H, ntx, smax;
    const unsigned* offsets;
    const unsigned* roffsets;
    unsigned* queue;
    unsigned* qoff;
    unsigned* ray_pix;
    uint8_t* ray_s;
    unsigned* ray_off;
};

__device__ __forceinline__ void scatter_body(const ScatterArgs& a, int bx, int by) {
    const uint8_t* __restrict__ spp = a.spp;
    const int W = a.W, H = a.H, ntx = a.ntx;
    const unsigned* __restrict__ offsets = a.offsets;
    const unsigned* __restrict__ roffsets = a.roffsets;
    unsigned* __restrict__ queue = a.queue;
    unsigned* __restrict__ qoff = a.qoff;
    unsigned* __restrict__ ray_pix = a.ray_pix;
    uint8_t* __restrict__ ray_s = a.ray_s;
    unsigned* __restrict__ ray_off = a.ray_off;
    const int t = threadIdx.x;  // Z-order index: x from the even bits, y from the odd bits
    const int mx = (t & 1) | ((t >> 1) & 2) | ((t >> 2) & 4) | ((t >> 3) & 8);
    const int my = ((t >> 1) & 1) | ((t >> 2) & 2) | ((t >> 3) & 4) | ((t >> 4) & 8);
    int i = bx * TB + mx, j = by * TB + my;
    unsigned n = (i < W && j < H) ? min((unsigned)spp[(size_t)j * W + i], (unsigned)a.smax) : 0u;
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
    const int tile = by * ntx + bx;
    unsigned base = offsets[tile], rbase = roffsets[tile];
    for (int k = 0; k < w; ++k) {
        base += wcnt[k];
        rbase += wray[k];
    }
    const unsigned q = (unsigned)(j * W + i);
    if (on) {
        const unsigned k = base + __popc(m & ((1u << lane) - 1u)), ro = rbase + r - n;
        queue[k] = q;
        qoff[k] = ro;
        if (ray_off) ray_off[q] = ro;
    }
    // the warp's rays are contiguous from rbase: lanes write them together,
    // entry e going to the lane whose inclusive spp prefix first exceeds e
    const unsigned total = __shfl_sync(0xffffffffu, r, 31), first = r - n;
    for (unsigned e0 = 0; e0 < total; e0 += 32) {
        const unsigned e = e0 + lane;
        unsigned owner = 0;  // lanes with prefix <= e
#pragma unroll
        for (unsigned b = 16; b > 0; b >>= 1) {
            const unsigned rt = __shfl_sync(0xffffffffu, r, owner + b - 1);
            if (rt <= e) owner += b;
        }
        const unsigned qo = __shfl_sync(0xffffffffu, q, owner), fo = __shfl_sync(0xffffffffu, first, owner);
        if (e < total) {
            ray_pix[rbase + e] = qo;
            ray_s[rbase + e] = (uint8_t)(e - fo);
        }
    }
}

__global__ void __launch_bounds__(256) k_scatter(ScatterArgs a) { scatter_body(a, blockIdx.x, blockIdx.y); }

struct TraceArgs {
    BvhView bvh;
    Cam cam;
    Coc coc;
    Lights L;
    float A, zf, miss_dist;
    int blades;              // aperture: 0 = disk, N >= 3 = regular N-gon inscribed in it
    float blade_rot;         // polygon rotation (radians)
    float aberration;        // sample weight 1 + aberration (2 rho^2 / A^2 - 1)
    uint2 key;
    int cap, smax;
    int packets;  // the view's default form is warp packets (packet_view)
    unsigned* status;
    const uint8_t* spp;
    const int* hint;   // optional per-pixel original id of the primary hit (< 0: none)
    const unsigned* queue;
    const unsigned* qoff;
    const unsigned* ray_pix;
    const uint8_t* ray_s;
    unsigned* totals;  // [0] queue length, [2] ray count, [3] ray head
    float2* recs;      // per ray (hit distance t, +inf for a miss; sorted triangle slot as int bits)
    float4* rt;        // 3 float4 per pixel
    float4* rec;       // optional per-ray (L rgb, view depth z) records, z = +inf for a miss
    const unsigned* ray_off;
};

// lens sample `smp` of pixel q: origin on the lens aperture (the disk, or
// the regular N-gon: sector k = floor(N u2), f = N u2 - k, point
// sqrt(u1) ((1 - f) V_k + f V_k+1), uniform over the sector's triangle),
// unit direction to the pixel's focus-plane point; *w (may be NULL): the
// sample's weight 1 + aberration (2 rho^2 / A^2 - 1)
__device__ __forceinline__ void lens_ray(const TraceArgs& a, unsigned q, unsigned smp, float3& O, float3& dir,
                                         float* w = nullptr) {
    const int W = a.cam.W;
    const int i = (int)(q % (unsigned)W), j = (int)(q / (unsigned)W);
    const float3 d = pinhole_dir(a.cam, i + 0.5f + a.cam.jx, j + 0.5f + a.cam.jy);
    const float3 Pf = a.cam.pos + a.zf * d;
    uint4 x = philox4x32_10(make_uint4(q, smp, 0u, 0u), a.key);
    float lx, ly;
    if (a.blades >= 3) {
        const float N = (float)a.blades, s = a.A * sqrtf(u01(x.x)), v = u01(x.y) * N;
        const float k = floorf(v), f = v - k;
        float s0, c0, s1, c1;
        sincosf(a.blade_rot + 6.28318530717958648f * k / N, &s0, &c0);
        sincosf(a.blade_rot + 6.28318530717958648f * (k + 1.f) / N, &s1, &c1);
        lx = s * ((1.f - f) * c0 + f * c1);
        ly = s * ((1.f - f) * s0 + f * s1);
    } else {
        float rho = a.A * sqrtf(u01(x.x));
        float sn, cs;
        sincospif(2.f * u01(x.y), &sn, &cs);
        lx = rho * cs;
        ly = rho * sn;
    }
    O = a.cam.pos + lx * a.cam.right + ly * a.cam.up;
    dir = normalize(Pf - O);
    if (w) *w = a.A > 0.f ? 1.f + a.aberration * (2.f * (lx * lx + ly * ly) / (a.A * a.A) - 1.f) : 1.f;
}

// where the rays of the trace come from: one view (the record is the kernel
// parameter) or many (a record table and the views' ray-count prefix)
struct OneView {
    const TraceArgs& a;
    __device__ __forceinline__ const TraceArgs& at(int) const { return a; }
    __device__ __forceinline__ int locate(unsigned g, unsigned& r) const {
        r = g;
        return 0;
    }
};
struct ManyViews {
    const TraceArgs* __restrict__ tab;
    const unsigned* __restrict__ gq;
    int n;
    __device__ __forceinline__ const TraceArgs& at(int v) const { return tab[v]; }
    __device__ __forceinline__ int locate(unsigned g, unsigned& r) const {
        int lo = 0, hi = n - 1;  // last view with gq[v] <= g
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (__ldg(&gq[mid]) <= g) lo = mid;
            else hi = mid - 1;
        }
        r = g - __ldg(&gq[lo]);
        return lo;
    }
};

// Persistent ray-level trace with dynamic fetch and speculative traversal.
// Per lane: one ray's traversal state (same node steps, stack discipline and
// tie rule as closest_hit) plus one postponed leaf.  A lane that reaches a
// leaf parks it and keeps descending; the warp runs node steps until no lane
// is still searching for a leaf, then tests every parked leaf together
// (Aila and Laine's speculative while-while), so the node and leaf code do not
// both run on almost every iteration.  Testing a leaf later than it was
// reached only delays culling: the closest hit is the same.  The fetch is
// warp-uniform: every lane takes part in the ballots; idle lanes are
// predicated off during the steps.
constexpr int DONE_REF = 0x7fffffff;  // stack exhausted
constexpr int NO_LEAF = 0;            // empty leaf slot (leaf references are negative)

// One lane's traversal state in the ray-level trace.
struct RayLane {
    bool live, done;
    int v, cur, leaf, sp, steps;
    unsigned r;
    Ray ray;
    Shear sh;
    Hit h;
};

// Steps of the ray-level trace between two fetches: node phases and leaf
// phases until fewer than `refill` lanes are still live.  OCT >= 0: every
// live lane's ray lies in that direction octant (box tests without per-axis
// min/max, same decisions); rays are fetched only between calls, so it holds
// throughout.
template <int OCT, class Src>
__device__ __forceinline__ void trace_rays_steps(const Src& src, RayLane& L, int (&stack)[HDOF_STACK], int refill) {
    const unsigned FULL = 0xffffffffu;
    const float INF = __int_as_float(0x7f800000);
    while (true) {
        // node phase: descend until no live lane is still looking for a leaf
        while (true) {
            // a lane past the step cap stops stepping (it is finished below)
            const bool can_step = L.live && L.cur >= 0 && L.cur != DONE_REF && L.steps <= src.at(L.v).cap;
            if (can_step) {
                const TraceArgs& a = src.at(L.v);
                const NodeBoxes nb = load_node(a.bvh.nodes + L.cur);
                const int4 ch = nb.ch;
                float t0, t1;
                const bool h0 = slab_hit_oct<OCT>(L.ray, nb.x0, nb.y0, nb.z0, L.h.t, t0);
                const bool h1 = slab_hit_oct<OCT>(L.ray, nb.x1, nb.y1, nb.z1, L.h.t, t1);
                if (h0 && h1) {
                    int nearc = t0 <= t1 ? ch.x : ch.y, farc = t0 <= t1 ? ch.y : ch.x;
                    if (L.sp < HDOF_STACK) stack[L.sp++] = farc;
                    else atomicOr(a.status, HDOF_STATUS_TIMEOUT);
                    L.cur = nearc;
                } else if (h0) {
                    L.cur = ch.x;
                } else if (h1) {
                    L.cur = ch.y;
                } else {
                    L.cur = L.sp ? stack[--L.sp] : DONE_REF;
                }
                if (L.cur < 0 && L.leaf == NO_LEAF) {  // park the leaf, keep descending
                    L.leaf = L.cur;
                    L.cur = L.sp ? stack[--L.sp] : DONE_REF;
                }
                ++L.steps;
            }
            const bool searching = can_step && L.leaf == NO_LEAF && L.cur >= 0 && L.cur != DONE_REF;
            if (!__any_sync(FULL, searching)) break;
        }
        // leaf phase: every parked leaf; a leaf waiting in cur moves into the slot
        if (L.live && L.leaf != NO_LEAF) {
            const TraceArgs& a = src.at(L.v);
            int e = ~L.leaf, first = e >> 3, count = (e & 7) + 1;
            for (int k = 0; k < count; ++k) hit_tri(a.bvh, first + k, L.ray.o, L.sh, L.h);
            L.leaf = NO_LEAF;
            if (L.cur < 0) {
                L.leaf = L.cur;
                L.cur = L.sp ? stack[--L.sp] : DONE_REF;
            }
            ++L.steps;
        }
        if (L.live) {
            const TraceArgs& a = src.at(L.v);
            bool fin = L.leaf == NO_LEAF && L.cur == DONE_REF;
            if (L.steps > a.cap) {
                atomicOr(a.status, HDOF_STATUS_TIMEOUT);
                fin = true;
            }
            if (fin) {
                const BvhView& bvh = a.bvh;
                for (int k = 0; k < bvh.big_count; ++k) {
                    float4 lo = __ldg(&bvh.big_box[2 * k]), hi = __ldg(&bvh.big_box[2 * k + 1]);
                    if (slab(L.ray, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, L.h.t) < INF)
                        hit_tri(bvh, bvh.big_first + k, L.ray.o, L.sh, L.h);
                }
                // shading happens per pixel in the resolve, not here where
                // few lanes of the warp finish at a time
                a.recs[L.r] = make_float2(L.h.slot >= 0 ? L.h.t : INF, __int_as_float(L.h.slot));
                L.live = false;
            }
        }
        if (__popc(__ballot_sync(FULL, L.live)) < refill) break;
    }
}

template <class Src>
__device__ __forceinline__ void trace_rays_body(const Src& src, unsigned total, unsigned* head, int refill,
                                                int chunk) {
    const unsigned FULL = 0xffffffffu;
    const float INF = __int_as_float(0x7f800000);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    RayLane L;
    L.live = L.done = false;
    L.v = L.cur = L.sp = L.steps = 0;
    L.leaf = NO_LEAF;
    L.r = 0;
    int stack[HDOF_STACK];
    // chunk > 0: the warp claims 32 x chunk rays per atomic into a warp-uniform
    // pool and serves its idle lanes from it; chunk 0: exactly the idle lanes'
    // count per atomic.  Which warp traces a ray does not change its hit.
    unsigned pool = 0, pool_end = 0;
    while (true) {
        const unsigned need = __ballot_sync(FULL, !L.live && !L.done);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned base = 0, navail = (unsigned)__popc(need);
            if (chunk <= 0) {
                if (lane == leader) base = atomicAdd(head, navail);
                base = __shfl_sync(FULL, base, leader);
            } else {
                if (pool == pool_end) {
                    unsigned b = 0;
                    if (lane == leader) b = atomicAdd(head, 32u * (unsigned)chunk);
                    b = __shfl_sync(FULL, b, leader);
                    pool = b;
                    pool_end = b + 32u * (unsigned)chunk;
                }
                base = pool;
                navail = min(pool_end - pool, navail);
                pool += navail;
            }
            const unsigned rk = __popc(need & lt);
            if (!L.live && !L.done && rk < navail) {
                const unsigned g = base + rk;
                if (g < total) {
                    L.v = src.locate(g, L.r);
                    const TraceArgs& a = src.at(L.v);
                    const unsigned qp = __ldg(&a.ray_pix[L.r]);
                    float3 O, dir;
                    lens_ray(a, qp, __ldg(&a.ray_s[L.r]), O, dir);
                    L.ray = make_ray(O, dir);
                    L.sh = make_shear(dir);
                    L.h.t = INF;
                    L.h.slot = -1;
                    L.h.id = 0x7fffffff;
                    L.h.b0 = L.h.b1 = L.h.b2 = 0.f;
                    if (a.hint) {
                        // the pixel's primary hit first: a lens ray often hits the same
                        // triangle, and the tight distance culls what lies behind it (the
                        // closest hit, the minimum of (t, id) over all hits, is unchanged)
                        const int id = __ldg(&a.hint[qp]);
                        if (id >= 0 && id < a.bvh.n_tris)
                            hit_tri(a.bvh, __ldg(&a.bvh.slot_of[id]), L.ray.o, L.sh, L.h);
                    }
                    L.cur = a.bvh.root;
                    L.leaf = NO_LEAF;
                    if (L.cur < 0) {  // the whole tree is one leaf
                        L.leaf = L.cur;
                        L.cur = DONE_REF;
                    }
                    L.sp = 0;
                    L.steps = 0;
                    L.live = true;
                } else {
                    L.done = true;
                }
            }
        }
        const unsigned lm = __ballot_sync(FULL, L.live);
        if (!lm) break;
        // the live lanes' common direction octant, if they share one
        const int oct = ray_octant(L.ray);
        const int o0 = __shfl_sync(FULL, oct, __ffs(lm) - 1);
        const int u = __all_sync(FULL, !L.live || oct == o0) ? o0 : -1;
        switch (u) {
            case 0: trace_rays_steps<0>(src, L, stack, refill); break;
            case 1: trace_rays_steps<1>(src, L, stack, refill); break;
            case 2: trace_rays_steps<2>(src, L, stack, refill); break;
            case 3: trace_rays_steps<3>(src, L, stack, refill); break;
            case 4: trace_rays_steps<4>(src, L, stack, refill); break;
            case 5: trace_rays_steps<5>(src, L, stack, refill); break;
            case 6: trace_rays_steps<6>(src, L, stack, refill); break;
            case 7: trace_rays_steps<7>(src, L, stack, refill); break;
            default: trace_rays_steps<-1>(src, L, stack, refill); break;
        }
    }
}

// Packet form of the trace: a warp takes 32 consecutive rays of the list
// (the lens samples of a few neighbouring pixels: nearly the same path
// through the tree) and finds their closest hits in one shared traversal
// (closest_hit_warp); in a batched list the rays of one view go together.
// Same records as the ray-level form.
template <class Src>
__device__ __forceinline__ void trace_packets_body(const Src& src, unsigned total, unsigned* head,
                                                   int chunk) {
    const unsigned FULL = 0xffffffffu;
    const float INF = __int_as_float(0x7f800000);
    const int lane = threadIdx.x & 31;
    const unsigned nc = chunk > 1 ? (unsigned)chunk : 1u;  // packets claimed per atomic
    unsigned base = 0, left = 0;
    while (true) {
        if (!left) {
            if (lane == 0) base = atomicAdd(head, 32u * nc);
            base = __shfl_sync(FULL, base, 0);
            left = nc;
        }
        if (base >= total) break;
        const unsigned g = base + lane;
        base += 32u;
        --left;
        bool pending = g < total;
        unsigned r = 0;
        int v = 0;
        if (pending) v = src.locate(g, r);
        while (true) {
            const unsigned pm = __ballot_sync(FULL, pending);
            if (!pm) break;
            const int v0 = __shfl_sync(FULL, v, __ffs(pm) - 1);
            const bool act = pending && v == v0;
            const TraceArgs& a = src.at(v0);
            Ray ray;
            Shear sh;
            Hit h;
            h.t = INF;
            h.slot = -1;
            h.id = 0x7fffffff;
            h.b0 = h.b1 = h.b2 = 0.f;
            float3 O = f3(0.f, 0.f, 0.f), dir = f3(0.f, 0.f, 1.f);
            if (act) {
                const unsigned qp = __ldg(&a.ray_pix[r]);
                lens_ray(a, qp, __ldg(&a.ray_s[r]), O, dir);
                if (a.hint) {  // the pixel's primary hit first (see trace_rays_body)
                    sh = make_shear(dir);
                    const int id = __ldg(&a.hint[qp]);
                    if (id >= 0 && id < a.bvh.n_tris) hit_tri(a.bvh, __ldg(&a.bvh.slot_of[id]), O, sh, h);
                }
            }
            ray = make_ray(O, dir);
            sh = make_shear(dir);
            closest_hit_warp(a.bvh, act, ray, O, sh, h, a.cap, a.status);
            if (act) {
                const BvhView& bvh = a.bvh;
                for (int k = 0; k < bvh.big_count; ++k) {
                    float4 lo = __ldg(&bvh.big_box[2 * k]), hi = __ldg(&bvh.big_box[2 * k + 1]);
                    if (slab(ray, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, h.t) < INF)
                        hit_tri(bvh, bvh.big_first + k, O, sh, h);
                }
                a.recs[r] = make_float2(h.slot >= 0 ? h.t : INF, __int_as_float(h.slot));
            }
            pending = pending && !act;
        }
    }
}

// register budget for 40 resident warps per SM (measured faster than 36 at 56 registers)
template <int BS>
__global__ void __launch_bounds__(BS, 1280 / BS) k_trace_packets(TraceArgs a, int chunk) {
    trace_packets_body(OneView{a}, __ldcg(&a.totals[2]), &a.totals[3], chunk);
}

template <int BS>
__global__ void __launch_bounds__(BS) k_trace_packets_batch(const TraceArgs* __restrict__ tab,
                                                            const unsigned* __restrict__ gq, int n, unsigned* head,
                                                            int chunk) {
    trace_packets_body(ManyViews{tab, gq, n}, __ldcg(&gq[n]), head, chunk);
}

template <int BS>
__global__ void __launch_bounds__(BS) k_trace_rays(TraceArgs a, int refill, int chunk) {
    trace_rays_body(OneView{a}, __ldcg(&a.totals[2]), &a.totals[3], refill, chunk);
}

template <int BS>
__global__ void __launch_bounds__(BS) k_trace_rays_batch(const TraceArgs* __restrict__ tab,
                                                         const unsigned* __restrict__ gq, int n, unsigned* head,
                                                         int refill, int chunk) {
    trace_rays_body(ManyViews{tab, gq, n}, __ldcg(&gq[n]), head, refill, chunk);
}

// per traced pixel (queue entry k): its samples' records in sample order ->
// shading of each hit (its barycentrics recomputed from the recorded
// triangle) -> near/far layer sums -> the normalised rt record (and the
// adjoint's per-ray (L, z) records when requested)
__device__ __forceinline__ void resolve_body(const TraceArgs& a, int bx) {
    const unsigned k = (unsigned)bx * 256u + threadIdx.x;
    if (k >= __ldcg(&a.totals[0])) return;
    const unsigned q = __ldg(&a.queue[k]), ro = __ldg(&a.qoff[k]);
    const int n = min((int)a.spp[q], a.smax);
    float3 SwL = f3(0, 0, 0), SfL = f3(0, 0, 0), SfP = f3(0, 0, 0);
    float Sw = 0.f, Sf = 0.f, Swc = 0.f, Sfc = 0.f, Ss = 0.f;
    for (int smp = 0; smp < n; ++smp) {
        float3 O, dir;
        float ws;
        lens_ray(a, q, (unsigned)smp, O, dir, &ws);
        const float2 rc = a.recs[ro + smp];
        const int slot = __float_as_int(rc.y);
        const bool hit = slot >= 0;
        float3 L = f3(0.f, 0.f, 0.f);
        float3 P;
        float c;
        if (hit) {
            Hit h;
            h.t = rc.x;
            h.slot = slot;
            const Tri* tr = a.bvh.tris + slot;
            const float4 p0 = __ldg(&tr->v0), p1 = __ldg(&tr->v1), p2 = __ldg(&tr->v2);
            h.id = __float_as_int(p0.w);
            tri_bary(O, make_shear(dir), f3(p0.x, p0.y, p0.z), f3(p1.x, p1.y, p1.z), f3(p2.x, p2.y, p2.z), h.b0, h.b1,
                     h.b2);
            float3 nrm;
            float spec;
            shade(a.bvh, a.L, h, dir, nrm, L, spec);
            P = O + rc.x * dir;
            c = a.coc(dot(P - a.cam.pos, a.cam.fwd));
        } else {
            P = O + a.miss_dist * dir;
            c = a.coc.at_infinity();
        }
        if (a.rec)
            a.rec[ro + smp] = make_float4(L.x, L.y, L.z, hit ? dot(P - a.cam.pos, a.cam.fwd)
                                                             : __int_as_float(0x7f800000));
        // split weight scaled by the sample's aperture weight (1 on the uniform disk)
        float w = ws * w_near(c), wf = ws - w, ac = fabsf(c);
        SwL = SwL + w * L;
        SfL = SfL + wf * L;
        SfP = SfP + wf * P;
        Sw += w;
        Sf += wf;
        Swc += w * ac;
        Sfc += wf * ac;
        Ss += ws;
    }
    bool nok = Sw >= HDOF_EMPTY_W, fok = Sf >= HDOF_EMPTY_W;
    float in = nok ? 1.f / Sw : 0.f, inf_ = fok ? 1.f / Sf : 0.f;
    float4* o = a.rt + 3 * (size_t)q;
    o[0] = make_float4(SwL.x * in, SwL.y * in, SwL.z * in, Sw / Ss);
    o[1] = make_float4(SfL.x * inf_, SfL.y * inf_, SfL.z * inf_, nok ? Swc * in : -1.f);
    o[2] = make_float4(SfP.x * inf_, SfP.y * inf_, SfP.z * inf_, fok ? Sfc * inf_ : -1.f);
}

__global__ void __launch_bounds__(256) k_resolve(TraceArgs a) { resolve_body(a, blockIdx.x); }

// Per-ray closest hits of the last trace on this workspace, in the order of
// its hit records: ids[qoff[k] + s] = original id of sample s of queue entry
// k (-1 for a miss), ts[...] = ray parameter of the hit (+inf for a miss).
struct HitsArgs {
    const Tri* tris;
    const uint8_t* spp;
    const unsigned* queue;
    const unsigned* qoff;
    const unsigned* totals;
    const float2* recs;
    int smax;
    int* ids;
    float* ts;
};
__global__ void __launch_bounds__(256) k_hits(HitsArgs a) {
    const unsigned k = blockIdx.x * 256u + threadIdx.x;
    if (k >= __ldg(&a.totals[0])) return;
    const unsigned q = __ldg(&a.queue[k]), ro = __ldg(&a.qoff[k]);
    const int n = min((int)__ldg(&a.spp[q]), a.smax);
    for (int smp = 0; smp < n; ++smp) {
        const float2 rc = a.recs[ro + smp];
        const int slot = __float_as_int(rc.y);
        a.ids[ro + smp] = slot >= 0 ? __float_as_int(__ldg(&a.tris[slot].v0.w)) : -1;
        if (a.ts) a.ts[ro + smp] = rc.x;
    }
}

TraceArgs trace_args(const hdof_bvh* b, const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p,
                     unsigned* st, const uint8_t* spp, const int* hint, const ViewWs& w, float* rt, float* rec,
                     const unsigned* ray_off) {
    TraceArgs a;
    a.bvh = b->view();
    a.cam = make_cam(*cam);
    a.coc = make_coc(*lens, cam->height, cam->tan_half_fovy);
    a.L = make_lights(*p);
    a.A = lens->aperture_radius;
    a.zf = lens->focus_dist;
    a.miss_dist = p->miss_dist;
    a.blades = p->blades;
    a.blade_rot = p->blade_rot;
    a.aberration = p->aberration;
    a.key = make_uint2(p->seed, (unsigned)p->view * 65536u + (unsigned)p->frame);
    a.cap = p->trav_cap > 0 ? p->trav_cap : 64 * (b->n_nodes + b->n_tris) + 64;
    a.smax = p->spp_max;
    a.packets = packet_view(*lens, *cam) ? 1 : 0;
    a.status = st;
    a.spp = spp;
    a.hint = hint;
    a.queue = w.queue;
    a.qoff = w.qoff;
    a.ray_pix = w.ray_pix;
    a.ray_s = w.ray_s;
    a.totals = w.totals;
    a.recs = w.rec;
    a.rt = reinterpret_cast<float4*>(rt);
    a.rec = reinterpret_cast<float4*>(rec);
    a.ray_off = ray_off;
    return a;
}

// ---- multi-view forms -------------------------------------------------------

__global__ void __launch_bounds__(256) k_count_batch(const CountArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    count_body(batch_record(a, v), bx, by);
}
__global__ void __launch_bounds__(1024) k_scan_batch(const ScanArgs* __restrict__ a) { scan_body(a[blockIdx.x]); }
__global__ void __launch_bounds__(256) k_scatter_batch(const ScatterArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    scatter_body(batch_record(a, v), bx, by);
}
__global__ void __launch_bounds__(256) k_resolve_batch(const TraceArgs* __restrict__ a, BatchGrid g) {
    int v, bx, by;
    g.locate(blockIdx.x, v, bx, by);
    resolve_body(batch_record(a, v), bx);
}

// exclusive prefix of the views' ray counts: gq[v] is the first ray of view
// v in the concatenated ray list, gq[n] the total; gq[n + 1] (the shared
// fetch head) is reset.  cls >= 0: only the views whose default form is
// warp packets (1) or ray level (0) count, the others hold no rays.  One
// block.
__global__ void __launch_bounds__(1024) k_ray_prefix(const ScanArgs* __restrict__ a, const TraceArgs* __restrict__ tab,
                                                     int n, int cls, unsigned* __restrict__ gq) {
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 1024) {
        int v = base + threadIdx.x;
        unsigned c = v < n && (cls < 0 || tab[v].packets == cls) ? __ldcg(&a[v].totals[2]) : 0u, x = c;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned sv = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += y;
            }
            wsum[lane] = sv;
        }
        __syncthreads();
        unsigned e = carry + (w ? wsum[w - 1] : 0u) + x - c;
        if (v < n) gq[v] = e;
        __syncthreads();
        if (threadIdx.x == 1023) carry = e + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        gq[n] = carry;
        gq[n + 1] = 0;
    }
}

template <int BS>
int rays_occupancy(bool batch, bool packets, int* nb) {
    cudaError_t e;
    if (packets)
        e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_trace_packets_batch<BS>, BS, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_trace_packets<BS>, BS, 0);
    else
        e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_trace_rays_batch<BS>, BS, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_trace_rays<BS>, BS, 0);
    if (e != cudaSuccess) return cuda_fail(e, "trace: occupancy");
    if (*nb < 1) *nb = 1;
    return HDOF_OK;
}

// resident grid of the persistent trace (cached per device, form and block size)
int rays_grid(bool batch, bool packets, int block, int* blocks) {
    static int cache[64][2][2][3] = {};
    int dev = 0;
    HDOF_CUDA(cudaGetDevice(&dev), "trace: device");
    const int bi = block == 64 ? 0 : (block == 256 ? 2 : 1);
    int nb = 0, rc = HDOF_OK;
    if (dev >= 0 && dev < 64 && cache[dev][batch][packets][bi]) {
        nb = cache[dev][batch][packets][bi];
    } else {
        if (bi == 0) rc = rays_occupancy<64>(batch, packets, &nb);
        else if (bi == 2) rc = rays_occupancy<256>(batch, packets, &nb);
        else rc = rays_occupancy<128>(batch, packets, &nb);
        if (rc) return rc;
        if (dev >= 0 && dev < 64) cache[dev][batch][packets][bi] = nb;
    }
    *blocks = sm_count() * nb;
    return HDOF_OK;
}

}  // namespace

size_t count_args_size() { return sizeof(CountArgs); }
void count_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TB - 1) / TB;
    *reinterpret_cast<CountArgs*>(dst) = CountArgs{v.spp, W, H, ntx, v.params.spp_max, w.counts};
    *gx = ntx;
    *gy = (H + TB - 1) / TB;
}
void count_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_trace_count", s);
    k_count_batch<<<blocks, 256, 0, s>>>(static_cast<const CountArgs*>(args), g);
}

size_t scan_args_size() { return sizeof(ScanArgs); }
void scan_fill(const hdof_view& v, const ViewWs& w, void* dst) {
    const int ntiles = ((v.cam.width + TB - 1) / TB) * ((v.cam.height + TB - 1) / TB);
    *reinterpret_cast<ScanArgs*>(dst) = ScanArgs{w.counts, ntiles, w.offsets, w.roffsets, w.totals, v.stats};
}
void scan_launch_batch(const void* args, int n, cudaStream_t s) {
    ProfScope ps_("batch_trace_scan", s);
    k_scan_batch<<<n, 1024, 0, s>>>(static_cast<const ScanArgs*>(args));
}

size_t scatter_args_size() { return sizeof(ScatterArgs); }
void scatter_fill(const hdof_view& v, const ViewWs& w, unsigned*, void* dst, int* gx, int* gy) {
    const int W = v.cam.width, H = v.cam.height, ntx = (W + TB - 1) / TB;
    *reinterpret_cast<ScatterArgs*>(dst) =
        ScatterArgs{v.spp, W, H, ntx, v.params.spp_max, w.offsets, w.roffsets, w.queue, w.qoff, w.ray_pix, w.ray_s,
                    nullptr};
    *gx = ntx;
    *gy = (H + TB - 1) / TB;
}
void scatter_launch_batch(const void* args, BatchGrid g, int blocks, cudaStream_t s) {
    ProfScope ps_("batch_trace_scatter", s);
    k_scatter_batch<<<blocks, 256, 0, s>>>(static_cast<const ScatterArgs*>(args), g);
}

size_t trace_args_size() { return sizeof(TraceArgs); }
void trace_fill(const hdof_view& v, const ViewWs& w, unsigned* st, void* dst, int* gx, int* gy) {
    *reinterpret_cast<TraceArgs*>(dst) =
        trace_args(v.bvh, &v.cam, &v.lens, &v.params, st, v.spp, v.g.tri, w, v.rt, nullptr, nullptr);
    *gx = (v.cam.width * v.cam.height + 255) / 256;  // resolve: one thread per possible queue entry
    *gy = 1;
}
int trace_batch_grid(int block, int refill, int* blocks) {
    if (refill == -1) {  // both forms run: the ray-level grid is cached for the launch
        int r = 0, rc = rays_grid(true, false, block, &r);
        if (rc) return rc;
    }
    return rays_grid(true, refill <= 0, block, blocks);
}

int trace_launch_batch(const void* scan_args, const void* trace_args, BatchGrid resolve, int resolve_blocks, int n,
                       unsigned* gq, int block, int refill, int chunk, int blocks, cudaStream_t s) {
    const ScanArgs* sa = static_cast<const ScanArgs*>(scan_args);
    const TraceArgs* a = static_cast<const TraceArgs*>(trace_args);
    if (refill == -1) {
        // each view in its default form: the packet views' rays in one list
        // (prefix gq, head gq[n + 1]), the ray-level views' in another (gq2)
        unsigned* gq2 = gq + n + 2;
        int rblocks = 0, rc = rays_grid(true, false, block, &rblocks);
        if (rc) return rc;
        k_ray_prefix<<<1, 1024, 0, s>>>(sa, a, n, 1, gq);
        k_ray_prefix<<<1, 1024, 0, s>>>(sa, a, n, 0, gq2);
        HDOF_LAUNCHED("batched trace: ray prefixes");
        {
            ProfScope ps_("batch_trace_packets", s);
            if (block == 64) k_trace_packets_batch<64><<<blocks, 64, 0, s>>>(a, gq, n, gq + n + 1, chunk);
            else if (block == 256) k_trace_packets_batch<256><<<blocks, 256, 0, s>>>(a, gq, n, gq + n + 1, chunk);
            else k_trace_packets_batch<128><<<blocks, 128, 0, s>>>(a, gq, n, gq + n + 1, chunk);
            HDOF_LAUNCHED("batched trace: packet views");
        }
        {
            ProfScope ps_("batch_trace_rays", s);
            if (block == 64) k_trace_rays_batch<64><<<rblocks, 64, 0, s>>>(a, gq2, n, gq2 + n + 1, 4, chunk);
            else if (block == 256) k_trace_rays_batch<256><<<rblocks, 256, 0, s>>>(a, gq2, n, gq2 + n + 1, 4, chunk);
            else k_trace_rays_batch<128><<<rblocks, 128, 0, s>>>(a, gq2, n, gq2 + n + 1, 4, chunk);
            HDOF_LAUNCHED("batched trace: ray-level views");
        }
        ProfScope ps_("batch_trace_resolve", s);
        k_resolve_batch<<<resolve_blocks, 256, 0, s>>>(a, resolve);
        HDOF_LAUNCHED("batched trace: resolve");
        return HDOF_OK;
    }
    k_ray_prefix<<<1, 1024, 0, s>>>(sa, a, n, -1, gq);
    HDOF_LAUNCHED("batched trace: ray prefix");
    {
        ProfScope ps_(refill == 0 ? "batch_trace_packets" : "batch_trace_rays", s);
        if (refill == 0) {  // warp packets
            if (block == 64) k_trace_packets_batch<64><<<blocks, 64, 0, s>>>(a, gq, n, gq + n + 1, chunk);
            else if (block == 256) k_trace_packets_batch<256><<<blocks, 256, 0, s>>>(a, gq, n, gq + n + 1, chunk);
            else k_trace_packets_batch<128><<<blocks, 128, 0, s>>>(a, gq, n, gq + n + 1, chunk);
        } else {  // ray level, dynamic fetch
            if (block == 64) k_trace_rays_batch<64><<<blocks, 64, 0, s>>>(a, gq, n, gq + n + 1, refill, chunk);
            else if (block == 256) k_trace_rays_batch<256><<<blocks, 256, 0, s>>>(a, gq, n, gq + n + 1, refill, chunk);
            else k_trace_rays_batch<128><<<blocks, 128, 0, s>>>(a, gq, n, gq + n + 1, refill, chunk);
    }
    HDOF_LAUNCHED("batched trace");
    }
    ProfScope ps_("batch_trace_resolve", s);
    k_resolve_batch<<<resolve_blocks, 256, 0, s>>>(a, resolve);
    HDOF_LAUNCHED("batched trace: resolve");
    return HDOF_OK;
}

}  // namespace hdof

using namespace hdof;

template <int BS>
void launch_trace(const TraceArgs& a, int refill, int chunk, int blocks, cudaStream_t s) {
    if (refill == 0) k_trace_packets<BS><<<blocks, BS, 0, s>>>(a, chunk);
    else k_trace_rays<BS><<<blocks, BS, 0, s>>>(a, refill, chunk);
}

extern "C" int hdof_trace(const hdof_bvh* b, const hdof_camera* cam, const hdof_lens* lens, const hdof_params* p,
                          const uint8_t* spp, const int32_t* hint_tri, float* rt, uint32_t* stats, float* rec,
                          uint32_t* ray_off, void* workspace, size_t workspace_bytes, const hdof_tuning* tune,
                          void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_trace: bvh is NULL");
    int rc;
    if ((rc = check_camera(cam, "hdof_trace")) || (rc = check_lens(lens, "hdof_trace")) ||
        (rc = check_params(p, "hdof_trace")))
        return rc;
    HDOF_CHECK_ARG(spp && rt, "hdof_trace: spp and rt are required");
    HDOF_CHECK_ARG(!rec == !ray_off, "hdof_trace: rec and ray_off go together");
    hdof_tuning t = {};
    if (tune) {
        t = *tune;
        HDOF_CHECK_ARG(t.trace_block == 64 || t.trace_block == 128 || t.trace_block == 256,
                       "hdof_trace: trace_block %d not in {64, 128, 256}", (int)t.trace_block);
        HDOF_CHECK_ARG(t.trace_refill >= -1 && t.trace_refill <= 32, "hdof_trace: trace_refill %d not in -1..32",
                       (int)t.trace_refill);
        HDOF_CHECK_ARG(t.trace_chunk >= 0 && t.trace_chunk <= 16, "hdof_trace: trace_chunk %d not in 0..16",
                       (int)t.trace_chunk);
    } else {
        t.trace_block = 128;
        t.trace_refill = -1;
    }
    if (t.trace_refill == -1) t.trace_refill = packet_view(*lens, *cam) ? 0 : 4;
    const int W = cam->width, H = cam->height;
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.trace, "hdof_trace: workspace of %zu bytes < %zu",
                   workspace_bytes, L.trace);
    unsigned* st = status_ptr();
    HDOF_CHECK_ARG(st, "hdof_trace: no status word on this device");
    cudaStream_t s = as_stream(stream);
    hdof_view v = {};
    v.cam = *cam;
    v.params = *p;
    v.workspace = workspace;
    const ViewWs w = view_ws(v);
    const int ntx = (W + TB - 1) / TB, nty = (H + TB - 1) / TB, ntiles = ntx * nty;
    dim3 tg(ntx, nty);
    {
        ProfScope ps_("trace_compact", s);
        k_count<<<tg, 256, 0, s>>>(CountArgs{spp, W, H, ntx, p->spp_max, w.counts});
        k_scan<<<1, 1024, 0, s>>>(ScanArgs{w.counts, ntiles, w.offsets, w.roffsets, w.totals, stats});
        k_scatter<<<tg, 256, 0, s>>>(
            ScatterArgs{spp, W, H, ntx, p->spp_max, w.offsets, w.roffsets, w.queue, w.qoff, w.ray_pix, w.ray_s, ray_off});
        HDOF_LAUNCHED("hdof_trace: compaction");
    }

    TraceArgs a = trace_args(b, cam, lens, p, st, spp, hint_tri, w, rt, rec, ray_off);
    int blocks = 0;
    if ((rc = rays_grid(false, t.trace_refill == 0, t.trace_block, &blocks))) return rc;
    {
        ProfScope ps_(t.trace_refill == 0 ? "trace_packets" : "trace_rays", s);
        if (t.trace_block == 64) launch_trace<64>(a, t.trace_refill, t.trace_chunk, blocks, s);
        else if (t.trace_block == 256) launch_trace<256>(a, t.trace_refill, t.trace_chunk, blocks, s);
        else launch_trace<128>(a, t.trace_refill, t.trace_chunk, blocks, s);
        HDOF_LAUNCHED("hdof_trace: trace");
    }
    ProfScope ps_("trace_resolve", s);
    k_resolve<<<(W * H + 255) / 256, 256, 0, s>>>(a);
    HDOF_LAUNCHED("hdof_trace: resolve");
    return HDOF_OK;
}

extern "C" int hdof_trace_hits(const hdof_bvh* b, const hdof_camera* cam, const hdof_params* p, const uint8_t* spp,
                               const void* workspace, size_t workspace_bytes, int32_t* ids, float* ts,
                               void* stream) {
    clear_error();
    HDOF_CHECK_ARG(b, "hdof_trace_hits: bvh is NULL");
    int rc;
    if ((rc = check_camera(cam, "hdof_trace_hits")) || (rc = check_params(p, "hdof_trace_hits"))) return rc;
    HDOF_CHECK_ARG(spp && ids, "hdof_trace_hits: spp and ids are required");
    const int W = cam->width, H = cam->height;
    WsLayout L = ws_layout(W, H, p);
    HDOF_CHECK_ARG(workspace && workspace_bytes >= L.trace, "hdof_trace_hits: workspace of %zu bytes < %zu",
                   workspace_bytes, L.trace);
    hdof_view v = {};
    v.cam = *cam;
    v.params = *p;
    v.workspace = const_cast<void*>(workspace);
    const ViewWs w = view_ws(v);
    HitsArgs a{b->tris, spp, w.queue, w.qoff, w.totals, w.rec, p->spp_max, ids, ts};
    k_hits<<<(W * H + 255) / 256, 256, 0, as_stream(stream)>>>(a);
    HDOF_LAUNCHED("hdof_trace_hits");
    return HDOF_OK;
}
