/* FP64 CPU oracle of the hybrid depth-of-field frame.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the library.  It shares no code with
 * the CUDA path.  Each stage follows the paper's design section in its order
 * (Design: G-buffer + post-process; Ray Trace: mask, lens rays, near/far split,
 * hit ratio; Reconstruction: temporal then spatial; Composite).  The paper is
 * prose only; where it is silent the numbered readings documented beside the
 * functions below are used (the same readings the CUDA library implements).
 *
 * Everything is double precision.  Loops are plain and unblocked; the
 * gathers run over their full defining window.
 */
#include "hdof_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SQRT2 1.41421356237309504880
#define PI_D 3.14159265358979323846
#define EMPTY_W 1e-6      /* layer weight below which a layer is empty */
#define HIST_MIN_W 1e-3   /* bilinear history weight below which history is invalid */
#define PP_MIN_W 1e-8     /* post-filter layer weight below which a layer is empty */
#define MV_OFFSCREEN 1e6  /* motion vector written when the previous camera cannot see P */

int32_t orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double* v) {
    double l = sqrt(dot3(v, v));
    v[0] /= l; v[1] /= l; v[2] /= l;
}
static double luminance(const double* c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies on a 4-word
 * counter, Weyl-sequence key schedule.  The lens sample is random per the
 * Ray Trace section; the generator is this reading's choice.
 * ---------------------------------------------------------------------- */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PH_W0; k1 += PH_W1; }
        uint64_t p0 = (uint64_t)PH_M0 * x0, p1 = (uint64_t)PH_M1 * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Second formulation of the same generator: 16-bit limb schoolbook products
 * and a key schedule computed as key + r*W, used only to cross-check the first. */
static void mul32_limbs(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint32_t a0 = a & 0xFFFF, a1 = a >> 16, b0 = b & 0xFFFF, b1 = b >> 16;
    uint32_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint32_t mid = (p00 >> 16) + (p01 & 0xFFFF) + (p10 & 0xFFFF);
    *lo = (p00 & 0xFFFF) | (mid << 16);
    *hi = p11 + (p01 >> 16) + (p10 >> 16) + (mid >> 16);
}
void orc_philox_limb(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    for (uint32_t r = 0; r < 10; ++r) {
        uint32_t k0 = key[0] + r * PH_W0, k1 = key[1] + r * PH_W1;
        uint32_t hi0, lo0, hi1, lo1;
        mul32_limbs(PH_M0, x[0], &hi0, &lo0);
        mul32_limbs(PH_M1, x[2], &hi1, &lo1);
        uint32_t y[4] = {hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0};
        memcpy(x, y, sizeof x);
    }
    memcpy(out, x, sizeof x);
}

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------
 * Thin lens (Potmesil & Chakravarty 1982, cited in the Design section).
 * Signed CoC diameter in pixels of a point at view depth z:
 *   c(z) = A * H * (zf - z) / (z * zf * tan(fovy/2)),  positive = near field.
 * (Sensor-plane CoC 2 A f |z - zf| / (z (zf - f)) divided by the pixel pitch of
 * a sensor at the focused image distance spanning fovy; f cancels.)
 * ---------------------------------------------------------------------- */
double orc_coc(double z, const orc_lens* lens, int32_t height, double t) {
    double A = lens->aperture_radius, zf = lens->focus_dist;
    if (isinf(z)) return -A * height / (zf * t);
    return A * height * (zf - z) / (z * zf * t);
}

/* Pinhole direction through continuous screen point (sx, sy) (pixel (i,j)
 * centre = (i+0.5, j+0.5)); its forward component is 1, so the point at view
 * depth z along it is pos + z*d. */
void orc_pinhole_dir(const orc_camera* c, double sx, double sy, double d[3]) {
    double t = c->tan_half_fovy, a = (double)c->width / c->height;
    double X = (2.0 * sx / c->width - 1.0) * a * t;
    double Y = (1.0 - 2.0 * sy / c->height) * t;
    for (int k = 0; k < 3; ++k) d[k] = X * c->right[k] + Y * c->up[k] + c->fwd[k];
}

/* Inverse of the above, into index space: u = screen point - 0.5 - jitter, so
 * that u = (i, j) is exactly the sample pixel (i, j) took this frame. */
int orc_project(const orc_camera* c, const double P[3], double u[2]) {
    double v[3];
    sub3(P, c->pos, v);
    double zc = dot3(v, c->fwd);
    if (!(zc > 0.0)) return 0;
    double t = c->tan_half_fovy, a = (double)c->width / c->height;
    double X = dot3(v, c->right) / zc, Y = dot3(v, c->up) / zc;
    double sx = (X / (a * t) + 1.0) * 0.5 * c->width;
    double sy = (1.0 - Y / t) * 0.5 * c->height;
    u[0] = sx - 0.5 - c->jitter[0];
    u[1] = sy - 0.5 - c->jitter[1];
    return 1;
}

/* ------------------------------------------------------------------------
 * Scene and closest hit.  The paper uses hardware ray tracing; what it
 * computes is the closest intersection along a ray.  Definition used here:
 * watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013) with edges
 * inclusive; hit requires t > 0; closest = smallest t, equal t -> lower
 * triangle id.  The BVH below (object-median split) only prunes; its result
 * equals the brute-force loop.
 * ---------------------------------------------------------------------- */
typedef struct {
    double lo[3], hi[3];
    int32_t left, right; /* internal: child node ids; leaf: left = first, right = -count */
} onode;

typedef struct {
    int32_t n;
    double* v;     /* [n][9] */
    double* mat;   /* [n][8] */
    double* uv;    /* [n][6] */
    onode* nodes;
    int32_t n_nodes;
    int32_t* order;
} oscene;

int32_t orc_intersect_tri(const double org[3], const double dir[3], const double* v9,
                          double* t, double bary[3]) {
    int kz = 0;
    double ax = fabs(dir[0]), ay = fabs(dir[1]), az = fabs(dir[2]);
    if (ay > ax && ay >= az) kz = 1;
    else if (az > ax && az > ay) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (dir[kz] < 0.0) { int tmp = kx; kx = ky; ky = tmp; }
    double Sx = dir[kx] / dir[kz], Sy = dir[ky] / dir[kz], Sz = 1.0 / dir[kz];
    double A[3], B[3], C[3];
    sub3(v9 + 0, org, A);
    sub3(v9 + 3, org, B);
    sub3(v9 + 6, org, C);
    double Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
    double Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
    double Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double T = U * (Sz * A[kz]) + V * (Sz * B[kz]) + W * (Sz * C[kz]);
    if (det > 0.0 ? !(T > 0.0) : !(T < 0.0)) return 0;
    *t = T / det;
    bary[0] = U / det; bary[1] = V / det; bary[2] = W / det;
    return 1;
}

static double g_sort_axis_key(const oscene* s, int32_t tri, int axis) {
    const double* v = s->v + 9 * (size_t)tri;
    return v[axis] + v[3 + axis] + v[6 + axis];
}

/* Reorder ord[0..n) so that ord[k] holds the element of rank k by centroid
 * (ties by triangle id) with smaller ranks before it and larger after it
 * (quickselect).  Any split serves the oracle's BVH, which only prunes. */
static int key_less(const oscene* s, int axis, int32_t a, int32_t b) {
    double ka = g_sort_axis_key(s, a, axis), kb = g_sort_axis_key(s, b, axis);
    return ka < kb || (ka == kb && a < b);
}
static void select_kth(const oscene* s, int axis, int32_t* ord, int32_t n, int32_t k) {
    int32_t lo = 0, hi = n - 1;
    while (hi > lo) {
        int32_t piv = ord[lo + (hi - lo) / 2];
        int32_t i = lo, j = hi;
        while (i <= j) {
            while (key_less(s, axis, ord[i], piv)) ++i;
            while (key_less(s, axis, piv, ord[j])) --j;
            if (i <= j) {
                int32_t t = ord[i]; ord[i] = ord[j]; ord[j] = t;
                ++i; --j;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return;
    }
}

static int32_t build_node(oscene* s, int32_t first, int32_t count) {
    int32_t id = s->n_nodes++;
    onode* nd = &s->nodes[id];
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    for (int32_t i = first; i < first + count; ++i) {
        const double* v = s->v + 9 * (size_t)s->order[i];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) {
                nd->lo[k] = fmin(nd->lo[k], v[3 * c + k]);
                nd->hi[k] = fmax(nd->hi[k], v[3 * c + k]);
            }
        for (int k = 0; k < 3; ++k) {
            double cen = g_sort_axis_key(s, s->order[i], k);
            clo[k] = fmin(clo[k], cen);
            chi[k] = fmax(chi[k], cen);
        }
    }
    /* conservative padding so the slab test never prunes a box the ray touches */
    for (int k = 0; k < 3; ++k) {
        double pad = 1e-9 * (fabs(nd->lo[k]) + fabs(nd->hi[k]) + 1.0);
        nd->lo[k] -= pad;
        nd->hi[k] += pad;
    }
    if (count <= 4) {
        nd->left = first;
        nd->right = -count;
        return id;
    }
    int axis = 0;
    double ext = chi[0] - clo[0];
    for (int k = 1; k < 3; ++k)
        if (chi[k] - clo[k] > ext) { ext = chi[k] - clo[k]; axis = k; }
    int32_t half = count / 2;
    select_kth(s, axis, s->order + first, count, half);
    int32_t l = build_node(s, first, half);
    int32_t r = build_node(s, first + half, count - half);
    s->nodes[id].left = l;
    s->nodes[id].right = r;
    return id;
}

void* orc_scene_create(int32_t n_tris, const double* tri_v, const double* mat, const double* uv) {
    oscene* s = (oscene*)calloc(1, sizeof(oscene));
    s->n = n_tris;
    s->v = (double*)malloc(sizeof(double) * 9 * (size_t)(n_tris > 0 ? n_tris : 1));
    s->mat = (double*)malloc(sizeof(double) * 8 * (size_t)(n_tris > 0 ? n_tris : 1));
    s->uv = (double*)malloc(sizeof(double) * 6 * (size_t)(n_tris > 0 ? n_tris : 1));
    memcpy(s->v, tri_v, sizeof(double) * 9 * (size_t)n_tris);
    memcpy(s->mat, mat, sizeof(double) * 8 * (size_t)n_tris);
    memcpy(s->uv, uv, sizeof(double) * 6 * (size_t)n_tris);
    s->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int32_t i = 0; i < n_tris; ++i) s->order[i] = i;
    s->nodes = (onode*)malloc(sizeof(onode) * (size_t)(2 * n_tris + 1));
    s->n_nodes = 0;
    if (n_tris > 0) build_node(s, 0, n_tris);
    return s;
}

void orc_scene_destroy(void* p) {
    oscene* s = (oscene*)p;
    if (!s) return;
    free(s->v); free(s->mat); free(s->uv); free(s->order); free(s->nodes);
    free(s);
}

static int slab_hit(const onode* nd, const double* org, const double* dir, double tmax) {
    double tn = 0.0, tf = tmax;
    for (int k = 0; k < 3; ++k) {
        if (dir[k] == 0.0) {
            if (org[k] < nd->lo[k] || org[k] > nd->hi[k]) return 0;
            continue;
        }
        double t0 = (nd->lo[k] - org[k]) / dir[k], t1 = (nd->hi[k] - org[k]) / dir[k];
        if (t0 > t1) { double tmp = t0; t0 = t1; t1 = tmp; }
        t1 *= 1.0 + 1e-9;
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
        if (tn > tf) return 0;
    }
    return 1;
}

static void consider(const oscene* s, int32_t tri, const double* org, const double* dir,
                     int32_t* best, double* bt, double* bb) {
    double t, b[3];
    if (!orc_intersect_tri(org, dir, s->v + 9 * (size_t)tri, &t, b)) return;
    if (t < *bt || (t == *bt && tri < *best)) {
        *bt = t; *best = tri;
        bb[0] = b[0]; bb[1] = b[1]; bb[2] = b[2];
    }
}

int32_t orc_closest_hit(const void* sp, const double org[3], const double dir[3], int32_t use_bvh,
                        double* t, double bary[3]) {
    const oscene* s = (const oscene*)sp;
    int32_t best = -1;
    double bt = INFINITY, bb[3] = {0, 0, 0};
    if (!use_bvh || s->n_nodes == 0) {
        for (int32_t i = 0; i < s->n; ++i) consider(s, i, org, dir, &best, &bt, bb);
    } else {
        int32_t stack[256];
        int sp_ = 0;
        stack[sp_++] = 0;
        while (sp_ > 0) {
            const onode* nd = &s->nodes[stack[--sp_]];
            if (!slab_hit(nd, org, dir, bt)) continue;
            if (nd->right <= 0) {
                for (int32_t k = 0; k < -nd->right; ++k)
                    consider(s, s->order[nd->left + k], org, dir, &best, &bt, bb);
            } else {
                stack[sp_++] = nd->left;
                stack[sp_++] = nd->right;
            }
        }
    }
    *t = bt;
    bary[0] = bb[0]; bary[1] = bb[1]; bary[2] = bb[2];
    return best;
}

void orc_closest_hits(const void* s, int32_t n, const double* org, const double* dir,
                      int32_t use_bvh, int32_t* ids, double* ts) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t i = 0; i < n; ++i) {
        double b[3];
        ids[i] = orc_closest_hit(s, org + 3 * (size_t)i, dir + 3 * (size_t)i, use_bvh, &ts[i], b);
    }
}

/* Shading of a hit (the paper's deferred shading; directional lights, no
 * shadows):
 *   L = albedo * (k_a + sum_l E_l max(0, n . w_l)) + S (1, 1, 1),
 *   S = k_s sum_{l: n . w_l > 0} E_l max(0, n . h_l)^32,  h_l = unit(w_l - dir),
 * n = geometric face normal turned to face the ray; albedo from the triangle's
 * material, a checkerboard of n x n cells over its (u,v) when checker_n > 0;
 * S is a white Blinn-Phong highlight (material k_s = mat[7]; the workloads'
 * materials are Lambertian, k_s = 0, S = 0), returned in *spec when asked.
 * dir is the unit direction of the ray that found the hit. */
static void shade_hit(const oscene* s, int32_t tri, const double* bary, const double* dir,
                      const orc_params* p, double n_out[3], double L[3], double* spec) {
    const double* v = s->v + 9 * (size_t)tri;
    double e1[3], e2[3], n[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, n);
    normalize3(n);
    if (dot3(n, dir) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
    const double* m = s->mat + 8 * (size_t)tri;
    const double* uv = s->uv + 6 * (size_t)tri;
    const double* alb = m;
    if (m[3] > 0.0) {
        double uu = bary[0] * uv[0] + bary[1] * uv[2] + bary[2] * uv[4];
        double vv = bary[0] * uv[1] + bary[1] * uv[3] + bary[2] * uv[5];
        long long cell = (long long)floor(m[3] * uu) + (long long)floor(m[3] * vv);
        if (cell & 1) alb = m + 4;
    }
    double irr = p->k_ambient;
    for (int l = 0; l < p->n_lights; ++l) irr += p->light_E[l] * fmax(0.0, dot3(n, p->light_dir[l]));
    double S = 0.0;
    if (m[7] > 0.0) {
        for (int l = 0; l < p->n_lights; ++l) {
            if (dot3(n, p->light_dir[l]) <= 0.0) continue;
            double h[3];
            sub3(p->light_dir[l], dir, h);
            normalize3(h);
            S += p->light_E[l] * pow(fmax(0.0, dot3(n, h)), 32.0);
        }
        S *= m[7];
    }
    for (int k = 0; k < 3; ++k) { L[k] = alb[k] * irr + S; n_out[k] = n[k]; }
    if (spec) *spec = S;
}

/* ------------------------------------------------------------------------
 * G-buffer (Design: deferred shading produces the G-buffer and the sharp
 * image).  Rasterisation is restated as the closest hit of the pinhole ray
 * through each pixel's sample point (i + 0.5 + jx, j + 0.5 + jy).
 * nd = (n, view depth z), col = (L, S) with S the specular part of L,
 * tri = hit id (-1 = miss).
 * mv = (i, j) - previous-frame index-space position of the hit point.
 * Misses: z = miss_dist, n = -fwd, L = 0.
 * ---------------------------------------------------------------------- */
void orc_gbuffer(const void* sp, const orc_camera* cam, const orc_camera* prev, const orc_params* p,
                 double* nd, double* col, double* mv, int32_t* tri) {
    const oscene* s = (const oscene*)sp;
    int32_t W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j) {
        for (int32_t i = 0; i < W; ++i) {
            size_t pix = (size_t)j * W + i;
            double d[3], dn[3];
            orc_pinhole_dir(cam, i + 0.5 + cam->jitter[0], j + 0.5 + cam->jitter[1], d);
            memcpy(dn, d, sizeof dn);
            normalize3(dn);
            double t, bary[3], n[3], L[3], P[3], S = 0.0;
            int32_t id = orc_closest_hit(s, cam->pos, dn, 1, &t, bary);
            double z;
            if (id >= 0) {
                for (int k = 0; k < 3; ++k) P[k] = cam->pos[k] + t * dn[k];
                double v[3];
                sub3(P, cam->pos, v);
                z = dot3(v, cam->fwd);
                shade_hit(s, id, bary, dn, p, n, L, &S);
            } else {
                z = p->miss_dist;
                for (int k = 0; k < 3; ++k) {
                    P[k] = cam->pos[k] + z * d[k];
                    n[k] = -cam->fwd[k];
                    L[k] = 0.0;
                }
            }
            nd[4 * pix + 0] = n[0]; nd[4 * pix + 1] = n[1]; nd[4 * pix + 2] = n[2];
            nd[4 * pix + 3] = z;
            col[4 * pix + 0] = L[0]; col[4 * pix + 1] = L[1]; col[4 * pix + 2] = L[2];
            col[4 * pix + 3] = S;
            tri[pix] = id;
            double u[2];
            if (orc_project(prev, P, u)) {
                mv[2 * pix + 0] = i - u[0];
                mv[2 * pix + 1] = j - u[1];
            } else {
                mv[2 * pix + 0] = MV_OFFSCREEN;
                mv[2 * pix + 1] = MV_OFFSCREEN;
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * Adaptive ray mask (Ray Trace section): Gaussian filter on the G-buffer,
 * Sobel gradient of normal and depth, threshold -> edge bits; tiled and
 * dilated; plus the temporally accumulated luminance variance term.
 * ---------------------------------------------------------------------- */
void orc_gaussian_weights(double sigma, double w[5]) {
    double s = 0.0;
    for (int k = -2; k <= 2; ++k) { w[k + 2] = exp(-(double)(k * k) / (2.0 * sigma * sigma)); s += w[k + 2]; }
    for (int k = 0; k < 5; ++k) w[k] /= s;
}

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* lens, t: the CoC-scaled mask (p->mask_coc = 1; the Discussion's mask resolution scaled by the CoC):
 * an edge tile reaches max(dilate, ceil(r / tile)) tiles (Chebyshev distance, at most 8), r = the
 * largest min(|c(z)| / 2, r_max) over its pixels; lens = NULL: every edge tile reaches `dilate` tiles. */
static void mask_impl(int32_t W, int32_t H, const double* nd, const double* mv, const double* hist_mom,
                      const uint8_t* hist_hlen, const orc_params* p, const orc_lens* lens, double t, uint8_t* edge,
                      uint8_t* spp, double* emetric) {
    size_t N = (size_t)W * H;
    double g[5];
    orc_gaussian_weights(p->gauss_sigma, g);
    double* f = (double*)malloc(sizeof(double) * 4 * N); /* Gaussian-filtered (nx,ny,nz,z) */
    /* 5x5 Gaussian (outer product of the 1-D weights), clamp-to-edge */
#pragma omp parallel for
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i)
            for (int c = 0; c < 4; ++c) {
                double acc = 0.0;
                for (int b = -2; b <= 2; ++b)
                    for (int a = -2; a <= 2; ++a) {
                        size_t q = (size_t)clampi(j + b, 0, H - 1) * W + clampi(i + a, 0, W - 1);
                        acc += g[a + 2] * g[b + 2] * nd[4 * q + c];
                    }
                f[4 * ((size_t)j * W + i) + c] = acc;
            }
    /* 3x3 Sobel scaled by 1/8 (a ramp of slope s gives gradient s), clamp-to-edge;
     * edge metric e = max(|grad n|, |grad z| / z~); edge bit = e > tau */
    static const double kw[3] = {1.0, 2.0, 1.0};
#pragma omp parallel for
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            double gx[4], gy[4];
            for (int c = 0; c < 4; ++c) {
                double sx = 0.0, sy = 0.0;
                for (int k = -1; k <= 1; ++k) {
                    size_t qr = (size_t)clampi(j + k, 0, H - 1) * W + clampi(i + 1, 0, W - 1);
                    size_t ql = (size_t)clampi(j + k, 0, H - 1) * W + clampi(i - 1, 0, W - 1);
                    size_t qd = (size_t)clampi(j + 1, 0, H - 1) * W + clampi(i + k, 0, W - 1);
                    size_t qu = (size_t)clampi(j - 1, 0, H - 1) * W + clampi(i + k, 0, W - 1);
                    sx += kw[k + 1] * (f[4 * qr + c] - f[4 * ql + c]);
                    sy += kw[k + 1] * (f[4 * qd + c] - f[4 * qu + c]);
                }
                gx[c] = sx / 8.0;
                gy[c] = sy / 8.0;
            }
            double en = sqrt(gx[0] * gx[0] + gy[0] * gy[0] + gx[1] * gx[1] + gy[1] * gy[1] +
                             gx[2] * gx[2] + gy[2] * gy[2]);
            double ez = sqrt(gx[3] * gx[3] + gy[3] * gy[3]) / f[4 * ((size_t)j * W + i) + 3];
            double e = en > ez ? en : ez;
            size_t pix = (size_t)j * W + i;
            if (emetric) emetric[pix] = e;
            edge[pix] = e > p->edge_tau ? 1 : 0;
        }
    /* tile OR; each edge tile's reach in tiles (fixed `dilate`, or from its pixels' largest CoC radius) */
    int32_t T = p->tile, ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    uint8_t* ton = (uint8_t*)calloc((size_t)ntx * nty, 1);
    int* reach = (int*)malloc(sizeof(int) * (size_t)ntx * nty);
    double* rt_ = (double*)calloc((size_t)ntx * nty, sizeof(double));
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t k = (size_t)(j / T) * ntx + i / T;
            if (edge[(size_t)j * W + i]) ton[k] = 1;
            if (lens && p->mask_coc) {
                double r = fmin(fabs(orc_coc(nd[4 * ((size_t)j * W + i) + 3], lens, H, t)) * 0.5, p->r_max);
                if (r > rt_[k]) rt_[k] = r;
            }
        }
    for (size_t k = 0; k < (size_t)ntx * nty; ++k) {
        int rc = p->dilate;
        if (lens && p->mask_coc) {
            int c = (int)ceil(rt_[k] / T);
            if (c > rc) rc = c;
            if (rc > 8) rc = 8;
        }
        reach[k] = rc;
    }
    int dmax = (lens && p->mask_coc) ? 8 : p->dilate;
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t pix = (size_t)j * W + i;
            int tx = i / T, ty = j / T, on = 0;
            for (int b = -dmax; b <= dmax && !on; ++b)
                for (int a = -dmax; a <= dmax; ++a) {
                    int x = tx + a, y = ty + b;
                    if (x < 0 || y < 0 || x >= ntx || y >= nty) continue;
                    size_t k = (size_t)y * ntx + x;
                    int cheb = abs(a) > abs(b) ? abs(a) : abs(b);
                    if (ton[k] && cheb <= reach[k]) { on = 1; break; }
                }
            int s = on ? p->spp_max : 0;
            if (!on && p->variance_on && hist_hlen && hist_mom) {
                /* previous frame's moments at the reprojected position (nearest pixel) */
                double ux = i - mv[2 * pix], uy = j - mv[2 * pix + 1];
                double fx = floor(ux + 0.5), fy = floor(uy + 0.5);
                int hl = 0;
                double m1 = 0.0, m2 = 0.0;
                if (fx >= 0.0 && fy >= 0.0 && fx < W && fy < H) {
                    size_t q = (size_t)fy * W + (size_t)fx;
                    hl = hist_hlen[q];
                    m1 = hist_mom[2 * q];
                    m2 = hist_mom[2 * q + 1];
                }
                double sig = sqrt(fmax(0.0, m2 - m1 * m1));
                int young = hl < p->hlen_young;
                if (hl >= 1 && (young || sig > p->var_tau)) {
                    if (young) s = p->spp_max;
                    else {
                        double c = ceil(p->spp_max * sig / p->var_scale);
                        s = (int)clampd(c, 1.0, (double)p->spp_max);
                    }
                }
            }
            spp[pix] = (uint8_t)s;
        }
    free(ton);
    free(reach);
    free(rt_);
    free(f);
}

void orc_mask(int32_t W, int32_t H, const double* nd, const double* mv, const double* hist_mom,
              const uint8_t* hist_hlen, const orc_params* p, uint8_t* edge, uint8_t* spp, double* emetric) {
    mask_impl(W, H, nd, mv, hist_mom, hist_hlen, p, NULL, 0.0, edge, spp, emetric);
}

void orc_mask_coc(int32_t W, int32_t H, const double* nd, const double* mv, const double* hist_mom,
                  const uint8_t* hist_hlen, const orc_params* p, const orc_lens* lens, double tan_half_fovy,
                  uint8_t* edge, uint8_t* spp, double* emetric) {
    mask_impl(W, H, nd, mv, hist_mom, hist_hlen, p, lens, tan_half_fovy, edge, spp, emetric);
}

/* ------------------------------------------------------------------------
 * Thin-lens distributed ray trace of the masked pixels (Ray Trace section).
 * Per sample s of pixel p: Philox(key = (seed, view*65536 + frame),
 * ctr = (p, s, 0, 0)) -> u1, u2; lens point rho = A sqrt(u1), theta = 2 pi u2
 * in the (right, up) plane; aim at the focus-plane point of the pixel's
 * pinhole ray; closest hit; Lambert radiance.  The split weight into the near
 * layer is linear across the focus zone |c| < sqrt2:
 *   w = clamp((c(z) + sqrt2) / (2 sqrt2), 0, 1).
 * Misses are far (c = c(inf), P = lens point + miss_dist * dir, L = 0).
 * Output rt[12] = (C_near rgb, h | C_far rgb, c_near | P_far xyz, c_far) with
 * h = sum w / n (hit ratio); empty layers (weight < 1e-6) give colour 0 and
 * CoC -1.
 * ---------------------------------------------------------------------- */
/* Aperture shape and sample weights (Discussion: alternative bokeh shapes
 * by the shape of the sampling kernel, spherical aberration by the relative
 * weight of its samples).  blades = 0: the disk of radius A; blades = N >= 3:
 * the regular N-gon inscribed in it, vertices at angles blade_rot + 2 pi k / N
 * in the (right, up) plane.  Its norm: D(v) = |v| / g(phi), g(phi) =
 * cos(pi/N) / cos(((phi - blade_rot) mod 2pi/N) - pi/N), so the aperture is
 * {D(v) <= A}.  A sample at lens-plane radius rho weighs
 * 1 + aberration (2 rho^2 / A^2 - 1) (mean 1 over the disk). */
static double aperture_norm(double vx, double vy, const orc_params* p) {
    double d = sqrt(vx * vx + vy * vy);
    if (p->blades < 3 || d == 0.0) return d;
    double sect = 2.0 * PI_D / p->blades;
    double m = fmod(atan2(vy, vx) - p->blade_rot, sect);
    if (m < 0.0) m += sect;
    return d * cos(m - PI_D / p->blades) / cos(PI_D / p->blades);
}
static double aperture_weight(double t, const orc_params* p) { return 1.0 + p->aberration * (2.0 * t * t - 1.0); }

/* Lens sample `smp` of pixel q (Ray Trace section: rays through random
 * points of the lens aperture, aimed at the pixel's point on the focus
 * plane): Philox(key = (seed, view*65536 + frame), ctr = (q, smp, 0, 0)) ->
 * u1, u2; on the disk, lens point rho = A sqrt(u1), theta = 2 pi u2 in the
 * (right, up) plane; on the N-gon, sector k = floor(N u2) and f = N u2 - k,
 * point sqrt(u1) ((1 - f) V_k + f V_k+1) (uniform over the sector's
 * triangle); unit direction towards the focus-plane point of the pixel's
 * pinhole ray; *weight (may be NULL) = the sample's weight. */
void orc_lens_ray(const orc_camera* cam, const orc_lens* lens, const orc_params* p, int64_t q, int32_t smp,
                  double O[3], double dir[3], double* weight) {
    int32_t W = cam->width, i = (int32_t)(q % W), j = (int32_t)(q / W);
    double A = lens->aperture_radius, zf = lens->focus_dist;
    uint32_t key[2] = {p->seed, (uint32_t)p->view * 65536u + (uint32_t)p->frame};
    double d[3], Pf[3];
    orc_pinhole_dir(cam, i + 0.5 + cam->jitter[0], j + 0.5 + cam->jitter[1], d);
    for (int k = 0; k < 3; ++k) Pf[k] = cam->pos[k] + zf * d[k];
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)smp, 0u, 0u}, x[4];
    orc_philox(ctr, key, x);
    double lx, ly;
    if (p->blades >= 3) {
        double N = p->blades, s_ = sqrt(u01(x[0])), v = u01(x[1]) * N;
        double k = floor(v), f = v - k;
        double t0 = p->blade_rot + 2.0 * PI_D * k / N, t1 = p->blade_rot + 2.0 * PI_D * (k + 1.0) / N;
        lx = A * s_ * ((1.0 - f) * cos(t0) + f * cos(t1));
        ly = A * s_ * ((1.0 - f) * sin(t0) + f * sin(t1));
    } else {
        double rho = A * sqrt(u01(x[0])), th = 2.0 * PI_D * u01(x[1]);
        lx = rho * cos(th);
        ly = rho * sin(th);
    }
    for (int k = 0; k < 3; ++k) O[k] = cam->pos[k] + lx * cam->right[k] + ly * cam->up[k];
    sub3(Pf, O, dir);
    normalize3(dir);
    if (weight) *weight = A > 0.0 ? aperture_weight(sqrt(lx * lx + ly * ly) / A, p) : 1.0;
}

static void trace_pixel(const oscene* s, const orc_camera* cam, const orc_lens* lens,
                        const orc_params* p, int32_t i, int32_t j, int n, double* rt) {
    int32_t W = cam->width, H = cam->height;
    double t = cam->tan_half_fovy;
    double SwL[3] = {0, 0, 0}, SfL[3] = {0, 0, 0}, SfP[3] = {0, 0, 0};
    double Sw = 0, Sf = 0, Swc = 0, Sfc = 0, Ss = 0;
    for (int smp = 0; smp < n; ++smp) {
        double O[3], dir[3], ws;
        orc_lens_ray(cam, lens, p, (int64_t)j * W + i, smp, O, dir, &ws);
        double th_, bary[3], n_[3], L[3], P[3], c;
        int32_t id = orc_closest_hit(s, O, dir, 1, &th_, bary);
        if (id >= 0) {
            for (int k = 0; k < 3; ++k) P[k] = O[k] + th_ * dir[k];
            double v[3];
            sub3(P, cam->pos, v);
            c = orc_coc(dot3(v, cam->fwd), lens, H, t);
            shade_hit(s, id, bary, dir, p, n_, L, NULL);
        } else {
            for (int k = 0; k < 3; ++k) { P[k] = O[k] + p->miss_dist * dir[k]; L[k] = 0.0; }
            c = orc_coc(INFINITY, lens, H, t);
        }
        /* split weight, scaled by the sample's aperture weight (1 for the uniform disk) */
        double w = ws * clampd((c + SQRT2) / (2.0 * SQRT2), 0.0, 1.0), wf = ws - w, ac = fabs(c);
        for (int k = 0; k < 3; ++k) {
            SwL[k] += w * L[k];
            SfL[k] += wf * L[k];
            SfP[k] += wf * P[k];
        }
        Sw += w; Sf += wf; Swc += w * ac; Sfc += wf * ac; Ss += ws;
    }
    int nok = Sw >= EMPTY_W, fok = Sf >= EMPTY_W;
    for (int k = 0; k < 3; ++k) {
        rt[k] = nok ? SwL[k] / Sw : 0.0;
        rt[4 + k] = fok ? SfL[k] / Sf : 0.0;
        rt[8 + k] = fok ? SfP[k] / Sf : 0.0;
    }
    rt[3] = Sw / Ss;
    rt[7] = nok ? Swc / Sw : -1.0;
    rt[11] = fok ? Sfc / Sf : -1.0;
}

void orc_trace(const void* sp, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
               const uint8_t* spp, double* rt, int32_t n_pix, const int32_t* pix) {
    const oscene* s = (const oscene*)sp;
    int32_t W = cam->width, H = cam->height;
    if (pix) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int32_t k = 0; k < n_pix; ++k) {
            int32_t q = pix[k];
            double* o = rt + 12 * (size_t)k;
            if (spp[q] == 0) { memset(o, 0, 12 * sizeof(double)); continue; }
            trace_pixel(s, cam, lens, p, q % W, q / W, spp[q], o);
        }
        return;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            double* o = rt + 12 * q;
            if (spp[q] == 0) { memset(o, 0, 12 * sizeof(double)); continue; }
            trace_pixel(s, cam, lens, p, i, j, spp[q], o);
        }
}

/* ------------------------------------------------------------------------
 * Temporal reconstruction (Reconstruction section).  History per pixel:
 * near = (EMA of h*C_near, EMA of h), far = (EMA of (1-h)*C_far, EMA of 1-h),
 * mom = (EMA of Y, EMA of Y^2) with Y the luminance of this frame's ray-traced
 * colour, hlen = frames accumulated (0 = none).  Near terms and moments are
 * reprojected with the motion vector; far terms with the previous-frame
 * projection of the far world position (average of the pixel's far hits; else
 * of its 3x3 neighbours' far hits; else the G-buffer surface point).  History
 * is sampled bilinearly over taps that hold history, renormalised, and is
 * invalid below a total weight of 1e-3.  EMA: x <- x_hist + alpha (x - x_hist).
 * Layer colours are normalised by their accumulated hit ratio; the composed
 * colour uses this frame's hit ratio when the camera moved, else the
 * accumulated one.  The CoC blends this frame's near and far CoC by the
 * accumulated hit ratio.  Untraced pixels drop their history.
 * ---------------------------------------------------------------------- */
static int hist_bilinear(int32_t W, int32_t H, double ux, double uy, const uint8_t* hlen,
                         const double* plane, int ch, double* out, int* hmax) {
    double x0 = floor(ux), y0 = floor(uy), fx = ux - x0, fy = uy - y0;
    double ws = 0.0;
    for (int c = 0; c < ch; ++c) out[c] = 0.0;
    if (hmax) *hmax = 0;
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            double x = x0 + a, y = y0 + b;
            if (x < 0.0 || y < 0.0 || x >= W || y >= H) continue;
            size_t q = (size_t)y * W + (size_t)x;
            if (hlen[q] == 0) continue;
            double w = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
            ws += w;
            for (int c = 0; c < ch; ++c) out[c] += w * plane[(size_t)ch * q + c];
            if (hmax && w > 0.0 && hlen[q] > *hmax) *hmax = hlen[q];
        }
    if (!(ws >= HIST_MIN_W)) return 0;
    for (int c = 0; c < ch; ++c) out[c] /= ws;
    return 1;
}

void orc_temporal(const orc_camera* cam, const orc_camera* prev, const orc_params* p,
                  const double* rt, const uint8_t* spp, const double* nd, const double* mv,
                  const double* h_near, const double* h_far, const double* h_mom,
                  const uint8_t* h_hlen, double* o_near, double* o_far, double* o_mom,
                  uint8_t* o_hlen, double* crt, double* hacc) {
    int32_t W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            if (spp[q] == 0) {
                memset(o_near + 4 * q, 0, 4 * sizeof(double));
                memset(o_far + 4 * q, 0, 4 * sizeof(double));
                memset(o_mom + 2 * q, 0, 2 * sizeof(double));
                memset(crt + 4 * q, 0, 4 * sizeof(double));
                hacc[q] = 0.0;
                o_hlen[q] = 0;
                continue;
            }
            const double* r = rt + 12 * q;
            double h = r[3], cn = r[7], cf = r[11];
            int nok = cn >= 0.0, fok = cf >= 0.0;
            double Ccur[3];
            for (int k = 0; k < 3; ++k)
                Ccur[k] = nok ? (fok ? h * r[k] + (1.0 - h) * r[4 + k] : r[k]) : r[4 + k];
            double Y = luminance(Ccur);
            /* near reprojection */
            double un = i - mv[2 * q], vn = j - mv[2 * q + 1];
            double hn[4], hm[2];
            int hl = 0;
            int vn_ok = hist_bilinear(W, H, un, vn, h_hlen, h_near, 4, hn, &hl);
            if (vn_ok) hist_bilinear(W, H, un, vn, h_hlen, h_mom, 2, hm, NULL);
            /* far world position */
            double P[3];
            if (fok) {
                for (int k = 0; k < 3; ++k) P[k] = r[8 + k];
            } else {
                double acc[3] = {0, 0, 0};
                int cnt = 0;
                for (int b = -1; b <= 1; ++b)
                    for (int a = -1; a <= 1; ++a) {
                        if (!a && !b) continue;
                        int x = i + a, y = j + b;
                        if (x < 0 || y < 0 || x >= W || y >= H) continue;
                        size_t qq = (size_t)y * W + x;
                        if (spp[qq] == 0 || rt[12 * qq + 11] < 0.0) continue;
                        for (int k = 0; k < 3; ++k) acc[k] += rt[12 * qq + 8 + k];
                        cnt++;
                    }
                if (cnt > 0) {
                    for (int k = 0; k < 3; ++k) P[k] = acc[k] / cnt;
                } else {
                    double d[3];
                    orc_pinhole_dir(cam, i + 0.5 + cam->jitter[0], j + 0.5 + cam->jitter[1], d);
                    for (int k = 0; k < 3; ++k) P[k] = cam->pos[k] + nd[4 * q + 3] * d[k];
                }
            }
            double uf[2], hf[4];
            int vf_ok = orc_project(prev, P, uf) && hist_bilinear(W, H, uf[0], uf[1], h_hlen, h_far, 4, hf, NULL);
            /* EMA weight: fixed, or per pixel (Discussion: per-pixel blend factors against ghosting, after
             * Schied et al.'s gradient-estimated temporal filtering): the normalised temporal gradient
             * lambda = clamp((|Y - mu1| - alpha_k sigma_L) / max(Y, mu1, 1e-3), 0, 1) of this frame's
             * luminance against the reprojected history, whose per-frame spread sigma_L counts as noise;
             * alpha = alpha_min + (1 - alpha_min) lambda */
            double al = p->ema_alpha;
            if (p->alpha_k > 0.0 && vn_ok) {
                double sg = sqrt(fmax(0.0, hm[1] - hm[0] * hm[0]));
                double den = fmax(fmax(Y, hm[0]), 1e-3);
                double lam = clampd((fabs(Y - hm[0]) - p->alpha_k * sg) / den, 0.0, 1.0);
                /* the hit ratio's change beyond alpha_k binomial standard errors of n samples */
                double hb = hn[3], se = sqrt(fmax(hb * (1.0 - hb), 0.0) / spp[q]);
                double lh = clampd(fabs(h - hb) - p->alpha_k * se, 0.0, 1.0);
                if (lh > lam) lam = lh;
                al += (1.0 - al) * lam;
            }
            /* EMA */
            double cur_n[4] = {h * r[0], h * r[1], h * r[2], h};
            double cur_f[4] = {(1 - h) * r[4], (1 - h) * r[5], (1 - h) * r[6], 1 - h};
            double cur_m[2] = {Y, Y * Y};
            double *on = o_near + 4 * q, *of = o_far + 4 * q, *om = o_mom + 2 * q;
            for (int k = 0; k < 4; ++k) {
                on[k] = vn_ok ? hn[k] + al * (cur_n[k] - hn[k]) : cur_n[k];
                of[k] = vf_ok ? hf[k] + al * (cur_f[k] - hf[k]) : cur_f[k];
            }
            for (int k = 0; k < 2; ++k) om[k] = vn_ok ? hm[k] + al * (cur_m[k] - hm[k]) : cur_m[k];
            int nh = vn_ok ? hl + 1 : 1;
            o_hlen[q] = (uint8_t)(nh > 255 ? 255 : nh);
            /* accumulated hit ratio, layer colours, composition */
            double Bn = on[3], Bf = of[3];
            double Hacc = (Bn + Bf >= EMPTY_W) ? Bn / (Bn + Bf) : h;
            int an = Bn >= EMPTY_W, af = Bf >= EMPTY_W;
            double hw = p->camera_moved ? h : Hacc;
            for (int k = 0; k < 3; ++k) {
                double Cn = an ? on[k] / Bn : 0.0, Cf = af ? of[k] / Bf : 0.0;
                crt[4 * q + k] = !an ? Cf : (!af ? Cn : hw * Cn + (1.0 - hw) * Cf);
            }
            crt[4 * q + 3] = !nok ? cf : (!fok ? cn : Hacc * cn + (1.0 - Hacc) * cf);
            hacc[q] = Hacc;
        }
}

/* ------------------------------------------------------------------------
 * Spatial reconstruction (Reconstruction section): circular gather over
 * traced pixels scaled by the pixel's CoC, rejecting samples whose CoC radius
 * is smaller than their distance, then blended by the clamped variance.
 *   r = min(c_rt / 2, R_s);  soft step s(x) = clamp(x + 0.5, 0, 1)
 *   C_sp = sum_q s(r_p - d) s(r_q - d) C_rt(q) / sum_q (same weight)
 *   beta = hlen < 2 ? 1 : clamp(sigma_L / var_ref, 0, 1)
 *   C_rec = C_rt + beta (C_sp - C_rt)
 * ---------------------------------------------------------------------- */
static double soft_step(double x) { return clampd(x + 0.5, 0.0, 1.0); }

static void spatial_pixel(int32_t W, int32_t H, const orc_params* p, const double* crt,
                          const uint8_t* spp, const double* mom, const uint8_t* hlen,
                          int32_t i, int32_t j, double* o) {
    size_t q = (size_t)j * W + i;
    if (spp[q] == 0) { o[0] = o[1] = o[2] = o[3] = 0.0; return; }
    double rp = fmin(crt[4 * q + 3] * 0.5, p->r_s);
    int K = (int)ceil(rp + 0.5);
    double S[3] = {0, 0, 0}, Ws = 0.0;
    for (int b = -K; b <= K; ++b)
        for (int a = -K; a <= K; ++a) {
            int x = i + a, y = j + b;
            if (x < 0 || y < 0 || x >= W || y >= H) continue;
            size_t qq = (size_t)y * W + x;
            if (spp[qq] == 0) continue;
            double d = sqrt((double)(a * a + b * b));
            double rq = fmin(crt[4 * qq + 3] * 0.5, p->r_s);
            double w = soft_step(rp - d) * soft_step(rq - d);
            if (w <= 0.0) continue;
            for (int k = 0; k < 3; ++k) S[k] += w * crt[4 * qq + k];
            Ws += w;
        }
    double m1 = mom[2 * q], m2 = mom[2 * q + 1];
    double sig = sqrt(fmax(0.0, m2 - m1 * m1));
    double beta = hlen[q] < 2 ? 1.0 : clampd(sig / p->var_ref, 0.0, 1.0);
    for (int k = 0; k < 3; ++k) {
        double c = crt[4 * q + k];
        o[k] = c + beta * (S[k] / Ws - c);
    }
    o[3] = 0.0;
}

void orc_spatial(int32_t W, int32_t H, const orc_params* p, const double* crt, const uint8_t* spp,
                 const double* mom, const uint8_t* hlen, double* crec, int32_t n_pix,
                 const int32_t* pix) {
    if (pix) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int32_t k = 0; k < n_pix; ++k)
            spatial_pixel(W, H, p, crt, spp, mom, hlen, pix[k] % W, pix[k] / W, crec + 4 * (size_t)k);
        return;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i)
            spatial_pixel(W, H, p, crt, spp, mom, hlen, i, j, crec + 4 * ((size_t)j * W + i));
}

/* ------------------------------------------------------------------------
 * Post-process CoC filter on the sharp image (Design section, adapted
 * gather; the same rejection rule as the spatial gather).  Scatter-as-gather:
 * pixel q spreads its colour over a soft disk s(r_q - d) of radius
 * r_q = min(|c(z_q)|/2, R_max), normalised by the disk's discrete area
 *   a(r) = sum over integer offsets o of s(r - |o|)
 * so that every pixel scatters a total weight of exactly 1.  Near layer:
 * weights w_near(q) s(r_q - d) / a(r_q); alpha = their sum clamped to [0,1].
 * Far layer: weights (1 - w_near(q)) s(r_q - d) k_z / a(r_q) with the soft
 * depth test k_z = clamp(1 - (z_q - z_p) / (kz_rel z_p), 0, 1); an empty far
 * layer takes the sharp colour.
 *   C_pp = alpha N + (1 - alpha) F,   pp = (C_pp, alpha)
 * ---------------------------------------------------------------------- */
double orc_disk_area(double r) {
    int K = (int)ceil(r + 0.5);
    double a = 0.0;
    for (int y = -K; y <= K; ++y)
        for (int x = -K; x <= K; ++x) a += soft_step(r - sqrt((double)(x * x + y * y)));
    return a;
}

/* Shaped bokeh (blades >= 3 or aberration != 0): the thin lens images an
 * aperture point O of a source at CoC c onto the screen offset
 * (c / 2A) (-O_right, O_up) (screen y grows downwards), so a near source's
 * bokeh is the aperture scaled to radius |c|/2 and mirrored left-right, a far
 * source's mirrored top-bottom.  A receiver at screen offset o = (ox, oy)
 * from source q lies at aperture norm D_near = D(-ox, oy) or D_far =
 * D(ox, -oy) in units of pixels, and its weight is s(r_q - D) times the
 * aperture weight at |o| / max(r_q, 1/2) (clamped to 1).  Normalised by the
 * lattice area of that weighted soft shape (the same for both mirrors: each
 * maps the integer lattice onto itself). */
static int shaped(const orc_params* p) { return p->blades >= 3 || p->aberration != 0.0; }

static double shaped_weight(double r, double D, double d, const orc_params* p) {
    double s = soft_step(r - D);
    if (s <= 0.0 || r < 1.0) return s;  /* a bokeh under a pixel wide shows no radial weighting */
    double tt = d / r;
    return s * aperture_weight(tt < 1.0 ? tt : 1.0, p);
}

double orc_shaped_area(double r, const orc_params* p) {
    int K = (int)ceil(r + 0.5);
    double a = 0.0;
    for (int y = -K; y <= K; ++y)
        for (int x = -K; x <= K; ++x)
            a += shaped_weight(r, aperture_norm(x, y, p), sqrt((double)(x * x + y * y)), p);
    return a;
}

static void postfilter_pixel(int32_t W, int32_t H, const orc_lens* lens, double t, const orc_params* p,
                             const double* nd, const double* col, const double* inv_area,
                             int32_t i, int32_t j, double* o) {
    int K = (int)ceil(p->r_max + 0.5);
    size_t pq = (size_t)j * W + i;
    double zp = nd[4 * pq + 3];
    double Sn[3] = {0, 0, 0}, Sf[3] = {0, 0, 0}, Wn = 0.0, Wf = 0.0;
    for (int b = -K; b <= K; ++b)
        for (int a = -K; a <= K; ++a) {
            int x = i + a, y = j + b;
            if (x < 0 || y < 0 || x >= W || y >= H) continue;
            size_t q = (size_t)y * W + x;
            double zq = nd[4 * q + 3];
            double c = orc_coc(zq, lens, H, t);
            double r = fmin(fabs(c) * 0.5, p->r_max);
            double d = sqrt((double)(a * a + b * b));
            double s = soft_step(r - d), sf = s;
            if (shaped(p)) {
                /* receiver p at offset o = (-a, -b) from source q: D_near = D(a, -b), D_far = D(-a, b) */
                s = shaped_weight(r, aperture_norm(a, -b, p), d, p);
                sf = shaped_weight(r, aperture_norm(-a, b, p), d, p);
            }
            if (s <= 0.0 && sf <= 0.0) continue;
            double ia = inv_area[q];
            double wn = clampd((c + SQRT2) / (2.0 * SQRT2), 0.0, 1.0);
            double kz = clampd(1.0 - (zq - zp) / (p->kz_rel * zp), 0.0, 1.0);
            double an = wn * s * ia, af = (1.0 - wn) * sf * ia * kz;
            for (int k = 0; k < 3; ++k) { Sn[k] += an * col[4 * q + k]; Sf[k] += af * col[4 * q + k]; }
            Wn += an;
            Wf += af;
        }
    double alpha = clampd(Wn, 0.0, 1.0);
    for (int k = 0; k < 3; ++k) {
        double N = Wn > PP_MIN_W ? Sn[k] / Wn : 0.0;
        double F = Wf > PP_MIN_W ? Sf[k] / Wf : col[4 * pq + k];
        o[k] = alpha * N + (1.0 - alpha) * F;
    }
    o[3] = alpha;
}

void orc_postfilter(int32_t W, int32_t H, const orc_lens* lens, double t, const orc_params* p,
                    const double* nd, const double* col, double* pp, int32_t n_pix, const int32_t* pix) {
    /* 1 / a(r_q) depends on pixel q alone: evaluate it once per pixel */
    double* inv_area = (double*)malloc(sizeof(double) * (size_t)W * H);
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t q = 0; q < W * H; ++q) {
        double r = fmin(fabs(orc_coc(nd[4 * (size_t)q + 3], lens, H, t)) * 0.5, p->r_max);
        inv_area[q] = 1.0 / (shaped(p) ? orc_shaped_area(r, p) : orc_disk_area(r));
    }
    if (pix) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int32_t k = 0; k < n_pix; ++k)
            postfilter_pixel(W, H, lens, t, p, nd, col, inv_area, pix[k] % W, pix[k] / W, pp + 4 * (size_t)k);
        free(inv_area);
        return;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i)
            postfilter_pixel(W, H, lens, t, p, nd, col, inv_area, i, j, pp + 4 * ((size_t)j * W + i));
    free(inv_area);
}

/* ------------------------------------------------------------------------
 * Composite (Composite section).  Focus-zone weight from the pixel's CoC (the
 * reconstructed ray-traced CoC where traced, else the G-buffer depth's):
 *   f = clamp(sqrt2 + 0.5 - |c|, 0, 1)   (the hard |c| < sqrt2 softened over one px)
 * near branch: traced ? lerp(C_rec, C_pp, clamp(spec_pref S_pp, 0, 1)) : C_pp,
 *   S_pp the specular part of the post-process colour (pp_spec, the post-filter
 *   of the specular plane; the preference for bright specular bokeh); without
 *   pp_spec, or with spec_pref = 0, traced ? C_rec : C_pp;
 * far branch: traced ? lerp(C_rec, C_pp, clamp(H_acc / h_tau, 0, 1)) : C_pp;
 * C_blur = w_near(c(z_p)) near + (1 - w_near) far;  out = lerp(C_blur, sharp, f).
 * ---------------------------------------------------------------------- */
void orc_composite(int32_t n, int32_t H, const orc_lens* lens, double t, const orc_params* p,
                   const double* nd, const double* col, const uint8_t* spp, const double* pp,
                   const double* pp_spec, const double* crt, const double* crec, const double* hacc,
                   double* out) {
    /* per-pixel: the planes are flat lists of n pixels of an image of height H */
#pragma omp parallel for
    for (int32_t qi = 0; qi < n; ++qi) {
            size_t q = (size_t)qi;
            double c = orc_coc(nd[4 * q + 3], lens, H, t);
            int traced = spp[q] > 0;
            double ce = traced ? crt[4 * q + 3] : fabs(c);
            double f = clampd(SQRT2 + 0.5 - ce, 0.0, 1.0);
            double wn = clampd((c + SQRT2) / (2.0 * SQRT2), 0.0, 1.0);
            double b = traced ? clampd(hacc[q] / p->h_tau, 0.0, 1.0) : 0.0;
            double sp = (traced && pp_spec && p->spec_pref > 0.0)
                            ? clampd(p->spec_pref * pp_spec[4 * q], 0.0, 1.0) : 0.0;
            for (int k = 0; k < 3; ++k) {
                double near_ = traced ? crec[4 * q + k] + sp * (pp[4 * q + k] - crec[4 * q + k]) : pp[4 * q + k];
                double far_ = traced ? crec[4 * q + k] + b * (pp[4 * q + k] - crec[4 * q + k]) : pp[4 * q + k];
                double blur = wn * near_ + (1.0 - wn) * far_;
                out[4 * q + k] = blur + f * (col[4 * q + k] - blur);
            }
            out[4 * q + 3] = 0.0;
        }
}

/* ------------------------------------------------------------------------
 * Differentiable post-path with frozen visibility.  The thin-lens samples of
 * a forward trace are recorded per ray as (L rgb, z) -- radiance and view
 * depth of the hit, z = +inf for a miss -- so the trace accumulation can be
 * re-evaluated at another focus distance and aperture with the same hits
 * (the visibility is held fixed; only each hit's CoC, split weight and CoC
 * magnitude change).  rec: [n_rays][4]; off[p]: first ray of pixel p
 * (row-major prefix of spp).
 * ---------------------------------------------------------------------- */
void orc_trace_records(const void* sp, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                       const uint8_t* spp, const int64_t* off, double* rec) {
    const oscene* s = (const oscene*)sp;
    int32_t W = cam->width, H = cam->height;
    (void)H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < cam->height; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            int n = spp[q];
            if (!n) continue;
            for (int smp = 0; smp < n; ++smp) {
                double O[3], dir[3];
                orc_lens_ray(cam, lens, p, (int64_t)q, smp, O, dir, NULL);
                double th_, bary[3], n_[3], L[3], P[3], z;
                int32_t id = orc_closest_hit(s, O, dir, 1, &th_, bary);
                if (id >= 0) {
                    for (int k = 0; k < 3; ++k) P[k] = O[k] + th_ * dir[k];
                    double v[3];
                    sub3(P, cam->pos, v);
                    z = dot3(v, cam->fwd);
                    shade_hit(s, id, bary, dir, p, n_, L, NULL);
                } else {
                    z = INFINITY;
                    L[0] = L[1] = L[2] = 0.0;
                }
                double* r = rec + 4 * (size_t)(off[q] + smp);
                r[0] = L[0]; r[1] = L[1]; r[2] = L[2]; r[3] = z;
            }
        }
}

/* Closest hit of every thin-lens sample (the visibility the trace shades):
 * for sample s of pixel q, ids[off[q] + s] = hit triangle (-1 = miss),
 * ts[...] = ray parameter along the unit direction, margin[...] = distance
 * of the hit point from the nearest edge of its triangle (world units,
 * +inf for a miss): a small margin marks a hit a slightly different ray can
 * miss (an epsilon-tie of the closest-hit decision). */
void orc_trace_hits(const void* sp, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                    const uint8_t* spp, const int64_t* off, int32_t* ids, double* ts, double* margin) {
    const oscene* s = (const oscene*)sp;
    int32_t W = cam->width;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < cam->height; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            for (int smp = 0; smp < spp[q]; ++smp) {
                double O[3], dir[3], th_, bary[3];
                orc_lens_ray(cam, lens, p, (int64_t)q, smp, O, dir, NULL);
                int32_t id = orc_closest_hit(s, O, dir, 1, &th_, bary);
                size_t r = (size_t)(off[q] + smp);
                ids[r] = id;
                ts[r] = id >= 0 ? th_ : INFINITY;
                margin[r] = INFINITY;
                if (id >= 0) {
                    /* distance to the edge opposite vertex k = bary_k * 2 area / |edge_k| */
                    const double* v = s->v + 9 * (size_t)id;
                    double e1[3], e2[3], nrm[3], ek[3];
                    sub3(v + 3, v, e1);
                    sub3(v + 6, v, e2);
                    cross3(e1, e2, nrm);
                    double twice_area = sqrt(dot3(nrm, nrm));
                    for (int k = 0; k < 3; ++k) {
                        sub3(v + 3 * ((k + 2) % 3), v + 3 * ((k + 1) % 3), ek);
                        double m = fabs(bary[k]) * twice_area / sqrt(dot3(ek, ek));
                        if (m < margin[r]) margin[r] = m;
                    }
                }
            }
        }
}

/* Full ray-traced depth of field (the reference the paper's Fig. 1 sets
 * beside the hybrid frame): the thin-lens image by distributed ray tracing,
 * every pixel, no mask.  out[q] = the mean over passes of each pass's
 * weighted mean Lambert radiance of the closest hits of spp_max lens samples
 * (sample weights as in the trace; 1 on the uniform disk, where this is the
 * plain mean of all samples); pass k draws its samples with the key of frame
 * (frame + k) mod 65536.  Misses contribute 0. */
void orc_reference_rt(const void* sp, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                      int32_t passes, double* out) {
    const oscene* s = (const oscene*)sp;
    int32_t W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            double S[3] = {0, 0, 0};
            for (int32_t k = 0; k < passes; ++k) {
                orc_params pk = *p;
                pk.frame = (int32_t)(((uint32_t)p->frame + (uint32_t)k) & 0xFFFFu);
                double Sk[3] = {0, 0, 0}, n = 0.0;
                for (int smp = 0; smp < p->spp_max; ++smp) {
                    double O[3], dir[3], th_, bary[3], n_[3], L[3], ws;
                    orc_lens_ray(cam, lens, &pk, (int64_t)q, smp, O, dir, &ws);
                    n += ws;
                    int32_t id = orc_closest_hit(s, O, dir, 1, &th_, bary);
                    if (id < 0) continue;
                    shade_hit(s, id, bary, dir, p, n_, L, NULL);
                    for (int c = 0; c < 3; ++c) Sk[c] += ws * L[c];
                }
                for (int c = 0; c < 3; ++c) S[c] += Sk[c] / n;
            }
            for (int c = 0; c < 3; ++c) out[4 * q + c] = S[c] / passes;
            out[4 * q + 3] = 0.0;
        }
}

/* The trace accumulation (same definitions as orc_trace) from recorded hits;
 * P_far is not recorded and is left 0. */
void orc_replay(int32_t W, int32_t H, const orc_lens* lens, double t, const uint8_t* spp, const int64_t* off,
                const double* rec, double* rt) {
#pragma omp parallel for
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            double* o = rt + 12 * q;
            int n = spp[q];
            memset(o, 0, 12 * sizeof(double));
            if (!n) continue;
            double SwL[3] = {0, 0, 0}, SfL[3] = {0, 0, 0}, Sw = 0, Sf = 0, Swc = 0, Sfc = 0;
            for (int smp = 0; smp < n; ++smp) {
                const double* r = rec + 4 * (size_t)(off[q] + smp);
                double c = orc_coc(r[3], lens, H, t);
                double w = clampd((c + SQRT2) / (2.0 * SQRT2), 0.0, 1.0), ac = fabs(c);
                for (int k = 0; k < 3; ++k) { SwL[k] += w * r[k]; SfL[k] += (1.0 - w) * r[k]; }
                Sw += w; Sf += 1.0 - w; Swc += w * ac; Sfc += (1.0 - w) * ac;
            }
            int nok = Sw >= EMPTY_W, fok = Sf >= EMPTY_W;
            for (int k = 0; k < 3; ++k) {
                o[k] = nok ? SwL[k] / Sw : 0.0;
                o[4 + k] = fok ? SfL[k] / Sf : 0.0;
            }
            o[3] = Sw / n;
            o[7] = nok ? Swc / Sw : -1.0;
            o[11] = fok ? Sfc / Sf : -1.0;
        }
}

/* Temporal reconstruction of orc_temporal with the history already sampled
 * at the reprojected positions and held fixed: hs[p][12] = (near rgb, B_near,
 * far rgb, B_far, mu1, mu2, flags = valid_near + 2 valid_far, hlen). */
void orc_temporal_frozen(int32_t W, int32_t H, const orc_params* p, const double* rt, const uint8_t* spp,
                         const double* hs, double* crt, double* hacc, double* mom, uint8_t* hlen) {
    double al = p->ema_alpha;
#pragma omp parallel for
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            size_t q = (size_t)j * W + i;
            if (spp[q] == 0) {
                crt[4 * q] = crt[4 * q + 1] = crt[4 * q + 2] = 0.0;
                crt[4 * q + 3] = -1.0;
                hacc[q] = 0.0;
                mom[2 * q] = mom[2 * q + 1] = 0.0;
                hlen[q] = 0;
                continue;
            }
            const double* r = rt + 12 * q;
            const double* s = hs + 12 * q;
            double h = r[3], cn = r[7], cf = r[11];
            int nok = cn >= 0.0, fok = cf >= 0.0;
            int flags = (int)s[10], vn = flags & 1, vf = (flags >> 1) & 1;
            double Ccur[3];
            for (int k = 0; k < 3; ++k)
                Ccur[k] = nok ? (fok ? h * r[k] + (1.0 - h) * r[4 + k] : r[k]) : r[4 + k];
            double Y = luminance(Ccur);
            double cur_n[4] = {h * r[0], h * r[1], h * r[2], h};
            double cur_f[4] = {(1 - h) * r[4], (1 - h) * r[5], (1 - h) * r[6], 1 - h};
            double on[4], of[4];
            for (int k = 0; k < 4; ++k) {
                on[k] = vn ? s[k] + al * (cur_n[k] - s[k]) : cur_n[k];
                of[k] = vf ? s[4 + k] + al * (cur_f[k] - s[4 + k]) : cur_f[k];
            }
            mom[2 * q] = vn ? s[8] + al * (Y - s[8]) : Y;
            mom[2 * q + 1] = vn ? s[9] + al * (Y * Y - s[9]) : Y * Y;
            int nh = vn ? (int)s[11] + 1 : 1;
            hlen[q] = (uint8_t)(nh > 255 ? 255 : nh);
            double Bn = on[3], Bf = of[3];
            double Hacc = (Bn + Bf >= EMPTY_W) ? Bn / (Bn + Bf) : h;
            int an = Bn >= EMPTY_W, af = Bf >= EMPTY_W;
            double hw = p->camera_moved ? h : Hacc;
            for (int k = 0; k < 3; ++k) {
                double Cn = an ? on[k] / Bn : 0.0, Cf = af ? of[k] / Bf : 0.0;
                crt[4 * q + k] = !an ? Cf : (!af ? Cn : hw * Cn + (1.0 - hw) * Cf);
            }
            crt[4 * q + 3] = !nok ? cf : (!fok ? cn : Hacc * cn + (1.0 - Hacc) * cf);
            hacc[q] = Hacc;
        }
}
