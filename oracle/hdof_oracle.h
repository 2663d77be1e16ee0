/* FP64 CPU oracle of the hybrid depth-of-field frame (Tan, Chua, Biette,
 * Bhojan, "Hybrid DoF: Ray-Traced and Post-Processed Hybrid Depth of Field
 * Effect for Real-Time Rendering", SIGGRAPH '20 Posters).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * statement of what the CUDA library computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Precision: double everywhere.  Inputs arrive as doubles converted exactly
 * from the float32 values the GPU reads.
 *
 * Image planes are row-major [H][W][C] (pixel (i,j) = column i, row j from the
 * top).  All functions are single-threaded per pixel; rows may run in
 * parallel under OpenMP, which does not change any result.
 */
#ifndef HDOF_ORACLE_H
#define HDOF_ORACLE_H
#include <stdint.h>

typedef struct {
    double pos[3], right[3], up[3], fwd[3];
    double tan_half_fovy;
    int32_t width, height;
    double jitter[2];
} orc_camera;

typedef struct {
    double focus_dist, aperture_radius, focal_length;
} orc_lens;

typedef struct {
    double gauss_sigma, edge_tau;
    int32_t tile, dilate, spp_max, variance_on;
    double var_tau, var_scale;
    int32_t hlen_young;
    uint32_t seed;
    int32_t frame, view;
    double k_ambient;
    int32_t n_lights;
    double light_dir[4][3];
    double light_E[4];
    double miss_dist;
    double ema_alpha;
    int32_t camera_moved;
    double r_s, var_ref;
    double r_max, kz_rel;
    double h_tau;
    double alpha_k;
    int32_t mask_coc, blades;
    double blade_rot, aberration;
    double spec_pref;
} orc_params;

/* ---- counter-based RNG (Philox4x32-10, Salmon et al. SC'11) ---- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_limb(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- thin lens ---- */
double orc_coc(double z, const orc_lens* lens, int32_t height, double tan_half_fovy);
void orc_pinhole_dir(const orc_camera* c, double sx, double sy, double d[3]);
int orc_project(const orc_camera* c, const double P[3], double u[2]);

/* ---- scene / closest hit ---- */
void* orc_scene_create(int32_t n_tris, const double* tri_v, const double* mat, const double* uv);
void orc_scene_destroy(void* s);
int32_t orc_intersect_tri(const double org[3], const double dir[3], const double* v9,
                          double* t, double bary[3]);
int32_t orc_closest_hit(const void* s, const double org[3], const double dir[3], int32_t use_bvh,
                        double* t, double bary[3]);
void orc_closest_hits(const void* s, int32_t n, const double* org, const double* dir,
                      int32_t use_bvh, int32_t* ids, double* ts);

/* ---- frame stages ---- */
void orc_gbuffer(const void* s, const orc_camera* cam, const orc_camera* prev, const orc_params* p,
                 double* nd, double* col, double* mv, int32_t* tri);
void orc_gaussian_weights(double sigma, double w[5]);
void orc_mask(int32_t W, int32_t H, const double* nd, const double* mv, const double* hist_mom,
              const uint8_t* hist_hlen, const orc_params* p, uint8_t* edge, uint8_t* spp,
              double* emetric);
void orc_mask_coc(int32_t W, int32_t H, const double* nd, const double* mv, const double* hist_mom,
                  const uint8_t* hist_hlen, const orc_params* p, const orc_lens* lens, double tan_half_fovy,
                  uint8_t* edge, uint8_t* spp, double* emetric);
void orc_trace(const void* s, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
               const uint8_t* spp, double* rt, int32_t n_pix, const int32_t* pix);
void orc_temporal(const orc_camera* cam, const orc_camera* prev, const orc_params* p,
                  const double* rt, const uint8_t* spp, const double* nd, const double* mv,
                  const double* h_near, const double* h_far, const double* h_mom,
                  const uint8_t* h_hlen, double* o_near, double* o_far, double* o_mom,
                  uint8_t* o_hlen, double* crt, double* hacc);
void orc_spatial(int32_t W, int32_t H, const orc_params* p, const double* crt, const uint8_t* spp,
                 const double* mom, const uint8_t* hlen, double* crec, int32_t n_pix,
                 const int32_t* pix);
void orc_postfilter(int32_t W, int32_t H, const orc_lens* lens, double tan_half_fovy,
                    const orc_params* p, const double* nd, const double* col, double* pp,
                    int32_t n_pix, const int32_t* pix);
void orc_composite(int32_t n, int32_t H, const orc_lens* lens, double tan_half_fovy,
                   const orc_params* p, const double* nd, const double* col, const uint8_t* spp,
                   const double* pp, const double* pp_spec, const double* crt, const double* crec,
                   const double* hacc, double* out);
double orc_disk_area(double r);
double orc_shaped_area(double r, const orc_params* p);
/* ---- differentiable post-path with frozen visibility ---- */
void orc_trace_records(const void* s, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                       const uint8_t* spp, const int64_t* off, double* rec);
void orc_replay(int32_t W, int32_t H, const orc_lens* lens, double tan_half_fovy, const uint8_t* spp,
                const int64_t* off, const double* rec, double* rt);
void orc_temporal_frozen(int32_t W, int32_t H, const orc_params* p, const double* rt, const uint8_t* spp,
                         const double* hs, double* crt, double* hacc, double* mom, uint8_t* hlen);
void orc_lens_ray(const orc_camera* cam, const orc_lens* lens, const orc_params* p, int64_t q, int32_t smp,
                  double O[3], double dir[3], double* weight);
void orc_trace_hits(const void* s, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                    const uint8_t* spp, const int64_t* off, int32_t* ids, double* ts, double* margin);
void orc_reference_rt(const void* s, const orc_camera* cam, const orc_lens* lens, const orc_params* p,
                      int32_t passes, double* out);
int32_t orc_num_threads(void);
#endif
