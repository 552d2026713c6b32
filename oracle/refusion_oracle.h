/*
 * ReFusion FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential restatement of the per-frame path of
 * "ReFusion: 3D Reconstruction in Dynamic Environments for RGB-D Cameras
 * Exploiting Residuals" (Palazzolo et al., IROS 2019): TSDF model with voxel
 * hashing (Sec. III-A), SDF + colour Levenberg-Marquardt registration
 * (Sec. III-B, Eq. 1-4), residual-based dynamic mask with Alg. 1 flood fill
 * (Sec. III-C, Eq. 5) and integration with free-space carving (Sec. III-D).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or table with the CUDA
 * library; the two are tied together only by the written definitions of the
 * method (and the readings of the paper where it is silent).
 */
#ifndef REFUSION_ORACLE_H
#define REFUSION_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double voxel_size;    /* m, Tab. I: 0.01 */
  double trunc;         /* tau, m, Tab. I: 0.1 */
  double w_c;           /* colour weight of Eq. 4, Tab. I: 0.025 */
  double theta;         /* flood-fill threshold of Alg. 1, Tab. I: 0.007 */
  double gamma;         /* residual threshold weight of Eq. 5, Tab. I: 0.5 */
  double depth_scale;   /* raw depth units per metre (1000 = mm) */
  double d_min;         /* valid depth range, m */
  double d_max;         /* also the carving clipping plane (Sec. III-D) */
  double z_near;        /* near plane of the carved frustum, m */
  int w_max;            /* weight cap of the running averages */
  int lm_iters[3];      /* LM candidate evaluations per level */
  int lm_strides[3];    /* pixel sub-sampling stride per level */
  double lm_lambda0;
  double lm_eps_trans;  /* convergence: |delta rho| (m) */
  double lm_eps_rot;    /* convergence: |delta phi| (rad) */
  int lm_min_valid;     /* minimum number of valid pixels for an evaluation */
} orc_params;

typedef struct {
  int height, width;
  double fx, fy, cx, cy;
  const uint16_t* depth; /* [H*W] raw units, 0 = invalid */
  const uint8_t* rgb;    /* [H*W*3] RGB8 */
} orc_frame;

typedef struct {
  int evals;          /* cost evaluations over all levels */
  int level_evals[3];
  int converged[3];
  double final_cost;  /* mean cost E/N at the returned pose (last level) */
  int64_t final_valid;
} orc_track_info;

void* orc_create(const orc_params* p);
void orc_destroy(void* vol);
int64_t orc_num_blocks(void* vol);
int orc_num_frames(void* vol);

/* Integration with free-space carving; returns number of updated voxels. */
int64_t orc_integrate(void* vol, const orc_frame* f, const double T[16], const uint8_t* mask);

/* Levenberg-Marquardt registration (three levels). */
void orc_track(void* vol, const orc_frame* f, const double T_init[16], const uint8_t* mask,
               double T_out[16], orc_track_info* info);
/* orc_track, also counting the distinct blocks its model lookups probed and
 * the distinct voxels they read (the footprint of a registration; bookkeeping
 * only, the result is orc_track's). */
void orc_track_footprint(void* vol, const orc_frame* f, const double T_init[16], const uint8_t* mask,
                         double T_out[16], orc_track_info* info, int64_t* n_blocks_probed, int64_t* n_voxels_read);

/* Normal equations at pose T: H[21] (upper triangle, row-major), g[6], E, N. */
void orc_eval(void* vol, const orc_frame* f, const double T[16], int stride, const uint8_t* mask,
              double H[21], double g[6], double* E, int64_t* N);

/* Trilinear model lookup at world point p. returns 1 if the SDF is valid. */
int orc_lookup(void* vol, const double p[3], double* sdf, double gsdf[3], double* inten,
               double ginten[3], int* colour_ok);

/* Residual r_i = V_SDF^2 per pixel at pose T (negative = invalid), seeds r_i > gamma tau^2. */
void orc_residual_seeds(void* vol, const orc_frame* f, const double T[16], double* r, uint8_t* seeds);
void orc_erode3(const uint8_t* in, int H, int W, uint8_t* out);
void orc_dilate3(const uint8_t* in, int H, int W, uint8_t* out);
void orc_floodfill(const uint8_t* MR, const uint16_t* depth, int H, int W, int64_t theta_ppm, uint8_t* MD);
void orc_compute_mask(void* vol, const orc_frame* f, const double T[16], uint8_t* mask);

/* Virtual depth (Sec. III-E, second option) of rows [row0, row1): zero pixels of f->depth take the first
 * positive-to-non-positive TSDF crossing along their ray seen from T (samples z_near + k voxel/2 up to
 * d_max, linear interpolation, rounded to raw units), far_raw where there is none; other pixels are copied. */
void orc_virtual_depth(void* vol, const orc_frame* f, const double T[16], uint16_t far_raw, int row0, int row1,
                       uint16_t* out);

/* Whole frame: track -> mask -> re-track -> integrate (first frame: integrate at T_init). */
void orc_process_frame(void* vol, const orc_frame* f, const double T_init[16], double T_out[16],
                       uint8_t* mask_out, orc_track_info* info);

/* se(3) exponential (xi = rho, phi) as 4x4 row-major; LM step solve. */
void orc_se3_exp(const double xi[6], double T[16]);
int orc_lm_solve(const double H[21], const double g[6], double lambda, double delta[6]);

/* Snapshot: blocks sorted by (bz, by, bx); voxel index x + 8 y + 64 z. */
void orc_export(void* vol, int32_t* coords, double* F, uint8_t* W, uint8_t* rgb, uint8_t* wc);
int orc_import(void* vol, int64_t n, const int32_t* coords, const double* F, const uint8_t* W,
               const uint8_t* rgb, const uint8_t* wc);

/* Marching tetrahedra: triangle soup, 3 vertices per triangle. Two calls:
 * pass NULL buffers to get the triangle count. */
int64_t orc_extract_mesh(void* vol, double* verts, uint8_t* colors, int64_t cap_tris);

#ifdef __cplusplus
}
#endif
#endif
