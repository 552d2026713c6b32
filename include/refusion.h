/*
 * refusion.h -- C ABI of the GB300 (sm_103a) ReFusion per-frame hot path.
 *
 * ReFusion (Palazzolo, Behley, Lottes, Giguere, Stachniss; IROS 2019) tracks
 * an RGB-D camera directly against a voxel-hashed TSDF with an SDF + colour
 * error (Sec. III-B, Eq. 1-4), detects dynamic pixels from the registration
 * residuals (Sec. III-C, Eq. 5, Alg. 1), registers again without them and
 * integrates the masked frame with explicit free-space carving (Sec. III-A,
 * III-D).  This library runs that loop in CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *  - Plain C types only.  `stream` is a cudaStream_t passed as void* (NULL =
 *    the legacy default stream).  Calls taking device pointers enqueue work on
 *    `stream` and return without synchronising; they are stream-ordered with
 *    respect to the caller's other work on that stream.
 *  - A pose T is a row-major 4x4 double matrix mapping camera coordinates to
 *    world coordinates (Eq. 2 applies T to back-projected camera points).
 *    Camera frame: x right, y down, z forward (pinhole, Eq. 1).
 *  - Depth: uint16, row-major, width*height, in units of 1/depth_scale metres;
 *    0 = invalid (Sec. III-E, first option).  Colour: RGB8 interleaved,
 *    width*height*3 bytes.  Masks: uint8 per pixel, nonzero = dynamic.
 *  - Ownership: the library owns every buffer it allocates (all inside
 *    rf_create_volume); caller buffers are borrowed for the duration of the
 *    enqueued work only.  No call allocates device memory after creation,
 *    except rf_volume_export/import staging on the host.
 *  - Errors: each call returns an rf_status.  Argument errors are detected on
 *    the host before anything is enqueued.  Errors found by kernels (hash or
 *    pool full, candidate overflow, flood fill not converged, grid-wide wait timeout)
 *    are OR-ed into a per-volume device status word; rf_sync_status()
 *    synchronises the stream, returns the first such error and clears it.
 *    rf_last_error() gives a readable message for the last failing call.
 *  - Every device loop is bounded; no kernel traps or spins without a limit.
 *  - A volume is not thread-safe: use one host thread (and one stream) per
 *    volume at a time.  Independent volumes may run concurrently.
 */
#ifndef REFUSION_H
#define REFUSION_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RF_ABI_VERSION 1

typedef enum rf_status {
  RF_OK = 0,
  RF_ERR_INVALID_ARG = 1,      /* bad pointer, size or parameter */
  RF_ERR_CUDA = 2,             /* a CUDA runtime call failed (message in rf_last_error) */
  RF_ERR_HASH_FULL = 3,        /* bounded hash probe found no free slot */
  RF_ERR_POOL_FULL = 4,        /* more blocks than max_blocks */
  RF_ERR_NOT_CONVERGED = 5,    /* flood fill exceeded max_ff_sweeps, or a grid-wide wait timed out */
  RF_ERR_BUFFER_TOO_SMALL = 6, /* caller buffer smaller than the result */
  RF_ERR_OUT_OF_RANGE = 7,     /* block coordinate outside +-8191 blocks per axis */
  RF_ERR_CAPACITY = 8          /* frustum candidate list overflow (raise max_candidates) */
} rf_status;

/* Parameters.  Defaults (rf_default_params) are Tab. I of the paper (voxel
 * 0.01 m, tau 0.1 m, w_c 0.025, theta 0.007, gamma 0.5) and the readings
 * for the quantities the paper leaves open. */
typedef struct rf_params {
  double voxel_size;   /* metres, at most 0.15; voxel_size * 1e6 must be an integer (micrometre lattice) */
  double trunc;        /* truncation distance tau (Sec. III-A), metres, below 2 */
  double w_c;          /* colour weight w_c of Eq. 4 */
  double theta;        /* flood-fill depth threshold of Alg. 1 (used as round(theta*1e6) ppm) */
  double gamma;        /* residual threshold weight of Eq. 5, t = gamma tau^2 */
  double depth_scale;  /* raw depth units per metre; 1e6/depth_scale must be an integer */
  double d_min;        /* valid depth range [d_min, d_max], metres */
  double d_max;        /* also the carving clipping plane (Sec. III-D); <= 50 m */
  double z_near;       /* near plane of the carved frustum, metres (> 0) */
  int w_max;           /* cap of the SDF and colour weights, 1..255 */
  int lm_iters[3];     /* LM candidate evaluations per level (coarse to fine) */
  int lm_strides[3];   /* pixel sub-sampling stride per level (Sec. III-B: 3 sub-samplings) */
  double lm_lambda0;   /* initial Marquardt damping */
  double lm_eps_trans; /* level converged when |delta rho| < eps_trans (m) ... */
  double lm_eps_rot;   /* ... and |delta phi| < eps_rot (rad) */
  int lm_min_valid;    /* an evaluation with fewer valid pixels is rejected */
  int max_ff_sweeps;   /* bound on flood-fill sweeps (RF_ERR_NOT_CONVERGED beyond) */
  int64_t max_candidates; /* capacity of the per-frame frustum block candidate list */
  int storage;         /* voxel storage: RF_STORAGE_FP32 (default) or RF_STORAGE_FP16 (compact) */
} rf_params;

/* Voxel storage modes.  FP32: SDF as float, weights and colour as uint8 (9 B
 * per voxel).  FP16 (the precision form): SDF as FP16 of F/tau, the SDF
 * weight and an 8-bit intensity (round(254 I), Sec. III-B) in one 4-byte
 * tracking word, colour and colour weight in a 4-byte colour word (8 B per
 * voxel); tracking reads 4 B per trilinear corner and free-space carving
 * rewrites 4 B per voxel.  Per-pixel maths, reductions and the LM step are
 * FP32 in both modes (the step's refinement residual formed exactly, the
 * pose carried as float pairs); hash indexing and the mask's decisions stay
 * exact (on the values stored).  rf_volume_export returns F = FP16 value x
 * tau (float multiply); rf_volume_import rounds F / tau to FP16 (nearest). */
#define RF_STORAGE_FP32 0
#define RF_STORAGE_FP16 1

/* One RGB-D frame in device memory (row-major, rows of exactly `width`). */
typedef struct rf_frame {
  int height, width;
  double fx, fy, cx, cy;   /* pinhole intrinsics (Eq. 1); fx*256 and (cx+0.5)*256 are rounded to integers */
  const uint16_t* depth;   /* height*width; device or page-locked host memory */
  const uint8_t* rgb;      /* height*width*3; device or page-locked host memory */
} rf_frame;

/* Registration summary (written to device memory by rf_track_frame). */
typedef struct rf_track_info {
  int evals;            /* cost evaluations over the three levels */
  int level_evals[3];
  int converged[3];     /* 1 if the level stopped on the step-size test or a failed solve */
  double final_cost;    /* mean cost E/N at the returned pose, last evaluated level */
  int64_t final_valid;  /* N: pixels with a valid model lookup at that evaluation */
} rf_track_info;

typedef struct rf_stats {
  int64_t n_blocks;       /* allocated 8x8x8 voxel blocks */
  int64_t max_blocks;
  int64_t n_buckets;      /* hash buckets (4 slots each) */
  int64_t frames;         /* frames processed by rf_process_frame */
  double load_factor;     /* n_blocks / (4 n_buckets) */
  int64_t device_bytes;   /* device memory owned by the volume */
} rf_stats;

/* Device-side timings and work counters of the last frame (rf_get_profile). */
typedef struct rf_profile {
  float frame_ms;            /* device time of the last rf_process_frame* call */
  float track_ms[2];         /* first and second registration */
  float mask_ms;             /* seeds, erosion, flood fill, dilation */
  float integrate_ms;        /* integration stage: frustum search, cull, update, neighbour tables */
  float integrate_kernel_ms; /* the per-voxel update kernel alone */
  int64_t candidates;        /* frustum candidate blocks of the last integration */
  int64_t updated_voxels;    /* voxels updated by the last integration */
  int64_t new_blocks;        /* blocks allocated by the last integration */
  int64_t guard_pixels;      /* mask seeds decided by the FP64 re-evaluation in the last mask */
} rf_profile;

typedef struct rf_volume rf_volume;

/* Fills `p` with the defaults described above.  Never fails for p != NULL. */
rf_status rf_default_params(rf_params* p);

/* Creates a voxel-hashed TSDF volume on the current CUDA device (Sec. III-A:
 * blocks allocated on demand, indexed by a spatial hash).  n_buckets must be
 * a power of two (4 slots per bucket); max_blocks <= 4,194,302.  max_width and
 * max_height bound the frames this volume accepts (per-frame scratch is sized
 * from them).  All device memory is allocated here.  On error *out is NULL. */
rf_status rf_create_volume(const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width,
                           int max_height, rf_volume** out);

/* Device bytes rf_create_volume would allocate for these arguments (the same
 * argument checks, no allocation, no device needed): what an admission
 * policy charges against its memory budget.  Equals rf_stats.device_bytes of
 * the created volume. */
rf_status rf_volume_footprint(const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width,
                              int max_height, int64_t* bytes);

/* Synchronises the device and frees everything the volume owns.  NULL is a no-op. */
rf_status rf_destroy_volume(rf_volume* vol);

/* Empties the volume (all blocks freed, frame counter 0; the next frame is
 * integrated at its T_init without tracking); synchronous. */
rf_status rf_volume_reset(rf_volume* vol);

/* Levenberg-Marquardt registration of a frame against the model (Sec. III-B):
 * minimises E = sum V_SDF(exp(xi) T x_i)^2 + w_c sum (V_I(exp(xi) T x_i) - I(p_i))^2
 * (Eq. 2-4) over the pixel strides lm_strides, starting at *T_init_dev.
 * mask_dev (device, nullable): pixels with nonzero mask are excluded (the
 * second registration of Sec. III-C).  T_init_dev/T_out_dev: device double[16]
 * (may alias).  info_dev: device rf_track_info or NULL.  Asynchronous. */
rf_status rf_track_frame(rf_volume* vol, const rf_frame* frame, const double* T_init_dev, const uint8_t* mask_dev,
                         double* T_out_dev, rf_track_info* info_dev, void* stream);

/* Dynamic mask at pose *T_dev (Sec. III-C): residual r_i = V_SDF(T x_i)^2
 * (Eq. 2), seeds r_i > gamma tau^2 (Eq. 5), 3x3 erosion, the depth-aware
 * flood fill of Alg. 1 (4-neighbours, |D(p)-D(n)| < theta D(p)), 3x3
 * dilation.  mask_dev: device uint8 height*width (caller-owned output).
 * Seeds are decided exactly: near the threshold the residual is re-evaluated
 * in FP64 in a fixed operation order.  Asynchronous. */
rf_status rf_compute_mask(rf_volume* vol, const rf_frame* frame, const double* T_dev, uint8_t* mask_dev,
                          void* stream);

/* Same result as rf_compute_mask, for callers that cannot call cudaMalloc
 * when they need a mask: an application whose own allocator or fixed memory
 * budget owns all device memory, or a frame loop with a latency bound that
 * cannot afford cudaMalloc's implicit device synchronisation.  The paper has
 * no counterpart; this is a property of the library only.
 *  - Allocates nothing: the per-call scratch (seed image, flood-fill working
 *    mask, barrier words, sweep flags) is one static device array of about
 *    1.9 MB that every GPU loading this library holds until the process exits.
 *  - Frames of at most 921,600 pixels (1280 x 720); larger frames return
 *    RF_ERR_INVALID_ARG with a message.  The flood fill is bounded by
 *    min(max_ff_sweeps, 4096) sweeps.
 *  - The current device must be the volume's device (RF_ERR_INVALID_ARG
 *    otherwise).  The first call on a device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current; make that first
 *    call before any stream capture.
 *  - All calls share the one array: calls whose GPU work overlaps (other
 *    streams, other volumes, other host threads) race and corrupt each other's
 *    masks.  Serialise them, e.g. on one stream.
 *  - The volume's own scratch is not touched.  Asynchronous like
 *    rf_compute_mask; kernel-detected errors go to rf_sync_status. */
rf_status rf_compute_mask_noalloc(rf_volume* vol, const rf_frame* frame, const double* T_dev, uint8_t* mask_dev,
                                  void* stream);

/* Integrates the frame at pose *T_dev (Sec. III-A running weighted average,
 * Sec. III-D free-space carving): every voxel projecting to a valid, unmasked
 * pixel with z in (z_near, d_max] and sdf = D - z >= -tau is updated with
 * sdf (|sdf| <= tau, colour too) or with tau (sdf > tau: free space).  Blocks
 * holding at least one such voxel are allocated.  Discrete decisions use exact
 * integer arithmetic.  mask_dev nullable.  Asynchronous. */
rf_status rf_integrate_frame(rf_volume* vol, const rf_frame* frame, const double* T_dev, const uint8_t* mask_dev,
                             void* stream);

/* Virtual depth (Sec. III-E, second option).  Call it on a temporary volume
 * that holds the n consecutive frames around the target frame, integrated at
 * their registered poses (the caller builds it with rf_volume_reset and
 * rf_integrate_frame; the paper uses n = 10).  Every zero pixel of
 * frame->depth gets the depth of the first crossing of the volume's TSDF from
 * V > 0 to V <= 0 along the pixel's ray seen from *T_dev: ray samples at
 * z_k = z_near + k voxel/2 (depth along the optical axis) up to d_max, a
 * sample counting when all 8 trilinear corners are observed, the crossing
 * interpolated linearly between the two bracketing samples and rounded to the
 * nearest raw unit.  Zero pixels without a crossing get far_raw (0 selects
 * round(d_max * depth_scale): the clipping plane, so that such rays carve free
 * space up to it); non-zero pixels are copied.  depth_out: device uint16
 * height*width; it may be frame->depth itself (in-place fill).  Decisions are
 * exact: FP32 with an error bound, FP64 re-evaluation near it.  Asynchronous. */
rf_status rf_virtual_depth(rf_volume* vol, const rf_frame* frame, const double* T_dev, int far_raw,
                           uint16_t* depth_out, void* stream);

/* The whole per-frame loop (Fig. 2 / Sec. III-C): track -> mask -> track
 * without masked pixels -> integrate with that pose and mask.  The first frame
 * of an empty volume (new, reset, or imported from an empty snapshot) is
 * integrated at *T_init_dev without tracking.  Device pointers:
 * T_init_dev (in), T_out_dev (out), mask_dev (out, nullable), info_dev (out,
 * nullable; info of the second registration).  The frame is copied into
 * volume-owned staging buffers first, so the caller may reuse its buffers once
 * the stream passes this call.  The device work is replayed from a CUDA graph
 * captured per (frame size, intrinsics, first-frame) combination.
 * Asynchronous. */
rf_status rf_process_frame(rf_volume* vol, const rf_frame* frame, const double* T_init_dev, double* T_out_dev,
                           uint8_t* mask_dev, rf_track_info* info_dev, void* stream);

/* Same loop from HOST buffers: copies depth/rgb/T_init to the device, runs
 * rf_process_frame, copies the pose (and the mask if mask_host != NULL) back
 * and synchronises the stream.  Returns kernel-detected errors too.
 * intrinsics = {fx, fy, cx, cy}. */
rf_status rf_process_frame_host(rf_volume* vol, int height, int width, const double intrinsics[4],
                                const uint16_t* depth_host, const uint8_t* rgb_host, const double T_init_host[16],
                                double T_out_host[16], uint8_t* mask_host, void* stream);

/* Batches: one frame for each of n volumes (independent camera streams, any
 * mix of resolutions and voxel sizes) per call.  Each of the two
 * registrations runs as cooperative launches over groups of at most
 * batch_group tracked streams (rf_launch_config), with one set of CTAs per
 * stream sized by its pixel count (the sets never wait on each other); the
 * residual seeds, erosions and dilations of all streams run as one launch
 * each, the flood fills as one cooperative launch per group, and the
 * integrations of the streams concurrently.  A
 * stream's result is bit-identical to processing it alone with
 * rf_process_frame (partial sums are taken over fixed pixel chunks, not per
 * CTA).
 * rf_batch_create: n <= number of SMs; volumes on the current device, each
 * at most once.  It allocates the batch's streams and events; each new batch
 * shape (frame sizes and intrinsics) captures a graph and allocates its small
 * descriptor buffers on first use.
 * rf_batch_process: frames, T_init_dev, T_out_dev, mask_dev (nullable, and
 * entries nullable) are arrays of n, device pointers as in rf_process_frame.
 * A stream whose frames[i].depth is NULL sits the call out: its volume is left
 * unchanged, T_out_dev[i] receives T_init_dev[i], its mask is not written (its
 * frame's size and intrinsics must still be the stream's).  A stream whose
 * volume is empty is integrated at T_init (as rf_process_frame does).  Which
 * streams track, start or sit out changes per call without a new capture: the
 * call uploads one small table (pointers, modes, the CTA split) and replays
 * the graph.  Asynchronous on `stream`; successive calls on one batch must be
 * ordered (same stream, or synchronised by the caller); kernel-detected errors
 * go to each volume's rf_sync_status.  A batch must not run concurrently with
 * other work on its volumes. */
typedef struct rf_batch rf_batch;
rf_status rf_batch_create(rf_volume* const* vols, int n, rf_batch** out);
rf_status rf_batch_destroy(rf_batch* batch);
rf_status rf_batch_process(rf_batch* batch, const rf_frame* frames, const double* const* T_init_dev,
                           double* const* T_out_dev, uint8_t* const* mask_dev, void* stream);
/* Message of the last failing batch call ("" for NULL). */
const char* rf_batch_last_error(rf_batch* batch);

/* Zero-crossing surface of the TSDF (the mesh of Sec. I) by marching
 * tetrahedra over cells whose 8 corners are observed; triangle soup, normals
 * towards positive SDF.  verts_dev: float [cap_tris][3][3]; colors_dev: uint8
 * [cap_tris][3][3].  With verts_dev == NULL only *n_tris_host is computed.
 * Synchronises `stream` (the count is returned on the host).
 * RF_ERR_BUFFER_TOO_SMALL if the mesh has more than cap_tris triangles. */
rf_status rf_extract_mesh(rf_volume* vol, float* verts_dev, uint8_t* colors_dev, int64_t cap_tris,
                          int64_t* n_tris_host, void* stream);

/* Host snapshot of the volume, blocks sorted by (bz, by, bx); voxel index
 * x + 8y + 64z.  coords int32 [n][3]; F float [n][512] (0 where W = 0);
 * W, wc uint8 [n][512] (SDF and colour weights); rgb uint8 [n][512][3].
 * With coords == NULL only *n_blocks is returned.  Synchronous. */
rf_status rf_volume_export(rf_volume* vol, int64_t cap_blocks, int32_t* coords, float* F, uint8_t* W,
                           uint8_t* rgb, uint8_t* wc, int64_t* n_blocks);

/* Replaces the volume content with a host snapshot in the export layout;
 * with n_blocks > 0 the next frame is tracked against it (eviction to the
 * host and back leaves a stream's results unchanged).  Synchronous. */
rf_status rf_volume_import(rf_volume* vol, int64_t n_blocks, const int32_t* coords, const float* F,
                           const uint8_t* W, const uint8_t* rgb, const uint8_t* wc);

/* Block count, capacity, frames processed, hash load factor and device bytes
 * of the volume: host-side bookkeeping plus one synchronous read of the
 * device block counter (synchronise the volume's stream first to count its
 * last frame). */
rf_status rf_volume_stats(rf_volume* vol, rf_stats* out);

/* Launch shapes of the kernels whose best grid depends on the device and the
 * workload: grid = number of SMs x CTAs per SM, and the stream grouping of batched
 * registrations.  Defaults {16, 8, 2, 8, 16}; the
 * package's autotuner (paper_1905_02082_gb300/autotune.py) measures them on
 * the current GPU and the Python binding applies its table.  Setting them
 * synchronises the device and drops the volume's captured graphs; batches
 * capture the shapes in force (batch_group: the first volume's) when they
 * first see a frame shape. */
typedef struct rf_launch_config {
  int integrate_ctas_per_sm;  /* per-voxel update (k_integrate, 128 threads) */
  int cull_ctas_per_sm;       /* frustum block cull (256 threads) */
  int fixup_ctas_per_sm;      /* neighbour-table fixup (256 threads) */
  int raycast_ctas_per_sm;    /* virtual-depth ray casting (256 threads) */
  int batch_group;            /* batches: tracked streams per registration launch at most, 0 = all in one
                                 (smaller groups keep more of each launch's models in L2; on GB300 for
                                 32 streams four launches of 8 beat one of 32 by ~12 %) */
} rf_launch_config;
rf_status rf_get_launch_config(rf_volume* vol, rf_launch_config* out);
rf_status rf_set_launch_config(rf_volume* vol, const rf_launch_config* cfg);

/* Bounded waits (a property of the library; the paper has no counterpart).
 * Every grid-wide wait of the cooperative kernels (the flood fill's grid
 * barrier; the registration's wait for every CTA's partial sums of a cost
 * evaluation) polls at most spin_limit times before it gives up: the kernel
 * then records RF_ERR_NOT_CONVERGED in the status word (rf_sync_status) and
 * returns, and the volume stays usable.  spin_limit 0 restores the default,
 * 2^24 polls (about one second).  extra_arrivals is fault injection for
 * tests: with extra_arrivals > 0 each wait expects that many arrivals beyond
 * the CTAs launched, which never come, so every wait runs out and the error
 * path is exercised; use 0 otherwise.  Synchronises the device and
 * drops the volume's captured graphs; batches keep the limits in force when
 * they first saw a frame shape. */
rf_status rf_set_wait_limits(rf_volume* vol, int64_t spin_limit, int extra_arrivals);

/* Registration tags (a property of the library; the paper has no
 * counterpart).  Each cost evaluation of a registration publishes its partial
 * sums tagged with a number from a per-volume sequence that only grows, and
 * starts over at 0, with the partial-sum buffer cleared, before it would reach
 * 2^31.  This call sets the sequence's next base (clearing the buffer, so no
 * stale tag can match), which lets tests reach the restart without 2^31
 * evaluations.  base must be at most 2^31 - 1 - (3 + the sum of lm_iters);
 * synchronises the device. */
rf_status rf_set_registration_tag_base(rf_volume* vol, uint32_t base);

/* Enables (1) or disables (0) device timing of the whole-frame calls: CUDA
 * events recorded on the caller's stream (kept inside the captured graphs)
 * around each stage and around the per-voxel update kernel.  Work counters
 * are always kept.  Takes effect for the next frame. */
rf_status rf_set_profiling(rf_volume* vol, int enable);

/* Synchronises `stream` and returns the timings (if profiling is enabled;
 * zeros otherwise) and the work counters of the last frame. */
rf_status rf_get_profile(rf_volume* vol, void* stream, rf_profile* out);

/* Synchronises `stream`, returns the first kernel-detected error since the
 * last call (RF_OK if none) and clears the device status word. */
rf_status rf_sync_status(rf_volume* vol, void* stream);

/* Message of the last failing call on this volume (vol == NULL: last
 * creation error).  The string stays valid until the next call. */
const char* rf_last_error(rf_volume* vol);

const char* rf_status_string(rf_status s);

#ifdef __cplusplus
}
#endif
#endif /* REFUSION_H */
