// Internal device structures of the ReFusion CUDA library (sm_103a).
//
// Model (ReFusion Sec. III-A): a TSDF on a voxel lattice, voxel k at world
// position voxel_size * k, stored sparsely in 8x8x8 blocks addressed through a
// spatial hash.  Per voxel:
//   vox[i].x : SDF value F as float bits; NaN marks a never-observed voxel
//              (this is exactly W == 0, so lookups need not read W)
//   vox[i].y : R | G << 8 | B << 16 | Wc << 24   (RGB8 colour, colour weight)
//   W[i]     : SDF weight (uint8, capped at w_max)
// Block b owns vox[b*512 .. b*512+511], voxel (x,y,z) at index x + 8y + 64z.
//
// Hash: n_buckets buckets of 4 slots; a slot holds one 64-bit word
//   key(42 bits: 14-bit two's complement bx, by, bz) << 22 | pool index (22 bits)
// or ~0 when empty.  Linear probing over buckets, at most kMaxProbe buckets.
// Entries are never deleted, so the first empty slot ends a search, and one
// 64-bit CAS publishes key and value together.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "refusion.h"

namespace rf {

constexpr int kBV = 512;  // voxels per block
constexpr int kSlots = 4;
constexpr unsigned long long kEmpty = ~0ull;
constexpr int kMaxProbe = 64;
constexpr int kMaxCoord = 8191;  // |block coordinate| bound of the 14-bit key fields
constexpr int kMaxPool = (1 << 22) - 2;
constexpr int kTile = 16;           // depth-max tiles used by the frustum cull

// device status bits (OR-ed by kernels, read by rf_sync_status)
enum : unsigned {
  ST_HASH_FULL = 1u,
  ST_POOL_FULL = 2u,
  ST_NOT_CONVERGED = 4u,
  ST_OUT_OF_RANGE = 8u,
  ST_CAPACITY = 16u,
  ST_BARRIER = 32u,
};

struct DevVol {
  unsigned long long* hash;  // n_buckets * kSlots
  unsigned long long bucket_mask;
  uint2* vox;
  uint8_t* W;
  int4* coords;  // block coordinate per pool index
  int4* nbr;     // per pool index, 2 x int4: pools of the blocks at offset (dx,dy,dz) in {0,1}^3,
                 // slot dx + 2 dy + 4 dz (slot 0 = itself), -1 where absent
  int* n_blocks;
  int max_blocks;
  unsigned* status;
};

// Per-volume constants derived from rf_params.
struct DevParams {
  float voxel, inv_voxel, tau, w_c, gamma_tau2;
  float gamma_tau2_f;  // (float)((gamma * tau) * tau), the mask threshold of Eq. 5 in float
  float inv_depth_scale, z_near, d_max;
  double voxel_d, tau_d, gamma_d, depth_scale_d;
  long long v_um, du_um, dmin_um, dmax_um, znear_tick, dmax_tick, tau_tick;
  int w_max;
  long long theta_ppm;
  int storage;    // voxel storage mode (0: FP32, 1: compact FP16)
  float inv_tau;  // 1 / tau (FP16 encoding of F / tau)
  unsigned du_tick;  // ticks (2^-10 um) per raw depth unit
};

// One frame in device memory plus its intrinsics in the three forms used:
// float (tracking), double (exact mask seeds) and quantised integers
// (integration: f*256 and (c+1/2)*256).
struct DevFrame {
  int H, W;
  float fx, fy, cx, cy, ifx, ify;
  double fxd, fyd, cxd, cyd;
  long long fxq, fyq, cxq, cyq;
  // float pixel estimates closer than this to a rounding boundary are decided
  // by the exact integer path (4x the bound on the estimate's error)
  float amb_u, amb_v;
  const uint16_t* depth;
  const uint8_t* rgb;
  // batches only: the stream's per-call mode (kMode*), read by every mask and
  // integration kernel of the stream; nullptr outside batches
  const int* gate;
};

// Per-call mode of a stream in a batch.  Track: the whole path.  First (empty
// volume): no registration or mask, integration at T_init.  Idle (no frame):
// nothing runs.
constexpr int kModeTrack = 0, kModeFirst = 1, kModeIdle = 2;

// True when a gated kernel has no work: the stream's mode is above max_mode.
__device__ __forceinline__ bool gated_off(const int* gate, int max_mode) {
  return gate != nullptr && __ldg(gate) > max_mode;
}

constexpr int kLambdaPow = 24;  // damping exponents k in [-kLambdaPow, kLambdaPow]
struct LMConst {
  double lambda0, eps_t, eps_r;
  float eps_t2f, eps_r2f;  // squared thresholds of the convergence test
  long long min_valid;
  int iters[3], strides[3];
  // lambda0 * 10^k rounded to float, k = -kLambdaPow .. kLambdaPow (the
  // Marquardt damping after k more rejections than acceptances)
  float lambda_pow[2 * kLambdaPow + 1];
};

// Everything one registration needs (one camera stream).
struct RegDesc {
  DevVol v;
  DevFrame f;
  DevParams p;
  const uint8_t* mask;
  const double* T_init;
  double* T_out;
  rf_track_info* info;
  LMConst c;
  // 2 x 29 x max_slots tagged partial sums (double-buffered by evaluation
  // parity; component-major)
  unsigned long long* partials;
  int max_slots;
  // tags[0]: the tag base of the next registration of this volume; tags[1]:
  // CTAs that have left the current one; tags[2]: arrivals at the current
  // one's evaluations (e * G after evaluation e).  The last CTA to leave
  // clears both counts and advances the base past every tag it used.
  unsigned* tags;
  unsigned* status;
  long long spin_limit;  // bound of each wait (polls)
  unsigned bar_extra;    // fault injection: arrivals each wait expects beyond the CTAs launched
  // per full-resolution pixel: the (block key << 22 | pool) its last sample
  // was found in, ~0 when none; a block's pool never changes until the
  // volume is reset or imported, which clear the cache.  nullptr: no cache
  unsigned long long* pxcache;
};

// Quantised pose and the frustum search region of one integration.
struct IntegState {
  long long A[9];  // llround(R^T * 2^30), world -> camera
  long long tq[3]; // llround(t * 1e6), camera centre in micrometres
  float R[9], t[3];
  int bmin[3];
  int dims[3];
  long long total;
  float zfar;
  int clipped;
  int max_um;
  int n_cand;
  int work;
  int new_blocks;
  int pool_before;  // pool size when the integration started (new blocks follow it)
  unsigned ticket;  // CTAs of the frustum search that have finished (reset by the last)
  unsigned long long updated;
  // constant of the per-voxel loop: one voxel step along world z in camera
  // coordinates, as a float estimate in ticks
  float szf[3];
};

// Everything one stream's residual seeds, erosion and dilation need.
struct MaskDesc {
  DevVol v;
  DevFrame f;
  DevParams p;
  const double* T;  // first-registration pose
  uint8_t* seeds;
  unsigned* guard;
  uint8_t* md;
  uint8_t* mask_out;
  const unsigned long long* pxcache;  // the volume's per-pixel block cache (read only)
};

__device__ __forceinline__ bool coord_ok(int bx, int by, int bz) {
  return bx >= -kMaxCoord && bx <= kMaxCoord && by >= -kMaxCoord && by <= kMaxCoord && bz >= -kMaxCoord &&
         bz <= kMaxCoord;
}

__device__ __forceinline__ unsigned long long pack_key(int bx, int by, int bz) {
  return ((unsigned long long)(bx & 0x3FFF) << 28) | ((unsigned long long)(by & 0x3FFF) << 14) |
         (unsigned long long)(bz & 0x3FFF);
}

// Bucket of a packed block key: murmur3's 32-bit finaliser applied to the
// two halves of the key folded together (32-bit integer ops only).
__device__ __forceinline__ unsigned long long bucket_of(unsigned long long key, unsigned long long mask) {
  unsigned k = (unsigned)key ^ ((unsigned)(key >> 32) * 0x9E3779B9u);
  k ^= k >> 16;
  k *= 0x85EBCA6Bu;
  k ^= k >> 13;
  k *= 0xC2B2AE35u;
  k ^= k >> 16;
  return (unsigned long long)k & mask;
}

// Read-only lookup for kernels that do not insert (tracking, mask, mesh).
__device__ __forceinline__ int hash_find(const DevVol& v, int bx, int by, int bz) {
  if (!coord_ok(bx, by, bz)) return -1;
  const unsigned long long key = pack_key(bx, by, bz);
  const unsigned long long b = bucket_of(key, v.bucket_mask);
  for (int p = 0; p < kMaxProbe; ++p) {
    const ulonglong2* bp = reinterpret_cast<const ulonglong2*>(v.hash + ((b + p) & v.bucket_mask) * kSlots);
    const ulonglong2 e01 = __ldg(bp);
    const ulonglong2 e23 = __ldg(bp + 1);
    const unsigned long long e[4] = {e01.x, e01.y, e23.x, e23.y};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (e[s] == kEmpty) return -1;
      if ((e[s] >> 22) == key) return (int)(e[s] & 0x3FFFFF);
    }
  }
  return -1;
}


// x < 2^23 as a float, exactly, without a conversion instruction: the float
// with exponent 2^23 and mantissa x is 2^23 + x, and subtracting 2^23 is exact.
__device__ __forceinline__ float u2f_exact(unsigned x) { return __uint_as_float(0x4B000000u | x) - 8388608.0f; }

// 2126 R + 7152 G + 722 B as a float: the intensity of Sec. III-B times
// 255e4 (exact integer arithmetic, one conversion).
constexpr float kIntensityScale = 1.0f / 2550000.0f;
__device__ __forceinline__ float rgb_intensity_raw(unsigned c) {
  // two 16x8-bit dot products: (2126, 7152) . (R, G) + (722, 0) . (B, byte 3)
  const unsigned s = __dp2a_hi(722u, c, __dp2a_lo(2126u | (7152u << 16), c, 0u));
  return u2f_exact(s);
}

// ---------------------------------------------------------------------------
// Voxel storage.  Mode 0 (FP32): per voxel a uint2 {F float bits (NaN when
// W = 0), R | G<<8 | B<<16 | Wc<<24} plus W in the uint8 array (9 B).
// Mode 1 (compact FP16): the block's 512 uint2 slots hold 512 tracking words
// followed by 512 colour words (8 B per voxel, no W array):
//   tracking word = F16(F / tau) (NaN when W = 0) | I8 << 16 | W << 24,
//   colour word   = R | G<<8 | B<<16 | Wc<<24,
// I8 = round(254 I) of the voxel's colour (Sec. III-B intensity), 255 when
// Wc = 0: tracking gathers 4 bytes per corner and free-space carving
// rewrites 4 bytes per voxel.
// ---------------------------------------------------------------------------
constexpr unsigned kTrkEmpty = 0x00FF7E00u;  // F16 NaN, I8 = 255, W = 0
constexpr float kI8Scale = 1.0f / 254.0f;

__device__ __forceinline__ const unsigned* trk_words(const DevVol& v, int pool) {
  return reinterpret_cast<const unsigned*>(v.vox + (size_t)pool * kBV);
}
__device__ __forceinline__ unsigned* trk_words_rw(const DevVol& v, int pool) {
  return reinterpret_cast<unsigned*>(v.vox + (size_t)pool * kBV);
}

// SDF of a tracking word, in metres: exactly F16 -> float, times tau (one
// float multiply, the value rf_volume_export returns).
__device__ __forceinline__ float trk_sdf(unsigned w, float tau) {
  return __fmul_rn(__half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu))), tau);
}

// I8 of an RGB8 colour: round half up of 254 (2126 R + 7152 G + 722 B) / 2550000.
__device__ __forceinline__ unsigned rgb_i8(unsigned c) {
  const unsigned s = __dp2a_hi(722u, c & 0x00FFFFFFu, __dp2a_lo(2126u | (7152u << 16), c, 0u));
  return (254u * s + 1275000u) / 2550000u;
}

// FP64 lerp in the oracle's operation order (no contraction).
__device__ __forceinline__ double lerp_rn(double a, double b, double t) {
  const double om = __dsub_rn(1.0, t);
  return __dadd_rn(__dmul_rn(a, om), __dmul_rn(b, t));
}

// Fetches the 8 corner SDF values of the cell with lattice origin k; false if
// any corner is missing or unobserved.  FP16 storage: the stored value F16 x
// tau (one float multiply, exactly what rf_volume_export returns).
// Pool of the block holding a lattice corner, from a block's neighbour table
// (n0, n1: slots 0-7, slot dx + 2 dy + 4 dz): sx, sy, sz tell whether the
// corner lies in the next block along x, y, z.  Selects only, so the table
// stays in registers (an indexed array would go to local memory).
__device__ __forceinline__ int nbr_pick(const int4& n0, const int4& n1, bool sx, bool sy, bool sz) {
  const int a = sx ? n0.y : n0.x, b = sx ? n0.w : n0.z;
  const int c = sx ? n1.y : n1.x, e = sx ? n1.w : n1.z;
  const int lo = sy ? b : a, hi = sy ? e : c;
  return sz ? hi : lo;
}

// The SDF values (metres) at the 8 corners n = dx + 2 dy + 4 dz of the
// lattice cell whose corner 0 is voxel (lx, ly, lz) of block `pool`.  All
// loads are issued before any value is tested, so their latencies overlap.
// False if a corner's block is missing or a corner was never observed.
template <int ST>
__device__ __forceinline__ bool corners_at(const DevVol& v, const DevParams& p, int pool, int lx, int ly, int lz,
                                           float F[8]) {
  auto value = [&](int pl, int i) -> float {
    if constexpr (ST == RF_STORAGE_FP32) return __uint_as_float(__ldg(&v.vox[(size_t)pl * kBV + i].x));
    else return trk_sdf(__ldg(trk_words(v, pl) + i), p.tau);
  };
  if (lx < 7 && ly < 7 && lz < 7) {  // all 8 corners in one block
    const int base = lx + 8 * ly + 64 * lz;
#pragma unroll
    for (int n = 0; n < 8; ++n) F[n] = value(pool, base + (n & 1) + 8 * ((n >> 1) & 1) + 64 * ((n >> 2) & 1));
  } else {
    const int4 n0 = __ldg(v.nbr + 2 * (size_t)pool), n1 = __ldg(v.nbr + 2 * (size_t)pool + 1);
    const bool ex = lx == 7, ey = ly == 7, ez = lz == 7;
    int pn[8];
    bool present = true;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      pn[n] = nbr_pick(n0, n1, (n & 1) && ex, ((n >> 1) & 1) && ey, ((n >> 2) & 1) && ez);
      present = present && pn[n] >= 0;
    }
    if (!present) return false;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int ix = (lx + (n & 1)) & 7, iy = (ly + ((n >> 1) & 1)) & 7, iz = (lz + ((n >> 2) & 1)) & 7;
      F[n] = value(pn[n], ix + 8 * iy + 64 * iz);
    }
  }
  bool observed = true;
#pragma unroll
  for (int n = 0; n < 8; ++n) observed = observed && F[n] == F[n];
  return observed;
}

template <int ST>
__device__ __forceinline__ bool corners_of(const DevVol& v, const DevParams& p, int kx, int ky, int kz, float F[8]) {
  const int pool = hash_find(v, kx >> 3, ky >> 3, kz >> 3);
  if (pool < 0) return false;
  return corners_at<ST>(v, p, pool, kx & 7, ky & 7, kz & 7, F);
}

// The same with a per-pixel cache of (block key << 22 | pool) entries: a
// matching entry saves the hash probe (entries of other blocks are ignored).
template <int ST>
__device__ __forceinline__ bool corners_cached(const DevVol& v, const DevParams& p, int kx, int ky, int kz,
                                               unsigned long long cached, float F[8]) {
  const int bx = kx >> 3, by = ky >> 3, bz = kz >> 3;
  int pool;
  if (cached != kEmpty && coord_ok(bx, by, bz) && (cached >> 22) == pack_key(bx, by, bz))
    pool = (int)(cached & 0x3FFFFFull);
  else
    pool = hash_find(v, bx, by, bz);
  if (pool < 0) return false;
  return corners_at<ST>(v, p, pool, kx & 7, ky & 7, kz & 7, F);
}

__device__ __forceinline__ bool pixel_valid(const DevParams& p, unsigned raw) {
  if (p.du_um < 32768) {  // raw * du fits 31 bits
    const int D = (int)raw * (int)p.du_um;
    return raw != 0 && D >= (int)p.dmin_um && D <= (int)p.dmax_um;
  }
  const long long D = (long long)raw * p.du_um;
  return raw != 0 && D >= p.dmin_um && D <= p.dmax_um;
}

// Default bound of a grid-barrier wait: 2^24 polls (after the first 4,096 each
// followed by a 64 ns sleep), about one second.
constexpr long long kDefaultSpinLimit = 1ll << 24;

// Grid-wide barrier for cooperative launches (all CTAs co-resident).  The
// spin is bounded: after spin_limit polls it records ST_BARRIER and returns
// false, and callers then leave the kernel.  extra > 0 (fault injection for
// tests) makes the barrier wait for arrivals that never come.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* status, long long spin_limit,
                                             unsigned extra) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned ticket = atomicAdd(bar, 1u);
    int ok = 1;
    if (ticket == nblocks + extra - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (++spins > spin_limit) {
          ok = 0;
          atomicOr(status, ST_BARRIER);
          break;
        }
        if (spins > 4096) __nanosleep(64);  // spin first: most waits are short
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Registration exchange.  Every CTA of a registration writes its partial
// sums of an evaluation as 64-bit words, the float in the low half and the
// evaluation's tag in the high half, then counts itself in an arrival counter
// with a relaxed reduction, and waits (one thread polling) until the count
// shows every CTA.  No fence orders the partials before the count (a release
// there cost a full L2 round trip per evaluation): the readers check each
// word's tag instead and read again the rare word that has not arrived.  A
// 64-bit access is single-copy atomic, so a word that shows the tag also
// shows the partial written with it.
//
// Accesses are relaxed at GPU scope (L1 bypassed).  On this GPU an acquire
// at GPU scope also invalidates the SM's L1, which holds the model the
// registration's samples gather; with one wait per cost evaluation every
// evaluation would start with a cold L1 (measured: the first sample's lookup
// took 2-5k cycles).  Nothing read after the wait needs it: the model is not
// written while the registration runs.  (Letting every thread poll its
// partials directly, without the count, was measured slower: tens of
// thousands of polling threads congest the L2 slices the stragglers need.)
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_relaxed_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Polls *count until it reaches target, at most spin_limit times (after the
// first 4,096 polls each followed by a 64 ns sleep); false when the wait ran
// out.
__device__ __forceinline__ bool await_count(const unsigned* count, unsigned target, long long spin_limit) {
  long long spins = 0;
  while (ld_relaxed_gpu(count) < target) {
    if (++spins > spin_limit) return false;
    if (spins > 4096) __nanosleep(64);
  }
  return true;
}

// Waits until the tagged word *p (last read into v) carries tag `want`,
// re-polling at most spin_limit times (the same schedule); false when the
// wait ran out.
__device__ __forceinline__ bool await_tag(const unsigned long long* p, unsigned long long& v, unsigned want,
                                          long long spin_limit) {
  long long spins = 0;
  while ((unsigned)(v >> 32) != want) {
    if (++spins > spin_limit) return false;
    if (spins > 4096) __nanosleep(64);
    v = ld_relaxed_gpu_u64(p);
  }
  return true;
}

// Tags stay below 2^31.
constexpr unsigned kTagLimit = 0x80000000u;

}  // namespace rf

// Host-side helpers shared by the translation units.
struct rf_volume;
namespace rf {
DevFrame make_dev_frame(const rf_frame* f);
bool frame_ok(const rf_volume* vol, const rf_frame* f);
rf_status set_error(rf_volume* vol, rf_status s, const char* fmt, ...);
rf_status check_cuda(rf_volume* vol, cudaError_t e, const char* what);
// stage launchers (stream-ordered, no host synchronisation)
rf_status launch_track(rf_volume* vol, const DevFrame& f, const double* T_init, const uint8_t* mask, double* T_out,
                       rf_track_info* info, cudaStream_t st);
rf_status launch_mask(rf_volume* vol, const DevFrame& f, const double* T, uint8_t* mask_out, cudaStream_t st);
rf_status launch_virtual_depth(rf_volume* vol, const DevFrame& f, const double* T, unsigned far_raw, uint16_t* out,
                               cudaStream_t st);
rf_status launch_integrate(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st);
// residual seeds + erosion, and dilation, of several streams in one launch
// each (grid y = stream; max_npix bounds every stream's pixel count; the
// guard counts and flood-fill words are reset by the caller)
MaskDesc make_mask_desc(rf_volume* vol, const DevFrame& f, const double* T, uint8_t* mask_out);
rf_status launch_mask_pre_batch(rf_volume* vol, const MaskDesc* descs, int n, int max_npix, cudaStream_t st);
rf_status launch_mask_post_batch(rf_volume* vol, const MaskDesc* descs, int n, int max_npix, cudaStream_t st);
// profiling events (no-ops unless profiling is enabled); ids below
enum ProfEvent { EV_FRAME0, EV_TRACK1_END, EV_MASK_END, EV_TRACK2_END, EV_INTEG0, EV_KERNEL0, EV_KERNEL1, EV_FRAME1,
                 EV_COUNT };
void prof_record(rf_volume* vol, int ev, cudaStream_t st);
rf_status run_mesh(rf_volume* vol, float* verts, uint8_t* colors, int64_t cap, int64_t* n, cudaStream_t st);
RegDesc make_reg_desc(rf_volume* vol, const DevFrame& f, const double* T_init, const uint8_t* mask, double* T_out,
                      rf_track_info* info);
rf_status launch_register_batch(rf_volume* vol, const RegDesc* descs, const int* cta_stream, const int* first,
                                int total_ctas, cudaStream_t st);
// the three parts of launch_mask (the flood fill is the cooperative one)
rf_status launch_mask_pre(rf_volume* vol, const DevFrame& f, const double* T, cudaStream_t st);
rf_status launch_mask_ff(rf_volume* vol, const DevFrame& f, cudaStream_t st);
// flood fills of several streams in one cooperative launch (the batches'
// CTA maps; total_ctas must not exceed floodfill_max_grid)
struct FloodDesc {
  uint8_t* md;
  const uint16_t* depth;
  int H, W;
  long long theta_ppm;
  unsigned* ff;
  int max_sweeps;
  unsigned* status;
  long long spin_limit;
  unsigned bar_extra;
};
FloodDesc make_flood_desc(rf_volume* vol, const DevFrame& f);
rf_status launch_floodfill_batch(rf_volume* vol, const FloodDesc* descs, const int* cta_stream, const int* first,
                                 int total_ctas, cudaStream_t st);
rf_status launch_mask_post(rf_volume* vol, const DevFrame& f, uint8_t* mask_out, cudaStream_t st);
// neighbour tables of the blocks allocated since *lo_ptr (or since lo when lo_ptr is null)
rf_status launch_nbr_fixup(rf_volume* vol, const int* lo_ptr, int lo, cudaStream_t st, const int* gate = nullptr);
}  // namespace rf
