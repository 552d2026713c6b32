// C entry points of refusion.h: volume lifecycle, argument checking, error
// reporting, snapshots and the whole-frame pipeline (ReFusion Fig. 2:
// track -> mask -> track without masked pixels -> integrate), which is
// captured once per frame geometry into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rf_cta_map.hpp"
#include "rf_half.hpp"
#include "rf_volume.hpp"

namespace rf {
int floodfill_max_grid(int device);
int register_max_grid(int device);

static thread_local std::string g_create_error;

rf_status set_error(rf_volume* vol, rf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (vol) vol->last_error = buf;
  else g_create_error = buf;
  return s;
}

rf_status check_cuda(rf_volume* vol, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RF_OK;
  return set_error(vol, RF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

DevFrame make_dev_frame(const rf_frame* f) {
  DevFrame d;
  d.H = f->height;
  d.W = f->width;
  d.fx = (float)f->fx;
  d.fy = (float)f->fy;
  d.cx = (float)f->cx;
  d.cy = (float)f->cy;
  d.ifx = (float)(1.0 / f->fx);
  d.ify = (float)(1.0 / f->fy);
  d.fxd = f->fx;
  d.fyd = f->fy;
  d.cxd = f->cx;
  d.cyd = f->cy;
  d.fxq = llround(f->fx * 256.0);
  d.fyq = llround(f->fy * 256.0);
  d.cxq = llround((f->cx + 0.5) * 256.0);
  d.cyq = llround((f->cy + 0.5) * 256.0);
  // |estimate - exact| <= 6e-7 |f x / z| + 2.5e-4 px, with |f x / z| bounded by
  // the image extent around the principal point (see the integration kernel)
  d.amb_u = (float)(4.0 * (6e-7 * 2.0 * (f->width + std::fabs(f->cx)) + 2.5e-4));
  d.amb_v = (float)(4.0 * (6e-7 * 2.0 * (f->height + std::fabs(f->cy)) + 2.5e-4));
  d.depth = f->depth;
  d.rgb = f->rgb;
  d.gate = nullptr;
  return d;
}

void prof_record(rf_volume* vol, int ev, cudaStream_t st) {
  if (!vol->profiling) return;
  // External records stay event-record nodes when captured into a graph;
  // outside a capture the flag is refused, so a plain record is taken there.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(vol->ev[ev], st, cudaEventRecordExternal);
  else
    cudaEventRecord(vol->ev[ev], st);
}

bool frame_ok(const rf_volume* vol, const rf_frame* f) {
  if (!f || !f->depth || !f->rgb) return false;
  if (f->height <= 0 || f->width <= 0 || f->height > vol->max_h || f->width > vol->max_w) return false;
  if (!(f->fx > 0.0 && f->fy > 0.0 && f->fx < 4096.0 && f->fy < 4096.0)) return false;
  if (!(std::fabs(f->cx) < 8192.0 && std::fabs(f->cy) < 8192.0)) return false;
  return true;
}

}  // namespace rf

using namespace rf;

namespace {

template <class T>
rf_status dalloc(rf_volume* vol, T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return set_error(vol, RF_ERR_CUDA, "cudaMalloc(%s, %zu bytes): %s", what, count * sizeof(T),
                                         cudaGetErrorString(e));
  vol->device_bytes += count * sizeof(T);
  return RF_OK;
}

bool is_integer(double x) { return std::fabs(x - std::llround(x)) < 1e-6; }

rf_status validate_params(const rf_params* p) {
  if (!(p->voxel_size > 0.0 && p->voxel_size <= 0.15) || !is_integer(p->voxel_size * 1e6))
    return set_error(nullptr, RF_ERR_INVALID_ARG,
                     "voxel_size must be a positive whole number of micrometres, at most 0.15 m");
  if (!(p->trunc > 0.0 && p->trunc < 2.0)) return set_error(nullptr, RF_ERR_INVALID_ARG, "trunc must be in (0, 2) m");
  if (!(p->depth_scale > 0.0) || !is_integer(1e6 / p->depth_scale))
    return set_error(nullptr, RF_ERR_INVALID_ARG, "1e6/depth_scale must be an integer");
  if (!(p->d_min >= 0.0 && p->d_max > p->d_min && p->d_max <= 50.0))
    return set_error(nullptr, RF_ERR_INVALID_ARG, "need 0 <= d_min < d_max <= 50 m");
  if (!(p->z_near > 0.0 && p->z_near < p->d_max)) return set_error(nullptr, RF_ERR_INVALID_ARG, "z_near out of range");
  if (p->w_max < 1 || p->w_max > 255) return set_error(nullptr, RF_ERR_INVALID_ARG, "w_max must be in 1..255");
  if (!(p->gamma >= 0.0 && p->gamma <= 1.0)) return set_error(nullptr, RF_ERR_INVALID_ARG, "gamma must be in [0,1]");
  if (!(p->theta >= 0.0 && p->theta < 1.0)) return set_error(nullptr, RF_ERR_INVALID_ARG, "theta must be in [0,1)");
  if (!(p->w_c >= 0.0)) return set_error(nullptr, RF_ERR_INVALID_ARG, "w_c must be >= 0");
  for (int l = 0; l < 3; ++l) {
    if (p->lm_iters[l] < 0 || p->lm_iters[l] > 1000) return set_error(nullptr, RF_ERR_INVALID_ARG, "lm_iters");
    if (p->lm_strides[l] < 1 || p->lm_strides[l] > 64) return set_error(nullptr, RF_ERR_INVALID_ARG, "lm_strides");
  }
  if (p->max_ff_sweeps < 1 || p->max_ff_sweeps > (1 << 20))
    return set_error(nullptr, RF_ERR_INVALID_ARG, "max_ff_sweeps");
  if (p->max_candidates < 1 || p->max_candidates > (int64_t)1 << 28)
    return set_error(nullptr, RF_ERR_INVALID_ARG, "max_candidates");
  if (p->storage != RF_STORAGE_FP32 && p->storage != RF_STORAGE_FP16)
    return set_error(nullptr, RF_ERR_INVALID_ARG, "storage must be RF_STORAGE_FP32 or RF_STORAGE_FP16");
  return RF_OK;
}

rf_status check_volume_args(const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width, int max_height) {
  rf_status s = validate_params(p);
  if (s) return s;
  if (n_buckets < 1 || (n_buckets & (n_buckets - 1)) != 0 || n_buckets > ((int64_t)1 << 30))
    return set_error(nullptr, RF_ERR_INVALID_ARG, "n_buckets must be a power of two <= 2^30");
  if (max_blocks < 1 || max_blocks > kMaxPool) return set_error(nullptr, RF_ERR_INVALID_ARG, "max_blocks out of range");
  if (max_width < 1 || max_height < 1 || max_width > 8192 || max_height > 8192)
    return set_error(nullptr, RF_ERR_INVALID_ARG, "frame size out of range");
  return RF_OK;
}

// Every device buffer of a volume, in one list: rf_create_volume allocates
// them, rf_volume_footprint adds up their sizes.
template <class Alloc>
rf_status volume_buffers(rf_volume* vol, const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width,
                         int max_height, Alloc&& A) {
  const size_t npix = (size_t)max_width * max_height;
  // partial-sum slots per component: the chunks of the smallest registration
  // chunk (128 pixels)
  const size_t max_slots = (npix + 127) / 128;
  const size_t ntiles = ((size_t)(max_width + kTile - 1) / kTile) * ((max_height + kTile - 1) / kTile);
  const size_t nslots = (size_t)n_buckets * kSlots;
  rf_status s;
  if ((s = A(&vol->d_hash, nslots, "hash")) || (s = A(&vol->d_vox, (size_t)max_blocks * kBV, "voxels")) ||
      (s = A(&vol->d_W, p->storage == RF_STORAGE_FP32 ? (size_t)max_blocks * kBV : 1, "weights")) ||
      (s = A(&vol->d_coords, (size_t)max_blocks, "coords")) ||
      (s = A(&vol->d_nbr, 2 * (size_t)max_blocks, "neighbour tables")) || (s = A(&vol->d_nblocks, 1, "pool")) ||
      (s = A(&vol->d_status, 1, "status")) || (s = A(&vol->d_regtags, 3, "registration tags")) ||
      (s = A(&vol->d_partials, 2 * 29 * max_slots, "partials")) || (s = A(&vol->d_seeds, npix, "seeds")) ||
      (s = A(&vol->d_md, npix, "mask work")) || (s = A(&vol->d_ff, (size_t)p->max_ff_sweeps + 2, "flood-fill words")) ||
      (s = A(&vol->d_integ, 1, "integ")) || (s = A(&vol->d_tilemax, ntiles, "tiles")) ||
      (s = A(&vol->d_dmask, npix, "masked depth")) ||
      (s = A(&vol->d_cand, (size_t)p->max_candidates, "candidates")) || (s = A(&vol->d_depth, npix, "depth staging")) ||
      (s = A(&vol->d_rgb, npix * 3, "rgb staging")) || (s = A(&vol->d_mask, npix, "mask staging")) ||
      (s = A(&vol->d_T, 48, "poses")) || (s = A(&vol->d_info, 1, "info")) || (s = A(&vol->d_guard, 1, "guard count")) ||
      (s = A(&vol->d_pxcache, npix, "pixel block cache")))
    return s;
  return RF_OK;
}


DevParams derive(const rf_params& p) {
  DevParams d;
  d.voxel = (float)p.voxel_size;
  d.inv_voxel = (float)(1.0 / p.voxel_size);
  d.tau = (float)p.trunc;
  d.w_c = (float)p.w_c;
  d.gamma_tau2 = (float)(p.gamma * p.trunc * p.trunc);
  d.gamma_tau2_f = (float)((p.gamma * p.trunc) * p.trunc);
  d.inv_depth_scale = (float)(1.0 / p.depth_scale);
  d.z_near = (float)p.z_near;
  d.d_max = (float)p.d_max;
  d.voxel_d = p.voxel_size;
  d.tau_d = p.trunc;
  d.gamma_d = p.gamma;
  d.depth_scale_d = p.depth_scale;
  d.v_um = llround(p.voxel_size * 1e6);
  d.du_um = llround(1e6 / p.depth_scale);
  d.dmin_um = llround(p.d_min * 1e6);
  d.dmax_um = llround(p.d_max * 1e6);
  d.znear_tick = llround(p.z_near * 1e6) * 1024;
  d.dmax_tick = d.dmax_um * 1024;
  d.tau_tick = llround(p.trunc * 1e6 * 1024.0);
  d.w_max = p.w_max;
  d.theta_ppm = llround(p.theta * 1e6);
  d.storage = p.storage;
  d.inv_tau = (float)(1.0 / p.trunc);
  d.du_tick = (unsigned)(d.du_um * 1024);
  return d;
}

__global__ void k_fill_u64(unsigned long long* p, size_t n, unsigned long long v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_import(DevVol v, const int4* __restrict__ coords, int n, int base) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = base + j;
  const int4 c = coords[j];
  if (!coord_ok(c.x, c.y, c.z)) {
    atomicOr(v.status, ST_OUT_OF_RANGE);
    return;
  }
  const unsigned long long key = pack_key(c.x, c.y, c.z);
  const unsigned long long b = bucket_of(key, v.bucket_mask);
  for (int pr = 0; pr < kMaxProbe; ++pr) {
    unsigned long long* bp = v.hash + ((b + pr) & v.bucket_mask) * kSlots;
    for (int s = 0; s < kSlots; ++s) {
      const unsigned long long prev = atomicCAS(bp + s, kEmpty, (key << 22) | (unsigned long long)i);
      if (prev == kEmpty) {
        v.coords[i] = make_int4(c.x, c.y, c.z, 1);
        return;
      }
      if ((prev >> 22) == key) return;  // duplicate coordinate in the snapshot: first one wins
    }
  }
  atomicOr(v.status, ST_HASH_FULL);
}

rf_status clear_model(rf_volume* vol, cudaStream_t st) {
  const size_t n = (size_t)vol->n_buckets * kSlots;
  k_fill_u64<<<vol->sm_count * 4, 256, 0, st>>>(vol->d_hash, n, kEmpty);
  rf_status s = check_cuda(vol, cudaGetLastError(), "hash clear");
  if (s) return s;
  if ((s = check_cuda(vol, cudaMemsetAsync(vol->d_nblocks, 0, sizeof(int), st), "pool reset"))) return s;
  if ((s = check_cuda(vol, cudaMemsetAsync(vol->d_coords, 0, sizeof(int4) * vol->max_blocks, st), "coords reset")))
    return s;
  // pools are reassigned from now on: forget every pixel's cached block
  if ((s = check_cuda(vol, cudaMemsetAsync(vol->d_pxcache, 0xFF,
                                           sizeof(unsigned long long) * (size_t)vol->max_w * vol->max_h, st),
                      "pixel cache reset")))
    return s;
  return RF_OK;
}

rf_status status_from_bits(rf_volume* vol, unsigned bits) {
  if (bits == 0) return RF_OK;
  if (bits & ST_HASH_FULL) return set_error(vol, RF_ERR_HASH_FULL, "hash table full (bounded probe exhausted)");
  if (bits & ST_POOL_FULL) return set_error(vol, RF_ERR_POOL_FULL, "block pool full (max_blocks reached)");
  if (bits & ST_CAPACITY) return set_error(vol, RF_ERR_CAPACITY, "frustum candidate list overflow");
  if (bits & ST_OUT_OF_RANGE) return set_error(vol, RF_ERR_OUT_OF_RANGE, "block coordinate outside +-8191");
  if (bits & ST_BARRIER) return set_error(vol, RF_ERR_NOT_CONVERGED, "grid-wide wait timed out (flood-fill barrier or registration partial sums)");
  if (bits & ST_NOT_CONVERGED) return set_error(vol, RF_ERR_NOT_CONVERGED, "flood fill exceeded max_ff_sweeps");
  return set_error(vol, RF_ERR_CUDA, "unknown device status 0x%x", bits);
}

// Enqueues the device work of one whole frame on `st`, reading the staging
// buffers of the volume only (so that it can be captured into a graph).
rf_status enqueue_frame(rf_volume* vol, const DevFrame& f, bool first, cudaStream_t st) {
  double* Tin = vol->d_T;
  double* T1 = vol->d_T + 16;
  double* T2 = vol->d_T + 32;
  rf_status s;
  prof_record(vol, EV_FRAME0, st);
  if (first) {
    if ((s = check_cuda(vol, cudaMemsetAsync(vol->d_mask, 0, (size_t)f.H * f.W, st), "mask clear"))) return s;
    prof_record(vol, EV_TRACK1_END, st);
    prof_record(vol, EV_MASK_END, st);
    prof_record(vol, EV_TRACK2_END, st);
    prof_record(vol, EV_INTEG0, st);
    if ((s = launch_integrate(vol, f, Tin, nullptr, st))) return s;
    s = check_cuda(vol, cudaMemcpyAsync(T2, Tin, 16 * sizeof(double), cudaMemcpyDeviceToDevice, st), "pose copy");
    prof_record(vol, EV_FRAME1, st);
    return s;
  }
  if ((s = launch_track(vol, f, Tin, nullptr, T1, nullptr, st))) return s;
  prof_record(vol, EV_TRACK1_END, st);
  if ((s = launch_mask(vol, f, T1, vol->d_mask, st))) return s;
  prof_record(vol, EV_MASK_END, st);
  if ((s = launch_track(vol, f, T1, vol->d_mask, T2, vol->d_info, st))) return s;
  prof_record(vol, EV_TRACK2_END, st);
  prof_record(vol, EV_INTEG0, st);
  s = launch_integrate(vol, f, T2, vol->d_mask, st);
  prof_record(vol, EV_FRAME1, st);
  return s;
}

constexpr size_t kMaxGraphs = 16;  // captured shapes kept per volume and per batch

rf_status frame_graph(rf_volume* vol, const rf_frame* fr, bool first, cudaGraphExec_t* out) {
  for (const auto& g : vol->graphs)
    if (g.H == fr->height && g.W == fr->width && g.fx == fr->fx && g.fy == fr->fy && g.cx == fr->cx &&
        g.cy == fr->cy && g.first == (int)first && g.profiling == (int)vol->profiling) {
      *out = g.exec;
      return RF_OK;
    }
  rf_frame staged = *fr;
  staged.depth = vol->d_depth;
  staged.rgb = vol->d_rgb;
  const DevFrame f = make_dev_frame(&staged);
  cudaStream_t cap;
  rf_status s = check_cuda(vol, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
  if (s) return s;
  s = check_cuda(vol, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (s) {
    cudaStreamDestroy(cap);
    return s;
  }
  rf_status es = enqueue_frame(vol, f, first, cap);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (es) {
    if (graph) cudaGraphDestroy(graph);
    return es;
  }
  if ((s = check_cuda(vol, ce, "end capture"))) return s;
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if ((s = check_cuda(vol, ce, "graph instantiate"))) return s;
  if (vol->graphs.size() >= kMaxGraphs) {
    // the oldest shape goes; it may still be running (a rare event: wait)
    if ((s = check_cuda(vol, cudaDeviceSynchronize(), "graph eviction sync"))) {
      cudaGraphExecDestroy(exec);
      return s;
    }
    cudaGraphExecDestroy(vol->graphs.front().exec);
    vol->graphs.erase(vol->graphs.begin());
  }
  vol->graphs.push_back(
      rf_graph_entry{fr->height, fr->width, fr->fx, fr->fy, fr->cx, fr->cy, (int)first, (int)vol->profiling, exec});
  *out = exec;
  return RF_OK;
}

// Replays the captured graph, or enqueues the kernels directly when graphs
// are disabled (RF_NO_GRAPHS=1 in the environment at volume creation).
rf_status run_frame(rf_volume* vol, const rf_frame* fr, bool first, cudaGraphExec_t exec, cudaStream_t st) {
  if (exec) return check_cuda(vol, cudaGraphLaunch(exec, st), "graph launch");
  rf_frame staged = *fr;
  staged.depth = vol->d_depth;
  staged.rgb = vol->d_rgb;
  return enqueue_frame(vol, make_dev_frame(&staged), first, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// batches: one frame for each of several volumes (independent camera streams)
// ---------------------------------------------------------------------------
// Per-stream, per-call part of a batch, uploaded with one copy before each
// replay: the staging kernel copies the caller's frame and pose into the
// volume, the output kernel copies the pose (and mask) back.
struct BatchStage {
  const uint16_t* depth_src;  // NULL: the stream sits this batch out
  const uint8_t* rgb_src;
  const double* T_src;
  uint16_t* depth_dst;
  uint8_t* rgb_dst;
  double* T_dst;  // the volume's [3][16] poses
  double* T_out;
  uint8_t* mask_out;  // nullable
  uint8_t* mask_buf;  // the volume's mask (zeroed for a first frame: nothing is masked)
  unsigned* guard;    // the volume's seed guard count and flood-fill words, zeroed
  unsigned* ff;       // for a tracked frame
  int ff_words;
  int npix;
  int mode;  // kModeTrack, kModeFirst or kModeIdle; the gate of the stream's kernels
};

struct rf_batch_graph {
  std::vector<double> sig;  // per stream: H, W, fx, fy, cx, cy
  cudaGraphExec_t exec = nullptr;
  RegDesc* d_desc = nullptr;   // [2][n]: first and second registration
  FloodDesc* d_flood = nullptr;  // [n]: the flood fills
  MaskDesc* d_mask = nullptr;    // [n]: seeds, erosion, dilation
  // [n] BatchStage, then per registration launch (ngroups of them): CTA ->
  // stream [total], then the n + 1 group starts
  void* d_table = nullptr;
  std::vector<unsigned char> h_table;
  int total_ctas = 0;
  int ngroups = 1;  // registration launches per registration
  int gsize = 1;    // tracked streams per launch at most
  int ff_ctas = 0;  // CTAs of a batched flood-fill launch (its own maps follow the registration's)
};

struct rf_batch {
  std::vector<rf_volume*> vols;
  int device = 0;
  static constexpr int kAux = 8;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kAux] = {};
  std::vector<rf_batch_graph> graphs;
  std::string last_error;
};

namespace {

__device__ __forceinline__ void copy_bytes(void* dst, const void* src, size_t n, size_t tid, size_t nth) {
  const bool vec = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
  size_t done = 0;
  if (vec) {
    const size_t n16 = n / 16;
    const uint4* s4 = static_cast<const uint4*>(src);
    uint4* d4 = static_cast<uint4*>(dst);
    for (size_t i = tid; i < n16; i += nth) d4[i] = __ldg(s4 + i);
    done = n16 * 16;
  }
  const uint8_t* s1 = static_cast<const uint8_t*>(src);
  uint8_t* d1 = static_cast<uint8_t*>(dst);
  for (size_t i = done + tid; i < n; i += nth) d1[i] = s1[i];
}

__device__ __forceinline__ void zero_bytes(void* dst, size_t n, size_t tid, size_t nth) {
  uint8_t* d1 = static_cast<uint8_t*>(dst);
  size_t done = 0;
  if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    uint4* d4 = static_cast<uint4*>(dst);
    for (size_t i = tid; i < n / 16; i += nth) d4[i] = make_uint4(0, 0, 0, 0);
    done = n / 16 * 16;
  }
  for (size_t i = done + tid; i < n; i += nth) d1[i] = 0;
}

// grid (x, n streams): frame and pose of every stream into its volume.
__global__ void __launch_bounds__(256) k_batch_stage(const BatchStage* __restrict__ table) {
  const BatchStage& b = table[blockIdx.y];
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
  if (b.mode != kModeIdle) {
    copy_bytes(b.depth_dst, b.depth_src, (size_t)b.npix * 2, tid, nth);
    copy_bytes(b.rgb_dst, b.rgb_src, (size_t)b.npix * 3, tid, nth);
  }
  if (b.mode == kModeFirst) zero_bytes(b.mask_buf, (size_t)b.npix, tid, nth);
  if (b.mode == kModeTrack && blockIdx.x == 0) {
    for (int k = threadIdx.x; k < b.ff_words; k += blockDim.x) b.ff[k] = 0u;
    if (threadIdx.x == 0) *b.guard = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < 48) {
    const int k = threadIdx.x;
    if (k < 16 || b.mode != kModeTrack) b.T_dst[k] = b.T_src[k & 15];
  }
}

// grid (x, n streams): final pose (and mask) of every stream to the caller.
__global__ void __launch_bounds__(256) k_batch_out(const BatchStage* __restrict__ table) {
  const BatchStage& b = table[blockIdx.y];
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
  if (b.mask_out && b.mode != kModeIdle) copy_bytes(b.mask_out, b.mask_buf, (size_t)b.npix, tid, nth);
  if (blockIdx.x == 0 && threadIdx.x < 16) b.T_out[threadIdx.x] = b.T_dst[32 + threadIdx.x];
}

rf_status batch_error(rf_batch* b, rf_status s, const std::string& msg) {
  b->last_error = msg;
  return s;
}

// Releases a captured batch graph and its device descriptors (not running).
void free_batch_graph(rf_batch_graph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  void* dev[] = {g.d_desc, g.d_table, g.d_flood, g.d_mask};
  for (void* p : dev)
    if (p) cudaFree(p);
  g = rf_batch_graph();
}

// Fork: every auxiliary stream waits for the work enqueued on cs so far.
void fork_aux(rf_batch* b, cudaStream_t cs) {
  cudaEventRecord(b->fork_ev, cs);
  for (int k = 0; k < rf_batch::kAux; ++k) cudaStreamWaitEvent(b->aux[k], b->fork_ev, 0);
}

// Join: cs waits for every auxiliary stream.
void join_aux(rf_batch* b, cudaStream_t cs) {
  for (int k = 0; k < rf_batch::kAux; ++k) {
    cudaEventRecord(b->join_ev[k], b->aux[k]);
    cudaStreamWaitEvent(cs, b->join_ev[k], 0);
  }
}

size_t table_bytes(int n, int total_ctas, int ff_ctas, int ngroups) {
  return sizeof(BatchStage) * n + sizeof(int) * (size_t)ngroups * ((total_ctas + n + 1) + (ff_ctas + n + 1));
}

// Captures the batch graph for one shape.  Every stream gets the full path;
// which streams actually track is decided per replay by the uploaded table.
rf_status batch_capture(rf_batch* b, const rf_frame* frames, const std::vector<double>& sig, rf_batch_graph* out) {
  const int n = (int)b->vols.size();
  out->total_ctas = b->vols[0]->reg_grid;
  // the tracked streams of a call run in groups of at most gsize per
  // registration launch (launch setting batch_group; 0: all in one)
  const int bg = b->vols[0]->launch.batch_group;
  out->gsize = bg > 0 ? std::min(bg, n) : n;
  out->ngroups = (n + out->gsize - 1) / out->gsize;
  out->ff_ctas = b->vols[0]->ff_grid;
  out->h_table.assign(table_bytes(n, out->total_ctas, out->ff_ctas, out->ngroups), 0);
  cudaError_t e = cudaMalloc(&out->d_table, out->h_table.size());
  if (e != cudaSuccess) return batch_error(b, RF_ERR_CUDA, std::string("batch table: ") + cudaGetErrorString(e));
  const void* out_table = out->d_table;
  std::vector<DevFrame> f(n);
  std::vector<RegDesc> desc(2 * n);
  for (int i = 0; i < n; ++i) {
    rf_volume* v = b->vols[i];
    rf_frame staged = frames[i];
    staged.depth = v->d_depth;
    staged.rgb = v->d_rgb;
    f[i] = make_dev_frame(&staged);
    f[i].gate = reinterpret_cast<const int*>(static_cast<const char*>(out_table) + i * sizeof(BatchStage) +
                                             offsetof(BatchStage, mode));
    desc[i] = make_reg_desc(v, f[i], v->d_T, nullptr, v->d_T + 16, nullptr);
    desc[n + i] = make_reg_desc(v, f[i], v->d_T + 16, v->d_mask, v->d_T + 32, v->d_info);
  }
  std::vector<FloodDesc> flood(n);
  std::vector<MaskDesc> mdesc(n);
  for (int i = 0; i < n; ++i) {
    rf_volume* v = b->vols[i];
    flood[i] = make_flood_desc(v, f[i]);
    mdesc[i] = make_mask_desc(v, f[i], v->d_T + 16, v->d_mask);
  }
  e = cudaMalloc(&out->d_desc, sizeof(RegDesc) * desc.size());
  if (e == cudaSuccess) e = cudaMemcpy(out->d_desc, desc.data(), sizeof(RegDesc) * desc.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&out->d_flood, sizeof(FloodDesc) * n);
  if (e == cudaSuccess) e = cudaMemcpy(out->d_flood, flood.data(), sizeof(FloodDesc) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&out->d_mask, sizeof(MaskDesc) * n);
  if (e == cudaSuccess) e = cudaMemcpy(out->d_mask, mdesc.data(), sizeof(MaskDesc) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return batch_error(b, RF_ERR_CUDA, std::string("batch descriptors: ") + cudaGetErrorString(e));
  std::vector<bool> prof(n);
  for (int i = 0; i < n; ++i) {
    prof[i] = b->vols[i]->profiling;
    b->vols[i]->profiling = false;  // per-volume profiling events are not used in batches
  }
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  rf_status s = RF_OK;
  if (e != cudaSuccess) {
    s = batch_error(b, RF_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  } else {
    const BatchStage* table = static_cast<const BatchStage*>(out->d_table);
    const int* maps = reinterpret_cast<const int*>(table + n);
    const int map_len = out->total_ctas + n + 1;
    const int* ff_maps = maps + out->ngroups * map_len;
    const int ff_len = out->ff_ctas + n + 1;
    int max_npix = 1;
    for (int i = 0; i < n; ++i) max_npix = std::max(max_npix, f[i].H * f[i].W);
    const dim3 copy_grid((unsigned)std::min((max_npix * 3 / 16 + 255) / 256, 64), (unsigned)n);
    k_batch_stage<<<copy_grid, 256, 0, cs>>>(table);
    for (int gi = 0; gi < out->ngroups && !s; ++gi)
      s = launch_register_batch(b->vols[0], out->d_desc, maps + gi * map_len, maps + gi * map_len + out->total_ctas,
                                out->total_ctas, cs);
    // residual seeds and erosion of every stream: one launch each (guard
    // counts and flood-fill words were reset by the staging kernel); flood
    // fills: one cooperative launch per group of streams; dilation: one launch
    if (!s) s = launch_mask_pre_batch(b->vols[0], out->d_mask, n, max_npix, cs);
    for (int gi = 0; gi < out->ngroups && !s; ++gi)
      s = launch_floodfill_batch(b->vols[0], out->d_flood, ff_maps + gi * ff_len,
                                 ff_maps + gi * ff_len + out->ff_ctas, out->ff_ctas, cs);
    if (!s) s = launch_mask_post_batch(b->vols[0], out->d_mask, n, max_npix, cs);
    for (int gi = 0; gi < out->ngroups && !s; ++gi)
      s = launch_register_batch(b->vols[0], out->d_desc + n, maps + gi * map_len,
                                maps + gi * map_len + out->total_ctas, out->total_ctas, cs);
    // integrations: concurrent (one launch over all streams' candidate
    // blocks is no faster: the per-voxel update is latency-bound at its
    // occupancy, and concurrent launches overlap the streams' frustum searches)
    fork_aux(b, cs);
    for (int i = 0; i < n && !s; ++i)
      s = launch_integrate(b->vols[i], f[i], b->vols[i]->d_T + 32, b->vols[i]->d_mask, b->aux[i % rf_batch::kAux]);
    join_aux(b, cs);
    k_batch_out<<<dim3(copy_grid.x, n), 256, 0, cs>>>(table);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (!s && ce != cudaSuccess) s = batch_error(b, RF_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ce));
    if (!s) {
      ce = cudaGraphInstantiate(&out->exec, graph, 0);
      if (ce != cudaSuccess) s = batch_error(b, RF_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    } else if (s != RF_OK && b->last_error.empty()) {
      b->last_error = b->vols[0]->last_error;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  if (cs) cudaStreamDestroy(cs);
  for (int i = 0; i < n; ++i) b->vols[i]->profiling = prof[i];
  out->sig = sig;
  return s;
}

}  // namespace

extern "C" {

rf_status rf_default_params(rf_params* p) {
  if (!p) return RF_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->voxel_size = 0.01;  // Tab. I
  p->trunc = 0.1;        // Tab. I
  p->w_c = 0.025;        // Tab. I
  p->theta = 0.007;      // Tab. I
  p->gamma = 0.5;        // Tab. I
  p->depth_scale = 1000.0;
  p->d_min = 0.2;
  p->d_max = 5.0;
  p->z_near = 0.2;
  p->w_max = 255;
  p->lm_iters[0] = 10;
  p->lm_iters[1] = 5;
  p->lm_iters[2] = 5;
  p->lm_strides[0] = 4;
  p->lm_strides[1] = 2;
  p->lm_strides[2] = 1;
  p->lm_lambda0 = 1e-4;
  p->lm_eps_trans = 1e-6;
  p->lm_eps_rot = 1e-6;
  p->lm_min_valid = 10;
  p->max_ff_sweeps = 4096;
  p->max_candidates = (int64_t)1 << 21;
  p->storage = RF_STORAGE_FP32;
  return RF_OK;
}

const char* rf_status_string(rf_status s) {
  switch (s) {
    case RF_OK: return "ok";
    case RF_ERR_INVALID_ARG: return "invalid argument";
    case RF_ERR_CUDA: return "CUDA error";
    case RF_ERR_HASH_FULL: return "hash table full";
    case RF_ERR_POOL_FULL: return "block pool full";
    case RF_ERR_NOT_CONVERGED: return "not converged";
    case RF_ERR_BUFFER_TOO_SMALL: return "buffer too small";
    case RF_ERR_OUT_OF_RANGE: return "block coordinate out of range";
    case RF_ERR_CAPACITY: return "candidate capacity exceeded";
  }
  return "unknown status";
}

const char* rf_last_error(rf_volume* vol) { return vol ? vol->last_error.c_str() : g_create_error.c_str(); }

rf_status rf_destroy_volume(rf_volume* vol) {
  if (!vol) return RF_OK;
  cudaDeviceSynchronize();
  for (auto& g : vol->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& e : vol->ev)
    if (e) cudaEventDestroy(e);
  void* dev[] = {vol->d_hash, vol->d_vox,  vol->d_W,       vol->d_coords, vol->d_nbr, vol->d_nblocks, vol->d_status,
                 vol->d_regtags, vol->d_partials, vol->d_seeds, vol->d_md,    vol->d_ff,      vol->d_integ,
                 vol->d_tilemax, vol->d_cand, vol->d_depth, vol->d_rgb,   vol->d_mask,    vol->d_T, vol->d_info,
                 vol->d_guard, vol->d_pxcache, vol->d_dmask};
  for (void* p : dev)
    if (p) cudaFree(p);
  delete vol;
  return RF_OK;
}

rf_status rf_create_volume(const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width, int max_height,
                           rf_volume** out) {
  if (!out) return set_error(nullptr, RF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!p) return set_error(nullptr, RF_ERR_INVALID_ARG, "params is NULL");
  rf_status s = check_volume_args(p, n_buckets, max_blocks, max_width, max_height);
  if (s) return s;
  rf_volume* vol = new rf_volume();
  vol->p = *p;
  vol->dp = derive(*p);
  vol->n_buckets = n_buckets;
  vol->max_blocks = max_blocks;
  vol->max_w = max_width;
  vol->max_h = max_height;
  cudaError_t e = cudaGetDevice(&vol->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&vol->sm_count, cudaDevAttrMultiProcessorCount, vol->device);
  if (e != cudaSuccess) {
    s = set_error(nullptr, RF_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    delete vol;
    return s;
  }
  const size_t npix = (size_t)max_width * max_height;
  vol->max_slots = (int)((npix + 127) / 128);
  vol->reg_grid = register_max_grid(vol->device);
  if (vol->reg_grid > vol->sm_count) vol->reg_grid = vol->sm_count;
  if (vol->reg_grid < 1) {
    s = set_error(nullptr, RF_ERR_CUDA, "registration kernel cannot be resident on this device");
    delete vol;
    return s;
  }
  if ((s = volume_buffers(vol, p, n_buckets, max_blocks, max_width, max_height,
                          [&](auto** ptr, size_t count, const char* what) { return dalloc(vol, ptr, count, what); }))) {
    g_create_error = vol->last_error;
    rf_destroy_volume(vol);
    return s;
  }
  vol->dv.hash = vol->d_hash;
  vol->dv.bucket_mask = (unsigned long long)n_buckets - 1;
  vol->dv.vox = vol->d_vox;
  vol->dv.W = vol->d_W;
  vol->dv.coords = vol->d_coords;
  vol->dv.nbr = vol->d_nbr;
  vol->dv.n_blocks = vol->d_nblocks;
  vol->dv.max_blocks = (int)max_blocks;
  vol->dv.status = vol->d_status;
  {
    const char* env = std::getenv("RF_NO_GRAPHS");
    vol->use_graphs = !(env && env[0] == '1');
  }
  vol->ff_grid = floodfill_max_grid(vol->device);
  if (vol->ff_grid < 1) vol->ff_grid = 1;
  s = clear_model(vol, 0);
  if (!s) s = check_cuda(vol, cudaMemset(vol->d_status, 0, sizeof(unsigned)), "status reset");
  // the frustum search's ticket counter starts at 0
  if (!s) s = check_cuda(vol, cudaMemset(vol->d_integ, 0, sizeof(IntegState)), "integration state reset");
  // registration tags start at 0 (base, counts) with every partial-sum word's tag 0
  if (!s) s = check_cuda(vol, cudaMemset(vol->d_regtags, 0, 3 * sizeof(unsigned)), "tag reset");
  if (!s)
    s = check_cuda(vol, cudaMemset(vol->d_partials, 0, (size_t)2 * 29 * vol->max_slots * sizeof(unsigned long long)),
                   "partials reset");
  if (!s) s = check_cuda(vol, cudaDeviceSynchronize(), "create sync");
  if (s) {
    g_create_error = vol->last_error;
    rf_destroy_volume(vol);
    return s;
  }
  *out = vol;
  return RF_OK;
}

rf_status rf_volume_footprint(const rf_params* p, int64_t n_buckets, int64_t max_blocks, int max_width, int max_height,
                              int64_t* bytes) {
  if (!bytes) return set_error(nullptr, RF_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  if (!p) return set_error(nullptr, RF_ERR_INVALID_ARG, "params is NULL");
  rf_status s = check_volume_args(p, n_buckets, max_blocks, max_width, max_height);
  if (s) return s;
  rf_volume shape;
  size_t total = 0;
  volume_buffers(&shape, p, n_buckets, max_blocks, max_width, max_height, [&](auto** ptr, size_t count, const char*) {
    total += (count ? count : 1) * sizeof(**ptr);
    return RF_OK;
  });
  *bytes = (int64_t)total;
  return RF_OK;
}

rf_status rf_volume_reset(rf_volume* vol) {
  if (!vol) return RF_ERR_INVALID_ARG;
  rf_status s = clear_model(vol, 0);
  if (!s) s = check_cuda(vol, cudaMemset(vol->d_status, 0, sizeof(unsigned)), "status reset");
  if (!s) s = check_cuda(vol, cudaDeviceSynchronize(), "reset sync");
  vol->frames = 0;
  vol->has_model = false;
  return s;
}

rf_status rf_track_frame(rf_volume* vol, const rf_frame* frame, const double* T_init_dev, const uint8_t* mask_dev,
                         double* T_out_dev, rf_track_info* info_dev, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_init_dev || !T_out_dev) return set_error(vol, RF_ERR_INVALID_ARG, "pose pointer is NULL");
  return launch_track(vol, make_dev_frame(frame), T_init_dev, mask_dev, T_out_dev, info_dev, (cudaStream_t)stream);
}

rf_status rf_compute_mask(rf_volume* vol, const rf_frame* frame, const double* T_dev, uint8_t* mask_dev, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_dev || !mask_dev) return set_error(vol, RF_ERR_INVALID_ARG, "NULL pose or mask");
  return launch_mask(vol, make_dev_frame(frame), T_dev, mask_dev, (cudaStream_t)stream);
}

rf_status rf_virtual_depth(rf_volume* vol, const rf_frame* frame, const double* T_dev, int far_raw,
                           uint16_t* depth_out, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_dev || !depth_out) return set_error(vol, RF_ERR_INVALID_ARG, "NULL pose or output");
  if (far_raw < 0 || far_raw > 65535) return set_error(vol, RF_ERR_INVALID_ARG, "far_raw must be in 0..65535");
  const unsigned far = far_raw > 0 ? (unsigned)far_raw : (unsigned)llround(vol->p.d_max * vol->p.depth_scale);
  return launch_virtual_depth(vol, make_dev_frame(frame), T_dev, far, depth_out, (cudaStream_t)stream);
}

rf_status rf_integrate_frame(rf_volume* vol, const rf_frame* frame, const double* T_dev, const uint8_t* mask_dev,
                             void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_dev) return set_error(vol, RF_ERR_INVALID_ARG, "NULL pose");
  return launch_integrate(vol, make_dev_frame(frame), T_dev, mask_dev, (cudaStream_t)stream);
}

rf_status rf_process_frame(rf_volume* vol, const rf_frame* frame, const double* T_init_dev, double* T_out_dev,
                           uint8_t* mask_dev, rf_track_info* info_dev, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_init_dev || !T_out_dev) return set_error(vol, RF_ERR_INVALID_ARG, "NULL pose");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t npix = (size_t)frame->height * frame->width;
  const bool first = !vol->has_model;
  cudaGraphExec_t exec = nullptr;
  rf_status s = vol->use_graphs ? frame_graph(vol, frame, first, &exec) : RF_OK;
  if (s) return s;
  if ((s = check_cuda(vol, cudaMemcpyAsync(vol->d_depth, frame->depth, npix * 2, cudaMemcpyDefault, st),
                      "depth staging")))
    return s;
  if ((s = check_cuda(vol, cudaMemcpyAsync(vol->d_rgb, frame->rgb, npix * 3, cudaMemcpyDefault, st),
                      "rgb staging")))
    return s;
  if ((s = check_cuda(vol, cudaMemcpyAsync(vol->d_T, T_init_dev, 16 * sizeof(double), cudaMemcpyDeviceToDevice, st),
                      "pose staging")))
    return s;
  if ((s = run_frame(vol, frame, first, exec, st))) return s;
  if ((s = check_cuda(vol, cudaMemcpyAsync(T_out_dev, vol->d_T + 32, 16 * sizeof(double), cudaMemcpyDeviceToDevice, st),
                      "pose out")))
    return s;
  if (mask_dev && (s = check_cuda(vol, cudaMemcpyAsync(mask_dev, vol->d_mask, npix, cudaMemcpyDeviceToDevice, st),
                                  "mask out")))
    return s;
  if (info_dev) {
    if (first) s = check_cuda(vol, cudaMemsetAsync(info_dev, 0, sizeof(rf_track_info), st), "info out");
    else s = check_cuda(vol, cudaMemcpyAsync(info_dev, vol->d_info, sizeof(rf_track_info), cudaMemcpyDeviceToDevice, st),
                        "info out");
    if (s) return s;
  }
  vol->frames++;
  vol->has_model = true;
  return RF_OK;
}

rf_status rf_process_frame_host(rf_volume* vol, int height, int width, const double intrinsics[4],
                                const uint16_t* depth_host, const uint8_t* rgb_host, const double T_init_host[16],
                                double T_out_host[16], uint8_t* mask_host, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!intrinsics || !depth_host || !rgb_host || !T_init_host || !T_out_host)
    return set_error(vol, RF_ERR_INVALID_ARG, "NULL host buffer");
  rf_frame fr{height, width, intrinsics[0], intrinsics[1], intrinsics[2], intrinsics[3], vol->d_depth, vol->d_rgb};
  if (!frame_ok(vol, &fr)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t npix = (size_t)height * width;
  const bool first = !vol->has_model;
  cudaGraphExec_t exec = nullptr;
  rf_status s = vol->use_graphs ? frame_graph(vol, &fr, first, &exec) : RF_OK;
  if (s) return s;
  if ((s = check_cuda(vol, cudaMemcpyAsync(vol->d_depth, depth_host, npix * 2, cudaMemcpyHostToDevice, st), "depth H2D")) ||
      (s = check_cuda(vol, cudaMemcpyAsync(vol->d_rgb, rgb_host, npix * 3, cudaMemcpyHostToDevice, st), "rgb H2D")) ||
      (s = check_cuda(vol, cudaMemcpyAsync(vol->d_T, T_init_host, 16 * sizeof(double), cudaMemcpyHostToDevice, st),
                      "pose H2D")) ||
      (s = run_frame(vol, &fr, first, exec, st)) ||
      (s = check_cuda(vol, cudaMemcpyAsync(T_out_host, vol->d_T + 32, 16 * sizeof(double), cudaMemcpyDeviceToHost, st),
                      "pose D2H")))
    return s;
  if (mask_host && (s = check_cuda(vol, cudaMemcpyAsync(mask_host, vol->d_mask, npix, cudaMemcpyDeviceToHost, st),
                                   "mask D2H")))
    return s;
  vol->frames++;
  vol->has_model = true;
  return rf_sync_status(vol, stream);
}

rf_status rf_extract_mesh(rf_volume* vol, float* verts_dev, uint8_t* colors_dev, int64_t cap_tris, int64_t* n_tris_host,
                          void* stream) {
  if (!vol || !n_tris_host) return RF_ERR_INVALID_ARG;
  if ((verts_dev == nullptr) != (colors_dev == nullptr))
    return set_error(vol, RF_ERR_INVALID_ARG, "verts and colors must both be given or both be NULL");
  if (verts_dev && cap_tris < 0) return set_error(vol, RF_ERR_INVALID_ARG, "negative capacity");
  return run_mesh(vol, verts_dev, colors_dev, cap_tris, n_tris_host, (cudaStream_t)stream);
}

rf_status rf_volume_export(rf_volume* vol, int64_t cap_blocks, int32_t* coords, float* F, uint8_t* W, uint8_t* rgb,
                           uint8_t* wc, int64_t* n_blocks) {
  if (!vol || !n_blocks) return RF_ERR_INVALID_ARG;
  rf_status s = check_cuda(vol, cudaDeviceSynchronize(), "export sync");
  if (s) return s;
  int nb = 0;
  if ((s = check_cuda(vol, cudaMemcpy(&nb, vol->d_nblocks, sizeof(int), cudaMemcpyDeviceToHost), "export count")))
    return s;
  nb = std::min<int64_t>(nb, vol->max_blocks);
  std::vector<int4> c(nb > 0 ? nb : 1);
  if (nb > 0 && (s = check_cuda(vol, cudaMemcpy(c.data(), vol->d_coords, sizeof(int4) * nb, cudaMemcpyDeviceToHost),
                                "export coords")))
    return s;
  std::vector<int> order;
  for (int i = 0; i < nb; ++i)
    if (c[i].w) order.push_back(i);
  *n_blocks = (int64_t)order.size();
  if (!coords) return RF_OK;
  if (!F || !W || !rgb || !wc) return set_error(vol, RF_ERR_INVALID_ARG, "export buffers must all be given");
  if ((int64_t)order.size() > cap_blocks)
    return set_error(vol, RF_ERR_BUFFER_TOO_SMALL, "volume has %zu blocks, buffer holds %lld", order.size(),
                     (long long)cap_blocks);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (c[a].z != c[b].z) return c[a].z < c[b].z;
    if (c[a].y != c[b].y) return c[a].y < c[b].y;
    return c[a].x < c[b].x;
  });
  // pools in chunks, each copied in one piece; unpacked into sorted positions
  std::vector<int64_t> pos(nb, -1);
  for (size_t n = 0; n < order.size(); ++n) pos[order[n]] = (int64_t)n;
  const bool fp16 = vol->p.storage == RF_STORAGE_FP16;
  const float tau = vol->dp.tau;
  const int kChunk = 8192;
  std::vector<uint2> vx((size_t)std::min(nb, kChunk) * kBV);
  std::vector<uint8_t> w(fp16 ? 1 : (size_t)std::min(nb, kChunk) * kBV);
  for (int c0 = 0; c0 < nb; c0 += kChunk) {
    const int cn = std::min(kChunk, nb - c0);
    if ((s = check_cuda(vol, cudaMemcpy(vx.data(), vol->d_vox + (size_t)c0 * kBV, sizeof(uint2) * kBV * cn,
                                        cudaMemcpyDeviceToHost), "export voxels")))
      return s;
    if (!fp16 && (s = check_cuda(vol, cudaMemcpy(w.data(), vol->d_W + (size_t)c0 * kBV, (size_t)kBV * cn,
                                                 cudaMemcpyDeviceToHost), "export weights")))
      return s;
    for (int pl = c0; pl < c0 + cn; ++pl) {
      const int64_t n = pos[pl];
      if (n < 0) continue;
      coords[n * 3 + 0] = c[pl].x;
      coords[n * 3 + 1] = c[pl].y;
      coords[n * 3 + 2] = c[pl].z;
      const uint2* bv = vx.data() + (size_t)(pl - c0) * kBV;
      const unsigned* trk = reinterpret_cast<const unsigned*>(bv);
      for (int i = 0; i < kBV; ++i) {
        const size_t k = (size_t)n * kBV + i;
        unsigned colour;
        if (fp16) {
          const unsigned t = trk[i];
          W[k] = (uint8_t)(t >> 24);
          F[k] = W[k] ? half_bits_to_float((uint16_t)(t & 0xFFFFu)) * tau : 0.0f;
          colour = trk[kBV + i];
        } else {
          float f;
          std::memcpy(&f, &bv[i].x, 4);
          const uint8_t wi = w[(size_t)(pl - c0) * kBV + i];
          W[k] = wi;
          F[k] = wi ? f : 0.0f;
          colour = bv[i].y;
        }
        rgb[k * 3 + 0] = (uint8_t)(colour & 255u);
        rgb[k * 3 + 1] = (uint8_t)((colour >> 8) & 255u);
        rgb[k * 3 + 2] = (uint8_t)((colour >> 16) & 255u);
        wc[k] = (uint8_t)(colour >> 24);
      }
    }
  }
  return RF_OK;
}

rf_status rf_volume_import(rf_volume* vol, int64_t n_blocks, const int32_t* coords, const float* F, const uint8_t* W,
                           const uint8_t* rgb, const uint8_t* wc) {
  if (!vol || n_blocks < 0) return RF_ERR_INVALID_ARG;
  if (n_blocks > 0 && (!coords || !F || !W || !rgb || !wc)) return set_error(vol, RF_ERR_INVALID_ARG, "NULL buffer");
  if (n_blocks > vol->max_blocks) return set_error(vol, RF_ERR_POOL_FULL, "snapshot larger than max_blocks");
  rf_status s = rf_volume_reset(vol);
  if (s) return s;
  if (n_blocks == 0) return RF_OK;
  const bool fp16 = vol->p.storage == RF_STORAGE_FP16;
  const float tau = vol->dp.tau;
  std::vector<uint2> vx((size_t)n_blocks * kBV);
  std::vector<int4> c(n_blocks);
  for (int64_t n = 0; n < n_blocks; ++n) {
    c[n] = make_int4(coords[n * 3], coords[n * 3 + 1], coords[n * 3 + 2], 0);
    unsigned* trk = reinterpret_cast<unsigned*>(vx.data() + (size_t)n * kBV);
    for (int i = 0; i < kBV; ++i) {
      const size_t k = (size_t)n * kBV + i;
      const unsigned colour = (unsigned)rgb[k * 3] | ((unsigned)rgb[k * 3 + 1] << 8) |
                              ((unsigned)rgb[k * 3 + 2] << 16) | ((unsigned)wc[k] << 24);
      if (fp16) {
        unsigned t = kTrkEmpty;
        if (W[k]) {
          const unsigned sI = 2126u * rgb[k * 3] + 7152u * rgb[k * 3 + 1] + 722u * rgb[k * 3 + 2];
          const unsigned i8 = wc[k] ? (254u * sI + 1275000u) / 2550000u : 255u;
          t = (unsigned)float_to_half_bits(F[k] / tau) | (i8 << 16) | ((unsigned)W[k] << 24);
        }
        trk[i] = t;
        trk[kBV + i] = colour;
      } else {
        float f = W[k] ? F[k] : std::nanf("");
        unsigned bits;
        std::memcpy(&bits, &f, 4);
        if (W[k] == 0) bits = 0x7fc00000u;
        vx[k] = make_uint2(bits, colour);
      }
    }
  }
  s = check_cuda(vol, cudaMemcpy(vol->d_vox, vx.data(), sizeof(uint2) * vx.size(), cudaMemcpyHostToDevice),
                 "import voxels");
  if (!s && !fp16)
    s = check_cuda(vol, cudaMemcpy(vol->d_W, W, (size_t)n_blocks * kBV, cudaMemcpyHostToDevice), "import weights");
  // block coordinates go through the candidate buffer (no allocation), in chunks
  const int64_t chunk = vol->p.max_candidates;
  for (int64_t base = 0; !s && base < n_blocks; base += chunk) {
    const int n = (int)std::min<int64_t>(chunk, n_blocks - base);
    s = check_cuda(vol, cudaMemcpy(vol->d_cand, c.data() + base, sizeof(int4) * n, cudaMemcpyHostToDevice),
                   "import coords");
    if (!s) {
      k_import<<<(n + 255) / 256, 256>>>(vol->dv, vol->d_cand, n, (int)base);
      s = check_cuda(vol, cudaGetLastError(), "import launch");
    }
    if (!s) s = check_cuda(vol, cudaDeviceSynchronize(), "import sync");
  }
  int nb = (int)n_blocks;
  if (!s) s = check_cuda(vol, cudaMemcpy(vol->d_nblocks, &nb, sizeof(int), cudaMemcpyHostToDevice), "import count");
  if (!s) s = launch_nbr_fixup(vol, nullptr, 0, nullptr);
  if (!s) s = check_cuda(vol, cudaDeviceSynchronize(), "import sync");
  if (s) return s;
  vol->has_model = true;  // the next frame is tracked against the imported model
  return rf_sync_status(vol, nullptr);
}

rf_status rf_get_launch_config(rf_volume* vol, rf_launch_config* out) {
  if (!vol || !out) return RF_ERR_INVALID_ARG;
  *out = vol->launch;
  return RF_OK;
}

rf_status rf_set_launch_config(rf_volume* vol, const rf_launch_config* cfg) {
  if (!vol || !cfg) return RF_ERR_INVALID_ARG;
  const int v[4] = {cfg->integrate_ctas_per_sm, cfg->cull_ctas_per_sm, cfg->fixup_ctas_per_sm,
                    cfg->raycast_ctas_per_sm};
  for (int x : v)
    if (x < 1 || x > 64) return set_error(vol, RF_ERR_INVALID_ARG, "CTAs per SM must be in 1..64");
  if (cfg->batch_group < 0) return set_error(vol, RF_ERR_INVALID_ARG, "batch_group must be >= 0");
  rf_status s = check_cuda(vol, cudaDeviceSynchronize(), "launch config sync");
  if (s) return s;
  for (auto& g : vol->graphs) cudaGraphExecDestroy(g.exec);  // they hold the old shapes
  vol->graphs.clear();
  vol->launch = *cfg;
  return RF_OK;
}

rf_status rf_set_wait_limits(rf_volume* vol, int64_t spin_limit, int extra_arrivals) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (spin_limit < 0 || spin_limit > ((int64_t)1 << 40) || extra_arrivals < 0 || extra_arrivals > 1024)
    return set_error(vol, RF_ERR_INVALID_ARG, "spin_limit must be in 0..2^40 and extra_arrivals in 0..1024");
  rf_status s = check_cuda(vol, cudaDeviceSynchronize(), "wait limits sync");
  if (s) return s;
  for (auto& g : vol->graphs) cudaGraphExecDestroy(g.exec);  // their kernels hold the old limits
  vol->graphs.clear();
  vol->wait_spins = spin_limit == 0 ? kDefaultSpinLimit : (long long)spin_limit;
  vol->wait_extra = (unsigned)extra_arrivals;
  return RF_OK;
}

rf_status rf_set_registration_tag_base(rf_volume* vol, uint32_t base) {
  if (!vol) return RF_ERR_INVALID_ARG;
  const uint64_t span = 3 + (uint64_t)vol->p.lm_iters[0] + vol->p.lm_iters[1] + vol->p.lm_iters[2];
  if ((uint64_t)base + span >= (uint64_t)kTagLimit)
    return set_error(vol, RF_ERR_INVALID_ARG, "tag base %u: must be below 2^31 - %llu", base,
                     (unsigned long long)span);
  rf_status s = check_cuda(vol, cudaDeviceSynchronize(), "tag base sync");
  if (!s)
    s = check_cuda(vol, cudaMemset(vol->d_partials, 0, (size_t)2 * 29 * vol->max_slots * sizeof(unsigned long long)),
                   "partials reset");
  const unsigned words[3] = {base, 0u, 0u};
  if (!s) s = check_cuda(vol, cudaMemcpy(vol->d_regtags, words, sizeof(words), cudaMemcpyHostToDevice), "tag base");
  return s;
}

rf_status rf_volume_stats(rf_volume* vol, rf_stats* out) {
  if (!vol || !out) return RF_ERR_INVALID_ARG;
  int nb = 0;
  rf_status s = check_cuda(vol, cudaMemcpy(&nb, vol->d_nblocks, sizeof(int), cudaMemcpyDeviceToHost), "stats");
  if (s) return s;
  out->n_blocks = std::min<int64_t>(nb, vol->max_blocks);
  out->max_blocks = vol->max_blocks;
  out->n_buckets = vol->n_buckets;
  out->frames = vol->frames;
  out->load_factor = (double)out->n_blocks / (double)(vol->n_buckets * kSlots);
  out->device_bytes = (int64_t)vol->device_bytes;
  return RF_OK;
}

rf_status rf_set_profiling(rf_volume* vol, int enable) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (enable && !vol->ev[0]) {
    for (auto& e : vol->ev) {
      rf_status s = check_cuda(vol, cudaEventCreate(&e), "event create");
      if (s) return s;
    }
  }
  vol->profiling = enable != 0;
  return RF_OK;
}

rf_status rf_get_profile(rf_volume* vol, void* stream, rf_profile* out) {
  if (!vol || !out) return RF_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  rf_status s = check_cuda(vol, cudaStreamSynchronize((cudaStream_t)stream), "profile sync");
  if (s) return s;
  if (vol->profiling) {
    auto ms = [&](int a, int b) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, vol->ev[a], vol->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        t = -1.0f;
      }
      return t;
    };
    out->frame_ms = ms(EV_FRAME0, EV_FRAME1);
    out->track_ms[0] = ms(EV_FRAME0, EV_TRACK1_END);
    out->mask_ms = ms(EV_TRACK1_END, EV_MASK_END);
    out->track_ms[1] = ms(EV_MASK_END, EV_TRACK2_END);
    out->integrate_ms = ms(EV_INTEG0, EV_FRAME1);
    out->integrate_kernel_ms = ms(EV_KERNEL0, EV_KERNEL1);
  }
  IntegState is;
  unsigned guard = 0;
  if ((s = check_cuda(vol, cudaMemcpy(&is, vol->d_integ, sizeof(is), cudaMemcpyDeviceToHost), "profile counters")) ||
      (s = check_cuda(vol, cudaMemcpy(&guard, vol->d_guard, sizeof(guard), cudaMemcpyDeviceToHost), "guard count")))
    return s;
  out->candidates = std::min<int64_t>(is.n_cand, vol->p.max_candidates);
  out->updated_voxels = (int64_t)is.updated;
  out->new_blocks = is.new_blocks;
  out->guard_pixels = guard;
  return RF_OK;
}

rf_status rf_batch_create(rf_volume* const* vols, int n, rf_batch** out) {
  if (!out) return RF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!vols || n < 1) return set_error(nullptr, RF_ERR_INVALID_ARG, "rf_batch_create: need at least one volume");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return set_error(nullptr, RF_ERR_CUDA, "no CUDA device");
  for (int i = 0; i < n; ++i) {
    if (!vols[i]) return set_error(nullptr, RF_ERR_INVALID_ARG, "rf_batch_create: NULL volume");
    if (vols[i]->device != dev) return set_error(nullptr, RF_ERR_INVALID_ARG, "volumes on different devices");
    for (int j = 0; j < i; ++j)
      if (vols[j] == vols[i]) return set_error(nullptr, RF_ERR_INVALID_ARG, "a volume appears twice in a batch");
    if (vols[i]->p.storage != vols[0]->p.storage)
      return set_error(nullptr, RF_ERR_INVALID_ARG, "volumes of one batch must share the storage mode");
  }
  // every tracked stream needs at least one CTA of a registration and of a flood-fill launch
  const int max_streams = std::min(vols[0]->reg_grid, vols[0]->ff_grid);
  if (n > max_streams)
    return set_error(nullptr, RF_ERR_INVALID_ARG, "rf_batch_create: at most %d streams per batch on this device",
                     max_streams);
  rf_batch* b = new rf_batch();
  b->vols.assign(vols, vols + n);
  b->device = dev;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int k = 0; k < rf_batch::kAux && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    rf_batch_destroy(b);
    return set_error(nullptr, RF_ERR_CUDA, "rf_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return RF_OK;
}

rf_status rf_batch_destroy(rf_batch* b) {
  if (!b) return RF_OK;
  cudaDeviceSynchronize();
  for (auto& g : b->graphs) {
    free_batch_graph(g);
  }
  for (int k = 0; k < rf_batch::kAux; ++k) {
    if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  delete b;
  return RF_OK;
}

const char* rf_batch_last_error(rf_batch* b) { return b ? b->last_error.c_str() : ""; }

rf_status rf_batch_process(rf_batch* b, const rf_frame* frames, const double* const* T_init_dev,
                           double* const* T_out_dev, uint8_t* const* mask_dev, void* stream) {
  if (!b || !frames || !T_init_dev || !T_out_dev) return RF_ERR_INVALID_ARG;
  const int n = (int)b->vols.size();
  std::vector<double> sig;
  std::vector<int> mode(n);
  for (int i = 0; i < n; ++i) {
    rf_volume* v = b->vols[i];
    const rf_frame& fr = frames[i];
    mode[i] = fr.depth == nullptr ? kModeIdle : (v->has_model ? kModeTrack : kModeFirst);
    rf_frame shape = fr;
    if (mode[i] == kModeIdle) {  // shape checks only
      shape.depth = v->d_depth;
      shape.rgb = v->d_rgb;
    }
    if (!frame_ok(v, &shape)) return batch_error(b, RF_ERR_INVALID_ARG, "invalid frame in batch");
    if (!T_init_dev[i] || !T_out_dev[i]) return batch_error(b, RF_ERR_INVALID_ARG, "NULL pose in batch");
    sig.insert(sig.end(), {(double)fr.height, (double)fr.width, fr.fx, fr.fy, fr.cx, fr.cy});
  }
  rf_batch_graph* g = nullptr;
  for (auto& x : b->graphs)
    if (x.sig == sig) g = &x;
  if (!g && b->graphs.size() >= kMaxGraphs) {
    // the oldest shape goes; it may still be running (a rare event: wait)
    cudaError_t se = cudaDeviceSynchronize();
    if (se != cudaSuccess) return batch_error(b, RF_ERR_CUDA, std::string("graph eviction: ") + cudaGetErrorString(se));
    rf_batch_graph& old = b->graphs.front();
    free_batch_graph(old);
    b->graphs.erase(b->graphs.begin());
  }
  if (!g) {
    b->graphs.emplace_back();
    g = &b->graphs.back();
    rf_status s = batch_capture(b, frames, sig, g);
    if (s != RF_OK) {
      free_batch_graph(*g);
      b->graphs.pop_back();
      return s;
    }
  }
  // per-call table: staging pointers and modes, then the registration CTA map
  BatchStage* tab = reinterpret_cast<BatchStage*>(g->h_table.data());
  int* maps = reinterpret_cast<int*>(tab + n);
  const int map_len = g->total_ctas + n + 1;
  int* ff_maps = maps + g->ngroups * map_len;
  const int ff_len = g->ff_ctas + n + 1;
  std::vector<int> tracked;
  for (int i = 0; i < n; ++i) {
    rf_volume* v = b->vols[i];
    BatchStage& t = tab[i];
    t.depth_src = frames[i].depth;
    t.rgb_src = frames[i].rgb;
    t.T_src = T_init_dev[i];
    t.depth_dst = v->d_depth;
    t.rgb_dst = v->d_rgb;
    t.T_dst = v->d_T;
    t.T_out = T_out_dev[i];
    t.mask_out = mask_dev ? mask_dev[i] : nullptr;
    t.mask_buf = v->d_mask;
    t.guard = v->d_guard;
    t.ff = v->d_ff;
    t.ff_words = 2 + v->p.max_ff_sweeps;
    t.npix = frames[i].height * frames[i].width;
    t.mode = mode[i];
    if (mode[i] == kModeTrack) tracked.push_back(i);
  }
  // registration launch gi takes the tracked streams gi*gsize .. gi*gsize+gsize-1
  // (in stream order), CTAs split among them by pixel count
  // (the flood fills use the same groups, with maps over their own CTA count)
  for (int gi = 0; gi < g->ngroups; ++gi) {
    std::vector<double> w(n, 0.0);
    for (int k = gi * g->gsize; k < std::min((int)tracked.size(), (gi + 1) * g->gsize); ++k)
      w[tracked[k]] = (double)tab[tracked[k]].npix;
    fill_cta_map(w, g->total_ctas, maps + gi * map_len);
    fill_cta_map(w, g->ff_ctas, ff_maps + gi * ff_len);
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(g->d_table, g->h_table.data(), g->h_table.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, st);
  if (e != cudaSuccess) return batch_error(b, RF_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) {
    if (mode[i] == kModeIdle) continue;
    b->vols[i]->frames++;
    b->vols[i]->has_model = true;
  }
  return RF_OK;
}

rf_status rf_sync_status(rf_volume* vol, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  rf_status s = check_cuda(vol, cudaStreamSynchronize(st), "stream sync");
  if (s) return s;
  unsigned bits = 0;
  if ((s = check_cuda(vol, cudaMemcpy(&bits, vol->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost), "status read")))
    return s;
  if (bits && (s = check_cuda(vol, cudaMemset(vol->d_status, 0, sizeof(unsigned)), "status clear"))) return s;
  return status_from_bits(vol, bits);
}

}  // extern "C"
