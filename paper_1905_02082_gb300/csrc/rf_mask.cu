// Dynamics detection (ReFusion Sec. III-C) on sm_103a.
//
//   k_seeds      r_i = V_SDF(T x_i)^2 (the residual of Eq. 2, V_SDF truncated to
//                [-tau, tau]) and the raw mask r_i > t = gamma tau^2 (Eq. 5), one
//                thread per pixel.  The
//                decision is exact: the FP32 evaluation carries an error bound;
//                when the lattice cell or the comparison is within it, the pixel
//                is re-evaluated in FP64 with a fixed operation order and no
//                contraction (__d*_rn), the order the FP64 oracle uses.
//   k_erode      M_R = 3x3 erosion of the raw mask (outside the image = 0), and
//                M_D initialised to M_R.
//   k_floodfill  Alg. 1 closure: n joins from p when |D(p) - D(n)| < theta D(p)
//                (4-neighbours, raw integer depth, theta in ppm).  The closure
//                is the set reachable from M_R, independent of visiting order,
//                so tiles propagate locally in shared memory until stable and
//                sweep globally (cooperative launch, bounded grid barrier) until
//                no tile changes; at most max_ff_sweeps sweeps.
//   k_dilate     final mask = 3x3 dilation of M_D.
#include <cmath>
#include <mutex>

#include "rf_volume.hpp"

namespace rf {
namespace {

// FP64 residual in the fixed evaluation order; r < 0 when the lookup is invalid.
template <int ST>
__device__ double residual_fp64(const DevVol& v, const DevFrame& f, const DevParams& p, const double* T, int u, int vv,
                                unsigned raw) {
  const double D = __ddiv_rn((double)raw, p.depth_scale_d);
  const double x = __dmul_rn(__ddiv_rn(__dsub_rn((double)u, f.cxd), f.fxd), D);
  const double y = __dmul_rn(__ddiv_rn(__dsub_rn((double)vv, f.cyd), f.fyd), D);
  const double z = D;
  double q[3];
  int k[3];
  double fr[3];
  for (int i = 0; i < 3; ++i) {
    const double pi = __dadd_rn(
        __dadd_rn(__dadd_rn(__dmul_rn(T[i * 4 + 0], x), __dmul_rn(T[i * 4 + 1], y)), __dmul_rn(T[i * 4 + 2], z)),
        T[i * 4 + 3]);
    q[i] = __ddiv_rn(pi, p.voxel_d);
    if (!(fabs(q[i]) < 1e9)) return -1.0;
    const double fl = floor(q[i]);
    k[i] = (int)fl;
    fr[i] = __dsub_rn(q[i], fl);
  }
  if (abs(k[0]) > 8 * kMaxCoord || abs(k[1]) > 8 * kMaxCoord || abs(k[2]) > 8 * kMaxCoord) return -1.0;
  float F[8];
  if (!corners_of<ST>(v, p, k[0], k[1], k[2], F)) return -1.0;
  const double c00 = lerp_rn(F[0], F[1], fr[0]), c10 = lerp_rn(F[2], F[3], fr[0]);
  const double c01 = lerp_rn(F[4], F[5], fr[0]), c11 = lerp_rn(F[6], F[7], fr[0]);
  const double c0 = lerp_rn(c00, c10, fr[1]), c1 = lerp_rn(c01, c11, fr[1]);
  const double V = fmin(fmax(lerp_rn(c0, c1, fr[2]), -p.tau_d), p.tau_d);  // truncated at tau
  return __dmul_rn(V, V);
}

// Seed decision of one valid pixel in FP32 with an error bound: 0 or 1, or
// 2 when the lattice cell or the comparison lies within the bound (the pixel
// is then decided in FP64).  Rf: the pose as floats (R row-major, then t).
template <int ST>
__device__ __forceinline__ int seed_fp32(const DevVol& v, const DevFrame& f, const DevParams& p, const float* Rf, int u,
                                         int vv, unsigned raw, unsigned long long cached) {
  const float t = p.gamma_tau2_f;
  const float D = (float)raw * p.inv_depth_scale;
  const float x = ((float)u - f.cx) * f.ifx * D, y = ((float)vv - f.cy) * f.ify * D;
  float q[3], fr[3];
  int k[3];
  const float mag_in = (fabsf(x) + fabsf(y) + fabsf(D) + fabsf(Rf[9]) + fabsf(Rf[10]) + fabsf(Rf[11])) * p.inv_voxel;
  float qmax = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float pi = Rf[i * 3] * x + Rf[i * 3 + 1] * y + Rf[i * 3 + 2] * D + Rf[9 + i];
    q[i] = pi * p.inv_voxel;
    qmax = fmaxf(qmax, fabsf(q[i]));
  }
  // bound on |q32 - q64| with an 8x margin (see the error budget in the design notes)
  const float eps_q = (mag_in + qmax) * 3.814697265625e-06f;  // 2^-18
  if (!(qmax < 8.0f * kMaxCoord - 2.0f)) return 2;
  bool ambiguous = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float fl = floorf(q[i]);
    k[i] = (int)fl;
    fr[i] = q[i] - fl;
    if (fr[i] < eps_q || fr[i] > 1.0f - eps_q) ambiguous = true;
  }
  if (ambiguous) return 2;
  float F[8];
  // an unambiguous cell with a missing corner is invalid in FP64 too: no seed
  if (!corners_cached<ST>(v, p, k[0], k[1], k[2], cached, F)) return 0;
  const float c00 = F[0] * (1.0f - fr[0]) + F[1] * fr[0], c10 = F[2] * (1.0f - fr[0]) + F[3] * fr[0];
  const float c01 = F[4] * (1.0f - fr[0]) + F[5] * fr[0], c11 = F[6] * (1.0f - fr[0]) + F[7] * fr[0];
  const float c0 = c00 * (1.0f - fr[1]) + c10 * fr[1], c1 = c01 * (1.0f - fr[1]) + c11 * fr[1];
  const float V = fminf(fmaxf(c0 * (1.0f - fr[2]) + c1 * fr[2], -p.tau), p.tau);
  float fmn = F[0], fmx = F[0], fab = fabsf(F[0]);
#pragma unroll
  for (int n = 1; n < 8; ++n) {
    fmn = fminf(fmn, F[n]);
    fmx = fmaxf(fmx, F[n]);
    fab = fmaxf(fab, fabsf(F[n]));
  }
  // + the gap between the float and double truncation bounds (<= 2^-24 tau)
  const float dV = 3.0f * (fmx - fmn) * eps_q + fab * 1.9073486328125e-06f + p.tau * 5.9604645e-08f;
  const float r = V * V;
  const float dr = 2.0f * fabsf(V) * dV + dV * dV + r * 2.384185791015625e-07f;  // 2^-22
  if (fabsf(r - t) <= 2.0f * dr + t * 2.384185791015625e-07f) return 2;
  return r > t ? 1 : 0;
}

// Seeds of the kSeedThreads * kSeedPx pixels of CTA `block` (blockDim.x =
// kSeedThreads; pixel block * kSeedThreads * kSeedPx + j * kSeedThreads + tid
// for j < kSeedPx).  Every thread first loads its pixels' depths and cache
// entries, then decides them in FP32; the ambiguous ones are queued in shared
// memory and decided in FP64 afterwards, side by side by consecutive threads:
// on GB300 the FP64 pipe is narrow, and a warp that takes the FP64 branch for
// one of its lanes costs as much as one that takes it for all 32.
// pxcache: the registration's per-pixel block cache (nullptr: none), read
// only, to skip hash probes.
constexpr int kSeedThreads = 256;
constexpr int kSeedPx = 4;

__host__ __device__ constexpr int seed_blocks(int npix) {
  return (npix + kSeedThreads * kSeedPx - 1) / (kSeedThreads * kSeedPx);
}

template <int ST>
__device__ __forceinline__ void seeds_body(const DevVol& v, const DevFrame& f, const DevParams& p,
                                           const double* __restrict__ T, uint8_t* __restrict__ seeds,
                                           unsigned* guard_count, const unsigned long long* __restrict__ pxcache,
                                           int block) {
  // pose and threshold converted once per CTA (conversions use the FP64 pipe)
  __shared__ float sR[12];
  __shared__ double s_t64;
  __shared__ int s_queue[kSeedThreads * kSeedPx];
  __shared__ int s_n;
  if (threadIdx.x < 12) {
    const int i = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
    const int j = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
    sR[threadIdx.x] = (float)T[i * 4 + j];
  }
  if (threadIdx.x == 12) s_t64 = __dmul_rn(__dmul_rn(p.gamma_d, p.tau_d), p.tau_d);
  if (threadIdx.x == 13) s_n = 0;
  __syncthreads();
  const int npix = f.H * f.W;
  const int first = block * kSeedThreads * kSeedPx + (int)threadIdx.x;
  unsigned raw[kSeedPx];
  unsigned long long cached[kSeedPx];
#pragma unroll
  for (int j = 0; j < kSeedPx; ++j) {
    const int idx = first + j * kSeedThreads;
    raw[j] = idx < npix ? __ldg(f.depth + idx) : 0u;
    cached[j] = idx < npix && pxcache ? __ldg(pxcache + idx) : kEmpty;
  }
#pragma unroll 1
  for (int j = 0; j < kSeedPx; ++j) {
    const int idx = first + j * kSeedThreads;
    if (idx >= npix) break;
    const unsigned rj = j == 0 ? raw[0] : (j == 1 ? raw[1] : (j == 2 ? raw[2] : raw[3]));
    const unsigned long long cj = j == 0 ? cached[0] : (j == 1 ? cached[1] : (j == 2 ? cached[2] : cached[3]));
    int seed = 0;
    if (pixel_valid(p, rj)) seed = seed_fp32<ST>(v, f, p, sR, idx % f.W, idx / f.W, rj, cj);
    if (seed == 2) s_queue[atomicAdd(&s_n, 1)] = idx;
    else seeds[idx] = (uint8_t)seed;
  }
  __syncthreads();
  const int n = s_n;
  for (int i = threadIdx.x; i < n; i += kSeedThreads) {
    const int idx = s_queue[i];
    const double r64 = residual_fp64<ST>(v, f, p, T, idx % f.W, idx / f.W, __ldg(f.depth + idx));
    seeds[idx] = (r64 >= 0.0 && r64 > s_t64) ? 1 : 0;
  }
  if (threadIdx.x == 0 && n > 0 && guard_count) atomicAdd(guard_count, (unsigned)n);
}

template <int ST>
__global__ void __launch_bounds__(kSeedThreads) k_seeds(DevVol v, DevFrame f, DevParams p,
                                                        const double* __restrict__ T, uint8_t* __restrict__ seeds,
                                                        unsigned* guard_count,
                                                        const unsigned long long* __restrict__ pxcache) {
  if (gated_off(f.gate, kModeTrack)) return;
  seeds_body<ST>(v, f, p, T, seeds, guard_count, pxcache, blockIdx.x);
}

// grid (x, n streams): the seeds of every tracked stream of a batch.
template <int ST>
__global__ void __launch_bounds__(kSeedThreads) k_seeds_batch(const MaskDesc* __restrict__ descs) {
  const MaskDesc& d = descs[blockIdx.y];
  if (gated_off(d.f.gate, kModeTrack) || (int)blockIdx.x >= seed_blocks(d.f.H * d.f.W)) return;
  seeds_body<ST>(d.v, d.f, d.p, d.T, d.seeds, d.guard, d.pxcache, blockIdx.x);
}

__device__ __forceinline__ void erode_px(const uint8_t* __restrict__ in, int H, int W, uint8_t* __restrict__ mr,
                                         int idx) {
  const int u = idx % W, v = idx / W;
  uint8_t all = 1;
  if (u == 0 || v == 0 || u == W - 1 || v == H - 1) {
    all = 0;
  } else {
#pragma unroll
    for (int dv = -1; dv <= 1; ++dv)
#pragma unroll
      for (int du = -1; du <= 1; ++du) all &= (__ldg(in + (v + dv) * W + (u + du)) != 0);
  }
  mr[idx] = all;
}

__global__ void __launch_bounds__(256) k_erode(const uint8_t* __restrict__ in, int H, int W, uint8_t* __restrict__ mr,
                                               const int* gate) {
  if (gated_off(gate, kModeTrack)) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < H * W) erode_px(in, H, W, mr, idx);
}

__device__ __forceinline__ void dilate_px(const uint8_t* __restrict__ in, int H, int W, uint8_t* __restrict__ out,
                                          int idx) {
  const int u = idx % W, v = idx / W;
  uint8_t any = 0;
  for (int dv = -1; dv <= 1; ++dv) {
    const int y = v + dv;
    if (y < 0 || y >= H) continue;
    for (int du = -1; du <= 1; ++du) {
      const int x = u + du;
      if (x < 0 || x >= W) continue;
      any |= (__ldg(in + y * W + x) != 0);
    }
  }
  out[idx] = any;
}

__global__ void __launch_bounds__(256) k_dilate(const uint8_t* __restrict__ in, int H, int W, uint8_t* __restrict__ out,
                                                const int* gate) {
  if (gated_off(gate, kModeTrack)) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < H * W) dilate_px(in, H, W, out, idx);
}

// grid (x, n streams): erosion and dilation of every tracked stream of a batch.
__global__ void __launch_bounds__(256) k_erode_batch(const MaskDesc* __restrict__ descs) {
  const MaskDesc& d = descs[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gated_off(d.f.gate, kModeTrack) || idx >= d.f.H * d.f.W) return;
  erode_px(d.seeds, d.f.H, d.f.W, d.md, idx);
}

__global__ void __launch_bounds__(256) k_dilate_batch(const MaskDesc* __restrict__ descs) {
  const MaskDesc& d = descs[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gated_off(d.f.gate, kModeTrack) || idx >= d.f.H * d.f.W) return;
  dilate_px(d.md, d.f.H, d.f.W, d.mask_out, idx);
}

constexpr int kFFW = 32, kFFH = 16;  // flood-fill tile (one thread per pixel)
constexpr int kFFThreads = kFFW * kFFH;

__device__ __forceinline__ bool ff_edge(unsigned Dsrc, unsigned Ddst, long long theta_ppm) {
  const long long diff = Dsrc > Ddst ? (long long)(Dsrc - Ddst) : (long long)(Ddst - Dsrc);
  return diff * 1000000ll < theta_ppm * (long long)Dsrc;
}

// ff words: [0] barrier count, [1] barrier generation, [2 + s] changed in sweep s
// Run by a group of G CTAs, this one being number lb of the group.
__device__ void floodfill_body(uint8_t* md, const uint16_t* __restrict__ depth, int H, int W, long long theta_ppm,
                               unsigned* ff, int max_sweeps, unsigned* status, long long spin_limit,
                               unsigned bar_extra, int lb, int G) {
  __shared__ uint8_t sm[kFFH + 2][kFFW + 2];
  __shared__ uint16_t sd[kFFH + 2][kFFW + 2];
  const int tiles_x = (W + kFFW - 1) / kFFW, tiles_y = (H + kFFH - 1) / kFFH;
  const int ntiles = tiles_x * tiles_y;
  const int tx = threadIdx.x % kFFW, ty = threadIdx.x / kFFW;
  unsigned* bar = ff;
  unsigned* changed = ff + 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int tile = lb; tile < ntiles; tile += G) {
      const int u0 = (tile % tiles_x) * kFFW, v0 = (tile / tiles_x) * kFFH;
      // tile + 1-pixel halo into shared memory
      for (int i = threadIdx.x; i < (kFFH + 2) * (kFFW + 2); i += kFFThreads) {
        const int hy = i / (kFFW + 2), hx = i % (kFFW + 2);
        const int u = u0 + hx - 1, v = v0 + hy - 1;
        const bool in = u >= 0 && u < W && v >= 0 && v < H;
        sm[hy][hx] = in ? *(volatile uint8_t*)(md + v * W + u) : 0;
        sd[hy][hx] = in ? __ldg(depth + v * W + u) : 0;
      }
      __syncthreads();
      const int u = u0 + tx, v = v0 + ty;
      const bool inside = u < W && v < H;
      bool grew = false;
      for (int it = 0; it < kFFThreads; ++it) {
        int c = 0;
        if (inside && !sm[ty + 1][tx + 1]) {
          const unsigned Dp = sd[ty + 1][tx + 1];
          if ((sm[ty + 1][tx] && ff_edge(sd[ty + 1][tx], Dp, theta_ppm)) ||
              (sm[ty + 1][tx + 2] && ff_edge(sd[ty + 1][tx + 2], Dp, theta_ppm)) ||
              (sm[ty][tx + 1] && ff_edge(sd[ty][tx + 1], Dp, theta_ppm)) ||
              (sm[ty + 2][tx + 1] && ff_edge(sd[ty + 2][tx + 1], Dp, theta_ppm))) {
            sm[ty + 1][tx + 1] = 1;
            grew = true;
            c = 1;
          }
        }
        if (!__syncthreads_or(c)) break;
      }
      if (grew) md[v * W + u] = 1;
      if (__syncthreads_or(grew) && threadIdx.x == 0) atomicExch(changed + sweep, 1u);
    }
    if (!grid_barrier(bar, G, status, spin_limit, bar_extra)) return;
    if (*(volatile unsigned*)(changed + sweep) == 0u) return;
  }
  if (lb == 0 && threadIdx.x == 0) atomicOr(status, ST_NOT_CONVERGED);
}

__global__ void __launch_bounds__(kFFThreads) k_floodfill(uint8_t* md, const uint16_t* __restrict__ depth, int H,
                                                           int W, long long theta_ppm, unsigned* ff, int max_sweeps,
                                                           unsigned* status, const int* gate, long long spin_limit,
                                                           unsigned bar_extra) {
  if (gated_off(gate, kModeTrack)) return;  // uniform over the grid: before any barrier
  floodfill_body(md, depth, H, W, theta_ppm, ff, max_sweeps, status, spin_limit, bar_extra, blockIdx.x, gridDim.x);
}

// The flood fills of several streams in one cooperative launch: CTA b runs
// stream cta_stream[b] (-1: none) as member b - first[s] of its group (the
// CTA maps of the batched registration).  Groups never wait on each other.
__global__ void __launch_bounds__(kFFThreads) k_floodfill_batch(const FloodDesc* __restrict__ descs,
                                                                 const int* __restrict__ cta_stream,
                                                                 const int* __restrict__ first) {
  const int s = cta_stream[blockIdx.x];
  if (s < 0) return;
  const FloodDesc d = descs[s];
  floodfill_body(d.md, d.depth, d.H, d.W, d.theta_ppm, d.ff, d.max_sweeps, d.status, d.spin_limit, d.bar_extra,
                 blockIdx.x - first[s], first[s + 1] - first[s]);
}

}  // namespace

rf_status launch_mask_pre(rf_volume* vol, const DevFrame& f, const double* T, cudaStream_t st) {
  const int n = f.H * f.W;
  const int blocks = (n + 255) / 256;
  rf_status s = check_cuda(vol, cudaMemsetAsync(vol->d_guard, 0, sizeof(unsigned), st), "guard reset");
  if (s != RF_OK) return s;
  if (vol->p.storage == RF_STORAGE_FP16)
    k_seeds<RF_STORAGE_FP16><<<seed_blocks(n), kSeedThreads, 0, st>>>(vol->dv, f, vol->dp, T, vol->d_seeds,
                                                                       vol->d_guard, vol->d_pxcache);
  else
    k_seeds<RF_STORAGE_FP32><<<seed_blocks(n), kSeedThreads, 0, st>>>(vol->dv, f, vol->dp, T, vol->d_seeds,
                                                                       vol->d_guard, vol->d_pxcache);
  k_erode<<<blocks, 256, 0, st>>>(vol->d_seeds, f.H, f.W, vol->d_md, f.gate);
  s = check_cuda(vol, cudaMemsetAsync(vol->d_ff, 0, sizeof(unsigned) * (2 + vol->p.max_ff_sweeps), st),
                 "flood-fill reset");
  if (s != RF_OK) return s;
  return check_cuda(vol, cudaGetLastError(), "mask launch");
}

rf_status launch_mask_ff(rf_volume* vol, const DevFrame& f, cudaStream_t st) {
  const int ntiles = ((f.W + kFFW - 1) / kFFW) * ((f.H + kFFH - 1) / kFFH);
  const int grid = ntiles < vol->ff_grid ? ntiles : vol->ff_grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kFFThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return check_cuda(vol,
                    cudaLaunchKernelEx(&cfg, k_floodfill, vol->d_md, f.depth, f.H, f.W, vol->dp.theta_ppm, vol->d_ff,
                                       vol->p.max_ff_sweeps, vol->d_status, f.gate, vol->wait_spins,
                                       vol->wait_extra),
                    "flood-fill launch");
}

MaskDesc make_mask_desc(rf_volume* vol, const DevFrame& f, const double* T, uint8_t* mask_out) {
  MaskDesc d;
  d.v = vol->dv;
  d.f = f;
  d.p = vol->dp;
  d.T = T;
  d.seeds = vol->d_seeds;
  d.guard = vol->d_guard;
  d.md = vol->d_md;
  d.mask_out = mask_out;
  d.pxcache = vol->d_pxcache;
  return d;
}

rf_status launch_mask_pre_batch(rf_volume* vol, const MaskDesc* descs, int n, int max_npix, cudaStream_t st) {
  const dim3 grid((unsigned)((max_npix + 255) / 256), (unsigned)n);
  const dim3 sgrid((unsigned)seed_blocks(max_npix), (unsigned)n);
  if (vol->p.storage == RF_STORAGE_FP16)
    k_seeds_batch<RF_STORAGE_FP16><<<sgrid, kSeedThreads, 0, st>>>(descs);
  else
    k_seeds_batch<RF_STORAGE_FP32><<<sgrid, kSeedThreads, 0, st>>>(descs);
  k_erode_batch<<<grid, 256, 0, st>>>(descs);
  return check_cuda(vol, cudaGetLastError(), "batched mask launch");
}

rf_status launch_mask_post_batch(rf_volume* vol, const MaskDesc* descs, int n, int max_npix, cudaStream_t st) {
  k_dilate_batch<<<dim3((unsigned)((max_npix + 255) / 256), (unsigned)n), 256, 0, st>>>(descs);
  return check_cuda(vol, cudaGetLastError(), "batched mask launch");
}

rf_status launch_mask_post(rf_volume* vol, const DevFrame& f, uint8_t* mask_out, cudaStream_t st) {
  const int n = f.H * f.W;
  k_dilate<<<(n + 255) / 256, 256, 0, st>>>(vol->d_md, f.H, f.W, mask_out, f.gate);
  return check_cuda(vol, cudaGetLastError(), "mask launch");
}

rf_status launch_mask(rf_volume* vol, const DevFrame& f, const double* T, uint8_t* mask_out, cudaStream_t st) {
  rf_status s = launch_mask_pre(vol, f, T, st);
  if (s == RF_OK) s = launch_mask_ff(vol, f, st);
  if (s == RF_OK) s = launch_mask_post(vol, f, mask_out, st);
  return s;
}

FloodDesc make_flood_desc(rf_volume* vol, const DevFrame& f) {
  FloodDesc d;
  d.md = vol->d_md;
  d.depth = f.depth;
  d.H = f.H;
  d.W = f.W;
  d.theta_ppm = vol->dp.theta_ppm;
  d.ff = vol->d_ff;
  d.max_sweeps = vol->p.max_ff_sweeps;
  d.status = vol->d_status;
  d.spin_limit = vol->wait_spins;
  d.bar_extra = vol->wait_extra;
  return d;
}

rf_status launch_floodfill_batch(rf_volume* vol, const FloodDesc* descs, const int* cta_stream, const int* first,
                                 int total_ctas, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(total_ctas);
  cfg.blockDim = dim3(kFFThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return check_cuda(vol, cudaLaunchKernelEx(&cfg, k_floodfill_batch, descs, cta_stream, first),
                    "batched flood-fill launch");
}

int floodfill_max_grid(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_floodfill, kFFThreads, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

// ---------------------------------------------------------------------------
// Mask without any allocation: the per-call scratch of rf_compute_mask (seed
// image, flood-fill working mask, barrier words, per-sweep change flags and the
// guard counter) lives in one file-scope device array instead of the buffers
// the volume owns.  Every GPU that loads this library holds the array (about
// 1.9 MB) until the process exits.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxPixels = 1280 * 720;  // largest frame: 921,600 pixels
constexpr int kNoAllocMaxSweeps = 4096;         // flood-fill sweep bound of this entry point
constexpr size_t kNoAllocWordsOff = 2 * (size_t)kNoAllocMaxPixels;  // multiple of 256
constexpr size_t kNoAllocWords = 2 + kNoAllocMaxSweeps + 1;         // barrier, change flags, guard count
constexpr size_t kNoAllocBytes = kNoAllocWordsOff + sizeof(unsigned) * kNoAllocWords;

static __device__ __align__(256) unsigned char g_mask_scratch[kNoAllocBytes];

// Device address of g_mask_scratch, looked up once per device with that
// device current.  In host code the symbol is only a host-side stand-in.
static void* mask_scratch_address(int device, cudaError_t* err) {
  static std::mutex mu;
  static void* addr[64] = {};
  *err = cudaSuccess;
  if (device < 0 || device >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_mask_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = p;
  }
  return addr[device];
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_compute_mask_noalloc(rf_volume* vol, const rf_frame* frame, const double* T_dev,
                                             uint8_t* mask_dev, void* stream) {
  if (!vol) return RF_ERR_INVALID_ARG;
  if (!frame_ok(vol, frame)) return set_error(vol, RF_ERR_INVALID_ARG, "invalid frame");
  if (!T_dev || !mask_dev) return set_error(vol, RF_ERR_INVALID_ARG, "NULL pose or mask");
  if ((int64_t)frame->height * frame->width > kNoAllocMaxPixels)
    return set_error(vol, RF_ERR_INVALID_ARG,
                     "rf_compute_mask_noalloc: frame of %d x %d pixels exceeds the static scratch limit of %d pixels",
                     frame->width, frame->height, kNoAllocMaxPixels);
  // the kernels run on the current device and read the volume's memory: the
  // two must be the same GPU (the scratch address is per device too)
  int device = 0;
  rf_status s = check_cuda(vol, cudaGetDevice(&device), "current device");
  if (s) return s;
  if (device != vol->device)
    return set_error(vol, RF_ERR_INVALID_ARG,
                     "rf_compute_mask_noalloc: current device %d is not the volume's device %d", device, vol->device);
  cudaError_t e;
  unsigned char* base = static_cast<unsigned char*>(mask_scratch_address(vol->device, &e));
  if (!base) return check_cuda(vol, e, "cudaGetSymbolAddress(mask scratch)");
  uint8_t* seeds = base;
  uint8_t* md = base + kNoAllocMaxPixels;
  unsigned* ff = reinterpret_cast<unsigned*>(base + kNoAllocWordsOff);
  unsigned* guard = ff + 2 + kNoAllocMaxSweeps;
  const int sweeps = vol->p.max_ff_sweeps < kNoAllocMaxSweeps ? vol->p.max_ff_sweeps : kNoAllocMaxSweeps;
  cudaStream_t st = (cudaStream_t)stream;
  const DevFrame f = make_dev_frame(frame);
  const int n = f.H * f.W;
  const int blocks = (n + 255) / 256;
  // the array keeps the previous call's contents: zero the words that count
  if ((s = check_cuda(vol, cudaMemsetAsync(ff, 0, sizeof(unsigned) * kNoAllocWords, st), "scratch clear"))) return s;
  if (vol->p.storage == RF_STORAGE_FP16)
    k_seeds<RF_STORAGE_FP16><<<seed_blocks(n), kSeedThreads, 0, st>>>(vol->dv, f, vol->dp, T_dev, seeds, guard,
                                                                       vol->d_pxcache);
  else
    k_seeds<RF_STORAGE_FP32><<<seed_blocks(n), kSeedThreads, 0, st>>>(vol->dv, f, vol->dp, T_dev, seeds, guard,
                                                                       vol->d_pxcache);
  k_erode<<<blocks, 256, 0, st>>>(seeds, f.H, f.W, md, nullptr);
  const int ntiles = ((f.W + kFFW - 1) / kFFW) * ((f.H + kFFH - 1) / kFFH);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntiles < vol->ff_grid ? ntiles : vol->ff_grid);
  cfg.blockDim = dim3(kFFThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((s = check_cuda(vol, cudaLaunchKernelEx(&cfg, k_floodfill, md, f.depth, f.H, f.W, vol->dp.theta_ppm, ff,
                                              sweeps, vol->d_status, (const int*)nullptr, vol->wait_spins,
                                              vol->wait_extra),
                      "flood-fill launch")))
    return s;
  k_dilate<<<blocks, 256, 0, st>>>(md, f.H, f.W, mask_dev, nullptr);
  return check_cuda(vol, cudaGetLastError(), "mask launch");
}
