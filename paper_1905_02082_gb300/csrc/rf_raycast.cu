// Virtual depth (Sec. III-E, second option): the zero pixels of a frame take
// the depth of the first crossing of a (temporary) model's TSDF along their
// ray, seen from a registered pose; rays without a crossing take a far value.
//
//   k_vd_holes       copies the non-zero pixels, lists the zero ones.
//   k_vd_cast        one warp per listed pixel casts its ray, 32
//                    consecutive samples at a time, at z_k = z_near + k v/2,
//                    k = 0..K, K = floor(2 (d_max - z_near) / v) (computed on
//                    micrometres).  A sample counts when the 8 trilinear
//                    corners of its cell are observed; the crossing is the
//                    first pair of consecutive counted samples with V > 0
//                    then V <= 0, and the depth is
//                    z* = z_{k-1} + (v/2) V_{k-1} / (V_{k-1} - V_k),
//                    rounded half up to raw units.
//
// Decisions are exact.  Each sample is first evaluated in FP32 with an error
// bound on its lattice position and on V; a sample whose cell or sign is
// within the bound is evaluated again in FP64 with a fixed operation order
// and no contraction (__d*_rn), the order of the FP64 oracle.  The two
// samples that bracket the crossing are always evaluated in FP64, and so is
// the final depth, so the written value is the oracle's.
#include "rf_volume.hpp"

namespace rf {
namespace {

struct Sample {
  bool valid;
  bool pos;  // V > 0
  double V;  // FP64 value (only when evaluated in FP64)
};

// FP64 sample k of pixel (u, vv) in the oracle's order.
template <int ST>
__device__ Sample sample_fp64(const DevVol& v, const DevFrame& f, const DevParams& p, const double* T, int u, int vv,
                              int k, double znear_d, double delta_d) {
  Sample s = {false, false, 0.0};
  const double z = __dadd_rn(znear_d, __dmul_rn((double)k, delta_d));
  const double x = __dmul_rn(__ddiv_rn(__dsub_rn((double)u, f.cxd), f.fxd), z);
  const double y = __dmul_rn(__ddiv_rn(__dsub_rn((double)vv, f.cyd), f.fyd), z);
  int kk[3];
  double fr[3];
  for (int i = 0; i < 3; ++i) {
    const double pi = __dadd_rn(
        __dadd_rn(__dadd_rn(__dmul_rn(__ldg(T + i * 4), x), __dmul_rn(__ldg(T + i * 4 + 1), y)),
                  __dmul_rn(__ldg(T + i * 4 + 2), z)),
        __ldg(T + i * 4 + 3));
    const double q = __ddiv_rn(pi, p.voxel_d);
    if (!(fabs(q) < 1e9)) return s;
    const double fl = floor(q);
    if (fabs(fl) > 8.0 * kMaxCoord) return s;  // outside every block: never observed
    kk[i] = (int)fl;
    fr[i] = __dsub_rn(q, fl);
  }
  float F[8];
  if (!corners_of<ST>(v, p, kk[0], kk[1], kk[2], F)) return s;
  const double c00 = lerp_rn(F[0], F[1], fr[0]), c10 = lerp_rn(F[2], F[3], fr[0]);
  const double c01 = lerp_rn(F[4], F[5], fr[0]), c11 = lerp_rn(F[6], F[7], fr[0]);
  const double c0 = lerp_rn(c00, c10, fr[1]), c1 = lerp_rn(c01, c11, fr[1]);
  s.V = lerp_rn(c0, c1, fr[2]);
  s.valid = true;
  s.pos = s.V > 0.0;
  return s;
}

// Decision of sample k of a ray (validity and sign of V): FP32 with an error
// bound, FP64 in the oracle's order when the cell or the sign is within it.
template <int ST>
__device__ __forceinline__ Sample decide_sample(const DevVol& v, const DevFrame& f, const DevParams& p,
                                                const double* T, const float* sR, int u, int vv, float xr, float yr,
                                                float tmag, int k, double znear_d, double delta_d, unsigned* n64) {
  const float z = (float)znear_d + (float)k * (float)delta_d;
  const float x = xr * z, y = yr * z;
  float q[3], qmax = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q[i] = (sR[i * 3] * x + sR[i * 3 + 1] * y + sR[i * 3 + 2] * z + sR[9 + i]) * p.inv_voxel;
    qmax = fmaxf(qmax, fabsf(q[i]));
  }
  // bound on |q32 - q64| with an 8x margin (the mask seeds' error budget)
  const float mag_in = (fabsf(x) + fabsf(y) + fabsf(z)) * p.inv_voxel + tmag;
  const float eps_q = (mag_in + qmax) * 3.814697265625e-06f;  // 2^-18
  bool ambiguous = !(qmax < 8.0f * kMaxCoord - 2.0f);
  int kk[3];
  float fr[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float fl = floorf(q[i]);
    kk[i] = (int)fl;
    fr[i] = q[i] - fl;
    if (fr[i] < eps_q || fr[i] > 1.0f - eps_q) ambiguous = true;
  }
  Sample s = {false, false, 0.0};
  if (!ambiguous) {
    float F[8];
    if (corners_of<ST>(v, p, kk[0], kk[1], kk[2], F)) {
      const float c00 = F[0] * (1.0f - fr[0]) + F[1] * fr[0], c10 = F[2] * (1.0f - fr[0]) + F[3] * fr[0];
      const float c01 = F[4] * (1.0f - fr[0]) + F[5] * fr[0], c11 = F[6] * (1.0f - fr[0]) + F[7] * fr[0];
      const float c0 = c00 * (1.0f - fr[1]) + c10 * fr[1], c1 = c01 * (1.0f - fr[1]) + c11 * fr[1];
      const float V = c0 * (1.0f - fr[2]) + c1 * fr[2];
      float fmn = F[0], fmx = F[0], fab = fabsf(F[0]);
#pragma unroll
      for (int n = 1; n < 8; ++n) {
        fmn = fminf(fmn, F[n]);
        fmx = fmaxf(fmx, F[n]);
        fab = fmaxf(fab, fabsf(F[n]));
      }
      const float dV = 3.0f * (fmx - fmn) * eps_q + fab * 1.9073486328125e-06f;
      if (fabsf(V) <= 2.0f * dV) {
        ambiguous = true;  // the sign needs FP64
      } else {
        s.valid = true;
        s.pos = V > 0.0f;
      }
    }
    // an unambiguous cell with a missing corner is invalid in FP64 too
  }
  if (ambiguous) {
    s = sample_fp64<ST>(v, f, p, T, u, vv, k, znear_d, delta_d);
    ++*n64;
  }
  return s;
}

// Copies the non-zero pixels and appends the zero ones to a list
// (warp-aggregated atomics); the list's order does not matter, each ray's
// result depends on its own pixel only.
__global__ void __launch_bounds__(256) k_vd_holes(DevFrame f, uint16_t* __restrict__ out, int* __restrict__ list,
                                                   unsigned* count) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int npix = f.H * f.W;
  const unsigned raw = idx < npix ? __ldg(f.depth + idx) : 1u;
  if (idx < npix && raw != 0u) out[idx] = (uint16_t)raw;
  const unsigned holes = __ballot_sync(0xffffffffu, idx < npix && raw == 0u);
  if (!holes) return;
  unsigned base = 0;
  if (lane == 0) base = atomicAdd(count, (unsigned)__popc(holes));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (raw == 0u && idx < npix) list[base + __popc(holes & ((1u << lane) - 1u))] = idx;
}

// One warp per zero pixel of the list (grid-stride over warps): the warp
// casts the ray 32 consecutive samples per step (lane l: sample k0 + l); the
// crossing is the first lane whose sample and its predecessor (the previous
// lane, or the last sample of the previous step) form a V > 0 -> V <= 0 pair.
template <int ST>
__global__ void __launch_bounds__(256) k_vd_cast(DevVol v, DevFrame f, DevParams p, const double* __restrict__ T,
                                                  unsigned far_raw, int K, double znear_d, double delta_d,
                                                  const int* __restrict__ list, const unsigned* count,
                                                  uint16_t* __restrict__ out, unsigned* fp64_count) {
  __shared__ float sR[12];
  if (threadIdx.x < 12) {
    const int i = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
    const int j = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
    sR[threadIdx.x] = (float)T[i * 4 + j];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nholes = *count;
  const float tmag = (fabsf(sR[9]) + fabsf(sR[10]) + fabsf(sR[11])) * p.inv_voxel;
  unsigned n64 = 0;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long h = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nholes; h += nwarps) {
    const int pix = __ldg(list + h);
    const int u = pix % f.W, vv = pix / f.W;
    const float xr = ((float)u - f.cx) * f.ifx, yr = ((float)vv - f.cy) * f.ify;
    unsigned result = far_raw;
    bool carry_valid = false, carry_pos = false;
    for (int k0 = 0; k0 <= K; k0 += 32) {
      const int k = k0 + lane;
      Sample cur = {false, false, 0.0};
      if (k <= K) cur = decide_sample<ST>(v, f, p, T, sR, u, vv, xr, yr, tmag, k, znear_d, delta_d, &n64);
      bool pv = __shfl_up_sync(0xffffffffu, cur.valid, 1), pp = __shfl_up_sync(0xffffffffu, cur.pos, 1);
      if (lane == 0) {
        pv = carry_valid;
        pp = carry_pos;
      }
      const unsigned cross = __ballot_sync(0xffffffffu, k <= K && pv && cur.valid && pp && !cur.pos);
      if (cross) {
        const int kc = k0 + __ffs(cross) - 1;
        // the bracketing pair and the depth in FP64, in the oracle's order
        if (lane == 0) {
          const Sample a = sample_fp64<ST>(v, f, p, T, u, vv, kc - 1, znear_d, delta_d);
          const Sample b = sample_fp64<ST>(v, f, p, T, u, vv, kc, znear_d, delta_d);
          const double zp = __dadd_rn(znear_d, __dmul_rn((double)(kc - 1), delta_d));
          const double t = __ddiv_rn(a.V, __dsub_rn(a.V, b.V));
          const double zs = __dadd_rn(zp, __dmul_rn(delta_d, t));
          const double r = floor(__dadd_rn(__dmul_rn(zs, p.depth_scale_d), 0.5));
          result = r < 0.0 ? 0u : (r > 65535.0 ? 65535u : (unsigned)r);
        }
        break;
      }
      carry_valid = __shfl_sync(0xffffffffu, cur.valid, 31);
      carry_pos = __shfl_sync(0xffffffffu, cur.pos, 31);
    }
    if (lane == 0) out[pix] = (uint16_t)result;
  }
  if (fp64_count) {
    n64 = __reduce_add_sync(0xffffffffu, n64);
    if (lane == 0 && n64) atomicAdd(fp64_count, n64);
  }
}

}  // namespace

rf_status launch_virtual_depth(rf_volume* vol, const DevFrame& f, const double* T, unsigned far_raw, uint16_t* out,
                               cudaStream_t st) {
  const long long znear_um = vol->dp.znear_tick / 1024;
  const int K = (int)((2 * (vol->dp.dmax_um - znear_um)) / vol->dp.v_um);
  const double znear_d = vol->p.z_near, delta_d = vol->p.voxel_size * 0.5;
  const long long npix = (long long)f.H * f.W;
  if (npix > 4 * vol->p.max_candidates)
    return set_error(vol, RF_ERR_CAPACITY, "frame larger than the hole list (4 x max_candidates pixels)");
  // scratch: the hole list in the candidate buffer, its count in the partials
  int* list = reinterpret_cast<int*>(vol->d_cand);
  unsigned* count = reinterpret_cast<unsigned*>(vol->d_partials);
  rf_status s = check_cuda(vol, cudaMemsetAsync(count, 0, sizeof(unsigned), st), "hole count reset");
  // the guard counter reports this call's FP64 re-evaluations
  if (s == RF_OK) s = check_cuda(vol, cudaMemsetAsync(vol->d_guard, 0, sizeof(unsigned), st), "guard reset");
  if (s != RF_OK) return s;
  k_vd_holes<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(f, out, list, count);
  const int grid = vol->sm_count * vol->launch.raycast_ctas_per_sm;
  if (vol->p.storage == RF_STORAGE_FP16)
    k_vd_cast<RF_STORAGE_FP16><<<grid, 256, 0, st>>>(vol->dv, f, vol->dp, T, far_raw, K, znear_d, delta_d, list, count,
                                                     out, vol->d_guard);
  else
    k_vd_cast<RF_STORAGE_FP32><<<grid, 256, 0, st>>>(vol->dv, f, vol->dp, T, far_raw, K, znear_d, delta_d, list, count,
                                                     out, vol->d_guard);
  return check_cuda(vol, cudaGetLastError(), "virtual depth launch");
}

}  // namespace rf
