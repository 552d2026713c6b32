// Virtual depth (Sec. III-E, second option): the zero pixels of a frame take
// the depth of the first crossing of a (temporary) model's TSDF along their
// ray, seen from a registered pose; rays without a crossing take a far value.
//
//   k_virtual_depth  one thread per pixel.  Non-zero pixels are copied.  A
//                    zero pixel marches its ray at z_k = z_near + k v/2,
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

template <int ST>
__global__ void __launch_bounds__(256) k_virtual_depth(DevVol v, DevFrame f, DevParams p, const double* __restrict__ T,
                                                        unsigned far_raw, int K, double znear_d, double delta_d,
                                                        uint16_t* __restrict__ out, unsigned* fp64_count) {
  __shared__ float sR[12];
  if (threadIdx.x < 12) {
    const int i = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
    const int j = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
    sR[threadIdx.x] = (float)T[i * 4 + j];
  }
  __syncthreads();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= f.H * f.W) return;
  const unsigned raw = __ldg(f.depth + idx);
  if (raw != 0u) {
    out[idx] = (uint16_t)raw;
    return;
  }
  const int u = idx % f.W, vv = idx / f.W;
  const float xr = ((float)u - f.cx) * f.ifx, yr = ((float)vv - f.cy) * f.ify;
  const float znear_f = (float)znear_d, delta_f = (float)delta_d;
  const float tmag = (fabsf(sR[9]) + fabsf(sR[10]) + fabsf(sR[11])) * p.inv_voxel;
  unsigned result = far_raw;
  unsigned n64 = 0;
  Sample prev = {false, false, 0.0};
  bool prev64 = false;
  for (int k = 0; k <= K; ++k) {
    const float z = znear_f + (float)k * delta_f;
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
    Sample cur = {false, false, 0.0};
    bool cur64 = false;
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
          cur.valid = true;
          cur.pos = V > 0.0f;
        }
      }
      // an unambiguous cell with a missing corner is invalid in FP64 too
    }
    if (ambiguous) {
      cur = sample_fp64<ST>(v, f, p, T, u, vv, k, znear_d, delta_d);
      cur64 = true;
      ++n64;
    }
    if (prev.valid && cur.valid && prev.pos && !cur.pos) {
      // the bracketing pair and the depth in FP64, in the oracle's order
      if (!prev64) prev = sample_fp64<ST>(v, f, p, T, u, vv, k - 1, znear_d, delta_d);
      if (!cur64) cur = sample_fp64<ST>(v, f, p, T, u, vv, k, znear_d, delta_d);
      const double zp = __dadd_rn(znear_d, __dmul_rn((double)(k - 1), delta_d));
      const double t = __ddiv_rn(prev.V, __dsub_rn(prev.V, cur.V));
      const double zs = __dadd_rn(zp, __dmul_rn(delta_d, t));
      const double r = floor(__dadd_rn(__dmul_rn(zs, p.depth_scale_d), 0.5));
      result = r < 0.0 ? 0u : (r > 65535.0 ? 65535u : (unsigned)r);
      break;
    }
    prev = cur;
    prev64 = cur64;
  }
  out[idx] = (uint16_t)result;
  if (fp64_count && n64) atomicAdd(fp64_count, n64);
}

}  // namespace

rf_status launch_virtual_depth(rf_volume* vol, const DevFrame& f, const double* T, unsigned far_raw, uint16_t* out,
                               cudaStream_t st) {
  const long long znear_um = vol->dp.znear_tick / 1024;
  const int K = (int)((2 * (vol->dp.dmax_um - znear_um)) / vol->dp.v_um);
  const double znear_d = vol->p.z_near, delta_d = vol->p.voxel_size * 0.5;
  const int n = f.H * f.W;
  const int blocks = (n + 255) / 256;
  // the guard counter reports this call's FP64 re-evaluations
  rf_status s = check_cuda(vol, cudaMemsetAsync(vol->d_guard, 0, sizeof(unsigned), st), "guard reset");
  if (s != RF_OK) return s;
  if (vol->p.storage == RF_STORAGE_FP16)
    k_virtual_depth<RF_STORAGE_FP16><<<blocks, 256, 0, st>>>(vol->dv, f, vol->dp, T, far_raw, K, znear_d, delta_d, out,
                                                             vol->d_guard);
  else
    k_virtual_depth<RF_STORAGE_FP32><<<blocks, 256, 0, st>>>(vol->dv, f, vol->dp, T, far_raw, K, znear_d, delta_d, out,
                                                             vol->d_guard);
  return check_cuda(vol, cudaGetLastError(), "virtual depth launch");
}

}  // namespace rf
