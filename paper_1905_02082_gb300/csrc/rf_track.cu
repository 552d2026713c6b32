// Registration (ReFusion Sec. III-B) on sm_103a: Levenberg-Marquardt on the
// joint error of Eq. 4, E = sum_i V_SDF(exp(xi) T x_i)^2
//                         + w_c sum_i (V_I(exp(xi) T x_i) - I(p_i))^2,
// over three pixel sub-samplings (strides), coarse to fine.
//
// One LM iteration is two launches with no host round trip:
//   k_track_accum  one thread per sampled pixel: Eq. 1 back-projection, rigid
//                  transform, hash lookup of the 8 lattice corners, trilinear
//                  SDF and intensity with analytic gradients, residuals and
//                  Jacobians J = dV/dp [I | -[p]x] (left perturbation), and a
//                  warp-shuffle + shared-memory reduction of the 21 entries of
//                  J^T J, the 6 of J^T r, the cost and the valid count into one
//                  per-CTA partial (FP32);
//   k_lm_update    one CTA: fixed-order FP64 reduction of the partials, accept or
//                  reject the candidate (mean cost E/N must decrease), lambda
//                  update, 6x6 Cholesky of H + lambda diag(H) in FP64, se(3)
//                  exponential and composition of the next candidate pose.
// A device flag ends a level early (step below the thresholds); the remaining
// launches of the level return at once.  Results are deterministic: fixed
// grids, fixed pixel-to-thread mapping and fixed reduction order.
#include <cmath>

#include "rf_volume.hpp"

namespace rf {
namespace {

constexpr int kTrackThreads = 256;

__device__ __forceinline__ float lerpf(float a, float b, float t) { return a * (1.0f - t) + b * t; }

// Trilinear SDF/intensity lookup with analytic gradients (per metre).
// Corner n = dx + 2 dy + 4 dz.  Returns false unless all 8 corners exist and
// were observed; *colour is true when all 8 also carry colour.
__device__ __forceinline__ bool model_sample(const DevVol& v, const DevParams& p, float px, float py, float pz,
                                             float* V, float gV[3], float* I, float gI[3], bool* colour) {
  const float qx = px * p.inv_voxel, qy = py * p.inv_voxel, qz = pz * p.inv_voxel;
  if (!(fabsf(qx) < 1.0e6f && fabsf(qy) < 1.0e6f && fabsf(qz) < 1.0e6f)) return false;
  const float fkx = floorf(qx), fky = floorf(qy), fkz = floorf(qz);
  const int kx = (int)fkx, ky = (int)fky, kz = (int)fkz;
  const float fx = qx - fkx, fy = qy - fky, fz = qz - fkz;
  const int lx = kx & 7, ly = ky & 7, lz = kz & 7;
  const int bx = kx >> 3, by = ky >> 3, bz = kz >> 3;
  uint2 c[8];
  if (lx < 7 && ly < 7 && lz < 7) {
    const int pool = hash_find(v, bx, by, bz);
    if (pool < 0) return false;
    const uint2* base = v.vox + (size_t)pool * kBV + lx + 8 * ly + 64 * lz;
    c[0] = __ldg(base);
    c[1] = __ldg(base + 1);
    c[2] = __ldg(base + 8);
    c[3] = __ldg(base + 9);
    c[4] = __ldg(base + 64);
    c[5] = __ldg(base + 65);
    c[6] = __ldg(base + 72);
    c[7] = __ldg(base + 73);
  } else {
    int pools[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) pools[n] = -2;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int ox = (n & 1) && lx == 7, oy = ((n >> 1) & 1) && ly == 7, oz = ((n >> 2) & 1) && lz == 7;
      const int slot = ox + 2 * oy + 4 * oz;
      if (pools[slot] == -2) pools[slot] = hash_find(v, bx + ox, by + oy, bz + oz);
      const int pool = pools[slot];
      if (pool < 0) return false;
      const int ix = (lx + (n & 1)) & 7, iy = (ly + ((n >> 1) & 1)) & 7, iz = (lz + ((n >> 2) & 1)) & 7;
      c[n] = __ldg(v.vox + (size_t)pool * kBV + ix + 8 * iy + 64 * iz);
    }
  }
  float F[8];
  bool col = true;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    F[n] = __uint_as_float(c[n].x);
    if (F[n] != F[n]) return false;  // never observed
    col &= (c[n].y >> 24) != 0u;
  }
  const float c00 = lerpf(F[0], F[1], fx), c10 = lerpf(F[2], F[3], fx);
  const float c01 = lerpf(F[4], F[5], fx), c11 = lerpf(F[6], F[7], fx);
  const float c0 = lerpf(c00, c10, fy), c1 = lerpf(c01, c11, fy);
  *V = lerpf(c0, c1, fz);
  gV[0] = lerpf(lerpf(F[1] - F[0], F[3] - F[2], fy), lerpf(F[5] - F[4], F[7] - F[6], fy), fz) * p.inv_voxel;
  gV[1] = lerpf(lerpf(F[2] - F[0], F[3] - F[1], fx), lerpf(F[6] - F[4], F[7] - F[5], fx), fz) * p.inv_voxel;
  gV[2] = (c1 - c0) * p.inv_voxel;
  *colour = col;
  if (col) {
    float In[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) In[n] = rgb_intensity(c[n].y);
    const float d00 = lerpf(In[0], In[1], fx), d10 = lerpf(In[2], In[3], fx);
    const float d01 = lerpf(In[4], In[5], fx), d11 = lerpf(In[6], In[7], fx);
    const float d0 = lerpf(d00, d10, fy), d1 = lerpf(d01, d11, fy);
    *I = lerpf(d0, d1, fz);
    gI[0] = lerpf(lerpf(In[1] - In[0], In[3] - In[2], fy), lerpf(In[5] - In[4], In[7] - In[6], fy), fz) * p.inv_voxel;
    gI[1] = lerpf(lerpf(In[2] - In[0], In[3] - In[1], fx), lerpf(In[6] - In[4], In[7] - In[5], fx), fz) * p.inv_voxel;
    gI[2] = (d1 - d0) * p.inv_voxel;
  }
  return true;
}

__device__ __forceinline__ void add_jtj(float* acc, const float J[6], float r, float w) {
  int n = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float wi = w * J[i];
#pragma unroll
    for (int j = i; j < 6; ++j) acc[n++] += wi * J[j];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) acc[21 + i] += w * J[i] * r;
  acc[27] += w * r * r;
}

__global__ void __launch_bounds__(kTrackThreads) k_track_accum(DevVol v, DevFrame f, DevParams p,
                                                                const uint8_t* __restrict__ mask, int stride, int Ws,
                                                                int npix, const LMState* __restrict__ lm,
                                                                int use_current, float* __restrict__ partials) {
  if (!use_current && *(volatile const int*)&lm->done) return;
  const float* Tf = use_current ? lm->Rf : lm->Rcf;
  const float R0 = Tf[0], R1 = Tf[1], R2 = Tf[2], R3 = Tf[3], R4 = Tf[4], R5 = Tf[5], R6 = Tf[6], R7 = Tf[7],
              R8 = Tf[8], t0 = Tf[9], t1 = Tf[10], t2 = Tf[11];
  float acc[29];
#pragma unroll
  for (int i = 0; i < 29; ++i) acc[i] = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    const int u = (i % Ws) * stride, vv = (i / Ws) * stride;
    const int idx = vv * f.W + u;
    const unsigned raw = __ldg(f.depth + idx);
    if (!pixel_valid(p, raw)) continue;
    if (mask && __ldg(mask + idx)) continue;
    const float D = (float)raw * p.inv_depth_scale;
    const float x = ((float)u - f.cx) * f.ifx * D, y = ((float)vv - f.cy) * f.ify * D;
    const float px = R0 * x + R1 * y + R2 * D + t0;
    const float py = R3 * x + R4 * y + R5 * D + t1;
    const float pz = R6 * x + R7 * y + R8 * D + t2;
    float V, gV[3], I, gI[3];
    bool colour;
    if (!model_sample(v, p, px, py, pz, &V, gV, &I, gI, &colour)) continue;
    const float Jd[6] = {gV[0], gV[1], gV[2], py * gV[2] - pz * gV[1], pz * gV[0] - px * gV[2],
                         px * gV[1] - py * gV[0]};
    add_jtj(acc, Jd, V, 1.0f);
    acc[28] += 1.0f;
    if (colour) {
      const uint8_t* c = f.rgb + 3 * (size_t)idx;
      const unsigned cc = (unsigned)__ldg(c) | ((unsigned)__ldg(c + 1) << 8) | ((unsigned)__ldg(c + 2) << 16);
      const float rc = I - rgb_intensity(cc);
      const float Jc[6] = {gI[0], gI[1], gI[2], py * gI[2] - pz * gI[1], pz * gI[0] - px * gI[2],
                           px * gI[1] - py * gI[0]};
      add_jtj(acc, Jc, rc, p.w_c);
    }
  }
  // warp-shuffle reduction, then across the CTA's warps in fixed order
  __shared__ float red[kTrackThreads / 32][29];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 29; ++i) {
    float s = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < 29) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kTrackThreads / 32; ++w) s += red[w][threadIdx.x];
    partials[blockIdx.x * kPartialStride + threadIdx.x] = s;
  }
}

struct LMConst {
  double lambda0, eps_t, eps_r;
  long long min_valid;
};

__device__ void se3_exp_d(const double xi[6], double T[16]) {
  const double th2 = xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5];
  const double th = sqrt(th2);
  double A, B, C;
  if (th < 1e-5) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    double s, c;
    sincos(th, &s, &c);
    A = s / th;
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
  }
  const double wx = xi[3], wy = xi[4], wz = xi[5];
  const double K[9] = {0, -wz, wy, wz, 0, -wx, -wy, wx, 0};
  double K2[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[i * 3 + j] = K[i * 3] * K[j] + K[i * 3 + 1] * K[3 + j] + K[i * 3 + 2] * K[6 + j];
  for (int i = 0; i < 3; ++i) {
    double t = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double I = (i == j) ? 1.0 : 0.0;
      T[i * 4 + j] = I + A * K[i * 3 + j] + B * K2[i * 3 + j];
      t += (I + B * K[i * 3 + j] + C * K2[i * 3 + j]) * xi[j];
    }
    T[i * 4 + 3] = t;
  }
  T[12] = T[13] = T[14] = 0.0;
  T[15] = 1.0;
}

// (H + lambda diag H) d = -g, H given as 21 upper-triangle entries.
__device__ bool lm_solve_d(const double* H, const double* g, double lambda, double d[6]) {
  double A[6][6], L[6][6];
  int n = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      A[i][j] = H[n];
      A[j][i] = H[n];
      ++n;
    }
  for (int i = 0; i < 6; ++i) A[i][i] *= (1.0 + lambda);
  for (int j = 0; j < 6; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0) || !isfinite(s)) return false;
    L[j][j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = -g[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
    y[i] = s / L[i][i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * d[k];
    d[i] = s / L[i][i];
  }
  return true;
}

__device__ void to_float(const double* T, float* Tf) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) Tf[i * 3 + j] = (float)T[i * 4 + j];
    Tf[9 + i] = (float)T[i * 4 + 3];
  }
}

__global__ void k_track_init(LMState* lm, const double* __restrict__ T_init) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < 16; ++i) {
    lm->T[i] = T_init[i];
    lm->Tc[i] = T_init[i];
  }
  to_float(lm->T, lm->Rf);
  to_float(lm->T, lm->Rcf);
  lm->done = 0;
  lm->E = 0.0;
  lm->N = 0;
  lm->lambda = 0.0;
  rf_track_info z = {};
  lm->info = z;
}

// mode 0: first evaluation of a level (at T, always taken); mode 1: candidate.
__global__ void __launch_bounds__(256) k_lm_update(LMState* lm, const float* __restrict__ partials, int G, int mode,
                                                   int level, int last, LMConst c) {
  if (mode == 1 && *(volatile int*)&lm->done) return;
  __shared__ double red[29];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int comp = warp; comp < 29; comp += 8) {
    double s = 0.0;
    for (int k = lane; k < G; k += 32) s += (double)partials[k * kPartialStride + comp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[comp] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double En = red[27];
  const long long Nn = llrint(red[28]);
  lm->info.evals++;
  lm->info.level_evals[level]++;
  if (mode == 0) {
    for (int i = 0; i < 21; ++i) lm->H[i] = red[i];
    for (int i = 0; i < 6; ++i) lm->g[i] = red[21 + i];
    lm->E = En;
    lm->N = Nn;
    lm->info.final_cost = Nn > 0 ? En / (double)Nn : 0.0;
    lm->info.final_valid = Nn;
    lm->done = 0;
    if (Nn < c.min_valid) {
      lm->done = 1;
      return;
    }
    lm->lambda = c.lambda0;
  } else {
    if (Nn >= c.min_valid && En / (double)Nn < lm->E / (double)lm->N) {
      for (int i = 0; i < 16; ++i) lm->T[i] = lm->Tc[i];
      for (int i = 0; i < 12; ++i) lm->Rf[i] = lm->Rcf[i];
      for (int i = 0; i < 21; ++i) lm->H[i] = red[i];
      for (int i = 0; i < 6; ++i) lm->g[i] = red[21 + i];
      lm->E = En;
      lm->N = Nn;
      lm->lambda /= 10.0;
      lm->info.final_cost = En / (double)Nn;
      lm->info.final_valid = Nn;
    } else {
      lm->lambda *= 10.0;
    }
    if (last) return;
  }
  double d[6];
  if (!lm_solve_d(lm->H, lm->g, lm->lambda, d)) {
    lm->info.converged[level] = 1;
    lm->done = 1;
    return;
  }
  const double nr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double nw = sqrt(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
  if (nr < c.eps_t && nw < c.eps_r) {
    lm->info.converged[level] = 1;
    lm->done = 1;
    return;
  }
  double Ex[16];
  se3_exp_d(d, Ex);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += Ex[i * 4 + k] * lm->T[k * 4 + j];
      lm->Tc[i * 4 + j] = s;
    }
  to_float(lm->Tc, lm->Rcf);
}

__global__ void k_track_final(const LMState* __restrict__ lm, double* T_out, rf_track_info* info) {
  const int i = threadIdx.x;
  if (i < 16) T_out[i] = lm->T[i];
  if (i == 0 && info) *info = lm->info;
}

}  // namespace

rf_status launch_track(rf_volume* vol, const DevFrame& f, const double* T_init, const uint8_t* mask, double* T_out,
                       rf_track_info* info, cudaStream_t st) {
  LMConst c{vol->p.lm_lambda0, vol->p.lm_eps_trans, vol->p.lm_eps_rot, (long long)vol->p.lm_min_valid};
  k_track_init<<<1, 32, 0, st>>>(vol->d_lm, T_init);
  for (int l = 0; l < 3; ++l) {
    const int s = vol->p.lm_strides[l];
    const int Ws = (f.W + s - 1) / s, Hs = (f.H + s - 1) / s;
    const int npix = Ws * Hs;
    int G = (npix + kTrackThreads - 1) / kTrackThreads;
    G = G < 1 ? 1 : (G > vol->max_partials ? vol->max_partials : G);
    const int iters = vol->p.lm_iters[l];
    k_track_accum<<<G, kTrackThreads, 0, st>>>(vol->dv, f, vol->dp, mask, s, Ws, npix, vol->d_lm, 1,
                                               vol->d_partials);
    k_lm_update<<<1, 256, 0, st>>>(vol->d_lm, vol->d_partials, G, 0, l, iters == 0, c);
    for (int it = 0; it < iters; ++it) {
      k_track_accum<<<G, kTrackThreads, 0, st>>>(vol->dv, f, vol->dp, mask, s, Ws, npix, vol->d_lm, 0,
                                                 vol->d_partials);
      k_lm_update<<<1, 256, 0, st>>>(vol->d_lm, vol->d_partials, G, 1, l, it == iters - 1, c);
    }
  }
  k_track_final<<<1, 32, 0, st>>>(vol->d_lm, T_out, info);
  return check_cuda(vol, cudaGetLastError(), "track launch");
}

}  // namespace rf
