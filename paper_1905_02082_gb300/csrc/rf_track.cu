// Registration (ReFusion Sec. III-B) on sm_103a: Levenberg-Marquardt on the
// joint error of Eq. 4, E = sum_i V_SDF(exp(xi) T x_i)^2
//                         + w_c sum_i (V_I(exp(xi) T x_i) - I(p_i))^2,
// over three pixel sub-samplings (strides), coarse to fine.
//
// A whole registration (three levels, every LM iteration) is ONE cooperative
// launch of k_register, one CTA of 512 threads per SM.  Per cost evaluation:
//   1. every thread takes sampled pixels: Eq. 1 back-projection, rigid
//      transform, hash lookup of the 8 lattice corners, trilinear SDF and
//      intensity with analytic gradients, residuals and Jacobians
//      J = dV/dp [I | -[p]x] (left perturbation);
//   2. a warp-shuffle + shared-memory reduction of the 21 entries of J^T J,
//      the 6 of J^T r, the cost and the valid count gives one FP32 partial
//      per CTA;
//   3. a bounded grid barrier;
//   4. EVERY CTA reduces all partials (FP32, the same fixed order) and runs
//      the same LM step on its shared-memory copy of the LM state, on one
//      warp: accept or reject the candidate (mean cost E/N must decrease),
//      update lambda, solve the damped 6x6 system in FP64 (3x3 block
//      elimination) and compose the next candidate pose exp(delta) T in FP64.
//      Identical inputs and code give identical states in all CTAs, so no
//      broadcast is needed.
// The LM state never leaves shared memory; a level ends early when the step
// falls below the thresholds.  Results are deterministic: fixed grid, fixed
// pixel-to-thread mapping, fixed reduction order.
#include <cmath>
#include <type_traits>

#include "rf_volume.hpp"

namespace rf {
namespace {

__device__ __forceinline__ float lerpf(float a, float b, float t) { return a * (1.0f - t) + b * t; }

// Trilinear SDF/intensity lookup with analytic gradients (per metre).
// Corner n = dx + 2 dy + 4 dz.  Returns false unless all 8 corners exist and
// were observed; *colour is true when all 8 also carry colour.
// cached: the pixel's (key << 22 | pool) from an earlier sample, ~0 if none;
// *fresh receives a new entry when the block had to be looked up.
template <int ST>
__device__ __forceinline__ bool model_sample(const DevVol& v, const DevParams& p, float px, float py, float pz,
                                             float* V, float gV[3], float* I, float gI[3], bool* colour,
                                             unsigned long long cached, unsigned long long* fresh) {
  const float qx = px * p.inv_voxel, qy = py * p.inv_voxel, qz = pz * p.inv_voxel;
  if (!(fabsf(qx) < 1.0e6f && fabsf(qy) < 1.0e6f && fabsf(qz) < 1.0e6f)) return false;
  const float fkx = floorf(qx), fky = floorf(qy), fkz = floorf(qz);
  const int kx = (int)fkx, ky = (int)fky, kz = (int)fkz;
  const float fx = qx - fkx, fy = qy - fky, fz = qz - fkz;
  const int lx = kx & 7, ly = ky & 7, lz = kz & 7;
  const int bx = kx >> 3, by = ky >> 3, bz = kz >> 3;
  // FP32 storage: the uint2 words; FP16 storage: the 4-byte tracking words
  using Word = typename std::conditional<ST == RF_STORAGE_FP32, uint2, unsigned>::type;
  Word c[8];
  if (!coord_ok(bx, by, bz)) return false;
  const unsigned long long key = pack_key(bx, by, bz);
  int pool;
  if (cached != kEmpty && (cached >> 22) == key) {
    pool = (int)(cached & 0x3FFFFFull);  // same block as last time: no hash probe
  } else {
    pool = hash_find(v, bx, by, bz);
    if (pool < 0) return false;
    *fresh = (key << 22) | (unsigned long long)pool;
  }
  const Word* words = reinterpret_cast<const Word*>(v.vox);
  const size_t stride = ST == RF_STORAGE_FP32 ? kBV : 2 * kBV;  // words per block
  if (lx < 7 && ly < 7 && lz < 7) {
    const Word* base = words + (size_t)pool * stride + lx + 8 * ly + 64 * lz;
    c[0] = __ldg(base);
    c[1] = __ldg(base + 1);
    c[2] = __ldg(base + 8);
    c[3] = __ldg(base + 9);
    c[4] = __ldg(base + 64);
    c[5] = __ldg(base + 65);
    c[6] = __ldg(base + 72);
    c[7] = __ldg(base + 73);
  } else {
    // the cell straddles blocks: the neighbours' pools come from the table
    const int4 n0 = __ldg(v.nbr + 2 * (size_t)pool), n1 = __ldg(v.nbr + 2 * (size_t)pool + 1);
    const int nb[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int ix = lx + (n & 1), iy = ly + ((n >> 1) & 1), iz = lz + ((n >> 2) & 1);
      const int slot = (ix >> 3) + 2 * (iy >> 3) + 4 * (iz >> 3);
      const int pn = nb[slot];
      if (pn < 0) return false;
      c[n] = __ldg(words + (size_t)pn * stride + (ix & 7) + 8 * (iy & 7) + 64 * (iz & 7));
    }
  }
  float F[8];
  if constexpr (ST == RF_STORAGE_FP32) {
#pragma unroll
    for (int n = 0; n < 8; ++n) F[n] = __uint_as_float(c[n].x);
  } else {
#pragma unroll
    for (int n = 0; n < 8; ++n) F[n] = __half2float(__ushort_as_half((unsigned short)(c[n] & 0xFFFFu)));
  }
  // FP16 storage holds F / tau: values and gradients are scaled by tau once
  const float sdf_scale = ST == RF_STORAGE_FP32 ? 1.0f : p.tau;
  const float c00 = lerpf(F[0], F[1], fx), c10 = lerpf(F[2], F[3], fx);
  const float c01 = lerpf(F[4], F[5], fx), c11 = lerpf(F[6], F[7], fx);
  const float c0 = lerpf(c00, c10, fy), c1 = lerpf(c01, c11, fy);
  *V = lerpf(c0, c1, fz) * sdf_scale;
  // a never-observed corner stores NaN; every corner enters V with its
  // weight (0 * NaN = NaN), so one test covers all eight
  if (*V != *V) return false;
  const float gs_v = p.inv_voxel * sdf_scale;
  gV[0] = lerpf(lerpf(F[1] - F[0], F[3] - F[2], fy), lerpf(F[5] - F[4], F[7] - F[6], fy), fz) * gs_v;
  gV[1] = lerpf(lerpf(F[2] - F[0], F[3] - F[1], fx), lerpf(F[6] - F[4], F[7] - F[5], fx), fz) * gs_v;
  gV[2] = (c1 - c0) * gs_v;
  float In[8];
  float iscale;
  if constexpr (ST == RF_STORAGE_FP32) {
    // colour weights in the top bytes: their minimum over the corners
    const unsigned wmin = __vminu4(__vminu4(__vminu4(c[0].y, c[1].y), __vminu4(c[2].y, c[3].y)),
                                   __vminu4(__vminu4(c[4].y, c[5].y), __vminu4(c[6].y, c[7].y)));
    *colour = (wmin >> 24) != 0u;
    if (!*colour) return true;
#pragma unroll
    for (int n = 0; n < 8; ++n) In[n] = rgb_intensity_raw(c[n].y);  // intensities x 255e4
    iscale = kIntensityScale;
  } else {
    // I8 = 255 marks a corner without colour: the byte maximum over the corners
    const unsigned imax = __vmaxu4(__vmaxu4(__vmaxu4(c[0], c[1]), __vmaxu4(c[2], c[3])),
                                   __vmaxu4(__vmaxu4(c[4], c[5]), __vmaxu4(c[6], c[7])));
    *colour = ((imax >> 16) & 255u) != 255u;
    if (!*colour) return true;
#pragma unroll
    for (int n = 0; n < 8; ++n) In[n] = (float)((c[n] >> 16) & 255u);  // intensities x 254
    iscale = kI8Scale;
  }
  const float d00 = lerpf(In[0], In[1], fx), d10 = lerpf(In[2], In[3], fx);
  const float d01 = lerpf(In[4], In[5], fx), d11 = lerpf(In[6], In[7], fx);
  const float d0 = lerpf(d00, d10, fy), d1 = lerpf(d01, d11, fy);
  const float gs = iscale * p.inv_voxel;
  *I = lerpf(d0, d1, fz) * iscale;
  gI[0] = lerpf(lerpf(In[1] - In[0], In[3] - In[2], fy), lerpf(In[5] - In[4], In[7] - In[6], fy), fz) * gs;
  gI[1] = lerpf(lerpf(In[2] - In[0], In[3] - In[1], fx), lerpf(In[6] - In[4], In[7] - In[5], fx), fz) * gs;
  gI[2] = (d1 - d0) * gs;
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


// float -> double conversions run on GB300's thin FP64 pipe; these build the
// same values from the IEEE bit fields with integer operations.
// Exact float -> double (normal numbers, zeros, infinities, NaN; a subnormal
// float takes the converting instruction).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0u && (b & 0x7FFFFFu) != 0u) return (double)f;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long ed = e == 0u ? 0ull : (e == 0xFFu ? 0x7FFull : (unsigned long long)(e - 127u + 1023u));
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// A float within 2^-20 (relative) of a double whose exponent is in the
// normal float range; flags the other cases.
__device__ __forceinline__ float d2f_approx(double d, bool* ok) {
  const unsigned hi = (unsigned)(__double_as_longlong(d) >> 32);
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  *ok = e > -126 && e < 127;
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)(e + 127) << 23) | ((hi & 0xFFFFFu) << 3));
}

// d > 0 and finite (no FP64 instruction): the bit pattern of a positive
// finite double lies strictly between those of +0 and +infinity.
__device__ __forceinline__ bool pos_finite(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0ll && b < 0x7FF0000000000000ll;
}

// For non-negative doubles the bit patterns order like the values.
__device__ __forceinline__ bool nonneg_less(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}

// FP64 reciprocal: FP32 seed refined by two FP64 Newton steps (relative
// error ~(2^-20)^4, i.e. full double precision), far cheaper than a double
// division on GB300's FP64 pipe.
__device__ __forceinline__ double rcp_d(double d) {
  bool ok;
  const float df = d2f_approx(d, &ok);
  if (!ok) return 1.0 / d;
  double r = f2d_exact(__frcp_rn(df));
  r = fma(fma(-d, r, 1.0), r, r);
  r = fma(fma(-d, r, 1.0), r, r);
  return r;
}

// LM state of one registration, one copy in the shared memory of every CTA,
// plus the scratch of the warp-cooperative FP64 step.
struct LMShared {
  double T[16];   // accepted pose
  double Tc[16];  // candidate pose under evaluation
  double H[21], g[6], E;
  double lambda, fin_E;
  double red[29];
  // scratch of the damped 6x6 solve and of the exponential map
  double A6[36], adjP[9], Pi[9], X[12], Y[12], adjS[9], d[6], coef[3], Ex[12];
  long long N, fin_N;
  float redf[29];  // FP32 sums of the partials
  float Rf[12];    // float copy of T  (R row-major, then t)
  float Rcf[12];   // float copy of Tc
  int done, accept, solve_ok;
  rf_track_info info;
};

// (row, column) of the 21 upper-triangle entries of H, row-major
__constant__ unsigned char kUpperRow[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__constant__ unsigned char kUpperCol[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};
// Taylor coefficients in th^2 of A = sin(th)/th, B = (1 - cos th)/th^2 and
// C = (th - sin th)/th^3, highest power first (th^10 ... th^0)
__constant__ double kExpCoef[3][6] = {
    {-1.0 / 39916800.0, 1.0 / 362880.0, -1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0, 1.0},
    {-1.0 / 479001600.0, 1.0 / 3628800.0, -1.0 / 40320.0, 1.0 / 720.0, -1.0 / 24.0, 0.5},
    {-1.0 / 6227020800.0, 1.0 / 39916800.0, -1.0 / 362880.0, 1.0 / 5040.0, -1.0 / 120.0, 1.0 / 6.0}};

// Cofactor (r, c) of a row-major 3x3 matrix; the adjugate is its transpose.
__device__ __forceinline__ double cofactor3(const double* a, int r, int c) {
  const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
  return fma(a[r1 * 3 + c1], a[r2 * 3 + c2], -a[r1 * 3 + c2] * a[r2 * 3 + c1]);
}

// One LM step, executed by the 32 lanes of one warp.  On GB300 every FP64
// warp instruction costs the FP64 pipe about the same whatever the number of
// active lanes, so the work is spread across lanes and the number of FP64
// instructions on the critical path is kept small (about 70).
//   mode 0: first evaluation of a level, at T (always taken);
//   mode 1: evaluation of the candidate Tc, accepted when the mean cost
//           decreases (En/Nn < E/N, compared as En N < E Nn).
// Solve of (H + lambda diag H) d = -g in FP64 by 3x3 block elimination over
// the translation / rotation blocks, A = [P Q; Q^T S]:
//   P^-1 = adj(P)/det P,  [M | y1] = P^-1 [Q | b1],
//   [Sc | r2] = [S | b2] - Q^T [M | y1]  (Schur complement),
//   d2 = adj(Sc) r2 / det Sc,  d1 = y1 - M d2,  with b = -g.
// Then the next candidate Tc = exp(d) T (FP64), with the se(3) exponential
// R = I + A K + B K^2, t = (I + B K + C K^2) rho, K = [phi]x, K^2 = phi phi^T - th^2 I.
__device__ void lm_step_warp(LMShared& S, int mode, int level, bool last, const LMConst& c, int lane) {
  if (lane < 29) S.red[lane] = f2d_exact(S.redf[lane]);
  __syncwarp();
  if (lane == 0) {
    const double En = S.red[27];
    const long long Nn = (long long)(S.redf[28] + 0.5f);
    S.info.evals++;
    S.info.level_evals[level]++;
    S.solve_ok = 1;
    if (mode == 0) {
      S.accept = 1;
      S.E = En;
      S.N = Nn;
      S.fin_E = En;
      S.fin_N = Nn;
      S.done = Nn < c.min_valid ? 1 : 0;
      S.lambda = c.lambda0;
    } else if (Nn >= c.min_valid && En * f2d_exact((float)S.N) < S.E * f2d_exact((float)Nn)) {  // N < 2^24: exact
      S.accept = 2;
      S.E = En;
      S.N = Nn;
      S.fin_E = En;
      S.fin_N = Nn;
      S.lambda *= 0.1;
    } else {
      S.accept = 0;
      S.lambda *= 10.0;
    }
  }
  __syncwarp();
  const int acc = S.accept;
  if (acc) {
    if (lane < 21) S.H[lane] = S.red[lane];
    else if (lane < 27) S.g[lane - 21] = S.red[lane];
    if (acc == 2) {
      if (lane < 16) S.T[lane] = S.Tc[lane];
      if (lane < 12) S.Rf[lane] = S.Rcf[lane];
    }
  }
  __syncwarp();
  if (S.done || last) return;
  // damped matrix
  if (lane < 21) {
    const int i = kUpperRow[lane], j = kUpperCol[lane];
    const double h = i == j ? S.H[lane] * (1.0 + S.lambda) : S.H[lane];
    S.A6[i * 6 + j] = h;
    S.A6[j * 6 + i] = h;
  }
  __syncwarp();
  const double* A6 = S.A6;
  // P^-1
  if (lane < 9) {
    double P[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) P[k] = A6[(k / 3) * 6 + (k % 3)];
    S.adjP[lane] = cofactor3(P, lane % 3, lane / 3);
  }
  __syncwarp();
  const double detP = fma(A6[0], S.adjP[0], fma(A6[1], S.adjP[3], A6[2] * S.adjP[6]));
  if (!pos_finite(detP) || !pos_finite(A6[0])) {
    if (lane == 0) S.solve_ok = 0;
  } else {
    const double rP = rcp_d(detP);
    if (lane < 9) S.Pi[lane] = S.adjP[lane] * rP;
    __syncwarp();
    // [M | y1] = P^-1 [Q | b1]
    if (lane < 12) {
      const int r = lane >> 2, cc = lane & 3;
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) v = fma(S.Pi[r * 3 + k], cc < 3 ? A6[k * 6 + 3 + cc] : -S.g[k], v);
      S.X[lane] = v;
    }
    __syncwarp();
    // [Sc | r2] = [S | b2] - Q^T [M | y1]
    if (lane < 12) {
      const int r = lane >> 2, cc = lane & 3;
      double v = cc < 3 ? A6[(3 + r) * 6 + 3 + cc] : -S.g[3 + r];
#pragma unroll
      for (int k = 0; k < 3; ++k) v = fma(-A6[k * 6 + 3 + r], S.X[k * 4 + cc], v);
      S.Y[lane] = v;
    }
    __syncwarp();
    if (lane < 9) {
      double Sc[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Sc[k] = S.Y[(k / 3) * 4 + (k % 3)];
      S.adjS[lane] = cofactor3(Sc, lane % 3, lane / 3);
    }
    __syncwarp();
    const double detS = fma(S.Y[0], S.adjS[0], fma(S.Y[1], S.adjS[3], S.Y[2] * S.adjS[6]));
    if (!pos_finite(detS) || !pos_finite(S.Y[0])) {
      if (lane == 0) S.solve_ok = 0;
    } else {
      const double rS = rcp_d(detS);
      if (lane < 3) {
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) v = fma(S.adjS[lane * 3 + k], S.Y[k * 4 + 3], v);
        S.d[3 + lane] = v * rS;
      }
      __syncwarp();
      if (lane < 3) {
        double v = S.X[lane * 4 + 3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v = fma(-S.X[lane * 4 + k], S.d[3 + k], v);
        S.d[lane] = v;
      }
    }
  }
  __syncwarp();
  const double d0 = S.d[0], d1 = S.d[1], d2 = S.d[2], w0 = S.d[3], w1 = S.d[4], w2 = S.d[5];
  // |rho|^2 on even lanes and |phi|^2 on odd lanes in one pass, then exchanged
  const int o = (lane & 1) * 3;
  const double sq = fma(S.d[o], S.d[o], fma(S.d[o + 1], S.d[o + 1], S.d[o + 2] * S.d[o + 2]));
  const double sq_other = __shfl_xor_sync(0xffffffffu, sq, 1);
  const double nr2 = (lane & 1) ? sq_other : sq;
  const double th2 = (lane & 1) ? sq : sq_other;
  const double inf = __longlong_as_double(0x7FF0000000000000ll);
  if (!S.solve_ok || !nonneg_less(nr2, inf) || !nonneg_less(th2, inf)) {
    if (lane == 0) {
      S.info.converged[level] = 1;
      S.done = 1;
    }
    __syncwarp();
    return;
  }
  if (nonneg_less(nr2, c.eps_t2) && nonneg_less(th2, c.eps_r2)) {
    if (lane == 0) {
      S.info.converged[level] = 1;
      S.done = 1;
    }
    __syncwarp();
    return;
  }
  // exponential map: coefficients A, B, C on lanes 0, 1, 2
  if (lane < 3) {
    double v;
    if (th2 < 0.01) {
      v = kExpCoef[lane][0];
#pragma unroll
      for (int k = 1; k < 6; ++k) v = fma(v, th2, kExpCoef[lane][k]);
    } else {
      const double th = sqrt(th2);
      double sn, cs;
      sincos(th, &sn, &cs);
      v = lane == 0 ? sn / th : (lane == 1 ? (1.0 - cs) / th2 : (th - sn) / (th2 * th));
    }
    S.coef[lane] = v;
  }
  __syncwarp();
  // R (lanes 0-8) = I + A K + B K^2 and V (lanes 9-17) = I + B K + C K^2
  if (lane < 18) {
    const int e = lane % 9, i = e / 3, j = e % 3;
    const double w[3] = {w0, w1, w2};
    const double kij = (i == j) ? 0.0 : ((j == (i + 1) % 3) ? -w[(i + 2) % 3] : w[(i + 1) % 3]);
    const double k2ij = fma(w[i], w[j], i == j ? -th2 : 0.0);
    const double a = lane < 9 ? S.coef[0] : S.coef[1], b = lane < 9 ? S.coef[1] : S.coef[2];
    S.A6[lane] = fma(a, kij, fma(b, k2ij, i == j ? 1.0 : 0.0));  // scratch reuse
  }
  __syncwarp();
  if (lane < 12) {
    const int i = lane >> 2, j = lane & 3;
    // Ex = [R | V rho]
    double v;
    if (j < 3) {
      v = S.A6[i * 3 + j];
    } else {
      v = fma(S.A6[9 + i * 3], d0, fma(S.A6[9 + i * 3 + 1], d1, S.A6[9 + i * 3 + 2] * d2));
    }
    S.Ex[lane] = v;
  }
  __syncwarp();
  // Tc = Ex T  (rows 0-2; the last row stays 0 0 0 1)
  if (lane < 12) {
    const int i = lane >> 2, j = lane & 3;
    double v = j == 3 ? S.Ex[i * 4 + 3] : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) v = fma(S.Ex[i * 4 + k], S.T[k * 4 + j], v);
    S.Tc[lane] = v;
    S.Rcf[j < 3 ? i * 3 + j : 9 + i] = (float)v;
  }
  if (lane >= 12 && lane < 16) S.Tc[lane] = lane == 15 ? 1.0 : 0.0;
  __syncwarp();
}

constexpr int kRegThreads = 512;
constexpr int kRegWarps = kRegThreads / 32;

// Pixels per partial sum: a fixed chunk of the sampled pixels of a level
// (128 below 2^16 pixels, 512 below 2^18, else 2048), so the partials, and
// thus the result, do not depend on how many CTAs run the registration.
__device__ __forceinline__ int chunk_pixels(int npix) {
  return npix >= (1 << 18) ? 4 * kRegThreads : (npix >= (1 << 16) ? kRegThreads : kRegThreads / 4);
}
constexpr int kMaxPerThread = 4;  // pixels of one chunk per thread (chunk_pixels / kRegThreads at most)

// One whole registration (see the file comment) run by a group of G CTAs,
// this CTA being number lb of the group.  d.partials: 2 x 29 x max chunks
// floats (double-buffered by evaluation parity); d.bar: a zeroed counter.
template <int ST>
__device__ void register_body(const RegDesc& d, int lb, int G) {
  __shared__ LMShared S;
  __shared__ float red[kRegWarps][29];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DevFrame& f = d.f;
  const DevParams& p = d.p;
  if (threadIdx.x < 16) {
    S.T[threadIdx.x] = d.T_init[threadIdx.x];
    S.Tc[threadIdx.x] = d.T_init[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    S.done = 0;
    S.E = 0.0;
    S.N = 0;
    S.fin_E = 0.0;
    S.fin_N = 0;
    S.lambda = 0.0;
    rf_track_info z = {};
    S.info = z;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int i = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
    const int j = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
    S.Rf[threadIdx.x] = (float)S.T[i * 4 + j];
    S.Rcf[threadIdx.x] = S.Rf[threadIdx.x];
  }
  __syncthreads();
  int eval = 0;
  for (int l = 0; l < 3; ++l) {
    const int stride = d.c.strides[l];
    const int Ws = (f.W + stride - 1) / stride, Hs = (f.H + stride - 1) / stride;
    const int npix = Ws * Hs;
    const int chunk = chunk_pixels(npix);
    const int nchunks = (npix + chunk - 1) / chunk;
    // row = i / Ws by a reciprocal multiply (off by at most one for i < 2^32),
    // then one integer correction step
    const unsigned long long magic = (0x100000000ull + Ws - 1) / Ws;
    const int iters = d.c.iters[l];
    for (int it = 0; it <= iters; ++it) {
      const int mode = it == 0 ? 0 : 1;
      if (mode == 1 && S.done) break;  // identical decision in every CTA of the group
      const float* Tf = mode == 0 ? S.Rf : S.Rcf;
      const float R0 = Tf[0], R1 = Tf[1], R2 = Tf[2], R3 = Tf[3], R4 = Tf[4], R5 = Tf[5], R6 = Tf[6], R7 = Tf[7],
                  R8 = Tf[8], t0 = Tf[9], t1 = Tf[10], t2 = Tf[11];
      float* part = d.partials + (size_t)(eval & 1) * 29 * d.max_chunks;
      // chunks narrower than the CTA run side by side, one per warp group
      // (slot): chunk lb + G (slot + slots it) at step it
      const int width = min(chunk, kRegThreads);  // threads per chunk
      const int slots = kRegThreads / width;
      const int slot = threadIdx.x / width, tin = threadIdx.x % width;
      for (int step = 0; lb + G * slots * step < nchunks; ++step) {
        const int ch = lb + G * (slot + slots * step);
        float acc[29];
#pragma unroll
        for (int i = 0; i < 29; ++i) acc[i] = 0.0f;
        const int end = ch < nchunks ? min(npix, (ch + 1) * chunk) : 0;
        // this thread's pixels of the chunk (at most kMaxPerThread): depth,
        // mask and colour loaded up front, so their latencies overlap; the
        // samples are then taken in the same order as the pixels
        unsigned praw[kMaxPerThread], puv[kMaxPerThread], prgb[kMaxPerThread];
        unsigned long long pcache[kMaxPerThread];
#pragma unroll
        for (int j = 0; j < kMaxPerThread; ++j) {
          const int i = ch * chunk + tin + j * kRegThreads;
          praw[j] = 0u;
          puv[j] = 0u;
          prgb[j] = 0u;
          pcache[j] = kEmpty;
          if (i < end) {
            int row = (int)(((unsigned long long)i * magic) >> 32);
            if (row * Ws > i) --row;
            else if ((row + 1) * Ws <= i) ++row;
            const int u = (i - row * Ws) * stride, vv = row * stride;
            const int idx = vv * f.W + u;
            unsigned raw = __ldg(f.depth + idx);
            if (d.mask && __ldg(d.mask + idx)) raw = 0u;  // masked: not sampled
            const uint8_t* cp = f.rgb + 3 * (size_t)idx;
            praw[j] = raw;
            puv[j] = (unsigned)u | ((unsigned)vv << 16);
            if (raw != 0u && d.pxcache) pcache[j] = __ldcg(d.pxcache + idx);
            prgb[j] = (unsigned)__ldg(cp) | ((unsigned)__ldg(cp + 1) << 8) | ((unsigned)__ldg(cp + 2) << 16);
          }
        }
#pragma unroll 1
        for (int j = 0; j < kMaxPerThread; ++j) {
          // the next pixel's values rotate into slot 0 (registers, no local memory)
          const unsigned raw = praw[0], uvj = puv[0], rgbj = prgb[0];
          const unsigned long long cj = pcache[0];
#pragma unroll
          for (int r = 0; r + 1 < kMaxPerThread; ++r) {
            praw[r] = praw[r + 1];
            puv[r] = puv[r + 1];
            prgb[r] = prgb[r + 1];
            pcache[r] = pcache[r + 1];
          }
          if (!pixel_valid(p, raw)) continue;
          const int u = (int)(uvj & 0xFFFFu), vv = (int)(uvj >> 16);
          const float D = (float)raw * p.inv_depth_scale;
          const float x = ((float)u - f.cx) * f.ifx * D, y = ((float)vv - f.cy) * f.ify * D;
          const float px = R0 * x + R1 * y + R2 * D + t0;
          const float py = R3 * x + R4 * y + R5 * D + t1;
          const float pz = R6 * x + R7 * y + R8 * D + t2;
          float V, gV[3], I, gI[3];
          bool colour;
          unsigned long long fresh = kEmpty;
          const bool found = model_sample<ST>(d.v, p, px, py, pz, &V, gV, &I, gI, &colour, cj, &fresh);
          if (fresh != kEmpty && d.pxcache) __stcg(d.pxcache + (size_t)vv * f.W + u, fresh);
          if (!found) continue;
          const float Jd[6] = {gV[0], gV[1], gV[2], py * gV[2] - pz * gV[1], pz * gV[0] - px * gV[2],
                               px * gV[1] - py * gV[0]};
          add_jtj(acc, Jd, V, 1.0f);
          acc[28] += 1.0f;
          if (colour) {
            const float rc = I - rgb_intensity_raw(rgbj) * kIntensityScale;
            const float Jc[6] = {gI[0], gI[1], gI[2], py * gI[2] - pz * gI[1], pz * gI[0] - px * gI[2],
                                 px * gI[1] - py * gI[0]};
            add_jtj(acc, Jc, rc, p.w_c);
          }
        }
        // chunk partial: a butterfly over the warp that halves the vector at
        // every step (31 shuffles for 32 slots) and leaves component c on
        // lane c, then the warps in fixed order
        {
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = i < 29 ? acc[i] : 0.0f;
#pragma unroll
          for (int h = 16; h > 0; h >>= 1) {
            const bool upper = (lane & h) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
              const float keep = upper ? v[i + h] : v[i];
              const float send = upper ? v[i] : v[i + h];
              v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
          }
          if (lane < 29) red[warp][lane] = v[0];
        }
        __syncthreads();
        // the chunk partial of each slot: its warps' sums in order
        if (warp < slots && lane < 29) {
          const int cs = lb + G * (warp + slots * step);
          if (cs < nchunks) {
            const int wpc = width / 32;
            float sv = 0.0f;
            for (int w = 0; w < wpc; ++w) sv += red[warp * wpc + w][lane];
            part[lane * nchunks + cs] = sv;
          }
        }
        __syncthreads();
      }
      if (!grid_sync_counter(d.bar, (unsigned)(eval + 1) * (unsigned)G + d.bar_extra, d.status, d.spin_limit))
        return;
      // every CTA of the group: FP32 reduction of the chunk partials in a fixed
      // order (lane-strided sums, then a shuffle tree); L1 bypassed
      {
        const int ca = warp, cb = warp + kRegWarps;  // warp w: components w and w + 16
        const float* ra = part + ca * nchunks;
        const float* rb = part + (cb < 29 ? cb : ca) * nchunks;
        float fa = 0.0f, fb = 0.0f;
        for (int k = lane; k < nchunks; k += 32) {
          fa += __ldcg(ra + k);
          fb += __ldcg(rb + k);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fa += __shfl_down_sync(0xffffffffu, fa, o);
          fb += __shfl_down_sync(0xffffffffu, fb, o);
        }
        if (lane == 0) {
          S.redf[ca] = fa;
          if (cb < 29) S.redf[cb] = fb;
        }
      }
      __syncthreads();
      if (warp == 0) lm_step_warp(S, mode, l, it == iters, d.c, lane);
      __syncthreads();
      ++eval;
    }
  }
  if (lb == 0) {
    if (threadIdx.x < 16) d.T_out[threadIdx.x] = S.T[threadIdx.x];
    if (threadIdx.x == 0 && d.info) {
      rf_track_info out = S.info;
      out.final_cost = S.fin_N > 0 ? S.fin_E / (double)S.fin_N : 0.0;
      out.final_valid = S.fin_N;
      *d.info = out;
    }
  }
}

// One registration on the whole grid.
template <int ST>
__global__ void __launch_bounds__(kRegThreads, 1) k_register(RegDesc d) { register_body<ST>(d, blockIdx.x, gridDim.x); }

// Several independent registrations in one cooperative launch: CTA b runs
// stream cta_stream[b] as member b - first[s] of a group of first[s+1] -
// first[s] CTAs.  Groups never wait on each other.  A CTA mapped to stream
// -1 has no work (streams that sit a batch out, or are on their first frame,
// get no CTAs; the map is rewritten per batch without re-capturing the graph).
template <int ST>
__global__ void __launch_bounds__(kRegThreads, 1)
    k_register_batch(const RegDesc* __restrict__ descs, const int* __restrict__ cta_stream,
                     const int* __restrict__ first) {
  __shared__ RegDesc sd;
  const int s = cta_stream[blockIdx.x];
  if (s < 0) return;
  if (threadIdx.x == 0) sd = descs[s];
  __syncthreads();
  register_body<ST>(sd, blockIdx.x - first[s], first[s + 1] - first[s]);
}

}  // namespace

int register_max_grid(int device) {
  // the smallest residency over the kernels launched with this grid
  const void* fns[] = {(const void*)k_register<RF_STORAGE_FP32>, (const void*)k_register<RF_STORAGE_FP16>,
                       (const void*)k_register_batch<RF_STORAGE_FP32>, (const void*)k_register_batch<RF_STORAGE_FP16>};
  int per_sm = 1 << 20, sms = 0;
  for (const void* fn : fns) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kRegThreads, 0);
    per_sm = n < per_sm ? n : per_sm;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

RegDesc make_reg_desc(rf_volume* vol, const DevFrame& f, const double* T_init, const uint8_t* mask, double* T_out,
                      rf_track_info* info) {
  RegDesc d;
  d.v = vol->dv;
  d.f = f;
  d.p = vol->dp;
  d.mask = mask;
  d.T_init = T_init;
  d.T_out = T_out;
  d.info = info;
  d.c.lambda0 = vol->p.lm_lambda0;
  d.c.eps_t = vol->p.lm_eps_trans;
  d.c.eps_r = vol->p.lm_eps_rot;
  d.c.eps_t2 = vol->p.lm_eps_trans * vol->p.lm_eps_trans;
  d.c.eps_r2 = vol->p.lm_eps_rot * vol->p.lm_eps_rot;
  d.c.min_valid = vol->p.lm_min_valid;
  for (int l = 0; l < 3; ++l) {
    d.c.iters[l] = vol->p.lm_iters[l];
    d.c.strides[l] = vol->p.lm_strides[l];
  }
  d.partials = vol->d_partials;
  d.max_chunks = vol->max_chunks;
  d.bar = vol->d_regbar;
  d.status = vol->d_status;
  d.spin_limit = vol->wait_spins;
  d.bar_extra = vol->wait_extra;
  d.pxcache = vol->d_pxcache;
  return d;
}

static rf_status launch_coop(rf_volume* vol, const void* fn, int grid, void** args, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kRegThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return check_cuda(vol, cudaLaunchKernelExC(&cfg, fn, args), "registration launch");
}

rf_status launch_track(rf_volume* vol, const DevFrame& f, const double* T_init, const uint8_t* mask, double* T_out,
                       rf_track_info* info, cudaStream_t st) {
  RegDesc d = make_reg_desc(vol, f, T_init, mask, T_out, info);
  rf_status s = check_cuda(vol, cudaMemsetAsync(vol->d_regbar, 0, 2 * sizeof(unsigned), st), "barrier reset");
  if (s != RF_OK) return s;
  void* args[] = {&d};
  const void* fn = vol->p.storage == RF_STORAGE_FP16 ? (const void*)k_register<RF_STORAGE_FP16>
                                                     : (const void*)k_register<RF_STORAGE_FP32>;
  return launch_coop(vol, fn, vol->reg_grid, args, st);
}

rf_status launch_register_batch(rf_volume* vol, const RegDesc* descs, const int* cta_stream, const int* first,
                                int total_ctas, cudaStream_t st) {
  void* args[] = {(void*)&descs, (void*)&cta_stream, (void*)&first};
  const void* fn = vol->p.storage == RF_STORAGE_FP16 ? (const void*)k_register_batch<RF_STORAGE_FP16>
                                                     : (const void*)k_register_batch<RF_STORAGE_FP32>;
  return launch_coop(vol, fn, total_ctas, args, st);
}

}  // namespace rf
