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
//      per fixed chunk of pixels, written with the evaluation's tag;
//   3. EVERY CTA reads all partials, each until it carries the tag (this is
//      the only grid-wide wait, bounded), reduces them (FP32, the same fixed
//      order) and runs the same LM step on its shared-memory copy of the LM
//      state, on one warp: accept or reject the candidate (mean cost E/N must
//      decrease), update lambda, solve the damped 6x6 system and compose the
//      next candidate pose exp(delta) T (FP32 with exactly formed residuals
//      and a pose carried as float pairs; see lm_step_warp).  Identical
//      inputs and code give identical states in all CTAs, so no broadcast is
//      needed.
// The LM state never leaves shared memory; a level ends early when the step
// falls below the thresholds.  Results are deterministic: fixed chunks, fixed
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
      c[n] = __ldg(words + (size_t)pn[n] * stride + ix + 8 * iy + 64 * iz);
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
    for (int n = 0; n < 8; ++n) In[n] = u2f_exact((c[n] >> 16) & 255u);  // intensities x 254
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


// LM state of one registration, one copy in the shared memory of every CTA.
struct LMShared {
  float Ef;       // FP32 cost sum E of the accepted pose
  long long N, fin_N;
  float fin_E;
  int lam_k;            // damping lambda0 * 10^lam_k
  float Hf[21], gf[6];  // normal equations of the accepted pose (FP32 sums)
  float redf[29];       // FP32 sums of the partials of the evaluation just reduced
  // the accepted pose T and the candidate Tc (R row-major, then t), each
  // entry an unevaluated sum hi + lo of two floats (about 48 bits): hi is the
  // float pose an evaluation uses, hi + lo the pose itself
  float Rf[12], Rlf[12];
  float Rcf[12], Rclf[12];
  double T0[12];  // the initial pose, returned unchanged when no candidate is accepted
  int moved;      // some candidate was accepted
  int done;
  rf_track_info info;
};

// Packed index of entry (i, j), i <= j, of the upper triangle of a symmetric
// 6x6 matrix (row-major: the order of the 21 sums of J^T J).
__host__ __device__ constexpr int up6(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }


// FP32 Cholesky factorisation of the damped matrix in place: A holds the
// upper triangle (row-major) on entry and L^T (L's column j stored as row j of
// the upper triangle) on exit; inv[j] = 1 / L[j][j] from the hardware
// reciprocal square root (the factor only preconditions the refined solve).
// False unless every pivot is positive and finite.  Fully unrolled.
__device__ __forceinline__ bool chol6(float A[21], float inv[6]) {
  // every loop has constant bounds (with guards) so that it unrolls fully and
  // A stays in registers
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float s = A[up6(j, j)];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < j) s = fmaf(-A[up6(k, j)], A[up6(k, j)], s);
    ok = ok && (s > 0.0f) && (s < 3.0e38f);
    const float r = rsqrtf(fmaxf(s, 1.0e-30f));
    A[up6(j, j)] = s * r;
    inv[j] = r;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (i > j) {
        float t = A[up6(j, i)];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          if (k < j) t = fmaf(-A[up6(k, i)], A[up6(k, j)], t);
        A[up6(j, i)] = t * r;
      }
    }
  }
  return ok;
}

// Solves L L^T x = b in place (b -> x) with the factor of chol6 (FP32).
__device__ __forceinline__ void chol6_solve(const float A[21], const float inv[6], float b[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float t = b[i];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < i) t = fmaf(-A[up6(k, i)], b[k], t);
    b[i] = t * inv[i];
  }
#pragma unroll
  for (int ii = 0; ii < 6; ++ii) {
    const int i = 5 - ii;
    float t = b[i];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k > i) t = fmaf(-A[up6(i, k)], b[k], t);
    b[i] = t * inv[i];
  }
}

// Error-free transformations (Knuth's TwoSum, the FMA form of Dekker's
// TwoProduct): a + b = s + e and a b = p + e exactly in FP32 arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// a * na < b * nb, exactly, for finite floats a, b >= 0 and integers
// 0 <= na, nb < 2^24 (each product is a 48-bit integer times a power of two).
__device__ __forceinline__ bool prod_less(float a, unsigned na, float b, unsigned nb) {
  const unsigned ba = __float_as_uint(a), bb = __float_as_uint(b);
  const unsigned ea = (ba >> 23) & 255u, eb = (bb >> 23) & 255u;
  const unsigned long long P = (unsigned long long)((ba & 0x7FFFFFu) | (ea ? 0x800000u : 0u)) * na;
  const unsigned long long Q = (unsigned long long)((bb & 0x7FFFFFu) | (eb ? 0x800000u : 0u)) * nb;
  if (P == 0ull || Q == 0ull) return P == 0ull && Q != 0ull;
  const int xa = (int)(ea ? ea : 1u), xb = (int)(eb ? eb : 1u);  // exponent of the integer mantissa, + 150
  const int ta = 63 - __clzll((long long)P) + xa, tb = 63 - __clzll((long long)Q) + xb;
  if (ta != tb) return ta < tb;
  return xa >= xb ? (P << (xa - xb)) < Q : P < (Q << (xb - xa));
}

// One LM step, executed by the 32 lanes of one warp.  On GB300 a dependent
// FP64 instruction costs hundreds of cycles (measured with clock64 stamps in
// this loop: about 300-400 per dependent FP64 operation), and the step lies
// on the registration's serial critical path; so the step works in FP32 and
// reaches FP64-class accuracy where it matters without FP64 latency:
//   mode 0: first evaluation of a level, at T (always taken);
//   mode 1: evaluation of the candidate Tc, accepted when the mean cost
//           decreases (En/Nn < E/N, compared exactly as En N < E Nn on the
//           integer mantissas);
//   damping lambda = lambda0 10^k, k counting rejections minus acceptances;
//   solve of (H + lambda diag H) d = -g: FP32 Cholesky, then one step of
//   iterative refinement whose residual -g - A d is formed exactly (FP32
//   error-free transformations: the products of FP32 numbers and their sum
//   carried to about 2^-46), which gives the solution to the accuracy of an
//   FP64 solve for the systems met here (condition numbers ~10^2);
//   exp(d) - I = [A K + B K^2 | rho + B K rho + C K^2 rho] in FP32 (its
//   entries are of the order of the step, so FP32 is relative to the step);
//   the candidate pose Tc = T + (exp(d) - I) T: the increment in FP32, added
//   to the pose carried as float pairs with an error-free sum (lanes 0-11 in
//   parallel); the pair's high float is what the next evaluation uses.
__device__ void lm_step_warp(LMShared& S, int mode, int level, bool last, const LMConst& c, int lane) {
  const float Enf = S.redf[27];
  const long long Nn = (long long)(S.redf[28] + 0.5f);
  int accept;
  bool done = false;
  int k = S.lam_k;
  if (mode == 0) {
    accept = 1;
    k = 0;
    done = Nn < c.min_valid;
  } else if (Nn >= c.min_valid && prod_less(Enf, (unsigned)S.N, S.Ef, (unsigned)Nn)) {  // N < 2^24
    accept = 2;
    k = max(k - 1, -kLambdaPow);
  } else {
    accept = 0;
    k = min(k + 1, kLambdaPow);
  }
  __syncwarp();  // every lane has read the state before lane 0 updates it
  if (lane == 0) {
    S.info.evals++;
    S.info.level_evals[level]++;
    S.lam_k = k;
    if (accept) {
      S.Ef = Enf;
      S.N = Nn;
      S.fin_E = Enf;
      S.fin_N = Nn;
    }
    if (accept == 2) S.moved = 1;
    if (mode == 0) S.done = done ? 1 : 0;  // every level starts undone unless it has too few pixels
  }
  if (accept) {
    if (lane < 21) S.Hf[lane] = S.redf[lane];
    else if (lane < 27) S.gf[lane - 21] = S.redf[lane];
    if (accept == 2 && lane < 12) {
      S.Rf[lane] = S.Rcf[lane];
      S.Rlf[lane] = S.Rclf[lane];
    }
  }
  __syncwarp();
  if (done || last) return;  // (a candidate is only evaluated while the level is not done)
  const float lam = c.lambda_pow[k + kLambdaPow];
  // FP32 Cholesky of the damped matrix and first solution (every lane)
  float A[21], inv[6], d[6], r[6];
#pragma unroll
  for (int q = 0; q < 21; ++q) A[q] = S.Hf[q];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    A[up6(i, i)] = fmaf(A[up6(i, i)], lam, A[up6(i, i)]);
    d[i] = -S.gf[i];
  }
  const bool ok = chol6(A, inv);
  chol6_solve(A, inv, d);
  // residual -g - (H + lambda diag H) d, exact to about 2^-46: row i on
  // lane i, then gathered on every lane
  {
    const int i = lane < 6 ? lane : 0;
    float sh = -S.gf[i], sl = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float h = S.Hf[i <= j ? up6(i, j) : up6(j, i)];
      float p, pe, e;
      two_prod(h, d[j], p, pe);
      two_sum(sh, -p, sh, e);
      sl += e - pe;
      if (i == j) {  // the damping term lambda h d
        float lh, lhe;
        two_prod(lam, h, lh, lhe);
        two_prod(lh, d[j], p, pe);
        two_sum(sh, -p, sh, e);
        sl += e - pe - lhe * d[j];
      }
    }
    const float ri = sh + sl;
#pragma unroll
    for (int q = 0; q < 6; ++q) r[q] = __shfl_sync(0xffffffffu, ri, q);
  }
  chol6_solve(A, inv, r);
#pragma unroll
  for (int q = 0; q < 6; ++q) d[q] += r[q];  // the refined step
  const float nr2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
  const float p0 = d[3], p1 = d[4], p2 = d[5];
  const float t2 = fmaf(p0, p0, fmaf(p1, p1, p2 * p2));
  if (!ok || !(nr2 < 3.0e38f) || !(t2 < 3.0e38f) || (nr2 < c.eps_t2f && t2 < c.eps_r2f)) {
    if (lane == 0) {
      S.info.converged[level] = 1;
      S.done = 1;
    }
    __syncwarp();
    return;
  }
  // exponential map minus identity: A, B, C of theta^2
  float cA, cB, cC;
  if (t2 < 0.01f) {  // Taylor series in theta^2, enough terms for FP32 below theta = 0.1
    cA = fmaf(t2, fmaf(t2, fmaf(t2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    cB = fmaf(t2, fmaf(t2, fmaf(t2, -1.0f / 40320.0f, 1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
    cC = fmaf(t2, fmaf(t2, fmaf(t2, -1.0f / 362880.0f, 1.0f / 5040.0f), -1.0f / 120.0f), 1.0f / 6.0f);
  } else {
    const float th = sqrtf(t2);
    float sn, cs;
    sincospif(th * 0.318309886183790672f, &sn, &cs);  // argument reduction by pi is exact
    cA = sn / th;
    cB = (1.0f - cs) / t2;
    cC = (th - sn) / (t2 * th);
  }
  // increment (exp(d) - I) T in FP32 from the float pose, added to the pose
  // carried as float pairs (lanes 0-11: rows 0-2, columns 0-3).  Row i of
  // exp(d) - I: Er = A K + B K^2 with K v = phi x v and K^2 = phi phi^T -
  // theta^2 I; et = rho + B K rho + C K^2 rho.
  if (lane < 12) {
    const int i = lane >> 2, j = lane & 3;
    const float pi = i == 0 ? p0 : (i == 1 ? p1 : p2);
    // row i of K: (K_i0, K_i1, K_i2)
    const float k0 = i == 0 ? 0.0f : (i == 1 ? p2 : -p1);
    const float k1 = i == 0 ? -p2 : (i == 1 ? 0.0f : p0);
    const float k2 = i == 0 ? p1 : (i == 1 ? -p0 : 0.0f);
    const float e0 = fmaf(cA, k0, cB * fmaf(pi, p0, i == 0 ? -t2 : 0.0f));
    const float e1 = fmaf(cA, k1, cB * fmaf(pi, p1, i == 1 ? -t2 : 0.0f));
    const float e2 = fmaf(cA, k2, cB * fmaf(pi, p2, i == 2 ? -t2 : 0.0f));
    const float c0 = S.Rf[j < 3 ? j : 9], c1 = S.Rf[j < 3 ? 3 + j : 10], c2 = S.Rf[j < 3 ? 6 + j : 11];
    float inc = fmaf(e0, c0, fmaf(e1, c1, e2 * c2));
    if (j == 3) {  // + (rho + B K rho + C K^2 rho)_i
      const float kr = fmaf(k0, d[0], fmaf(k1, d[1], k2 * d[2]));  // (K rho)_i
      const float kr0 = p1 * d[2] - p2 * d[1], kr1 = p2 * d[0] - p0 * d[2], kr2 = p0 * d[1] - p1 * d[0];
      const float kk = fmaf(k0, kr0, fmaf(k1, kr1, k2 * kr2));  // (K K rho)_i
      const float rho_i = i == 0 ? d[0] : (i == 1 ? d[1] : d[2]);
      inc += fmaf(cC, kk, fmaf(cB, kr, rho_i));
    }
    const int fi = j < 3 ? i * 3 + j : 9 + i;
    float hi, lo;
    two_sum(S.Rf[fi], inc, hi, lo);
    lo += S.Rlf[fi];
    const float h2 = hi + lo;  // renormalised: h2 is the nearest float of the pair's sum
    S.Rcf[fi] = h2;
    S.Rclf[fi] = lo - (h2 - hi);
  }
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
constexpr int kReduceBatch = 8;   // partials per lane and component loaded at once in the reduction

// The pixels of chunk ch that thread tin of its slot samples (at most
// kMaxPerThread, kRegThreads apart): raw depth (0 where masked), (u, v) and
// packed RGB, and the pixel's cached block entry.  All loads are issued
// before any is used, so their latencies overlap.
struct PixelRegs {
  unsigned raw[kMaxPerThread], uv[kMaxPerThread], rgb[kMaxPerThread];
  unsigned long long cache[kMaxPerThread];
};

__device__ __forceinline__ void load_pixels(const RegDesc& d, PixelRegs& P, int ch, int chunk, int npix, int nchunks,
                                            int Ws, unsigned long long magic, int stride, int tin) {
  const DevFrame& f = d.f;
  const int end = ch < nchunks ? min(npix, (ch + 1) * chunk) : 0;
#pragma unroll
  for (int j = 0; j < kMaxPerThread; ++j) {
    const int i = ch * chunk + tin + j * kRegThreads;
    P.raw[j] = 0u;
    P.uv[j] = 0u;
    P.rgb[j] = 0u;
    P.cache[j] = kEmpty;
    if (i < end) {
      // row = i / Ws by a reciprocal multiply (off by at most one for
      // i < 2^32), then one integer correction step
      int row = (int)(((unsigned long long)i * magic) >> 32);
      if (row * Ws > i) --row;
      else if ((row + 1) * Ws <= i) ++row;
      const int u = (i - row * Ws) * stride, vv = row * stride;
      const int idx = vv * f.W + u;
      unsigned raw = __ldg(f.depth + idx);
      if (d.mask && __ldg(d.mask + idx)) raw = 0u;  // masked: not sampled
      const uint8_t* cp = f.rgb + 3 * (size_t)idx;
      P.raw[j] = raw;
      P.uv[j] = (unsigned)u | ((unsigned)vv << 16);
      if (raw != 0u && d.pxcache) P.cache[j] = __ldcg(d.pxcache + idx);
      P.rgb[j] = (unsigned)__ldg(cp) | ((unsigned)__ldg(cp + 1) << 8) | ((unsigned)__ldg(cp + 2) << 16);
    }
  }
}

// Every CTA of a registration group calls this once, after its last read of
// the partial sums.  The last CTA to leave clears the arrival count and
// advances the tag base past the
// registration's tags (at most 3 + the sum of the level iteration caps); when
// the tags would reach kTagLimit it first clears the whole partial buffer,
// whose tags then all read 0, and restarts the base at 0.  Either way every
// tag left in the buffer is below the next registration's tags.
__device__ __forceinline__ void leave_registration(const RegDesc& d, int lb, int G, unsigned tag0) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(d.tags + 1, 1u) == (unsigned)G - 1u;
  __syncthreads();
  if (!s_last) return;
  const unsigned span = (unsigned)(d.c.iters[0] + d.c.iters[1] + d.c.iters[2] + 3);
  unsigned next = tag0 + span;
  if (next >= kTagLimit - span) {
    const size_t n = (size_t)2 * 29 * d.max_slots;
    for (size_t i = threadIdx.x; i < n; i += kRegThreads) d.partials[i] = 0ull;
    next = 0u;
  }
  if (threadIdx.x == 0) {
    d.tags[2] = 0u;
    d.tags[1] = 0u;
    d.tags[0] = next;
  }
}

// One whole registration (see the file comment) run by a group of G CTAs,
// this CTA being number lb of the group.
//
// Exchange of the partial sums: evaluation e of the registration tags its
// partials with base + e + 1 (base: d.tags[0]) and then counts the CTA in
// d.tags[2] with a relaxed reduction; every CTA waits until the count shows
// all G arrivals of e, then reads the partials, re-polling any word that does
// not carry the tag yet (no fence orders a CTA's partials before its count,
// so the tags carry the ordering).  The count also makes double buffering by
// evaluation parity safe: a CTA writes evaluation e + 2 only after all G CTAs
// arrived at e + 1, each after it had read all of evaluation e.
template <int ST>
__device__ void register_body(const RegDesc& d, int lb, int G) {
  __shared__ LMShared S;
  __shared__ float red[2][kRegWarps][29];  // per-warp sums of a chunk, double-buffered by step parity
  __shared__ int s_arrived;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DevFrame& f = d.f;
  const DevParams& p = d.p;

  if (threadIdx.x == 0) {
    S.done = 0;
    S.Ef = 0.0f;
    S.N = 0;
    S.fin_E = 0.0f;
    S.fin_N = 0;
    S.lam_k = 0;
    S.moved = 0;
    rf_track_info z = {};
    S.info = z;
  }
  __syncthreads();
  if (threadIdx.x < 12) {  // the initial pose as float pairs (FP64 once per registration)
    const int i = threadIdx.x < 9 ? threadIdx.x / 3 : threadIdx.x - 9;
    const int j = threadIdx.x < 9 ? threadIdx.x % 3 : 3;
    const double t = d.T_init[i * 4 + j];
    S.T0[threadIdx.x] = t;
    const float hi = (float)t;
    S.Rf[threadIdx.x] = hi;
    S.Rlf[threadIdx.x] = (float)(t - (double)hi);
    S.Rcf[threadIdx.x] = hi;
    S.Rclf[threadIdx.x] = S.Rlf[threadIdx.x];
  }
  __syncthreads();
  const unsigned tag0 = ld_relaxed_gpu(d.tags);  // written by the previous registration's last CTA
  int eval = 0;
  bool failed = false;
  PixelRegs P;
  for (int l = 0; l < 3 && !failed; ++l) {
    const int stride = d.c.strides[l];
    const int Ws = (f.W + stride - 1) / stride, Hs = (f.H + stride - 1) / stride;
    const int npix = Ws * Hs;
    const int chunk = chunk_pixels(npix);
    const int nchunks = (npix + chunk - 1) / chunk;
    const unsigned long long magic = (0x100000000ull + Ws - 1) / Ws;
    const int iters = d.c.iters[l];
    bool pre = false;  // P already holds the pixels of the next step to run
    for (int it = 0; it <= iters; ++it) {
      const int mode = it == 0 ? 0 : 1;
      if (mode == 1 && S.done) break;  // identical decision in every CTA of the group
      const float* Tf = mode == 0 ? S.Rf : S.Rcf;
      const float R0 = Tf[0], R1 = Tf[1], R2 = Tf[2], R3 = Tf[3], R4 = Tf[4], R5 = Tf[5], R6 = Tf[6], R7 = Tf[7],
                  R8 = Tf[8], t0 = Tf[9], t1 = Tf[10], t2 = Tf[11];
      unsigned long long* part = d.partials + (size_t)(eval & 1) * 29 * d.max_slots;
      const unsigned tag = tag0 + (unsigned)eval + 1u;
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
        if (!pre) load_pixels(d, P, ch, chunk, npix, nchunks, Ws, magic, stride, tin);
#pragma unroll 1
        for (int j = 0; j < kMaxPerThread; ++j) {
          // the next pixel's values rotate into slot 0 (registers, no local memory)
          const unsigned raw = P.raw[0], uvj = P.uv[0], rgbj = P.rgb[0];
          const unsigned long long cj = P.cache[0];
#pragma unroll
          for (int r = 0; r + 1 < kMaxPerThread; ++r) {
            P.raw[r] = P.raw[r + 1];
            P.uv[r] = P.uv[r + 1];
            P.rgb[r] = P.rgb[r + 1];
            P.cache[r] = P.cache[r + 1];
          }
          if (!pixel_valid(p, raw)) continue;
          const int u = (int)(uvj & 0xFFFFu), vv = (int)(uvj >> 16);
          const float D = u2f_exact(raw) * p.inv_depth_scale;
          const float x = (u2f_exact((unsigned)u) - f.cx) * f.ifx * D, y = (u2f_exact((unsigned)vv) - f.cy) * f.ify * D;
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
          if (lane < 29) red[step & 1][warp][lane] = v[0];
        }
        // the next step's pixels: loads issued now, used after the partials
        pre = lb + G * slots * (step + 1) < nchunks;
        if (pre) load_pixels(d, P, ch + G * slots, chunk, npix, nchunks, Ws, magic, stride, tin);
        __syncthreads();
        // the chunk partial of each slot: its warps' sums in order, tagged.
        // No barrier after it: the next step writes the other buffer, and
        // this one again only after the next step's barrier, which these
        // reads precede.
        if (warp < slots && lane < 29) {
          const int cs = lb + G * (warp + slots * step);
          if (cs < nchunks) {
            const int wpc = width / 32;
            float sv = 0.0f;
            for (int w = 0; w < wpc; ++w) sv += red[step & 1][warp * wpc + w][lane];
            st_relaxed_gpu_u64(part + lane * nchunks + cs, ((unsigned long long)tag << 32) | __float_as_uint(sv));
          }
        }
      }
      // arrival: one relaxed count per CTA (other warps' partial stores may
      // still be on their way: the readers check the tags)
      if (threadIdx.x == 0) red_relaxed_gpu_add(d.tags + 2, 1u);
      // the next evaluation of this level samples the same pixels: their
      // loads are issued now and complete while the CTA waits for the others
      pre = it < iters;
      if (pre) load_pixels(d, P, lb + G * slot, chunk, npix, nchunks, Ws, magic, stride, tin);
      if (threadIdx.x == 0)
        s_arrived = await_count(d.tags + 2, (unsigned)(eval + 1) * (unsigned)G + d.bar_extra, d.spin_limit);
      __syncthreads();
      if (!s_arrived) {
        if (threadIdx.x == 0) atomicOr(d.status, ST_BARRIER);
        failed = true;
        break;
      }
      // every CTA of the group: FP32 reduction of the chunk partials in a fixed
      // order (lane-strided sums, then a shuffle tree); a word without this
      // evaluation's tag is read again until it has it
      bool ok = true;
      {
        const int ca = warp, cb = warp + kRegWarps;  // warp w: components w and w + 16
        const unsigned long long* ra = part + ca * nchunks;
        const unsigned long long* rb = part + (cb < 29 ? cb : ca) * nchunks;
        float fa = 0.0f, fb = 0.0f;
        for (int k0 = lane; k0 < nchunks && ok; k0 += 32 * kReduceBatch) {
          // the loads of a batch are issued together (one L2 round trip),
          // then checked and added in order
          unsigned long long va[kReduceBatch], vb[kReduceBatch];
#pragma unroll
          for (int u = 0; u < kReduceBatch; ++u) {
            const int k = k0 + 32 * u;
            va[u] = k < nchunks ? ld_relaxed_gpu_u64(ra + k) : 0ull;
            vb[u] = k < nchunks ? ld_relaxed_gpu_u64(rb + k) : 0ull;
          }
#pragma unroll
          for (int u = 0; u < kReduceBatch; ++u) {
            const int k = k0 + 32 * u;
            if (k < nchunks) {
              ok = ok && await_tag(ra + k, va[u], tag, d.spin_limit) && await_tag(rb + k, vb[u], tag, d.spin_limit);
              fa += __uint_as_float((unsigned)va[u]);
              fb += __uint_as_float((unsigned)vb[u]);
            }
          }
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
      if (!__syncthreads_and(ok)) {  // some wait ran out: leave, reporting it once per CTA
        if (threadIdx.x == 0) atomicOr(d.status, ST_BARRIER);
        failed = true;
        break;
      }
      if (warp == 0) lm_step_warp(S, mode, l, it == iters, d.c, lane);
      __syncthreads();
      ++eval;
    }
  }
  leave_registration(d, lb, G, tag0);
  if (failed) return;
  if (lb == 0) {
    if (threadIdx.x < 16) {  // the pose in FP64: hi + lo of each entry, the last row 0 0 0 1
      const int i = threadIdx.x >> 2, j = threadIdx.x & 3;
      const int fi = j < 3 ? i * 3 + j : 9 + i;
      d.T_out[threadIdx.x] = i == 3   ? (j == 3 ? 1.0 : 0.0)
                             : S.moved ? (double)S.Rf[fi] + (double)S.Rlf[fi]
                                       : S.T0[fi];
    }
    if (threadIdx.x == 0 && d.info) {
      rf_track_info out = S.info;
      out.final_cost = S.fin_N > 0 ? (double)S.fin_E / (double)S.fin_N : 0.0;
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
  d.c.eps_t2f = (float)(vol->p.lm_eps_trans * vol->p.lm_eps_trans);
  d.c.eps_r2f = (float)(vol->p.lm_eps_rot * vol->p.lm_eps_rot);
  for (int k = -kLambdaPow; k <= kLambdaPow; ++k)
    d.c.lambda_pow[k + kLambdaPow] = (float)(vol->p.lm_lambda0 * std::pow(10.0, (double)k));
  d.c.min_valid = vol->p.lm_min_valid;
  for (int l = 0; l < 3; ++l) {
    d.c.iters[l] = vol->p.lm_iters[l];
    d.c.strides[l] = vol->p.lm_strides[l];
  }
  d.partials = vol->d_partials;
  d.max_slots = vol->max_slots;
  d.tags = vol->d_regtags;
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
