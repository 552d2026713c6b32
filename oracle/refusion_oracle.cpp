// ReFusion FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (tests, smoke check,
// benchmark CPU baseline).  Plain sequential C++17: std::unordered_map of
// 8x8x8 voxel blocks, double-precision arithmetic in the paper's order, and
// 128-bit integers for every discrete geometric decision.  See
// refusion_oracle.h for the entry points.  Compile with -ffp-contract=off so
// that the specified FP64 evaluation order of the mask residual is kept.
//
// Passages followed (ReFusion, Palazzolo et al., IROS 2019):
//   Sec. III-A  TSDF voxels with weight and colour, running weighted average,
//               voxel hashing of blocks allocated on demand.
//   Sec. III-B  Eq. 1 back-projection, exp map of se(3), intensity
//               I = 0.2126 R + 0.7152 G + 0.0722 B, trilinear interpolation,
//               Eq. 2 depth error, Eq. 3 colour error, Eq. 4 joint error,
//               Levenberg-Marquardt on three coarse-to-fine sub-samplings.
//   Sec. III-C  Eq. 5 threshold t = gamma tau^2 on the residuals r_i of Eq. 2,
//               erosion, Alg. 1 depth-aware flood fill, dilation, second
//               registration without masked pixels, masked integration.
//   Sec. III-D  free-space carving: every non-occluded frustum voxel outside
//               the truncation band (up to a clipping plane) is averaged
//               towards tau.
//   Sec. III-E  invalid (zero) depth is ignored (first option); the second
//               option's virtual depth: zero pixels filled from a temporary
//               model by casting each pixel's ray through its TSDF.
//   Tab. I      default parameters.
//
// Readings where the paper is silent (shared definition with the CUDA path):
//   * pose T maps camera to world; voxel k sits at world position v*k;
//   * integration is projective: sdf = D(pixel) - z_cam(voxel), nearest pixel
//     u = floor(fx x/z + cx + 1/2); sdf < -tau: occluded (no update);
//     sdf > tau: free (value tau); colour averaged only inside the band;
//   * every discrete decision of integration is taken on exact integers:
//     positions in micrometres, world->camera rotation quantised as
//     llround(R^T 2^30), translation llround(t 1e6), camera coordinates
//     floor(. / 2^20) ("ticks" of 2^-10 um), intrinsics llround(f 256) and
//     llround((c + 1/2) 256);
//   * a block is allocated when at least one of its voxels is updated;
//   * weights count observations (1 each), capped at w_max; colour has its
//     own weight and is stored as RGB8, rounded half up at every update;
//   * the residual of the mask is V_SDF^2 (the underbraced term of Eq. 2),
//     V_SDF clamped to [-tau, tau] (the TSDF is truncated at tau), and seeds
//     are r_i > t; erosion/dilation are 3x3 squares (outside = 0);
//     Alg. 1 uses 4-neighbours and the test |D(p)-D(n)| 1e6 < theta_ppm D(p)
//     on raw integer depth;
//   * LM: H + lambda diag(H), lambda0 = 1e-4, /10 on accept, x10 on reject,
//     acceptance on decrease of the mean cost E/N, left update exp(d) T;
//     sub-sampling = pixel stride (4, 2, 1).
#include "refusion_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <unordered_set>
#include <vector>

typedef __int128 i128;

namespace {

constexpr int BS = 8;          // block edge in voxels
constexpr int BV = BS * BS * BS;

struct Block {
  double F[BV];
  int W[BV];
  int Wc[BV];
  uint8_t rgb[BV * 3];
  Block() {
    for (int i = 0; i < BV; ++i) { F[i] = 0.0; W[i] = 0; Wc[i] = 0; }
    std::memset(rgb, 0, sizeof(rgb));
  }
};

struct BlockKey {
  int64_t x, y, z;
  bool operator==(const BlockKey& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct BlockKeyHash {
  size_t operator()(const BlockKey& k) const {
    uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

struct Volume {
  orc_params p;
  std::unordered_map<BlockKey, Block, BlockKeyHash> blocks;
  int frames = 0;
  // integer forms of the parameters
  int64_t v_um, du_um, dmin_um, dmax_um, znear_tick, dmax_tick, tau_tick;
  // bookkeeping only (no effect on any result): when set, model lookups
  // record the distinct blocks they probe and voxels they read
  std::unordered_set<BlockKey, BlockKeyHash>* probed = nullptr;
  std::unordered_set<int64_t>* read = nullptr;
};

// floor(a / b) for b > 0
i128 floor_div(i128 a, i128 b) {
  i128 q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

int64_t floor_div64(int64_t a, int64_t b) { return (int64_t)floor_div((i128)a, (i128)b); }

void derive(Volume& V) {
  const orc_params& p = V.p;
  V.v_um = llround(p.voxel_size * 1e6);
  V.du_um = llround(1e6 / p.depth_scale);
  V.dmin_um = llround(p.d_min * 1e6);
  V.dmax_um = llround(p.d_max * 1e6);
  V.znear_tick = llround(p.z_near * 1e6) * 1024;
  V.dmax_tick = V.dmax_um * 1024;
  V.tau_tick = llround(p.trunc * 1e6 * 1024.0);
}

Block* find_block(Volume& V, int64_t bx, int64_t by, int64_t bz) {
  auto it = V.blocks.find(BlockKey{bx, by, bz});
  return it == V.blocks.end() ? nullptr : &it->second;
}

int vidx(int x, int y, int z) { return x + BS * y + BS * BS * z; }

// Depth of a raw pixel in micrometres; valid iff raw > 0 and inside [d_min, d_max].
bool pixel_depth(const Volume& V, uint16_t raw, int64_t* D_um) {
  if (raw == 0) return false;
  *D_um = (int64_t)raw * V.du_um;
  return *D_um >= V.dmin_um && *D_um <= V.dmax_um;
}

// Intensity of an RGB8 triple (Sec. III-B), scaled to [0, 1].
double intensity(const uint8_t* c) {
  return (0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]) / 255.0;
}

// ---------------------------------------------------------------------------
// quantised pose and exact voxel -> pixel association (integration)
// ---------------------------------------------------------------------------
struct QPose {
  i128 A[3][3];  // world->camera rotation R^T scaled by 2^30
  i128 t[3];     // camera centre in micrometres
};

QPose quantise(const double T[16]) {
  QPose q;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) q.A[i][j] = (i128)llround(T[j * 4 + i] * 1073741824.0);
  for (int i = 0; i < 3; ++i) q.t[i] = (i128)llround(T[i * 4 + 3] * 1e6);
  return q;
}

struct QIntr {
  i128 fx, fy, cx, cy;  // f * 256 and (c + 1/2) * 256
};

QIntr quantise_intr(const orc_frame* f) {
  QIntr q;
  q.fx = llround(f->fx * 256.0);
  q.fy = llround(f->fy * 256.0);
  q.cx = llround((f->cx + 0.5) * 256.0);
  q.cy = llround((f->cy + 0.5) * 256.0);
  return q;
}

// Observation of voxel k in this frame.  Returns false when the voxel is not
// updated (behind the near plane or beyond the clipping plane, outside the
// image, invalid or masked pixel, or occluded: sdf < -tau).
bool observe_voxel(const Volume& V, const orc_frame* f, const QPose& q, const QIntr& K,
                   const uint8_t* mask, const int64_t k[3], double* x, bool* band, int* pix) {
  i128 C[3];
  for (int i = 0; i < 3; ++i) {
    i128 s = 0;
    for (int j = 0; j < 3; ++j) s += q.A[i][j] * ((i128)V.v_um * k[j] - q.t[j]);
    C[i] = floor_div(s, (i128)1 << 20);
  }
  if (C[2] <= V.znear_tick || C[2] > V.dmax_tick) return false;
  i128 u = floor_div(K.fx * C[0] + K.cx * C[2], 256 * C[2]);
  i128 v = floor_div(K.fy * C[1] + K.cy * C[2], 256 * C[2]);
  if (u < 0 || u >= f->width || v < 0 || v >= f->height) return false;
  int idx = (int)v * f->width + (int)u;
  int64_t D_um;
  if (!pixel_depth(V, f->depth[idx], &D_um)) return false;
  if (mask && mask[idx]) return false;
  i128 sdf = (i128)D_um * 1024 - C[2];
  if (sdf < -(i128)V.tau_tick) return false;
  if (sdf > (i128)V.tau_tick) {
    *x = V.p.trunc;
    *band = false;
  } else {
    *x = (double)(int64_t)sdf / 1.024e9;
    *band = true;
  }
  *pix = idx;
  return true;
}

void apply_update(const Volume& V, Block& B, int vi, double x, bool band, const uint8_t* rgb) {
  int w = B.W[vi];
  B.F[vi] = (w == 0) ? x : (w * B.F[vi] + x) / (w + 1);
  B.W[vi] = std::min(w + 1, V.p.w_max);
  if (band) {
    int wc = B.Wc[vi];
    for (int ch = 0; ch < 3; ++ch) {
      int num = wc * B.rgb[vi * 3 + ch] + rgb[ch];
      B.rgb[vi * 3 + ch] = (uint8_t)((2 * num + (wc + 1)) / (2 * (wc + 1)));
    }
    B.Wc[vi] = std::min(wc + 1, V.p.w_max);
  }
}

int64_t integrate(Volume& V, const orc_frame* f, const double T[16], const uint8_t* mask) {
  const int H = f->height, W = f->width;
  int64_t maxD = -1;
  for (int i = 0; i < H * W; ++i) {
    int64_t D_um;
    if (pixel_depth(V, f->depth[i], &D_um) && !(mask && mask[i])) maxD = std::max(maxD, D_um);
  }
  if (maxD < 0) return 0;
  const double zfar = std::min(maxD * 1e-6 + V.p.trunc, V.p.d_max);
  // axis-aligned box around the truncated frustum (brute-force search region)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  const double us[2] = {-0.5, W - 0.5}, vs[2] = {-0.5, H - 0.5}, zs[2] = {V.p.z_near, zfar};
  for (double z : zs)
    for (double u : us)
      for (double v : vs) {
        double c[3] = {(u - f->cx) / f->fx * z, (v - f->cy) / f->fy * z, z};
        for (int i = 0; i < 3; ++i) {
          double w = T[i * 4 + 0] * c[0] + T[i * 4 + 1] * c[1] + T[i * 4 + 2] * c[2] + T[i * 4 + 3];
          lo[i] = std::min(lo[i], w);
          hi[i] = std::max(hi[i], w);
        }
      }
  const double bsize = BS * V.p.voxel_size, margin = 2 * V.p.voxel_size;
  int64_t bmin[3], bmax[3];
  for (int i = 0; i < 3; ++i) {
    bmin[i] = (int64_t)std::floor((lo[i] - margin) / bsize);
    bmax[i] = (int64_t)std::floor((hi[i] + margin) / bsize);
  }
  const QPose q = quantise(T);
  const QIntr K = quantise_intr(f);
  int64_t updated = 0;
  struct Obs { int vi; double x; bool band; int pix; };
  std::vector<Obs> obs;
  obs.reserve(BV);
  for (int64_t bz = bmin[2]; bz <= bmax[2]; ++bz)
    for (int64_t by = bmin[1]; by <= bmax[1]; ++by)
      for (int64_t bx = bmin[0]; bx <= bmax[0]; ++bx) {
        obs.clear();
        for (int z = 0; z < BS; ++z)
          for (int y = 0; y < BS; ++y)
            for (int x = 0; x < BS; ++x) {
              int64_t k[3] = {bx * BS + x, by * BS + y, bz * BS + z};
              Obs o;
              if (observe_voxel(V, f, q, K, mask, k, &o.x, &o.band, &o.pix)) {
                o.vi = vidx(x, y, z);
                obs.push_back(o);
              }
            }
        if (obs.empty()) continue;
        Block& B = V.blocks[BlockKey{bx, by, bz}];
        for (const Obs& o : obs) apply_update(V, B, o.vi, o.x, o.band, f->rgb + 3 * (size_t)o.pix);
        updated += (int64_t)obs.size();
      }
  return updated;
}

// ---------------------------------------------------------------------------
// model lookup: trilinear interpolation of SDF and intensity (Sec. III-B)
// ---------------------------------------------------------------------------
double lerp(double a, double b, double t) {
  double om = 1.0 - t;
  return a * om + b * t;
}

struct Corners {
  double F[8], I[8];
  bool colour;
};

// Gathers the 8 lattice corners k0 + (dx,dy,dz), corner index dx + 2 dy + 4 dz.
bool gather(Volume& V, const int64_t k0[3], Corners* c) {
  c->colour = true;
  for (int n = 0; n < 8; ++n) {
    int64_t k[3] = {k0[0] + (n & 1), k0[1] + ((n >> 1) & 1), k0[2] + ((n >> 2) & 1)};
    int64_t b[3];
    int l[3];
    for (int i = 0; i < 3; ++i) {
      b[i] = floor_div64(k[i], BS);
      l[i] = (int)(k[i] - b[i] * BS);
    }
    Block* B = find_block(V, b[0], b[1], b[2]);
    if (V.probed) V.probed->insert(BlockKey{b[0], b[1], b[2]});
    if (!B) return false;
    int vi = vidx(l[0], l[1], l[2]);
    if (V.read) V.read->insert((k[0] & 0x1FFFFF) | ((k[1] & 0x1FFFFF) << 21) | ((k[2] & 0x1FFFFF) << 42));
    if (B->W[vi] <= 0) return false;
    c->F[n] = B->F[vi];
    c->I[n] = intensity(B->rgb + 3 * vi);
    if (B->Wc[vi] <= 0) c->colour = false;
  }
  return true;
}

// V(f) by nested lerps: along x, then y, then z (the fixed evaluation order).
double trilinear(const double v[8], const double f[3]) {
  double c00 = lerp(v[0], v[1], f[0]);
  double c10 = lerp(v[2], v[3], f[0]);
  double c01 = lerp(v[4], v[5], f[0]);
  double c11 = lerp(v[6], v[7], f[0]);
  double c0 = lerp(c00, c10, f[1]);
  double c1 = lerp(c01, c11, f[1]);
  return lerp(c0, c1, f[2]);
}

// Analytic gradient of the trilinear interpolant w.r.t. f (per voxel unit).
void trilinear_grad(const double v[8], const double f[3], double g[3]) {
  for (int a = 0; a < 3; ++a) {
    double s = 0.0;
    for (int n = 0; n < 8; ++n) {
      double w = 1.0;
      for (int d = 0; d < 3; ++d) {
        int bit = (n >> d) & 1;
        if (d == a) w *= bit ? 1.0 : -1.0;
        else w *= bit ? f[d] : 1.0 - f[d];
      }
      s += w * v[n];
    }
    g[a] = s;
  }
}

bool cell_of(const Volume& V, const double p[3], int64_t k0[3], double fr[3]) {
  for (int i = 0; i < 3; ++i) {
    double q = p[i] / V.p.voxel_size;
    if (!(std::fabs(q) < 1e9)) return false;
    double fl = std::floor(q);
    k0[i] = (int64_t)fl;
    fr[i] = q - fl;
  }
  return true;
}

bool lookup(Volume& V, const double p[3], double* sdf, double gs[3], double* I, double gI[3],
            bool* colour) {
  int64_t k0[3];
  double fr[3];
  if (!cell_of(V, p, k0, fr)) return false;
  Corners c;
  if (!gather(V, k0, &c)) return false;
  *sdf = trilinear(c.F, fr);
  trilinear_grad(c.F, fr, gs);
  for (int i = 0; i < 3; ++i) gs[i] /= V.p.voxel_size;
  *colour = c.colour;
  if (c.colour) {
    *I = trilinear(c.I, fr);
    trilinear_grad(c.I, fr, gI);
    for (int i = 0; i < 3; ++i) gI[i] /= V.p.voxel_size;
  } else {
    *I = 0.0;
    gI[0] = gI[1] = gI[2] = 0.0;
  }
  return true;
}

// Eq. 1 back-projection followed by the rigid transform T (camera -> world),
// in the fixed evaluation order.
void backproject_world(const orc_frame* f, int u, int v, double D, const double T[16], double p[3]) {
  double x = ((u - f->cx) / f->fx) * D;
  double y = ((v - f->cy) / f->fy) * D;
  double z = D;
  for (int i = 0; i < 3; ++i) p[i] = ((T[i * 4 + 0] * x + T[i * 4 + 1] * y) + T[i * 4 + 2] * z) + T[i * 4 + 3];
}

// ---------------------------------------------------------------------------
// registration (Sec. III-B)
// ---------------------------------------------------------------------------
void eval_normal_eq(Volume& V, const orc_frame* f, const double T[16], int s, const uint8_t* mask,
                    double Hm[6][6], double g[6], double* E, int64_t* N) {
  for (int i = 0; i < 6; ++i) {
    g[i] = 0.0;
    for (int j = 0; j < 6; ++j) Hm[i][j] = 0.0;
  }
  *E = 0.0;
  *N = 0;
  for (int v = 0; v < f->height; v += s)
    for (int u = 0; u < f->width; u += s) {
      int idx = v * f->width + u;
      int64_t D_um;
      if (!pixel_depth(V, f->depth[idx], &D_um)) continue;
      if (mask && mask[idx]) continue;
      double D = f->depth[idx] / V.p.depth_scale;
      double p[3];
      backproject_world(f, u, v, D, T, p);
      double sdf, gs[3], I, gI[3];
      bool colour;
      if (!lookup(V, p, &sdf, gs, &I, gI, &colour)) continue;
      // d p / d xi = [I | -[p]x] for the left perturbation exp(xi) T
      double Jd[6] = {gs[0], gs[1], gs[2], p[1] * gs[2] - p[2] * gs[1], p[2] * gs[0] - p[0] * gs[2],
                      p[0] * gs[1] - p[1] * gs[0]};
      for (int i = 0; i < 6; ++i) {
        g[i] += Jd[i] * sdf;
        for (int j = 0; j < 6; ++j) Hm[i][j] += Jd[i] * Jd[j];
      }
      *E += sdf * sdf;
      *N += 1;
      if (colour) {
        double rc = I - intensity(f->rgb + 3 * (size_t)idx);
        double Jc[6] = {gI[0], gI[1], gI[2], p[1] * gI[2] - p[2] * gI[1], p[2] * gI[0] - p[0] * gI[2],
                        p[0] * gI[1] - p[1] * gI[0]};
        const double wc = V.p.w_c;
        for (int i = 0; i < 6; ++i) {
          g[i] += wc * Jc[i] * rc;
          for (int j = 0; j < 6; ++j) Hm[i][j] += wc * Jc[i] * Jc[j];
        }
        *E += wc * rc * rc;
      }
    }
}

void mat4_mul(const double A[16], const double B[16], double C[16]) {
  double R[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[i * 4 + k] * B[k * 4 + j];
      R[i * 4 + j] = s;
    }
  std::memcpy(C, R, sizeof(R));
}

void se3_exp(const double xi[6], double T[16]) {
  const double* rho = xi;
  const double* phi = xi + 3;
  double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  double th = std::sqrt(th2);
  double A, B, C;
  if (th < 1e-5) {
    A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
    B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
  } else {
    A = std::sin(th) / th;
    B = (1.0 - std::cos(th)) / th2;
    C = (th - std::sin(th)) / (th2 * th);
  }
  double K[3][3] = {{0, -phi[2], phi[1]}, {phi[2], 0, -phi[0]}, {-phi[1], phi[0], 0}};
  double K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += K[i][k] * K[k][j];
      K2[i][j] = s;
    }
  double R[3][3], Vm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double I = (i == j) ? 1.0 : 0.0;
      R[i][j] = I + A * K[i][j] + B * K2[i][j];
      Vm[i][j] = I + B * K[i][j] + C * K2[i][j];
    }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T[i * 4 + j] = R[i][j];
    T[i * 4 + 3] = Vm[i][0] * rho[0] + Vm[i][1] * rho[1] + Vm[i][2] * rho[2];
  }
  T[12] = T[13] = T[14] = 0.0;
  T[15] = 1.0;
}

// (H + lambda diag H) delta = -g by Cholesky; false if not positive definite.
bool lm_solve(const double Hm[6][6], const double g[6], double lambda, double delta[6]) {
  double A[6][6], L[6][6] = {{0}};
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) A[i][j] = Hm[i][j];
  for (int i = 0; i < 6; ++i) A[i][i] = Hm[i][i] * (1.0 + lambda);
  for (int j = 0; j < 6; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    L[j][j] = std::sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
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
    for (int k = i + 1; k < 6; ++k) s -= L[k][i] * delta[k];
    delta[i] = s / L[i][i];
  }
  return true;
}

void track(Volume& V, const orc_frame* f, const double T_init[16], const uint8_t* mask, double T_out[16],
           orc_track_info* info) {
  double T[16];
  std::memcpy(T, T_init, sizeof(T));
  orc_track_info inf;
  std::memset(&inf, 0, sizeof(inf));
  for (int l = 0; l < 3; ++l) {
    const int s = V.p.lm_strides[l];
    double Hm[6][6], g[6], E;
    int64_t N;
    eval_normal_eq(V, f, T, s, mask, Hm, g, &E, &N);
    inf.evals++;
    inf.level_evals[l]++;
    inf.final_cost = N > 0 ? E / N : 0.0;
    inf.final_valid = N;
    if (N < V.p.lm_min_valid) continue;
    double lambda = V.p.lm_lambda0;
    for (int it = 0; it < V.p.lm_iters[l]; ++it) {
      double d[6];
      if (!lm_solve(Hm, g, lambda, d)) { inf.converged[l] = 1; break; }
      double nr = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double nphi = std::sqrt(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
      if (nr < V.p.lm_eps_trans && nphi < V.p.lm_eps_rot) { inf.converged[l] = 1; break; }
      double Ex[16], Tc[16];
      se3_exp(d, Ex);
      mat4_mul(Ex, T, Tc);
      double Hc[6][6], gc[6], Ec;
      int64_t Nc;
      eval_normal_eq(V, f, Tc, s, mask, Hc, gc, &Ec, &Nc);
      inf.evals++;
      inf.level_evals[l]++;
      if (Nc >= V.p.lm_min_valid && Ec / Nc < E / N) {
        std::memcpy(T, Tc, sizeof(T));
        std::memcpy(Hm, Hc, sizeof(Hm));
        std::memcpy(g, gc, sizeof(g));
        E = Ec;
        N = Nc;
        lambda /= 10.0;
        inf.final_cost = E / N;
        inf.final_valid = N;
      } else {
        lambda *= 10.0;
      }
    }
  }
  std::memcpy(T_out, T, sizeof(T));
  if (info) *info = inf;
}

// ---------------------------------------------------------------------------
// dynamics detection (Sec. III-C)
// ---------------------------------------------------------------------------
void residual_seeds(Volume& V, const orc_frame* f, const double T[16], double* r, uint8_t* seeds) {
  const double t = (V.p.gamma * V.p.trunc) * V.p.trunc;  // Eq. 5
  for (int v = 0; v < f->height; ++v)
    for (int u = 0; u < f->width; ++u) {
      int idx = v * f->width + u;
      double ri = -1.0;
      int64_t D_um;
      if (pixel_depth(V, f->depth[idx], &D_um)) {
        double D = f->depth[idx] / V.p.depth_scale;
        double p[3];
        backproject_world(f, u, v, D, T, p);
        int64_t k0[3];
        double fr[3];
        Corners c;
        if (cell_of(V, p, k0, fr) && gather(V, k0, &c)) {
          // the model is a TSDF truncated at tau (Sec. III-A)
          double sdf = std::min(std::max(trilinear(c.F, fr), -V.p.trunc), V.p.trunc);
          ri = sdf * sdf;  // r_i of Eq. 2
        }
      }
      if (r) r[idx] = ri;
      if (seeds) seeds[idx] = (ri >= 0.0 && ri > t) ? 1 : 0;
    }
}

void erode3(const uint8_t* in, int H, int W, uint8_t* out) {
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      int all = 1;
      for (int dv = -1; dv <= 1; ++dv)
        for (int du = -1; du <= 1; ++du) {
          int y = v + dv, x = u + du;
          if (y < 0 || y >= H || x < 0 || x >= W || !in[y * W + x]) all = 0;
        }
      out[v * W + u] = (uint8_t)all;
    }
}

void dilate3(const uint8_t* in, int H, int W, uint8_t* out) {
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      int any = 0;
      for (int dv = -1; dv <= 1; ++dv)
        for (int du = -1; du <= 1; ++du) {
          int y = v + dv, x = u + du;
          if (y >= 0 && y < H && x >= 0 && x < W && in[y * W + x]) any = 1;
        }
      out[v * W + u] = (uint8_t)any;
    }
}

// Alg. 1: grow M_D from the pixels of M_R through 4-neighbours n of p with
// |D(p) - D(n)| < theta D(p), on raw integer depth with theta in ppm.
void floodfill(const uint8_t* MR, const uint16_t* depth, int H, int W, int64_t theta_ppm, uint8_t* MD) {
  std::vector<uint8_t> queued(H * W, 0);
  std::deque<int> Q;
  for (int i = 0; i < H * W; ++i) {
    MD[i] = 0;
    if (MR[i]) { Q.push_back(i); queued[i] = 1; }
  }
  const int du[4] = {1, -1, 0, 0}, dv[4] = {0, 0, 1, -1};
  while (!Q.empty()) {
    int p = Q.front();
    Q.pop_front();
    MD[p] = 1;
    int pu = p % W, pv = p / W;
    int64_t Dp = depth[p];
    for (int n = 0; n < 4; ++n) {
      int x = pu + du[n], y = pv + dv[n];
      if (x < 0 || x >= W || y < 0 || y >= H) continue;
      int q = y * W + x;
      if (queued[q]) continue;
      int64_t Dn = depth[q];
      int64_t diff = Dp > Dn ? Dp - Dn : Dn - Dp;
      if (diff * 1000000 < theta_ppm * Dp) {
        queued[q] = 1;
        Q.push_back(q);
      }
    }
  }
}

void compute_mask(Volume& V, const orc_frame* f, const double T[16], uint8_t* mask) {
  const int H = f->height, W = f->width;
  std::vector<uint8_t> seeds(H * W), MR(H * W), MD(H * W);
  residual_seeds(V, f, T, nullptr, seeds.data());
  erode3(seeds.data(), H, W, MR.data());
  floodfill(MR.data(), f->depth, H, W, llround(V.p.theta * 1e6), MD.data());
  dilate3(MD.data(), H, W, mask);
}

// ---------------------------------------------------------------------------
// mesh: marching tetrahedra over cells with 8 observed corners
// ---------------------------------------------------------------------------
int perm_parity(const int* a, int n) {
  int inv = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (a[i] > a[j]) inv++;
  return inv & 1;
}

struct MeshOut {
  double* verts;
  uint8_t* colors;
  int64_t cap, n;
};

void emit_vertex(MeshOut& M, int64_t slot, const double pa[3], const double pb[3], double Fa, double Fb,
                 const uint8_t* ca, bool oka, const uint8_t* cb, bool okb) {
  double t = Fa / (Fa - Fb);
  for (int i = 0; i < 3; ++i) M.verts[slot * 3 + i] = pa[i] + t * (pb[i] - pa[i]);
  for (int ch = 0; ch < 3; ++ch) {
    double c;
    if (oka && okb) c = ca[ch] + t * ((double)cb[ch] - ca[ch]);
    else if (oka) c = ca[ch];
    else if (okb) c = cb[ch];
    else c = 0.0;
    M.colors[slot * 3 + ch] = (uint8_t)std::lround(c);
  }
}

int64_t extract_mesh(Volume& V, double* verts, uint8_t* colors, int64_t cap) {
  std::vector<BlockKey> keys;
  for (auto& kv : V.blocks) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end(), [](const BlockKey& a, const BlockKey& b) {
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  MeshOut M{verts, colors, cap, 0};
  const bool write = verts && colors;
  const int axes_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (const BlockKey& bk : keys)
    for (int z = 0; z < BS; ++z)
      for (int y = 0; y < BS; ++y)
        for (int x = 0; x < BS; ++x) {
          int64_t k0[3] = {bk.x * BS + x, bk.y * BS + y, bk.z * BS + z};
          double F[8], P[8][3];
          uint8_t C[8][3];
          bool ok[8];
          bool valid = true;
          for (int n = 0; n < 8 && valid; ++n) {
            int64_t k[3] = {k0[0] + (n & 1), k0[1] + ((n >> 1) & 1), k0[2] + ((n >> 2) & 1)};
            int64_t b[3];
            int l[3];
            for (int i = 0; i < 3; ++i) {
              b[i] = floor_div64(k[i], BS);
              l[i] = (int)(k[i] - b[i] * BS);
            }
            Block* B = find_block(V, b[0], b[1], b[2]);
            int vi = vidx(l[0], l[1], l[2]);
            if (!B || B->W[vi] <= 0) { valid = false; break; }
            F[n] = B->F[vi];
            for (int i = 0; i < 3; ++i) P[n][i] = k[i] * V.p.voxel_size;
            std::memcpy(C[n], B->rgb + 3 * vi, 3);
            ok[n] = B->Wc[vi] > 0;
          }
          if (!valid) continue;
          for (int pi = 0; pi < 6; ++pi) {
            // Kuhn tetrahedron: 0 -> e_a -> e_a + e_b -> 7
            int a = axes_perm[pi][0], b = axes_perm[pi][1];
            int tv[4] = {0, 1 << a, (1 << a) | (1 << b), 7};
            int par = perm_parity(axes_perm[pi], 3);
            if (par) std::swap(tv[1], tv[2]);  // positive orientation
            int inside[4], outside[4], ni = 0, no = 0;
            for (int i = 0; i < 4; ++i) {
              if (F[tv[i]] < 0.0) inside[ni++] = i;
              else outside[no++] = i;
            }
            if (ni == 0 || ni == 4) continue;
            // orderings of tetra positions with even parity relative to tv
            auto edge = [&](int64_t slot, int i, int j) {
              int va = tv[i], vb = tv[j];
              emit_vertex(M, slot, P[va], P[vb], F[va], F[vb], C[va], ok[va], C[vb], ok[vb]);
            };
            if (ni == 1 || ni == 3) {
              int apex = ni == 1 ? inside[0] : outside[0];
              int ord[4], m = 0;
              ord[m++] = apex;
              for (int i = 0; i < 4; ++i)
                if (i != apex) ord[m++] = i;
              if (perm_parity(ord, 4)) std::swap(ord[2], ord[3]);
              if (ni == 3) std::swap(ord[2], ord[3]);  // normal towards the outside apex
              if (write && M.n < cap) {
                edge(M.n * 3 + 0, ord[0], ord[1]);
                edge(M.n * 3 + 1, ord[0], ord[2]);
                edge(M.n * 3 + 2, ord[0], ord[3]);
              }
              M.n++;
            } else {
              int ord[4] = {inside[0], inside[1], outside[0], outside[1]};
              if (perm_parity(ord, 4)) std::swap(ord[2], ord[3]);
              int i1 = ord[0], i2 = ord[1], o1 = ord[2], o2 = ord[3];
              if (write && M.n + 1 < cap) {
                edge(M.n * 3 + 0, i1, o1);
                edge(M.n * 3 + 1, i1, o2);
                edge(M.n * 3 + 2, i2, o2);
                edge(M.n * 3 + 3, i1, o1);
                edge(M.n * 3 + 4, i2, o2);
                edge(M.n * 3 + 5, i2, o1);
              }
              M.n += 2;
            }
          }
        }
  return M.n;
}

void unpack_H(const double Hm[6][6], double H21[21]) {
  int n = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) H21[n++] = Hm[i][j];
}

void pack_H(const double H21[21], double Hm[6][6]) {
  int n = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j) {
      Hm[i][j] = H21[n];
      Hm[j][i] = H21[n];
      n++;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// virtual depth (Sec. III-E, second option)
// ---------------------------------------------------------------------------
// Readings: ray samples at z_k = z_near + k v/2 (z along the optical axis),
// k = 0 .. floor(2 (d_max - z_near) / v), computed on micrometres; a sample
// counts when all 8 trilinear corners are observed; the virtual depth is the
// first crossing from V > 0 to V <= 0 between two consecutive counted samples,
// z* = z_{k-1} + (v/2) V_{k-1} / (V_{k-1} - V_k), rounded to the nearest raw
// unit (half up); zero pixels without a crossing get far_raw.
void virtual_depth(Volume& V, const orc_frame* f, const double T[16], uint16_t far_raw, int row0, int row1,
                   uint16_t* out) {
  const double delta = V.p.voxel_size * 0.5;
  const int64_t K = (2 * (V.dmax_um - llround(V.p.z_near * 1e6))) / V.v_um;
  for (int v = row0; v < row1; ++v)
    for (int u = 0; u < f->width; ++u) {
      const int idx = v * f->width + u;
      if (f->depth[idx] != 0) {
        out[idx] = f->depth[idx];
        continue;
      }
      uint16_t result = far_raw;
      bool prev_valid = false;
      double prev_V = 0.0, prev_z = 0.0;
      for (int64_t k = 0; k <= K; ++k) {
        const double z = V.p.z_near + (double)k * delta;
        double p[3];
        backproject_world(f, u, v, z, T, p);
        int64_t k0[3];
        double fr[3];
        Corners c;
        const bool valid = cell_of(V, p, k0, fr) && gather(V, k0, &c);
        const double Vk = valid ? trilinear(c.F, fr) : 0.0;
        if (prev_valid && valid && prev_V > 0.0 && Vk <= 0.0) {
          const double t = prev_V / (prev_V - Vk);
          const double zs = prev_z + delta * t;
          result = (uint16_t)std::floor(zs * V.p.depth_scale + 0.5);
          break;
        }
        prev_valid = valid;
        prev_V = Vk;
        prev_z = z;
      }
      out[idx] = result;
    }
}

extern "C" {

void* orc_create(const orc_params* p) {
  Volume* V = new Volume();
  V->p = *p;
  derive(*V);
  return V;
}

void orc_destroy(void* vol) { delete static_cast<Volume*>(vol); }

int64_t orc_num_blocks(void* vol) { return (int64_t) static_cast<Volume*>(vol)->blocks.size(); }

int orc_num_frames(void* vol) { return static_cast<Volume*>(vol)->frames; }

int64_t orc_integrate(void* vol, const orc_frame* f, const double T[16], const uint8_t* mask) {
  return integrate(*static_cast<Volume*>(vol), f, T, mask);
}

void orc_track(void* vol, const orc_frame* f, const double T_init[16], const uint8_t* mask, double T_out[16],
               orc_track_info* info) {
  track(*static_cast<Volume*>(vol), f, T_init, mask, T_out, info);
}

void orc_track_footprint(void* vol, const orc_frame* f, const double T_init[16], const uint8_t* mask,
                         double T_out[16], orc_track_info* info, int64_t* n_blocks_probed, int64_t* n_voxels_read) {
  Volume& V = *static_cast<Volume*>(vol);
  std::unordered_set<BlockKey, BlockKeyHash> probed;
  std::unordered_set<int64_t> read;
  V.probed = &probed;
  V.read = &read;
  track(V, f, T_init, mask, T_out, info);
  V.probed = nullptr;
  V.read = nullptr;
  *n_blocks_probed = (int64_t)probed.size();
  *n_voxels_read = (int64_t)read.size();
}

void orc_eval(void* vol, const orc_frame* f, const double T[16], int stride, const uint8_t* mask, double H[21],
              double g[6], double* E, int64_t* N) {
  double Hm[6][6];
  eval_normal_eq(*static_cast<Volume*>(vol), f, T, stride, mask, Hm, g, E, N);
  unpack_H(Hm, H);
}

int orc_lookup(void* vol, const double p[3], double* sdf, double gsdf[3], double* inten, double ginten[3],
               int* colour_ok) {
  bool c = false;
  bool ok = lookup(*static_cast<Volume*>(vol), p, sdf, gsdf, inten, ginten, &c);
  *colour_ok = c ? 1 : 0;
  return ok ? 1 : 0;
}

void orc_residual_seeds(void* vol, const orc_frame* f, const double T[16], double* r, uint8_t* seeds) {
  residual_seeds(*static_cast<Volume*>(vol), f, T, r, seeds);
}

void orc_erode3(const uint8_t* in, int H, int W, uint8_t* out) { erode3(in, H, W, out); }
void orc_dilate3(const uint8_t* in, int H, int W, uint8_t* out) { dilate3(in, H, W, out); }
void orc_floodfill(const uint8_t* MR, const uint16_t* depth, int H, int W, int64_t theta_ppm, uint8_t* MD) {
  floodfill(MR, depth, H, W, theta_ppm, MD);
}

void orc_compute_mask(void* vol, const orc_frame* f, const double T[16], uint8_t* mask) {
  compute_mask(*static_cast<Volume*>(vol), f, T, mask);
}

void orc_process_frame(void* vol, const orc_frame* f, const double T_init[16], double T_out[16],
                       uint8_t* mask_out, orc_track_info* info) {
  Volume& V = *static_cast<Volume*>(vol);
  const int HW = f->height * f->width;
  std::vector<uint8_t> mask(HW, 0);
  if (V.frames == 0) {
    integrate(V, f, T_init, nullptr);
    std::memcpy(T_out, T_init, 16 * sizeof(double));
    if (info) std::memset(info, 0, sizeof(*info));
  } else {
    double T1[16], T2[16];
    track(V, f, T_init, nullptr, T1, nullptr);
    compute_mask(V, f, T1, mask.data());
    track(V, f, T1, mask.data(), T2, info);
    integrate(V, f, T2, mask.data());
    std::memcpy(T_out, T2, sizeof(T2));
  }
  if (mask_out) std::memcpy(mask_out, mask.data(), HW);
  V.frames++;
}

void orc_virtual_depth(void* vol, const orc_frame* f, const double T[16], uint16_t far_raw, int row0, int row1,
                       uint16_t* out) {
  virtual_depth(*static_cast<Volume*>(vol), f, T, far_raw, row0, row1, out);
}

void orc_se3_exp(const double xi[6], double T[16]) { se3_exp(xi, T); }

int orc_lm_solve(const double H[21], const double g[6], double lambda, double delta[6]) {
  double Hm[6][6];
  pack_H(H, Hm);
  return lm_solve(Hm, g, lambda, delta) ? 1 : 0;
}

void orc_export(void* vol, int32_t* coords, double* F, uint8_t* W, uint8_t* rgb, uint8_t* wc) {
  Volume& V = *static_cast<Volume*>(vol);
  std::vector<BlockKey> keys;
  for (auto& kv : V.blocks) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end(), [](const BlockKey& a, const BlockKey& b) {
    if (a.z != b.z) return a.z < b.z;
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  for (size_t n = 0; n < keys.size(); ++n) {
    const Block& B = V.blocks[keys[n]];
    coords[n * 3 + 0] = (int32_t)keys[n].x;
    coords[n * 3 + 1] = (int32_t)keys[n].y;
    coords[n * 3 + 2] = (int32_t)keys[n].z;
    for (int i = 0; i < BV; ++i) {
      F[n * BV + i] = B.W[i] > 0 ? B.F[i] : 0.0;
      W[n * BV + i] = (uint8_t)std::min(B.W[i], 255);
      wc[n * BV + i] = (uint8_t)std::min(B.Wc[i], 255);
      for (int ch = 0; ch < 3; ++ch) rgb[(n * BV + i) * 3 + ch] = B.rgb[i * 3 + ch];
    }
  }
}

int orc_import(void* vol, int64_t n, const int32_t* coords, const double* F, const uint8_t* W, const uint8_t* rgb,
               const uint8_t* wc) {
  Volume& V = *static_cast<Volume*>(vol);
  for (int64_t b = 0; b < n; ++b) {
    Block& B = V.blocks[BlockKey{coords[b * 3 + 0], coords[b * 3 + 1], coords[b * 3 + 2]}];
    for (int i = 0; i < BV; ++i) {
      B.F[i] = F[b * BV + i];
      B.W[i] = W[b * BV + i];
      B.Wc[i] = wc[b * BV + i];
      for (int ch = 0; ch < 3; ++ch) B.rgb[i * 3 + ch] = rgb[(b * BV + i) * 3 + ch];
    }
  }
  return 0;
}

int64_t orc_extract_mesh(void* vol, double* verts, uint8_t* colors, int64_t cap_tris) {
  return extract_mesh(*static_cast<Volume*>(vol), verts, colors, cap_tris);
}

}  // extern "C"
