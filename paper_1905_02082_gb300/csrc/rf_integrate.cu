// Integration with free-space carving (ReFusion Sec. III-A, III-C last
// paragraph, III-D) on sm_103a.
//
// Definition (shared with the FP64 oracle): voxel k (world position v k) is
// updated by a frame at pose T when, with camera coordinates computed from
// the quantised pose,
//     z in (z_near, d_max],  u = floor(fx x / z + cx + 1/2) inside the image,
//     D(u) valid and not masked,  sdf = D(u) - z >= -tau;
// the update is F <- (W F + s) / (W + 1), W <- min(W + 1, w_max) with
// s = sdf inside the band |sdf| <= tau (colour averaged too) and s = tau in
// front of it (free space).  A block is allocated when at least one of its
// voxels is updated.  All decisions use exact integers: camera coordinates in
// ticks of 2^-10 um from R^T quantised to 2^30 and t to micrometres, pixel
// rounding verified with int64 products after a float guess.
//
// Kernels, in stream order:
//   k_frustum      16x16-tile maximum of valid unmasked depth        (tile/CTA),
//                  then in its last CTA: quantised pose, counters reset,
//                  block range of the truncated frustum
//   k_cull         conservative per-block frustum/depth test, warp-aggregated
//                  append to the candidate list                     (block/thread)
//   k_integrate    exact per-voxel predicate, lock-free hash insert of blocks
//                  with updates, read-modify-write of updated voxels (one warp
//                  per block, persistent grid, static round-robin)
#include <cmath>

#include "rf_volume.hpp"

namespace rf {
namespace {

// Largest frustum search region (blocks); beyond it the frame is rejected
// with RF_ERR_OUT_OF_RANGE (d_max / voxel_size far too large, or a
// non-finite pose).
constexpr long long kMaxSearchBlocks = 1ll << 28;

// Quantised pose (one entry per lane of warp 0: conversions run on the FP64
// pipe, so they are spread over lanes), the per-frame constants of the voxel
// loop and the reset of the per-frame counters.
__device__ __forceinline__ void integ_prep(const double* __restrict__ T, IntegState* st, const int* __restrict__ n_blocks,
                                           const DevParams& p, int max_um) {
  const int a = threadIdx.x;
  if (a < 9) {
    const int i = a / 3, j = a % 3;
    st->A[a] = llround(T[j * 4 + i] * 1073741824.0);  // world -> camera rotation R^T, 2^30 scale
    st->R[a] = (float)T[i * 4 + j];
  } else if (a < 12) {
    st->tq[a - 9] = llround(T[(a - 9) * 4 + 3] * 1e6);
    st->t[a - 9] = (float)T[(a - 9) * 4 + 3];
  } else if (a == 12) {
    st->max_um = max_um;
    st->n_cand = 0;
    st->work = 0;
    st->clipped = 0;
    st->new_blocks = 0;
    st->updated = 0ull;
    st->pool_before = *n_blocks;
  } else if (a < 16) {
    // one voxel step along world z, camera coordinate i = a - 13, in ticks
    const int i = a - 13;
    st->szf[i] = (float)((double)(llround(T[8 + i] * 1073741824.0) * p.v_um) * (1.0 / 1048576.0));
  }
}

// Block range of the truncated frustum z in (z_near, zfar], zfar =
// min(max valid depth + tau, d_max), over the pixel rectangle.  Float math on
// 8 lanes of one warp (one frustum corner each); the 2-voxel margin covers
// its rounding.  R, t: the pose as floats (already in st).
__device__ __forceinline__ void integ_aabb(const DevFrame& f, const DevParams& p, IntegState* st, int max_um,
                                           int lane) {
  if (max_um < 0) {
    if (lane == 0) {
      st->total = 0;
      st->zfar = 0.0f;
    }
    return;
  }
  const float zfar = fminf((float)max_um * 1e-6f + p.tau, (float)p.dmax_um * 1e-6f);
  bool finite = true;
  for (int i = 0; i < 9; ++i) finite &= isfinite(st->R[i]) != 0;
  for (int i = 0; i < 3; ++i) finite &= isfinite(st->t[i]) != 0;
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  if (lane < 8) {
    const float z = (lane & 4) ? zfar : p.z_near;
    const float u = (lane & 1) ? (float)f.W - 0.5f : -0.5f, v = (lane & 2) ? (float)f.H - 0.5f : -0.5f;
    const float x = (u - f.cx) * f.ifx * z, y = (v - f.cy) * f.ify * z;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float w = st->R[i * 3] * x + st->R[i * 3 + 1] * y + st->R[i * 3 + 2] * z + st->t[i];
      lo[i] = w;
      hi[i] = w;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lo[i] = fminf(lo[i], __shfl_xor_sync(0xffffffffu, lo[i], o));
      hi[i] = fmaxf(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
    }
  if (lane != 0) return;
  const float bs = 8.0f * p.voxel, margin = 2.0f * p.voxel;
  long long total = 1;
  bool clipped = !finite;
  for (int i = 0; i < 3 && !clipped; ++i) {
    const float f0 = fmaxf(fminf(floorf((lo[i] - margin) / bs), 1e9f), -1e9f);
    const float f1 = fmaxf(fminf(floorf((hi[i] + margin) / bs), 1e9f), -1e9f);
    if (!(f0 == f0) || !(f1 == f1)) {
      clipped = true;
      break;
    }
    long long b0 = (long long)f0, b1 = (long long)f1;
    if (b0 < -kMaxCoord) { b0 = -kMaxCoord; clipped = true; }
    if (b1 > kMaxCoord) { b1 = kMaxCoord; clipped = true; }
    if (b1 < b0) b1 = b0 - 1;
    st->bmin[i] = (int)b0;
    st->dims[i] = (int)(b1 - b0 + 1);
    total *= (b1 - b0 + 1);
  }
  if (!finite || total > kMaxSearchBlocks) total = 0;
  st->total = total > 0 ? total : 0;
  st->zfar = zfar;
  st->clipped = clipped ? 1 : 0;  // blocks beyond the key range cannot be stored (reported by k_cull)
}

// Frustum search, first kernel of an integration.  Per 16x16 tile: the
// largest valid unmasked depth, and the frame's depth with invalid and masked
// pixels zeroed (the per-voxel loop then tests one value per pixel).  The
// last CTA to finish (a ticket counter it resets) then takes the maximum over
// the tiles and writes the quantised pose, the per-frame constants, the reset
// counters and the block range of the truncated frustum.
__global__ void __launch_bounds__(256) k_frustum(DevFrame f, DevParams p, const uint8_t* __restrict__ mask,
                                                 int* __restrict__ tilemax, IntegState* st, int tiles_x, int ntiles,
                                                 uint16_t* __restrict__ dm, const double* __restrict__ T,
                                                 const int* __restrict__ n_blocks) {
  if (gated_off(f.gate, kModeFirst)) return;
  const int tile = blockIdx.x;
  const int u = (tile % tiles_x) * kTile + (threadIdx.x % kTile);
  const int v = (tile / tiles_x) * kTile + (threadIdx.x / kTile);
  int d = -1;
  if (u < f.W && v < f.H) {
    const int idx = v * f.W + u;
    const unsigned raw = f.depth[idx];
    const bool use = pixel_valid(p, raw) && !(mask && mask[idx]);
    if (use) d = (int)(raw * p.du_um);
    dm[idx] = use ? (uint16_t)raw : (uint16_t)0;
  }
  d = __reduce_max_sync(0xffffffffu, d);
  __shared__ int s[8];
  __shared__ int s_last;
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = s[0];
    for (int w = 1; w < 8; ++w) m = max(m, s[w]);
    tilemax[tile] = m;
    __threadfence();  // the tile maximum before the ticket
    s_last = atomicAdd(&st->ticket, 1u) == (unsigned)ntiles - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int m = -1;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) m = max(m, __ldcg(tilemax + t));
  m = __reduce_max_sync(0xffffffffu, m);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  int max_um = s[0];
  for (int w = 1; w < 8; ++w) max_um = max(max_um, s[w]);
  if (threadIdx.x < 32) integ_prep(T, st, n_blocks, p, max_um);
  if (threadIdx.x == 0) st->ticket = 0u;
  __syncthreads();  // R and t in st are visible to the whole CTA
  if (threadIdx.x >= 32 && threadIdx.x < 64) integ_aabb(f, p, st, max_um, threadIdx.x - 32);
}

// Conservative test: may keep blocks without updated voxels, never drops one.
__device__ bool cull_keep(int bx, int by, int bz, const DevFrame& f, const DevParams& p, const IntegState& st,
                          const int* __restrict__ tilemax, int tiles_x, int tiles_y, int max_um) {
  float zmin = 3.0e38f, zmax = -3.0e38f;
  float pcx[8], pcy[8], pcz[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float wx = (float)(bx * 8 + ((c & 1) ? 7 : 0)) * p.voxel - st.t[0];
    const float wy = (float)(by * 8 + ((c & 2) ? 7 : 0)) * p.voxel - st.t[1];
    const float wz = (float)(bz * 8 + ((c & 4) ? 7 : 0)) * p.voxel - st.t[2];
    // camera = R^T (w - t); R row-major camera->world
    pcx[c] = st.R[0] * wx + st.R[3] * wy + st.R[6] * wz;
    pcy[c] = st.R[1] * wx + st.R[4] * wy + st.R[7] * wz;
    pcz[c] = st.R[2] * wx + st.R[5] * wy + st.R[8] * wz;
    zmin = fminf(zmin, pcz[c]);
    zmax = fmaxf(zmax, pcz[c]);
  }
  const float eps = 1e-3f + 1e-5f * fabsf(zmax);
  if (zmax <= p.z_near - eps) return false;
  if (zmin > st.zfar + eps) return false;
  if (!(zmin > 0.5f * p.z_near)) return true;  // straddles the near plane: keep
  float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float iz = 1.0f / pcz[c];
    const float u = f.fx * pcx[c] * iz + f.cx, v = f.fy * pcy[c] * iz + f.cy;
    umin = fminf(umin, u);
    umax = fmaxf(umax, u);
    vmin = fminf(vmin, v);
    vmax = fmaxf(vmax, v);
  }
  // pixel range of the voxels (nearest-pixel rounding, one pixel of margin)
  const float lu = floorf(umin + 0.5f) - 1.0f, hu = floorf(umax + 0.5f) + 1.0f;
  const float lv = floorf(vmin + 0.5f) - 1.0f, hv = floorf(vmax + 0.5f) + 1.0f;
  if (hu < 0.0f || hv < 0.0f || lu > (float)(f.W - 1) || lv > (float)(f.H - 1)) return false;
  const int u0 = max(0, (int)lu), u1 = min(f.W - 1, (int)fminf(hu, 1.0e9f));
  const int v0 = max(0, (int)lv), v1 = min(f.H - 1, (int)fminf(hv, 1.0e9f));
  const int tx0 = u0 / kTile, tx1 = u1 / kTile, ty0 = v0 / kTile, ty1 = v1 / kTile;
  int m = -1;
  if ((tx1 - tx0 + 1) * (ty1 - ty0 + 1) <= 64) {
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) m = max(m, __ldg(tilemax + ty * tiles_x + tx));
  } else {
    m = max_um;
  }
  if (m < 0) return false;
  return (float)m * 1e-6f + p.tau + eps >= zmin;
}

__global__ void __launch_bounds__(256) k_cull(DevFrame f, DevParams p, IntegState* st, const int* __restrict__ tilemax,
                                              int tiles_x, int tiles_y, int4* __restrict__ cand, long long max_cand,
                                              unsigned* status) {
  if (gated_off(f.gate, kModeFirst)) return;
  __shared__ IntegState s;
  if (threadIdx.x == 0) s = *st;
  __syncthreads();
  const int max_um = s.max_um;
  if (s.clipped && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OUT_OF_RANGE);
  const long long total = s.total;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long idx = base + threadIdx.x;
    bool keep = false;
    int bx = 0, by = 0, bz = 0;
    if (idx < total) {
      const long long dx = s.dims[0], dy = s.dims[1];
      bx = s.bmin[0] + (int)(idx % dx);
      by = s.bmin[1] + (int)((idx / dx) % dy);
      bz = s.bmin[2] + (int)(idx / (dx * dy));
      keep = cull_keep(bx, by, bz, f, p, s, tilemax, tiles_x, tiles_y, max_um);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    if (ballot) {
      int off = 0;
      const int leader = __ffs(ballot) - 1;
      if (lane == leader) off = atomicAdd(&st->n_cand, __popc(ballot));
      off = __shfl_sync(0xffffffffu, off, leader);
      if (keep) {
        const long long slot = off + __popc(ballot & ((1u << lane) - 1u));
        if (slot < max_cand) cand[slot] = make_int4(bx, by, bz, 0);
        else atomicOr(status, ST_CAPACITY);
      }
    }
  }
}

constexpr int kIntegThreads = 128;  // 4 warps; one warp integrates one block at a time
constexpr int kIntegWarps = kIntegThreads / 32;
constexpr float kTickMetres = 9.765625e-10f;  // 2^-10 um

// Colour running average of one band voxel (Sec. III-A, reading: RGB8 kept
// rounded half up, own weight Wc): (Wc C + c) / (Wc + 1) per channel as an
// exact integer quotient from a float reciprocal, corrected one step either way.
__device__ __forceinline__ unsigned colour_update(unsigned word, const uint8_t* c, int w_max) {
  const unsigned wc = word >> 24;
  const unsigned den = 2 * (wc + 1);
  const float rden = __frcp_rn((float)den);
  unsigned out = 0;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const unsigned num = 2 * (wc * ((word >> (8 * ch)) & 255u) + __ldg(c + ch)) + wc + 1;
    unsigned q = (unsigned)((float)num * rden);
    if (q * den > num) q -= 1;
    else if ((q + 1) * den <= num) q += 1;
    out |= q << (8 * ch);
  }
  return out | (min(wc + 1, (unsigned)w_max) << 24);
}

// Float of an int64 count of 2^-20 ticks, in ticks, without the FP64 pipe:
// the two 32-bit halves are converted separately (error below 2^-12 ticks plus
// one float rounding).
__device__ __forceinline__ float ticks_f(long long s) {
  const float hi = (float)(int)(s >> 32), lo = (float)(unsigned)(s & 0xffffffffll);
  return fmaf(hi, 4096.0f, lo * 9.5367431640625e-07f);  // hi 2^32 / 2^20, lo / 2^20
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Floor of a pixel estimate and whether it lies within `amb` of a rounding
// boundary (the exact integer path then decides).  Adding 1.5 * 2^23 rounds a
// float below 2^22 in magnitude to an integer in the low mantissa bits, so
// floor(e) = round(e - 1/2) costs a few FP32 adds and no conversion.
__device__ __forceinline__ int pixel_floor(float est, float amb, bool& ambiguous) {
  const float e = fminf(fmaxf(est, -4194304.0f), 4194304.0f);
  const float t = (e - 0.5f) + 12582912.0f;
  const float fr = e - (t - 12582912.0f);
  ambiguous = fabsf(fr - 0.5f) > 0.5f - amb;
  return __float_as_int(t) - 0x4B400000;
}

// Everything the voxel loop of one frame needs (shared memory, per CTA).
struct IntegShared {
  long long A[9], tq[3];
  float szf[3];
  float zlo_f, zhi_f;  // z_near and d_max in ticks (float)
  float tau_t, du_f;   // tau and one raw depth unit in ticks (float)
  float rcpw[256];     // 1 / (W + 1), W = 0..255 (running-average divisor)
};

// Per-lane constants: lane l owns voxels (x, y, z) = (l & 7, (l >> 3) + 4 h, z),
// h = 0, 1, z = 0..7, i.e. block indices l + 32 h + 64 z.  Their offsets from
// the block origin in camera coordinates, as float estimates (ticks).
struct LaneConsts {
  float lf[3][2];
};

__device__ __forceinline__ void lane_consts(const IntegShared& sh, long long v_um, int lane, LaneConsts& c) {
  const long long x = (long long)(lane & 7) * v_um;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const long long y = (long long)((lane >> 3) + 4 * h) * v_um;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const long long L = sh.A[i * 3] * x + sh.A[i * 3 + 1] * y;
      c.lf[i][h] = ticks_f(L);
    }
  }
}

// Per-block state: origin voxel (0, 0, 0) of block b in camera coordinates.
struct BlockState {
  long long* S;    // exact sums, 2^-20 ticks (the warp's shared memory)
  long long Qb;    // floor(S_z / 2^20): camera z of the origin in ticks
  float base[3][2];  // float estimates of the lane's two voxel columns at z = 0
};

// lc: this thread's LaneConsts (shared memory); S: the warp's 3 shared words.
__device__ __forceinline__ void block_state(const IntegShared& sh, const DevParams& p, const LaneConsts& lc, int4 b,
                                            long long* S, int lane, BlockState& bs) {
  const long long d0 = (long long)b.x * 8 * p.v_um - sh.tq[0], d1 = (long long)b.y * 8 * p.v_um - sh.tq[1],
                  d2 = (long long)b.z * 8 * p.v_um - sh.tq[2];
  long long s2 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long si = sh.A[i * 3] * d0 + sh.A[i * 3 + 1] * d1 + sh.A[i * 3 + 2] * d2;
    if (lane == i) S[i] = si;
    if (i == 2) s2 = si;
    const float bf = ticks_f(si);
    bs.base[i][0] = bf + lc.lf[i][0];
    bs.base[i][1] = bf + lc.lf[i][1];
  }
  bs.S = S;
  bs.Qb = s2 >> 20;
  __syncwarp();
}

// Update value of a voxel given its pixel's masked raw depth and its camera
// z (Qb + dz): false when not updated (invalid or masked pixel, or occluded:
// sdf < -tau).  sdf = D - z exactly in ticks; |sdf| <= tau: the band (tau
// below 2 m keeps the band's sdf within 32 bits).
__device__ __forceinline__ bool sdf_value(unsigned raw, long long Qb, int dz, const DevParams& p, float& x,
                                          bool& band) {
  const long long sdf = (long long)raw * p.du_tick - Qb - dz;
  band = sdf <= p.tau_tick;
  x = band ? (float)(int)sdf * kTickMetres : p.tau;
  return raw != 0u && sdf >= -p.tau_tick;
}

// Fast decision of one voxel, in FP32 with error bounds and no branches: -1
// when not updated, else the pixel index (bit 31 set inside the band) and x
// the update value.  (bx, by, bz): float camera coordinates (ticks) of the
// voxel's column at block z = 0; zr: its z as a float.  The camera z estimate
// is within ez = 1e-6 z + 64 ticks of the exact one (it carries a few float
// roundings of at most 2^-24 relative each, and the exact value is floored to
// whole ticks), and the sdf estimate within 2 ez.  amb: a decision lies within
// those bounds (the z range, the sdf thresholds +-tau) or the pixel estimate
// lies too close to a rounding boundary; the voxel is then left to the exact
// path (reported here as not updated).  Non-candidate voxels read pixel 0
// (always in bounds) instead of branching around the load.
__device__ __forceinline__ int decide_fast(const IntegShared& sh, const DevFrame& f, const DevParams& p, float bx,
                                           float by, float bz, float zr, float fxg, float fyg, float cxg,
                                           float cyg, const uint16_t* __restrict__ dm, float& x, bool& amb) {
  const float zf = fmaf(zr, sh.szf[2], bz);
  const float xf = fmaf(zr, sh.szf[0], bx);
  const float yf = fmaf(zr, sh.szf[1], by);
  const float ez = fmaf(1e-6f, fabsf(zf), 64.0f);
  const bool zin = zf > sh.zlo_f && zf <= sh.zhi_f;
  const bool zamb = fabsf(zf - sh.zlo_f) <= ez || fabsf(zf - sh.zhi_f) <= ez;
  const float iz = rcp_approx(zf);
  bool au, av;
  const int u = pixel_floor(fmaf(fxg * xf, iz, cxg), f.amb_u, au);
  const int v = pixel_floor(fmaf(fyg * yf, iz, cyg), f.amb_v, av);
  const bool cand = zin && !(au || av) && (unsigned)u < (unsigned)f.W && (unsigned)v < (unsigned)f.H;
  const int pix = cand ? v * f.W + u : 0;
  const unsigned raw = __ldg(dm + pix);
  const float sdf = fmaf(__uint_as_float(0x4B000000u | raw) - 8388608.0f, sh.du_f, -zf);  // exact float of raw
  const bool live = cand && raw != 0u;
  amb = zamb || (zin && (au || av)) || (live && fabsf(fabsf(sdf) - sh.tau_t) <= 2.0f * ez);
  const bool band = sdf <= sh.tau_t;
  x = band ? sdf * kTickMetres : p.tau;
  return (live && sdf >= -sh.tau_t && !amb) ? (band ? (pix | (int)0x80000000) : pix) : -1;
}

// floor(num / den) for den > 0 when it lies in [0, n), else -1.  `guess` is
// a float estimate of num / den (within one unit when the result is in
// range); it is corrected and verified with exact int64 products.
__device__ __forceinline__ int pixel_of(float guess, long long num, long long den, int n) {
  const float g = fminf(fmaxf(floorf(guess), -2.0f), (float)n + 1.0f);
  long long u = (long long)(int)g;
  if (u * den > num) u -= 1;
  else if ((u + 1) * den <= num) u += 1;
  if (u * den > num || (u + 1) * den <= num) return -1;
  return (u >= 0 && u < n) ? (int)u : -1;
}

// Exact decision of voxel (x, y, z) of the block: camera coordinates
// C = floor(S / 2^20) from int64 sums, pixel u = floor((fxq Cx + cxq Cz) /
// (256 Cz)) verified with int64 products.  Same return convention as
// decide_fast.  Taken for the few voxels whose estimate is ambiguous.
__device__ int decide_exact(const IntegShared& sh, const BlockState& bs, const DevFrame& f, const DevParams& p,
                            float fxg, float fyg, float cxg, float cyg, const uint16_t* __restrict__ dm, int vx,
                            int vy, int vz, float& x) {
  long long C[3];
  float cf[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long s = bs.S[i] + sh.A[i * 3] * (vx * p.v_um) + sh.A[i * 3 + 1] * (vy * p.v_um) +
                        sh.A[i * 3 + 2] * (vz * p.v_um);
    C[i] = s >> 20;
    cf[i] = ticks_f(s);
  }
  if (C[2] <= p.znear_tick || C[2] > p.dmax_tick) return -1;
  const long long den = C[2] << 8;
  const float iz = __frcp_rn(cf[2]);
  const int u = pixel_of(fxg * cf[0] * iz + cxg, f.fxq * C[0] + f.cxq * C[2], den, f.W);
  if (u < 0) return -1;
  const int v = pixel_of(fyg * cf[1] * iz + cyg, f.fyq * C[1] + f.cyq * C[2], den, f.H);
  if (v < 0) return -1;
  const int pix = v * f.W + u;
  bool band;
  if (!sdf_value(__ldg(dm + pix), bs.Qb, (int)(C[2] - bs.Qb), p, x, band)) return -1;
  return band ? (pix | (int)0x80000000) : pix;
}

// Lookup-or-insert of a block; only called for blocks no other CTA of the
// launch handles, so racing inserts only ever involve different keys.
__device__ int hash_insert(const DevVol& v, int bx, int by, int bz, bool* is_new) {
  *is_new = false;
  if (!coord_ok(bx, by, bz)) {
    atomicOr(v.status, ST_OUT_OF_RANGE);
    return -1;
  }
  const unsigned long long key = pack_key(bx, by, bz);
  const unsigned long long b = bucket_of(key, v.bucket_mask);
  int pool = -1;
  for (int pr = 0; pr < kMaxProbe; ++pr) {
    unsigned long long* bp = v.hash + ((b + pr) & v.bucket_mask) * kSlots;
    for (int s = 0; s < kSlots; ++s) {
      unsigned long long e = *(volatile unsigned long long*)(bp + s);
      if (e == kEmpty) {
        if (pool < 0) {
          pool = atomicAdd(v.n_blocks, 1);
          if (pool >= v.max_blocks) {
            atomicOr(v.status, ST_POOL_FULL);
            return -1;
          }
        }
        const unsigned long long ent = (key << 22) | (unsigned long long)pool;
        e = atomicCAS(bp + s, kEmpty, ent);
        if (e == kEmpty) {
          v.coords[pool] = make_int4(bx, by, bz, 1);
          *is_new = true;
          return pool;
        }
      }
      if ((e >> 22) == key) return (int)(e & 0x3FFFFF);
    }
  }
  atomicOr(v.status, ST_HASH_FULL);
  return -1;
}

// Running-average update of one voxel (Sec. III-A; free space, Sec. III-D:
// value tau).  FP32 storage: the uint2 word {F, RGB | Wc << 24} and the
// weight byte.  dec: decide_* result (>= 0: updated).
__device__ __forceinline__ void update_fp32(uint2& w, unsigned& W, int dec, float x, const IntegShared& sh,
                                            const uint8_t* __restrict__ rgb, int w_max) {
  const float F = __uint_as_float(w.x);
  const float Wf = __uint_as_float(0x4B000000u | W) - 8388608.0f;  // exact float of W <= 255
  const float Fn = W == 0u ? x : fmaf(Wf, F, x) * sh.rcpw[W];
  w.x = __float_as_uint(Fn);
  if (dec < 0) w.y = colour_update(w.y, rgb + 3 * (size_t)(dec & 0x7fffffff), w_max);  // band
  W = min(W + 1u, (unsigned)w_max);
}

// FP16 storage: tracking word {F16(F / tau) | I8 << 16 | W << 24} always,
// colour word {RGB | Wc << 24} inside the band (I8 derived from the colour).
__device__ __forceinline__ void update_fp16(unsigned& t, unsigned& col, bool& col_written, int dec, float x,
                                            const IntegShared& sh, const uint8_t* __restrict__ rgb,
                                            const DevParams& p) {
  const unsigned W = t >> 24;
  const float F = __half2float(__ushort_as_half((unsigned short)(t & 0xFFFFu))) * p.tau;
  const float Wf = __uint_as_float(0x4B000000u | W) - 8388608.0f;
  const float Fn = W == 0u ? x : fmaf(Wf, F, x) * sh.rcpw[W];
  const unsigned h = (unsigned)__half_as_ushort(__float2half_rn(Fn * p.inv_tau));
  unsigned i8 = (t >> 16) & 255u;
  if (dec < 0) {  // band: colour, and the intensity derived from it
    col = colour_update(col, rgb + 3 * (size_t)(dec & 0x7fffffff), p.w_max);
    col_written = true;
    i8 = rgb_i8(col);
  }
  t = h | (i8 << 16) | (min(W + 1u, (unsigned)p.w_max) << 24);
}

// Read-modify-write of voxel (lane, h, z0 + k) for k = 0..3 of block `pool`
// after their decisions `dec` (-1: not updated); a fresh block gets every
// voxel written (empty unless updated).  `o`: lane + 32 h + 64 z0.
template <int ST>
__device__ __forceinline__ void rmw4(const DevVol& v, const DevFrame& f, const DevParams& p, const IntegShared& sh,
                                     int pool, bool fresh, int o, const int dec[4], const float xv[4]) {
  if constexpr (ST == RF_STORAGE_FP32) {
    uint2* vb = v.vox + (size_t)pool * kBV + o;
    uint8_t* wb = v.W + (size_t)pool * kBV + o;
    uint2 w[4];
    unsigned W[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ld = dec[k] != -1 && !fresh;
      w[k] = ld ? vb[64 * k] : make_uint2(0x7fc00000u, 0u);
      W[k] = ld ? (unsigned)wb[64 * k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (dec[k] != -1) update_fp32(w[k], W[k], dec[k], xv[k], sh, f.rgb, p.w_max);
      if (dec[k] != -1 || fresh) {
        vb[64 * k] = w[k];
        wb[64 * k] = (uint8_t)W[k];
      }
    }
  } else {
    unsigned* tb = trk_words_rw(v, pool) + o;
    unsigned* cb = tb + kBV;
    unsigned t[4], col[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ld = dec[k] != -1 && !fresh;
      t[k] = ld ? tb[64 * k] : kTrkEmpty;
      col[k] = (ld && dec[k] < -2) ? cb[64 * k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool cw = fresh;
      if (dec[k] != -1) update_fp16(t[k], col[k], cw, dec[k], xv[k], sh, f.rgb, p);
      if (dec[k] != -1 || fresh) tb[64 * k] = t[k];
      if (cw) cb[64 * k] = col[k];
    }
  }
}

// One candidate block b, integrated by one warp (see k_integrate).
template <int ST>
__device__ __forceinline__ void integrate_block(const DevVol& v, const DevFrame& f, const DevParams& p,
                                                const uint16_t* __restrict__ dm, const IntegShared& sh,
                                                const LaneConsts& lc, const int4 b, int lane, unsigned short* aq,
                                                long long* S, unsigned& my_updated, unsigned& my_new) {
  const unsigned long long key = pack_key(b.x, b.y, b.z);
  const bool in_range = coord_ok(b.x, b.y, b.z);
  const unsigned long long bucket = bucket_of(key, v.bucket_mask);
  unsigned long long e = kEmpty;
  if (lane < kSlots && in_range) e = __ldcg(v.hash + bucket * kSlots + lane);  // first bucket
  const float fxg = (float)f.fxq * (1.0f / 256.0f), fyg = (float)f.fyq * (1.0f / 256.0f);
  const float cxg = (float)f.cxq * (1.0f / 256.0f), cyg = (float)f.cyq * (1.0f / 256.0f);
  BlockState bs;
  block_state(sh, p, lc, b, S, lane, bs);
  const unsigned found = __ballot_sync(0xffffffffu, lane < kSlots && e != kEmpty && (e >> 22) == key);
  int pool = -1;
  bool fresh = false;
  if (found) {
    pool = (int)(__shfl_sync(0xffffffffu, e, __ffs(found) - 1) & 0x3FFFFFull);
  } else {
    // not in its first bucket: allocate only if some voxel is updated
    bool any = false;
#pragma unroll 1
    for (int j = 0; j < 16; ++j) {
      const int h = j & 1, z = j >> 1;
      float x;
      bool amb;
      int dec = decide_fast(sh, f, p, h ? bs.base[0][1] : bs.base[0][0], h ? bs.base[1][1] : bs.base[1][0],
                            h ? bs.base[2][1] : bs.base[2][0], (float)z, fxg, fyg, cxg, cyg, dm, x, amb);
      if (amb) dec = decide_exact(sh, bs, f, p, fxg, fyg, cxg, cyg, dm, lane & 7, (lane >> 3) + 4 * h, z, x);
      any |= dec != -1;
    }
    if (!__any_sync(0xffffffffu, any)) return;
    int pl = -1, nw = 0;
    if (lane == 0) {
      bool is_new;
      pl = hash_insert(v, b.x, b.y, b.z, &is_new);
      nw = is_new;
    }
    pool = __shfl_sync(0xffffffffu, pl, 0);
    fresh = __shfl_sync(0xffffffffu, nw, 0) != 0;
    if (pool < 0) return;
  }
  my_new += (lane == 0 && fresh) ? 1u : 0u;
  // main pass: 16 voxels per lane, four at a time (decisions, loads, stores)
  unsigned ambmask = 0u;  // bit 8 h + z
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    const int h = g & 1, z0 = (g >> 1) * 4;
    const float bx = h ? bs.base[0][1] : bs.base[0][0], by = h ? bs.base[1][1] : bs.base[1][0];
    const float bz = h ? bs.base[2][1] : bs.base[2][0];
    const float z0f = (g >> 1) ? 4.0f : 0.0f;
    int dec[4];
    float xv[4];
    unsigned am = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bool a;
      dec[k] = decide_fast(sh, f, p, bx, by, bz, z0f + (float)k, fxg, fyg, cxg, cyg, dm, xv[k], a);
      am |= a ? (1u << k) : 0u;
      my_updated += dec[k] != -1 ? 1u : 0u;
    }
    ambmask |= am << (8 * h + z0);
    rmw4<ST>(v, f, p, sh, pool, fresh, lane + 32 * h + 64 * z0, dec, xv);
  }
  // ambiguous voxels: queued across the warp, then one exact decision each
  const int cnt = __popc(ambmask);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  int pos = incl - cnt;
  for (unsigned m = ambmask; m; m &= m - 1u) {
    const int bit = __ffs(m) - 1;
    aq[pos++] = (unsigned short)(lane + 32 * (bit >> 3) + 64 * (bit & 7));
  }
  __syncwarp();  // the queue and the main pass's stores (fresh blocks: every voxel) are visible to the warp
  for (int q = lane; q < total; q += 32) {
    const int j = aq[q];
    const int vx = j & 7, vy = (j >> 3) & 7, vz = j >> 6;
    float x;
    const int dec = decide_exact(sh, bs, f, p, fxg, fyg, cxg, cyg, dm, vx, vy, vz, x);
    if (dec == -1) continue;
    my_updated += 1u;
    if constexpr (ST == RF_STORAGE_FP32) {
      uint2* wp = v.vox + (size_t)pool * kBV + j;
      uint8_t* Wp = v.W + (size_t)pool * kBV + j;
      uint2 w = *wp;
      unsigned W = *Wp;
      update_fp32(w, W, dec, x, sh, f.rgb, p.w_max);
      *wp = w;
      *Wp = (uint8_t)W;
    } else {
      unsigned* tp = trk_words_rw(v, pool) + j;
      unsigned t = *tp;
      unsigned col = dec < 0 ? tp[kBV] : 0u;
      bool cw = false;
      update_fp16(t, col, cw, dec, x, sh, f.rgb, p);
      *tp = t;
      if (cw) tp[kBV] = col;
    }
  }
  __syncwarp();  // the queue is reused by the warp's next block
}

// Counts of one warp for one stream's integration statistics.
__device__ __forceinline__ void integ_flush(IntegState* st, unsigned updated, unsigned fresh, int lane) {
  updated = __reduce_add_sync(0xffffffffu, updated);
  fresh = __reduce_add_sync(0xffffffffu, fresh);
  if (lane == 0 && updated) atomicAdd(&st->updated, (unsigned long long)updated);
  if (lane == 0 && fresh) atomicAdd(&st->new_blocks, (int)fresh);
}

// Per-voxel update: one warp per candidate block (static round-robin over all
// warps, no CTA barriers inside the loop).  Per block: the origin's exact
// camera coordinates (int64) and their float estimates; per voxel only FP32
// work without branches: the camera coordinates, the pixel, one load of the
// masked depth and the sdf, each decision taken in FP32 when it lies outside
// the estimate's error bound; then the read-modify-write of the updated
// voxels, four at a time.  The ~2 % of voxels with a decision inside an error
// bound (almost all: a pixel estimate near a rounding boundary) are queued and
// decided by the exact int64 path after the main pass.
template <int ST>
__global__ void __launch_bounds__(kIntegThreads, 8) k_integrate(DevVol v, DevFrame f, DevParams p,
                                                             const uint16_t* __restrict__ dm, IntegState* st,
                                                             const int4* __restrict__ cand, long long max_cand) {
  __shared__ IntegShared sh;
  __shared__ unsigned short s_aq[kIntegWarps][kBV];  // voxels queued for the exact path
  __shared__ LaneConsts s_lc[kIntegThreads];
  __shared__ long long s_S[kIntegWarps][4];
  if (gated_off(f.gate, kModeFirst)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < 9) sh.A[threadIdx.x] = st->A[threadIdx.x];
  if (threadIdx.x < 3) {
    sh.tq[threadIdx.x] = st->tq[threadIdx.x];
    sh.szf[threadIdx.x] = st->szf[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    sh.zlo_f = (float)p.znear_tick;
    sh.zhi_f = (float)p.dmax_tick;
    sh.tau_t = (float)p.tau_tick;
    sh.du_f = (float)p.du_tick;
  }
  for (int w = threadIdx.x; w < 256; w += kIntegThreads) sh.rcpw[w] = 1.0f / (float)(w + 1);
  __syncthreads();
  const long long n_cand = min((long long)*(volatile int*)&st->n_cand, max_cand);
  lane_consts(sh, p.v_um, lane, s_lc[threadIdx.x]);
  const long long warp0 = ((long long)blockIdx.x * kIntegThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kIntegThreads) >> 5;
  unsigned my_updated = 0, my_new = 0;
  for (long long ci = warp0; ci < n_cand; ci += nwarps)
    integrate_block<ST>(v, f, p, dm, sh, s_lc[threadIdx.x], cand[ci], lane, s_aq[wid], s_S[wid], my_updated,
                        my_new);
  integ_flush(st, my_updated, my_new, lane);
}

// Neighbour tables of the blocks allocated since `lo`: each new block gets
// the pools of its 7 positive neighbours, and each existing negative
// neighbour gets the new block in the matching slot.  Runs after the
// integration (the hash is complete and read-only here).  One thread per
// table entry (15 per new block: its own slot 0, 7 forward lookups, 7
// reverse ones), so the hash probes of a block run side by side.  Two new
// neighbours write each other's entries from both sides with the same value.
constexpr int kFixupWork = 15;

__device__ __forceinline__ void fixup_entry(const DevVol& v, int b, int k) {
  const int4 c = v.coords[b];
  if (c.w == 0) return;
  int* flat = reinterpret_cast<int*>(v.nbr);
  if (k == 0) {
    flat[8 * (size_t)b] = b;
  } else if (k < 8) {
    flat[8 * (size_t)b + k] = hash_find(v, c.x + (k & 1), c.y + ((k >> 1) & 1), c.z + ((k >> 2) & 1));
  } else {
    const int o = k - 7;
    const int n = hash_find(v, c.x - (o & 1), c.y - ((o >> 1) & 1), c.z - ((o >> 2) & 1));
    if (n >= 0) flat[8 * (size_t)n + o] = b;
  }
}

__global__ void __launch_bounds__(256) k_nbr_fixup(DevVol v, const int* __restrict__ lo_ptr, int lo_value,
                                                   const int* gate) {
  if (gated_off(gate, kModeFirst)) return;
  const int lo = lo_ptr ? *lo_ptr : lo_value;
  const int hi = min(*(volatile int*)v.n_blocks, v.max_blocks);
  const long long n = (long long)max(hi - lo, 0) * kFixupWork;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    fixup_entry(v, lo + (int)(i / kFixupWork), (int)(i % kFixupWork));
}

}  // namespace

rf_status launch_nbr_fixup(rf_volume* vol, const int* lo_ptr, int lo, cudaStream_t st, const int* gate) {
  k_nbr_fixup<<<vol->sm_count * vol->launch.fixup_ctas_per_sm, 256, 0, st>>>(vol->dv, lo_ptr, lo, gate);
  return check_cuda(vol, cudaGetLastError(), "neighbour table launch");
}

// The frustum search of an integration: prep, tile maxima, AABB, cull.
static rf_status launch_frustum(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st) {
  const int tiles_x = (f.W + kTile - 1) / kTile, tiles_y = (f.H + kTile - 1) / kTile;
  k_frustum<<<tiles_x * tiles_y, 256, 0, st>>>(f, vol->dp, mask, vol->d_tilemax, vol->d_integ, tiles_x,
                                               tiles_x * tiles_y, vol->d_dmask, T, vol->d_nblocks);
  k_cull<<<vol->sm_count * vol->launch.cull_ctas_per_sm, 256, 0, st>>>(f, vol->dp, vol->d_integ, vol->d_tilemax, tiles_x, tiles_y, vol->d_cand,
                                            vol->p.max_candidates, vol->d_status);
  return check_cuda(vol, cudaGetLastError(), "frustum launch");
}

rf_status launch_integrate(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st) {
  rf_status s = launch_frustum(vol, f, T, mask, st);
  if (s != RF_OK) return s;
  prof_record(vol, EV_KERNEL0, st);
  if (vol->p.storage == RF_STORAGE_FP16)
    k_integrate<RF_STORAGE_FP16><<<vol->sm_count * vol->launch.integrate_ctas_per_sm, kIntegThreads, 0, st>>>(vol->dv, f, vol->dp, vol->d_dmask, vol->d_integ,
                                                                             vol->d_cand, vol->p.max_candidates);
  else
    k_integrate<RF_STORAGE_FP32><<<vol->sm_count * vol->launch.integrate_ctas_per_sm, kIntegThreads, 0, st>>>(vol->dv, f, vol->dp, vol->d_dmask, vol->d_integ,
                                                                             vol->d_cand, vol->p.max_candidates);
  prof_record(vol, EV_KERNEL1, st);
  s = check_cuda(vol, cudaGetLastError(), "integrate launch");
  if (s != RF_OK) return s;
  return launch_nbr_fixup(vol, &vol->d_integ->pool_before, 0, st, f.gate);
}

}  // namespace rf
