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
//   k_integ_prep   quantise the pose, reset counters                 (1 thread)
//   k_tilemax      16x16-tile maximum of valid unmasked depth        (tile/CTA)
//   k_integ_aabb   block range of the truncated frustum              (1 thread)
//   k_cull         conservative per-block frustum/depth test, warp-aggregated
//                  append to the candidate list                     (block/thread)
//   k_integrate    exact per-voxel predicate, lock-free hash insert of blocks
//                  with updates, read-modify-write of updated voxels (one warp
//                  per block, persistent grid, static round-robin)
#include <cmath>

#include "rf_volume.hpp"

namespace rf {
namespace {

// Quantised pose (one entry per lane: conversions run on the FP64 pipe, so
// they are spread over lanes) and reset of the per-frame counters.
__global__ void k_integ_prep(const double* __restrict__ T, IntegState* st, const int* __restrict__ n_blocks,
                             const int* gate) {
  if (gated_off(gate, kModeFirst)) return;
  const int a = threadIdx.x;
  if (a < 9) {
    const int i = a / 3, j = a % 3;
    st->A[a] = llround(T[j * 4 + i] * 1073741824.0);  // world -> camera rotation R^T, 2^30 scale
    st->R[a] = (float)T[i * 4 + j];
  } else if (a < 12) {
    st->tq[a - 9] = llround(T[(a - 9) * 4 + 3] * 1e6);
    st->t[a - 9] = (float)T[(a - 9) * 4 + 3];
  } else if (a == 12) {
    st->max_um = -1;
    st->n_cand = 0;
    st->work = 0;
    st->total = 0;
    st->clipped = 0;
    st->new_blocks = 0;
    st->updated = 0ull;
    st->pool_before = *n_blocks;
  }
}

__global__ void __launch_bounds__(256) k_tilemax(DevFrame f, DevParams p, const uint8_t* __restrict__ mask,
                                                 int* __restrict__ tilemax, IntegState* st, int tiles_x) {
  if (gated_off(f.gate, kModeFirst)) return;
  const int tile = blockIdx.x;
  const int u = (tile % tiles_x) * kTile + (threadIdx.x % kTile);
  const int v = (tile / tiles_x) * kTile + (threadIdx.x / kTile);
  int d = -1;
  if (u < f.W && v < f.H) {
    const int idx = v * f.W + u;
    const unsigned raw = f.depth[idx];
    if (pixel_valid(p, raw) && !(mask && mask[idx])) d = (int)(raw * p.du_um);
  }
  d = __reduce_max_sync(0xffffffffu, d);
  __shared__ int s[8];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = s[0];
    for (int w = 1; w < 8; ++w) m = max(m, s[w]);
    tilemax[tile] = m;
    if (m >= 0) atomicMax(&st->max_um, m);
  }
}

// Largest frustum search region (blocks); beyond it the frame is rejected
// with RF_ERR_OUT_OF_RANGE (d_max / voxel_size far too large, or a
// non-finite pose).
constexpr long long kMaxSearchBlocks = 1ll << 28;

// Block range of the truncated frustum z in (z_near, zfar], zfar =
// min(max valid depth + tau, d_max), over the pixel rectangle.  Float math on
// 8 lanes (one frustum corner each); the 2-voxel margin covers its rounding.
__global__ void k_integ_aabb(const double* __restrict__ T, DevFrame f, DevParams p, IntegState* st) {
  if (gated_off(f.gate, kModeFirst)) return;
  const int lane = threadIdx.x;
  const int max_um = st->max_um;
  if (max_um < 0) {
    if (lane == 0) st->total = 0;
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

// floor(num / den) for den > 0 when it lies in [0, n), else -1.  `guess` is
// a float estimate of num / den (within one unit when the result is in
// range); it is corrected and verified with exact int64 products.  No
// int64 <-> float conversion is used: those run on the FP64 pipe.
__device__ __forceinline__ int pixel_of(float guess, long long num, long long den, int n) {
  const float g = fminf(fmaxf(floorf(guess), -2.0f), (float)n + 1.0f);
  long long u = (long long)(int)g;
  if (u * den > num) u -= 1;
  else if ((u + 1) * den <= num) u += 1;
  if (u * den > num || (u + 1) * den <= num) return -1;
  return (u >= 0 && u < n) ? (int)u : -1;
}

// Exact nearest pixel of a voxel with camera coordinates (Cx, Cy, Cz) in
// ticks, or -1 when z is outside (z_near, d_max] or the pixel is outside the
// image.  (xf, yf, zf): float estimates used only for the guess.
__device__ __forceinline__ int voxel_pixel(long long Cx, long long Cy, long long Cz, float xf, float yf, float zf,
                                           const DevFrame& f, const DevParams& p, float fxg, float fyg, float cxg,
                                           float cyg) {
  if (Cz <= p.znear_tick || Cz > p.dmax_tick) return -1;
  const long long den = Cz << 8;
  const float iz = __fdividef(1.0f, zf);
  const int u = pixel_of(fxg * xf * iz + cxg, f.fxq * Cx + f.cxq * Cz, den, f.W);
  if (u < 0) return -1;
  const int v = pixel_of(fyg * yf * iz + cyg, f.fyq * Cy + f.cyq * Cz, den, f.H);
  if (v < 0) return -1;
  return v * f.W + u;
}

// Fast path of the nearest-pixel rounding: floor of the float estimate when
// it is farther than `amb` from a rounding boundary (then provably equal to
// the exact floor), else kAmbiguous.  Out-of-range results give -1.
constexpr int kAmbiguous = -2;
__device__ __forceinline__ int pixel_fast(float est, float amb, int n) {
  const float fl = floorf(est);
  const float fr = est - fl;
  if (fr < amb || fr > 1.0f - amb) return kAmbiguous;
  return (fl >= 0.0f && fl < (float)n) ? (int)fl : -1;
}

// Update value of a voxel whose pixel has raw depth `raw`: false when the
// voxel is not updated (invalid pixel or occluded: sdf < -tau).
__device__ __forceinline__ bool voxel_value(unsigned raw, long long Cz, const DevParams& p, float* x, bool* band) {
  if (!pixel_valid(p, raw)) return false;
  const long long sdf = (long long)raw * p.du_um * 1024 - Cz;
  if (sdf < -p.tau_tick) return false;
  *band = sdf <= p.tau_tick;
  if (*band) {
    // |sdf| <= tau_tick: a 32-bit conversion (exact below 2^31 ticks = 2.1 m)
    *x = p.tau_tick < (1ll << 31) ? __int2float_rn((int)sdf) * 9.765625e-10f
                                  : __int2float_rn((int)(sdf >> 8)) * 2.5e-7f;
  } else {
    *x = p.tau;
  }
  return true;
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

constexpr int kIntegThreads = 128;  // 4 warps; one warp integrates one block at a time
constexpr int kIntegWarps = kIntegThreads / 32;
constexpr int kVPL = kBV / 32;       // 16 voxels per lane: voxel lane + 32 j

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

// Per-lane constants of the voxel loop for one stream: lane l's offsets
// within a block (from the quantised rotation) and the intrinsics in pixels.
struct IntegConsts {
  long long O[3], SY4[3], SZ[3];
  float SY4f[3], SZf[3];
  float fxg, fyg, cxg, cyg;
};

__device__ __forceinline__ void integ_consts(const long long* A, const DevFrame& f, const DevParams& p, int lane,
                                             IntegConsts& c) {
  const long long lx = (long long)(lane & 7) * p.v_um, ly = (long long)(lane >> 3) * p.v_um;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c.O[i] = A[i * 3] * lx + A[i * 3 + 1] * ly;
    c.SY4[i] = A[i * 3 + 1] * (4 * p.v_um);
    c.SZ[i] = A[i * 3 + 2] * p.v_um;
    c.SY4f[i] = (float)(c.SY4[i] >> 20);  // float estimates in ticks, converted once per thread
    c.SZf[i] = (float)(c.SZ[i] >> 20);
  }
  c.fxg = (float)f.fxq * (1.0f / 256.0f);
  c.fyg = (float)f.fyq * (1.0f / 256.0f);
  c.cxg = (float)f.cxq * (1.0f / 256.0f);
  c.cyg = (float)f.cyq * (1.0f / 256.0f);
}

// One candidate block b, integrated by one warp.  Lane l owns voxels
// (x, y, z) = (l & 7, (l >> 3) + 4 (j & 1), j >> 1), j = 0..15, whose exact
// camera coordinates follow from the block's by int64 additions.  (1) nearest
// pixels of the 16 voxels (float estimate, exact integer path only near
// rounding boundaries), (2) depth loads four at a time and the exact
// truncation tests, (3) hash lookup (first bucket prefetched by lanes 0-3) or
// insert, (4) read-modify-write of the updated voxels.  Per-voxel values are
// staged in the warp's shared memory (spx, sx), not registers.  A and tq: the
// quantised pose (shared memory).
template <int ST>
__device__ __forceinline__ void integrate_block(const DevVol& v, const DevFrame& f, const DevParams& p,
                                                const uint8_t* __restrict__ mask, const long long* A,
                                                const long long* tq, const IntegConsts& c, const int4 b, int lane,
                                                int (*spx)[32], float (*sx)[32], unsigned& my_updated,
                                                unsigned& my_new) {
  const unsigned nan_bits = 0x7fc00000u;
  const unsigned long long key = pack_key(b.x, b.y, b.z);
  const bool in_range = coord_ok(b.x, b.y, b.z);
  const unsigned long long bucket = bucket_of(key, v.bucket_mask);
  unsigned long long e = kEmpty;
  if (lane < kSlots && in_range) e = __ldcg(v.hash + bucket * kSlots + lane);  // prefetch
  // exact camera coordinates of voxel (lane & 7, lane >> 3, 0) of this block
  long long c0[3];
  float c0f[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long d0 = (long long)b.x * 8 * p.v_um - tq[0], d1 = (long long)b.y * 8 * p.v_um - tq[1],
                    d2 = (long long)b.z * 8 * p.v_um - tq[2];
    c0[i] = A[i * 3] * d0 + A[i * 3 + 1] * d1 + A[i * 3 + 2] * d2 + c.O[i];
    c0f[i] = (float)(c0[i] >> 20);
  }
  // 1) nearest pixel of each voxel
#pragma unroll 2
  for (int j = 0; j < kVPL; ++j) {
    const int h = j & 1, zz = j >> 1;
    const long long Cz = (c0[2] + (h ? c.SY4[2] : 0ll) + zz * c.SZ[2]) >> 20;
    int pix = -1;
    if (Cz > p.znear_tick && Cz <= p.dmax_tick) {
      const float xf = c0f[0] + (h ? c.SY4f[0] : 0.0f) + (float)zz * c.SZf[0];
      const float yf = c0f[1] + (h ? c.SY4f[1] : 0.0f) + (float)zz * c.SZf[1];
      const float zf = c0f[2] + (h ? c.SY4f[2] : 0.0f) + (float)zz * c.SZf[2];
      const float iz = __frcp_rn(zf);
      const int u = pixel_fast(c.fxg * xf * iz + c.cxg, f.amb_u, f.W);
      const int vv = pixel_fast(c.fyg * yf * iz + c.cyg, f.amb_v, f.H);
      pix = (u == kAmbiguous || vv == kAmbiguous) ? kAmbiguous : ((u < 0 || vv < 0) ? -1 : vv * f.W + u);
      if (pix == kAmbiguous) {
        const long long Cx = (c0[0] + (h ? c.SY4[0] : 0ll) + zz * c.SZ[0]) >> 20;
        const long long Cy = (c0[1] + (h ? c.SY4[1] : 0ll) + zz * c.SZ[1]) >> 20;
        pix = voxel_pixel(Cx, Cy, Cz, xf, yf, zf, f, p, c.fxg, c.fyg, c.cxg, c.cyg);
      }
    }
    spx[j][lane] = pix;
  }
  // 2) depth (and mask) loads, four voxels at a time, and the exact tests
  unsigned passbits = 0;
#pragma unroll 4
  for (int j = 0; j < kVPL; ++j) {
    const int pix = spx[j][lane];
    unsigned raw = pix >= 0 ? (unsigned)__ldg(f.depth + pix) : 0u;
    if (mask && pix >= 0 && __ldg(mask + pix)) raw = 0u;  // masked pixel: as invalid
    const int h = j & 1, zz = j >> 1;
    const long long Cz = (c0[2] + (h ? c.SY4[2] : 0ll) + zz * c.SZ[2]) >> 20;
    float x = 0.0f;
    bool band = false;
    const bool ok = pix >= 0 && voxel_value(raw, Cz, p, &x, &band);
    sx[j][lane] = x;
    if (band) spx[j][lane] = pix | (int)0x80000000;
    passbits |= ok ? (1u << j) : 0u;
  }
  if (!__any_sync(0xffffffffu, passbits != 0)) return;
  // 3) pool index: from the prefetched bucket, else probe/insert by lane 0
  const unsigned found = __ballot_sync(0xffffffffu, lane < kSlots && e != kEmpty && (e >> 22) == key);
  int pool;
  bool fresh = false;
  if (found) {
    pool = (int)(__shfl_sync(0xffffffffu, e, __ffs(found) - 1) & 0x3FFFFFull);
  } else {
    int pl = -1, nw = 0;
    if (lane == 0) {
      bool is_new;
      pl = hash_insert(v, b.x, b.y, b.z, &is_new);
      nw = is_new;
    }
    pool = __shfl_sync(0xffffffffu, pl, 0);
    fresh = __shfl_sync(0xffffffffu, nw, 0) != 0;
  }
  if (pool < 0) return;
  my_new += (lane == 0 && fresh) ? 1u : 0u;
  my_updated += __popc(passbits);
  if constexpr (ST == RF_STORAGE_FP32) {
    uint2* vb = v.vox + (size_t)pool * kBV + lane;
    uint8_t* wb = v.W + (size_t)pool * kBV + lane;
    // 4) read-modify-write
#pragma unroll 4
    for (int j = 0; j < kVPL; ++j) {
      const bool pass = (passbits >> j) & 1u;
      uint2 w;
      unsigned W;
      if (fresh) {
        w = make_uint2(nan_bits, 0u);
        W = 0;
      } else {
        if (!pass) continue;
        w = vb[32 * j];
        W = wb[32 * j];
      }
      if (pass) {
        const float F = __uint_as_float(w.x);
        const float x = sx[j][lane];
        const int px = spx[j][lane];
        const float Fn = (W == 0) ? x : __fdividef((float)W * F + x, (float)(W + 1));
        w.x = __float_as_uint(Fn);
        if (px < 0) w.y = colour_update(w.y, f.rgb + 3 * (size_t)(px & 0x7fffffff), p.w_max);  // band
        W = min(W + 1, (unsigned)p.w_max);
      }
      vb[32 * j] = w;
      wb[32 * j] = (uint8_t)W;
    }
  } else {
    // FP16 storage: the tracking word always, the colour word inside the band
    unsigned* tb = trk_words_rw(v, pool) + lane;
    unsigned* cb = tb + kBV;
#pragma unroll 4
    for (int j = 0; j < kVPL; ++j) {
      const bool pass = (passbits >> j) & 1u;
      unsigned t;
      if (fresh) {
        t = kTrkEmpty;
      } else {
        if (!pass) continue;
        t = tb[32 * j];
      }
      unsigned col = 0u;
      bool col_written = fresh;
      if (pass) {
        const unsigned W = t >> 24;
        const float x = sx[j][lane];
        const int px = spx[j][lane];
        const float F = __half2float(__ushort_as_half((unsigned short)(t & 0xFFFFu))) * p.tau;
        const float Fn = (W == 0) ? x : __fdividef((float)W * F + x, (float)(W + 1));
        const unsigned h = (unsigned)__half_as_ushort(__float2half_rn(Fn * p.inv_tau));
        unsigned i8 = (t >> 16) & 255u;
        if (px < 0) {  // band: colour, and the intensity derived from it
          col = colour_update(fresh ? 0u : cb[32 * j], f.rgb + 3 * (size_t)(px & 0x7fffffff), p.w_max);
          col_written = true;
          i8 = rgb_i8(col);
        }
        t = h | (i8 << 16) | (min(W + 1, (unsigned)p.w_max) << 24);
      }
      tb[32 * j] = t;
      if (col_written) cb[32 * j] = col;
    }
  }
}

// Counts of one warp for one stream's integration statistics.
__device__ __forceinline__ void integ_flush(IntegState* st, unsigned updated, unsigned fresh, int lane) {
  updated = __reduce_add_sync(0xffffffffu, updated);
  fresh = __reduce_add_sync(0xffffffffu, fresh);
  if (lane == 0 && updated) atomicAdd(&st->updated, (unsigned long long)updated);
  if (lane == 0 && fresh) atomicAdd(&st->new_blocks, (int)fresh);
}

// One warp per candidate block (static round-robin over all warps): no CTA
// barriers.
template <int ST>
__global__ void __launch_bounds__(kIntegThreads) k_integrate(DevVol v, DevFrame f, DevParams p,
                                                             const uint8_t* __restrict__ mask, IntegState* st,
                                                             const int4* __restrict__ cand, long long max_cand) {
  __shared__ int s_px[kIntegWarps][kVPL][32];    // pixel index | band << 31, or -1
  __shared__ float s_x[kIntegWarps][kVPL][32];   // update value
  __shared__ long long A[9], tq[3];              // quantised pose
  if (gated_off(f.gate, kModeFirst)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < 9) A[threadIdx.x] = st->A[threadIdx.x];
  if (threadIdx.x < 3) tq[threadIdx.x] = st->tq[threadIdx.x];
  __syncthreads();
  const long long n_cand = min((long long)*(volatile int*)&st->n_cand, max_cand);
  IntegConsts c;
  integ_consts(A, f, p, lane, c);
  const long long warp0 = ((long long)blockIdx.x * kIntegThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kIntegThreads) >> 5;
  unsigned my_updated = 0, my_new = 0;
  for (long long ci = warp0; ci < n_cand; ci += nwarps)
    integrate_block<ST>(v, f, p, mask, A, tq, c, cand[ci], lane, s_px[wid], s_x[wid], my_updated, my_new);
  integ_flush(st, my_updated, my_new, lane);
}

// Neighbour tables of the blocks allocated since `lo`: each new block gets
// the pools of its 7 positive neighbours, and each existing negative
// neighbour gets the new block in the matching slot.  Runs after the
// integration (the hash is complete and read-only here).
__device__ __forceinline__ void fixup_block(const DevVol& v, int b) {
  const int4 c = v.coords[b];
  if (c.w == 0) return;
  int* flat = reinterpret_cast<int*>(v.nbr);
  int t[8];
  t[0] = b;
#pragma unroll
  for (int o = 1; o < 8; ++o) t[o] = hash_find(v, c.x + (o & 1), c.y + ((o >> 1) & 1), c.z + ((o >> 2) & 1));
  v.nbr[2 * (size_t)b] = make_int4(t[0], t[1], t[2], t[3]);
  v.nbr[2 * (size_t)b + 1] = make_int4(t[4], t[5], t[6], t[7]);
#pragma unroll
  for (int o = 1; o < 8; ++o) {
    const int n = hash_find(v, c.x - (o & 1), c.y - ((o >> 1) & 1), c.z - ((o >> 2) & 1));
    if (n >= 0) flat[8 * (size_t)n + o] = b;
  }
}

__global__ void __launch_bounds__(256) k_nbr_fixup(DevVol v, const int* __restrict__ lo_ptr, int lo_value,
                                                   const int* gate) {
  if (gated_off(gate, kModeFirst)) return;
  const int lo = lo_ptr ? *lo_ptr : lo_value;
  const int hi = min(*(volatile int*)v.n_blocks, v.max_blocks);
  for (int b = lo + blockIdx.x * blockDim.x + threadIdx.x; b < hi; b += gridDim.x * blockDim.x) fixup_block(v, b);
}

}  // namespace

rf_status launch_nbr_fixup(rf_volume* vol, const int* lo_ptr, int lo, cudaStream_t st, const int* gate) {
  k_nbr_fixup<<<vol->sm_count * vol->launch.fixup_ctas_per_sm, 256, 0, st>>>(vol->dv, lo_ptr, lo, gate);
  return check_cuda(vol, cudaGetLastError(), "neighbour table launch");
}

// The frustum search of an integration: prep, tile maxima, AABB, cull.
static rf_status launch_frustum(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st) {
  const int tiles_x = (f.W + kTile - 1) / kTile, tiles_y = (f.H + kTile - 1) / kTile;
  k_integ_prep<<<1, 32, 0, st>>>(T, vol->d_integ, vol->d_nblocks, f.gate);
  k_tilemax<<<tiles_x * tiles_y, 256, 0, st>>>(f, vol->dp, mask, vol->d_tilemax, vol->d_integ, tiles_x);
  k_integ_aabb<<<1, 32, 0, st>>>(T, f, vol->dp, vol->d_integ);
  k_cull<<<vol->sm_count * vol->launch.cull_ctas_per_sm, 256, 0, st>>>(f, vol->dp, vol->d_integ, vol->d_tilemax, tiles_x, tiles_y, vol->d_cand,
                                            vol->p.max_candidates, vol->d_status);
  return check_cuda(vol, cudaGetLastError(), "frustum launch");
}

rf_status launch_integrate(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st) {
  rf_status s = launch_frustum(vol, f, T, mask, st);
  if (s != RF_OK) return s;
  prof_record(vol, EV_KERNEL0, st);
  if (vol->p.storage == RF_STORAGE_FP16)
    k_integrate<RF_STORAGE_FP16><<<vol->sm_count * vol->launch.integrate_ctas_per_sm, kIntegThreads, 0, st>>>(vol->dv, f, vol->dp, mask, vol->d_integ,
                                                                             vol->d_cand, vol->p.max_candidates);
  else
    k_integrate<RF_STORAGE_FP32><<<vol->sm_count * vol->launch.integrate_ctas_per_sm, kIntegThreads, 0, st>>>(vol->dv, f, vol->dp, mask, vol->d_integ,
                                                                             vol->d_cand, vol->p.max_candidates);
  prof_record(vol, EV_KERNEL1, st);
  s = check_cuda(vol, cudaGetLastError(), "integrate launch");
  if (s != RF_OK) return s;
  return launch_nbr_fixup(vol, &vol->d_integ->pool_before, 0, st, f.gate);
}

}  // namespace rf
