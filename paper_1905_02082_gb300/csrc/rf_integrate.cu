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
//                  with updates, read-modify-write of updated voxels (block/CTA,
//                  persistent, blocks taken from an atomic work counter)
#include <cmath>

#include "rf_volume.hpp"

namespace rf {
namespace {

__global__ void k_integ_prep(const double* __restrict__ T, IntegState* st) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      st->A[i * 3 + j] = llround(T[j * 4 + i] * 1073741824.0);
      st->R[i * 3 + j] = (float)T[i * 4 + j];
    }
  for (int i = 0; i < 3; ++i) {
    st->tq[i] = llround(T[i * 4 + 3] * 1e6);
    st->t[i] = (float)T[i * 4 + 3];
  }
  st->max_um = -1;
  st->n_cand = 0;
  st->work = 0;
  st->total = 0;
  st->clipped = 0;
  st->new_blocks = 0;
  st->updated = 0ull;
}

__global__ void __launch_bounds__(256) k_tilemax(DevFrame f, DevParams p, const uint8_t* __restrict__ mask,
                                                 int* __restrict__ tilemax, IntegState* st, int tiles_x) {
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

__global__ void k_integ_aabb(const double* __restrict__ T, DevFrame f, DevParams p, IntegState* st) {
  if (threadIdx.x != 0) return;
  if (st->max_um < 0) {
    st->total = 0;
    return;
  }
  for (int i = 0; i < 12; ++i)
    if (!isfinite(T[i])) {
      st->total = 0;
      st->clipped = 1;
      return;
    }
  const double zfar = fmin(st->max_um * 1e-6 + p.tau_d, (double)p.dmax_um * 1e-6);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  const double us[2] = {-0.5, f.W - 0.5}, vs[2] = {-0.5, f.H - 0.5};
  const double zs[2] = {(double)p.z_near, zfar};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        const double z = zs[a];
        const double x = (us[b] - f.cxd) / f.fxd * z, y = (vs[c] - f.cyd) / f.fyd * z;
        for (int i = 0; i < 3; ++i) {
          const double w = T[i * 4 + 0] * x + T[i * 4 + 1] * y + T[i * 4 + 2] * z + T[i * 4 + 3];
          lo[i] = fmin(lo[i], w);
          hi[i] = fmax(hi[i], w);
        }
      }
  const double bs = 8.0 * p.voxel_d, margin = 2.0 * p.voxel_d;
  long long total = 1;
  bool clipped = false;
  for (int i = 0; i < 3; ++i) {
    const double f0 = fmax(fmin(floor((lo[i] - margin) / bs), 1e9), -1e9);
    const double f1 = fmax(fmin(floor((hi[i] + margin) / bs), 1e9), -1e9);
    long long b0 = (long long)f0;
    long long b1 = (long long)f1;
    if (b0 < -kMaxCoord) { b0 = -kMaxCoord; clipped = true; }
    if (b1 > kMaxCoord) { b1 = kMaxCoord; clipped = true; }
    if (b1 < b0) b1 = b0 - 1;
    st->bmin[i] = (int)b0;
    st->dims[i] = (int)(b1 - b0 + 1);
    total *= (b1 - b0 + 1);
  }
  if (total > kMaxSearchBlocks) {
    total = 0;
    clipped = true;
  }
  st->total = total > 0 ? total : 0;
  st->zfar = (float)zfar;
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

// floor(num / den) for den > 0 when it lies in [0, n), else -1.  A float
// guess is corrected and verified with exact int64 products.
__device__ __forceinline__ int pixel_of(long long num, long long den, int n) {
  float g = floorf(__fdividef(__ll2float_rn(num), __ll2float_rn(den)));
  g = fminf(fmaxf(g, -2.0f), (float)n + 1.0f);
  long long u = (long long)g;
  if (u * den > num) u -= 1;
  else if ((u + 1) * den <= num) u += 1;
  if (u * den > num || (u + 1) * den <= num) return -1;
  return (u >= 0 && u < n) ? (int)u : -1;
}

struct Obs {
  float x;
  int pix;
  bool band;
};

__device__ __forceinline__ bool observe(long long Cx, long long Cy, long long Cz, const DevFrame& f,
                                        const DevParams& p, const uint8_t* __restrict__ mask, Obs* o) {
  if (Cz <= p.znear_tick || Cz > p.dmax_tick) return false;
  const long long den = Cz << 8;
  const int u = pixel_of(f.fxq * Cx + f.cxq * Cz, den, f.W);
  if (u < 0) return false;
  const int v = pixel_of(f.fyq * Cy + f.cyq * Cz, den, f.H);
  if (v < 0) return false;
  const int idx = v * f.W + u;
  const unsigned raw = __ldg(f.depth + idx);
  if (!pixel_valid(p, raw)) return false;
  if (mask && __ldg(mask + idx)) return false;
  const long long sdf = (long long)raw * p.du_um * 1024 - Cz;
  if (sdf < -p.tau_tick) return false;
  o->band = sdf <= p.tau_tick;
  o->x = o->band ? __ll2float_rn(sdf) * 9.765625e-10f : p.tau;
  o->pix = idx;
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
  const unsigned long long b = mix64(key) & v.bucket_mask;
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

constexpr int kIntegThreads = 256;
constexpr int kVPT = kBV / kIntegThreads;  // voxels per thread

__global__ void __launch_bounds__(kIntegThreads) k_integrate(DevVol v, DevFrame f, DevParams p,
                                                             const uint8_t* __restrict__ mask, IntegState* st,
                                                             const int4* __restrict__ cand, long long max_cand) {
  __shared__ long long sA[9], sT[3];
  __shared__ long long sC0[3];
  __shared__ int s_idx, s_pool, s_new;
  if (threadIdx.x < 9) sA[threadIdx.x] = st->A[threadIdx.x];
  if (threadIdx.x < 3) sT[threadIdx.x] = st->tq[threadIdx.x];
  __syncthreads();
  const long long n_cand = min((long long)*(volatile int*)&st->n_cand, max_cand);
  // per-thread lattice offsets A * (v_um * o) of the voxels this thread owns
  long long off[kVPT][3];
#pragma unroll
  for (int j = 0; j < kVPT; ++j) {
    const int li = threadIdx.x + j * kIntegThreads;
    const long long o[3] = {(long long)(li & 7) * p.v_um, (long long)((li >> 3) & 7) * p.v_um,
                            (long long)(li >> 6) * p.v_um};
#pragma unroll
    for (int i = 0; i < 3; ++i) off[j][i] = sA[i * 3] * o[0] + sA[i * 3 + 1] * o[1] + sA[i * 3 + 2] * o[2];
  }
  const unsigned nan_bits = 0x7fc00000u;
  unsigned my_updated = 0;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(&st->work, 1);
    __syncthreads();
    const int ci = s_idx;
    if (ci >= n_cand) break;
    const int4 b = cand[ci];
    if (threadIdx.x < 3) {
      const int i = threadIdx.x;
      const long long d0 = (long long)b.x * 8 * p.v_um - sT[0];
      const long long d1 = (long long)b.y * 8 * p.v_um - sT[1];
      const long long d2 = (long long)b.z * 8 * p.v_um - sT[2];
      sC0[i] = sA[i * 3] * d0 + sA[i * 3 + 1] * d1 + sA[i * 3 + 2] * d2;
    }
    __syncthreads();
    Obs ob[kVPT];
    bool pass[kVPT];
    int any = 0;
#pragma unroll
    for (int j = 0; j < kVPT; ++j) {
      const long long Cx = (sC0[0] + off[j][0]) >> 20;
      const long long Cy = (sC0[1] + off[j][1]) >> 20;
      const long long Cz = (sC0[2] + off[j][2]) >> 20;
      pass[j] = observe(Cx, Cy, Cz, f, p, mask, &ob[j]);
      any |= pass[j];
    }
    if (!__syncthreads_or(any)) continue;
#pragma unroll
    for (int j = 0; j < kVPT; ++j) my_updated += pass[j];
    if (threadIdx.x == 0) {
      bool is_new;
      s_pool = hash_insert(v, b.x, b.y, b.z, &is_new);
      s_new = is_new;
      if (is_new) atomicAdd(&st->new_blocks, 1);
    }
    __syncthreads();
    const int pool = s_pool;
    if (pool < 0) continue;
    const bool fresh = s_new != 0;
    uint2* vb = v.vox + (size_t)pool * kBV;
    uint8_t* wb = v.W + (size_t)pool * kBV;
#pragma unroll
    for (int j = 0; j < kVPT; ++j) {
      const int li = threadIdx.x + j * kIntegThreads;
      uint2 w;
      unsigned W;
      if (fresh) {
        w = make_uint2(nan_bits, 0u);
        W = 0;
      } else {
        if (!pass[j]) continue;
        w = vb[li];
        W = wb[li];
      }
      if (pass[j]) {
        const float F = __uint_as_float(w.x);
        const float x = ob[j].x;
        const float Fn = (W == 0) ? x : ((float)W * F + x) / (float)(W + 1);
        w.x = __float_as_uint(Fn);
        if (ob[j].band) {
          const uint8_t* c = f.rgb + 3 * (size_t)ob[j].pix;
          const unsigned wc = w.y >> 24;
          unsigned out = 0;
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            const unsigned num = wc * ((w.y >> (8 * ch)) & 255u) + __ldg(c + ch);
            out |= ((2 * num + wc + 1) / (2 * (wc + 1))) << (8 * ch);
          }
          w.y = out | (min(wc + 1, (unsigned)p.w_max) << 24);
        }
        W = min(W + 1, (unsigned)p.w_max);
      }
      vb[li] = w;
      wb[li] = (uint8_t)W;
    }
  }
  my_updated = __reduce_add_sync(0xffffffffu, my_updated);
  if ((threadIdx.x & 31) == 0 && my_updated) atomicAdd(&st->updated, (unsigned long long)my_updated);
}

}  // namespace

rf_status launch_integrate(rf_volume* vol, const DevFrame& f, const double* T, const uint8_t* mask, cudaStream_t st) {
  const int tiles_x = (f.W + kTile - 1) / kTile, tiles_y = (f.H + kTile - 1) / kTile;
  k_integ_prep<<<1, 32, 0, st>>>(T, vol->d_integ);
  k_tilemax<<<tiles_x * tiles_y, 256, 0, st>>>(f, vol->dp, mask, vol->d_tilemax, vol->d_integ, tiles_x);
  k_integ_aabb<<<1, 32, 0, st>>>(T, f, vol->dp, vol->d_integ);
  k_cull<<<vol->sm_count * 8, 256, 0, st>>>(f, vol->dp, vol->d_integ, vol->d_tilemax, tiles_x, tiles_y, vol->d_cand,
                                            vol->p.max_candidates, vol->d_status);
  prof_record(vol, EV_KERNEL0, st);
  k_integrate<<<vol->sm_count * 4, kIntegThreads, 0, st>>>(vol->dv, f, vol->dp, mask, vol->d_integ, vol->d_cand,
                                                           vol->p.max_candidates);
  prof_record(vol, EV_KERNEL1, st);
  return check_cuda(vol, cudaGetLastError(), "integrate launch");
}

}  // namespace rf
