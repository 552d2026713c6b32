// Zero-crossing surface of the TSDF (the mesh ReFusion produces, Sec. I) by
// marching tetrahedra: every cell whose 8 lattice corners are observed is cut
// into the 6 Kuhn tetrahedra 0 -> e_a -> e_a + e_b -> 7 (one per axis order
// a, b, c), and each tetrahedron with corners of both signs (inside: F < 0)
// emits one triangle (1 or 3 inside) or two (2 inside).  Vertices are linear
// zero crossings on the edges; triangles are wound so that their normal points
// towards positive SDF.  One CTA per allocated block; pass 0 counts, pass 1
// writes (slots from an atomic counter, so the triangle order is arbitrary).
#include "rf_volume.hpp"

namespace rf {
namespace {

__device__ __forceinline__ int parity3(int a, int b, int c) {
  return ((a > b) + (a > c) + (b > c)) & 1;
}

__device__ __forceinline__ int parity4(const int* o) {
  int inv = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i + 1; j < 4; ++j) inv += o[i] > o[j];
  return inv & 1;
}

struct Cell {
  float F[8];
  float P[8][3];
  unsigned C[8];  // rgb | wc << 24
};

__device__ void put_vertex(const Cell& c, int a, int b, float* vout, uint8_t* cout) {
  const float t = c.F[a] / (c.F[a] - c.F[b]);
#pragma unroll
  for (int i = 0; i < 3; ++i) vout[i] = c.P[a][i] + t * (c.P[b][i] - c.P[a][i]);
  const bool oka = (c.C[a] >> 24) != 0u, okb = (c.C[b] >> 24) != 0u;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float ca = (float)((c.C[a] >> (8 * ch)) & 255u), cb = (float)((c.C[b] >> (8 * ch)) & 255u);
    float v = 0.0f;
    if (oka && okb) v = ca + t * (cb - ca);
    else if (oka) v = ca;
    else if (okb) v = cb;
    cout[ch] = (uint8_t)fminf(fmaxf(rintf(v), 0.0f), 255.0f);
  }
}

// Emits the triangles of one tetrahedron (corner ids tv[0..3], positively
// oriented); returns the number emitted (written only when out != nullptr).
__device__ int tet_tris(const Cell& c, const int tv[4], float* vout, uint8_t* cout) {
  int inside[4], outside[4], ni = 0, no = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (c.F[tv[i]] < 0.0f) inside[ni++] = i;
    else outside[no++] = i;
  }
  if (ni == 0 || ni == 4) return 0;
  if (ni == 1 || ni == 3) {
    int o[4];
    o[0] = ni == 1 ? inside[0] : outside[0];
    int m = 1;
    for (int i = 0; i < 4; ++i)
      if (i != o[0]) o[m++] = i;
    if (parity4(o)) { const int t = o[2]; o[2] = o[3]; o[3] = t; }
    if (ni == 3) { const int t = o[2]; o[2] = o[3]; o[3] = t; }
    if (vout) {
      put_vertex(c, tv[o[0]], tv[o[1]], vout + 0, cout + 0);
      put_vertex(c, tv[o[0]], tv[o[2]], vout + 3, cout + 3);
      put_vertex(c, tv[o[0]], tv[o[3]], vout + 6, cout + 6);
    }
    return 1;
  }
  int o[4] = {inside[0], inside[1], outside[0], outside[1]};
  if (parity4(o)) { const int t = o[2]; o[2] = o[3]; o[3] = t; }
  if (vout) {
    put_vertex(c, tv[o[0]], tv[o[2]], vout + 0, cout + 0);
    put_vertex(c, tv[o[0]], tv[o[3]], vout + 3, cout + 3);
    put_vertex(c, tv[o[1]], tv[o[3]], vout + 6, cout + 6);
    put_vertex(c, tv[o[0]], tv[o[2]], vout + 9, cout + 9);
    put_vertex(c, tv[o[1]], tv[o[3]], vout + 12, cout + 12);
    put_vertex(c, tv[o[1]], tv[o[2]], vout + 15, cout + 15);
  }
  return 2;
}

template <int ST>
__global__ void __launch_bounds__(256) k_mesh(DevVol v, float voxel, float tau, int pass, unsigned long long* counter,
                                              float* verts, uint8_t* colors, long long cap) {
  const int pool = blockIdx.x;
  const int4 bc = v.coords[pool];
  if (bc.w == 0) return;
  __shared__ int nb[8];
  if (threadIdx.x < 8) {
    const int t = threadIdx.x;
    nb[t] = t == 0 ? pool : hash_find(v, bc.x + (t & 1), bc.y + ((t >> 1) & 1), bc.z + ((t >> 2) & 1));
  }
  __syncthreads();
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int cell = threadIdx.x; cell < kBV; cell += blockDim.x) {
    const int x = cell & 7, y = (cell >> 3) & 7, z = cell >> 6;
    Cell c;
    bool ok = true;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int xx = x + (n & 1), yy = y + ((n >> 1) & 1), zz = z + ((n >> 2) & 1);
      const int nbi = (xx >> 3) + 2 * (yy >> 3) + 4 * (zz >> 3);
      const int p = nb[nbi];
      if (p < 0) { ok = false; break; }
      const int i = (xx & 7) + 8 * (yy & 7) + 64 * (zz & 7);
      if constexpr (ST == RF_STORAGE_FP32) {
        const uint2 w = v.vox[(size_t)p * kBV + i];
        c.F[n] = __uint_as_float(w.x);
        c.C[n] = w.y;
      } else {
        const unsigned* tw = trk_words(v, p);
        c.F[n] = trk_sdf(tw[i], tau);
        c.C[n] = tw[kBV + i];
      }
      if (c.F[n] != c.F[n]) { ok = false; break; }
      c.P[n][0] = (float)(bc.x * 8 + xx) * voxel;
      c.P[n][1] = (float)(bc.y * 8 + yy) * voxel;
      c.P[n][2] = (float)(bc.z * 8 + zz) * voxel;
    }
    if (!ok) continue;
    int tvs[6][4];
    int total = 0;
#pragma unroll
    for (int pi = 0; pi < 6; ++pi) {
      const int a = perms[pi][0], b = perms[pi][1];
      tvs[pi][0] = 0;
      tvs[pi][1] = 1 << a;
      tvs[pi][2] = (1 << a) | (1 << b);
      tvs[pi][3] = 7;
      if (parity3(perms[pi][0], perms[pi][1], perms[pi][2])) {
        const int t = tvs[pi][1]; tvs[pi][1] = tvs[pi][2]; tvs[pi][2] = t;
      }
      total += tet_tris(c, tvs[pi], nullptr, nullptr);
    }
    if (total == 0) continue;
    const unsigned long long slot = atomicAdd(counter, (unsigned long long)total);
    if (pass == 0 || slot + total > (unsigned long long)cap) continue;
    unsigned long long s = slot;
    for (int pi = 0; pi < 6; ++pi) s += tet_tris(c, tvs[pi], verts + s * 9, colors + s * 9);
  }
}

}  // namespace

rf_status run_mesh(rf_volume* vol, float* verts, uint8_t* colors, int64_t cap, int64_t* n, cudaStream_t st) {
  int nb = 0;
  rf_status s = check_cuda(vol, cudaMemcpyAsync(&nb, vol->d_nblocks, sizeof(int), cudaMemcpyDeviceToHost, st),
                           "mesh block count");
  if (s != RF_OK) return s;
  s = check_cuda(vol, cudaStreamSynchronize(st), "mesh sync");
  if (s != RF_OK) return s;
  if (nb > vol->max_blocks) nb = (int)vol->max_blocks;
  unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(vol->d_partials);  // scratch reuse
  unsigned long long cnt = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && (verts == nullptr || colors == nullptr)) break;
    s = check_cuda(vol, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st), "mesh reset");
    if (s != RF_OK) return s;
    if (nb > 0 && vol->p.storage == RF_STORAGE_FP16)
      k_mesh<RF_STORAGE_FP16><<<nb, 256, 0, st>>>(vol->dv, vol->dp.voxel, vol->dp.tau, pass, d_cnt, verts, colors, cap);
    else if (nb > 0)
      k_mesh<RF_STORAGE_FP32><<<nb, 256, 0, st>>>(vol->dv, vol->dp.voxel, vol->dp.tau, pass, d_cnt, verts, colors, cap);
    s = check_cuda(vol, cudaGetLastError(), "mesh launch");
    if (s != RF_OK) return s;
    s = check_cuda(vol, cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st), "mesh count");
    if (s != RF_OK) return s;
    s = check_cuda(vol, cudaStreamSynchronize(st), "mesh sync");
    if (s != RF_OK) return s;
    if (pass == 0 && verts != nullptr && (int64_t)cnt > cap) {
      *n = (int64_t)cnt;
      return set_error(vol, RF_ERR_BUFFER_TOO_SMALL, "mesh has %lld triangles, buffer holds %lld", (long long)cnt,
                       (long long)cap);
    }
  }
  *n = (int64_t)cnt;
  return RF_OK;
}

}  // namespace rf
