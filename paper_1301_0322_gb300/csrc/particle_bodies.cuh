// Per-particle device bodies of a COLA force evaluation (Sec. 2 PM code; App. A.3 eq. KDKALC),
// shared by the single-box kernels and the multi-box (ensemble) kernels.  The binning bodies
// (count_key, place_record and the four-particle keys_x4_body, scatter_x4_body) use warp-wide
// votes and must be called by all 32 lanes of a warp (live marks the lanes that own a
// particle); the gather and kick/drift bodies handle the one particle p of the calling thread.
#pragma once
#include "cola_internal.cuh"
#include "pm_common.cuh"

namespace cola {

// key = tile_bin(ty_tile, tz_tile) * 4 + ry + 2 rz, where ry (rz) marks a particle whose cell
// is the last row of its tile along y (z): its cloud also reaches the next tile.
// Tile sizes are powers of two (4 x 2 rows for a plan, 2 .. 16 rows per axis in an ensemble).
__device__ __forceinline__ int tile_key(const Tiles& tl, int cy, int cz) {
  const int ty = cy >> (__ffs(tl.ty) - 1), tz = cz >> (__ffs(tl.tz) - 1);
  const int ry = ((cy & (tl.ty - 1)) == tl.ty - 1) ? 1 : 0;
  const int rz = ((cz & (tl.tz - 1)) == tl.tz - 1) ? 2 : 0;
  return tile_bin(tl, ty, tz) * 4 + ry + rz;
}

// Tile key of particle p with displacement (sx, sy, sz); flags a non-finite displacement.
__device__ __forceinline__ int particle_key(const Geometry& g, const Tiles& tl, int64_t p, float sx, float sy,
                                            float sz, int* __restrict__ err) {
  int ix, iy, iz;
  lattice_index(g, p, ix, iy, iz);
  if (!isfinite(sx) || !isfinite(sy) || !isfinite(sz)) atomicOr(err, kErrNonFinite);
  int cy, ty, cz, tz;
  fixed_axis(g, iy, sy, cy, ty);
  fixed_axis(g, iz, sz, cz, tz);
  return tile_key(tl, cy, cz);
}

// counts[key] += 1 for the key of every live lane, one atomic per distinct key in the warp
__device__ __forceinline__ void count_key(int key, bool live, int* __restrict__ counts) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (live && lane == __ffs(peers) - 1) atomicAdd(&counts[key], __popc(peers));
}

// Record of particle p: its fixed-point CIC coordinates f_d = (cell << F) | t (each < ng 2^F <=
// 2^31) and its lattice index, so the deposit and the gather read them in bin order with one
// 16-byte access.
__device__ __forceinline__ uint4 particle_record(const Geometry& g, int64_t p, float sx, float sy, float sz) {
  int ix, iy, iz;
  lattice_index(g, p, ix, iy, iz);
  const int li[3] = {ix, iy, iz};
  const float sd[3] = {sx, sy, sz};
  uint32_t f[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int c, t;
    fixed_axis(g, li[d], sd[d], c, t);
    f[d] = ((uint32_t)c << g.fbits) | (uint32_t)t;
  }
  return make_uint4(f[0], f[1], f[2], (uint32_t)p);
}

// rec[cursor[key]++] = r for every live lane (one atomic per distinct key in the warp; lanes
// with the same key take consecutive slots in lane order)
__device__ __forceinline__ void place_record(int key, bool live, uint4 r, int* __restrict__ cursor,
                                             uint4* __restrict__ rec) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int base = 0;
  if (live && lane == leader) base = atomicAdd(&cursor[key], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  if (live) rec[base + __popc(peers & ((1u << lane) - 1u))] = r;
}

// Four particles per thread in warp-strided rounds: the block of nt threads takes the 4 nt
// particles from q0, warp w the 128 from q0 + 128 w, lane l of it the particles 32 u + l
// (u = 0..3).  All four loads of a thread are in flight together (four times the bytes of one
// particle per thread, which leaves these kernels bound by memory latency), and each round u
// still covers 32 consecutive particles: as few distinct keys per warp as one particle per
// thread, and the records of a bin stay in lattice order within each warp.
constexpr int kPartPerThread = 4;
__device__ __forceinline__ int64_t x4_first(int64_t q0) {
  return q0 + (int64_t)(threadIdx.x & ~31) * kPartPerThread + (threadIdx.x & 31);
}

// keys (plus bin_base) and bin counts of the particles of this thread (see x4_first)
__device__ __forceinline__ void keys_x4_body(const Geometry& g, const Tiles& tl, const float* __restrict__ s,
                                             int64_t q0, int bin_base, int* __restrict__ keys,
                                             int* __restrict__ counts, int* __restrict__ err) {
  constexpr int U = kPartPerThread;
  const int64_t p0 = x4_first(q0);
  float sx[U], sy[U], sz[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = p0 + 32 * u;
    if (p < g.np3) {
      sx[u] = __ldg(s + p);
      sy[u] = __ldg(s + g.np3 + p);
      sz[u] = __ldg(s + 2 * g.np3 + p);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = p0 + 32 * u;
    const bool live = p < g.np3;
    int key = -1;
    if (live) {
      key = bin_base + particle_key(g, tl, p, sx[u], sy[u], sz[u], err);
      keys[p] = key;
    }
    count_key(key, live, counts);
  }
}

// records of the particles of this thread into their bins (see x4_first)
__device__ __forceinline__ void scatter_x4_body(const Geometry& g, const float* __restrict__ s, int64_t q0,
                                                const int* __restrict__ keys, int* __restrict__ cursor,
                                                uint4* __restrict__ rec) {
  constexpr int U = kPartPerThread;
  const int64_t p0 = x4_first(q0);
  int k[U];
  float sx[U], sy[U], sz[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = p0 + 32 * u;
    k[u] = -1;
    if (p < g.np3) {
      k[u] = __ldg(keys + p);
      sx[u] = __ldg(s + p);
      sy[u] = __ldg(s + g.np3 + p);
      sz[u] = __ldg(s + 2 * g.np3 + p);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t p = p0 + 32 * u;
    const bool live = p < g.np3;
    place_record(k[u], live, live ? particle_record(g, p, sx[u], sy[u], sz[u]) : uint4{}, cursor, rec);
  }
}

// CIC gather of the three force meshes fmesh [3][ng^3] for a cloud that starts at cells c with
// upper-neighbour weights t / 2^F (the deposit's weights).
__device__ __forceinline__ void gather_force(const Geometry& g, const float* __restrict__ fmesh, const int (&c)[3],
                                             const int (&t)[3], float (&f)[3]) {
  const int ng = g.ng;
  const int64_t ng3 = (int64_t)ng * ng * ng;
  const float inv_one = __int_as_float((127 - g.fbits) << 23);  // 2^-F from its bit pattern
  float w1[3], w0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    w1[d] = (float)t[d] * inv_one;  // exact
    w0[d] = 1.0f - w1[d];           // exact
  }
  const int xs[2] = {c[0], wrap_inc(c[0], ng)};
  const int ys[2] = {c[1], wrap_inc(c[1], ng)};
  const int zs[2] = {c[2], wrap_inc(c[2], ng)};
  f[0] = f[1] = f[2] = 0.f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float wzy = (dz ? w1[2] : w0[2]) * (dy ? w1[1] : w0[1]);
      const int64_t row = ((int64_t)zs[dz] * ng + ys[dy]) * ng;
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = wzy * (dx ? w1[0] : w0[0]);
        const int64_t gi = row + xs[dx];
#pragma unroll
        for (int j = 0; j < 3; ++j) f[j] = fmaf(w, __ldg(fmesh + j * ng3 + gi), f[j]);
      }
    }
}

// With the gathered force f of particle p: (mode 0) Kick + Drift of eq. KDKALC, (mode 1) the
// final Kick + L+ of eq. Lops.
__device__ __forceinline__ void kick_drift_update(const Geometry& g, float* __restrict__ s, float* __restrict__ v,
                                                  const float* __restrict__ s1, const float* __restrict__ s2,
                                                  const float* __restrict__ coef, int mode, int64_t p,
                                                  const float (&f)[3]) {
  const int64_t n3 = g.np3;
  // explicit FMA chains: the same rounding in every kernel this body is inlined into
  const float cKF = __ldg(coef + kCKF), cK1 = __ldg(coef + kCK1), cK2 = __ldg(coef + kCK2);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float a1 = s1[j * n3 + p], a2 = s2[j * n3 + p];
    float vj = v[j * n3 + p];
    vj = __fadd_rn(vj, fmaf(cKF, f[j], fmaf(-cK1, a1, __fmul_rn(-cK2, a2))));  // Kick (eq. KDKALC)
    if (mode == 0) {
      const float dj = fmaf(__ldg(coef + kCD), vj, fmaf(__ldg(coef + kDD1), a1, __fmul_rn(__ldg(coef + kDD2), a2)));
      s[j * n3 + p] = __fadd_rn(s[j * n3 + p], dj);  // Drift
    } else {
      vj = __fadd_rn(vj, fmaf(__ldg(coef + kTD1), a1, __fmul_rn(__ldg(coef + kTD2), a2)));  // L+ (eq. Lops)
    }
    v[j * n3 + p] = vj;
  }
}

// Gather at particle p (lattice order, its cells from s), then the kick/drift of `mode` (0, 1)
// or (mode 2) the gathered force alone into gout [3][np^3].
__device__ __forceinline__ void gather_kick_drift_body(const Geometry& g, const float* __restrict__ fmesh,
                                                       float* __restrict__ s, float* __restrict__ v,
                                                       const float* __restrict__ s1, const float* __restrict__ s2,
                                                       const float* __restrict__ coef, int mode,
                                                       float* __restrict__ gout, int64_t p) {
  int ix, iy, iz;
  lattice_index(g, p, ix, iy, iz);
  int c[3], t[3];
  fixed_axis(g, ix, s[p], c[0], t[0]);
  fixed_axis(g, iy, s[g.np3 + p], c[1], t[1]);
  fixed_axis(g, iz, s[2 * g.np3 + p], c[2], t[2]);
  float f[3];
  gather_force(g, fmesh, c, t, f);
  if (mode == 2) {
#pragma unroll
    for (int j = 0; j < 3; ++j) gout[j * g.np3 + p] = f[j];
    return;
  }
  kick_drift_update(g, s, v, s1, s2, coef, mode, p, f);
}

}  // namespace cola
