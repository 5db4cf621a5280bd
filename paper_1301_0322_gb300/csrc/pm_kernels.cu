// Particle-mesh kernels of a COLA force evaluation (Sec. 2 PM code; App. A.1 eq. eom;
// App. A.3 eq. KDKALC):
//   binning  : particles -> (y, z) row tiles of the mesh (counting sort, integer atomics)
//   deposit  : CIC mass of every particle touching a tile, int64 fixed point in shared memory
//              (integer sums: the result does not depend on the order of the atomics)
//   k-space  : g_j = i k_j delta_k / (k^2 W^p) / ng^3 (Nyquist plane of j and k = 0 set to 0)
//   gather   : CIC interpolation of g with the deposit's weights, fused with the COLA Kick and
//              Drift (or the final L+ of eq. Lops)
#include "cola_internal.cuh"
#include "pm_common.cuh"
#include "particle_bodies.cuh"

namespace cola {

// ---- binning -------------------------------------------------------------------------------
// four particles per thread (keys_x4_body)
__global__ void __launch_bounds__(256) k_keys_x4(Geometry g, Tiles tl, const float* __restrict__ s,
                                                 int* __restrict__ keys, int* __restrict__ counts,
                                                 int* __restrict__ err) {
  keys_x4_body(g, tl, s, (int64_t)blockIdx.x * blockDim.x * kPartPerThread, 0, keys, counts, err);
}

// Exclusive scan of the bin counts in three launches (block sums, scan of the block sums,
// per-block scan); resets the counts for the next use.  kScanTile bins per block.
constexpr int kScanTile = 1024;

// inclusive block scan of one int per thread (blockDim.x == 1024)
__device__ __forceinline__ int block_inclusive_scan(int x, int* warp_sums) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int ws = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    warp_sums[lane] = ws;
  }
  __syncthreads();
  return x + (wid > 0 ? warp_sums[wid - 1] : 0);
}

__global__ void __launch_bounds__(1024) k_scan_reduce(int n, const int* __restrict__ counts, int* __restrict__ block_sums) {
  __shared__ int warp_sums[32];
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  const int x = i < n ? counts[i] : 0;
  const int incl = block_inclusive_scan(x, warp_sums);
  if (threadIdx.x == kScanTile - 1) block_sums[blockIdx.x] = incl;
}

// exclusive scan of nb block sums in place (single block; nb <= 1024 * per)
__global__ void __launch_bounds__(1024) k_scan_blocks(int nb, int* __restrict__ block_sums) {
  __shared__ int warp_sums[32];
  const int per = (nb + 1023) / 1024;
  const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
  int local = 0;
  for (int b = b0; b < b1; ++b) local += block_sums[b];
  int run = block_inclusive_scan(local, warp_sums) - local;
  for (int b = b0; b < b1; ++b) {
    const int c = block_sums[b];
    block_sums[b] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(int n, int* __restrict__ counts, const int* __restrict__ block_sums,
                                                    int* __restrict__ offsets, int* __restrict__ cursor) {
  __shared__ int warp_sums[32];
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  const int x = i < n ? counts[i] : 0;
  const int excl = block_inclusive_scan(x, warp_sums) - x + block_sums[blockIdx.x];
  if (i < n) {
    offsets[i] = excl;
    cursor[i] = excl;
    counts[i] = 0;
  }
  if (i == n - 1) offsets[n] = excl + x;
}

// four particles per thread (scatter_x4_body)
__global__ void __launch_bounds__(256) k_scatter_x4(Geometry g, const float* __restrict__ s,
                                                    const int* __restrict__ keys, int* __restrict__ cursor,
                                                    uint4* __restrict__ rec) {
  scatter_x4_body(g, s, (int64_t)blockIdx.x * blockDim.x * kPartPerThread, keys, cursor, rec);
}

// ---- deposit ----------------------------------------------------------------------------------
// One block per tile of TY x TZ mesh rows (whole x extent).  It reads the bin-ordered records
// (fixed-point CIC coordinates, stored by the scatter) of the particles binned to the tile and to
// the boundary regions of its three lower neighbours, accumulates exact int64 CIC weights in
// shared memory and writes the rows once (int64 and/or float overdensity).
template <int TY, int TZ>
__global__ void __launch_bounds__(256) k_deposit(Geometry g, Tiles tl, const uint4* __restrict__ rec,
                                                 const int* __restrict__ offsets, int64_t* __restrict__ rho,
                                                 float* __restrict__ delta, float dscale, int* __restrict__ err) {
  extern __shared__ unsigned long long acc[];
  __shared__ int rbeg[9], rpre[10];
  const int ng = g.ng;
  int tyi, tzi;
  tile_of_bin(tl, blockIdx.x, tyi, tzi);
  const int y0 = tyi * TY, z0 = tzi * TZ;
  const int ncell = TZ * TY * ng;
  for (int i = threadIdx.x; i < ncell; i += blockDim.x) acc[i] = 0ull;
  if (threadIdx.x == 0) {
    const int tym = tyi == 0 ? tl.nty - 1 : tyi - 1;
    const int tzm = tzi == 0 ? tl.ntz - 1 : tzi - 1;
    const int tys[9] = {tyi, tyi, tyi, tyi, tym, tym, tyi, tyi, tym};
    const int tzs[9] = {tzi, tzi, tzi, tzi, tzi, tzi, tzm, tzm, tzm};
    const int reg[9] = {0, 1, 2, 3, 1, 3, 2, 3, 3};
    int run = 0;
    for (int k = 0; k < 9; ++k) {
      const int b = tile_bin(tl, tys[k], tzs[k]) * 4 + reg[k];
      rbeg[k] = offsets[b];
      rpre[k] = run;
      run += offsets[b + 1] - offsets[b];
    }
    rpre[9] = run;
  }
  __syncthreads();
  const int total = rpre[9];
  const unsigned long long one = 1ull << g.fbits;
  unsigned* lo = reinterpret_cast<unsigned*>(acc);
  unsigned* hi = lo + ncell;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    int r = 0;
#pragma unroll
    for (int k = 1; k < 9; ++k) r += (i >= rpre[k]) ? 1 : 0;
    const int64_t pos = rbeg[r] + (i - rpre[r]);
    const uint32_t fmask = (uint32_t)one - 1u;
    const uint4 q = __ldg(rec + pos);
    const uint32_t fx = q.x, fy = q.y, fz = q.z;
    const int cx = (int)(fx >> g.fbits), tx = (int)(fx & fmask);
    const int cy = (int)(fy >> g.fbits), ty = (int)(fy & fmask);
    const int cz = (int)(fz >> g.fbits), tz = (int)(fz & fmask);
    const int cx1 = wrap_inc(cx, ng);
    const unsigned long long wx0 = one - tx, wx1 = tx;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      const int z = dz ? wrap_inc(cz, ng) : cz;
      const int lz = z - z0;
      if (lz < 0 || lz >= TZ) continue;
      const unsigned long long wz = dz ? (unsigned long long)tz : one - tz;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int y = dy ? wrap_inc(cy, ng) : cy;
        const int ly = y - y0;
        if (ly < 0 || ly >= TY) continue;
        const unsigned long long wzy = wz * (dy ? (unsigned long long)ty : one - ty);
        const int row = (lz * TY + ly) * ng;
        acc_add64(lo, hi, row + cx, wzy * wx0);
        acc_add64(lo, hi, row + cx1, wzy * wx1);
      }
    }
  }
  __syncthreads();
  bool overflow = false;
  for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
    const int lz = i / (TY * ng), rem = i - lz * (TY * ng);
    const int ly = rem / ng, x = rem - ly * ng;
    const int64_t gi = ((int64_t)(z0 + lz) * ng + (y0 + ly)) * ng + x;
    const unsigned long long v = acc_value(lo, hi, i);
    overflow |= (v >> 62) != 0ull;
    if (rho) rho[gi] = (int64_t)v;
    if (delta) delta[gi] = fmaf(__ull2float_rn(v), dscale, -1.0f);
  }
  if (overflow) atomicOr(err, kErrOverflow);
}

// ---- k-space force --------------------------------------------------------------------------
__device__ __forceinline__ float sinc_pi(int n, int ng) {
  if (n == 0) return 1.0f;
  const float x = (float)n / (float)ng;
  return sinpif(x) / (3.14159265358979323846f * x);
}

__global__ void k_kspace_force(int ng, int P, float kf, int deconv, float norm, const float2* __restrict__ dk,
                               float2* __restrict__ gx, float2* __restrict__ gy, float2* __restrict__ gz) {
  const int nh = ng / 2 + 1;
  const int64_t total = (int64_t)ng * ng * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nh);
    const int64_t r = i / nh;
    const int ky = (int)(r % ng), kz = (int)(r / ng);
    const int nx = kx, ny = ky < ng / 2 ? ky : ky - ng, nz = kz < ng / 2 ? kz : kz - ng;
    const int64_t o = r * P + kx;
    const int m2 = nx * nx + ny * ny + nz * nz;
    float2 out[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (m2 != 0) {
      float green = norm / (kf * kf * (float)m2);
      if (deconv) {
        const float sx = sinc_pi(nx, ng), sy = sinc_pi(ny, ng), sz = sinc_pi(nz, ng);
        const float w = (sx * sx) * (sy * sy) * (sz * sz);
        green /= (deconv == 2 ? w * w : w);
      }
      const float2 d = dk[o];
      const float2 val = make_float2(d.x * green, d.y * green);
      const int half = ng / 2;
      const float kx_ = (nx == half) ? 0.f : kf * nx;
      const float ky_ = (ny == -half) ? 0.f : kf * ny;
      const float kz_ = (nz == -half) ? 0.f : kf * nz;
      // i k (a + i b) = k (-b + i a)
      out[0] = make_float2(-kx_ * val.y, kx_ * val.x);
      out[1] = make_float2(-ky_ * val.y, ky_ * val.x);
      out[2] = make_float2(-kz_ * val.y, kz_ * val.x);
    }
    gx[o] = out[0];
    gy[o] = out[1];
    gz[o] = out[2];
  }
}

// ---- gather + kick + drift -------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather_kick_drift(Geometry g, const float* __restrict__ fmesh,
                                                            float* __restrict__ s, float* __restrict__ v,
                                                            const float* __restrict__ s1, const float* __restrict__ s2,
                                                            const float* __restrict__ coef, int mode,
                                                            float* __restrict__ gout) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < g.np3) gather_kick_drift_body(g, fmesh, s, v, s1, s2, coef, mode, gout, p);
}

// Gather in bin order: thread i takes the particle of bin position i from its record (lattice
// index p and the fixed-point coordinates, which equal fixed_axis of the current s), so the
// threads of a block read neighbouring mesh rows however clustered the particles are; the
// force goes to fj[p].
__global__ void __launch_bounds__(256) k_gather_binned(Geometry g, const float* __restrict__ fmesh,
                                                        const uint4* __restrict__ rec, float* __restrict__ f0,
                                                        float* __restrict__ f1, float* __restrict__ f2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.np3) return;
  const uint4 q = __ldg(rec + i);
  const int64_t p = q.w;
  const uint32_t fmask = (1u << g.fbits) - 1u;
  const uint32_t fq[3] = {q.x, q.y, q.z};
  int c[3], t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c[d] = (int)(fq[d] >> g.fbits);
    t[d] = (int)(fq[d] & fmask);
  }
  float f[3];
  gather_force(g, fmesh, c, t, f);
  f0[p] = f[0];
  f1[p] = f[1];
  f2[p] = f[2];
}

// As k_gather_binned, with the three components written as one 16-byte float4 at the particle's
// lattice index: once the particles cluster, consecutive bin positions belong to scattered
// lattice indices, and one 16-byte write touches one 32-byte sector where three 4-byte writes
// to three arrays touch three.
__global__ void __launch_bounds__(256) k_gather_binned4(Geometry g, const float* __restrict__ fmesh,
                                                         const uint4* __restrict__ rec, float4* __restrict__ f4) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.np3) return;
  const uint4 q = __ldg(rec + i);
  const uint32_t fmask = (1u << g.fbits) - 1u;
  const uint32_t fq[3] = {q.x, q.y, q.z};
  int c[3], t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c[d] = (int)(fq[d] >> g.fbits);
    t[d] = (int)(fq[d] & fmask);
  }
  float f[3];
  gather_force(g, fmesh, c, t, f);
  f4[q.w] = make_float4(f[0], f[1], f[2], 0.0f);
}

// Kick/drift in lattice order with the forces of k_gather_binned4.
__global__ void __launch_bounds__(256) k_kick_drift4(Geometry g, const float4* __restrict__ f4,
                                                      float* __restrict__ s, float* __restrict__ v,
                                                      const float* __restrict__ s1, const float* __restrict__ s2,
                                                      const float* __restrict__ coef, int mode) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.np3) return;
  const float4 q = __ldg(f4 + p);
  const float f[3] = {q.x, q.y, q.z};
  kick_drift_update(g, s, v, s1, s2, coef, mode, p, f);
}

// Kick/drift in lattice order with the gathered force fj[p].
__global__ void __launch_bounds__(256) k_kick_drift(Geometry g, const float* __restrict__ f0,
                                                     const float* __restrict__ f1, const float* __restrict__ f2,
                                                     float* __restrict__ s, float* __restrict__ v,
                                                     const float* __restrict__ s1, const float* __restrict__ s2,
                                                     const float* __restrict__ coef, int mode) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.np3) return;
  const float f[3] = {f0[p], f1[p], f2[p]};
  kick_drift_update(g, s, v, s1, s2, coef, mode, p, f);
}

// ---- launchers ------------------------------------------------------------------------------------
static unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int launch_keys(const Geometry& g, const Tiles& t, const float* s, int* keys, int* counts, int* err, cudaStream_t st) {
  { LaunchScope ls_("keys", st);
  k_keys_x4<<<blocks_for(g.np3, 256 * kPartPerThread), 256, 0, st>>>(g, t, s, keys, counts, err); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int scan_block_count(const Tiles& t) { return (t.nbins + kScanTile - 1) / kScanTile; }

int launch_scan(const Tiles& t, int* counts, int* offsets, int* cursor, int* block_sums, cudaStream_t st) {
  const int nb = scan_block_count(t);
  {
    LaunchScope ls_("scan_reduce", st);
    k_scan_reduce<<<nb, kScanTile, 0, st>>>(t.nbins, counts, block_sums);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("scan_blocks", st);
    k_scan_blocks<<<1, 1024, 0, st>>>(nb, block_sums);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("scan_apply", st);
    k_scan_apply<<<nb, kScanTile, 0, st>>>(t.nbins, counts, block_sums, offsets, cursor);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_scatter(const Geometry& g, const float* s, const int* keys, int* cursor, uint4* rec,
                   cudaStream_t st) {
  { LaunchScope ls_("scatter", st);
  k_scatter_x4<<<blocks_for(g.np3, 256 * kPartPerThread), 256, 0, st>>>(g, s, keys, cursor, rec); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

template <int TY, int TZ>
static int deposit_t(const Geometry& g, const Tiles& t, const uint4* rec, const int* offsets, int64_t* rho,
                     float* delta, int* err, cudaStream_t st) {
  const size_t smem = (size_t)TY * TZ * g.ng * sizeof(unsigned long long);
  if (smem > 227 * 1024) return fail(COLA_EUNSUPPORTED, "deposit tile does not fit in shared memory");
  if (smem > 32 * 1024)
    COLA_CUDA_CHECK(cudaFuncSetAttribute(k_deposit<TY, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const double ng3 = (double)g.ng * g.ng * g.ng;
  const float dscale = (float)(ng3 / ((double)g.np3 * std::ldexp(1.0, 3 * g.fbits)));
  { LaunchScope ls_(TY == 2 ? "deposit_2x2" : (TZ == 2 ? "deposit_4x2" : "deposit_4x4"), st);
  k_deposit<TY, TZ><<<t.nty * t.ntz, 256, smem, st>>>(g, t, rec, offsets, rho, delta, dscale, err); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_deposit(const Geometry& g, const Tiles& t, const uint4* rec, const int* offsets, int64_t* rho,
                   float* delta, int* err, cudaStream_t st) {
  if (t.ty == 4 && t.tz == 4) return deposit_t<4, 4>(g, t, rec, offsets, rho, delta, err, st);
  if (t.ty == 4 && t.tz == 2) return deposit_t<4, 2>(g, t, rec, offsets, rho, delta, err, st);
  if (t.ty == 2 && t.tz == 2) return deposit_t<2, 2>(g, t, rec, offsets, rho, delta, err, st);
  return fail(COLA_EUNSUPPORTED, "deposit: unsupported tile shape");
}

int launch_kspace_force(int ng, int P, double box, int deconv, const float2* dk, float2* gx, float2* gy, float2* gz,
                        cudaStream_t st) {
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const float norm = (float)(1.0 / ((double)ng * ng * ng));
  const int64_t total = (int64_t)ng * ng * (ng / 2 + 1);
  const unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(total, 256), 152 * 64);
  { LaunchScope ls_("kspace_force", st);
  k_kspace_force<<<blocks, 256, 0, st>>>(ng, P, kf, deconv, norm, dk, gx, gy, gz); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_gather_kick_drift(const Geometry& g, const float* fmesh, float* s, float* v, const float* s1,
                             const float* s2, const float* coef_row, int mode, float* gout, cudaStream_t st) {
  { LaunchScope ls_("gather_kick_drift", st);
  k_gather_kick_drift<<<blocks_for(g.np3, 256), 256, 0, st>>>(g, fmesh, s, v, s1, s2, coef_row, mode, gout); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_gather_binned(const Geometry& g, const float* fmesh, const uint4* rec,
                         float* f0, float* f1, float* f2, cudaStream_t st) {
  { LaunchScope ls_("gather_binned", st);
  k_gather_binned<<<blocks_for(g.np3, 256), 256, 0, st>>>(g, fmesh, rec, f0, f1, f2); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_gather_binned4(const Geometry& g, const float* fmesh, const uint4* rec, float4* f4, cudaStream_t st) {
  { LaunchScope ls_("gather_binned4", st);
  k_gather_binned4<<<blocks_for(g.np3, 256), 256, 0, st>>>(g, fmesh, rec, f4); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_kick_drift4(const Geometry& g, const float4* f4, float* s, float* v, const float* s1, const float* s2,
                       const float* coef_row, int mode, cudaStream_t st) {
  { LaunchScope ls_("kick_drift4", st);
  k_kick_drift4<<<blocks_for(g.np3, 256), 256, 0, st>>>(g, f4, s, v, s1, s2, coef_row, mode); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_kick_drift(const Geometry& g, const float* f0, const float* f1, const float* f2, float* s, float* v,
                      const float* s1, const float* s2, const float* coef_row, int mode, cudaStream_t st) {
  { LaunchScope ls_("kick_drift", st);
  k_kick_drift<<<blocks_for(g.np3, 256), 256, 0, st>>>(g, f0, f1, f2, s, v, s1, s2, coef_row, mode); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

}  // namespace cola
