// Shell-averaged power spectrum (Sec. 3.1) and small layout utilities.
//
// Shell b of integer m = |n|^2 is the b with b(b-1) < m <= b(b+1), i.e.
// (b - 1/2) k_F <= |k| < (b + 1/2) k_F, decided in integers.  Over the r2c half spectrum the
// planes n_x = 0 and n_x = ng/2 count once, the others twice.
#include "cola_internal.cuh"

namespace cola {

constexpr int kPowerChunks = 4;  // chunks of 32 modes whose loads a warp issues together

__device__ __forceinline__ int shell_of(int m) {
  int r = (int)sqrtf((float)m);
  while ((r + 1) * (r + 1) <= m) ++r;
  while (r * r > m) --r;
  return m <= r * (r + 1) ? r : r + 1;
}

__device__ __forceinline__ float sinc_pi_p(int n, int ng) {
  if (n == 0) return 1.0f;
  const float x = (float)n / (float)ng;
  return sinpif(x) / (3.14159265358979323846f * x);
}

// Power-spectrum binning.  A warp takes 32 consecutive k_x of one (k_y, k_z) row; lanes in
// the same shell are contiguous, so a segmented shuffle reduction (float32, at most 31 adds)
// leaves each shell's sum in its first lane, which adds it in float64 to the warp's own
// shared-memory accumulators (no atomics).  Each block then writes its per-shell totals in a
// fixed order and the finish kernel adds the blocks in block order: the result is
// deterministic.  NF = 1: one field, partial layout [block][shell][3] = (sum w |k|, sum w P,
// sum w); NF = 2: two fields a, b, [block][shell][5] = (sum w |k|, sum w P_a, sum w P_b,
// sum w P_ab, sum w) with P_ab from Re(a b^*).  One launch bins the shells b0 .. b1 - 1 of the
// nbins (the accumulators of a range of shells per warp leave room for more warps than those of
// all shells); chunks of modes outside the range are skipped.
template <int NF>
__global__ void k_power_bin(int ng, int P, float kf, float pnorm, int nbins, int b0, int b1,
                            const float2* __restrict__ dk, const float2* __restrict__ dk2,
                            double* __restrict__ partial) {
  constexpr int NQ = NF == 1 ? 3 : 5;
  static_assert(NQ <= kPowerQuantities, "partial sums beyond the sized buffers");
  extern __shared__ double pacc[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nh = ng / 2 + 1;
  // 1 / W_x^2 = sinc^-4 of every k_x, once per block (after the accumulators)
  const int nb = b1 - b0;
  float* inv_wx2 = reinterpret_cast<float*>(pacc + (size_t)nwarps * nb * NQ);
  for (int i = threadIdx.x; i < nwarps * nb * NQ; i += blockDim.x) pacc[i] = 0.0;
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    const float sx = sinc_pi_p(i, ng), wx = sx * sx;
    inv_wx2[i] = 1.0f / (wx * wx);
  }
  __syncthreads();
  double* mine = pacc + (size_t)warp * nb * NQ;
  // the shells of the range hold the modes with lo_m < |n|^2 <= hi_m
  const int lo_m = b0 * (b0 + 1), hi_m = b1 * (b1 + 1);
  const int64_t nrows = (int64_t)ng * ng;
  for (int64_t row = (int64_t)blockIdx.x * nwarps + warp; row < nrows; row += (int64_t)gridDim.x * nwarps) {
    const int ky = (int)(row % ng), kz = (int)(row / ng);
    const int ny = ky < ng / 2 ? ky : ky - ng, nz = kz < ng / 2 ? kz : kz - ng;
    const int myz = ny * ny + nz * nz;
    // rows and chunks with no mode of the range's shells are skipped (warp-uniform)
    const int lim = hi_m - myz;
    if (lim < 0) continue;
    // the first chunk group with a mode above lo_m: c^2 > lo_m - myz for some c in the group
    int gstart = 0;
    if (lo_m - myz > 0) {
      int c = (int)sqrtf((float)(lo_m - myz));
      while (c > 0 && c * c > lo_m - myz) --c;
      gstart = (c / (32 * kPowerChunks)) * (32 * kPowerChunks);
    }
    const float sy = sinc_pi_p(ny, ng), sz = sinc_pi_p(nz, ng);
    const float wyz = (sy * sy) * (sz * sz);
    const float row_scale = pnorm / (wyz * wyz);
    const float2* rowp = dk + row * P;
    const float2* rowq = NF == 2 ? dk2 + row * P : nullptr;
    // chunks of 32 k_x in groups of kPowerChunks whose loads are all issued first
    for (int g0 = gstart; g0 < nh && g0 * g0 <= lim; g0 += 32 * kPowerChunks) {
      float2 dv[kPowerChunks], ev[kPowerChunks];
#pragma unroll
      for (int u = 0; u < kPowerChunks; ++u) {
        const int kx = g0 + 32 * u + lane;
        dv[u] = kx < nh ? rowp[kx] : make_float2(0.f, 0.f);
        if constexpr (NF == 2) ev[u] = kx < nh ? rowq[kx] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kPowerChunks; ++u) {
        const int c0 = g0 + 32 * u;
        if (c0 >= nh || c0 * c0 > lim) break;  // warp-uniform
        const int kx = c0 + lane;
        int b = -1;
        float q[NQ];
#pragma unroll
        for (int j = 0; j < NQ; ++j) q[j] = 0.f;
        if (kx < nh) {
          const int m = kx * kx + myz;
          const int sb = shell_of(m);
          if (sb - 1 >= b0 && sb - 1 < b1) {
            b = sb - 1 - b0;
            const float w = (kx == 0 || kx == ng / 2) ? 1.f : 2.f;
            const float2 d = dv[u];
            const float scale = w * (row_scale * inv_wx2[kx]);  // w P-normalisation / W(k)^2
            q[0] = w * kf * sqrtf((float)m);
            q[1] = (d.x * d.x + d.y * d.y) * scale;
            if constexpr (NF == 2) {
              const float2 e = ev[u];
              q[2] = (e.x * e.x + e.y * e.y) * scale;
              q[3] = (d.x * e.x + d.y * e.y) * scale;
            }
            q[NQ - 1] = w;
          }
        }
        // segmented reduction toward the first lane of each run of equal shells
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int bo = __shfl_down_sync(0xffffffffu, b, o);
          float qo[NQ];
#pragma unroll
          for (int j = 0; j < NQ; ++j) qo[j] = __shfl_down_sync(0xffffffffu, q[j], o);
          if (lane + o < 32 && bo == b) {
#pragma unroll
            for (int j = 0; j < NQ; ++j) q[j] += qo[j];
          }
        }
        const int bprev = __shfl_up_sync(0xffffffffu, b, 1);
        if (b >= 0 && (lane == 0 || bprev != b)) {
#pragma unroll
          for (int j = 0; j < NQ; ++j) mine[NQ * b + j] += (double)q[j];
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb * NQ; i += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += pacc[(size_t)wv * nb * NQ + i];
    partial[((size_t)blockIdx.x * nbins + b0) * NQ + i] = t;
  }
}

__global__ void k_power_finish(int nbins, int nblocks, const double* __restrict__ partial, double* __restrict__ k,
                               double* __restrict__ pk, int64_t* __restrict__ nmodes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  double ks = 0.0, ps = 0.0, cs = 0.0;
  for (int blk = 0; blk < nblocks; ++blk) {
    const double* r = partial + ((size_t)blk * nbins + b) * 3;
    ks += r[0];
    ps += r[1];
    cs += r[2];
  }
  k[b] = cs > 0 ? ks / cs : 0.0;
  pk[b] = cs > 0 ? ps / cs : 0.0;
  nmodes[b] = (int64_t)cs;
}

// shell means of the two spectra and the cross term, rho = P_ab / sqrt(P_a P_b) (Sec. 3.1) and
// n_max = (2/3) rho / sqrt(1 - rho^2) (eq. nmax)
__global__ void k_cross_finish(int nbins, int nblocks, const double* __restrict__ partial, double* __restrict__ k,
                               double* __restrict__ pa, double* __restrict__ pb, double* __restrict__ pab,
                               double* __restrict__ rho, double* __restrict__ nmax, int64_t* __restrict__ nmodes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int blk = 0; blk < nblocks; ++blk) {
    const double* r = partial + ((size_t)blk * nbins + b) * 5;
#pragma unroll
    for (int j = 0; j < 5; ++j) s[j] += r[j];
  }
  const double cs = s[4];
  const double ma = cs > 0 ? s[1] / cs : 0.0, mb = cs > 0 ? s[2] / cs : 0.0, mab = cs > 0 ? s[3] / cs : 0.0;
  const double r = mab / sqrt(ma * mb);
  k[b] = cs > 0 ? s[0] / cs : 0.0;
  pa[b] = ma;
  pb[b] = mb;
  pab[b] = mab;
  rho[b] = r;
  nmax[b] = (2.0 / 3.0) * r / sqrt(1.0 - r * r);
  nmodes[b] = (int64_t)cs;
}

__global__ void k_unpad(int n, int P, const float2* __restrict__ in, float2* __restrict__ out) {
  const int nh = n / 2 + 1;
  const int64_t total = (int64_t)n * n * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nh;
    out[i] = in[r * P + (i - r * nh)];
  }
}

// 8 warps per block: the shells in one launch if their per-warp float64 accumulators still let
// two blocks share an SM (at most 110 KB a block), else in equal ranges whose accumulators let
// three (at most 64 KB)
constexpr int kPowerWarps = 8;
static int power_range(int nbins, int nq) {
  const size_t per_shell = (size_t)kPowerWarps * nq * sizeof(double);
  const int two = (int)((110 * 1024) / per_shell), three = (int)((64 * 1024) / per_shell);
  if (nbins <= two) return nbins;
  const int launches = (nbins + three - 1) / three;
  return (nbins + launches - 1) / launches;
}

int power_partial_doubles(int nbins) { return kPowerBlocks * nbins * kPowerQuantities; }

template <int NF>
static int power_bin_t(int ng, int P, double box, int nbins, const float2* dk, const float2* dk2, double* partial,
                       cudaStream_t st) {
  constexpr int NQ = NF == 1 ? 3 : 5;
  static_assert(NQ <= kPowerQuantities, "partial sums beyond the sized buffers");
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const double ng6 = std::pow((double)ng, 6.0);
  const float pnorm = (float)(box * box * box / ng6);
  const int range = power_range(nbins, NQ);
  const size_t smem = (size_t)kPowerWarps * range * NQ * sizeof(double) + sizeof(float) * (ng / 2 + 1);
  if (smem > 227 * 1024) return fail(COLA_EUNSUPPORTED, "power spectrum: mesh too large for shared memory");
  if (smem > 32 * 1024)
    COLA_CUDA_CHECK(cudaFuncSetAttribute(k_power_bin<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int b0 = 0; b0 < nbins; b0 += range) {
    const int b1 = std::min(nbins, b0 + range);
    {
      LaunchScope ls_(NF == 1 ? "power_bin" : "cross_bin", st);
      k_power_bin<NF><<<kPowerBlocks, 32 * kPowerWarps, smem, st>>>(ng, P, kf, pnorm, nbins, b0, b1, dk, dk2,
                                                                      partial);
    }
    COLA_LAUNCH_CHECK();
  }
  return COLA_OK;
}

int launch_power_bin(int ng, int P, double box, int nbins, const float2* dk, double* partial, cudaStream_t st) {
  return power_bin_t<1>(ng, P, box, nbins, dk, nullptr, partial, st);
}

int launch_cross_bin(int ng, int P, double box, int nbins, const float2* da, const float2* db, double* partial,
                     cudaStream_t st) {
  return power_bin_t<2>(ng, P, box, nbins, da, db, partial, st);
}

int launch_cross_finish(int nbins, const double* partial, double* k, double* pa, double* pb, double* pab, double* rho,
                        double* nmax, int64_t* nmodes, cudaStream_t st) {
  {
    LaunchScope ls_("cross_finish", st);
    k_cross_finish<<<(nbins + 127) / 128, 128, 0, st>>>(nbins, kPowerBlocks, partial, k, pa, pb, pab, rho, nmax,
                                                         nmodes);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_power_finish(int nbins, const double* partial, double* k, double* pk, int64_t* nmodes, cudaStream_t st) {
  {
    LaunchScope ls_("power_finish", st);
    k_power_finish<<<(nbins + 127) / 128, 128, 0, st>>>(nbins, kPowerBlocks, partial, k, pk, nmodes);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_unpad(int n, int P, const float2* in, float2* out, cudaStream_t st) {
  const int64_t total = (int64_t)n * n * (n / 2 + 1);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  { LaunchScope ls_("unpad", st);
  k_unpad<<<blocks, 256, 0, st>>>(n, P, in, out); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

}  // namespace cola
