// Shell-averaged power spectrum (Sec. 3.1) and small layout utilities.
//
// Shell b of integer m = |n|^2 is the b with b(b-1) < m <= b(b+1), i.e.
// (b - 1/2) k_F <= |k| < (b + 1/2) k_F, decided in integers.  Over the r2c half spectrum the
// planes n_x = 0 and n_x = ng/2 count once, the others twice.
#include "cola_internal.cuh"

namespace cola {

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
// fixed order and k_power_finish adds the blocks in block order: the result is deterministic.
// partial layout: [block][shell][3] = (sum w |k|, sum w P, sum w).
__global__ void k_power_bin(int ng, int P, float kf, float pnorm, int nbins, const float2* __restrict__ dk,
                            double* __restrict__ partial) {
  extern __shared__ double pacc[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nh = ng / 2 + 1;
  for (int i = threadIdx.x; i < nwarps * nbins * 3; i += blockDim.x) pacc[i] = 0.0;
  __syncthreads();
  double* mine = pacc + (size_t)warp * nbins * 3;
  const int64_t nrows = (int64_t)ng * ng;
  for (int64_t row = (int64_t)blockIdx.x * nwarps + warp; row < nrows; row += (int64_t)gridDim.x * nwarps) {
    const int ky = (int)(row % ng), kz = (int)(row / ng);
    const int ny = ky < ng / 2 ? ky : ky - ng, nz = kz < ng / 2 ? kz : kz - ng;
    const int myz = ny * ny + nz * nz;
    const float sy = sinc_pi_p(ny, ng), sz = sinc_pi_p(nz, ng);
    const float wyz = (sy * sy) * (sz * sz);
    const float2* rowp = dk + row * P;
    for (int c0 = 0; c0 < nh; c0 += 32) {
      const int kx = c0 + lane;
      int b = -1;
      float kw = 0.f, pw = 0.f, w = 0.f;
      if (kx < nh) {
        const int m = kx * kx + myz;
        const int sb = shell_of(m);
        if (sb >= 1 && sb <= nbins) {
          b = sb - 1;
          w = (kx == 0 || kx == ng / 2) ? 1.f : 2.f;
          const float2 d = rowp[kx];
          const float sx = sinc_pi_p(kx, ng);
          const float win = (sx * sx) * wyz;
          kw = w * kf * sqrtf((float)m);
          pw = w * (d.x * d.x + d.y * d.y) * pnorm / (win * win);
        }
      }
      // segmented reduction toward the first lane of each run of equal shells
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int bo = __shfl_down_sync(0xffffffffu, b, o);
        const float ko = __shfl_down_sync(0xffffffffu, kw, o);
        const float po = __shfl_down_sync(0xffffffffu, pw, o);
        const float wo = __shfl_down_sync(0xffffffffu, w, o);
        if (lane + o < 32 && bo == b) {
          kw += ko;
          pw += po;
          w += wo;
        }
      }
      const int bprev = __shfl_up_sync(0xffffffffu, b, 1);
      if (b >= 0 && (lane == 0 || bprev != b)) {
        mine[3 * b] += (double)kw;
        mine[3 * b + 1] += (double)pw;
        mine[3 * b + 2] += (double)w;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins * 3; i += blockDim.x) {
    double t = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) t += pacc[(size_t)wv * nbins * 3 + i];
    partial[(size_t)blockIdx.x * nbins * 3 + i] = t;
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

__global__ void k_unpad(int n, int P, const float2* __restrict__ in, float2* __restrict__ out) {
  const int nh = n / 2 + 1;
  const int64_t total = (int64_t)n * n * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nh;
    out[i] = in[r * P + (i - r * nh)];
  }
}

static int power_warps(int nbins) {
  const int w = (int)((160 * 1024) / ((size_t)nbins * 3 * sizeof(double)));
  return std::max(1, std::min(8, w));
}

int power_partial_doubles(int nbins) { return kPowerBlocks * nbins * 3; }

int launch_power_bin(int ng, int P, double box, int nbins, const float2* dk, double* partial, cudaStream_t st) {
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const double ng6 = std::pow((double)ng, 6.0);
  const float pnorm = (float)(box * box * box / ng6);
  const int warps = power_warps(nbins);
  const size_t smem = (size_t)warps * nbins * 3 * sizeof(double);
  if (smem > 32 * 1024)
    COLA_CUDA_CHECK(cudaFuncSetAttribute(k_power_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    LaunchScope ls_("power_bin", st);
    k_power_bin<<<kPowerBlocks, 32 * warps, smem, st>>>(ng, P, kf, pnorm, nbins, dk, partial);
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
