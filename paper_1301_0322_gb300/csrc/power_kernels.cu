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

// acc[2 b] += sum w |k|, acc[2 b + 1] += sum w P(k), cnt[b] += sum w, for shells b = 1..nbins
// (stored at b - 1).  Lanes of a warp that share a shell are summed by their leader in lane
// order, so each warp issues one float64 atomic per distinct shell.
__global__ void k_power_bin(int ng, int P, float kf, float pnorm, int nbins, const float2* __restrict__ dk,
                            double* __restrict__ acc, unsigned long long* __restrict__ cnt) {
  const int nh = ng / 2 + 1;
  const int64_t total = (int64_t)ng * ng * nh;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int b = -1;
    float kw = 0.f, pw = 0.f;
    int w = 0;
    if (i < total) {
      const int kx = (int)(i % nh);
      const int64_t r = i / nh;
      const int ky = (int)(r % ng), kz = (int)(r / ng);
      const int nx = kx, ny = ky < ng / 2 ? ky : ky - ng, nz = kz < ng / 2 ? kz : kz - ng;
      const int m = nx * nx + ny * ny + nz * nz;
      const int sb = shell_of(m);
      if (sb >= 1 && sb <= nbins) {
        b = sb - 1;
        w = (nx == 0 || nx == ng / 2) ? 1 : 2;
        const float2 d = dk[r * P + kx];
        const float sx = sinc_pi_p(nx, ng), sy = sinc_pi_p(ny, ng), sz = sinc_pi_p(nz, ng);
        const float win = (sx * sx) * (sy * sy) * (sz * sz);
        const float p = (d.x * d.x + d.y * d.y) * pnorm / (win * win);
        kw = w * kf * sqrtf((float)m);
        pw = w * p;
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    double ks = 0.0, ps = 0.0;
    unsigned long long cs = 0;
    for (int l = 0; l < 32; ++l) {
      const float kl = __shfl_sync(0xffffffffu, kw, l);
      const float pl = __shfl_sync(0xffffffffu, pw, l);
      const int wl = __shfl_sync(0xffffffffu, w, l);
      if ((peers >> l) & 1u) {
        ks += (double)kl;
        ps += (double)pl;
        cs += (unsigned long long)wl;
      }
    }
    if (b >= 0 && lane == leader) {
      atomicAdd(&acc[2 * b], ks);
      atomicAdd(&acc[2 * b + 1], ps);
      atomicAdd(&cnt[b], cs);
    }
  }
}

__global__ void k_power_finish(int nbins, const double* __restrict__ acc, const unsigned long long* __restrict__ cnt,
                               double* __restrict__ k, double* __restrict__ pk, int64_t* __restrict__ nmodes) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const unsigned long long c = cnt[b];
  k[b] = c ? acc[2 * b] / (double)c : 0.0;
  pk[b] = c ? acc[2 * b + 1] / (double)c : 0.0;
  nmodes[b] = (int64_t)c;
}

__global__ void k_unpad(int n, int P, const float2* __restrict__ in, float2* __restrict__ out) {
  const int nh = n / 2 + 1;
  const int64_t total = (int64_t)n * n * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nh;
    out[i] = in[r * P + (i - r * nh)];
  }
}

int launch_power_bin(int ng, int P, double box, int nbins, const float2* dk, double* acc, unsigned long long* cnt,
                     cudaStream_t st) {
  COLA_CUDA_CHECK(cudaMemsetAsync(acc, 0, sizeof(double) * 2 * nbins, st));
  COLA_CUDA_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nbins, st));
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const double ng6 = std::pow((double)ng, 6.0);
  const float pnorm = (float)(box * box * box / ng6);
  const int64_t total = (int64_t)ng * ng * (ng / 2 + 1);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  { LaunchScope ls_("power_bin", st);
  k_power_bin<<<blocks, 256, 0, st>>>(ng, P, kf, pnorm, nbins, dk, acc, cnt); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_power_finish(int nbins, const double* acc, const unsigned long long* cnt, double* k, double* pk,
                        int64_t* nmodes, cudaStream_t st) {
  { LaunchScope ls_("power_finish", st);
  k_power_finish<<<(nbins + 127) / 128, 128, 0, st>>>(nbins, acc, cnt, k, pk, nmodes); }
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
