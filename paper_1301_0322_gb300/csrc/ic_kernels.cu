// Initial-condition kernels: Philox white noise, the linear density filter and the 2LPT
// derivative fields of App. A.3 (s1 = i k delta_k / k^2, mu2, s2 = D2u(1) (-i k mu2_k / k^2)).
#include "cola_internal.cuh"

namespace cola {

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) ------------------------------------
__device__ __forceinline__ void philox_round(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
  const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
  const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
  const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c, k0, k1);
  }
}

// Cell m of the lattice uses counter block g = m >> 2 (counter = (g lo, g hi, 0, 0),
// key = (seed lo, seed hi)); uniforms u = ((r >> 8) + 1) 2^-24; Box-Muller pairs (r0, r1) ->
// cells 4g, 4g+1 (cos, sin) and (r2, r3) -> cells 4g+2, 4g+3.
__global__ void k_noise(int64_t n3, uint32_t key0, uint32_t key1, float* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 4 >= n3) return;
  uint32_t c[4] = {(uint32_t)(g & 0xFFFFFFFFll), (uint32_t)(g >> 32), 0u, 0u};
  philox4x32_10(c, key0, key1);
  float z[4];
#pragma unroll
  for (int pair = 0; pair < 2; ++pair) {
    const float ua = (float)((c[2 * pair] >> 8) + 1u) * 5.9604644775390625e-8f;  // 2^-24, exact
    const float ub = (float)((c[2 * pair + 1] >> 8) + 1u) * 5.9604644775390625e-8f;
    const float rho = sqrtf(-2.0f * logf(ua));
    float sn, cs;
    sincospif(2.0f * ub, &sn, &cs);
    z[2 * pair] = rho * cs;
    z[2 * pair + 1] = rho * sn;
  }
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (g * 4 + l < n3) out[g * 4 + l] = z[l];
}

// ---- Fourier-space helpers ----------------------------------------------------------------------
struct Mode {
  int nx, ny, nz;
  int64_t off;  // index in the padded half spectrum
};

__device__ __forceinline__ Mode mode_of(int64_t i, int n, int P) {
  const int nh = n / 2 + 1;
  Mode m;
  const int kx = (int)(i % nh);
  const int64_t r = i / nh;
  const int ky = (int)(r % n), kz = (int)(r / n);
  m.nx = kx;
  m.ny = ky < n / 2 ? ky : ky - n;
  m.nz = kz < n / 2 ? kz : kz - n;
  m.off = r * P + kx;
  return m;
}

// delta_k = w_k sqrt(P(k) n^3 / L^3), P = A k^ns T_BBKS(k)^2, k = 0 removed.
__global__ void k_ic_filter(int n, int P, float kf, float amp_scale, float n_s, float gamma, float2* __restrict__ wk) {
  const int64_t total = (int64_t)n * n * (n / 2 + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const Mode m = mode_of(i, n, P);
    const int m2 = m.nx * m.nx + m.ny * m.ny + m.nz * m.nz;
    float f = 0.0f;
    if (m2 != 0) {
      const float k = kf * sqrtf((float)m2);
      const float q = k / gamma;
      const float x = 2.34f * q;
      const float lead = log1pf(x) / x;
      const float poly = 1.0f + 3.89f * q + (16.1f * q) * (16.1f * q) + (5.46f * q) * (5.46f * q) * (5.46f * q) +
                         (6.71f * q) * (6.71f * q) * (6.71f * q) * (6.71f * q);
      const float tk = lead * rsqrtf(sqrtf(poly));  // poly^(-1/4)
      f = amp_scale * expf(0.5f * n_s * logf(k)) * tk;  // sqrt(A n^3/L^3) k^(ns/2) T(k)
    }
    const float2 w = wk[m.off];
    wk[m.off] = make_float2(w.x * f, w.y * f);
  }
}

// First derivative factor i k_j, zero on the Nyquist plane |n_j| = n/2.
__device__ __forceinline__ float kcomp(const Mode& m, int j, int n, float kf) {
  const int c = j == 0 ? m.nx : (j == 1 ? m.ny : m.nz);
  return (c == n / 2 || c == -n / 2) ? 0.0f : kf * (float)c;
}

// kind 0: out = scale * (i k_i) / k^2 * in                (s1_i; with scale < 0: s2 from mu2)
// kind 1: out = scale * (i k_i)(i k_j) / k^2 * in         (psi1_{i,j})
__global__ void k_kmul(int n, int P, float kf, int kind, int i_, int j_, float scale, const float2* __restrict__ in,
                       float2* __restrict__ out) {
  const int64_t total = (int64_t)n * n * (n / 2 + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const Mode m = mode_of(i, n, P);
    const int m2 = m.nx * m.nx + m.ny * m.ny + m.nz * m.nz;
    float2 r = make_float2(0.f, 0.f);
    if (m2 != 0) {
      const float inv_k2 = scale / (kf * kf * (float)m2);
      const float2 a = in[m.off];
      const float ki = kcomp(m, i_, n, kf);
      if (kind == 0) {  // i ki a / k^2
        r = make_float2(-ki * a.y * inv_k2, ki * a.x * inv_k2);
      } else {  // -ki kj a / k^2
        const float kk = -ki * kcomp(m, j_, n, kf) * inv_k2;
        r = make_float2(kk * a.x, kk * a.y);
      }
    }
    out[m.off] = r;
  }
}

// acc = fxx fyy + fxx fzz + fyy fzz  (diagonal part of mu2)
__global__ void k_source_diag(int64_t n3, const float* __restrict__ fxx, const float* __restrict__ fyy,
                              const float* __restrict__ fzz, float* __restrict__ acc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = fxx[i], b = fyy[i], c = fzz[i];
    acc[i] = a * b + a * c + b * c;
  }
}

// acc -= f^2  (off-diagonal part of mu2)
__global__ void k_source_sub_sq(int64_t n3, const float* __restrict__ f, float* __restrict__ acc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = f[i];
    acc[i] = fmaf(-x, x, acc[i]);
  }
}

// s = D1 s1 + D2 s2, v = 0 (2LPT position at a_init; velocity after L-).
__global__ void k_ic_assemble(int64_t m, float d1, float d2, float t1, float t2, const float* __restrict__ s1,
                              const float* __restrict__ s2, float* __restrict__ s, float* __restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = s1[i], b = s2[i];
    s[i] = fmaf(d1, a, d2 * b);
    v[i] = fmaf(t1, a, t2 * b);
  }
}

static unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)std::min<int64_t>(b, 152 * 32);
}

int launch_noise(int np, uint64_t seed, float* out, cudaStream_t st) {
  const int64_t n3 = (int64_t)np * np * np;
  const int64_t groups = (n3 + 3) / 4;
  {
    LaunchScope ls_("noise", st);
    k_noise<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(n3, (uint32_t)(seed & 0xFFFFFFFFull),
                                                              (uint32_t)(seed >> 32), out);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_ic_filter(int np, int P, double box, double amp, double n_s, double omega_m, double h, float2* wk,
                     cudaStream_t st) {
  const double n3 = (double)np * np * np;
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const float amp_scale = (float)std::sqrt(amp * n3 / (box * box * box));
  const int64_t total = (int64_t)np * np * (np / 2 + 1);
  { LaunchScope ls_("ic_filter", st);
  k_ic_filter<<<grid_for(total), 256, 0, st>>>(np, P, kf, amp_scale, (float)n_s, (float)(omega_m * h), wk); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_kmul(int n, int P, double box, int kind, int i, int j, float scale, const float2* in, float2* out,
                cudaStream_t st) {
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const int64_t total = (int64_t)n * n * (n / 2 + 1);
  { LaunchScope ls_("kmul", st);
  k_kmul<<<grid_for(total), 256, 0, st>>>(n, P, kf, kind, i, j, scale, in, out); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_source_2lpt(int64_t n3, const float* fxx, const float* fyy, const float* fzz, float* out_acc,
                       cudaStream_t st) {
  { LaunchScope ls_("source_diag", st);
  k_source_diag<<<grid_for(n3), 256, 0, st>>>(n3, fxx, fyy, fzz, out_acc); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_source_sub_sq(int64_t n3, const float* f, float* acc, cudaStream_t st) {
  { LaunchScope ls_("source_sub_sq", st);
  k_source_sub_sq<<<grid_for(n3), 256, 0, st>>>(n3, f, acc); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_ic_assemble(int64_t n3, float d1, float d2, float t1, float t2, const float* s1, const float* s2,
                       float* s, float* v, cudaStream_t st) {
  { LaunchScope ls_("ic_assemble", st);
  k_ic_assemble<<<grid_for(3 * n3), 256, 0, st>>>(3 * n3, d1, d2, t1, t2, s1, s2, s, v); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

}  // namespace cola
