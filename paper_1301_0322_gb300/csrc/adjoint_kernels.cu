// Reverse-mode (adjoint) kernels: the transpose of one force evaluation of eq. ALCtimestep, of
// the CIC density and of the 2LPT initial conditions.  The paper has no derivatives; these are
// the exact transposes of the forward kernels (the CIC weights' gradient is taken almost
// everywhere, at the same quantised positions the forward path uses).
//
// One force evaluation maps (s, v) -> (s', v') with g the unit PM force at s:
//   v1 = v + cKF g(s) - cK1 s1 - cK2 s2;  s' = s + cD v1 + dD1 s1 + dD2 s2, v' = v1   (steps < n)
//   v' = v1 + TD1 s1 + TD2 s2, s' = s                                                  (step n, L+)
// so, given the adjoints (lam_s, lam_v) of (s', v'):
//   lam_v1 = lam_v + cD lam_s (or lam_v),  lam_s1 += dD1 lam_s - cK1 lam_v1 (or (TD1 - cK1) lam_v),
//   lam_s2 likewise,  lam_s <- lam_s + cKF (dg/ds)^T lam_v1,  lam_v <- lam_v1.
// (dg/ds)^T lam = (N/L) [ sum_i lam_i sum_c dW F_i(c) + (1/rho_bar) sum_c dW Phi(c) ],
// Phi = sum_i IFFT(conj(m_i) FFT(Lam_i)) / N^3, Lam_i = CIC deposit of lam_i, m_i = i k_i/(k^2 W^p).
#include "cola_internal.cuh"
#include "pm_common.cuh"

namespace cola {

__device__ __forceinline__ float sinc_pi_a(int n, int ng) {
  if (n == 0) return 1.0f;
  const float x = (float)n / (float)ng;
  return sinpif(x) / (3.14159265358979323846f * x);
}

// adjoint of the Kick/Drift/L+ algebra (before the force VJP), elementwise over particles
__global__ void k_adjoint_pre(int64_t n3, int mode, const float* __restrict__ coef, float* __restrict__ lam_s,
                              float* __restrict__ lam_v, float* __restrict__ lam_s1, float* __restrict__ lam_s2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n3) return;
  const float cK1 = __ldg(coef + kCK1), cK2 = __ldg(coef + kCK2);
  const float ls = lam_s[i];
  float lv = lam_v[i];
  if (mode == 0) {
    lv += __ldg(coef + kCD) * ls;
    lam_s1[i] += __ldg(coef + kDD1) * ls - cK1 * lv;
    lam_s2[i] += __ldg(coef + kDD2) * ls - cK2 * lv;
    lam_v[i] = lv;
  } else {
    lam_s1[i] += (__ldg(coef + kTD1) - cK1) * lv;
    lam_s2[i] += (__ldg(coef + kTD2) - cK2) * lv;
  }
}

// Lam_i(c) = sum_p W(u_p - c) lam_p,i  (float atomics; the summation order is not fixed)
__global__ void k_lambda_deposit(Geometry g, const float* __restrict__ s, const float* __restrict__ lam,
                                 float* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.np3) return;
  const int ng = g.ng;
  const int64_t ng3 = (int64_t)ng * ng * ng, n3 = g.np3;
  int ix, iy, iz;
  lattice_index(g, p, ix, iy, iz);
  int c[3], t[3];
  fixed_axis(g, ix, s[p], c[0], t[0]);
  fixed_axis(g, iy, s[n3 + p], c[1], t[1]);
  fixed_axis(g, iz, s[2 * n3 + p], c[2], t[2]);
  const float inv_one = __int_as_float((127 - g.fbits) << 23);  // 2^-F from its bit pattern
  float w1[3], w0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    w1[d] = (float)t[d] * inv_one;
    w0[d] = 1.0f - w1[d];
  }
  const float l[3] = {lam[p], lam[n3 + p], lam[2 * n3 + p]};
  const int xs[2] = {c[0], wrap_inc(c[0], ng)}, ys[2] = {c[1], wrap_inc(c[1], ng)}, zs[2] = {c[2], wrap_inc(c[2], ng)};
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float w = (dz ? w1[2] : w0[2]) * (dy ? w1[1] : w0[1]) * (dx ? w1[0] : w0[0]);
        const int64_t gi = ((int64_t)zs[dz] * ng + ys[dy]) * ng + xs[dx];
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(out + j * ng3 + gi, w * l[j]);
      }
}

// Phi_k = sum_i conj(m_i) Lam_i,k / N^3 with m_i = i k_i / (k^2 W^p): in place into lx.
__global__ void k_kspace_adjoint(int ng, int P, float kf, int deconv, float norm, float2* __restrict__ lx,
                                 const float2* __restrict__ ly, const float2* __restrict__ lz) {
  const int nh = ng / 2 + 1;
  const int64_t total = (int64_t)ng * ng * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nh);
    const int64_t r = i / nh;
    const int ky = (int)(r % ng), kz = (int)(r / ng);
    const int nx = kx, ny = ky < ng / 2 ? ky : ky - ng, nz = kz < ng / 2 ? kz : kz - ng;
    const int64_t o = r * P + kx;
    const int m2 = nx * nx + ny * ny + nz * nz;
    float2 out = make_float2(0.f, 0.f);
    if (m2 != 0) {
      float green = norm / (kf * kf * (float)m2);
      if (deconv) {
        const float sx = sinc_pi_a(nx, ng), sy = sinc_pi_a(ny, ng), sz = sinc_pi_a(nz, ng);
        const float w = (sx * sx) * (sy * sy) * (sz * sz);
        green /= (deconv == 2 ? w * w : w);
      }
      const int half = ng / 2;
      const float kx_ = (nx == half) ? 0.f : kf * nx;
      const float ky_ = (ny == -half) ? 0.f : kf * ny;
      const float kz_ = (nz == -half) ? 0.f : kf * nz;
      const float2 a = lx[o], b = ly[o], c = lz[o];
      // -i k (x + i y) = k (y - i x)
      const float re = kx_ * a.y + ky_ * b.y + kz_ * c.y;
      const float im = -(kx_ * a.x + ky_ * b.x + kz_ * c.x);
      out = make_float2(re * green, im * green);
    }
    lx[o] = out;
  }
}

// mode 0: lam_s += cKF (N/L) [ sum_i lam_v,i sum_c dW F_i(c) + (1/rho_bar) sum_c dW Phi(c) ]
// mode 1: lam_s  = (N/L) (1/rho_bar) sum_c dW Phi(c)   (density VJP, Phi = delta_bar)
__global__ void __launch_bounds__(256) k_gather_adjoint(Geometry g, const float* __restrict__ s,
                                                         const float* __restrict__ F, const float* __restrict__ phi,
                                                         const float* __restrict__ lam_v, float* __restrict__ lam_s,
                                                         float scale_a, float scale_b, int mode) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.np3) return;
  const int ng = g.ng;
  const int64_t ng3 = (int64_t)ng * ng * ng, n3 = g.np3;
  int ix, iy, iz;
  lattice_index(g, p, ix, iy, iz);
  int c[3], t[3];
  fixed_axis(g, ix, s[p], c[0], t[0]);
  fixed_axis(g, iy, s[n3 + p], c[1], t[1]);
  fixed_axis(g, iz, s[2 * n3 + p], c[2], t[2]);
  const float inv_one = __int_as_float((127 - g.fbits) << 23);  // 2^-F from its bit pattern
  float w1[3], w0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    w1[d] = (float)t[d] * inv_one;
    w0[d] = 1.0f - w1[d];
  }
  float lv[3] = {0.f, 0.f, 0.f};
  if (mode == 0) {
    lv[0] = lam_v[p];
    lv[1] = lam_v[n3 + p];
    lv[2] = lam_v[2 * n3 + p];
  }
  const int xs[2] = {c[0], wrap_inc(c[0], ng)}, ys[2] = {c[1], wrap_inc(c[1], ng)}, zs[2] = {c[2], wrap_inc(c[2], ng)};
  float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float wx = dx ? w1[0] : w0[0], wy = dy ? w1[1] : w0[1], wz = dz ? w1[2] : w0[2];
        const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
        const float dW[3] = {sx * wy * wz, wx * sy * wz, wx * wy * sz};
        const int64_t gi = ((int64_t)zs[dz] * ng + ys[dy]) * ng + xs[dx];
        const float ph = __ldg(phi + gi);
        float lf = 0.f;
        if (mode == 0) lf = lv[0] * __ldg(F + gi) + lv[1] * __ldg(F + ng3 + gi) + lv[2] * __ldg(F + 2 * ng3 + gi);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ga[d] = fmaf(dW[d], lf, ga[d]);
          gb[d] = fmaf(dW[d], ph, gb[d]);
        }
      }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float mu = scale_a * ga[d] + scale_b * gb[d];
    if (mode == 0)
      lam_s[d * n3 + p] += mu;
    else
      lam_s[d * n3 + p] = mu;
  }
}

// ---- initial conditions ----------------------------------------------------------------------------
// out (+)= scale * factor(k) * in; kind 0: i k_i / k^2; kind 1: (i k_i)(i k_j) / k^2
__global__ void k_kmul_acc(int n, int P, float kf, int kind, int i_, int j_, float scale, int accumulate,
                           const float2* __restrict__ in, float2* __restrict__ out) {
  const int nh = n / 2 + 1;
  const int64_t total = (int64_t)n * n * nh;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nh);
    const int64_t r = i / nh;
    const int ky = (int)(r % n), kz = (int)(r / n);
    const int c[3] = {kx, ky < n / 2 ? ky : ky - n, kz < n / 2 ? kz : kz - n};
    const int64_t o = r * P + kx;
    const int m2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    float2 res = make_float2(0.f, 0.f);
    if (m2 != 0) {
      const float inv_k2 = scale / (kf * kf * (float)m2);
      const float2 a = in[o];
      const float ki = (c[i_] == n / 2 || c[i_] == -n / 2) ? 0.f : kf * (float)c[i_];
      if (kind == 0) {
        res = make_float2(-ki * a.y * inv_k2, ki * a.x * inv_k2);
      } else {
        const float kj = (c[j_] == n / 2 || c[j_] == -n / 2) ? 0.f : kf * (float)c[j_];
        const float kk = -ki * kj * inv_k2;
        res = make_float2(kk * a.x, kk * a.y);
      }
    }
    if (accumulate) {
      const float2 prev = out[o];
      res = make_float2(prev.x + res.x, prev.y + res.y);
    }
    out[o] = res;
  }
}

// lam_s1 += d1 lam_s, lam_s2 += d2 lam_s
__global__ void k_ic_adjoint_assemble(int64_t m, float d1, float d2, const float* __restrict__ lam_s,
                                      float* __restrict__ lam_s1, float* __restrict__ lam_s2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float l = lam_s[i];
    lam_s1[i] += d1 * l;
    lam_s2[i] += d2 * l;
  }
}

// out = a * (b + c)   or (with c == nullptr)  out = -2 a b
__global__ void k_ic_adjoint_product(int64_t n3, const float* __restrict__ a, const float* __restrict__ b,
                                     const float* __restrict__ c, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = c ? a[i] * (b[i] + c[i]) : -2.0f * a[i] * b[i];
}

// ---- launchers -----------------------------------------------------------------------------------------
static unsigned grid_of(int64_t n, int threads = 256) {
  return (unsigned)std::min<int64_t>((n + threads - 1) / threads, (int64_t)152 * 32);
}
static unsigned full_grid(int64_t n, int threads = 256) { return (unsigned)((n + threads - 1) / threads); }

int launch_adjoint_pre(int64_t n3, int mode, const float* coef, float* lam_s, float* lam_v, float* lam_s1,
                       float* lam_s2, cudaStream_t st) {
  {
    LaunchScope ls_("adjoint_pre", st);
    k_adjoint_pre<<<full_grid(3 * n3), 256, 0, st>>>(n3, mode, coef, lam_s, lam_v, lam_s1, lam_s2);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_lambda_deposit(const Geometry& g, const float* s, const float* lam, float* out, cudaStream_t st) {
  const int64_t ng3 = (int64_t)g.ng * g.ng * g.ng;
  COLA_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(float) * 3 * ng3, st));
  {
    LaunchScope ls_("lambda_deposit", st);
    k_lambda_deposit<<<full_grid(g.np3), 256, 0, st>>>(g, s, lam, out);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_kspace_adjoint(int ng, int P, double box, int deconv, float2* lx, const float2* ly, const float2* lz,
                          cudaStream_t st) {
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const float norm = (float)(1.0 / ((double)ng * ng * ng));
  {
    LaunchScope ls_("kspace_adjoint", st);
    k_kspace_adjoint<<<grid_of((int64_t)ng * ng * (ng / 2 + 1)), 256, 0, st>>>(ng, P, kf, deconv, norm, lx, ly, lz);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_gather_adjoint(const Geometry& g, const float* s, const float* F, const float* phi, const float* lam_v,
                          float* lam_s, float scale_a, float scale_b, int mode, cudaStream_t st) {
  {
    LaunchScope ls_(mode == 0 ? "gather_adjoint" : "density_adjoint", st);
    k_gather_adjoint<<<full_grid(g.np3), 256, 0, st>>>(g, s, F, phi, lam_v, lam_s, scale_a, scale_b, mode);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_kmul_acc(int n, int P, double box, int kind, int i, int j, float scale, int accumulate, const float2* in,
                    float2* out, cudaStream_t st) {
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  {
    LaunchScope ls_("kmul_acc", st);
    k_kmul_acc<<<grid_of((int64_t)n * n * (n / 2 + 1)), 256, 0, st>>>(n, P, kf, kind, i, j, scale, accumulate, in,
                                                                         out);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_ic_adjoint_assemble(int64_t n3, float d1, float d2, const float* lam_s, float* lam_s1, float* lam_s2,
                               cudaStream_t st) {
  {
    LaunchScope ls_("ic_adjoint_assemble", st);
    k_ic_adjoint_assemble<<<grid_of(3 * n3), 256, 0, st>>>(3 * n3, d1, d2, lam_s, lam_s1, lam_s2);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int launch_ic_adjoint_product(int64_t n3, const float* a, const float* b, const float* c, float* out,
                              cudaStream_t st) {
  {
    LaunchScope ls_("ic_adjoint_product", st);
    k_ic_adjoint_product<<<grid_of(n3), 256, 0, st>>>(n3, a, b, c, out);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

}  // namespace cola
