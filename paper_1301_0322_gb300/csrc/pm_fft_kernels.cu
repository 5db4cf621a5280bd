// Fused mesh passes of one PM force evaluation (App. A.1 eq. eom: the force
// -(3/2) Om a d_x d_x^-2 delta; readings: CIC, spectral gradient, 1/W^p deconvolution).
//
// With A the half spectrum [z][y][kx] (rows of P complex), one force evaluation runs
//   1. k_deposit_fftx   CIC deposit of a tile of TY x TZ rows (int64 in shared memory), the
//                       overdensity, and the real-to-complex FFT of those rows -> A
//   2. k_fft_cols       forward y pass on A (fft_kernels.cu)
//   3. k_fft_z_green    forward z pass, then two inverse z passes of
//                       phi_k = delta_k / (k^2 W^p N^3) and of i k_z phi_k   -> B (in A), Gz
//   4. k_fft_y_inv3     inverse y passes: C = IFFT_y(B), Gy = IFFT_y(i k_y B), Gz' = IFFT_y(Gz)
//   5. k_fft_x_c2r3     inverse x passes of (i k_x C, Gy, Gz') -> the three real force meshes
// Steps 3-5 use linearity: i k_x and i k_y are constant along z, so the x and y components
// share the inverse z transform of phi_k, and the x component shares the inverse y transform.
#include "cola_internal.cuh"
#include "fft.cuh"
#include "pm_common.cuh"

namespace cola {

// ---- helpers -----------------------------------------------------------------------------
__device__ __forceinline__ float sinc_pi_f(int n, int ng) {
  if (n == 0) return 1.0f;
  const float x = (float)n / (float)ng;
  return sinpif(x) / (3.14159265358979323846f * x);
}
__device__ __forceinline__ int signed_mode(int k, int n) { return k < n / 2 ? k : k - n; }

// first-derivative factor i k_j (zero on the Nyquist plane |n_j| = N/2)
__device__ __forceinline__ float2 mul_ik(float2 a, float k) { return make_float2(-k * a.y, k * a.x); }


template <int N>
__host__ __device__ constexpr int green_width() {
  return FFTConf<N>::T * 16 <= 256 ? 16 : (FFTConf<N>::T * 8 <= 256 ? 8 : (FFTConf<N>::T * 4 <= 512 ? 4 : 2));
}

// ---- 1. deposit + x r2c -----------------------------------------------------------------------
template <int N, int TY, int TZ>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * TY * TZ)
    k_deposit_fftx(Geometry g, Tiles tl, const float* __restrict__ s, const unsigned* __restrict__ idx,
                   const int* __restrict__ offsets, float2* __restrict__ out, int P, const float2* __restrict__ tw,
                   float dscale, int* __restrict__ err) {
  constexpr int M = N / 2, T = FFTConf<M>::T, ROWS = TY * TZ, LD = xrow_ld<M>();
  extern __shared__ unsigned long long acc[];
  __shared__ int rbeg[9], rpre[10];
  const int tyi = blockIdx.x % tl.nty, tzi = blockIdx.x / tl.nty;
  const int y0 = tyi * TY, z0 = tzi * TZ;
  for (int i = threadIdx.x; i < ROWS * N; i += blockDim.x) acc[i] = 0ull;
  // the tile's own 4 bins and the boundary bins of its 3 lower neighbours, loaded in parallel
  __shared__ int rlen[9];
  if (threadIdx.x < 9) {
    const int k = threadIdx.x;
    const int tym = tyi == 0 ? tl.nty - 1 : tyi - 1;
    const int tzm = tzi == 0 ? tl.ntz - 1 : tzi - 1;
    const int ty_ = (k == 4 || k == 5 || k == 8) ? tym : tyi;
    const int tz_ = k >= 6 ? tzm : tzi;
    const int reg = k < 4 ? k : ((k == 4 || k == 5) ? (k == 4 ? 1 : 3) : (k == 6 ? 2 : 3));
    const int b = (tz_ * tl.nty + ty_) * 4 + reg;
    const int o0 = offsets[b];
    rbeg[k] = o0;
    rlen[k] = offsets[b + 1] - o0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < 9; ++k) {
      rpre[k] = run;
      run += rlen[k];
    }
    rpre[9] = run;
  }
  __syncthreads();
  const int total = rpre[9];
  const unsigned long long one = 1ull << g.fbits;
  constexpr int U = 4;  // particles in flight per thread
  for (int base = threadIdx.x; base < total; base += blockDim.x * U) {
    int64_t pp[U];
    float sv[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * blockDim.x;
      pp[u] = -1;
      if (i < total) {
        int r = 0;
#pragma unroll
        for (int k = 1; k < 9; ++k) r += (i >= rpre[k]) ? 1 : 0;
        pp[u] = idx[rbeg[r] + (i - rpre[r])];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (pp[u] >= 0) {
        sv[u][0] = s[pp[u]];
        sv[u][1] = s[g.np3 + pp[u]];
        sv[u][2] = s[2 * g.np3 + pp[u]];
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pp[u] < 0) continue;
      int ix, iy, iz;
      lattice_index(g, pp[u], ix, iy, iz);
      int cx, tx, cy, ty, cz, tz;
      fixed_axis(g, ix, sv[u][0], cx, tx);
      fixed_axis(g, iy, sv[u][1], cy, ty);
      fixed_axis(g, iz, sv[u][2], cz, tz);
      const int cx1 = wrap_inc(cx, N);
      const unsigned long long wx0 = one - tx, wx1 = tx;
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        const int lz = (dz ? wrap_inc(cz, N) : cz) - z0;
        if (lz < 0 || lz >= TZ) continue;
        const unsigned long long wz = dz ? (unsigned long long)tz : one - tz;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          const int ly = (dy ? wrap_inc(cy, N) : cy) - y0;
          if (ly < 0 || ly >= TY) continue;
          const unsigned long long wzy = wz * (dy ? (unsigned long long)ty : one - ty);
          unsigned long long* row = acc + (lz * TY + ly) * N;
          atomicAdd(row + cx, wzy * wx0);
          atomicAdd(row + cx1, wzy * wx1);
        }
      }
    }
  }
  __syncthreads();
  // real-to-complex FFT of each tile row; z[n] = (delta[2n], delta[2n+1])
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  const unsigned long long* arow = acc + w * N;
  float2* buf = reinterpret_cast<float2*>(acc) + w * LD;
  bool overflow = false;
  auto load = [&](int n) -> float2 {
    const unsigned long long a = arow[2 * n], b = arow[2 * n + 1];
    overflow |= ((a | b) >> 62) != 0ull;
    return make_float2(fmaf(__ull2float_rn(a), dscale, -1.0f), fmaf(__ull2float_rn(b), dscale, -1.0f));
  };
  auto mem = [&](int n) -> float2& { return buf[xpad(n)]; };
  auto store = [&](int n, float2 x) { buf[xpad(n)] = x; };
  fft_1d<M, 2, false>(t, tw, load, mem, store);
  if (overflow) atomicOr(err, kErrOverflow);
  __syncthreads();
  const int lz = w / TY, ly = w - lz * TY;
  float2* dst = out + ((int64_t)(z0 + lz) * N + (y0 + ly)) * P;
  for (int k = t; k <= M; k += T) {
    const float2 a = buf[xpad(k == M ? 0 : k)];
    const float2 b = c_conj(buf[xpad(k == 0 ? 0 : M - k)]);
    const float2 e = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
    const float2 d = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y - b.y));
    dst[k] = c_add(e, c_mul(__ldg(tw + k), make_float2(d.y, -d.x)));
  }
}

// ---- 3. z pass with the Green's function ------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * green_width<N>(), 2)
    k_fft_z_green(float2* __restrict__ A, float2* __restrict__ Gz, int P, float kf, int deconv, float norm,
                  const float2* __restrict__ tw) {
  constexpr int W = green_width<N>(), nh = N / 2 + 1;
  extern __shared__ float2 sm[];
  float2* S0 = sm;           // delta_k of the slab, [n][W]
  float2* S1 = sm + N * W;   // exchange buffer
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int ky = blockIdx.y, kx = blockIdx.x * W + w;
  const bool valid = kx < nh;
  const int64_t zstride = (int64_t)N * P;
  float2* a = A + (int64_t)ky * P + (valid ? kx : 0);
  float2* gz = Gz + (int64_t)ky * P + (valid ? kx : 0);
  auto mem = [&](int n) -> float2& { return S1[n * W + w]; };
  {
    auto load = [&](int n) -> float2 { return valid ? a[n * zstride] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) { S0[n * W + w] = x; };
    fft_1d<N, 1, false>(t, tw, load, mem, store);
  }
  // sinc^2 table of the z index, then phi_k = delta_k g(k) in place in S0 (one pass)
  float* sz2 = reinterpret_cast<float*>(S1);  // S1 is free between the transforms
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const float sz = sinc_pi_f(signed_mode(n, N), N);
    sz2[n] = sz * sz;
  }
  __syncthreads();
  {
    const int ny = signed_mode(ky, N);
    const float sy = sinc_pi_f(ny, N);
    const float wy = sy * sy;
    for (int i = threadIdx.x; i < N * W; i += blockDim.x) {
      const int n = i / W, c = i - n * W;
      const int nx = blockIdx.x * W + c;
      const int nz = signed_mode(n, N);
      const int m2 = nx * nx + ny * ny + nz * nz;
      float gk = 0.0f;
      if (m2 != 0 && nx < nh) {
        gk = norm / (kf * kf * (float)m2);
        if (deconv) {
          const float sx = sinc_pi_f(nx, N);
          const float wk = (sx * sx) * wy * sz2[n];
          gk /= (deconv == 2 ? wk * wk : wk);
        }
      }
      S0[i] = c_scale(S0[i], gk);
    }
  }
  __syncthreads();
  {
    auto load = [&](int n) -> float2 { return S0[n * W + w]; };
    auto store = [&](int n, float2 x) {
      if (valid) a[n * zstride] = x;
    };
    fft_1d<N, 1, true>(t, tw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 {
      const float kz = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return mul_ik(S0[n * W + w], kz);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gz[n * zstride] = x;
    };
    fft_1d<N, 1, true>(t, tw, load, mem, store);
  }
}

// ---- 4. inverse y passes ------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * green_width<N>(), 2)
    k_fft_y_inv3(float2* __restrict__ B, float2* __restrict__ Gy, float2* __restrict__ Gz, int P, float kf,
                 const float2* __restrict__ tw) {
  constexpr int W = green_width<N>(), nh = N / 2 + 1, T = FFTConf<N>::T;
  extern __shared__ float2 sm[];
  float2* S0 = sm;
  float2* S1 = sm + N * W;
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int z = blockIdx.y, kx = blockIdx.x * W + w;
  const bool valid = kx < nh;
  const int64_t slab = (int64_t)z * N * P + (valid ? kx : 0);
  float2* b = B + slab;
  float2* gy = Gy + slab;
  float2* gz = Gz + slab;
  for (int n = t; n < N; n += T) S0[n * W + w] = valid ? b[(int64_t)n * P] : make_float2(0.f, 0.f);
  __syncthreads();
  auto mem = [&](int n) -> float2& { return S1[n * W + w]; };
  {
    auto load = [&](int n) -> float2 { return S0[n * W + w]; };
    auto store = [&](int n, float2 x) {
      if (valid) b[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true>(t, tw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 {
      const float ky = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return mul_ik(S0[n * W + w], ky);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gy[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true>(t, tw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 { return valid ? gz[(int64_t)n * P] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      if (valid) gz[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true>(t, tw, load, mem, store);
  }
}

// ---- 5. inverse x passes of the three components -------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int c2r3_rows() {
  return FFTConf<N / 2>::T >= 256 ? 1 : 256 / FFTConf<N / 2>::T;
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * c2r3_rows<N>(), 2)
    k_fft_x_c2r3(const float2* __restrict__ C, const float2* __restrict__ Gy, const float2* __restrict__ Gz,
                 float* __restrict__ F, int P, float kf, const float2* __restrict__ tw) {
  constexpr int M = N / 2, T = FFTConf<M>::T, RB = c2r3_rows<N>(), LD = xrow_ld<M>();
  extern __shared__ float2 smem[];
  const int comp = blockIdx.y;
  const float2* srcm = comp == 0 ? C : (comp == 1 ? Gy : Gz);
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  const int64_t row = (int64_t)blockIdx.x * RB + w;
  const float2* src = srcm + row * P;
  float2* buf = smem + w * LD;
  for (int k = t; k <= M; k += T) {
    float2 x = src[k];
    if (comp == 0) x = mul_ik(x, k == M ? 0.0f : kf * (float)k);
    buf[xpad(k)] = x;
  }
  __syncthreads();
  auto load = [&](int n) -> float2 {
    const float2 a = buf[xpad(n)], bb = c_conj(buf[xpad(M - n)]);
    const float2 e = c_add(a, bb);
    const float2 o = c_mul(c_sub(a, bb), c_conj(__ldg(tw + n)));
    return make_float2(e.x - o.y, e.y + o.x);
  };
  auto mem = [&](int n) -> float2& { return buf[xpad(n)]; };
  float2* dst = reinterpret_cast<float2*>(F + (int64_t)comp * N * N * N + row * N);
  auto store = [&](int n, float2 x) { dst[n] = x; };
  fft_1d<M, 2, true>(t, tw, load, mem, store);
}

// ---- launchers ---------------------------------------------------------------------------------------------------
template <class K>
static int set_smem(K kernel, size_t bytes) {
  if (bytes > 227 * 1024) return fail(COLA_EUNSUPPORTED, "fused FFT kernel: shared memory request too large");
  if (bytes > 32 * 1024)
    COLA_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return COLA_OK;
}

template <int N>
static const char* flabel(int kind) {
  static const std::string names[4] = {std::string("deposit_fftx_") + std::to_string(N),
                                       std::string("fft_z_green_") + std::to_string(N),
                                       std::string("fft_y_inv3_") + std::to_string(N),
                                       std::string("fft_x_c2r3_") + std::to_string(N)};
  return names[kind].c_str();
}

template <int N>
static int force_passes_t(const Geometry& g, const Tiles& tl, const float* s, const unsigned* idx, const int* offsets,
                          float2* A, float2* Gy, float2* Gz, float* F, int P, double box, int deconv,
                          const float2* tw, int* err, cudaStream_t st) {
  constexpr int M = N / 2, W = green_width<N>(), nh = N / 2 + 1;
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const float norm = (float)(1.0 / ((double)N * N * N));
  int rc;
  // 1. deposit + x r2c
  {
    const double n3 = (double)N * N * N;
    const float dscale = (float)(n3 / ((double)g.np3 * std::ldexp(1.0, 3 * g.fbits)));
    if (tl.ty == 4 && tl.tz == 2) {
      const size_t smem = sizeof(unsigned long long) * 8 * std::max(N, xrow_ld<M>());
      if ((rc = set_smem(k_deposit_fftx<N, 4, 2>, smem))) return rc;
      LaunchScope ls_(flabel<N>(0), st);
      k_deposit_fftx<N, 4, 2><<<tl.nty * tl.ntz, FFTConf<M>::T * 8, smem, st>>>(g, tl, s, idx, offsets, A, P, tw,
                                                                                  dscale, err);
    } else if (tl.ty == 2 && tl.tz == 2) {
      const size_t smem = sizeof(unsigned long long) * 4 * std::max(N, xrow_ld<M>());
      if ((rc = set_smem(k_deposit_fftx<N, 2, 2>, smem))) return rc;
      LaunchScope ls_(flabel<N>(0), st);
      k_deposit_fftx<N, 2, 2><<<tl.nty * tl.ntz, FFTConf<M>::T * 4, smem, st>>>(g, tl, s, idx, offsets, A, P, tw,
                                                                                  dscale, err);
    } else {
      return fail(COLA_EUNSUPPORTED, "fused deposit: unsupported tile shape");
    }
    COLA_LAUNCH_CHECK();
  }
  // 2. forward y pass
  if ((rc = launch_fft_cols(N, false, A, N, (int64_t)N * P, P, nh, tw, st))) return rc;
  // 3. z pass with the Green's function
  {
    const size_t smem = sizeof(float2) * 2 * N * W;
    if ((rc = set_smem(k_fft_z_green<N>, smem))) return rc;
    dim3 grid((nh + W - 1) / W, N);
    LaunchScope ls_(flabel<N>(1), st);
    k_fft_z_green<N><<<grid, FFTConf<N>::T * W, smem, st>>>(A, Gz, P, kf, deconv, norm, tw);
    COLA_LAUNCH_CHECK();
  }
  // 4. inverse y passes
  {
    const size_t smem = sizeof(float2) * 2 * N * W;
    if ((rc = set_smem(k_fft_y_inv3<N>, smem))) return rc;
    dim3 grid((nh + W - 1) / W, N);
    LaunchScope ls_(flabel<N>(2), st);
    k_fft_y_inv3<N><<<grid, FFTConf<N>::T * W, smem, st>>>(A, Gy, Gz, P, kf, tw);
    COLA_LAUNCH_CHECK();
  }
  // 5. inverse x passes
  {
    constexpr int RB = c2r3_rows<N>();
    const size_t smem = sizeof(float2) * RB * xrow_ld<M>();
    if ((rc = set_smem(k_fft_x_c2r3<N>, smem))) return rc;
    const int64_t nrows = (int64_t)N * N;
    if (nrows % RB) return fail(COLA_EINVAL, "fused c2r: row count not a multiple of the block rows");
    dim3 grid((unsigned)(nrows / RB), 3);
    LaunchScope ls_(flabel<N>(3), st);
    k_fft_x_c2r3<N><<<grid, FFTConf<M>::T * RB, smem, st>>>(A, Gy, Gz, F, P, kf, tw);
    COLA_LAUNCH_CHECK();
  }
  return COLA_OK;
}

int launch_force_passes(const Geometry& g, const Tiles& tl, const float* s, const unsigned* idx, const int* offsets,
                        float2* A, float2* Gy, float2* Gz, float* F, int P, double box, int deconv, const float2* tw,
                        int* err, cudaStream_t st) {
  switch (g.ng) {
#define X(N) \
  case N:    \
    return force_passes_t<N>(g, tl, s, idx, offsets, A, Gy, Gz, F, P, box, deconv, tw, err, st);
    X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "force passes: unsupported mesh size");
  }
}

}  // namespace cola
