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
#include "pm_bodies.cuh"

namespace cola {

// ---- single-box kernels ------------------------------------------------------------------------
template <int N, int TY, int TZ>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * TY * TZ)
    k_deposit_fftx(Geometry g, Tiles tl, const float* __restrict__ s, const unsigned* __restrict__ idx,
                   const int* __restrict__ offsets, float2* __restrict__ out, int P, const float2* __restrict__ tw,
                   float dscale, int* __restrict__ err) {
  extern __shared__ unsigned long long acc[];
  __shared__ int ints[28];
  deposit_fftx_body<N, TY, TZ>(g, tl, s, idx, offsets, out, P, tw, dscale, err, blockIdx.x, acc, ints);
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * green_width<N>(), 2)
    k_fft_z_green(float2* __restrict__ A, float2* __restrict__ Gz, int P, float kf, int deconv, float norm,
                  const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  z_green_body<N, green_width<N>()>(A, Gz, P, kf, deconv, norm, tw, blockIdx.x, blockIdx.y, sm);
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * green_width<N>(), 2)
    k_fft_y_inv3(float2* __restrict__ B, float2* __restrict__ Gy, float2* __restrict__ Gz, int P, float kf,
                 const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  y_inv3_body<N, green_width<N>()>(B, Gy, Gz, P, kf, tw, blockIdx.x, blockIdx.y, sm);
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * c2r3_rows<N>(), 2)
    k_fft_x_c2r3(const float2* __restrict__ C, const float2* __restrict__ Gy, const float2* __restrict__ Gz,
                 float* __restrict__ F, int P, float kf, const float2* __restrict__ tw) {
  extern __shared__ float2 smem[];
  c2r3_body<N, c2r3_rows<N>()>(C, Gy, Gz, F, P, kf, tw, blockIdx.x, blockIdx.y, smem);
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
