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
// resident blocks per SM the fused deposit is compiled for: 512 threads per SM, and three blocks
// of 2 x 2 tiles at N = 2048 (64 KB of cell sums each; 80 registers, no spills)
template <int N, int TY, int TZ>
__host__ __device__ constexpr int deposit_min_blocks() {
  return N == 2048 && TY * TZ == 4 ? 3 : ((512 / (FFTConf<N / 2>::T * TY * TZ)) > 0 ? 512 / (FFTConf<N / 2>::T * TY * TZ) : 1);
}

// cell sums (8 bytes per cell) of a TY x TZ tile, which later hold the rows' transform buffers
template <int N, int TY, int TZ>
__host__ __device__ constexpr int deposit_acc_cells() {
  return TY * TZ * (N > xrow_ld<N / 2>() ? N : xrow_ld<N / 2>());
}
// A tight stage twiddle table (fft.cuh) behind the cell sums at N = 2048 (10.3 KB: three blocks
// of 2 x 2 tiles per SM still fit); below 2048 the table costs more in resident blocks than the
// twiddle loads it saves.
template <int N>
__host__ __device__ constexpr int deposit_table_size() {
  return N == 2048 ? stw_size<FFTConf<N / 2>, true>() : 0;
}

template <int N, int TY, int TZ>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * TY * TZ, deposit_min_blocks<N, TY, TZ>())
    k_deposit_fftx(Geometry g, Tiles tl, const uint4* __restrict__ rec, const int* __restrict__ offsets,
                   float2* __restrict__ out, int P, const float2* __restrict__ tw, float dscale,
                   int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned long long acc[];
  __shared__ int ints[28];
  if constexpr (deposit_table_size<N>() > 0) {
    float2* stab = reinterpret_cast<float2*>(acc + deposit_acc_cells<N, TY, TZ>());
    stw_fill<FFTConf<N / 2>, 2, true>(stab, tw, threadIdx.x, blockDim.x);
    deposit_fftx_body<N, TY, TZ>(g, tl, rec, offsets, out, P, tw, SmemTw<FFTConf<N / 2>, true>{stab}, dscale, err,
                                 blockIdx.x, acc, ints);
  } else {
    deposit_fftx_body<N, TY, TZ>(g, tl, rec, offsets, out, P, tw, tw, dscale, err, blockIdx.x, acc, ints);
  }
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * col_width<N>(), 2)
    k_fft_z_green(float2* __restrict__ A, float2* __restrict__ Gz, int P, float kf, int deconv, float norm,
                  const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  z_green_body<N, col_width<N>()>(A, Gz, P, kf, deconv, norm, tw, blockIdx.x, blockIdx.y, sm);
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N>::T * col_width<N>(), 2)
    k_fft_y_inv3(float2* __restrict__ B, float2* __restrict__ Gy, float2* __restrict__ Gz, int P, float kf,
                 const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  y_inv3_body<N, col_width<N>()>(B, Gy, Gz, P, kf, tw, blockIdx.x, blockIdx.y, sm);
}

// Strip widths of the single-buffer (wide-strip) z, forward y and inverse y passes, 0 where the
// two-buffer bodies (z, inverse y) or the stand-alone column pass (forward y) are used.  At 256,
// 16-column strips: z 0.88 -> 0.75, forward y 0.34 -> 0.31 ms per 128^3/256^3 run; at 768 the
// stand-alone forward y pass stays faster.
template <int N>
__host__ __device__ constexpr int wide_width() {
  return (N == 2048 || N == 768) ? 8 : ((N >= 128 && N <= 256) ? 16 : 0);
}
template <int N>
__host__ __device__ constexpr int wide_fwd_width() {
  return N == 768 ? 0 : wide_width<N>();
}
// the same for the inverse y passes (768: 27.0 -> 23.5 ms per 256^3/768^3 run; 16-column strips
// at 128-256: 1.43 -> 0.75 ms per 128^3/256^3 run)
template <int N>
__host__ __device__ constexpr int wide_inv_width() {
  return (N == 2048 || N == 768) ? 8 : ((N >= 128 && N <= 256) ? 16 : 0);
}
template <int N, int W>
__host__ __device__ constexpr int wide_min_blocks() {
  return FFTConf<N>::T * W >= 1024 ? 1 : 2;
}

// scratch slots per SM of the wide z pass: the SM's own slot where one block fits (2048), four
// claimed slots at 768 (at most three blocks of 58 KB fit), none elsewhere
template <int N, int W>
__host__ __device__ constexpr int wide_z_slots() {
  return wide_min_blocks<N, W>() == 1 ? 1 : (N == 768 ? 4 : 0);
}
// slot flags of the claimed scratch slots (zero between launches: every block frees its slot)
__device__ int g_zslot_busy[kZScratchSlots * 4];

template <int N, int W>
__global__ void __launch_bounds__(FFTConf<N>::T * W, wide_min_blocks<N, W>())
    k_fft_z_green_wide(float2* __restrict__ A, float2* __restrict__ Gz, float2* __restrict__ scratch, float kf,
                       int deconv, float norm, const float2* __restrict__ tw, int* __restrict__ err) {
  extern __shared__ __align__(16) float2 sm[];
  z_green_wide_body<N, W, wide_z_slots<N, W>()>(A, Gz, scratch, g_zslot_busy, kf, deconv, norm, tw, err,
                                                 blockIdx.x, blockIdx.y, sm);
}
// the scratch slot of an SM belongs to one block only if two blocks cannot share the SM
template <int N, int W>
constexpr size_t wide_z_smem() {
  return sizeof(float2) * (wide_z_table_offset<N, W>() + stw_size<FFTConf<N>>());
}
static_assert(2 * wide_z_smem<2048, 8>() > 228 * 1024, "two wide z blocks would fit on one SM");
static_assert(4 * (wide_z_smem<768, 8>() + 1024) > 228 * 1024, "four wide z blocks would fit on one SM");

template <int N, int W>
__global__ void __launch_bounds__(FFTConf<N>::T * W, wide_min_blocks<N, W>())
    k_fft_y_inv3_wide(float2* __restrict__ B, float2* __restrict__ Gy, float2* __restrict__ Gz, float kf,
                      const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 sm[];
  y_inv3_wide_body<N, W>(B, Gy, Gz, kf, tw, blockIdx.x, blockIdx.y, sm);
}

// forward y pass of the half spectrum in strips of W columns (slab = z)
template <int N, int W>
__global__ void __launch_bounds__(FFTConf<N>::T * W, wide_min_blocks<N, W>())
    k_fft_y_fwd_wide(float2* __restrict__ A, const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 sm[];
  constexpr int P = half_pitch<N>();
  float2* stab = sm + N * W;
  stw_fill<FFTConf<N>, 1>(stab, tw, threadIdx.x, FFTConf<N>::T * W);
  const SmemTw<FFTConf<N>> stw{stab};
  cols_body<N, W, false>(A, (int64_t)N * P, P, N / 2 + 1, stw, blockIdx.x, blockIdx.y, sm);
}

// Persistent: each block walks items blockIdx.x, blockIdx.x + gridDim.x, ... with the bulk
// copies of its next NB - 1 items in flight during the transform of the current one (NB buffers).
template <int N>
__host__ __device__ constexpr int c2r3_stages() {
  return 2;
}

// resident blocks per SM of the inverse-x pass: four at N = 2048 (128 registers, no spills;
// 16 warps to cover the shared-memory latency of the staged rows), three otherwise
template <int N>
__host__ __device__ constexpr int c2r3_min_blocks() {
  return N == 2048 ? 4 : 3;
}

template <int N>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * c2r3_rows<N>(), c2r3_min_blocks<N>())
    k_fft_x_c2r3(const float2* __restrict__ C, const float2* __restrict__ Gy, const float2* __restrict__ Gz,
                 float* __restrict__ F, int P, float kf, const float2* __restrict__ tw, int* __restrict__ err) {
  constexpr int M = N / 2, RB = c2r3_rows<N>(), LD = xrow_ld<M>(), NB = c2r3_stages<N>();
  extern __shared__ __align__(128) float2 c2r_stage[];
  __shared__ __align__(8) uint64_t bars[NB];
  const int64_t nrb = (int64_t)N * N / RB, total = 3 * nrb;
  auto src_of = [&](int64_t item) -> const float2* {
    const int comp = (int)(item / nrb);
    const float2* m = comp == 0 ? C : (comp == 1 ? Gy : Gz);
    return m + (item - comp * nrb) * RB * P;
  };
  // stage twiddles, copied once per block (persistent) behind the staging buffers
  float2* stab = c2r_stage + NB * RB * LD;
  stw_fill<FFTConf<M>, 2>(stab, tw, threadIdx.x, blockDim.x);
  const SmemTw<FFTConf<M>> stw{stab};
  if (threadIdx.x == 0) {
    for (int k = 0; k < NB; ++k) mbar_init(&bars[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // prologue: the first NB - 1 items
  for (int k = 0; k < NB - 1; ++k) {
    const int64_t item = blockIdx.x + (int64_t)k * gridDim.x;
    if (item < total && threadIdx.x < 32) c2r3_issue(c2r_stage + k * RB * LD, src_of(item), RB, P, LD, &bars[k]);
  }
  int64_t item = blockIdx.x;
  for (int it = 0; item < total; ++it, item += gridDim.x) {
    const int b = it % NB;
    const int64_t ahead = item + (int64_t)(NB - 1) * gridDim.x;
    const int ba = (it + NB - 1) % NB;  // consumed at iteration it - 1, free after its closing barrier
    if (ahead < total && threadIdx.x < 32) c2r3_issue(c2r_stage + ba * RB * LD, src_of(ahead), RB, P, LD, &bars[ba]);
    const bool ok = mbar_wait(&bars[b], (it / NB) & 1);
    if (__syncthreads_or(!ok)) {
      // leave no bulk copy in flight into shared memory the block releases: wait again (bounded)
      // for the copy that timed out and for every later one already issued
      if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
      for (int k = 0; k < NB; ++k)
        if (item + (int64_t)k * gridDim.x < total) mbar_wait(&bars[(it + k) % NB], ((it + k) / NB) & 1);
      return;
    }
    const int comp = (int)(item / nrb);
    const int64_t row0 = (item - comp * nrb) * RB;
    c2r3_compute<N, RB>(c2r_stage + b * RB * LD, F + (int64_t)comp * N * N * N + row0 * N, comp, kf, tw, stw);
    __syncthreads();
  }
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
  static const std::string names[5] = {std::string("deposit_fftx_") + std::to_string(N),
                                       std::string("fft_z_green_") + std::to_string(N),
                                       std::string("fft_y_inv3_") + std::to_string(N),
                                       std::string("fft_x_c2r3_") + std::to_string(N),
                                       std::string("fft_cols_fwd_") + std::to_string(N)};
  return names[kind].c_str();
}

// 1. deposit + x r2c of every tile into the half spectrum A
template <int N>
static int deposit_fftx_t(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets, float2* A, int P,
                          const float2* tw, int* err, cudaStream_t st) {
  constexpr int M = N / 2;
  int rc;
  const double n3 = (double)N * N * N;
  const float dscale = (float)(n3 / ((double)g.np3 * std::ldexp(1.0, 3 * g.fbits)));
  if (tl.ty == 4 && tl.tz == 2) {
    const size_t smem = sizeof(unsigned long long) * (deposit_acc_cells<N, 4, 2>() + deposit_table_size<N>());
    if ((rc = set_smem(k_deposit_fftx<N, 4, 2>, smem))) return rc;
    LaunchScope ls_(flabel<N>(0), st);
    k_deposit_fftx<N, 4, 2><<<tl.nty * tl.ntz, FFTConf<M>::T * 8, smem, st>>>(g, tl, rec, offsets, A, P, tw,
                                                                                dscale, err);
  } else if (tl.ty == 2 && tl.tz == 2) {
    const size_t smem = sizeof(unsigned long long) * (deposit_acc_cells<N, 2, 2>() + deposit_table_size<N>());
    if ((rc = set_smem(k_deposit_fftx<N, 2, 2>, smem))) return rc;
    LaunchScope ls_(flabel<N>(0), st);
    k_deposit_fftx<N, 2, 2><<<tl.nty * tl.ntz, FFTConf<M>::T * 4, smem, st>>>(g, tl, rec, offsets, A, P, tw,
                                                                                dscale, err);
  } else {
    return fail(COLA_EUNSUPPORTED, "fused deposit: unsupported tile shape");
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

// 2. forward y pass of the half spectrum A
template <int N>
static int forward_y_t(float2* A, int P, const float2* tw, cudaStream_t st) {
  constexpr int nh = N / 2 + 1, WF = wide_fwd_width<N>();
  if constexpr (WF > 0) {
    if (P != half_pitch<N>()) return fail(COLA_EINVAL, "wide column passes: unexpected half-spectrum pitch");
    int rc;
    const dim3 grid((nh + WF - 1) / WF, N);
    const size_t smem = sizeof(float2) * (N * WF + stw_size<FFTConf<N>>());
    if ((rc = set_smem(k_fft_y_fwd_wide<N, WF>, smem))) return rc;
    LaunchScope ls_(flabel<N>(4), st);
    k_fft_y_fwd_wide<N, WF><<<grid, FFTConf<N>::T * WF, smem, st>>>(A, tw);
    COLA_LAUNCH_CHECK();
    return COLA_OK;
  } else {
    return launch_fft_cols(N, false, A, N, (int64_t)N * P, P, nh, tw, st);
  }
}

template <int N>
static int force_passes_t(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets,
                          float2* A, float2* Gy, float2* Gz, float* F, int P, double box, int deconv,
                          const float2* tw, int* err, cudaStream_t st) {
  constexpr int M = N / 2, W = col_width<N>(), nh = N / 2 + 1;
  const float kf = (float)(2.0 * 3.14159265358979323846 / box);
  const float norm = (float)(1.0 / ((double)N * N * N));
  int rc;
  if ((rc = deposit_fftx_t<N>(g, tl, rec, offsets, A, P, tw, err, st))) return rc;
  constexpr int WW = wide_width<N>(), WI = wide_inv_width<N>();
  if constexpr (WW > 0 || WI > 0) {
    if (P != half_pitch<N>()) return fail(COLA_EINVAL, "wide column passes: unexpected half-spectrum pitch");
  }
  if ((rc = forward_y_t<N>(A, P, tw, st))) return rc;
  if constexpr (WW > 0) {
    const dim3 grid((nh + WW - 1) / WW, N);
    constexpr int NT = FFTConf<N>::T * WW;
    // 3. z pass with the Green's function; its scratch slots sit at the start of Gy, which the
    // inverse y passes write only afterwards
    {
      static_assert((int64_t)kZScratchSlots * wide_z_slots<N, WW>() * N * WW <= (int64_t)N * N * half_pitch<N>(),
                    "scratch exceeds Gy");
      const size_t smem = wide_z_smem<N, WW>();
      if ((rc = set_smem(k_fft_z_green_wide<N, WW>, smem))) return rc;
      LaunchScope ls_(flabel<N>(1), st);
      k_fft_z_green_wide<N, WW><<<grid, NT, smem, st>>>(A, Gz, Gy, kf, deconv, norm, tw, err);
      COLA_LAUNCH_CHECK();
    }
  } else {
    // 3. z pass with the Green's function
    {
      const size_t smem = sizeof(float2) * 2 * N * W;
      if ((rc = set_smem(k_fft_z_green<N>, smem))) return rc;
      dim3 grid((nh + W - 1) / W, N);
      LaunchScope ls_(flabel<N>(1), st);
      k_fft_z_green<N><<<grid, FFTConf<N>::T * W, smem, st>>>(A, Gz, P, kf, deconv, norm, tw);
      COLA_LAUNCH_CHECK();
    }
  }
  // 4. inverse y passes
  if constexpr (WI > 0) {
    const dim3 grid((nh + WI - 1) / WI, N);
    const size_t smem = sizeof(float2) * (N * WI + stw_size<FFTConf<N>>());
    if ((rc = set_smem(k_fft_y_inv3_wide<N, WI>, smem))) return rc;
    LaunchScope ls_(flabel<N>(2), st);
    k_fft_y_inv3_wide<N, WI><<<grid, FFTConf<N>::T * WI, smem, st>>>(A, Gy, Gz, kf, tw);
    COLA_LAUNCH_CHECK();
  } else {
    const size_t smem = sizeof(float2) * 2 * N * W;
    if ((rc = set_smem(k_fft_y_inv3<N>, smem))) return rc;
    dim3 grid((nh + W - 1) / W, N);
    LaunchScope ls_(flabel<N>(2), st);
    k_fft_y_inv3<N><<<grid, FFTConf<N>::T * W, smem, st>>>(A, Gy, Gz, P, kf, tw);
    COLA_LAUNCH_CHECK();
  }
  // 5. inverse x passes (persistent, bulk-copy pipelined)
  {
    constexpr int RB = c2r3_rows<N>(), T = FFTConf<M>::T;
    const size_t smem = sizeof(float2) * (c2r3_stages<N>() * RB * xrow_ld<M>() + stw_size<FFTConf<M>>());
    if ((rc = set_smem(k_fft_x_c2r3<N>, smem))) return rc;
    const int64_t nrows = (int64_t)N * N;
    if (nrows % RB) return fail(COLA_EINVAL, "fused c2r: row count not a multiple of the block rows");
    if (P % 4) return fail(COLA_EINVAL, "fused c2r: row pitch must be a multiple of 4 complex");
    // resident blocks x SMs of the current device (cached per device)
    static int grid_cap[64] = {};
    int dev = 0;
    COLA_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(COLA_EUNSUPPORTED, "device index above 63");
    if (!grid_cap[dev]) {
      int occ = 0, sms = 0;
      COLA_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_x_c2r3<N>, T * RB, smem));
      COLA_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      if (occ < 1) return fail(COLA_EUNSUPPORTED, "fused c2r does not fit on an SM");
      grid_cap[dev] = occ * sms;
    }
    const int64_t items = 3 * nrows / RB;
    const unsigned grid = (unsigned)std::min<int64_t>(items, grid_cap[dev]);
    LaunchScope ls_(flabel<N>(3), st);
    k_fft_x_c2r3<N><<<grid, T * RB, smem, st>>>(A, Gy, Gz, F, P, kf, tw, err);
    COLA_LAUNCH_CHECK();
  }
  return COLA_OK;
}

int launch_density_spectrum(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets, float2* A,
                            int P, const float2* tw, int* err, cudaStream_t st) {
  switch (g.ng) {
#define X(N)                                                                                          \
  case N: {                                                                                           \
    int rc;                                                                                           \
    if ((rc = deposit_fftx_t<N>(g, tl, rec, offsets, A, P, tw, err, st))) return rc;                  \
    if ((rc = forward_y_t<N>(A, P, tw, st))) return rc;                                               \
    return launch_fft_cols(N, false, A, N, P, (int64_t)N * P, N / 2 + 1, tw, st); /* z: slab = y */ \
  }
    X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "density spectrum: unsupported mesh size");
  }
}

int launch_force_passes(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets,
                        float2* A, float2* Gy, float2* Gz, float* F, int P, double box, int deconv, const float2* tw,
                        int* err, cudaStream_t st) {
  switch (g.ng) {
#define X(N) \
  case N:    \
    return force_passes_t<N>(g, tl, rec, offsets, A, Gy, Gz, F, P, box, deconv, tw, err, st);
    X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "force passes: unsupported mesh size");
  }
}

}  // namespace cola
