// Batched 1-D FFT passes of the 3-D real-to-complex / complex-to-real transforms.
//
// Layout of a half spectrum of an n^3 real mesh: [z][y][kx], kx in [0, n/2], rows padded to
// P >= n/2 + 1 complex entries.  A 3-D r2c is: x pass (real rows -> half rows), y pass and
// z pass (strided complex columns, in place).  The c2r runs the same passes in reverse.
#include "cola_internal.cuh"
#include "fft.cuh"
#include "pm_bodies.cuh"

namespace cola {

// rows per block of the contiguous x passes (about 256 threads per block)
template <int N>
__host__ __device__ constexpr int x_rows() {
  return FFTConf<N / 2>::T >= 256 ? 1 : 256 / FFTConf<N / 2>::T;
}

// Columns per block of the stand-alone column passes: 8 (64-byte row segments) for the 16-element
// transforms of length 1024 and 2048, whose one exchange buffer leaves room for them (the
// two-buffer force passes at those lengths use col_width).
template <int N>
__host__ __device__ constexpr int cols_pass_width() {
  return (N == 1024 || N == 2048) ? 8 : col_width<N>();
}
template <int N>
__host__ __device__ constexpr int cols_pass_min_blocks() {
  return FFTConf<N>::T * cols_pass_width<N>() >= 1024 ? 1 : 2;
}

// Stage twiddles from a shared-memory table (fft.cuh) at N = 2048, where one block per SM leaves
// room for it; at the other lengths the table would cost resident blocks.
template <int N>
__host__ __device__ constexpr int cols_table_size() {
  return N == 2048 ? stw_size<FFTConf<N>>() : 0;
}

// In-place FFT of ncols columns per slab: element (n, col) at data[slab*slab_stride + n*row_stride + col].
template <int N, bool INV>
__global__ void __launch_bounds__(FFTConf<N>::T * cols_pass_width<N>(), cols_pass_min_blocks<N>())
    k_fft_cols(float2* __restrict__ data, int64_t slab_stride, int64_t row_stride, int ncols,
               const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 smem[];
  constexpr int W = cols_pass_width<N>();
  if constexpr (cols_table_size<N>() > 0) {
    float2* stab = smem + N * W;
    stw_fill<FFTConf<N>, 1>(stab, tw, threadIdx.x, FFTConf<N>::T * W);
    cols_body<N, W, INV>(data, slab_stride, row_stride, ncols, SmemTw<FFTConf<N>>{stab}, blockIdx.x, blockIdx.y,
                         smem);
  } else {
    cols_body<N, W, INV>(data, slab_stride, row_stride, ncols, tw, blockIdx.x, blockIdx.y, smem);
  }
}

// Real rows of length N -> half-spectrum rows (N/2 + 1 entries, stride P), via a complex
// FFT of length M = N/2 of z[n] = x[2n] + i x[2n+1] and the split
//   X[k] = (Z[k] + conj Z[M-k]) / 2 - (i/2) exp(-2 pi i k/N) (Z[k] - conj Z[M-k]).
// The x passes read their stage twiddles from a shared-memory table behind the row buffers
// (fft.cuh; filled per block, first read after the transform's first barrier).
template <int N>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * x_rows<N>())
    k_fft_x_r2c(const float* __restrict__ in, float2* __restrict__ out, int P, const float2* __restrict__ tw) {
  constexpr int M = N / 2, T = FFTConf<M>::T, RB = x_rows<N>(), LD = xrow_ld<M>();
  constexpr int R0 = first_radix<FFTConf<M>>();
  extern __shared__ __align__(16) float2 smem[];
  float2* stab = smem + RB * LD;
  stw_fill<FFTConf<M>, 2>(stab, tw, threadIdx.x, T * RB);
  const SmemTw<FFTConf<M>> stw{stab};
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  const int64_t row = (int64_t)blockIdx.x * RB + w;
  const float2* src = reinterpret_cast<const float2*>(in + row * N);
  float2* buf = smem + w * LD;
  auto load = [&](int n) -> float2 { return src[n]; };
  auto mem = [&](int n) -> float2& { return buf[xpad<R0>(n)]; };
  auto store = [&](int n, float2 x) { buf[xpad<R0>(n)] = x; };
  fft_1d<M, 2, false>(t, stw, load, mem, store);
  __syncthreads();
  float2* dst = out + row * P;
  // X[k] = e + p and X[M - k] = conj(e - p) from one pair Z[k], Z[M - k] (p = W^k (-i d))
  for (int k = t; k <= M / 2; k += T) {
    const float2 a = buf[xpad<R0>(k)];
    const float2 b = c_conj(buf[xpad<R0>(k == 0 ? 0 : M - k)]);
    const float2 e = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y + b.y));
    const float2 d = make_float2(0.5f * (a.x - b.x), 0.5f * (a.y - b.y));
    const float2 p = c_mul(__ldg(tw + k), make_float2(d.y, -d.x));
    dst[k] = c_add(e, p);
    if (2 * k != M) dst[M - k] = c_conj(c_sub(e, p));
  }
}

// Half-spectrum rows -> real rows of length N (unscaled inverse, times `scale`).
template <int N>
__global__ void __launch_bounds__(FFTConf<N / 2>::T * x_rows<N>())
    k_fft_x_c2r(const float2* __restrict__ in, float* __restrict__ out, int P, const float2* __restrict__ tw,
                float scale) {
  constexpr int M = N / 2, T = FFTConf<M>::T, RB = x_rows<N>(), LD = xrow_ld<M>();
  constexpr int R0 = first_radix<FFTConf<M>>();
  extern __shared__ __align__(16) float2 smem[];
  float2* stab = smem + RB * LD;
  stw_fill<FFTConf<M>, 2>(stab, tw, threadIdx.x, T * RB);
  const SmemTw<FFTConf<M>> stw{stab};
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  const int64_t row = (int64_t)blockIdx.x * RB + w;
  const float2* src = in + row * P;
  float2* buf = smem + w * LD;
  for (int k = t; k <= M; k += T) buf[xpad<R0>(k)] = src[k];
  __syncthreads();
  auto load = [&](int n) -> float2 {
    const float2 a = buf[xpad<R0>(n)], b = c_conj(buf[xpad<R0>(M - n)]);
    const float2 e = c_add(a, b);
    const float2 o = c_mul(c_sub(a, b), c_conj(__ldg(tw + n)));
    return make_float2(e.x - o.y, e.y + o.x);  // e + i o
  };
  auto mem = [&](int n) -> float2& { return buf[xpad<R0>(n)]; };
  float2* dst = reinterpret_cast<float2*>(out + row * N);
  auto store = [&](int n, float2 x) { dst[n] = c_scale(x, scale); };
  fft_1d<M, 2, true>(t, stw, load, mem, store);
}

// persistent per-size kernel labels for the profiler
template <int N>
static const char* label(const char* kind) {
  static const std::string names[4] = {std::string("fft_x_r2c_") + std::to_string(N),
                                       std::string("fft_x_c2r_") + std::to_string(N),
                                       std::string("fft_cols_fwd_") + std::to_string(N),
                                       std::string("fft_cols_inv_") + std::to_string(N)};
  const int i = kind[0] == 'r' ? 0 : kind[0] == 'c' ? 1 : kind[0] == 'f' ? 2 : 3;
  return names[i].c_str();
}

template <class K>
static void allow_smem(K kernel, size_t bytes) {
  if (bytes > 32 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N>
static int x_r2c(const float* in, float2* out, int64_t nrows, int P, const float2* tw, cudaStream_t st) {
  constexpr int M = N / 2, RB = x_rows<N>();
  const size_t smem = (size_t)(RB * xrow_ld<M>() + stw_size<FFTConf<M>>()) * sizeof(float2);
  if (nrows % RB) return fail(COLA_EINVAL, "fft x pass: row count not a multiple of the block rows");
  allow_smem(k_fft_x_r2c<N>, smem);
  { LaunchScope ls_(label<N>("r2c"), st);
  k_fft_x_r2c<N><<<(unsigned)(nrows / RB), FFTConf<M>::T * RB, smem, st>>>(in, out, P, tw); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

template <int N>
static int x_c2r(const float2* in, float* out, int64_t nrows, int P, const float2* tw, float scale, cudaStream_t st) {
  constexpr int M = N / 2, RB = x_rows<N>();
  const size_t smem = (size_t)(RB * xrow_ld<M>() + stw_size<FFTConf<M>>()) * sizeof(float2);
  if (nrows % RB) return fail(COLA_EINVAL, "fft x pass: row count not a multiple of the block rows");
  allow_smem(k_fft_x_c2r<N>, smem);
  { LaunchScope ls_(label<N>("c2r"), st);
  k_fft_x_c2r<N><<<(unsigned)(nrows / RB), FFTConf<M>::T * RB, smem, st>>>(in, out, P, tw, scale); }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

template <int N>
static int cols(bool inverse, float2* data, int64_t nslabs, int64_t slab_stride, int64_t row_stride, int ncols,
                const float2* tw, cudaStream_t st) {
  constexpr int W = cols_pass_width<N>();
  const size_t smem = (size_t)(N * W + cols_table_size<N>()) * sizeof(float2);
  if (nslabs > 65535) return fail(COLA_EINVAL, "fft column pass: too many slabs");
  dim3 grid((ncols + W - 1) / W, (unsigned)nslabs);
  if (inverse) {
    allow_smem(k_fft_cols<N, true>, smem);
    { LaunchScope ls_(label<N>("inv"), st);
    k_fft_cols<N, true><<<grid, FFTConf<N>::T * W, smem, st>>>(data, slab_stride, row_stride, ncols, tw); }
  } else {
    allow_smem(k_fft_cols<N, false>, smem);
    { LaunchScope ls_(label<N>("fwd"), st);
    k_fft_cols<N, false><<<grid, FFTConf<N>::T * W, smem, st>>>(data, slab_stride, row_stride, ncols, tw); }
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

#define COLA_FOR_SIZES(X) \
  X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048)

bool fft_size_supported(int n) {
  switch (n) {
#define X(N) case N:
    COLA_FOR_SIZES(X)
#undef X
    return true;
    default:
      return false;
  }
}

int launch_fft_x_r2c(int n, const float* in, float2* out, int64_t nrows, int P, const float2* tw, cudaStream_t st) {
  switch (n) {
#define X(N) \
  case N:    \
    return x_r2c<N>(in, out, nrows, P, tw, st);
    COLA_FOR_SIZES(X)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "fft: unsupported length " + std::to_string(n));
  }
}

int launch_fft_x_c2r(int n, const float2* in, float* out, int64_t nrows, int P, const float2* tw, float scale,
                     cudaStream_t st) {
  switch (n) {
#define X(N) \
  case N:    \
    return x_c2r<N>(in, out, nrows, P, tw, scale, st);
    COLA_FOR_SIZES(X)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "fft: unsupported length " + std::to_string(n));
  }
}

int launch_fft_cols(int n, bool inverse, float2* data, int64_t nslabs, int64_t slab_stride, int64_t row_stride,
                    int ncols, const float2* tw, cudaStream_t st) {
  switch (n) {
#define X(N) \
  case N:    \
    return cols<N>(inverse, data, nslabs, slab_stride, row_stride, ncols, tw, st);
    COLA_FOR_SIZES(X)
#undef X
    default:
      return fail(COLA_EUNSUPPORTED, "fft: unsupported length " + std::to_string(n));
  }
}

int fft3d_r2c(int n, int P, const float* in, float2* out, const float2* tw, cudaStream_t st) {
  const int64_t nn = n;
  int rc = launch_fft_x_r2c(n, in, out, nn * nn, P, tw, st);
  if (rc) return rc;
  rc = launch_fft_cols(n, false, out, nn, nn * P, P, n / 2 + 1, tw, st);  // y: slab = z
  if (rc) return rc;
  return launch_fft_cols(n, false, out, nn, P, nn * P, n / 2 + 1, tw, st);  // z: slab = y
}

int fft3d_c2r(int n, int P, float2* in, float* out, const float2* tw, float scale, cudaStream_t st) {
  const int64_t nn = n;
  int rc = launch_fft_cols(n, true, in, nn, P, nn * P, n / 2 + 1, tw, st);  // z
  if (rc) return rc;
  rc = launch_fft_cols(n, true, in, nn, nn * P, P, n / 2 + 1, tw, st);  // y
  if (rc) return rc;
  return launch_fft_x_c2r(n, in, out, nn * nn, P, tw, scale, st);
}

}  // namespace cola
