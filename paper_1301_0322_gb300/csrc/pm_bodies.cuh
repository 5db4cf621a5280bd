// Device bodies of the mesh passes, shared by the single-box kernels and the multi-box
// (ensemble) kernels.  Each body processes one block's share of work given by explicit block
// indices and shared-memory pointers, so that a persistent kernel can run the bodies of
// different boxes (and mesh sizes) one after another.
#pragma once
#include "cola_internal.cuh"
#include "fft.cuh"
#include "pm_common.cuh"
#include "tma.cuh"

namespace cola {

// ---- helpers -----------------------------------------------------------------------------
__device__ __forceinline__ float sinc_pi_f(int n, int ng) {
  if (n == 0) return 1.0f;
  const float x = (float)n / (float)ng;
  return sinpif(x) / (3.14159265358979323846f * x);
}
__device__ __forceinline__ int signed_mode(int k, int n) { return k < n / 2 ? k : k - n; }

// first-derivative factor i k_j (zero on the Nyquist plane |n_j| = N/2)
__device__ __forceinline__ float2 mul_ik(float2 a, float k) { return make_float2(__fmul_rn(-k, a.y), __fmul_rn(k, a.x)); }

// columns per block of the strided passes (16 columns = 128 contiguous bytes per row); blocks
// of at most 256 threads (512 for the longest transforms) so that two blocks fit on an SM with
// every thread's E elements in registers, and one block's loads overlap the other's FFT
template <int N>
__host__ __device__ constexpr int col_width() {
  return FFTConf<N>::T * 16 <= 256 ? 16 : (FFTConf<N>::T * 8 <= 256 ? 8 : (FFTConf<N>::T * 4 <= 512 ? 4 : 2));
}

// row pitch (complex entries) of a half spectrum of an N^3 mesh: N/2 + 1 rounded up to a multiple
// of 4 (32-byte rows, the alignment the bulk copies need)
template <int N>
__host__ __device__ constexpr int half_pitch() {
  return ((N / 2 + 1) + 3) / 4 * 4;
}

// block (bx, slab): W columns of one slab of the in-place strided FFT (T(N) * W threads);
// smem: N W float2.  Element (n, col) at data[slab * slab_stride + n * row_stride + col].
// (tw: the base twiddle table or an SmemTw stage table)
template <int N, int W, bool INV, class C = FFTConf<N>, class TW>
__device__ __forceinline__ void cols_body(float2* __restrict__ data, int64_t slab_stride, int64_t row_stride,
                                          int ncols, const TW& tw, int bx, int slab, float2* smem) {
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int col = bx * W + w;
  const bool valid = col < ncols;
  float2* base = data + (int64_t)slab * slab_stride + (valid ? col : 0);
  auto load = [&](int n) -> float2 { return valid ? base[(int64_t)n * row_stride] : make_float2(0.f, 0.f); };
  auto mem = [&](int n) -> float2& { return smem[n * W + w]; };
  auto store = [&](int n, float2 x) {
    if (valid) base[(int64_t)n * row_stride] = x;
  };
  fft_1d<N, 1, INV, C>(t, tw, load, mem, store);
}

// ---- 1. deposit + x r2c -----------------------------------------------------------------------
// block: one tile of TY x TZ rows (T(N/2) * TY * TZ threads); acc: max(TY TZ N, TY TZ LD) x 8
// bytes of shared memory (the cells' low 32-bit words, then their high words; afterwards the
// rows' transform buffers); ints: 28 ints of shared memory
// rec: the bin-ordered particle records (fixed-point CIC coordinates; offsets index them directly)
// (stw: the row transform's stage twiddles, the base table tw or an SmemTw table)
template <int N, int TY, int TZ, class CM = FFTConf<N / 2>, class STW>
__device__ __forceinline__ void deposit_fftx_body(const Geometry& g, const Tiles& tl, const uint4* __restrict__ rec,
                                                  const int* __restrict__ offsets, float2* __restrict__ out, int P,
                                                  const float2* __restrict__ tw, const STW& stw, float dscale,
                                                  int* __restrict__ err, int tile, unsigned long long* acc,
                                                  int* ints) {
  constexpr int M = N / 2, T = CM::T, ROWS = TY * TZ, LD = xrow_ld<M>(), NT = T * ROWS, R0 = first_radix<CM>();
  int* rbeg = ints;
  int* rpre = ints + 9;
  int* rlen = ints + 19;
  int tyi, tzi;
  tile_of_bin(tl, tile, tyi, tzi);
  const int y0 = tyi * TY, z0 = tzi * TZ;
  for (int i = threadIdx.x; i < ROWS * N; i += NT) acc[i] = 0ull;
  // the tile's own 4 bins and the boundary bins of its 3 lower neighbours, loaded in parallel
  // (a loop: at N = 32 and 48 a block has only 8 threads)
  for (int k = threadIdx.x; k < 9; k += NT) {
    const int tym = tyi == 0 ? tl.nty - 1 : tyi - 1;
    const int tzm = tzi == 0 ? tl.ntz - 1 : tzi - 1;
    const int ty_ = (k == 4 || k == 5 || k == 8) ? tym : tyi;
    const int tz_ = k >= 6 ? tzm : tzi;
    const int reg = k < 4 ? k : ((k == 4 || k == 5) ? (k == 4 ? 1 : 3) : (k == 6 ? 2 : 3));
    const int b = tile_bin(tl, ty_, tz_) * 4 + reg;
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
  unsigned* lo = reinterpret_cast<unsigned*>(acc);
  unsigned* hi = lo + ROWS * N;
  constexpr int U = 4;  // particles in flight per thread
  const uint32_t fmask = (uint32_t)one - 1u;
  for (int base = threadIdx.x; base < total; base += NT * U) {
    uint32_t f[U][3];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * NT;
      ok[u] = i < total;
      if (ok[u]) {
        int r = 0;
#pragma unroll
        for (int k = 1; k < 9; ++k) r += (i >= rpre[k]) ? 1 : 0;
        const uint4 q = __ldg(rec + rbeg[r] + (i - rpre[r]));
        f[u][0] = q.x;
        f[u][1] = q.y;
        f[u][2] = q.z;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int cx = (int)(f[u][0] >> g.fbits), tx = (int)(f[u][0] & fmask);
      const int cy = (int)(f[u][1] >> g.fbits), ty = (int)(f[u][1] & fmask);
      const int cz = (int)(f[u][2] >> g.fbits), tz = (int)(f[u][2] & fmask);
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
          const int row = (lz * TY + ly) * N;
          acc_add64(lo, hi, row + cx, wzy * wx0);
          acc_add64(lo, hi, row + cx1, wzy * wx1);
        }
      }
    }
  }
  __syncthreads();
  // real-to-complex FFT of each tile row; z[n] = (delta[2n], delta[2n+1]).  The transform
  // buffers overlay the accumulators: fft_1d reads all its inputs before a block barrier
  // that precedes its first shared-memory write.
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  const uint2* lrow = reinterpret_cast<const uint2*>(lo + w * N);
  const uint2* hrow = reinterpret_cast<const uint2*>(hi + w * N);
  float2* buf = reinterpret_cast<float2*>(acc) + w * LD;
  bool overflow = false;
  auto load = [&](int n) -> float2 {
    const uint2 l = lrow[n], h = hrow[n];
    overflow |= ((h.x | h.y) >> 30) != 0u;
    const unsigned long long a = ((unsigned long long)h.x << 32) | l.x;
    const unsigned long long b = ((unsigned long long)h.y << 32) | l.y;
    return make_float2(fmaf(u64_to_f32_rn(a), dscale, -1.0f), fmaf(u64_to_f32_rn(b), dscale, -1.0f));
  };
  auto mem = [&](int n) -> float2& { return buf[xpad<R0>(n)]; };
  auto store = [&](int n, float2 x) { buf[xpad<R0>(n)] = x; };
  fft_1d<M, 2, false, CM>(t, stw, load, mem, store);
  if (overflow) atomicOr(err, kErrOverflow);
  __syncthreads();
  const int lz = w / TY, ly = w - lz * TY;
  float2* dst = out + ((int64_t)(z0 + lz) * N + (y0 + ly)) * P;
  // X[k] and X[M - k] from one pair Z[k], Z[M - k]: with e = (Z[k] + conj Z[M - k]) / 2,
  // d = (Z[k] - conj Z[M - k]) / 2 and p = W^k (-i d), X[k] = e + p and X[M - k] = conj(e - p)
  // (as W^(M - k) = -conj W^k); k = 0 gives X[0] and X[M] from Z[0]
  for (int k = t; k <= M / 2; k += T) {
    const float2 a = buf[xpad<R0>(k)];
    const float2 b = c_conj(buf[xpad<R0>(k == 0 ? 0 : M - k)]);
    const float2 e = c_scale(c_add(a, b), 0.5f);
    const float2 d = c_scale(c_sub(a, b), 0.5f);
    const float2 p = c_mul(__ldg(tw + k), make_float2(d.y, -d.x));
    dst[k] = c_add(e, p);
    if (2 * k != M) dst[M - k] = c_conj(c_sub(e, p));
  }
}

// ---- 3. z pass with the Green's function ------------------------------------------------------------
// block (bx, ky): W columns kx of the slab ky (T(N) * W threads); sm: 2 N W float2
// (stw: the stage twiddles, the base table tw or an SmemTw table)
template <int N, int W, class C = FFTConf<N>, class STW>
__device__ __forceinline__ void z_green_body(float2* __restrict__ A, float2* __restrict__ Gz, int P, float kf,
                                             int deconv, float norm, const STW& stw, int bx, int ky, float2* sm) {
  constexpr int nh = N / 2 + 1, NT = C::T * W;
  float2* S0 = sm;           // delta_k of the slab, [n][W]
  float2* S1 = sm + N * W;   // exchange buffer
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = bx * W + w;
  const bool valid = kx < nh;
  const int64_t zstride = (int64_t)N * P;
  float2* a = A + (int64_t)ky * P + (valid ? kx : 0);
  float2* gz = Gz + (int64_t)ky * P + (valid ? kx : 0);
  auto mem = [&](int n) -> float2& { return S1[n * W + w]; };
  {
    auto load = [&](int n) -> float2 { return valid ? a[n * zstride] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) { S0[n * W + w] = x; };
    fft_1d<N, 1, false, C>(t, stw, load, mem, store);
  }
  // sinc^2 tables of the z index and of the block's W columns, then
  // phi_k = delta_k norm / (k^2 W(k)^p) in place in S0 with one division per mode
  float* sz2 = reinterpret_cast<float*>(S1);  // S1 is free between the transforms
  float* sx2 = sz2 + N;
  for (int n = threadIdx.x; n < N + W; n += NT) {
    const float sv = n < N ? sinc_pi_f(signed_mode(n, N), N) : sinc_pi_f(bx * W + (n - N), N);
    (n < N ? sz2[n] : sx2[n - N]) = sv * sv;
  }
  __syncthreads();
  {
    const int ny = signed_mode(ky, N);
    const float sy = sinc_pi_f(ny, N);
    const float wy = sy * sy;
    const float kf2 = kf * kf;
    for (int i = threadIdx.x; i < N * W; i += NT) {
      const int n = i / W, c = i - n * W;
      const int nx = bx * W + c;
      const int nz = signed_mode(n, N);
      const int m2 = nx * nx + ny * ny + nz * nz;
      float gk = 0.0f;
      if (m2 != 0 && nx < nh) {
        float den = kf2 * (float)m2;
        if (deconv) {
          const float wk = sx2[c] * wy * sz2[n];
          den *= deconv == 2 ? wk * wk : wk;
        }
        gk = __fdividef(norm, den);  // fast reciprocal: <= 2 ulp, far below the transforms' rounding
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
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 {
      const float kz = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return mul_ik(S0[n * W + w], kz);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gz[n * zstride] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
}

// ---- 4. inverse y passes ------------------------------------------------------------------------------------
// block (bx, z): W columns kx of the slab z (T(N) * W threads); sm: 2 N W float2
template <int N, int W, class C = FFTConf<N>, class STW>
__device__ __forceinline__ void y_inv3_body(float2* __restrict__ B, float2* __restrict__ Gy, float2* __restrict__ Gz,
                                            int P, float kf, const STW& stw, int bx, int z, float2* sm) {
  constexpr int nh = N / 2 + 1, T = C::T;
  float2* S0 = sm;
  float2* S1 = sm + N * W;
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = bx * W + w;
  const bool valid = kx < nh;
  const int64_t slab = (int64_t)z * N * P + (valid ? kx : 0);
  float2* b = B + slab;
  float2* gy = Gy + slab;
  float2* gz = Gz + slab;
  // the Gz strip is read only by the third transform: start pulling it into L2 now
  if (w == 0)
    for (int n = t; n < N; n += T) prefetch_l2_line(Gz + (int64_t)z * N * P + bx * W + (int64_t)n * P);
  for (int n = t; n < N; n += T) S0[n * W + w] = valid ? b[(int64_t)n * P] : make_float2(0.f, 0.f);
  __syncthreads();
  auto mem = [&](int n) -> float2& { return S1[n * W + w]; };
  {
    auto load = [&](int n) -> float2 { return S0[n * W + w]; };
    auto store = [&](int n, float2 x) {
      if (valid) b[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 {
      const float ky = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return mul_ik(S0[n * W + w], ky);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gy[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 { return valid ? gz[(int64_t)n * P] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      if (valid) gz[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
}

// ---- 3'/4'. single-buffer (wide-strip) variants of the z and inverse y passes ------------------------------
// For long columns the two-buffer bodies above leave room for only narrow strips (4 columns =
// 32-byte row segments at N = 2048).  These variants keep one exchange buffer of N x W complex
// and re-read their input strip from global memory (an L2 hit) for each transform instead of
// holding it in shared memory, so the strips can be twice as wide.
//
// z pass: forward transform of the strip, phi = delta_k norm / (k^2 W(k)^p) written back to A in
// the forward transform's last stage, then the inverse transforms of i k_z phi (-> Gz) and of phi
// (-> A, in place).  block (bx, ky): W columns kx of the slab ky (T(N) * W threads);
// sm: N W float2 + (N + W) floats (sinc^2 tables).
// shared-memory layout of the wide z pass: strip (N W float2), sinc^2 tables (N + W floats,
// rounded up to 16 bytes), stage twiddle table
template <int N, int W>
__host__ __device__ constexpr int wide_z_table_offset() {
  return N * W + (N + W + 3) / 4 * 2;
}
// scratch slots of the wide z pass (one per SM id, N W float2 each)
constexpr int kZScratchSlots = 512;

// z pass with the Green's function, one exchange buffer.  With KS > 0 scratch slots per SM the
// forward transform of the strip (Green's function applied as it is stored) goes to a slot of
// this SM, contiguous [n][w], and the inverse transforms of i k_z phi (-> Gz) and of phi (-> A)
// read it back from L2 as whole 128-byte lines (the strip itself spans N rows N (N/2+1) 8 bytes
// apart: 16.8 MB at N = 2048).  KS = 1: one block fits per SM (shared memory), so the slot of
// %smid is the block's own while it runs; KS > 1: a block claims one of its SM's KS slots
// (compare-and-swap on busy[], a bounded number of rounds) and frees it when it is done, KS
// being above the blocks that fit on an SM.  KS = 0: phi goes to A and the inverse transforms
// read it back from there (an L2 hit).
// block (bx, ky): W columns kx of the slab ky (T(N) W threads); scratch: kZScratchSlots KS N W
// float2; busy: kZScratchSlots KS ints, zero between launches
template <int N, int W, int KS, class C = FFTConf<N>>
__device__ __forceinline__ void z_green_wide_body(float2* __restrict__ A, float2* __restrict__ Gz,
                                                  float2* __restrict__ scratch, int* __restrict__ busy, float kf,
                                                  int deconv, float norm, const float2* __restrict__ tw,
                                                  int* __restrict__ err, int bx, int ky, float2* sm) {
  constexpr int nh = N / 2 + 1, NT = C::T * W, P = half_pitch<N>();
  constexpr bool SCRATCH = KS > 0;
  float2* sc = nullptr;
  int* my_flag = nullptr;
  if constexpr (SCRATCH) {
    unsigned smid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    if (nsmid > (unsigned)kZScratchSlots) {
      if (threadIdx.x == 0) atomicOr(err, kErrSmIds);
      return;
    }
    int slot = (int)smid * KS;
    if constexpr (KS > 1) {
      __shared__ int claimed;
      if (threadIdx.x == 0) {
        int got = -1;
        for (int round = 0; round < 1024 && got < 0; ++round)
          for (int k = 0; k < KS && got < 0; ++k)
            if (atomicCAS(busy + slot + k, 0, 1) == 0) got = k;
        claimed = got;
      }
      __syncthreads();
      if (claimed < 0) {
        if (threadIdx.x == 0) atomicOr(err, kErrSmIds);
        return;
      }
      slot += claimed;
      my_flag = busy + slot;
    }
    sc = scratch + (int64_t)slot * (N * W);
  }
  float2* S = sm;
  float* sz2 = reinterpret_cast<float*>(sm + N * W);
  float* sx2 = sz2 + N;
  float2* stab = sm + wide_z_table_offset<N, W>();
  stw_fill<C, 1>(stab, tw, threadIdx.x, NT);
  const SmemTw<C> stw{stab};
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = bx * W + w;
  const bool valid = kx < nh;
  constexpr int64_t zstride = (int64_t)N * P;
  float2* a = A + (int64_t)ky * P + (valid ? kx : 0);
  float2* gz = Gz + (int64_t)ky * P + (valid ? kx : 0);
  for (int n = threadIdx.x; n < N + W; n += NT) {
    const float sv = n < N ? sinc_pi_f(signed_mode(n, N), N) : sinc_pi_f(bx * W + (n - N), N);
    (n < N ? sz2[n] : sx2[n - N]) = sv * sv;
  }
  if constexpr (SCRATCH) {
    // the slot still holds the previous block's strip, dead now: drop its lines from L2 rather
    // than let them be written back (the barrier orders this before the slot's new writes)
    for (int l = threadIdx.x; l < N * W * (int)sizeof(float2) / 128; l += NT)
      discard_l2_line(reinterpret_cast<char*>(sc) + 128 * l);
  }
  __syncthreads();
  // phi of element n of this thread's column: where the forward transform leaves it
  auto phi_at = [&](int n) -> float2* { return SCRATCH ? sc + n * W + w : a + n * zstride; };
  auto mem = [&](int n) -> float2& { return S[n * W + w]; };
  {
    const int ny = signed_mode(ky, N);
    const float sy = sinc_pi_f(ny, N);
    const float wy = sy * sy;
    const float kf2 = kf * kf;
    auto load = [&](int n) -> float2 { return valid ? a[n * zstride] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      const int nz = signed_mode(n, N);
      const int m2 = kx * kx + ny * ny + nz * nz;
      float gk = 0.0f;
      if (m2 != 0) {
        float den = kf2 * (float)m2;
        if (deconv) {
          const float wk = sx2[w] * wy * sz2[n];
          den *= deconv == 2 ? wk * wk : wk;
        }
        gk = __fdividef(norm, den);
      }
      if (SCRATCH || valid) __stcg(phi_at(n), c_scale(x, gk));
    };
    fft_1d<N, 1, false, C>(t, stw, load, mem, store);
  }
  __syncthreads();  // phi of the strip is in the scratch slot or in A (visible to the block after the barrier)
  {
    auto load = [&](int n) -> float2 {
      const float kz = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return (SCRATCH || valid) ? mul_ik(__ldcg(phi_at(n)), kz) : make_float2(0.f, 0.f);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gz[n * zstride] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 { return (SCRATCH || valid) ? __ldcg(phi_at(n)) : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      if (valid) a[n * zstride] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  if constexpr (KS > 1) {
    __syncthreads();  // every read of the slot is done: free it (the exchange returns when done)
    if (threadIdx.x == 0) atomicExch(my_flag, 0);
  }
}

// inverse y passes, one exchange buffer: Gy = IFFT_y(i k_y B), then B = IFFT_y(B) in place (the
// strip of B read again, from L2), then Gz = IFFT_y(Gz).  block (bx, z): W columns kx of the slab
// z (T(N) * W threads); sm: N W float2
template <int N, int W, class C = FFTConf<N>>
__device__ __forceinline__ void y_inv3_wide_body(float2* __restrict__ B, float2* __restrict__ Gy,
                                                 float2* __restrict__ Gz, float kf, const float2* __restrict__ tw,
                                                 int bx, int z, float2* sm) {
  constexpr int nh = N / 2 + 1, T = C::T, P = half_pitch<N>();
  float2* stab = sm + N * W;
  stw_fill<C, 1>(stab, tw, threadIdx.x, T * W);
  const SmemTw<C> stw{stab};
  const int w = threadIdx.x % W, t = threadIdx.x / W;
  const int kx = bx * W + w;
  const bool valid = kx < nh;
  const int64_t slab = (int64_t)z * N * P + (valid ? kx : 0);
  float2* b = B + slab;
  float2* gy = Gy + slab;
  float2* gz = Gz + slab;
  // the Gz strip is read only by the third transform: start pulling it into L2 now
  if (w == 0)
    for (int n = t; n < N; n += T) prefetch_l2_line(Gz + (int64_t)z * N * P + bx * W + (int64_t)n * P);
  auto mem = [&](int n) -> float2& { return sm[n * W + w]; };
  {
    auto load = [&](int n) -> float2 {
      const float ky = (n == N / 2) ? 0.0f : kf * (float)signed_mode(n, N);
      return valid ? mul_ik(b[(int64_t)n * P], ky) : make_float2(0.f, 0.f);
    };
    auto store = [&](int n, float2 x) {
      if (valid) gy[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 { return valid ? b[(int64_t)n * P] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      if (valid) b[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
  {
    auto load = [&](int n) -> float2 { return valid ? gz[(int64_t)n * P] : make_float2(0.f, 0.f); };
    auto store = [&](int n, float2 x) {
      if (valid) gz[(int64_t)n * P] = x;
    };
    fft_1d<N, 1, true, C>(t, stw, load, mem, store);
  }
}

// ---- 5. inverse x passes of the three components -------------------------------------------------------------
// Work item: RB consecutive rows of one component (C, Gy or Gz; P complex per row).  The rows
// arrive in shared memory by bulk copy (TMA) at pitch LD = xrow_ld(N/2) while the block
// computes the previous item; the first FFT stage reads them there, and later stages reuse
// the same rows as their exchange buffer (the first stage has read all its inputs by then).
template <int N>
__host__ __device__ constexpr int c2r3_rows() {
  return FFTConf<N / 2>::T >= 128 ? 1 : 128 / FFTConf<N / 2>::T;
}

// Called by the 32 threads of warp 0: lane 0 registers the bytes on `bar`, lanes < rb copy one
// row each (P complex; P is a multiple of 4, so every row is a multiple of 32 bytes).
__device__ __forceinline__ void c2r3_issue(float2* stage, const float2* src_rows, int rb, int P, int LD,
                                           uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  fence_proxy_async_smem();
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)rb * (uint32_t)P * 8u);
  __syncwarp();
  for (int w = lane; w < rb; w += 32) bulk_copy_g2s(stage + w * LD, src_rows + (int64_t)w * P, (uint32_t)P * 8u, bar);
}

// Inverse x transform of the staged rows into F rows (pitch N floats); comp 0 applies i k_x.
// tw: the base twiddle table; stw: the stage twiddles (the base table or an SmemTw table)
template <int N, int RB, class CM = FFTConf<N / 2>, class STW>
__device__ __forceinline__ void c2r3_compute(float2* stage, float* __restrict__ Frows, int comp, float kf,
                                             const float2* __restrict__ tw, const STW& stw) {
  constexpr int M = N / 2, T = CM::T, LD = xrow_ld<M>(), R0 = first_radix<CM>();
  static_assert(T * RB <= 1024, "block too large");
  const int t = threadIdx.x % T, w = threadIdx.x / T;
  float2* buf = stage + w * LD;
  auto X = [&](int k) -> float2 {
    const float2 x = buf[k];
    return comp == 0 ? mul_ik(x, k == M ? 0.0f : kf * (float)k) : x;
  };
  auto load = [&](int n) -> float2 {
    const float2 a = X(n), bb = c_conj(X(M - n));
    const float2 e = c_add(a, bb);
    const float2 o = c_mul(c_sub(a, bb), c_conj(__ldg(tw + n)));
    return make_float2(__fsub_rn(e.x, o.y), __fadd_rn(e.y, o.x));
  };
  auto mem = [&](int n) -> float2& { return buf[xpad<R0>(n)]; };
  float2* dst = reinterpret_cast<float2*>(Frows + (int64_t)w * N);
  auto store = [&](int n, float2 x) { dst[n] = x; };
  fft_1d<M, 2, true, CM>(t, stw, load, mem, store);
}
template <int N, int RB, class CM = FFTConf<N / 2>>
__device__ __forceinline__ void c2r3_compute(float2* stage, float* __restrict__ Frows, int comp, float kf,
                                             const float2* __restrict__ tw) {
  c2r3_compute<N, RB, CM>(stage, Frows, comp, kf, tw, tw);
}

}  // namespace cola
