// Ensembles of independent COLA boxes of different sizes (the many-realisation use of Sec. 1
// and Sec. 4) evolved together: one launch per kernel class per force evaluation for all
// boxes, each launch a persistent kernel whose blocks walk a work list of (box, item) pairs.
//
// Each box keeps a full single-box plan (its coefficient table, twiddles and mesh buffers);
// the ensemble adds a description of every box for the device, the shared particle-sort
// buffers and the work lists.  The bins of all boxes form one array (box b's bins start at
// bin_base), so one scan serves every box, and box b's bin-ordered particle records land in
// positions [poff[b], poff[b+1]) of the shared record array.
//
// One step (eq. ALCtimestep) = keys, 3 scan phases, scatter, deposit + x r2c, y pass, z pass
// with the Green's function, inverse y passes, inverse x passes, gather in bin order, kick +
// drift: 12 launches for the whole ensemble, recorded once per step as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cola_internal.cuh"
#include "particle_bodies.cuh"
#include "pm_bodies.cuh"

namespace cola {

#define COLA_ENS_SIZES(X) X(64) X(96) X(128) X(192) X(256)

// per-box description read by the ensemble kernels
struct BoxDesc {
  Geometry g;
  Tiles tl;
  int P, deconv, bin_base, c2r_rb;  // c2r_rb: rows per inverse-x work item
  float kf, norm, dscale;
  int c2r_ld;                        // row pitch (complex) of the staged inverse-x rows
  int64_t pbase;            // first particle of the box in the ensemble arrays
  float2* A;                // half spectrum [ng][ng][P]
  float2* Gy;
  float2* Gz;
  float* F;                 // force meshes [3][ng^3]
  const float2* tw;         // exp(-2 pi i m / ng)
  const float* coef;        // (nsteps + 1) x kCoef32
  int* err;
};

// work lists: particles (one per thread), particles four per thread, deposit tiles, column
// strips, inverse-x row blocks
enum { kEParticles, kEParticles4, kEDeposit, kECols, kEC2r, kENumLists };
enum { kKKeys, kKScatter, kKDeposit, kKYfwd, kKZgreen, kKYinv, kKC2r, kKGather, kKGatherB, kKKick, kKNum };

constexpr int kEnsMaxBoxes = 4096;

namespace {

// largest b with starts[b] <= item (starts ascending, starts[0] = 0)
__device__ __forceinline__ int find_box(const int* __restrict__ starts, int nbox, int item) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(starts + mid) <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The box of the items a block walks (blockIdx.x, + gridDim.x, ...): found once by bisection,
// then moved forward, as the items only increase (a bisection per item costs a chain of
// dependent loads every time).
struct BoxCursor {
  int b, first, end;  // box, its first item, one past its last
  __device__ __forceinline__ BoxCursor(const int* __restrict__ starts, int nbox, int item) {
    b = item < __ldg(starts + nbox) ? find_box(starts, nbox, item) : 0;
    first = __ldg(starts + b);
    end = __ldg(starts + b + 1);
  }
  // box of `item` (item >= every item passed before, item < the total)
  __device__ __forceinline__ int operator()(const int* __restrict__ starts, int item) {
    while (item >= end) {
      ++b;
      first = end;
      end = __ldg(starts + b + 1);
    }
    return b;
  }
};

// position of mesh size n in COLA_ENS_SIZES
__host__ __device__ constexpr int ens_size_index(int n) {
  return n == 64 ? 0 : n == 96 ? 1 : n == 128 ? 2 : n == 192 ? 3 : 4;
}

// rows of a deposit tile (y) for a tile of `rows` rows and its two shapes (tile_shape 0 / 1):
// 8 -> 4x2 / 2x4, 16 -> 4x4 / 8x2, 32 -> 8x4 / 4x8, 64 -> 8x8 / 16x4, 128 -> 16x8 / 8x16
__host__ __device__ constexpr int ens_tile_ty(int rows, int shape) {
  return rows == 8 ? (shape == 0 ? 4 : 2)
                   : rows == 16 ? (shape == 0 ? 4 : 8)
                                : rows == 32 ? (shape == 0 ? 8 : 4) : rows == 64 ? (shape == 0 ? 8 : 16) : (shape == 0 ? 16 : 8);
}

// ---- persistent kernels -----------------------------------------------------------------------
// Each kernel walks the items of all boxes: boxes[0 .. nbox), item list starts[0 .. nbox].

// binning, four particles per thread (keys_x4_body, scatter_x4_body)
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ke_keys(const BoxDesc* __restrict__ boxes, const int* __restrict__ starts,
                                              int nbox, const float* __restrict__ s, int* __restrict__ keys,
                                              int* __restrict__ counts) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int64_t q0 = (int64_t)(item - cur.first) * NT * kPartPerThread;
    keys_x4_body(d.g, d.tl, s + 3 * d.pbase, q0, d.bin_base, keys + d.pbase, counts, d.err);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ke_scatter(const BoxDesc* __restrict__ boxes,
                                                           const int* __restrict__ starts, int nbox,
                                                           const float* __restrict__ s, const int* __restrict__ keys,
                                                           int* __restrict__ cursor, uint4* __restrict__ rec) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int64_t q0 = (int64_t)(item - cur.first) * NT * kPartPerThread;
    scatter_x4_body(d.g, s + 3 * d.pbase, q0, keys + d.pbase, cursor, rec);
  }
}

// One tile of one box.  Not inlined: every (size, tile) instantiation gets its own register
// allocation instead of the union of all of them.
template <int N, int TY, int TZ, class CM>
__device__ __noinline__ void deposit_tile(const BoxDesc* __restrict__ d, const uint4* __restrict__ rec,
                                          const int* __restrict__ offsets, int tile) {
  extern __shared__ __align__(16) unsigned long long ens_smem[];
  __shared__ int ints[28];
  deposit_fftx_body<N, TY, TZ, CM>(d->g, d->tl, rec, offsets, d->A, d->P, d->tw, d->tw, d->dscale, d->err, tile, ens_smem,
                                   ints);
}

template <int N, int NT, int V>
__device__ __forceinline__ void deposit_item(const BoxDesc* d, const uint4* rec, const int* offsets, int tile) {
  using CM = FFTConfV<N / 2, V>;
  constexpr int ROWS = NT / CM::T;
  constexpr int TY0 = ens_tile_ty(ROWS, 0), TY1 = ens_tile_ty(ROWS, 1);
  if (d->tl.ty == TY0)
    deposit_tile<N, TY0, ROWS / TY0, CM>(d, rec, offsets, tile);
  else
    deposit_tile<N, TY1, ROWS / TY1, CM>(d, rec, offsets, tile);
}

template <int NT, int V>
__global__ void __launch_bounds__(NT, 512 / NT) ke_deposit(const BoxDesc* __restrict__ boxes,
                                                           const int* __restrict__ starts, int nbox,
                                                           const uint4* __restrict__ rec,
                                                           const int* __restrict__ offsets) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc* d = boxes + b;
    const int local = item - cur.first;
    const int* ob = offsets + d->bin_base;
    switch (d->g.ng) {
#define X(N)                                              \
  case N:                                                 \
    deposit_item<N, NT, V>(d, rec, ob, local);            \
    break;
      COLA_ENS_SIZES(X)
#undef X
      default:
        break;
    }
    __syncthreads();
  }
}

// column passes: kind 0 = forward y, 1 = z with the Green's function, 2 = inverse y (three
// outputs); single-buffer strips of W = NT / T(N) columns, stage twiddles from shared memory
// (the bodies of the single-box passes at 128-256; the z pass keeps phi in A)
template <int NT, int KIND, int V>
__global__ void __launch_bounds__(NT, 512 / NT) ke_cols(const BoxDesc* __restrict__ boxes, const int* __restrict__ starts,
                                              int nbox) {
  extern __shared__ __align__(16) unsigned long long ens_smem[];
  float2* sm = reinterpret_cast<float2*>(ens_smem);
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int local = item - cur.first;
    switch (d.g.ng) {
#define X(N)                                                                                              \
  case N: {                                                                                               \
    using C = FFTConfV<N, V>;                                                                             \
    constexpr int W = NT / C::T, nbx = (N / 2 + 1 + W - 1) / W;                                           \
    const int bx = local % nbx, slab = local / nbx;                                                       \
    if (KIND == 0) {                                                                                      \
      float2* stab = sm + N * W;                                                                          \
      stw_fill<C, 1>(stab, d.tw, threadIdx.x, NT);                                                        \
      cols_body<N, W, false, C>(d.A, (int64_t)N * d.P, d.P, N / 2 + 1, SmemTw<C>{stab}, bx, slab, sm);    \
    } else if (KIND == 1) {                                                                               \
      z_green_wide_body<N, W, 0, C>(d.A, d.Gz, nullptr, nullptr, d.kf, d.deconv, d.norm, d.tw, d.err, bx, \
                                    slab, sm);                                                            \
    } else {                                                                                              \
      y_inv3_wide_body<N, W, C>(d.A, d.Gy, d.Gz, d.kf, d.tw, bx, slab, sm);                               \
    }                                                                                                     \
  } break;
      COLA_ENS_SIZES(X)
#undef X
      default:
        break;
    }
    __syncthreads();
  }
}

// Stage twiddle tables (fft.cuh) of the inverse-x transforms of every ensemble size, behind the
// two stage buffers of ke_c2r3: ens_c2r_tab_offset(n) float2 entries from their start.
constexpr int kEnsSizes[] = {64, 96, 128, 192, 256};
constexpr int kEnsNumSizes = 5;
template <int V>
__host__ __device__ constexpr int ens_c2r_tab_size(int n) {
  return n == 64    ? stw_size<FFTConfV<32, V>>()
         : n == 96  ? stw_size<FFTConfV<48, V>>()
         : n == 128 ? stw_size<FFTConfV<64, V>>()
         : n == 192 ? stw_size<FFTConfV<96, V>>()
                    : stw_size<FFTConfV<128, V>>();
}
template <int V>
__host__ __device__ constexpr int ens_c2r_tab_offset(int n) {
  int off = 0;
  for (int k = 0; k < kEnsNumSizes && kEnsSizes[k] != n; ++k) off += ens_c2r_tab_size<V>(kEnsSizes[k]);
  return off;
}
// base twiddle table of a box of each size (nullptr: no box of that size)
struct EnsTw {
  const float2* tw[kEnsNumSizes];
};

// Inverse x passes of all boxes: persistent, with the bulk copy of the next item (which may
// belong to another box and mesh size) in flight during the transform of the current one.
// half: float2 capacity of each of the two stage buffers.
template <int NT, int V>
__global__ void __launch_bounds__(NT, 512 / NT) ke_c2r3(const BoxDesc* __restrict__ boxes,
                                                        const int* __restrict__ starts, int nbox, int half, EnsTw tws,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned long long ens_smem[];
  float2* sm = reinterpret_cast<float2*>(ens_smem);
  float2* tabs = sm + 2 * half;
  __shared__ __align__(8) uint64_t bars[2];
  const int total = __ldg(starts + nbox);
#define X(N)                                                                                                   \
  if (tws.tw[ens_size_index(N)])                                                                             \
    stw_fill<FFTConfV<N / 2, V>, 2>(tabs + ens_c2r_tab_offset<V>(N), tws.tw[ens_size_index(N)], threadIdx.x, NT);
  COLA_ENS_SIZES(X)
#undef X
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  BoxCursor icur(starts, nbox, blockIdx.x), cur(starts, nbox, blockIdx.x);  // items issued / computed
  auto issue = [&](int item, int buf) {
    const int b = icur(starts, item);
    const BoxDesc& d = boxes[b];
    const int local = item - icur.first;
    const int rb = d.c2r_rb, n = d.g.ng;
    const int nrb = n * n / rb;
    const int comp = local / nrb;
    const float2* m = comp == 0 ? d.A : (comp == 1 ? d.Gy : d.Gz);
    c2r3_issue(sm + buf * half, m + (int64_t)(local - comp * nrb) * rb * d.P, rb, d.P, d.c2r_ld, &bars[buf]);
  };
  int item = blockIdx.x;
  if (item < total && threadIdx.x < 32) issue(item, 0);
  for (int it = 0; item < total; ++it, item += gridDim.x) {
    const int buf = it & 1;
    const int next = item + gridDim.x;
    if (next < total && threadIdx.x < 32) issue(next, buf ^ 1);
    const bool ok = mbar_wait(&bars[buf], (it >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      // leave no bulk copy in flight into shared memory the block releases: wait again (bounded)
      // for the copy that timed out and for the next item's copy
      if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
      mbar_wait(&bars[buf], (it >> 1) & 1);
      if (next < total) mbar_wait(&bars[buf ^ 1], ((it + 1) >> 1) & 1);
      return;
    }
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int local = item - cur.first;
    switch (d.g.ng) {
#define X(N)                                                                                       \
  case N: {                                                                                        \
    using CM = FFTConfV<N / 2, V>;                                                                 \
    constexpr int RB = NT / CM::T, nrb = N * N / RB;                                               \
    const int comp = local / nrb;                                                                  \
    c2r3_compute<N, RB, CM>(sm + buf * half, d.F + (int64_t)comp * N * N * N + (int64_t)(local - comp * nrb) * RB * N, \
                            comp, d.kf, d.tw, SmemTw<CM>{tabs + ens_c2r_tab_offset<V>(N)});          \
  } break;
      COLA_ENS_SIZES(X)
#undef X
      default:
        break;
    }
    __syncthreads();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ke_gather(const BoxDesc* __restrict__ boxes, const int* __restrict__ starts,
                                                int nbox, float* __restrict__ s, float* __restrict__ v,
                                                const float* __restrict__ s1, const float* __restrict__ s2, int step,
                                                int mode) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int64_t p = (int64_t)(item - cur.first) * NT + threadIdx.x;
    if (p < d.g.np3) {
      const int64_t o = 3 * d.pbase;
      gather_kick_drift_body(d.g, d.F, s + o, v + o, s1 + o, s2 + o, d.coef + (size_t)step * kCoef32, mode, nullptr,
                             p);
    }
  }
}

// Gather in bin order into each box's half-spectrum buffers (free once its force meshes exist):
// the particles of box b hold bin positions pbase .. pbase + np^3 - 1 (the boxes' bins follow
// one another and every particle has one bin).
// f4: the forces go to A as one float4 per particle (every box's half spectrum holds 16 bytes per
// particle), else as three float arrays in A, Gy and Gz.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ke_gather_binned(const BoxDesc* __restrict__ boxes,
                                                                 const int* __restrict__ starts, int nbox,
                                                                 const uint4* __restrict__ rec, bool f4) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int64_t q = (int64_t)(item - cur.first) * NT + threadIdx.x;
    if (q < d.g.np3) {
      const uint4 r = __ldg(rec + d.pbase + q);
      const int64_t p = r.w;
      const uint32_t fmask = (1u << d.g.fbits) - 1u;
      const uint32_t fq[3] = {r.x, r.y, r.z};
      int c[3], t[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        c[k] = (int)(fq[k] >> d.g.fbits);
        t[k] = (int)(fq[k] & fmask);
      }
      float f[3];
      gather_force(d.g, d.F, c, t, f);
      if (f4) {
        reinterpret_cast<float4*>(d.A)[p] = make_float4(f[0], f[1], f[2], 0.0f);
      } else {
        reinterpret_cast<float*>(d.A)[p] = f[0];
        reinterpret_cast<float*>(d.Gy)[p] = f[1];
        reinterpret_cast<float*>(d.Gz)[p] = f[2];
      }
    }
  }
}

// Kick/drift in lattice order with the forces of ke_gather_binned.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ke_kick_drift(const BoxDesc* __restrict__ boxes,
                                                              const int* __restrict__ starts, int nbox,
                                                              float* __restrict__ s, float* __restrict__ v,
                                                              const float* __restrict__ s1,
                                                              const float* __restrict__ s2, int step, int mode,
                                                              bool f4) {
  const int total = __ldg(starts + nbox);
  BoxCursor cur(starts, nbox, blockIdx.x);
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int b = cur(starts, item);
    const BoxDesc& d = boxes[b];
    const int64_t p = (int64_t)(item - cur.first) * NT + threadIdx.x;
    if (p < d.g.np3) {
      const int64_t o = 3 * d.pbase;
      float f[3];
      if (f4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(d.A) + p);
        f[0] = q.x;
        f[1] = q.y;
        f[2] = q.z;
      } else {
        f[0] = reinterpret_cast<const float*>(d.A)[p];
        f[1] = reinterpret_cast<const float*>(d.Gy)[p];
        f[2] = reinterpret_cast<const float*>(d.Gz)[p];
      }
      kick_drift_update(d.g, s + o, v + o, s1 + o, s2 + o, d.coef + (size_t)step * kCoef32, mode, p, f);
    }
  }
}

// ---- host side ----------------------------------------------------------------------------------
// threads per transform of length n in radix variant v
int host_T(int n, int v) {
  switch (n) {
#define X(N) \
  case N:    \
    return v ? FFTConfV<N, 1>::T : FFTConfV<N, 0>::T;
    X(32) X(48) X(64) X(96) X(128) X(192) X(256)
#undef X
    default:
      return 0;
  }
}

bool ens_size_supported(int n) {
  switch (n) {
#define X(N) case N:
    COLA_ENS_SIZES(X)
#undef X
    return true;
    default:
      return false;
  }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Shape {
  int W, nbx, RB, rows, ty, tz;
};

Shape box_shape(int n, int nt, int tile_shape, int v) {
  Shape s{};
  s.W = nt / host_T(n, v);
  s.nbx = (n / 2 + 1 + s.W - 1) / s.W;
  s.RB = nt / host_T(n / 2, v);
  s.rows = s.RB;
  s.ty = ens_tile_ty(s.rows, tile_shape);
  s.tz = s.rows / s.ty;
  return s;
}

int xrow_ld_host(int m) { return ((m + 1 + ((m + 1) >> 3) + 1) + 15) / 16 * 16 + 8; }

}  // namespace
}  // namespace cola

using namespace cola;

struct cola_ensemble {
  std::vector<cola_plan*> plans;
  int nbox = 0, nsteps = 0, min_ng = 0;
  bool binned_gather = true;  // every box gathers in bin order (as its single-box plan does)
  bool gather_f4 = true;      // ... into one float4 per particle (as its single-box plan does)
  std::vector<int64_t> poff, moff;
  std::vector<size_t> plan_off;
  size_t ens_off = 0, ws_bytes = 0;
  int max_bins_total = 0;
  void* ws_base = nullptr;
  // shared device buffers
  int* keys = nullptr;
  uint4* rec = nullptr;  // [all particles] bin-ordered records (fixed-point coordinates, lattice index)
  int* counts = nullptr;
  int* offsets = nullptr;
  int* cursor = nullptr;
  int* scan_blocks = nullptr;
  BoxDesc* d_boxes = nullptr;
  int* d_starts = nullptr;
  // current launch configuration
  cola_ensemble_tuning tuning{256, 0, 0, 0, 0, 0};
  std::vector<BoxDesc> h_boxes;
  std::vector<int> h_starts;  // work list l at h_starts[l (nbox + 1)]
  int total_bins = 0;
  int grid[kKNum] = {};
  size_t smem[kKNum] = {};
  int c2r_half = 0;     // float2 capacity of each inverse-x stage buffer
  EnsTw tws{};
  int version = 0;
  int num_sms = 0;
  // graphs
  bool use_graphs = true;
  cudaStream_t cap = nullptr;
  // per-box work outside the step (noise, initial conditions, density, P(k)) runs on kForks
  // side streams forked from and joined back into the caller's (or the capture) stream
  static constexpr int kForks = 8;
  cudaStream_t side[kForks] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kForks] = {};
  struct Cached {
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;  // pointers and scalars the recorded launches baked in
    int version = -1;
    unsigned long long kernels = 0;
  };
  std::vector<Cached> graphs;  // one per step, then the noise, initial conditions, density, P(k)
  Profiler prof;

  ~cola_ensemble() {
    for (auto& c : graphs)
      if (c.exec) cudaGraphExecDestroy(c.exec);
    if (cap) cudaStreamDestroy(cap);
    for (int k = 0; k < kForks; ++k) {
      if (side[k]) cudaStreamDestroy(side[k]);
      if (join_ev[k]) cudaEventDestroy(join_ev[k]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (auto* p : plans) cola_plan_destroy(p);
  }
};

namespace cola {
namespace {

// multi-box binning, gather and kick around every box's own mesh passes on forked streams
bool hybrid(const cola_ensemble* e) { return e->tuning.launch == 0 && e->tuning.mesh_streams > 0; }

template <int NT, int V>
int kernel_attrs(cola_ensemble* e) {
  const void* fns[kKNum] = {(const void*)ke_keys<NT>,       (const void*)ke_scatter<NT>,
                            (const void*)ke_deposit<NT, V>, (const void*)ke_cols<NT, 0, V>,
                            (const void*)ke_cols<NT, 1, V>, (const void*)ke_cols<NT, 2, V>,
                            (const void*)ke_c2r3<NT, V>,    (const void*)ke_gather<NT>,
                            (const void*)ke_gather_binned<NT>, (const void*)ke_kick_drift<NT>};
  const int lists[kKNum] = {kEParticles4, kEParticles4, kEDeposit,   kECols,      kECols,
                            kECols,       kEC2r,        kEParticles, kEParticles, kEParticles};
  for (int k = 0; k < kKNum; ++k) {
    if (e->smem[k] > 227 * 1024) return fail(COLA_EUNSUPPORTED, "ensemble kernel: shared memory request too large");
    COLA_CUDA_CHECK(cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem[k]));
    int occ = 0;
    COLA_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[k], NT, e->smem[k]));
    if (occ < 1) return fail(COLA_EUNSUPPORTED, "ensemble kernel does not fit on an SM");
    const int per_sm = e->tuning.blocks_per_sm > 0 ? std::min(occ, (int)e->tuning.blocks_per_sm) : occ;
    const int items = e->h_starts[(size_t)lists[k] * (e->nbox + 1) + e->nbox];
    e->grid[k] = std::max(1, std::min(items, per_sm * e->num_sms));
  }
  return COLA_OK;
}

// stage twiddle table of an n-point column transform in radix variant v (float2 entries)
int ens_stw_size(int n, int v) {
  switch (n) {
#define X(N) \
  case N:    \
    return v ? stw_size<FFTConfV<N, 1>>() : stw_size<FFTConfV<N, 0>>();
    COLA_ENS_SIZES(X)
#undef X
    default:
      return 0;
  }
}

// inverse-x stage twiddle tables of every ensemble size (float2 entries)
int ens_c2r_tab_total(int v) {
  return v ? ens_c2r_tab_offset<1>(0) : ens_c2r_tab_offset<0>(0);
}

// (re)build the box descriptions, work lists and launch shapes for e->tuning
int configure(cola_ensemble* e, cudaStream_t st) {
  const int nt = e->tuning.threads;
  const int nb = e->nbox;
  e->h_boxes.assign(nb, BoxDesc{});
  std::vector<int64_t> items((size_t)nb * kENumLists);
  std::fill(e->smem, e->smem + kKNum, (size_t)0);
  size_t c2r_buf = 0;
  for (int k = 0; k < kEnsNumSizes; ++k) e->tws.tw[k] = nullptr;
  int bins = 0;
  for (int b = 0; b < nb; ++b) {
    cola_plan* p = e->plans[b];
    const int n = p->geo.ng;
    const Shape sh = box_shape(n, nt, e->tuning.tile_shape, e->tuning.radix);
    BoxDesc& d = e->h_boxes[b];
    d.g = p->geo;
    if ((sh.ty & (sh.ty - 1)) || (sh.tz & (sh.tz - 1)))
      return fail(COLA_EUNSUPPORTED, "ensemble: deposit tile sides must be powers of two");
    if (hybrid(e)) {
      d.tl = p->tiles;  // the box's own mesh passes read its bins in its plan's tile layout
    } else {
      d.tl.ty = sh.ty;
      d.tl.tz = sh.tz;
      d.tl.nty = n / sh.ty;
      d.tl.ntz = n / sh.tz;
      d.tl.nbins = d.tl.nty * d.tl.ntz * 4;
      d.tl.lband = tile_band_log2(d.tl.nty);
    }
    d.P = p->Pg;
    d.deconv = p->cfg.deconv;
    d.bin_base = bins;
    bins += d.tl.nbins;
    d.kf = (float)(2.0 * 3.14159265358979323846 / p->cfg.box);
    d.norm = (float)(1.0 / ((double)n * n * n));
    d.dscale = (float)((double)n * n * n / ((double)p->geo.np3 * std::ldexp(1.0, 3 * p->geo.fbits)));
    d.pbase = e->poff[b];
    d.A = p->ws.meshA;
    d.Gy = p->ws.meshG[1];
    d.Gz = p->ws.meshG[2];
    d.F = p->ws.freal;
    d.tw = p->ws.tw_g;
    d.coef = p->ws.coef;
    d.err = p->ws.err;
    if (!e->tws.tw[ens_size_index(n)]) e->tws.tw[ens_size_index(n)] = p->ws.tw_g;
    const int64_t part_items = (p->geo.np3 + nt - 1) / nt;
    const int64_t part4_items = (p->geo.np3 + (int64_t)nt * kPartPerThread - 1) / ((int64_t)nt * kPartPerThread);
    const int64_t it[kENumLists] = {part_items, part4_items, (int64_t)d.tl.nty * d.tl.ntz, (int64_t)sh.nbx * n,
                                    (int64_t)n * n / sh.RB * 3};
    for (int l = 0; l < kENumLists; ++l) items[(size_t)b * kENumLists + l] = it[l];
    const int M = n / 2;
    const size_t dep = sizeof(unsigned long long) * sh.rows * std::max(n, xrow_ld_host(M));
    const size_t cols = sizeof(float2) * (n * sh.W + ens_stw_size(n, e->tuning.radix));
    d.c2r_rb = sh.RB;
    d.c2r_ld = xrow_ld_host(M);
    c2r_buf = std::max(c2r_buf, (size_t)sh.RB * xrow_ld_host(M));
    e->smem[kKDeposit] = std::max(e->smem[kKDeposit], dep);
    e->smem[kKYfwd] = std::max(e->smem[kKYfwd], cols);
    e->smem[kKZgreen] = std::max(e->smem[kKZgreen], cols + sizeof(float2) * ((n + sh.W + 3) / 4 * 2));
    e->smem[kKYinv] = std::max(e->smem[kKYinv], cols);
  }
  if (bins > e->max_bins_total) return fail(COLA_EINVAL, "ensemble: bin count above the workspace sizing");
  e->total_bins = bins;
  e->c2r_half = (int)c2r_buf;  // two stage buffers, then the stage twiddle tables
  e->smem[kKC2r] = sizeof(float2) * (2 * c2r_buf + ens_c2r_tab_total(e->tuning.radix));
  e->h_starts.assign((size_t)kENumLists * (nb + 1), 0);
  for (int l = 0; l < kENumLists; ++l) {
    int* st_l = &e->h_starts[(size_t)l * (nb + 1)];
    for (int b = 0; b < nb; ++b) {
      const int64_t next = (int64_t)st_l[b] + items[(size_t)b * kENumLists + l];
      if (next > 0x7fffffff) return fail(COLA_EINVAL, "ensemble: too many work items");
      st_l[b + 1] = (int)next;
    }
  }
  const int v = e->tuning.radix;
  int rc = nt == 128 ? (v ? kernel_attrs<128, 1>(e) : kernel_attrs<128, 0>(e))
                     : (v ? kernel_attrs<256, 1>(e) : kernel_attrs<256, 0>(e));
  if (rc) return rc;
  if (e->ws_base) {
    COLA_CUDA_CHECK(cudaMemcpyAsync(e->d_boxes, e->h_boxes.data(), sizeof(BoxDesc) * nb, cudaMemcpyHostToDevice, st));
    COLA_CUDA_CHECK(cudaMemcpyAsync(e->d_starts, e->h_starts.data(), sizeof(int) * e->h_starts.size(),
                                    cudaMemcpyHostToDevice, st));
    // the pageable source vectors may change before an asynchronous copy reads them
    COLA_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  ++e->version;
  return COLA_OK;
}

// work list l on the device
const int* work_list(const cola_ensemble* e, int l) { return e->d_starts + (size_t)l * (e->nbox + 1); }

// Run per_box(b, stream) for every box with the boxes spread over K side streams, forked from
// and joined back into `st` (inside a capture the forks become parallel graph branches; the
// boxes use disjoint workspaces, so their work is independent).
template <class F>
int fork_join(cola_ensemble* e, cudaStream_t st, F&& per_box, int K = cola_ensemble::kForks) {
  COLA_CUDA_CHECK(cudaEventRecord(e->fork_ev, st));
  for (int k = 0; k < K; ++k) COLA_CUDA_CHECK(cudaStreamWaitEvent(e->side[k], e->fork_ev, 0));
  int rc = COLA_OK;
  for (int b = 0; b < e->nbox && !rc; ++b) rc = per_box(b, e->side[b % K]);
  for (int k = 0; k < K; ++k) {  // join even after a failure: no stream may stay forked
    const cudaError_t r1 = cudaEventRecord(e->join_ev[k], e->side[k]);
    const cudaError_t r2 = cudaStreamWaitEvent(st, e->join_ev[k], 0);
    if (!rc && (r1 != cudaSuccess || r2 != cudaSuccess)) rc = fail(COLA_ECUDA, "ensemble stream join failed");
  }
  return rc;
}

// binning of all boxes: one keys, scan and scatter launch for the whole ensemble
template <int NT>
int enqueue_binning(cola_ensemble* e, const float* s, cudaStream_t st) {
  const int nb = e->nbox;
  const int* sp4 = work_list(e, kEParticles4);
  {
    LaunchScope ls_("ens_keys", st);
    ke_keys<NT><<<e->grid[kKKeys], NT, 0, st>>>(e->d_boxes, sp4, nb, s, e->keys, e->counts);
  }
  COLA_LAUNCH_CHECK();
  Tiles all{};
  all.nbins = e->total_bins;
  int rc = launch_scan(all, e->counts, e->offsets, e->cursor, e->scan_blocks, st);
  if (rc) return rc;
  {
    LaunchScope ls_("ens_scatter", st);
    ke_scatter<NT><<<e->grid[kKScatter], NT, 0, st>>>(e->d_boxes, sp4, nb, s, e->keys, e->cursor, e->rec);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

// Mesh passes of all boxes: the multi-box kernels, or (hybrid) every box's own passes from the
// ensemble's records, the boxes dealt over mesh_streams forked streams.
template <int NT, int V>
int enqueue_mesh_passes(cola_ensemble* e, cudaStream_t st) {
  if (hybrid(e)) {
    auto box_passes = [&](int b, cudaStream_t sb) {
      return plan_force_passes(e->plans[b], e->rec, e->offsets + e->h_boxes[b].bin_base, sb);
    };
    if (e->tuning.mesh_streams > 1) return fork_join(e, st, box_passes, e->tuning.mesh_streams);
    for (int b = 0; b < e->nbox; ++b)
      if (const int rc = box_passes(b, st)) return rc;
    return COLA_OK;
  }
  const int nb = e->nbox;
  const int* sd = work_list(e, kEDeposit);
  const int* sc = work_list(e, kECols);
  const int* sr = work_list(e, kEC2r);
  {
    LaunchScope ls_("ens_deposit_fftx", st);
    ke_deposit<NT, V><<<e->grid[kKDeposit], NT, e->smem[kKDeposit], st>>>(e->d_boxes, sd, nb, e->rec, e->offsets);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("ens_fft_y", st);
    ke_cols<NT, 0, V><<<e->grid[kKYfwd], NT, e->smem[kKYfwd], st>>>(e->d_boxes, sc, nb);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("ens_fft_z_green", st);
    ke_cols<NT, 1, V><<<e->grid[kKZgreen], NT, e->smem[kKZgreen], st>>>(e->d_boxes, sc, nb);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("ens_fft_y_inv3", st);
    ke_cols<NT, 2, V><<<e->grid[kKYinv], NT, e->smem[kKYinv], st>>>(e->d_boxes, sc, nb);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("ens_fft_x_c2r3", st);
    ke_c2r3<NT, V><<<e->grid[kKC2r], NT, e->smem[kKC2r], st>>>(e->d_boxes, sr, nb, e->c2r_half, e->tws,
                                                              e->plans[0]->ws.err);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

template <int NT>
int enqueue_gather_binned(cola_ensemble* e, cudaStream_t st) {
  {
    LaunchScope ls_("ens_gather_binned", st);
    ke_gather_binned<NT><<<e->grid[kKGatherB], NT, 0, st>>>(e->d_boxes, work_list(e, kEParticles), e->nbox, e->rec,
                                                            e->gather_f4);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

template <int NT, int V>
int enqueue_step(cola_ensemble* e, int step, float* s, float* v, const float* s1, const float* s2, cudaStream_t st) {
  int rc = enqueue_binning<NT>(e, s, st);
  if (!rc) rc = enqueue_mesh_passes<NT, V>(e, st);
  if (rc) return rc;
  const int nb = e->nbox;
  const int* sp = work_list(e, kEParticles);
  const int mode = step == e->nsteps ? 1 : 0;
  if (!e->binned_gather) {
    {
      LaunchScope ls_("ens_gather_kick_drift", st);
      ke_gather<NT><<<e->grid[kKGather], NT, 0, st>>>(e->d_boxes, sp, nb, s, v, s1, s2, step, mode);
    }
    COLA_LAUNCH_CHECK();
    return COLA_OK;
  }
  if ((rc = enqueue_gather_binned<NT>(e, st))) return rc;
  {
    LaunchScope ls_("ens_kick_drift", st);
    ke_kick_drift<NT><<<e->grid[kKKick], NT, 0, st>>>(e->d_boxes, sp, nb, s, v, s1, s2, step, mode, e->gather_f4);
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

int enqueue_step_any(cola_ensemble* e, int step, float* s, float* v, const float* s1, const float* s2,
                     cudaStream_t st) {
  const bool r = e->tuning.radix != 0;
  if (e->tuning.threads == 128)
    return r ? enqueue_step<128, 1>(e, step, s, v, s1, s2, st) : enqueue_step<128, 0>(e, step, s, v, s1, s2, st);
  return r ? enqueue_step<256, 1>(e, step, s, v, s1, s2, st) : enqueue_step<256, 0>(e, step, s, v, s1, s2, st);
}

// The force evaluation without the particle update (what the autotuner times): the binning and
// mesh passes, and the gather in bin order, whose mesh locality depends on the tile shape (it
// writes only the half-spectrum buffers, so the particle state is left untouched).
template <int NT, int V>
int enqueue_force(cola_ensemble* e, const float* s, cudaStream_t st) {
  int rc = enqueue_binning<NT>(e, s, st);
  if (!rc) rc = enqueue_mesh_passes<NT, V>(e, st);
  if (rc || !e->binned_gather) return rc;
  return enqueue_gather_binned<NT>(e, st);
}

int enqueue_force_any(cola_ensemble* e, const float* s, cudaStream_t st) {
  const bool r = e->tuning.radix != 0;
  if (e->tuning.threads == 128) return r ? enqueue_force<128, 1>(e, s, st) : enqueue_force<128, 0>(e, s, st);
  return r ? enqueue_force<256, 1>(e, s, st) : enqueue_force<256, 0>(e, s, st);
}

int check_ens(const cola_ensemble* e) {
  if (!e) return fail(COLA_EINVAL, "null ensemble");
  if (!e->ws_base) return fail(COLA_ENOWORKSPACE, "cola_ensemble_set_workspace has not been called");
  return COLA_OK;
}

bool valid_tuning(const cola_ensemble_tuning& t) {
  return (t.threads == 128 || t.threads == 256) && (t.tile_shape == 0 || t.tile_shape == 1) &&
         (t.radix == 0 || t.radix == 1) && t.blocks_per_sm >= 0 && t.blocks_per_sm <= 64 &&
         (t.launch == 0 || t.launch == 1 || t.launch == 2 || t.launch == 4) &&
         (t.mesh_streams == 0 || t.mesh_streams == 1 || t.mesh_streams == 2 || t.mesh_streams == 4);
}

// Run `enqueue` on `st`: directly (graphs off or profiling), or as a CUDA graph recorded on
// the private capture stream the first time these `key` values are seen, then replayed.
template <class F>
int replay(cola_ensemble* e, cola_ensemble::Cached& c, const std::vector<uintptr_t>& key, F&& enqueue,
           cudaStream_t st) {
  if (!e->use_graphs || e->prof.on) {
    ProfilerGuard pg(&e->prof);
    return enqueue(st);
  }
  if (!c.exec || c.version != e->version || c.key != key) {
    if (c.exec) {
      COLA_CUDA_CHECK(cudaGraphExecDestroy(c.exec));
      c.exec = nullptr;
    }
    ProfilerGuard pg(nullptr);
    const unsigned long long before = g_launches.load();
    COLA_CUDA_CHECK(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeRelaxed));
    const int rc = enqueue(e->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->cap, &graph);
    const unsigned long long kernels = g_launches.load() - before;
    g_launches.fetch_sub(kernels);  // counted when the graph runs
    if (rc || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return rc ? rc : fail(COLA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    const cudaError_t ie = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      c.exec = nullptr;
      return fail(COLA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    c.key = key;
    c.version = e->version;
    c.kernels = kernels;
  }
  COLA_CUDA_CHECK(cudaGraphLaunch(c.exec, st));
  g_launches.fetch_add(c.kernels);
  return COLA_OK;
}

uintptr_t u(const void* p) { return reinterpret_cast<uintptr_t>(p); }

}  // namespace
}  // namespace cola

extern "C" {

int cola_ensemble_create(const cola_config* boxes, int32_t nbox, cola_ensemble** out) {
  if (!boxes || !out) return fail(COLA_EINVAL, "null argument");
  *out = nullptr;
  if (nbox < 1 || nbox > kEnsMaxBoxes) return fail(COLA_EINVAL, "nbox must be in [1, 4096]");
  for (int b = 0; b < nbox; ++b) {
    if (!ens_size_supported((int)boxes[b].ng))
      return fail(COLA_EUNSUPPORTED, "ensemble boxes need ng in {64, 96, 128, 192, 256} (box " + std::to_string(b) +
                                         ")");
    if (boxes[b].nsteps != boxes[0].nsteps) return fail(COLA_EINVAL, "every ensemble box needs the same nsteps");
    if (boxes[b].adjoint) return fail(COLA_EINVAL, "ensemble boxes do not carry adjoint buffers");
  }
  cola_ensemble* e = new cola_ensemble();
  e->nbox = nbox;
  e->nsteps = boxes[0].nsteps;
  e->poff.assign(nbox + 1, 0);
  e->moff.assign(nbox + 1, 0);
  e->plan_off.assign(nbox, 0);
  size_t off = 0;
  int64_t max_bins = 0;
  e->min_ng = (int)boxes[0].ng;
  for (int b = 0; b < nbox; ++b) {
    cola_plan* p = nullptr;
    int rc = cola_plan_create(&boxes[b], &p);
    if (rc) {
      const std::string why = std::string("ensemble box ") + std::to_string(b) + ": " + cola_last_error();
      delete e;
      return fail(rc, why);
    }
    e->plans.push_back(p);
    e->binned_gather = e->binned_gather && p->binned_gather;
    e->gather_f4 = e->gather_f4 && p->binned_gather4;
    e->poff[b + 1] = e->poff[b] + p->geo.np3;
    e->moff[b + 1] = e->moff[b] + p->ng3;
    e->plan_off[b] = off;
    off += align256(p->ws_bytes);
    e->min_ng = std::min(e->min_ng, p->geo.ng);
    // most bins over the candidate launch shapes: the fewest tile rows (128 threads)
    const int n = p->geo.ng;
    const int rows = 128 / std::max(host_T(n / 2, 0), host_T(n / 2, 1));
    // (the hybrid mode bins as the box's plan does)
    max_bins += std::max(4LL * n * n / rows, (long long)p->tiles.nbins);
  }
  if (e->poff[nbox] >= 0x7fffffffLL || max_bins >= 0x7fffffffLL) {
    delete e;
    return fail(COLA_EINVAL, "ensemble: more than 2^31 particles or bins");
  }
  e->max_bins_total = (int)max_bins;
  e->ens_off = off;
  const int64_t np_all = e->poff[nbox];
  Tiles all{};
  all.nbins = e->max_bins_total;
  off += align256(sizeof(int) * np_all);                   // keys
  off += align256(sizeof(uint4) * np_all);                 // bin-ordered records
  off += align256(sizeof(int) * all.nbins);                // counts
  off += align256(sizeof(int) * (all.nbins + 1));          // offsets
  off += align256(sizeof(int) * all.nbins);                // cursor
  off += align256(sizeof(int) * scan_block_count(all));    // scan block sums
  off += align256(sizeof(BoxDesc) * nbox);                 // box descriptions
  off += align256(sizeof(int) * kENumLists * (nbox + 1));  // work lists
  e->ws_bytes = off;
  e->graphs.resize(e->nsteps + 1 + 4);
  *out = e;
  return COLA_OK;
}

int cola_ensemble_destroy(cola_ensemble* ens) {
  delete ens;
  return COLA_OK;
}

int cola_ensemble_workspace_bytes(const cola_ensemble* ens, size_t* bytes) {
  if (!ens || !bytes) return fail(COLA_EINVAL, "null argument");
  *bytes = ens->ws_bytes;
  return COLA_OK;
}

int cola_ensemble_set_workspace(cola_ensemble* ens, void* dev_ptr, size_t bytes, cola_stream stream) {
  if (!ens || !dev_ptr) return fail(COLA_EINVAL, "null argument");
  if (bytes < ens->ws_bytes) return fail(COLA_EINVAL, "workspace too small");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) return fail(COLA_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)dev_ptr;
  for (int b = 0; b < ens->nbox; ++b) {
    cola_plan* p = ens->plans[b];
    const int rc = cola_set_workspace(p, base + ens->plan_off[b], p->ws_bytes, stream);
    if (rc) return rc;
  }
  size_t off = ens->ens_off;
  auto take = [&](size_t n) {
    char* ptr = base + off;
    off += align256(n);
    return ptr;
  };
  const int64_t np_all = ens->poff[ens->nbox];
  Tiles all{};
  all.nbins = ens->max_bins_total;
  ens->keys = (int*)take(sizeof(int) * np_all);
  ens->rec = (uint4*)take(sizeof(uint4) * np_all);
  ens->counts = (int*)take(sizeof(int) * all.nbins);
  ens->offsets = (int*)take(sizeof(int) * (all.nbins + 1));
  ens->cursor = (int*)take(sizeof(int) * all.nbins);
  ens->scan_blocks = (int*)take(sizeof(int) * scan_block_count(all));
  ens->d_boxes = (BoxDesc*)take(sizeof(BoxDesc) * ens->nbox);
  ens->d_starts = (int*)take(sizeof(int) * kENumLists * (ens->nbox + 1));
  COLA_CUDA_CHECK(cudaMemsetAsync(ens->counts, 0, sizeof(int) * all.nbins, st));
  int dev = 0;
  COLA_CUDA_CHECK(cudaGetDevice(&dev));
  COLA_CUDA_CHECK(cudaDeviceGetAttribute(&ens->num_sms, cudaDevAttrMultiProcessorCount, dev));
  if (!ens->cap) COLA_CUDA_CHECK(cudaStreamCreateWithFlags(&ens->cap, cudaStreamNonBlocking));
  if (!ens->fork_ev) {
    COLA_CUDA_CHECK(cudaEventCreateWithFlags(&ens->fork_ev, cudaEventDisableTiming));
    for (int k = 0; k < cola_ensemble::kForks; ++k) {
      COLA_CUDA_CHECK(cudaStreamCreateWithFlags(&ens->side[k], cudaStreamNonBlocking));
      COLA_CUDA_CHECK(cudaEventCreateWithFlags(&ens->join_ev[k], cudaEventDisableTiming));
    }
  }
  ens->ws_base = dev_ptr;
  return configure(ens, st);
}

int cola_ensemble_offsets(const cola_ensemble* ens, int64_t* poff, int64_t* moff) {
  if (!ens || !poff || !moff) return fail(COLA_EINVAL, "null argument");
  std::memcpy(poff, ens->poff.data(), sizeof(int64_t) * ens->poff.size());
  std::memcpy(moff, ens->moff.data(), sizeof(int64_t) * ens->moff.size());
  return COLA_OK;
}

int cola_ensemble_noise(cola_ensemble* ens, const uint64_t* seeds, float* noise, cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!seeds || !noise) return fail(COLA_EINVAL, "null array");
  std::vector<uintptr_t> key{u(noise)};
  for (int b = 0; b < ens->nbox; ++b) key.push_back((uintptr_t)seeds[b]);
  return replay(ens, ens->graphs[ens->nsteps + 1], key, [&](cudaStream_t st) {
    return fork_join(ens, st, [&](int b, cudaStream_t sb) {
      return cola_noise(ens->plans[b], seeds[b], noise + ens->poff[b], (cola_stream)sb);
    });
  }, (cudaStream_t)stream);
}

int cola_ensemble_ic_2lpt(cola_ensemble* ens, const float* noise, float* s, float* v, float* s1, float* s2,
                          cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!noise || !s || !v || !s1 || !s2) return fail(COLA_EINVAL, "null array");
  return replay(ens, ens->graphs[ens->nsteps + 2], {u(noise), u(s), u(v), u(s1), u(s2)}, [&](cudaStream_t st) {
    return fork_join(ens, st, [&](int b, cudaStream_t sb) {
      const int64_t o = ens->poff[b], o3 = 3 * ens->poff[b];
      return cola_ic_2lpt(ens->plans[b], noise + o, s + o3, v + o3, s1 + o3, s2 + o3, (cola_stream)sb);
    });
  }, (cudaStream_t)stream);
}

int cola_ensemble_step(cola_ensemble* ens, int32_t step, float* s, float* v, const float* s1, const float* s2,
                       cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!s || !v || !s1 || !s2) return fail(COLA_EINVAL, "null array");
  if (step < 0 || step > ens->nsteps) return fail(COLA_EINVAL, "step out of range");
  return replay(ens, ens->graphs[step], {u(s), u(v), u(s1), u(s2)},
                [&](cudaStream_t st) {
                  if (ens->tuning.launch == 0) return enqueue_step_any(ens, step, s, v, s1, s2, st);
                  // per-box launch modes: every box's single-box step, the boxes dealt over
                  // `launch` streams (one box after another on each)
                  auto box_step = [&](int b, cudaStream_t sb) {
                    const int64_t o3 = 3 * ens->poff[b];
                    return cola_step(ens->plans[b], step, s + o3, v + o3, s1 + o3, s2 + o3, (cola_stream)sb);
                  };
                  if (ens->tuning.launch > 1) return fork_join(ens, st, box_step, ens->tuning.launch);
                  for (int b = 0; b < ens->nbox; ++b)
                    if (const int rc = box_step(b, st)) return rc;
                  return (int)COLA_OK;
                },
                (cudaStream_t)stream);
}

int cola_ensemble_density(cola_ensemble* ens, const float* s, float* delta, cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!s || !delta) return fail(COLA_EINVAL, "null array");
  return replay(ens, ens->graphs[ens->nsteps + 3], {u(s), u(delta)}, [&](cudaStream_t st) {
    return fork_join(ens, st, [&](int b, cudaStream_t sb) {
      return cola_density(ens->plans[b], s + 3 * ens->poff[b], nullptr, delta + ens->moff[b], (cola_stream)sb);
    });
  }, (cudaStream_t)stream);
}

int cola_ensemble_power(cola_ensemble* ens, const float* delta, int32_t nbins, double* k, double* pk,
                        int64_t* nmodes, cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!delta || !k || !pk || !nmodes) return fail(COLA_EINVAL, "null array");
  if (nbins < 1 || nbins > ens->min_ng) return fail(COLA_EINVAL, "nbins must be in [1, smallest ng]");
  return replay(ens, ens->graphs[ens->nsteps + 4], {u(delta), (uintptr_t)nbins, u(k), u(pk), u(nmodes)},
                [&](cudaStream_t st) {
                  return fork_join(ens, st, [&](int b, cudaStream_t sb) {
                    const size_t o = (size_t)b * nbins;
                    return cola_power(ens->plans[b], delta + ens->moff[b], nbins, k + o, pk + o, nmodes + o,
                                      (cola_stream)sb);
                  });
                },
                (cudaStream_t)stream);
}

int cola_ensemble_get_tuning(const cola_ensemble* ens, cola_ensemble_tuning* tuning) {
  if (!ens || !tuning) return fail(COLA_EINVAL, "null argument");
  *tuning = ens->tuning;
  return COLA_OK;
}

int cola_ensemble_set_tuning(cola_ensemble* ens, const cola_ensemble_tuning* tuning, cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!tuning || !valid_tuning(*tuning))
    return fail(COLA_EINVAL, "tuning: threads 128 or 256, tile_shape and radix 0 or 1, blocks_per_sm 0..64, "
                             "launch 0, 1, 2 or 4, mesh_streams 0, 1, 2 or 4");
  const cola_ensemble_tuning old = ens->tuning;
  ens->tuning = *tuning;
  if ((rc = configure(ens, (cudaStream_t)stream))) {
    ens->tuning = old;
    configure(ens, (cudaStream_t)stream);
    return rc;
  }
  return COLA_OK;
}

int cola_ensemble_tune(cola_ensemble* ens, const float* s, int32_t reps, cola_ensemble_tuning* best, double* ms,
                       cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  if (!s) return fail(COLA_EINVAL, "null array");
  if (reps < 1 || reps > 1000) return fail(COLA_EINVAL, "reps must be in [1, 1000]");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  COLA_CUDA_CHECK(cudaEventCreate(&e0));
  COLA_CUDA_CHECK(cudaEventCreate(&e1));
  const cola_ensemble_tuning start = ens->tuning;
  cola_ensemble_tuning winner = start;
  double best_ms = 1e300;
  ProfilerGuard pg(nullptr);
  // one force evaluation of all boxes without the particle update, in the candidate's mode
  auto force = [&](cudaStream_t fs) -> int {
    if (ens->tuning.launch == 0) return enqueue_force_any(ens, s, fs);
    auto box_force = [&](int b, cudaStream_t sb) { return plan_force_scratch(ens->plans[b], s + 3 * ens->poff[b], sb); };
    if (ens->tuning.launch > 1) return fork_join(ens, fs, box_force, ens->tuning.launch);
    for (int b = 0; b < ens->nbox; ++b)
      if (const int r = box_force(b, fs)) return r;
    return COLA_OK;
  };
  for (int i = 0; i < COLA_ENSEMBLE_TUNE_CANDIDATES && !rc; ++i) {
    ens->tuning = i < 16   ? cola_ensemble_tuning{(i & 8) ? 256 : 128, (i >> 2) & 1, (i & 2) ? 2 : 0, i & 1, 0, 0}
                  : i < 19 ? cola_ensemble_tuning{128, 0, 0, 0, 1 << (i - 16), 0}
                           : cola_ensemble_tuning{(i - 19) & 1 ? 256 : 128, 0, 0, 0, 0, 1 << ((i - 19) >> 1)};
    if ((rc = configure(ens, st))) break;
    // timed as the steps run: replayed from a CUDA graph (or launched directly with graphs off)
    cudaGraphExec_t exec = nullptr;
    if (ens->use_graphs) {
      const unsigned long long before = g_launches.load();
      if (cudaStreamBeginCapture(ens->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rc = fail(COLA_ECUDA, "tuner: graph capture");
        break;
      }
      const int frc = force(ens->cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(ens->cap, &graph);
      g_launches.fetch_sub(g_launches.load() - before);  // not launched yet
      if (frc || ce != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        rc = frc ? frc : fail(COLA_ECUDA, std::string("tuner: graph capture: ") + cudaGetErrorString(ce));
        break;
      }
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        rc = fail(COLA_ECUDA, std::string("tuner: graph instantiate: ") + cudaGetErrorString(ie));
        break;
      }
    }
    auto run = [&]() -> int {
      if (!exec) return force(st);
      return cudaGraphLaunch(exec, st) == cudaSuccess ? (int)COLA_OK : fail(COLA_ECUDA, "tuner: graph launch");
    };
    rc = run();  // warm-up
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = fail(COLA_ECUDA, "event record");
    for (int r = 0; r < reps && !rc; ++r) rc = run();
    float el = 0.f;
    if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&el, e0, e1) != cudaSuccess))
      rc = fail(COLA_ECUDA, "event timing");
    if (exec) {
      cudaStreamSynchronize(st);
      cudaGraphExecDestroy(exec);
    }
    if (rc) break;
    const double t = (double)el / reps;
    if (ms) ms[i] = t;
    if (t < best_ms) {
      best_ms = t;
      winner = ens->tuning;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ens->tuning = rc ? start : winner;
  const int rc2 = configure(ens, st);
  if (rc) return rc;
  if (rc2) return rc2;
  if (best) *best = ens->tuning;
  return COLA_OK;
}

int cola_ensemble_use_graphs(cola_ensemble* ens, int32_t enable) {
  if (!ens) return fail(COLA_EINVAL, "null ensemble");
  ens->use_graphs = enable != 0;
  return COLA_OK;
}

int cola_ensemble_status(cola_ensemble* ens, cola_stream stream) {
  int rc = check_ens(ens);
  if (rc) return rc;
  for (int b = 0; b < ens->nbox; ++b)
    if ((rc = cola_status(ens->plans[b], stream)))
      return fail(rc, std::string("ensemble box ") + std::to_string(b) + ": " + cola_last_error());
  return COLA_OK;
}

int cola_ensemble_profile(cola_ensemble* ens, int32_t enable) {
  if (!ens) return fail(COLA_EINVAL, "null ensemble");
  ens->prof.on = enable != 0;
  return COLA_OK;
}

int cola_ensemble_profile_read(cola_ensemble* ens, int32_t max_entries, char* names, int64_t* launches, double* ms,
                               int32_t* count) {
  if (!ens) return fail(COLA_EINVAL, "null ensemble");
  return profile_read(ens->prof, max_entries, names, launches, ms, count);
}

}  // extern "C"
