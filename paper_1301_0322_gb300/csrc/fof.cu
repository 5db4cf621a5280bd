// Friends-of-friends halo groups (Sec. 3.2) on the GPU.
//
// Positions are the particles' fixed-point CIC coordinates f (mesh cells x 2^F, the PM
// force's own quantised positions).  Two particles are friends iff den^2 |d|^2 < num^2 s^2
// with d the periodic minimum-image separation and s = (ng/np) 2^F the mean separation
// (b = num/den, 1/5 in the paper): an exact integer test, so the groups do not depend on
// rounding or on the order of the atomics.
//
//   1. cell keys: cubic cells of `csize` mesh cells (>= the linking length), counting sort of
//      the particles into them (the binning scan and scatter of the PM step; the scatter also
//      stores f in cell order)
//   2. link: one thread per particle (cell order) visits the 27 neighbouring cells and unites
//      it with every friend of higher sorted position: lock-free union-find whose roots
//      always point to smaller positions (compare-and-swap, bounded retries)
//   3. compress every path to its root, count group sizes, smallest original index per group
//   4. per particle: group label (smallest particle index of its group, -1 below nmin) and
//      group size; per threshold: number of halos with at least that many particles
#include <climits>
#include <cstring>

#include "cola_internal.cuh"
#include "particle_bodies.cuh"

namespace cola {
namespace {

constexpr int kMaxThresholds = 32;

struct Thresholds {
  int n;
  int v[kMaxThresholds];
};

__global__ void k_fof_keys(Geometry g, const float* __restrict__ s, int csize, int nc, int* __restrict__ keys,
                           int* __restrict__ counts, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < g.np3;
  int key = -1;
  if (live) {
    int ix, iy, iz;
    lattice_index(g, p, ix, iy, iz);
    const float sx = s[p], sy = s[g.np3 + p], sz = s[2 * g.np3 + p];
    if (!isfinite(sx) || !isfinite(sy) || !isfinite(sz)) atomicOr(err, kErrNonFinite);
    int cx, cy, cz, t;
    fixed_axis(g, ix, sx, cx, t);
    fixed_axis(g, iy, sy, cy, t);
    fixed_axis(g, iz, sz, cz, t);
    key = ((cz / csize) * nc + cy / csize) * nc + cx / csize;
    keys[p] = key;
  }
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (live && lane == __ffs(peers) - 1) atomicAdd(&counts[key], __popc(peers));
}

__global__ void k_fof_init(int64_t n, int* __restrict__ parent, int* __restrict__ gsize, int* __restrict__ minp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    parent[i] = (int)i;
    gsize[i] = 0;
    minp[i] = INT_MAX;
  }
}

// root of x: parents only ever point to smaller positions, so the walk ends within x steps
__device__ __forceinline__ int fof_find(const int* parent, int x) {
  int p = __ldcg(parent + x);
  while (p != x) {
    x = p;
    p = __ldcg(parent + x);
  }
  return x;
}

// link the larger of the two roots under the smaller one; false if the `tries` attempts ran out
__device__ __forceinline__ bool fof_union(int* parent, int a, int b, int tries) {
  for (int it = 0; it < tries; ++it) {
    a = fof_find(parent, a);
    b = fof_find(parent, b);
    if (a == b) return true;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + a, a, b) == a) return true;
  }
  return false;
}

__device__ __forceinline__ int64_t min_image(int64_t d, int64_t period) {
  if (d > period / 2) return d - period;
  if (d < -(period / 2)) return d + period;
  return d;
}

__global__ void k_fof_link(Geometry g, const uint4* __restrict__ rec, const int* __restrict__ offsets, int csize,
                           int nc, int64_t den2, int64_t lim, int tries, int* __restrict__ parent,
                           int* __restrict__ err) {
  const int64_t n = g.np3;
  const int64_t period = (int64_t)g.ng << g.fbits;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 qi = rec[i];
    const int64_t fx = qi.x, fy = qi.y, fz = qi.z;
    const int cx = (int)(fx >> g.fbits) / csize, cy = (int)(fy >> g.fbits) / csize, cz = (int)(fz >> g.fbits) / csize;
    bool ok = true;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = (cz + dz + nc) % nc;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = (cy + dy + nc) % nc;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = (cx + dx + nc) % nc;
          const int cell = (zz * nc + yy) * nc + xx;
          const int j1 = offsets[cell + 1];
          for (int j = max(offsets[cell], (int)i + 1); j < j1; ++j) {
            const uint4 qj = rec[j];
            const int64_t ex = min_image((int64_t)qj.x - fx, period);
            const int64_t ey = min_image((int64_t)qj.y - fy, period);
            const int64_t ez = min_image((int64_t)qj.z - fz, period);
            const int64_t d2 = ex * ex + ey * ey + ez * ez;
            if (den2 * d2 < lim) ok = fof_union(parent, (int)i, j, tries) && ok;
          }
        }
      }
    }
    if (!ok) atomicOr(err, kErrUnion);
  }
}

__global__ void k_fof_groups(int64_t n, const uint4* __restrict__ rec, int* __restrict__ parent,
                             int* __restrict__ gsize, int* __restrict__ minp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = fof_find(parent, (int)i);
    parent[i] = r;
    atomicAdd(gsize + r, 1);
    atomicMin(minp + r, (int)rec[i].w);
  }
}

__global__ void k_fof_output(int64_t n, const uint4* __restrict__ rec, const int* __restrict__ parent,
                             const int* __restrict__ gsize, const int* __restrict__ minp, int nmin, Thresholds thr,
                             int* __restrict__ group, int* __restrict__ size, unsigned long long* __restrict__ n_ge) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = parent[i];
    const int gs = gsize[r];
    const unsigned p = rec[i].w;
    if (size) size[p] = gs;
    if (group) group[p] = gs >= nmin ? minp[r] : -1;
    if (r == (int)i && gs >= nmin)
      for (int k = 0; k < thr.n; ++k)
        if (gs >= thr.v[k]) atomicAdd(n_ge + k, 1ULL);
  }
}

unsigned grid_of(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 64); }

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" int cola_fof(cola_plan* plan, const float* s, int32_t b_num, int32_t b_den, int32_t nmin, int32_t* group,
                        int32_t* size, int32_t nthr, const int32_t* thresholds, int64_t* n_ge, cola_stream stream) {
  if (!plan) return fail(COLA_EINVAL, "null plan");
  if (!plan->ws_base) return fail(COLA_ENOWORKSPACE, "cola_set_workspace has not been called");
  ProfilerGuard pg(&plan->prof);
  if (!s || (!group && !size)) return fail(COLA_EINVAL, "null array");
  if (b_num < 1 || b_den < 1 || b_den > 50 || b_num > b_den)
    return fail(COLA_EINVAL, "linking length b = b_num / b_den needs 1 <= b_num <= b_den <= 50");
  if (nmin < 1) return fail(COLA_EINVAL, "nmin must be >= 1");
  if (nthr < 0 || nthr > kMaxThresholds || (nthr > 0 && (!thresholds || !n_ge)))
    return fail(COLA_EINVAL, "0..32 thresholds with host thresholds and a device n_ge array");
  const Geometry& g = plan->geo;
  if (g.ratio < 1) return fail(COLA_EUNSUPPORTED, "FOF needs ng to be a multiple of np");
  if (g.np3 >= 0x7fffffffLL) return fail(COLA_EUNSUPPORTED, "FOF supports fewer than 2^31 particles");
  // cells of csize mesh cells: at least the linking length b * (ng/np), a divisor of ng, and few
  // enough cells for int32 bin offsets
  int csize = (b_num * g.ratio + b_den - 1) / b_den;
  while (csize <= g.ng && (g.ng % csize != 0 || (int64_t)(g.ng / csize) * (g.ng / csize) * (g.ng / csize) >= (1LL << 30)))
    ++csize;
  const int nc = csize <= g.ng ? g.ng / csize : 0;
  if (nc < 3) return fail(COLA_EUNSUPPORTED, "FOF needs at least 3 linking cells per side");
  // exact int64 tests: den^2 d^2 with |d| < 2 csize 2^F per axis, and num^2 s^2
  if (((int64_t)csize << g.fbits) >= (1LL << 24) || (((int64_t)g.ratio << g.fbits) >= (1LL << 24)))
    return fail(COLA_EUNSUPPORTED, "FOF: linking cells or mean separation too large for exact int64 distances");
  Thresholds thr{};
  thr.n = nthr;
  for (int k = 0; k < nthr; ++k) thr.v[k] = thresholds[k];
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  // scratch: cell bins in the force-mesh region, union-find arrays in the half spectra
  Tiles cells{};
  cells.nbins = nc * nc * nc;
  int* counts = reinterpret_cast<int*>(w.freal);
  int* offsets = counts + cells.nbins;
  int* cursor = offsets + cells.nbins + 1;
  int* scan_blocks = cursor + cells.nbins;
  int* parent = reinterpret_cast<int*>(w.meshA);
  int* gsize = reinterpret_cast<int*>(w.meshG[1]);
  int* minp = reinterpret_cast<int*>(w.meshG[2]);
  const int64_t n = g.np3;
  COLA_CUDA_CHECK(cudaMemsetAsync(counts, 0, sizeof(int) * cells.nbins, st));
  if (nthr > 0) COLA_CUDA_CHECK(cudaMemsetAsync(n_ge, 0, sizeof(int64_t) * nthr, st));
  {
    LaunchScope ls_("fof_keys", st);
    k_fof_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, s, csize, nc, w.keys, counts, w.err);
  }
  COLA_LAUNCH_CHECK();
  int rc = launch_scan(cells, counts, offsets, cursor, scan_blocks, st);
  if (rc) return rc;
  if ((rc = launch_scatter(g, s, w.keys, cursor, w.rec, st))) return rc;
  {
    LaunchScope ls_("fof_init", st);
    k_fof_init<<<grid_of(n), 256, 0, st>>>(n, parent, gsize, minp);
  }
  COLA_LAUNCH_CHECK();
  const int64_t sfix = (int64_t)g.ratio << g.fbits;
  const int64_t lim = (int64_t)b_num * b_num * sfix * sfix;
  {
    LaunchScope ls_("fof_link", st);
    k_fof_link<<<grid_of(n), 256, 0, st>>>(g, w.rec, offsets, csize, nc, (int64_t)b_den * b_den, lim,
                                           plan->fof_union_tries, parent, w.err);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("fof_groups", st);
    k_fof_groups<<<grid_of(n), 256, 0, st>>>(n, w.rec, parent, gsize, minp);
  }
  COLA_LAUNCH_CHECK();
  {
    LaunchScope ls_("fof_output", st);
    k_fof_output<<<grid_of(n), 256, 0, st>>>(n, w.rec, parent, gsize, minp, nmin, thr, group, size,
                                             reinterpret_cast<unsigned long long*>(n_ge));
  }
  COLA_LAUNCH_CHECK();
  return COLA_OK;
}

extern "C" int cola_set_fof_union_tries(cola_plan* plan, int32_t tries) {
  if (!plan) return fail(COLA_EINVAL, "null plan");
  if (tries < 0 || tries > (1 << 30)) return fail(COLA_EINVAL, "tries must be in [0, 2^30]");
  plan->fof_union_tries = tries;
  return COLA_OK;
}
