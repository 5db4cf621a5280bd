// Internal declarations shared by the CUDA translation units of the COLA library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cola.h"
#include "profiler.cuh"

namespace cola {

// error bits latched in the workspace by kernels
enum : int { kErrOverflow = 1, kErrNonFinite = 2, kErrTimeout = 4, kErrUnion = 8, kErrSmIds = 16 };

// per-step float32 coefficients on the device (row of kCoef32 floats per force evaluation)
enum Coef32 : int {
  kCKF = 0,   // c_K * (3/2) Om a_i     (multiplies the unit force g)
  kCK1 = 1,   // c_K * T^2[D1](a_i)
  kCK2 = 2,   // c_K * T^2[D2](a_i)
  kCD = 3,    // drift coefficient
  kDD1 = 4,   // D1(a_i+1) - D1(a_i)
  kDD2 = 5,   // D2(a_i+1) - D2(a_i)
  kTD1 = 6,   // T[D1](a_i)  (used by L+ on the last row)
  kTD2 = 7,   // T[D2](a_i)
  kLast = 8,  // 1 on the last row
  kCoef32 = 16
};

// Fixed-point CIC geometry shared by the deposit, the gather and the binning:
//   f_d = (floor(i_d ng 2^F / np) + floor(fl32(s_d * fl32(ng/L)) * 2^F)) mod (ng 2^F)
struct Geometry {
  int np, ng;
  int64_t np3;
  int fbits;
  int ratio;      // ng / np when ng is a multiple of np, else 0
  float scale32;  // fl32(ng / L)
  // division of a 32-bit index by np as a multiply-high and shifts (set_np_divider)
  uint32_t np_mul;
  int np_sh1, np_sh2;
  // fixed_axis may take its 32-bit path: ratio != 0 and 2^22 <= ng 2^F <= 2^30
  int fast32;
};

// Unsigned 32-bit division by an invariant d >= 1 (Granlund & Montgomery 1994, Sec. 4): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, every n < 2^32 has
//   n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),  t = mulhi(m, n).
inline void set_np_divider(Geometry& g) {
  const uint64_t d = (uint64_t)g.np;
  int l = 0;
  while ((1ull << l) < d) ++l;
  g.np_mul = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  g.np_sh1 = l < 1 ? l : 1;
  g.np_sh2 = l > 1 ? l - 1 : 0;
  const int64_t period = (int64_t)g.ng << g.fbits;
  g.fast32 = g.ratio != 0 && period >= (1LL << 22) && period <= (1LL << 30);
}

struct Tiles {
  int ty, tz;     // rows per tile along y and z (the tile spans the whole x row)
  int nty, ntz;   // tiles per axis
  int nbins;      // nty * ntz * 4 (4 boundary regions per tile)
  int lband;      // log2 of the tiles per band along y (bins run band by band, see tile_bin)
};

// Tiles are numbered band by band: a band is 2^lband consecutive tiles along y, and within a band
// the tiles run along y, then z.  Consecutive bins then cover the whole z range of a narrow band
// of y rows, so the rows that neighbouring tiles share along z (and y) are still in L2 when the
// next tile reads them.
__host__ __device__ __forceinline__ int tile_bin(const Tiles& tl, int ty, int tz) {
  return (((ty >> tl.lband) * tl.ntz + tz) << tl.lband) + (ty & ((1 << tl.lband) - 1));
}
__host__ __device__ __forceinline__ void tile_of_bin(const Tiles& tl, int bin, int& ty, int& tz) {
  const int per_band = tl.ntz << tl.lband;
  const int band = bin / per_band, rem = bin - band * per_band;
  tz = rem >> tl.lband;
  ty = (band << tl.lband) + (rem & ((1 << tl.lband) - 1));
}
// the largest power of two <= 32 that divides nty
inline int tile_band_log2(int nty) {
  int l = 0;
  while (l < 5 && nty % (2 << l) == 0) ++l;
  return l;
}

struct Workspace {
  float2* tw_g = nullptr;   // exp(-2 pi i m / ng), m < ng
  float2* tw_p = nullptr;   // exp(-2 pi i m / np), m < np
  float* coef = nullptr;    // (nsteps+1) x kCoef32
  int* err = nullptr;       // latched error bits
  // PM step (aliases the IC region)
  float2* meshA = nullptr;  // half spectrum, ng x ng x Pg
  float2* meshG[3] = {nullptr, nullptr, nullptr};  // [1], [2]: y and z force half spectra ([0] unused)
  float* freal = nullptr;   // 3 x ng^3 force meshes (freal[0..ng^3) doubles as delta)
  // particle binning
  int* keys = nullptr;
  // [np^3] in bin order: the particle's fixed-point CIC coordinates f_x, f_y, f_z and its
  // lattice index (one 16-byte record, written and read with one access)
  uint4* rec = nullptr;
  int* counts = nullptr;    // nbins
  int* offsets = nullptr;   // nbins + 1
  int* cursor = nullptr;    // nbins
  int* scan_blocks = nullptr;  // one partial sum per scan tile
  // power spectrum per-block partial sums: kPowerBlocks x ng x 3 doubles
  double* pk_partial = nullptr;
  // initial conditions (alias the PM meshes)
  float2* icC0 = nullptr;
  float2* icC1 = nullptr;
  float2* icC2 = nullptr;
  float* icR[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // adjoint only: three real meshes for the deposited adjoint (the first doubles as Phi)
  float* lam_real = nullptr;
};

}  // namespace cola

struct cola_plan {
  cola_config cfg;
  cola::Geometry geo;
  cola::Tiles tiles;
  int Pg = 0, Pp = 0;  // padded half-spectrum row lengths (complex) for ng and np
  int64_t ng3 = 0;
  // the step gathers in bin order into the half-spectrum buffers (each holds np^3 floats), as
  // one float4 per particle into the first of them when it holds 16 bytes per particle
  bool binned_gather = false;
  bool binned_gather4 = false;
  // retry limit of the friends-of-friends union-find (cola_set_fof_union_tries)
  int fof_union_tries = 1 << 20;
  std::vector<double> coef64;
  std::vector<float> coef32;
  std::vector<float2> tw_g, tw_p;
  double pk_amp = 0.0;  // A of P(k) = A k^ns T^2(k)
  double d2u1 = 0.0;
  size_t ws_bytes = 0;
  void* ws_base = nullptr;
  cola::Workspace ws;
  cola::Profiler prof;
};

namespace cola {

// ---- host helpers (api.cu) ------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
struct Profiler;
int profile_read(Profiler& pr, int32_t max_entries, char* names, int64_t* launches, double* ms, int32_t* count);
bool fft_size_supported(int n);

// ---- host coefficient module (coeffs.cpp) -----------------------------------------------
struct HostCosmo;
int build_coefficients(const cola_config& cfg, std::vector<double>& table, double& pk_amp, double& d2u1,
                       std::string& why);
void twiddle_table(int n, std::vector<float2>& out);

// ---- launchers (kernels_*.cu) ------------------------------------------------------------
// FFT passes (fft_kernels.cu)
int launch_fft_x_r2c(int n, const float* in, float2* out, int64_t nrows, int P, const float2* tw, cudaStream_t st);
int launch_fft_x_c2r(int n, const float2* in, float* out, int64_t nrows, int P, const float2* tw, float scale,
                     cudaStream_t st);
int launch_fft_cols(int n, bool inverse, float2* data, int64_t nslabs, int64_t slab_stride, int64_t row_stride,
                    int ncols, const float2* tw, cudaStream_t st);
// 3-D helpers built on the passes: r2c (x then y then z) and c2r (z, y, x), layout [n][n][P]
int fft3d_r2c(int n, int P, const float* in, float2* out, const float2* tw, cudaStream_t st);
int fft3d_c2r(int n, int P, float2* in_destroyed, float* out, const float2* tw, float scale, cudaStream_t st);

// PM kernels (pm_kernels.cu)
int launch_keys(const Geometry& g, const Tiles& t, const float* s, int* keys, int* counts, int* err, cudaStream_t st);
int scan_block_count(const Tiles& t);
int launch_scan(const Tiles& t, int* counts, int* offsets, int* cursor, int* block_sums, cudaStream_t st);
int launch_scatter(const Geometry& g, const float* s, const int* keys, int* cursor, uint4* rec,
                   cudaStream_t st);
int launch_deposit(const Geometry& g, const Tiles& t, const uint4* rec, const int* offsets, int64_t* rho,
                   float* delta, int* err, cudaStream_t st);
int launch_kspace_force(int ng, int P, double box, int deconv, const float2* dk, float2* gx, float2* gy, float2* gz,
                        cudaStream_t st);
// the fused mesh passes of one force evaluation (pm_fft_kernels.cu): deposit + x r2c, y pass,
// z pass with the Green's function, inverse y passes, inverse x passes -> F [3][ng^3]
// the half spectrum A of the density of the binned particles: the force evaluation's fused
// deposit + x r2c, then the forward y and z passes (no Green's function)
int launch_density_spectrum(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets, float2* A,
                            int P, const float2* tw, int* err, cudaStream_t st);
int launch_force_passes(const Geometry& g, const Tiles& tl, const uint4* rec, const int* offsets,
                        float2* A, float2* Gy, float2* Gz, float* F, int P, double box, int deconv, const float2* tw,
                        int* err, cudaStream_t st);
// mode 0: kick + drift, 1: kick + L+ (last force evaluation), 2: write the gathered unit force to gout
int launch_gather_kick_drift(const Geometry& g, const float* fmesh, float* s, float* v, const float* s1,
                             const float* s2, const float* coef_row, int mode, float* gout, cudaStream_t st);
// the gather in bin order of the last binning (records rec) into fj[p], and the kick/drift in
// lattice order from those forces
// one force evaluation of a plan without the particle update (binning, mesh passes, and the
// gather into the free half-spectrum buffers when the plan gathers in bin order): what the
// ensemble autotuner times for the per-box launch mode
int plan_force_scratch(cola_plan* p, const float* s, cudaStream_t st);
// the mesh passes of plan p (deposit + x r2c .. inverse x) from bin-ordered records rec and bin
// offsets `offsets` in the layout of p->tiles, supplied by the caller
int plan_force_passes(cola_plan* p, const uint4* rec, const int* offsets, cudaStream_t st);
int launch_gather_binned(const Geometry& g, const float* fmesh, const uint4* rec,
                         float* f0, float* f1, float* f2, cudaStream_t st);
int launch_kick_drift(const Geometry& g, const float* f0, const float* f1, const float* f2, float* s, float* v,
                      const float* s1, const float* s2, const float* coef_row, int mode, cudaStream_t st);
// the same with the force of particle p as one float4 f4[p] (used when a half spectrum holds
// 16 bytes per particle)
int launch_gather_binned4(const Geometry& g, const float* fmesh, const uint4* rec, float4* f4, cudaStream_t st);
int launch_kick_drift4(const Geometry& g, const float4* f4, float* s, float* v, const float* s1, const float* s2,
                       const float* coef_row, int mode, cudaStream_t st);

// IC kernels (ic_kernels.cu)
int launch_noise(int np, uint64_t seed, float* out, cudaStream_t st);
int launch_ic_filter(int np, int P, double box, double amp, double n_s, double omega_m, double h, float2* wk,
                     cudaStream_t st);
// out = factor(k) * in on the half spectrum; kind selects the operator (see ic_kernels.cu)
int launch_kmul(int n, int P, double box, int kind, int i, int j, float scale, const float2* in, float2* out,
                cudaStream_t st);
int launch_source_2lpt(int64_t n3, const float* fxx, const float* fyy, const float* fzz, float* out_acc,
                       cudaStream_t st);
int launch_source_sub_sq(int64_t n3, const float* f, float* acc, cudaStream_t st);
int launch_ic_assemble(int64_t n3, float d1, float d2, float t1, float t2, const float* s1, const float* s2,
                       float* s, float* v, cudaStream_t st);

// adjoint kernels (adjoint_kernels.cu)
int launch_adjoint_pre(int64_t n3, int mode, const float* coef, float* lam_s, float* lam_v, float* lam_s1,
                       float* lam_s2, cudaStream_t st);
int launch_lambda_deposit(const Geometry& g, const float* s, const float* lam, float* out, cudaStream_t st);
int launch_kspace_adjoint(int ng, int P, double box, int deconv, float2* lx, const float2* ly, const float2* lz,
                          cudaStream_t st);
int launch_gather_adjoint(const Geometry& g, const float* s, const float* F, const float* phi, const float* lam_v,
                          float* lam_s, float scale_a, float scale_b, int mode, cudaStream_t st);
int launch_kmul_acc(int n, int P, double box, int kind, int i, int j, float scale, int accumulate, const float2* in,
                    float2* out, cudaStream_t st);
int launch_ic_adjoint_assemble(int64_t n3, float d1, float d2, const float* lam_s, float* lam_s1, float* lam_s2,
                               cudaStream_t st);
int launch_ic_adjoint_product(int64_t n3, const float* a, const float* b, const float* c, float* out,
                              cudaStream_t st);

// power spectrum and utilities (power_kernels.cu)
// blocks of the binning kernel (fixed, so that the per-block partial sums and their reduction
// order, hence the result, do not depend on the launch)
constexpr int kPowerBlocks = 456;  // 3 blocks per SM of 152
// partial sums per block and shell: 3 (k, P, modes) for P(k), 5 for the cross spectrum
constexpr int kPowerQuantities = 5;
int power_partial_doubles(int nbins);  // size of the partial-sum buffer
int launch_power_bin(int ng, int P, double box, int nbins, const float2* dk, double* partial, cudaStream_t st);
int launch_power_finish(int nbins, const double* partial, double* k, double* pk, int64_t* nmodes, cudaStream_t st);
int launch_cross_bin(int ng, int P, double box, int nbins, const float2* da, const float2* db, double* partial,
                     cudaStream_t st);
int launch_cross_finish(int nbins, const double* partial, double* k, double* pa, double* pb, double* pab, double* rho,
                        double* nmax, int64_t* nmodes, cudaStream_t st);
int launch_unpad(int n, int P, const float2* in, float2* out, cudaStream_t st);

}  // namespace cola

#define COLA_CUDA_CHECK(expr)                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return ::cola::fail(COLA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define COLA_LAUNCH_CHECK() COLA_CUDA_CHECK(cudaGetLastError())
