// C ABI of the COLA library (declarations and documentation in include/cola.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "cola_internal.cuh"

namespace cola {

static thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
thread_local Profiler* t_profiler = nullptr;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Assigns the workspace regions (when base != nullptr) and returns the total size.
static size_t layout(cola_plan* p, char* base) {
  const int64_t ng = p->geo.ng, np = p->geo.np;
  const int64_t ng3 = ng * ng * ng, np3 = np * np * np;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  Workspace& w = p->ws;
  w.tw_g = (float2*)take(sizeof(float2) * ng);
  w.tw_p = (float2*)take(sizeof(float2) * np);
  w.coef = (float*)take(sizeof(float) * kCoef32 * (p->cfg.nsteps + 1));
  w.err = (int*)take(sizeof(int) * 4);
  w.keys = (int*)take(sizeof(int) * np3);
  w.rec = (uint4*)take(sizeof(uint4) * np3);
  w.counts = (int*)take(sizeof(int) * p->tiles.nbins);
  w.offsets = (int*)take(sizeof(int) * (p->tiles.nbins + 1));
  w.cursor = (int*)take(sizeof(int) * p->tiles.nbins);
  w.scan_blocks = (int*)take(sizeof(int) * scan_block_count(p->tiles));
  w.pk_partial = (double*)take(sizeof(double) * power_partial_doubles((int)ng));
  // mesh region: the PM step and the initial conditions reuse the same bytes
  const size_t region = off;
  const size_t half_g = sizeof(float2) * ng * ng * p->Pg;
  w.meshA = (float2*)take(half_g);
  w.meshG[0] = nullptr;  // the x component is never stored as a half spectrum
  for (int j = 1; j < 3; ++j) w.meshG[j] = (float2*)take(half_g);
  w.freal = (float*)take(sizeof(float) * 3 * ng3);
  const size_t pm_end = off;
  off = region;
  const size_t half_p = sizeof(float2) * np * np * p->Pp;
  w.icC0 = (float2*)take(half_p);
  w.icC1 = (float2*)take(half_p);
  w.icC2 = (float2*)take(half_p);
  for (int j = 0; j < 5; ++j) w.icR[j] = (float*)take(sizeof(float) * np3);
  off = std::max(off, pm_end);
  w.lam_real = p->cfg.adjoint ? (float*)take(sizeof(float) * 3 * ng3) : nullptr;
  return off;
}

static int check_ws(const cola_plan* p) {
  if (!p) return fail(COLA_EINVAL, "null plan");
  if (!p->ws_base) return fail(COLA_ENOWORKSPACE, "cola_set_workspace has not been called");
  return COLA_OK;
}

static int padded_half(int n) { return ((n / 2 + 1) + 3) / 4 * 4; }

// particle binning for positions s: keys -> counts -> offsets -> bin-ordered records
static int bin_particles(cola_plan* p, const float* s, cudaStream_t st) {
  Workspace& w = p->ws;
  int rc = launch_keys(p->geo, p->tiles, s, w.keys, w.counts, w.err, st);
  if (rc) return rc;
  rc = launch_scan(p->tiles, w.counts, w.offsets, w.cursor, w.scan_blocks, st);
  if (rc) return rc;
  return launch_scatter(p->geo, s, w.keys, w.cursor, w.rec, st);
}

// unit force meshes g_j (freal[j]) for positions s
static int force_meshes(cola_plan* p, const float* s, cudaStream_t st) {
  Workspace& w = p->ws;
  int rc = bin_particles(p, s, st);
  if (rc) return rc;
  return launch_force_passes(p->geo, p->tiles, w.rec, w.offsets, w.meshA, w.meshG[1], w.meshG[2], w.freal, p->Pg,
                             p->cfg.box, p->cfg.deconv, w.tw_g, w.err, st);
}

int plan_force_scratch(cola_plan* p, const float* s, cudaStream_t st) {
  int rc = force_meshes(p, s, st);
  if (rc || !p->binned_gather) return rc;
  Workspace& w = p->ws;
  if (p->binned_gather4) return launch_gather_binned4(p->geo, w.freal, w.rec, reinterpret_cast<float4*>(w.meshA), st);
  return launch_gather_binned(p->geo, w.freal, w.rec, reinterpret_cast<float*>(w.meshA),
                              reinterpret_cast<float*>(w.meshG[1]), reinterpret_cast<float*>(w.meshG[2]), st);
}

int plan_force_passes(cola_plan* p, const uint4* rec, const int* offsets, cudaStream_t st) {
  Workspace& w = p->ws;
  return launch_force_passes(p->geo, p->tiles, rec, offsets, w.meshA, w.meshG[1], w.meshG[2], w.freal, p->Pg,
                             p->cfg.box, p->cfg.deconv, w.tw_g, w.err, st);
}

}  // namespace cola

namespace cola {
int profile_read(Profiler& pr, int32_t max_entries, char* names, int64_t* launches, double* ms, int32_t* count) {
  if (!names || !launches || !ms || !count || max_entries < 1) return fail(COLA_EINVAL, "null argument");
  std::vector<std::string> keys;
  std::vector<int64_t> n;
  std::vector<double> t;
  for (auto& r : pr.recs) {
    COLA_CUDA_CHECK(cudaEventSynchronize(r.stop));
    float el = 0.f;
    COLA_CUDA_CHECK(cudaEventElapsedTime(&el, r.start, r.stop));
    size_t i = 0;
    while (i < keys.size() && keys[i] != r.name) ++i;
    if (i == keys.size()) {
      keys.emplace_back(r.name);
      n.push_back(0);
      t.push_back(0.0);
    }
    n[i] += 1;
    t[i] += el;
    pr.pool.push_back(r.start);
    pr.pool.push_back(r.stop);
  }
  pr.recs.clear();
  const int m = std::min<int>((int)keys.size(), max_entries);
  for (int i = 0; i < m; ++i) {
    std::memset(names + 64 * i, 0, 64);
    std::strncpy(names + 64 * i, keys[i].c_str(), 63);
    launches[i] = n[i];
    ms[i] = t[i];
  }
  *count = m;
  return COLA_OK;
}

}  // namespace cola

using namespace cola;

extern "C" {

int cola_config_default(cola_config* cfg) {
  if (!cfg) return fail(COLA_EINVAL, "null config");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->np = 32;
  cfg->ng = 64;
  cfg->box = 100.0;
  cfg->cosmo = {0.27, 0.73, 0.7, 0.8, 0.96};
  cfg->n_lpt = -2.5;
  cfg->nsteps = 10;
  cfg->a_init = 0.1;
  cfg->a_final = 1.0;
  cfg->deconv = 1;
  cfg->fixed_bits = 16;
  cfg->adjoint = 0;
  cfg->scheme = COLA_SCHEME_COLA;
  cfg->log_a = 0;
  return COLA_OK;
}

int cola_plan_create(const cola_config* cfg, cola_plan** out) {
  if (!cfg || !out) return fail(COLA_EINVAL, "null argument");
  *out = nullptr;
  const cola_config& c = *cfg;
  if (!fft_size_supported((int)c.np) || !fft_size_supported((int)c.ng) || c.np > 1536)
    return fail(COLA_EUNSUPPORTED, "np and ng must be one of 32,48,64,96,128,192,256,384,512,768,1024,1536,2048 "
                                   "(np <= 1536)");
  if (c.ng % 4) return fail(COLA_EINVAL, "ng must be a multiple of 4");
  if (!(c.box > 0) || !std::isfinite(c.box)) return fail(COLA_EINVAL, "box must be positive");
  if (c.nsteps < 1 || c.nsteps > 100000) return fail(COLA_EINVAL, "nsteps out of range");
  if (!(c.a_init > 0) || !(c.a_final > c.a_init)) return fail(COLA_EINVAL, "need 0 < a_init < a_final");
  if (c.deconv < 0 || c.deconv > 2) return fail(COLA_EINVAL, "deconv must be 0, 1 or 2");
  if (c.fixed_bits < 8 || c.fixed_bits > 20) return fail(COLA_EINVAL, "fixed_bits must be in [8, 20]");
  if (c.adjoint != 0 && c.adjoint != 1) return fail(COLA_EINVAL, "adjoint must be 0 or 1");
  if (c.scheme < COLA_SCHEME_COLA || c.scheme > COLA_SCHEME_COLA_U1) return fail(COLA_EINVAL, "unknown scheme");
  if (c.log_a != 0 && c.log_a != 1) return fail(COLA_EINVAL, "log_a must be 0 or 1");
  if (c.adjoint && c.scheme == COLA_SCHEME_PM)
    return fail(COLA_EINVAL, "the adjoint calls assume the LPT frame (v = 0 after L-): not with COLA_SCHEME_PM");
  if (!(c.cosmo.omega_m > 0) || !(c.cosmo.h > 0) || !(c.cosmo.sigma8 > 0))
    return fail(COLA_EINVAL, "omega_m, h and sigma8 must be positive");
  cola_plan* p = new cola_plan();
  p->cfg = c;
  p->geo.np = (int)c.np;
  p->geo.ng = (int)c.ng;
  p->geo.np3 = c.np * c.np * c.np;
  p->geo.fbits = c.fixed_bits;
  p->geo.ratio = (c.ng % c.np == 0) ? (int)(c.ng / c.np) : 0;
  p->geo.scale32 = (float)((double)c.ng / c.box);
  set_np_divider(p->geo);
  p->ng3 = c.ng * c.ng * c.ng;
  // deposit tiles of 4 x 2 mesh rows (y, z), each spanning the whole x extent (2 x 2 at ng = 2048,
  // where a 4 x 2 tile of int64 cells fills the shared memory of an SM: two blocks per SM)
  p->tiles.ty = c.ng == 2048 ? 2 : 4;
  p->tiles.tz = 2;
  p->tiles.nty = (int)c.ng / p->tiles.ty;
  p->tiles.ntz = (int)c.ng / 2;
  p->tiles.nbins = p->tiles.nty * p->tiles.ntz * 4;
  p->tiles.lband = tile_band_log2(p->tiles.nty);
  p->Pg = padded_half((int)c.ng);
  p->Pp = padded_half((int)c.np);
  p->binned_gather = (double)sizeof(float2) * c.ng * c.ng * p->Pg >= (double)sizeof(float) * p->geo.np3;
  p->binned_gather4 = (double)sizeof(float2) * c.ng * c.ng * p->Pg >= (double)sizeof(float4) * p->geo.np3;
  std::string why;
  int rc = build_coefficients(c, p->coef64, p->pk_amp, p->d2u1, why);
  if (rc) {
    delete p;
    return fail(rc, why);
  }
  p->coef32.assign((size_t)(c.nsteps + 1) * kCoef32, 0.0f);
  for (int i = 0; i <= c.nsteps; ++i) {
    const double* r = &p->coef64[(size_t)i * COLA_NCOEF];
    float* o = &p->coef32[(size_t)i * kCoef32];
    // the standard leapfrog has no LPT frame: no -T^2[D] s terms, no dD s drift, no L+
    const double frame = c.scheme == COLA_SCHEME_PM ? 0.0 : 1.0;
    o[kCKF] = (float)(r[2] * r[1]);
    o[kCK1] = (float)(frame * r[2] * r[3]);
    o[kCK2] = (float)(frame * r[2] * r[4]);
    o[kCD] = (float)r[5];
    o[kDD1] = (float)(frame * r[6]);
    o[kDD2] = (float)(frame * r[7]);
    o[kTD1] = (float)(frame * r[8]);
    o[kTD2] = (float)(frame * r[9]);
    o[kLast] = i == c.nsteps ? 1.0f : 0.0f;
  }
  twiddle_table((int)c.ng, p->tw_g);
  twiddle_table((int)c.np, p->tw_p);
  p->ws_bytes = layout(p, nullptr);
  *out = p;
  return COLA_OK;
}

int cola_plan_destroy(cola_plan* plan) {
  delete plan;
  return COLA_OK;
}

int cola_workspace_bytes(const cola_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return fail(COLA_EINVAL, "null argument");
  *bytes = plan->ws_bytes;
  return COLA_OK;
}

int cola_set_workspace(cola_plan* plan, void* dev_ptr, size_t bytes, cola_stream stream) {
  if (!plan || !dev_ptr) return fail(COLA_EINVAL, "null argument");
  if (bytes < plan->ws_bytes) return fail(COLA_EINVAL, "workspace too small");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) return fail(COLA_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  plan->ws_base = dev_ptr;
  layout(plan, (char*)dev_ptr);
  Workspace& w = plan->ws;
  COLA_CUDA_CHECK(cudaMemcpyAsync(w.tw_g, plan->tw_g.data(), sizeof(float2) * plan->tw_g.size(),
                                  cudaMemcpyHostToDevice, st));
  COLA_CUDA_CHECK(cudaMemcpyAsync(w.tw_p, plan->tw_p.data(), sizeof(float2) * plan->tw_p.size(),
                                  cudaMemcpyHostToDevice, st));
  COLA_CUDA_CHECK(cudaMemcpyAsync(w.coef, plan->coef32.data(), sizeof(float) * plan->coef32.size(),
                                  cudaMemcpyHostToDevice, st));
  COLA_CUDA_CHECK(cudaMemsetAsync(w.err, 0, sizeof(int) * 4, st));
  COLA_CUDA_CHECK(cudaMemsetAsync(w.counts, 0, sizeof(int) * plan->tiles.nbins, st));
  return COLA_OK;
}

int cola_coeffs(const cola_plan* plan, double* table) {
  if (!plan || !table) return fail(COLA_EINVAL, "null argument");
  std::memcpy(table, plan->coef64.data(), sizeof(double) * plan->coef64.size());
  return COLA_OK;
}

int cola_noise(cola_plan* plan, uint64_t seed, float* noise, cola_stream stream) {
  if (!plan || !noise) return fail(COLA_EINVAL, "null argument");
  ProfilerGuard pg(&plan->prof);
  return launch_noise(plan->geo.np, seed, noise, (cudaStream_t)stream);
}

int cola_ic_2lpt(cola_plan* plan, const float* noise, float* s, float* v, float* s1, float* s2, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!noise || !s || !v || !s1 || !s2) return fail(COLA_EINVAL, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  const int n = plan->geo.np, P = plan->Pp;
  const int64_t n3 = plan->geo.np3;
  const float norm = (float)(1.0 / (double)n3);
  const double box = plan->cfg.box;
  // white noise -> linear density at a = 1
  if ((rc = fft3d_r2c(n, P, noise, w.icC0, w.tw_p, st))) return rc;
  if ((rc = launch_ic_filter(n, P, box, plan->pk_amp, plan->cfg.cosmo.n_s, plan->cfg.cosmo.omega_m,
                             plan->cfg.cosmo.h, w.icC0, st)))
    return rc;
  // s1 = i k delta / k^2
  for (int j = 0; j < 3; ++j) {
    if ((rc = launch_kmul(n, P, box, 0, j, 0, norm, w.icC0, w.icC1, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC1, s1 + j * n3, w.tw_p, 1.0f, st))) return rc;
  }
  // mu2 = psi_xx psi_yy + psi_xx psi_zz + psi_yy psi_zz - psi_xy^2 - psi_xz^2 - psi_yz^2
  for (int j = 0; j < 3; ++j) {
    if ((rc = launch_kmul(n, P, box, 1, j, j, norm, w.icC0, w.icC1, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC1, w.icR[j], w.tw_p, 1.0f, st))) return rc;
  }
  if ((rc = launch_source_2lpt(n3, w.icR[0], w.icR[1], w.icR[2], w.icR[0], st))) return rc;
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (auto& ij : pairs) {
    if ((rc = launch_kmul(n, P, box, 1, ij[0], ij[1], norm, w.icC0, w.icC1, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC1, w.icR[1], w.tw_p, 1.0f, st))) return rc;
    if ((rc = launch_source_sub_sq(n3, w.icR[1], w.icR[0], st))) return rc;
  }
  // s2 = D2u(1) * (-i k mu2_k / k^2)
  if ((rc = fft3d_r2c(n, P, w.icR[0], w.icC1, w.tw_p, st))) return rc;
  const float s2scale = (float)(-plan->d2u1 / (double)n3);
  for (int j = 0; j < 3; ++j) {
    if ((rc = launch_kmul(n, P, box, 0, j, 0, s2scale, w.icC1, w.icC0, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC0, s2 + j * n3, w.tw_p, 1.0f, st))) return rc;
  }
  // v = T[s] after L- (eq. Lops): 0 in the LPT frame; the standard leapfrog starts from the
  // full 2LPT velocity T[D1] s1 + T[D2] s2
  const double* row0 = plan->coef64.data();
  const bool pm = plan->cfg.scheme == COLA_SCHEME_PM;
  return launch_ic_assemble(n3, (float)row0[10], (float)row0[11], pm ? (float)row0[8] : 0.0f,
                            pm ? (float)row0[9] : 0.0f, s1, s2, s, v, st);
}

int cola_step(cola_plan* plan, int32_t step, float* s, float* v, const float* s1, const float* s2,
              cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!s || !v || !s1 || !s2) return fail(COLA_EINVAL, "null array");
  if (step < 0 || step > plan->cfg.nsteps) return fail(COLA_EINVAL, "step out of range");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = force_meshes(plan, s, st))) return rc;
  const int mode = step == plan->cfg.nsteps ? 1 : 0;
  const float* coef = plan->ws.coef + (size_t)step * kCoef32;
  const Workspace& w = plan->ws;
  if (!plan->binned_gather)
    return launch_gather_kick_drift(plan->geo, w.freal, s, v, s1, s2, coef, mode, nullptr, st);
  // the gathered forces go to the half-spectrum buffers, free once the force meshes exist
  if (plan->binned_gather4) {
    float4* f4 = reinterpret_cast<float4*>(w.meshA);
    if ((rc = launch_gather_binned4(plan->geo, w.freal, w.rec, f4, st))) return rc;
    return launch_kick_drift4(plan->geo, f4, s, v, s1, s2, coef, mode, st);
  }
  float* f[3] = {reinterpret_cast<float*>(w.meshA), reinterpret_cast<float*>(w.meshG[1]),
                 reinterpret_cast<float*>(w.meshG[2])};
  if ((rc = launch_gather_binned(plan->geo, w.freal, w.rec, f[0], f[1], f[2], st))) return rc;
  return launch_kick_drift(plan->geo, f[0], f[1], f[2], s, v, s1, s2, coef, mode, st);
}

int cola_force(cola_plan* plan, const float* s, float* g, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!s || !g) return fail(COLA_EINVAL, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = force_meshes(plan, s, st))) return rc;
  const int64_t n3 = plan->geo.np3;
  return launch_gather_binned(plan->geo, plan->ws.freal, plan->ws.rec, g, g + n3, g + 2 * n3, st);
}

int cola_density(cola_plan* plan, const float* s, int64_t* rho_fix, float* delta, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!s || (!rho_fix && !delta)) return fail(COLA_EINVAL, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = bin_particles(plan, s, st))) return rc;
  return launch_deposit(plan->geo, plan->tiles, plan->ws.rec, plan->ws.offsets, rho_fix, delta, plan->ws.err, st);
}

int cola_power(cola_plan* plan, const float* delta, int32_t nbins, double* k, double* pk, int64_t* nmodes,
               cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!delta || !k || !pk || !nmodes) return fail(COLA_EINVAL, "null array");
  if (nbins < 1 || nbins > plan->geo.ng) return fail(COLA_EINVAL, "nbins must be in [1, ng]");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  if ((rc = fft3d_r2c(plan->geo.ng, plan->Pg, delta, w.meshA, w.tw_g, st))) return rc;
  if ((rc = launch_power_bin(plan->geo.ng, plan->Pg, plan->cfg.box, nbins, w.meshA, w.pk_partial, st))) return rc;
  return launch_power_finish(nbins, w.pk_partial, k, pk, nmodes, st);
}

int cola_density_power(cola_plan* plan, const float* s, int32_t nbins, double* k, double* pk, int64_t* nmodes,
                       cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!s || !k || !pk || !nmodes) return fail(COLA_EINVAL, "null array");
  if (nbins < 1 || nbins > plan->geo.ng) return fail(COLA_EINVAL, "nbins must be in [1, ng]");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  if ((rc = bin_particles(plan, s, st))) return rc;
  if ((rc = launch_density_spectrum(plan->geo, plan->tiles, w.rec, w.offsets, w.meshA, plan->Pg, w.tw_g, w.err, st)))
    return rc;
  if ((rc = launch_power_bin(plan->geo.ng, plan->Pg, plan->cfg.box, nbins, w.meshA, w.pk_partial, st))) return rc;
  return launch_power_finish(nbins, w.pk_partial, k, pk, nmodes, st);
}

int cola_cross_power(cola_plan* plan, const float* delta_a, const float* delta_b, int32_t nbins, double* k,
                     double* pk_a, double* pk_b, double* pk_ab, double* rho, double* nmax, int64_t* nmodes,
                     cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!delta_a || !delta_b || !k || !pk_a || !pk_b || !pk_ab || !rho || !nmax || !nmodes)
    return fail(COLA_EINVAL, "null array");
  if (nbins < 1 || nbins > plan->geo.ng) return fail(COLA_EINVAL, "nbins must be in [1, ng]");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  if ((rc = fft3d_r2c(plan->geo.ng, plan->Pg, delta_a, w.meshA, w.tw_g, st))) return rc;
  if ((rc = fft3d_r2c(plan->geo.ng, plan->Pg, delta_b, w.meshG[1], w.tw_g, st))) return rc;
  if ((rc = launch_cross_bin(plan->geo.ng, plan->Pg, plan->cfg.box, nbins, w.meshA, w.meshG[1], w.pk_partial, st)))
    return rc;
  return launch_cross_finish(nbins, w.pk_partial, k, pk_a, pk_b, pk_ab, rho, nmax, nmodes, st);
}

int cola_fft_r2c(cola_plan* plan, int32_t which, const float* in, float* out, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!in || !out) return fail(COLA_EINVAL, "null array");
  if (which != 0 && which != 1) return fail(COLA_EINVAL, "which must be 0 (mesh) or 1 (lattice)");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = which == 0 ? plan->geo.ng : plan->geo.np;
  const int P = which == 0 ? plan->Pg : plan->Pp;
  const float2* tw = which == 0 ? plan->ws.tw_g : plan->ws.tw_p;
  float2* tmp = which == 0 ? plan->ws.meshA : plan->ws.icC0;
  if ((rc = fft3d_r2c(n, P, in, tmp, tw, st))) return rc;
  return launch_unpad(n, P, tmp, reinterpret_cast<float2*>(out), st);
}

int cola_status(cola_plan* plan, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  COLA_CUDA_CHECK(cudaStreamSynchronize(st));
  int err = 0;
  COLA_CUDA_CHECK(cudaMemcpy(&err, plan->ws.err, sizeof(int), cudaMemcpyDeviceToHost));
  COLA_CUDA_CHECK(cudaMemset(plan->ws.err, 0, sizeof(int)));
  if (err & kErrTimeout) return fail(COLA_ETIMEOUT, "a kernel gave up waiting for its bulk copies");
  if (err & kErrUnion) return fail(COLA_ETIMEOUT, "friends-of-friends: union-find retries ran out");
  if (err & kErrSmIds)
    return fail(COLA_EUNSUPPORTED, "the wide z pass found no scratch slot for its SM (more SM ids than slots)");
  if (err & kErrNonFinite) return fail(COLA_EOVERFLOW, "non-finite particle displacement");
  if (err & kErrOverflow) return fail(COLA_EOVERFLOW, "fixed-point density overflow (too many particles per cell)");
  return COLA_OK;
}

int cola_step_adjoint(cola_plan* plan, int32_t step, const float* s_ckpt, float* lam_s, float* lam_v, float* lam_s1,
                      float* lam_s2, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!plan->cfg.adjoint) return fail(COLA_EINVAL, "plan was created without adjoint buffers (cola_config.adjoint)");
  if (!s_ckpt || !lam_s || !lam_v || !lam_s1 || !lam_s2) return fail(COLA_EINVAL, "null array");
  if (step < 0 || step > plan->cfg.nsteps) return fail(COLA_EINVAL, "step out of range");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  const int ng = plan->geo.ng;
  const int64_t ng3 = plan->ng3;
  const int mode = step == plan->cfg.nsteps ? 1 : 0;
  const float* coef = w.coef + (size_t)step * kCoef32;
  // adjoint of the Kick/Drift/L+ algebra: lam_v becomes the adjoint of the kicked velocity
  if ((rc = launch_adjoint_pre(plan->geo.np3, mode, coef, lam_s, lam_v, lam_s1, lam_s2, st))) return rc;
  // the force meshes at the checkpointed positions (term A of the force VJP)
  if ((rc = force_meshes(plan, s_ckpt, st))) return rc;
  // term B: deposit lam_v, apply the transposed force operator, gather with the weight gradient
  if ((rc = launch_lambda_deposit(plan->geo, s_ckpt, lam_v, w.lam_real, st))) return rc;
  float2* half[3] = {w.meshA, w.meshG[1], w.meshG[2]};
  for (int j = 0; j < 3; ++j)
    if ((rc = fft3d_r2c(ng, plan->Pg, w.lam_real + j * ng3, half[j], w.tw_g, st))) return rc;
  if ((rc = launch_kspace_adjoint(ng, plan->Pg, plan->cfg.box, plan->cfg.deconv, half[0], half[1], half[2], st)))
    return rc;
  float* phi = w.lam_real;
  if ((rc = fft3d_c2r(ng, plan->Pg, half[0], phi, w.tw_g, 1.0f, st))) return rc;
  const double* row = &plan->coef64[(size_t)step * COLA_NCOEF];
  const double to_cells = (double)ng / plan->cfg.box;
  const double inv_rho_bar = (double)ng3 / (double)plan->geo.np3;
  const double ckf = row[2] * row[1];
  return launch_gather_adjoint(plan->geo, s_ckpt, w.freal, phi, lam_v, lam_s, (float)(ckf * to_cells),
                               (float)(ckf * to_cells * inv_rho_bar), 0, st);
}

int cola_density_adjoint(cola_plan* plan, const float* s, const float* delta_bar, float* lam_s, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!s || !delta_bar || !lam_s) return fail(COLA_EINVAL, "null array");
  const double to_cells = (double)plan->geo.ng / plan->cfg.box;
  const double inv_rho_bar = (double)plan->ng3 / (double)plan->geo.np3;
  return launch_gather_adjoint(plan->geo, s, plan->ws.freal, delta_bar, nullptr, lam_s, 0.0f,
                               (float)(to_cells * inv_rho_bar), 1, (cudaStream_t)stream);
}

int cola_ic_2lpt_adjoint(cola_plan* plan, const float* noise, const float* lam_s, float* lam_s1, float* lam_s2,
                         float* grad_noise, cola_stream stream) {
  int rc = check_ws(plan);
  if (rc) return rc;
  ProfilerGuard pg(&plan->prof);
  if (!noise || !lam_s || !lam_s1 || !lam_s2 || !grad_noise) return fail(COLA_EINVAL, "null array");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = plan->ws;
  const int n = plan->geo.np, P = plan->Pp;
  const int64_t n3 = plan->geo.np3;
  const float norm = (float)(1.0 / (double)n3);
  const double box = plan->cfg.box;
  const double* row0 = plan->coef64.data();
  // s = D1 s1 + D2 s2 at a_init
  if ((rc = launch_ic_adjoint_assemble(n3, (float)row0[10], (float)row0[11], lam_s, lam_s1, lam_s2, st))) return rc;
  // lam_mu2 = IFFT( sum_j (+i k_j / k^2) FFT(D2u(1) lam_s2_j) ) / n^3   (transpose of s2 = D2u(1) psi2)
  for (int j = 0; j < 3; ++j) {
    if ((rc = fft3d_r2c(n, P, lam_s2 + j * n3, w.icC1, w.tw_p, st))) return rc;
    if ((rc = launch_kmul_acc(n, P, box, 0, j, 0, (float)(plan->d2u1 / (double)n3), j > 0, w.icC1, w.icC2, st)))
      return rc;
  }
  float* lam_mu2 = w.icR[3];
  if ((rc = fft3d_c2r(n, P, w.icC2, lam_mu2, w.tw_p, 1.0f, st))) return rc;
  // the linear density and the diagonal second derivatives psi_ii
  if ((rc = fft3d_r2c(n, P, noise, w.icC0, w.tw_p, st))) return rc;
  if ((rc = launch_ic_filter(n, P, box, plan->pk_amp, plan->cfg.cosmo.n_s, plan->cfg.cosmo.omega_m,
                             plan->cfg.cosmo.h, w.icC0, st)))
    return rc;
  for (int i = 0; i < 3; ++i) {
    if ((rc = launch_kmul(n, P, box, 1, i, i, norm, w.icC0, w.icC1, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC1, w.icR[i], w.tw_p, 1.0f, st))) return rc;
  }
  // lam_delta_k = sum_ij M_ij FFT(lam_psi_ij) + sum_j (-i k_j / k^2) FFT(lam_s1_j)
  float* tmp = w.icR[4];
  for (int i = 0; i < 3; ++i) {  // lam_psi_ii = lam_mu2 * (psi_jj + psi_kk)
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    if ((rc = launch_ic_adjoint_product(n3, lam_mu2, w.icR[j], w.icR[k], tmp, st))) return rc;
    if ((rc = fft3d_r2c(n, P, tmp, w.icC1, w.tw_p, st))) return rc;
    if ((rc = launch_kmul_acc(n, P, box, 1, i, i, 1.0f, i > 0, w.icC1, w.icC2, st))) return rc;
  }
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (auto& ij : pairs) {  // lam_psi_ij = -2 lam_mu2 psi_ij
    if ((rc = launch_kmul(n, P, box, 1, ij[0], ij[1], norm, w.icC0, w.icC1, st))) return rc;
    if ((rc = fft3d_c2r(n, P, w.icC1, tmp, w.tw_p, 1.0f, st))) return rc;
    if ((rc = launch_ic_adjoint_product(n3, lam_mu2, tmp, nullptr, tmp, st))) return rc;
    if ((rc = fft3d_r2c(n, P, tmp, w.icC1, w.tw_p, st))) return rc;
    if ((rc = launch_kmul_acc(n, P, box, 1, ij[0], ij[1], 1.0f, 1, w.icC1, w.icC2, st))) return rc;
  }
  for (int j = 0; j < 3; ++j) {
    if ((rc = fft3d_r2c(n, P, lam_s1 + j * n3, w.icC1, w.tw_p, st))) return rc;
    if ((rc = launch_kmul_acc(n, P, box, 0, j, 0, -1.0f, 1, w.icC1, w.icC2, st))) return rc;
  }
  // noise gradient = IFFT(amp(k) lam_delta_k) / n^3
  if ((rc = launch_ic_filter(n, P, box, plan->pk_amp, plan->cfg.cosmo.n_s, plan->cfg.cosmo.omega_m,
                             plan->cfg.cosmo.h, w.icC2, st)))
    return rc;
  return fft3d_c2r(n, P, w.icC2, grad_noise, w.tw_p, norm, st);
}

int cola_profile(cola_plan* plan, int32_t enable) {
  if (!plan) return fail(COLA_EINVAL, "null plan");
  plan->prof.on = enable != 0;
  return COLA_OK;
}

int cola_profile_read(cola_plan* plan, int32_t max_entries, char* names, int64_t* launches, double* ms,
                      int32_t* count) {
  if (!plan) return fail(COLA_EINVAL, "null plan");
  return profile_read(plan->prof, max_entries, names, launches, ms, count);
}

int cola_launch_count(uint64_t* count) {
  if (!count) return fail(COLA_EINVAL, "null argument");
  *count = g_launches.load();
  return COLA_OK;
}

const char* cola_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
