// cola_power_noalloc: the shell-averaged power spectrum of a small density mesh without any
// plan, workspace or device allocation.
//
// Who needs it: code that measures P(k) from inside a host application that owns every byte
// of device memory through its own pool allocator (so a library may not call cudaMalloc /
// cudaFree behind its back, and those calls would also synchronise the whole device), and
// monitoring tools attached to a running simulation that must not change its memory
// footprint.  Such callers still pass their own input and output buffers.
//
// The scratch (the half spectrum, the shell accumulators and one twiddle table per supported
// mesh size) lives in the file-scope device array below, sized for meshes up to
// COLA_NOALLOC_MAX_NG^3.  Every GPU that loads this library keeps that array (about 10.7 MiB)
// until the process exits.  Host code must not pass the array's name to a kernel: on the host
// that name is only a stand-in for the device symbol, so its device address is looked up once
// per device with cudaGetSymbolAddress and that address is what the kernels receive.  The
// twiddle table of a mesh size is uploaded once per device, by the first call with that size;
// later calls issue no host-to-device copy.
#include <mutex>
#include <vector>

#include "cola_internal.cuh"

namespace cola {
namespace {

constexpr int kMaxNg = COLA_NOALLOC_MAX_NG;
constexpr int kSizes[] = {32, 48, 64, 96, 128};  // the supported mesh sizes up to kMaxNg
constexpr int kNumSizes = sizeof(kSizes) / sizeof(kSizes[0]);
static_assert(kSizes[kNumSizes - 1] == kMaxNg, "size list must end at the scratch limit");
constexpr int kMaxP = ((kMaxNg / 2 + 1) + 3) / 4 * 4;
constexpr size_t kSpecBytes = sizeof(float2) * kMaxNg * kMaxNg * kMaxP;
// per-block shell sums, sized as the plan's (power_partial_doubles) for nbins <= kMaxNg
constexpr size_t kPartOff = kSpecBytes;
constexpr size_t kPartBytes = sizeof(double) * kPowerBlocks * kMaxNg * kPowerQuantities;
constexpr size_t kTwOff = kPartOff + (kPartBytes + 255) / 256 * 256;  // float2[kNumSizes][kMaxNg]
constexpr size_t kScratchBytes = kTwOff + sizeof(float2) * kNumSizes * kMaxNg;
static_assert(kPartOff % 256 == 0 && kTwOff % 256 == 0, "scratch regions must stay aligned");

static __device__ __align__(256) unsigned char g_power_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
bool g_tw_ready[kMaxDevices][kNumSizes] = {};  // twiddle table of kSizes[i] uploaded on this device

int size_slot(int ng) {
  for (int i = 0; i < kNumSizes; ++i)
    if (kSizes[i] == ng) return i;
  return -1;
}

// Device address of the scratch array on the current device (looked up on the first call), with
// the twiddle table of mesh size ng in place (uploaded by the first call with that size).
int scratch_address(int ng, unsigned char** out) {
  int dev = 0;
  COLA_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(COLA_EINVAL, "cola_power_noalloc: device index out of range");
  const int slot = size_slot(ng);
  if (slot < 0) return fail(COLA_EUNSUPPORTED, "cola_power_noalloc: unsupported ng");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_power_scratch);
    if (e != cudaSuccess || !p)
      return fail(COLA_ECUDA, std::string("cola_power_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  if (!g_tw_ready[dev][slot]) {
    std::vector<float2> tw;
    twiddle_table(ng, tw);
    COLA_CUDA_CHECK(cudaMemcpy(base + kTwOff + sizeof(float2) * kMaxNg * slot, tw.data(), sizeof(float2) * ng,
                               cudaMemcpyHostToDevice));
    g_tw_ready[dev][slot] = true;
  }
  *out = base;
  return COLA_OK;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" int cola_power_noalloc(const float* delta, int32_t ng, double box, int32_t nbins, double* k, double* pk,
                                  int64_t* nmodes, cola_stream stream) {
  if (!delta || !k || !pk || !nmodes) return fail(COLA_EINVAL, "cola_power_noalloc: null array");
  if (ng > kMaxNg)
    return fail(COLA_EINVAL, "cola_power_noalloc: ng = " + std::to_string(ng) + " exceeds the static scratch limit of " +
                                 std::to_string(kMaxNg) + " cells per side; use cola_power with a workspace");
  if (size_slot(ng) < 0 || !fft_size_supported(ng)) return fail(COLA_EUNSUPPORTED, "cola_power_noalloc: unsupported ng");
  if (!(box > 0)) return fail(COLA_EINVAL, "cola_power_noalloc: box must be positive");
  if (nbins < 1 || nbins > ng) return fail(COLA_EINVAL, "cola_power_noalloc: nbins must be in [1, ng]");
  unsigned char* base = nullptr;
  int rc = scratch_address(ng, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  float2* spec = reinterpret_cast<float2*>(base);
  double* partial = reinterpret_cast<double*>(base + kPartOff);
  const float2* tw = reinterpret_cast<const float2*>(base + kTwOff + sizeof(float2) * kMaxNg * size_slot(ng));
  static_assert((size_t)kPowerBlocks * kMaxNg * kPowerQuantities * sizeof(double) <= kPartBytes,
                "the shell sums of nbins = ng must fit");
  const int P = ((ng / 2 + 1) + 3) / 4 * 4;
  if ((rc = fft3d_r2c(ng, P, delta, spec, tw, st))) return rc;
  // the binning kernel overwrites every partial sum it later reads, so what the previous call
  // left in the scratch never enters this result
  if ((rc = launch_power_bin(ng, P, box, nbins, spec, partial, st))) return rc;
  return launch_power_finish(nbins, partial, k, pk, nmodes, st);
}
