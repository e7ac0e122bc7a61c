// Read-out of macroscopic fields that allocates no memory.
//
// For callers that cannot call cudaMalloc (for example code running under an
// external memory manager that forbids allocations, or a plugin that only
// receives device buffers from its host application).  It runs the same
// read-out kernel as rlbm_moments, but every piece of device scratch it needs
// -- the sticky error word, the R(zeta) table and the staging planes of the
// result -- lives in one file-scope static device array, so the only device
// memory touched is that array and the caller's own buffers.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "rlbm_kernels.cuh"
#include "rlbm_stencil.h"

namespace rlbm {
namespace {

// Static scratch, present on every GPU that loads the library until exit.
constexpr size_t kScratchBytes = size_t(8) << 20;          // 8 MiB
constexpr size_t kErrOffset = 0;                           // one unsigned
constexpr size_t kTableOffset = 256;                       // R(zeta) FP64 table
constexpr size_t kTableBytes = size_t(RT_NSEG) * RT_NC64 * sizeof(double);
constexpr size_t kOutOffset = (kTableOffset + kTableBytes + 255) / 256 * 256;
constexpr size_t kOutDoubles = (kScratchBytes - kOutOffset) / sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
bool g_ready[kMaxDevices] = {};
unsigned char* g_addr[kMaxDevices] = {};

// host cache of the last stencil (host-side tables only)
bool g_have_stencil = false;
int g_groups[6];
double g_m = 0, g_v0 = 0;
int g_Nx = 0, g_Ny = 0;
StepParams<double> g_params;
rlbm_status fail(rlbm_status s, const std::string& msg) {
  set_global_error(msg);   // readable with rlbm_last_error(NULL)
  return s;
}

}  // namespace
}  // namespace rlbm

using namespace rlbm;

extern "C" rlbm_status rlbm_moments_noalloc(const int* groups, int ngroups, double m, double v0, int Nx,
                                            int Ny, const double* f_dev, double* out_host, unsigned mask,
                                            void* cuda_stream) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!groups || !f_dev || !out_host || Nx < 1 || Ny < 1 || !(v0 > 0))
    return fail(RLBM_EINVAL, "invalid argument");
  if (ngroups != 6)
    return fail(RLBM_EINVAL, "rlbm_moments_noalloc takes six-group (second-order) stencils only; got " +
                                 std::to_string(ngroups) + " groups");
  if (mask == 0 || (mask & ~0x7Fu)) return fail(RLBM_EINVAL, "mask must select 1..7 known fields");
  size_t planes = 0;
  for (unsigned b : {RLBM_M_N, RLBM_M_UX, RLBM_M_UY, RLBM_M_T, RLBM_M_E})
    if (mask & b) ++planes;
  if (mask & RLBM_M_NVEC) planes += 3;
  if (mask & RLBM_M_TMN) planes += 6;
  const size_t nsite = (size_t)Nx * (size_t)Ny;   // < 2^62: no wrap
  // compared by division: planes * nsite could wrap for huge Nx, Ny
  if (nsite > kOutDoubles / planes) {
    return fail(RLBM_EINVAL, "result of " + std::to_string(planes) + " planes x " + std::to_string(nsite) +
                                 " sites exceeds the static scratch of " + std::to_string(kOutDoubles) +
                                 " doubles (8 MiB array)");
  }
  // set-up, once per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(RLBM_ENOTSUP, "device index beyond 64");
  if (!g_ready[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const auto& t64 = ratio_table64();
    e = cudaMemcpy(static_cast<unsigned char*>(ptr) + kTableOffset, t64.data(), kTableBytes,
                   cudaMemcpyHostToDevice);
    // a pageable upload may return before the copy lands; the read-outs run on
    // caller streams that need not be ordered after the legacy stream
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<unsigned char*>(ptr);
    g_ready[dev] = true;
  }
  unsigned char* base = g_addr[dev];
  // host tables of the stencil (rebuilt only when the parameters change)
  int sorted[6];
  for (int k = 0; k < 6; ++k) sorted[k] = groups[k];
  std::sort(sorted, sorted + 6);
  bool same = g_have_stencil && g_m == m && g_v0 == v0 && g_Nx == Nx && g_Ny == Ny;
  for (int k = 0; k < 6 && same; ++k) same = (g_groups[k] == sorted[k]);
  if (!same) {
    StencilBuild sb;
    std::string err;
    rlbm_stencil st{6, sorted, v0};
    const rlbm_status s = build_stencil(&st, m, &sb, &err);
    if (s != RLBM_OK) return fail(s, err);
    std::memset(&g_params, 0, sizeof g_params);
    g_params.Nx = Nx;
    g_params.Ny = Ny;
    g_params.Q = (int)sb.pops.size();
    g_params.halo = sb.halo;
    g_params.pitch = Nx;                      // compact [Q][Ny][Nx] layout
    g_params.plane = (long long)Nx * Ny;
    g_params.inv_tau = 1.0;
    g_params.v0 = sb.v0;
    g_params.sc = sb.sc;
    fill_pop_table<double>(sb, Nx, Ny, &g_params.pt);
    // the populations passed in are f(., t) itself: no pull
    for (int i = 0; i < QMAX; ++i) g_params.pt.dxm[i] = g_params.pt.dym[i] = 0;
    for (int k = 0; k < 6; ++k) g_groups[k] = sorted[k];
    g_m = m;
    g_v0 = v0;
    g_Nx = Nx;
    g_Ny = Ny;
    g_have_stencil = true;
  }
  g_params.rt64 = reinterpret_cast<const double*>(base + kTableOffset);
  g_params.rt32 = nullptr;
  g_params.err = reinterpret_cast<unsigned*>(base + kErrOffset);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the error word must start at zero; the staging planes are fully written
  e = cudaMemsetAsync(base + kErrOffset, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("memset: ") + cudaGetErrorString(e));
  MomentOut mo{reinterpret_cast<double*>(base + kOutOffset), mask};
  e = launch_moments(RLBM_F64, g_params, f_dev, mo, s);
  if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  unsigned flags = 0;
  e = cudaMemcpyAsync(out_host, base + kOutOffset, planes * nsite * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, base + kErrOffset, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(RLBM_ECUDA, std::string("read-back: ") + cudaGetErrorString(e));
  if (flags) return fail(RLBM_ENONPHYS, "non-physical site(s) in the populations");
  return RLBM_OK;
}
