// C ABI of the native 3D lattices (include/rlbm.h, "native 3D lattices").
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "rlbm_fieldscan.h"
#include "rlbm_devmem.h"
#include "rlbm_o3_3d.h"
#include "rlbm_stencil.h"
#include "rlbm_stencils.h"

using namespace rlbm;

struct rlbm_ctx3 {
  int Nx = 0, Ny = 0, Nz = 0;
  rlbm_dtype dtype = RLBM_F64;
  cudaStream_t stream = nullptr;
  double m = 0, tau = 0;
  StencilBuild3 sb;
  int Q = 0;
  long long pitch = 0, plane = 0;
  size_t elem = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;                 // buffer the next step pulls from
  long long t = 0;
  unsigned* d_err = nullptr;
  double* d_rt64 = nullptr;
  float* d_rt32 = nullptr;
  double* d_dr64 = nullptr;      // the lattice's dR(Td) table (compiled kernel's EOS step)
  int* d_shift = nullptr;
  long long* d_off = nullptr;
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  double* d_fields = nullptr;  // 5 planes for rlbm3_init, then the field check's scratch
  double* d_out = nullptr;
  size_t out_cap = 0;
  size_t device_bytes = 0;
  bool initialised = false;
  Step3Params p{};
  int fused = 0;               // 0 generic kernel; 1..4: {5,12,14,17,21,26}, {1..6},
                               // {1,14,49,51,60,70}, {3,9,10,14,17,21} (FP32)
  Fused3Params fp{};
  // third-order (eleven-group) stencils: the dual-basis tables and the
  // kernel parameters (q.b mirrors p at every launch)
  int order = 2;
  double* d_w64 = nullptr;
  float* d_w32 = nullptr;
  Step3O3Params q{};
  DevMem mem;                  // device allocator (rlbm_set_allocator at creation)
  std::string last_error;
};

namespace {

thread_local std::string g_create_error3;

rlbm_status fail3(rlbm_ctx3* c, rlbm_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  else g_create_error3 = msg;
  return s;
}

rlbm_status cuda_fail3(rlbm_ctx3* c, cudaError_t e, const char* where) {
  return fail3(c, RLBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void release3(rlbm_ctx3* c) {
  if (c->buf[0] || c->buf[1]) cudaStreamSynchronize(c->stream);
  for (void* p : {c->buf[0], c->buf[1], (void*)c->d_err, (void*)c->d_rt64, (void*)c->d_rt32, (void*)c->d_dr64,
                  (void*)c->d_shift, (void*)c->d_off,
                  (void*)c->d_tab64, (void*)c->d_tab32, (void*)c->d_fields, (void*)c->d_out, (void*)c->d_w64,
                  (void*)c->d_w32})
    c->mem.put(p);
  c->buf[0] = c->buf[1] = nullptr;
}

HL split3(double v) {
  HL h;
  h.hi = (float)v;
  h.lo = (float)(v - (double)h.hi);
  return h;
}

// The compiled 3D stencil for these groups, when its population order is the
// host's (the storage planes) and the lattice is at least a halo wide.
template <class D>
bool same_order(const rlbm_ctx3* c) {
  for (int k = 0; k < 6; ++k)
    if (c->sb.sb.groups[k] != D::groups[k]) return false;
  if (D::Q != c->Q) return false;
  for (int i = 0; i < D::Q; ++i) {
    const Pop3& q = c->sb.pops[i];
    if (q.group != D::U.grp[i] || q.nx != D::U.nx[i] || q.ny != D::U.ny[i] || q.nz != D::U.nz[i]) return false;
  }
  const int h = D::U.halo;
  return c->Nx >= h && c->Ny >= h && c->Nz >= h;
}

int fused3_kind(const rlbm_ctx3* c) {
  if (c->dtype != RLBM_F32) return 0;
  if (same_order<Stencil3M1>(c)) return 1;
  if (same_order<Stencil3G16>(c)) return 2;
  if (same_order<Stencil3E5>(c)) return 3;
  if (same_order<Stencil3S2>(c)) return 4;
  return 0;
}

// Parameters of the stencil-specialised 3D kernel at reference density nref.
void fill_fused3(rlbm_ctx3* c, double nref) {
  Fused3Params& f = c->fp;
  std::memset(&f, 0, sizeof f);
  const StencilBuild& sb = c->sb.sb;
  f.Nx = c->Nx;
  f.Ny = c->Ny;
  f.Nz = c->Nz;
  f.pitch = c->pitch;
  f.zstride = c->pitch * c->Ny;
  f.plane = c->plane;
  f.inv_tau = (float)(1.0 / c->tau);
  f.v0 = (float)sb.v0;
  f.mb = (float)sb.mbar;
  f.k21 = (float)sb.sc.k21;
  f.cb00_1 = (float)sb.sc.cb00_1;
  f.mY = (float)sb.sc.mY;
  f.cv_r = (float)sb.cv_r;
  f.Rr = split3(sb.sc.Rr);
  const double N0r = nref * c->sb.mref1[0];
  const double er = nref * c->sb.mref1[4];
  f.nr = split3(N0r);
  f.yr = split3(er / N0r);
  for (int k = 0; k < 14; ++k) f.mref[k] = split3(nref * c->sb.mref1[k]);
  f.Rr64 = sb.sc.Rr;
  f.mb64 = sb.mbar;
  for (int g = 0; g < 6; ++g) {
    for (int q = 0; q < 5; ++q) f.gm[g][q] = split3(sb.gm[g][q]);
    for (int q = 0; q < 10; ++q) f.gf[g][q] = split3(c->sb.gf3[g][q]);
  }
  f.rt64 = c->d_rt64;
  f.rt32 = c->d_rt32;
  f.dr64 = c->d_dr64;
  f.err = c->d_err;
}

// Reference r_i of the FP32 storage at density nref (FP64 storage: none).
void set_reference3(rlbm_ctx3* c, double nref) {
  if (c->dtype == RLBM_F64) nref = 0.0;
  c->p.nref = nref;
  c->p.b0ref = c->order == 3 ? 0.0 : nref * c->sb.sb.b0ref1;
  for (int k = 0; k < 14; ++k) c->p.mref[k] = nref * c->sb.mref1[k];
  if (c->fused) fill_fused3(c, nref);
}

rlbm_status check_error3(rlbm_ctx3* c) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail3(c, e, "device synchronisation");
  if (h) {
    cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    std::string msg = "non-physical site(s):";
    if (h & ERR_LANDAU) msg += " Landau frame failed or |u| >= 1;";
    if (h & ERR_DENSITY) msg += " n <= 0;";
    if (h & ERR_EOS) msg += " e/n <= m or T <= 0;";
    if (h & ERR_ZETA) msg += " zeta = m/T invalid;";
    return fail3(c, RLBM_ENONPHYS, msg);
  }
  return RLBM_OK;
}

}  // namespace

extern "C" {

rlbm_status rlbm3_create(const rlbm_stencil* st, double m, double tau, int Nx, int Ny, int Nz,
                         rlbm_dtype dtype, void* cuda_stream, rlbm_ctx3** out) {
  if (!out) return fail3(nullptr, RLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (Nx < 1 || Ny < 1 || Nz < 1) return fail3(nullptr, RLBM_EINVAL, "Nx, Ny and Nz must be >= 1");
  if ((long long)Nx * Ny * Nz > INT_MAX)
    return fail3(nullptr, RLBM_EINVAL, "Nx * Ny * Nz exceeds 2^31 - 1 (the kernels index sites with 32-bit integers)");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail3(nullptr, RLBM_EINVAL, "tau must exceed 1/2");
  if (dtype == RLBM_BF16_DEV) return fail3(nullptr, RLBM_ENOTSUP, "3D lattices store FP64 or FP32");
  if (dtype != RLBM_F64 && dtype != RLBM_F32) return fail3(nullptr, RLBM_EINVAL, "unknown dtype");
  std::unique_ptr<rlbm_ctx3> c(new (std::nothrow) rlbm_ctx3);
  if (!c) return fail3(nullptr, RLBM_ENOMEM, "host allocation failed");
  std::string err;
  std::unique_ptr<StencilBuild3O3> s3;
  if (st && st->ngroups == 11) {
    s3.reset(new StencilBuild3O3);
    rlbm_status s = build_stencil3d_o3(st, m, s3.get(), &err);
    if (s != RLBM_OK) return fail3(nullptr, s, err);
    c->sb = s3->base;
    c->order = 3;
  } else {
    rlbm_status s = build_stencil3d(st, m, &c->sb, &err);
    if (s != RLBM_OK) return fail3(nullptr, s, err);
  }
  c->Nx = Nx;
  c->Ny = Ny;
  c->Nz = Nz;
  c->dtype = dtype;
  c->m = m;
  c->tau = tau;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->Q = (int)c->sb.pops.size();
  c->elem = dtype == RLBM_F64 ? sizeof(double) : sizeof(float);
  c->pitch = ((long long)Nx + 31) / 32 * 32;
  c->plane = c->pitch * Ny * Nz;
  if (c->plane >= (1LL << 32))
    return fail3(nullptr, RLBM_ENOTSUP, "a population plane exceeds 2^32 elements (32-bit element indices)");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail3(nullptr, RLBM_ECUDA, "no CUDA device available");
  c->mem = current_devmem(c->stream);
  // constant table [Q][kRow3], shifts [3][Q], interior offsets [Q]
  const int Q = c->Q;
  const long long pitch = ((long long)Nx + 31) / 32 * 32;
  std::vector<double> t64((size_t)kRow3 * Q, 0.0);
  std::vector<float> t32((size_t)kRow3 * Q, 0.0f);
  std::vector<int> sh((size_t)3 * Q);
  std::vector<long long> off(Q);
  for (int i = 0; i < Q; ++i) {
    const Pop3& q = c->sb.pops[i];
    for (int k = 0; k < kPop3; ++k) {
      t64[(size_t)i * kRow3 + k] = q.c[k];
      t32[(size_t)i * kRow3 + k] = (float)q.c[k];
    }
    sh[i] = ((q.nx % Nx) + Nx) % Nx;
    sh[Q + i] = ((q.ny % Ny) + Ny) % Ny;
    sh[2 * Q + i] = ((q.nz % Nz) + Nz) % Nz;
    off[i] = -(((long long)q.nz * Ny + q.ny) * pitch + q.nx);
  }
  const size_t fbytes = (size_t)Q * (size_t)c->plane * c->elem;
  const size_t nsite = (size_t)Nx * Ny * Nz;
  const auto& r64 = ratio_table64();
  const auto& r32 = ratio_table32();
  const std::vector<double> drt = dr_table(m);
  bool ok = c->mem.get(&c->buf[0], fbytes) == cudaSuccess && c->mem.get(&c->buf[1], fbytes) == cudaSuccess &&
            c->mem.get(&c->d_err, sizeof(unsigned)) == cudaSuccess &&
            c->mem.get(&c->d_rt64, r64.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_rt32, r32.size() * sizeof(float)) == cudaSuccess &&
            c->mem.get(&c->d_dr64, drt.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_shift, sh.size() * sizeof(int)) == cudaSuccess &&
            c->mem.get(&c->d_off, off.size() * sizeof(long long)) == cudaSuccess &&
            c->mem.get(&c->d_tab64, t64.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_tab32, t32.size() * sizeof(float)) == cudaSuccess &&
            c->mem.get(&c->d_fields, (5 * nsite + kScanBlocks + 1) * sizeof(double)) == cudaSuccess;
  std::vector<double> w64;
  std::vector<float> w32;
  if (ok && c->order == 3) {
    w64.assign((size_t)kRowW3 * Q, 0.0);
    w32.assign((size_t)kRowW3 * Q, 0.0f);
    for (int i = 0; i < Q; ++i)
      for (int l = 0; l < kRowW3; ++l) {
        w64[(size_t)i * kRowW3 + l] = s3->wrows[i][l];
        w32[(size_t)i * kRowW3 + l] = (float)s3->wrows[i][l];
      }
    ok = c->mem.get(&c->d_w64, w64.size() * sizeof(double)) == cudaSuccess &&
         c->mem.get(&c->d_w32, w32.size() * sizeof(float)) == cudaSuccess;
  }
  if (!ok) {
    release3(c.get());
    return fail3(nullptr, RLBM_ENOMEM, "device allocation failed");
  }
  c->device_bytes = 2 * fbytes + r64.size() * 8 + r32.size() * 4 + drt.size() * 8 + sh.size() * 4 + off.size() * 8 + t64.size() * 12 +
                    (5 * nsite + kScanBlocks + 1) * 8 + 4;
  e = cudaMemcpy(c->d_rt64, r64.data(), r64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_rt32, r32.data(), r32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_dr64, drt.data(), drt.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_shift, sh.data(), sh.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tab64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tab32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->order == 3) {
    e = cudaMemcpy(c->d_w64, w64.data(), w64.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_w32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice);
    c->device_bytes += w64.size() * 12;
  }
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
  // pageable uploads may return before their DMA lands: finish them before
  // any kernel runs on a stream that is not ordered after the legacy stream
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    release3(c.get());
    return fail3(nullptr, RLBM_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  Step3Params& p = c->p;
  p.Nx = Nx;
  p.Ny = Ny;
  p.Nz = Nz;
  p.Q = Q;
  p.pitch = c->pitch;
  p.plane = c->plane;
  p.inv_tau = 1.0 / tau;
  p.sc = c->sb.sb.sc;
  p.rt64 = c->d_rt64;
  p.rt32 = c->d_rt32;
  p.shift = c->d_shift;
  p.off = c->d_off;
  p.halo = c->sb.halo;
  p.tab64 = c->d_tab64;
  p.tab32 = c->d_tab32;
  p.err = c->d_err;
  c->fused = c->order == 3 ? 0 : fused3_kind(c.get());
  if (c->order == 3) {
    c->q.c = s3->c;
    c->q.w64 = c->d_w64;
    c->q.w32 = c->d_w32;
  }
  set_reference3(c.get(), 1.0);
  *out = c.release();
  return RLBM_OK;
}

rlbm_status rlbm3_init(rlbm_ctx3* c, const double* n, const double* ux, const double* uy, const double* uz,
                       const double* T) {
  if (!c) return RLBM_EINVAL;
  if (!n || !ux || !uy || !uz || !T) return fail3(c, RLBM_EINVAL, "NULL field pointer");
  const size_t N = (size_t)c->Nx * c->Ny * c->Nz;
  // upload, then a device check of the copy; populations are written after it passed
  const double* src[5] = {n, ux, uy, uz, T};
  for (int k = 0; k < 5; ++k) {
    cudaError_t e = cudaMemcpyAsync(c->d_fields + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(c->stream);
      return cuda_fail3(c, e, "field upload");
    }
  }
  const double* d = c->d_fields;
  const FieldScan fs = check_fields(d, d + N, d + 2 * N, d + 3 * N, d + 4 * N, N, c->d_fields + 5 * N, c->stream);
  if (fs.err != cudaSuccess) return cuda_fail3(c, fs.err, "field check");
  if (fs.first_bad < N) {
    const size_t s = fs.first_bad;
    char b[200];
    std::snprintf(b, sizeof b, "invalid field at site %zu (x=%zu, y=%zu, z=%zu): need n>0, T>0, |u|<1", s,
                  s % (size_t)c->Nx, (s / (size_t)c->Nx) % (size_t)c->Ny, s / ((size_t)c->Nx * c->Ny));
    return fail3(c, RLBM_EINVAL, b);
  }
  set_reference3(c, fs.nsum / (double)N);
  Field3Ptrs fp{c->d_fields, c->d_fields + N, c->d_fields + 2 * N, c->d_fields + 3 * N, c->d_fields + 4 * N};
  c->q.b = c->p;
  cudaError_t e = c->order == 3 ? launch_init3d_o3(c->dtype, c->q, fp, c->buf[0], c->buf[1], c->stream)
                                : launch_init3d(c->dtype, c->p, fp, c->buf[0], c->buf[1], c->stream);
  if (e != cudaSuccess) return cuda_fail3(c, e, "init launch");
  c->cur = 0;
  c->t = 0;
  c->initialised = true;
  return check_error3(c);
}

rlbm_status rlbm3_step(rlbm_ctx3* c, int nsteps) {
  if (!c) return RLBM_EINVAL;
  if (nsteps < 0) return fail3(c, RLBM_EINVAL, "nsteps < 0");
  if (!c->initialised) return fail3(c, RLBM_EINVAL, "rlbm3_init has not been called");
  c->q.b = c->p;
  for (int k = 0; k < nsteps; ++k) {
    cudaError_t e;
    if (c->order == 3) e = launch_step3d_o3(c->dtype, c->q, c->buf[c->cur], c->buf[1 - c->cur], c->stream);
    else if (c->fused) e = launch_fused3d(c->fused, c->fp, c->buf[c->cur], c->buf[1 - c->cur], c->stream);
    else e = launch_step3d(c->dtype, c->p, c->buf[c->cur], c->buf[1 - c->cur], c->stream);
    if (e != cudaSuccess) return cuda_fail3(c, e, "step launch");
    c->cur = 1 - c->cur;
    ++c->t;
  }
  return RLBM_OK;
}

size_t rlbm3_moments_size(const rlbm_ctx3* c, unsigned mask) {
  if (!c) return 0;
  size_t planes = 0;
  for (unsigned b : {RLBM_M_N, RLBM_M_UX, RLBM_M_UY, RLBM_M_T, RLBM_M_E, RLBM_M_UZ})
    if (mask & b) ++planes;
  if (mask & RLBM_M_NVEC) planes += 4;
  if (mask & RLBM_M_TMN) planes += 10;
  return planes * (size_t)c->Nx * c->Ny * c->Nz;
}

rlbm_status rlbm3_moments(rlbm_ctx3* c, double* out, unsigned mask) {
  if (!c) return RLBM_EINVAL;
  if (!out) return fail3(c, RLBM_EINVAL, "out is NULL");
  if (!c->initialised) return fail3(c, RLBM_EINVAL, "rlbm3_init has not been called");
  if (mask & ~0xFFu) return fail3(c, RLBM_EINVAL, "unknown mask bits");
  const size_t need = rlbm3_moments_size(c, mask);
  if (need == 0) return RLBM_OK;
  // page-locked caller memory: the read-out kernel writes it directly
  double* direct = mapped_alias(out);
  if (!direct && need > c->out_cap) {
    c->mem.put(c->d_out);
    c->d_out = nullptr;
    c->out_cap = 0;
    cudaError_t e = c->mem.get(&c->d_out, need * sizeof(double));
    if (e != cudaSuccess) return fail3(c, RLBM_ENOMEM, "read-out buffer");
    c->out_cap = need;
  }
  MomentOut mo{direct ? direct : c->d_out, mask};
  // the pre-collision state at t is the pull of S_{t-1}, the buffer the last step read
  cudaError_t e = launch_moments3d(c->dtype, c->p, c->buf[1 - c->cur], mo, c->stream);
  if (e == cudaSuccess && !direct)
    e = cudaMemcpyAsync(out, c->d_out, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail3(c, e, "read-out");
  return check_error3(c);
}

rlbm_status rlbm3_sync(rlbm_ctx3* c) {
  if (!c) return RLBM_EINVAL;
  return check_error3(c);
}

rlbm_status rlbm3_get_info(const rlbm_ctx3* c, rlbm3_info* info) {
  if (!c || !info) return RLBM_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->Nx = c->Nx;
  info->Ny = c->Ny;
  info->Nz = c->Nz;
  info->Q = c->Q;
  info->halo = c->sb.halo;
  info->dtype = c->dtype;
  info->m = c->m;
  info->tau = c->tau;
  info->v0 = c->sb.sb.v0;
  info->t = c->t;
  info->bytes_per_site = 2 * (size_t)c->Q * c->elem;
  info->device_bytes = c->device_bytes + c->out_cap * sizeof(double);
  info->kernel = c->fused;
  info->order = c->order;
  return RLBM_OK;
}

const char* rlbm3_last_error(const rlbm_ctx3* c) {
  return c ? c->last_error.c_str() : g_create_error3.c_str();
}

void rlbm3_destroy(rlbm_ctx3* c) {
  if (!c) return;
  release3(c);
  delete c;
}

}  // extern "C"
