// C ABI of the library (include/rlbm.h): context lifetime, validation,
// device buffers, launches and error reporting.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "rlbm_devmem.h"
#include "rlbm_fieldscan.h"
#include "rlbm_fused_launch.h"
#include "rlbm_stencil.h"

using namespace rlbm;

struct rlbm_ctx {
  int Nx = 0, Ny = 0;
  rlbm_dtype dtype = RLBM_F32;
  cudaStream_t stream = nullptr;
  double m = 0, tau = 0;
  StencilBuild sb;
  int Q = 0, qb = 0;
  long long pitch = 0, plane = 0;
  size_t elem = 0;
  void* buf[2] = {nullptr, nullptr};
  void* coef[2] = {nullptr, nullptr};   // BF16 storage: per-site reference coefficients
  int cur = 0;              // buffer holding S_t
  long long t = 0;
  unsigned* d_err = nullptr;
  double* d_rt64 = nullptr;
  float* d_rt32 = nullptr;
  double* d_dr64 = nullptr;      // the lattice's dR(Td) table (FP32 kernels' EOS step)
  double* d_fields = nullptr;   // 4 planes for rlbm_init, then the field check's scratch
  double* d_out = nullptr;      // read-out planes
  size_t out_cap = 0;
  size_t device_bytes = 0;
  bool initialised = false;
  bool host_init = false;   // rlbm_init in progress (it sets the reference itself)
  bool fresh = false;       // FP32 compiled path: S_0 written in place by the init, not stepped yet
  std::unique_ptr<StepParams<double>> p64;
  std::unique_ptr<StepParams<float>> p32;
  int fused = 0;                 // 1: M1, 2: G1..G6, 3: E5, 4: S2; 0: generic kernel
  int ext = 0;                   // FP32 storage on a compiled stencil: extended moment sums
  std::unique_ptr<FusedParams> fp;
  // third-order stencils (eleven groups)
  int order = 2;
  std::unique_ptr<StencilBuildO3> sb3;
  std::unique_ptr<O3Params> o3;
  std::unique_ptr<FusedO3Params> fo3;   // compiled third-order kernel (fused == 5)
  int* d_shift = nullptr;
  long long* d_off = nullptr;
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  DevMem mem;                    // device allocator (rlbm_set_allocator at creation)
  std::string last_error;
};

static thread_local std::string g_create_error;
static void batch_forget(const rlbm_ctx* c);   // drop cached batch graphs that use c

// Variant of the compiled second-order kernel: 0 FP32, 1 BF16 deviation,
// 2 / 3 FP32 with extended moment sums of level 1 / 2.
static int fused_mode(const rlbm_ctx* c) {
  return c->dtype == RLBM_BF16_DEV ? 1 : (c->ext ? 1 + c->ext : 0);
}

// The allocator installed by rlbm_set_allocator (all null: cudaMalloc).
static std::mutex g_alloc_mutex;
static DevMem g_alloc;

DevMem rlbm::current_devmem(cudaStream_t stream) {
  DevMem m;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    m = g_alloc;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) m.device = dev;
  m.stream = stream;
  return m;
}

void rlbm::set_global_error(const std::string& msg) { g_create_error = msg; }

static rlbm_status fail(rlbm_ctx* c, rlbm_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  else g_create_error = msg;
  return s;
}

static rlbm_status cuda_fail(rlbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, RLBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static void release(rlbm_ctx* c) {
  if (!c) return;
  if (c->buf[0]) cudaStreamSynchronize(c->stream);
  for (void* p : {c->buf[0], c->buf[1], c->coef[0], c->coef[1], (void*)c->d_err, (void*)c->d_rt64, (void*)c->d_rt32,
                  (void*)c->d_dr64,
                  (void*)c->d_fields, (void*)c->d_out, (void*)c->d_shift, (void*)c->d_off, (void*)c->d_tab64,
                  (void*)c->d_tab32})
    c->mem.put(p);
}

template <typename CT>
static void fill_params(rlbm_ctx* c, StepParams<CT>* p) {
  std::memset(p, 0, sizeof(*p));
  p->Nx = c->Nx;
  p->Ny = c->Ny;
  p->Q = c->Q;
  p->halo = c->sb.halo;
  p->pitch = c->pitch;
  p->plane = c->plane;
  p->inv_tau = 1.0 / c->tau;
  p->v0 = c->sb.v0;
  p->sc = c->sb.sc;
  p->rt64 = c->d_rt64;
  p->rt32 = c->d_rt32;
  p->err = c->d_err;
  fill_pop_table<CT>(c->sb, c->Nx, c->Ny, &p->pt);
}

static HL split(double x) {
  HL h;
  h.hi = (float)x;
  h.lo = (float)(x - (double)h.hi);
  return h;
}

// Which stencil-specialised kernel serves this context (0: none).
static int fused_kind(const rlbm_ctx* c) {
  if (c->dtype == RLBM_F64) return 0;
  auto same = [&](const int* g) {
    for (int k = 0; k < 6; ++k)
      if (c->sb.groups[k] != g[k]) return false;
    return true;
  };
  int kind = 0;
  const Folded* F = nullptr;
  if (same(StencilM1::groups)) kind = 1, F = &StencilM1::F;
  else if (same(StencilG16::groups)) kind = 2, F = &StencilG16::F;
  else if (same(StencilE5::groups)) kind = 3, F = &StencilE5::F;
  else if (same(StencilS2::groups)) kind = 4, F = &StencilS2::F;
  if (!kind || F->Q != c->Q || F->halo != c->sb.halo) return 0;
  // the compiled population order must be the host's (same storage planes)
  for (int i = 0; i < F->Q; ++i) {
    const FoldedPop& fp = c->sb.pops[i];
    if (fp.nx != F->nx[i] || fp.ny != F->ny[i] || fp.group != F->grp[i] || fp.mult != F->mult[i]) return 0;
  }
  const int halo = F->halo;
  // the kernels wrap a source coordinate at most once
  if (c->Nx < halo || c->Ny < halo) return 0;
  return kind;
}

static void fill_fused(rlbm_ctx* c, double nref) {
  FusedParams& f = *c->fp;
  std::memset(&f, 0, sizeof f);
  const StencilBuild& sb = c->sb;
  f.Nx = c->Nx;
  f.Ny = c->Ny;
  f.pitch = c->pitch;
  f.plane = c->plane;
  f.inv_tau = (float)(1.0 / c->tau);
  f.v0 = (float)sb.v0;
  f.mb = (float)sb.mbar;
  f.k21 = (float)sb.sc.k21;
  f.mk32 = (float)sb.sc.mk32;
  f.cb00_1 = (float)sb.sc.cb00_1;
  f.mY = (float)sb.sc.mY;
  f.cv_r = (float)sb.cv_r;
  f.Rr = split(sb.sc.Rr);
  const double N0r = nref * sb.mref1[0];
  const double er = nref * sb.mref1[3];
  const double pr = nref * sb.mref1[6];
  f.nr = split(N0r);
  f.yr = split(er / N0r);
  for (int k = 0; k < 9; ++k) f.mref[k] = split(nref * sb.mref1[k]);
  f.Rr64 = sb.sc.Rr;
  f.hr64 = er + pr;
  f.mb64 = sb.mbar;
  f.nr64 = N0r;
  for (int g = 0; g < 6; ++g) {
    for (int q = 0; q < 5; ++q) f.gm[g][q] = split(sb.gm[g][q]);
    for (int q = 0; q < 10; ++q) f.gf[g][q] = split(sb.gf[g][q]);
    for (int q = 0; q < 2; ++q) f.gk[g][q] = split(sb.gk[g][q]);
    for (int q = 0; q < 5; ++q) f.gm64[g][q] = sb.gm[g][q];
    // split grid q = 2^(ceil(log2 r_g) - 11), r_g the group's largest
    // reference population: its h-sums (at most 24 members, weights up to 6)
    // stay exact while the pulled values stay below about 50 r_g
    const int e = (int)std::ceil(std::log2(nref * sb.rmax1[g]));
    f.exC[g] = (float)std::ldexp(1.5, 23 + e - 11);
  }
  for (int g = 0; g < 6; ++g) {
    const HL* m = f.gm[g];
    const HL pairs[4][2] = {{m[0], m[1]}, {m[2], m[2]}, {m[3], m[3]}, {m[4], m[4]}};
    for (int q = 0; q < 4; ++q) {
      f.gm2[g][2 * q] = make_float2(pairs[q][0].hi, pairs[q][1].hi);
      f.gm2[g][2 * q + 1] = make_float2(pairs[q][0].lo, pairs[q][1].lo);
    }
  }
  for (int j = 0; j < 3; ++j)
    for (int q = 0; q < 10; ++q) {
      f.gf2[j][q][0] = make_float2(f.gf[2 * j][q].hi, f.gf[2 * j + 1][q].hi);
      f.gf2[j][q][1] = make_float2(f.gf[2 * j][q].lo, f.gf[2 * j + 1][q].lo);
    }
  {
    // multiplier of the exact division by Nx (Granlund-Montgomery): with
    // 2^(l-1) < Nx <= 2^l, m = ceil(2^(31+l) / Nx) = (2^(31+l) + e) / Nx,
    // 0 <= e < Nx, is below 2^32, and s m / 2^(31+l) exceeds s / Nx by
    // s e / (Nx 2^(31+l)) < 2^-l <= 1/Nx for s < 2^31: too little to reach
    // the next integer, so the floor is s / Nx
    int l = 0;
    while ((1LL << l) < c->Nx) ++l;
    f.nx_m = (unsigned)(((1ULL << (31 + l)) + (unsigned long long)c->Nx - 1) / (unsigned long long)c->Nx);
    f.nx_sh = 31 + l;
  }
  // fixed pull offsets of the sites that need no wrapping (BF16 kernels):
  // bfloat16 slots (two per word, population i in half half[i] of word plane
  // word[i]) from the site's slot 0 of word plane 0, coefficient words from
  // its word of group 0
  const BfWords* bw = c->fused == 1 ? &StencilM1::B : c->fused == 2 ? &StencilG16::B
                    : c->fused == 3 ? &StencilE5::B : &StencilS2::B;
  const int H = sb.halo;
  const long long span = 2LL * (c->Q + 1) * c->plane + 2LL * H * (c->pitch + 1);
  if (c->Q <= kMaxQ2 && span < INT_MAX && c->Nx > 2 * H && c->Ny > 2 * H) {
    f.inner_nx = c->Nx - 2 * H;
    f.inner_ny = c->Ny - 2 * H;
    for (int i = 0; i < c->Q; ++i) {
      const FoldedPop& fp = sb.pops[i];
      const long long back = (long long)fp.ny * c->pitch + fp.nx;
      f.doff[i] = (int)(2 * ((long long)bw->word[i] * c->plane - back) + bw->half[i]);
      f.dcoff[i] = (int)((long long)fp.group * c->plane - back);
    }
  }
  f.k0r = split(nref * sb.kref1);
  f.ykr = split(sb.ykr1);
  f.rt64 = c->d_rt64;
  f.rt32 = c->d_rt32;
  f.dr64 = c->d_dr64;
  f.err = c->d_err;
}

// Compiled third-order kernels (rlbm_fused_o3.cu): kind 5..10 for the
// groups of StencilO3M5, StencilO3D, StencilO3E, StencilO3A, StencilO3B,
// StencilO3C.
template <class D>
static bool fused_o3_is(const rlbm_ctx* c) {
  if (c->Q != D::Q || c->sb3->halo != D::halo) return false;
  for (int k = 0; k < 11; ++k)
    if (c->sb3->groups[k] != D::groups[k]) return false;
  for (int i = 0; i < D::Q; ++i) {
    const FoldedPop& fp = c->sb3->pops[i];
    if (fp.nx != D::F.nx[i] || fp.ny != D::F.ny[i] || fp.group != D::F.grp[i] || fp.mult != D::F.mult[i])
      return false;
  }
  return true;
}

// Which compiled third-order kernel serves this context (0: none): FP32,
// compiled groups in the host's population order, Nx, Ny >= halo.
static int fused_o3_kind(const rlbm_ctx* c) {
  if (c->dtype != RLBM_F32 || c->Nx < c->sb3->halo || c->Ny < c->sb3->halo) return 0;
  if (fused_o3_is<StencilO3M5>(c)) return 5;
  if (fused_o3_is<StencilO3D>(c)) return 6;
  if (fused_o3_is<StencilO3E>(c)) return 7;
  if (fused_o3_is<StencilO3A>(c)) return 8;
  if (fused_o3_is<StencilO3B>(c)) return 9;
  if (fused_o3_is<StencilO3C>(c)) return 10;
  return 0;
}

template <class D>
static void fill_orbits_o3(const StencilBuildO3& sb, FusedO3Params& f) {
  for (int k = 0; k < D::O.K; ++k) {
    const auto& row = sb.rows[D::O.idx[k][0]];
    for (int l = 0; l <= kO3Mono; ++l) f.ow[k][l] = split(row[9 + l]);
  }
}

static void fill_fused_o3(rlbm_ctx* c, double nref) {
  FusedO3Params& f = *c->fo3;
  std::memset(&f, 0, sizeof f);
  const StencilBuildO3& sb = *c->sb3;
  f.Nx = c->Nx;
  f.Ny = c->Ny;
  f.pitch = c->pitch;
  f.plane = c->plane;
  f.inv_tau = (float)(1.0 / c->tau);
  f.v0 = (float)sb.v0;
  f.mb = (float)sb.mbar;
  f.cv_r = (float)sb.cv_r;
  f.c = (float)sb.c;
  f.Rr = split(sb.sc.Rr);
  const double N0r = nref * sb.mref1[0];
  const double er = nref * sb.mref1[3];
  f.nr = split(N0r);
  f.yr = split(er / N0r);
  for (int k = 0; k < 9; ++k) f.mref[k] = split(nref * sb.mref1[k]);
  f.Rr64 = sb.sc.Rr;
  f.mb64 = sb.mbar;
  for (int g = 0; g < 11; ++g)
    for (int q = 0; q < 5; ++q) f.gm[g][q] = split(sb.gm[g][q]);
  switch (c->fused) {
    case 5: fill_orbits_o3<StencilO3M5>(sb, f); break;
    case 6: fill_orbits_o3<StencilO3D>(sb, f); break;
    case 7: fill_orbits_o3<StencilO3E>(sb, f); break;
    case 8: fill_orbits_o3<StencilO3A>(sb, f); break;
    case 9: fill_orbits_o3<StencilO3B>(sb, f); break;
    default: fill_orbits_o3<StencilO3C>(sb, f); break;
  }
  f.rt64 = c->d_rt64;
  f.rt32 = c->d_rt32;
  f.dr64 = c->d_dr64;
  f.err = c->d_err;
}

// Reference density of the FP32 deviation storage (see StepParams).
static void set_reference(rlbm_ctx* c, double nref) {
  if (c->dtype == RLBM_F64) return;
  if (c->order == 3) {
    c->o3->nref = nref;
    for (int k = 0; k < 9; ++k) c->o3->mref[k] = nref * c->sb3->mref1[k];
    if (c->fo3) fill_fused_o3(c, nref);
    return;
  }
  for (StepParams<double>* p : {c->p64.get()}) {
    p->nref = nref;
    p->b0ref = nref * c->sb.b0ref1;
    for (int k = 0; k < 9; ++k) p->mref[k] = nref * c->sb.mref1[k];
  }
  StepParams<float>* q = c->p32.get();
  q->nref = nref;
  q->b0ref = nref * c->sb.b0ref1;
  for (int k = 0; k < 9; ++k) q->mref[k] = nref * c->sb.mref1[k];
  if (c->fused) fill_fused(c, nref);
}

static rlbm_status check_device_error(rlbm_ctx* c) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device synchronisation");
  if (h) {
    cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream);
    cudaStreamSynchronize(c->stream);
    if (h & ERR_TIMEOUT)
      return fail(c, RLBM_ETIMEOUT,
                  "a bounded device-side wait of the persistent batch kernel ran out; the lattice's state is "
                  "undefined until rlbm_init");
    std::string msg = "non-physical site(s):";
    if (h & ERR_LANDAU) msg += " Landau frame failed or |u| >= 1;";
    if (h & ERR_DENSITY) msg += " n <= 0;";
    if (h & ERR_EOS) msg += " e/n <= m or T <= 0;";
    if (h & ERR_ZETA) msg += " zeta = m/T invalid;";
    return fail(c, RLBM_ENONPHYS, msg);
  }
  return RLBM_OK;
}

// Context of a third-order (eleven-group) stencil: FP64 or FP32 storage,
// generic kernels over a device table (rlbm_kernels_o3.cu).
static rlbm_status create_o3(const rlbm_stencil* st, double m, double tau, int Nx, int Ny, rlbm_dtype dtype,
                             void* cuda_stream, rlbm_ctx** out) {
  if (dtype == RLBM_BF16_DEV)
    return fail(nullptr, RLBM_ENOTSUP, "third-order stencils support FP64 and FP32 storage only");
  std::unique_ptr<rlbm_ctx> c(new (std::nothrow) rlbm_ctx);
  if (!c) return fail(nullptr, RLBM_ENOMEM, "host allocation failed");
  c->sb3.reset(new StencilBuildO3);
  std::string err;
  rlbm_status s = build_stencil_o3(st, m, c->sb3.get(), &err);
  if (s != RLBM_OK) return fail(nullptr, s, err);
  const StencilBuildO3& sb = *c->sb3;
  c->order = 3;
  c->Nx = Nx;
  c->Ny = Ny;
  c->dtype = dtype;
  c->m = m;
  c->tau = tau;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->Q = (int)sb.pops.size();
  c->elem = (dtype == RLBM_F64) ? sizeof(double) : sizeof(float);
  c->pitch = ((long long)Nx + 31) / 32 * 32;
  c->plane = c->pitch * Ny;
  c->sb.halo = sb.halo;
  if (c->plane >= (1LL << 32))
    return fail(nullptr, RLBM_ENOTSUP, "a population plane exceeds 2^32 elements (32-bit element indices)");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(nullptr, RLBM_ECUDA, "no CUDA device available");
  c->mem = current_devmem(c->stream);
  const int Q = c->Q;
  const size_t fbytes = (size_t)Q * (size_t)c->plane * c->elem;
  for (int b = 0; b < 2; ++b) {
    e = c->mem.get(&c->buf[b], fbytes);
    if (e != cudaSuccess) {
      release(c.get());
      return fail(nullptr, RLBM_ENOMEM, "population buffers: " + std::string(cudaGetErrorString(e)));
    }
  }
  const auto& t64 = ratio_table64();
  const auto& t32 = ratio_table32();
  const std::vector<double> drt = dr_table(m);
  const size_t nsite = (size_t)Nx * Ny;
  const size_t tbytes = (size_t)Q * kRowO3;
  bool ok = c->mem.get(&c->d_err, sizeof(unsigned)) == cudaSuccess &&
            c->mem.get(&c->d_rt64, t64.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_rt32, t32.size() * sizeof(float)) == cudaSuccess &&
            c->mem.get(&c->d_dr64, drt.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_fields, (4 * nsite + kScanBlocks + 1) * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_shift, 2 * Q * sizeof(int)) == cudaSuccess &&
            c->mem.get(&c->d_off, Q * sizeof(long long)) == cudaSuccess &&
            c->mem.get(&c->d_tab64, tbytes * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_tab32, tbytes * sizeof(float)) == cudaSuccess;
  if (!ok) {
    release(c.get());
    return fail(nullptr, RLBM_ENOMEM, "device allocation failed");
  }
  c->device_bytes = 2 * fbytes + sizeof(unsigned) + t64.size() * 8 + t32.size() * 4 + drt.size() * 8 +
                    (4 * nsite + kScanBlocks + 1) * 8 + 2 * Q * sizeof(int) + Q * sizeof(long long) + tbytes * 12;
  std::vector<int> shift(2 * Q);
  std::vector<long long> off(Q);
  std::vector<double> tab64(tbytes);
  std::vector<float> tab32(tbytes);
  for (int i = 0; i < Q; ++i) {
    const FoldedPop& fp = sb.pops[i];
    shift[i] = ((fp.nx % Nx) + Nx) % Nx;
    shift[Q + i] = ((fp.ny % Ny) + Ny) % Ny;
    off[i] = -((long long)fp.ny * c->pitch + fp.nx);
    for (int k = 0; k < kRowO3; ++k) {
      tab64[(size_t)i * kRowO3 + k] = sb.rows[i][k];
      tab32[(size_t)i * kRowO3 + k] = (float)sb.rows[i][k];
    }
  }
  e = cudaMemcpy(c->d_rt64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_rt32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_shift, shift.data(), shift.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tab64, tab64.data(), tbytes * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tab32, tab32.data(), tbytes * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_dr64, drt.data(), drt.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
  // pageable uploads may return before their DMA lands: finish them before
  // any kernel runs on a stream that is not ordered after the legacy stream
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    release(c.get());
    return fail(nullptr, RLBM_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  c->o3.reset(new O3Params);
  O3Params& p = *c->o3;
  std::memset(&p, 0, sizeof p);
  p.Nx = Nx;
  p.Ny = Ny;
  p.Q = Q;
  p.halo = sb.halo;
  p.pitch = c->pitch;
  p.plane = c->plane;
  p.inv_tau = 1.0 / tau;
  p.c = sb.c;
  p.sc = sb.sc;
  p.rt64 = c->d_rt64;
  p.rt32 = c->d_rt32;
  p.shift = c->d_shift;
  p.off = c->d_off;
  p.tab64 = c->d_tab64;
  p.tab32 = c->d_tab32;
  p.err = c->d_err;
  c->fused = fused_o3_kind(c.get());
  if (c->fused) {
    c->fo3.reset(new FusedO3Params);
    fill_fused_o3(c.get(), 1.0);
  }
  *out = c.release();
  return RLBM_OK;
}

extern "C" {

const char* rlbm_version(void) { return "rlbm-gb300 0.1 (sm_103a)"; }

rlbm_status rlbm_set_allocator(rlbm_alloc_fn alloc, rlbm_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, RLBM_EINVAL, "rlbm_set_allocator: give both alloc and free_fn, or neither");
  std::lock_guard<std::mutex> lock(g_alloc_mutex);
  g_alloc.alloc = alloc;
  g_alloc.release = free_fn;
  g_alloc.user = alloc ? user : nullptr;
  return RLBM_OK;
}

rlbm_status rlbm_create(const rlbm_stencil* st, double m, double tau, int Nx, int Ny,
                        rlbm_dtype dtype, void* cuda_stream, rlbm_ctx** out) {
  if (!out) return fail(nullptr, RLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (Nx < 1 || Ny < 1) return fail(nullptr, RLBM_EINVAL, "Nx and Ny must be >= 1");
  if ((long long)Nx * Ny > INT_MAX)
    return fail(nullptr, RLBM_EINVAL, "Nx * Ny exceeds 2^31 - 1 (the kernels index sites with 32-bit integers)");
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, RLBM_EINVAL, "tau must exceed 1/2");
  if (dtype != RLBM_F64 && dtype != RLBM_F32 && dtype != RLBM_BF16_DEV)
    return fail(nullptr, RLBM_EINVAL, "unknown dtype");
  if (st && st->ngroups == 11) return create_o3(st, m, tau, Nx, Ny, dtype, cuda_stream, out);
  std::unique_ptr<rlbm_ctx> c(new (std::nothrow) rlbm_ctx);
  if (!c) return fail(nullptr, RLBM_ENOMEM, "host allocation failed");
  std::string err;
  rlbm_status s = build_stencil(st, m, &c->sb, &err);
  if (s != RLBM_OK) return fail(nullptr, s, err);
  c->Nx = Nx;
  c->Ny = Ny;
  c->dtype = dtype;
  c->m = m;
  c->tau = tau;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->Q = (int)c->sb.pops.size();
  c->qb = 0;
  for (int q : QBUCKETS)
    if (c->Q <= q) {
      c->qb = q;
      break;
    }
  if (!c->qb) return fail(nullptr, RLBM_ENOTSUP, "too many populations");
  c->elem = (dtype == RLBM_F64) ? sizeof(double) : (dtype == RLBM_F32) ? sizeof(float) : 2;
  c->pitch = ((long long)Nx + 31) / 32 * 32;
  c->plane = c->pitch * Ny;
  if (c->plane >= (1LL << 32))
    return fail(nullptr, RLBM_ENOTSUP, "a population plane exceeds 2^32 elements (32-bit element indices)");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(nullptr, RLBM_ECUDA, "no CUDA device available");
  c->mem = current_devmem(c->stream);
  // BF16: two bfloat16 values a 32-bit word, so Q rounded up to even slots
  const size_t slots = dtype == RLBM_BF16_DEV ? (size_t)((c->Q + 1) / 2 * 2) : (size_t)c->Q;
  const size_t fbytes = slots * (size_t)c->plane * c->elem;
  for (int b = 0; b < 2; ++b) {
    e = c->mem.get(&c->buf[b], fbytes);
    if (e != cudaSuccess) {
      release(c.get());
      return fail(nullptr, RLBM_ENOMEM, "population buffers: " + std::string(cudaGetErrorString(e)));
    }
  }
  const auto& t64 = ratio_table64();
  const auto& t32 = ratio_table32();
  const std::vector<double> drt = dr_table(m);
  const size_t nsite = (size_t)Nx * Ny;
  bool ok = c->mem.get(&c->d_err, sizeof(unsigned)) == cudaSuccess &&
            c->mem.get(&c->d_rt64, t64.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_rt32, t32.size() * sizeof(float)) == cudaSuccess &&
            c->mem.get(&c->d_dr64, drt.size() * sizeof(double)) == cudaSuccess &&
            c->mem.get(&c->d_fields, (4 * nsite + kScanBlocks + 1) * sizeof(double)) == cudaSuccess;
  if (!ok) {
    release(c.get());
    return fail(nullptr, RLBM_ENOMEM, "device allocation failed");
  }
  c->device_bytes = 2 * fbytes + sizeof(unsigned) + t64.size() * 8 + t32.size() * 4 + drt.size() * 8 +
                    (4 * nsite + kScanBlocks + 1) * 8;
  e = cudaMemcpy(c->d_rt64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_rt32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_dr64, drt.data(), drt.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
  // pageable uploads may return before their DMA lands: finish them before
  // any kernel runs on a stream that is not ordered after the legacy stream
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    release(c.get());
    return fail(nullptr, RLBM_ECUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  c->p64.reset(new StepParams<double>);
  fill_params<double>(c.get(), c->p64.get());
  if (dtype != RLBM_F64) {
    c->p32.reset(new StepParams<float>);
    fill_params<float>(c.get(), c->p32.get());
  }
  c->fused = fused_kind(c.get());
  if (c->fused) {
    c->fp.reset(new FusedParams);
    fill_fused(c.get(), 1.0);
  }
  if (dtype == RLBM_BF16_DEV) {
    if (!c->fused) {
      release(c.get());
      return fail(nullptr, RLBM_ENOTSUP,
                  "BF16 deviation storage needs a compiled stencil ({5,12,14,17,21,26}, {1..6}, "
                  "{1,14,49,51,60,70} or {3,9,10,14,17,21}) and Nx, Ny >= its halo");
    }
    const size_t cbytes = (size_t)6 * (size_t)c->plane * 8;
    for (int b = 0; b < 2; ++b) {
      e = c->mem.get(&c->coef[b], cbytes);
      if (e != cudaSuccess) {
        release(c.get());
        return fail(nullptr, RLBM_ENOMEM, "coefficient buffers: " + std::string(cudaGetErrorString(e)));
      }
    }
    c->device_bytes += 2 * cbytes;
  }
  *out = c.release();
  return RLBM_OK;
}

rlbm_status rlbm_init_device(rlbm_ctx* c, const double* n, const double* ux, const double* uy,
                             const double* T) {
  if (!c) return RLBM_EINVAL;
  if (!n || !ux || !uy || !T) return fail(c, RLBM_EINVAL, "NULL field pointer");
  FieldPtrs fp{n, ux, uy, T};
  batch_forget(c);   // its parameters change below
  if (!c->host_init) set_reference(c, 1.0);
  cudaError_t e;
  if (c->order == 3) {
    e = launch_init_o3(c->dtype, *c->o3, fp, c->buf[0], c->buf[1], c->stream);
  } else if (c->dtype == RLBM_BF16_DEV) {
    MomentOut none{nullptr, 0};
    if (c->fused == 1) e = launch_bf16_io<StencilM1>(0, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], c->coef[0], c->coef[1], none, c->stream);
    else if (c->fused == 2) e = launch_bf16_io<StencilG16>(0, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], c->coef[0], c->coef[1], none, c->stream);
    else if (c->fused == 3) e = launch_bf16_io<StencilE5>(0, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], c->coef[0], c->coef[1], none, c->stream);
    else e = launch_bf16_io<StencilS2>(0, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], c->coef[0], c->coef[1], none, c->stream);
  } else if (c->dtype == RLBM_F32 && c->fused) {
    MomentOut none{nullptr, 0};
    if (c->fused == 1) e = launch_bf16_io<StencilM1>(2, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], nullptr, nullptr, none, c->stream);
    else if (c->fused == 2) e = launch_bf16_io<StencilG16>(2, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], nullptr, nullptr, none, c->stream);
    else if (c->fused == 3) e = launch_bf16_io<StencilE5>(2, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], nullptr, nullptr, none, c->stream);
    else e = launch_bf16_io<StencilS2>(2, *c->fp, *c->p64, fp, c->buf[0], c->buf[1], nullptr, nullptr, none, c->stream);
  } else {
    e = launch_init(c->dtype, *c->p64, fp, c->buf[0], c->buf[1], c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "init launch");
  c->cur = 0;
  c->t = 0;
  c->initialised = true;
  c->fresh = c->order == 2 && c->dtype == RLBM_F32 && c->fused;
  return RLBM_OK;
}

rlbm_status rlbm_init(rlbm_ctx* c, const double* n, const double* ux, const double* uy,
                      const double* T) {
  if (!c) return RLBM_EINVAL;
  if (!n || !ux || !uy || !T) return fail(c, RLBM_EINVAL, "NULL field pointer");
  const size_t N = (size_t)c->Nx * c->Ny;
  // upload, then a device check of the copy (first invalid site, density
  // sum); the populations are written only after the check has passed
  const double* src[4] = {n, ux, uy, T};
  for (int k = 0; k < 4; ++k) {
    cudaError_t e = cudaMemcpyAsync(c->d_fields + k * N, src[k], N * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(c->stream);
      return cuda_fail(c, e, "field upload");
    }
  }
  const double* d = c->d_fields;
  const FieldScan fs = check_fields(d, d + N, d + 2 * N, nullptr, d + 3 * N, N, c->d_fields + 4 * N, c->stream);
  if (fs.err != cudaSuccess) return cuda_fail(c, fs.err, "field check");
  if (fs.first_bad < N) {
    const size_t s = fs.first_bad;
    char b[160];
    std::snprintf(b, sizeof b, "invalid field at site %zu (x=%zu, y=%zu): need n>0, T>0, |u|<1",
                  s, s % (size_t)c->Nx, s / (size_t)c->Nx);
    return fail(c, RLBM_EINVAL, b);
  }
  set_reference(c, fs.nsum / (double)N);
  c->host_init = true;
  rlbm_status s = rlbm_init_device(c, c->d_fields, c->d_fields + N, c->d_fields + 2 * N,
                                   c->d_fields + 3 * N);
  c->host_init = false;
  if (s != RLBM_OK) return s;
  return check_device_error(c);
}

rlbm_status rlbm_set_extended_sums(rlbm_ctx* c, int on) {
  if (!c) return RLBM_EINVAL;
  if (c->order != 2 || c->dtype != RLBM_F32 || !c->fused)
    return fail(c, RLBM_ENOTSUP, "extended moment sums need FP32 storage on a compiled second-order stencil");
  if (on < 0 || on > 2) return fail(c, RLBM_EINVAL, "extended sums level must be 0, 1 or 2");
  const int v = on;
  if (v != c->ext) batch_forget(c);
  c->ext = v;
  return RLBM_OK;
}

rlbm_status rlbm_step(rlbm_ctx* c, int nsteps) {
  if (!c) return RLBM_EINVAL;
  if (nsteps < 0) return fail(c, RLBM_EINVAL, "nsteps < 0");
  if (!c->initialised) return fail(c, RLBM_EINVAL, "rlbm_init has not been called");
  for (int k = 0; k < nsteps; ++k) {
    const void* fin = c->buf[c->cur];
    void* fout = c->buf[1 - c->cur];
    cudaError_t e;
    if (c->order == 3)
      e = c->fo3 ? launch_fused_o3(c->fused, *c->fo3, fin, fout, c->stream)
                 : launch_step_o3(c->dtype, *c->o3, fin, fout, c->stream);
    else if (c->dtype == RLBM_F64) e = launch_step_f64(*c->p64, fin, fout, c->qb, c->stream);
    else if (c->fused) {
      const int mode = fused_mode(c);
      c->fp->cin = c->coef[c->cur];
      c->fp->cout = c->coef[1 - c->cur];
      if (c->fused == 1) e = launch_fused<StencilM1>(*c->fp, fin, fout, mode, c->stream);
      else if (c->fused == 2) e = launch_fused<StencilG16>(*c->fp, fin, fout, mode, c->stream);
      else if (c->fused == 3) e = launch_fused<StencilE5>(*c->fp, fin, fout, mode, c->stream);
      else e = launch_fused<StencilS2>(*c->fp, fin, fout, mode, c->stream);
    }
    else e = launch_step_f32(*c->p32, fin, fout, c->qb, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    c->cur = 1 - c->cur;
    ++c->t;
    c->fresh = false;
  }
  return RLBM_OK;
}

size_t rlbm_moments_size(const rlbm_ctx* c, unsigned mask) {
  if (!c) return 0;
  size_t planes = 0;
  for (unsigned b : {RLBM_M_N, RLBM_M_UX, RLBM_M_UY, RLBM_M_T, RLBM_M_E})
    if (mask & b) ++planes;
  if (mask & RLBM_M_NVEC) planes += 3;
  if (mask & RLBM_M_TMN) planes += 6;
  return planes * (size_t)c->Nx * c->Ny;
}

rlbm_status rlbm_moments(rlbm_ctx* c, double* out, unsigned mask) {
  if (!c) return RLBM_EINVAL;
  if (!out) return fail(c, RLBM_EINVAL, "out is NULL");
  if (!c->initialised) return fail(c, RLBM_EINVAL, "rlbm_init has not been called");
  if (mask & ~0x7Fu) return fail(c, RLBM_EINVAL, "unknown mask bits");
  const size_t need = rlbm_moments_size(c, mask);
  if (need == 0) return RLBM_OK;
  // page-locked caller memory: the read-out kernel writes it directly
  double* direct = mapped_alias(out);
  if (!direct && need > c->out_cap) {
    c->mem.put(c->d_out);
    c->d_out = nullptr;
    c->out_cap = 0;
    cudaError_t e = c->mem.get(&c->d_out, need * sizeof(double));
    if (e != cudaSuccess) return fail(c, RLBM_ENOMEM, "read-out buffer");
    c->out_cap = need;
  }
  MomentOut mo{direct ? direct : c->d_out, mask};
  cudaError_t e;
  if (c->order == 3) {
    e = launch_moments_o3(c->dtype, *c->o3, c->buf[1 - c->cur], mo, c->stream);
  } else if (c->dtype == RLBM_BF16_DEV) {
    FieldPtrs none{nullptr, nullptr, nullptr, nullptr};
    void* pv = c->buf[1 - c->cur];
    void* cp = c->coef[1 - c->cur];
    if (c->fused == 1) e = launch_bf16_io<StencilM1>(1, *c->fp, *c->p64, none, nullptr, pv, nullptr, cp, mo, c->stream);
    else if (c->fused == 2) e = launch_bf16_io<StencilG16>(1, *c->fp, *c->p64, none, nullptr, pv, nullptr, cp, mo, c->stream);
    else if (c->fused == 3) e = launch_bf16_io<StencilE5>(1, *c->fp, *c->p64, none, nullptr, pv, nullptr, cp, mo, c->stream);
    else e = launch_bf16_io<StencilS2>(1, *c->fp, *c->p64, none, nullptr, pv, nullptr, cp, mo, c->stream);
  } else if (c->dtype == RLBM_F32 && c->fused) {
    // the state at t is the pull of S_{t-1}; right after the init, S_0 read in place
    FieldPtrs none{nullptr, nullptr, nullptr, nullptr};
    void* pv = c->fresh ? c->buf[c->cur] : c->buf[1 - c->cur];
    const int what = c->fresh ? 4 : 3;
    if (c->fused == 1) e = launch_bf16_io<StencilM1>(what, *c->fp, *c->p64, none, nullptr, pv, nullptr, nullptr, mo, c->stream);
    else if (c->fused == 2) e = launch_bf16_io<StencilG16>(what, *c->fp, *c->p64, none, nullptr, pv, nullptr, nullptr, mo, c->stream);
    else if (c->fused == 3) e = launch_bf16_io<StencilE5>(what, *c->fp, *c->p64, none, nullptr, pv, nullptr, nullptr, mo, c->stream);
    else e = launch_bf16_io<StencilS2>(what, *c->fp, *c->p64, none, nullptr, pv, nullptr, nullptr, mo, c->stream);
  } else {
    e = launch_moments(c->dtype, *c->p64, c->buf[1 - c->cur], mo, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "moments launch");
  if (!direct) {
    e = cudaMemcpyAsync(out, c->d_out, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read-out copy");
  }
  return check_device_error(c);
}

rlbm_status rlbm_sync(rlbm_ctx* c) {
  if (!c) return RLBM_EINVAL;
  return check_device_error(c);
}

rlbm_status rlbm_get_info(const rlbm_ctx* c, rlbm_info* info) {
  if (!c || !info) return RLBM_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->Nx = c->Nx;
  info->Ny = c->Ny;
  info->Q = c->Q;
  info->halo = c->sb.halo;
  info->dtype = c->dtype;
  info->m = c->m;
  info->tau = c->tau;
  info->order = c->order;
  if (c->order == 3) {
    info->v0 = c->sb3->v0;
    for (int k = 0; k < 11; ++k) info->w_group[k] = c->sb3->w_group[k];
  } else {
    info->v0 = c->sb.v0;
    for (int k = 0; k < 6; ++k) info->w_group[k] = c->sb.w_group[k];
  }
  info->t = c->t;
  info->bytes_per_site = 2 * (size_t)c->Q * c->elem;
  info->extra_bytes_per_site = (c->dtype == RLBM_BF16_DEV) ? 2 * 6 * 8 : 0;   // coefficients read + written
  info->device_bytes = c->device_bytes + c->out_cap * sizeof(double);
  info->kernel = c->fused;
  info->extended_sums = c->ext;
  return RLBM_OK;
}

const char* rlbm_last_error(const rlbm_ctx* c) {
  return c ? c->last_error.c_str() : g_create_error.c_str();
}

void rlbm_destroy(rlbm_ctx* c) {
  if (!c) return;
  batch_forget(c);
  release(c);
  delete c;
}

rlbm_status rlbm_quadrature_weights(const int* groups, int ngroups, double m, double v0,
                                    double* w_out) {
  if (!groups || (ngroups != 6 && ngroups != 11) || !w_out || !(m > 0) || !(v0 > 0)) return RLBM_EINVAL;
  for (int k = 0; k < ngroups; ++k)
    if (groups[k] < 1 || groups[k] > 84) return RLBM_EINVAL;
  return quadrature_weights(groups, ngroups, m, v0, w_out) ? RLBM_OK : RLBM_ENOQUAD;
}

rlbm_status rlbm_quadrature_window(const int* groups, int ngroups, double m, double* lo, double* hi,
                                   int* nwindows) {
  if (!groups || (ngroups != 6 && ngroups != 11) || !lo || !hi || !(m > 0)) return RLBM_EINVAL;
  for (int k = 0; k < ngroups; ++k)
    if (groups[k] < 1 || groups[k] > 84) return RLBM_EINVAL;
  const int n = quadrature_window(groups, ngroups, m, lo, hi);
  if (nwindows) *nwindows = n;
  return n > 0 ? RLBM_OK : RLBM_ENOQUAD;
}

double rlbm_bessel_ratio(double zeta, int precision) { return ratio_eval_host(zeta, precision); }

}  // extern "C"

// ------------------------------------------------------------------ batches
// Independent lattices advanced together: one CUDA graph per batch holds, for
// every lattice, a chain of G step-kernel nodes (step k+1 depends on step k
// of the same lattice) and no edge between lattices, so the GPU overlaps the
// chains; each node runs the single-lattice kernel (second or third order)
// with that lattice's parameters in its own constant bank.  G (steps per
// graph) is autotuned.
namespace {

const void* kernel_of(const rlbm_ctx* c) {
  if (c->order == 3) return fused_o3_kernel_fn(c->fused);
  const int mode = fused_mode(c);
  switch (c->fused) {
    case 1: return fused_kernel_fn<StencilM1>(mode);
    case 2: return fused_kernel_fn<StencilG16>(mode);
    case 3: return fused_kernel_fn<StencilE5>(mode);
    default: return fused_kernel_fn<StencilS2>(mode);
  }
}

// Arguments of the k-th step from now (buffers by parity); params[0] points
// at the FusedParams copy (second order) or at the context's FusedO3Params.
struct NodeArgs {
  FusedParams p;
  const void* fin;
  void* fout;
  void* params[3];
};

void args_of(const rlbm_ctx* c, int k, NodeArgs& a) {
  const int cur = c->cur ^ (k & 1);
  if (c->order == 3) {
    a.params[0] = c->fo3.get();
  } else {
    a.p = *c->fp;
    a.p.cin = c->coef[cur];
    a.p.cout = c->coef[1 - cur];
    a.params[0] = &a.p;
  }
  a.fin = c->buf[cur];
  a.fout = c->buf[1 - cur];
  a.params[1] = &a.fin;
  a.params[2] = &a.fout;
}

unsigned grid_of(const rlbm_ctx* c) { return (unsigned)(((long long)c->Nx * c->Ny + 127) / 128); }

struct BatchPlan {
  int gsteps = 0;
  cudaGraphExec_t exec = nullptr;
};

// The autotuner's choice for a batch: the graph engine with G steps per
// replay, or the persistent engine with spt sites per thread.
struct BatchChoice {
  int engine = RLBM_BATCH_GRAPH;
  int param = 8;
};

// A persistent launch: the lattices of a batch that share a compiled stencil
// and storage variant, in claim order (largest first), with their device
// descriptors, the units of one step and the launch's control words.
struct PersistGroup {
  const void* fn = nullptr;
  std::vector<rlbm_ctx*> lats;
  PersistLattice* d_lat = nullptr;
  int2* d_units = nullptr;
  int* d_par0 = nullptr;
  unsigned* d_ctl = nullptr;      // ticket, abort, done[nlat]
  std::vector<int> par0;          // host copy uploaded before each launch
  int units_per_step = 0;
  int grid = 0;
};

struct PersistPlan {
  int spt = 0;
  std::vector<PersistGroup> groups;
};

std::mutex g_batch_mutex;
std::map<std::string, BatchChoice> g_tuned;  // batch signature -> engine choice
std::map<std::string, BatchPlan> g_plans;    // signature with parities and G -> graph
std::map<std::string, PersistPlan> g_pplans; // signature and spt -> persistent launches
rlbm_batch_options g_bopt = {RLBM_BATCH_AUTO, 0u, 0u};

constexpr unsigned kDefaultSpinLimit = 1u << 23;   // polls of ~0.3 us: about 2.5 s

void free_pplan(PersistPlan& pl) {
  for (PersistGroup& g : pl.groups)
    for (void* q : {(void*)g.d_lat, (void*)g.d_units, (void*)g.d_par0, (void*)g.d_ctl})
      if (q) cudaFree(q);
  pl.groups.clear();
}

std::string signature(rlbm_ctx* const* ctxs, int n, bool with_parity) {
  std::string s;
  for (int i = 0; i < n; ++i) {
    char b[64];
    std::snprintf(b, sizeof b, "%p:%d:%d:%d;", (void*)ctxs[i], ctxs[i]->fused, (int)ctxs[i]->dtype,
                  with_parity ? ctxs[i]->cur : 0);
    s += b;
  }
  return s;
}

// Lattices by decreasing size: the chains of the largest lattices are
// created (and so issued) first.
std::vector<rlbm_ctx*> by_size(const std::vector<rlbm_ctx*>& v) {
  std::vector<rlbm_ctx*> o(v);
  std::stable_sort(o.begin(), o.end(), [](rlbm_ctx* a, rlbm_ctx* b) {
    return (long long)a->Nx * a->Ny > (long long)b->Nx * b->Ny;
  });
  return o;
}

cudaError_t build_graph(const std::vector<rlbm_ctx*>& v, int gsteps, cudaStream_t s, BatchPlan& plan) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  for (rlbm_ctx* c : by_size(v)) {
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < gsteps && e == cudaSuccess; ++k) {
      NodeArgs a;
      args_of(c, k, a);
      cudaKernelNodeParams kp = {};
      kp.func = const_cast<void*>(kernel_of(c));
      kp.gridDim = dim3(grid_of(c));
      kp.blockDim = dim3(128);
      kp.sharedMemBytes = 0;
      kp.kernelParams = a.params;
      cudaGraphNode_t node = nullptr;
      e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
      prev = node;
    }
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&plan.exec, g, 0);
  if (e == cudaSuccess) e = cudaGraphUpload(plan.exec, s);
  cudaGraphDestroy(g);
  plan.gsteps = gsteps;
  return e;
}

cudaError_t single_step(const std::vector<rlbm_ctx*>& v, cudaStream_t s) {
  for (rlbm_ctx* c : by_size(v)) {
    NodeArgs a;
    args_of(c, 0, a);
    cudaError_t e = cudaLaunchKernel(kernel_of(c), dim3(grid_of(c)), dim3(128), a.params, 0, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void advance_all(const std::vector<rlbm_ctx*>& v, int k) {
  for (rlbm_ctx* c : v) {
    c->cur ^= (k & 1);
    c->t += k;
    if (k > 0) c->fresh = false;
  }
}

// The graph for the contexts' current parities and G, built on first use.
cudaError_t plan_for(rlbm_ctx* const* ctxs, int count, const std::vector<rlbm_ctx*>& v, int gsteps,
                     cudaStream_t s, BatchPlan** out) {
  const std::string key = signature(ctxs, count, true) + "/" + std::to_string(gsteps);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    BatchPlan plan;
    cudaError_t e = build_graph(v, gsteps, s, plan);
    if (e != cudaSuccess) {
      if (plan.exec) cudaGraphExecDestroy(plan.exec);
      return e;
    }
    it = g_plans.emplace(key, plan).first;
  }
  *out = &it->second;
  return cudaSuccess;
}

const void* persist_fn_of(const rlbm_ctx* c) {
  const int mode = fused_mode(c);
  switch (c->fused) {
    case 1: return persist_kernel_fn<StencilM1>(mode);
    case 2: return persist_kernel_fn<StencilG16>(mode);
    case 3: return persist_kernel_fn<StencilE5>(mode);
    default: return persist_kernel_fn<StencilS2>(mode);
  }
}

// Lattices grouped by kernel (stencil and variant), each group largest first.
cudaError_t build_pplan(const std::vector<rlbm_ctx*>& v, int spt, PersistPlan& plan) {
  plan.spt = spt;
  std::map<const void*, std::vector<rlbm_ctx*>> by_fn;
  std::vector<const void*> order;
  for (rlbm_ctx* c : by_size(v)) {
    const void* fn = persist_fn_of(c);
    if (!by_fn.count(fn)) order.push_back(fn);
    by_fn[fn].push_back(c);
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (const void* fn : order) {
    if (e != cudaSuccess) break;
    PersistGroup g;
    g.fn = fn;
    g.lats = by_fn[fn];
    const int nl = (int)g.lats.size();
    std::vector<PersistLattice> hl(nl);
    std::vector<int2> units;
    const int tile = 128 * spt;
    for (int l = 0; l < nl; ++l) {
      rlbm_ctx* c = g.lats[l];
      PersistLattice& L = hl[l];
      std::memset(&L, 0, sizeof L);
      for (int par = 0; par < 2; ++par) {
        L.p[par] = *c->fp;
        L.p[par].cin = c->coef[par];
        L.p[par].cout = c->coef[1 - par];
      }
      L.buf[0] = c->buf[0];
      L.buf[1] = c->buf[1];
      L.nsite = c->Nx * c->Ny;
      L.ntiles = (L.nsite + tile - 1) / tile;
      for (int t = 0; t < L.ntiles; ++t) units.push_back(make_int2(l, t));
    }
    g.units_per_step = (int)units.size();
    g.par0.assign(nl, 0);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 128, 0);
    if (e == cudaSuccess && nb < 1) e = cudaErrorInvalidConfiguration;
    g.grid = std::max(1, std::min(nb * sms, g.units_per_step));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_lat, nl * sizeof(PersistLattice));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_units, units.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_par0, nl * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g.d_ctl, (2 + nl) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(g.d_lat, hl.data(), nl * sizeof(PersistLattice), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(g.d_units, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);   // pageable uploads landed
    plan.groups.push_back(std::move(g));
  }
  return e;
}

// nsteps steps of every group, one cooperative launch per group and chunk of
// steps (tickets stay below 2^31).
cudaError_t persist_launch(PersistPlan& plan, int nsteps, unsigned spin_limit, unsigned wait_offset,
                           cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (PersistGroup& g : plan.groups) {
    const int nl = (int)g.lats.size();
    const int chunk = std::max(1, (int)std::min<long long>(nsteps, (1LL << 31) / std::max(1, g.units_per_step)));
    for (int done = 0; done < nsteps && e == cudaSuccess; done += chunk) {
      const int k = std::min(chunk, nsteps - done);
      for (int l = 0; l < nl; ++l) g.par0[l] = g.lats[l]->cur ^ (done & 1);
      e = cudaMemsetAsync(g.d_ctl, 0, (2 + nl) * sizeof(unsigned), s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(g.d_par0, g.par0.data(), nl * sizeof(int), cudaMemcpyHostToDevice, s);
      PersistParams pp;
      std::memset(&pp, 0, sizeof pp);
      pp.lat = g.d_lat;
      pp.units = g.d_units;
      pp.nlat = nl;
      pp.units_per_step = g.units_per_step;
      pp.nsteps = k;
      pp.spt = plan.spt;
      pp.spin_limit = spin_limit;
      pp.wait_offset = wait_offset;
      pp.ticket = g.d_ctl;
      pp.abort = g.d_ctl + 1;
      pp.done = g.d_ctl + 2;
      pp.par0 = g.d_par0;
      void* args[1] = {&pp};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)g.grid);
      cfg.blockDim = dim3(128);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (e == cudaSuccess) e = cudaLaunchKernelExC(&cfg, g.fn, args);
      // the pageable par0 copy returns once staged, so par0 may change below
    }
  }
  return e;
}

cudaError_t pplan_for(rlbm_ctx* const* ctxs, int count, const std::vector<rlbm_ctx*>& v, int spt,
                      PersistPlan** out) {
  const std::string key = signature(ctxs, count, false) + "/p" + std::to_string(spt);
  auto it = g_pplans.find(key);
  if (it == g_pplans.end()) {
    PersistPlan plan;
    cudaError_t e = build_pplan(v, spt, plan);
    if (e != cudaSuccess) {
      free_pplan(plan);
      return e;
    }
    it = g_pplans.emplace(key, std::move(plan)).first;
  }
  *out = &it->second;
  return cudaSuccess;
}

}  // namespace

static void batch_forget(const rlbm_ctx* c) {
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  char b[32];
  std::snprintf(b, sizeof b, "%p:", (const void*)c);
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (it->first.find(b) != std::string::npos) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = g_pplans.begin(); it != g_pplans.end();) {
    if (it->first.find(b) != std::string::npos) {
      free_pplan(it->second);
      it = g_pplans.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = g_tuned.begin(); it != g_tuned.end();) {
    if (it->first.find(b) != std::string::npos) it = g_tuned.erase(it);
    else ++it;
  }
}

extern "C" rlbm_status rlbm_batch_step(rlbm_ctx* const* ctxs, int count, int nsteps) {
  if (!ctxs || count < 1 || nsteps < 0) return fail(nullptr, RLBM_EINVAL, "batch: bad arguments");
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  for (int i = 0; i < count; ++i) {
    rlbm_ctx* c = ctxs[i];
    if (!c || !c->initialised) return fail(nullptr, RLBM_EINVAL, "batch: a context is missing or not initialised");
    if (c->order == 3 ? !c->fo3 : ((c->dtype != RLBM_F32 && c->dtype != RLBM_BF16_DEV) || !c->fused))
      return fail(nullptr, RLBM_ENOTSUP,
                  "batch: every context needs a compiled stencil and FP32 storage (or BF16 at second order)");
    if (c->stream != ctxs[0]->stream) return fail(nullptr, RLBM_EINVAL, "batch: contexts on different streams");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(nullptr, RLBM_EINVAL, "batch: a context is listed twice");
  }
  if (nsteps == 0) return RLBM_OK;
  std::vector<rlbm_ctx*> v(ctxs, ctxs + count);
  cudaStream_t user = ctxs[0]->stream;
  // graph launches need a non-legacy stream: bridge a NULL stream with events
  static cudaStream_t bridge = nullptr;
  cudaStream_t s = user;
  struct Events {
    cudaEvent_t in = nullptr, out = nullptr, a = nullptr, b = nullptr;
    ~Events() {
      for (cudaEvent_t e : {in, out, a, b})
        if (e) cudaEventDestroy(e);
    }
  } ev;
  cudaError_t e = cudaSuccess;
  if (!user) {
    if (!bridge) e = cudaStreamCreateWithFlags(&bridge, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev.in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev.out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev.in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bridge, ev.in, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch stream bridge");
    s = bridge;
  }
  const std::string sig = signature(ctxs, count, false);
  bool any_o3 = false;
  for (rlbm_ctx* c : v) any_o3 = any_o3 || c->order == 3;
  const unsigned spin = g_bopt.spin_limit ? g_bopt.spin_limit : kDefaultSpinLimit;
  int done = 0;
  BatchChoice ch;
  auto tuned = g_tuned.find(sig);
  if (tuned != g_tuned.end()) {
    ch = tuned->second;
  } else if (g_bopt.engine == RLBM_BATCH_PERSISTENT && !any_o3) {
    ch.engine = RLBM_BATCH_PERSISTENT;
    ch.param = 2;
    g_tuned[sig] = ch;
  } else {
    // autotune: time each candidate on steps that count towards nsteps
    const int cand[3] = {2, 8, 32};
    const int spts[3] = {1, 2, 4};
    const bool try_persist = g_bopt.engine == RLBM_BATCH_AUTO && !any_o3;
    const int kp = 8;
    const int total = cand[0] + cand[1] + cand[2] + (try_persist ? 3 * kp : 0);
    if (nsteps >= total) {
      e = cudaEventCreate(&ev.a);
      if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
      float best = 1e30f;
      auto timed = [&](auto&& run, int k, int engine, int param) {
        if (e == cudaSuccess) e = cudaEventRecord(ev.a, s);
        if (e == cudaSuccess) e = run();
        if (e == cudaSuccess) e = cudaEventRecord(ev.b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.a, ev.b);
        if (e != cudaSuccess) return;
        advance_all(v, k);
        done += k;
        if (ms / k < best) {
          best = ms / k;
          ch.engine = engine;
          ch.param = param;
        }
      };
      for (int g : cand) {
        BatchPlan* pl = nullptr;
        if (e == cudaSuccess) e = plan_for(ctxs, count, v, g, s, &pl);
        timed([&] { return cudaGraphLaunch(pl->exec, s); }, g, RLBM_BATCH_GRAPH, g);
      }
      if (try_persist)
        for (int spt : spts) {
          PersistPlan* pp = nullptr;
          if (e == cudaSuccess) e = pplan_for(ctxs, count, v, spt, &pp);
          timed([&] { return persist_launch(*pp, kp, spin, g_bopt.wait_offset, s); }, kp,
                RLBM_BATCH_PERSISTENT, spt);
        }
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch autotune");
      g_tuned[sig] = ch;
    } else {
      ch.engine = RLBM_BATCH_GRAPH;          // too few steps to tune: not cached
      ch.param = nsteps >= cand[1] ? cand[1] : cand[0];
    }
  }
  if (ch.engine == RLBM_BATCH_PERSISTENT && nsteps > done) {
    PersistPlan* pp = nullptr;
    e = pplan_for(ctxs, count, v, ch.param, &pp);
    if (e == cudaSuccess) e = persist_launch(*pp, nsteps - done, spin, g_bopt.wait_offset, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch persistent launch");
    advance_all(v, nsteps - done);
    done = nsteps;
  }
  const int G = ch.engine == RLBM_BATCH_GRAPH ? ch.param : 2;
  for (int g : {G, 2}) {
    if (nsteps - done < g) continue;
    BatchPlan* pl = nullptr;
    e = plan_for(ctxs, count, v, g, s, &pl);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch graph");
    while (nsteps - done >= g) {
      e = cudaGraphLaunch(pl->exec, s);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch graph launch");
      advance_all(v, g);   // g is even: parities unchanged, the same graph serves again
      done += g;
    }
  }
  if (nsteps - done == 1) {
    e = single_step(v, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch step");
    advance_all(v, 1);
    done += 1;
  }
  if (!user) {
    e = cudaEventRecord(ev.out, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev.out, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch stream bridge");
  }
  return RLBM_OK;
}

extern "C" rlbm_status rlbm_batch_tuning(rlbm_ctx* const* ctxs, int count, int* steps_per_graph,
                                         int* launches_per_step) {
  if (!ctxs || count < 1) return fail(nullptr, RLBM_EINVAL, "batch tuning: bad arguments");
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return fail(nullptr, RLBM_EINVAL, "batch tuning: a context is missing");
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  auto tuned = g_tuned.find(signature(ctxs, count, false));
  if (tuned == g_tuned.end()) return fail(nullptr, RLBM_EINVAL, "batch tuning: this batch has not been tuned");
  const bool graph = tuned->second.engine == RLBM_BATCH_GRAPH;
  if (steps_per_graph) *steps_per_graph = graph ? tuned->second.param : 0;
  if (launches_per_step) *launches_per_step = graph ? count : 0;
  return RLBM_OK;
}

extern "C" rlbm_status rlbm_batch_engine(rlbm_ctx* const* ctxs, int count, int* engine, int* param,
                                         int* launches) {
  if (!ctxs || count < 1) return fail(nullptr, RLBM_EINVAL, "batch engine: bad arguments");
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return fail(nullptr, RLBM_EINVAL, "batch engine: a context is missing");
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  const std::string sig = signature(ctxs, count, false);
  auto tuned = g_tuned.find(sig);
  if (tuned == g_tuned.end()) return fail(nullptr, RLBM_EINVAL, "batch engine: no engine chosen for this batch yet");
  const BatchChoice ch = tuned->second;
  int nl = count;
  if (ch.engine == RLBM_BATCH_PERSISTENT) {
    auto it = g_pplans.find(sig + "/p" + std::to_string(ch.param));
    nl = it == g_pplans.end() ? 0 : (int)it->second.groups.size();
  }
  if (engine) *engine = ch.engine;
  if (param) *param = ch.param;
  if (launches) *launches = nl;
  return RLBM_OK;
}

extern "C" rlbm_status rlbm_batch_set_options(const rlbm_batch_options* opt) {
  rlbm_batch_options o = {RLBM_BATCH_AUTO, 0u, 0u};
  if (opt) o = *opt;
  if (o.engine < RLBM_BATCH_AUTO || o.engine > RLBM_BATCH_PERSISTENT)
    return fail(nullptr, RLBM_EINVAL, "batch options: unknown engine");
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  g_bopt = o;
  g_tuned.clear();
  return RLBM_OK;
}
