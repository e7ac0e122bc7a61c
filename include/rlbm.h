/*
 * rlbm.h -- C ABI of the GB300 relativistic lattice Boltzmann step.
 *
 * Method: Gabbana, Mendoza, Succi & Tripiccione, "Towards a unified lattice
 * kinetic scheme for relativistic hydrodynamics" (arXiv:1703.04605).  One call
 * of rlbm_step advances a periodic Nx x Ny lattice by the discrete
 * relativistic Boltzmann equation with Anderson-Witting relaxation (Eq. 49,
 * Sec. III C):
 *
 *   f_i(x + n_i, t + 1) = f_i(x, t) - (p_i.U / (p_i^0 tau)) (f_i - f_i^eq),
 *
 * where, per site, N^a = sum_i f_i p_i^a and T^ab = sum_i f_i p_i^a p_i^b
 * (Eq. 4-5, 18), e and U solve the Landau-frame eigenproblem T^ab U_b = e U^a
 * (Eq. 20), n = U_a N^a (Eq. 19), T solves e/n = 3T + m K1(m/T)/K2(m/T)
 * (Eq. 28), and f_i^eq = n w_i sum_k b^(k)(U, T) J^(k)(p_i) is the
 * second-order expansion (Eq. 16, App. A and B) -- or, on an eleven-group
 * stencil, the third-order one (polynomials of degree <= 3, Sec. III A-D).
 *
 * Units: c = k_B = T_R = 1 (so mbar = m), lattice spacing 1, one time step 1.
 * Metric diag(1,-1,-1,-1).  The velocity set is a second-order stencil of six
 * groups (or a third-order one of eleven) of Table I (App. C) with common
 * velocity parameter v0 (Eq. 48),
 * folded onto the xy plane: the +-n_z members of a group merge into one
 * population of doubled weight, which reproduces the 3D model on an
 * Nx x Ny x 1 lattice exactly while U^z = 0.
 *
 * Conventions for every function:
 *  - Status codes only; nothing throws across the ABI.  On failure the
 *    context keeps its previous state and rlbm_last_error() describes why.
 *  - Host arrays are owned by the caller, row-major [Ny][Nx] doubles.
 *  - Device work is issued on the CUDA stream given at creation.  Device-side
 *    errors (non-physical sites) are sticky: they are reported by the next
 *    call that synchronises (rlbm_moments, rlbm_sync) as RLBM_ENONPHYS.
 *  - The library never falls back to host computation: without a usable
 *    CUDA device every call that needs one returns RLBM_ECUDA.
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlbm_ctx rlbm_ctx;

typedef enum {
  RLBM_OK = 0,
  RLBM_EINVAL = 1,   /* invalid argument, detected before any launch          */
  RLBM_ENOQUAD = 2,  /* no positive-weight quadrature for these groups at m   */
  RLBM_ENOMEM = 3,   /* device or host allocation failed                       */
  RLBM_ECUDA = 4,    /* CUDA runtime error (including: no device)              */
  RLBM_ENONPHYS = 5, /* a site left the physical domain (n<=0, |u|>=1, T<=0,
                        non-finite); sticky until reported                     */
  RLBM_ETIMEOUT = 6, /* a bounded device-side wait expired                     */
  RLBM_ENOTSUP = 7   /* valid but unsupported (e.g. more populations than the
                        compiled maximum)                                      */
} rlbm_status;

/* Population storage.  Arithmetic: F64 computes everything in FP64.  F32
 * and BF16_DEV accumulate the moments in FP32, solve the Landau frame in
 * FP32 and the EOS by FP32 Newton iterations finished by one FP64 Newton
 * step with the FP64 R(zeta) table (the only FP64 work of their step).
 * BF16_DEV stores, per population, the bfloat16 deviation of f_i from a
 * reference polynomial mult_i (a + b_x n_x + b_y n_y + q (n_x^2 + n_y^2))
 * of the writing site's equilibrium, and beside the populations the four
 * bfloat16 coefficients (a, b_x, b_y, q) of each of the six groups per site
 * (6 x 8 bytes), from which the reader rebuilds f_i. */
typedef enum { RLBM_F64 = 0, RLBM_F32 = 1, RLBM_BF16_DEV = 2 } rlbm_dtype;

/* A stencil (Sec. III C-D): six distinct groups of Table I (ids 1..84) for
 * the second-order scheme, or eleven for the third-order one, and v0.  v0 > 0
 * is used as given (it must make every weight positive and v0 ||n_k|| < 1);
 * v0 == 0 selects the centre of the widest interval of v0 where all weights
 * are positive (Sec. III D).  Third-order contexts take FP64 or FP32 storage
 * (ENOTSUP for BF16_DEV), join rlbm_batch_step on a compiled stencil with
 * FP32 storage, and their
 * equilibrium is the unique w_i times a polynomial of degree <= 3 in p_i
 * whose moments up to rank 3 (N^a, T^ab, T^abc, Eq. 4-6) equal those of the
 * Maxwell-Juttner distribution. */
typedef struct {
  int ngroups;
  const int* groups;
  double v0;
} rlbm_stencil;

/* Read-only description of a context (rlbm_get_info). */
typedef struct {
  int Nx, Ny;
  int Q;            /* folded populations                                   */
  int halo;         /* largest |n_x| or |n_y| of the stencil                */
  rlbm_dtype dtype;
  double m, tau, v0;
  double w_group[11];       /* weights of the groups (Eq. 47/52): six, or
                               eleven for a third-order stencil             */
  long long t;              /* current time step                             */
  size_t bytes_per_site;    /* populations read + written per site update:
                               2 Q sizeof(storage)                           */
  size_t extra_bytes_per_site; /* other per-site traffic of one step (macros) */
  size_t device_bytes;      /* device memory owned by the context            */
  int kernel;               /* step kernel: 0 generic; 1..4 compiled for the
                               stencils {5,12,14,17,21,26}, {1..6},
                               {1,14,49,51,60,70}, {3,9,10,14,17,21}; 5..10
                               the compiled third-order stencils
                               {1,2,5,6,7,9,10,11,12,13,15},
                               {2,3,5,6,7,8,9,10,11,13,15},
                               {1,2,3,6,7,8,9,10,11,13,15},
                               {8,15,20,24,26,27,28,30,36,37,42},
                               {4,10,15,20,24,26,27,28,30,36,37},
                               {4,8,14,15,16,17,18,21,22,23,26} (FP32
                               storage, lattice at least a halo wide)          */
  int order;                /* expansion order of f^eq: 2 or 3               */
  int extended_sums;        /* level of extended-precision moment sums of the
                               FP32 step, 0..2 (rlbm_set_extended_sums)      */
} rlbm_info;

/* Create a lattice context.
 *  st     stencil (copied); m = particle mass in units of T_R (m > 0);
 *  tau    relaxation time in lattice steps (tau > 1/2);
 *  Nx,Ny  lattice size (>= 1 each, Nx Ny <= 2^31 - 1: the kernels index
 *         sites with 32-bit integers);  dtype  population storage;
 *  cuda_stream  a cudaStream_t (NULL = legacy default stream), borrowed.
 * Builds the stencil tables on the host (weights of Eq. 52 in binary128),
 * uploads them and allocates two population buffers.  *out is set only on
 * success.  Errors: EINVAL, ENOQUAD, ENOTSUP (also: a population plane of
 * (Nx rounded up to 32) * Ny elements must stay below 2^32, the kernels'
 * 32-bit element indices), ENOMEM, ECUDA. */
rlbm_status rlbm_create(const rlbm_stencil* st, double m, double tau, int Nx, int Ny,
                        rlbm_dtype dtype, void* cuda_stream, rlbm_ctx** out);

/* Set f_i = f_i^eq(n, U, T) everywhere (Eq. 16) and t = 0.  Host arrays of
 * Nx*Ny doubles: density n > 0, three-velocity (ux, uy) with ux^2+uy^2 < 1,
 * temperature T > 0.  Copies the fields to the device (page-locked arrays
 * make the copy direct), checks the copy there (EINVAL names the first bad
 * site; the lattice is then left as it was) and waits for the check on the
 * context stream; the reference density of the FP32/BF16 storage is the
 * mean of n.  The arrays may be reused when the call returns. */
rlbm_status rlbm_init(rlbm_ctx* ctx, const double* n, const double* ux, const double* uy,
                      const double* T);

/* Same as rlbm_init with the four fields already in device memory (each
 * Nx*Ny doubles, row-major).  Asynchronous on the context stream; no
 * validation beyond the device-side physicality flags. */
rlbm_status rlbm_init_device(rlbm_ctx* ctx, const double* n, const double* ux, const double* uy,
                             const double* T);

/* Advance nsteps >= 0 time steps (Eq. 49 applied nsteps times).
 * Asynchronous on the context stream: returns after enqueueing. */
rlbm_status rlbm_step(rlbm_ctx* ctx, int nsteps);

/* Moment sums of the FP32 step on a compiled second-order stencil
 * (rlbm_info.kernel 1..4, FP32 storage).  level 1: N^0 and the kinetic
 * moment K^0 = T^00 - m N^0 (Eq. 4-5, 18) are accumulated to about 2^-40
 * relative -- each pulled value split exactly into a part on a per-group
 * grid and a small remainder, the group sums combined by error-free products
 * and sums -- and e - m n (Eq. 19-20) is formed from K^a = T^0a - m N^a
 * without cancelling the rest-mass energy; level 2: N^x, N^y, K^x, K^y
 * extended as well.  This keeps FP32 storage close to FP64 over thousands of
 * steps on steep, sloshing flows of massive particles, where plain FP32
 * moment sums drift (they break mass and energy conservation by about one
 * rounding per step and site).  level 0: plain FP32 sums (fewest
 * instructions).  Takes effect at the next step; cached batch graphs of the
 * context are dropped.  Errors: EINVAL (NULL ctx, level not 0..2), ENOTSUP
 * (no compiled FP32 second-order kernel for this context). */
rlbm_status rlbm_set_extended_sums(rlbm_ctx* ctx, int level);

/* Macroscopic fields of the current pre-collision state f(., t).
 * mask selects fields (bits below); out (host memory, rlbm_moments_size
 * doubles) receives, in bit order, one Nx*Ny plane per scalar (RLBM_M_NVEC:
 * 3 planes N^0,N^x,N^y; RLBM_M_TMN: 6 planes T^00,T^0x,T^0y,T^xx,T^xy,T^yy).
 * Page-locked (mapped) memory is written directly by the read-out kernel;
 * other memory through a device buffer of the context and one copy.  The
 * library cannot see the buffer's length: a page-locked buffer shorter than
 * rlbm_moments_size would be overrun by the device (the Python binding
 * checks the length before the call).
 * Synchronises the stream, then reports any sticky device error. */
#define RLBM_M_N    0x01u  /* n = U_a N^a (Eq. 19)             */
#define RLBM_M_UX   0x02u  /* u_x = U^x / U^0                  */
#define RLBM_M_UY   0x04u  /* u_y = U^y / U^0                  */
#define RLBM_M_T    0x08u  /* temperature (Eq. 28)             */
#define RLBM_M_E    0x10u  /* energy density e (Eq. 20)        */
#define RLBM_M_NVEC 0x20u  /* N^a, 3 planes                    */
#define RLBM_M_TMN  0x40u  /* T^ab, 6 planes                   */
#define RLBM_M_UZ   0x80u  /* u_z = U^z / U^0 (3D lattices only) */
rlbm_status rlbm_moments(rlbm_ctx* ctx, double* out, unsigned mask);

/* Number of doubles rlbm_moments writes for a mask (0 on a NULL ctx). */
size_t rlbm_moments_size(const rlbm_ctx* ctx, unsigned mask);

/* Block until the context stream is idle; report sticky device errors. */
rlbm_status rlbm_sync(rlbm_ctx* ctx);

/* Fill *info.  Never touches the device. */
rlbm_status rlbm_get_info(const rlbm_ctx* ctx, rlbm_info* info);

/* Human-readable description of the last failure on ctx (or of the last
 * failed rlbm_create when ctx is NULL).  Valid until the next call. */
const char* rlbm_last_error(const rlbm_ctx* ctx);

/* Release the context and its device memory (synchronises its stream). */
void rlbm_destroy(rlbm_ctx* ctx);

/* ---- device memory ---------------------------------------------------
 * Contexts own their device buffers (populations, tables, staging) and by
 * default take them from cudaMalloc.  rlbm_set_allocator installs a
 * caller-supplied allocator instead -- a framework's caching allocator, for
 * instance -- for the contexts (2D and 3D) created after the call:
 *   alloc(bytes, device, stream, user) returns device memory of at least
 *     bytes on that device, aligned to 256 bytes, for use on that stream
 *     (the context's; NULL = legacy default stream), or NULL (ENOMEM; a
 *     block that is not 256-byte aligned is handed back and counts as NULL);
 *   free_fn(ptr, user) takes back a block alloc returned.
 * A context keeps the pair it was created with and frees through it, on
 * rlbm_destroy (after synchronising its stream) and when rlbm_moments grows
 * its read-out buffer.  alloc and free_fn both NULL restore cudaMalloc and
 * cudaFree; exactly one NULL is EINVAL.  Process-wide; the setting is
 * copied under a lock, so it may change while other threads create contexts.
 * The paper has no counterpart.  rlbm_moments_noalloc allocates nothing. */
typedef void* (*rlbm_alloc_fn)(size_t bytes, int device, void* cuda_stream, void* user);
typedef void (*rlbm_free_fn)(void* ptr, void* user);
rlbm_status rlbm_set_allocator(rlbm_alloc_fn alloc, rlbm_free_fn free_fn, void* user);

/* Advance count contexts by nsteps each, as one batch (the independent
 * lattices of a parameter sweep or an ensemble).  Equivalent to calling
 * rlbm_step(ctxs[i], nsteps) for every i, with identical results.  Two
 * engines run the steps:
 *  - graph: replays of one CUDA graph per batch that holds, for every
 *    lattice, a chain of G step kernels (step k+1 of a lattice depends on its
 *    step k) and no dependency between lattices, so the GPU overlaps the
 *    lattices' kernels; each kernel is the single-lattice step kernel with
 *    that lattice's parameters;
 *  - persistent: one cooperative launch per stencil and storage variant
 *    covers all nsteps steps of its lattices; its blocks claim tiles of
 *    128 x spt sites in step-major order and wait, with a bounded poll, until
 *    the tile's lattice has finished the previous step (second-order lattices
 *    only).  A wait that runs out of polls ends the launch; the lattices'
 *    next synchronising call returns RLBM_ETIMEOUT and their state is
 *    undefined until rlbm_init.
 * With the engine left to the autotuner (rlbm_batch_set_options), the first
 * call for a batch with enough steps times one replay of each graph length G
 * in {2, 8, 32} (42 steps) and, on a batch of second-order lattices, 8 steps
 * of the persistent engine at each spt in {1, 2, 4} (24 more steps; so
 * nsteps >= 66, or >= 42 with third-order members), those steps counting
 * towards nsteps, and caches the fastest; rlbm_batch_engine reports it.
 * Shorter calls run the graph engine untuned.
 * Graphs and persistent plans are cached per batch; rlbm_init,
 * rlbm_set_extended_sums or rlbm_destroy of a member drops them.  A
 * persistent plan holds a few small device descriptors of its own (about
 * 3 KB per lattice, taken with cudaMalloc, not from rlbm_set_allocator's
 * allocator, which serves the contexts' buffers).
 * Requirements: every context initialised, a compiled stencil
 * (rlbm_info.kernel != 0) with FP32 or BF16-deviation storage (FP32 only at
 * third order; second- and third-order contexts may be mixed), all on the
 * same CUDA stream, no context listed twice.  Asynchronous on that stream (a
 * NULL stream is bridged to an internal stream with events).  Not thread-safe
 * against rlbm_step on the same contexts.  The paper has no counterpart (it
 * advances one lattice at a time).  Errors: EINVAL (violated requirement),
 * ENOTSUP, ECUDA. */
rlbm_status rlbm_batch_step(rlbm_ctx* const* ctxs, int count, int nsteps);

/* Batch engines and the persistent engine's bounded waits.  Process-wide;
 * a change drops every cached tuning choice. */
#define RLBM_BATCH_AUTO 0        /* the autotuner picks (default)             */
#define RLBM_BATCH_GRAPH 1       /* graph of per-lattice step kernels         */
#define RLBM_BATCH_PERSISTENT 2  /* persistent cooperative kernel            */
typedef struct {
  int engine;              /* RLBM_BATCH_AUTO, _GRAPH or _PERSISTENT; a batch
                              the persistent engine cannot run (third-order
                              members) uses the graph engine                 */
  unsigned spin_limit;     /* polls (about 0.3 us each) of one device-side
                              wait before it gives up; 0 = default 2^23       */
  unsigned wait_offset;    /* fault injection for tests of the timeout path:
                              added to every wait target, so that a wait can
                              never be met; 0 in normal use                   */
} rlbm_batch_options;
/* opt NULL restores the defaults.  Errors: EINVAL (unknown engine). */
rlbm_status rlbm_batch_set_options(const rlbm_batch_options* opt);

/* The engine used for a batch (same contexts, same order) once it has been
 * chosen: *engine = RLBM_BATCH_GRAPH (*param = G, steps per graph replay,
 * *launches = kernel launches per step = count) or RLBM_BATCH_PERSISTENT
 * (*param = sites per thread, *launches = cooperative launches per call).
 * Output pointers may be NULL.  Never touches the device.  Errors: EINVAL (bad
 * arguments, or no choice made for this batch yet). */
rlbm_status rlbm_batch_engine(rlbm_ctx* const* ctxs, int count, int* engine, int* param, int* launches);

/* The autotuner's choice for a batch that rlbm_batch_step has tuned (same
 * contexts, same order): *steps_per_graph = G, *launches_per_step = kernel
 * launches of one step (one per lattice), or both 0 when the persistent
 * engine was chosen (rlbm_batch_engine describes it).  Either output pointer
 * may be NULL.  Never touches the device.  Errors: EINVAL (bad arguments, or
 * no choice cached for this batch). */
rlbm_status rlbm_batch_tuning(rlbm_ctx* const* ctxs, int count, int* steps_per_graph, int* launches_per_step);

/* ---- native 3D lattices ----------------------------------------------
 * The paper's model is three-dimensional (Sec. II-III, App. C); these entry
 * points run it on an Nx x Ny x Nz periodic lattice with the unfolded
 * stencil (every vector of the six Table I orbits, signed n_z), all three
 * velocity components and the 14 polynomials of App. A.  They use generic
 * kernels (any six-group stencil): FP64 storage (f_i), or FP32 storage of
 * d_i = f_i - r_i with FP32 accumulation; the site solve (Landau frame by
 * Newton iteration on the three velocities, Eq. 20; EOS, Eq. 28) is FP64.
 * Fields are [Nz][Ny][Nx] arrays, x fastest.  A separate context type. */
typedef struct rlbm_ctx3 rlbm_ctx3;

typedef struct {
  int Nx, Ny, Nz;
  int Q;                    /* populations of the unfolded stencil            */
  int halo;                 /* largest |n| component                          */
  rlbm_dtype dtype;
  double m, tau, v0;
  long long t;
  size_t bytes_per_site;    /* 2 Q sizeof(storage)                            */
  size_t device_bytes;
  int kernel;               /* step kernel: 0 generic; 1..4 compiled for the
                               stencils {5,12,14,17,21,26}, {1..6},
                               {1,14,49,51,60,70}, {3,9,10,14,17,21} (FP32
                               storage, lattice at least a halo wide)         */
  int order;                /* expansion order of f^eq: 2 or 3 (eleven groups:
                               the thirty-monomial third-order equilibrium on
                               the generic kernels)                           */
} rlbm3_info;

/* As rlbm_create, with Nz >= 1 and Nx Ny Nz <= 2^31 - 1; dtype RLBM_F64 or RLBM_F32 (ENOTSUP for
 * BF16).  Six groups: the second-order equilibrium (App. A-B); eleven: the
 * third-order one, exact to the third moment T^abc (generic kernels).  More
 * than 160 unfolded populations: ENOTSUP. */
rlbm_status rlbm3_create(const rlbm_stencil* st, double m, double tau, int Nx, int Ny, int Nz,
                         rlbm_dtype dtype, void* cuda_stream, rlbm_ctx3** out);

/* f = f^eq(n, U, T) (Eq. 16), t = 0.  Host FP64 arrays of Nx*Ny*Nz values;
 * n > 0, T > 0, |u| < 1 checked on the device copy (EINVAL names the first
 * bad site), as rlbm_init. */
rlbm_status rlbm3_init(rlbm_ctx3* ctx, const double* n, const double* ux, const double* uy,
                       const double* uz, const double* T);

/* nsteps steps (Eq. 49), asynchronous on the context's stream. */
rlbm_status rlbm3_step(rlbm_ctx3* ctx, int nsteps);

/* Macroscopic fields of the pre-collision state at t into host memory, one
 * Nx*Ny*Nz plane per scalar, in the order of the mask bits: RLBM_M_N, _UX,
 * _UY, _T, _E, _NVEC (4 planes N^0..N^z), _TMN (10 planes T^00 T^0x T^0y
 * T^0z T^xx T^xy T^xz T^yy T^yz T^zz), _UZ; rlbm3_moments_size doubles.
 * Page-locked memory is written directly, as rlbm_moments (same length
 * caveat).  Synchronises the stream and reports sticky device errors
 * (ENONPHYS). */
rlbm_status rlbm3_moments(rlbm_ctx3* ctx, double* out, unsigned mask);
size_t rlbm3_moments_size(const rlbm_ctx3* ctx, unsigned mask);

rlbm_status rlbm3_sync(rlbm_ctx3* ctx);
rlbm_status rlbm3_get_info(const rlbm_ctx3* ctx, rlbm3_info* info);
/* Last failure on ctx, or of the last failed rlbm3_create when ctx is NULL. */
const char* rlbm3_last_error(const rlbm_ctx3* ctx);
void rlbm3_destroy(rlbm_ctx3* ctx);

/* ---- read-out without memory allocation -------------------------------
 * The paper has no counterpart of this entry point; it serves callers that
 * may not allocate device memory -- e.g. code running inside a host
 * application that owns every allocation (a plugin handed device buffers),
 * or under a memory manager that forbids cudaMalloc at the point of call.
 *
 * Computes the same fields as rlbm_moments, for FP64 populations the caller
 * holds in device memory: f_dev = f_i(x, t) in the library's population
 * order (groups ascending, inside a group (n_x, n_y) lexicographic), compact
 * layout [Q][Ny][Nx] doubles.  The populations are read as they are (no
 * streaming).  out_host receives the planes selected by mask (same layout as
 * rlbm_moments).  groups/m/v0 describe the stencil as in rlbm_create
 * (v0 > 0 required); only six-group (second-order) stencils are accepted,
 * any other ngroups is RLBM_EINVAL.
 *
 * Synchronisation: every call copies the result and the error word back to
 * the host and synchronises cuda_stream before it returns, so it must never
 * be called while any stream is being captured into a CUDA graph.
 *
 * Memory: allocates no device memory.  Its device scratch -- the error
 * word, the R(zeta) table and the result staging -- is one static 8 MiB
 * array that every GPU loading the library holds until exit; results larger
 * than 1,045,728 doubles (planes x Nx x Ny) are rejected with RLBM_EINVAL.
 * The first call on a device sets the array up (symbol address, table copy,
 * then a device synchronisation); the first call for a new stencil or
 * lattice size builds host tables.  All calls share the array, which keeps
 * the last call's contents (the error word is cleared per call).  Within one
 * process the calls are serialised by a lock and each one synchronises its
 * stream, so they cannot overlap; two processes on one GPU have separate
 * copies of the array.  Errors are described by rlbm_last_error(NULL). */
rlbm_status rlbm_moments_noalloc(const int* groups, int ngroups, double m, double v0, int Nx, int Ny,
                                 const double* f_dev, double* out_host, unsigned mask,
                                 void* cuda_stream);

/* ---- host-only helpers (no device needed) ---------------------------- */

/* Weights of the groups at (m, v0) from Eq. 52 (ngroups = 6: the six
 * second-order conditions; 11: the eleven third-order ones), solved in
 * binary128 and rounded to FP64 into w_out[ngroups].  Returns ENOQUAD if the
 * system is singular; the weights are returned whatever their sign. */
rlbm_status rlbm_quadrature_weights(const int* groups, int ngroups, double m, double v0,
                                    double* w_out);

/* The widest v0 interval (lo, hi) in which all weights (6 or 11 groups) are
 * positive (Sec. III D: v0 is free inside it), and the count of disjoint
 * positive intervals; ENOQUAD if there is none. */
rlbm_status rlbm_quadrature_window(const int* groups, int ngroups, double m, double* lo,
                                   double* hi, int* nwindows);

/* R(zeta) = K1(zeta)/K2(zeta), the Bessel ratio of the equation of state
 * (Eq. 28), from the library's piecewise-polynomial tables, evaluated on the
 * host by the same formulas the kernels use (precision 64 or 32).  For
 * validation of the tables. */
double rlbm_bessel_ratio(double zeta, int precision);

/* Measurement helper (not part of the method): the device's FP64 fused
 * multiply-add throughput in TFLOP/s (2 flops per FMA), timed with CUDA
 * events on cuda_stream (NULL = legacy default stream) as the best of five
 * launches of a kernel whose threads run eight independent FMA chains each,
 * on register operands (constant-bank operands would read about 16 % lower).
 * The denominator of the FP64 step kernels' ALU roofline.  Synchronises the
 * stream; about 0.1 s.  Errors: EINVAL (NULL tflops), ECUDA. */
rlbm_status rlbm_fp64_fma_rate(void* cuda_stream, double* tflops);

/* Library version string. */
const char* rlbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RLBM_H */
