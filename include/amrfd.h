/*
 * amrfd.h -- C ABI of the GB300 FP64 conservative finite-difference update of
 * Porth et al., "MPI-AMRVAC for solar and astrophysics" (ApJS 2014).
 *
 * One call advances the conserved state of many domains by one strong-stability-
 * preserving Runge-Kutta step of the paper's FD scheme:
 *   conserved -> primitive, maximal characteristic speed per cell, global
 *   Lax-Friedrichs flux splitting F^{+-} = (F +- c_max U)/2 (Sec. 2.2), MP5
 *   reconstruction of the split fluxes at faces (Suresh & Huynh 1997, cited in
 *   Sec. 2.2), the flux difference L(U) = -sum_j dF_j/dx_j (Sec. 2.1), the
 *   Shu-Osher stage combination of SSPRK3 or SSPRK(5,4) (Sec. 2.3), GLM psi
 *   damping (Sec. 4.2), and the CFL time step (Sec. 4.4).
 *
 * Conventions for every entry point:
 *  - All state, time-step and gradient arrays are DEVICE pointers owned by the
 *    caller (e.g. torch tensors). FP64 only.
 *  - State layout: the caller's buffer holds every domain at its `offset`
 *    (elements), each domain as U[v][z][y][x], x fastest, interior cells only
 *    (no ghost cells; halos are synthesised from the boundary kinds).
 *      Euler   (nv = 2 + ndim): rho, m_1..m_ndim, E
 *      MHD+GLM (nv = 9):        rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi
 *    E = p/(gamma-1) + rho v^2/2 + B^2/2 (Sec. 3, Sec. 4.3); units with no
 *    4 pi or mu_0 (B^2/2 is the magnetic pressure).
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) and does not synchronise, except where stated.
 *  - Return value: AMRFD_OK or an AMRFD_ERR_* code (see amrfd_strerror).
 *    Argument errors are detected on the host before anything is launched.
 *    Conditions found on the device (non-physical states) are latched in the
 *    handle and read with amrfd_get_error.
 *  - A handle is not thread-safe; calls on one handle must be serialised.
 */
#ifndef AMRFD_H
#define AMRFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* physics, integrator, boundary and time-step scope selectors */
#define AMRFD_EULER 0
#define AMRFD_MHD_GLM 1
#define AMRFD_SSPRK3 0
#define AMRFD_SSPRK54 1
#define AMRFD_SSPRK43 2
#define AMRFD_MP5 0
#define AMRFD_LIMO3 1
#define AMRFD_BC_PERIODIC 0
#define AMRFD_BC_OUTFLOW 1
#define AMRFD_BC_SYMMETRIC 2 /* mirror ghosts, per-variable sign: see amrfd_domain.asym */
#define AMRFD_DT_PER_DOMAIN 0
#define AMRFD_DT_GLOBAL 1

/* return codes */
#define AMRFD_OK 0
#define AMRFD_ERR_INVALID_ARG 1
#define AMRFD_ERR_CUDA 2
#define AMRFD_ERR_UNSUPPORTED 3
#define AMRFD_ERR_NONPHYSICAL 4 /* device found rho <= 0, p <= 0 or a non-finite value */
#define AMRFD_ERR_CHECK 5       /* checked build (-DAMRFD_CHECKS): a work descriptor or index
                                   check failed in a kernel; the access was skipped */

typedef struct amrfd_config {
  int physics;    /* AMRFD_EULER | AMRFD_MHD_GLM */
  int ndim;       /* 1, 2 or 3 */
  int integrator; /* AMRFD_SSPRK3 (Gottlieb-Shu RK3, Sec. 2.3) | AMRFD_SSPRK54 | AMRFD_SSPRK43 (printed tables, Sec. 2.3) */
  int dt_scope;   /* AMRFD_DT_PER_DOMAIN | AMRFD_DT_GLOBAL (min over domains) */
  double gamma;   /* ratio of specific heats, > 1 */
  double cfl;     /* Courant number used by amrfd_dt */
  double glm_cr;  /* MHD: psi damping length c_r = c_p^2/c_h (Sec. 4.2); <= 0 disables damping */
  int recon;      /* AMRFD_MP5 (Suresh & Huynh, Sec. 2.2) | AMRFD_LIMO3 (Cada & Torrilhon, Sec. 2.2) */
  int reserved_;  /* set to 0 */
  double limo3_r; /* LIMO3: radius r of the asymptotic region, > 0; the switch compares
                     (delta_-^2 + delta_+^2) of the split fluxes with (r dx)^2 */
} amrfd_config;

typedef struct amrfd_domain {
  int n[3];        /* interior cells per dimension; 1 for dimensions >= ndim */
  int nb[3];       /* blocks per dimension (n[d] % nb[d] == 0); a block is the unit of activity */
  double dx[3];    /* cell size per dimension (> 0) */
  int bc[3][2];    /* AMRFD_BC_* of the low and high face of each dimension; periodic must pair */
  uint32_t asym[3][2]; /* AMRFD_BC_SYMMETRIC faces: bit v set = conserved variable v is odd
                          (antisymmetric) across the face, clear = even (symmetric). Ghost
                          layer m = 1..3 outside the face holds interior cell m-1 inside it,
                          odd variables negated (the per-variable symmetric/antisymmetric
                          ghost kinds of Sec. 4.5.10); a reflecting wall sets the normal
                          momentum (MHD: and the tangential field and psi) odd. Ignored on
                          other faces; bits >= nv are invalid. */
  int64_t offset;  /* element offset of U[0][0][0][0] of this domain in the state buffer */
} amrfd_domain;

typedef struct amrfd_handle amrfd_handle;

/* Create a handle for `ndomain` domains (copied). `active_host` has one flag per
   block, blocks numbered domain by domain and, inside a domain, x-fastest; NULL
   means all active (App. C: only active blocks are advanced). Allocates the
   workspace (stage states, per-direction residuals, speeds, work lists) with
   cudaMalloc on the current device. Constraints: n[d] >= 3 along periodic
   dimensions and at mirror (AMRFD_BC_SYMMETRIC) faces, n[d] >= 1 otherwise;
   domains must not overlap. Returns
   AMRFD_ERR_INVALID_ARG on bad arguments, AMRFD_ERR_CUDA on allocation failure. */
int amrfd_create(amrfd_handle **h, const amrfd_config *cfg, const amrfd_domain *domains, int ndomain,
                 const uint8_t *active_host, void *stream);

/* Replace the per-block active flags from DEVICE memory (uint8, one per block)
   and rebuild the device work lists of active blocks. Synchronises `stream`
   once to keep a host copy for the per-domain path. */
int amrfd_set_active(amrfd_handle *h, const uint8_t *active_dev, void *stream);

/* Dynamic grid activation, App. C step 1 with a built-in criterion: writes
   flag_dev[b] = 1 (candidate for de-activation) for every block b whose cells
   all lie within tol (absolute, every conserved variable) of U_ref, e.g. the
   initial or an analytic stationary state, else 0 (a NaN counts as a
   deviation). U, U_ref: device, state layout; flag_dev: device, one byte per
   block (caller-owned). Asynchronous; every block is tested, active or not. */
int amrfd_flag_steady(amrfd_handle *h, const double *U, const double *U_ref, double tol, uint8_t *flag_dev,
                      void *stream);

/* Dynamic grid activation, App. C steps 2 and 3: blocks with flag_dev[b] = 0
   become active, candidates (flag 1) passive; then `belt` times (>= 0) every
   passive block with an active neighbour (sharing a face, edge or corner in its
   domain; neighbours wrap across periodic faces) is re-activated, each round
   testing against the previous round's flags; the device work lists are then
   rebuilt on the device. Asynchronous on `stream`, no host synchronisation; the
   next amrfd_step or amrfd_adjoint synchronises once to refresh the host copy
   of the flags (amrfd_step_batched and amrfd_dt need none). Returns
   AMRFD_ERR_INVALID_ARG for belt < 0. */
int amrfd_activate(amrfd_handle *h, const uint8_t *flag_dev, int belt, void *stream);

/* Copy the current per-block active flags to active_dev (device, one byte per
   block). Asynchronous. */
int amrfd_get_active(amrfd_handle *h, uint8_t *active_dev, void *stream);

/* CFL time step per domain (Sec. 4.4, unsplit multi-D form):
   dt = cfl / max over active cells of sum_d c_d/dx_d, where c_d = |v_d| + fast
   (MHD) or sound (Euler) speed and, with GLM, every c_d is raised to the GLM
   speed c_h = max_d max_cells c_d; then dt = min(dt, t_end - t). With
   AMRFD_DT_GLOBAL every entry receives the minimum over domains. Writes
   dt_dev[ndomain] (device). Domains with no active block get t_end - t. */
int amrfd_dt(amrfd_handle *h, const double *U, double *dt_dev, double t, double t_end, void *stream);

/* One SSPRK step of every active block, in place, with per-domain time steps
   dt_dev[ndomain] (device). Plain path: one launch per domain for each pass
   (flux pass and stage combination of every RK stage). Passive blocks are
   neither read as interior nor written; active blocks read their passive
   neighbours' U^n as halo. */
int amrfd_step(amrfd_handle *h, double *U, const double *dt_dev, void *stream);

/* Same update as amrfd_step, bitwise identical, issued as one persistent launch
   per pass over a device-side work list of active (block, tile) items sorted
   largest first; the whole step is replayed from a CUDA graph captured on the
   first call for a given (U, dt_dev) pair (the 16 most recently used pairs are
   kept; evicting one synchronises `stream` once). */
int amrfd_step_batched(amrfd_handle *h, double *U, const double *dt_dev, void *stream);

/* One CFL-limited step: writes dt_dev[ndomain] (device) exactly as
   amrfd_dt(h, U, dt_dev, t, t_end) would and advances U with it, bitwise as
   amrfd_dt followed by amrfd_step_batched, with the speed maxima of U^n (Sec. 2.2,
   4.4) evaluated once for both. Persistent launches, no graph (t and t_end are
   arguments of every call). */
int amrfd_step_cfl(amrfd_handle *h, double *U, double *dt_dev, double t, double t_end, void *stream);

/* Discrete adjoint of one amrfd_step with the same U^n and dt: given
   gU_np1 = dJ/dU^{n+1}, writes gU_n = dJ/dU^n (both device, state layout).
   Splitting speeds c_max, c_h and the psi damping factor are held fixed at
   the values the forward step used; the pieces the MP5 or LIMO3 limiter took
   at every face are replayed from a forward recomputation (inside LIMO3's
   2e-12-wide blend band, the piece of the nearer half). Passive blocks
   (App. C) are the identity map, and where an active block's fluxes read a
   passive neighbour's U^n as halo, that dependence is transposed into gU_n
   too. Returns AMRFD_ERR_UNSUPPORTED for a periodic dimension of fewer than
   6 cells, a mirror dimension whose blocks hold fewer than 3 cells along it,
   or a partly active domain whose blocks hold fewer than 3 cells along a
   dimension. */
int amrfd_adjoint(amrfd_handle *h, const double *U_n, const double *dt_dev, const double *gU_np1,
                  double *gU_n, void *stream);

/* A step that keeps what its adjoint needs, so that the adjoint need not recompute it
   (no counterpart in the paper: the discrete adjoint above, split at its forward
   recomputation). amrfd_record_bytes(h): size of one record of this handle (the splitting
   speeds of every stage input, the stage states U^(1..s-1), the limiter pieces of every
   flux pass); 0 for a NULL handle. amrfd_step_record: one SSPRK step of U in place, exactly
   as amrfd_step_batched, that also fills `record` (device memory of at least
   amrfd_record_bytes bytes, 16-byte aligned, caller-owned). amrfd_adjoint_recorded: the
   gradient amrfd_adjoint would give for the step that wrote `record`, from U_n = the state
   before that step (the caller keeps a copy: the step overwrote U) and the same dt_dev,
   without the forward recomputation. A record serves only the handle that wrote it, with
   its active flags unchanged since. Both are asynchronous; AMRFD_ERR_INVALID_ARG for NULL
   or misaligned pointers, AMRFD_ERR_UNSUPPORTED as amrfd_adjoint. */
size_t amrfd_record_bytes(const amrfd_handle *h);
int amrfd_step_record(amrfd_handle *h, double *U, const double *dt_dev, void *record, void *stream);
int amrfd_adjoint_recorded(amrfd_handle *h, const double *U_n, const double *dt_dev, const void *record,
                           const double *gU_np1, double *gU_n, void *stream);

/* Choose the flux-pass tile (segment length along the sweep, lines per tile,
   threads per block) by timing the candidates on this handle's work, using U
   and dt_dev as the sample state (U is restored). Synchronises `stream`. */
int amrfd_autotune(amrfd_handle *h, double *U, const double *dt_dev, void *stream);

/* Set the flux-pass tile explicitly: seg = max cells per sweep segment
   (8..64), lines = lines per tile (1..32), threads per block (multiple of 32,
   32..320). Every tile gives bitwise the same results. */
int amrfd_set_tile(amrfd_handle *h, int seg, int lines, int threads);
/* Read back the current tile. */
int amrfd_get_tile(const amrfd_handle *h, int *seg, int *lines, int *threads);

/* Set the tile of amrfd_adjoint's transposed flux pass (no counterpart in the paper; a
   tuning knob like amrfd_set_tile; default 16 cells, 16 lines, 192 threads): seg = max
   cells per segment (6..64), lines = lines
   per tile (1..32), threads per block (multiple of 32, 32..256); its shared memory must
   stay within 227 KB (AMRFD_ERR_INVALID_ARG beyond). Every tile gives bitwise the same
   gradients. Synchronous when the adjoint's workspace exists (its items are rebuilt). */
int amrfd_set_adjoint_tile(amrfd_handle *h, int seg, int lines, int threads);

/* Kernel timing for measurement. After amrfd_timing_begin(h, capacity), every
   kernel that amrfd_dt, amrfd_step and amrfd_step_batched launch is bracketed by
   a pair of CUDA events recorded on the launching stream (amrfd_step_batched
   then issues its persistent launches directly instead of replaying the graph;
   the kernels are the same). At most `capacity` launches are recorded.
   amrfd_timing_end synchronises `stream`, writes per kernel kind
   (0 speeds, 1 flux pass, 2 stage combination, 3 time step) the summed elapsed
   milliseconds and the launch counts, and stops timing. */
int amrfd_timing_begin(amrfd_handle *h, int capacity);
int amrfd_timing_end(amrfd_handle *h, double ms[4], int counts[4], void *stream);

/* FP64 throughput of this GPU, the denominator of the flux pass's roofline (the
   paper has no counterpart: a measurement utility). Runs a kernel of independent
   FP64 fused multiply-adds on `stream`: five single launches after a warm-up
   (burst: the best) and then back-to-back launches for about `seconds` (0..60;
   sustained). out[0] = burst TFLOP/s, out[1] = sustained TFLOP/s (2 flop per
   FMA), out[2] = milliseconds of the best launch, out[3] = FMAs per launch.
   Synchronises `stream`; AMRFD_ERR_INVALID_ARG for a bad `seconds` or NULL out. */
int amrfd_fp64_peak(double seconds, double out[4], void *stream);

/* Per-stage splitting speeds of the last step, raw (before raising to c_h):
   out[stage][domain][3], host memory, `nstage` = stages to copy. Synchronises. */
int amrfd_get_alpha(amrfd_handle *h, double *out, int nstage, void *stream);

/* Synchronise `stream`, return the latched device condition (AMRFD_OK,
   AMRFD_ERR_CHECK in a checked build, else AMRFD_ERR_NONPHYSICAL) and clear it. */
int amrfd_get_error(amrfd_handle *h, void *stream);

/* Free the handle and its workspace (synchronises the device first). */
void amrfd_destroy(amrfd_handle *h);

/* CFL time step of amrfd_dt for callers that cannot allocate device memory
   (no handle, no cudaMalloc, no heap use). The paper has no counterpart: this is
   a deployment variant of amrfd_dt. Inputs as for amrfd_create plus amrfd_dt:
   `domains[ndomain]` (host), optional per-block `active_dev` (device, NULL = all
   active), state `U` and output `dt_dev[ndomain]` (device). Scratch is a fixed
   ~116 KB __device__ array inside the library, held by every GPU that loads it
   until the process exits; ndomain is limited to 1024 (AMRFD_ERR_INVALID_ARG,
   with a message on stderr, beyond). The descriptors travel as kernel arguments:
   the call neither copies from host memory nor waits for the GPU. The first call
   on a device looks up the array's device address (cudaGetSymbolAddress); that
   address is kept for the life of the process, so the library must not outlive a
   reset of the device's primary context. All calls
   share the one array and each leaves its contents behind: calls whose work
   overlaps on the GPU (other streams, other host threads) race; serialise them.
   A domain holding a non-physical cell (rho <= 0, p <= 0 or a non-finite value,
   among its active cells) gets dt = NaN, and with AMRFD_DT_GLOBAL every domain
   does; amrfd_dt instead leaves such cells out and latches AMRFD_ERR_NONPHYSICAL. */
int amrfd_dt_noalloc(const amrfd_config *cfg, const amrfd_domain *domains, int ndomain,
                     const uint8_t *active_dev, const double *U, double *dt_dev, double t, double t_end,
                     void *stream);

/* Static description of a return code. */
const char *amrfd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
