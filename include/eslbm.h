/*
 * eslbm.h -- C ABI of the GB300 (sm_103a) implementation of the fourth-order,
 * entropy-stable, vectorial lattice Boltzmann scheme of Bellotti, Helluy and
 * Navoret, "Fourth-order entropy-stable lattice Boltzmann schemes for
 * hyperbolic systems" (arXiv 2403.13406).
 *
 * The calls follow the paper's statement of the problem:
 *   - initialise the distributions at equilibrium from conserved fields
 *     (Section 3.1: data taken at equilibrium, f_k = f^eq_k(u0));
 *   - run n composite steps Phi(dt) = psi(dt/6)^4 psi(-dt/3) psi(dt/6)^4 of the
 *     basic brick psi(dt) = T(dt/4) R T(dt/2) R T(dt/4) (eqs. splittingToUse
 *     and basicBrickSplitting), dt = 24 kappa dx / V (Section 2.3), with the
 *     relaxation R_omega of eq. relaxationDiscretizationOmega and either a
 *     fixed omega or the per-cell entropic omega of eq. variableOmegaProblem
 *     (Section 4);
 *   - read back the conserved moments u = sum_k f_k and the total microscopic
 *     and macroscopic entropies (Section 4).
 *
 * Conventions
 *   - Velocity sets (Section 1.2): D1Q2 with velocities (+V, -V); D2Q4 with
 *     (+V,0), (0,+V), (-V,0), (0,-V), in that order.
 *   - Distributions are stored structure-of-arrays: plane (k*M + m) holds the
 *     m-th conserved component of population k for every cell, cells row-major
 *     with x fastest (cell = y*nx + x).  Conserved fields use M planes with the
 *     same cell order.  Host-side fields are always double precision; device
 *     state is float or double according to eslbm_config.precision.
 *   - The grid is periodic with cells at x_j = j dx.
 *   - Memory: the caller owns every buffer.  The library never allocates device
 *     memory: eslbm_create receives two state buffers (ping-pong) and a
 *     workspace, sized by eslbm_query.  Buffers passed with on_device = 0 are
 *     host buffers; the call then copies through the spare state buffer and
 *     synchronizes the stream before it returns.  Device buffers are used
 *     asynchronously on the handle's stream.
 *   - Errors: nothing throws across the ABI.  Every call returns an
 *     eslbm_status; eslbm_last_error(h) describes the last failure of h.
 */
#ifndef ESLBM_H
#define ESLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESLBM_ABI_VERSION 3

typedef enum {
    ESLBM_OK = 0,
    ESLBM_ERR_ARG = 1,          /* invalid argument (null pointer, size, enum value) */
    ESLBM_ERR_DOMAIN = 2,       /* data outside the convexity / sub-characteristic domain */
    ESLBM_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    ESLBM_ERR_NAN = 4,          /* non-finite values in the input or the state */
    ESLBM_ERR_UNSUPPORTED = 5,  /* valid but not implemented combination */
    ESLBM_WARN_OMEGA_FALLBACK = 100 /* some cells had no entropic root; omega = 1 was used */
} eslbm_status;

/* Conservation laws of Section 1.2.  LINEAR: phi^j = a_j u (Examples 1, 4).
   BURGERS: phi^j = c_j u^2/2 (Example 2; Section 3.3 uses c = (1, 3/5)).
   SHALLOW_WATER: (h, hu[, hv]) with gravity g (Example 3).  EULER: (rho, rho u,
   rho v, E) with gamma-law pressure (Section 6.3), fixed omega only. */
enum { ESLBM_LINEAR = 0, ESLBM_BURGERS = 1, ESLBM_SHALLOW_WATER = 2, ESLBM_EULER = 3 };
/* Precision.  FP32 / FP64: storage and all arithmetic of the relaxation in that
   type (the reported reductions are FP64 in every mode).  FP32_MIXED (no
   counterpart in the paper): FP32 storage and FP32 root-find iterations, with the
   entropy difference of the entropic omega evaluated in FP64 -- E0 = B(-1) and
   the residual F(t) = B(t) - E0 at the returned root, B(t) = sum_k B_k(t delta_k)
   (Section 4, eq. variableOmegaProblem); when F(t) > 0 the chord root through
   (0, -E0) and (t, F(t)), which never exceeds the root of the convex F, replaces
   t.  With a fixed omega FP32_MIXED is FP32. */
enum { ESLBM_FP32 = 0, ESLBM_FP64 = 1, ESLBM_FP32_MIXED = 2 };
/* Temporal blocking (eslbm_config.blocking): AUTO runs the fastest measured path
   -- 1D: every step in one launch from shared memory; 2D: the temporally blocked
   2D kernel two stages a launch for Euler (16 planes) in FP32 with a fixed omega,
   one launch per fused stage otherwise.  OFF runs one launch per fused stage in
   1D and 2D (the same per-cell
   arithmetic; used to cross-check the blocked kernels).  A value n in [2, 32]
   runs the temporally blocked 2D kernel where rows start on 16-byte boundaries
   (nx a multiple of 4 in FP32 and FP32_MIXED, of 2 in FP64), at most n stages
   per launch (1D as AUTO). */
enum { ESLBM_BLOCKING_AUTO = 0, ESLBM_BLOCKING_OFF = 1 };
enum { ESLBM_OMEGA_FIXED = 0, ESLBM_OMEGA_ENTROPIC = 1 };
/* Schemes (I)-(IV) of Section 6.1; PLAIN is the standard scheme R T(kappa dx/V)
   of Section 2.1 (one stage per step); B is scheme (B) of Section 6.3,
   R_1 T(dt/4) R T(dt/2) R T(dt/4) with dt = 4 kappa dx / V. */
enum { ESLBM_SCHEME_I = 1, ESLBM_SCHEME_II = 2, ESLBM_SCHEME_III = 3, ESLBM_SCHEME_IV = 4,
       ESLBM_SCHEME_PLAIN = 5, ESLBM_SCHEME_B = 6 };
/* Relaxation kinds for eslbm_relax: the scheme's main relaxation (fixed omega
   or entropic omega) or the projection on the equilibrium R_1 (Section 6.1). */
enum { ESLBM_RELAX_MAIN = 0, ESLBM_RELAX_PROJECT = 1 };

typedef struct {
    int32_t dim;        /* 1 (D1Q2) or 2 (D2Q4) */
    int32_t system;     /* ESLBM_LINEAR, ESLBM_BURGERS, ESLBM_SHALLOW_WATER, ESLBM_EULER */
    int32_t precision;  /* ESLBM_FP32, ESLBM_FP64 or ESLBM_FP32_MIXED (see above) */
    int32_t omega_mode; /* ESLBM_OMEGA_FIXED or ESLBM_OMEGA_ENTROPIC */
    int32_t scheme;     /* ESLBM_SCHEME_* */
    int32_t kappa;      /* shift unit V dt / (24 dx) >= 1 (Section 2.3; the paper uses 1) */
    int64_t nx, ny;     /* cells per direction; ny = 1 when dim = 1 */
    double V;           /* lattice velocity V > 0 */
    double omega;       /* fixed relaxation parameter (fixed mode), e.g. 2 */
    double a[2];        /* linear transport velocity */
    double c[2];        /* Burgers flux coefficients */
    double g;           /* gravity (shallow water) */
    double gamma;       /* ratio of specific heats (Euler) */
    double t_max;       /* entropic mode: omega - 1 is searched in [0, t_max]; 0 -> 3 */
    int32_t diagnostics;/* 1: check every entropic relaxation per cell and track omega min/max
                           (eslbm_diagnostics); the same kernels run, the results do not change */
    int32_t shifted;    /* 1: store g = f - fbar with fbar_k = f^eq_k(u_ref) (see below); 0: store f */
    double u_ref[4];    /* reference conserved state of the shifted storage (M values used) */
    int32_t blocking;   /* ESLBM_BLOCKING_AUTO, ESLBM_BLOCKING_OFF, or 2..32 (see above) */
    int32_t reserved;   /* 0 */
} eslbm_config;

/* Shifted storage (no counterpart in the paper).  With shifted = 1 the state
   buffers hold g_k = f_k - fbar_k, fbar_k = f^eq_k(u_ref) rounded to the storage
   precision, and the relaxation works on deviations from the reference state
   (the conserved moments as u_ref + sum_k g_k, the equilibrium as
   f^eq(u) - f^eq(u_ref) in a cancellation-free form).  The rounding of the
   stored values is then relative to |f - fbar| instead of |f|: for data close to
   a background state (e.g. a depth of 1 plus waves of amplitude 0.1) the FP32
   rounding error of a long run drops by the ratio of the two.  The scheme and
   every call's inputs and outputs are unchanged (f and u in, f and u out); only
   the raw buffers differ, so eslbm_read_totals_noalloc must receive the same
   configuration.  u_ref must lie in the domain of Section 1.2 (else
   ESLBM_ERR_DOMAIN from eslbm_query and eslbm_create). */

typedef struct {
    int64_t q;               /* velocities: 2 (D1Q2) or 4 (D2Q4) */
    int64_t M;               /* conserved components */
    int64_t planes;          /* q * M */
    int64_t ncell;           /* nx * ny */
    uint64_t state_bytes;    /* bytes of one distribution buffer (planes * ncell * element) */
    uint64_t workspace_bytes;/* bytes of the workspace */
    int64_t stages_per_step; /* fused relax-plus-shift stages per step of the scheme */
    int64_t step_cells;      /* lattice time of one step in units of dx / V (24 kappa for I-IV) */
    double launches_per_step;/* relaxation kernel launches per step in steady state (1D: one per
                                step, or one per 24 steps of the short schemes; 2D blocked: one per
                                group of stages; otherwise one per stage); diagnostics add one
                                check launch after each */
} eslbm_sizes;

/* Per-cell entropy check (diagnostics = 1, entropic omega, Section 4): for every
   relaxation the kernel evaluates, in FP64 from the moments and deviations it
   used and with its own constants, F(omega - 1) = B(omega - 1) - B(-1), the change
   of the cell's microscopic entropy under R_omega.  entropy_increases counts the
   cells where F exceeds 64 unit roundoffs of B(-1) in the arithmetic that chose
   omega (FP32, or FP64 for FP64 and FP32_MIXED); entropy_excess_max is the largest
   F / B(-1) seen (0 if never positive). */
typedef struct {
    uint64_t relaxations;        /* cell relaxations since the last reset */
    uint64_t fallbacks;          /* cells that used omega = 1 (no entropic root) */
    uint64_t entropy_increases;  /* cells whose Sigma increased (diagnostics = 1, see above) */
    double omega_min, omega_max; /* range of omega used (diagnostics = 1) */
    double entropy_excess_max;   /* largest F(omega - 1) / B(-1) (diagnostics = 1, see above) */
} eslbm_diagnostics;

typedef struct eslbm_handle eslbm_handle;

/* Version of this ABI (ESLBM_ABI_VERSION). */
int32_t eslbm_abi_version(void);

/* Human-readable name of a status code; never NULL. */
const char *eslbm_status_string(eslbm_status s);

/* Sizes of the buffers for cfg.  Validates cfg (ESLBM_ERR_ARG on a bad
   field, ESLBM_ERR_UNSUPPORTED for entropic Euler). */
eslbm_status eslbm_query(const eslbm_config *cfg, eslbm_sizes *out);

/* Create a handle.  f_a, f_b: device buffers of sizes.state_bytes each (16-byte
   aligned); workspace: device buffer of sizes.workspace_bytes; stream: a
   cudaStream_t (NULL = legacy default stream).  The buffers stay owned by the
   caller and must outlive the handle.  The handle is allocated on the host. */
eslbm_status eslbm_create(const eslbm_config *cfg, void *f_a, void *f_b, void *workspace,
                          void *stream, eslbm_handle **out);

/* Release the handle (not the buffers).  Safe on NULL. */
eslbm_status eslbm_destroy(eslbm_handle *h);

/* Switch the stream used by later calls. */
eslbm_status eslbm_set_stream(eslbm_handle *h, void *stream);

/* Message describing the last failure on h (empty if none); never NULL. */
const char *eslbm_last_error(const eslbm_handle *h);

/* f_k = f^eq_k(u0) in every cell (Section 3.1).  u0: M double planes of ncell
   cells.  Checks the convexity / sub-characteristic domain of Section 1.2 on the
   device (synchronizes) and returns ESLBM_ERR_DOMAIN if a cell violates it,
   ESLBM_ERR_NAN for non-finite input; the state is then written but not
   meaningful.  Resets the pending shift. */
eslbm_status eslbm_init_equilibrium(eslbm_handle *h, const double *u0, int32_t u0_on_device);

/* Set the distributions directly (q*M double planes, rounded to the storage
   precision), e.g. off-equilibrium data (Section 6.2).  No domain check. */
eslbm_status eslbm_init_distributions(eslbm_handle *h, const double *f0, int32_t on_device);

/* Advance n composite steps of the configured scheme (eq. splittingToUse for
   scheme I).  Asynchronous on the stream; adjacent transports are merged into
   one pull-shift per fused stage and the trailing shift of the last step is
   kept pending until the next stage or readback. */
eslbm_status eslbm_step(eslbm_handle *h, int64_t n);

/* Apply the transport T(s) (eq. transportPhase, s cells along each
   population's velocity, negative s reverses it): recorded as a pending shift
   and folded into the next stage or readback (a pure permutation). */
eslbm_status eslbm_transport(eslbm_handle *h, int64_t s);

/* One relaxation sweep (eq. relaxationDiscretizationOmega) of the given kind,
   fused with the pending shift. */
eslbm_status eslbm_relax(eslbm_handle *h, int32_t kind);

/* Conserved moments u = sum_k f_k (M double planes) of the current state. */
eslbm_status eslbm_read_moments(eslbm_handle *h, double *u_out, int32_t on_device);

/* Distributions in logical order (q*M double planes, pending shift applied). */
eslbm_status eslbm_read_distributions(eslbm_handle *h, double *f_out, int32_t on_device);

/* Totals reduced in double precision with a fixed order (deterministic):
   out[0] = sum_x Sigma(f(x)) (total microscopic entropy, Section 4),
   out[1] = sum_x S(u(x)) (total entropy of the moments),
   out[2 .. 2+M-1] = sum_x u_m(x) (conserved totals).
   Entropies are NaN for EULER (no kinetic entropy is defined). */
eslbm_status eslbm_read_totals(eslbm_handle *h, double *out, int32_t on_device);

/* Counters accumulated by the stage kernels since the last reset (synchronizes).
   Returns ESLBM_WARN_OMEGA_FALLBACK when fallbacks > 0, and ESLBM_ERR_CUDA if a
   2D stage staged by bulk copies gave up waiting for them (its cells were then
   not relaxed; not expected to happen). */
eslbm_status eslbm_get_diagnostics(eslbm_handle *h, eslbm_diagnostics *out);
eslbm_status eslbm_reset_diagnostics(eslbm_handle *h);

/* Totals of a caller-held state, for callers that cannot allocate device memory
   (no counterpart in the paper).  eslbm_read_totals needs a handle, whose
   workspace the caller must allocate; code that runs while a CUDA graph is being
   captured, or a host that gives the library a fixed pre-sized pool, cannot.
   This call allocates nothing: its scratch is a file-scope device array of
   64 KiB (8 x 1024 partial sums plus 8 totals) that every device loading the
   library keeps until the process exits.
   cfg: the state's configuration; f: device buffer of planes * ncell values in the
   storage precision (16-byte aligned), physical layout; pending_shift: transport
   still to apply (the totals are those of T(pending_shift) f); out: 2 + M doubles
   as in eslbm_read_totals, device memory if out_on_device, else host memory (the
   call then synchronizes the stream).  Same fixed-order reduction as
   eslbm_read_totals.
   The first call on a device looks up the scratch's device address on the current
   device; make that first call before any stream capture.  The address is then
   cached for the life of the process: after cudaDeviceReset, or any other teardown
   of the device's primary context, it is stale, and the call must not be used again
   in that process.  All calls share the scratch (it keeps the last call's contents;
   every call overwrites what it reads), so calls that overlap on the GPU, e.g. on
   two streams, race.
   A call made while `stream` is being captured into a CUDA graph must pass
   out_on_device = 1: the host copy of out_on_device = 0 ends with a stream
   synchronization, which capture forbids, so such a call returns ESLBM_ERR_ARG and
   records nothing.
   Errors: ESLBM_ERR_ARG for a bad cfg, a null or misaligned pointer, totals that
   do not fit the scratch (more than 8, i.e. M > 6), or out_on_device = 0 on a
   capturing stream; ESLBM_ERR_CUDA on a failed CUDA call. */
eslbm_status eslbm_read_totals_noalloc(const eslbm_config *cfg, const void *f, int64_t pending_shift,
                                       double *out, int32_t out_on_device, void *stream);

/* Bytes of the device workspace eslbm_gradient needs for n steps checkpointed
   every K steps: (ceil(n/K) + min(K, n) + stages_per_step + 2) state buffers,
   each rounded up to 256 bytes. */
eslbm_status eslbm_gradient_workspace(const eslbm_config *cfg, int64_t n, int64_t K, uint64_t *bytes);

/* Reverse mode (no counterpart in the paper, which does not differentiate the
   scheme): gradient dJ/du0 of a scalar J(u_T) for u_T = the moments after n steps
   of the configured scheme from f_0 = f^eq(u0).  u0, dJ_duT, dJ_du0: M double
   planes in device memory.  The forward pass keeps the state every K steps in ws;
   the reverse pass recomputes each K-step segment (keeping every step's starting
   state), then each step stage by stage (keeping every stage's input; in 1D one
   launch of the temporally blocked kernel that also writes every stage's output),
   and applies
   the adjoint stages in reverse: the reverse shift of the transport and the
   transposed Jacobian of the relaxation, including the derivative of the entropic
   omega by the implicit function theorem on eq. variableOmegaProblem.  On return
   the handle holds the final forward state.  ws: device workspace of at least
   eslbm_gradient_workspace bytes, 256-byte aligned.  Synchronizes (the forward
   init checks the domain). */
eslbm_status eslbm_gradient(eslbm_handle *h, const double *u0, const double *dJ_duT, double *dJ_du0, int64_t n,
                            int64_t K, void *ws, uint64_t ws_bytes);

/* Capture the launches of one step (two for an odd number of stages) in a CUDA
   graph and replay it inside eslbm_step (enable = 1), or launch directly
   (enable = 0, the default). */
eslbm_status eslbm_use_graph(eslbm_handle *h, int32_t enable);

/* ------------------------------------------------------------------------
   Batched execution (no counterpart in the paper, which runs one lattice at a
   time): `count` independent periodic 2D lattices of sizes nx[i] x ny[i] that
   share one configuration (system, precision, omega mode, scheme, V and the
   physical constants; the nx, ny of `base` are ignored) advance together.  One
   composite step of all of them is ONE cooperative launch: the blocks sweep a
   work list of row segments of every instance for each fused stage, with a grid
   barrier between stages.  Every instance computes exactly what a single
   handle with its sizes computes (same per-cell arithmetic, same stage list).
   Only dim = 2 is supported (ESLBM_ERR_UNSUPPORTED otherwise).
   ------------------------------------------------------------------------ */
typedef struct eslbm_batch eslbm_batch;

typedef struct {
    int32_t count;           /* instances */
    int64_t q, M, planes;    /* as in eslbm_sizes */
    int64_t total_cells;     /* sum of nx[i] * ny[i] */
    uint64_t pool_bytes;     /* bytes of one state pool: the instances' states, each 256-byte aligned */
    uint64_t workspace_bytes;/* bytes of the workspace (counters, instance and work lists, one
                                single-lattice workspace for eslbm_batch_gradient) */
    int64_t stages_per_step; /* fused stages of one composite step */
    int64_t step_cells;      /* lattice time of one step, as in eslbm_sizes */
} eslbm_batch_sizes;

/* Sizes for `count` instances; validates every instance as eslbm_query does.
   Errors: ESLBM_ERR_ARG (null pointer, count < 1, bad field), ESLBM_ERR_UNSUPPORTED. */
eslbm_status eslbm_batch_query(const eslbm_config *base, int32_t count, const int64_t *nx, const int64_t *ny,
                               eslbm_batch_sizes *out);

/* Create a batch.  pool_a, pool_b: distinct device buffers of pool_bytes each;
   workspace: device buffer of workspace_bytes; all 256-byte aligned, owned by the
   caller and outliving the batch.  Instance i occupies planes * nx[i] * ny[i]
   values of each pool in the layout of a single handle, starting at the pool
   offset sum_{j<i} round_up(state_bytes_j, 256).  stream: a cudaStream_t.
   Synchronizes once (uploads the work list).  The default schedule is 256-cell
   segments, the kernel's full residency, instance-major order. */
eslbm_status eslbm_batch_create(const eslbm_config *base, int32_t count, const int64_t *nx, const int64_t *ny,
                                void *pool_a, void *pool_b, void *workspace, void *stream, eslbm_batch **out);
eslbm_status eslbm_batch_destroy(eslbm_batch *b);
const char *eslbm_batch_last_error(const eslbm_batch *b);

/* f = f^eq(u0) for every instance (Section 3.1).  u0: the instances' moments one
   after the other, each M double planes of nx[i] * ny[i] cells; device memory if
   on_device, else host memory (staged through the spare pool).  Synchronizes.
   ESLBM_ERR_DOMAIN / ESLBM_ERR_NAN as in eslbm_init_equilibrium (the state is then
   written but not meaningful). */
eslbm_status eslbm_batch_init_equilibrium(eslbm_batch *b, const double *u0, int32_t on_device);

/* Advance every instance n composite steps (one cooperative launch per step;
   asynchronous).  ESLBM_ERR_CUDA if the cooperative launch is refused. */
eslbm_status eslbm_batch_step(eslbm_batch *b, int64_t n);

/* Moments of every instance in the layout of eslbm_batch_init_equilibrium's u0;
   device memory if on_device, else host memory (synchronizes). */
eslbm_status eslbm_batch_read_moments(eslbm_batch *b, double *u_out, int32_t on_device);

/* Schedule of the batched launch: row segments of `segment` cells (>= 128),
   blocks_per_sm resident blocks per SM (1 .. the kernel's occupancy), order 0 =
   instance-major work list, 1 = rows of all instances interleaved.  Results do not
   depend on the schedule (bitwise).  Synchronizes. */
eslbm_status eslbm_batch_set_schedule(eslbm_batch *b, int64_t segment, int32_t blocks_per_sm, int32_t order);
eslbm_status eslbm_batch_get_schedule(const eslbm_batch *b, int64_t *segment, int32_t *blocks_per_sm,
                                      int32_t *order);

/* Autotuner: times `steps` steps of every candidate schedule (segments 128, 256,
   512, 1024; full, half and single residency; both orders) with CUDA events from
   the current state, keeps the fastest, and restores the state.  scratch: device
   buffer of at least pool_bytes.  Synchronizes. */
eslbm_status eslbm_batch_tune(eslbm_batch *b, void *scratch, uint64_t scratch_bytes, int32_t steps);

/* Replay each step from a CUDA graph of its cooperative launch (enable = 1) or
   launch directly (0, the default).  Needs a non-NULL stream. */
eslbm_status eslbm_batch_use_graph(eslbm_batch *b, int32_t enable);

/* Reverse mode per instance: workspace bytes (the largest instance's
   eslbm_gradient_workspace) and the gradients.  u0, dJ_duT, dJ_du0: device
   memory in the layout of eslbm_batch_init_equilibrium's u0.  Each instance runs
   eslbm_gradient on a temporary handle over its part of the pools; on return the
   batch holds f^eq(u0) (the state at step 0).  Synchronizes. */
eslbm_status eslbm_batch_gradient_workspace(const eslbm_config *base, int32_t count, const int64_t *nx,
                                            const int64_t *ny, int64_t n, int64_t K, uint64_t *bytes);
eslbm_status eslbm_batch_gradient(eslbm_batch *b, const double *u0, const double *dJ_duT, double *dJ_du0, int64_t n,
                                  int64_t K, void *ws, uint64_t ws_bytes);

/* Counters of the batched kernels since creation (synchronizes): fallbacks, and
   with base.diagnostics = 1 the per-cell entropy check and the omega range as in
   eslbm_get_diagnostics (relaxations is not tracked, returned as 0).
   ESLBM_WARN_OMEGA_FALLBACK when fallbacks > 0. */
eslbm_status eslbm_batch_get_diagnostics(eslbm_batch *b, eslbm_diagnostics *out);

#ifdef __cplusplus
}
#endif
#endif /* ESLBM_H */
