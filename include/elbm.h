/*
 * elbm.h -- C ABI of the GB300 library for the essentially entropic lattice
 * Boltzmann step of Atif, Kolluru & Ansumali, "Essentially entropic lattice
 * Boltzmann model: Theory and simulations" (arXiv:2203.12946).
 *
 * One time step, per lattice node (Sec. I, Sec. III, Appendix D):
 *   1. pull-stream the Q populations from the neighbours (Eq. advection),
 *   2. form rho and u (Sec. I) and the product-form entropic equilibrium,
 *   3. x_i = f_i^eq / f_i - 1 (Eq. xdef),
 *   4. the closed-form path length alpha: alpha = 2 when |x|max < 1e-3,
 *      otherwise alpha_Lower (Eq. alphaLowerSoln), the upper bound h (Eq.
 *      gaplhah0) and alpha_Higher (Eq. qaud_tight, qaud_tight_coeff), then the
 *      positivity clamp (Appendix D),
 *   5. relax f* = f + alpha beta (f^eq - f) (Eq. fstar_def) and store.
 *
 * Conventions shared by every entry point
 *  - All functions return an int status (ELBM_OK or a negative ELBM_ERR_*).
 *    No exception, abort or exit crosses the ABI.  A failed call leaves a
 *    message in elbm_last_error(handle) (or elbm_last_error(NULL) when no
 *    handle exists yet).
 *  - Lattices: D2Q9 and D3Q27, the tensor products of D1Q3 (Sec. I).
 *    Velocity i enumerates (c_x, c_y[, c_z]) in {-1,0,1}^D lexicographically
 *    with the last axis fastest: i = sum_a (c_a + 1) 3^(D-1-a); the opposite
 *    velocity of i is Q-1-i.  Weights are products of the D1Q3 weights
 *    {1/6, 4/6, 1/6}.
 *  - Populations are stored structure-of-arrays: element (i, n) at offset
 *    i*N + n, with node index n = (z*ny + y)*nx + x, N = nx*ny*nz (nz = 1 for
 *    D2Q9).  The element type is the storage type of the handle (see
 *    ELBM_STORE_*).  The stored state is the post-collision field f*.
 *  - Macroscopic arrays are IEEE double: rho[n] (N values) and u[a*N + n]
 *    (D x N values).
 *  - Asynchrony: entry points enqueue work on the handle's CUDA stream.
 *    Functions that return data to the host (elbm_diagnostics, elbm_moments
 *    and elbm_alpha_field with host outputs, elbm_get_populations with a host
 *    destination) synchronise that stream; a device fault raised by earlier
 *    asynchronous work is reported by the next synchronising call as
 *    ELBM_ERR_CUDA.
 *  - Boundary conditions: periodic only (the paper's wall condition is cited,
 *    not specified).
 */
#ifndef ELBM_H_
#define ELBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define ELBM_OK 0
#define ELBM_ERR_ARG (-1)         /* invalid argument (lattice, dims, beta, null pointer, size) */
#define ELBM_ERR_UNSUPPORTED (-2) /* valid but not implemented (boundary condition, option)   */
#define ELBM_ERR_CUDA (-3)        /* a CUDA call failed; see elbm_last_error                  */
#define ELBM_ERR_NONPHYSICAL (-4) /* a population is <= 0 or not finite (positivity polytope) */
#define ELBM_ERR_TIMEOUT (-5)     /* a bounded device-side wait expired                       */

/* Lattices (value = Q). */
#define ELBM_D2Q9 9
#define ELBM_D3Q27 27

/* Boundary conditions. */
#define ELBM_BC_PERIODIC 0

/* Storage of the populations.  F64 and F32 store f_i and compute in the same
 * precision.  F32DEV, F16DEV and BF16DEV store the deviation d_i = f_i - c_i
 * from the reference c_i = w_i rho0 rounded to FP32 (exactly k_i R with
 * w_i = k_i 6^-D, k_i a power of two, and R = 6^-D rho0 rounded to FP32), in
 * IEEE single, half or bfloat16, and compute in FP32.  F32DEV collides on the
 * deviations themselves, so every rounding of the step (the relaxation and the
 * store) happens at the scale of d_i instead of w_i, for the same 4 bytes per
 * population as F32.  elbm_get_populations / elbm_set_populations transfer the
 * stored values (d_i for the deviation storages). */
#define ELBM_STORE_F64 0
#define ELBM_STORE_F32 1
#define ELBM_STORE_F16DEV 2
#define ELBM_STORE_BF16DEV 3
#define ELBM_STORE_F32DEV 4

/* Path-length rule.  HIGHER is the paper's alpha_Higher (default); LOWER the
 * more dissipative alpha_Lower (Sec. III A); LBGK the constant alpha = 2;
 * ITERATE1 one Newton step of the mirror-state entropy equation (Eq. deltaH_)
 * started from alpha_Lower, the alpha_Iterate1 of Sec. IV (Table III) -- a
 * comparison variant that evaluates logarithms, off the FP32 fast path.  The
 * cutoff and the positivity clamp apply to every rule but LBGK. */
#define ELBM_ALPHA_HIGHER 0
#define ELBM_ALPHA_LOWER 1
#define ELBM_ALPHA_LBGK 2
#define ELBM_ALPHA_ITERATE1 3

/* Reading of the Omega+ denominators in the b coefficient (Eq.
 * qaud_tight_coeff): DERIVED uses 4 + m alpha_Lower beta x (m = 1, 2, 3), as
 * the lower-bound split of Appendix C gives; PRINTED uses 4 + m alpha_Lower x
 * as typeset. */
#define ELBM_B_DERIVED 0
#define ELBM_B_PRINTED 1

/* Kernel of elbm_step.  DIRECT: one node per thread, neighbours loaded
 * through the L1 cache; any dims.  ROWS: persistent CTAs stage every source
 * row of an x-row in shared memory with bulk asynchronous copies (TMA engine,
 * mbarrier pipeline); needs FP32 or 16-bit storage, nx * element size a
 * multiple of 16 bytes and nx <= 1024 (D2Q9) or 512 (D3Q27).  AUTO (default)
 * takes DIRECT, the faster of the two on GB300.  Both kernels evaluate the same
 * per-node arithmetic; they agree to rounding (the compiler may fuse
 * multiply-adds differently in each). */
#define ELBM_KERNEL_AUTO 0
#define ELBM_KERNEL_DIRECT 1
#define ELBM_KERNEL_ROWS 2

/* Location of a caller buffer. */
#define ELBM_MEM_DEVICE 0
#define ELBM_MEM_HOST 1

/* Per-node flags written by elbm_alpha_field. */
#define ELBM_BRANCH_CUTOFF 0  /* alpha = 2 (|x|max < 1e-3, or x == 0, or LBGK) */
#define ELBM_BRANCH_SOLVED 1  /* alpha from the closed form                   */
#define ELBM_BRANCH_CLAMPED 2 /* alpha reduced by the positivity clamp        */

/* Number of interior bins of the alpha histogram (on [1.9, 2.1)); the
 * histogram array has ELBM_HIST_BINS + 2 entries: [0] counts alpha < 1.9,
 * [ELBM_HIST_BINS + 1] counts alpha >= 2.1. */
#define ELBM_HIST_BINS 256

typedef struct elbm_opts {
    int storage;    /* ELBM_STORE_*, default ELBM_STORE_F32                          */
    int alpha_mode; /* ELBM_ALPHA_*, default ELBM_ALPHA_HIGHER                       */
    int cutoff;     /* 1: alpha = 2 when |x|max < 1e-3 (Appendix D, default); 0: off */
    int b_variant;  /* ELBM_B_*, default ELBM_B_DERIVED                              */
    int device;     /* CUDA device ordinal, default 0                                */
    double rho0;    /* reference density of deviation storage, default 1.0           */
    void *stream;   /* cudaStream_t for all work; NULL = the legacy default stream   */
    int kernel;     /* ELBM_KERNEL_*, default ELBM_KERNEL_AUTO                       */
} elbm_opts;

/* Domain-wide diagnostics of the current state and of the collision that the
 * next step will apply (Eq. hdef, Eq. deltaH3), accumulated in FP64. */
typedef struct elbm_diag {
    double mass;        /* sum over nodes of rho                                      */
    double momentum[3]; /* sum over nodes of rho u (zero beyond D)                        */
    double H;           /* sum over nodes of H[f] = <f, log(f/w) - 1> (streamed state)    */
    double dH_max;      /* max over nodes of H[f*] - H[f] of the next collision           */
    double alpha_min;   /* min / max / mean over nodes of the next collision's alpha      */
    double alpha_max;
    double alpha_mean;
    int64_t n_nodes;
    int64_t n_cutoff;      /* nodes on the alpha = 2 branch                             */
    int64_t n_solved;      /* nodes with the closed-form alpha                          */
    int64_t n_clamped;     /* nodes where the positivity clamp acted                    */
    int64_t n_nonpositive; /* nodes with a population <= 0 or not finite                */
    int64_t n_dH_positive; /* nodes with H[f*] - H[f] > 1e-6 <f, x^2> (an H-theorem
                              violation beyond the rounding of alpha)                   */
    int64_t n_xmax_band[4]; /* nodes by |x|max of the next collision (Eq. xdef) in
                               [0, 1e-3) (the cutoff of Appendix D), [1e-3, 5e-3),
                               [5e-3, 4e-2) and [4e-2, inf) (where the FP32 path
                               takes its short series, long series and per-population
                               forms of the path-length coefficients)                   */
} elbm_diag;

typedef struct elbm elbm_t;

/* Fills *opts with the defaults listed in elbm_opts. */
void elbm_default_opts(elbm_opts *opts);

/* Bytes of ONE population buffer (Q * N * sizeof(storage element)) for the
 * given lattice, dims and storage.  Returns ELBM_ERR_ARG on invalid input. */
int elbm_population_bytes(int lattice, const int64_t dims[3], int storage, size_t *bytes);

/* Creates a handle for a periodic lattice of dims = {nx, ny, nz} nodes (nz = 1
 * for D2Q9) with relaxation parameter beta = dt/(2 tau + dt), 0 < beta < 1
 * (Sec. I).  opts may be NULL (defaults).  No device memory is allocated for
 * the populations until elbm_bind_buffers or the first call that needs them;
 * a small device scratch block for the diagnostics reductions is allocated
 * here.  Errors: ELBM_ERR_ARG (null out, lattice not 9/27, any dim < 1, nz != 1
 * for D2Q9, beta outside (0,1), rho0 <= 0, unknown storage/mode/variant),
 * ELBM_ERR_UNSUPPORTED (bc != ELBM_BC_PERIODIC), ELBM_ERR_CUDA. */
int elbm_create(elbm_t **out, int lattice, const int64_t dims[3], double beta, int bc,
                const elbm_opts *opts);

/* Frees the handle and every buffer the library allocated.  Borrowed buffers
 * are not freed.  Safe on NULL. */
void elbm_destroy(elbm_t *h);

/* Message of the last failed call on h (or of the last failed elbm_create when
 * h is NULL).  The string is owned by the library and valid until the next
 * call on the same handle. */
const char *elbm_last_error(const elbm_t *h);

/* Binds two caller-owned device buffers of at least elbm_population_bytes
 * bytes each, 256-byte aligned (ping-pong pair: each step reads one and writes
 * the other).  The library never frees them; they must outlive the handle or
 * the next bind.  Any buffers the library had allocated are freed.  The
 * contents become the state: call elbm_init_equilibrium or
 * elbm_set_populations before stepping.  Errors: ELBM_ERR_ARG (null, aliasing,
 * too small, misaligned). */
int elbm_bind_buffers(elbm_t *h, void *pop_a, void *pop_b, size_t bytes);

/* Sets the stream used by all later work of h (NULL = legacy default stream). */
int elbm_set_stream(elbm_t *h, void *stream);

/* Initial state f = f^eq(rho, u) at every node (Sec. I equilibrium), computed
 * in FP64 (for FP32 storage in double-length FP32 arithmetic of ~44 bits) and
 * rounded once to the storage type.  rho: N doubles (NULL = uniform rho0); u:
 * D*N doubles, u[a*N + n].  where = ELBM_MEM_DEVICE or ELBM_MEM_HOST (host
 * arrays are copied through a library-owned staging buffer, in node ranges
 * that overlap the copies with the computation; the first host call creates
 * the buffer, a copy stream and its events).  Host inputs synchronise the
 * stream: the caller may reuse its arrays on return.  Resets the step
 * counter.  Errors: ELBM_ERR_ARG (u NULL, bad where), ELBM_ERR_CUDA. */
int elbm_init_equilibrium(elbm_t *h, const double *rho, const double *u, int where);

/* Advances the state by n >= 0 time steps (one fused pull-stream + collide
 * kernel launch per step, ping-pong between the two buffers).  Asynchronous.
 * Errors: ELBM_ERR_ARG (n < 0), ELBM_ERR_UNSUPPORTED (opts.kernel ==
 * ELBM_KERNEL_ROWS where it does not apply), ELBM_ERR_CUDA (launch failure).
 * A bounded device-side wait of the ROWS kernel that expires is reported as
 * ELBM_ERR_TIMEOUT by the next synchronising call. */
int elbm_step(elbm_t *h, int64_t n);

/* rho and u of the current (post-collision) state at every node, from the
 * stored populations: rho and rho u are their exact sums rounded once to FP64
 * (FP64 storage: FP64 sums), u = (rho u) (1/rho).  rho_out: N doubles (may be
 * NULL); u_out: D*N doubles (may be NULL).  Host outputs are copied in node
 * ranges behind the computation and synchronise the stream. */
int elbm_moments(elbm_t *h, double *rho_out, double *u_out, int where);

/* Per-node path length that the NEXT collision will apply (the current state
 * is pull-streamed and alpha evaluated exactly as elbm_step does, in the
 * storage's compute precision; nothing is written back).  alpha_out: N
 * doubles; flags_out: N bytes of ELBM_BRANCH_* (may be NULL).  Both in the
 * same memory space (where).  Host outputs synchronise the stream. */
int elbm_alpha_field(elbm_t *h, double *alpha_out, uint8_t *flags_out, int where);

/* Subgrid (turbulent) viscosity implied by the path length of the next
 * collision at every node, nu_T = theta dt (2 - alpha) / (2 alpha beta) with
 * theta = 1/3, dt = 1 (Sec. VI, Eq. nuT): positive where alpha < 2 adds
 * dissipation, negative where alpha > 2 removes it.  nut_out: N doubles in
 * memory space `where`.  Host output synchronises the stream. */
int elbm_subgrid_viscosity(elbm_t *h, double *nut_out, int where);

/* Domain-wide diagnostics: mass, momentum and H of the current state, and the
 * alpha statistics, per-node entropy change H[f*] - H[f] (Eq. deltaH3, FP64)
 * and branch counts of the next collision.  alpha_hist (host, may be NULL)
 * receives ELBM_HIST_BINS + 2 counts.  Synchronises the stream.  Returns
 * ELBM_ERR_NONPHYSICAL (after filling *out) when any node has a population
 * <= 0 or not finite. */
int elbm_diagnostics(elbm_t *h, elbm_diag *out, int64_t *alpha_hist);

/* n >= 1 steps (as elbm_step) whose first step also takes the diagnostics of
 * elbm_diagnostics: *out and alpha_hist describe the state before the n steps
 * and the collision its first step applies (Eq. hdef, Eq. deltaH3), as
 * elbm_diagnostics called before elbm_step(h, n) would, up to the order of
 * floating-point sums.  On the DIRECT kernel without body force the first
 * step and the diagnostics are one pass over the populations; otherwise the
 * diagnostics pass runs first.  Synchronises the stream.  Errors: as
 * elbm_diagnostics and elbm_step; ELBM_ERR_ARG for n < 1. */
int elbm_step_diag(elbm_t *h, int64_t n, elbm_diag *out, int64_t *alpha_hist);

/* Copies the current population buffer (Q*N storage elements, layout above)
 * to dst / from src.  where selects host or device memory.  Host copies
 * synchronise the stream.  set resets the step counter. */
int elbm_get_populations(elbm_t *h, void *dst, int where);
int elbm_set_populations(elbm_t *h, const void *src, int where);

/* ---------------------------------------------------------------------------
 * Reverse-mode derivatives.  The paper has no adjoint; these are the chain
 * rule through the step, for gradient-based studies (sensitivities of a loss
 * with respect to the initial state).  Gradient arrays are SoA [Q][N] in the
 * compute type of the handle (double for ELBM_STORE_F64, float otherwise),
 * device memory, caller-owned.  All calls enqueue on the handle's stream.
 * ------------------------------------------------------------------------- */

/* One backward step.  f_t: the state BEFORE the step (storage type, Q*N,
 * device); g_next = dL/df^{t+1}; writes g_t = dL/df^t, where
 * f^{t+1} = collide(stream(f^t)).  The collision is differentiated through the
 * equilibrium, x, the sign-split sums, alpha_Lower, h, alpha_Higher and the
 * positivity clamp (the cutoff and clamp branches on the side the forward
 * pass takes; Omega+/- membership held fixed).  g_t must not alias g_next. */
int elbm_adjoint_step(elbm_t *h, const void *f_t, const void *g_next, void *g_t);

/* As elbm_adjoint_step, and also adds to dforce[0..D-1] (DEVICE pointer, FP64,
 * accumulated, not overwritten) the derivative of sum_x <g_next(x), f^{t+1}(x)>
 * with respect to the uniform body force of elbm_set_force, taken at the force
 * currently set (zero included).  Summing over the steps of a reverse sweep
 * gives dL/dF.  The paper defines no force and no adjoint; see elbm_set_force.
 * Errors: ELBM_ERR_ARG (null pointer, g_t == g_next), ELBM_ERR_CUDA. */
int elbm_adjoint_step_force(elbm_t *h, const void *f_t, const void *g_next, void *g_t, double *dforce);

/* Uniform body force F (D host doubles; NULL = none), applied by every later
 * elbm_step after the collision as the exact-difference term
 *   f_i += f^eq_i(rho, u + F/rho) - f^eq_i(rho, u),
 * rho, u the node's moments.  Not from the paper (which has no forcing): it
 * serves gradient studies such as dL/dF.  It keeps the mass and adds exactly F
 * to the momentum of every node per step.  A nonzero force uses the DIRECT
 * kernel.  Errors: ELBM_ERR_ARG (non-finite component), ELBM_ERR_UNSUPPORTED
 * (opts.kernel == ELBM_KERNEL_ROWS). */
int elbm_set_force(elbm_t *h, const double *force);

/* L = 1/2 sum_x rho |u|^2 of the field f (storage type, device; NULL = the
 * current state), accumulated in FP64 into *L (host; synchronises), and, if
 * grad is not NULL, dL/df_i = c_i . u - |u|^2/2 (compute type, device). */
int elbm_kinetic_energy(elbm_t *h, const void *f, double *L, void *grad);

/* Derivatives of the initial state f = f^eq(rho, u) (elbm_init_equilibrium)
 * with respect to rho and u, given g = dL/df (compute type): drho (N doubles,
 * may be NULL) and du (D*N doubles, may be NULL); rho may be NULL (rho0).
 * All arrays in device memory. */
int elbm_equilibrium_vjp(elbm_t *h, const double *rho, const double *u, const void *g, double *drho, double *du);

/* Steps taken since the last init/set. */
int elbm_step_count(const elbm_t *h, int64_t *steps);

/* Waits for all work enqueued on the handle's stream; reports deferred
 * device errors as ELBM_ERR_CUDA and an expired device-side wait as
 * ELBM_ERR_TIMEOUT (the flag is cleared when reported). */
int elbm_synchronize(elbm_t *h);

/* ---------------------------------------------------------------------------
 * Batched ensembles.  The paper has no counterpart (a library service): many
 * independent periodic domains of one lattice, each with its own dims and
 * beta, held in one pair of device buffers and advanced together, so that
 * domains too small to fill the GPU alone share every launch.
 *
 * Each domain's populations are one block in the layout described above
 * (Q*N_d elements, SoA), so the per-domain calls below behave like their
 * single-handle counterparts.  All calls enqueue on the batch's stream
 * (opts->stream, or a stream the batch creates when that is NULL, since CUDA
 * graphs cannot be captured on the legacy default stream); host transfers
 * synchronise it.  Errors as for the single-domain calls; messages in
 * elbm_batch_last_error.
 * ------------------------------------------------------------------------- */
typedef struct elbm_batch elbm_batch_t;

/* How elbm_batch_step issues its n steps.  GRAPH: one launch per step over the
 * work items of every domain, the n launches captured once (per n and buffer
 * parity) into a CUDA graph that is replayed; LAUNCHES: the same launches
 * issued one by one; PER_DOMAIN: one single-domain launch per domain and step
 * (the baseline the batched forms are measured against); PERSISTENT: one
 * cooperative launch advances every domain by n steps (up to 2^20 steps per
 * launch), captured into a CUDA graph like GRAPH.  Its blocks, one per resident
 * slot, own fixed runs of work items and wait only for the other owners of the
 * same domain between steps; those waits are bounded (1 s), and one that
 * expires leaves the steps incomplete and makes the next elbm_batch_synchronize
 * return ELBM_ERR_TIMEOUT.  AUTO: whichever of GRAPH and PERSISTENT
 * elbm_batch_tune_persistent found faster (GRAPH until it has run). */
#define ELBM_BATCH_GRAPH 0
#define ELBM_BATCH_LAUNCHES 1
#define ELBM_BATCH_PER_DOMAIN 2
#define ELBM_BATCH_PERSISTENT 3
#define ELBM_BATCH_AUTO 4

/* ndomains >= 1 domains; dims: 3 values per domain (each in [1, 65535], nz = 1
 * for D2Q9); beta: one value per domain in (0, 1).  opts as for elbm_create
 * (kernel is ignored).  Allocates both population buffers.  A domain of more
 * than 2^32 - 1 populations (Q nx ny nz) is ELBM_ERR_UNSUPPORTED: the batched
 * kernels address each domain with 32-bit offsets (advance such a domain with
 * elbm_create / elbm_step). */
int elbm_batch_create(elbm_batch_t **out, int lattice, int ndomains, const int64_t *dims, const double *beta,
                      const elbm_opts *opts);
void elbm_batch_destroy(elbm_batch_t *b);
const char *elbm_batch_last_error(const elbm_batch_t *b);
/* Number of domains, total nodes and the current work-item width. */
int elbm_batch_info(const elbm_batch_t *b, int *ndomains, int64_t *nodes, int *block_width);
/* Per-domain initial state f = f^eq(rho, u) (rho may be NULL: rho0). */
int elbm_batch_init_equilibrium(elbm_batch_t *b, int domain, const double *rho, const double *u, int where);
/* Advances every domain by n >= 0 steps in the given mode (ELBM_BATCH_*). */
int elbm_batch_step(elbm_batch_t *b, int64_t n, int mode);
/* Times the candidate work-item widths (64, 128, 256 nodes) on the current
 * state -- trial steps read the current buffer and write the other, so the
 * state is unchanged -- and keeps the fastest.  chosen (may be NULL) receives
 * it; ms_per_step (may be NULL) three timings in that order.  Synchronises. */
int elbm_batch_tune(elbm_batch_t *b, int *chosen, double *ms_per_step);
/* Times the PERSISTENT mode at the work-item widths 64, 128 and 256 and the
 * batched launches at the width elbm_batch_tune chose (run first if it has not
 * been), 2 untimed and 50 timed steps each, advancing a copy of the state (the
 * state is restored afterwards); keeps the fastest width for PERSISTENT and sets
 * what ELBM_BATCH_AUTO issues: PERSISTENT if its steps were faster, else GRAPH.  chosen_mode
 * (may be NULL) receives that mode; ms_per_step (may be NULL) the three
 * persistent timings.  Allocates one temporary copy of a population buffer;
 * synchronises. */
int elbm_batch_tune_persistent(elbm_batch_t *b, int *chosen_mode, double *ms_per_step);
int elbm_batch_moments(elbm_batch_t *b, int domain, double *rho_out, double *u_out, int where);
int elbm_batch_diagnostics(elbm_batch_t *b, int domain, elbm_diag *out, int64_t *alpha_hist);
int elbm_batch_get_populations(elbm_batch_t *b, int domain, void *dst, int where);
int elbm_batch_set_populations(elbm_batch_t *b, int domain, const void *src, int where);
int elbm_batch_synchronize(elbm_batch_t *b);
/* Self-test of the PERSISTENT mode's failure detection (no counterpart in the
 * paper).  Runs one two-step persistent launch in which every domain counts one
 * owner more than hold a part of it, so that every wait before the second step
 * expires after the bounded limit (1 s) -- no fault, no hang -- and checks that
 * the launch ended and reported ELBM_ERR_TIMEOUT.  Returns ELBM_OK when it did
 * (the error flag is cleared again); ELBM_ERR_CUDA if the expiry went unreported.
 * The state is unchanged: the first step writes the spare buffer only.
 * Synchronises; takes about a second. */
int elbm_batch_check_wait_timeout(elbm_batch_t *b);

/* ---------------------------------------------------------------------------
 * Allocation-free diagnostics.  The paper has no counterpart: this is a
 * service of the library for callers that cannot allocate device memory (an
 * application whose GPU memory belongs to another allocator or a fixed pool,
 * code that must not grow its footprint after start-up, a monitoring hook
 * inside someone else's time step).  elbm_create allocates, so these callers
 * have no handle; this entry point needs none.
 *
 * Computes exactly what elbm_diagnostics computes, for a caller-owned device
 * buffer `populations` (Q*N elements of opts->storage, the layout above)
 * holding a post-collision state.  lattice, dims, beta and opts mean what they
 * mean for elbm_create (opts may be NULL: the defaults on the current device
 * and the legacy default stream; only storage, alpha_mode, cutoff, b_variant,
 * rho0, device and stream are used; opts->device must be the current device).
 * populations must be device or managed memory of the current device, aligned
 * to its storage element.  *out and alpha_hist (ELBM_HIST_BINS + 2 counts, may
 * be NULL) are host memory.  Synchronises opts->stream.
 *
 * Scratch: the reduction accumulator lives in a file-scope device array of
 * ELBM_NOALLOC_SCRATCH_BYTES bytes, present on every GPU that loads the
 * library until the process exits.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  A call whose scratch would exceed that maximum
 * is rejected with ELBM_ERR_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for the
 * life of the process, so the call is not valid after a cudaDeviceReset of
 * that device.  Every call clears the array before use, but all calls share
 * it: calls that overlap on the GPU (from different streams or host threads)
 * race and must be serialised by the caller.
 *
 * Errors (message in elbm_last_error(NULL)): ELBM_ERR_ARG (null pointer,
 * lattice, dims or their product above 2^31 nodes, beta, options, a buffer
 * that is misaligned or not device memory of the current device, device not
 * current, scratch too small) -- all decided before any work reaches the GPU;
 * ELBM_ERR_CUDA, ELBM_ERR_NONPHYSICAL (after filling *out). */
#define ELBM_NOALLOC_SCRATCH_BYTES 4096
int elbm_diagnostics_noalloc(int lattice, const int64_t dims[3], double beta, const elbm_opts *opts,
                             const void *populations, elbm_diag *out, int64_t *alpha_hist);

#ifdef __cplusplus
}
#endif

#endif /* ELBM_H_ */
