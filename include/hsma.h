/*
 * hsma.h -- C ABI of the GB300 (sm_103a) implementation of the harmonic surface mapping
 * algorithm (HSMA) for electrostatic reaction potentials of a spherical cavity in a
 * linearized Poisson-Boltzmann continuum (Fu & Gan, arXiv:1907.01724).
 *
 * The problem (Sec. 2.1): N point charges q_i at x_i inside the sphere |x| < a with
 * dielectric constant eps1; outside, dielectric eps2 and inverse Debye length kappa.
 * Inside, Phi_1 = Phi_Coul + Phi_RF (Sec. 2.2).  HSMA writes Phi_RF as a Coulomb sum over
 * N trapezoid-modified Kelvin images plus 3M discrete surface images on the auxiliary
 * sphere R_tau = (1+tau) a (Sec. 2.4, eq. phirffinall).  Every step runs in CUDA kernels
 * on one GPU; no call falls back to the CPU.
 *
 * Conventions for every entry point:
 *   - Return value: HSMA_OK (0) or a negative HSMA_E_* code.  No call aborts the process;
 *     hsma_last_error() gives a one-line message for the failing handle.
 *   - "host" pointers are ordinary CPU memory owned by the caller and only read/written
 *     during the call; "device" pointers are CUDA global memory of the handle's device,
 *     owned by the caller, accessed in stream order on the handle's stream.
 *   - Positions are row-major (n, 3) float64 arrays, charges and potentials float64.
 *   - Potentials are in units of coulomb_k * charge / length (coulomb_k = 1/(4 pi)
 *     reproduces the paper's Phi = q / (4 pi eps1 r)).
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef HSMA_H
#define HSMA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HSMA_API __attribute__((visibility("default")))
#else
#define HSMA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HSMA_OK 0
#define HSMA_E_INVALID_ARG (-1)   /* bad parameter, size or pointer */
#define HSMA_E_OUTSIDE (-2)       /* a charge has |x_i| >= a, or a non-finite coordinate */
#define HSMA_E_STATE (-3)         /* call out of order (e.g. potential before sources) */
#define HSMA_E_OOM (-4)           /* device allocation failed or workspace too small */
#define HSMA_E_CUDA (-5)          /* a CUDA runtime call failed */
#define HSMA_E_TIMEOUT (-6)       /* a host-side wait reached its deadline (hsma_server_poll) */
#define HSMA_E_BUSY (-7)          /* server queue full / no admission */
#define HSMA_E_NONFINITE (-8)     /* non-finite potential (e.g. coincident charges) */

/* precision of the pair sums */
#define HSMA_FP32 0   /* FP32 pair sums (hi/lo split coordinates near, compensated partials);
                         moments, coefficients, surface synthesis and reductions in
                         double-float arithmetic (FP32 pairs, ~2^-46 relative); record
                         geometry in FP64 */
#define HSMA_FP64 1   /* FP64 everywhere */

/* which potential hsma_potential returns */
#define HSMA_TOTAL 0      /* Phi_Coul (j != i) + Phi_RF */
#define HSMA_REACTION 1   /* Phi_RF only */
#define HSMA_COULOMB 2    /* Phi_Coul only */

#define HSMA_P_MAX 80     /* largest truncation order p */

/* Numerical parameters (Sec. 2.4 and Sec. 4). */
typedef struct {
  int p;            /* truncation order: n = 0..p (Sec. 2.4 eq. phim); 0 <= p <= HSMA_P_MAX */
  int M;            /* quadrature points per shell, M = 2(F2+1) (Sec. 2.4, Fibonacci rule);
                       ignored when F2 > 0 */
  int F1, F2;       /* successive Fibonacci numbers; F2 = 0 derives F2 = M/2 - 1,
                       F1 = round(F2 (sqrt5 - 1)/2) (gives 987 for 1597) */
  double tau;       /* auxiliary sphere R_tau = (1 + tau) a, tau > 0 (Sec. 2.4) */
  double dy_rel;    /* central-difference step dy = dy_rel * R_tau (Sec. 2.4 eq. approxG;
                       Sec. 4 uses 1e-5) */
  double coulomb_k; /* Coulomb prefactor; 1/(4 pi) = the paper's units */
  int precision;    /* HSMA_FP32 or HSMA_FP64 */
  int device;       /* CUDA device ordinal */
  void* stream;     /* cudaStream_t for all work of the handle; NULL = a non-blocking stream
                       that the handle creates and owns */
} hsma_params;

typedef struct hsma_t hsma_t;

/* Fill *p with defaults: p=20, M=1000, tau=0.1, dy_rel=1e-5, coulomb_k=1/(4pi), FP32,
 * device 0, NULL stream (the CPU-time parameters of Sec. 4.2, P=20, tau=0.1). */
HSMA_API int hsma_default_params(hsma_params* p);

/* Create a handle for one cavity of radius a (Sec. 2.1: eps1 inside, eps2 and kappa
 * outside).  a > 0, eps1 > 0, eps2 > 0, kappa >= 0.  Allocates nothing on the device until
 * sources are built.  *out receives the handle (caller destroys it). */
HSMA_API int hsma_create(double a, double eps1, double eps2, double kappa, const hsma_params* params, hsma_t** out);

/* Destroy a handle and free the device memory it owns (not an attached workspace). */
HSMA_API void hsma_destroy(hsma_t* h);

/* Last error message of a handle (static storage of the handle; never NULL). */
HSMA_API const char* hsma_last_error(const hsma_t* h);

/* Device workspace.  hsma_workspace_size returns in *bytes the device memory the handle
 * needs for n charges; hsma_attach_workspace hands the handle caller-owned device memory
 * (256-byte aligned, at least that size, alive until detached/destroyed) so that it never
 * calls cudaMalloc itself (the Python binding passes memory from PyTorch's allocator).
 * Without an attached workspace the handle allocates (and grows) its own. */
HSMA_API int hsma_workspace_size(hsma_t* h, int64_t n, size_t* bytes);
HSMA_API int hsma_attach_workspace(hsma_t* h, void* device_ptr, size_t bytes);

/* Build the source set of eq. phirffinall for n charges (Sec. 2.4, Algorithm 1 step 4):
 * trapezoid-modified Kelvin images (one per charge), the truncated correction
 * coefficients, and the 3M monopole/dipole surface images on R_tau.  xyz: host (n,3),
 * q: host (n).  n >= 0.  Every |x_i| must be < a with finite coordinates and charges: the
 * first kernel of the pass checks every charge on the device (host and device inputs alike),
 * and the evaluation that runs the pass (hsma_potential, hsma_energy, hsma_field) returns
 * HSMA_E_OUTSIDE.  Pageable host arrays are copied before the call returns (it is then
 * asynchronous with respect to the host); page-locked host arrays (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister) are read in place by the next evaluation, as device arrays
 * are (see hsma_build_sources_device): keep them unchanged until its work has run. */
HSMA_API int hsma_build_sources(hsma_t* h, int64_t n, const double* xyz, const double* q);

/* Same as hsma_build_sources with inputs already resident on the device, read in place: this
 * call copies nothing; the next evaluation on the handle (the call that runs the build pass)
 * reads xyz_dev and q_dev on the handle's stream and keeps its own copy of them.  Until that
 * evaluation's work has run, the arrays must stay allocated and unchanged (stream-ordered
 * writes enqueued after that call are fine). */
HSMA_API int hsma_build_sources_device(hsma_t* h, int64_t n, const double* xyz_dev, const double* q_dev);

/* Potentials at the n charges (Algorithm 1 step 5, by direct tiled summation):
 * what = HSMA_TOTAL, HSMA_REACTION or HSMA_COULOMB.  phi: host array of n doubles (a
 * page-locked one is written by the device itself, without a staging copy).
 * Synchronises the handle's stream; returns HSMA_E_NONFINITE for coincident charges. */
HSMA_API int hsma_potential(hsma_t* h, double* phi, int what);

/* Same, writing n doubles to device memory (stream-ordered; no host synchronisation). */
HSMA_API int hsma_potential_device(hsma_t* h, double* phi_dev, int what);

/* Fields E = -grad phi at the n charges: the gradient, with every source held fixed, of each
 * term of the potential above (real charges other than the charge itself, Kelvin images, the
 * monopole and dipole layers of Sec. 2.4), so that the force on charge i is q_i E_i.
 * what = HSMA_TOTAL, HSMA_REACTION or HSMA_COULOMB.  E: host array of n x 3 doubles (row-major,
 * caller-owned).  The same pass refreshes the potentials and energies, so hsma_potential and
 * hsma_energy then return without another pair sum.  The first call allocates the pass's
 * buffers (32 bytes per pair partial, 72 bytes per charge; HSMA_E_OOM if that fails).
 * Synchronises the handle's stream; HSMA_E_NONFINITE for coincident charges. */
HSMA_API int hsma_field(hsma_t* h, double* E, int what);

/* Same, writing n x 3 doubles to device memory (stream-ordered; no host synchronisation). */
HSMA_API int hsma_field_device(hsma_t* h, double* E_dev, int what);

/* Energies (Sec. 4.1 generalised to N charges): E_total = 1/2 sum_i q_i [Phi_Coul(x_i) +
 * Phi_RF(x_i)], E_reaction = 1/2 sum_i q_i Phi_RF(x_i) (either pointer may be NULL).
 * Host doubles; synchronises the handle's stream. */
HSMA_API int hsma_energy(hsma_t* h, double* e_total, double* e_reaction);

/* Energy change of moving charge k to x_new (host double[3], |x_new| < a):
 * *de = E_total(after) - E_total(before), from the resident state without rebuilding all
 * sources (a Monte Carlo trial move; the paper's method is linear in the charges, Sec. 2.4).
 * The state is unchanged. */
HSMA_API int hsma_delta_energy(hsma_t* h, int64_t k, const double* x_new, double* de);

/* Commit a move (an accepted Monte Carlo step): charge k is now at x_new.  Updates the
 * resident sources incrementally; equivalent to rebuilding with the moved charge. */
HSMA_API int hsma_apply_move(hsma_t* h, int64_t k, const double* x_new);

/* Truncated correction coefficients of the current sources (eq. phim), in the real
 * normalised solid-harmonic basis T_nm (sum_m T_nm(x) T_nm(y) = |x|^n |y|^n P_n(cos angle)):
 * Phi_corr(y) = sum_{n<=p, |m|<=n} out[n^2 + n + m] T_nm(y/a), with m < 0 the sine part.
 * out: host array of len >= (p+1)^2 doubles.  Synchronises the stream. */
HSMA_API int hsma_coefficients(hsma_t* h, double* out, int64_t len);

/* Number of the library's kernel launches issued so far by this handle (for accounting). */
HSMA_API int64_t hsma_kernel_launches(const hsma_t* h);

/* Scheduling of a build followed by a potential/energy evaluation.  hsma_build_sources copies
 * the inputs and defers the source kernels to the first call that needs them.  on = 1 (the
 * default): a potential or energy evaluation right after a build runs the build and the pair
 * sum as one graph (the spatial order and the image records beside the coefficient and surface
 * kernels; a single cavity also runs the real-charge/Kelvin part of the pair sum beside them,
 * see hsma_batch_set_pair_schedule); on = 0: separate passes (the pair kernel then runs alone
 * on the GPU, which is how hsma_last_pair_time times it in isolation).  Results are bitwise
 * the same either way. */
HSMA_API int hsma_set_overlap(hsma_t* h, int on);

/* Device time in milliseconds of the most recent pair-sum kernel launch of the handle (the
 * potential pass's or, after hsma_field, the field pass's; CUDA events recorded on the
 * handle's stream just before and after that launch).  Synchronises
 * the stream.  HSMA_E_STATE if no pair sum has run yet. */
HSMA_API int hsma_last_pair_time(hsma_t* h, float* ms);

/* Far field of the pair sum by a treecode, for large cavities (the paper accelerates the pair
 * sum of eq. phirffinall with the FMM for N up to 1e6, Sec. 4.2).  With theta in (0, 1) the
 * real-charge and Kelvin-image parts of the pair sum of a single FP32 handle run as a GPU
 * treecode over the spatial order of the charges: an octree of the charges (and, node by node,
 * of their Kelvin images), multipole moments of the given order (8, 12 or 16) per node, and per
 * group of 32 charges a traversal that takes a node through its moments when
 * node radius <= theta * (its distance from each charge of the group) and it holds at least
 * (order + 1)^2 / 3 charges, else opens it or sums it directly; Kelvin images farther than 2a
 * from the centre enter through one expansion of order 24 about the centre.  The surface images
 * keep their direct sum.  theta = 0 (the default) restores the direct sum.  Takes effect at the
 * next hsma_build_sources (call this first; it discards the current sources).  With the tree on,
 * hsma_field, hsma_delta_energy and hsma_apply_move return HSMA_E_STATE.  HSMA_E_INVALID_ARG for
 * theta outside [0, 1), another order, or an FP64 handle.  Its error against the direct sum
 * falls with theta and rises with the order; theta = 0.5 with order 12 stays below 5e-7 relative
 * (norm-wise) against the exact sums, uniform or clustered charges. */
HSMA_API int hsma_set_far_field(hsma_t* h, double theta, int order);

/* Device time in milliseconds of the most recent treecode evaluation (the traversal kernel,
 * after the tree's build; CUDA events).  Synchronises the stream; HSMA_E_STATE if none ran. */
HSMA_API int hsma_last_far_time(hsma_t* h, float* ms);

/* Library version string. */
HSMA_API const char* hsma_version(void);

/* ---------------------------------------------------------------------------------------
 * Batched API: many independent cavities (each its own a, eps1, eps2, kappa and charge set;
 * common numerical parameters) evaluated by the same kernels in single launches.  Arrays
 * over systems are indexed s = 0..nsys-1; charges are concatenated in system order (system s
 * owns n[s] consecutive rows).  The work is split over the whole batch (a system's share of
 * items follows its share of the work), so a batched system's results equal those of the same
 * system alone up to the rounding of a different summation split (within the path's
 * tolerance); for a given batch they are deterministic (no dependence on scheduling).
 * --------------------------------------------------------------------------------------- */
typedef struct hsma_batch_t hsma_batch_t;

/* Create a batch of nsys cavities (host arrays of length nsys; the same constraints as
 * hsma_create for each system). */
HSMA_API int hsma_batch_create(int nsys, const double* a, const double* eps1, const double* eps2,
                               const double* kappa, const hsma_params* params, hsma_batch_t** out);
HSMA_API void hsma_batch_destroy(hsma_batch_t* b);
HSMA_API const char* hsma_batch_last_error(const hsma_batch_t* b);

/* Workspace for charge counts n[nsys] (host; the largest over all pair-sum tile
 * configurations, so it also serves hsma_batch_autotune), and attaching caller-owned device
 * memory, as for a single handle. */
HSMA_API int hsma_batch_workspace_size(hsma_batch_t* b, const int64_t* n, size_t* bytes);
HSMA_API int hsma_batch_attach_workspace(hsma_batch_t* b, void* device_ptr, size_t bytes);

/* Reserve room for up to max_requests single-charge moves per call of hsma_batch_delta_energy
 * / hsma_batch_apply_moves (default 1; takes effect at the next build). */
HSMA_API int hsma_batch_set_max_requests(hsma_batch_t* b, int max_requests);

/* Build all sources (Sec. 2.4) for n[nsys] charges per system: xyz (sum n, 3) and q (sum n),
 * host or device memory respectively (device and page-locked host inputs are read in place by
 * the next evaluation, as for hsma_build_sources).  A charge outside its cavity or a non-finite value is
 * reported as HSMA_E_OUTSIDE by the evaluation that runs the pass (see hsma_build_sources). */
HSMA_API int hsma_batch_build_sources(hsma_batch_t* b, const int64_t* n, const double* xyz, const double* q);
HSMA_API int hsma_batch_build_sources_device(hsma_batch_t* b, const int64_t* n, const double* xyz_dev,
                                             const double* q_dev);

/* Potentials of all charges (sum n doubles, concatenated), host or device output (a
 * page-locked host array is written by the device itself, as for hsma_potential). */
HSMA_API int hsma_batch_potential(hsma_batch_t* b, double* phi, int what);
HSMA_API int hsma_batch_potential_device(hsma_batch_t* b, double* phi_dev, int what);

/* Fields of all charges (sum n x 3 doubles, concatenated; see hsma_field), host or device. */
HSMA_API int hsma_batch_field(hsma_batch_t* b, double* E, int what);
HSMA_API int hsma_batch_field_device(hsma_batch_t* b, double* E_dev, int what);

/* Energies of every system: e_total[nsys], e_reaction[nsys] (host; either may be NULL). */
HSMA_API int hsma_batch_energy(hsma_batch_t* b, double* e_total, double* e_reaction);

/* Energy changes of nreq independent trial moves (system sys[r], charge k[r] moved to
 * x_new[3r..3r+2]); de[r] receives E(after) - E(before) of that system alone.  Host arrays.
 * The state is unchanged.  nreq <= the reserved maximum. */
HSMA_API int hsma_batch_delta_energy(hsma_batch_t* b, int nreq, const int* sys, const int64_t* k,
                                     const double* x_new, double* de);

/* Commit nreq moves, at most one per system per call. */
HSMA_API int hsma_batch_apply_moves(hsma_batch_t* b, int nreq, const int* sys, const int64_t* k,
                                    const double* x_new);

HSMA_API int64_t hsma_batch_kernel_launches(const hsma_batch_t* b);
HSMA_API int hsma_batch_last_pair_time(hsma_batch_t* b, float* ms);

/* Build/potential scheduling of the batch (see hsma_set_overlap). */
HSMA_API int hsma_batch_set_overlap(hsma_batch_t* b, int on);

/* Where the graph of a build followed by a potential/energy evaluation (overlap on) runs the
 * pair sum of the real charges and Kelvin images, which needs only the image records:
 * mode = 1 in a launch of its own right after the records, beside the coefficient and surface
 * kernels (at the lowest launch priority, leaving one CTA slot per SM to those kernels);
 * mode = 2 the same, leaving room for one CTA of the largest of those kernels per SM; mode = 0
 * in one launch with the surface images after those kernels; mode = -1 (the default) the
 * autotuned choice for this size class if there is one (hsma_batch_autotune times all three),
 * else 1 for up to 8 cavities and 0 for more.  Results are bitwise the same either way; the
 * choice takes effect at the next build (as hsma_batch_set_pair_config does).
 * HSMA_E_INVALID_ARG for another mode.  hsma_batch_pair_schedule writes the schedule of the
 * current layout (0, 1 or 2) to *mode. */
HSMA_API int hsma_batch_set_pair_schedule(hsma_batch_t* b, int mode);
HSMA_API int hsma_batch_pair_schedule(const hsma_batch_t* b, int* mode);

/* Pair-sum tile configurations: CTA threads x targets per thread, and the number of pair work
 * items per resident CTA slot the layout aims for (any pointer may be NULL).
 * hsma_batch_set_pair_config forces one (-1 = automatic); hsma_batch_autotune times every
 * configuration on the current inputs (reps runs each, CUDA events: the build + potential step
 * in one graph, or with overlap off the potential pass alone; the three fastest again in
 * interleaved rounds; then, with overlap on and no forced schedule, the winner with the three pair
 * schedules of hsma_batch_set_pair_schedule) and keeps the fastest for this size class;
 * *best and *best_ms (nullable) receive the configuration and its time. */
HSMA_API int hsma_pair_config_count(void);
HSMA_API int hsma_pair_config_info(int idx, int* threads, int* targets_per_thread, int* items_per_slot);
HSMA_API int hsma_batch_set_pair_config(hsma_batch_t* b, int cfg);
HSMA_API int hsma_batch_autotune(hsma_batch_t* b, int reps, int* best, float* best_ms);

/* ---------------------------------------------------------------------------------------
 * Serving: Monte Carlo chains (independent cavities) kept on the device, answering
 * single-charge-move energy changes and full energies as requests arrive (the Monte Carlo
 * use of the method, Sec. 1; the paper itself defines no serving loop).  The request loop is
 * native: hsma_server_start runs it on a thread of its own; any thread then submits requests
 * (hsma_server_submit) and takes answers (hsma_server_poll) while it runs; hsma_server_stop
 * ends it.  Continuous batching: a chain has one request in flight at a time and its released
 * requests wait in a FIFO (a chain's results follow its own order); every ready move request
 * of every idle chain joins the next batched Delta-E launch (high-priority stream; accepted
 * moves are committed in the same launch sequence), while full-energy requests run on
 * low-priority streams as bounded chunks of pair work on a grid limited to part of the GPU,
 * so move batches keep running between and beside them.  Admission by device footprint: a
 * request for a chain that is not resident waits until that chain fits the budget once idle
 * resident chains (least recently used first) are evicted; the resident set is then rebuilt
 * from every chain's committed state at a point where no work is in flight.
 * --------------------------------------------------------------------------------------- */
typedef struct hsma_server_t hsma_server_t;

#define HSMA_REQ_DELTA 0   /* energy change of moving charge k of the chain to x; commit if accept */
#define HSMA_REQ_ENERGY 1  /* total energy of the chain's current configuration */

typedef struct {
  double t_arrival;  /* hsma_server_run only: release time in seconds after the start of the run */
  int chain;         /* chain (system) index */
  int kind;          /* HSMA_REQ_DELTA or HSMA_REQ_ENERGY */
  int accept;        /* DELTA: commit the move after computing Delta E (the caller's MC decision) */
  int pad;
  int64_t k;         /* DELTA: charge index */
  double x[3];       /* DELTA: new position, |x| < a */
  int64_t id;        /* caller's tag, copied to the result */
} hsma_request;

typedef struct {
  int64_t id;        /* the request's tag */
  int status;        /* HSMA_OK, HSMA_E_BUSY (chain closed, larger than the budget, or cancelled
                        by hsma_server_stop(s, 0)), HSMA_E_OUTSIDE, HSMA_E_INVALID_ARG, ... */
  int chain;         /* the request's chain */
  double value;      /* Delta E, or E_total */
  double t_arrival;  /* submission time (s; hsma_server_run: the release time, run clock) */
  double t_done;     /* completion seen by the loop (s, same clock) */
  int64_t ticket;    /* the ticket hsma_server_submit returned (counted from 0 at each start) */
} hsma_result;

/* Create a server for nchains cavities (arrays as for hsma_batch_create; common params).
 * hbm_budget_bytes bounds the device memory of the resident chains (0 = no bound);
 * max_batch bounds the move requests per batched launch; energy_slots is the number of
 * full-energy requests that may run at once; energy_sm_frac in (0, 1] is the fraction of the
 * GPU's resident-block slots a full-energy pair kernel may occupy. */
HSMA_API int hsma_server_create(int nchains, const double* a, const double* eps1, const double* eps2,
                                const double* kappa, const hsma_params* params, size_t hbm_budget_bytes,
                                int max_batch, int energy_slots, double energy_sm_frac, hsma_server_t** out);
/* Destroy a server (stops a running loop first, cancelling what has not started). */
HSMA_API void hsma_server_destroy(hsma_server_t* s);
HSMA_API const char* hsma_server_last_error(const hsma_server_t* s);

/* Initial charges of every chain: n[nchains], xyz (sum n, 3), q (sum n), host.  Chains are
 * admitted in index order while their device footprint fits the budget; their sources are
 * built on the device.  *admitted (nullable) receives the number of resident chains.
 * HSMA_E_STATE while the loop runs. */
HSMA_API int hsma_server_load(hsma_server_t* s, const int64_t* n, const double* xyz, const double* q,
                              int* admitted);

/* Close chain c for good (its later requests are answered HSMA_E_BUSY), free its share of the
 * budget and admit waiting chains that now fit, in index order.  HSMA_E_STATE while the loop
 * runs. */
HSMA_API int hsma_server_close_chain(hsma_server_t* s, int c, int* admitted);

/* Start the request loop on a native thread (HSMA_E_STATE if it runs already or nothing is
 * loaded).  From here until hsma_server_stop the loop alone issues the server's device work. */
HSMA_API int hsma_server_start(hsma_server_t* s);

/* Submit one request (thread-safe; any number of producer threads).  It is released at once:
 * its submission time on the server clock becomes its arrival time.  *ticket (nullable)
 * receives its ticket.  HSMA_E_BUSY: 65536 requests are submitted and not yet answered (try
 * again after polling); HSMA_E_STATE: the loop is not running or is stopping; a loop that
 * ended on a CUDA error returns that error.  Invalid requests are accepted here and answered
 * with their error status. */
HSMA_API int hsma_server_submit(hsma_server_t* s, const hsma_request* req, int64_t* ticket);

/* Take up to max_results answers, in completion order, into out (thread-safe); *count receives
 * how many.  timeout_s = 0: return at once; timeout_s > 0: wait up to that long for at least
 * one answer and return HSMA_E_TIMEOUT if none came.  Answers stay available after
 * hsma_server_stop until taken. */
HSMA_API int hsma_server_poll(hsma_server_t* s, hsma_result* out, int max_results, double timeout_s, int* count);

/* Stop the loop and join its thread.  drain = 1: every submitted request is answered first;
 * drain = 0: requests that have not started are answered HSMA_E_BUSY, those in flight
 * complete.  Returns HSMA_OK, or the CUDA error that ended the loop. */
HSMA_API int hsma_server_stop(hsma_server_t* s, int drain);

/* Replay nreq requests (any order of t_arrival) in real time: starts the loop, submits each
 * request from the calling thread at its release time, polls the answers, stops the loop with
 * drain = 1, and returns when all are answered; results[r] answers reqs[r].  HSMA_E_STATE if
 * the loop is already running. */
HSMA_API int hsma_server_run(hsma_server_t* s, int nreq, const hsma_request* reqs, hsma_result* results);

/* Current positions of chain c (n_c x 3 doubles, host) after the committed moves (thread-safe). */
HSMA_API int hsma_server_positions(hsma_server_t* s, int c, double* xyz_out, int64_t n);

/* ---------------------------------------------------------------------------------------
 * Allocation-free Coulomb sum.  The paper has no counterpart: this is a service for callers
 * that may not allocate device memory (code inside allocator or memory-pool callbacks, where
 * an allocation would re-enter the allocator; plugins whose host application owns and
 * accounts for all device memory; real-time loops with a fixed memory budget).  It computes phi[i] = k_over_eps1 * sum_{j != i} q[j] / |x_i - x_j| for n charges
 * with the library's FP32 tiled pair sum (hi/lo split coordinates, compensated partials;
 * the same numbers as hsma_potential(..., HSMA_COULOMB) up to the FP32 tolerance).
 *   xyz_dev (n,3), q_dev (n): device inputs; phi_dev (n): device output; stream: a
 *   cudaStream_t or NULL (legacy default stream); the call is asynchronous on it.
 *   n <= HSMA_NOALLOC_MAX_N, else HSMA_E_INVALID_ARG (nothing is launched).
 * It calls no cudaMalloc/cudaFree or other allocating routine.  Its scratch memory (8 MB of
 * partial sums and counters) is a static device array that every GPU loading the library
 * keeps until the process exits.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress, with the device current): make that first call before any stream
 * capture.  The address is kept for the life of the process and does not survive
 * cudaDeviceReset (do not call this entry point again after a reset).  All calls share the
 * array, which keeps the last call's contents (the call clears its completion counters
 * itself): calls that may overlap on the GPU (different streams without ordering, or several
 * host threads) race and must be serialised by the caller.  A CUDA error left pending by
 * earlier work is returned as HSMA_E_CUDA before anything is launched, and left pending. */
#define HSMA_NOALLOC_MAX_N 32768
HSMA_API int hsma_coulomb_potential_noalloc(int64_t n, const double* xyz_dev, const double* q_dev,
                                            double k_over_eps1, double* phi_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HSMA_H */
