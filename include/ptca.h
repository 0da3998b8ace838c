/*
 * ptca.h -- C ABI of the GB300 traveling-cluster Monte Carlo library (libptca.so).
 *
 * The library runs the hot path of the parallelised traveling cluster
 * approximation (PTCA, Sec. III of Mukherjee, Patel, Bishop, Dagotto,
 * arXiv:1502.07028).  The headline model is the double-exchange spin-fermion
 * model: classical unit spins S_i, electrons with nearest-neighbour hopping
 * -t and a Hund coupling -J_H S_i . sigma.  The Hubbard mean-field model
 * (Eq. 1) and the adiabatic Holstein model (Sec. VII.b) run on the same path
 * (ptca_params.model), on chains, square and cubic lattices.  For an update
 * site i_s the traveling cluster is the window of L_c sites per axis around
 * it (Sec. II.b, Fig. 1); its Hamiltonian is a 2N_c x 2N_c complex Hermitian
 * matrix (two spin species, Sec. IV).  Its eigenvalues eps_k give the cluster
 * free energy
 *     F = -T sum_k ln(1 + exp(-(eps_k - mu)/T))
 * (the periodic cluster is a grand-canonical ensemble, Sec. II.b; the Hubbard
 * and Holstein models add a classical energy), and
 * Metropolis on dF = F_new - F_old accepts or rejects a proposed spin
 * (Sec. II.c steps a-f).  A sweep is a list of stages; the update sites of a
 * stage are processed at once from the configuration at the start of the
 * stage (Sec. III.a), which the schedule guarantees is the same as visiting
 * them one after another.
 *
 * Conventions for every entry point:
 *   - All compute runs in hand-written CUDA kernels on the device that was
 *     current when ptca_init was called.  There is no CPU fallback: without a
 *     usable GPU, ptca_init returns PTCA_ERR_CUDA.
 *   - Buffers are owned by the caller unless stated.  "device pointer" means
 *     memory the GPU can dereference (cudaMalloc / torch CUDA tensors).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous unless stated.
 *   - No exception crosses the ABI.  On failure a call returns a status other
 *     than PTCA_OK and ptca_last_error() describes it (per thread).  Invalid
 *     arguments are rejected before any launch (PTCA_ERR_INVALID).
 *   - Complex matrices are stored as the packed lower triangle, row-major:
 *     element (r, c), c <= r, at index r(r+1)/2 + c, each element an
 *     interleaved (re, im) pair of double (PTCA_FP64) or float (PTCA_MIXED).
 *   - Spins are N x 3 row-major doubles (S_x, S_y, S_z), site
 *     i = (z*Ly + y)*Lx + x.
 */
#ifndef PTCA_H
#define PTCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTCA_VERSION_MAJOR 0
#define PTCA_VERSION_MINOR 1

typedef struct ptca_ctx ptca_ctx; /* opaque; created by ptca_init, freed by ptca_destroy */

typedef enum {
    PTCA_OK = 0,
    PTCA_ERR_INVALID = 1,     /* bad argument or unsupported size, nothing launched  */
    PTCA_ERR_CUDA = 2,        /* a CUDA call failed (no device, launch error, ...)    */
    PTCA_ERR_OOM = 3,         /* device allocation failed                            */
    PTCA_ERR_TIMEOUT = 4,     /* a bounded device-wide wait gave up                  */
    PTCA_ERR_NUMERIC = 5,     /* NaN/Inf met in a free energy or eigenvalue          */
    PTCA_ERR_UNSUPPORTED = 6  /* valid request that this build does not implement    */
} ptca_status;

enum { PTCA_SCHEDULE_TILED = 0, PTCA_SCHEDULE_BLOCK = 1 };
enum { PTCA_FP64 = 0, PTCA_MIXED = 1 };
enum { PTCA_PROPOSAL_SPHERE = 0, PTCA_PROPOSAL_CONE = 1 };
enum { PTCA_MODEL_DOUBLE_EXCHANGE = 0, PTCA_MODEL_HUBBARD_MF = 1, PTCA_MODEL_HOLSTEIN = 2 };
enum { PTCA_PIPELINE_STAGES = 0, PTCA_PIPELINE_PERSISTENT = 1, PTCA_PIPELINE_GRAPH = 2, PTCA_PIPELINE_OVERLAP = 3 };
enum { PTCA_REDUCTION_ROWS = 0, PTCA_REDUCTION_TILED = 1, PTCA_REDUCTION_SHARED = 2 };

/* Square lattice, chain or cubic lattice.  Ly == 1 is a one-dimensional chain
 * (Sec. III.a, Fig. 3); Lz > 1 (with Ly > 1) a cubic lattice of Lx*Ly*Lz
 * sites, index (z*Ly + y)*Lx + x, with L_c^3 traveling clusters and 2^3 blocks
 * (Sec. III.a, IV).  Lz of 0 or 1 means a square lattice or chain. */
typedef struct {
    int32_t Lx, Ly;
    int32_t periodic; /* 1: torus; 0: open edges (windows are clipped at the edges) */
    int32_t Lz;
} ptca_lattice;

/* Problem parameters.  Three models share the lattice, the hopping -t and the
 * two spin species per site:
 *   PTCA_MODEL_DOUBLE_EXCHANGE  on-site -J_H S_i . sigma, classical unit spins S_i
 *                               (proposals: sphere or cone);
 *   PTCA_MODEL_HUBBARD_MF       Eq. 1 with <n_i> = 1: on-site (U/2)(1 - m_i . sigma)
 *                               with classical vectors m_i of any length, and the
 *                               classical energy (U/4)(m_i^2 - 1) of every window
 *                               site in the cluster free energy; proposals
 *                               m_new = m_old + a step uniform in the ball of
 *                               radius m_step.  Spins, S(q) and the records then
 *                               hold the fields m_i;
 *   PTCA_MODEL_HOLSTEIN         the adiabatic Holstein model (Sec. VII.b):
 *                               one classical distortion x_i per site (component
 *                               0 of the site's vector, the others 0), the
 *                               one-body term lambda x_i n_i, and the classical
 *                               energy K/2 x_i^2 - lambda x_i + mu of every window
 *                               site in the cluster free energy; initial x
 *                               uniform in [-1, 1], proposals x + m_step (2u - 1).
 *                               S(q) is then the charge structure factor N(q). */
typedef struct {
    double t;                 /* hopping                                              */
    double J_H;               /* Hund coupling (double exchange)                      */
    double mu;                /* chemical potential                                   */
    double T;                 /* temperature (> 0)                                    */
    int32_t L_c;              /* linear cluster size, 2 <= L_c <= every extent > 1    */
    int32_t cluster_periodic; /* -1: same as the lattice; 1: wrap inside the window   */
                              /* (Sec. II.b); 0: open cluster                         */
    int32_t update_offset;    /* position of the update site inside the window along  */
                              /* each axis; -1: floor(L_c/2) for the tiled schedule,  */
                              /* 0 (corner, Sec. III.a) for the block schedule        */
    int32_t schedule;         /* PTCA_SCHEDULE_TILED or PTCA_SCHEDULE_BLOCK            */
    int32_t stride;           /* tiled schedule: spacing of the update sites in a     */
                              /* stage along each axis; 0: L_c                        */
    int32_t precision;        /* PTCA_FP64 or PTCA_MIXED (FP32 reduction to tridiagonal */
                              /* form, double-float eigenvalue finish, FP64 free      */
                              /* energies and dF)                                     */
    int32_t proposal;         /* PTCA_PROPOSAL_SPHERE or PTCA_PROPOSAL_CONE            */
    int32_t model;            /* PTCA_MODEL_DOUBLE_EXCHANGE, _HUBBARD_MF or _HOLSTEIN   */
    double cone_deg;          /* half-angle of the cone proposal, degrees             */
    uint64_t seed;            /* key of the counter-based generator                   */
    double U;                 /* Hubbard U (PTCA_MODEL_HUBBARD_MF), finite            */
    double m_step;            /* Hubbard: radius of the field proposal ball; Holstein: */
                              /* half-width of the distortion step; > 0               */
    double lam;               /* Holstein electron-lattice coupling lambda, finite    */
    double K;                 /* Holstein elastic constant, finite                    */
} ptca_params;

/* Per-call sweep statistics (host struct filled by ptca_sweep when non-NULL). */
typedef struct {
    int64_t attempts;   /* proposals made (N per sweep)                               */
    int64_t accepted;   /* proposals accepted                                          */
    int64_t eigensolves;/* cluster matrices diagonalised (2 per proposal)              */
    int64_t resolved;   /* PTCA_MIXED: proposals re-solved at FP64-class precision     */
                        /* near the threshold                                          */
    int64_t sweeps;     /* sweeps run so far on this context (RNG sweep counter)       */
    double  seconds;    /* device time of the call, from CUDA events                   */
    int64_t screened;   /* surrogate on: proposals rejected at stage 1 (no cluster     */
                        /* diagonalisation)                                           */
} ptca_sweep_stats;

/* Observables of the current configuration (ptca_observables). */
typedef struct {
    double S_00;        /* S(q) at q = 0, Eq. 2 for one configuration                  */
    double S_pipi;      /* S(q) at q = (pi,pi), or (pi,pi,pi) on a cubic lattice        */
    double F_site;      /* last sweep: mean over solved visits of F of the accepted      */
                        /* state / N_c                                                 */
    double acceptance;  /* last sweep: accepted / attempts                              */
    double filling;     /* last sweep: mean over solved visits of sum_k f(eps_k) / N_c, f the */
                        /* Fermi function, for the accepted state                      */
} ptca_obs;

/* ----------------------------------------------------------------------- */
/* Context lifetime                                                          */
/* ----------------------------------------------------------------------- */

/* Validate the problem, build the stage schedule (Sec. III.a), allocate the
 * device state and draw the initial spins uniformly on the sphere from
 * `seed` (counter-based Philox4x32-10; Holstein: distortions uniform in
 * [-1, 1]).  Rejects with PTCA_ERR_INVALID:
 * L_c out of range, a stride that lets a window of one stage contain another
 * update site of the same stage that precedes it, a block schedule with
 * L_c > floor(L/2)+1 on a torus, a tiled stride that does not divide L on a
 * torus, T <= 0, a matrix order n = 2 N_c above 512 (orders above the
 * shared-memory kernels' -- 224 in PTCA_MIXED, 144 in PTCA_FP64 -- run with
 * the matrix in global memory).
 * Synchronous.  *out receives the context (owned by the library). */
ptca_status ptca_init(const ptca_lattice* lattice, const ptca_params* params, ptca_ctx** out);

/* Free every device buffer of the context.  Synchronous.  NULL is a no-op. */
ptca_status ptca_destroy(ptca_ctx* ctx);

/* Change the temperature (T > 0) or the chemical potential for later calls. */
ptca_status ptca_set_T(ptca_ctx* ctx, double T);
ptca_status ptca_set_mu(ptca_ctx* ctx, double mu);

/* Copy the N x 3 spins out of / into the context.  on_device != 0: dst/src are
 * device pointers and the copy is stream-ordered; on_device == 0: host
 * pointers, and the call synchronises `stream` before returning.
 * ptca_set_spins does not renormalise. */
ptca_status ptca_get_spins(ptca_ctx* ctx, double* dst, int on_device, void* stream);
ptca_status ptca_set_spins(ptca_ctx* ctx, const double* src, int on_device, void* stream);

/* ----------------------------------------------------------------------- */
/* Batched building blocks (each step of Sec. II.c, for many clusters)       */
/* ----------------------------------------------------------------------- */

/* Largest matrix order n (= 2 N_c) of this context and the element stride of
 * the packed-triangle slots that ptca_build_clusters uses (nmax(nmax+1)/2). */
ptca_status ptca_dims(const ptca_ctx* ctx, int32_t* nmax, int64_t* packed_stride);

/* Sec. II.c step b (and d, with new_spins): build the cluster Hamiltonians
 * H_clus of m update sites from the current spins.
 *   sites      device int32[m], lattice sites (0 <= site < N)
 *   new_spins  device double[m*3] replacing the spin of each update site, or NULL
 *   H_out      device buffer of m * packed_stride complex elements in the
 *              context precision; matrix i starts at offsets_out[i]
 *   offsets_out device int64[m]  (= i * packed_stride)
 *   n_out      device int32[m]   matrix order 2 * (window sites)
 * Window, boundary and basis follow the module comment; basis index of window
 * site (wx, wy, wz) and spin s is 2*((wz*ey + wy)*ex + wx) + s. */
ptca_status ptca_build_clusters(ptca_ctx* ctx, const int32_t* sites, int32_t m,
                                const double* new_spins, void* H_out, int64_t* offsets_out,
                                int32_t* n_out, void* stream);

/* Sec. II.c steps b/d: all eigenvalues, ascending, of m packed Hermitian
 * matrices (the exact diagonalisation of each cluster).
 *   H        device, packed lower triangles in the context precision
 *   offsets  device int64[m], element offset of matrix i in H
 *   n        device int32[m], order of matrix i (1 <= n <= nmax)
 *   eig_out  device double[], eigenvalues of matrix i at eig_out + eig_offsets[i]
 *   eig_offsets device int64[m]
 * Every eigenvalue is first bracketed by FP32 multisection with Sturm counts.
 * PTCA_FP64: FP64 Householder reduction to tridiagonal form; the bracket is
 * confirmed by FP64 Sturm counts and refined by safeguarded FP64 Newton.
 * PTCA_MIXED: FP32 reduction; one double-float Newton step on the FP64
 * tridiagonal.  Sizes are checked on the device; a matrix with n outside
 * [1, nmax] gets NaN eigenvalues.  In a large-cluster context (orders above
 * the shared-memory kernels', Sec. VII.a) each matrix is copied into one of
 * the context's global matrix slots and reduced there by a 16-warp CTA; the
 * call is then ordered after the context's earlier work on `stream` (a
 * sweep running on another stream must finish first). */
ptca_status ptca_cluster_eigvals(ptca_ctx* ctx, const void* H, const int64_t* offsets,
                                 const int32_t* n, int32_t m, double* eig_out,
                                 const int64_t* eig_offsets, void* stream);

/* Grand-canonical free energy of each eigenvalue list (the cluster free
 * energy of Sec. II.b, without a model's classical term):
 * F_i = -T sum_k ln(1 + exp(-(eig_k - mu)/T)), FP64, written to F_out[i]
 * (device double[m]).  eig/eig_offsets/n as in ptca_cluster_eigvals. */
ptca_status ptca_free_energy(ptca_ctx* ctx, const double* eig, const int64_t* eig_offsets,
                             const int32_t* n, int32_t m, double mu, double T, double* F_out,
                             void* stream);

/* ----------------------------------------------------------------------- */
/* The hot path: whole sweeps                                                */
/* ----------------------------------------------------------------------- */

/* Run n_sweeps PTCA sweeps (Sec. III.a-b): for every stage, every update site
 * of the stage gathers its window, proposes a spin (Philox, counter =
 * (site, purpose, sweep)), builds H_old and H_new, reduces both to tridiagonal
 * form, computes their eigenvalues and free energies, and accepts iff
 * ln u < -(F_new - F_old)/T; accepted spins become visible to the next stage.
 * Asynchronous when stats_out == NULL; otherwise synchronises `stream` and
 * fills *stats_out.  In PTCA_PIPELINE_OVERLAP a call without statistics
 * leaves its last stage's re-solve running on the context's side stream for
 * the next call to overlap (see ptca_flush); the library's own calls see a
 * complete configuration. */
ptca_status ptca_sweep(ptca_ctx* ctx, int32_t n_sweeps, ptca_sweep_stats* stats_out, void* stream);

/* How ptca_sweep launches the stages of a sweep (the paper's MPI gather and
 * broadcast between blocks, Sec. III.b, become device-wide barriers):
 *   PTCA_PIPELINE_STAGES      one kernel launch per stage;
 *   PTCA_PIPELINE_PERSISTENT  one persistent launch for all stages of all
 *                             requested sweeps: co-resident CTAs take
 *                             (site, old/new) items of a stage from an atomic
 *                             queue, largest window first, and meet at a
 *                             device-wide barrier between stages;
 *   PTCA_PIPELINE_GRAPH       (default; large clusters default to
 *                             PTCA_PIPELINE_STAGES) the persistent launch
 *                             captured once in a CUDA graph per sweep count
 *                             and replayed;
 *   PTCA_PIPELINE_OVERLAP     per-stage launches in which the re-solve of
 *                             the decisions a stage deferred (PTCA_MIXED
 *                             guard) runs on a high-priority stream of the
 *                             context, concurrently with the visits of the
 *                             next stage whose windows hold no site of that
 *                             stage; the visits whose windows do hold one
 *                             run after the re-solve, on that stream.  Three
 *                             rotating spin buffers keep every read on a
 *                             stable configuration.  Falls back to
 *                             PTCA_PIPELINE_STAGES when nothing is deferred
 *                             (PTCA_FP64, margin 0), with the precision
 *                             checker on and with surrogate screening.
 * Every pipeline computes the same chain, bit for bit.  Every barrier wait is
 * bounded by barrier_timeout_s (default 30 s): past it the kernel stops and
 * ptca_sweep (with stats) returns PTCA_ERR_TIMEOUT.  The persistent kernels
 * run the row-chunked reduction, one per matrix: selecting
 * PTCA_PIPELINE_PERSISTENT or PTCA_PIPELINE_GRAPH here resets the launch
 * configuration's reduction and panel_width to 0 (and a default re-solve
 * margin to that reduction's, ptca_set_resolve_margin). */
ptca_status ptca_set_pipeline(ptca_ctx* ctx, int32_t mode, double barrier_timeout_s);

/* Launch configuration of the sweep kernels:
 *   pipeline       PTCA_PIPELINE_STAGES / _PERSISTENT / _GRAPH / _OVERLAP
 *                  (as above);
 *   warps_per_cta  8: one 8-warp CTA per cluster matrix (every precision
 *                  and order); 4: one warp group per matrix, more resident
 *                  matrices per SM (PTCA_MIXED, orders up to 128); 1: one
 *                  warp per matrix (PTCA_MIXED, orders up to 32).  Orders
 *                  above the shared-memory kernels' (large clusters,
 *                  Sec. VII.a): 8 runs PTCA_MIXED stages on a thread-block
 *                  cluster of 2, 4 or 8 CTAs per matrix holding it in
 *                  distributed shared memory (every precision else: one
 *                  16-warp CTA, matrix in global memory); 16 runs the
 *                  16-warp, global-memory kernel;
 *   ctas_per_sm    CTAs per SM of the persistent kernel, 0 = as many as fit
 *                  (large clusters: the persistent pipelines run width 16,
 *                  the matrix in each CTA's global slot);
 *   reduction      organisation of the FP32 Householder pass (Sec. II.c
 *                  step b): PTCA_REDUCTION_ROWS = lanes on columns of the
 *                  packed triangle, rows in batches (every width);
 *                  PTCA_REDUCTION_TILED = register tiles, 4x4
 *                  complex tiles per lane over pairs of block rows, the
 *                  matrix stored as tiles (PTCA_MIXED, 4-warp CTAs, orders
 *                  up to 128, per-stage and overlapped pipelines);
 *                  PTCA_REDUCTION_SHARED = one reduction for both matrices
 *                  of a visit: H_new differs from H_old only in the update
 *                  site's 2x2 on-site block, so a block Householder
 *                  reduction in 2-column panels started below that block
 *                  gives both 2x2 block-tridiagonal forms at once; each is
 *                  then made tridiagonal by a Givens bulge chase and solved
 *                  (PTCA_MIXED, 4-warp CTAs, one per update site, orders up
 *                  to 128; large clusters: 16-warp CTAs striding over the
 *                  update sites, the matrix in a global slot; per-stage and
 *                  overlapped pipelines).  Orders up to 128: opt-in, since
 *                  its FP32 free-energy differences carry about twice the
 *                  row-chunked pass's error, which narrows the re-solve
 *                  guard's safety factor (ptca_autotune does not select it).
 *                  Large clusters: the chases run in double-float, the dF
 *                  error falls about 400-fold below the per-matrix kernel's,
 *                  and it is faster; it is the default of PTCA_MIXED large
 *                  contexts and an autotuner candidate;
 *   panel_width    0 or 1: the unblocked reduction above; 2, 4 or 8: the
 *                  blocked form, panels of that many reflectors with one
 *                  rank-2b update of the trailing block per panel (the
 *                  LAPACK LATRD scheme; PTCA_MIXED, 8-warp CTAs, orders up to
 *                  128, per-stage and overlapped pipelines, reduction 0).
 * Every configuration computes the same chain (decisions and spins; free
 * energies to rounding). */
typedef struct {
    int32_t pipeline;
    int32_t warps_per_cta;
    int32_t ctas_per_sm;
    int32_t reduction;
    int32_t panel_width;
} ptca_launch_config;

/* Apply a launch configuration.  PTCA_ERR_UNSUPPORTED for a width the
 * problem cannot use, PTCA_ERR_INVALID for values out of range. */
ptca_status ptca_set_launch_config(ptca_ctx* ctx, const ptca_launch_config* cfg);
ptca_status ptca_get_launch_config(const ptca_ctx* ctx, ptca_launch_config* out);

/* Autotuner: times every launch configuration the problem admits (CTA width
 * x pipeline x persistent CTAs per SM x reduction x panel width) on this context's own lattice -- one
 * warm-up sweep and trial_sweeps (1..100) timed sweeps each, CUDA events on
 * `stream` -- restoring the spins and the sweep counter before every trial
 * and at the end, so the chain is left where it was (the per-visit record
 * of the last sweep is overwritten).  Applies the fastest configuration,
 * writes it to *best (may be NULL) and, if json is not NULL, a JSON table of
 * every candidate's ms per sweep (NUL-terminated, at most json_cap bytes;
 * PTCA_ERR_INVALID if it does not fit).  Synchronises `stream`.  The
 * precision checker must be off. */
ptca_status ptca_autotune(ptca_ctx* ctx, int32_t trial_sweeps, ptca_launch_config* best, char* json, int32_t json_cap,
                          void* stream);

/* Per-kernel timing of the per-stage pipelines (off by default).  While on,
 * every stage-kernel launch and every re-solve launch of ptca_sweep is
 * bracketed by CUDA events on the stream it runs on.  ptca_kernel_times
 * synchronises `stream` and writes, into a host array of 9 doubles:
 *   out[0], out[1]  total ms and launch count of the stage kernels (whole
 *                   stages; in PTCA_PIPELINE_OVERLAP the visits that do not
 *                   wait for the previous stage's re-solve);
 *   out[2], out[3]  total ms and launch count of the re-solve kernels;
 *   out[4], out[5]  total ms and launch count of the stage kernels of
 *                   PTCA_PIPELINE_OVERLAP that run after a re-solve;
 *   out[6], out[7]  cluster matrices solved by the launches of out[0] and of
 *                   out[4] (two per visit);
 *   out[8]          ms during which at least one launch of out[0] ran (the
 *                   union of their intervals: in PTCA_PIPELINE_OVERLAP a
 *                   stage's independent visits start beside the previous
 *                   stage's, so the launches overlap);
 * then clears the record.  Launches of one pipeline may overlap in time, so
 * the totals can exceed the elapsed time.  The persistent pipelines time as
 * one launch per call of ptca_sweep (ptca_sweep_stats.seconds). */
ptca_status ptca_set_kernel_timing(ptca_ctx* ctx, int32_t on);
ptca_status ptca_kernel_times(ptca_ctx* ctx, double* out, void* stream);

/* PTCA_MIXED decision guard.  The FP32 reduction leaves an error of about
 * 1e-4 in dF at n = 128, so a Metropolis decision whose margin
 * |ln u + dF/T| is below `margin` is deferred: both cluster matrices of that
 * update site are solved again at FP64-class precision (reduction and
 * eigenvalues in double-float arithmetic, about 48 significant bits) and the
 * decision is taken on that dF, before the next stage starts.  With a
 * margin above T^-1 times the largest dF error this makes decisions identical
 * to the FP64 path wherever the FP64 margin exceeds its own error.  Default
 * in PTCA_MIXED: 1e-2; 1e-4 for large clusters on the shared reduction
 * (launch configuration reduction = PTCA_REDUCTION_SHARED, their default),
 * whose dF error is about 5e-7.  The default follows the launch
 * configuration until the caller sets a margin here; 0 disables it.  The
 * count of re-solved updates is ptca_sweep_stats.resolved.  Rejected
 * (PTCA_ERR_INVALID) for PTCA_FP64. */
ptca_status ptca_set_resolve_margin(ptca_ctx* ctx, double margin);

/* Precision checker (PTCA_MIXED only; PTCA_ERR_UNSUPPORTED otherwise).  While
 * on, every stage of ptca_sweep first solves both cluster matrices of each of
 * its visits twice from the stage-start spins -- with the FP32 reduction the
 * sweep uses and fully in FP64 -- and records per stage (per batch of
 * concurrent clusters) the largest eigenvalue error max|eps32 - eps64| and
 * free-energy-difference error max|dF32 - dF64|.  The chain itself is
 * unchanged; sweeps run the per-stage pipeline while the checker is on.
 * Large clusters are checked in the context's global matrix slots (FP32 in
 * the stage kernel's, FP64 in the re-solve's). */
ptca_status ptca_set_checker(ptca_ctx* ctx, int32_t on);

/* Checker results since the last read (or since the checker was first turned
 * on), then reset.  out: host array of n_rows x 5 doubles, n_rows >= the
 * number of stages; row s = stage s: [0] max |d eps|, [1] max |d dF|,
 * [2] max |d eps| / (J_H + 4|t|) (the spectral-norm bound of a cluster
 * matrix), [3] max |d dF| / max(1, |F_old|, |F_new|), [4] max |d dF| / s,
 * s = max(|dF|, sum_k |eps_k - mu| f(eps_k) / n) from the FP64 spectrum of
 * the old cluster (f the Fermi function, n the matrix order): the scale of
 * a free-energy difference, about 1 on the double-exchange headline where
 * |F| is about 100.  Maxima over every
 * sweep since the last read; a NaN anywhere reads as NaN.  Synchronises
 * `stream`. */
ptca_status ptca_checker_read(ptca_ctx* ctx, double* out, int32_t n_rows, void* stream);

/* Per-visit record of the last sweep, in flattened stage order (length N):
 * update site, F_old, F_new, ln u and the decision (1 accepted).  Device
 * pointers; any of them may be NULL.  Stream-ordered. */
/* Completes, stream-ordered on `stream`, what the last ptca_sweep call left
 * running beside the caller's stream: in PTCA_PIPELINE_OVERLAP a call
 * without statistics leaves its last stage's re-solve to the next call, which
 * runs it beside its own first stage (as a multi-sweep call does between its
 * sweeps).  Every other call that reads or changes the configuration, the
 * records, the counters or the launch configuration does this itself; a
 * caller that times sweeps with its own events calls this before the last
 * event.  No-op when nothing is pending. */
ptca_status ptca_flush(ptca_ctx* ctx, void* stream);

ptca_status ptca_sweep_record(ptca_ctx* ctx, int32_t* site, double* F_old, double* F_new,
                              double* lnu, uint8_t* accepted, void* stream);

/* Observables of the current configuration and the last sweep (see
 * ptca_obs).  S(q) follows Eq. 2 for one configuration.  Synchronises
 * `stream` and writes the host struct *out. */
ptca_status ptca_observables(ptca_ctx* ctx, ptca_obs* out, void* stream);

/* ----------------------------------------------------------------------- */
/* Partial stages: a lattice split over several GPUs                         */
/* ----------------------------------------------------------------------- */

/* The paper distributes the independent clusters of a block over processes
 * and, once the block is done, gathers the accepted updates and broadcasts the
 * new configuration before the next block (Sec. III.b, Fig. 4).  With the
 * lattice split into strips, one per GPU, each GPU runs the visits of a stage
 * that lie in its strip (ptca_stage_run) and then receives, from its
 * neighbours, the spins of that stage's visits that lie in the windows of its
 * own visits (ptca_get_sites on the sender, ptca_set_sites on the receiver);
 * the partition and the exchange live in the Python package (strips.py).
 *
 * ptca_stage_run: Sec. II.c steps a-f for the given visits of ONE stage of
 * this context's schedule, all reading the configuration at the call's start
 * and writing their decisions together, as a stage of ptca_sweep does, with
 * the random stream of sweep `sweep_index` (the PTCA_MIXED re-solve guard
 * included).  sites: HOST int32[count], update sites of a single stage,
 * without repeats (checked: PTCA_ERR_INVALID otherwise); any subset of the
 * stage, in any order.  The sweep record (ptca_sweep_record) then holds these
 * visits, entries 0 .. count-1 in the order given.  The context's sweep
 * counter is not advanced.  PTCA_ERR_UNSUPPORTED while surrogate screening is
 * on.  Stream-ordered (the site list is staged before the call returns). */
ptca_status ptca_stage_run(ptca_ctx* ctx, int64_t sweep_index, const int32_t* sites, int32_t count, void* stream);

/* Spins of `count` sites (HOST int32 list, indices in [0, N), no repeats) out
 * of / into the context: out/spins hold 3 doubles per listed site, in list
 * order, on the device if on_device != 0 (stream-ordered) else on the host
 * (ptca_get_sites then synchronises `stream`). */
ptca_status ptca_get_sites(ptca_ctx* ctx, const int32_t* sites, int32_t count, double* out, int32_t on_device,
                           void* stream);
ptca_status ptca_set_sites(ptca_ctx* ctx, const int32_t* sites, int32_t count, const double* spins, int32_t on_device,
                           void* stream);

/* ----------------------------------------------------------------------- */
/* Surrogate network and delayed acceptance                                  */
/* ----------------------------------------------------------------------- */
/* A multilayer perceptron h: 150 -> 256 -> 256 -> 256 -> 1 (SiLU), reading the
 * 7x7 patch of the cluster window around the update site (as centred as the
 * window allows; 147 values, the update site's entry holding a spin s) and a
 * second spin.  Its estimate of the proposal's free-energy change is
 *     dF~ = scale * ( h([P(s_old), s_new]) - h([P(s_new), s_old]) ),
 * antisymmetric in the two states.  Matrix products run on the tensor cores
 * with bfloat16 operands and FP32 accumulation (this library's mma.sync
 * kernels); parameters,
 * AdamW moments and the rest are FP32.  With the surrogate enabled,
 * ptca_sweep uses delayed acceptance (Christen and Fox 2005): stage 1 passes
 * a proposal with probability min(1, exp(-dF~/T)); only passing proposals get
 * the exact cluster solves, and stage 2 accepts with probability
 * min(1, exp(-(dF - dF~)/T)).  Detailed balance with respect to the exact
 * cluster free energy holds for any network; the network only changes how
 * many exact solves are spent.  Screening runs with the per-stage pipeline.
 * The paper has no surrogate; its exact TCA step has the final say here.  */

/* Number of FP32 parameters (layout W1[256x160] b1 W2[256x256] b2 W3 b3
 * W4[8x256] b4[8]; W1 columns 150..159 and W4/b4 rows 1..7 are padding). */
int32_t ptca_surrogate_param_count(void);
/* Allocate the network (once) and draw fresh parameters from `seed`. */
ptca_status ptca_surrogate_init(ptca_ctx* ctx, uint64_t seed, void* stream);
/* Copy parameters out/in (device or host pointers; synchronous). */
ptca_status ptca_surrogate_get_params(ptca_ctx* ctx, float* theta, float* scale, void* stream);
ptca_status ptca_surrogate_set_params(ptca_ctx* ctx, const float* theta, float scale, void* stream);
/* Run n_sweeps exact sweeps (no screening) and record, per visit in
 * flattened stage order, the 150 inputs [P(s_old), s_new] (feat, device
 * float[n_sweeps*N*150]), the patch index of the update site (center,
 * int32[n_sweeps*N]) and the exact dF (dF, float[n_sweeps*N]). */
ptca_status ptca_surrogate_collect(ptca_ctx* ctx, int32_t n_sweeps, float* feat, int32_t* center, float* dF,
                                   void* stream);
/* `steps` AdamW steps (betas 0.9/0.999, eps 1e-8, decoupled weight decay) on
 * mini-batches of `batch` samples drawn from n collected samples with the
 * counter generator (seed), minimising mean((dF~ - dF)^2)/scale^2; scale is
 * the standard deviation of dF, fixed at the first step.  loss_trace: device
 * float[steps] or NULL.  Stream-ordered. */
ptca_status ptca_surrogate_train(ptca_ctx* ctx, const float* feat, const int32_t* center, const float* dF, int64_t n,
                                 int32_t steps, int32_t batch, float lr, float weight_decay, uint64_t seed,
                                 float* loss_trace, void* stream);
/* Loss and its gradient (float[param_count]) over the n samples given, with
 * no update (gradient checks).  Synchronous. */
ptca_status ptca_surrogate_grad(ptca_ctx* ctx, const float* feat, const int32_t* center, const float* dF, int32_t n,
                                float* grad_out, float* loss_out, void* stream);
/* dF~ for n samples (device float[n]).  Stream-ordered. */
ptca_status ptca_surrogate_predict(ptca_ctx* ctx, const float* feat, const int32_t* center, int32_t n, float* dF_out,
                                   void* stream);
/* Turn delayed-acceptance screening in ptca_sweep on (1) or off (0). */
ptca_status ptca_surrogate_enable(ptca_ctx* ctx, int32_t on);

/* ----------------------------------------------------------------------- */
/* Sweep without device allocation                                           */
/* ----------------------------------------------------------------------- */

/* One sweep as ptca_sweep runs it in the per-stage pipeline (same stage and
 * re-solve kernels, same decisions and spins), for callers that cannot
 * allocate device memory: hosts whose own pool owns the device memory or
 * that forbid loaded libraries to allocate, and loops that cannot afford
 * cudaMalloc/cudaFree (cudaFree synchronises the device).  The paper has no
 * counterpart; this is a property of the library.
 *   spins        device double[N*3]: the configuration, updated in place
 *   sweep_index  counter of the random stream (the sweep number, >= 0)
 *   F_out        device double[2N] or NULL: F_old of every visit, then F_new
 *   accepted_out device uint8[N] or NULL: decisions, in the flattened stage
 *                order of ptca_schedule for the same lattice and params
 *   status_out   device int32[1] or NULL: receives, stream-ordered after the
 *                sweep, 0 or the ptca_status of a device-side failure
 *                (PTCA_ERR_NUMERIC: a free-energy difference was not finite)
 * The schedule is built and checked on the host, as ptca_init does, and
 * copied into the library's array.  In PTCA_MIXED the decisions within 1e-2
 * of the Metropolis threshold are re-solved at FP64-class precision, as
 * ptca_sweep's default margin does; that re-solve keeps its matrix in shared
 * memory, so PTCA_MIXED is limited to the orders where that fits (128 on a
 * GB300; PTCA_ERR_UNSUPPORTED above).
 * No context and no device allocation: working memory is one array of about
 * 2.2 MB that the library defines in device global memory and that every GPU
 * loading the library holds until the process exits.  Limit: N <= 16384
 * sites (larger lattices return PTCA_ERR_INVALID).  All calls share that
 * array and its contents persist between calls; calls that overlap on the GPU
 * (other streams or threads on the same device) race and must be serialised.
 * The first call on a device looks up the array's address with that device
 * current; make it before any stream capture.  Stream-ordered, asynchronous
 * (the host-to-device copy of the schedule is staged before it returns). */
ptca_status ptca_sweep_noalloc(const ptca_lattice* lattice, const ptca_params* params, double* spins,
                               int64_t sweep_index, double* F_out, uint8_t* accepted_out, int32_t* status_out,
                               void* stream);

/* ----------------------------------------------------------------------- */
/* Full-system spectrum                                                      */
/* ----------------------------------------------------------------------- */

/* All 2N eigenvalues, ascending, of the one-body Hamiltonian of the whole
 * lattice in the current configuration (the context's model: hopping and
 * on-site terms; the classical energy is not part of it).  The paper
 * diagonalises saved configurations of the whole system with ScaLAPACK
 * (Sec. VI); here the dense 2N x 2N matrix is built on the device, reduced to
 * real tridiagonal form by this library's Householder reduction spread over
 * the whole GPU (one pass over the trailing triangle per reflector: FP64 for
 * a PTCA_FP64 context; double-float, about 48 significant bits on the FP32
 * pipe, for a PTCA_MIXED context, with the per-reflector scalars in FP64),
 * and its eigenvalues found one thread each (FP32 bisection finished by
 * double-float Sturm counts and Newton).  No library eigensolver is used.
 *   eig_out  device double[2N]
 * N <= 16384 sites (PTCA_ERR_INVALID otherwise).  Allocates about
 * 8 (2N)^2 bytes of device memory for the call (the packed triangle; plus
 * 32 (2N)^2 / 64 bytes of partial sums), PTCA_ERR_OOM when it does not fit.
 * Synchronises `stream`. */
ptca_status ptca_full_spectrum(ptca_ctx* ctx, double* eig_out, void* stream);

/* ----------------------------------------------------------------------- */
/* Host-only helpers (no GPU needed)                                         */
/* ----------------------------------------------------------------------- */

/* The stage schedule ptca_init would use (Sec. III.a), without a GPU.
 * stage_start: host int32[N+1], sites: host int32[N]; *n_stages receives the
 * number of stages; stage s holds sites[stage_start[s] .. stage_start[s+1]).
 * Same validation as ptca_init. */
ptca_status ptca_schedule(const ptca_lattice* lattice, const ptca_params* params,
                          int32_t* stage_start, int32_t* sites, int32_t* n_stages);

/* Dependence of each stage on the one before it (the last stage of a sweep
 * precedes stage 0 of the next), as PTCA_PIPELINE_OVERLAP uses it.  A visit of
 * stage s depends on stage s-1 iff its window (Sec. II.b, as ptca_init builds
 * it) holds a site of stage s-1; the others read only sites that were final
 * before stage s-1 began.  order: host int32[N]; order[stage_start[s] + k] for
 * k < stage_start[s+1] - stage_start[s] lists the indices into stage s's site
 * list: first the n_indep[s] visits that do not depend on stage s-1, then the
 * rest, each part largest window first and otherwise in schedule order.
 * n_indep: host int32[n_stages].  stage_start, n_stages as ptca_schedule.
 * Same validation as ptca_init; no GPU. */
ptca_status ptca_stage_split(const ptca_lattice* lattice, const ptca_params* params, int32_t* order,
                             int32_t* n_indep);

/* Self-test of the bounded device-wide barrier: `blocks` CTAs wait at a
 * barrier sized for blocks + 1 participants, so the wait can only end by its
 * time limit.  Returns PTCA_ERR_TIMEOUT when every wait gave up and reported
 * it (the expected outcome), PTCA_OK if the barrier completed, PTCA_ERR_CUDA
 * on a CUDA error.  The GPU stays usable.  Synchronous; allocates 16 bytes. */
ptca_status ptca_selftest_barrier_timeout(int32_t blocks, double timeout_s, void* stream);

/* Description of the last failure on this thread (never NULL). */
const char* ptca_last_error(void);

/* Library version as major*100 + minor. */
int32_t ptca_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTCA_H */
