/*
 * gcmc.h -- C ABI of the GB300 grand canonical Monte Carlo (GCMC) hot path
 * for Lennard-Jones fluids with cell lists, after "An Efficient Cell List
 * Implementation for Monte Carlo Simulation on GPUs" (Schwiebert et al.,
 * arXiv 1408.3764).
 *
 * Conventions shared by every call
 * --------------------------------
 * - One context = one simulation box on one GPU.  All work of a call is
 *   issued on the CUDA stream given to gcmc_create (NULL = legacy default
 *   stream); calls that return host results synchronise that stream.
 * - Pointers marked "device" must point to memory of the context's device;
 *   "host" pointers to ordinary host memory.  The library never keeps a
 *   caller pointer beyond the call and never frees caller memory.  All
 *   internal buffers belong to the context and are freed by gcmc_destroy.
 * - Errors come back as gcmc_status codes; no C++ exception crosses the ABI.
 *   gcmc_last_error(ctx) gives a one-line description of the last failure.
 *   Errors detected on the device (cell overflow, capacity, non-finite
 *   energy) are read back by the call that launched the work.
 * - Positions.  The box is cubic with edge L and periodic.  A coordinate x
 *   is stored on a grid of 2^32 points per edge: X = floor(x * (2^32/L))
 *   mod 2^32 evaluated in IEEE double exactly in that order; the stored
 *   position is X * L / 2^32.  Minimum-image separations are exact integer
 *   differences, the cutoff test r^2 < rc^2 is decided exactly on the
 *   integer squared grid distance (threshold ceil((rc * 2^32/L)^2), IEEE
 *   double in that order).
 * - Cells (Sec. 3.2.2 of the paper): T = floor(L/rc) cells per side, T = 3
 *   when L < 3 rc; S = L/T.  The cell of grid coordinate X is
 *   floor(X * T / 2^32); cell id = (cz * T + cy) * T + cx.
 * - Particles.  Species s owns the dense indices 0 .. N_s-1.  A particle is
 *   named by the 64-bit id (s << 32) | i.  At gcmc_build_cells the index of a
 *   particle within its species is its rank among the input particles of
 *   that species ("species-major order" below lists species 0's particles
 *   by index, then species 1's, ...).
 */
#ifndef GCMC_H
#define GCMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCMC_MAX_SPECIES 8

typedef enum {
    GCMC_OK = 0,
    GCMC_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
    GCMC_ERR_CELL_OVERFLOW = 2, /* a cell would exceed its capacity (Sec. 3.2.2) */
    GCMC_ERR_CAPACITY = 3,      /* a species would exceed max_particles */
    GCMC_ERR_NONFINITE = 4,     /* the running energy is not finite */
    GCMC_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    GCMC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    GCMC_ERR_STATE = 7          /* the call needs cells that were never built */
} gcmc_status;

typedef enum {
    GCMC_FP64 = 0, /* pair terms and sums in FP64 */
    GCMC_FP32 = 1  /* pair terms in FP32, sums and the Metropolis test in FP64 */
} gcmc_precision;

/* Box, cutoff and force field (Eq. 1 with per-species-pair eps and sigma). */
typedef struct {
    double L;              /* box edge, > 0 */
    double rc;             /* cutoff radius, 0 < rc <= L/2 */
    int32_t n_species;     /* 1 .. GCMC_MAX_SPECIES */
    int32_t precision;     /* gcmc_precision */
    const double *eps;     /* host, n_species x n_species row-major, symmetric, >= 0 */
    const double *sigma;   /* host, n_species x n_species row-major, symmetric, > 0 */
    int64_t max_particles; /* per-species index capacity; 0 = 2 * N at first build (>= 1024) */
    int32_t cell_capacity; /* particles per cell slot array; 0 = automatic (Sec. 3.2.2) */
    int32_t reserved;      /* must be 0 */
} gcmc_params;

/* Move mix and thermodynamic state of a GCMC run (Sec. 2, Algorithm 1). */
typedef struct {
    double p_disp, p_ins, p_del;       /* move probabilities, >= 0, summing to 1 */
    double max_disp;                   /* displacement half-width delta, 0 <= delta < L/2 */
    double beta;                       /* 1 / kT */
    double log_z[GCMC_MAX_SPECIES];    /* ln z_s = beta mu_s - 3 ln Lambda_s */
    int32_t flags;                     /* GCMC_MIX_* bits; 0: energy only */
    int32_t reserved;                  /* must be 0 */
} gcmc_move_mix;

/* Also keep the running virial W = sum_{i<j} r U'(r) over the pairs within
 * rc (the pair sum of the virial pressure P = rho k T - W / (3V), updated
 * on each accepted move, Sec. 3.1.2, and averaged on the GPU, Sec. 3.3.4):
 * each accepted trial adds its dW, the same 27-cell sum with
 * r U'(r) in place of U.  Reported in gcmc_move_stats.virial/sum_virial.
 * The first run with the flag after a build, a restore or a run without it
 * starts from the full 27-cell sum (the running energy is left as it is);
 * later runs with it continue the running value.  The flag changes no
 * decision: the moves are those of a run without it (dU to rounding). */
#define GCMC_MIX_VIRIAL 1

/* Counters of one gcmc_run_moves call (averages over the moves of the call). */
typedef struct {
    int64_t attempted[3];  /* displacement, insertion, deletion */
    int64_t accepted[3];
    int64_t flagged;       /* trials within tolerance of the acceptance threshold */
    int64_t moves_done;    /* moves completed (less than asked only on error) */
    double energy;         /* running total energy after the last move */
    double sum_energy;     /* sum over the moves of the running energy after the move */
    double sum_n;          /* sum over the moves of N after the move */
    int64_t n[GCMC_MAX_SPECIES]; /* particles per species after the last move */
    double virial;         /* running virial after the last move (GCMC_MIX_VIRIAL; else NaN) */
    double sum_virial;     /* sum over the moves of the running virial after the move */
    double chain_ms;       /* device time of the chain's CTA, start to finish, summed over the
                            * call's launches (global timer; 0 for the microcell chain) */
} gcmc_move_stats;

/* One record per move of gcmc_run_moves (32 bytes). */
typedef struct {
    double dU;        /* energy change of the trial (the value added on acceptance) */
    double lnA;       /* log acceptance ratio; -inf when the move is impossible */
    double uabs;      /* sum over the evaluated pairs of |4 eps s^12| + |4 eps s^6| */
    int32_t index;    /* particle index within its species; -1 when none */
    uint8_t type;     /* 0 displacement, 1 insertion, 2 deletion */
    uint8_t species;
    uint8_t accepted;
    uint8_t flagged;  /* bit 0: near the threshold; bit 1: decided in FP64 */
} gcmc_trace;

/* Geometry derived from the parameters. */
typedef struct {
    int64_t T;             /* cells per side */
    int64_t n_cells;       /* T^3 */
    int64_t cell_capacity; /* slot array length per cell */
    int64_t max_particles; /* per species */
    uint64_t cutoff_grid2; /* squared-grid-distance cutoff */
    double h;              /* grid spacing L / 2^32 */
} gcmc_geometry;

typedef struct gcmc_ctx gcmc_ctx;

/* Creates a context for one box.  Copies the eps/sigma tables (Eq. 1) and
 * derives the cell grid of Sec. 3.2.2.  stream: a cudaStream_t or NULL.
 * Allocates only a few words of device memory (status, running energy,
 * counts) until gcmc_build_cells.
 * Errors: INVALID_ARG (L, rc, species, tables, precision), CUDA. */
gcmc_status gcmc_create(const gcmc_params *params, void *stream, gcmc_ctx **out);

/* Frees the context and all its device buffers (after its stream drains).
 * NULL is accepted.  Errors: none (always OK). */
gcmc_status gcmc_destroy(gcmc_ctx *ctx);

/* Bins n particles into the cell list (Sec. 3.2.1, "Building the Initial
 * Cell List"): quantises pos, computes each particle's cell, and builds the
 * cell list with an integer counting sort that keeps input order within a
 * cell.  pos: device, n x 3 FP64 row-major; species: device, n int32 in
 * [0, n_species).  Replaces any previous configuration and invalidates the
 * running energy.  Errors: INVALID_ARG (n < 0, bad species, non-finite
 * coordinate), CAPACITY, CELL_OVERFLOW (explicit cell_capacity too small),
 * CUDA. */
gcmc_status gcmc_build_cells(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n);

/* The current configuration as input for gcmc_build_cells: pos (device,
 * N x 3 FP64) receives each particle's coordinates (the centre of its grid
 * point, which quantises back to the same point) and species (device, N
 * int32) its species, in species-major order (species 0 by index, then
 * species 1, ...), so that building from them reproduces the configuration
 * with the same particle ids.  n (host, may be NULL) receives N.  Launches
 * one kernel on the context's stream; nothing waits.
 * Errors: STATE (no cells), INVALID_ARG (NULL arrays while N > 0), CUDA. */
gcmc_status gcmc_export_positions(gcmc_ctx *ctx, double *pos, int32_t *species, int64_t *n);

/* The compact cell list of the last gcmc_build_cells: cell_start and
 * cell_count (device, n_cells int32 each) and order (device, n int32: input
 * indices sorted by cell, input order within a cell).  Any pointer may be
 * NULL.  Valid only before the first gcmc_run_moves after the build.
 * Errors: STATE, CUDA. */
gcmc_status gcmc_cell_list(gcmc_ctx *ctx, int32_t *cell_start, int32_t *cell_count,
                           int32_t *order);

/* Trial energies (Algorithms 6 and 7; Eq. 1 over the 27 cells around each
 * point): out[k] = sum over particles j != exclude[k] in the 27 cells of the
 * cell of pos[k] of U_{species[k], s_j}(r) for r < rc.
 * pos: device m x 3 FP64 (quantised as above); species: device m int32;
 * exclude: device m int64 particle ids, -1 = none, or NULL for none;
 * out: device m FP64; out_abs: device m FP64 (the uabs of gcmc_trace) or NULL.
 * Errors: STATE, INVALID_ARG, CUDA. */
gcmc_status gcmc_trial_energy(gcmc_ctx *ctx, const double *pos, const int32_t *species,
                              const int64_t *exclude, int64_t m, double *out, double *out_abs);

/* Runs moves first_move .. first_move + n_moves - 1 of the Markov chain
 * (Sec. 2 and Algorithm 1, with the acceptance rules of Eqs. 3-5 read with
 * the textbook sign of mu) entirely on the device: no host round trip per
 * move.  Move m draws two Philox4x32-10 blocks with counter
 * (m mod 2^32, m / 2^32, chain, 0|1) and key (seed mod 2^32, seed / 2^32),
 * chain = 0 for a single box.  Accepted moves update the cell list in place
 * (Sec. 3.2.5): swap-with-last removal, append, and a deleted index refilled
 * by the last index of its species.  The running energy starts from
 * gcmc_total_energy (computed here when not yet known) and grows by dU.
 * In FP32 mode a trial within 1e-5 * beta * uabs of the threshold is
 * re-evaluated in FP64 and decided on that value (trace flag bit 1).
 * stats: host, may be NULL; trace: device n_moves records, may be NULL.
 * Errors: STATE, INVALID_ARG (mix), CELL_OVERFLOW, CAPACITY (the chain stops
 * before the offending move: stats->moves_done tells where), NONFINITE, CUDA. */
gcmc_status gcmc_run_moves(gcmc_ctx *ctx, uint64_t seed, uint64_t first_move, int64_t n_moves,
                           const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace);

/* Checks the configuration on the host (a consistency checker, in place of
 * a device sanitizer): every particle of every species is listed exactly
 * once, in the cell of its grid position, with an entry equal to its
 * record; cell counts are within capacity and sum to N; the same for the
 * microcells when they are up to date.  Copies the state to the host;
 * synchronises the stream.  Errors: STATE (with the first violation in
 * gcmc_last_error), CUDA. */
gcmc_status gcmc_check_state(gcmc_ctx *ctx);

/* Diagnostic hook for the failure path: ns = the limit, in ns of the GPU's
 * global timer, of every wait inside the chain kernel (0: the default,
 * 1 s); stall_move >= 0: in later gcmc_run_moves calls the committer, about
 * to commit move stall_move of the call, waits on a flag that nothing sets
 * (-1: no stall).  A wait that runs out stops the chain before its next
 * move: every committed move is applied and booked, the kernel returns and
 * gcmc_run_moves returns TIMEOUT with moves_done = the moves committed; the
 * context stays usable.  Errors: INVALID_ARG. */
gcmc_status gcmc_set_wait_limit(gcmc_ctx *ctx, uint64_t ns, int64_t stall_move);

/* Microcell list (Sec. 3.3): the box cut into M^3 microcells of edge about
 * one sigma, each holding at most `capacity` particles in a slot array
 * stored slot-major (slot k of every cell contiguous, Sec. 3.3.1).
 * M = ceil(L / edge) cells per side of equal edge L / M (the paper's unit
 * cells with a thinner last one have the same count); the microcell of grid
 * coordinate X is floor(X * M / 2^32).  Builds the microcells of the
 * current particles, listed species by species, index by index.
 * capacity: 1 .. 15, or 0 = automatic (5, raised to the fullest cell's
 * count and grown by gcmc_run_moves_micro when a move needs a fuller cell).
 * Valid until a build, a restore or a gcmc_run_moves / batch run (which
 * keep only the 27-cell lists); gcmc_run_moves_micro rebuilds them then.
 * Errors: STATE (no cells), INVALID_ARG (edge, capacity, too many
 * microcells for the chain's on-chip counters), CELL_OVERFLOW (a cell holds
 * more than capacity, or more than 15), CUDA. */
gcmc_status gcmc_build_microcells(gcmc_ctx *ctx, double edge, int32_t capacity);

/* The microcells: per_side = M, capacity = slots per cell (host, or NULL);
 * counts: host, M^3 bytes, or NULL; slots: host, capacity * M^3 records of
 * four uint32 (X, Y, Z, tag), slot-major, or NULL (slots at or past a cell's
 * count hold stale data).  Errors: STATE (none up to date), CUDA. */
gcmc_status gcmc_microcells(gcmc_ctx *ctx, int64_t *per_side, int32_t *capacity, uint8_t *counts,
                            uint32_t *slots);

/* The chain of gcmc_run_moves evaluated over the microcell list (Sec. 3.3.3
 * and 3.3.4): one CTA runs the moves one after another; each trial's energy
 * is the sum over the (2D+1)^3 microcells around the old and the new
 * position, D = 1 + floor((rcg - 1) M / 2^32) with rcg the smallest integer
 * with rcg^2 >= the grid cutoff (every cell at most D cells away along each
 * axis; all M when 2D+1 > M).  Same moves, decisions, trace and statistics
 * as gcmc_run_moves (the flag GCMC_MIX_VIRIAL is not accepted); accepted
 * moves update the microcells (append; removal by swap-with-last) and the
 * 27-cell lists exactly as gcmc_run_moves does, so every other call stays
 * valid.  Rebuilds stale microcells first with the last edge and capacity.
 * Errors: as gcmc_run_moves; STATE when gcmc_build_microcells was never
 * called; CELL_OVERFLOW when a microcell of fixed capacity is full. */
gcmc_status gcmc_run_moves_micro(gcmc_ctx *ctx, uint64_t seed, uint64_t first_move, int64_t n_moves,
                                 const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace);

/* Full-system cell-list energy E = 1/2 sum_i sum_{j != i in the 27 cells}
 * U(r_ij), r < rc (Sec. 3.1.1 computes the same sum over all pairs).
 * Also resets the running energy of the chain to this value.
 * energy: host.  Errors: STATE, CUDA. */
gcmc_status gcmc_total_energy(gcmc_ctx *ctx, double *energy);

/* The same full-system energy, computed without allocating any memory.  The
 * paper has no counterpart; this call exists for callers that cannot
 * allocate device memory where they need the energy: code whose device
 * memory is all owned by another allocator or held to a fixed budget, and
 * real-time loops that must not enter the driver's allocator (an allocation
 * can block on the device or fail when memory runs short).  It calls no
 * cudaMalloc, cudaFree or other
 * allocating routine: it reads the padded cell layout that gcmc_build_cells
 * and gcmc_run_moves keep current, and keeps its per-cell partial sums in a
 * static device array of GCMC_NOALLOC_MAX_CELLS doubles (1 MiB) built into
 * the library.
 *   energy: device pointer to one double; written on the context's stream,
 *           stream-ordered (no host synchronisation; read it after the
 *           stream reaches the call).  The running energy of the chain is
 *           not changed.
 * The first call on a device looks up the static array's device address
 * (once per device, with the context's device made current for the call);
 * make that first call before any stream capture begins.  Every call on a
 * device shares the one array: calls whose kernels overlap on the GPU (on
 * different streams, or from different contexts) race and give wrong
 * energies; serialise them.
 * Errors: INVALID_ARG (NULL or host energy pointer, memory of another
 * device, more than GCMC_NOALLOC_MAX_CELLS cells), STATE (cells not built),
 * CUDA. */
#define GCMC_NOALLOC_MAX_CELLS 131072
gcmc_status gcmc_total_energy_noalloc(gcmc_ctx *ctx, double *energy);

/* Gradient of the full-system energy (Eq. 1 differentiated):
 *   dpos[k]   = dE/dr_k (device, N x 3 FP32, species-major order) or NULL;
 *   deps      = dE/deps[a][b], half of the sum over ordered type pairs (a,b)
 *               (host, n_species^2 FP64) or NULL;
 *   dsigma    = dE/dsigma[a][b], same convention, rc fixed (host) or NULL;
 *   energy    = E (host) or NULL;  virial = sum_{i<j} r U'(r) (host) or NULL.
 * Errors: STATE, CUDA. */
gcmc_status gcmc_energy_grad(gcmc_ctx *ctx, float *dpos, double *deps, double *dsigma,
                             double *energy, double *virial);

/* Particle counts per species (host, n_species int64; zeros before the
 * first build).  Errors: INVALID_ARG (NULL). */
gcmc_status gcmc_counts(gcmc_ctx *ctx, int64_t *n_per_species);

/* Copies the current configuration out (all host pointers, any may be NULL):
 * pos_grid: N x 3 uint32 grid coordinates in species-major order;
 * cell_count: n_cells int32; cell_refs: N uint32 = (i << 8) | s, the
 * particles of cell 0 in cell order, then cell 1, ...;
 * energy: the running energy (NaN when unknown).  Errors: STATE, CUDA. */
gcmc_status gcmc_get_state(gcmc_ctx *ctx, uint32_t *pos_grid, int32_t *cell_count,
                           uint32_t *cell_refs, double *energy);

/* Restores a configuration written by gcmc_get_state (host pointers), with
 * n_per_species (host, n_species int64) and the running energy (NaN =
 * unknown).  Together with the counter-based moves this resumes a chain bit
 * for bit.  Errors: INVALID_ARG (inconsistent arrays), CAPACITY,
 * CELL_OVERFLOW, CUDA. */
gcmc_status gcmc_set_state(gcmc_ctx *ctx, const int64_t *n_per_species, const uint32_t *pos_grid,
                           const int32_t *cell_count, const uint32_t *cell_refs, double energy);

/* Geometry of the context (host out).  Errors: INVALID_ARG. */
gcmc_status gcmc_get_geometry(gcmc_ctx *ctx, gcmc_geometry *out);

/* Number of CUDA kernels this context has launched so far (host out; a
 * diagnostic for launch accounting).  Errors: INVALID_ARG. */
gcmc_status gcmc_kernel_launches(gcmc_ctx *ctx, int64_t *out);

/* Diagnostics of the last gcmc_run_moves (host out, either may be NULL):
 * refetched = moves whose prefetched neighbour data or particle record was
 * invalidated by the previous move and loaded again; refined = trials whose
 * FP32 decision fell inside the error band and were decided in FP64.
 * Errors: INVALID_ARG. */
gcmc_status gcmc_chain_counters(gcmc_ctx *ctx, int64_t *refetched, int64_t *refined);

/* Where the chain kernel's time went in the last gcmc_run_moves (or batch
 * run) of this context, in SM clock cycles summed over the run (host, 12
 * doubles): [0] the committer waiting for evaluations, [1] checking their
 * validity, [2] deciding (partial sums, Metropolis test, FP64 refinement),
 * [3] applying accepted moves, [4] the committer's whole loop; [5] the team
 * leaders waiting for an eligible move and [6] the teams evaluating (summed
 * over teams), [7] evaluations; [8] .. [10] the parts of [1]: the count
 * epoch, the logged moves, the particle pick; [11] booking a decided move.
 * Zeros for the microcell chain, and for a run without the counters
 * (gcmc_set_chain_profile).
 * Errors: INVALID_ARG. */
gcmc_status gcmc_chain_profile(gcmc_ctx *ctx, double *cycles);

/* Whether the chain runs of this context count the cycles gcmc_chain_profile
 * reports (on = 1; 0, the default, leaves the clock reads out of the
 * kernel, which runs about 2.5 % faster).  A batch counts them when any of
 * its contexts asks.  No paper counterpart (a diagnostic).
 * Errors: INVALID_ARG (NULL, on not 0 or 1). */
gcmc_status gcmc_set_chain_profile(gcmc_ctx *ctx, int32_t on);

/* Team shape of the chain kernel (how its warps split the evaluation of
 * upcoming moves; warps per team, teams, look-ahead L -- a move is
 * evaluated once fewer than L moves separate it from the last committed
 * one: 0 = (6, 2, 4), 1 = (7, 2, 4), 2 = (4, 3, 6), 3 = (3, 4, 8)):
 * 0 .. GCMC_CHAIN_CONFIGS-1, or -1 to time every shape
 * during the next gcmc_run_moves (after a first quarter of its moves under
 * shape 0) and keep the fastest.  Every shape takes the same moves and
 * decisions and reaches the same configuration.  How a trial's pair terms
 * are split among warps depends on the shape and, under speculation, on
 * which counts an evaluation read, so dU and the running energy may differ
 * between runs in their last bits (within the precision's tolerance).
 * Errors: INVALID_ARG. */
#define GCMC_CHAIN_CONFIGS 4
gcmc_status gcmc_set_chain_config(gcmc_ctx *ctx, int32_t config);
/* The current team shape (host int32; -1 until the tuner has run).
 * Errors: INVALID_ARG (NULL). */
gcmc_status gcmc_get_chain_config(gcmc_ctx *ctx, int32_t *config);

/* Last error message of the context (never NULL; "" when none). */
const char *gcmc_last_error(gcmc_ctx *ctx);

/* ---- Batches of independent chains (the points of an isotherm) ----------
 * A batch runs the chains of several built contexts (same device, same
 * precision) in one launch, one CTA per chain, captured as a CUDA graph on
 * the batch's own stream and replayed for later rounds.  Chain k draws
 * Philox counters (m_lo, m_hi, k, 0|1) with its own seed.  The batch keeps
 * pointers to the contexts; they must outlive it. */
typedef struct gcmc_batch gcmc_batch;

/* Errors: INVALID_ARG (NULL or repeated contexts, mixed precision or
 * device), CUDA. */
gcmc_status gcmc_batch_create(gcmc_ctx *const *ctxs, int32_t n_chains, gcmc_batch **out);
/* Frees the batch (its stream and buffers); the contexts stay.  NULL is
 * accepted.  Errors: none (always OK). */
gcmc_status gcmc_batch_destroy(gcmc_batch *batch);

/* Moves first_move .. first_move + n_moves - 1 of every chain, as
 * gcmc_run_moves would run them one context at a time.  seeds, mixes:
 * host, n_chains each; stats: host, n_chains, or NULL.  On the first call
 * with the automatic team shape, the first quarter of the moves runs under
 * shape 0, then every shape is timed on two short chunks (in ascending, then
 * descending shape order) and the shape with the smallest total is kept.  Errors: as gcmc_run_moves, the first
 * failing chain's status (its context has the message); INVALID_ARG. */
gcmc_status gcmc_batch_run_moves(gcmc_batch *batch, const uint64_t *seeds, uint64_t first_move, int64_t n_moves,
                                 const gcmc_move_mix *mixes, gcmc_move_stats *stats);

/* gcmc_build_cells and gcmc_total_energy for every chain of the batch, the
 * work of all contexts issued on their own streams with two host
 * synchronisations in all (the per-context calls synchronise six times
 * each).  pos, species: host arrays of n_chains device pointers (FP64 N x 3,
 * int32 N); n: host, n_chains counts; energies: host, n_chains doubles, or
 * NULL.  Errors: as gcmc_build_cells and gcmc_total_energy, the first
 * failing chain's (gcmc_batch_last_error names it). */
gcmc_status gcmc_batch_prepare(gcmc_batch *batch, const double *const *pos, const int32_t *const *species,
                               const int64_t *n, double *energies);

/* gcmc_energy_grad for every chain (forces, energy and virial; no table
 * derivatives), one host synchronisation in all.  dpos: host array of
 * n_chains device pointers (FP32 N x 3, species-major) or NULL entries, or
 * dpos = NULL; energies, virials: host, n_chains doubles, or NULL.
 * Errors: as gcmc_energy_grad, the first failing chain's. */
gcmc_status gcmc_batch_energy_grad(gcmc_batch *batch, float *const *dpos, double *energies, double *virials);

/* gcmc_export_positions for every chain of the batch (no paper counterpart:
 * the next step's build input).  pos, species: host arrays of n_chains
 * device pointers, each large enough for that chain's N; n: host, n_chains
 * counts out, or NULL.  Launches one kernel per chain on its context's
 * stream; nothing waits.  Errors: as gcmc_export_positions, the first
 * failing chain's; INVALID_ARG (NULL arrays). */
gcmc_status gcmc_batch_export_positions(gcmc_batch *batch, double *const *pos, int32_t *const *species, int64_t *n);

/* Per-chain move records for the following gcmc_batch_run_moves calls:
 * traces is a host array of n_chains device pointers, each NULL or room for
 * the n_moves records (gcmc_trace, the format of gcmc_run_moves) of a call,
 * written at [0, n_moves) of every call; traces = NULL stops the records.
 * The batch keeps the pointers, not the memory.  Errors: INVALID_ARG. */
gcmc_status gcmc_batch_set_traces(gcmc_batch *batch, gcmc_trace *const *traces);

/* Sets the team shape (-1 automatic, -2 leave unchanged) and reports the
 * current one and the per-shape probe times in ms of the last tuning (the
 * sum of the shape's two chunks; host,
 * GCMC_CHAIN_CONFIGS doubles, or NULL).  Errors: INVALID_ARG. */
gcmc_status gcmc_batch_config(gcmc_batch *batch, int32_t set_config, int32_t *config_out, double *probe_ms);

/* Chain-kernel launches (graph replays included) made by the batch (host
 * int64).  Errors: INVALID_ARG (NULL). */
gcmc_status gcmc_batch_launches(gcmc_batch *batch, int64_t *out);

/* Device time in ms of the chain-kernel launches of the last
 * gcmc_batch_run_moves (tuning launches included), taken with CUDA events on
 * the batch's stream around each launch; each launch's few-hundred-byte
 * argument upload and result download fall inside.  ms: host.
 * Errors: INVALID_ARG. */
gcmc_status gcmc_batch_device_ms(gcmc_batch *batch, double *ms);

const char *gcmc_batch_last_error(gcmc_batch *batch);

/* Library version string. */
const char *gcmc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GCMC_H */
