/*
 * sph.h -- C ABI of the GB300 SPH timestep library (libsph_gb300.so).
 *
 * One timestep of the SPH-EXA mini-app's vanilla SPH solver on the rotating
 * square patch (arXiv 1905.03344): neighbour discovery (Table 1), density
 * summation and equation of state, momentum and energy equations with
 * artificial viscosity, Courant time-step, Press (leapfrog) positions and
 * Adams-Bashforth energy (Sec. 3), for one or many independent patches.
 * The paper describes the mini-app's parts as independent libraries with
 * interfaces generic enough to be called from any production code (Sec. 1);
 * this header is that interface: plain C types, no C++ or torch types.
 *
 * Conventions (apply to every entry point):
 *  - Every call returns sph_status; no exception, exit() or device trap ever
 *    crosses this boundary.  sph_last_error(ctx) gives a one-line message.
 *  - A CUDA error that poisons the context (a sticky error) puts the context
 *    in SPH_ESTATE; afterwards only sph_destroy is valid.
 *  - Particle fields are exchanged in the caller's particle order ("original
 *    order").  Internally particles are kept sorted by (patch, Morton cell)
 *    and the library keeps the permutation.
 *  - on_device = 1: pointers are device pointers readable/writable on the
 *    context's stream (e.g. torch tensors' data_ptr()).  on_device = 0: host
 *    pointers; the call copies synchronously.
 *  - All work is issued on the stream given in sph_config.cuda_stream (or a
 *    library-owned stream when NULL).  Calls that return host-visible values
 *    synchronise that stream.
 *  - Inputs are copied: the caller keeps ownership of every pointer it
 *    passes.  Pointers the library returns are borrowed and stay valid until
 *    the next call that changes the particles or the neighbour lists.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_EINVAL = 1,      /* bad argument or configuration */
    SPH_ENOMEM = 2,      /* device or host allocation failed */
    SPH_ECUDA = 3,       /* a CUDA call failed (non-sticky) */
    SPH_EOVERFLOW = 4,   /* neighbour list exceeded max_pairs; state left at the
                            start of the failing step, particles re-sorted */
    SPH_ENONFINITE = 5,  /* NaN/Inf in density, pressure, dt or inputs, or
                            (grad_h) Omega = 0: a particle with no
                            neighbour inside its support */
    SPH_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    SPH_ESTATE = 7       /* call out of order, or context poisoned */
} sph_status;

enum { SPH_FP64 = 0, SPH_MIXED = 1 };               /* sph_config.precision */
enum { SPH_KERNEL_WENDLAND = 0, SPH_KERNEL_SINC = 1 }; /* sph_config.kernel */

/* How the pair sums find their pairs (sph_config.pair_mode). */
enum {
    SPH_PAIRS_LISTS = 0,    /* the step writes neighbour lists and the
                               density and momentum sums read them */
    SPH_PAIRS_FUSED = 1,    /* no lists: the density and the momentum sums each
                               run the neighbour search themselves and take
                               the same pairs in the same order */
    SPH_PAIRS_AUTO = 2      /* SPH_PAIRS_LISTS until sph_autotune, which times
                               both and keeps the faster */
};

/* Fields for sph_get_field (all returned as double, original order). */
enum {
    SPH_FIELD_X = 0, SPH_FIELD_Y, SPH_FIELD_Z,
    SPH_FIELD_VX, SPH_FIELD_VY, SPH_FIELD_VZ,     /* v_{n+1/2} after a step */
    SPH_FIELD_M, SPH_FIELD_H, SPH_FIELD_U,
    SPH_FIELD_DU_PREV,                            /* du of the last step */
    SPH_FIELD_AXP, SPH_FIELD_AYP, SPH_FIELD_AZP,  /* a of the last step */
    SPH_FIELD_RHO, SPH_FIELD_P, SPH_FIELD_C,      /* from the last density call */
    SPH_FIELD_AX, SPH_FIELD_AY, SPH_FIELD_AZ, SPH_FIELD_DU, /* last momentum call */
    SPH_FIELD_NOWN,                               /* n_i = #{j : r^2 < 4 h_i^2} */
    SPH_FIELD_NNB,                                /* |N(i)| (symmetric union) */
    SPH_FIELD_COUNT
};

typedef struct {
    int32_t precision;      /* SPH_FP64 or SPH_MIXED (FP32 pair sums, Kahan) */
    int32_t kernel;         /* SPH_KERNEL_WENDLAND (Eq. 2, the default) or
                               SPH_KERNEL_SINC: W = B_n / h^3 sinc^n(pi v / 2),
                               0 <= v <= 2 (Sec. 3), B_n normalising it */
    int32_t kernel_n;       /* n of the Sinc kernel, 2..16 (default 6) */
    double gamma;           /* ideal-gas exponent, 5/3 */
    double n_target;        /* target neighbour count of h adaptation, 100 */
    double courant;         /* Courant factor C, 0.2 */
    double dt_growth;       /* dt_n <= dt_growth * dt_{n-1}, 1.1 */
    double av_alpha, av_beta, av_eps;  /* Monaghan viscosity, 1, 2, 0.01 */
    double lz;              /* period along z, 1 */
    double dt_fixed;        /* > 0: fixed dt instead of the Courant condition */
    int32_t adapt_h;        /* 1: h adaptation after each step */
    int32_t grad_h;         /* 1: the grad-h momentum and energy form of
                               [rosswog2009]: each side's pressure term with
                               its own kernel, divided by
                               Omega = 1 - dh/drho sum_j m_j dW/dh (h ~ rho^-1/3),
                               evaluated as sum_{j != i} m_j (-v S'(v)) /
                               (3 sum_j m_j S(v)) for W = B h^-3 S(r/h), which
                               is never negative and has no cancellation;
                               Omega = 0 (no neighbour inside the support)
                               fails the step with SPH_ENONFINITE;
                               0 (default): the symmetrised-kernel form */
    int32_t threads_per_particle; /* 0 = auto; else 1, 2, 4, 8, 16 or 32 */
    int32_t pair_mode;      /* SPH_PAIRS_LISTS (default), _FUSED or _AUTO */
    double cell_factor;     /* cell edge = 2 h_s * cell_factor, in [1/3, 4]
                               (h_s: the patch's class threshold of h);
                               below 1/2 the stencil reaches 3 cells and the
                               edge is at least min(h_s, 1.3 h_median).
                               0 (default): 1/2, switched by sph_step between
                               1/2 and 0.4 as the state's spread of h asks;
                               any other value stays fixed */
    double list_skin;       /* 0 (default): every step sorts and searches.
                               skin > 0 (at most 1; list mode only): the search
                               lists the candidate superset r < 2 (1 + skin)
                               max(h_i, h_j), and each step takes its exact
                               lists from that superset with the same
                               predicate as the search; the sort and search
                               run again only once some particle has moved
                               farther than min_k ((1 + skin) h_k0 - h_k)
                               since the superset was built (h_k0: h then),
                               which keeps every pair in the superset.  The
                               lists are the same sets; within a row the
                               order is the superset's.  sph_find_neighbors
                               also takes a superset that still holds (no
                               sort then); a state restored by sph_set_state
                               rebuilds at its first step. */
    int64_t max_particles;  /* capacity, <= 2^25 */
    int64_t max_pairs;      /* neighbour-list capacity (total list entries);
                               0 = 160 * max_particles.  The list pool holds
                               5/2 max_pairs + 24 max_particles + 64 entries of
                               4 bytes: rows are reserved ahead of the search
                               with a margin over their previous length. */
    int32_t max_patches;    /* capacity of independent patches, <= 256 */
    int32_t use_graph;      /* 1: sph_step replays a captured CUDA graph */
    int32_t pair_bins;      /* load balance of the pair sums over lists of
                               uneven length (the imbalance Sec. 4.1 finds
                               across ranks, here across the lanes of a
                               warp): the particles are binned by row-length
                               octave after each search and each octave is
                               summed with the lanes per particle that keep a
                               lane at pair_bins list words or fewer (8, 16,
                               32, 64, 128 or 256; 1 to 32 lanes), so the rows
                               summed side by side differ by less than 2x.
                               0 (default): uniform lanes until sph_autotune,
                               which times bins against uniform lanes;
                               -1: never bins */
    int32_t reserved;       /* set to 0 */
    void* cuda_stream;      /* cudaStream_t or NULL */
} sph_config;

/* Fills the defaults listed above (max_particles = 1<<20, max_patches = 1).
 * The physical defaults are the readings of Sec. 3 (gamma = 5/3, C = 0.2,
 * alpha = 1, beta = 2, 100 neighbours); the rest are library settings. */
void sph_config_default(sph_config* cfg);

/* One instance of the solver library the paper describes (its parts are
 * independent libraries callable from other codes, Sec. 1).
 * Creates a context and allocates all device memory for the capacities in
 * cfg.  Errors: SPH_EINVAL (bad cfg), SPH_ENOMEM, SPH_ECUDA (no device). */
sph_status sph_create(const sph_config* cfg, sph_ctx** out);

/* Frees everything; ctx may be NULL.  (Library housekeeping; no paper
 * counterpart.) */
void sph_destroy(sph_ctx* ctx);

/* Message of the last failing call on ctx (ctx may be NULL: global message).
 * (Library housekeeping; no paper counterpart.) */
const char* sph_last_error(const sph_ctx* ctx);
const char* sph_status_string(sph_status s);

/* Sets n particles (0 <= n <= max_particles); arrays of n doubles each, in the
 * caller's order: position, velocity (v_{-1/2} := v_0), mass, smoothing
 * length, specific internal energy.  These are the particle fields of the
 * square-patch test of Sec. 4 (lattice positions in a periodic-z box, the
 * rotation velocity of Eq. 3, the internal energy of the series pressure);
 * any other particle set is accepted the same way.  Resets the time state
 * (step 0, dt_{-1} = 0, du_{-1} = 0, a_{-1} = 0) and makes all particles one
 * patch.  The arrays are copied; the caller keeps them.
 * Errors: SPH_EINVAL (n out of range, NULL pointer), SPH_ECUDA. */
sph_status sph_set_particles(sph_ctx* ctx, int64_t n, const double* x, const double* y,
                             const double* z, const double* vx, const double* vy,
                             const double* vz, const double* m, const double* h,
                             const double* u, int on_device);

/* The paper has no counterpart: it runs one patch per job.  This call
 * batches many independent problems into one launch per phase.
 * Splits the particles into independent patches: patch p is particles
 * [offsets[p], offsets[p+1]) of the original order, offsets[0] = 0,
 * offsets[n_patches] = n.  Each patch has its own grid, time-step and
 * conserved sums, and its own z period lz.  Valid only right after
 * sph_set_particles (or sph_set_state).  offsets is a host array.
 * Errors: SPH_EINVAL, SPH_ESTATE. */
sph_status sph_set_patches(sph_ctx* ctx, int32_t n_patches, const int64_t* offsets);

/* Neighbour discovery (Table 1): per patch bounding box, h histogram and
 * class threshold, Morton keys, radix sort into cells, cell ranges, and one
 * search per particle that writes its row into the list pool.  j is a
 * neighbour of i iff j != i and r_ij^2 < 4 h_i^2 or r_ij^2 < 4 h_j^2
 * (minimum image along z), decided exactly in FP64.
 * Errors: SPH_EOVERFLOW (more than max_pairs entries), SPH_ESTATE. */
sph_status sph_find_neighbors(sph_ctx* ctx);

/* The result of the neighbour discovery of Table 1 as lists.
 * Borrowed device pointers to the last neighbour lists as a canonical CSR in
 * sorted order: row k (sorted particle k) holds col[off[k] .. off[k+1]) as
 * sorted indices; perm[k] is the original index of sorted particle k.  Within
 * a row, the neighbours with h below the patch's class threshold come first,
 * grouped by cell and ascending inside each cell, then the few above it
 * (grouped by coarse cell, ascending inside each).  (The
 * timestep itself reads the rows where the search wrote them -- contiguous
 * rows with a start and a length each; this call lays them out with prefix
 * offsets.)  Any output pointer may be NULL. */
sph_status sph_get_neighbors(sph_ctx* ctx, const uint64_t** off, const uint32_t** col,
                             const uint32_t** perm, int64_t* nnz);

/* The neighbour lists of Table 1's discovery, copied out.
 * Copies the last neighbour lists into caller buffers (device or host per
 * on_device): off (n+1 uint64), col (nnz uint32, sorted indices), perm (n
 * uint32).  Any pointer may be NULL.  Same layout as sph_get_neighbors. */
sph_status sph_copy_neighbors(sph_ctx* ctx, uint64_t* off, uint32_t* col, uint32_t* perm,
                              int on_device);

/* Density summation rho_i = m_i W(0,h_i) + sum_j m_j W(r_ij, h_i) (Sec. 3,
 * Eq. 2) and the ideal-gas EOS P = (gamma-1) rho u, c = sqrt(gamma P/rho), on
 * the current neighbour lists, or (SPH_PAIRS_FUSED in effect) over the
 * neighbour search itself, which then also sets |N(i)| and n_i.  Needs
 * sph_find_neighbors on the current particles.  Errors: SPH_ESTATE,
 * SPH_ENONFINITE. */
sph_status sph_density(sph_ctx* ctx);

/* Momentum and energy pair sums with Monaghan viscosity (Sec. 3):
 *   a_i  = -sum_j m_j (P_i/rho_i^2 + P_j/rho_j^2 + Pi_ij) grad_i Wbar_ij
 *   du_i =  sum_j m_j (P_i/rho_i^2 + Pi_ij/2) v_ij . grad_i Wbar_ij
 * with Wbar_ij = (W(r,h_i) + W(r,h_j))/2 and the time-centred velocity
 * v_{n-1/2} + a_{n-1} dt_{n-1}/2.  Errors: SPH_ESTATE (no density). */
sph_status sph_momentum_energy(sph_ctx* ctx);

/* nsteps full timesteps of the mini-app's solver (Sec. 3): the Courant
 * condition on a global time-step (Table 1 "Global"), positions by the Press
 * (leapfrog) method and the energy by Adams-Bashforth.  Each step runs
 * neighbours, density + EOS, momentum + energy,
 * Courant dt_n = min(C min h/c, dt_growth dt_{n-1}) per patch, kick
 * v_{n+1/2} = v_{n-1/2} + a_n (dt_n + dt_{n-1})/2, drift x += v_{n+1/2} dt_n
 * (z wrapped), Adams-Bashforth energy, h adaptation, conserved sums.
 * dt_last (nullable, host) receives patch 0's last dt.  With a cell factor
 * of 1/2 or 0.4 that came from the default or from sph_autotune, the call
 * ends by taking the cell grid's vote of its last sort for the next call:
 * 0.4 once the spread of h is wide but smooth in space, 1/2 again when it is
 * not (see cell_factor); the choice depends on the state alone.
 * Errors: SPH_EOVERFLOW, SPH_ENONFINITE, SPH_ETIMEOUT, SPH_ESTATE. */
sph_status sph_step(sph_ctx* ctx, int32_t nsteps, double* dt_last);

/* The quantities whose conservation the square-patch test of Sec. 4 is used
 * to check (Sec. 4 stresses enforcing the fundamental conservation laws).
 * Conserved sums of patch (or all patches for patch = -1) from the current
 * state, out (host) = { M, Px, Py, Pz, Lz, Ekin, Eint }: M = sum m,
 * P = sum m v, Lz = sum m (x v_y - y v_x), Ekin = sum m v^2/2, Eint = sum m u,
 * computed in FP64 with a deterministic two-level reduction. */
sph_status sph_conserved(sph_ctx* ctx, int32_t patch, double out[7]);

/* Copies one field (SPH_FIELD_*) in original order into dst (n doubles): the
 * particle state and the quantities of the Sec. 3 solver (rho, P, c, a,
 * du/dt, n_i, |N(i)|). */
sph_status sph_get_field(sph_ctx* ctx, int32_t field, double* dst, int on_device);

/* Time state of a patch: last dt (the Courant step of Sec. 3), the dt used
 * as dt_{n-1}, steps taken. */
sph_status sph_get_dt(sph_ctx* ctx, int32_t patch, double* dt, double* dt_prev, int64_t* step);

/* The mini-app has no checkpoint/restart (Table 2); the paper lists
 * checkpointing as future work (Sec. 5).  Here it is a state save/restore.
 * Checkpoint: with buf = NULL, *bytes receives the size needed; otherwise the
 * full time state (particle fields in internal order, permutation, patch
 * table, dt state) is written to the host buffer buf.  sph_set_state restores
 * it; stepping then continues bit for bit as without the checkpoint. */
sph_status sph_get_state(sph_ctx* ctx, void* buf, size_t* bytes);
sph_status sph_set_state(sph_ctx* ctx, const void* buf, size_t bytes);

/* The paper has no counterpart (it tunes nothing at run time): a launch-shape
 * autotuner of this library.
 * Times the neighbour and pair-sum phases for a few candidate launch
 * configurations (threads per particle, cell factor and, with
 * SPH_PAIRS_AUTO, lists against the list-free sums) on the current
 * particles and keeps the fastest; the particle state is left unchanged. */
sph_status sph_autotune(sph_ctx* ctx);

/* No paper counterpart (launch settings of this library).
 * Current launch configuration (after sph_autotune or as configured): the
 * momentum sum's lanes per particle and the cell factor. */
sph_status sph_get_tuning(sph_ctx* ctx, int32_t* threads_per_particle, double* cell_factor);

/* No paper counterpart (launch settings of this library).
 * Lanes per particle of the density sum (sph_autotune tunes it apart from the
 * momentum sum's). */
sph_status sph_get_density_tpp(sph_ctx* ctx, int32_t* threads_per_particle);

/* The load-balance settings for the imbalance Sec. 4.1 describes.
 * Row-length bins in effect (sph_config.pair_bins, or the autotuner's
 * choice): the list-word target per lane of the density and of the momentum
 * sum, 0 where that sum runs with uniform lanes per particle. */
sph_status sph_get_pair_bins(sph_ctx* ctx, int32_t* words_density, int32_t* words_momentum);

/* No paper counterpart (a choice of this library's design).
 * The pair mode in effect: SPH_PAIRS_LISTS or SPH_PAIRS_FUSED (SPH_PAIRS_AUTO
 * resolves to one of them in sph_autotune). */
sph_status sph_get_pair_mode(sph_ctx* ctx, int32_t* mode);

/* No paper counterpart (reused candidate supersets are this library's).
 * Candidate supersets built so far (list_skin > 0: sph_find_neighbors and
 * the steps that had to sort and search again). */
sph_status sph_get_list_rebuilds(sph_ctx* ctx, int64_t* n);

/* The paper profiles its runs to find imbalance and idle time (Sec. 4.1);
 * these are this library's timers for its own phases.
 * Phase timers: when enabled, every phase of sph_step/sph_find_neighbors/
 * sph_density/sph_momentum_energy is bracketed by CUDA events on the
 * context's stream (graph replay is then off).  sph_get_profile returns the
 * accumulated milliseconds and launch counts per phase (SPH_PHASE_*) and
 * resets them. */
enum {
    SPH_PHASE_BBOX = 0,      /* per-patch bounding box, largest h, grid */
    SPH_PHASE_KEYS,          /* Morton cell keys */
    SPH_PHASE_SORT,          /* radix sort */
    SPH_PHASE_GATHER,        /* gather into sorted order, cell table */
    SPH_PHASE_NB_RESET,      /* list pool reset */
    SPH_PHASE_NB,            /* neighbour lists, one warp per 32 particles */
    SPH_PHASE_DENSITY,       /* density + EOS */
    SPH_PHASE_MOMENTUM,      /* momentum + energy */
    SPH_PHASE_UPDATE,        /* dt, kick/drift/AB2, h, conserved sums */
    SPH_PHASE_COUNT
};
sph_status sph_set_profiling(sph_ctx* ctx, int enable);
sph_status sph_get_profile(sph_ctx* ctx, double* ms, int64_t* launches, int32_t nphase);

/* No paper counterpart (instrumentation).
 * Number of kernels this context has launched so far (graph replays count
 * every kernel node). */
sph_status sph_get_launch_count(sph_ctx* ctx, int64_t* launches);

/* Neighbour-list size of the last sph_find_neighbors (Table 1's discovery). */
sph_status sph_get_nnz(sph_ctx* ctx, int64_t* nnz);

/* No paper counterpart (instrumentation: the benchmark's pair count).
 * Sum of |N(i)| over all particles and all sph_step steps since the last
 * reset (the pair-interaction count of the steps); reset != 0 zeroes it. */
sph_status sph_get_pair_count(sph_ctx* ctx, int64_t* total, int reset);

/* Conserved sums { M, Px, Py, Pz, Lz, Ekin, Eint } (as sph_conserved) of n
 * particles whose fields the caller already holds on the device, computed
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code that runs
 * while a stream is being captured into a CUDA graph, host frameworks that
 * own the device allocator and forbid other allocations, processes that have
 * handed all device memory to their own pool.
 * Arguments: device pointers x, y, vx, vy, vz, m, u (n doubles each) and out
 * (7 doubles, device); cuda_stream is a cudaStream_t or NULL (default
 * stream).  The call is asynchronous on that stream: read out after
 * synchronising it.  No context is needed.
 * Scratch: a fixed array of 4096 partial-sum slots in the library's own
 * device memory (256 KB, kept by every GPU that loads the library until the
 * process exits), so n is limited to 16,777,216; larger n returns
 * SPH_EINVAL.  The first call on a device looks up the array's device
 * address (do that first call before any stream capture) and keeps it for
 * the life of the process: after cudaDeviceReset, or anything else that
 * replaces the device's primary context, the kept address is stale and this
 * entry point must not be called again on that device.  Every call
 * overwrites the array: calls whose work overlaps on the GPU race.
 * Errors: SPH_EINVAL (n out of range, NULL pointer), SPH_ECUDA;
 * sph_noalloc_last_error() gives the message. */
sph_status sph_conserved_noalloc(int64_t n, const double* x, const double* y, const double* vx,
                                 const double* vy, const double* vz, const double* m,
                                 const double* u, double* out, void* cuda_stream);
const char* sph_noalloc_last_error(void);

/* The fused multiply-add rate of this GPU in FLOP/s (an FMA counts 2): a
 * kernel of independent FMA chains on every SM, 8 CTAs of 256 threads per SM,
 * timed with CUDA events over runs of at least 50 ms, best of three.
 * precision: SPH_MIXED measures FP32 FMA, SPH_FP64 measures FP64 FMA.  It is
 * the roofline denominator of the pair sums, which are bound by those pipes.
 * The paper has no counterpart.  Synchronous on cuda_stream (a cudaStream_t
 * or NULL); runs for about 0.3 s on the current device; allocates nothing
 * but two events.  Errors: SPH_EINVAL, SPH_ECUDA;
 * sph_fma_peak_last_error() gives the message. */
sph_status sph_fma_peak(int32_t precision, double* flop_per_s, void* cuda_stream);
const char* sph_fma_peak_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPH_GB300_H */
