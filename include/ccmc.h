/*
 * ccmc.h -- C ABI of the GB300 coupled cluster Monte Carlo (CCMC) library.
 *
 * One call of ccmc_step advances the stochastic coupled cluster wavefunction
 * by one imaginary-time step as defined in Spencer et al., "Large Scale
 * Parallelization in Stochastic Coupled Cluster" (arXiv:1807.03749):
 *   - selection of clusters of excitors (Sec. II: cluster size from
 *     p_size(s) = 2^-(s+1), s in [0, l+2]; excitors with probability
 *     |t_i| / (N_total - t_HF)), or the full non-composite sweep (Sec. IV.B);
 *   - collapse of each cluster to one determinant with its fermionic sign
 *     (Sec. II, Eq. 3-5);
 *   - spawning through an excitation generator and Slater-Condon matrix
 *     elements, with multi-spawn attempts (Sec. II; Sec. IV.C, Eq. 7-8);
 *   - death, the diagonal part of the propagator (Sec. II, Eq. CCMC);
 *   - annihilation: radix sort of the spawned particles by determinant key,
 *     reduction of equal keys and merge into the excip list (Sec. II);
 *   - the projected-energy numerator (Sec. II, Eq. E_proj) and the shift.
 * Everything runs in CUDA kernels on one GPU; the host only sequences the
 * launches and evaluates the logarithm of the shift update every shift_a steps.
 *
 * Conventions
 *   - Spin-orbital p is bit (p & 63) of word (p >> 6) of a determinant;
 *     spin-orbital 2q is alpha and 2q+1 beta of spatial orbital q.  A
 *     determinant with M spin-orbitals uses K = ceil(M/64) words (M <= 384;
 *     the FP32 form M <= 192).
 *   - Determinants are ordered as unsigned integers compared from the most
 *     significant word; the Hartree-Fock (HF) reference is the lowest N bits.
 *   - Populations are int64 fixed point: value = pop / 2^16.
 *   - A "key" is the rank of a determinant among all determinants of
 *     excitation level <= l in that order (HF has key 0).
 *   - Every function returns a ccmc_status; nothing traps or aborts.  Errors
 *     found by kernels (buffer overflow, numeric overflow, a runaway
 *     population) are recorded in a device status word and reported by the
 *     next synchronising call.  No kernel waits on another.
 *   - One context per CUDA stream; calls on one context are not thread-safe.
 *   - Host pointers are read during the call only (the library copies what it
 *     keeps).  Device memory is owned by the context and released by ccmc_free.
 */
#ifndef CCMC_H
#define CCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccmc_ctx ccmc_ctx;

typedef enum {
    CCMC_OK = 0,
    CCMC_ERR_ARG = 1,             /* invalid argument or description            */
    CCMC_ERR_CUDA = 2,            /* a CUDA runtime call failed                 */
    CCMC_ERR_OOM = 3,             /* device or host allocation failed           */
    CCMC_ERR_SPAWN_OVERFLOW = 4,  /* more spawned particles than spawn_capacity */
    CCMC_ERR_TIMEOUT = 5,         /* a bounded device wait gave up              */
    CCMC_ERR_NUMERIC = 6,         /* a weight left the fixed-point range        */
    CCMC_ERR_LIST_OVERFLOW = 7,   /* more occupied excitors than list_capacity  */
    CCMC_ERR_STATE = 8,           /* call not valid in the context's state      */
    CCMC_ERR_RUNAWAY = 9          /* population runaway: a step would need more
                                     than max(64 x target_pop, 2^24) samples, or
                                     spawning attempts; it was abandoned        */
} ccmc_status;

enum { CCMC_UEG = 0, CCMC_GENERIC = 1 };
enum { CCMC_FP64 = 0, CCMC_FP32 = 1 };

/* Hamiltonian description (caller-owned; copied by ccmc_init).
 *   kind = CCMC_UEG: three-dimensional uniform electron gas in a cubic box of
 *     side L = rs (4 pi N / 3)^(1/3); the n_spinorb/2 plane waves of lowest
 *     |n|^2 (ties in lexicographic order of n; the count must close a shell);
 *     kinetic |k|^2/2 and Coulomb 4 pi / (L^3 |q|^2) without q = 0.
 *   kind = CCMC_GENERIC: spatial integrals h1[p*norb+q] and chemists' (pq|rs)
 *     at eri[((p*norb+q)*norb+r)*norb+s], norb = n_spinorb/2, both symmetric. */
typedef struct {
    int32_t kind;
    int32_t n_electrons;   /* N */
    int32_t n_spinorb;     /* M, even, N < M <= 384 (FP32 form: <= 192) */
    int32_t reserved;
    double rs;             /* UEG density parameter (bohr) */
    const double *h1;      /* GENERIC only */
    const double *eri;     /* GENERIC only */
    double e_core;         /* GENERIC only: constant added to energies */
} ccmc_hamiltonian;

/* Reference determinant (caller-owned, K words).  It must be the lowest N
 * spin-orbitals; any other reference is rejected with CCMC_ERR_ARG. */
typedef struct {
    const uint64_t *bits;
} ccmc_reference;

/* Optional device allocator (e.g. a framework's caching allocator).  When
 * alloc is NULL the library uses cudaMalloc/cudaFree. */
typedef void *(*ccmc_alloc_fn)(size_t bytes, void *user);
typedef void (*ccmc_free_fn)(void *ptr, void *user);

typedef struct {
    double tau;              /* time step delta tau */
    double target_pop;       /* population at which the shift starts to vary */
    double d0_init;          /* initial weight on HF */
    int32_t shift_a;         /* steps between shift updates (A) */
    int32_t fnc;             /* 1: full non-composite sampling (Sec. IV.B) */
    double zeta;             /* shift damping */
    double spawn_cutoff;     /* spawned weights below this are rounded stochastically to it */
    int32_t multispawn;      /* 1: n_attempts = max(1, floor(|A|/a_thresh)) (Sec. IV.C) */
    int32_t precision;       /* CCMC_FP64 or CCMC_FP32 matrix elements */
    double a_thresh;         /* multi-spawn threshold */
    uint64_t seed;           /* Philox key word 0 */
    uint64_t replica;        /* Philox key word 1 */
    uint64_t list_capacity;  /* 0 = default from target_pop */
    uint64_t spawn_capacity; /* 0 = default from target_pop */
    void *cuda_stream;       /* cudaStream_t, NULL = legacy default stream */
    ccmc_alloc_fn alloc;
    ccmc_free_fn free;
    void *alloc_user;
    int32_t radix_bits;      /* digit width of the radix sort, 0 = default */
    int32_t flags;           /* CCMC_NO_GRAPH, CCMC_SORT_ALL (below) */
    int32_t n_ranks;         /* simulated processors N_p of the paper's distributed
                                cluster sampling (Sec. III, Eq. ccmc_dist); 0 or 1:
                                none (the plain single-GPU step) */
    int32_t nu_move;         /* excitors move between the simulated processors every
                                2^nu_move iterations; >= 64: never */
} ccmc_params;

/* ccmc_params.flags
 *   CCMC_NO_GRAPH  launch the step's kernels one by one instead of replaying a
 *                  captured CUDA graph of the step.
 *   CCMC_SORT_ALL  send every spawned record through the radix sort.  By
 *                  default a record whose determinant is already in the excip
 *                  list is added to that entry directly (an integer atomic)
 *                  and only records onto new determinants are sorted; the
 *                  merged list is identical either way (integer sums), but
 *                  ccmc_get_spawned then returns the sorted records onto new
 *                  determinants only.  With this flag it returns all of them. */
#define CCMC_NO_GRAPH 1
#define CCMC_SORT_ALL 2

/* Per-step record; one is kept for every step in a device ring buffer. */
typedef struct {
    uint64_t iter;        /* iteration index of the step */
    double shift;         /* S used in the step (relative to E_HF) */
    int64_t n0;           /* t_HF at the start of the step (fixed point) */
    int64_t ntot;         /* N_total at the start (fixed point) */
    int64_t n_sel;        /* cluster samples drawn */
    int64_t n_visit;      /* full non-composite visits */
    int64_t n_attempts;   /* spawning attempts */
    int64_t n_spawned;    /* spawned records entering the sort */
    double e_num;         /* projected-energy numerator of the step */
    int64_t ntot_after;   /* N_total after annihilation */
    int64_t nocc_after;   /* occupied excitors after annihilation */
    int64_t n_keys;       /* distinct keys among the spawned records */
    int64_t n_clusters;   /* composite clusters buffered for multi-spawn attempts */
    int64_t n_direct;     /* spawned records added directly to listed determinants
                             (included in n_spawned; not sorted) */
} ccmc_record;

/* Creates a context: copies the Hamiltonian, builds orbital and matrix-element
 * tables, allocates device state and places d0_init on HF.  truncation_level
 * is l (1..4); clusters up to size l+2 are sampled.  Asynchronous work is
 * issued on params->cuda_stream.  Returns CCMC_ERR_ARG for an invalid
 * description, CCMC_ERR_OOM when device memory is exhausted. */
ccmc_status ccmc_init(const ccmc_hamiltonian *ham, const ccmc_reference *ref, int truncation_level,
                      const ccmc_params *params, ccmc_ctx **out);

/* Issues nsteps time steps (Sec. II) on the context's stream.  The host
 * synchronises only at shift-update boundaries (every shift_a steps) to take
 * the logarithm of the population ratio; otherwise the call is asynchronous.
 * On a non-NULL stream the step's kernels are captured once into a CUDA graph
 * and replayed (unless CCMC_NO_GRAPH or profiling is set); the first step of
 * a context should therefore not be issued inside another stream capture.
 * Kernel-detected errors are returned by the first synchronising call. */
ccmc_status ccmc_step(ccmc_ctx *ctx, int nsteps);

/* Synchronises and returns the estimators of the latest step:
 * e_proj = e_num / t_HF (correlation energy), the numerator, t_HF, the shift
 * and N_total after annihilation, all in population units.  Any pointer may
 * be NULL. */
ccmc_status ccmc_energy(ccmc_ctx *ctx, double *e_proj, double *e_num, double *n0, double *shift,
                        double *n_total);

/* Reference energy E_HF (+ e_core) of the context's Hamiltonian. */
ccmc_status ccmc_reference_energy(ccmc_ctx *ctx, double *e_hf);

/* Copies the records of the last min(cap, steps since the previous call,
 * ring size) steps, oldest first; *n receives the count. */
ccmc_status ccmc_get_records(ccmc_ctx *ctx, ccmc_record *out, size_t cap, size_t *n);

/* Number of occupied excitors in the list. */
ccmc_status ccmc_list_size(ccmc_ctx *ctx, size_t *n);

/* Copies the excip list in key order to host buffers: bits (n*K words,
 * determinant i at bits[i*K..]), keys (n) and pop (n); NULL buffers are
 * skipped.  Returns CCMC_ERR_ARG if cap < n. */
ccmc_status ccmc_get_list(ccmc_ctx *ctx, uint64_t *bits, uint64_t *keys, int64_t *pop, size_t cap,
                          size_t *n);

/* Replaces the excip list from host buffers (n determinants of K words and
 * their populations).  The list must be sorted, unique, start with HF, stay
 * within the truncation level and within the reference's sector (its S_z,
 * and for the gas its total momentum: the sector every spawn stays in);
 * otherwise CCMC_ERR_ARG and the context keeps its previous list.  The checks
 * run on the device; the list is uploaded into the context's spare list
 * buffer, which becomes current only if it passes. */
ccmc_status ccmc_set_list(ccmc_ctx *ctx, const uint64_t *bits, const int64_t *pop, size_t n);

/* The spawned records of the latest step that went through the sort (keys
 * and fixed-point weights, sorted by key; composite deaths included): with
 * CCMC_SORT_ALL the whole multiset entering the annihilation, otherwise the
 * records onto determinants not in the list at the start of the step. */
ccmc_status ccmc_get_spawned(ccmc_ctx *ctx, uint64_t *keys, int64_t *pop, size_t cap, size_t *n);

/* The death deltas of the latest step for the list entries of that step's
 * start (same order as the list then). */
ccmc_status ccmc_get_death(ccmc_ctx *ctx, int64_t *death, size_t cap, size_t *n);

/* Iteration index, shift, shift-varying flag and the population at the last
 * shift boundary (checkpoint state besides the list). */
ccmc_status ccmc_set_state(ccmc_ctx *ctx, uint64_t iter, double shift, int32_t vary, double nprev);
ccmc_status ccmc_get_state(ccmc_ctx *ctx, uint64_t *iter, double *shift, int32_t *vary, double *nprev);

/* Checkpoint to / restore from a file (state + list).  Because every random
 * number is a function of (seed, replica, iteration, index), a restored run
 * continues bit-identically. */
ccmc_status ccmc_save(ccmc_ctx *ctx, const char *path);
ccmc_status ccmc_load(ccmc_ctx *ctx, const char *path);

/* Phases of a step for the opt-in timers: a1 scans, a2-a5 sampling, a4/a6
 * expanded attempts, a7 radix sort, a8 key reduction, a9 merge, a10 estimator
 * reduction. */
enum {
    CCMC_PHASE_SCAN = 0,
    CCMC_PHASE_SAMPLE = 1,
    CCMC_PHASE_ATTEMPTS = 2,
    CCMC_PHASE_SORT = 3,
    CCMC_PHASE_REDUCE = 4,
    CCMC_PHASE_MERGE = 5,
    CCMC_PHASE_FINALIZE = 6,
    CCMC_NPHASES = 7
};

/* Enables (1) or disables (0) per-phase timing.  While enabled, ccmc_step
 * records CUDA events between phases on the context's stream and waits for
 * each step to finish, so timed runs should leave it disabled.  Enabling
 * resets the accumulated times. */
ccmc_status ccmc_profile(ccmc_ctx *ctx, int32_t enable);

/* Accumulated milliseconds and kernel launches per phase since profiling was
 * enabled (ms and launches hold nphases entries, NULL to skip), and the total
 * number of kernels launched by ccmc_step since the context was created. */
ccmc_status ccmc_phase_times(ccmc_ctx *ctx, double *ms, int64_t *launches, int32_t nphases, int64_t *total_launches);

/* ---- Batched form: many independent contexts stepped together ----------
 * Every phase of the step is one kernel launch over all replicas that share
 * a determinant word count and precision (a CUDA grid dimension indexes the
 * replica), and the whole step is captured once in a CUDA graph and replayed.
 * The cluster sampler, the bulk of the work, is one persistent launch whose
 * blocks take shares of the replicas' samples from a plan written on the
 * device each step, so replicas of very different sizes keep the GPU busy.
 * Per-replica grid sizes, the sampler's samples per share and the radix digit
 * width are chosen by timing candidates on real steps, again whenever the
 * batch's total population has changed by a factor of two since the last
 * choice (the trajectory does not depend on them).
 * Replicas keep their own Philox keys, shift control and checkpoints; results
 * are bit-identical to stepping each context alone. */
typedef struct ccmc_batch ccmc_batch;

/* Groups n contexts (which must all use the same shift_a) into a batch whose
 * work is issued on cuda_stream (must not be NULL).  The contexts stay owned
 * by the caller; while in the batch, ccmc_step on them returns
 * CCMC_ERR_STATE, and a context in another batch is rejected with
 * CCMC_ERR_STATE.  Reading a member (lists, records, energies, spawned
 * records, death deltas), ccmc_set_list, ccmc_set_state and checkpoints
 * remain allowed: each such call first waits for the batch's stream, so it
 * sees (or replaces) the state after the batch's last issued step.  Free the
 * batch before its contexts; a member freed first is detached from the batch
 * (after waiting for the batch's stream), and the batch then refuses to step
 * (CCMC_ERR_STATE) and can only be freed. */
ccmc_status ccmc_batch_create(ccmc_ctx **ctxs, int32_t n, void *cuda_stream, ccmc_batch **out);

/* nsteps steps of every context in the batch.  The host synchronises at each
 * context's shift-update boundary (every shift_a steps).  Tuning steps are
 * issued one by one and timed; the graph is captured after each tuning. */
ccmc_status ccmc_step_batched(ccmc_batch *b, int32_t nsteps);

/* The current per-replica work-grid blocks, the sampler's samples per share
 * (sample_tile), the radix digit width, the number of replica groups and how
 * many times the shapes have been tuned (any pointer may be NULL). */
ccmc_status ccmc_batch_info(ccmc_batch *b, int32_t *work_blocks, int32_t *sample_tile, int32_t *digit_bits,
                            int32_t *groups, int32_t *tunings);

/* Per-phase timers of the batch, as ccmc_profile / ccmc_phase_times for a
 * context (phases summed over the replica groups). */
ccmc_status ccmc_batch_profile(ccmc_batch *b, int32_t enable);
ccmc_status ccmc_batch_phase_times(ccmc_batch *b, double *ms, int64_t *launches, int32_t nphases,
                                   int64_t *total_launches);

/* Releases the batch (not its contexts). */
void ccmc_batch_free(ccmc_batch *b);

/* Largest record count accepted by ccmc_reduce_records_noalloc. */
#define CCMC_NOALLOC_MAX_RECORDS 65536

/* Sorts n spawned records by key and sums each run of equal keys -- the
 * annihilation's sort and reduction as a standalone call -- without
 * allocating any device memory.  The paper has no counterpart.  It is for
 * callers that may not call cudaMalloc or an allocating library routine:
 * plugins whose host application owns the device allocator, and loops that
 * must keep a fixed device-memory footprint once set up.
 *   keys_in, pops_in   device arrays of n records (read only)
 *   key_bits           significant bits of the keys (1..64); keys with bits
 *                      set above key_bits are outside the contract and are
 *                      not sorted correctly
 *   keys_out, pops_out device arrays with room for n records; receive the
 *                      distinct keys in increasing order and their summed
 *                      weights (runs that sum to zero are kept)
 *   n_out              host pointer; receives the number of distinct keys
 *   cuda_stream        cudaStream_t for the work (NULL = legacy stream); the
 *                      call waits for it before returning
 * Scratch is one fixed device array inside the library of about 2.07 MiB
 * (two ping-pong buffers of CCMC_NOALLOC_MAX_RECORDS keys and weights, 2 MiB,
 * plus histograms, block partials and counters), held by every GPU that
 * loads the library until the process exits.  n above
 * CCMC_NOALLOC_MAX_RECORDS is rejected with CCMC_ERR_ARG before any work.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  The array is shared per device by every caller in the process
 * (other streams, other threads, other library contexts) and keeps the last
 * call's contents; calls that overlap on the GPU race and must be
 * serialised by the caller. */
ccmc_status ccmc_reduce_records_noalloc(const uint64_t *keys_in, const int64_t *pops_in, size_t n, int32_t key_bits,
                                        uint64_t *keys_out, int64_t *pops_out, size_t *n_out, void *cuda_stream);

/* ---- The paper's distribution over processors, simulated ----------------
 * Sec. III distributes excitors over N_p processors with the owner
 *   o(D, i) = (hash(D) + i) >> nu_move,  p(D, i) = hash(D xor o) mod N_p
 * (Eq. ccmc_dist; i the iteration, o xor-ed into the first word of D), and
 * each processor forms composite clusters only from its own excitors.  Here
 * the hash is Philox-4x64-10 under a fixed key used as a mixing function over
 * the bit string (three words per call, each call chained through the fourth
 * counter word).  With ccmc_params.n_ranks = N_p > 1 (at most 65535) a
 * composite cluster of size s is drawn as a processor would draw it from the
 * excitors it holds: its first excitor from the whole list (a processor
 * samples in proportion to its population), the others from the first one's
 * processor q only, in proportion to |t| among q's excitors (N_q their sum).
 * Its amplitude is N_ex (N_q N_p)^(s-1) / (|t_HF|^(s-1) n_sel p(s) s!): the
 * inverse selection probability times N_p^(s-1), the inverse of the
 * probability that s excitors share a processor, so that the step is
 * unbiased averaged over owners while each iteration samples a subspace --
 * the source of the parallelisation bias the paper studies.
 *
 * ccmc_colocation computes the co-location statistics of Fig. excitdistrib
 * for n determinants (host array, n rows of n_words words): for every
 * checkpoint T (ascending, at most 64, the last <= 2^20), the sums over pairs
 * i < j of C_ij(T) and C_ij(T)^2, C_ij(T) being the number of iterations
 * t < T at which excitors i and j have the same owner.  The mean co-location
 * probability is sum_c / (P T) and its variance over pairs
 * sum_c2 / (P T^2) - mean^2, with P = n(n-1)/2.  n_ranks <= 65535, n <= 2^20.
 * Allocates temporary device memory; synchronises cuda_stream. */
ccmc_status ccmc_colocation(const uint64_t *dets, size_t n, int32_t n_words, int64_t n_ranks, int32_t nu_move,
                            const int64_t *checkpoints, int32_t n_checkpoints, uint64_t *sum_c, uint64_t *sum_c2,
                            void *cuda_stream);

/* Waits for the context's stream and reports kernel-detected errors. */
ccmc_status ccmc_sync(ccmc_ctx *ctx);

/* Human-readable description of the last error on this context. */
const char *ccmc_last_error(ccmc_ctx *ctx);

/* Releases the context and all its device memory. */
void ccmc_free(ccmc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CCMC_H */
