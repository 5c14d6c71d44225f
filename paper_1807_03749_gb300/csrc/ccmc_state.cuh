// ccmc_state.cuh -- device-resident state of a CCMC context, shared by the
// step kernels (ccmc_step.cu) and the host API (ccmc_api.cu).  Every kernel
// uses a fixed grid and reads its element counts from device memory, so a
// whole step is issued without a host round trip.
#pragma once

#include "ccmc_device.cuh"

namespace ccmc {

constexpr int SCAN_THREADS = 512;
constexpr int WORK_THREADS = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int MAX_DIGIT_BITS = 8;
// resident blocks of the cluster sampler per SM (its register budget)
#ifndef CCMC_SAMPLE_BLOCKS_PER_SM
#define CCMC_SAMPLE_BLOCKS_PER_SM 4
#endif
constexpr int SAMPLE_BLOCKS_PER_SM = CCMC_SAMPLE_BLOCKS_PER_SM;
constexpr int RING = 1 << 14;             // per-step records kept on the device
constexpr int CL_SHIFT = 38;              // packed (clusters << 38) | attempts
constexpr u64 CL_MASK = (1ULL << CL_SHIFT) - 1ULL;

// Run parameters read by the kernels.
struct RunParams {
    double tau;
    double spawn_cutoff;
    double a_thresh;
    u64 seed, replica;
    int fnc, multispawn;
    int int_round;        // rounding decisions from the FP64 bit pattern (cutoff 0 or 2^k)
    int a_thresh_one;     // A_thresh == 1: floor(|A|) without a division
    int direct;           // spawns onto listed determinants are added to them directly (not sorted)
    int buffered;         // original sampler: each valid cluster's one attempt runs in the attempts kernel
    int nranks;           // simulated processors (Sec. III): composite clusters from one processor's excitors
    int nu_move;          // owners move every 2^nu_move iterations (>= 64: never)
    i64 work_cap;         // samples, visit attempts or cluster attempts per step beyond which the step is abandoned
    RoundSpec spawn_rs;   // spawn rounding (with the cutoff)
    RoundSpec death_rs;   // death rounding (no cutoff)
};

// Excip list, structure of arrays with capacity cap.
struct ListView {
    u64 *bits;      // bits[w * cap + i]
    u64 *key;
    i64 *pop;
    double *diag;   // H_DD - E_HF
    i64 cap;
};

// Per-step record as stored on the device (same layout as ccmc_record).
struct Record {
    u64 iter;
    double shift;
    i64 n0, ntot, n_sel, n_visit, n_attempts, n_spawned;
    double e_num;
    i64 ntot_after, nocc_after, n_keys;
    i64 n_clusters;
    i64 n_direct;
};

// Mutable per-step scalars living in device memory.
struct DevStep {
    u64 iter;
    double shift;
    i64 n_occ;          // list size at the start of the step
    i64 ntot, n0, nex, n_sel, fnc_attempts;
    double mag[8];      // |A_s| of a cluster of size s
    double cmag[8];     // |A_s| / n_att(s): magnitude of one attempt's coefficient
    i64 natt_s[8];      // attempts of a cluster of size s
    int bucket_shift;   // selection buckets cover 2^bucket_shift positions each
    int pad0;
    i64 nbuckets;
    i64 n_sp;           // spawned records appended (may exceed capacity on overflow)
    u64 cl_packed;      // (clusters << CL_SHIFT) | attempts of buffered clusters
    i64 n_attempts;
    i64 n_keys;         // distinct keys after the reduction
    i64 kept_list, kept_new;
    i64 ntot_after;
    i64 n_start;        // list size at the start of the latest finished step
    double cl_att;      // attempts of the buffered clusters (runaway check; exact below 2^53)
    unsigned err;
    int cur;            // list buffer holding the current list
    int kshift;         // key buckets cover 2^kshift keys each
    int pad1;
    i64 nkb;            // key buckets in use (0: no direct accumulation this step)
    i64 n_direct;       // spawned records added directly to listed determinants
    i64 n_hit;          // listed determinants that received such records
    i64 prev_spawned;   // spawned records of the previous step (0 after a list upload)
    // simulated distribution (Sec. III): the denominators of |A_s| (a
    // composite's amplitude depends on its processor's population), and the
    // chunks of the per-processor position table
    double mden[8];
    int lcs;            // chunks cover 2^lcs list entries
    int pad2;
    i64 nlc;            // chunks in use
};

// Spawn buffer pair for the radix sort (ping-pong).
struct SpawnBuf {
    u64 *key[2];
    i64 *pop[2];
    i64 cap;
};

// Clusters buffered for expanded multi-spawn attempts.
struct ClusterBuf {
    u64 *bits;      // bits[w * cap + c]
    double *catt;   // coefficient of one attempt
    u64 *index;     // sample index g (Philox counter)
    i64 *end;       // inclusive attempt prefix
    i64 cap;
};

// The cluster sampler's view of one list entry besides its bit string,
// written by the scans each step and gathered by a pick as one 32-byte
// sector: selection prefix, population, death factor and <HF|H|D>.
struct __align__(64) PickEntry {
    i64 prefix;     // inclusive |pop| prefix over entries >= 1 (entry 0: 0)
    i64 pop;
    double tdeath;  // tau (Delta E_i - S): the death factor of this step
    double href;    // <HF|H|D_i> (levels 1-2; 0 otherwise; 0 with full non-composite sampling)
    u64 w[4];       // the determinant's words (up to four; more are read from the list)
};
static_assert(sizeof(PickEntry) == 64, "pick table rows are one 64-byte granule");

// Per-step work arrays over the list and the merge.
struct WorkArrays {
    PickEntry *picks; // one row per list entry
    int *bucket;      // owner of the first position of each selection bucket
    int bucket_bits;  // log2 of the bucket capacity
    i64 *att_end;     // inclusive prefix of full non-composite attempts
    double *catt;     // attempt coefficient of each list entry
    i64 *death;       // death deltas (fixed point)
    i64 *acc;         // spawned weight matched to each list entry (direct and reduced)
    int *kbucket;     // first list entry of each key bucket (key >> kshift)
    int kbucket_bits; // log2 of the key-bucket capacity
    unsigned char *hit;  // list entries that received directly added spawns this step
    i64 *part;        // block partials of the scans (4 per block)
    i64 *wpart;       // warp partials of the list scan (4 per warp of the scan grid)
    u64 *enum_part;   // 128-bit fixed-point E_num partial (lo, hi) per producing block
    i64 *newpop;      // list values after the merge (threshold applied)
    i64 *keep_l;      // keep flag | before << 32 of list entries; exclusive prefix where new keys go in
    int *before;      // kept new keys inserted just before each list entry
    i64 *keep_s;      // keep flags of reduced spawns -> exclusive prefix
    i64 *ins;         // insertion position of a new key, -1 when matched
    unsigned *hist;   // radix histograms, digit-major (2^bits x sort grid)
    unsigned *hist_tot;  // per-digit totals of the current pass
    Record *ring;     // per-step records
    // simulated distribution (Sec. III), allocated only with N_p > 1
    unsigned short *owner;  // processor of each list entry at this iteration
    i64 *lcp;         // [q][chunk]: |pop| of processor q's entries before the chunk
    i64 *nq;          // N_q: |pop| held by processor q
    i64 lcp_cap;      // capacity of lcp
};

// Grid shapes chosen once per context.
struct Shapes {
    int scan_grid;    // blocks of SCAN_THREADS for list scans
    int work_grid;    // blocks of WORK_THREADS for sampling and attempts
    int sort_grid;    // blocks of SORT_THREADS for sort passes
    int digit_bits;   // radix digit width
    int key_bits;     // significant key bits
    int enum_slots;   // scan_grid + work_grid (E_num partials of the scans and the sampler)
    int nranks;       // simulated processors (largest over the replicas; 1: none)
};

// Per-replica arguments of the step kernels (device-resident; a single
// context has one, a batch an array indexed by blockIdx.y).
struct StepArgs {
    SysDev s;
    RunParams p;
    ListView list[2];
    SpawnBuf sp;
    ClusterBuf cl;
    WorkArrays wa;
    DevStep *st;
};

// Everything the step launcher needs.
struct StepCtx {
    int K;
    bool fp32;            // FP32 matrix elements and generation probabilities
    SysDev sys;
    RunParams prm;
    ListView list[2];
    int cur;              // list buffer holding the current list
    SpawnBuf sp;
    ClusterBuf cl;
    WorkArrays wa;
    DevStep *st;          // device scalars
    Shapes sh;
    cudaStream_t stream;
    int sorted_buf;       // spawn buffer holding the sorted records after a step
    // opt-in phase timers: events[p] is recorded before phase p, events[NPH] after the last
    bool profile;
    cudaEvent_t events[8];
    i64 launches[8];      // kernels launched per phase (cumulative)
    i64 total_launches;
    StepArgs h_args;      // host copy of this context's kernel arguments
    StepArgs *d_args;     // device copy
};

constexpr int NPHASES = 7;

// Work plan of a batch's cluster sampler: replica r owns the virtual blocks
// [vstart[r], vstart[r+1]), about one per per_block samples (at least one, at
// most wmax), and a persistent grid of `grid` blocks takes virtual blocks
// from `counter` until all are done.  Written on the device every step.
struct FlatPlan {
    int *vstart;          // nrep + 1 entries
    unsigned *counter;    // next virtual block
    int per_block;        // samples per virtual block
    int wmax;             // virtual blocks per replica at most (<= its work-array slots)
    int grid;             // blocks of the persistent sampler
};

// Issues one full time step on ctx.stream.  Returns a CUDA error code.
cudaError_t launch_step(StepCtx &ctx);

// Issues one step for nrep replicas of the same word count and precision
// whose arguments are A[0..nrep); launch counts are added to launches[7].
// With a work plan the sampler runs as one persistent launch over all of
// them, with blocks shared out in proportion to each replica's samples.
cudaError_t launch_group(const StepArgs *A, int nrep, int K, bool fp32, const Shapes &sh, bool multi_att,
                         cudaStream_t sm, i64 *launches, const cudaEvent_t *ev, const FlatPlan *plan = nullptr);

// Number of radix passes for the shapes.
int sort_passes(const Shapes &sh);

// Copies the rank-key bit count needed for a key bound.
int bits_for(u64 bound);

}  // namespace ccmc
