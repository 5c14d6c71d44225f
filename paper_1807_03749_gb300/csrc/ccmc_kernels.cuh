// ccmc_kernels.cuh -- device code of one CCMC time step (Spencer et al.,
// arXiv:1807.03749, Sec. II and Sec. IV.B-C): the building blocks a1-a10,
// the kernels templated on the determinant word count K and the precision R
// of the matrix elements, and the template that issues a whole step.  Each
// (K, R) pair is instantiated in its own translation unit
// (ccmc_step_k<K>.cu) so that the word counts compile in parallel; the
// kernels that do not depend on K are defined once, in ccmc_step.cu.
//
//  a1  k_scan_partial / k_scan_top / k_scan_final : |t_i| prefix, N_total,
//      t_HF, N_ex, n_sel, cluster amplitudes; full non-composite visits
//      (death and estimator of every list entry, Sec. IV.B)
//  a2-a5 k_sample  : cluster selection, collapse with sign, death, estimator,
//      one spawning attempt inline or the cluster queued for multi-spawn
//  a4/a6 k_attempts: expanded multi-spawn attempts (Sec. IV.C)
//  a7  k_sort_*    : LSD radix sort of spawned records by rank key
//  a8  k_seg_*     : sum of each run of equal keys
//  a9  k_merge_*   : merge into the list, occupation threshold, compaction
//  a10 k_finalize  : projected-energy numerator, per-step record
//  batch k_sample_plan / k_sample_flat: the sampler as one persistent launch
//      over many replicas, with a work plan written on the device each step
#pragma once

#include "ccmc_state.cuh"

namespace ccmc {

#define FULLMASK 0xFFFFFFFFu

// ---------------------------------------------------------------------------
// Block and warp helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(FULLMASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    return v;
}

// inclusive scan of one value per thread; sm must hold 32 elements
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T *sm, T &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) sm[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = lane < nw ? sm[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < nw) sm[lane] = wi;
    }
    __syncthreads();
    T off = wid > 0 ? sm[wid - 1] : T(0);
    total = sm[nw - 1];
    __syncthreads();
    return incl + off;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sm)
{
    T tot;
    block_incl_scan(v, sm, tot);
    return tot;
}

// compensated block reduction in a fixed tree order (deterministic): a
// shuffle tree inside each warp, then one more over the warp results, so the
// chain of dependent FP64 operations is logarithmic in the block size
__device__ __forceinline__ KSum warp_ksum(KSum k)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        KSum t;
        t.s = __shfl_xor_sync(FULLMASK, k.s, o);
        t.c = __shfl_xor_sync(FULLMASK, k.c, o);
        k.merge(t);
    }
    return k;
}

__device__ __forceinline__ KSum block_ksum(KSum k, double *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    k = warp_ksum(k);
    if (lane == 0) {
        sm[2 * wid] = k.s;
        sm[2 * wid + 1] = k.c;
    }
    __syncthreads();
    KSum r = {0.0, 0.0};
    if (wid == 0) {
        if (lane < nw) {
            r.s = sm[2 * lane];
            r.c = sm[2 * lane + 1];
        }
        r = warp_ksum(r);
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ Fix128 warp_fix(Fix128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Fix128 t;
        t.lo = __shfl_xor_sync(FULLMASK, v.lo, o);
        t.hi = __shfl_xor_sync(FULLMASK, v.hi, o);
        v.add(t);
    }
    return v;
}

// integer block sum of Fix128 values; sm holds 64 u64; the result is valid in thread 0
__device__ __forceinline__ Fix128 block_fix(Fix128 v, u64 *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_fix(v);
    if (lane == 0) {
        sm[2 * wid] = v.lo;
        sm[2 * wid + 1] = v.hi;
    }
    __syncthreads();
    Fix128 r = {0, 0};
    if (wid == 0) {
        if (lane < nw) {
            r.lo = sm[2 * lane];
            r.hi = sm[2 * lane + 1];
        }
        r = warp_fix(r);
    }
    __syncthreads();
    return r;
}

// contiguous share [lo, hi) of n elements for this block
__device__ __forceinline__ void chunk_of(i64 n, i64 &lo, i64 &hi)
{
    i64 c = (n + gridDim.x - 1) / gridDim.x;
    lo = (i64)blockIdx.x * c;
    if (lo > n) lo = n;
    hi = lo + c;
    if (hi > n) hi = n;
}

// Warp-granular chunks of a list: warp q of the grid's W warps gets
// [q c, (q + 1) c), c = ceil(n / W); its scans need no block barrier.
__device__ __forceinline__ i64 warp_chunk_of(i64 n, i64 &lo, i64 &hi)
{
    const i64 W = (i64)gridDim.x * (blockDim.x >> 5);
    const i64 q = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const i64 c = (n + W - 1) / W;
    lo = q * c < n ? q * c : n;
    hi = lo + c < n ? lo + c : n;
    return q;
}

// All 32 lanes call; returns this lane's exclusive offset in a global
// counter after reserving the warp's total with one atomic.
__device__ __forceinline__ i64 warp_reserve(i64 *counter, i64 count)
{
    const int lane = threadIdx.x & 31;
    i64 incl = warp_incl_scan(count);
    i64 total = __shfl_sync(FULLMASK, incl, 31);
    i64 base = 0;
    if (lane == 31 && total) base = (i64)atomicAdd((unsigned long long *)counter, (unsigned long long)total);
    base = __shfl_sync(FULLMASK, base, 31);
    return base + incl - count;
}

__device__ __forceinline__ u64 warp_reserve_u64(u64 *counter, u64 count)
{
    const int lane = threadIdx.x & 31;
    u64 incl = warp_incl_scan(count);
    u64 total = __shfl_sync(FULLMASK, incl, 31);
    u64 base = 0;
    if (lane == 31 && total) base = atomicAdd((unsigned long long *)counter, (unsigned long long)total);
    base = __shfl_sync(FULLMASK, base, 31);
    return base + incl - count;
}

// Every thread of the block calls; one atomic per block reserves the
// block's total and each thread receives its exclusive offset.
template <typename T>
__device__ __forceinline__ T block_reserve(T *counter, T count, T *sm, T *sbase)
{
    T tot;
    T incl = block_incl_scan(count, sm, tot);
    if (threadIdx.x == 0) *sbase = tot ? (T)atomicAdd((unsigned long long *)counter, (unsigned long long)tot) : T(0);
    __syncthreads();
    T base = *sbase;
    __syncthreads();
    return base + incl - count;
}

template <int K>
__device__ __forceinline__ Det<K> load_det(const u64 *bits, i64 cap, i64 i)
{
    Det<K> d;
#pragma unroll
    for (int w = 0; w < K; w++) d.w[w] = bits[w * cap + i];
    return d;
}

template <int K>
__device__ __forceinline__ void store_det(u64 *bits, i64 cap, i64 i, const Det<K> &d)
{
#pragma unroll
    for (int w = 0; w < K; w++) bits[w * cap + i] = d.w[w];
}

template <int K>
__device__ __forceinline__ Det<K> hf_det(const SysDev &s)
{
    Det<K> d;
#pragma unroll
    for (int w = 0; w < K; w++) d.w[w] = s.hf[w];
    return d;
}

// n_attempts = max(1, floor(|A| / A_thresh)) with multi-spawn, else 1
__device__ __forceinline__ i64 attempts_of(double amp_abs, const RunParams &p)
{
    if (!p.multispawn) return 1;
    if (p.a_thresh_one) {
        // floor(|A|) from the bit pattern (A / 1.0 == A exactly)
        u64 M;
        int E;
        split_double((u64)__double_as_longlong(amp_abs) & 0x7FFFFFFFFFFFFFFFULL, M, E);
        u64 q = E >= 0 ? (E >= 10 ? (1ULL << 62) : (M << E)) : (E <= -64 ? 0 : (M >> -E));
        return q < 1 ? 1 : (i64)q;
    }
    double q = floor(amp_abs / p.a_thresh);
    return q < 1.0 ? 1 : (i64)q;
}

// stochastic rounding of a spawned (with cutoff) or death (without) value
__device__ __forceinline__ bool round_value(double x, u64 r, const RunParams &p, bool spawn, i64 &out)
{
    if (p.int_round) return stoch_round_bits((u64)__double_as_longlong(x), r, spawn ? p.spawn_rs : p.death_rs, out);
    return stoch_round(x, unif(r), spawn ? p.spawn_cutoff : 0.0, out);
}

// the determinant of a picked entry: from its pick row (one granule with
// the prefix and population just searched) when it has at most four words
template <int K>
__device__ __forceinline__ Det<K> pick_det(const PickEntry *pk, const ListView &L, i64 id)
{
    Det<K> d;
    if constexpr (K <= 4) {
#pragma unroll
        for (int w = 0; w < K; w++) d.w[w] = __ldg(&pk[id].w[w]);
    } else {
        d = load_det<K>(L.bits, L.cap, id);
    }
    return d;
}

// smallest i in [1, n-1] with prefix[i] > x (excitor owning position x);
// the bucket of x brackets the answer between the owners of its first
// position and of the next bucket's first position
__device__ __forceinline__ i64 pick_index(const PickEntry *pk, const int *bucket, int shift, i64 nbuckets, i64 n,
                                          u64 x)
{
    i64 b = (i64)(x >> shift);
    i64 lo = __ldg(&bucket[b]);
    i64 hi = b + 1 < nbuckets ? __ldg(&bucket[b + 1]) : n - 1;
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if ((u64)__ldg(&pk[mid].prefix) > x) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Simulated distribution (Sec. III): the excitor of processor q holding
// position x in [0, N_q) of that processor's entries in list order -- the
// chunk whose processor-q prefix brackets x, then a walk over the chunk;
// -1 only if the tables were inconsistent
__device__ __forceinline__ i64 local_pick(const WorkArrays &wa, const PickEntry *pk, i64 n, int lcs, i64 nlc, u64 q,
                                          u64 x)
{
    const i64 *row = wa.lcp + (i64)q * nlc;
    i64 lo = 0, hi = nlc - 1;   // last chunk c with row[c] <= x
    while (lo < hi) {
        const i64 mid = (lo + hi + 1) >> 1;
        if ((u64)__ldg(&row[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    u64 acc = (u64)__ldg(&row[lo]);
    const i64 b = lo << lcs, e = b + (1LL << lcs) < n ? b + (1LL << lcs) : n;
    for (i64 i = b > 1 ? b : 1; i < e; i++) {
        if (__ldg(&wa.owner[i]) != q) continue;
        const i64 v = __ldg(&pk[i].pop);
        acc += (u64)(v < 0 ? -v : v);
        if (acc > x) return i;
    }
    return -1;
}

// smallest i in [lo, hi] with end[i] > t (the answer is known to lie there)
__device__ __forceinline__ i64 owner_in(const i64 *end, i64 lo, i64 hi, i64 t)
{
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (__ldg(&end[mid]) > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Attempt ranges: entry e owns attempts [end[e-1], end[e]) with end strictly
// increasing (every entry has at least one attempt), so 32 consecutive
// entries always cover 32 consecutive attempts.  A warp walks a contiguous
// chunk of attempts with a sliding window of 32 entry ends (one coalesced
// load per 32 attempts) and finds each lane's owner by a 5-step search over
// the window held in registers.
struct AttemptWindow {
    i64 cur;      // owner of the first attempt of the current 32
    i64 prev;     // end[cur - 1] (0 when cur == 0)
};

__device__ __forceinline__ AttemptWindow window_start(const i64 *end, i64 n, i64 t0)
{
    const int lane = threadIdx.x & 31;
    AttemptWindow w;
    i64 c = lane == 0 ? owner_in(end, 0, n - 1, t0) : 0;
    w.cur = __shfl_sync(FULLMASK, c, 0);
    i64 pv = (lane == 0 && w.cur > 0) ? end[w.cur - 1] : 0;
    w.prev = __shfl_sync(FULLMASK, pv, 0);
    return w;
}

// owner and attempt number of t = t0 + lane; advances the window past t0 + 31
__device__ __forceinline__ void window_step(const i64 *end, i64 n, i64 t0, AttemptWindow &w, i64 &owner, i64 &m)
{
    const int lane = threadIdx.x & 31;
    const i64 t = t0 + lane;
    const i64 e = w.cur + lane;
    const i64 ev = e < n ? __ldg(&end[e]) : 0x7FFFFFFFFFFFFFFFLL;
    int L = 0;
#pragma unroll
    for (int st = 16; st >= 1; st >>= 1) {
        i64 v = __shfl_sync(FULLMASK, ev, L + st - 1);
        if (v <= t) L += st;
    }
    i64 before = __shfl_sync(FULLMASK, ev, L > 0 ? L - 1 : 0);
    owner = w.cur + L;
    m = t - (L > 0 ? before : w.prev);
    // entries whose attempts all lie before t0 + 32 are finished; the next
    // window starts at the owner of attempt t0 + 32
    unsigned done = __ballot_sync(FULLMASK, ev <= t0 + 32);
    int adv = __popc(done);
    if (adv > 0) w.prev = __shfl_sync(FULLMASK, ev, adv - 1);
    w.cur += adv;
}

// first i in [0, n) with keys[i] >= k (n if none)
__device__ __forceinline__ i64 lower_bound_key(const u64 *keys, i64 n, u64 k)
{
    i64 lo = 0, hi = n;
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (__ldg(&keys[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One spawning attempt from dj carrying coefficient c_att (Sec. II):
// value -dtau H_ij c_att s_D(i) / p_gen, stochastically rounded.
// A spawning attempt in two halves.  attempt_draw runs the excitation
// generator and the truncation check (about nine draws in ten end here for
// the gas); attempt_finish computes the matrix element, the value, its
// stochastic rounding and the rank key.  The expanded-attempt kernel queues
// the surviving draws and finishes them 32 at a time, so the second half
// runs on full warps.
// the drawn excitation (holes i, j and particles a, b: 16 bits each, M <= 384)
template <int K>
__device__ __forceinline__ bool attempt_draw(const SysDev &s, const Det<K> &dj, const R4 &r, u64 &code, int &gc)
{
    Det<K> di;
    int nh, i, j, a, b;
    if (!excite(s, dj, r, di, nh, i, j, a, b, gc)) return false;
    if (level_of(s, di) > s.lmax) return false;
    code = (u64)i | ((u64)j << 16) | ((u64)a << 32) | ((u64)b << 48);
    return true;
}

template <int K, typename R>
__device__ __forceinline__ bool attempt_finish(const SysDev &s, const RunParams &p, const Det<K> &dj, double c_att,
                                               u64 r3, u64 code, int gc, u64 &key, i64 &val, unsigned &err)
{
    const int i = (int)(code & 0xFFFF), j = (int)((code >> 16) & 0xFFFF), a = (int)((code >> 32) & 0xFFFF),
              b = (int)(code >> 48);
    const int nh = (gc == 1 || gc == 2) ? 1 : 2;
    Det<K> di = dj;
    flip(di, i);
    if (nh == 2) flip(di, j);
    flip(di, a);
    if (nh == 2) flip(di, b);
    // matrix element and 1/p_gen in the precision R; the value itself in FP64
    double h = h_offdiag<K, R>(s, dj, nh, i, j, a, b);
    double x = ((p.tau * h) * inv_pgen_of<R>(s, gc)) * c_att;
    if (excitor_sign(s, di) > 0) x = -x;
    i64 v;
    if (!round_value(x, r3, p, true, v)) {
        err |= ERRB_NUMERIC;
        return false;
    }
    if (v == 0) return false;
    key = rank_key(s, di);
    val = v;
    return true;
}

// Per-warp queue of drawn attempts waiting for attempt_finish.
template <int K>
struct AttQueue {
    u64 det[K][64];
    double c[64];
    u64 r[64];
    u64 code[64];
    unsigned char gc[64];
};

// All 32 lanes call; lanes with ok append their attempt (qn < 32 on entry).
template <int K>
__device__ __forceinline__ void q_push(AttQueue<K> &q, int &qn, bool ok, const Det<K> &dj, double c, u64 r3, u64 code,
                                       int gc)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(FULLMASK, ok);
    if (ok) {
        const int e = qn + __popc(m & ((1u << lane) - 1u));
#pragma unroll
        for (int w = 0; w < K; w++) q.det[w][e] = dj.w[w];
        q.c[e] = c;
        q.r[e] = r3;
        q.code[e] = code;
        q.gc[e] = (unsigned char)gc;
    }
    qn += __popc(m);
    __syncwarp();
}

// Per-warp staging of spawned records: appended by ballot, written to the
// spawn buffer 32 at a time (one atomic per 32 records, 256-byte runs).
struct RecStage {
    u64 key[64];
    i64 val[64];
};

// All 32 lanes call; lanes with has append their record (rn < 32 on entry).
__device__ __forceinline__ void rec_push(RecStage &rs, int &rn, bool has, u64 k, i64 v)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(FULLMASK, has);
    if (has) {
        const int e = rn + __popc(m & ((1u << lane) - 1u));
        rs.key[e] = k;
        rs.val[e] = v;
    }
    rn += __popc(m);
    __syncwarp();
}

// Direct accumulation (annihilation fast path): a spawned record whose key
// is already in the sorted excip list is added to that entry's matched-spawn
// sum with an integer atomic instead of going through the sort; only keys new
// to the list are appended to the spawn buffer.  Integer sums make the merged
// list identical either way.  The key buckets (entries whose key >> kshift
// equals b start at kbucket[b]) narrow each search to a few entries.
struct DirectView {
    const u64 *key;      // the list's keys, ascending
    const int *kb;       // key buckets
    i64 *acc;            // matched-spawn sums per entry
    unsigned char *hit;  // entries that received a direct record
    i64 n, nkb;          // list size, buckets in use (0: off)
    int ks;              // key-bucket shift
};

__device__ __forceinline__ DirectView direct_view(const ListView &L, const WorkArrays &wa, const DevStep *st)
{
    DirectView d;
    d.key = L.key;
    d.kb = wa.kbucket;
    d.acc = wa.acc;
    d.hit = wa.hit;
    d.n = st->n_occ;
    d.nkb = st->nkb;
    d.ks = st->kshift;
    return d;
}

// index of key k in the list, or -1
__device__ __forceinline__ i64 find_key(const DirectView &d, u64 k)
{
    const u64 b = k >> d.ks;
    if (b >= (u64)d.nkb) return -1;
    i64 lo = __ldg(&d.kb[b]);
    i64 hi = b + 1 < (u64)d.nkb ? (i64)__ldg(&d.kb[b + 1]) : d.n;
    while (lo < hi) {
        const i64 mid = lo + (hi - lo) / 2;
        if (__ldg(&d.key[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return (lo < d.n && __ldg(&d.key[lo]) == k) ? lo : -1;
}

// All 32 lanes call: takes the newest 32 staged records while 32 or more are
// waiting (with all, every staged record); records onto listed determinants
// are added to them directly, the others appended to the spawn buffer with
// one atomic per warp.
__device__ __forceinline__ void rec_flush(RecStage &rs, int &rn, bool all, DevStep *st, const SpawnBuf &sp,
                                          const DirectView &dv, i64 &ndirect, unsigned &err)
{
    const int lane = threadIdx.x & 31;
    while (rn >= 32 || (all && rn > 0)) {
        const int take = rn >= 32 ? 32 : rn;
        const bool have = lane < take;
        u64 k = 0;
        i64 v = 0;
        if (have) {
            const int e = rn - take + lane;
            k = rs.key[e];
            v = rs.val[e];
        }
        __syncwarp();   // the stage is read before later pushes reuse it
        rn -= take;
        bool app = have;
        if (have && dv.nkb > 0) {
            const i64 pos = find_key(dv, k);
            if (pos >= 0) {
                atomicAdd((unsigned long long *)&dv.acc[pos], (unsigned long long)v);
                dv.hit[pos] = 1;
                ndirect++;
                app = false;
            }
        }
        const unsigned m = __ballot_sync(FULLMASK, app);
        if (m == 0) continue;
        i64 base = 0;
        if (lane == 0) base = (i64)atomicAdd((unsigned long long *)&st->n_sp, (unsigned long long)__popc(m));
        base = __shfl_sync(FULLMASK, base, 0);
        if (app) {
            const i64 off = base + __popc(m & ((1u << lane) - 1u));
            if (off < sp.cap) {
                sp.key[0][off] = k;
                sp.pop[0][off] = v;
            } else {
                err |= ERRB_SPAWN_OVERFLOW;
            }
        }
    }
}

// All 32 lanes call: finishes the newest 32 queued attempts while 32 or more
// are waiting (with all, every waiting attempt) into the record stage.
template <int K, typename R>
__device__ __forceinline__ void q_drain_staged(AttQueue<K> &q, int &qn, bool all, RecStage &rs, int &rn,
                                               const SysDev &s, const RunParams &p, DevStep *st, const SpawnBuf &sp,
                                               const DirectView &dv, i64 &ndirect, unsigned &err)
{
    const int lane = threadIdx.x & 31;
    while (qn >= 32 || (all && qn > 0)) {
        const int take = qn >= 32 ? 32 : qn;
        bool has = false;
        u64 k = 0;
        i64 v = 0;
        if (lane < take) {
            const int e = qn - take + lane;
            Det<K> dj;
#pragma unroll
            for (int w = 0; w < K; w++) dj.w[w] = q.det[w][e];
            has = attempt_finish<K, R>(s, p, dj, q.c[e], q.r[e], q.code[e], q.gc[e], k, v, err);
        }
        __syncwarp();   // the entries are read before later pushes reuse them
        qn -= take;
        rec_push(rs, rn, has, k, v);
        rec_flush(rs, rn, false, st, sp, dv, ndirect, err);
    }
}

// occupation threshold: 0 < |v| < 1 becomes +-1 with probability |v|, else 0
__device__ __forceinline__ i64 threshold(const RunParams &p, u64 it, u64 key, i64 v)
{
    i64 av = v < 0 ? -v : v;
    if (av > 0 && av < (i64)FIX_ONE) {
        R4 r = draw(p.seed, p.replica, it, TAG_THRESH, key, 0);
        bool keep = (r.v[0] >> 11) < ((u64)av << 37);
        return keep ? (v < 0 ? -(i64)FIX_ONE : (i64)FIX_ONE) : 0;
    }
    return v;
}

// ---------------------------------------------------------------------------
// a1: scans over the list
// ---------------------------------------------------------------------------

__device__ __forceinline__ void d_scan_partial(const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa)
{
    i64 n = st->n_occ, lo, hi;
    const i64 q = warp_chunk_of(n, lo, hi);
    i64 sw = 0, sa = 0;
    for (i64 i = lo + (threadIdx.x & 31); i < hi; i += 32) {
        i64 v = L.pop[i], av = v < 0 ? -v : v;
        if (i > 0) sw += av;
        if (p.fnc) sa += attempts_of(fabs((double)v / FIX_ONE), p);
    }
    sw = warp_sum(sw);
    sa = warp_sum(sa);
    if ((threadIdx.x & 31) == 0) {
        wa.wpart[4 * q] = sw;
        wa.wpart[4 * q + 1] = sa;
    }
}

// Exclusive prefixes of W warp partials (wpart[4 (off + q) + f] into
// wpart[4 (off + q) + f + 2]) by one block of 1024 threads: warp v takes a
// contiguous run, read 32 at a time (coalesced); the warps' totals are scanned
// in shared memory.  Returns the grand total (every thread).
__device__ __forceinline__ i64 partials_prefix(i64 *wpart, int off, int W, int f)
{
    __shared__ i64 s_tot[32];
    __shared__ i64 s_all;
    const int lane = threadIdx.x & 31, v = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int S = 32 * ((W + blockDim.x - 1) / blockDim.x);
    const int s0 = v * S < W ? v * S : W, s1 = s0 + S < W ? s0 + S : W;
    i64 tot = 0;
    for (int j = s0; j < s1; j += 32) {
        const int q = j + lane;
        tot += warp_sum(q < s1 ? wpart[4 * (off + q) + f] : (i64)0);
    }
    __syncthreads();   // s_tot is free (an earlier call may still read it)
    if (lane == 0) s_tot[v] = tot;
    __syncthreads();
    if (v == 0) {
        const i64 x = lane < nwarp ? s_tot[lane] : 0;
        const i64 incl = warp_incl_scan(x);
        if (lane < nwarp) s_tot[lane] = incl - x;
        if (lane == 31) s_all = incl;
    }
    __syncthreads();
    i64 carry = s_tot[v];
    for (int j = s0; j < s1; j += 32) {
        const int q = j + lane;
        const i64 x = q < s1 ? wpart[4 * (off + q) + f] : 0;
        const i64 incl = warp_incl_scan(x);
        if (q < s1) wpart[4 * (off + q) + f + 2] = carry + incl - x;
        carry += __shfl_sync(FULLMASK, incl, 31);
    }
    return s_all;
}

// one block of 1024 threads over the W = grid x warps-per-block partials of
// the warp-granular chunks
__device__ __forceinline__ void d_scan_top(const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa, int grid, int lmax)
{
    const int t = threadIdx.x;
    const int W = grid * (SCAN_THREADS / 32);
    const i64 tw = partials_prefix(wa.wpart, 0, W, 0);
    i64 ta = p.fnc ? partials_prefix(wa.wpart, 0, W, 1) : 0;
    if (t == 0) {
        i64 n0 = st->n_occ > 0 ? L.pop[0] : 0;
        i64 an0 = n0 < 0 ? -n0 : n0;
        i64 ntot = an0 + tw;
        i64 n_sel = (ntot + 32768) >> 16;
        // a runaway population: abandon the step instead of sampling it
        if (n_sel > p.work_cap || (p.fnc && ta > p.work_cap)) {
            atomicOr(&st->err, (unsigned)ERRB_RUNAWAY);
            n_sel = 0;
            ta = 0;
        }
        st->n0 = n0;
        st->ntot = ntot;
        st->nex = tw;
        // selection buckets: the smallest power of two 2^k with N_ex <= 2^(k + bucket_bits)
        // about two buckets per list entry (bounded by the bucket array)
        int bb = 4;
        while (bb < wa.bucket_bits && (1LL << bb) < 2 * st->n_occ) bb++;
        int k = 0;
        while (k < 62 && ((u64)tw >> (k + bb)) != 0) k++;
        st->bucket_shift = k;
        st->nbuckets = tw > 0 ? (i64)(((u64)tw + (1ULL << k) - 1) >> k) : 0;
        st->n_sel = n_sel;
        st->fnc_attempts = p.fnc ? ta : 0;
        // key buckets for direct accumulation: about two per list entry over
        // the list's key range, within the table's capacity
        st->n_direct = 0;
        st->n_hit = 0;
        // direct accumulation pays once the step spawns more than about one
        // record per ten list entries (the buckets cost a pass over the
        // list, a sorted record several); the choice follows the previous
        // step and does not change any result
        if (p.direct && st->n_occ > 0 && 10 * st->prev_spawned > st->n_occ) {
            const u64 kmax = L.key[st->n_occ - 1];
            i64 want = 2 * st->n_occ;
            if (want > (1LL << wa.kbucket_bits)) want = 1LL << wa.kbucket_bits;
            int ks = 0;
            while (ks < 63 && (i64)(kmax >> ks) + 1 > want) ks++;
            st->kshift = ks;
            st->nkb = (i64)(kmax >> ks) + 1;
        } else {
            st->kshift = 0;
            st->nkb = 0;
        }
        // |A_s| = N_ex^s / (|t_HF|^(s-1) n_sel p(s) s!), fixed operation order
        double nex_d = (double)tw / FIX_ONE;
        double n0_d = (double)an0 / FIX_ONE;
        int smax = lmax + 2;
        for (int s = 0; s < 8; s++) {
            st->mag[s] = 0.0;
            st->mden[s] = 0.0;
        }
        for (int s = 0; s <= smax && n_sel > 0; s++) {
            double pr;
            if (p.fnc) {
                if (s < 2) continue;
                pr = s < smax ? ldexp(1.0, -(s - 1)) : ldexp(1.0, -lmax);
            } else {
                pr = s < smax ? ldexp(1.0, -(s + 1)) : ldexp(1.0, -(lmax + 2));
            }
            if (s == 0) {
                st->mag[0] = n0_d / ((double)n_sel * pr);
                continue;
            }
            double num = 1.0, den = 1.0, fact = 1.0;
            for (int e = 0; e < s; e++) num = num * nex_d;
            for (int e = 0; e < s - 1; e++) den = den * n0_d;
            for (int e = 2; e <= s; e++) fact = fact * (double)e;
            den = den * (double)n_sel;
            den = den * pr;
            den = den * fact;
            st->mag[s] = num / den;
            st->mden[s] = den;
        }
        // simulated distribution: chunks of 2^lcs entries, as fine as the
        // per-processor position table allows
        if (p.nranks > 1) {
            const i64 n = st->n_occ;
            int c = 5;
            while (c < 40 && (i64)p.nranks * ((n + (1LL << c) - 1) >> c) > wa.lcp_cap) c++;
            st->lcs = c;
            st->nlc = (n + (1LL << c) - 1) >> c;
        }
        // every cluster of size s has |A| = mag[s]: its attempt count and
        // the magnitude of one attempt's coefficient, once per step
        for (int s = 0; s < 8; s++) {
            const i64 na = attempts_of(st->mag[s], p);
            st->natt_s[s] = na;
            st->cmag[s] = na > 1 ? st->mag[s] / (double)na : st->mag[s];
        }
        st->n_sp = 0;
        st->cl_packed = 0;
        st->cl_att = 0.0;
        st->n_attempts = 0;
        st->n_keys = 0;
        st->kept_list = 0;
        st->kept_new = 0;
        st->ntot_after = 0;
    }
}

// prefix arrays; with full non-composite sampling also every visit's death,
// estimator contribution and attempt coefficient (Sec. IV.B)
template <int K, typename R>
__device__ __forceinline__ void d_scan_final(const SysDev &s, const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa)
{
    __shared__ u64 smf[64];
    i64 n = st->n_occ, lo, hi;
    const i64 q = warp_chunk_of(n, lo, hi);
    i64 cw = wa.wpart[4 * q + 2], ca = wa.wpart[4 * q + 3];
    const u64 it = st->iter;
    const double S = st->shift;
    Fix128 es = {0, 0};
    unsigned err = 0;
    const bool kb = st->nkb > 0;
    // each warp scans its own chunk 32 entries at a time (no block barrier)
    for (i64 base = lo; base < hi; base += 32) {
        i64 i = base + (threadIdx.x & 31);
        bool ok = i < hi;
        // every read of the entry is issued before the warp scans, so that
        // one memory latency per tile is exposed instead of two
        i64 v = ok ? L.pop[i] : 0, av = v < 0 ? -v : v;
        const u64 key_i = ok && kb ? L.key[i] : 0, key_p = ok && kb && i > 0 ? L.key[i - 1] : 0;
        const double diag_i = ok && i > 0 ? L.diag[i] : 0.0;
        Det<K> d;
        if (ok) d = load_det<K>(L.bits, L.cap, i);
        i64 w = (ok && i > 0) ? av : 0;
        double amp = (double)v / FIX_ONE;
        i64 na = (ok && p.fnc) ? attempts_of(fabs(amp), p) : 0;
        i64 ta = 0, ia = 0;
        const i64 iw = warp_incl_scan(w);
        const i64 tw = __shfl_sync(FULLMASK, iw, 31);
        if (p.fnc) {   // attempt prefix: full non-composite visits only
            ia = warp_incl_scan(na);
            ta = __shfl_sync(FULLMASK, ia, 31);
        }
        if (ok) {
            PickEntry pe;
            pe.prefix = cw + iw;
            pe.pop = v;
            pe.href = 0.0;
            if (i > 0 && w > 0) {
                // buckets whose first position falls in [prefix[i-1], prefix[i]) start at entry i
                const int k = st->bucket_shift;
                u64 p0 = (u64)(cw + iw - w), p1 = (u64)(cw + iw);
                u64 b0 = (p0 + (1ULL << k) - 1) >> k, b1 = (p1 + (1ULL << k) - 1) >> k;
                for (u64 b = b0; b < b1; b++) wa.bucket[b] = (int)i;
            }
            wa.acc[i] = 0;
            wa.before[i] = 0;
            if (kb) {
                // buckets whose first key falls in (key[i-1], key[i]] start at entry i
                const int ks = st->kshift;
                const u64 b0 = i == 0 ? 0 : (key_p >> ks) + 1, b1 = key_i >> ks;
                for (u64 b = b0; b <= b1; b++) wa.kbucket[b] = (int)i;
                wa.hit[i] = 0;
            }
            const double td = p.tau * ((i == 0 ? 0.0 : diag_i) - S);
            pe.tdeath = td;
            i64 dv = 0;
            if (p.fnc) {
                wa.att_end[i] = ca + ia;
                int sd = excitor_sign(s, d);
                double coef = sd > 0 ? amp : -amp;
                int lev = level_of(s, d);
                if (lev == 1 || lev == 2) es.add(to_fix(h_ref<K, R>(s, d) * coef));
                R4 r = draw(p.seed, p.replica, it, TAG_VISIT, (u64)i, 0);
                double x = td * coef;
                if (sd > 0) x = -x;
                if (!round_value(x, r.v[0], p, false, dv)) err |= ERRB_NUMERIC;
                wa.catt[i] = na > 1 ? coef / (double)na : coef;
            } else {
                // <HF|H|D_i> for the single-excitor clusters of the sampler
                const int lev = level_of(s, d);
                pe.href = (lev == 1 || lev == 2) ? h_ref<K, R>(s, d) : 0.0;
            }
            // the words ride in the row a pick reads anyway (up to four)
#pragma unroll
            for (int q = 0; q < 4; q++) pe.w[q] = q < K ? d.w[q < K ? q : 0] : 0;
            wa.picks[i] = pe;
            wa.death[i] = dv;
        }
        cw += tw;
        ca += ta;
    }
    es = block_fix(es, smf);
    if (threadIdx.x == 0) {
        wa.enum_part[2 * blockIdx.x] = es.lo;
        wa.enum_part[2 * blockIdx.x + 1] = es.hi;
    }
    if (err) atomicOr(&st->err, err);   // every thread reports its own bits
}

// Simulated distribution (Sec. III): the owner of every excitor at this
// iteration (Eq. ccmc_dist) and, per chunk of 2^lcs list entries, the |pop|
// each processor holds in it; one warp per chunk, which clears its column of
// the table first (integer sums: the table does not depend on the order)
template <int K>
__device__ __forceinline__ void d_local_table(const ListView &L, const DevStep *st, const RunParams &p, const WorkArrays &wa)
{
    if (p.nranks <= 1) return;
    const i64 n = st->n_occ, nlc = st->nlc;
    const int lcs = st->lcs, lane = threadIdx.x & 31;
    const u64 it = st->iter;
    const i64 nw = (i64)gridDim.x * (blockDim.x / 32);
    for (i64 c = (i64)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); c < nlc; c += nw) {
        for (i64 q = lane; q < p.nranks; q += 32) wa.lcp[q * nlc + c] = 0;
        __syncwarp();
        const i64 b = c << lcs, e = b + (1LL << lcs) < n ? b + (1LL << lcs) : n;
        for (i64 i = b + lane; i < e; i += 32) {
            if (i == 0) continue;   // the reference is not an excitor
            const Det<K> d = load_det<K>(L.bits, L.cap, i);
            const u64 q = words_owner(d.w, K, it, p.nu_move, (u64)p.nranks);
            wa.owner[i] = (unsigned short)q;
            const i64 v = L.pop[i];
            atomicAdd((unsigned long long *)&wa.lcp[(i64)q * nlc + c], (unsigned long long)(v < 0 ? -v : v));
        }
        __syncwarp();
    }
}

// each processor's row of the table turned into exclusive prefixes over the
// chunks; its total is N_q
__device__ __forceinline__ void d_local_scan(const DevStep *st, const RunParams &p, const WorkArrays &wa)
{
    __shared__ i64 sm[32];
    if (p.nranks <= 1) return;
    const i64 nlc = st->nlc;
    for (i64 q = blockIdx.x; q < p.nranks; q += gridDim.x) {
        i64 *row = wa.lcp + q * nlc;
        i64 carry = 0;
        for (i64 base = 0; base < nlc; base += blockDim.x) {
            const i64 c = base + threadIdx.x;
            const i64 v = c < nlc ? row[c] : 0;
            i64 tot;
            const i64 incl = block_incl_scan(v, sm, tot);
            if (c < nlc) row[c] = carry + incl - v;
            carry += tot;
        }
        if (threadIdx.x == 0) wa.nq[q] = carry;
    }
}

// ---------------------------------------------------------------------------
// a2-a5: cluster sampling (Sec. II; composites only with FNC, Sec. IV.B)
// ---------------------------------------------------------------------------

// DIST: the simulated distribution's restricted composite draw is compiled
// in (a separate instantiation keeps it out of the plain sampler's loop)
template <int K, typename R, bool DIST>
__device__ __forceinline__ void d_sample(const SysDev &s, const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa,
                                                         const SpawnBuf &sp, const ClusterBuf &cl, int enum_base,
                                                         int vb, int vg)
{
    __shared__ double smag[8], scmag[8], smden[8];
    __shared__ i64 snatt[8];
    __shared__ u64 smf[64];
    __shared__ i64 sm[32];
    // per-warp queues: drawn spawning attempts waiting for attempt_finish,
    // and spawned records waiting to be written 32 at a time
    __shared__ AttQueue<K> aq[WORK_THREADS / 32];
    __shared__ RecStage rsb[WORK_THREADS / 32];
    if (threadIdx.x < 8) {
        smag[threadIdx.x] = st->mag[threadIdx.x];
        scmag[threadIdx.x] = st->cmag[threadIdx.x];
        snatt[threadIdx.x] = st->natt_s[threadIdx.x];
        smden[threadIdx.x] = st->mden[threadIdx.x];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    AttQueue<K> &q = aq[wid];
    RecStage &rb = rsb[wid];
    int qn = 0, rn = 0;   // warp-uniform queue fills
    const i64 n_sel = st->n_sel, n = st->n_occ, nex = st->nex, n0 = st->n0;
    const int bshift = st->bucket_shift;
    const i64 nbk = st->nbuckets;
    const int lcs = st->lcs;
    const i64 nlc = st->nlc;
    const u64 it = st->iter;
    const double S = st->shift;
    Fix128 es = {0, 0};
    unsigned err = 0;
    i64 inline_att = 0;
    u64 cl_att = 0;        // attempts of the clusters this thread buffers
    i64 death_hf = 0;      // reference-cluster deaths, summed per block at the end
    i64 ndirect = 0;       // records added directly to listed determinants
    const DirectView dv = direct_view(L, wa, st);
    const PickEntry *pk = wa.picks;
    // each warp runs its 32 samples of every block tile on its own: the
    // appends are staged per warp, so no block barrier is needed in the loop
    for (i64 g0 = (i64)vb * blockDim.x + 32 * wid; g0 < n_sel; g0 += (i64)vg * blockDim.x) {
        const i64 g = g0 + lane;
        bool rec = false;       // a composite death record
        u64 rk = 0;
        i64 rv = 0;
        bool valid_cl = false;  // a cluster that makes spawning attempts
        Det<K> dj;
        double coef = 0.0, catt = 0.0;
        i64 natt = 0;
        if (g < n_sel) {
            R4 r0 = draw(p.seed, p.replica, it, TAG_SAMPLE, (u64)g, 0);
            u64 nr = ~r0.v[0];
            int lz = nr ? __clzll((long long)nr) : 64;
            int sz = p.fnc ? 2 + min(lz, s.lmax) : min(lz, s.lmax + 2);
            bool valid = true;
            int par = 0;
            i64 idx0 = 0;
            double amp = 0.0;
            dj = hf_det<K>(s);
            if (sz == 0) {
                amp = n0 < 0 ? -smag[0] : smag[0];
            } else if (nex == 0 || (sz >= 2 && n0 == 0) || sz * s.lmin_exc > s.lmax + 2) {
                // the last test: a valid cluster's level is the sum of its
                // excitors' levels, so this size cannot stay within l + 2
                // and the sample contributes nothing (its picks are skipped)
                valid = false;
            } else {
                R4 r1;
                if (sz > 2) r1 = draw(p.seed, p.replica, it, TAG_SAMPLE, (u64)g, 1);
                i64 idx[6];
                int neg = 0;
                // simulated distribution: a composite's later excitors come
                // from the first one's processor q (Sec. III)
                const bool local = DIST && p.nranks > 1 && sz >= 2;
                i64 nq = 0;
                if (!local) {
                    // the picks are independent: issue all searches before using them
                    for (int e = 0; e < sz; e++) {
                        u64 rr = e < 2 ? r0.v[2 + e] : r1.v[e - 2];
                        idx[e] = pick_index(pk, wa.bucket, bshift, nbk, n, below(rr, (u64)nex));
                    }
                } else {
                    idx[0] = pick_index(pk, wa.bucket, bshift, nbk, n, below(r0.v[2], (u64)nex));
                    const u64 q = __ldg(&wa.owner[idx[0]]);
                    nq = __ldg(&wa.nq[q]);
                    for (int e = 1; e < sz; e++) {
                        u64 rr = e < 2 ? r0.v[2 + e] : r1.v[e - 2];
                        idx[e] = local_pick(wa, pk, n, lcs, nlc, q, below(rr, (u64)nq));
                        if (idx[e] < 0) {   // tables inconsistent (cannot happen): a sticky error, not a guess
                            valid = false;
                            err |= ERRB_NUMERIC;
                        }
                    }
                }
                for (int e = 1; e < sz; e++)
                    for (int f = 0; f < e; f++)
                        if (idx[f] == idx[e]) valid = false;   // repeated excitor: discarded
                if (sz == 1) {
                    // one excitor: its own determinant, with the sign s_D of
                    // applying it to HF (the closed form of the same product)
                    const i64 id = idx[0];
                    if (__ldg(&pk[id].pop) < 0) neg ^= 1;
                    dj = pick_det<K>(pk, L, id);
                    par = excitor_sign(s, dj) < 0 ? 1 : 0;
                } else {
                    for (int e = 0; e < sz && valid; e++) {
                        const i64 id = idx[e];
                        if (__ldg(&pk[id].pop) < 0) neg ^= 1;
                        const Det<K> de = pick_det<K>(pk, L, id);
                        if (!apply_excitor(s, de, dj, par)) valid = false;   // shared orbital
                    }
                }
                if (valid) {
                    if (n0 < 0 && ((sz - 1) & 1)) neg ^= 1;
                    double a = smag[sz];
                    if (local) {
                        // |A| = N_ex (N_q N_p)^(s-1) / (|t_HF|^(s-1) n_sel p(s) s!):
                        // selection within q times co-location N_p^-(s-1)
                        const double f = ((double)nq / FIX_ONE) * (double)p.nranks;
                        double num = (double)nex / FIX_ONE;
                        for (int e = 1; e < sz; e++) num = num * f;
                        a = num / smden[sz];
                    }
                    amp = neg ? -a : a;
                    idx0 = idx[0];
                }
            }
            int lev = valid ? level_of(s, dj) : 0;
            if (valid && lev <= s.lmax + 2) {
                coef = (par & 1) ? -amp : amp;
                // a single excitor collapses to its own determinant: <HF|H|D> cached per entry
                if (lev == 1 || lev == 2)
                    es.add(to_fix((sz == 1 && !p.fnc ? __ldg(&pk[idx0].href) : h_ref<K, R>(s, dj)) * coef));
                // s_D of the collapsed determinant (HF: +1; one excitor: known)
                const int sdj = sz == 0 ? 1 : (sz == 1 ? ((par & 1) ? -1 : 1) : excitor_sign(s, dj));
                if (sz <= 1) {
                    double x = __ldg(&pk[idx0].tdeath) * coef;   // tau (Delta E - S) C (idx0 = 0 for the reference)
                    if (sdj > 0) x = -x;
                    i64 dv;
                    if (!round_value(x, r0.v[1], p, false, dv)) err |= ERRB_NUMERIC;
                    if (dv != 0) {
                        if (idx0 == 0) death_hf += dv;   // hot entry: one atomic per block below
                        else atomicAdd((unsigned long long *)&wa.death[idx0], (unsigned long long)dv);
                    }
                } else if (lev <= s.lmax) {
                    double x = (p.tau * (diag_rel<K, R>(s, dj) - S)) * coef;
                    if (sdj > 0) x = -x;
                    i64 dv;
                    if (!round_value(x, r0.v[1], p, false, dv)) err |= ERRB_NUMERIC;
                    if (dv != 0) {
                        rk = rank_key(s, dj);
                        rv = dv;
                        rec = true;
                    }
                }
                // = attempts_of(|amp|): |amp| = mag[sz] for every cluster of
                // size sz, unless its processor's population sets it
                const bool local_amp = DIST && p.nranks > 1 && sz >= 2;
                natt = local_amp ? attempts_of(fabs(amp), p) : snatt[sz];
                valid_cl = true;
                if (p.buffered) {
                    catt = coef;    // the original sampler's one attempt
                    cl_att += 1;
                } else if (p.multispawn) {
                    // coef / natt: the same division, done once per size
                    if (local_amp) catt = natt > 1 ? coef / (double)natt : coef;
                    else catt = natt > 1 ? (coef < 0.0 ? -scmag[sz] : scmag[sz]) : coef;
                    if (natt > p.work_cap) {   // runaway: the attempts kernel will not run them
                        err |= ERRB_RUNAWAY;
                        natt = p.work_cap + 1;
                    }
                    cl_att += (u64)natt;
                }
            }
        }
        rec_push(rb, rn, rec, rk, rv);
        rec_flush(rb, rn, false, st, sp, dv, ndirect, err);   // the stage holds fewer than 32 again
        if (p.multispawn || p.buffered) {
            // the cluster is queued for the attempts kernel: multi-spawn
            // packs (clusters << CL_SHIFT | attempts) into one counter; the
            // original sampler's one attempt per cluster counts clusters only
            u64 mine = valid_cl ? (p.buffered ? 1ULL : ((1ULL << CL_SHIFT) | (u64)natt)) : 0ULL;
            u64 o = warp_reserve_u64(&st->cl_packed, mine);
            if (valid_cl) {
                const i64 c = p.buffered ? (i64)o : (i64)(o >> CL_SHIFT);
                if (c < cl.cap) {
                    store_det<K>(cl.bits, cl.cap, c, dj);
                    cl.catt[c] = catt;
                    cl.index[c] = (u64)g;
                    cl.end[c] = p.buffered ? c + 1 : (i64)(o & CL_MASK) + natt;
                } else {
                    err |= ERRB_CLUSTER_OVERFLOW;
                }
            }
        } else {
            // one attempt per valid cluster, drawn and generated with the
            // valid lanes together; the few that survive the generator and
            // the truncation wait in the queue and are finished 32 at a time
            bool ok = false;
            u64 code = 0;
            int gc = 0;
            u64 r3 = 0;
            if (valid_cl) {
                inline_att++;
                R4 ra = draw(p.seed, p.replica, it, TAG_SAMPLE_ATT, (u64)g, 0);
                ok = attempt_draw<K>(s, dj, ra, code, gc);
                r3 = ra.v[3];
            }
            q_push<K>(q, qn, ok, dj, coef, r3, code, gc);
            q_drain_staged<K, R>(q, qn, false, rb, rn, s, p, st, sp, dv, ndirect, err);
        }
        rec_flush(rb, rn, false, st, sp, dv, ndirect, err);
    }
    q_drain_staged<K, R>(q, qn, true, rb, rn, s, p, st, sp, dv, ndirect, err);
    rec_flush(rb, rn, true, st, sp, dv, ndirect, err);
    es = block_fix(es, smf);
    inline_att = block_sum(inline_att, sm);
    death_hf = block_sum(death_hf, sm);
    ndirect = block_sum(ndirect, sm);
    if (p.multispawn || p.buffered) {
        __shared__ double smd[32];
        double ca = block_sum((double)cl_att, smd);
        if (threadIdx.x == 0 && ca != 0.0) atomicAdd(&st->cl_att, ca);
    }
    if (threadIdx.x == 0) {
        if (death_hf) atomicAdd((unsigned long long *)&wa.death[0], (unsigned long long)death_hf);
        wa.enum_part[2 * (enum_base + vb)] = es.lo;
        wa.enum_part[2 * (enum_base + vb) + 1] = es.hi;
        if (inline_att) atomicAdd((unsigned long long *)&st->n_attempts, (unsigned long long)inline_att);
        if (ndirect) atomicAdd((unsigned long long *)&st->n_direct, (unsigned long long)ndirect);
    }
    if (err) atomicOr(&st->err, err);   // every thread reports its own bits
}

// ---------------------------------------------------------------------------
// a4/a6: expanded spawning attempts -- full non-composite visits first, then
// buffered composite clusters (Sec. IV.B-C)
// ---------------------------------------------------------------------------

template <int K, typename R>
__device__ __forceinline__ void d_attempts(const SysDev &s, const ListView &L, DevStep *st, const RunParams &p,
                                                              const WorkArrays &wa, const SpawnBuf &sp, const ClusterBuf &cl)
{
    // the cluster attempts of a runaway population are not run (their
    // packed count may have wrapped); the step reports the error instead
    if ((st->err & ERRB_RUNAWAY) || st->cl_att > (double)p.work_cap) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&st->err, (unsigned)ERRB_RUNAWAY);
        return;
    }
    const i64 n = st->n_occ, tf = st->fnc_attempts;
    i64 ncl = p.buffered ? (i64)st->cl_packed : (i64)(st->cl_packed >> CL_SHIFT);
    if (ncl > cl.cap) ncl = cl.cap;
    const i64 tc = ncl > 0 ? cl.end[ncl - 1] : 0;
    const u64 it = st->iter;
    const int lane = threadIdx.x & 31;
    const i64 nwarps = (i64)gridDim.x * blockDim.x / 32;
    const i64 wglob = ((i64)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    unsigned err = 0;
    __shared__ AttQueue<K> aq[WORK_THREADS / 32];
    __shared__ RecStage rsb[WORK_THREADS / 32];
    __shared__ i64 sm[32];
    AttQueue<K> &q = aq[threadIdx.x >> 5];
    RecStage &rb = rsb[threadIdx.x >> 5];
    int qn = 0, rn = 0;   // drawn attempts and staged records of this warp (warp-uniform)
    i64 ndirect = 0;
    const DirectView dv = direct_view(L, wa, st);
    for (int part = 0; part < 2; part++) {
        // part 0: full non-composite attempts (owners: list entries);
        // part 1: attempts of the composite clusters queued by k_sample
        const i64 total = part == 0 ? tf : tc;
        const i64 *end = part == 0 ? wa.att_end : cl.end;
        const i64 nown = part == 0 ? n : ncl;
        const i64 per = ((total + nwarps - 1) / nwarps + 31) & ~31LL;
        const i64 a0 = wglob * per, a1 = a0 + per < total ? a0 + per : total;
        if (a0 >= a1) continue;
        AttemptWindow w = window_start(end, nown, a0);
        for (i64 t0 = a0; t0 < a1; t0 += 32) {
            i64 o, m;
            window_step(end, nown, t0, w, o, m);
            bool ok = false;
            Det<K> dj;
            double ca = 0.0;
            u64 r3 = 0;
            u64 code = 0;
            int gc = 0;
            if (t0 + lane < a1) {
                u64 tag, idx;
                if (part == 0) {
                    dj = load_det<K>(L.bits, L.cap, o);
                    ca = wa.catt[o];
                    tag = TAG_VISIT_ATT;
                    idx = (u64)o;
                } else {
                    dj = load_det<K>(cl.bits, cl.cap, o);
                    ca = cl.catt[o];
                    tag = TAG_SAMPLE_ATT;
                    idx = cl.index[o];
                }
                R4 r = draw(p.seed, p.replica, it, tag, idx, (u64)m);
                ok = attempt_draw<K>(s, dj, r, code, gc);
                r3 = r.v[3];
            }
            q_push<K>(q, qn, ok, dj, ca, r3, code, gc);
            q_drain_staged<K, R>(q, qn, false, rb, rn, s, p, st, sp, dv, ndirect, err);
        }
    }
    q_drain_staged<K, R>(q, qn, true, rb, rn, s, p, st, sp, dv, ndirect, err);
    rec_flush(rb, rn, true, st, sp, dv, ndirect, err);
    ndirect = block_sum(ndirect, sm);
    if (threadIdx.x == 0 && ndirect) atomicAdd((unsigned long long *)&st->n_direct, (unsigned long long)ndirect);
    if (err) atomicOr(&st->err, err);
}

// ---------------------------------------------------------------------------
// a7: LSD radix sort by rank key (stable, fixed grid, digit-major offsets)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void d_sort_hist(const u64 *keys, const DevStep *st, i64 cap, int shift, int bits,
                                                             unsigned *hist)
{
    __shared__ unsigned h[1 << MAX_DIGIT_BITS];
    const int nd = 1 << bits;
    for (int d = threadIdx.x; d < nd; d += blockDim.x) h[d] = 0;
    __syncthreads();
    i64 n = st->n_sp < cap ? st->n_sp : cap, lo, hi;
    chunk_of(n, lo, hi);
    const u64 mask = (u64)nd - 1;
    for (i64 i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += blockDim.x) hist[(size_t)d * gridDim.x + blockIdx.x] = h[d];
}

// exclusive scan of row d (one digit across all sort blocks) in place, and
// the row total; one block per digit
__device__ __forceinline__ void d_sort_scan(unsigned *hist, int grid, unsigned *totals)
{
    __shared__ i64 sm[32];
    const int d = blockIdx.x;
    unsigned *row = hist + (size_t)d * grid;
    i64 carry = 0;
    for (int base = 0; base < grid; base += blockDim.x) {
        int b = base + threadIdx.x;
        i64 v = b < grid ? row[b] : 0, tot;
        i64 incl = block_incl_scan(v, sm, tot);
        if (b < grid) row[b] = (unsigned)(carry + incl - v);
        carry += tot;
    }
    if (threadIdx.x == 0) totals[d] = (unsigned)carry;
}

__device__ __forceinline__ void d_sort_scatter(const u64 *kin, const i64 *vin, u64 *kout, i64 *vout,
                                                                const DevStep *st, i64 cap, int shift, int bits,
                                                                const unsigned *hist, const unsigned *totals)
{
    constexpr int NW = SORT_THREADS / 32;
    static_assert((1 << MAX_DIGIT_BITS) <= SORT_THREADS, "one thread per digit in the tile scans");
    __shared__ unsigned s_off[1 << MAX_DIGIT_BITS];
    __shared__ unsigned s_tot[1 << MAX_DIGIT_BITS];
    __shared__ unsigned s_tpre[1 << MAX_DIGIT_BITS];
    __shared__ unsigned s_w[NW][1 << MAX_DIGIT_BITS];
    // the tile in digit order, so that each digit's run is written out by
    // consecutive threads to consecutive addresses
    __shared__ u64 s_tk[SORT_TILE];
    __shared__ i64 s_tv[SORT_TILE];
    __shared__ i64 s_sc[32];
    const int nd = 1 << bits;
    const u64 mask = (u64)nd - 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    {
        // digit base = exclusive scan of the digit totals; plus this block's row prefix
        __shared__ i64 sm64[32];
        for (int d0 = 0; d0 < nd; d0 += blockDim.x) {
            int d = d0 + threadIdx.x;
            i64 v = d < nd ? totals[d] : 0, tot;
            i64 incl = block_incl_scan(v, sm64, tot);
            if (d < nd) s_off[d] = (unsigned)(incl - v);
            __syncthreads();
        }
        for (int d = threadIdx.x; d < nd; d += blockDim.x) s_off[d] += hist[(size_t)d * gridDim.x + blockIdx.x];
    }
    i64 n = st->n_sp < cap ? st->n_sp : cap, lo, hi;
    chunk_of(n, lo, hi);
    for (i64 tb = lo; tb < hi; tb += SORT_TILE) {
        for (int q = threadIdx.x; q < NW * nd; q += blockDim.x) s_w[q / nd][q % nd] = 0;
        __syncthreads();
        u64 kk[SORT_ITEMS];
        i64 vv[SORT_ITEMS];
        unsigned dg[SORT_ITEMS], rk[SORT_ITEMS];
        bool ok[SORT_ITEMS];
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; j++) {
            i64 idx = tb + (i64)wid * (32 * SORT_ITEMS) + j * 32 + lane;
            ok[j] = idx < hi;
            kk[j] = ok[j] ? kin[idx] : 0;
            vv[j] = ok[j] ? vin[idx] : 0;
            unsigned d = (unsigned)((kk[j] >> shift) & mask);
            dg[j] = d;
            unsigned peers = __ballot_sync(FULLMASK, ok[j]);
            for (int b = 0; b < bits; b++) {
                unsigned bb = __ballot_sync(FULLMASK, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bb : ~bb;
            }
            unsigned base = 0;
            if (ok[j]) base = s_w[wid][d];
            __syncwarp();
            if (ok[j] && (peers & lt) == 0) s_w[wid][d] = base + __popc(peers);
            __syncwarp();
            rk[j] = base + __popc(peers & lt);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < nd; d += blockDim.x) {
            unsigned run = 0;
            for (int w = 0; w < NW; w++) {
                unsigned t = s_w[w][d];
                s_w[w][d] = run;
                run += t;
            }
            s_tot[d] = run;
        }
        __syncthreads();
        {
            // exclusive prefix of the tile's digit counts (nd <= blockDim)
            const int d = threadIdx.x;
            const i64 v = d < nd ? (i64)s_tot[d] : 0;
            i64 tot;
            const i64 incl = block_incl_scan(v, s_sc, tot);
            if (d < nd) s_tpre[d] = (unsigned)(incl - v);
        }
        __syncthreads();
        // stable order within the tile: digit, then warp, then item, then lane
#pragma unroll
        for (int j = 0; j < SORT_ITEMS; j++) {
            if (ok[j]) {
                const unsigned tp = s_tpre[dg[j]] + s_w[wid][dg[j]] + rk[j];
                s_tk[tp] = kk[j];
                s_tv[tp] = vv[j];
            }
        }
        __syncthreads();
        const int tn = (int)(hi - tb < (i64)SORT_TILE ? hi - tb : (i64)SORT_TILE);
        for (int q = threadIdx.x; q < tn; q += blockDim.x) {
            const u64 k = s_tk[q];
            const unsigned d = (unsigned)((k >> shift) & mask);
            const unsigned pos = s_off[d] + (unsigned)q - s_tpre[d];
            kout[pos] = k;
            vout[pos] = s_tv[q];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < nd; d += blockDim.x) s_off[d] += s_tot[d];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// a8: one record per distinct key with the summed weight
// ---------------------------------------------------------------------------

__device__ __forceinline__ void d_seg_count(const u64 *keys, const DevStep *st, i64 cap, i64 *outpop,
                                                             const WorkArrays &wa)
{
    __shared__ i64 sm[32];
    i64 n = st->n_sp < cap ? st->n_sp : cap, lo, hi;
    chunk_of(n, lo, hi);
    i64 c = 0;
    for (i64 i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        c += (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
        outpop[i] = 0;
    }
    c = block_sum(c, sm);
    if (threadIdx.x == 0) wa.part[4 * blockIdx.x] = c;
}

// generic: exclusive scan of part[4b + src] into part[4b + dst], total to *out
__device__ __forceinline__ void d_part_scan(const WorkArrays &wa, int grid, int src, int dst, i64 *out)
{
    __shared__ i64 sm[32];
    int t = threadIdx.x;
    i64 v = t < grid ? wa.part[4 * t + src] : 0, tot;
    i64 incl = block_incl_scan(v, sm, tot);
    if (t < grid) wa.part[4 * t + dst] = incl - v;
    if (t == 0) *out = tot;
}

__device__ __forceinline__ void d_seg_write(const u64 *keys, const i64 *pops, const DevStep *st, i64 cap,
                                                             u64 *outkey, i64 *outpop, const WorkArrays &wa)
{
    __shared__ i64 sm[32];
    i64 n = st->n_sp < cap ? st->n_sp : cap, lo, hi;
    chunk_of(n, lo, hi);
    i64 carry = wa.part[4 * blockIdx.x + 2];
    const int lane = threadIdx.x & 31;
    for (i64 base = lo; base < hi; base += blockDim.x) {
        i64 i = base + threadIdx.x;
        bool ok = i < hi;
        u64 k = ok ? keys[i] : 0;
        i64 v = ok ? pops[i] : 0;
        i64 head = (ok && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
        i64 tot;
        i64 incl = block_incl_scan(head, sm, tot);
        i64 seg = ok ? carry + incl - 1 : -1;
        if (head) outkey[seg] = k;
        // segmented warp sum; the last lane of each run adds it
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            i64 tv = __shfl_up_sync(FULLMASK, v, o);
            i64 ts = __shfl_up_sync(FULLMASK, seg, o);
            if (lane >= o && ts == seg) v += tv;
        }
        i64 nxt = __shfl_down_sync(FULLMASK, seg, 1);
        bool last = lane == 31 || nxt != seg;
        if (ok && last && v != 0) atomicAdd((unsigned long long *)&outpop[seg], (unsigned long long)v);
        carry += tot;
    }
}

// ---------------------------------------------------------------------------
// a9: merge into the list with the occupation threshold
// ---------------------------------------------------------------------------

// each reduced key: add to its list entry, or mark it new (thresholded)
__device__ __forceinline__ void d_merge_match(const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa,
                                                               const u64 *rkey, i64 *rpop)
{
    const i64 n = st->n_occ, m = st->n_keys;
    const u64 it = st->iter;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (i64)gridDim.x * blockDim.x) {
        u64 k = rkey[j];
        i64 pos = lower_bound_key(L.key, n, k);
        if (pos < n && L.key[pos] == k) {
            wa.acc[pos] += rpop[j];
            wa.ins[j] = -1;
            wa.keep_s[j] = 0;
        } else {
            i64 v = threshold(p, it, k, rpop[j]);
            rpop[j] = v;
            wa.ins[j] = pos;
            wa.keep_s[j] = v != 0 ? 1 : 0;
            // a kept new key lands right before list entry pos
            if (v != 0 && pos < n) atomicAdd(&wa.before[pos], 1);
        }
    }
}

// New populations of the list entries (old + death + matched spawns, then the
// occupation threshold) with their keep flags packed with the kept new keys
// inserted before them (blocks [0, G), contiguous chunks), and the keep counts
// of the new keys (blocks [G, 2G)); each block's sum goes to the partials.
__device__ __forceinline__ void d_merge_count(const ListView &L, DevStep *st, const RunParams &p, const WorkArrays &wa,
                                              int G)
{
    __shared__ i64 sm[32];
    const bool second = blockIdx.x >= G;
    const i64 n = second ? st->n_keys : st->n_occ;
    const i64 c = (n + G - 1) / G;
    const i64 b = second ? blockIdx.x - G : blockIdx.x;
    const i64 lo = b * c < n ? b * c : n, hi = lo + c < n ? lo + c : n;
    i64 sum = 0;
    if (second) {
        for (i64 i = lo + threadIdx.x; i < hi; i += blockDim.x) sum += wa.keep_s[i];
    } else {
        const u64 it = st->iter;
        const bool direct = st->nkb > 0;
        i64 hits = 0;   // entries that received directly added spawns: distinct keys of the step
        for (i64 i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            i64 v = L.pop[i] + wa.death[i] + wa.acc[i];
            // the key is read only for the few entries the threshold decides
            const i64 av = v < 0 ? -v : v;
            if (i > 0 && av > 0 && av < (i64)FIX_ONE) v = threshold(p, it, L.key[i], v);
            wa.newpop[i] = v;
            // two counts in one word (each below 2^31): the entry's keep flag
            // and the kept new keys that go before it; one prefix gives both
            const i64 w = ((i == 0 || v != 0) ? 1 : 0) | ((i64)wa.before[i] << 32);
            wa.keep_l[i] = w;
            sum += w;
            if (direct) hits += wa.hit[i];
        }
        if (direct) {
            hits = block_sum(hits, sm);
            if (threadIdx.x == 0 && hits) atomicAdd((unsigned long long *)&st->n_hit, (unsigned long long)hits);
        }
    }
    sum = block_sum(sum, sm);
    if (threadIdx.x == 0) wa.part[4 * blockIdx.x] = sum;
}

// scan of the 2G partials: list part then spawn part
__device__ __forceinline__ void d_keep_top(DevStep *st, const WorkArrays &wa, int G)
{
    __shared__ i64 sm[32];
    int t = threadIdx.x;
    i64 a = t < G ? wa.part[4 * t] : 0, ta;
    i64 ia = block_incl_scan(a, sm, ta);
    if (t < G) wa.part[4 * t + 2] = ia - a;
    i64 b = t < G ? wa.part[4 * (G + t)] : 0, tb;
    i64 ib = block_incl_scan(b, sm, tb);
    if (t < G) wa.part[4 * (G + t) + 2] = ib - b;
    if (t == 0) {
        st->kept_list = ta & 0xFFFFFFFFLL;   // the low count of the packed list flags
        st->kept_new = tb;
    }
}

// The keep prefixes and the list's scatter in one pass.  Blocks [G, 2G):
// exclusive prefix of the new keys' keep flags in place.  Blocks [0, G): the
// exclusive prefix e of the packed list words (kept entries | kept new keys
// before the entry << 32) over the block's chunk, four rows of counts read
// before their scans; each kept entry goes to e_lo + e_hi + (new keys right
// before it), and e is stored only where kept new keys are inserted (the
// new-key scatter reads it there).
template <int K>
__device__ __forceinline__ void d_keep_scatter(const ListView &L, const ListView &O, DevStep *st, const WorkArrays &wa,
                                               int G)
{
    __shared__ i64 sm[32];
    const bool second = blockIdx.x >= G;
    const i64 n = second ? st->n_keys : st->n_occ;
    const i64 c = (n + G - 1) / G;
    const i64 b = second ? blockIdx.x - G : blockIdx.x;
    const i64 lo = b * c < n ? b * c : n, hi = lo + c < n ? lo + c : n;
    i64 carry = wa.part[4 * blockIdx.x + 2];
    if (second) {
        for (i64 base = lo; base < hi; base += blockDim.x) {
            const i64 i = base + threadIdx.x;
            const i64 v = i < hi ? wa.keep_s[i] : 0;
            i64 tot;
            const i64 incl = block_incl_scan(v, sm, tot);
            if (i < hi) wa.keep_s[i] = carry + incl - v;
            carry += tot;
        }
        return;
    }
    constexpr int ROWS = 4;
    i64 asum = 0;
    unsigned err = 0;
    for (i64 base = lo; base < hi; base += ROWS * (i64)blockDim.x) {
        i64 w[ROWS], v[ROWS], e[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const i64 i = base + r * (i64)blockDim.x + threadIdx.x;
            w[r] = i < hi ? wa.keep_l[i] : 0;
            v[r] = i < hi ? wa.newpop[i] : 0;
        }
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            i64 tot;
            const i64 incl = block_incl_scan(w[r], sm, tot);
            e[r] = carry + incl - w[r];
            carry += tot;
        }
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const i64 i = base + r * (i64)blockDim.x + threadIdx.x;
            if (i >= hi) continue;
            const i64 nb = w[r] >> 32;   // kept new keys inserted right before entry i
            if (nb) wa.keep_l[i] = e[r];
            if (!(i == 0 || v[r] != 0)) continue;
            const i64 out = (e[r] & 0xFFFFFFFFLL) + (e[r] >> 32) + nb;
            if (out >= O.cap) {
                err |= ERRB_LIST_OVERFLOW;
                continue;
            }
            store_det<K>(O.bits, O.cap, out, load_det<K>(L.bits, L.cap, i));
            O.key[out] = L.key[i];
            O.pop[out] = v[r];
            O.diag[out] = L.diag[i];
            asum += v[r] < 0 ? -v[r] : v[r];
        }
    }
    asum = block_sum(asum, sm);
    if (threadIdx.x == 0) {
        if (asum) atomicAdd((unsigned long long *)&st->ntot_after, (unsigned long long)asum);
    }
    if (err) atomicOr(&st->err, err);   // every thread reports its own bits
}

template <int K, typename R>
__device__ __forceinline__ void d_scatter_new(const SysDev &s, const ListView &O, DevStep *st, const WorkArrays &wa,
                                                               const u64 *rkey, const i64 *rpop)
{
    __shared__ i64 sm[32];
    const i64 n = st->n_occ, m = st->n_keys, kl = st->kept_list;
    i64 asum = 0;
    unsigned err = 0;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (i64)gridDim.x * blockDim.x) {
        i64 il = wa.ins[j];
        i64 v = rpop[j];
        if (il < 0 || v == 0) continue;
        i64 out = wa.keep_s[j] + (il < n ? (wa.keep_l[il] & 0xFFFFFFFFLL) : kl);
        if (out >= O.cap) {
            err |= ERRB_LIST_OVERFLOW;
            continue;
        }
        u64 k = rkey[j];
        Det<K> d = unrank_key<K>(s, k);
        store_det<K>(O.bits, O.cap, out, d);
        O.key[out] = k;
        O.pop[out] = v;
        O.diag[out] = diag_rel<K, R>(s, d);
        asum += v < 0 ? -v : v;
    }
    asum = block_sum(asum, sm);
    if (threadIdx.x == 0) {
        if (asum) atomicAdd((unsigned long long *)&st->ntot_after, (unsigned long long)asum);
    }
    if (err) atomicOr(&st->err, err);   // every thread reports its own bits
}

// ---------------------------------------------------------------------------
// a10: estimator reduction and the per-step record
// ---------------------------------------------------------------------------

__device__ __forceinline__ void d_finalize(DevStep *st, const RunParams &p, const WorkArrays &wa, const ClusterBuf &cl, int slots,
                                                   i64 list_cap)
{
    __shared__ u64 smf[64];
    Fix128 k = {0, 0};
    for (int q = threadIdx.x; q < slots; q += blockDim.x) {
        Fix128 t = {wa.enum_part[2 * q], wa.enum_part[2 * q + 1]};
        k.add(t);
    }
    k = block_fix(k, smf);
    if (threadIdx.x == 0) {
        i64 ncl = p.buffered ? (i64)st->cl_packed : (i64)(st->cl_packed >> CL_SHIFT);
        if (ncl > cl.cap) ncl = cl.cap;
        i64 tc = ncl > 0 ? cl.end[ncl - 1] : 0;
        Record r;
        r.iter = st->iter;
        r.shift = st->shift;
        r.n0 = st->n0;
        r.ntot = st->ntot;
        r.n_sel = st->n_sel;
        r.n_visit = p.fnc ? st->n_occ : 0;
        r.n_attempts = st->fnc_attempts + tc + st->n_attempts;
        r.n_spawned = st->n_sp + st->n_direct;
        r.e_num = fix_to_double(k);
        r.ntot_after = st->ntot_after;
        r.nocc_after = st->kept_list + st->kept_new;
        r.n_keys = st->n_keys + st->n_hit;
        r.n_clusters = ncl;
        r.n_direct = st->n_direct;
        st->prev_spawned = r.n_spawned;
        wa.ring[st->iter % RING] = r;
        st->n_start = st->n_occ;
        st->n_occ = r.nocc_after < list_cap ? r.nocc_after : list_cap;
        st->cur ^= 1;   // the merged list becomes the current one
        st->iter = st->iter + 1;
    }
}

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------


// ---------------------------------------------------------------------------
// Kernels: each block serves replica blockIdx.y of an array of per-replica
// arguments (one entry for a single context, many for a batch).
// ---------------------------------------------------------------------------

#define REPLICA                               \
    const StepArgs &a = A[blockIdx.y];        \
    const int cur_ = a.st->cur

// the replica's arguments copied to shared memory (hot kernels)
#define REPLICA_SMEM                                                              \
    __shared__ StepArgs a_sm;                                                     \
    {                                                                             \
        const u64 *src_ = (const u64 *)&A[blockIdx.y];                            \
        u64 *dst_ = (u64 *)&a_sm;                                                 \
        for (int q_ = threadIdx.x; q_ < (int)(sizeof(StepArgs) / 8); q_ += blockDim.x) dst_[q_] = src_[q_]; \
    }                                                                             \
    __syncthreads();                                                              \
    const StepArgs &a = a_sm;                                                     \
    const int cur_ = a.st->cur

// Kernels that do not depend on the word count (defined in ccmc_step.cu).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_partial(const StepArgs *__restrict__ A);
__global__ void __launch_bounds__(1024) k_scan_top(const StepArgs *__restrict__ A, int grid);
__global__ void __launch_bounds__(1024) k_sample_plan(const StepArgs *__restrict__ A, int nrep, FlatPlan fp,
                                                       int enum_base);
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const StepArgs *__restrict__ A, int src, int shift, int bits);
__global__ void __launch_bounds__(1024) k_sort_scan(const StepArgs *__restrict__ A, int grid);
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const StepArgs *__restrict__ A, int src, int shift, int bits);
__global__ void __launch_bounds__(SCAN_THREADS) k_seg_count(const StepArgs *__restrict__ A, int src);
__global__ void __launch_bounds__(1024) k_part_scan(const StepArgs *__restrict__ A, int grid);
__global__ void __launch_bounds__(SCAN_THREADS) k_seg_write(const StepArgs *__restrict__ A, int src);
__global__ void __launch_bounds__(WORK_THREADS) k_merge_match(const StepArgs *__restrict__ A, int src);
__global__ void __launch_bounds__(SCAN_THREADS) k_merge_count(const StepArgs *__restrict__ A, int G);
__global__ void __launch_bounds__(SCAN_THREADS) k_local_scan(const StepArgs *__restrict__ A);
__global__ void __launch_bounds__(1024) k_keep_top(const StepArgs *__restrict__ A, int G);
__global__ void __launch_bounds__(1024) k_finalize(const StepArgs *__restrict__ A, int slots);

template <int K, typename R>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_final(const StepArgs *__restrict__ A)
{
    REPLICA_SMEM;
    d_scan_final<K, R>(a.s, a.list[cur_], a.st, a.p, a.wa);
}

template <int K, typename R, bool DIST>
__global__ void __launch_bounds__(WORK_THREADS, SAMPLE_BLOCKS_PER_SM) k_sample(const StepArgs *__restrict__ A, int enum_base)
{
    REPLICA_SMEM;
    d_sample<K, R, DIST>(a.s, a.list[cur_], a.st, a.p, a.wa, a.sp, a.cl, enum_base, blockIdx.x, gridDim.x);
}

// Persistent batch sampler: each block takes the next virtual block of the
// plan, finds its replica and runs that share of the replica's samples.
template <int K, typename R, bool DIST>
__global__ void __launch_bounds__(WORK_THREADS, SAMPLE_BLOCKS_PER_SM) k_sample_flat(const StepArgs *__restrict__ A, int nrep, FlatPlan fp,
                                                                 int enum_base)
{
    __shared__ StepArgs a_sm;
    __shared__ int s_v, s_r;
    const int total = fp.vstart[nrep];
    int have = -1;
    for (;;) {
        __syncthreads();   // the previous share is finished with a_sm and s_v
        if (threadIdx.x == 0) {
            const int v = (int)atomicAdd(fp.counter, 1u);
            int r = 0;
            if (v < total) {
                int lo = 0, hi = nrep - 1;   // last r with vstart[r] <= v
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (fp.vstart[mid] <= v) lo = mid;
                    else hi = mid - 1;
                }
                r = lo;
            }
            s_v = v;
            s_r = r;
        }
        __syncthreads();
        const int v = s_v;
        if (v >= total) break;
        const int r = s_r;
        if (r != have) {
            const u64 *src = (const u64 *)&A[r];
            u64 *dst = (u64 *)&a_sm;
            for (int q = threadIdx.x; q < (int)(sizeof(StepArgs) / 8); q += blockDim.x) dst[q] = src[q];
            __syncthreads();
            have = r;
        }
        const StepArgs &a = a_sm;
        const int v0 = fp.vstart[r];
        d_sample<K, R, DIST>(a.s, a.list[a.st->cur], a.st, a.p, a.wa, a.sp, a.cl, enum_base, v - v0,
                       fp.vstart[r + 1] - v0);
    }
}

template <int K, typename R>
__global__ void __launch_bounds__(WORK_THREADS, 4) k_attempts(const StepArgs *__restrict__ A)
{
    REPLICA_SMEM;
    d_attempts<K, R>(a.s, a.list[cur_], a.st, a.p, a.wa, a.sp, a.cl);
}

template <int K>
__global__ void __launch_bounds__(WORK_THREADS) k_local_table(const StepArgs *__restrict__ A)
{
    REPLICA;
    d_local_table<K>(a.list[cur_], a.st, a.p, a.wa);
}

template <int K>
__global__ void __launch_bounds__(SCAN_THREADS) k_keep_scatter(const StepArgs *__restrict__ A, int G)
{
    REPLICA;
    d_keep_scatter<K>(a.list[cur_], a.list[cur_ ^ 1], a.st, a.wa, G);
}

template <int K, typename R>
__global__ void __launch_bounds__(WORK_THREADS) k_scatter_new(const StepArgs *__restrict__ A, int src)
{
    REPLICA;
    d_scatter_new<K, R>(a.s, a.list[cur_ ^ 1], a.st, a.wa, a.sp.key[src ^ 1], a.sp.pop[src ^ 1]);
}

// ---------------------------------------------------------------------------
// The whole step for nrep replicas (grid dimension y), the same sequence
// every step, so it can be captured once in a CUDA graph.
// ---------------------------------------------------------------------------

template <int K, typename R>
cudaError_t launch_phases(const StepArgs *A, int nrep, const Shapes &sh, bool multi_att, cudaStream_t sm,
                          i64 *launches, const cudaEvent_t *ev, const FlatPlan *plan)
{
    auto mark = [&](int phase) {
        if (ev) cudaEventRecord(ev[phase], sm);
    };
    const dim3 gscan(sh.scan_grid, nrep), gwork(sh.work_grid, nrep), gsort(sh.sort_grid, nrep), gone(1, nrep);
    mark(0);
    k_scan_partial<<<gscan, SCAN_THREADS, 0, sm>>>(A);
    k_scan_top<<<gone, 1024, 0, sm>>>(A, sh.scan_grid);
    k_scan_final<K, R><<<gscan, SCAN_THREADS, 0, sm>>>(A);
    launches[0] += 3;
    if (sh.nranks > 1) {
        // simulated distribution: owners and per-processor position tables
        k_local_table<K><<<gwork, WORK_THREADS, 0, sm>>>(A);
        k_local_scan<<<dim3(sh.nranks < 1024 ? sh.nranks : 1024, nrep), SCAN_THREADS, 0, sm>>>(A);
        launches[0] += 2;
    }
    mark(1);
    if (plan) {
        k_sample_plan<<<1, 1024, 0, sm>>>(A, nrep, *plan, sh.scan_grid);
        if (sh.nranks > 1) k_sample_flat<K, R, true><<<plan->grid, WORK_THREADS, 0, sm>>>(A, nrep, *plan, sh.scan_grid);
        else k_sample_flat<K, R, false><<<plan->grid, WORK_THREADS, 0, sm>>>(A, nrep, *plan, sh.scan_grid);
        launches[1] += 2;
    } else {
        if (sh.nranks > 1) k_sample<K, R, true><<<gwork, WORK_THREADS, 0, sm>>>(A, sh.scan_grid);
        else k_sample<K, R, false><<<gwork, WORK_THREADS, 0, sm>>>(A, sh.scan_grid);
        launches[1] += 1;
    }
    mark(2);
    if (multi_att) {
        k_attempts<K, R><<<gwork, WORK_THREADS, 0, sm>>>(A);
        launches[2] += 1;
    }
    mark(3);
    int src = 0;
    for (int shift = 0; shift < sh.key_bits; shift += sh.digit_bits) {
        int bits = min(sh.digit_bits, sh.key_bits - shift);
        k_sort_hist<<<gsort, SORT_THREADS, 0, sm>>>(A, src, shift, bits);
        k_sort_scan<<<dim3(1 << bits, nrep), 1024, 0, sm>>>(A, sh.sort_grid);
        k_sort_scatter<<<gsort, SORT_THREADS, 0, sm>>>(A, src, shift, bits);
        src ^= 1;
        launches[3] += 3;
    }
    mark(4);
    k_seg_count<<<gscan, SCAN_THREADS, 0, sm>>>(A, src);
    k_part_scan<<<gone, 1024, 0, sm>>>(A, sh.scan_grid);
    k_seg_write<<<gscan, SCAN_THREADS, 0, sm>>>(A, src);
    launches[4] += 3;
    mark(5);
    k_merge_match<<<gwork, WORK_THREADS, 0, sm>>>(A, src);
    k_merge_count<<<dim3(2 * sh.scan_grid, nrep), SCAN_THREADS, 0, sm>>>(A, sh.scan_grid);
    k_keep_top<<<gone, 1024, 0, sm>>>(A, sh.scan_grid);
    k_keep_scatter<K><<<dim3(2 * sh.scan_grid, nrep), SCAN_THREADS, 0, sm>>>(A, sh.scan_grid);
    k_scatter_new<K, R><<<gwork, WORK_THREADS, 0, sm>>>(A, src);
    launches[5] += 5;
    mark(6);
    k_finalize<<<gone, 1024, 0, sm>>>(A, plan ? sh.scan_grid + plan->wmax : sh.enum_slots);
    launches[6] += 1;
    mark(7);
    return cudaGetLastError();
}

}  // namespace ccmc
