// ccmc_device.cuh -- device building blocks of the CCMC time step.
//
// Conventions (shared with the rest of the library, see include/ccmc.h):
// spin-orbital p is bit (p & 63) of word (p >> 6); 2q = alpha, 2q+1 = beta;
// the Hartree-Fock (HF) determinant is the lowest N bits; populations are
// int64 multiples of 2^-16.  Floating point is FP64 without fused
// multiply-add (the library is compiled with -fmad=false) and every
// expression below keeps the operation order documented beside it, so that
// decisions taken from FP64 values (stochastic rounding) are reproducible.
#pragma once

#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace ccmc {

typedef unsigned long long u64;
typedef long long i64;

constexpr int MAXK = 6;            // words per determinant (M <= 384)
constexpr int RANK_STRIDE = 384;   // row stride of the rank tables (positions < M)
constexpr double FIX_ONE = 65536.0;

// Philox counter tags (bits 56..63 of counter word 1).
enum : u64 {
    TAG_SAMPLE = 1,      // cluster selection of sample g
    TAG_SAMPLE_ATT = 2,  // spawning attempt m of sample g
    TAG_VISIT = 3,       // full non-composite death draw of list entry i
    TAG_VISIT_ATT = 4,   // full non-composite attempt m of list entry i
    TAG_THRESH = 5       // occupation threshold of the excitor with a given key
};

// Device error bits (sticky status word).
enum : unsigned {
    ERRB_SPAWN_OVERFLOW = 1u,
    ERRB_NUMERIC = 2u,
    ERRB_LIST_OVERFLOW = 4u,
    ERRB_CLUSTER_OVERFLOW = 8u,
    ERRB_RUNAWAY = 16u
};

// Hamiltonian and generator tables as seen by the kernels (passed by value).
struct SysDev {
    int kind;            // 0 UEG, 1 generic
    int nel, nso, lmax;
    int nw;
    u64 hf[MAXK];
    u64 valid[MAXK];     // bits < nso
    u64 virt[MAXK];      // bits in [nel, nso)
    // UEG
    int nmax, side;
    const int *grid;     // (2 nmax + 1)^3 -> spatial orbital or -1
    const int *kv;       // 3 ints per spatial orbital
    const double *tkin;  // per spin-orbital
    const double *vtab;  // Coulomb by integer |n|^2
    double inv_pgen_ueg;
    u64 npairs, nvirt;
    // generic integrals
    int norb;
    const double *h1;
    const double *eri;
    int nv[2];
    u64 ns_nd, ns;
    u64 ndcase[3];
    double inv_pgen_single[2];
    double inv_pgen_double[3];
    // rank key: tab[c * RANK_STRIDE + q] = sum_{j=0}^{l-c} C(q, j)
    const u64 *rank_tab;
    u64 cocc;
    int lmin_exc;        // smallest excitation level of any non-reference list entry
    const double *fock;  // reference Fock diagonal per spin-orbital
    // FP32 form: tables rounded from the FP64 ones
    const float *tkin_f, *vtab_f, *h1_f, *eri_f;
    const float *fock_f;
    float inv_pgen_ueg_f;
    float inv_pgen_single_f[2];
    float inv_pgen_double_f[3];
};

// table selection by real type
template <typename R> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ const double *tkin(const SysDev &s) { return s.tkin; }
    static __device__ __forceinline__ const double *vtab(const SysDev &s) { return s.vtab; }
    static __device__ __forceinline__ const double *h1(const SysDev &s) { return s.h1; }
    static __device__ __forceinline__ const double *eri(const SysDev &s) { return s.eri; }
    static __device__ __forceinline__ const double *fock(const SysDev &s) { return s.fock; }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ const float *tkin(const SysDev &s) { return s.tkin_f; }
    static __device__ __forceinline__ const float *vtab(const SysDev &s) { return s.vtab_f; }
    static __device__ __forceinline__ const float *h1(const SysDev &s) { return s.h1_f; }
    static __device__ __forceinline__ const float *eri(const SysDev &s) { return s.eri_f; }
    static __device__ __forceinline__ const float *fock(const SysDev &s) { return s.fock_f; }
};

template <int K>
struct Det {
    u64 w[K];
};

// ---------------------------------------------------------------------------
// Philox-4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11)
// ---------------------------------------------------------------------------

struct R4 {
    u64 v[4];
};

// 64x64 -> 128-bit product (host builds: four 32x32 -> 64 multiply-adds):
// x*m = p0 + 2^32 (xL mH + xH mL) + 2^64 xH mH; with t = xL mH + hi32(p0) and
// u = xH mL + lo32(t) (neither overflows), lo = lo32(p0) | lo32(u) << 32 and
// hi = xH mH + hi32(t) + hi32(u).
__host__ __device__ __forceinline__ void mulhilo64(u64 x, u64 m, u64 &hi, u64 &lo)
{
#ifdef __CUDA_ARCH__
    hi = __umul64hi(x, m);   // measured faster on sm_103a than the limb form below
    lo = x * m;
    return;
#endif
    const u64 xl = x & 0xFFFFFFFFULL, xh = x >> 32, ml = m & 0xFFFFFFFFULL, mh = m >> 32;
    const u64 p0 = xl * ml;
    const u64 t = xl * mh + (p0 >> 32);
    const u64 u = xh * ml + (t & 0xFFFFFFFFULL);
    hi = xh * mh + (t >> 32) + (u >> 32);
    lo = (p0 & 0xFFFFFFFFULL) | (u << 32);
}

__host__ __device__ __forceinline__ R4 philox(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1)
{
    // two rounds per loop iteration: the sampler inlines several draws, and
    // fully unrolled rounds made its loop overflow the instruction cache
#pragma unroll 2
    for (int r = 0; r < 10; r++) {
        const u64 m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
        u64 hi0, lo0, hi1, lo1;
        mulhilo64(c0, m0, hi0, lo0);
        mulhilo64(c2, m1, hi1, lo1);
        u64 n0 = hi1 ^ c1 ^ k0;
        u64 n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    R4 o;
    o.v[0] = c0;
    o.v[1] = c1;
    o.v[2] = c2;
    o.v[3] = c3;
    return o;
}

__host__ __device__ __forceinline__ R4 draw(u64 k0, u64 k1, u64 it, u64 tag, u64 index, u64 block)
{
    return philox(it, (tag << 56) | index, block, 0, k0, k1);
}

// ---------------------------------------------------------------------------
// The paper's distribution of excitors over N_p processors (Sec. III, Eq.
// ccmc_dist), simulated on one GPU: a determinant hash (Philox-4x64-10 under
// a fixed key as a mixing function over the bit string, three words per
// call, each call taking the previous result as its fourth counter word)
// and the owner o = (hash(D) + i) >> nu_move, p = hash(D xor o) mod N_p,
// with o xor-ed into the first word; nu_move >= 64 never moves an excitor.
// ---------------------------------------------------------------------------

constexpr u64 HASH_K0 = 0x243F6A8885A308D3ULL, HASH_K1 = 0x13198A2E03707344ULL;

__host__ __device__ __forceinline__ u64 words_hash(const u64 *w, int nw)
{
    u64 h = 0;
    for (int g = 0; g < nw; g += 3)
        h = philox(w[g], g + 1 < nw ? w[g + 1] : 0, g + 2 < nw ? w[g + 2] : 0, h, HASH_K0, HASH_K1).v[0];
    return h;
}

__host__ __device__ __forceinline__ u64 words_owner(const u64 *w, int nw, u64 it, int nu_move, u64 n_ranks)
{
    const u64 h = words_hash(w, nw);
    const u64 o = nu_move >= 64 ? 0 : (h + it) >> nu_move;
    u64 x[6];
    for (int i = 0; i < nw; i++) x[i] = w[i];
    x[0] ^= o;
    return words_hash(x, nw) % n_ranks;
}

// uniform in [0,1) from the top 53 bits
__device__ __forceinline__ double unif(u64 r) { return (double)(r >> 11) * 0x1p-53; }

// integer in [0, n): high word of r*n
__device__ __forceinline__ u64 below(u64 r, u64 n) { return __umul64hi(r, n); }

// ---------------------------------------------------------------------------
// Bit strings
// ---------------------------------------------------------------------------

template <int K>
__device__ __forceinline__ int bit(const Det<K> &d, int p) { return (int)((d.w[p >> 6] >> (p & 63)) & 1ULL); }

template <int K>
__device__ __forceinline__ void flip(Det<K> &d, int p) { d.w[p >> 6] ^= 1ULL << (p & 63); }

// number of set bits strictly below position p
template <int K>
__device__ __forceinline__ int count_below(const Det<K> &d, int p)
{
    int c = 0, wp = p >> 6;
#pragma unroll
    for (int i = 0; i < K; i++) {
        if (i < wp) c += __popcll(d.w[i]);
        else if (i == wp) c += __popcll(d.w[i] & ((1ULL << (p & 63)) - 1ULL));
    }
    return c;
}

// position of the k-th (0-based) set bit of x; x must have more than k bits
__device__ __forceinline__ int kth_bit64(u64 x, int k)
{
    int pos = 0, c;
    c = __popc((unsigned)x);
    if (k >= c) { k -= c; x >>= 32; pos += 32; }
    c = __popc((unsigned)(x & 0xFFFFULL));
    if (k >= c) { k -= c; x >>= 16; pos += 16; }
    c = __popc((unsigned)(x & 0xFFULL));
    if (k >= c) { k -= c; x >>= 8; pos += 8; }
    c = __popc((unsigned)(x & 0xFULL));
    if (k >= c) { k -= c; x >>= 4; pos += 4; }
    c = __popc((unsigned)(x & 0x3ULL));
    if (k >= c) { k -= c; x >>= 2; pos += 2; }
    if (k >= (int)(x & 1ULL)) pos += 1;
    return pos;
}

__device__ __forceinline__ u64 spin_mask(int spin)
{
    return spin < 0 ? ~0ULL : (spin == 0 ? 0x5555555555555555ULL : 0xAAAAAAAAAAAAAAAAULL);
}

// k-th occupied spin-orbital (ascending)
template <int K>
__device__ __forceinline__ int kth_occupied(const Det<K> &d, int k)
{
#pragma unroll
    for (int w = 0; w < K; w++) {
        int c = __popcll(d.w[w]);
        if (k < c) return 64 * w + kth_bit64(d.w[w], k);
        k -= c;
    }
    return -1;
}

// k-th empty spin-orbital (ascending), optionally of one spin
template <int K>
__device__ __forceinline__ int kth_empty(const SysDev &s, const Det<K> &d, u64 k, int spin)
{
    u64 sm = spin_mask(spin);
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 m = ~d.w[w] & s.valid[w] & sm;
        u64 c = (u64)__popcll(m);
        if (k < c) return 64 * w + kth_bit64(m, (int)k);
        k -= c;
    }
    return -1;
}

// excitation level relative to HF = number of holes
template <int K>
__device__ __forceinline__ int level_of(const SysDev &s, const Det<K> &d)
{
    int c = 0;
#pragma unroll
    for (int w = 0; w < K; w++) c += __popcll(s.hf[w] & ~d.w[w]);
    return c;
}

template <int K>
__device__ __forceinline__ bool is_hf(const SysDev &s, const Det<K> &d)
{
    bool e = true;
#pragma unroll
    for (int w = 0; w < K; w++) e = e && (d.w[w] == s.hf[w]);
    return e;
}

// s_D = <D|c_D|HF>: annihilating the holes h_1 < ... < h_n of HF in ascending
// order meets h_m - (m-1) occupied orbitals below h_m; creating the particles
// in descending order meets the N - n remaining electrons each time.  The sign
// is therefore (-1)^(sum h_m - n(n-1)/2 + n(N-n)).
template <int K>
__device__ __forceinline__ int excitor_sign(const SysDev &s, const Det<K> &d)
{
    int n = 0, hsum = 0;
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 m = s.hf[w] & ~d.w[w];
        while (m) {
            int b = __ffsll((long long)m) - 1;
            hsum += 64 * w + b;
            n++;
            m &= m - 1;
        }
    }
    int par = hsum - n * (n - 1) / 2 + n * (s.nel - n);
    return (par & 1) ? -1 : 1;
}

// Applies excitor c_e (given by its determinant) to cur: annihilators of its
// holes in ascending order, then creators of its particles in descending
// order, accumulating the parity of the occupied orbitals passed.  Returns
// false if the product vanishes.
template <int K>
__device__ __forceinline__ bool apply_excitor(const SysDev &s, const Det<K> &e, Det<K> &cur, int &parity)
{
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 m = s.hf[w] & ~e.w[w];
        while (m) {
            int p = 64 * w + (__ffsll((long long)m) - 1);
            if (!bit(cur, p)) return false;
            parity += count_below(cur, p);
            flip(cur, p);
            m &= m - 1;
        }
    }
#pragma unroll
    for (int w = K - 1; w >= 0; w--) {
        u64 m = e.w[w] & s.virt[w];
        while (m) {
            int b = 63 - __clzll((long long)m);
            int p = 64 * w + b;
            if (bit(cur, p)) return false;
            parity += count_below(cur, p);
            flip(cur, p);
            m &= ~(1ULL << b);
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Rank key: key = rank_V * C_O - rank_H (order-preserving on level <= l)
// ---------------------------------------------------------------------------

template <int K>
__device__ __forceinline__ u64 rank_key(const SysDev &s, const Det<K> &d)
{
    u64 rv = 0, rh = 0;
    int c = 0;
#pragma unroll
    for (int w = K - 1; w >= 0; w--) {
        u64 m = d.w[w] & s.virt[w];
        while (m) {
            int b = 63 - __clzll((long long)m);
            rv += __ldg(&s.rank_tab[c * RANK_STRIDE + (64 * w + b - s.nel)]);
            c++;
            m &= ~(1ULL << b);
        }
    }
    c = 0;
#pragma unroll
    for (int w = K - 1; w >= 0; w--) {
        u64 m = s.hf[w] & ~d.w[w];
        while (m) {
            int b = 63 - __clzll((long long)m);
            rh += __ldg(&s.rank_tab[c * RANK_STRIDE + (64 * w + b)]);
            c++;
            m &= ~(1ULL << b);
        }
    }
    return rv * s.cocc - rh;
}

template <int K>
__device__ __forceinline__ Det<K> unrank_key(const SysDev &s, u64 key)
{
    Det<K> d;
#pragma unroll
    for (int w = 0; w < K; w++) d.w[w] = s.hf[w];
    u64 rv = (key + s.cocc - 1) / s.cocc;
    u64 rh = rv * s.cocc - key;
    // digit c of a rank: the largest position q below the previous digit with
    // tab[c][q] <= rank (tab[c][q] grows with q; tab[c][0] = 1, so a zero
    // rank has no further digits) -- a binary search per digit
    int top = s.nso - s.nel;
    for (int c = 0; c <= s.lmax && rv > 0 && top > 0; c++) {
        const u64 *t = s.rank_tab + c * RANK_STRIDE;
        int lo = 0, hi = top - 1;   // tab[c][0] = 1 <= rv
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&t[mid]) <= rv) lo = mid;
            else hi = mid - 1;
        }
        rv -= __ldg(&t[lo]);
        flip(d, lo + s.nel);
        top = lo;
    }
    top = s.nel;
    for (int c = 0; c <= s.lmax && rh > 0 && top > 0; c++) {
        const u64 *t = s.rank_tab + c * RANK_STRIDE;
        int lo = 0, hi = top - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&t[mid]) <= rh) lo = mid;
            else hi = mid - 1;
        }
        rh -= __ldg(&t[lo]);
        flip(d, lo);
        top = lo;
    }
    return d;
}

// ---------------------------------------------------------------------------
// Matrix elements (Slater-Condon rules)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int ueg_n2(const SysDev &s, int p, int q)
{
    const int *a = s.kv + 3 * (p >> 1), *b = s.kv + 3 * (q >> 1);
    int dx = __ldg(a) - __ldg(b), dy = __ldg(a + 1) - __ldg(b + 1), dz = __ldg(a + 2) - __ldg(b + 2);
    return dx * dx + dy * dy + dz * dz;
}

template <typename R>
__device__ __forceinline__ R eri_at(const SysDev &s, int p, int q, int r, int t)
{
    size_t n = (size_t)s.norb;
    return __ldg(&Tab<R>::eri(s)[((p * n + q) * n + r) * n + t]);
}

// physicists' <pq|rs> for a momentum-conserving (UEG) or any (generic) quadruple
template <typename R>
__device__ __forceinline__ R g2(const SysDev &s, int p, int q, int r, int t)
{
    if (((p ^ r) & 1) || ((q ^ t) & 1)) return R(0);
    if (s.kind == 0) return __ldg(&Tab<R>::vtab(s)[ueg_n2(s, p, r)]);
    return eri_at<R>(s, p >> 1, r >> 1, q >> 1, t >> 1);
}

// <pq||pq> for p != q in the precision R: gas, minus the exchange Coulomb
// term (callers skip opposite spins, whose pair term is the omitted q = 0
// Coulomb term); molecule, (pp|qq) minus (pq|qp) for equal spins.
template <typename R>
__device__ __forceinline__ R pair_ex(const SysDev &s, int p, int q)
{
    if (s.kind == 0) return -__ldg(&Tab<R>::vtab(s)[ueg_n2(s, p, q)]);
    const int P = p >> 1, Q = q >> 1;
    R t = eri_at<R>(s, P, P, Q, Q);
    if (((p ^ q) & 1) == 0) t = t - eri_at<R>(s, P, Q, Q, P);
    return t;
}

__device__ __forceinline__ bool pair_zero(const SysDev &s, int p, int q)
{
    return s.kind == 0 && ((p ^ q) & 1);
}

// H_DD - E_HF from the excitation of D relative to HF: holes H and particles
// P ascending, sum_P F_a - sum_H F_i + sum_{i<j in H} <ij||ij>
// + sum_{a<b in P} <ab||ab> - sum_{a in P, i in H} <ai||ai>, in this order,
// in the precision R and promoted to double.  D is within the truncation
// (at most 8 holes are read).
template <int K, typename R>
__device__ __forceinline__ double diag_rel(const SysDev &s, const Det<K> &d)
{
    int hol[8], par[8], nh = 0, np = 0;
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 hm = s.hf[w] & ~d.w[w];
        u64 pm = d.w[w] & ~s.hf[w];
        while (hm) {
            if (nh < 8) hol[nh++] = 64 * w + (__ffsll((long long)hm) - 1);
            hm &= hm - 1;
        }
        while (pm) {
            if (np < 8) par[np++] = 64 * w + (__ffsll((long long)pm) - 1);
            pm &= pm - 1;
        }
    }
    const R *f = Tab<R>::fock(s);
    R e = R(0);
    for (int x = 0; x < np; x++) e = e + __ldg(&f[par[x]]);
    for (int x = 0; x < nh; x++) e = e - __ldg(&f[hol[x]]);
    for (int x = 0; x < nh; x++)
        for (int y = x + 1; y < nh; y++)
            if (!pair_zero(s, hol[x], hol[y])) e = e + pair_ex<R>(s, hol[x], hol[y]);
    for (int x = 0; x < np; x++)
        for (int y = x + 1; y < np; y++)
            if (!pair_zero(s, par[x], par[y])) e = e + pair_ex<R>(s, par[x], par[y]);
    for (int x = 0; x < np; x++)
        for (int y = 0; y < nh; y++)
            if (!pair_zero(s, par[x], hol[y])) e = e - pair_ex<R>(s, par[x], hol[y]);
    return (double)e;
}

// <bra|H|ket> for determinants differing by one or two spin-orbitals.
// holes i<j are in ket only, particles a<b in bra only; gamma is the phase of
// a+_a a+_b a_j a_i |ket> = gamma |bra>.  Computed in R, returned as double.
template <int K, typename R>
__device__ double h_offdiag(const SysDev &s, const Det<K> &ket, int nh, int i, int j, int a, int b)
{
    Det<K> cur = ket;
    int par = count_below(cur, i);
    flip(cur, i);
    if (nh == 2) {
        par += count_below(cur, j);
        flip(cur, j);
        par += count_below(cur, b);
        flip(cur, b);
    }
    par += count_below(cur, a);
    if (nh == 2) {
        R v1 = g2<R>(s, a, b, i, j);
        R v2 = g2<R>(s, a, b, j, i);
        R d = v1 - v2;
        return (double)((par & 1) ? -d : d);
    }
    if (s.kind == 0 || ((i ^ a) & 1)) return 0.0;
    int A = a >> 1, I = i >> 1;
    R acc = __ldg(&Tab<R>::h1(s)[A * s.norb + I]);
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 m = ket.w[w];
        while (m) {
            int k = 64 * w + (__ffsll((long long)m) - 1);
            m &= m - 1;
            if (k == i) continue;
            int Kk = k >> 1;
            R t = eri_at<R>(s, A, I, Kk, Kk);
            if (((a ^ k) & 1) == 0) t = t - eri_at<R>(s, A, Kk, Kk, I);
            acc = acc + t;
        }
    }
    return (double)((par & 1) ? -acc : acc);
}

// <bra|H|ket> for bra != ket by at most two spin-orbitals (else 0)
template <int K, typename R>
__device__ double h_between(const SysDev &s, const Det<K> &bra, const Det<K> &ket)
{
    int hol[2], par[2], nh = 0, np = 0;
#pragma unroll
    for (int w = 0; w < K; w++) {
        u64 hm = ket.w[w] & ~bra.w[w];
        u64 pm = bra.w[w] & ~ket.w[w];
        while (hm) {
            if (nh < 2) hol[nh] = 64 * w + (__ffsll((long long)hm) - 1);
            nh++;
            hm &= hm - 1;
        }
        while (pm) {
            if (np < 2) par[np] = 64 * w + (__ffsll((long long)pm) - 1);
            np++;
            pm &= pm - 1;
        }
    }
    if (nh != np || nh == 0 || nh > 2) return 0.0;
    return h_offdiag<K, R>(s, ket, nh, hol[0], nh == 2 ? hol[1] : 0, par[0], nh == 2 ? par[1] : 0);
}

// <HF|H|D> for D at level 1 or 2
template <int K, typename R>
__device__ __forceinline__ double h_ref(const SysDev &s, const Det<K> &d)
{
    Det<K> hf;
#pragma unroll
    for (int w = 0; w < K; w++) hf.w[w] = s.hf[w];
    return h_between<K, R>(s, hf, d);
}

// ---------------------------------------------------------------------------
// Excitation generators
// ---------------------------------------------------------------------------

// pair index -> (x < y) with index = y(y-1)/2 + x
__device__ __forceinline__ void pair_of(u64 idx, int &x, int &y)
{
    int yy = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)idx)) * 0.5f);
    if (yy < 1) yy = 1;
    while ((u64)yy * (yy - 1) / 2 > idx) yy--;
    while ((u64)(yy + 1) * yy / 2 <= idx) yy++;
    y = yy;
    x = (int)(idx - (u64)yy * (yy - 1) / 2);
}

// 1/p_gen of a generator case (0: gas double; 1, 2: molecule single of spin
// 0, 1; 3, 4, 5: molecule double of spin case 0, 1, mixed) in the precision
// R, promoted to double.
template <typename R>
__device__ __forceinline__ double inv_pgen_of(const SysDev &s, int gc)
{
    if (sizeof(R) == 4) {
        float f = gc == 0 ? s.inv_pgen_ueg_f : (gc < 3 ? s.inv_pgen_single_f[gc - 1] : s.inv_pgen_double_f[gc - 3]);
        return (double)f;
    }
    return gc == 0 ? s.inv_pgen_ueg : (gc < 3 ? s.inv_pgen_single[gc - 1] : s.inv_pgen_double[gc - 3]);
}

// One draw of the excitation generator from dj.  Returns false for a null
// draw; otherwise di, the holes (i<j) and particles (a<b) relative to dj, the
// number of holes nh and the generator case gc (see inv_pgen_of).
template <int K>
__device__ bool excite(const SysDev &s, const Det<K> &dj, const R4 &r, Det<K> &di, int &nh, int &i, int &j,
                       int &a, int &b, int &gc)
{
    if (s.kind == 0) {
        int x, y;
        pair_of(below(r.v[1], s.npairs), x, y);
        i = kth_occupied(dj, x);
        j = kth_occupied(dj, y);
        int aa = kth_empty(s, dj, below(r.v[2], s.nvirt), -1);
        if (aa < 0) return false;
        int sb = (i & 1) + (j & 1) - (aa & 1);
        if (sb < 0 || sb > 1) return false;
        const int *ki = s.kv + 3 * (i >> 1), *kj = s.kv + 3 * (j >> 1), *ka = s.kv + 3 * (aa >> 1);
        int nb0 = __ldg(ki) + __ldg(kj) - __ldg(ka);
        int nb1 = __ldg(ki + 1) + __ldg(kj + 1) - __ldg(ka + 1);
        int nb2 = __ldg(ki + 2) + __ldg(kj + 2) - __ldg(ka + 2);
        int nm = s.nmax;
        if (nb0 < -nm || nb0 > nm || nb1 < -nm || nb1 > nm || nb2 < -nm || nb2 > nm) return false;
        int bs = __ldg(&s.grid[((nb0 + nm) * s.side + (nb1 + nm)) * s.side + (nb2 + nm)]);
        if (bs < 0) return false;
        int bb = 2 * bs + sb;
        if (bb == aa || bit(dj, bb)) return false;
        a = aa < bb ? aa : bb;
        b = aa < bb ? bb : aa;
        nh = 2;
        gc = 0;
    } else if (below(r.v[0], s.ns_nd) < s.ns) {
        i = kth_occupied(dj, (int)below(r.v[1], (u64)s.nel));
        int sg = i & 1;
        if (s.nv[sg] == 0) return false;
        a = kth_empty(s, dj, below(r.v[2], (u64)s.nv[sg]), sg);
        if (a < 0) return false;
        j = b = 0;
        nh = 1;
        gc = 1 + sg;
    } else {
        int x, y;
        pair_of(below(r.v[1], s.npairs), x, y);
        i = kth_occupied(dj, x);
        j = kth_occupied(dj, y);
        int aa, bb, c;
        if (((i ^ j) & 1) == 0) {
            int sg = i & 1;
            c = sg;
            if (s.ndcase[c] == 0) return false;
            int xa, ya;
            pair_of(below(r.v[2], s.ndcase[c]), xa, ya);
            aa = kth_empty(s, dj, (u64)xa, sg);
            bb = kth_empty(s, dj, (u64)ya, sg);
        } else {
            c = 2;
            if (s.ndcase[c] == 0) return false;
            u64 q = below(r.v[2], s.ndcase[c]);
            aa = kth_empty(s, dj, q / (u64)s.nv[1], 0);
            bb = kth_empty(s, dj, q % (u64)s.nv[1], 1);
        }
        if (aa < 0 || bb < 0) return false;
        a = aa < bb ? aa : bb;
        b = aa < bb ? bb : aa;
        nh = 2;
        gc = 3 + c;
    }
    di = dj;
    flip(di, i);
    if (nh == 2) flip(di, j);
    flip(di, a);
    if (nh == 2) flip(di, b);
    return true;
}

// ---------------------------------------------------------------------------
// Stochastic rounding onto the 2^-16 grid (below cutoff: +-cutoff with
// probability |x|/cutoff).  Returns false on overflow of the fixed-point range.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool stoch_round(double x, double u, double cutoff, i64 &out)
{
    double ax = fabs(x);
    if (!(ax < 0x1p46)) {
        out = 0;
        return false;
    }
    i64 n;
    if (ax < cutoff) {
        n = (u * cutoff < ax) ? (i64)(cutoff * FIX_ONE) : 0;
    } else {
        double q = ax * FIX_ONE;
        double f = floor(q);
        n = (i64)f + ((u < q - f) ? 1 : 0);
    }
    out = x < 0.0 ? -n : n;
    return true;
}

// The same decision taken with integer arithmetic on the FP64 bit pattern.
// Every FP64 operation of stoch_round is exact -- scaling by 2^16, floor, the
// subtraction q - f, the 53-bit uniform u and, for a power-of-two cutoff,
// u * cutoff -- so comparing the exact values as scaled integers reproduces
// it bit for bit without using the (narrow) FP64 pipe.

// a * 2^sa < b * 2^sb for unsigned a, b
__host__ __device__ __forceinline__ bool lt_scaled(u64 a, int sa, u64 b, int sb)
{
    int d = sa - sb;
    if (d >= 0) {                       // a * 2^d < b
        if (a == 0) return b != 0;
        if (d >= 64) return false;
        if (d > 0 && (a >> (64 - d)) != 0) return false;
        return (a << d) < b;
    }
    int e = -d;                         // a < b * 2^e
    if (b == 0) return false;
    if (e >= 64) return true;
    if ((b >> (64 - e)) != 0) return true;
    return a < (b << e);
}

// |x| = M * 2^E exactly (M < 2^53)
__host__ __device__ __forceinline__ void split_double(u64 abits, u64 &M, int &E)
{
    u64 ex = abits >> 52, fr = abits & ((1ULL << 52) - 1ULL);
    if (ex == 0) {
        M = fr;
        E = -1074;
    } else {
        M = fr | (1ULL << 52);
        E = (int)ex - 1075;
    }
}

// Rounding parameters: cutoff must be 0 or a power of two (checked on the host).
struct RoundSpec {
    u64 cutoff_bits;   // bit pattern of the cutoff (0 = no cutoff)
    int cutoff_e;      // u * cutoff = m_u * 2^cutoff_e
    i64 cutoff_fixed;  // cutoff in fixed point
};

__host__ __device__ __forceinline__ bool stoch_round_bits(u64 xbits, u64 r, const RoundSpec &rs, i64 &out)
{
    const bool neg = (xbits >> 63) != 0;
    const u64 ab = xbits & 0x7FFFFFFFFFFFFFFFULL;
    if (!(ab < 0x42D0000000000000ULL)) {   // |x| < 2^46 (also rejects inf and NaN)
        out = 0;
        return false;
    }
    const u64 mu = r >> 11;                // u = mu * 2^-53
    u64 M;
    int E;
    split_double(ab, M, E);
    i64 n;
    if (ab < rs.cutoff_bits) {             // |x| < cutoff
        n = lt_scaled(mu, rs.cutoff_e, M, E) ? rs.cutoff_fixed : 0;
    } else {
        int e = E + 16;                    // q = |x| 2^16 = M 2^e
        if (e >= 0) {
            n = (i64)(M << e);
        } else {
            int t = -e;
            u64 f = t >= 64 ? 0 : (M >> t);
            u64 fr = t >= 64 ? M : (M & ((1ULL << t) - 1ULL));
            n = (i64)f + (lt_scaled(mu, -53, fr, -t) ? 1 : 0);
        }
    }
    out = neg ? -n : n;
    return true;
}

// ---------------------------------------------------------------------------
// Exact fixed-point accumulation of FP64 terms: each term is truncated to a
// multiple of 2^-64 and summed as a 128-bit two's-complement integer, so the
// sum is independent of the order of the terms and uses no FP64 operations.
// ---------------------------------------------------------------------------

struct Fix128 {
    u64 lo, hi;
    __host__ __device__ __forceinline__ void add(const Fix128 &b)
    {
        u64 l = lo + b.lo;
        hi = hi + b.hi + (l < lo ? 1ULL : 0ULL);
        lo = l;
    }
};

__host__ __device__ __forceinline__ Fix128 to_fix(double x)
{
    u64 bits;
    memcpy(&bits, &x, 8);
    Fix128 r = {0, 0};
    u64 ab = bits & 0x7FFFFFFFFFFFFFFFULL;
    if (ab >= 0x43E0000000000000ULL) return r;   // |x| >= 2^63: out of range (not produced by the step)
    u64 M;
    int E;
    split_double(ab, M, E);
    int sft = E + 64;                            // value * 2^64 = M * 2^sft
    if (sft >= 64) {
        r.hi = M << (sft - 64);
    } else if (sft > 0) {
        r.lo = M << sft;
        r.hi = M >> (64 - sft);
    } else if (sft > -64) {
        r.lo = M >> (-sft);
    }
    if (bits >> 63) {                            // negate
        r.lo = ~r.lo;
        r.hi = ~r.hi;
        u64 l = r.lo + 1;
        r.hi += (l == 0) ? 1ULL : 0ULL;
        r.lo = l;
    }
    return r;
}

__host__ __device__ __forceinline__ double fix_to_double(Fix128 v)
{
    bool neg = (v.hi >> 63) != 0;
    if (neg) {
        v.lo = ~v.lo;
        v.hi = ~v.hi;
        u64 l = v.lo + 1;
        v.hi += (l == 0) ? 1ULL : 0ULL;
        v.lo = l;
    }
    double d = (double)v.hi + (double)v.lo * 0x1p-64;
    return neg ? -d : d;
}

// ---------------------------------------------------------------------------
// Neumaier-compensated accumulation
// ---------------------------------------------------------------------------

struct KSum {
    double s, c;
    __device__ __forceinline__ void add(double x)
    {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ void merge(const KSum &o)
    {
        add(o.s);
        add(o.c);
    }
};

}  // namespace ccmc
