/*
 * ccmc_oracle.c -- plain, slow, CPU reference of one coupled cluster Monte
 * Carlo (CCMC) time step, written from Spencer et al., "Large Scale
 * Parallelization in Stochastic Coupled Cluster" (arXiv:1807.03749).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file.  It shares no code with the CUDA
 * path: both sides implement the same written conventions independently.
 *
 * Everything is FP64, compiled with -ffp-contract=off so that no multiply-add
 * is fused (aarch64 GCC fuses by default).  Populations are int64 fixed point
 * with 2^-16 resolution.  Random numbers come from Philox-4x64-10 (Salmon et
 * al., SC'11), keyed by (seed, replica) and counted by (iteration, tag|index,
 * block, 0), so every sample is a pure function of its counter.
 *
 * Paper passages followed:
 *   Sec. II, Eq. 1-2        CC ansatz Psi = t_HF exp(T/t_HF)|D_HF>
 *   Sec. II, Eq. (CCMC)     linearised propagator t_i -= dtau sum_j (H_ij - S d_ij) t~_j
 *   Sec. II (+footnote)     p_size(s) = 2^-(s+1), s in [0, l+2], last bin = remainder;
 *                           excitors drawn with |t_i|/(N_total - t_HF); repeats discarded
 *   Sec. II                 spawn / death / annihilation, truncation discard
 *   Sec. II, Eq. 3-5        excitor and determinant operator ordering, s_D(i)
 *   Sec. II, Eq. (E_proj)   projected energy estimator
 *   Sec. II                 shift held then varied to keep the population stable
 *   Sec. IV.B               full non-composite (FNC) sampling
 *   Sec. IV.C, Eq. 7-8      multi-spawn: n_attempts = max(1, floor(A/A_thresh))
 *   Sec. III, Eq. ccmc_dist simulated distribution over N_p processors: owner
 *                           hash; composite clusters from one processor's excitors
 *
 * Diagonal energies H_DD - E_HF use the excitation form (reference Fock
 * diagonal plus pair corrections among holes and particles), pinned against
 * the plain Slater-Condon diagonal.  The FP32 mode (matrix elements,
 * diagonal energies and 1/p_gen in single precision from tables rounded from
 * FP64) is a convention shared with the CUDA path; its energies are pinned
 * only to an accuracy band: parity unpinned for the FP32 energies.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OW 6                 /* maximum words per bit string (M <= 384) */
#define OBINOM 385           /* binomial table rows C(n, k), n <= 384 */
#define FIX_ONE 65536.0      /* populations are multiples of 2^-16 */
#define FIX_SHIFT 16
#define ORC_PI 3.14159265358979323846

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_OOM = 3, ORC_ERR_NUMERIC = 6 };

/* Philox counter tags (word 1 of the counter, bits 56..63). */
enum {
    TAG_SAMPLE = 1,      /* cluster selection of sample g                  */
    TAG_SAMPLE_ATT = 2,  /* spawning attempt m of sample g                 */
    TAG_VISIT = 3,       /* FNC death draw of list entry i                 */
    TAG_VISIT_ATT = 4,   /* FNC spawning attempt m of list entry i         */
    TAG_THRESH = 5       /* occupation threshold of excitor with rank key  */
};

typedef struct { uint64_t w[OW]; } det_t;

/* ------------------------------------------------------------------------- */
/* Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).                        */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, x0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B97F4A7C15ULL;   /* Weyl key schedule */
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* The paper's distribution of excitors over N_p processors (Sec. III,       */
/* Eq. ccmc_dist), simulated: a determinant hash (any good hash will do;     */
/* here Philox-4x64-10 under a fixed key used as a mixing function over the  */
/* bit string, three words per call, each call taking the previous result as */
/* its fourth counter word) and the owner                                    */
/*   o(D, i) = (hash(D) + i) >> nu_move,   p(D, i) = hash(D xor o) mod N_p,  */
/* with o xor-ed into the first word of the bit string.                     */
/* ------------------------------------------------------------------------- */

static const uint64_t HASH_KEY[2] = { 0x243F6A8885A308D3ULL, 0x13198A2E03707344ULL };

static uint64_t det_hash(const uint64_t *w, int nw)
{
    uint64_t h = 0;
    for (int g = 0; g < nw; g += 3) {
        uint64_t c[4] = { w[g], g + 1 < nw ? w[g + 1] : 0, g + 2 < nw ? w[g + 2] : 0, h }, out[4];
        orc_philox(c, HASH_KEY, out);
        h = out[0];
    }
    return h;
}

uint64_t orc_det_hash(const uint64_t *w, int nw) { return det_hash(w, nw); }

uint64_t orc_owner(const uint64_t *w, int nw, uint64_t iter, int nu_move, uint64_t n_ranks)
{
    uint64_t h = det_hash(w, nw);
    uint64_t o = nu_move >= 64 ? 0 : (h + iter) >> nu_move;
    uint64_t x[OW];
    for (int i = 0; i < nw; i++) x[i] = w[i];
    x[0] ^= o;
    return det_hash(x, nw) % n_ranks;
}

/* Co-location of excitor pairs (Fig. excitdistrib): for T = 1..t_max, the
   sums over pairs i < j of C_ij(T) and C_ij(T)^2, where C_ij(T) counts the
   iterations t < T at which excitors i and j have the same owner; reported
   at the nck checkpoints tcheck[] (ascending). */
void orc_colocation(const uint64_t *dets, int64_t n, int nw, int64_t n_ranks, int nu_move, int64_t t_max,
                    const int64_t *tcheck, int nck, uint64_t *sum_c, uint64_t *sum_c2)
{
    int64_t *own = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n * t_max));
    int64_t *cnt = (int64_t *)calloc((size_t)(n * (n - 1) / 2 + 1), sizeof(int64_t));
    for (int64_t t = 0; t < t_max; t++)
        for (int64_t i = 0; i < n; i++)
            own[t * n + i] = (int64_t)orc_owner(dets + i * nw, nw, (uint64_t)t, nu_move, (uint64_t)n_ranks);
    for (int k = 0; k < nck; k++) { sum_c[k] = 0; sum_c2[k] = 0; }
    int k = 0;
    for (int64_t t = 0; t < t_max && k < nck; t++) {
        int64_t q = 0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = i + 1; j < n; j++, q++)
                if (own[t * n + i] == own[t * n + j]) cnt[q]++;
        while (k < nck && tcheck[k] == t + 1) {
            q = 0;
            for (int64_t i = 0; i < n; i++)
                for (int64_t j = i + 1; j < n; j++, q++) {
                    sum_c[k] += (uint64_t)cnt[q];
                    sum_c2[k] += (uint64_t)(cnt[q] * cnt[q]);
                }
            k++;
        }
    }
    free(own);
    free(cnt);
}

static void draw4(const uint64_t key[2], uint64_t it, uint64_t tag, uint64_t index,
                  uint64_t block, uint64_t out[4])
{
    uint64_t ctr[4] = { it, (tag << 56) | index, block, 0 };
    orc_philox(ctr, key, out);
}

/* Uniform double in [0,1) from the top 53 bits. */
static double unif(uint64_t r) { return (double)(r >> 11) * 0x1p-53; }

/* Integer in [0, n) as the high word of r*n. */
static uint64_t below(uint64_t r, uint64_t n)
{
    uint64_t hi, lo;
    mulhilo64(r, n, &hi, &lo);
    return hi;
}

/* ------------------------------------------------------------------------- */
/* Bit strings: spin-orbital p is bit p&63 of word p>>6; 2q = alpha, 2q+1 =   */
/* beta of spatial orbital q.  Determinants are ordered as unsigned integers   */
/* compared from the most significant word.                                    */
/* ------------------------------------------------------------------------- */

static int det_bit(const det_t *d, int p) { return (int)((d->w[p >> 6] >> (p & 63)) & 1ULL); }
static void det_set(det_t *d, int p) { d->w[p >> 6] |= 1ULL << (p & 63); }
static void det_clr(det_t *d, int p) { d->w[p >> 6] &= ~(1ULL << (p & 63)); }

/* Number of occupied spin-orbitals strictly below p. */
static int det_count_below(const det_t *d, int p)
{
    int c = 0;
    for (int q = 0; q < p; q++) c += det_bit(d, q);
    return c;
}

static int det_popcount(const det_t *d, int nw)
{
    int c = 0;
    for (int i = 0; i < nw; i++) c += __builtin_popcountll(d->w[i]);
    return c;
}

static int det_equal(const det_t *a, const det_t *b, int nw)
{
    for (int i = 0; i < nw; i++) if (a->w[i] != b->w[i]) return 0;
    return 1;
}

/* Sign of applying the annihilator a_p (p occupied) or creator a+_p (p empty):
 * (-1)^(number of occupied orbitals below p), Sec. II Eq. 4 ordering. */
static int op_phase(const det_t *d, int p) { return (det_count_below(d, p) & 1) ? -1 : 1; }

/* ------------------------------------------------------------------------- */
/* Systems                                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int kind;            /* 0 = uniform electron gas, 1 = generic integrals */
    int nel, nso, nw, lmax;
    det_t hf;
    /* UEG (plane waves sorted by |n|^2 then lexicographic n) */
    double rs, L;
    int npw, nmax;       /* largest |component| of any basis vector */
    int (*kv)[3];        /* integer wave vector per spatial orbital */
    int *grid;           /* (2 nmax+1)^3 lookup: spatial index or -1 */
    double *tkin;        /* kinetic energy per spin-orbital */
    double *vtab;        /* Coulomb 1/(pi L n^2) by integer n^2 */
    int n2tab;
    /* generic integrals */
    int norb;
    double *h1;          /* norb x norb */
    double *eri;         /* norb^4, chemists' (pq|rs), fully symmetric */
    double ecore;
    /* common */
    double ehf_rel;      /* <HF|H|HF> without the constant ecore */
    double *fock;        /* F_p = h_pp + sum_{k in HF, k != p} <pk||pk>, per spin-orbital */
    uint64_t binom[OBINOM][8];
    uint64_t cocc;       /* number of hole sets with <= l holes */
    uint64_t nvranks;    /* number of particle sets with <= l particles */
    /* excitation generator constants */
    uint64_t npairs, nvirt;
    double inv_pgen_ueg;
    int no[2], nv[2];
    uint64_t ns, nd, ndcase[3];
    double inv_pgen_single[2], inv_pgen_double[3];
    /* FP32 form: matrix elements and generation probabilities in single
     * precision from tables rounded from the FP64 ones */
    int fp32;
    float *tkin_f, *vtab_f, *h1_f, *eri_f;
    float *fock_f;       /* F rounded to single precision */
    float ehf_rel_f;
    float inv_pgen_ueg_f, inv_pgen_single_f[2], inv_pgen_double_f[3];
} orc_system;

static int spin_of(int p) { return p & 1; }
static int spat_of(int p) { return p >> 1; }

static void fill_binom(orc_system *s)
{
    for (int n = 0; n < OBINOM; n++)
        for (int k = 0; k < 8; k++) {
            if (k == 0) s->binom[n][k] = 1;
            else if (n == 0) s->binom[n][k] = 0;
            else s->binom[n][k] = s->binom[n - 1][k - 1] + s->binom[n - 1][k];
        }
}

static uint64_t count_upto(const orc_system *s, int n, int kmax)
{
    uint64_t c = 0;
    for (int j = 0; j <= kmax; j++) c += s->binom[n][j];
    return c;
}

static double h_diag_abs(const orc_system *s, const det_t *d);
static int fock_setup(orc_system *s);

static int common_setup(orc_system *s)
{
    fill_binom(s);
    s->nw = (s->nso + 63) / 64;
    memset(&s->hf, 0, sizeof(det_t));
    for (int p = 0; p < s->nel; p++) det_set(&s->hf, p);
    s->cocc = count_upto(s, s->nel, s->lmax);
    s->nvranks = count_upto(s, s->nso - s->nel, s->lmax);
    s->npairs = (uint64_t)s->nel * (uint64_t)(s->nel - 1) / 2;
    s->nvirt = (uint64_t)(s->nso - s->nel);
    s->ehf_rel = h_diag_abs(s, &s->hf);
    return fock_setup(s);
}

static int cmp_kvec(const void *a, const void *b)
{
    const int *x = (const int *)a, *y = (const int *)b;
    int nx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    int ny = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if (nx != ny) return nx < ny ? -1 : 1;
    for (int i = 0; i < 3; i++) if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

void orc_system_free(orc_system *s)
{
    if (!s) return;
    free(s->kv); free(s->grid); free(s->tkin); free(s->vtab);
    free(s->h1); free(s->eri);
    free(s->tkin_f); free(s->vtab_f); free(s->h1_f); free(s->eri_f);
    free(s->fock); free(s->fock_f);
    free(s);
}

/* Uniform electron gas in a cubic box: plane waves k = 2 pi n / L with
 * L = r_s (4 pi N / 3)^(1/3); kinetic energy |k|^2/2; Coulomb
 * 4 pi/(Omega |q|^2) = 1/(pi L |n_q|^2) with the q = 0 term omitted. */
orc_system *orc_ueg_new(int nel, int nso, double rs, int lmax)
{
    if (nel < 2 || nso <= nel || nso > 64 * OW || (nso & 1) || lmax < 1 || lmax > 4) return NULL;
    orc_system *s = (orc_system *)calloc(1, sizeof(orc_system));
    if (!s) return NULL;
    s->kind = 0; s->nel = nel; s->nso = nso; s->lmax = lmax; s->rs = rs;
    s->npw = nso / 2;
    /* smallest cutoff |n|^2 <= ecut whose shell count equals npw */
    int found = -1, cnt = 0;
    for (int ecut = 0; ecut < 100 && found < 0; ecut++) {
        cnt = 0;
        int r = (int)ceil(sqrt((double)ecut)) + 1;
        for (int x = -r; x <= r; x++)
            for (int y = -r; y <= r; y++)
                for (int z = -r; z <= r; z++)
                    if (x * x + y * y + z * z <= ecut) cnt++;
        if (cnt == s->npw) found = ecut;
        if (cnt > s->npw) break;
    }
    if (found < 0) { free(s); return NULL; }
    s->kv = (int (*)[3])calloc((size_t)s->npw, sizeof(int[3]));
    int r = (int)ceil(sqrt((double)found)) + 1, m = 0;
    for (int x = -r; x <= r; x++)
        for (int y = -r; y <= r; y++)
            for (int z = -r; z <= r; z++)
                if (x * x + y * y + z * z <= found) {
                    s->kv[m][0] = x; s->kv[m][1] = y; s->kv[m][2] = z; m++;
                }
    qsort(s->kv, (size_t)s->npw, sizeof(int[3]), cmp_kvec);
    s->nmax = 0;
    for (int i = 0; i < s->npw; i++)
        for (int c = 0; c < 3; c++) {
            int a = abs(s->kv[i][c]);
            if (a > s->nmax) s->nmax = a;
        }
    int side = 2 * s->nmax + 1;
    s->grid = (int *)malloc(sizeof(int) * (size_t)side * side * side);
    for (int i = 0; i < side * side * side; i++) s->grid[i] = -1;
    for (int i = 0; i < s->npw; i++) {
        int gx = s->kv[i][0] + s->nmax, gy = s->kv[i][1] + s->nmax, gz = s->kv[i][2] + s->nmax;
        s->grid[(gx * side + gy) * side + gz] = i;
    }
    s->L = rs * cbrt((4.0 * ORC_PI * (double)nel) / 3.0);
    s->tkin = (double *)malloc(sizeof(double) * (size_t)nso);
    for (int p = 0; p < nso; p++) {
        const int *k = s->kv[spat_of(p)];
        int n2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        s->tkin[p] = ((2.0 * ORC_PI * ORC_PI) * (double)n2) / (s->L * s->L);
    }
    s->n2tab = 12 * s->nmax * s->nmax + 1;
    s->vtab = (double *)malloc(sizeof(double) * (size_t)s->n2tab);
    s->vtab[0] = 0.0;
    for (int n2 = 1; n2 < s->n2tab; n2++) s->vtab[n2] = 1.0 / ((ORC_PI * s->L) * (double)n2);
    if (common_setup(s)) { orc_system_free(s); return NULL; }
    s->inv_pgen_ueg = (double)(s->npairs * s->nvirt) * 0.5;
    return s;
}

/* Generic Hamiltonian from spatial integrals: h1[p][q] and chemists'
 * (pq|rs) stored densely (norb^4), used for the molecule-like system. */
orc_system *orc_generic_new(int nel, int norb, const double *h1, const double *eri, double ecore, int lmax)
{
    int nso = 2 * norb;
    if (nel < 2 || nso <= nel || nso > 64 * OW || lmax < 1 || lmax > 4) return NULL;
    orc_system *s = (orc_system *)calloc(1, sizeof(orc_system));
    if (!s) return NULL;
    s->kind = 1; s->nel = nel; s->nso = nso; s->lmax = lmax; s->norb = norb; s->ecore = ecore;
    size_t n2 = (size_t)norb * norb, n4 = n2 * n2;
    s->h1 = (double *)malloc(sizeof(double) * n2);
    s->eri = (double *)malloc(sizeof(double) * n4);
    if (!s->h1 || !s->eri) { orc_system_free(s); return NULL; }
    memcpy(s->h1, h1, sizeof(double) * n2);
    memcpy(s->eri, eri, sizeof(double) * n4);
    if (common_setup(s)) { orc_system_free(s); return NULL; }
    /* spin-resolved occupied / virtual counts of the reference */
    s->no[0] = s->no[1] = 0;
    for (int p = 0; p < nel; p++) s->no[spin_of(p)]++;
    s->nv[0] = norb - s->no[0];
    s->nv[1] = norb - s->no[1];
    s->ns = (uint64_t)s->no[0] * s->nv[0] + (uint64_t)s->no[1] * s->nv[1];
    s->ndcase[0] = s->binom[s->nv[0]][2];                   /* alpha-alpha */
    s->ndcase[1] = s->binom[s->nv[1]][2];                   /* beta-beta   */
    s->ndcase[2] = (uint64_t)s->nv[0] * (uint64_t)s->nv[1];  /* alpha-beta  */
    s->nd = s->binom[s->no[0]][2] * s->ndcase[0] + s->binom[s->no[1]][2] * s->ndcase[1]
          + (uint64_t)s->no[0] * s->no[1] * s->ndcase[2];
    for (int sg = 0; sg < 2; sg++)
        s->inv_pgen_single[sg] = ((double)((uint64_t)nel * (uint64_t)s->nv[sg]) * (double)(s->ns + s->nd)) / (double)s->ns;
    for (int c = 0; c < 3; c++)
        s->inv_pgen_double[c] = ((double)(s->npairs * s->ndcase[c]) * (double)(s->ns + s->nd)) / (double)s->nd;
    return s;
}

/* ------------------------------------------------------------------------- */
/* Integrals and Slater-Condon rules                                          */
/* ------------------------------------------------------------------------- */

static double eri_at(const orc_system *s, int p, int q, int r, int t)
{
    size_t n = (size_t)s->norb;
    return s->eri[((p * n + q) * n + r) * n + t];
}

static int ueg_n2_between(const orc_system *s, int p, int q)
{
    const int *a = s->kv[spat_of(p)], *b = s->kv[spat_of(q)];
    int dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Physicists' <pq|rs> = integral p*(1) q*(2) r12^-1 r(1) s(2). */
static double g2(const orc_system *s, int p, int q, int r, int t)
{
    if (spin_of(p) != spin_of(r) || spin_of(q) != spin_of(t)) return 0.0;
    if (s->kind == 0) {
        const int *kp = s->kv[spat_of(p)], *kq = s->kv[spat_of(q)];
        const int *kr = s->kv[spat_of(r)], *kt = s->kv[spat_of(t)];
        for (int c = 0; c < 3; c++) if (kp[c] + kq[c] != kr[c] + kt[c]) return 0.0;
        return s->vtab[ueg_n2_between(s, p, r)];
    }
    return eri_at(s, spat_of(p), spat_of(r), spat_of(q), spat_of(t));
}

/* <D|H|D> without the constant core energy, canonical summation order:
 * one-body terms over occupied p ascending, then pairs p<q ascending. */
static double h_diag_abs(const orc_system *s, const det_t *d)
{
    int occ[64 * OW], n = 0;
    for (int p = 0; p < s->nso; p++) if (det_bit(d, p)) occ[n++] = p;
    if (s->kind == 0) {
        double tsum = 0.0, xsum = 0.0;
        for (int i = 0; i < n; i++) tsum = tsum + s->tkin[occ[i]];
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++)
                if (spin_of(occ[i]) == spin_of(occ[j]))
                    xsum = xsum + s->vtab[ueg_n2_between(s, occ[i], occ[j])];
        return tsum - xsum;
    }
    double e1 = 0.0, e2 = 0.0;
    for (int i = 0; i < n; i++) {
        int P = spat_of(occ[i]);
        e1 = e1 + s->h1[P * s->norb + P];
    }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            int P = spat_of(occ[i]), Q = spat_of(occ[j]);
            double t = eri_at(s, P, P, Q, Q);
            if (spin_of(occ[i]) == spin_of(occ[j])) t = t - eri_at(s, P, Q, Q, P);
            e2 = e2 + t;
        }
    return e1 + e2;
}

/* <pq||pq> = <pq|pq> - <pq|qp> for p != q.  Gas: the direct term is the
 * omitted q = 0 Coulomb term, so only the exchange of equal spins remains
 * (callers skip pairs of opposite spin there).  Molecule: (pp|qq) minus
 * (pq|qp) for equal spins. */
static double pair_ex(const orc_system *s, int p, int q)
{
    if (s->kind == 0) return -s->vtab[ueg_n2_between(s, p, q)];
    int P = spat_of(p), Q = spat_of(q);
    double t = eri_at(s, P, P, Q, Q);
    if (spin_of(p) == spin_of(q)) t = t - eri_at(s, P, Q, Q, P);
    return t;
}

static int pair_zero(const orc_system *s, int p, int q)
{
    return s->kind == 0 && spin_of(p) != spin_of(q);
}

/* Fock diagonal of the reference, per spin-orbital: one-body term, then
 * <pk||pk> over the occupied k != p ascending. */
static int fock_setup(orc_system *s)
{
    s->fock = (double *)malloc(sizeof(double) * (size_t)s->nso);
    if (!s->fock) return ORC_ERR_OOM;
    for (int p = 0; p < s->nso; p++) {
        double f = s->kind == 0 ? s->tkin[p] : s->h1[spat_of(p) * s->norb + spat_of(p)];
        for (int k = 0; k < s->nel; k++) {
            if (k == p || pair_zero(s, p, k)) continue;
            f = f + pair_ex(s, p, k);
        }
        s->fock[p] = f;
    }
    return 0;
}

/* H_DD - E_HF from the excitation of D relative to HF (holes H, particles P,
 * both ascending): sum_P F_a - sum_H F_i + sum_{i<j in H} <ij||ij>
 * + sum_{a<b in P} <ab||ab> - sum_{a in P, i in H} <ai||ai>, in this order.
 * It equals the difference of the two Slater-Condon diagonals (both without
 * the core constant). */
static double h_diag_rel(const orc_system *s, const det_t *d)
{
    int hol[64 * OW], par[64 * OW], nh = 0, np = 0;
    for (int p = 0; p < s->nso; p++) {
        int b = det_bit(d, p), r = det_bit(&s->hf, p);
        if (r && !b) hol[nh++] = p;
        if (b && !r) par[np++] = p;
    }
    double e = 0.0;
    for (int x = 0; x < np; x++) e = e + s->fock[par[x]];
    for (int x = 0; x < nh; x++) e = e - s->fock[hol[x]];
    for (int x = 0; x < nh; x++)
        for (int y = x + 1; y < nh; y++)
            if (!pair_zero(s, hol[x], hol[y])) e = e + pair_ex(s, hol[x], hol[y]);
    for (int x = 0; x < np; x++)
        for (int y = x + 1; y < np; y++)
            if (!pair_zero(s, par[x], par[y])) e = e + pair_ex(s, par[x], par[y]);
    for (int x = 0; x < np; x++)
        for (int y = 0; y < nh; y++)
            if (!pair_zero(s, par[x], hol[y])) e = e - pair_ex(s, par[x], hol[y]);
    return e;
}

/* <bra|H|ket> for canonical determinants.  The phase gamma is that of
 * a+_a a+_b a_j a_i |ket> = gamma |bra> (holes i<j annihilated in ascending
 * order, particles a<b created in descending order). */
double orc_hij(const orc_system *s, const uint64_t *bra_w, const uint64_t *ket_w)
{
    det_t bra = {{0}}, ket = {{0}};
    for (int i = 0; i < s->nw; i++) { bra.w[i] = bra_w[i]; ket.w[i] = ket_w[i]; }
    int holes[64 * OW], parts[64 * OW], nh = 0, np = 0;
    for (int p = 0; p < s->nso; p++) {
        int b = det_bit(&bra, p), k = det_bit(&ket, p);
        if (k && !b) holes[nh++] = p;
        if (b && !k) parts[np++] = p;
    }
    if (nh != np) return 0.0;
    if (nh == 0) return h_diag_abs(s, &ket) + s->ecore;
    if (nh > 2) return 0.0;
    det_t cur = ket;
    int gamma = 1;
    for (int m = 0; m < nh; m++) { gamma *= op_phase(&cur, holes[m]); det_clr(&cur, holes[m]); }
    for (int m = np - 1; m >= 0; m--) { gamma *= op_phase(&cur, parts[m]); det_set(&cur, parts[m]); }
    if (nh == 1) {
        int i = holes[0], a = parts[0];
        if (spin_of(i) != spin_of(a) || s->kind == 0) return 0.0;
        int A = spat_of(a), I = spat_of(i);
        double acc = s->h1[A * s->norb + I];
        for (int k = 0; k < s->nso; k++) {
            if (!det_bit(&ket, k) || k == i) continue;
            int K = spat_of(k);
            double t = eri_at(s, A, I, K, K);
            if (spin_of(a) == spin_of(k)) t = t - eri_at(s, A, K, K, I);
            acc = acc + t;
        }
        return gamma > 0 ? acc : -acc;
    }
    int i = holes[0], j = holes[1], a = parts[0], b = parts[1];
    double v1 = g2(s, a, b, i, j);
    double v2 = g2(s, a, b, j, i);
    double d = v1 - v2;
    return gamma > 0 ? d : -d;
}

/* ------------------------------------------------------------------------- */
/* FP32 form of the same matrix elements (same operation order, float        */
/* arithmetic on float tables).                                              */
/* ------------------------------------------------------------------------- */

static float eri_f_at(const orc_system *s, int p, int q, int r, int t)
{
    size_t n = (size_t)s->norb;
    return s->eri_f[((p * n + q) * n + r) * n + t];
}

static float g2_f(const orc_system *s, int p, int q, int r, int t)
{
    if (spin_of(p) != spin_of(r) || spin_of(q) != spin_of(t)) return 0.0f;
    if (s->kind == 0) {
        const int *kp = s->kv[spat_of(p)], *kq = s->kv[spat_of(q)];
        const int *kr = s->kv[spat_of(r)], *kt = s->kv[spat_of(t)];
        for (int c = 0; c < 3; c++) if (kp[c] + kq[c] != kr[c] + kt[c]) return 0.0f;
        return s->vtab_f[ueg_n2_between(s, p, r)];
    }
    return eri_f_at(s, spat_of(p), spat_of(r), spat_of(q), spat_of(t));
}

static float h_diag_abs_f(const orc_system *s, const det_t *d)
{
    int occ[64 * OW], n = 0;
    for (int p = 0; p < s->nso; p++) if (det_bit(d, p)) occ[n++] = p;
    if (s->kind == 0) {
        float tsum = 0.0f, xsum = 0.0f;
        for (int i = 0; i < n; i++) tsum = tsum + s->tkin_f[occ[i]];
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++)
                if (spin_of(occ[i]) == spin_of(occ[j]))
                    xsum = xsum + s->vtab_f[ueg_n2_between(s, occ[i], occ[j])];
        return tsum - xsum;
    }
    float e1 = 0.0f, e2 = 0.0f;
    for (int i = 0; i < n; i++) {
        int P = spat_of(occ[i]);
        e1 = e1 + s->h1_f[P * s->norb + P];
    }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            int P = spat_of(occ[i]), Q = spat_of(occ[j]);
            float t = eri_f_at(s, P, P, Q, Q);
            if (spin_of(occ[i]) == spin_of(occ[j])) t = t - eri_f_at(s, P, Q, Q, P);
            e2 = e2 + t;
        }
    return e1 + e2;
}

static float pair_ex_f(const orc_system *s, int p, int q)
{
    if (s->kind == 0) return -s->vtab_f[ueg_n2_between(s, p, q)];
    int P = spat_of(p), Q = spat_of(q);
    float t = eri_f_at(s, P, P, Q, Q);
    if (spin_of(p) == spin_of(q)) t = t - eri_f_at(s, P, Q, Q, P);
    return t;
}

/* The excitation form of H_DD - E_HF in single precision: Fock diagonal
 * rounded from FP64, pair terms from the rounded tables, same order. */
static float h_diag_rel_f(const orc_system *s, const det_t *d)
{
    int hol[64 * OW], par[64 * OW], nh = 0, np = 0;
    for (int p = 0; p < s->nso; p++) {
        int b = det_bit(d, p), r = det_bit(&s->hf, p);
        if (r && !b) hol[nh++] = p;
        if (b && !r) par[np++] = p;
    }
    float e = 0.0f;
    for (int x = 0; x < np; x++) e = e + s->fock_f[par[x]];
    for (int x = 0; x < nh; x++) e = e - s->fock_f[hol[x]];
    for (int x = 0; x < nh; x++)
        for (int y = x + 1; y < nh; y++)
            if (!pair_zero(s, hol[x], hol[y])) e = e + pair_ex_f(s, hol[x], hol[y]);
    for (int x = 0; x < np; x++)
        for (int y = x + 1; y < np; y++)
            if (!pair_zero(s, par[x], par[y])) e = e + pair_ex_f(s, par[x], par[y]);
    for (int x = 0; x < np; x++)
        for (int y = 0; y < nh; y++)
            if (!pair_zero(s, par[x], hol[y])) e = e - pair_ex_f(s, par[x], hol[y]);
    return e;
}

/* <bra|H|ket> in single precision for bra != ket (0 for the diagonal). */
static float hij_f(const orc_system *s, const det_t *bra, const det_t *ket)
{
    int holes[64 * OW], parts[64 * OW], nh = 0, np = 0;
    for (int p = 0; p < s->nso; p++) {
        int b = det_bit(bra, p), k = det_bit(ket, p);
        if (k && !b) holes[nh++] = p;
        if (b && !k) parts[np++] = p;
    }
    if (nh != np || nh == 0 || nh > 2) return 0.0f;
    det_t cur = *ket;
    int gamma = 1;
    for (int m = 0; m < nh; m++) { gamma *= op_phase(&cur, holes[m]); det_clr(&cur, holes[m]); }
    for (int m = np - 1; m >= 0; m--) { gamma *= op_phase(&cur, parts[m]); det_set(&cur, parts[m]); }
    if (nh == 1) {
        int i = holes[0], a = parts[0];
        if (spin_of(i) != spin_of(a) || s->kind == 0) return 0.0f;
        int A = spat_of(a), I = spat_of(i);
        float acc = s->h1_f[A * s->norb + I];
        for (int k = 0; k < s->nso; k++) {
            if (!det_bit(ket, k) || k == i) continue;
            int K = spat_of(k);
            float t = eri_f_at(s, A, I, K, K);
            if (spin_of(a) == spin_of(k)) t = t - eri_f_at(s, A, K, K, I);
            acc = acc + t;
        }
        return gamma > 0 ? acc : -acc;
    }
    float v1 = g2_f(s, parts[0], parts[1], holes[0], holes[1]);
    float v2 = g2_f(s, parts[0], parts[1], holes[1], holes[0]);
    float d = v1 - v2;
    return gamma > 0 ? d : -d;
}

/* Switch a system to the FP32 form. */
int orc_system_set_fp32(orc_system *s)
{
    if (s->kind == 0) {
        s->tkin_f = (float *)malloc(sizeof(float) * (size_t)s->nso);
        s->vtab_f = (float *)malloc(sizeof(float) * (size_t)s->n2tab);
        if (!s->tkin_f || !s->vtab_f) return ORC_ERR_OOM;
        for (int p = 0; p < s->nso; p++) s->tkin_f[p] = (float)s->tkin[p];
        for (int n2 = 0; n2 < s->n2tab; n2++) s->vtab_f[n2] = (float)s->vtab[n2];
        s->inv_pgen_ueg_f = (float)s->inv_pgen_ueg;
    } else {
        size_t n2 = (size_t)s->norb * s->norb;
        s->h1_f = (float *)malloc(sizeof(float) * n2);
        s->eri_f = (float *)malloc(sizeof(float) * n2 * n2);
        if (!s->h1_f || !s->eri_f) return ORC_ERR_OOM;
        for (size_t i = 0; i < n2; i++) s->h1_f[i] = (float)s->h1[i];
        for (size_t i = 0; i < n2 * n2; i++) s->eri_f[i] = (float)s->eri[i];
        for (int g = 0; g < 2; g++) s->inv_pgen_single_f[g] = (float)s->inv_pgen_single[g];
        for (int c = 0; c < 3; c++) s->inv_pgen_double_f[c] = (float)s->inv_pgen_double[c];
    }
    s->fock_f = (float *)malloc(sizeof(float) * (size_t)s->nso);
    if (!s->fock_f) return ORC_ERR_OOM;
    for (int p = 0; p < s->nso; p++) s->fock_f[p] = (float)s->fock[p];
    s->fp32 = 1;
    s->ehf_rel_f = h_diag_abs_f(s, &s->hf);
    return 0;
}

double orc_hij_f(const orc_system *s, const uint64_t *bra_w, const uint64_t *ket_w)
{
    det_t bra = {{0}}, ket = {{0}};
    for (int i = 0; i < s->nw; i++) { bra.w[i] = bra_w[i]; ket.w[i] = ket_w[i]; }
    if (det_equal(&bra, &ket, s->nw)) return (double)h_diag_abs_f(s, &ket);
    return (double)hij_f(s, &bra, &ket);
}

/* ------------------------------------------------------------------------- */
/* Excitors: s_D(i) = <D_i|c_i|D_HF> (Sec. II Eq. 5), collapse of clusters.   */
/* ------------------------------------------------------------------------- */

/* Apply excitor c_e (given by its determinant de) to the state cur: its
 * annihilators (HF orbitals absent from de) in ascending order, then its
 * creators (virtuals present in de) in descending order.  Returns 0 when the
 * product vanishes (an orbital already emptied or already filled). */
static int apply_excitor(const orc_system *s, const det_t *de, det_t *cur, int *sign)
{
    for (int p = 0; p < s->nel; p++) {
        if (det_bit(de, p)) continue;
        if (!det_bit(cur, p)) return 0;
        *sign *= op_phase(cur, p);
        det_clr(cur, p);
    }
    for (int p = s->nso - 1; p >= s->nel; p--) {
        if (!det_bit(de, p)) continue;
        if (det_bit(cur, p)) return 0;
        *sign *= op_phase(cur, p);
        det_set(cur, p);
    }
    return 1;
}

static int excitor_sign(const orc_system *s, const det_t *d)
{
    det_t cur = s->hf;
    int sign = 1;
    apply_excitor(s, d, &cur, &sign);
    return sign;
}

static int level_of(const orc_system *s, const det_t *d)
{
    int c = 0;
    for (int p = 0; p < s->nel; p++) c += !det_bit(d, p);
    return c;
}

/* Collapse the cluster prod_e c_e |HF> = sigma |D>.  Returns 0 if it vanishes. */
static int collapse(const orc_system *s, int ns, const det_t *ex, det_t *out, int *sigma)
{
    det_t cur = s->hf;
    int sign = 1;
    for (int e = 0; e < ns; e++)
        if (!apply_excitor(s, &ex[e], &cur, &sign)) return 0;
    *out = cur;
    *sigma = sign;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Rank key: an order-preserving integer for determinants of level <= l.     */
/* key = rank(particle set) * C_O - rank(hole set), where rank(X) counts the */
/* sets of at most l positions that are numerically smaller than X.          */
/* ------------------------------------------------------------------------- */

static uint64_t rank_positions(const orc_system *s, const int *pos_desc, int npos)
{
    /* pos_desc: set positions (relative), in descending order */
    uint64_t r = 0;
    for (int c = 0; c < npos; c++) {
        int q = pos_desc[c];
        for (int j = 0; j <= s->lmax - c; j++) r += s->binom[q][j];
    }
    return r;
}

static uint64_t rank_key(const orc_system *s, const det_t *d)
{
    int pos[64 * OW], n = 0;
    for (int p = s->nso - 1; p >= s->nel; p--) if (det_bit(d, p)) pos[n++] = p - s->nel;
    uint64_t rv = rank_positions(s, pos, n);
    n = 0;
    for (int p = s->nel - 1; p >= 0; p--) if (!det_bit(d, p)) pos[n++] = p;
    uint64_t rh = rank_positions(s, pos, n);
    return rv * s->cocc - rh;
}

static void unrank_positions(const orc_system *s, uint64_t r, int m, int *pos, int *npos)
{
    int c = 0;
    for (int q = m - 1; q >= 0; q--) {
        if (c > s->lmax) break;
        uint64_t cnt = 0;
        for (int j = 0; j <= s->lmax - c; j++) cnt += s->binom[q][j];
        if (r >= cnt) { r -= cnt; pos[c++] = q; }
    }
    *npos = c;
}

static void unrank_key(const orc_system *s, uint64_t key, det_t *d)
{
    uint64_t rv = (key + s->cocc - 1) / s->cocc;
    uint64_t rh = rv * s->cocc - key;
    int pos[64 * OW], n;
    *d = s->hf;
    unrank_positions(s, rv, s->nso - s->nel, pos, &n);
    for (int c = 0; c < n; c++) det_set(d, pos[c] + s->nel);
    unrank_positions(s, rh, s->nel, pos, &n);
    for (int c = 0; c < n; c++) det_clr(d, pos[c]);
}

/* ------------------------------------------------------------------------- */
/* Excitation generators (the paper names them only; the forms used here are */
/* uniform ones with exactly known generation probabilities).                */
/* ------------------------------------------------------------------------- */

/* k-th (0-based) empty spin-orbital of d, optionally restricted to one spin */
static int kth_empty(const orc_system *s, const det_t *d, uint64_t k, int spin)
{
    for (int p = 0; p < s->nso; p++) {
        if (det_bit(d, p)) continue;
        if (spin >= 0 && spin_of(p) != spin) continue;
        if (k == 0) return p;
        k--;
    }
    return -1;
}

static void pair_from_index(uint64_t idx, int *x, int *y)
{
    uint64_t yy = 1;
    while ((yy + 1) * yy / 2 <= idx) yy++;
    *y = (int)yy;
    *x = (int)(idx - yy * (yy - 1) / 2);
}

/* Returns 1 and fills di, h = <di|H|dj>, inv_pgen = 1/p_gen; 0 for a null draw. */
static int excite(const orc_system *s, const det_t *dj, const uint64_t r[4],
                  det_t *di, double *h, double *inv_pgen)
{
    int occ[64 * OW], n = 0;
    for (int p = 0; p < s->nso; p++) if (det_bit(dj, p)) occ[n++] = p;
    if (s->kind == 0) {
        int x, y;
        pair_from_index(below(r[1], s->npairs), &x, &y);
        int i = occ[x], j = occ[y];
        int a = kth_empty(s, dj, below(r[2], s->nvirt), -1);
        int sb = spin_of(i) + spin_of(j) - spin_of(a);
        if (sb < 0 || sb > 1) return 0;
        int nb[3];
        for (int c = 0; c < 3; c++)
            nb[c] = s->kv[spat_of(i)][c] + s->kv[spat_of(j)][c] - s->kv[spat_of(a)][c];
        for (int c = 0; c < 3; c++) if (nb[c] < -s->nmax || nb[c] > s->nmax) return 0;
        int side = 2 * s->nmax + 1;
        int bs = s->grid[((nb[0] + s->nmax) * side + (nb[1] + s->nmax)) * side + (nb[2] + s->nmax)];
        if (bs < 0) return 0;
        int b = 2 * bs + sb;
        if (b == a || det_bit(dj, b)) return 0;
        *di = *dj;
        det_clr(di, i); det_clr(di, j); det_set(di, a); det_set(di, b);
        *h = orc_hij(s, di->w, dj->w);
        *inv_pgen = s->inv_pgen_ueg;
        return 1;
    }
    if (below(r[0], s->ns + s->nd) < s->ns) {
        int i = occ[below(r[1], (uint64_t)s->nel)];
        int sg = spin_of(i);
        if (s->nv[sg] == 0) return 0;
        int a = kth_empty(s, dj, below(r[2], (uint64_t)s->nv[sg]), sg);
        *di = *dj;
        det_clr(di, i); det_set(di, a);
        *h = orc_hij(s, di->w, dj->w);
        *inv_pgen = s->inv_pgen_single[sg];
        return 1;
    }
    int x, y;
    pair_from_index(below(r[1], s->npairs), &x, &y);
    int i = occ[x], j = occ[y], a, b, c;
    if (spin_of(i) == spin_of(j)) {
        int sg = spin_of(i);
        c = sg;
        if (s->ndcase[c] == 0) return 0;
        int xa, ya;
        pair_from_index(below(r[2], s->ndcase[c]), &xa, &ya);
        a = kth_empty(s, dj, (uint64_t)xa, sg);
        b = kth_empty(s, dj, (uint64_t)ya, sg);
    } else {
        c = 2;
        if (s->ndcase[c] == 0) return 0;
        uint64_t q = below(r[2], s->ndcase[c]);
        a = kth_empty(s, dj, q / (uint64_t)s->nv[1], 0);
        b = kth_empty(s, dj, q % (uint64_t)s->nv[1], 1);
    }
    *di = *dj;
    det_clr(di, i); det_clr(di, j); det_set(di, a); det_set(di, b);
    *h = orc_hij(s, di->w, dj->w);
    *inv_pgen = s->inv_pgen_double[c];
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Stochastic rounding onto the 2^-16 grid.  Values below the spawn cutoff   */
/* become +-cutoff with probability |x|/cutoff (unbiased), else 0.           */
/* ------------------------------------------------------------------------- */

static int64_t stoch_round(double x, double u, double cutoff, int *err)
{
    double ax = fabs(x);
    int64_t n;
    if (!(ax < 0x1p46)) { *err = ORC_ERR_NUMERIC; return 0; }
    if (ax < cutoff) {
        n = (u * cutoff < ax) ? (int64_t)(cutoff * FIX_ONE) : 0;
    } else {
        double q = ax * FIX_ONE;
        double f = floor(q);
        n = (int64_t)f + ((u < q - f) ? 1 : 0);
    }
    return x < 0.0 ? -n : n;
}

/* ------------------------------------------------------------------------- */
/* Simulation                                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    double tau;
    double target_pop;
    double d0_init;
    int32_t shift_a;
    int32_t fnc;
    double zeta;
    double spawn_cutoff;
    int32_t multispawn;
    int32_t n_ranks;      /* processors of the simulated distribution (<= 1: none) */
    double a_thresh;
    uint64_t seed;
    uint64_t replica;
    int32_t nu_move;      /* owners move every 2^nu_move iterations (>= 64: never) */
    int32_t pad1;
} orc_params;

typedef struct {
    uint64_t iter;
    double shift;
    int64_t n0;
    int64_t ntot;
    int64_t n_sel;
    int64_t n_visit;
    int64_t n_attempts;
    int64_t n_spawned;
    double e_num;
    int64_t ntot_after;
    int64_t nocc_after;
    int64_t n_keys;       /* distinct keys among the spawn records */
} orc_record;

typedef struct {
    const orc_system *sys;
    orc_params prm;
    int64_t n, cap;
    det_t *bits;
    uint64_t *key;
    int64_t *pop;
    /* per-step outputs */
    int64_t *death;
    int64_t death_n;     /* list size at the start of the latest step */
    int64_t nsp, spcap;
    uint64_t *spkey;
    int64_t *sppop;
    double enum_sum, enum_comp;
    /* shift state */
    double shift;
    int vary;
    double nprev;
    uint64_t iter;
    orc_record rec;
} orc_sim;

static int sim_reserve(orc_sim *m, int64_t n)
{
    if (n <= m->cap) return 0;
    int64_t c = m->cap ? m->cap : 16;
    while (c < n) c *= 2;
    det_t *b = (det_t *)realloc(m->bits, sizeof(det_t) * (size_t)c);
    if (!b) return ORC_ERR_OOM;
    m->bits = b;
    uint64_t *k = (uint64_t *)realloc(m->key, sizeof(uint64_t) * (size_t)c);
    if (!k) return ORC_ERR_OOM;
    m->key = k;
    int64_t *p = (int64_t *)realloc(m->pop, sizeof(int64_t) * (size_t)c);
    if (!p) return ORC_ERR_OOM;
    m->pop = p;
    int64_t *d = (int64_t *)realloc(m->death, sizeof(int64_t) * (size_t)c);
    if (!d) return ORC_ERR_OOM;
    m->death = d;
    m->cap = c;
    return 0;
}

static int push_spawn(orc_sim *m, uint64_t key, int64_t v)
{
    if (m->nsp == m->spcap) {
        int64_t c = m->spcap ? 2 * m->spcap : 1024;
        uint64_t *k = (uint64_t *)realloc(m->spkey, sizeof(uint64_t) * (size_t)c);
        if (!k) return ORC_ERR_OOM;
        m->spkey = k;
        int64_t *p = (int64_t *)realloc(m->sppop, sizeof(int64_t) * (size_t)c);
        if (!p) return ORC_ERR_OOM;
        m->sppop = p;
        m->spcap = c;
    }
    m->spkey[m->nsp] = key;
    m->sppop[m->nsp] = v;
    m->nsp++;
    return 0;
}

/* Neumaier-compensated accumulation of the projected-energy numerator. */
static void enum_add(orc_sim *m, double x)
{
    double t = m->enum_sum + x;
    if (fabs(m->enum_sum) >= fabs(x)) m->enum_comp += (m->enum_sum - t) + x;
    else m->enum_comp += (x - t) + m->enum_sum;
    m->enum_sum = t;
}

orc_sim *orc_sim_new(const orc_system *s, const orc_params *prm)
{
    orc_sim *m = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!m) return NULL;
    m->sys = s;
    m->prm = *prm;
    if (sim_reserve(m, 16)) { free(m); return NULL; }
    m->n = 1;
    m->bits[0] = s->hf;
    m->key[0] = rank_key(s, &s->hf);
    m->pop[0] = (int64_t)llround(prm->d0_init * FIX_ONE);
    m->shift = 0.0;
    m->vary = 0;
    m->nprev = prm->d0_init;
    m->iter = 0;
    return m;
}

void orc_sim_free(orc_sim *m)
{
    if (!m) return;
    free(m->bits); free(m->key); free(m->pop); free(m->death);
    free(m->spkey); free(m->sppop);
    free(m);
}

/* The FP32 counterpart of a generation probability (1/p_gen) of this system. */
static float pgen_f_of(const orc_system *s, double inv_pgen)
{
    if (s->kind == 0) return s->inv_pgen_ueg_f;
    for (int g = 0; g < 2; g++) if (inv_pgen == s->inv_pgen_single[g]) return s->inv_pgen_single_f[g];
    for (int c = 0; c < 3; c++) if (inv_pgen == s->inv_pgen_double[c]) return s->inv_pgen_double_f[c];
    return (float)inv_pgen;
}

/* Diagonal energy relative to HF in the system's precision. */
static double diag_rel_p(const orc_system *s, const det_t *d)
{
    return s->fp32 ? (double)h_diag_rel_f(s, d) : h_diag_rel(s, d);
}

/* <HF|H|D> in the system's precision. */
static double href_p(const orc_system *s, const det_t *d)
{
    return s->fp32 ? (double)hij_f(s, &s->hf, d) : orc_hij(s, s->hf.w, d->w);
}

/* Spawning attempts from one cluster, Sec. II and Sec. IV.C: each attempt
 * carries the cluster coefficient divided by n_attempts.  The spawned value
 * onto excitor i is -dtau H_ij C s_D(i) / p_gen. */
static int spawn_attempts(orc_sim *m, const det_t *dj, double coef, int64_t n_att,
                          uint64_t tag, uint64_t index)
{
    const orc_system *s = m->sys;
    const uint64_t pkey[2] = { m->prm.seed, m->prm.replica };
    double c_att = (n_att > 1) ? coef / (double)n_att : coef;
    int err = 0;
    for (int64_t a = 0; a < n_att; a++) {
        uint64_t r[4];
        draw4(pkey, m->iter, tag, index, (uint64_t)a, r);
        det_t di;
        double h, inv_pgen;
        m->rec.n_attempts++;
        if (!excite(s, dj, r, &di, &h, &inv_pgen)) continue;
        if (level_of(s, &di) > s->lmax) continue;
        if (s->fp32) {
            h = (double)hij_f(s, &di, dj);
            inv_pgen = (double)pgen_f_of(s, inv_pgen);
        }
        double x = ((m->prm.tau * h) * inv_pgen) * c_att;
        if (excitor_sign(s, &di) > 0) x = -x;
        int64_t v = stoch_round(x, unif(r[3]), m->prm.spawn_cutoff, &err);
        if (err) return err;
        if (v != 0) {
            int rc = push_spawn(m, rank_key(s, &di), v);
            if (rc) return rc;
        }
    }
    return 0;
}

/* Death of a cluster (Sec. II): -dtau (H_jj - E_HF - S) C s_D(j). */
static double death_value(const orc_sim *m, double dE, double coef, int sdj)
{
    double x = (m->prm.tau * (dE - m->shift)) * coef;
    return sdj > 0 ? -x : x;
}

static int64_t n_attempts_for(const orc_sim *m, double amp)
{
    if (!m->prm.multispawn) return 1;
    double q = floor(fabs(amp) / m->prm.a_thresh);
    return q < 1.0 ? 1 : (int64_t)q;
}

/* Index of the excitor holding position x in [0, N_ex): the smallest i >= 1
 * with prefix[i] > x, where prefix[i] = sum_{1<=k<=i} |pop_k|. */
static int64_t pick_index(const int64_t *prefix, int64_t n, uint64_t x)
{
    int64_t lo = 1, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((uint64_t)prefix[mid] > x) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Simulated distribution (Sec. III): a processor forms composite clusters
 * only from the excitors it holds.  The excitors (entries i >= 1) grouped by
 * their owner at this iteration, ascending within each group, with running
 * sums of |t_i| per group; N_q is processor q's total. */
typedef struct {
    int64_t *own, *start, *count, *order, *lpre, *nq;
} orc_local;

static void local_free(orc_local *l)
{
    free(l->own); free(l->start); free(l->count); free(l->order); free(l->lpre); free(l->nq);
}

static int local_build(const orc_sim *m, orc_local *l)
{
    const int64_t n = m->n, np_ = m->prm.n_ranks;
    l->own = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    l->order = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    l->lpre = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    l->start = (int64_t *)calloc((size_t)np_, sizeof(int64_t));
    l->count = (int64_t *)calloc((size_t)np_, sizeof(int64_t));
    l->nq = (int64_t *)calloc((size_t)np_, sizeof(int64_t));
    if (!l->own || !l->order || !l->lpre || !l->start || !l->count || !l->nq) return ORC_ERR_OOM;
    for (int64_t i = 1; i < n; i++) {
        l->own[i] = (int64_t)orc_owner(m->bits[i].w, m->sys->nw, m->iter, m->prm.nu_move, (uint64_t)np_);
        l->count[l->own[i]]++;
    }
    for (int64_t q = 1; q < np_; q++) l->start[q] = l->start[q - 1] + l->count[q - 1];
    int64_t *fill = (int64_t *)calloc((size_t)np_, sizeof(int64_t));
    if (!fill) return ORC_ERR_OOM;
    for (int64_t i = 1; i < n; i++) {
        const int64_t q = l->own[i], k = l->start[q] + fill[q]++;
        const int64_t a = m->pop[i] < 0 ? -m->pop[i] : m->pop[i];
        l->order[k] = i;
        l->nq[q] += a;
        l->lpre[k] = l->nq[q];
    }
    free(fill);
    return 0;
}

/* The excitor of processor q holding position x in [0, N_q): the first in
 * the group whose running sum exceeds x. */
static int64_t local_pick(const orc_local *l, int64_t q, uint64_t x)
{
    int64_t lo = l->start[q], hi = l->start[q] + l->count[q] - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((uint64_t)l->lpre[mid] > x) hi = mid; else lo = mid + 1;
    }
    return l->order[lo];
}

/* Cluster sample g (Sec. II; FNC composites per Sec. IV.B). */
static int sample_cluster(orc_sim *m, uint64_t g, const int64_t *prefix, int64_t nex,
                          const double *mag, const double *den, const orc_local *loc, int fnc)
{
    const orc_system *s = m->sys;
    const uint64_t pkey[2] = { m->prm.seed, m->prm.replica };
    uint64_t r[8];
    draw4(pkey, m->iter, TAG_SAMPLE, g, 0, r);
    draw4(pkey, m->iter, TAG_SAMPLE, g, 1, r + 4);
    uint64_t nr = ~r[0];
    int lz = nr ? __builtin_clzll(nr) : 64;
    int sz;
    if (fnc) sz = 2 + (lz < s->lmax ? lz : s->lmax);
    else sz = lz < s->lmax + 2 ? lz : s->lmax + 2;
    int64_t n0 = m->pop[0];
    det_t dj;
    int sigma = 1;
    int64_t idx[8];
    double amp;
    if (sz == 0) {
        dj = s->hf;
        amp = n0 < 0 ? -mag[0] : mag[0];
        idx[0] = 0;
    } else {
        if (nex == 0) return 0;
        if (sz >= 2 && n0 == 0) return 0;
        det_t ex[8];
        int neg = 0;
        /* simulated distribution (Sec. III): the first excitor is drawn from
           the whole list (a processor draws in proportion to the population
           it holds), the others from the first one's processor q only */
        const int local = loc && sz >= 2;
        int64_t q = 0;
        for (int e = 0; e < sz; e++) {
            if (local && e >= 1) {
                idx[e] = local_pick(loc, q, below(r[2 + e], (uint64_t)loc->nq[q]));
            } else {
                idx[e] = pick_index(prefix, m->n, below(r[2 + e], (uint64_t)nex));
                if (local) q = loc->own[idx[0]];
            }
            for (int f = 0; f < e; f++) if (idx[f] == idx[e]) return 0;   /* repeated excitor */
            ex[e] = m->bits[idx[e]];
            if (m->pop[idx[e]] < 0) neg ^= 1;
        }
        if (!collapse(s, sz, ex, &dj, &sigma)) return 0;
        if (n0 < 0 && ((sz - 1) & 1)) neg ^= 1;
        double a = mag[sz];
        if (local) {
            /* |A| = N_ex (N_q N_p)^(s-1) / (|t_HF|^(s-1) n_sel p(s) s!): the
               selection probability p(s) s! prod|t| / (N_ex N_q^(s-1)) times
               the co-location probability N_p^-(s-1) of the cluster */
            const double f = ((double)loc->nq[q] / FIX_ONE) * (double)m->prm.n_ranks;
            double num = (double)nex / FIX_ONE;
            for (int e = 1; e < sz; e++) num = num * f;
            a = num / den[sz];
        }
        amp = neg ? -a : a;
    }
    int lev = level_of(s, &dj);
    if (lev > s->lmax + 2) return 0;
    double coef = sigma > 0 ? amp : -amp;
    if (lev == 1 || lev == 2) enum_add(m, href_p(s, &dj) * coef);
    /* death */
    int err = 0;
    int sdj = excitor_sign(s, &dj);
    if (sz <= 1) {
        double dE = (sz == 0) ? 0.0 : diag_rel_p(s, &dj);
        int64_t v = stoch_round(death_value(m, dE, coef, sdj), unif(r[1]), 0.0, &err);
        if (err) return err;
        m->death[idx[0]] += v;
    } else if (lev <= s->lmax) {
        int64_t v = stoch_round(death_value(m, diag_rel_p(s, &dj), coef, sdj), unif(r[1]), 0.0, &err);
        if (err) return err;
        if (v != 0) {
            int rc = push_spawn(m, rank_key(s, &dj), v);
            if (rc) return rc;
        }
    }
    return spawn_attempts(m, &dj, coef, n_attempts_for(m, amp), TAG_SAMPLE_ATT, g);
}

/* FNC non-composite visit of list entry i (Sec. IV.B): p = 1, A = t_i. */
static int visit_excitor(orc_sim *m, int64_t i)
{
    const orc_system *s = m->sys;
    const uint64_t pkey[2] = { m->prm.seed, m->prm.replica };
    const det_t *dj = &m->bits[i];
    double amp = (double)m->pop[i] / FIX_ONE;
    int sdj = excitor_sign(s, dj);
    double coef = sdj > 0 ? amp : -amp;
    int lev = level_of(s, dj);
    if (lev == 1 || lev == 2) enum_add(m, href_p(s, dj) * coef);
    uint64_t r[4];
    draw4(pkey, m->iter, TAG_VISIT, (uint64_t)i, 0, r);
    double dE = (i == 0) ? 0.0 : diag_rel_p(s, dj);
    int err = 0;
    int64_t v = stoch_round(death_value(m, dE, coef, sdj), unif(r[0]), 0.0, &err);
    if (err) return err;
    m->death[i] += v;
    return spawn_attempts(m, dj, coef, n_attempts_for(m, amp), TAG_VISIT_ATT, (uint64_t)i);
}

static int cmp_spawn(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return 0;
}

/* Annihilation (Sec. II): combine the list, its death deltas and the spawned
 * particles per excitor; then the occupation threshold; drop empty excitors. */
static int annihilate(orc_sim *m)
{
    const orc_system *s = m->sys;
    const uint64_t pkey[2] = { m->prm.seed, m->prm.replica };
    /* sort the spawn records by key and sum runs of equal keys */
    uint64_t *rec = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)(m->nsp + 1));
    if (!rec) return ORC_ERR_OOM;
    for (int64_t i = 0; i < m->nsp; i++) { rec[2 * i] = m->spkey[i]; rec[2 * i + 1] = (uint64_t)m->sppop[i]; }
    qsort(rec, (size_t)m->nsp, 2 * sizeof(uint64_t), cmp_spawn);
    int64_t nu = 0;
    for (int64_t i = 0; i < m->nsp; i++) {
        if (nu > 0 && rec[2 * (nu - 1)] == rec[2 * i]) {
            rec[2 * (nu - 1) + 1] = (uint64_t)((int64_t)rec[2 * (nu - 1) + 1] + (int64_t)rec[2 * i + 1]);
        } else {
            rec[2 * nu] = rec[2 * i];
            rec[2 * nu + 1] = rec[2 * i + 1];
            nu++;
        }
    }
    m->rec.n_keys = nu;
    /* merge */
    int64_t cap = m->n + nu;
    det_t *nb = (det_t *)malloc(sizeof(det_t) * (size_t)(cap + 1));
    uint64_t *nk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap + 1));
    int64_t *np = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap + 1));
    if (!nb || !nk || !np) { free(rec); free(nb); free(nk); free(np); return ORC_ERR_OOM; }
    int64_t a = 0, b = 0, out = 0;
    while (a < m->n || b < nu) {
        uint64_t key;
        int64_t v;
        det_t d;
        if (b >= nu || (a < m->n && m->key[a] < rec[2 * b])) {
            key = m->key[a]; d = m->bits[a]; v = m->pop[a] + m->death[a]; a++;
        } else if (a >= m->n || rec[2 * b] < m->key[a]) {
            key = rec[2 * b]; unrank_key(s, key, &d); v = (int64_t)rec[2 * b + 1]; b++;
        } else {
            key = m->key[a]; d = m->bits[a]; v = m->pop[a] + m->death[a] + (int64_t)rec[2 * b + 1]; a++; b++;
        }
        int is_hf = (out == 0 && det_equal(&d, &s->hf, s->nw));
        if (!is_hf) {
            int64_t av = v < 0 ? -v : v;
            if (av > 0 && av < (int64_t)FIX_ONE) {
                uint64_t r[4];
                draw4(pkey, m->iter, TAG_THRESH, key, 0, r);
                int keep = (r[0] >> 11) < ((uint64_t)av << 37);
                v = keep ? (v < 0 ? -(int64_t)FIX_ONE : (int64_t)FIX_ONE) : 0;
            }
            if (v == 0) continue;
        }
        nb[out] = d; nk[out] = key; np[out] = v; out++;
    }
    free(rec);
    int rc = sim_reserve(m, out);
    if (rc) { free(nb); free(nk); free(np); return rc; }
    memcpy(m->bits, nb, sizeof(det_t) * (size_t)out);
    memcpy(m->key, nk, sizeof(uint64_t) * (size_t)out);
    memcpy(m->pop, np, sizeof(int64_t) * (size_t)out);
    m->n = out;
    free(nb); free(nk); free(np);
    return 0;
}

static int sim_step_range(orc_sim *m, int propagate_only, int64_t i_lo, int64_t i_hi, int64_t g_lo, int64_t g_hi);

/* One time step.  With propagate_only the spawned records and the death
 * deltas are produced but not annihilated and the iteration does not advance
 * (used to check the mean of one step against the exact action). */
int orc_sim_step(orc_sim *m, int propagate_only)
{
    return sim_step_range(m, propagate_only, 0, INT64_MAX, 0, INT64_MAX);
}

/* Propagation (no annihilation) restricted to the non-composite visits
 * [i_lo, i_hi) and the cluster samples [g_lo, g_hi) of the current step: the
 * same per-sample work as a full step, for timing bounded samples of it. */
int orc_sim_sample_range(orc_sim *m, int64_t i_lo, int64_t i_hi, int64_t g_lo, int64_t g_hi)
{
    return sim_step_range(m, 1, i_lo, i_hi, g_lo, g_hi);
}

static int sim_step_range(orc_sim *m, int propagate_only, int64_t i_lo, int64_t i_hi, int64_t g_lo, int64_t g_hi)
{
    const orc_system *s = m->sys;
    int64_t n = m->n;
    memset(&m->rec, 0, sizeof(m->rec));
    m->rec.iter = m->iter;
    m->rec.shift = m->shift;
    m->nsp = 0;
    m->enum_sum = 0.0;
    m->enum_comp = 0.0;
    for (int64_t i = 0; i < n; i++) m->death[i] = 0;
    m->death_n = n;
    /* selection weights |t_i|/(N_total - t_HF), Sec. II */
    int64_t *prefix = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!prefix) return ORC_ERR_OOM;
    int64_t ntot = m->pop[0] < 0 ? -m->pop[0] : m->pop[0];
    prefix[0] = 0;
    for (int64_t i = 1; i < n; i++) {
        int64_t a = m->pop[i] < 0 ? -m->pop[i] : m->pop[i];
        prefix[i] = prefix[i - 1] + a;
        ntot += a;
    }
    int64_t n0 = m->pop[0];
    int64_t nex = ntot - (n0 < 0 ? -n0 : n0);
    int64_t n_sel = (ntot + 32768) >> FIX_SHIFT;
    m->rec.n0 = n0;
    m->rec.ntot = ntot;
    m->rec.n_sel = n_sel;
    /* |A| of a cluster of size s: N_ex^s / (|t_HF|^(s-1) n_sel p(s) s!) */
    double mag[8] = { 0 }, den_s[8] = { 0 };
    double nex_d = (double)nex / FIX_ONE;
    double n0_d = (double)(n0 < 0 ? -n0 : n0) / FIX_ONE;
    int smax = s->lmax + 2;
    for (int sz = 0; sz <= smax; sz++) {
        if (n_sel == 0) break;
        double p;
        if (m->prm.fnc) {
            if (sz < 2) continue;
            p = (sz < smax) ? ldexp(1.0, -(sz - 1)) : ldexp(1.0, -s->lmax);
        } else {
            p = (sz < smax) ? ldexp(1.0, -(sz + 1)) : ldexp(1.0, -(s->lmax + 2));
        }
        if (sz == 0) { mag[0] = n0_d / ((double)n_sel * p); continue; }
        double num = 1.0, den = 1.0, fact = 1.0;
        for (int e = 0; e < sz; e++) num = num * nex_d;
        for (int e = 0; e < sz - 1; e++) den = den * n0_d;
        for (int e = 2; e <= sz; e++) fact = fact * (double)e;
        den = den * (double)n_sel;
        den = den * p;
        den = den * fact;
        mag[sz] = num / den;
        den_s[sz] = den;
    }
    orc_local loc = { 0 };
    int rc = 0;
    if (m->prm.n_ranks > 1) {
        rc = local_build(m, &loc);
        if (rc) { local_free(&loc); free(prefix); return rc; }
    }
    if (m->prm.fnc) {
        int64_t hi = i_hi < n ? i_hi : n;
        m->rec.n_visit = hi > i_lo ? hi - i_lo : 0;
        for (int64_t i = i_lo; i < hi && !rc; i++) rc = visit_excitor(m, i);
    }
    {
        int64_t hi = g_hi < n_sel ? g_hi : n_sel;
        for (int64_t g = g_lo; g < hi && !rc; g++)
            rc = sample_cluster(m, (uint64_t)g, prefix, nex, mag, den_s, m->prm.n_ranks > 1 ? &loc : NULL, m->prm.fnc);
    }
    local_free(&loc);
    free(prefix);
    if (rc) return rc;
    m->rec.n_spawned = m->nsp;
    m->rec.e_num = m->enum_sum + m->enum_comp;
    if (propagate_only) return 0;
    rc = annihilate(m);
    if (rc) return rc;
    int64_t nt = 0;
    for (int64_t i = 0; i < m->n; i++) nt += m->pop[i] < 0 ? -m->pop[i] : m->pop[i];
    m->rec.ntot_after = nt;
    m->rec.nocc_after = m->n;
    /* shift update every A steps once the target population was exceeded */
    if (((m->iter + 1) % (uint64_t)m->prm.shift_a) == 0) {
        double nt_d = (double)nt / FIX_ONE;
        if (m->vary && nt_d > 0.0 && m->nprev > 0.0)
            m->shift = m->shift - (m->prm.zeta / ((double)m->prm.shift_a * m->prm.tau)) * log(nt_d / m->nprev);
        if (!m->vary && nt_d > m->prm.target_pop) m->vary = 1;
        m->nprev = nt_d;
    }
    m->iter++;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exported helpers for the tests                                             */
/* ------------------------------------------------------------------------- */

static det_t load_det(const orc_system *s, const uint64_t *w)
{
    det_t d = {{0}};
    for (int i = 0; i < s->nw; i++) d.w[i] = w[i];
    return d;
}

void orc_sys_info(const orc_system *s, int32_t *out)
{
    out[0] = s->nel; out[1] = s->nso; out[2] = s->nw; out[3] = s->lmax; out[4] = s->kind;
}

double orc_ehf(const orc_system *s) { return s->ehf_rel + s->ecore; }
double orc_ueg_length(const orc_system *s) { return s->L; }
void orc_hf(const orc_system *s, uint64_t *out) { for (int i = 0; i < s->nw; i++) out[i] = s->hf.w[i]; }

void orc_ueg_kvec(const orc_system *s, int32_t *out)
{
    for (int i = 0; i < s->npw; i++) for (int c = 0; c < 3; c++) out[3 * i + c] = s->kv[i][c];
}

double orc_ueg_tkin(const orc_system *s, int p) { return s->tkin[p]; }
double orc_ueg_vq(const orc_system *s, int n2) { return (n2 >= 0 && n2 < s->n2tab) ? s->vtab[n2] : 0.0; }

double orc_hdiag_rel(const orc_system *s, const uint64_t *w)
{
    det_t d = load_det(s, w);
    return h_diag_rel(s, &d);
}

double orc_hdiag_rel_f(const orc_system *s, const uint64_t *w)
{
    det_t d = load_det(s, w);
    return s->fp32 ? (double)h_diag_rel_f(s, &d) : 0.0;
}

int orc_excitor_sign(const orc_system *s, const uint64_t *w)
{
    det_t d = load_det(s, w);
    return excitor_sign(s, &d);
}

int orc_level(const orc_system *s, const uint64_t *w)
{
    det_t d = load_det(s, w);
    return level_of(s, &d);
}

int orc_collapse(const orc_system *s, int ns, const uint64_t *ex_w, uint64_t *out, int32_t *sigma)
{
    det_t ex[8], d;
    if (ns > 8) return -1;
    for (int e = 0; e < ns; e++) ex[e] = load_det(s, ex_w + e * s->nw);
    int sg = 0;
    int ok = collapse(s, ns, ex, &d, &sg);
    if (ok) { for (int i = 0; i < s->nw; i++) out[i] = d.w[i]; *sigma = sg; }
    return ok;
}

uint64_t orc_rank(const orc_system *s, const uint64_t *w)
{
    det_t d = load_det(s, w);
    return rank_key(s, &d);
}

void orc_unrank(const orc_system *s, uint64_t key, uint64_t *out)
{
    det_t d;
    unrank_key(s, key, &d);
    for (int i = 0; i < s->nw; i++) out[i] = d.w[i];
}

uint64_t orc_key_bound(const orc_system *s) { return s->nvranks * s->cocc; }

int orc_excite(const orc_system *s, const uint64_t *dj_w, const uint64_t *r, uint64_t *di_w,
               double *h, double *inv_pgen)
{
    det_t dj = load_det(s, dj_w), di;
    int ok = excite(s, &dj, r, &di, h, inv_pgen);
    if (ok) for (int i = 0; i < s->nw; i++) di_w[i] = di.w[i];
    return ok;
}

int orc_size_draw(uint64_t r0, int lmax, int fnc)
{
    uint64_t nr = ~r0;
    int lz = nr ? __builtin_clzll(nr) : 64;
    if (fnc) return 2 + (lz < lmax ? lz : lmax);
    return lz < lmax + 2 ? lz : lmax + 2;
}

int64_t orc_pick_index(const int64_t *prefix, int64_t n, uint64_t x) { return pick_index(prefix, n, x); }
uint64_t orc_below(uint64_t r, uint64_t n) { return below(r, n); }

int64_t orc_stoch_round(double x, double u, double cutoff)
{
    int err = 0;
    int64_t v = stoch_round(x, u, cutoff, &err);
    return err ? INT64_MIN : v;
}

int orc_sim_set_list(orc_sim *m, int64_t n, const uint64_t *bits_w, const int64_t *pop)
{
    const orc_system *s = m->sys;
    if (n < 1) return ORC_ERR_ARG;
    int rc = sim_reserve(m, n);
    if (rc) return rc;
    for (int64_t i = 0; i < n; i++) {
        m->bits[i] = load_det(s, bits_w + i * s->nw);
        if (level_of(s, &m->bits[i]) > s->lmax) return ORC_ERR_ARG;
        if (det_popcount(&m->bits[i], s->nw) != s->nel) return ORC_ERR_ARG;
        m->key[i] = rank_key(s, &m->bits[i]);
        m->pop[i] = pop[i];
        if (i > 0 && m->key[i] <= m->key[i - 1]) return ORC_ERR_ARG;
    }
    if (!det_equal(&m->bits[0], &s->hf, s->nw)) return ORC_ERR_ARG;
    m->n = n;
    return 0;
}

int64_t orc_sim_size(const orc_sim *m) { return m->n; }

void orc_sim_get_list(const orc_sim *m, uint64_t *bits_w, uint64_t *keys, int64_t *pop)
{
    const orc_system *s = m->sys;
    for (int64_t i = 0; i < m->n; i++) {
        if (bits_w) for (int w = 0; w < s->nw; w++) bits_w[i * s->nw + w] = m->bits[i].w[w];
        if (keys) keys[i] = m->key[i];
        if (pop) pop[i] = m->pop[i];
    }
}

int64_t orc_sim_nspawned(const orc_sim *m) { return m->nsp; }

void orc_sim_get_spawned(const orc_sim *m, uint64_t *keys, int64_t *pop)
{
    for (int64_t i = 0; i < m->nsp; i++) { keys[i] = m->spkey[i]; pop[i] = m->sppop[i]; }
}

int64_t orc_sim_ndeath(const orc_sim *m) { return m->death_n; }

void orc_sim_get_death(const orc_sim *m, int64_t *out)
{
    for (int64_t i = 0; i < m->death_n; i++) out[i] = m->death[i];
}

void orc_sim_get_record(const orc_sim *m, orc_record *out) { *out = m->rec; }

void orc_sim_set_state(orc_sim *m, uint64_t iter, double shift, int32_t vary, double nprev)
{
    m->iter = iter; m->shift = shift; m->vary = vary; m->nprev = nprev;
}

void orc_sim_get_state(const orc_sim *m, uint64_t *iter, double *shift, int32_t *vary, double *nprev)
{
    *iter = m->iter; *shift = m->shift; *vary = m->vary; *nprev = m->nprev;
}

int orc_sim_run(orc_sim *m, int nsteps, orc_record *records)
{
    for (int k = 0; k < nsteps; k++) {
        int rc = orc_sim_step(m, 0);
        if (rc) return rc;
        if (records) records[k] = m->rec;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Test helper: closure of HF under the excitation generator, visiting every */
/* draw outcome once from each determinant reached (only from those below   */
/* max_level unless expand_top is set), keeping the targets of level <=     */
/* max_level.  The restricted form is complete when every top-level         */
/* determinant is one excitation from a lower level.                        */
/* Returns the number of determinants reached (HF included), or -1 when the */
/* key bitmap would be too large.                                           */
/* ------------------------------------------------------------------------- */

static uint64_t r_for_index(uint64_t idx, uint64_t n)
{
    /* smallest r with floor(r n / 2^64) == idx */
    unsigned __int128 num = ((unsigned __int128)idx << 64) + (n - 1);
    return (uint64_t)(num / n);
}

int64_t orc_generator_closure(const orc_system *s, int max_level, int expand_top, uint64_t *keys_out, int64_t cap)
{
    uint64_t bound = s->nvranks * s->cocc;
    if (bound > (1ULL << 34)) return -1;
    uint8_t *seen = (uint8_t *)calloc((size_t)(bound / 8 + 1), 1);
    int64_t qcap = 1024, qn = 0, qh = 0;
    det_t *queue = (det_t *)malloc(sizeof(det_t) * (size_t)qcap);
    if (!seen || !queue) { free(seen); free(queue); return -1; }
    queue[qn++] = s->hf;
    uint64_t k0 = rank_key(s, &s->hf);
    seen[k0 >> 3] |= (uint8_t)(1u << (k0 & 7));
    while (qh < qn) {
        det_t dj = queue[qh++];
        if (!expand_top && level_of(s, &dj) >= max_level) continue;
        /* enumerate all draw tuples (r0, r1, r2) that select distinct outcomes */
        uint64_t n0 = (s->kind == 0) ? 1 : 2;
        for (uint64_t t = 0; t < n0; t++) {
            uint64_t r0 = (s->kind == 0) ? 0 : (t == 0 ? r_for_index(0, s->ns + s->nd) : r_for_index(s->ns, s->ns + s->nd));
            int single = (s->kind == 1 && t == 0);
            uint64_t n1 = single ? (uint64_t)s->nel : s->npairs;
            for (uint64_t i1 = 0; i1 < n1; i1++) {
                uint64_t n2max = (s->kind == 0) ? s->nvirt : 0;
                if (s->kind == 1) {
                    int occ[64 * OW], n = 0;
                    for (int p = 0; p < s->nso; p++) if (det_bit(&dj, p)) occ[n++] = p;
                    if (single) {
                        n2max = (uint64_t)s->nv[spin_of(occ[i1])];
                    } else {
                        int x, y;
                        pair_from_index(i1, &x, &y);
                        int c = (spin_of(occ[x]) == spin_of(occ[y])) ? spin_of(occ[x]) : 2;
                        n2max = s->ndcase[c];
                    }
                }
                for (uint64_t i2 = 0; i2 < n2max; i2++) {
                    uint64_t r[4] = { r0, r_for_index(i1, n1), r_for_index(i2, n2max), 0 };
                    det_t di;
                    double h, ip;
                    if (!excite(s, &dj, r, &di, &h, &ip)) continue;
                    if (level_of(s, &di) > max_level) continue;
                    uint64_t k = rank_key(s, &di);
                    if (seen[k >> 3] & (1u << (k & 7))) continue;
                    seen[k >> 3] |= (uint8_t)(1u << (k & 7));
                    if (qn == qcap) {
                        qcap *= 2;
                        det_t *nq = (det_t *)realloc(queue, sizeof(det_t) * (size_t)qcap);
                        if (!nq) { free(seen); free(queue); return -1; }
                        queue = nq;
                    }
                    queue[qn++] = di;
                }
            }
        }
    }
    if (keys_out) {
        /* keys in increasing order (bit-string order) */
        int64_t m = 0;
        for (uint64_t k = 0; k < bound && m < cap; k++)
            if (seen[k >> 3] & (1u << (k & 7))) keys_out[m++] = k;
    }
    free(seen);
    free(queue);
    return qn;
}
