// ccmc_api.cu -- host side of the C ABI declared in include/ccmc.h.
//
// Builds the Hamiltonian tables (uniform electron gas: plane waves sorted by
// |n|^2 then lexicographically, kinetic |k|^2/2, Coulomb 1/(pi L |n_q|^2);
// generic: dense h1 and (pq|rs)), the rank-key tables, allocates the device
// state and sequences the kernels of ccmc_step.cu.  The host evaluates only
// the logarithm of the shift update (Sec. II: the shift is held, then varied
// to keep the population stable) every shift_a steps.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ccmc.h"
#include "ccmc_state.cuh"

using namespace ccmc;

namespace {

constexpr double PI_D = 3.14159265358979323846;

struct HostSys {
    int kind = 0, nel = 0, nso = 0, lmax = 0, nw = 0;
    double rs = 0.0, L = 0.0, ecore = 0.0;
    int npw = 0, nmax = 0, side = 0;
    std::vector<int> kv, grid;
    std::vector<double> tkin, vtab, h1, eri;
    int norb = 0;
    std::vector<u64> rank_tab;
    u64 cocc = 0, nvranks = 0;
    u64 binom[RANK_STRIDE][8];
    double ehf_rel = 0.0;
    u64 npairs = 0, nvirt = 0, ns = 0, nd = 0, ndcase[3] = {0, 0, 0};
    int no[2] = {0, 0}, nv[2] = {0, 0};
    double inv_pgen_ueg = 0.0, inv_pgen_single[2] = {0, 0}, inv_pgen_double[3] = {0, 0, 0};
    std::vector<double> fock;     // reference Fock diagonal per spin-orbital
    // FP32 form
    std::vector<float> tkin_f, vtab_f, h1_f, eri_f, fock_f;
};

void fill_binom(HostSys &h)
{
    for (int n = 0; n < RANK_STRIDE; n++)
        for (int k = 0; k < 8; k++)
            h.binom[n][k] = k == 0 ? 1 : (n == 0 ? 0 : h.binom[n - 1][k - 1] + h.binom[n - 1][k]);
}

// <D|H|D> without core energy, same operation order as the device code
double host_diag(const HostSys &h, const std::vector<int> &occ)
{
    const int n = (int)occ.size();
    if (h.kind == CCMC_UEG) {
        double tsum = 0.0, xsum = 0.0;
        for (int i = 0; i < n; i++) tsum = tsum + h.tkin[occ[i]];
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++)
                if (((occ[i] ^ occ[j]) & 1) == 0) {
                    const int *a = &h.kv[3 * (occ[i] >> 1)], *b = &h.kv[3 * (occ[j] >> 1)];
                    int dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
                    xsum = xsum + h.vtab[dx * dx + dy * dy + dz * dz];
                }
        return tsum - xsum;
    }
    double e1 = 0.0, e2 = 0.0;
    const size_t no = (size_t)h.norb;
    for (int i = 0; i < n; i++) {
        int P = occ[i] >> 1;
        e1 = e1 + h.h1[P * no + P];
    }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            size_t P = occ[i] >> 1, Q = occ[j] >> 1;
            double t = h.eri[((P * no + P) * no + Q) * no + Q];
            if (((occ[i] ^ occ[j]) & 1) == 0) t = t - h.eri[((P * no + Q) * no + Q) * no + P];
            e2 = e2 + t;
        }
    return e1 + e2;
}

// <pq||pq> for p != q (same definition and operation order as the device)
double host_pair_ex(const HostSys &h, int p, int q)
{
    if (h.kind == CCMC_UEG) {
        const int *a = &h.kv[3 * (p >> 1)], *b = &h.kv[3 * (q >> 1)];
        int dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
        return -h.vtab[dx * dx + dy * dy + dz * dz];
    }
    const size_t no = (size_t)h.norb, P = p >> 1, Q = q >> 1;
    double t = h.eri[((P * no + P) * no + Q) * no + Q];
    if (((p ^ q) & 1) == 0) t = t - h.eri[((P * no + Q) * no + Q) * no + P];
    return t;
}

// F_p = one-body term + <pk||pk> over the reference's occupied k != p ascending
void host_fock(HostSys &h)
{
    h.fock.assign(h.nso, 0.0);
    const size_t no = (size_t)h.norb;
    for (int p = 0; p < h.nso; p++) {
        double f = h.kind == CCMC_UEG ? h.tkin[p] : h.h1[(size_t)(p >> 1) * no + (size_t)(p >> 1)];
        for (int k = 0; k < h.nel; k++) {
            if (k == p || (h.kind == CCMC_UEG && ((p ^ k) & 1))) continue;
            f = f + host_pair_ex(h, p, k);
        }
        h.fock[p] = f;
    }
    h.fock_f.assign(h.fock.begin(), h.fock.end());
}

bool build_ueg(HostSys &h)
{
    h.npw = h.nso / 2;
    // plane waves with |n|^2 <= ecut; the smallest ecut whose count is npw
    int ecut = -1;
    for (int e = 0; e < 100; e++) {
        int r = (int)std::ceil(std::sqrt((double)e)) + 1, c = 0;
        for (int x = -r; x <= r; x++)
            for (int y = -r; y <= r; y++)
                for (int z = -r; z <= r; z++)
                    if (x * x + y * y + z * z <= e) c++;
        if (c == h.npw) { ecut = e; break; }
        if (c > h.npw) break;
    }
    if (ecut < 0) return false;
    std::vector<std::array<int, 3>> v;
    int r = (int)std::ceil(std::sqrt((double)ecut)) + 1;
    for (int x = -r; x <= r; x++)
        for (int y = -r; y <= r; y++)
            for (int z = -r; z <= r; z++)
                if (x * x + y * y + z * z <= ecut) v.push_back({x, y, z});
    std::sort(v.begin(), v.end(), [](const std::array<int, 3> &a, const std::array<int, 3> &b) {
        int na = a[0] * a[0] + a[1] * a[1] + a[2] * a[2], nb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        if (na != nb) return na < nb;
        return a < b;
    });
    h.kv.resize(3 * h.npw);
    h.nmax = 0;
    for (int i = 0; i < h.npw; i++)
        for (int c = 0; c < 3; c++) {
            h.kv[3 * i + c] = v[i][c];
            h.nmax = std::max(h.nmax, std::abs(v[i][c]));
        }
    h.side = 2 * h.nmax + 1;
    h.grid.assign((size_t)h.side * h.side * h.side, -1);
    for (int i = 0; i < h.npw; i++)
        h.grid[((h.kv[3 * i] + h.nmax) * h.side + (h.kv[3 * i + 1] + h.nmax)) * h.side + (h.kv[3 * i + 2] + h.nmax)] = i;
    h.L = h.rs * std::cbrt((4.0 * PI_D * (double)h.nel) / 3.0);
    h.tkin.resize(h.nso);
    for (int p = 0; p < h.nso; p++) {
        const int *k = &h.kv[3 * (p >> 1)];
        int n2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        h.tkin[p] = ((2.0 * PI_D * PI_D) * (double)n2) / (h.L * h.L);
    }
    int n2tab = 12 * h.nmax * h.nmax + 1;
    h.vtab.assign(n2tab, 0.0);
    for (int n2 = 1; n2 < n2tab; n2++) h.vtab[n2] = 1.0 / ((PI_D * h.L) * (double)n2);
    return true;
}

struct Alloc {
    ccmc_alloc_fn fa = nullptr;
    ccmc_free_fn ff = nullptr;
    void *user = nullptr;
    std::vector<void *> blocks;
    bool failed = false;

    void *get(size_t bytes)
    {
        if (bytes == 0) bytes = 256;
        bytes = (bytes + 255) & ~(size_t)255;
        void *p = nullptr;
        if (fa) p = fa(bytes, user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
        if (!p) { failed = true; return nullptr; }
        blocks.push_back(p);
        return p;
    }
    template <typename T>
    T *arr(size_t n) { return (T *)get(n * sizeof(T)); }
    void release()
    {
        for (void *p : blocks) {
            if (ff) ff(p, user);
            else if (!fa) cudaFree(p);
        }
        blocks.clear();
    }
};

}  // namespace

constexpr int UPLOAD_CHUNKS = 8;   // pieces of a list upload whose copy and check overlap

struct ccmc_ctx {
    HostSys hs;
    StepCtx sc;
    Alloc al;
    ccmc_params prm;
    cudaStream_t stream = nullptr;
    // host mirror of the shift state
    u64 iter = 0;
    double shift = 0.0;
    int vary = 0;
    double nprev = 0.0;
    u64 records_read = 0;
    bool stepped = false;
    // pinned staging
    DevStep *h_st = nullptr;
    double *h_shift = nullptr;
    std::string err;
    i64 list_cap = 0, spawn_cap = 0, cl_cap = 0;
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    i64 phase_launch0[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // captured CUDA graph of one step (replayed on non-NULL streams)
    cudaGraphExec_t graph = nullptr;
    i64 graph_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // list upload/download: row-major determinants (K words per entry) and
    // the validation word of the last upload
    u64 *io = nullptr;
    unsigned *d_bad = nullptr, *h_bad = nullptr;
    // chunked upload: the copies run on their own stream, each chunk's check
    // on the context's stream once its copy has landed (created on first use)
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_ev[UPLOAD_CHUNKS + 1] = {};
    // the batch that steps this context, if any (it is not stepped alone
    // then), and the stream its batched steps run on
    ccmc_batch *batch = nullptr;
    cudaStream_t batch_stream = nullptr;
};

// Removes a context that is being freed from its batch (defined with the batch).
static void batch_detach(ccmc_batch *b, ccmc_ctx *c);

namespace {

ccmc_status fail(ccmc_ctx *c, ccmc_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

ccmc_status cuda_fail(ccmc_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, CCMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

// A batch member's device state is written by the batch's graph on the
// batch's stream: every call that reads or writes that state waits for it.
cudaError_t wait_batch(ccmc_ctx *ctx)
{
    return ctx->batch ? cudaStreamSynchronize(ctx->batch_stream) : cudaSuccess;
}

ccmc_status status_from_bits(ccmc_ctx *ctx, unsigned bits)
{
    // a runaway population overflows the buffers too; it is the cause to report
    if (bits & ERRB_RUNAWAY)
        return fail(ctx, CCMC_ERR_RUNAWAY, "population runaway: a step needed more than max(64 x target_pop, 2^24) "
                                           "samples or spawning attempts");
    if (bits & ERRB_SPAWN_OVERFLOW) return fail(ctx, CCMC_ERR_SPAWN_OVERFLOW, "spawned particles exceeded spawn_capacity");
    if (bits & ERRB_CLUSTER_OVERFLOW) return fail(ctx, CCMC_ERR_SPAWN_OVERFLOW, "multi-spawn clusters exceeded capacity");
    if (bits & ERRB_LIST_OVERFLOW) return fail(ctx, CCMC_ERR_LIST_OVERFLOW, "occupied excitors exceeded list_capacity");
    if (bits & ERRB_NUMERIC) return fail(ctx, CCMC_ERR_NUMERIC, "a weight left the fixed-point range");
    return CCMC_OK;
}

// validation bits of an uploaded list
enum : unsigned {
    BAD_COUNT = 1u, BAD_RANGE = 2u, BAD_SZ = 4u, BAD_MOMENTUM = 8u, BAD_LEVEL = 16u, BAD_FIRST = 32u, BAD_ORDER = 64u
};

// Uploaded list: row-major determinants -> the list's word-major layout,
// each entry checked (electron count, orbital range, the reference's S_z,
// zero total momentum for the gas, truncation level, HF first), then its
// key and diagonal energy.
template <int K, typename R>
__global__ void k_load_list(SysDev s, ListView L, const u64 *rows, i64 i0, i64 i1, unsigned *bad)
{
    const u64 alpha = 0x5555555555555555ULL;
    unsigned b = 0;
    for (i64 i = i0 + (i64)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (i64)gridDim.x * blockDim.x) {
        Det<K> d;
        int pc = 0, na = 0, holes = 0, kx = 0, ky = 0, kz = 0;
        unsigned e = 0;
#pragma unroll
        for (int w = 0; w < K; w++) {
            const u64 x = rows[i * K + w];
            d.w[w] = x;
            L.bits[w * L.cap + i] = x;
            pc += __popcll(x);
            na += __popcll(x & alpha);
            holes += __popcll(s.hf[w] & ~x);
            if (x & ~s.valid[w]) e |= BAD_RANGE;
            if (s.kind == 0)
                for (u64 m = x & s.valid[w]; m; m &= m - 1) {
                    const int q = (64 * w + __ffsll((long long)m) - 1) >> 1;
                    kx += __ldg(&s.kv[3 * q]);
                    ky += __ldg(&s.kv[3 * q + 1]);
                    kz += __ldg(&s.kv[3 * q + 2]);
                }
        }
        int na_ref = 0;
#pragma unroll
        for (int w = 0; w < K; w++) na_ref += __popcll(s.hf[w] & alpha);
        if (pc != s.nel) e |= BAD_COUNT;
        if (na != na_ref) e |= BAD_SZ;
        if (kx != 0 || ky != 0 || kz != 0) e |= BAD_MOMENTUM;
        if (holes > s.lmax) e |= BAD_LEVEL;
        if (i == 0 && holes != 0) e |= BAD_FIRST;
        if (e == 0) {
            L.key[i] = rank_key(s, d);
            L.diag[i] = holes == 0 ? 0.0 : diag_rel<K, R>(s, d);
        } else {
            L.key[i] = 0;
            L.diag[i] = 0.0;
        }
        b |= e;
    }
    if (b) atomicOr(bad, b);
}

__global__ void k_check_order(const u64 *key, i64 n, unsigned *bad)
{
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n; i += (i64)gridDim.x * blockDim.x)
        if (key[i] <= key[i - 1]) {
            atomicOr(bad, (unsigned)BAD_ORDER);
            return;
        }
}

// the list in row-major order for download
template <int K>
__global__ void k_store_list(ListView L, u64 *rows, i64 n)
{
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
#pragma unroll
        for (int w = 0; w < K; w++) rows[i * K + w] = L.bits[w * L.cap + i];
}

// the device check of entries [i0, i1) of an upload (key and Delta E computed)
cudaError_t load_list(ccmc_ctx *ctx, ListView &L, i64 i0, i64 i1)
{
    const i64 n = i1 - i0;
    const int g = (int)std::min<i64>(4096, (n + 255) / 256 + 1);
    const bool f = ctx->sc.fp32;
    cudaStream_t sm = ctx->stream;
    const SysDev &s = ctx->sc.sys;
    switch (ctx->sc.K) {
    case 1:
        if (f) k_load_list<1, float><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        else k_load_list<1, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        break;
    case 2:
        if (f) k_load_list<2, float><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        else k_load_list<2, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        break;
    case 3:
        if (f) k_load_list<3, float><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        else k_load_list<3, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad);
        break;
    case 4: k_load_list<4, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad); break;   // FP64 only
    case 5: k_load_list<5, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad); break;
    default: k_load_list<6, double><<<g, 256, 0, sm>>>(s, L, ctx->io, i0, i1, ctx->d_bad); break;
    }
    return cudaGetLastError();
}

cudaError_t store_list(ccmc_ctx *ctx, const ListView &L, i64 n)
{
    const int g = (int)std::min<i64>(4096, (n + 255) / 256 + 1);
    switch (ctx->sc.K) {
    case 1: k_store_list<1><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    case 2: k_store_list<2><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    case 3: k_store_list<3><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    case 4: k_store_list<4><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    case 5: k_store_list<5><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    default: k_store_list<6><<<g, 256, 0, ctx->stream>>>(L, ctx->io, n); break;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

ccmc_status ccmc_init(const ccmc_hamiltonian *ham, const ccmc_reference *ref, int truncation_level,
                      const ccmc_params *params, ccmc_ctx **out)
{
    if (!out) return CCMC_ERR_ARG;
    *out = nullptr;
    if (!ham || !params) return CCMC_ERR_ARG;
    const int nel = ham->n_electrons, nso = ham->n_spinorb, l = truncation_level;
    if (nel < 2 || nso <= nel || nso > 64 * MAXK || (nso & 1) || l < 1 || l > 4) return CCMC_ERR_ARG;
    if (ham->kind != CCMC_UEG && ham->kind != CCMC_GENERIC) return CCMC_ERR_ARG;
    if (ham->kind == CCMC_GENERIC && (!ham->h1 || !ham->eri)) return CCMC_ERR_ARG;
    if (!(params->tau > 0.0) || params->shift_a < 1 || !(params->d0_init > 0.0)) return CCMC_ERR_ARG;
    if (params->multispawn && !(params->a_thresh > 0.0)) return CCMC_ERR_ARG;
    if (params->radix_bits < 0 || params->radix_bits > MAX_DIGIT_BITS) return CCMC_ERR_ARG;
    if (params->precision != CCMC_FP64 && params->precision != CCMC_FP32) return CCMC_ERR_ARG;
    if (params->precision == CCMC_FP32 && nso > 192) return CCMC_ERR_ARG;   // FP32 form: up to three words
    if (params->n_ranks < 0 || params->n_ranks > 65535 || params->nu_move < 0) return CCMC_ERR_ARG;

    ccmc_ctx *ctx = new (std::nothrow) ccmc_ctx();
    if (!ctx) return CCMC_ERR_OOM;
    ctx->prm = *params;
    HostSys &h = ctx->hs;
    h.kind = ham->kind;
    h.nel = nel;
    h.nso = nso;
    h.lmax = l;
    h.nw = (nso + 63) / 64;
    h.rs = ham->rs;
    h.ecore = ham->kind == CCMC_GENERIC ? ham->e_core : 0.0;
    // the reference must be the lowest N spin-orbitals
    if (ref && ref->bits) {
        for (int w = 0; w < h.nw; w++) {
            u64 want = 0;
            for (int p = 64 * w; p < std::min(64 * w + 64, nel); p++) want |= 1ULL << (p & 63);
            if (ref->bits[w] != want) { delete ctx; return CCMC_ERR_ARG; }
        }
    }
    if (h.kind == CCMC_UEG) {
        if (!(h.rs > 0.0) || !build_ueg(h)) { delete ctx; return CCMC_ERR_ARG; }
    } else {
        h.norb = nso / 2;
        size_t n2 = (size_t)h.norb * h.norb;
        h.h1.assign(ham->h1, ham->h1 + n2);
        h.eri.assign(ham->eri, ham->eri + n2 * n2);
    }
    fill_binom(h);
    // rank tables
    h.rank_tab.assign((size_t)(l + 1) * RANK_STRIDE, 0);
    for (int c = 0; c <= l; c++)
        for (int q = 0; q < RANK_STRIDE; q++) {
            u64 s = 0;
            for (int j = 0; j <= l - c; j++) s += h.binom[q][j];
            h.rank_tab[(size_t)c * RANK_STRIDE + q] = s;
        }
    h.cocc = h.rank_tab[nel];                        // c = 0 row at q = N
    h.nvranks = h.rank_tab[nso - nel];
    // reference energy and generator constants
    std::vector<int> hfocc(nel);
    for (int p = 0; p < nel; p++) hfocc[p] = p;
    h.ehf_rel = host_diag(h, hfocc);
    host_fock(h);
    // FP32 tables: rounded from the FP64 ones
    h.tkin_f.assign(h.tkin.begin(), h.tkin.end());
    h.vtab_f.assign(h.vtab.begin(), h.vtab.end());
    h.h1_f.assign(h.h1.begin(), h.h1.end());
    h.eri_f.assign(h.eri.begin(), h.eri.end());
    h.npairs = (u64)nel * (u64)(nel - 1) / 2;
    h.nvirt = (u64)(nso - nel);
    if (h.kind == CCMC_UEG) {
        h.inv_pgen_ueg = (double)(h.npairs * h.nvirt) * 0.5;
    } else {
        for (int p = 0; p < nel; p++) h.no[p & 1]++;
        h.nv[0] = h.norb - h.no[0];
        h.nv[1] = h.norb - h.no[1];
        h.ns = (u64)h.no[0] * h.nv[0] + (u64)h.no[1] * h.nv[1];
        h.ndcase[0] = h.binom[h.nv[0]][2];
        h.ndcase[1] = h.binom[h.nv[1]][2];
        h.ndcase[2] = (u64)h.nv[0] * (u64)h.nv[1];
        h.nd = h.binom[h.no[0]][2] * h.ndcase[0] + h.binom[h.no[1]][2] * h.ndcase[1] +
               (u64)h.no[0] * h.no[1] * h.ndcase[2];
        for (int sg = 0; sg < 2; sg++)
            h.inv_pgen_single[sg] = ((double)((u64)nel * (u64)h.nv[sg]) * (double)(h.ns + h.nd)) / (double)h.ns;
        for (int c = 0; c < 3; c++)
            h.inv_pgen_double[c] = ((double)(h.npairs * h.ndcase[c]) * (double)(h.ns + h.nd)) / (double)h.nd;
    }

    // capacities
    double tgt = std::max(params->target_pop, params->d0_init);
    u64 key_bound = h.nvranks * h.cocc;
    ctx->list_cap = params->list_capacity ? (i64)params->list_capacity
                                          : (i64)std::min<double>((double)key_bound, 2.0 * tgt + 4096.0);
    // spawned records per step: about one per attempt; multi-spawn makes several attempts per cluster
    const double per = params->multispawn ? 8.0 : (params->fnc ? 3.0 : 2.0);
    ctx->spawn_cap = params->spawn_capacity ? (i64)params->spawn_capacity : (i64)(per * tgt + 65536.0);
    // the original sampler on a generic Hamiltonian queues its clusters for
    // the attempts kernel (their attempts are long and divergent); the
    // trajectory is the same either way
    const bool buffered = !params->multispawn && ham->kind == CCMC_GENERIC;
    ctx->cl_cap = params->multispawn ? (i64)(3.0 * tgt + 65536.0) : (buffered ? (i64)(4.0 * tgt + 65536.0) : 1);
    if (ctx->list_cap < 2 || ctx->spawn_cap < 1 || ctx->spawn_cap >= (i64)0xFFFFFFFFLL) {
        delete ctx;
        return CCMC_ERR_ARG;
    }

    ctx->stream = (cudaStream_t)params->cuda_stream;
    ctx->al.fa = params->alloc;
    ctx->al.ff = params->free;
    ctx->al.user = params->alloc_user;
    Alloc &al = ctx->al;

    // device tables
    SysDev &s = ctx->sc.sys;
    memset(&s, 0, sizeof(s));
    s.kind = h.kind;
    s.nel = nel;
    s.nso = nso;
    s.lmax = l;
    s.nw = h.nw;
    for (int w = 0; w < MAXK; w++) {
        u64 hf = 0, valid = 0, virt = 0;
        for (int b = 0; b < 64; b++) {
            int p = 64 * w + b;
            if (p < nel) hf |= 1ULL << b;
            if (p < nso) valid |= 1ULL << b;
            if (p >= nel && p < nso) virt |= 1ULL << b;
        }
        s.hf[w] = hf;
        s.valid[w] = valid;
        s.virt[w] = virt;
    }
    auto upload = [&](const void *src, size_t bytes) -> void * {
        void *d = al.get(bytes);
        if (d && bytes) cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
        return d;
    };
    if (h.kind == CCMC_UEG) {
        s.nmax = h.nmax;
        s.side = h.side;
        s.grid = (const int *)upload(h.grid.data(), h.grid.size() * sizeof(int));
        s.kv = (const int *)upload(h.kv.data(), h.kv.size() * sizeof(int));
        s.tkin = (const double *)upload(h.tkin.data(), h.tkin.size() * sizeof(double));
        s.vtab = (const double *)upload(h.vtab.data(), h.vtab.size() * sizeof(double));
        s.inv_pgen_ueg = h.inv_pgen_ueg;
    } else {
        s.norb = h.norb;
        s.h1 = (const double *)upload(h.h1.data(), h.h1.size() * sizeof(double));
        s.eri = (const double *)upload(h.eri.data(), h.eri.size() * sizeof(double));
        s.nv[0] = h.nv[0];
        s.nv[1] = h.nv[1];
        s.ns = h.ns;
        s.ns_nd = h.ns + h.nd;
        for (int c = 0; c < 3; c++) {
            s.ndcase[c] = h.ndcase[c];
            s.inv_pgen_double[c] = h.inv_pgen_double[c];
        }
        s.inv_pgen_single[0] = h.inv_pgen_single[0];
        s.inv_pgen_single[1] = h.inv_pgen_single[1];
    }
    s.npairs = h.npairs;
    s.nvirt = h.nvirt;
    s.rank_tab = (const u64 *)upload(h.rank_tab.data(), h.rank_tab.size() * sizeof(u64));
    if (h.kind == CCMC_UEG) {
        s.tkin_f = (const float *)upload(h.tkin_f.data(), h.tkin_f.size() * sizeof(float));
        s.vtab_f = (const float *)upload(h.vtab_f.data(), h.vtab_f.size() * sizeof(float));
    } else {
        s.h1_f = (const float *)upload(h.h1_f.data(), h.h1_f.size() * sizeof(float));
        s.eri_f = (const float *)upload(h.eri_f.data(), h.eri_f.size() * sizeof(float));
    }
    s.fock = (const double *)upload(h.fock.data(), h.fock.size() * sizeof(double));
    s.fock_f = (const float *)upload(h.fock_f.data(), h.fock_f.size() * sizeof(float));
    s.inv_pgen_ueg_f = (float)h.inv_pgen_ueg;
    for (int g = 0; g < 2; g++) s.inv_pgen_single_f[g] = (float)h.inv_pgen_single[g];
    for (int c = 0; c < 3; c++) s.inv_pgen_double_f[c] = (float)h.inv_pgen_double[c];
    s.cocc = h.cocc;
    // smallest excitation level a list entry can have: the gas sector has no
    // single excitations (momentum), the molecule has them
    s.lmin_exc = h.kind == CCMC_UEG ? 2 : 1;

    RunParams &rp = ctx->sc.prm;
    rp.tau = params->tau;
    rp.spawn_cutoff = params->spawn_cutoff;
    rp.a_thresh = params->a_thresh;
    rp.seed = params->seed;
    rp.replica = params->replica;
    rp.fnc = params->fnc ? 1 : 0;
    rp.multispawn = params->multispawn ? 1 : 0;
    rp.buffered = buffered ? 1 : 0;
    rp.a_thresh_one = params->a_thresh == 1.0 ? 1 : 0;
    rp.direct = (params->flags & CCMC_SORT_ALL) ? 0 : 1;
    rp.nranks = params->n_ranks > 1 ? params->n_ranks : 1;
    rp.nu_move = params->nu_move;
    {
        // work per step beyond which a runaway population is reported
        // instead of sampled: 64x the target, at least 2^24, at most 2^36
        double cap = 64.0 * params->target_pop;
        if (!(cap >= 16777216.0)) cap = 16777216.0;
        if (cap > 68719476736.0) cap = 68719476736.0;
        rp.work_cap = (i64)cap;
    }
    {
        // integer rounding needs a cutoff of 0 or an exact power of two
        double c = params->spawn_cutoff;
        int ex = 0;
        double m = std::frexp(c, &ex);
        bool pow2 = c == 0.0 || (c > 0.0 && m == 0.5 && ex > -1000 && ex < 1000);
        rp.int_round = pow2 ? 1 : 0;
        u64 cb;
        memcpy(&cb, &c, 8);
        rp.spawn_rs.cutoff_bits = c > 0.0 ? cb : 0;
        rp.spawn_rs.cutoff_e = c > 0.0 ? (ex - 1) - 53 : 0;   // u * 2^(ex-1) = mu * 2^(ex-1-53)
        rp.spawn_rs.cutoff_fixed = (i64)(c * 65536.0);
        rp.death_rs.cutoff_bits = 0;
        rp.death_rs.cutoff_e = 0;
        rp.death_rs.cutoff_fixed = 0;
    }

    // shapes
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    Shapes &sh = ctx->sc.sh;
    sh.scan_grid = std::min(1024, 2 * nsm);
    sh.work_grid = 4 * nsm;   // one wave of the sampler and attempt kernels (four blocks per SM)
    sh.sort_grid = 2 * nsm;
    sh.key_bits = bits_for(key_bound);
    sh.digit_bits = params->radix_bits ? params->radix_bits : MAX_DIGIT_BITS;
    sh.enum_slots = sh.scan_grid + sh.work_grid;
    sh.nranks = rp.nranks;
    ctx->sc.K = h.nw;
    ctx->sc.fp32 = params->precision == CCMC_FP32;

    // lists
    const int K = h.nw;
    for (int b = 0; b < 2; b++) {
        ListView &L = ctx->sc.list[b];
        L.cap = ctx->list_cap;
        L.bits = al.arr<u64>((size_t)K * L.cap);
        L.key = al.arr<u64>(L.cap);
        L.pop = al.arr<i64>(L.cap);
        L.diag = al.arr<double>(L.cap);
    }
    SpawnBuf &sp = ctx->sc.sp;
    sp.cap = ctx->spawn_cap;
    for (int b = 0; b < 2; b++) {
        sp.key[b] = al.arr<u64>(sp.cap);
        sp.pop[b] = al.arr<i64>(sp.cap);
    }
    ClusterBuf &cl = ctx->sc.cl;
    cl.cap = ctx->cl_cap;
    cl.bits = al.arr<u64>((size_t)K * cl.cap);
    cl.catt = al.arr<double>(cl.cap);
    cl.index = al.arr<u64>(cl.cap);
    cl.end = al.arr<i64>(cl.cap);
    WorkArrays &wa = ctx->sc.wa;
    const i64 lc = ctx->list_cap;
    wa.picks = al.arr<PickEntry>(lc);
    wa.bucket_bits = 10;
    while (wa.bucket_bits < 24 && (1LL << wa.bucket_bits) < lc / 2) wa.bucket_bits++;
    wa.bucket = al.arr<int>(((size_t)1 << wa.bucket_bits) + 1);
    wa.att_end = al.arr<i64>(lc);
    wa.catt = al.arr<double>(lc);
    wa.death = al.arr<i64>(lc);
    wa.acc = al.arr<i64>(lc);
    wa.kbucket_bits = 10;
    while (wa.kbucket_bits < 25 && (1LL << wa.kbucket_bits) < 2 * lc) wa.kbucket_bits++;
    wa.kbucket = al.arr<int>((size_t)1 << wa.kbucket_bits);
    wa.hit = al.arr<unsigned char>(lc);
    wa.newpop = al.arr<i64>(lc);
    wa.keep_l = al.arr<i64>(lc);
    wa.before = al.arr<int>(lc);
    wa.keep_s = al.arr<i64>(sp.cap);
    wa.ins = al.arr<i64>(sp.cap);
    wa.part = al.arr<i64>(4 * 2 * (size_t)std::max(sh.scan_grid, sh.work_grid));
    wa.wpart = al.arr<i64>(4 * (size_t)sh.scan_grid * (SCAN_THREADS / 32));
    wa.enum_part = al.arr<u64>(2 * (size_t)sh.enum_slots);
    wa.hist = al.arr<unsigned>((size_t)(1 << MAX_DIGIT_BITS) * sh.sort_grid);
    wa.hist_tot = al.arr<unsigned>((size_t)(1 << MAX_DIGIT_BITS));
    wa.ring = al.arr<Record>(RING);
    wa.owner = nullptr;
    wa.lcp = nullptr;
    wa.nq = nullptr;
    wa.lcp_cap = 0;
    if (rp.nranks > 1) {
        // per-processor position table: chunks of at least 32 entries, at
        // most 2^22 cells (chunks grow with the list beyond that)
        const i64 want = (i64)rp.nranks * ((lc + 31) / 32);
        wa.lcp_cap = std::max<i64>((i64)rp.nranks, std::min<i64>(want, 1LL << 22));
        wa.owner = al.arr<unsigned short>(lc);
        wa.lcp = al.arr<i64>(wa.lcp_cap);
        wa.nq = al.arr<i64>(rp.nranks);
    }
    ctx->io = al.arr<u64>((size_t)K * (size_t)lc);
    ctx->d_bad = al.arr<unsigned>(1);
    ctx->sc.st = al.arr<DevStep>(1);
    ctx->sc.d_args = al.arr<StepArgs>(1);
    if (al.failed) {
        al.release();
        delete ctx;
        return CCMC_ERR_OOM;
    }
    if (cudaMallocHost(&ctx->h_st, sizeof(DevStep)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_shift, sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_bad, sizeof(unsigned)) != cudaSuccess) {
        ccmc_free(ctx);
        return CCMC_ERR_OOM;
    }
    ctx->sc.stream = ctx->stream;
    ctx->sc.cur = 0;
    ctx->sc.sorted_buf = 0;
    {
        StepArgs &ha = ctx->sc.h_args;
        ha.s = ctx->sc.sys;
        ha.p = ctx->sc.prm;
        ha.list[0] = ctx->sc.list[0];
        ha.list[1] = ctx->sc.list[1];
        ha.sp = ctx->sc.sp;
        ha.cl = ctx->sc.cl;
        ha.wa = ctx->sc.wa;
        ha.st = ctx->sc.st;
        if (cudaMemcpy(ctx->sc.d_args, &ha, sizeof(StepArgs), cudaMemcpyHostToDevice) != cudaSuccess) {
            al.release();
            delete ctx;
            return CCMC_ERR_CUDA;
        }
    }
    ctx->sc.profile = false;
    for (int e = 0; e < 8; e++) {
        ctx->sc.launches[e] = 0;
        if (cudaEventCreate(&ctx->sc.events[e]) != cudaSuccess) {
            al.release();
            delete ctx;
            return CCMC_ERR_CUDA;
        }
    }

    // initial state: d0_init on HF
    ctx->iter = 0;
    ctx->shift = 0.0;
    ctx->vary = 0;
    ctx->nprev = params->d0_init;
    std::vector<uint64_t> hfw(K);
    for (int w = 0; w < K; w++) hfw[w] = s.hf[w];
    int64_t pop0 = (int64_t)std::llround(params->d0_init * 65536.0);
    ccmc_status st = ccmc_set_list(ctx, hfw.data(), &pop0, 1);
    if (st != CCMC_OK) {
        ccmc_free(ctx);
        return st;
    }
    *out = ctx;
    return CCMC_OK;
}

ccmc_status ccmc_set_list(ccmc_ctx *ctx, const uint64_t *bits, const int64_t *pop, size_t n)
{
    if (!ctx || !bits || !pop || n < 1) return fail(ctx, CCMC_ERR_ARG, "empty list");
    if ((i64)n > ctx->list_cap) return fail(ctx, CCMC_ERR_LIST_OVERFLOW, "list larger than list_capacity");
    const int K = ctx->hs.nw;
    // upload, then check every entry on the device: electron count, orbital
    // range, the reference's S_z and (gas) its total momentum -- the sector
    // every spawn stays in, so a gas list has no single excitations --,
    // truncation level, HF first, strictly increasing keys.  The upload goes
    // to the spare list buffer, which becomes current only if it passes.
    CK(wait_batch(ctx));
    const int nb = ctx->sc.cur ^ 1;
    ListView &L = ctx->sc.list[nb];
    CK(cudaMemsetAsync(ctx->d_bad, 0, sizeof(unsigned), ctx->stream));
    if (!ctx->up_stream) {
        CK(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
        for (int c = 0; c <= UPLOAD_CHUNKS; c++) CK(cudaEventCreateWithFlags(&ctx->up_ev[c], cudaEventDisableTiming));
    }
    // the copies start after the context's earlier work (which may still use
    // the staging rows and the spare list); the check of each piece waits
    // for its copy, so copies of later pieces overlap checks of earlier ones
    CK(cudaEventRecord(ctx->up_ev[UPLOAD_CHUNKS], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->up_stream, ctx->up_ev[UPLOAD_CHUNKS], 0));
    const i64 chunk = std::max<i64>(1 << 20, ((i64)n + UPLOAD_CHUNKS - 1) / UPLOAD_CHUNKS);
    int c = 0;
    cudaError_t ue = cudaSuccess;
    for (i64 a = 0; a < (i64)n && ue == cudaSuccess; a += chunk, c++) {
        const i64 m = std::min<i64>(chunk, (i64)n - a);
        ue = cudaMemcpyAsync(ctx->io + a * K, bits + a * K, (size_t)m * K * sizeof(u64), cudaMemcpyHostToDevice,
                             ctx->up_stream);
        if (ue == cudaSuccess)
            ue = cudaMemcpyAsync(L.pop + a, pop + a, (size_t)m * sizeof(i64), cudaMemcpyHostToDevice, ctx->up_stream);
        if (ue == cudaSuccess) ue = cudaEventRecord(ctx->up_ev[c], ctx->up_stream);
        if (ue == cudaSuccess) ue = cudaStreamWaitEvent(ctx->stream, ctx->up_ev[c], 0);
        if (ue == cudaSuccess) ue = load_list(ctx, L, a, a + m);
    }
    if (ue != cudaSuccess) {
        // no copy may still read the caller's buffers once the call returns
        cudaStreamSynchronize(ctx->up_stream);
        return cuda_fail(ctx, ue, "list upload");
    }
    {
        const int g = (int)std::min<i64>(4096, ((i64)n + 255) / 256 + 1);
        k_check_order<<<g, 256, 0, ctx->stream>>>(L.key, (i64)n, ctx->d_bad);
        CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(ctx->h_bad, ctx->d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const unsigned bad = *ctx->h_bad;
    if (bad & BAD_COUNT) return fail(ctx, CCMC_ERR_ARG, "wrong electron count");
    if (bad & BAD_RANGE) return fail(ctx, CCMC_ERR_ARG, "orbital beyond M");
    if (bad & BAD_SZ) return fail(ctx, CCMC_ERR_ARG, "determinant outside the reference's S_z sector");
    if (bad & BAD_MOMENTUM) return fail(ctx, CCMC_ERR_ARG, "determinant outside the zero-momentum sector");
    if (bad & BAD_LEVEL) return fail(ctx, CCMC_ERR_ARG, "excitor beyond the truncation level");
    if (bad & BAD_FIRST) return fail(ctx, CCMC_ERR_ARG, "first entry must be HF");
    if (bad & BAD_ORDER) return fail(ctx, CCMC_ERR_ARG, "list not sorted and unique");
    ctx->sc.cur = nb;
    DevStep st;
    memset(&st, 0, sizeof(st));
    st.iter = ctx->iter;
    st.shift = ctx->shift;
    st.n_occ = (i64)n;
    st.cur = ctx->sc.cur;
    CK(cudaMemcpy(ctx->sc.st, &st, sizeof(DevStep), cudaMemcpyHostToDevice));
    ctx->stepped = false;
    return CCMC_OK;
}

static ccmc_status check_device(ccmc_ctx *ctx)
{
    CK(wait_batch(ctx));
    CK(cudaMemcpyAsync(ctx->h_st, ctx->sc.st, sizeof(DevStep), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return status_from_bits(ctx, ctx->h_st->err);
}

// One step: replay of the captured graph when possible, else kernel launches.
static cudaError_t issue_step(ccmc_ctx *ctx)
{
    StepCtx &c = ctx->sc;
    const bool use_graph = ctx->stream != nullptr && !c.profile && !(ctx->prm.flags & CCMC_NO_GRAPH);
    if (!use_graph) return launch_step(c);
    if (!ctx->graph) {
        i64 before[8];
        for (int i = 0; i < 8; i++) before[i] = c.launches[i];
        int cur = c.cur;
        cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        e = launch_step(c);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        for (int i = 0; i < 8; i++) {
            ctx->graph_launches[i] = c.launches[i] - before[i];
            c.launches[i] = before[i];
        }
        c.cur = cur;
        if (e != cudaSuccess) {
            ctx->graph = nullptr;
            return e;
        }
    }
    cudaError_t e = cudaGraphLaunch(ctx->graph, ctx->stream);
    for (int i = 0; i < 8; i++) c.launches[i] += ctx->graph_launches[i];
    c.sorted_buf = sort_passes(c.sh) & 1;
    c.cur ^= 1;
    return e;
}

ccmc_status ccmc_step(ccmc_ctx *ctx, int nsteps)
{
    if (!ctx || nsteps < 0) return CCMC_ERR_ARG;
    if (ctx->batch) return fail(ctx, CCMC_ERR_STATE, "the context is stepped by its batch");
    const int A = ctx->prm.shift_a;
    for (int k = 0; k < nsteps; k++) {
        cudaError_t e = issue_step(ctx);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "launch_step");
        ctx->stepped = true;
        if (ctx->sc.profile) {
            CK(cudaEventSynchronize(ctx->sc.events[NPHASES]));
            for (int ph = 0; ph < NPHASES; ph++) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, ctx->sc.events[ph], ctx->sc.events[ph + 1]));
                ctx->phase_ms[ph] += ms;
            }
        }
        u64 it = ctx->iter;
        ctx->iter++;
        if ((it + 1) % (u64)A == 0) {
            ccmc_status s = check_device(ctx);
            if (s != CCMC_OK) return s;
            Record r;
            CK(cudaMemcpy(&r, ctx->sc.wa.ring + (it % RING), sizeof(Record), cudaMemcpyDeviceToHost));
            double nt = (double)r.ntot_after / 65536.0;
            double prev = ctx->shift;
            if (ctx->vary && nt > 0.0 && ctx->nprev > 0.0)
                ctx->shift = ctx->shift - (ctx->prm.zeta / ((double)A * ctx->prm.tau)) * std::log(nt / ctx->nprev);
            if (!ctx->vary && nt > ctx->prm.target_pop) ctx->vary = 1;
            ctx->nprev = nt;
            if (ctx->shift != prev) {
                *ctx->h_shift = ctx->shift;
                CK(cudaMemcpyAsync(&ctx->sc.st->shift, ctx->h_shift, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
            }
        }
    }
    return CCMC_OK;
}

ccmc_status ccmc_profile(ccmc_ctx *ctx, int32_t enable)
{
    if (!ctx) return CCMC_ERR_ARG;
    CK(wait_batch(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->sc.profile = enable != 0;
    for (int ph = 0; ph < 8; ph++) {
        ctx->phase_ms[ph] = 0.0;
        ctx->phase_launch0[ph] = ctx->sc.launches[ph];
    }
    return CCMC_OK;
}

ccmc_status ccmc_phase_times(ccmc_ctx *ctx, double *ms, int64_t *launches, int32_t nphases, int64_t *total_launches)
{
    if (!ctx || nphases < 0) return CCMC_ERR_ARG;
    for (int ph = 0; ph < nphases && ph < NPHASES; ph++) {
        if (ms) ms[ph] = ctx->phase_ms[ph];
        if (launches) launches[ph] = ctx->sc.launches[ph] - ctx->phase_launch0[ph];
    }
    if (total_launches) {
        i64 t = 0;
        for (int ph = 0; ph < NPHASES; ph++) t += ctx->sc.launches[ph];
        *total_launches = t;
    }
    return CCMC_OK;
}

ccmc_status ccmc_sync(ccmc_ctx *ctx)
{
    if (!ctx) return CCMC_ERR_ARG;
    return check_device(ctx);
}

ccmc_status ccmc_energy(ccmc_ctx *ctx, double *e_proj, double *e_num, double *n0, double *shift, double *n_total)
{
    if (!ctx) return CCMC_ERR_ARG;
    ccmc_status s = check_device(ctx);
    if (s != CCMC_OK) return s;
    if (!ctx->stepped && ctx->iter == 0) {
        if (e_proj) *e_proj = 0.0;
        if (e_num) *e_num = 0.0;
        if (n0) *n0 = ctx->prm.d0_init;
        if (shift) *shift = ctx->shift;
        if (n_total) *n_total = ctx->prm.d0_init;
        return CCMC_OK;
    }
    Record r;
    CK(cudaMemcpy(&r, ctx->sc.wa.ring + ((ctx->iter - 1) % RING), sizeof(Record), cudaMemcpyDeviceToHost));
    double n0d = (double)r.n0 / 65536.0;
    if (e_proj) *e_proj = n0d != 0.0 ? r.e_num / n0d : 0.0;
    if (e_num) *e_num = r.e_num;
    if (n0) *n0 = n0d;
    if (shift) *shift = r.shift;
    if (n_total) *n_total = (double)r.ntot_after / 65536.0;
    return CCMC_OK;
}

ccmc_status ccmc_reference_energy(ccmc_ctx *ctx, double *e_hf)
{
    if (!ctx || !e_hf) return CCMC_ERR_ARG;
    *e_hf = ctx->hs.ehf_rel + ctx->hs.ecore;
    return CCMC_OK;
}

ccmc_status ccmc_get_records(ccmc_ctx *ctx, ccmc_record *out, size_t cap, size_t *n)
{
    if (!ctx || !n) return CCMC_ERR_ARG;
    *n = 0;
    ccmc_status s = check_device(ctx);
    if (s != CCMC_OK) return s;
    u64 first = ctx->records_read;
    if (ctx->iter > (u64)RING && first < ctx->iter - RING) first = ctx->iter - RING;
    u64 count = ctx->iter - first;
    if (count > cap) {
        first = ctx->iter - cap;
        count = cap;
    }
    static_assert(sizeof(Record) == sizeof(ccmc_record), "record layout");
    for (u64 k = 0; k < count; k++)
        CK(cudaMemcpy(out + k, ctx->sc.wa.ring + ((first + k) % RING), sizeof(Record), cudaMemcpyDeviceToHost));
    ctx->records_read = ctx->iter;
    *n = (size_t)count;
    return CCMC_OK;
}

ccmc_status ccmc_list_size(ccmc_ctx *ctx, size_t *n)
{
    if (!ctx || !n) return CCMC_ERR_ARG;
    ccmc_status s = check_device(ctx);
    if (s != CCMC_OK) return s;
    *n = (size_t)ctx->h_st->n_occ;
    return CCMC_OK;
}

ccmc_status ccmc_get_list(ccmc_ctx *ctx, uint64_t *bits, uint64_t *keys, int64_t *pop, size_t cap, size_t *n)
{
    size_t m = 0;
    ccmc_status s = ccmc_list_size(ctx, &m);
    if (s != CCMC_OK) return s;
    if (n) *n = m;
    if (m > cap) return fail(ctx, CCMC_ERR_ARG, "buffer too small");
    const ListView &L = ctx->sc.list[ctx->sc.cur];
    const int K = ctx->hs.nw;
    if (bits) {
        CK(store_list(ctx, L, (i64)m));
        CK(cudaMemcpyAsync(bits, ctx->io, m * (size_t)K * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (keys) CK(cudaMemcpyAsync(keys, L.key, m * sizeof(u64), cudaMemcpyDeviceToHost, ctx->stream));
    if (pop) CK(cudaMemcpyAsync(pop, L.pop, m * sizeof(i64), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return CCMC_OK;
}

ccmc_status ccmc_get_spawned(ccmc_ctx *ctx, uint64_t *keys, int64_t *pop, size_t cap, size_t *n)
{
    if (!ctx || !n) return CCMC_ERR_ARG;
    ccmc_status s = check_device(ctx);
    if (s != CCMC_OK) return s;
    if (!ctx->stepped) {
        *n = 0;
        return CCMC_OK;
    }
    i64 m = std::min<i64>(ctx->h_st->n_sp, ctx->spawn_cap);
    *n = (size_t)m;
    if ((size_t)m > cap) return fail(ctx, CCMC_ERR_ARG, "buffer too small");
    if (keys) CK(cudaMemcpy(keys, ctx->sc.sp.key[ctx->sc.sorted_buf], m * sizeof(u64), cudaMemcpyDeviceToHost));
    if (pop) CK(cudaMemcpy(pop, ctx->sc.sp.pop[ctx->sc.sorted_buf], m * sizeof(i64), cudaMemcpyDeviceToHost));
    return CCMC_OK;
}

ccmc_status ccmc_get_death(ccmc_ctx *ctx, int64_t *death, size_t cap, size_t *n)
{
    if (!ctx || !n) return CCMC_ERR_ARG;
    CK(wait_batch(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->stepped) {
        *n = 0;
        return CCMC_OK;
    }
    // the death deltas belong to the list at the start of the latest step
    CK(cudaMemcpy(ctx->h_st, ctx->sc.st, sizeof(DevStep), cudaMemcpyDeviceToHost));
    size_t m = (size_t)ctx->h_st->n_start;
    *n = m;
    if (m > cap) return fail(ctx, CCMC_ERR_ARG, "buffer too small");
    if (death) CK(cudaMemcpy(death, ctx->sc.wa.death, m * sizeof(i64), cudaMemcpyDeviceToHost));
    return CCMC_OK;
}

ccmc_status ccmc_set_state(ccmc_ctx *ctx, uint64_t iter, double shift, int32_t vary, double nprev)
{
    if (!ctx) return CCMC_ERR_ARG;
    ctx->iter = iter;
    ctx->shift = shift;
    ctx->vary = vary ? 1 : 0;
    ctx->nprev = nprev;
    ctx->records_read = iter;
    CK(wait_batch(ctx));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(&ctx->sc.st->iter, &iter, sizeof(u64), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(&ctx->sc.st->shift, &shift, sizeof(double), cudaMemcpyHostToDevice));
    return CCMC_OK;
}

ccmc_status ccmc_get_state(ccmc_ctx *ctx, uint64_t *iter, double *shift, int32_t *vary, double *nprev)
{
    if (!ctx) return CCMC_ERR_ARG;
    if (iter) *iter = ctx->iter;
    if (shift) *shift = ctx->shift;
    if (vary) *vary = ctx->vary;
    if (nprev) *nprev = ctx->nprev;
    return CCMC_OK;
}

ccmc_status ccmc_save(ccmc_ctx *ctx, const char *path)
{
    if (!ctx || !path) return CCMC_ERR_ARG;
    size_t n = 0;
    ccmc_status s = ccmc_list_size(ctx, &n);
    if (s != CCMC_OK) return s;
    const int K = ctx->hs.nw;
    std::vector<uint64_t> bits((size_t)K * n);
    std::vector<int64_t> pop(n);
    s = ccmc_get_list(ctx, bits.data(), nullptr, pop.data(), n, &n);
    if (s != CCMC_OK) return s;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ctx, CCMC_ERR_ARG, "cannot open checkpoint for writing");
    const char magic[8] = {'C', 'C', 'M', 'C', 'C', 'K', '0', '1'};
    int32_t hdr[4] = {ctx->hs.nel, ctx->hs.nso, ctx->hs.lmax, K};
    u64 nn = n;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(&ctx->iter, 8, 1, f) == 1 && fwrite(&ctx->shift, 8, 1, f) == 1 &&
              fwrite(&ctx->vary, 4, 1, f) == 1 && fwrite(&ctx->nprev, 8, 1, f) == 1 && fwrite(&nn, 8, 1, f) == 1 &&
              fwrite(bits.data(), 8, bits.size(), f) == bits.size() && fwrite(pop.data(), 8, n, f) == n;
    fclose(f);
    return ok ? CCMC_OK : fail(ctx, CCMC_ERR_ARG, "checkpoint write failed");
}

ccmc_status ccmc_load(ccmc_ctx *ctx, const char *path)
{
    if (!ctx || !path) return CCMC_ERR_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ctx, CCMC_ERR_ARG, "cannot open checkpoint");
    char magic[8];
    int32_t hdr[4];
    u64 iter, nn;
    double shift, nprev;
    int32_t vary;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "CCMCCK01", 8) == 0 && fread(hdr, sizeof(hdr), 1, f) == 1 &&
              fread(&iter, 8, 1, f) == 1 && fread(&shift, 8, 1, f) == 1 && fread(&vary, 4, 1, f) == 1 &&
              fread(&nprev, 8, 1, f) == 1 && fread(&nn, 8, 1, f) == 1;
    if (!ok || hdr[0] != ctx->hs.nel || hdr[1] != ctx->hs.nso || hdr[2] != ctx->hs.lmax || hdr[3] != ctx->hs.nw ||
        nn < 1 || nn > (u64)ctx->list_cap) {
        fclose(f);
        return fail(ctx, CCMC_ERR_ARG, "checkpoint does not match this context");
    }
    const int K = ctx->hs.nw;
    std::vector<uint64_t> bits((size_t)K * nn);
    std::vector<int64_t> pop(nn);
    ok = fread(bits.data(), 8, bits.size(), f) == bits.size() && fread(pop.data(), 8, nn, f) == nn;
    fclose(f);
    if (!ok) return fail(ctx, CCMC_ERR_ARG, "truncated checkpoint");
    ccmc_status s = ccmc_set_state(ctx, iter, shift, vary, nprev);
    if (s != CCMC_OK) return s;
    return ccmc_set_list(ctx, bits.data(), pop.data(), nn);
}

const char *ccmc_last_error(ccmc_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

void ccmc_free(ccmc_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->batch) batch_detach(ctx->batch, ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->al.release();
    for (int e = 0; e < 8; e++)
        if (ctx->sc.events[e]) cudaEventDestroy(ctx->sc.events[e]);
    if (ctx->up_stream) {
        cudaStreamSynchronize(ctx->up_stream);
        cudaStreamDestroy(ctx->up_stream);
    }
    for (int c = 0; c <= UPLOAD_CHUNKS; c++)
        if (ctx->up_ev[c]) cudaEventDestroy(ctx->up_ev[c]);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    if (ctx->h_shift) cudaFreeHost(ctx->h_shift);
    if (ctx->h_bad) cudaFreeHost(ctx->h_bad);
    delete ctx;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form
// ---------------------------------------------------------------------------

namespace {

// latest record and error word of every replica, for the host's shift control
__global__ void k_batch_gather(const StepArgs *A, int n, Record *out, unsigned *err)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const DevStep *st = A[r].st;
    out[r] = A[r].wa.ring[(st->iter + RING - 1) % RING];
    err[r] = st->err;
}

__global__ void k_batch_shift(const StepArgs *A, int n, const double *shift)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) A[r].st->shift = shift[r];
}

struct BatchGroup {
    int K = 1;
    bool fp32 = false, multi = false;
    std::vector<int> members;
    StepArgs *d_args = nullptr;
    int key_bits = 1;
    int *d_vstart = nullptr;        // sampler plan (members + 1 entries)
    unsigned *d_counter = nullptr;
};

// Shapes the tuner chooses between.
struct BatchShape {
    int work = 64;      // per-replica blocks of the list, merge and sort kernels
    int tile = 1024;    // samples per share of the persistent sampler
    int digit = 8;      // radix digit bits
};

constexpr int TUNE_STAGES = 3;
const int TUNE_WORK[] = {32, 64, 128, 256};
const int TUNE_TILE[] = {256, 512, 1024, 2048, 4096};
const int TUNE_DIGIT[] = {8, 6};

int tune_count(int stage)
{
    return stage == 0 ? 4 : stage == 1 ? 5 : 2;
}

}  // namespace

struct ccmc_batch {
    std::vector<ccmc_ctx *> ctxs;
    cudaStream_t stream = nullptr;
    bool member_freed = false;        // a member context was freed: the batch can no longer step
    std::vector<BatchGroup> groups;
    StepArgs *d_all = nullptr;       // every replica, for gather / shift scatter
    Record *d_rec = nullptr, *h_rec = nullptr;
    unsigned *d_err = nullptr, *h_err = nullptr;
    double *d_shift = nullptr, *h_shift = nullptr;
    Shapes sh;                        // per-replica shapes (key_bits set per group)
    Shapes lim;                       // what every context allocated for
    BatchShape shape;                 // current choice
    int flat_grid = 0;                // blocks of the persistent sampler
    bool tuned = false;
    int tune_stage = 0, tune_idx = 0, tunings = 0;
    BatchShape tune_best;
    float tune_best_ms = 0.0f;
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    double pop_now = 0.0, pop_tuned = 0.0;   // batch population at the last boundary / last tuning
    cudaGraphExec_t graph = nullptr;
    i64 launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    i64 graph_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<void *> blocks;
    // opt-in phase timers
    bool profile = false;
    std::vector<cudaEvent_t> events;   // 8 per group
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    i64 launch0[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// A member freed while in the batch: wait for the batch's work, drop the
// member's slot and refuse further batched steps (the captured graph and
// the per-replica argument arrays still point at the member's memory).
static void batch_detach(ccmc_batch *b, ccmc_ctx *c)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (ccmc_ctx *&m : b->ctxs)
        if (m == c) m = nullptr;
    b->member_freed = true;
    c->batch = nullptr;
    c->batch_stream = nullptr;
}

namespace {

// per-replica shapes for a tuner choice, within what every context allocated
Shapes shapes_for(const ccmc_batch *b, const BatchShape &c)
{
    Shapes sh = b->lim;
    sh.work_grid = std::min(c.work, b->lim.work_grid);
    sh.scan_grid = std::min(std::max(2, c.work / 2), b->lim.scan_grid);
    sh.sort_grid = std::min(std::max(2, c.work / 2), b->lim.sort_grid);
    sh.digit_bits = c.digit;
    sh.enum_slots = sh.scan_grid + sh.work_grid;
    return sh;
}

cudaError_t batch_launch(ccmc_batch *b, const Shapes &base)
{
    for (size_t gi = 0; gi < b->groups.size(); gi++) {
        BatchGroup &g = b->groups[gi];
        Shapes sh = base;
        sh.key_bits = g.key_bits;
        FlatPlan plan;
        plan.vstart = g.d_vstart;
        plan.counter = g.d_counter;
        plan.per_block = b->shape.tile;
        plan.wmax = b->lim.work_grid;
        plan.grid = b->flat_grid;
        const cudaEvent_t *ev = b->profile ? &b->events[8 * gi] : nullptr;
        cudaError_t e = launch_group(g.d_args, (int)g.members.size(), g.K, g.fp32, sh, g.multi, b->stream,
                                     b->launches, ev, &plan);
        if (e != cudaSuccess) return e;
    }
    if (b->profile) {
        for (size_t gi = 0; gi < b->groups.size(); gi++) {
            if (cudaEventSynchronize(b->events[8 * gi + NPHASES]) != cudaSuccess) return cudaErrorUnknown;
            for (int ph = 0; ph < NPHASES; ph++) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, b->events[8 * gi + ph], b->events[8 * gi + ph + 1]);
                b->phase_ms[ph] += ms;
            }
        }
    }
    return cudaSuccess;
}

void batch_after_step(ccmc_batch *b, const Shapes &launched)
{
    for (BatchGroup &g : b->groups) {
        Shapes sh = launched;
        sh.key_bits = g.key_bits;
        for (int m : g.members) {
            ccmc_ctx *c = b->ctxs[m];
            c->sc.cur ^= 1;
            c->sc.sorted_buf = sort_passes(sh) & 1;
            c->stepped = true;
            c->iter++;
        }
    }
}

// shift control for the contexts that reached a boundary with this step
ccmc_status batch_boundaries(ccmc_batch *b)
{
    const int n = (int)b->ctxs.size();
    bool any = false;
    for (ccmc_ctx *c : b->ctxs) any = any || (c->iter % (u64)c->prm.shift_a) == 0;
    if (!any) return CCMC_OK;
    k_batch_gather<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_all, n, b->d_rec, b->d_err);
    if (cudaMemcpyAsync(b->h_rec, b->d_rec, sizeof(Record) * n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->h_err, b->d_err, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return CCMC_ERR_CUDA;
    bool changed = false;
    double pop = 0.0;
    for (int r = 0; r < n; r++) pop += (double)b->h_rec[r].ntot_after / 65536.0;
    b->pop_now = pop;
    // a population twice or half as large as at the last tuning: tune again
    if (b->tuned && (pop > 2.0 * b->pop_tuned || pop < 0.5 * b->pop_tuned)) {
        b->tuned = false;
        b->tune_stage = 0;
        b->tune_idx = 0;
        b->tune_best = b->shape;
        b->tune_best_ms = 1e30f;
    }
    for (int r = 0; r < n; r++) {
        ccmc_ctx *c = b->ctxs[r];
        if (b->h_err[r]) return status_from_bits(c, b->h_err[r]);
        b->h_shift[r] = c->shift;
        if ((c->iter % (u64)c->prm.shift_a) != 0) continue;
        const int A = c->prm.shift_a;
        double nt = (double)b->h_rec[r].ntot_after / 65536.0;
        double prev = c->shift;
        if (c->vary && nt > 0.0 && c->nprev > 0.0)
            c->shift = c->shift - (c->prm.zeta / ((double)A * c->prm.tau)) * std::log(nt / c->nprev);
        if (!c->vary && nt > c->prm.target_pop) c->vary = 1;
        c->nprev = nt;
        b->h_shift[r] = c->shift;
        changed = changed || c->shift != prev;
    }
    if (changed) {
        if (cudaMemcpyAsync(b->d_shift, b->h_shift, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess)
            return CCMC_ERR_CUDA;
        k_batch_shift<<<(n + 127) / 128, 128, 0, b->stream>>>(b->d_all, n, b->d_shift);
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CCMC_ERR_CUDA;
    }
    return CCMC_OK;
}

}  // namespace

extern "C" {

ccmc_status ccmc_batch_create(ccmc_ctx **ctxs, int32_t n, void *cuda_stream, ccmc_batch **out)
{
    if (!out) return CCMC_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n < 1 || !cuda_stream) return CCMC_ERR_ARG;
    for (int r = 0; r < n; r++) {
        if (!ctxs[r] || ctxs[r]->prm.shift_a != ctxs[0]->prm.shift_a) return CCMC_ERR_ARG;
        if (ctxs[r]->batch) return CCMC_ERR_STATE;   // already in a batch
        for (int q = 0; q < r; q++)
            if (ctxs[q] == ctxs[r]) return CCMC_ERR_ARG;
    }
    ccmc_batch *b = new (std::nothrow) ccmc_batch();
    if (!b) return CCMC_ERR_OOM;
    b->ctxs.assign(ctxs, ctxs + n);
    b->stream = (cudaStream_t)cuda_stream;
    for (int r = 0; r < n; r++) {
        ccmc_ctx *c = ctxs[r];
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            delete b;
            return CCMC_ERR_CUDA;
        }
        bool multi = c->prm.fnc || c->prm.multispawn || c->sc.prm.buffered;
        bool fp32 = c->sc.fp32;
        BatchGroup *g = nullptr;
        for (BatchGroup &x : b->groups)
            if (x.K == c->sc.K && x.fp32 == fp32) g = &x;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->K = c->sc.K;
            g->fp32 = fp32;
        }
        g->multi = g->multi || multi;
        g->members.push_back(r);
        g->key_bits = std::max(g->key_bits, c->sc.sh.key_bits);
    }
    auto dalloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        b->blocks.push_back(p);
        return p;
    };
    std::vector<StepArgs> all(n);
    for (int r = 0; r < n; r++) all[r] = ctxs[r]->sc.h_args;
    b->d_all = (StepArgs *)dalloc(sizeof(StepArgs) * n);
    b->d_rec = (Record *)dalloc(sizeof(Record) * n);
    b->d_err = (unsigned *)dalloc(sizeof(unsigned) * n);
    b->d_shift = (double *)dalloc(sizeof(double) * n);
    bool ok = b->d_all && b->d_rec && b->d_err && b->d_shift &&
              cudaMallocHost(&b->h_rec, sizeof(Record) * n) == cudaSuccess &&
              cudaMallocHost(&b->h_err, sizeof(unsigned) * n) == cudaSuccess &&
              cudaMallocHost(&b->h_shift, sizeof(double) * n) == cudaSuccess &&
              cudaMemcpy(b->d_all, all.data(), sizeof(StepArgs) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    for (BatchGroup &g : b->groups) {
        std::vector<StepArgs> ga;
        for (int m : g.members) ga.push_back(all[m]);
        g.d_args = (StepArgs *)dalloc(sizeof(StepArgs) * ga.size());
        g.d_vstart = (int *)dalloc(sizeof(int) * (ga.size() + 1));
        g.d_counter = (unsigned *)dalloc(sizeof(unsigned));
        ok = ok && g.d_args && g.d_vstart && g.d_counter &&
             cudaMemcpy(g.d_args, ga.data(), sizeof(StepArgs) * ga.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    // per-replica shapes may not exceed what every context allocated for
    Shapes lim = ctxs[0]->sc.sh;
    for (int r = 1; r < n; r++) {
        lim.scan_grid = std::min(lim.scan_grid, ctxs[r]->sc.sh.scan_grid);
        lim.work_grid = std::min(lim.work_grid, ctxs[r]->sc.sh.work_grid);
        lim.sort_grid = std::min(lim.sort_grid, ctxs[r]->sc.sh.sort_grid);
        lim.nranks = std::max(lim.nranks, ctxs[r]->sc.sh.nranks);
    }
    lim.digit_bits = MAX_DIGIT_BITS;
    b->lim = lim;
    b->sh = shapes_for(b, b->shape);
    int dev = 0, sms = 0;
    ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
         cudaEventCreate(&b->tune_ev[0]) == cudaSuccess && cudaEventCreate(&b->tune_ev[1]) == cudaSuccess;
    b->flat_grid = SAMPLE_BLOCKS_PER_SM * std::max(1, sms);   // resident blocks of the persistent sampler
    for (int r = 0; r < n; r++) b->pop_now += ctxs[r]->prm.d0_init;
    b->tune_best = b->shape;
    b->tune_best_ms = 1e30f;
    if (!ok) {
        ccmc_batch_free(b);
        return CCMC_ERR_OOM;
    }
    for (ccmc_ctx *c : b->ctxs) {
        c->batch = b;
        c->batch_stream = b->stream;
    }
    *out = b;
    return CCMC_OK;
}

// the candidate for the current tuning position
static BatchShape tune_candidate(const ccmc_batch *b)
{
    BatchShape c = b->tune_best;
    if (b->tune_stage == 0) c.work = TUNE_WORK[b->tune_idx];
    else if (b->tune_stage == 1) c.tile = TUNE_TILE[b->tune_idx];
    else c.digit = TUNE_DIGIT[b->tune_idx];
    return c;
}

// One timed tuning step: the candidates of one stage are tried in turn with
// the best of the earlier stages (coordinate search); after the last stage
// the best choice is kept and the graph is captured again.
static ccmc_status batch_tune_step(ccmc_batch *b, Shapes &launched)
{
    b->shape = tune_candidate(b);
    b->sh = shapes_for(b, b->shape);
    launched = b->sh;
    if (cudaEventRecord(b->tune_ev[0], b->stream) != cudaSuccess) return CCMC_ERR_CUDA;
    if (batch_launch(b, b->sh) != cudaSuccess) return CCMC_ERR_CUDA;
    if (cudaEventRecord(b->tune_ev[1], b->stream) != cudaSuccess) return CCMC_ERR_CUDA;
    if (cudaEventSynchronize(b->tune_ev[1]) != cudaSuccess) return CCMC_ERR_CUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, b->tune_ev[0], b->tune_ev[1]);
    if (ms < b->tune_best_ms) {
        b->tune_best_ms = ms;
        b->tune_best = b->shape;
    }
    if (++b->tune_idx == tune_count(b->tune_stage)) {
        b->tune_idx = 0;
        b->tune_stage++;
        b->tune_best_ms = 1e30f;   // the next stage is timed afresh
        if (b->tune_stage == TUNE_STAGES) {
            b->shape = b->tune_best;
            b->sh = shapes_for(b, b->shape);
            b->tuned = true;
            b->tunings++;
            b->pop_tuned = b->pop_now;
            if (b->graph) {
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
        }
    }
    return CCMC_OK;
}

static ccmc_status batch_capture(ccmc_batch *b)
{
    i64 before[8];
    for (int i = 0; i < 8; i++) before[i] = b->launches[i];
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return CCMC_ERR_CUDA;
    e = batch_launch(b, b->sh);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int i = 0; i < 8; i++) {
        b->graph_launches[i] = b->launches[i] - before[i];
        b->launches[i] = before[i];
    }
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return CCMC_ERR_CUDA;
    }
    return CCMC_OK;
}

ccmc_status ccmc_step_batched(ccmc_batch *b, int32_t nsteps)
{
    if (!b || nsteps < 0) return CCMC_ERR_ARG;
    if (b->member_freed) return CCMC_ERR_STATE;
    for (int k = 0; k < nsteps; k++) {
        Shapes launched = b->sh;
        if (!b->tuned) {
            ccmc_status st = batch_tune_step(b, launched);
            if (st != CCMC_OK) return st;
        } else if (b->profile) {
            if (batch_launch(b, b->sh) != cudaSuccess) return CCMC_ERR_CUDA;
        } else {
            if (!b->graph) {
                ccmc_status st = batch_capture(b);
                if (st != CCMC_OK) return st;
            }
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return CCMC_ERR_CUDA;
            for (int i = 0; i < 8; i++) b->launches[i] += b->graph_launches[i];
        }
        batch_after_step(b, launched);
        ccmc_status st = batch_boundaries(b);
        if (st != CCMC_OK) return st;
    }
    return CCMC_OK;
}

ccmc_status ccmc_batch_profile(ccmc_batch *b, int32_t enable)
{
    if (!b) return CCMC_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CCMC_ERR_CUDA;
    if (enable && b->events.empty()) {
        b->events.resize(8 * b->groups.size());
        for (cudaEvent_t &e : b->events)
            if (cudaEventCreate(&e) != cudaSuccess) return CCMC_ERR_CUDA;
    }
    b->profile = enable != 0;
    for (int i = 0; i < 8; i++) {
        b->phase_ms[i] = 0.0;
        b->launch0[i] = b->launches[i];
    }
    return CCMC_OK;
}

ccmc_status ccmc_batch_phase_times(ccmc_batch *b, double *ms, int64_t *launches, int32_t nphases,
                                   int64_t *total_launches)
{
    if (!b || nphases < 0) return CCMC_ERR_ARG;
    for (int ph = 0; ph < nphases && ph < NPHASES; ph++) {
        if (ms) ms[ph] = b->phase_ms[ph];
        if (launches) launches[ph] = b->launches[ph] - b->launch0[ph];
    }
    if (total_launches) {
        i64 t = 0;
        for (int ph = 0; ph < NPHASES; ph++) t += b->launches[ph];
        *total_launches = t;
    }
    return CCMC_OK;
}

ccmc_status ccmc_batch_info(ccmc_batch *b, int32_t *work_blocks, int32_t *sample_tile, int32_t *digit_bits,
                            int32_t *groups, int32_t *tunings)
{
    if (!b) return CCMC_ERR_ARG;
    if (work_blocks) *work_blocks = b->sh.work_grid;
    if (sample_tile) *sample_tile = b->shape.tile;
    if (digit_bits) *digit_bits = b->sh.digit_bits;
    if (groups) *groups = (int32_t)b->groups.size();
    if (tunings) *tunings = b->tunings;
    return CCMC_OK;
}

void ccmc_batch_free(ccmc_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (ccmc_ctx *c : b->ctxs)
        if (c && c->batch == b) {
            c->batch = nullptr;
            c->batch_stream = nullptr;
        }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (cudaEvent_t e : b->tune_ev)
        if (e) cudaEventDestroy(e);
    for (void *p : b->blocks) cudaFree(p);
    if (b->h_rec) cudaFreeHost(b->h_rec);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->h_shift) cudaFreeHost(b->h_shift);
    delete b;
}

}  // extern "C"
