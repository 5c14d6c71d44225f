// ccmc_step.cu -- the kernels of one CCMC time step (Spencer et al.,
// arXiv:1807.03749, Sec. II and Sec. IV.B-C) that do not depend on the
// determinant word count, the dispatch of a step to the word count's
// instantiation (ccmc_step_k<K>.cu) and the allocation-free sort-and-reduce
// entry point.  The device building blocks are in ccmc_kernels.cuh.
//
//  a1  k_scan_partial / k_scan_top           a7  k_sort_hist / scan / scatter
//  a8  k_seg_count / k_part_scan / k_seg_write
//  a9  k_merge_match / k_merge_count / k_keep_top (k_keep_scatter, k_scatter_new: per word count)
//  a10 k_finalize      batch: k_sample_plan
//  ccmc_reduce_records_noalloc (end of file): the sort and reduction as a
//      standalone call on a static scratch array
#include <mutex>

#include "../../include/ccmc.h"
#include "ccmc_kernels.cuh"

namespace ccmc {

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_partial(const StepArgs *__restrict__ A)
{
    REPLICA;
    d_scan_partial(a.list[cur_], a.st, a.p, a.wa);
}

__global__ void __launch_bounds__(1024) k_scan_top(const StepArgs *__restrict__ A, int grid)
{
    REPLICA;
    d_scan_top(a.list[cur_], a.st, a.p, a.wa, grid, a.s.lmax);
}

// Batch work plan for the sampler: virtual blocks per replica from its
// sample count, their prefix, the reset work counter, and zeroed E_num
// partials for the slots a replica does not use this step (the final
// reduction reads wmax of them).  One block.
__global__ void __launch_bounds__(1024) k_sample_plan(const StepArgs *__restrict__ A, int nrep, FlatPlan fp,
                                                       int enum_base)
{
    __shared__ int sm[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int r0 = 0; r0 < nrep; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        int want = 0;
        if (r < nrep) {
            const i64 ns = A[r].st->n_sel;
            const i64 w = (ns + fp.per_block - 1) / fp.per_block;
            want = (int)(w < 1 ? 1 : (w > fp.wmax ? fp.wmax : w));
        }
        int tot;
        const int incl = block_incl_scan(want, sm, tot);
        if (r < nrep) fp.vstart[r] = carry + incl - want;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        fp.vstart[nrep] = carry;
        *fp.counter = 0u;
    }
    __syncthreads();
    // unused E_num slots of every replica
    for (int r = 0; r < nrep; r++) {
        const i64 ns = A[r].st->n_sel;
        const i64 w = (ns + fp.per_block - 1) / fp.per_block;
        const int used = (int)(w < 1 ? 1 : (w > fp.wmax ? fp.wmax : w));
        u64 *ep = A[r].wa.enum_part;
        for (int q = used + (int)threadIdx.x; q < fp.wmax; q += blockDim.x) {
            ep[2 * (enum_base + q)] = 0;
            ep[2 * (enum_base + q) + 1] = 0;
        }
    }
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const StepArgs *__restrict__ A, int src, int shift, int bits)
{
    const StepArgs &a = A[blockIdx.y];
    d_sort_hist(a.sp.key[src], a.st, a.sp.cap, shift, bits, a.wa.hist);
}

__global__ void __launch_bounds__(1024) k_sort_scan(const StepArgs *__restrict__ A, int grid)
{
    const StepArgs &a = A[blockIdx.y];
    d_sort_scan(a.wa.hist, grid, a.wa.hist_tot);
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const StepArgs *__restrict__ A, int src, int shift, int bits)
{
    const StepArgs &a = A[blockIdx.y];
    d_sort_scatter(a.sp.key[src], a.sp.pop[src], a.sp.key[src ^ 1], a.sp.pop[src ^ 1], a.st, a.sp.cap, shift, bits,
                   a.wa.hist, a.wa.hist_tot);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_count(const StepArgs *__restrict__ A, int src)
{
    const StepArgs &a = A[blockIdx.y];
    d_seg_count(a.sp.key[src], a.st, a.sp.cap, a.sp.pop[src ^ 1], a.wa);
}

__global__ void __launch_bounds__(1024) k_part_scan(const StepArgs *__restrict__ A, int grid)
{
    const StepArgs &a = A[blockIdx.y];
    d_part_scan(a.wa, grid, 0, 2, &a.st->n_keys);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_write(const StepArgs *__restrict__ A, int src)
{
    const StepArgs &a = A[blockIdx.y];
    d_seg_write(a.sp.key[src], a.sp.pop[src], a.st, a.sp.cap, a.sp.key[src ^ 1], a.sp.pop[src ^ 1], a.wa);
}

__global__ void __launch_bounds__(WORK_THREADS) k_merge_match(const StepArgs *__restrict__ A, int src)
{
    REPLICA;
    d_merge_match(a.list[cur_], a.st, a.p, a.wa, a.sp.key[src ^ 1], a.sp.pop[src ^ 1]);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_merge_count(const StepArgs *__restrict__ A, int G)
{
    REPLICA;
    d_merge_count(a.list[cur_], a.st, a.p, a.wa, G);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_local_scan(const StepArgs *__restrict__ A)
{
    const StepArgs &a = A[blockIdx.y];
    d_local_scan(a.st, a.p, a.wa);
}

__global__ void __launch_bounds__(1024) k_keep_top(const StepArgs *__restrict__ A, int G)
{
    const StepArgs &a = A[blockIdx.y];
    d_keep_top(a.st, a.wa, G);
}

__global__ void __launch_bounds__(1024) k_finalize(const StepArgs *__restrict__ A, int slots)
{
    REPLICA;
    d_finalize(a.st, a.p, a.wa, a.cl, slots, a.list[cur_ ^ 1].cap);
}

// pointer-argument forms of the sort and reduction kernels (used without a context)
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist_p(const u64 *keys, const DevStep *st, i64 cap, int shift,
                                                               int bits, unsigned *hist)
{
    d_sort_hist(keys, st, cap, shift, bits, hist);
}

__global__ void __launch_bounds__(1024) k_sort_scan_p(unsigned *hist, int grid, unsigned *totals)
{
    d_sort_scan(hist, grid, totals);
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter_p(const u64 *kin, const i64 *vin, u64 *kout, i64 *vout,
                                                                  const DevStep *st, i64 cap, int shift, int bits,
                                                                  const unsigned *hist, const unsigned *totals)
{
    d_sort_scatter(kin, vin, kout, vout, st, cap, shift, bits, hist, totals);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_count_p(const u64 *keys, const DevStep *st, i64 cap, i64 *outpop,
                                                               WorkArrays wa)
{
    d_seg_count(keys, st, cap, outpop, wa);
}

__global__ void __launch_bounds__(1024) k_part_scan_p(WorkArrays wa, int grid, int src, int dst, i64 *out)
{
    d_part_scan(wa, grid, src, dst, out);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_seg_write_p(const u64 *keys, const i64 *pops, const DevStep *st,
                                                               i64 cap, u64 *outkey, i64 *outpop, WorkArrays wa)
{
    d_seg_write(keys, pops, st, cap, outkey, outpop, wa);
}

// ---------------------------------------------------------------------------
// Launcher
// ---------------------------------------------------------------------------

int bits_for(u64 bound)
{
    int b = 1;
    while (b < 64 && (bound - 1) >> b) b++;
    return b;
}

int sort_passes(const Shapes &sh)
{
    return (sh.key_bits + sh.digit_bits - 1) / sh.digit_bits;
}

// instantiated in ccmc_step_k<K>.cu
#define CCMC_EXTERN_LAUNCH(K, R)                                                                              \
    extern template cudaError_t launch_phases<K, R>(const StepArgs *, int, const Shapes &, bool, cudaStream_t, \
                                                    i64 *, const cudaEvent_t *, const FlatPlan *)
CCMC_EXTERN_LAUNCH(1, double);
CCMC_EXTERN_LAUNCH(2, double);
CCMC_EXTERN_LAUNCH(3, double);
CCMC_EXTERN_LAUNCH(4, double);
CCMC_EXTERN_LAUNCH(5, double);
CCMC_EXTERN_LAUNCH(6, double);
CCMC_EXTERN_LAUNCH(1, float);
CCMC_EXTERN_LAUNCH(2, float);
CCMC_EXTERN_LAUNCH(3, float);

cudaError_t launch_group(const StepArgs *A, int nrep, int K, bool fp32, const Shapes &sh, bool multi_att,
                         cudaStream_t sm, i64 *launches, const cudaEvent_t *ev, const FlatPlan *plan)
{
    if (fp32) {   // the FP32 form: up to three words (M <= 192)
        switch (K) {
        case 1: return launch_phases<1, float>(A, nrep, sh, multi_att, sm, launches, ev, plan);
        case 2: return launch_phases<2, float>(A, nrep, sh, multi_att, sm, launches, ev, plan);
        case 3: return launch_phases<3, float>(A, nrep, sh, multi_att, sm, launches, ev, plan);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (K) {
    case 1: return launch_phases<1, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    case 2: return launch_phases<2, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    case 3: return launch_phases<3, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    case 4: return launch_phases<4, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    case 5: return launch_phases<5, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    case 6: return launch_phases<6, double>(A, nrep, sh, multi_att, sm, launches, ev, plan);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(StepCtx &c)
{
    cudaError_t e = launch_group(c.d_args, 1, c.K, c.fp32, c.sh, c.prm.fnc || c.prm.multispawn || c.prm.buffered, c.stream, c.launches,
                                 c.profile ? c.events : nullptr);
    c.sorted_buf = sort_passes(c.sh) & 1;
    c.cur ^= 1;
    return e;
}

}  // namespace ccmc

// ---------------------------------------------------------------------------
// Sort-and-reduce of spawned records without any allocation
//
// For callers that may not allocate device memory: plugins whose host
// application owns the device allocator, and loops that must keep a fixed
// device-memory footprint once set up.  The scratch lives in one file-scope
// device array that every GPU loading this library holds until the process
// exits; every call on a device shares it and leaves its contents behind
// (the counters the kernels rely on are reset by k_noalloc_begin and the
// output weights are zeroed before the per-run atomics).
// ---------------------------------------------------------------------------

namespace ccmc {
namespace {

constexpr size_t NOALLOC_MAX = (size_t)1 << 16;   // records per call
constexpr int NOALLOC_GRID = 64;                   // blocks of the sort and reduce kernels

struct NoAllocScratch {
    u64 key[2][NOALLOC_MAX];
    i64 pop[2][NOALLOC_MAX];
    unsigned hist[(1 << MAX_DIGIT_BITS) * NOALLOC_GRID];
    unsigned tot[1 << MAX_DIGIT_BITS];
    i64 part[8 * NOALLOC_GRID];
    DevStep st;
};

__device__ __align__(256) NoAllocScratch g_noalloc;

std::mutex g_noalloc_mutex;
NoAllocScratch *g_noalloc_ptr[256];

// Device address of the scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device address).
cudaError_t noalloc_scratch(NoAllocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (NoAllocScratch *)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

__global__ void k_noalloc_begin(DevStep *st, i64 n)
{
    if (threadIdx.x == 0) {
        st->n_sp = n;
        st->n_keys = 0;
        st->err = 0;
    }
}

}  // namespace

}  // namespace ccmc

extern "C" ccmc_status ccmc_reduce_records_noalloc(const uint64_t *keys_in, const int64_t *pops_in, size_t n,
                                                   int32_t key_bits, uint64_t *keys_out, int64_t *pops_out,
                                                   size_t *n_out, void *cuda_stream)
{
    using namespace ccmc;
    if (!n_out) return CCMC_ERR_ARG;
    *n_out = 0;
    if (n > NOALLOC_MAX || key_bits < 1 || key_bits > 64) return CCMC_ERR_ARG;
    if (n == 0) return CCMC_OK;
    if (!keys_in || !pops_in || !keys_out || !pops_out) return CCMC_ERR_ARG;
    cudaStream_t sm = (cudaStream_t)cuda_stream;
    NoAllocScratch *S = nullptr;
    if (noalloc_scratch(&S) != cudaSuccess) return CCMC_ERR_CUDA;
    const i64 cap = (i64)NOALLOC_MAX;
    k_noalloc_begin<<<1, 32, 0, sm>>>(&S->st, (i64)n);
    // LSD radix passes: the caller's input, then the two scratch buffers
    const u64 *kin = (const u64 *)keys_in;
    const i64 *vin = (const i64 *)pops_in;
    int dst = 0;
    for (int shift = 0; shift < key_bits; shift += MAX_DIGIT_BITS) {
        int bits = key_bits - shift < MAX_DIGIT_BITS ? key_bits - shift : MAX_DIGIT_BITS;
        k_sort_hist_p<<<NOALLOC_GRID, SORT_THREADS, 0, sm>>>(kin, &S->st, cap, shift, bits, S->hist);
        k_sort_scan_p<<<1 << bits, 1024, 0, sm>>>(S->hist, NOALLOC_GRID, S->tot);
        k_sort_scatter_p<<<NOALLOC_GRID, SORT_THREADS, 0, sm>>>(kin, vin, S->key[dst], S->pop[dst], &S->st, cap, shift,
                                                               bits, S->hist, S->tot);
        kin = S->key[dst];
        vin = S->pop[dst];
        dst ^= 1;
    }
    // one record per distinct key with the summed weight
    WorkArrays wa;
    memset(&wa, 0, sizeof(wa));
    wa.part = S->part;
    k_seg_count_p<<<NOALLOC_GRID, SCAN_THREADS, 0, sm>>>(kin, &S->st, cap, (i64 *)pops_out, wa);
    k_part_scan_p<<<1, 1024, 0, sm>>>(wa, NOALLOC_GRID, 0, 2, &S->st.n_keys);
    k_seg_write_p<<<NOALLOC_GRID, SCAN_THREADS, 0, sm>>>(kin, vin, &S->st, cap, (u64 *)keys_out, (i64 *)pops_out, wa);
    if (cudaGetLastError() != cudaSuccess) return CCMC_ERR_CUDA;
    i64 m = 0;
    if (cudaMemcpyAsync(&m, &S->st.n_keys, sizeof(i64), cudaMemcpyDeviceToHost, sm) != cudaSuccess) return CCMC_ERR_CUDA;
    if (cudaStreamSynchronize(sm) != cudaSuccess) return CCMC_ERR_CUDA;
    *n_out = (size_t)m;
    return CCMC_OK;
}
