// ccmc_dist.cu -- co-location statistics of the paper's distribution of
// excitors over processors (Sec. III, Eq. ccmc_dist, Fig. excitdistrib),
// simulated on one GPU: the owner of every excitor at every iteration, then,
// for every pair of excitors, the number of iterations they shared a
// processor, summed (with its square) over pairs at each checkpoint.
#include <vector>

#include "../../include/ccmc.h"
#include "ccmc_device.cuh"

namespace ccmc {
namespace {

constexpr int PAIR_TILE = 32;       // excitors per side of a pair tile
constexpr int MAX_CHECKPOINTS = 64;

// own[t * n + i] = owner of excitor i at iteration t
__global__ void k_owners(const u64 *dets, i64 n, int nw, i64 t_max, int nu_move, u64 n_ranks, unsigned short *own)
{
    const i64 total = n * t_max;
    for (i64 q = (i64)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (i64)gridDim.x * blockDim.x) {
        const i64 t = q / n, i = q - t * n;
        own[q] = (unsigned short)words_owner(dets + i * nw, nw, (u64)t, nu_move, n_ranks);
    }
}

// One 32 x 32 tile of pairs (i in the row tile, j in the column tile, j > i)
// per block of 32 x 8 threads; each thread walks 4 pairs of its row through
// the iterations, staging 32 iterations of owners of both tiles in shared
// memory, and adds C and C^2 of its pairs at each checkpoint.
__global__ void __launch_bounds__(256) k_pairs(const unsigned short *own, i64 n, i64 t_max, const i64 *ck, int nck,
                                               u64 *sum_c, u64 *sum_c2)
{
    const i64 bi = blockIdx.y, bj = blockIdx.x;
    if (bj < bi) return;
    __shared__ unsigned short si[32][PAIR_TILE + 1], sj[32][PAIR_TILE + 1];
    __shared__ i64 sck[MAX_CHECKPOINTS];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // column lane, row group
    if (threadIdx.x < nck) sck[threadIdx.x] = ck[threadIdx.x];
    const i64 j = bj * PAIR_TILE + tx;
    unsigned c[4] = {0, 0, 0, 0};
    int k = 0;
    for (i64 t0 = 0; t0 < t_max; t0 += 32) {
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const i64 t = t0 + r;
            const i64 ii = bi * PAIR_TILE + tx, jj = bj * PAIR_TILE + tx;
            si[r][tx] = (t < t_max && ii < n) ? own[t * n + ii] : 0;
            sj[r][tx] = (t < t_max && jj < n) ? own[t * n + jj] : 0;
        }
        __syncthreads();
        const int tn = t_max - t0 < 32 ? (int)(t_max - t0) : 32;
        for (int r = 0; r < tn; r++) {
            const unsigned short oj = sj[r][tx];
#pragma unroll
            for (int a = 0; a < 4; a++) c[a] += si[r][ty * 4 + a] == oj ? 1u : 0u;
            // checkpoint after iteration t0 + r (i.e. T = t0 + r + 1)
            while (k < nck && sck[k] == t0 + r + 1) {
                u64 s1 = 0, s2 = 0;
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const i64 i = bi * PAIR_TILE + ty * 4 + a;
                    if (i < n && j < n && j > i) {
                        s1 += c[a];
                        s2 += (u64)c[a] * c[a];
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
                    s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
                }
                if (tx == 0) {
                    atomicAdd((unsigned long long *)&sum_c[k], (unsigned long long)s1);
                    atomicAdd((unsigned long long *)&sum_c2[k], (unsigned long long)s2);
                }
                k++;
            }
        }
    }
}

}  // namespace
}  // namespace ccmc

extern "C" ccmc_status ccmc_colocation(const uint64_t *dets, size_t n, int32_t n_words, int64_t n_ranks,
                                       int32_t nu_move, const int64_t *checkpoints, int32_t n_checkpoints,
                                       uint64_t *sum_c, uint64_t *sum_c2, void *cuda_stream)
{
    using namespace ccmc;
    if (!dets || !checkpoints || !sum_c || !sum_c2 || n < 2 || n > ((size_t)1 << 20) || n_words < 1 ||
        n_words > MAXK || n_ranks < 1 || n_ranks > 65535 || nu_move < 0 || n_checkpoints < 1 ||
        n_checkpoints > MAX_CHECKPOINTS)
        return CCMC_ERR_ARG;
    for (int k = 0; k < n_checkpoints; k++)
        if (checkpoints[k] < 1 || (k > 0 && checkpoints[k] <= checkpoints[k - 1])) return CCMC_ERR_ARG;
    const i64 t_max = checkpoints[n_checkpoints - 1];
    if (t_max > ((i64)1 << 20)) return CCMC_ERR_ARG;
    cudaStream_t sm = (cudaStream_t)cuda_stream;
    u64 *d_dets = nullptr, *d_s1 = nullptr, *d_s2 = nullptr;
    i64 *d_ck = nullptr;
    unsigned short *d_own = nullptr;
    ccmc_status st = CCMC_OK;
    const size_t nn = n, nw = (size_t)n_words, nck = (size_t)n_checkpoints;
    if (cudaMalloc(&d_dets, nn * nw * 8) != cudaSuccess || cudaMalloc(&d_s1, nck * 8) != cudaSuccess ||
        cudaMalloc(&d_s2, nck * 8) != cudaSuccess || cudaMalloc(&d_ck, nck * 8) != cudaSuccess ||
        cudaMalloc(&d_own, nn * (size_t)t_max * 2) != cudaSuccess) {
        st = CCMC_ERR_OOM;
    } else if (cudaMemcpyAsync(d_dets, dets, nn * nw * 8, cudaMemcpyHostToDevice, sm) != cudaSuccess ||
               cudaMemcpyAsync(d_ck, checkpoints, nck * 8, cudaMemcpyHostToDevice, sm) != cudaSuccess ||
               cudaMemsetAsync(d_s1, 0, nck * 8, sm) != cudaSuccess ||
               cudaMemsetAsync(d_s2, 0, nck * 8, sm) != cudaSuccess) {
        st = CCMC_ERR_CUDA;
    } else {
        k_owners<<<1024, 256, 0, sm>>>(d_dets, (i64)n, n_words, t_max, nu_move, (u64)n_ranks, d_own);
        const unsigned tiles = (unsigned)((n + PAIR_TILE - 1) / PAIR_TILE);
        k_pairs<<<dim3(tiles, tiles), 256, 0, sm>>>(d_own, (i64)n, t_max, d_ck, n_checkpoints, d_s1, d_s2);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(sum_c, d_s1, nck * 8, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
            cudaMemcpyAsync(sum_c2, d_s2, nck * 8, cudaMemcpyDeviceToHost, sm) != cudaSuccess ||
            cudaStreamSynchronize(sm) != cudaSuccess)
            st = CCMC_ERR_CUDA;
    }
    cudaFree(d_dets);
    cudaFree(d_s1);
    cudaFree(d_s2);
    cudaFree(d_ck);
    cudaFree(d_own);
    return st;
}
