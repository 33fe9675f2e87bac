// Pair screening by the overlap of moduli (Eq. 4) and the kept pair list
// of the truncated potential (Eq. 5): an occupied pair (i, k) is dropped
// when S_ik < S_thr, which removes both u^(ik) and u^(ki); pairs with an
// extra (virtual) orbital are always kept (Sec. 4.1).  Also the exchange
// energy sum over the pair-energy matrix.
#include <algorithm>

#include "lace_internal.cuh"

namespace lace {

namespace {

constexpr int SC_THREADS = 256;

// counts[i] = number of kept j in [i, n_occ) plus n_extra.
__global__ void count_kernel(int n_occ, int n_extra, const double* __restrict__ S, double thr, int use_S,
                             int* __restrict__ counts) {
    const int i = blockIdx.x;
    __shared__ int sh[SC_THREADS];
    int c = 0;
    for (int j = i + threadIdx.x; j < n_occ; j += blockDim.x)
        c += (!use_S || S[(size_t)i * n_occ + j] >= thr) ? 1 : 0;
    sh[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[i] = sh[0] + n_extra;
}

// Exclusive scan of counts[0..n) into offs[0..n], offs[n] = total (one block).
__global__ void scan_kernel(int n, const int* __restrict__ counts, int* __restrict__ offs) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < n; ++i) {
            offs[i] = acc;
            acc += counts[i];
        }
        offs[n] = acc;
    }
}

// Row i writes its kept (i, j), j ascending, then (i, n_occ + e).
__global__ void write_pairs_kernel(int n_occ, int n_extra, const double* __restrict__ S, double thr, int use_S,
                                   const int* __restrict__ offs, int2* __restrict__ pairs) {
    const int i = blockIdx.x;
    __shared__ int base;
    __shared__ int warp_tot[SC_THREADS / 32];
    if (threadIdx.x == 0) base = offs[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j0 = i; j0 < n_occ; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool keep = j < n_occ && (!use_S || S[(size_t)i * n_occ + j] >= thr);
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        const int rank = __popc(ballot & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(ballot);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += warp_tot[w];
        if (keep) pairs[base + before + rank] = make_int2(i, j);
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_tot[w];
            base += t;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n_extra; e += blockDim.x) pairs[base + e] = make_int2(i, n_occ + e);
}

__global__ void pack_kernel(const int2* __restrict__ pairs, long long n_pairs, PairGrid* __restrict__ grids,
                            long long n_grids) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_grids) return;
    const int2 a = pairs[2 * g];
    PairGrid d;
    d.i1 = a.x;
    d.j1 = a.y;
    if (2 * g + 1 < n_pairs) {
        const int2 b = pairs[2 * g + 1];
        d.i2 = b.x;
        d.j2 = b.y;
    } else {
        d.i2 = a.x;
        d.j2 = -1;
    }
    grids[g] = d;
}

// Fixed-order FP64 sums over many blocks (FP64 issues slowly: a one-block
// sum of 65,536 values took ~120 us).  Block b sums the contiguous range b
// of m values (x, or x^2 with SQUARE) into part[b]; a second one-block
// kernel adds the partials in order and scales them.
template <bool SQUARE>
__global__ void partial_sum_kernel(size_t m, size_t chunk, const double* __restrict__ x, double* __restrict__ part) {
    __shared__ double sh[SC_THREADS];
    const size_t lo = (size_t)blockIdx.x * chunk, hi = lo + chunk < m ? lo + chunk : m;
    double s0 = 0.0, s1 = 0.0;
    size_t i = lo + threadIdx.x;
    for (; i + SC_THREADS < hi; i += 2 * SC_THREADS) {
        const double a = x[i], b = x[i + SC_THREADS];
        s0 += SQUARE ? a * a : a;
        s1 += SQUARE ? b * b : b;
    }
    if (i < hi) s0 += SQUARE ? x[i] * x[i] : x[i];
    sh[threadIdx.x] = s0 + s1;
    __syncthreads();
    for (int o = SC_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void finish_sum_kernel(int nb, const double* __restrict__ part, double scale, double* __restrict__ out) {
    __shared__ double sh[SC_THREADS];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += SC_THREADS) s += part[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = SC_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale * sh[0];
}

cudaError_t fixed_sum(size_t m, const double* d_x, bool square, double scale, double* d_part, double* d_out,
                      cudaStream_t s, int* launches) {
    const int nb = (int)std::max<size_t>(1, std::min<size_t>(kSumBlocks, (m + 2047) / 2048));
    const size_t chunk = (m + nb - 1) / nb;
    if (square) partial_sum_kernel<true><<<nb, SC_THREADS, 0, s>>>(m, chunk, d_x, d_part);
    else partial_sum_kernel<false><<<nb, SC_THREADS, 0, s>>>(m, chunk, d_x, d_part);
    finish_sum_kernel<<<1, SC_THREADS, 0, s>>>(nb, d_part, scale, d_out);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace

cudaError_t neg_sum_squares(size_t m, const double* d_X, double* d_part, double* d_out, cudaStream_t s,
                            int* launches) {
    return fixed_sum(m, d_X, true, -1.0, d_part, d_out, s, launches);
}

cudaError_t build_pair_list(int n_occ, int n_extra, const double* d_S, double thr, bool use_S, int2* d_pairs,
                            int* d_counts, long long* n_pairs, cudaStream_t s, int* launches) {
    int* offs = d_counts + n_occ;  // caller provides 2*n_occ + 1 ints
    count_kernel<<<n_occ, SC_THREADS, 0, s>>>(n_occ, n_extra, d_S, thr, use_S ? 1 : 0, d_counts);
    scan_kernel<<<1, 32, 0, s>>>(n_occ, d_counts, offs);
    write_pairs_kernel<<<n_occ, SC_THREADS, 0, s>>>(n_occ, n_extra, d_S, thr, use_S ? 1 : 0, offs, d_pairs);
    *launches += 3;
    int total = 0;
    cudaMemcpyAsync(&total, offs + n_occ, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    *n_pairs = total;
    return e;
}

cudaError_t pack_pair_grids(const int2* d_pairs, long long n_pairs, PairGrid* d_grids, cudaStream_t s,
                            int* launches) {
    const long long n_grids = (n_pairs + 1) / 2;
    if (n_grids == 0) return cudaSuccess;
    pack_kernel<<<(unsigned)((n_grids + 255) / 256), 256, 0, s>>>(d_pairs, n_pairs, d_grids, n_grids);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t exchange_energy_sum(int n_occ, const double* d_E, double* d_part, double* d_ex, cudaStream_t s,
                                int* launches) {
    return fixed_sum((size_t)n_occ * n_occ, d_E, false, -0.5, d_part, d_ex, s, launches);
}

}  // namespace lace
