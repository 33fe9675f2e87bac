// SCDM localisation support (Sec. 2): pivoted QR (Businger-Golub, modified
// Gram-Schmidt with exact column norms at every step) on the grid subsample,
// and the gathers that feed it and the U = phi_C^T (phi_C phi_C^T)^{-1/2}
// rotation computed by the caller.
#include <algorithm>

#include "grid_sync.cuh"
#include "lace_internal.cuh"

namespace lace {

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_MAXROWS = 1024;

struct Best {
    double v;
    int idx;
};

__device__ __forceinline__ bool better(double v, int i, double bv, int bi) { return v > bv || (v == bv && i < bi); }

// One column per thread: apply the previous reflection-free MGS step
// R[:,c] -= q (q . R[:,c]), then the exact squared norm of the column.
// Chosen columns report -1.  Per-block argmax (ties: lowest index).
template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_update_kernel(int nrow, int ncol, T* __restrict__ R, size_t ld,
                                                               const T* __restrict__ q, int has_q,
                                                               const unsigned char* __restrict__ chosen,
                                                               Best* __restrict__ block_best) {
    __shared__ T qs[QR_MAXROWS];
    __shared__ double bv[QR_THREADS];
    __shared__ int bi[QR_THREADS];
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) qs[r] = has_q ? q[r] : T(0);
    __syncthreads();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double best = -2.0;
    int bidx = 0x7fffffff;
    if (c < ncol) {
        T* col = R + c;
        if (has_q) {
            T dot = T(0);
            for (int r = 0; r < nrow; ++r) dot += qs[r] * col[(size_t)r * ld];
            T nrm = T(0);
            for (int r = 0; r < nrow; ++r) {
                T v = col[(size_t)r * ld] - qs[r] * dot;
                col[(size_t)r * ld] = v;
                nrm += v * v;
            }
            best = chosen[c] ? -1.0 : (double)nrm;
        } else {
            T nrm = T(0);
            for (int r = 0; r < nrow; ++r) {
                T v = col[(size_t)r * ld];
                nrm += v * v;
            }
            best = chosen[c] ? -1.0 : (double)nrm;
        }
        bidx = c;
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            if (better(bv[threadIdx.x + o], bi[threadIdx.x + o], bv[threadIdx.x], bi[threadIdx.x])) {
                bv[threadIdx.x] = bv[threadIdx.x + o];
                bi[threadIdx.x] = bi[threadIdx.x + o];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) block_best[blockIdx.x] = Best{bv[0], bi[0]};
}

// Pick the pivot among the block winners, mark it, form q = R[:,p]/||R[:,p]||.
template <typename T>
__global__ void __launch_bounds__(QR_THREADS) qr_select_kernel(int nrow, int nblocks, const T* __restrict__ R,
                                                               size_t ld, const Best* __restrict__ block_best,
                                                               unsigned char* __restrict__ chosen, T* __restrict__ q,
                                                               int* __restrict__ piv, int step) {
    __shared__ double bv[QR_THREADS];
    __shared__ int bi[QR_THREADS];
    __shared__ double nrm_sh[QR_THREADS];
    double best = -3.0;
    int bidx = 0x7fffffff;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const Best x = block_best[b];
        if (better(x.v, x.idx, best, bidx)) { best = x.v; bidx = x.idx; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o && better(bv[threadIdx.x + o], bi[threadIdx.x + o], bv[threadIdx.x], bi[threadIdx.x])) {
            bv[threadIdx.x] = bv[threadIdx.x + o];
            bi[threadIdx.x] = bi[threadIdx.x + o];
        }
        __syncthreads();
    }
    const int p = bi[0];
    double s = 0.0;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
        const double v = (double)R[(size_t)r * ld + p];
        s += v * v;
    }
    nrm_sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) nrm_sh[threadIdx.x] += nrm_sh[threadIdx.x + o];
        __syncthreads();
    }
    const double inv = nrm_sh[0] > 0.0 ? 1.0 / sqrt(nrm_sh[0]) : 0.0;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) q[r] = (T)((double)R[(size_t)r * ld + p] * inv);
    if (threadIdx.x == 0) {
        piv[step] = p;
        chosen[p] = 1;
    }
}

// Persistent pivoted QR: one cooperative launch runs every step.  One CTA
// of 512 threads (16 warps) per SM.  A group of WPT warps owns a 32-column
// tile (lane = column); warp g of the group holds rows g*RPW .. g*RPW+RPW-1
// of the tile in registers, so a step loads each element once, forms q.r
// (partial sums exchanged through shared memory behind a named barrier of
// the group), updates the registers, stores them and forms the exact new
// norm.  One grid-wide barrier per step; the block winners are
// double-buffered by step parity and a chosen column is never written
// again, so every CTA can read the pivot column while the next step runs.
constexpr int QC_THREADS = 512, QC_WARPS = 16, QC_MAXROWS = 1024;

__device__ __forceinline__ void best_merge(double& v, int& i, double v2, int i2) {
    if (better(v2, i2, v, i)) { v = v2; i = i2; }
}

template <typename T> struct Vec4 {
    T a, b, c, d;
};
// four consecutive shared-memory values as 16-byte loads (16-byte aligned p)
__device__ __forceinline__ Vec4<float> load4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Vec4<double> load4(const double* p) {
    const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
    return {v0.x, v0.y, v1.x, v1.y};
}

__device__ __forceinline__ void group_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename T, int RPW>
__global__ void __launch_bounds__(QC_THREADS) qr_persistent_kernel(int nrow, int ncol, T* __restrict__ R,
                                                                   int npiv, int wpt, Best* __restrict__ block_best,
                                                                   unsigned char* __restrict__ chosen,
                                                                   int* __restrict__ piv, unsigned* bar) {
    __shared__ __align__(16) T qs[QC_MAXROWS + RPW];
    __shared__ T part[QC_WARPS][32];
    __shared__ double gv[QC_WARPS];
    __shared__ int gi[QC_WARPS];
    __shared__ double red[QC_WARPS];
    __shared__ int pivot_sh;
    __shared__ int abort_sh;
    unsigned gen = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ngroups = QC_WARPS / wpt;
    const int group = warp / wpt, wig = warp % wpt;
    const int ntiles = (ncol + 31) / 32;
    const int ggroup = blockIdx.x * ngroups + group, total_groups = gridDim.x * ngroups;
    const int rbase = wig * RPW;
    for (int r = threadIdx.x; r < QC_MAXROWS + RPW; r += blockDim.x) qs[r] = T(0);
    __syncthreads();
    for (int step = 0; step < npiv; ++step) {
        double best = -2.0;
        int bidx = 0x7fffffff;
        if (group < ngroups) {
            for (int tile = ggroup; tile < ntiles; tile += total_groups) {
                const int c = tile * 32 + lane;
                const bool live = c < ncol && !chosen[c];
                T v[RPW];
                // all RPW rows of this warp exist: no per-row guard (the common case)
                const bool full = rbase + RPW <= nrow;
                if (full) {
#pragma unroll
                    for (int j = 0; j < RPW; ++j) v[j] = live ? R[(size_t)(rbase + j) * ncol + c] : T(0);
                } else {
#pragma unroll
                    for (int j = 0; j < RPW; ++j)
                        v[j] = (live && rbase + j < nrow) ? R[(size_t)(rbase + j) * ncol + c] : T(0);
                }
                if (step > 0) {
                    T pd = T(0);
#pragma unroll
                    for (int j = 0; j < RPW; j += 4) {
                        const Vec4<T> q4 = load4(qs + rbase + j);
                        pd += q4.a * v[j] + q4.b * v[j + 1] + q4.c * v[j + 2] + q4.d * v[j + 3];
                    }
                    part[warp][lane] = pd;
                    group_bar(1 + group, wpt * 32);
                    T dot = T(0);
                    for (int w = 0; w < wpt; ++w) dot += part[group * wpt + w][lane];
                    group_bar(1 + group, wpt * 32);
#pragma unroll
                    for (int j = 0; j < RPW; j += 4) {
                        const Vec4<T> q4 = load4(qs + rbase + j);
                        v[j] -= q4.a * dot;
                        v[j + 1] -= q4.b * dot;
                        v[j + 2] -= q4.c * dot;
                        v[j + 3] -= q4.d * dot;
                    }
                    if (live) {
                        if (full) {
#pragma unroll
                            for (int j = 0; j < RPW; ++j) R[(size_t)(rbase + j) * ncol + c] = v[j];
                        } else {
#pragma unroll
                            for (int j = 0; j < RPW; ++j)
                                if (rbase + j < nrow) R[(size_t)(rbase + j) * ncol + c] = v[j];
                        }
                    }
                }
                T pn = T(0);
#pragma unroll
                for (int j = 0; j < RPW; ++j) pn += v[j] * v[j];
                part[warp][lane] = pn;
                group_bar(1 + group, wpt * 32);
                if (wig == 0) {
                    T tot = T(0);
                    for (int w = 0; w < wpt; ++w) tot += part[group * wpt + w][lane];
                    double cv = live ? (double)tot : (c < ncol ? -1.0 : -2.0);
                    int ci = c < ncol ? c : 0x7fffffff;
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ov = __shfl_xor_sync(0xffffffffu, cv, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
                        best_merge(cv, ci, ov, oi);
                    }
                    best_merge(best, bidx, cv, ci);
                }
                group_bar(1 + group, wpt * 32);
            }
        }
        if (lane == 0 && wig == 0 && group < ngroups) { gv[group] = best; gi[group] = bidx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = gv[0];
            int bi_ = gi[0];
            for (int w = 1; w < ngroups; ++w) best_merge(b, bi_, gv[w], gi[w]);
            block_best[(step & 1) * gridDim.x + blockIdx.x] = Best{b, bi_};
        }
        if (!grid_barrier(bar, gen, &abort_sh)) return;
        // every CTA: global argmax, then q = R[:,p] / ||R[:,p]|| into shared memory
        if (warp == 0) {
            double gb = -3.0;
            int gbi = 0x7fffffff;
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const Best x = block_best[(step & 1) * gridDim.x + b];
                best_merge(gb, gbi, x.v, x.idx);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, gb, o);
                const int oi = __shfl_xor_sync(0xffffffffu, gbi, o);
                best_merge(gb, gbi, ov, oi);
            }
            if (lane == 0) pivot_sh = gbi;
        }
        __syncthreads();
        const int p = pivot_sh;
        const T xr = threadIdx.x < nrow ? R[(size_t)threadIdx.x * ncol + p] : T(0);
        const int r2 = threadIdx.x + QC_THREADS;
        const T xr2 = r2 < nrow ? R[(size_t)r2 * ncol + p] : T(0);
        double s2 = (double)xr * (double)xr + (double)xr2 * (double)xr2;
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) red[warp] = s2;
        __syncthreads();
        if (warp == 0) {
            double t = lane < QC_WARPS ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[0] = t;
        }
        __syncthreads();
        const double inv = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
        if (threadIdx.x < nrow) qs[threadIdx.x] = (T)((double)xr * inv);
        if (r2 < nrow) qs[r2] = (T)((double)xr2 * inv);
        if (threadIdx.x == 0) {
            chosen[p] = 1;
            if (blockIdx.x == 0) piv[step] = p;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void gather_subsample_kernel(int n1, int n2, int n3, int stride, int m1, int m2, int m3,
                                        const T* __restrict__ psi, size_t ng, T* __restrict__ out, size_t ncol) {
    const int o = blockIdx.y;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(c % m3);
        const int j = (int)((c / m3) % m2);
        const int i = (int)(c / ((size_t)m3 * m2));
        const size_t full = ((size_t)(i * stride) * n2 + (size_t)(j * stride)) * n3 + (size_t)(k * stride);
        out[(size_t)o * ncol + c] = psi[(size_t)o * ng + full];
    }
    (void)n1;
    (void)m1;
}

template <typename T>
__global__ void gather_columns_kernel(const T* __restrict__ psi, size_t ldpsi, int norb,
                                      const long long* __restrict__ idx, int npts, double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npts * norb) return;
    const int p = e / norb, o = e % norb;
    out[e] = (double)psi[(size_t)o * ldpsi + (size_t)idx[p]];
}

}  // namespace

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Capacity (in Best entries) of the block-winner buffer of qrcp_aux_bytes.
static int nblocks_cap(int ncol) { return std::max((ncol + QR_THREADS - 1) / QR_THREADS, 2 * 152 * 8); }

size_t qrcp_aux_bytes(int nrow, int ncol) {
    const int nblocks = nblocks_cap(ncol);
    return align256(sizeof(Best) * nblocks) + align256((size_t)ncol) + align256(sizeof(double) * nrow) + 256;
}

// R (nrow x ncol, row-major, leading dimension ncol) is overwritten.  aux is
// caller-provided scratch of qrcp_aux_bytes(nrow, ncol) bytes.
template <typename T>
cudaError_t qrcp_pivots(int nrow, int ncol, T* R, int npiv, int* d_piv, void* aux, int* h_timeout, cudaStream_t s,
                        int* launches) {
    *h_timeout = 0;
    if (nrow > QR_MAXROWS || npiv > ncol) return cudaErrorInvalidValue;
    const int nblocks = (ncol + QR_THREADS - 1) / QR_THREADS;
    unsigned char* base = static_cast<unsigned char*>(aux);
    Best* best = reinterpret_cast<Best*>(base);
    unsigned char* chosen = base + align256(sizeof(Best) * nblocks_cap(ncol));
    T* q = reinterpret_cast<T*>(chosen + align256((size_t)ncol));
    unsigned* bar = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(q) + align256(sizeof(double) * nrow));
    cudaMemsetAsync(chosen, 0, ncol, s);
    // persistent cooperative version when the rows fit the per-thread registers
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    constexpr int RPW = sizeof(T) == 4 ? 64 : 32;  // rows per warp held in registers
    int wpt = 2;  // >= 2 keeps the named-barrier ids (1 + group) within 1..8
    while (wpt * RPW < nrow) wpt *= 2;
    const void* fn = (const void*)qr_persistent_kernel<T, RPW>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_persistent_kernel<T, RPW>, QC_THREADS, 0);
    const int gridn = sms * std::min(per_sm, 1);
    if (coop && per_sm > 0 && wpt <= QC_WARPS && nrow <= QC_MAXROWS && 2 * gridn <= nblocks_cap(ncol)) {
        Best* bb = best;
        cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s);
        if (e) return e;
        void* args[] = {(void*)&nrow, (void*)&ncol, (void*)&R, (void*)&npiv, (void*)&wpt, (void*)&bb,
                        (void*)&chosen, (void*)&d_piv, (void*)&bar};
        e = cudaLaunchCooperativeKernel(fn, dim3(gridn), dim3(QC_THREADS), args, 0, s);
        *launches += 1;
        if (e) return e;
        unsigned flag = 0;
        if ((e = cudaMemcpyAsync(&flag, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s))) return e;
        if ((e = cudaStreamSynchronize(s))) return e;
        *h_timeout = flag != 0u;
        return cudaSuccess;
    }
    for (int step = 0; step < npiv; ++step) {
        qr_update_kernel<T><<<nblocks, QR_THREADS, 0, s>>>(nrow, ncol, R, (size_t)ncol, q, step > 0, chosen, best);
        qr_select_kernel<T><<<1, QR_THREADS, 0, s>>>(nrow, nblocks, R, (size_t)ncol, best, chosen, q, d_piv, step);
        *launches += 2;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_subsample(const GridGeom& g, int stride, const T* psi, int norb, T* out, int* ncol_out,
                             cudaStream_t s, int* launches) {
    const int m1 = (g.n[0] + stride - 1) / stride, m2 = (g.n[1] + stride - 1) / stride,
              m3 = (g.n[2] + stride - 1) / stride;
    const size_t ncol = (size_t)m1 * m2 * m3;
    *ncol_out = (int)ncol;
    dim3 grid((unsigned)std::min<size_t>((ncol + 255) / 256, 1024), norb);
    gather_subsample_kernel<T><<<grid, 256, 0, s>>>(g.n[0], g.n[1], g.n[2], stride, m1, m2, m3, psi, g.ng, out, ncol);
    *launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_columns(const T* psi, size_t ldpsi, int norb, const long long* d_full_idx, int npts, double* out,
                           cudaStream_t s, int* launches) {
    const int tot = npts * norb;
    gather_columns_kernel<T><<<(tot + 255) / 256, 256, 0, s>>>(psi, ldpsi, norb, d_full_idx, npts, out);
    *launches += 1;
    return cudaGetLastError();
}

template cudaError_t qrcp_pivots<float>(int, int, float*, int, int*, void*, int*, cudaStream_t, int*);
template cudaError_t qrcp_pivots<double>(int, int, double*, int, int*, void*, int*, cudaStream_t, int*);
template cudaError_t gather_subsample<float>(const GridGeom&, int, const float*, int, float*, int*, cudaStream_t, int*);
template cudaError_t gather_subsample<double>(const GridGeom&, int, const double*, int, double*, int*, cudaStream_t,
                                              int*);
template cudaError_t gather_columns<float>(const float*, size_t, int, const long long*, int, double*, cudaStream_t,
                                           int*);
template cudaError_t gather_columns<double>(const double*, size_t, int, const long long*, int, double*, cudaStream_t,
                                            int*);

}  // namespace lace
