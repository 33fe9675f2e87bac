// SCDM localisation support (Sec. 2): pivoted QR (Businger-Golub, modified
// Gram-Schmidt with exact column norms at every step) on the grid subsample,
// and the gathers that feed it and the U = phi_C^T (phi_C phi_C^T)^{-1/2}
// rotation computed by the caller.
#include <algorithm>

#include "f32x2.cuh"
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

// Persistent pivoted QR: one cooperative launch runs every step, one CTA of
// 512 threads (16 warps) per SM.  A group of wpt warps owns 32-column tiles
// (lane = column); warp w of the group holds rows w*RPW .. w*RPW+RPW-1 of a
// tile.  The matrix stays on chip across the steps where it fits: the first
// NREG tiles of a group live in registers, the next nsm tiles in shared
// memory, and only the rest is streamed from and back to global memory
// every step.  A step forms q.r (partial sums exchanged through shared
// memory behind the group's named barrier), updates the column, forms its
// exact new norm and the group's argmax; each CTA then publishes its best
// column's values, so one grid-wide barrier per step suffices: after it,
// every CTA picks the global winner and reads the winner's published column
// as the next q.  Block winners and published columns are double-buffered by
// step parity.
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

// q . v over this warp's RPW rows, four independent partial sums
template <typename T, int RPW>
__device__ __forceinline__ T dot_rows(const T* v, const T* qs, int rbase) {
    T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
#pragma unroll
    for (int j = 0; j < RPW; j += 4) {
        const Vec4<T> q4 = load4(qs + rbase + j);
        p0 += q4.a * v[j];
        p1 += q4.b * v[j + 1];
        p2 += q4.c * v[j + 2];
        p3 += q4.d * v[j + 3];
    }
    return (p0 + p1) + (p2 + p3);
}

// v -= q dot over the warp's rows, and the new squared norm of v
template <typename T, int RPW>
__device__ __forceinline__ T update_rows(T* v, const T* qs, int rbase, T dot) {
    T n0 = T(0), n1 = T(0), n2 = T(0), n3 = T(0);
#pragma unroll
    for (int j = 0; j < RPW; j += 4) {
        const Vec4<T> q4 = load4(qs + rbase + j);
        v[j] -= q4.a * dot;
        v[j + 1] -= q4.b * dot;
        v[j + 2] -= q4.c * dot;
        v[j + 3] -= q4.d * dot;
        n0 += v[j] * v[j];
        n1 += v[j + 1] * v[j + 1];
        n2 += v[j + 2] * v[j + 2];
        n3 += v[j + 3] * v[j + 3];
    }
    return (n0 + n1) + (n2 + n3);
}

template <typename T, int RPW>
__device__ __forceinline__ T norm_rows(const T* v) {
    T n0 = T(0), n1 = T(0), n2 = T(0), n3 = T(0);
#pragma unroll
    for (int j = 0; j < RPW; j += 4) {
        n0 += v[j] * v[j];
        n1 += v[j + 1] * v[j + 1];
        n2 += v[j + 2] * v[j + 2];
        n3 += v[j + 3] * v[j + 3];
    }
    return (n0 + n1) + (n2 + n3);
}

// Warp argmax of the 32 columns of a tile (lane = column), merged into (best, bidx).
__device__ __forceinline__ void tile_argmax(double cv, int ci, double& best, int& bidx) {
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, cv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
        best_merge(cv, ci, ov, oi);
    }
    best_merge(best, bidx, cv, ci);
}

template <typename T, int RPW, int NREG>
__global__ void __launch_bounds__(QC_THREADS, 1)
    qr_persistent_kernel(int nrow, int ncol, T* __restrict__ R, int npiv, int wpt, int nsm,
                         Best* __restrict__ block_best, T* __restrict__ pub, unsigned char* __restrict__ chosen,
                         int* __restrict__ piv, unsigned* bar, unsigned long long limit_ns) {
    extern __shared__ __align__(16) unsigned char qr_smem_raw[];
    const int ngroups = QC_WARPS / wpt;
    const int kres_max = NREG + nsm;                 // resident tiles per group at most
    T* stiles = reinterpret_cast<T*>(qr_smem_raw);  // [ngroups][nsm][wpt][RPW][32]
    T* pdot = stiles + (size_t)ngroups * nsm * wpt * RPW * 32;  // [kres_max][QC_WARPS][32]
    T* pnrm = pdot + (size_t)kres_max * QC_WARPS * 32;            // [kres_max][QC_WARPS][32]
    __shared__ __align__(16) T qs[QC_MAXROWS + RPW];
    __shared__ T part[QC_WARPS * 32];
    __shared__ double gv[QC_WARPS];
    __shared__ int gi[QC_WARPS];
    __shared__ int wsel[QC_WARPS];
    __shared__ double red[QC_WARPS];
    __shared__ int pivot_sh, winner_sh, mybest_sh;
    __shared__ int abort_sh;
    unsigned gen = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int group = warp / wpt, wig = warp % wpt;
    const int ntiles = (ncol + 31) / 32;
    const int ggroup = blockIdx.x * ngroups + group, total_groups = gridDim.x * ngroups;
    const int ktot = ggroup < ntiles ? (ntiles - ggroup + total_groups - 1) / total_groups : 0;
    const int kres = min(ktot, kres_max);  // this group's resident tiles
    const int rbase = wig * RPW;
    const int rows_pad = wpt * RPW;
    T vr[NREG > 0 ? NREG : 1][RPW];
    // chosen columns among this lane's resident tiles (bit k: resident tile k),
    // kept in a register so that a step reads no global flag for them
    unsigned cmask = 0u;
    for (int r = threadIdx.x; r < QC_MAXROWS + RPW; r += blockDim.x) qs[r] = T(0);
    __syncthreads();
    for (int step = 0; step < npiv; ++step) {
        double best = -2.0;
        int bidx = 0x7fffffff;
        // resident tiles: all dot partials, one barrier, all updates and norm
        // partials, one barrier, then the argmax over the tiles
        if (step == 0) {
#pragma unroll
            for (int k = 0; k < NREG; ++k) {
                if (k < kres) {
                    const int c = (ggroup + k * total_groups) * 32 + lane;
#pragma unroll
                    for (int j = 0; j < RPW; ++j)
                        vr[k][j] = (c < ncol && rbase + j < nrow) ? R[(size_t)(rbase + j) * ncol + c] : T(0);
                    pnrm[(k * QC_WARPS + warp) * 32 + lane] = norm_rows<T, RPW>(vr[k]);
                }
            }
            for (int k = NREG; k < kres; ++k) {
                const int c = (ggroup + k * total_groups) * 32 + lane;
                T* st = stiles + ((((size_t)group * nsm + (k - NREG)) * wpt + wig) * RPW) * 32 + lane;
                T v[RPW];
#pragma unroll
                for (int j = 0; j < RPW; ++j) {
                    v[j] = (c < ncol && rbase + j < nrow) ? R[(size_t)(rbase + j) * ncol + c] : T(0);
                    st[j * 32] = v[j];
                }
                pnrm[(k * QC_WARPS + warp) * 32 + lane] = norm_rows<T, RPW>(v);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NREG; ++k)
                if (k < kres) pdot[(k * QC_WARPS + warp) * 32 + lane] = dot_rows<T, RPW>(vr[k], qs, rbase);
            for (int k = NREG; k < kres; ++k) {
                const T* st = stiles + ((((size_t)group * nsm + (k - NREG)) * wpt + wig) * RPW) * 32 + lane;
                T v[RPW];
#pragma unroll
                for (int j = 0; j < RPW; ++j) v[j] = st[j * 32];
                pdot[(k * QC_WARPS + warp) * 32 + lane] = dot_rows<T, RPW>(v, qs, rbase);
            }
            if (kres > 0) group_bar(1 + group, wpt * 32);
#pragma unroll
            for (int k = 0; k < NREG; ++k) {
                if (k < kres) {
                    T dot = T(0);
                    for (int w = 0; w < wpt; ++w) dot += pdot[(k * QC_WARPS + group * wpt + w) * 32 + lane];
                    pnrm[(k * QC_WARPS + warp) * 32 + lane] = update_rows<T, RPW>(vr[k], qs, rbase, dot);
                }
            }
            for (int k = NREG; k < kres; ++k) {
                T* st = stiles + ((((size_t)group * nsm + (k - NREG)) * wpt + wig) * RPW) * 32 + lane;
                T dot = T(0);
                for (int w = 0; w < wpt; ++w) dot += pdot[(k * QC_WARPS + group * wpt + w) * 32 + lane];
                T v[RPW];
#pragma unroll
                for (int j = 0; j < RPW; ++j) v[j] = st[j * 32];
                pnrm[(k * QC_WARPS + warp) * 32 + lane] = update_rows<T, RPW>(v, qs, rbase, dot);
#pragma unroll
                for (int j = 0; j < RPW; ++j) st[j * 32] = v[j];
            }
        }
        if (kres > 0) group_bar(1 + group, wpt * 32);
        if (wig == 0) {
            for (int k = 0; k < kres; ++k) {
                T tot = T(0);
                for (int w = 0; w < wpt; ++w) tot += pnrm[(k * QC_WARPS + group * wpt + w) * 32 + lane];
                const int c = (ggroup + k * total_groups) * 32 + lane;
                const bool live = c < ncol && !((cmask >> k) & 1u);
                tile_argmax(live ? (double)tot : (c < ncol ? -1.0 : -2.0), c < ncol ? c : 0x7fffffff, best, bidx);
            }
        }
        // the rest: streamed from and back to global memory, one tile at a time
        for (int tile = ggroup + kres_max * total_groups; tile < ntiles; tile += total_groups) {
            const int c = tile * 32 + lane;
            const bool live = c < ncol && !chosen[c];
            T v[RPW];
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
                part[warp * 32 + lane] = dot_rows<T, RPW>(v, qs, rbase);
                group_bar(1 + group, wpt * 32);
                T dot = T(0);
                for (int w = 0; w < wpt; ++w) dot += part[(group * wpt + w) * 32 + lane];
                group_bar(1 + group, wpt * 32);
                part[warp * 32 + lane] = update_rows<T, RPW>(v, qs, rbase, dot);
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
            } else {
                part[warp * 32 + lane] = norm_rows<T, RPW>(v);
            }
            group_bar(1 + group, wpt * 32);
            if (wig == 0) {
                T tot = T(0);
                for (int w = 0; w < wpt; ++w) tot += part[(group * wpt + w) * 32 + lane];
                tile_argmax(live ? (double)tot : (c < ncol ? -1.0 : -2.0), c < ncol ? c : 0x7fffffff, best, bidx);
            }
            group_bar(1 + group, wpt * 32);
        }
        if (lane == 0 && wig == 0) { gv[group] = best; gi[group] = bidx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = gv[0];
            int bi_ = gi[0];
            for (int w = 1; w < ngroups; ++w) best_merge(b, bi_, gv[w], gi[w]);
            block_best[(step & 1) * gridDim.x + blockIdx.x] = Best{b, bi_};
            mybest_sh = (b >= 0.0 && bi_ < ncol) ? bi_ : -1;
        }
        __syncthreads();
        // publish this CTA's candidate column (its current residual values) and,
        // in slot rows_pad, the inverse of its FP64 norm
        {
            T* out = pub + ((size_t)(step & 1) * gridDim.x + blockIdx.x) * (rows_pad + 4);
            const int cb = mybest_sh;
            if (cb >= 0) {
                const int tile = cb / 32, cl = cb % 32;
                const int kk = tile / total_groups, gg = tile % total_groups - blockIdx.x * ngroups;
                T x = T(0);
                if (kk < NREG) {
                    // the lane holding the column, in each warp of its group
                    if (group == gg && lane == cl) {
#pragma unroll
                        for (int k = 0; k < NREG; ++k)
                            if (k == kk) {
#pragma unroll
                                for (int j = 0; j < RPW; ++j) out[rbase + j] = vr[k][j];
                            }
                    }
                    __syncthreads();
                    if (threadIdx.x < rows_pad) x = out[threadIdx.x];
                } else if (kk < kres_max) {
                    const T* st = stiles + (((size_t)gg * nsm + (kk - NREG)) * wpt) * RPW * 32 + cl;
                    if (threadIdx.x < rows_pad) {
                        x = st[(size_t)threadIdx.x * 32];
                        out[threadIdx.x] = x;
                    }
                } else {
                    if (threadIdx.x < rows_pad) {
                        x = threadIdx.x < nrow ? R[(size_t)threadIdx.x * ncol + cb] : T(0);
                        out[threadIdx.x] = x;
                    }
                }
                const int r2 = threadIdx.x + QC_THREADS;
                T x2 = T(0);
                if (r2 < rows_pad) {
                    if (kk < NREG) x2 = out[r2];
                    else if (kk < kres_max)
                        x2 = stiles[((((size_t)gg * nsm + (kk - NREG)) * wpt) * RPW + r2) * 32 + cl];
                    else x2 = r2 < nrow ? R[(size_t)r2 * ncol + cb] : T(0);
                    if (kk >= NREG) out[r2] = x2;
                }
                double s2 = (double)x * (double)x + (double)x2 * (double)x2;
                for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                if (lane == 0) red[warp] = s2;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double t = 0.0;
                    for (int w = 0; w < QC_WARPS; ++w) t += red[w];
                    out[rows_pad] = (T)(t > 0.0 ? 1.0 / sqrt(t) : 0.0);
                }
            }
        }
        if (!grid_barrier(bar, gen, &abort_sh, limit_ns)) return;
        // every CTA: global argmax (one block winner per thread: a single round
        // of loads), then q = (winner's column) x (its inverse norm)
        {
            double gb = -3.0;
            int gbi = 0x7fffffff, gw = 0;
            if (threadIdx.x < gridDim.x) {
                const Best x = block_best[(step & 1) * gridDim.x + threadIdx.x];
                gb = x.v;
                gbi = x.idx;
                gw = threadIdx.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, gb, o);
                const int oi = __shfl_xor_sync(0xffffffffu, gbi, o);
                const int ow = __shfl_xor_sync(0xffffffffu, gw, o);
                if (better(ov, oi, gb, gbi)) { gb = ov; gbi = oi; gw = ow; }
            }
            if (lane == 0) { gv[warp] = gb; gi[warp] = gbi; wsel[warp] = gw; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < QC_WARPS; ++w)
                    if (better(gv[w], gi[w], gb, gbi)) { gb = gv[w]; gbi = gi[w]; gw = wsel[w]; }
                pivot_sh = gbi;
                winner_sh = gw;
            }
        }
        __syncthreads();
        const int p = pivot_sh;
        {
            const T* col = pub + ((size_t)(step & 1) * gridDim.x + winner_sh) * (rows_pad + 4);
            const double inv = (double)col[rows_pad];
            for (int r = threadIdx.x; r < nrow; r += blockDim.x) qs[r] = (T)((double)col[r] * inv);
        }
        if (threadIdx.x == 0) {
            chosen[p] = 1;
            if (blockIdx.x == 0) piv[step] = p;
        }
        {
            const int tile = p / 32, gg = tile % total_groups, kk = tile / total_groups;
            if (gg / ngroups == (int)blockIdx.x && group == gg % ngroups && lane == p % 32 && kk < kres_max)
                cmask |= 1u << kk;
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


// ---------------------------------------------------------------------------
// Register-resident pivoted QR (FP32): the same Businger-Golub steps as the
// kernels above (take the live column with the largest residual norm, ties
// to the lowest index; remove its direction from every column), laid out so
// that one step is a short dependent chain.  LPC lanes hold one column (RPL
// rows each), so the q.r dot products and the norms reduce with lane
// shuffles alone; the columns of a CTA that do not fit in registers live in
// shared memory with a padded row pitch (16-byte accesses free of bank
// conflicts).  The row work runs on packed FP32 pairs.  A step makes one
// pass over each column (the previous step's projection, this step's dot and
// the squared norm before this step's projection: the residual norm is the
// difference, |v|^2 - (q.v)^2).  Per step each warp publishes its best
// column, projected, with its exact squared norm to global memory; the CTAs
// then agree on the global winner through one 64-bit atomicMax per CTA
// (key = the FP32 squared norm's bits above the complemented column index:
// the largest norm, then the lowest index) and a grid barrier on a monotone
// arrival counter; every CTA reads the winner's published column and scales
// it by the inverse square root of its published norm (in FP32: FP64 runs
// at a small fraction of the FP32 rate on this GPU).
constexpr int QR2_THREADS = 512, QR2_WARPS = QR2_THREADS / 32;

__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// sum over the LPC lanes of one column (consecutive lanes)
template <int LPC>
__device__ __forceinline__ float lane_sum(float x) {
#pragma unroll
    for (int o = 1; o < LPC; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One pass over a column chunk held in registers: v <- v - dp qp (the
// previous step's projection, deferred to this pass), then the partial dot
// q.v and squared norm v.v of the result.  The stored values and the dot are
// those of the two-pass form (same products in the same order); only the
// norm after this step's projection, |v|^2 - (q.v)^2, is formed differently.
template <int RPL>
__device__ __forceinline__ void qpass(const float* __restrict__ qp, const float* __restrict__ q, float* v, float dp,
                                      float& dot, float& ss) {
    const f2 nd = bc2(-dp);
    f2 a0 = bc2(0.f), a1 = bc2(0.f), n0 = bc2(0.f), n1 = bc2(0.f);
#pragma unroll
    for (int j = 0; j < RPL; j += 4) {
        const float4 p4 = *reinterpret_cast<const float4*>(qp + j);
        const float4 q4 = *reinterpret_cast<const float4*>(q + j);
        const f2 u0 = fma2(mk2(p4.x, p4.y), nd, mk2(v[j], v[j + 1]));
        const f2 u1 = fma2(mk2(p4.z, p4.w), nd, mk2(v[j + 2], v[j + 3]));
        a0 = fma2(mk2(q4.x, q4.y), u0, a0);
        a1 = fma2(mk2(q4.z, q4.w), u1, a1);
        n0 = fma2(u0, u0, n0);
        n1 = fma2(u1, u1, n1);
        unpk2(u0, v[j], v[j + 1]);
        unpk2(u1, v[j + 2], v[j + 3]);
    }
    float x0, x1;
    unpk2(a0 + a1, x0, x1);
    dot = x0 + x1;
    unpk2(n0 + n1, x0, x1);
    ss = x0 + x1;
}
// The same pass over a column chunk in shared memory: one read and (store)
// one write of the chunk per step.
template <int RPL>
__device__ __forceinline__ void spass(const float* __restrict__ qp, const float* __restrict__ q, float* w, float dp,
                                      bool store, float& dot, float& ss) {
    const f2 nd = bc2(-dp);
    f2 a0 = bc2(0.f), a1 = bc2(0.f), n0 = bc2(0.f), n1 = bc2(0.f);
#pragma unroll 4
    for (int j = 0; j < RPL; j += 4) {
        const float4 p4 = *reinterpret_cast<const float4*>(qp + j);
        const float4 q4 = *reinterpret_cast<const float4*>(q + j);
        const float4 x = *reinterpret_cast<const float4*>(w + j);
        const f2 u0 = fma2(mk2(p4.x, p4.y), nd, mk2(x.x, x.y));
        const f2 u1 = fma2(mk2(p4.z, p4.w), nd, mk2(x.z, x.w));
        a0 = fma2(mk2(q4.x, q4.y), u0, a0);
        a1 = fma2(mk2(q4.z, q4.w), u1, a1);
        n0 = fma2(u0, u0, n0);
        n1 = fma2(u1, u1, n1);
        if (store) {
            float4 o;
            unpk2(u0, o.x, o.y);
            unpk2(u1, o.z, o.w);
            *reinterpret_cast<float4*>(w + j) = o;
        }
    }
    float x0, x1;
    unpk2(a0 + a1, x0, x1);
    dot = x0 + x1;
    unpk2(n0 + n1, x0, x1);
    ss = x0 + x1;
}

__device__ __forceinline__ unsigned long long col_key(float nrm, int col) {
    return ((unsigned long long)__float_as_uint(nrm) << 32) | (unsigned long long)(0xffffffffu - (unsigned)col);
}

// The columns of CTA b are [b cpb, (b + 1) cpb): the first G = 512 / LPC in
// registers (group g = thread / LPC), the rest (s = 0, 1, ...) in shared
// memory, handled by group s % G.  Rows: lane l of a group holds rows
// [l RPL, (l + 1) RPL); q is kept as LPC row chunks of RPL + 4 floats, so
// the LPC distinct chunks a warp reads at once fall on different banks.
//
// Each step makes one pass over every column: it applies the previous step's
// projection (v -= d_{k-1} q_{k-1}, deferred from that step), and forms
// d_k = q_k.v and |v|^2, so the column's norm after step k's projection is
// |v|^2 - d_k^2 (clamped at 0).  A shared-memory column is read and written
// once per step instead of read twice and written once.  The published
// candidate is the projected column v - d_k q_k with its exact squared norm
// (pnorm), from which the next q is normalised.  keys[npiv] and bar[0] are
// zero at launch.
template <int RPL, int LPC>
__global__ void __launch_bounds__(QR2_THREADS, 1)
    qr_resident_kernel(int nrow, int ncol, const float* __restrict__ R, int npiv, int cpb, float* __restrict__ pub,
                       unsigned long long* __restrict__ keys, int* __restrict__ piv, unsigned* bar,
                       unsigned long long limit_ns) {
    constexpr int G = QR2_THREADS / LPC;
    constexpr int NPAD = RPL * LPC;     // padded rows
    constexpr int PITCH = RPL + 4;      // shared-memory row-chunk pitch (floats)
    extern __shared__ __align__(16) float qr2_smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid / LPC, l = tid % LPC;
    const int c0 = blockIdx.x * cpb;
    const int ncta = min(cpb, ncol - c0);  // columns of this CTA
    const int SC = max(0, ncta - G);       // of them in shared memory
    const int rounds = (SC + G - 1) / G;
    const int myreg = g < ncta ? c0 + g : -1;
    float* qbuf = qr2_smem;                            // 2 x [LPC][PITCH]: q of steps k (k & 1) and k - 1
    float* sc = qr2_smem + 2 * LPC * PITCH;            // [SC][LPC][PITCH] shared-memory columns
    float* dsm = sc + (size_t)SC * LPC * PITCH;        // [SC] each shared column's last dot
    float* pnorm = pub + (size_t)2 * gridDim.x * QR2_WARPS * NPAD;  // [2][CTAs][warps] exact squared norms
    __shared__ unsigned long long wkey[QR2_WARPS];
    __shared__ int abort_sh;
    float v[RPL];
    float dreg = 0.f;      // the register column's last dot
    unsigned chosen = 0u;  // bit 0: the register column; bit 1 + r: shared column of round r
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int row = l * RPL + j;
        v[j] = (myreg >= 0 && row < nrow) ? R[(size_t)row * ncol + myreg] : 0.f;
    }
    for (int r = 0; r < rounds; ++r) {
        const int s = r * G + g;
        if (s < SC) {
            float* dst = sc + ((size_t)s * LPC + l) * PITCH;
            const int col = c0 + G + s;
            for (int j = 0; j < RPL; ++j) {
                const int row = l * RPL + j;
                dst[j] = row < nrow ? R[(size_t)row * ncol + col] : 0.f;
            }
        }
    }
    for (int j = tid; j < 2 * LPC * PITCH; j += QR2_THREADS) qbuf[j] = 0.f;
    for (int j = tid; j < SC; j += QR2_THREADS) dsm[j] = 0.f;
    __syncthreads();
    for (int step = 0; step < npiv; ++step) {
        const float* qrow = qbuf + (step & 1) * LPC * PITCH + l * PITCH;        // q_k (zero at step 0)
        const float* prow = qbuf + ((step + 1) & 1) * LPC * PITCH + l * PITCH;  // q_{k-1}
        unsigned long long best = 0ull;
        // register column
        {
            float d, ss;
            qpass<RPL>(prow, qrow, v, dreg, d, ss);
            d = lane_sum<LPC>(d);
            ss = lane_sum<LPC>(ss);
            dreg = d;
            const float nrm = fmaxf(ss - d * d, 0.f);
            if (myreg >= 0 && !(chosen & 1u)) best = col_key(nrm, myreg);
        }
        // shared-memory columns
        for (int r = 0; r < rounds; ++r) {
            const int s = r * G + g;
            const bool has = s < SC;  // uniform over the LPC lanes of the group
            float* w = sc + ((size_t)(has ? s : 0) * LPC + l) * PITCH;
            const float dp = has ? dsm[s] : 0.f;
            float d, ss;
            spass<RPL>(prow, qrow, w, dp, has, d, ss);
            d = lane_sum<LPC>(d);
            ss = lane_sum<LPC>(ss);
            if (has && l == 0) dsm[s] = d;
            if (has && !((chosen >> (1 + r)) & 1u)) {
                const unsigned long long k = col_key(fmaxf(ss - d * d, 0.f), c0 + G + s);
                best = k > best ? k : best;
            }
        }
        // warp argmax of the keys
        unsigned long long wb = best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, wb, o);
            wb = x > wb ? x : wb;
        }
        // the lanes holding the warp's best column publish it projected
        // (v - d q) with its exact squared norm
        __syncwarp();  // this step's dsm writes are visible to the group's lanes
        const size_t slot = ((size_t)(step & 1) * gridDim.x + blockIdx.x) * QR2_WARPS + warp;
        const int wcol = (int)(0xffffffffu - (unsigned)(wb & 0xffffffffu));
        const int ws = wcol - c0 - G;
        const bool own_reg = wb != 0ull && wcol == myreg;
        const bool own_sh = wb != 0ull && ws >= 0 && ws < SC && ws % G == g;
        float pn = 0.f;
        if (own_reg || own_sh) {
            float* out = pub + slot * NPAD + l * RPL;
            const float* src = own_sh ? sc + ((size_t)ws * LPC + l) * PITCH : nullptr;
            const float d = own_sh ? dsm[ws] : dreg;
#pragma unroll
            for (int j = 0; j < RPL; j += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(qrow + j);
                const float4 x = own_sh ? *reinterpret_cast<const float4*>(src + j)
                                        : make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                const float4 o = make_float4(fmaf(-d, q4.x, x.x), fmaf(-d, q4.y, x.y), fmaf(-d, q4.z, x.z),
                                             fmaf(-d, q4.w, x.w));
                pn = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, pn))));
                *reinterpret_cast<float4*>(out + j) = o;
            }
        }
        pn = lane_sum<LPC>(pn);  // every lane takes part; the owner group's lanes get its norm
        if ((own_reg || own_sh) && l == 0) pnorm[slot] = pn;
        if (lane == 0) wkey[warp] = wb;
        // grid barrier: arrive with this CTA's best key, wait for every CTA.
        // The key goes in first (a relaxed reduction, ordered before the
        // arrival by its release); waiting CTAs poll with relaxed loads and
        // a short back-off, then take one acquire fence.
        __syncthreads();
        if (tid == 0) {
            unsigned long long kb = 0ull;
#pragma unroll
            for (int w = 0; w < QR2_WARPS; ++w) kb = wkey[w] > kb ? wkey[w] : kb;
            if (kb) asm volatile("red.relaxed.gpu.global.max.u64 [%0], %1;" ::"l"(keys + step), "l"(kb) : "memory");
            const unsigned target = (unsigned)(step + 1) * gridDim.x;
            unsigned cnt;
            asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(cnt) : "l"(bar) : "memory");
            int timed_out = 0;
            if (cnt + 1 < target) {
                const unsigned long long t0 = global_ns();
                for (;;) {
                    unsigned vv;
                    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(vv) : "l"(bar) : "memory");
                    if (vv >= target) break;
                    if (global_ns() - t0 > limit_ns) {
                        atomicExch(bar + 2, 1u);
                        timed_out = 1;
                        break;
                    }
                    __nanosleep(40);
                }
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            abort_sh = timed_out;
        }
        __syncthreads();
        if (abort_sh) return;
        const unsigned long long key = ld_cg_u64(keys + step);
        if (key == 0ull) {  // no live column left: cannot happen for npiv <= ncol
            if (tid == 0) atomicExch(bar + 2, 2u);
            return;
        }
        const int p = (int)(0xffffffffu - (unsigned)(key & 0xffffffffu));
        const int wcta = p / cpb, li = p - wcta * cpb;
        const int wg = li < G ? li : (li - G) % G;
        const size_t wslot = ((size_t)(step & 1) * gridDim.x + wcta) * QR2_WARPS + (wg * LPC) / 32;
        // the winner's exact squared norm, published with its column; the
        // inverse square root in FP32 (FP64 arithmetic in every thread of
        // every CTA cost ~5 us a step on this GPU's FP64 rate)
        const float nn = __ldcg(pnorm + wslot);
        const float inv = nn > 0.f ? 1.f / sqrtf(nn) : 0.f;
        float* qnext = qbuf + ((step + 1) & 1) * LPC * PITCH;  // q_{k-1} is no longer read
        for (int j = tid; j < NPAD; j += QR2_THREADS)
            qnext[(j / RPL) * PITCH + j % RPL] = __ldcg(pub + wslot * NPAD + j) * inv;
        if (wcta == (int)blockIdx.x && wg == g) {
            if (li < G) chosen |= 1u;
            else chosen |= 1u << (1 + (li - G) / G);
        }
        if (tid == 0 && blockIdx.x == 0) piv[step] = p;
        __syncthreads();
    }
}

}  // namespace

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Capacity (in Best entries) of the block-winner buffer of qrcp_aux_bytes.
static int nblocks_cap(int ncol) { return std::max((ncol + QR_THREADS - 1) / QR_THREADS, 2 * 152 * 8); }

// Row layout of the register-resident QR: RPL rows per lane, LPC lanes per column.
static void qr2_layout(int nrow, int* rpl, int* lpc) {
    *rpl = nrow <= 32 ? 32 : 64;
    *lpc = nrow <= 64 ? 1 : (nrow + 63) / 64 <= 2 ? 2 : (nrow + 63) / 64 <= 4 ? 4 : (nrow + 63) / 64 <= 8 ? 8 : 16;
}

// Published candidate columns: of the persistent kernel, 2 (step parity) x
// CTAs (up to 304) x padded rows (< 2 nrow + 64), FP64 at most; of the
// register-resident kernel, 2 x CTAs x 16 warps x padded rows (FP32).
static size_t pub_bytes(int nrow) {
    int rpl = 0, lpc = 0;
    qr2_layout(nrow, &rpl, &lpc);
    const size_t old = (size_t)2 * 304 * (2 * (size_t)nrow + 64) * sizeof(double);
    const size_t res = align256((size_t)2 * 304 * 16 * rpl * lpc * sizeof(float)) + (size_t)2 * 304 * 16 * lpc * sizeof(double);
    return align256(std::max(old, res));
}

size_t qrcp_aux_bytes(int nrow, int ncol) {
    const int nblocks = nblocks_cap(ncol);
    return align256(sizeof(Best) * nblocks) + align256((size_t)ncol) + align256(sizeof(double) * nrow) + 256 +
           pub_bytes(nrow);
}

// The persistent kernel for one (T, RPW, NREG); *ran = false when the rows
// do not fit its warp layout or the device cannot co-schedule it.
template <typename T, int RPW, int NREG>
static cudaError_t qr_persistent_launch(int nrow, int ncol, T* R, int npiv, Best* best, T* pub,
                                        unsigned char* chosen, int* d_piv, unsigned* bar,
                                        unsigned long long limit_ns, cudaStream_t s, int* launches, bool* ran) {
    *ran = false;
    int dev = 0, sms = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int wpt = 2;  // >= 2 keeps the named-barrier ids (1 + group) within 1..8
    while (wpt * RPW < nrow) wpt *= 2;
    if (!coop || wpt > QC_WARPS || nrow > QC_MAXROWS || sms > 304 || 2 * sms > nblocks_cap(ncol) ||
        (size_t)2 * sms * (wpt * RPW + 4) * sizeof(T) > pub_bytes(nrow))
        return cudaSuccess;
    const void* fn = (const void*)qr_persistent_kernel<T, RPW, NREG>;
    cudaFuncAttributes fa{};
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, fn))) return e;
    // one limit for every caller of this kernel: the opt-in maximum
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)))
        return e;
    const int ngroups = QC_WARPS / wpt;
    const int ntiles = (ncol + 31) / 32;
    // no more CTAs than it takes to hold every tile in registers: a small
    // matrix then syncs fewer CTAs per step and leaves SMs to other work
    const int ctas = std::min(sms, std::max(1, (ntiles + ngroups * std::max(NREG, 1) - 1) / (ngroups * std::max(NREG, 1))));
    const int total_groups = ctas * ngroups;
    const int max_k = (ntiles + total_groups - 1) / total_groups;
    const size_t tile_bytes = (size_t)wpt * RPW * 32 * sizeof(T);  // one tile slot of one group
    const size_t red_bytes = (size_t)2 * QC_WARPS * 32 * sizeof(T);  // dot and norm partials of one tile slot
    const size_t budget = (size_t)std::max(0, optin - (int)fa.sharedSizeBytes - 1024);
    if constexpr (NREG > 0) {
        if (budget < NREG * red_bytes) return cudaSuccess;
    }
    int nsm = std::max(0, max_k - NREG);
    nsm = (int)std::min<size_t>((size_t)nsm, (budget - NREG * red_bytes) / (ngroups * tile_bytes + red_bytes));
    nsm = std::min(nsm, 30 - NREG);  // the per-lane chosen mask has 32 bits
    const size_t dyn = (size_t)ngroups * nsm * tile_bytes + (size_t)(NREG + nsm) * red_bytes;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, QC_THREADS, dyn))) return e;
    if (per_sm < 1) return cudaSuccess;
    if ((e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s))) return e;
    void* args[] = {(void*)&nrow, (void*)&ncol, (void*)&R,   (void*)&npiv,   (void*)&wpt,  (void*)&nsm,
                    (void*)&best, (void*)&pub,  (void*)&chosen, (void*)&d_piv, (void*)&bar, (void*)&limit_ns};
    if ((e = cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(QC_THREADS), args, dyn, s))) return e;
    *launches += 1;
    *ran = true;
    return cudaSuccess;
}

// The register-resident kernel for one (RPL, LPC); *ran = false when the
// matrix does not fit on chip (registers of 256 threads an SM plus shared
// memory) or the device cannot co-schedule the CTAs.
template <int RPL, int LPC>
static cudaError_t qr_resident_launch(int nrow, int ncol, const float* R, int npiv, unsigned long long* keys,
                                      float* pub, int* d_piv, unsigned* bar, unsigned long long limit_ns,
                                      cudaStream_t s, int* launches, bool* ran) {
    *ran = false;
    int dev = 0, sms = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    constexpr int G = QR2_THREADS / LPC, NPAD = RPL * LPC, PITCH = RPL + 4;
    if (!coop || nrow > NPAD || sms > 304 || npiv > 4864) return cudaSuccess;
    int ctas = std::min(sms, (ncol + G - 1) / G);
    const int cpb = (ncol + ctas - 1) / ctas;
    ctas = (ncol + cpb - 1) / cpb;
    const int sc = std::max(0, cpb - G);
    if ((sc + G - 1) / G > 31) return cudaSuccess;  // the per-thread chosen mask has 32 bits
    const void* fn = (const void*)qr_resident_kernel<RPL, LPC>;
    cudaFuncAttributes fa{};
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, fn))) return e;
    // two q buffers, the shared-memory columns and their last dots
    const size_t dyn = (2 * (size_t)LPC * PITCH + (size_t)sc * LPC * PITCH + (((size_t)sc + 3) & ~(size_t)3)) *
                       sizeof(float);
    if (dyn + fa.sharedSizeBytes + 1024 > (size_t)optin) return cudaSuccess;
    // one limit for every caller of this kernel: the opt-in maximum
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)))
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, QR2_THREADS, dyn))) return e;
    if (per_sm < 1 || ctas > per_sm * sms) return cudaSuccess;
    if ((e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s))) return e;
    if ((e = cudaMemsetAsync(keys, 0, (size_t)npiv * sizeof(unsigned long long), s))) return e;
    int cpb_arg = cpb;
    void* args[] = {(void*)&nrow, (void*)&ncol, (void*)&R,     (void*)&npiv,     (void*)&cpb_arg,
                    (void*)&pub,  (void*)&keys, (void*)&d_piv, (void*)&bar, (void*)&limit_ns};
    if ((e = cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(QR2_THREADS), args, dyn, s))) return e;
    *launches += 1;
    *ran = true;
    return cudaSuccess;
}

static bool qr_resident_enabled() {
    static const int on = [] {
        const char* e = getenv("LACE_QR_RESIDENT");  // tuning: 0 selects the tile-group persistent kernel
        return (e && e[0] == '0') ? 0 : 1;
    }();
    return on != 0;
}

// R (nrow x ncol, row-major, leading dimension ncol) is overwritten.  aux is
// caller-provided scratch of qrcp_aux_bytes(nrow, ncol) bytes.
template <typename T>
cudaError_t qrcp_pivots(int nrow, int ncol, T* R, int npiv, int* d_piv, void* aux, int* h_timeout,
                        unsigned long long wait_limit_ns, cudaStream_t s, int* launches) {
    *h_timeout = 0;
    if (nrow > QR_MAXROWS || npiv > ncol) return cudaErrorInvalidValue;
    const int nblocks = (ncol + QR_THREADS - 1) / QR_THREADS;
    unsigned char* base = static_cast<unsigned char*>(aux);
    Best* best = reinterpret_cast<Best*>(base);
    unsigned char* chosen = base + align256(sizeof(Best) * nblocks_cap(ncol));
    T* q = reinterpret_cast<T*>(chosen + align256((size_t)ncol));
    unsigned* bar = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(q) + align256(sizeof(double) * nrow));
    T* pub = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(bar) + 256);
    cudaMemsetAsync(chosen, 0, ncol, s);
    // persistent cooperative version: float rows <= 512 keep two tiles per group
    // in registers (32 rows per warp); otherwise shared memory and streaming only
    bool ran = false;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        // register-resident kernel where the matrix fits on chip, else the
        // tile-group persistent kernel
        e = cudaSuccess;
        if (qr_resident_enabled()) {
            int rpl = 0, lpc = 0;
            qr2_layout(nrow, &rpl, &lpc);
            unsigned long long* keys = reinterpret_cast<unsigned long long*>(best);
            auto go = [&](auto launch) {
                return launch(nrow, ncol, R, npiv, keys, pub, d_piv, bar, wait_limit_ns, s, launches, &ran);
            };
            if (rpl == 32) e = go(qr_resident_launch<32, 1>);
            else if (lpc == 1) e = go(qr_resident_launch<64, 1>);
            else if (lpc == 2) e = go(qr_resident_launch<64, 2>);
            else if (lpc == 4) e = go(qr_resident_launch<64, 4>);
            else if (lpc == 8) e = go(qr_resident_launch<64, 8>);
            else e = go(qr_resident_launch<64, 16>);
        }
        if (!e && !ran) {
            if (nrow <= 512)
                e = qr_persistent_launch<T, 32, 2>(nrow, ncol, R, npiv, best, pub, chosen, d_piv, bar, wait_limit_ns,
                                                  s, launches, &ran);
            else
                e = qr_persistent_launch<T, 64, 0>(nrow, ncol, R, npiv, best, pub, chosen, d_piv, bar, wait_limit_ns,
                                                  s, launches, &ran);
        }
    } else {
        e = qr_persistent_launch<T, 32, 0>(nrow, ncol, R, npiv, best, pub, chosen, d_piv, bar, wait_limit_ns, s,
                                          launches, &ran);
    }
    if (e) return e;
    if (ran) {
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

template cudaError_t qrcp_pivots<float>(int, int, float*, int, int*, void*, int*, unsigned long long, cudaStream_t,
                                         int*);
template cudaError_t qrcp_pivots<double>(int, int, double*, int, int*, void*, int*, unsigned long long, cudaStream_t,
                                          int*);
template cudaError_t gather_subsample<float>(const GridGeom&, int, const float*, int, float*, int*, cudaStream_t, int*);
template cudaError_t gather_subsample<double>(const GridGeom&, int, const double*, int, double*, int*, cudaStream_t,
                                              int*);
template cudaError_t gather_columns<float>(const float*, size_t, int, const long long*, int, double*, cudaStream_t,
                                           int*);
template cudaError_t gather_columns<double>(const double*, size_t, int, const long long*, int, double*, cudaStream_t,
                                            int*);

}  // namespace lace
