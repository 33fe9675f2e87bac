// Pair convolutions of many independent systems in one persistent launch
// (batched uneven instances: different grids, orbital counts and pair
// counts).  Eq. 2 with FFTs (Sec. 2), as in pairconv.cu, for every kept pair
// of every instance.
//
// The complex grids of all instances form one list (instance by instance),
// cut into chunks that fit the scratch pool; one cooperative launch of
// ctas_per_sm x SMs CTAs per chunk (one launch in all when the pool holds
// every kept grid), in which the CTAs sweep
//   A  (planes: rho and the 2D FFT over y, z)          -> barrier
//   B  (slabs: FFT along x, K(G)/Ng, inverse FFT)      -> barrier
//   C  (planes: inverse 2D FFT, W -= w v, energies)    -> barrier
//   D  (grids: per-plane energies -> pair-energy matrix)
// with every work item (plane, slab, grid) taken round-robin by the CTAs.
// The number of grids of each instance is read from device memory at run
// time, so a captured graph of these launches serves any pair counts that
// need no more chunks than it has launches (a launch without a chunk exits).
// The barriers have a time limit (grid_sync.cuh) and report through bar[2].
#include <algorithm>
#include <cstring>

#include "grid_sync.cuh"
#include "lace_internal.cuh"
#include "pairconv_generic.cuh"

namespace lace {

namespace {

constexpr int kMaxEntries = 256;  // instance pieces per chunk

struct ChunkTable {
    int n;                       // entries
    int q[kMaxEntries];          // instance
    int g0[kMaxEntries];         // first grid (instance-local index)
    int cnt[kMaxEntries];        // grids
    size_t pool[kMaxEntries];    // pool offset of the first grid (complex elements)
    size_t ep[kMaxEntries];      // epart offset (doubles)
    int item[kMaxEntries + 1];   // item prefix of the current phase
    // where the next chunk starts
    int next_q, next_g;
};

// Thread 0: the chunk starting at grid g of instance q.
__device__ void build_chunk(const MultiArgs& A, int q, int g, ChunkTable& t) {
    size_t pool_used = 0, ep_used = 0;
    int n = 0;
    while (q < A.n_inst && n < kMaxEntries) {
        const int total = A.n_grids[q];
        const int rem = total - g;
        if (rem <= 0) {
            ++q;
            g = 0;
            continue;
        }
        const MultiInst& I = A.inst[q];
        const size_t ng = I.P.ng;
        const size_t per_ep = 2 * (size_t)I.n1;
        const size_t fit_pool = (A.pool_elems - pool_used) / ng;
        const size_t fit_ep = (A.epart_elems - ep_used) / per_ep;
        const int fit = (int)std::min<size_t>((size_t)rem, std::min(fit_pool, fit_ep));
        if (fit <= 0) break;
        t.q[n] = q;
        t.g0[n] = g;
        t.cnt[n] = fit;
        t.pool[n] = pool_used;
        t.ep[n] = ep_used;
        pool_used += (size_t)fit * ng;
        ep_used += (size_t)fit * per_ep;
        ++n;
        g += fit;
        if (g >= total) {
            ++q;
            g = 0;
        }
    }
    t.n = n;
    t.next_q = q;
    t.next_g = g;
}

// Thread 0: item prefix for a phase (0: planes n1, 1: slabs n2, 2: grids).
__device__ void build_items(const MultiArgs& A, ChunkTable& t, int phase) {
    int acc = 0;
    for (int e = 0; e < t.n; ++e) {
        t.item[e] = acc;
        const MultiInst& I = A.inst[t.q[e]];
        const int per = phase == 0 ? I.n1 : (phase == 1 ? I.n2 : 1);
        acc += t.cnt[e] * per;
    }
    t.item[t.n] = acc;
}

__device__ __forceinline__ int find_entry(const ChunkTable& t, int it) {
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.item[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Chunk `chunk` of the grid list, all four phases.  Thread 0 finds the
// chunk by walking the chunks before it (O(chunks x instances), negligible).
// One chunk per launch: around a chunk loop the inlined phases need twice the
// registers.
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT > 0 ? 512 / NT : 1) pairconv_multi_kernel(MultiArgs A, int chunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<float>* work = reinterpret_cast<cplx<float>*>(smem_raw);
    __shared__ ChunkTable t;
    __shared__ double red[2 * 32];
    __shared__ int abort_sh;
    unsigned gen = 0;
    if (threadIdx.x == 0) {
        int q = 0, g = 0;
        for (int c = 0;; ++c) {
            build_chunk(A, q, g, t);
            if (c == chunk || t.n == 0) break;
            q = t.next_q;
            g = t.next_g;
        }
    }
    __syncthreads();
    if (t.n == 0) return;
    // A: planes
    if (threadIdx.x == 0) build_items(A, t, 0);
    __syncthreads();
    for (int it = blockIdx.x; it < t.item[t.n]; it += gridDim.x) {
        const int e = find_entry(t, it);
        const MultiInst& I = A.inst[t.q[e]];
        const int loc = it - t.item[e], k = loc / I.n1, x = loc - k * I.n1;
        gen::pass_a_plane<float>(I.P, I.P.grids[t.g0[e] + k], A.pool + t.pool[e] + (size_t)k * I.P.ng, x, work);
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // B: slabs
    if (threadIdx.x == 0) build_items(A, t, 1);
    __syncthreads();
    for (int it = blockIdx.x; it < t.item[t.n]; it += gridDim.x) {
        const int e = find_entry(t, it);
        const MultiInst& I = A.inst[t.q[e]];
        const int loc = it - t.item[e], k = loc / I.n2, ky = loc - k * I.n2;
        gen::pass_b_slab<float>(I.P, A.pool + t.pool[e] + (size_t)k * I.P.ng, ky, work);
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // C: planes
    if (threadIdx.x == 0) build_items(A, t, 0);
    __syncthreads();
    for (int it = blockIdx.x; it < t.item[t.n]; it += gridDim.x) {
        const int e = find_entry(t, it);
        const MultiInst& I = A.inst[t.q[e]];
        const int loc = it - t.item[e], k = loc / I.n1, x = loc - k * I.n1;
        gen::pass_c_plane<float>(I.P, I.P.grids[t.g0[e] + k], A.pool + t.pool[e] + (size_t)k * I.P.ng, x, work, red,
                                 A.epart + t.ep[e] + ((size_t)k * I.n1 + x) * 2);
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // D: per grid, the plane energies in a fixed order -> E[i][j] = E[j][i]
    if (threadIdx.x == 0) build_items(A, t, 2);
    __syncthreads();
    for (int it = blockIdx.x * NT + threadIdx.x; it < t.item[t.n]; it += gridDim.x * NT) {
        const int e = find_entry(t, it);
        const MultiInst& I = A.inst[t.q[e]];
        const int k = it - t.item[e];
        const PairGrid d = I.P.grids[t.g0[e] + k];
        const double* ep = A.epart + t.ep[e] + (size_t)k * I.n1 * 2;
        double sa = 0.0, sb = 0.0;
        for (int x = 0; x < I.n1; ++x) {
            sa += ep[2 * x];
            sb += ep[2 * x + 1];
        }
        const int no = I.P.n_occ;
        if (d.j1 < no) {
            I.E[(size_t)d.i1 * no + d.j1] = sa;
            I.E[(size_t)d.j1 * no + d.i1] = sa;
        }
        if (d.j2 >= 0 && d.j2 < no) {
            I.E[(size_t)d.i2 * no + d.j2] = sb;
            I.E[(size_t)d.j2 * no + d.i2] = sb;
        }
    }
}

template <int NT>
const void* multi_fn() {
    return (const void*)pairconv_multi_kernel<NT>;
}

const void* fn_for(int threads) {
    switch (threads) {
        case 128: return multi_fn<128>();
        case 256: return multi_fn<256>();
        case 512: return multi_fn<512>();
        default: return nullptr;
    }
}

}  // namespace

int pairconv_multi_chunks(const std::vector<int>& n_grids, const std::vector<size_t>& ng, const std::vector<int>& n1,
                          size_t pool_elems, size_t epart_elems) {
    const int n_inst = (int)n_grids.size();
    int chunks = 0, q = 0, g = 0;
    for (;;) {
        size_t pool_used = 0, ep_used = 0;
        int n = 0;
        while (q < n_inst && n < kMaxEntries) {
            const int rem = n_grids[q] - g;
            if (rem <= 0) {
                ++q;
                g = 0;
                continue;
            }
            const size_t per_ep = 2 * (size_t)n1[q];
            const size_t fit_pool = (pool_elems - pool_used) / ng[q];
            const size_t fit_ep = (epart_elems - ep_used) / per_ep;
            const int fit = (int)std::min<size_t>((size_t)rem, std::min(fit_pool, fit_ep));
            if (fit <= 0) break;
            pool_used += (size_t)fit * ng[q];
            ep_used += (size_t)fit * per_ep;
            ++n;
            g += fit;
            if (g >= n_grids[q]) {
                ++q;
                g = 0;
            }
        }
        if (n == 0) return chunks;
        ++chunks;
    }
}

size_t pairconv_multi_smem(int n1, int n2, int n3) {
    GridGeom g{};
    g.n[0] = n1;
    g.n[1] = n2;
    g.n[2] = n3;
    return std::max(pairconv_smem_bytes(g, 4, 0), pairconv_smem_bytes(g, 4, 1));
}

int pairconv_multi_occupancy(int threads, size_t smem) {
    const void* fn = fn_for(threads);
    if (!fn) return 0;
    int dev = 0, per_sm = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // the limit is shared by every caller of this kernel: the opt-in maximum
    if (smem + fa.sharedSizeBytes > (size_t)optin ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

cudaError_t pairconv_multi_run(const MultiArgs& A, int n_chunks, size_t smem, int threads, int ctas_per_sm,
                               cudaStream_t s, int* launches) {
    const void* fn = fn_for(threads);
    if (!fn || ctas_per_sm < 1) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, coop = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaMemsetAsync(A.bar, 0, 4 * sizeof(unsigned), s))) return e;
    MultiArgs a = A;
    for (int c = 0; c < n_chunks; ++c) {
        // fresh barrier counters per launch; the timeout flag bar[2] stays set
        if (c > 0 && (e = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), s))) return e;
        void* args[] = {(void*)&a, (void*)&c};
        if ((e = cudaLaunchCooperativeKernel(fn, dim3(sms * ctas_per_sm), dim3(threads), args, smem, s))) return e;
        *launches += 1;
    }
    return cudaSuccess;
}

}  // namespace lace
