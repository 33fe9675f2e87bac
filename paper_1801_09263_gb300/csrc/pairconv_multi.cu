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
// With 256 or 512 threads a CTA, instances on a cubic grid with
// size-specialised passes (24 ... 64) run their items through those pass
// bodies (pairconv_spec2.cuh) in thread groups: a CTA splits into as many
// groups of the size's thread count as its threads and shared memory hold
// (four of 128 threads at 24^3, two of 256 at 32^3-48^3, one of 512 at 60^3
// and 64^3 in a 512-thread CTA), each on its own plane or slab with its own
// named barrier; the other instances run the generic-radix bodies on the
// whole CTA.  Each launch gets all the shared memory its CTAs per SM leave.
// The number of grids of each instance is read from device memory at run
// time, so a captured graph of these launches serves any pair counts that
// need no more chunks than it has launches (a launch without a chunk exits).
// The barriers have a time limit (grid_sync.cuh) and report through bar[2].
#include <algorithm>
#include <cstring>

#include "pairconv_multi.cuh"

namespace lace {

namespace {

using multi::kMaxEntries;

const void* fn_for(int threads, int ctas_per_sm) {
    switch (threads) {
        case 128: return (const void*)multi::pairconv_multi_kernel<128, false>;
        case 256: return multi_kernel_256();
        case 512: return ctas_per_sm >= 2 ? multi_kernel_512x2() : multi_kernel_512();
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

int multi_spec_size(int n1, int n2, int n3) {
    if (n1 != n2 || n2 != n3) return 0;
    switch (n1) {
        case 24: case 32: case 36: case 40: case 48: case 50: case 54: case 60: case 64: return n1;
        default: return 0;
    }
}

size_t multi_spec_smem(int n) {
    switch (n) {
        case 24: return spec2::smem_max(24);
        case 32: return spec2::smem_max(32);
        case 36: return spec2::smem_max(36);
        case 40: return spec2::smem_max(40);
        case 48: return spec2::smem_max(48);
        case 50: return spec2::smem_max(50);
        case 54: return spec2::smem_max(54);
        case 60: return spec2::smem_max(60);
        case 64: return spec2::smem_max(64);
        default: return 0;
    }
}

size_t pairconv_multi_cta_smem(int threads, int ctas_per_sm, size_t need) {
    const void* fn = fn_for(threads, ctas_per_sm);
    if (!fn || ctas_per_sm < 1) return 0;
    int dev = 0, optin = 0, per_sm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // the SM's shared memory split evenly (1 KB reserved per CTA), within
    // the per-CTA opt-in limit; the limit of the kernel is shared by every
    // caller: the opt-in maximum
    const long long share = (long long)per_sm / ctas_per_sm - 1024 - (long long)fa.sharedSizeBytes;
    const long long cap = (long long)optin - (long long)fa.sharedSizeBytes;
    const long long smem = (std::min(share, cap) / 16) * 16;
    if (smem < (long long)need ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, (size_t)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ >= ctas_per_sm ? (size_t)smem : 0;
}

cudaError_t pairconv_multi_run(const MultiArgs& A, int n_chunks, size_t smem, int threads, int ctas_per_sm,
                               cudaStream_t s, int* launches) {
    const void* fn = fn_for(threads, ctas_per_sm);
    if (!fn || ctas_per_sm < 1) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, coop = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaMemsetAsync(A.bar, 0, 4 * sizeof(unsigned), s))) return e;
    MultiArgs a = A;
    a.smem_cta = smem;
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
