// Allocation-free variant of the FP64 pair convolutions.
//
// Some host programs cannot call cudaMalloc at the point where they need the
// exchange applied: a latency-critical loop in which cudaMalloc/cudaFree
// would synchronise the device and stall every other stream, or a program
// whose device memory is owned end to end by its own pool allocator and
// leaves no headroom for a library's private buffers.  For them,
// lace_exchange_pairs_noalloc runs the same three FFT passes as
// lace_apply_exchange in FP64, but takes all of its scratch from one
// file-scope device array of fixed size instead of allocating.  The caller
// passes its own device inputs and outputs.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/lace.h"
#include "lace_internal.cuh"

using namespace lace;

namespace {

// 32 MiB, held on every device that loads the library until the process exits.
constexpr size_t kNoallocScratchBytes = 32u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Set-up cache: the array's device address per device, valid for the
// context it was looked up in.  A cudaDeviceReset destroys that context;
// the device code is then loaded again in a new one and the array can sit
// at another address, so the address is looked up again whenever the
// current context's id (unique for the life of the process) has changed.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult(CUDAAPI*)(CUcontext*);
using CtxGetIdFn = CUresult(CUDAAPI*)(CUcontext, unsigned long long*);

// Id of the current context, 0 when it cannot be read (the address is then
// looked up on every call).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                       q == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<CtxGetCurrentFn>(f)
                   : nullptr;
    }();
    static CtxGetIdFn get_id = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        return cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                       q == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<CtxGetIdFn>(f)
                   : nullptr;
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

constexpr size_t kFlagBytes = 256;
constexpr size_t kTableBytes = 16384;  // 3 twiddle tables (<= 128 x 16 B) + 3 |G|^2 tables (<= 128 x 8 B)

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// FFT tables on the device: tw_a[m] = exp(-2 pi i m / n_a), g2_a[m] = (2 pi m_fft / L_a)^2.
__global__ void noalloc_tables_kernel(int n1, int n2, int n3, double a1, double a2, double a3, double2* tw,
                                      double* g2) {
    const int ns[3] = {n1, n2, n3};
    const double ls[3] = {a1, a2, a3};
    for (int a = 0; a < 3; ++a) {
        const int n = ns[a];
        for (int m = threadIdx.x; m < n; m += blockDim.x) {
            double s, c;
            sincospi(-2.0 * (double)m / (double)n, &s, &c);
            tw[a * kMaxN + m] = make_double2(c, s);
            const int mm = (m < (n + 1) / 2) ? m : m - n;
            const double gv = 2.0 * 3.141592653589793238462643383279502884 * (double)mm / ls[a];
            g2[a * kMaxN + m] = gv * gv;
        }
    }
}

// Every pair must name an occupied i and a row j of Psi, with i <= j when j
// is occupied, and appear once: bit i * n_p + j of seen (cleared by the
// caller) marks a pair already listed.  Pass C adds each pair's potential
// into W; a repeated pair would count twice in W but once in the pair
// energies.
__global__ void noalloc_check_pairs_kernel(const int2* __restrict__ pairs, long long n_pairs, int n_occ, int n_p,
                                           unsigned* __restrict__ seen, int* __restrict__ bad) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (long long)gridDim.x * blockDim.x) {
        const int2 q = pairs[p];
        const bool ok = q.x >= 0 && q.x < n_occ && q.y >= 0 && q.y < n_p && (q.y >= n_occ || q.x <= q.y);
        if (!ok) {
            atomicExch(bad, 1);
            continue;
        }
        const long long bit = (long long)q.x * n_p + q.y;
        const unsigned m = 1u << (bit & 31);
        if (atomicOr(seen + (bit >> 5), m) & m) atomicExch(bad, 1);
    }
}

bool good_axis(int n) {
    if (n < 4 || n > kMaxN) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

}  // namespace

extern "C" lace_status lace_exchange_pairs_noalloc(const double cell[3], int n1, int n2, int n3,
                                                   const double* d_psi, int n_occ, int n_p, const int* d_pairs,
                                                   long long n_pairs, double* d_W, double* d_pair_e,
                                                   void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!cell || !(cell[0] > 0) || !(cell[1] > 0) || !(cell[2] > 0)) return LACE_ERR_ARG;
    if (!d_psi || !d_W || !d_pair_e || (n_pairs > 0 && !d_pairs)) return LACE_ERR_ARG;
    if (n_occ < 1 || n_p < n_occ || n_pairs < 0) return LACE_ERR_ARG;
    if (!good_axis(n1) || !good_axis(n2) || !good_axis(n3)) return LACE_ERR_UNSUPPORTED;

    GridGeom g{};
    const int ns[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = ns[a];
        g.cell[a] = cell[a];
        if (!plan_axis(ns[a], &g.ax[a])) return LACE_ERR_UNSUPPORTED;
    }
    g.ng = (size_t)n1 * n2 * n3;
    g.omega = cell[0] * cell[1] * cell[2];
    g.dv = g.omega / (double)g.ng;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LACE_ERR_CUDA;
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return LACE_ERR_CUDA;
    if (std::max(pairconv_smem_bytes(g, 8, 0), pairconv_smem_bytes(g, 8, 1)) > (size_t)smem_optin)
        return LACE_ERR_UNSUPPORTED;

    // Scratch layout: [flag][tables][pair bitmap][grid descriptors]
    // [energy partials x batch][complex grids x batch]
    const long long n_grids = (n_pairs + 1) / 2;
    const size_t seen_bytes = round256(((size_t)n_occ * (size_t)n_p + 31) / 32 * sizeof(unsigned));
    const size_t desc_bytes = round256((size_t)std::max<long long>(n_grids, 1) * sizeof(PairGrid));
    const size_t fixed = kFlagBytes + kTableBytes + seen_bytes + desc_bytes;
    const size_t epart_per_grid = (size_t)n1 * 2 * sizeof(double);
    const size_t per_grid = g.ng * sizeof(double2) + epart_per_grid;
    auto need = [&](size_t nb) { return fixed + round256(nb * epart_per_grid) + nb * g.ng * sizeof(double2); };
    if (need(1) > kNoallocScratchBytes) return LACE_ERR_UNSUPPORTED;  // grid, pair list or bitmap too large
    size_t nb = (kNoallocScratchBytes - fixed) > 256 ? (kNoallocScratchBytes - fixed - 256) / per_grid : 0;
    nb = std::max<size_t>(std::min<size_t>(nb, 1024), 1);
    while (nb > 1 && need(nb) > kNoallocScratchBytes) --nb;
    const int batch = (int)nb;

    // Set-up, once per device (and again after a device reset), with that
    // device current: the array's device address.  The array's name in host
    // code is only a host-side stand-in for it.  cudaSetDevice makes the
    // device's primary context current (and creates it if needed), so the
    // context id read next is the one the kernels below run in.
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return LACE_ERR_CUDA;
    }
    void* base = nullptr;
    {
        const unsigned long long ctx = current_context_id();
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                g_scratch_addr[dev] = nullptr;
                return LACE_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
            g_scratch_ctx[dev] = ctx;
        }
        base = g_scratch_addr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    int* d_flag = reinterpret_cast<int*>(b);
    double2* tw = reinterpret_cast<double2*>(b + kFlagBytes);
    double* g2 = reinterpret_cast<double*>(b + kFlagBytes + 3 * kMaxN * sizeof(double2));
    unsigned* seen = reinterpret_cast<unsigned*>(b + kFlagBytes + kTableBytes);
    PairGrid* grids = reinterpret_cast<PairGrid*>(b + kFlagBytes + kTableBytes + seen_bytes);
    double* epart = reinterpret_cast<double*>(b + fixed);
    double2* grid_scratch = reinterpret_cast<double2*>(b + fixed + round256((size_t)batch * epart_per_grid));

    // Validate the pair list on the device before any pass reads Psi through
    // it.  The flag and the bitmap keep the previous call's contents: clear them.
    if (cudaMemsetAsync(d_flag, 0, sizeof(int), s) != cudaSuccess) return LACE_ERR_CUDA;
    if (n_pairs > 0) {
        if (cudaMemsetAsync(seen, 0, seen_bytes, s) != cudaSuccess) return LACE_ERR_CUDA;
        const unsigned blocks = (unsigned)std::min<long long>((n_pairs + 255) / 256, 1024);
        noalloc_check_pairs_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const int2*>(d_pairs), n_pairs, n_occ,
                                                          n_p, seen, d_flag);
    }
    int h_bad = 0;
    if (cudaMemcpyAsync(&h_bad, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return LACE_ERR_CUDA;
    }
    if (h_bad) return LACE_ERR_ARG;

    // Outputs accumulate: clear them.  The scratch itself is fully rewritten
    // before it is read, so it needs no clearing.
    int launches = 0;
    if (cudaMemsetAsync(d_W, 0, (size_t)n_p * g.ng * sizeof(double), s) != cudaSuccess) return LACE_ERR_CUDA;
    if (fill_zero_f64(d_pair_e, (size_t)n_occ * n_occ, s, &launches) != cudaSuccess) return LACE_ERR_CUDA;
    noalloc_tables_kernel<<<1, 128, 0, s>>>(n1, n2, n3, cell[0], cell[1], cell[2], tw, g2);
    FFTTables<double> tb;
    for (int a = 0; a < 3; ++a) {
        tb.tw[a] = tw + a * kMaxN;
        tb.g2[a] = g2 + a * kMaxN;
    }
    if (n_grids > 0) {
        if (pack_pair_grids(reinterpret_cast<const int2*>(d_pairs), n_pairs, grids, s, &launches) != cudaSuccess)
            return LACE_ERR_CUDA;
        if (pairconv_run<double>(g, tb, d_psi, n_occ, d_W, grids, (int)n_grids, grid_scratch, batch, epart,
                                 d_pair_e, s, &launches, nullptr, nullptr) != cudaSuccess)
            return LACE_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? LACE_OK : LACE_ERR_CUDA;
}
