// Pair convolutions of the exchange operator (Eq. 2 evaluated with FFTs,
// Sec. 2; truncated to the kept pairs of Eq. 5).
//
// For each kept pair (i, j) the pair density rho = w_i psi_j is transformed
// to reciprocal space, multiplied by K(G) = 4 pi/|G|^2 (K(0) = 0), and
// transformed back: v_ij = IFFT(K FFT(rho)).  Then W_j -= w_i v_ij and, for
// an occupied j != i, W_i -= w_j v_ij (v_ij = v_ji).  Two real pairs share
// one complex FFT grid (rho_a + i rho_b): K is real and even, so the real
// and imaginary parts of the inverse transform are v_a and v_b exactly.
//
// Three passes per batch of complex grids, grid layout [x][y][z] (z fastest):
//   A: per x-plane: form rho, 2D FFT over (y, z) in shared memory, store.
//   B: per y-slab: FFT along x, multiply by K(G)/Ng, inverse FFT along x.
//   C: per x-plane: inverse 2D FFT, then accumulate -w v into W (atomic
//      adds) and the real-space pair energies dV sum rho v (FP64).
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <type_traits>
#include <vector>

#include "lace_internal.cuh"
#include "pairconv_generic.cuh"

namespace lace {

namespace {

constexpr int kThreads = 256;

// Pass A: rho for plane x of complex grid g, forward FFT over z then y.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_a_kernel(ConvArgs<T> P, int g0) {
    extern __shared__ unsigned char smem_raw[];
    const int g = blockIdx.y;
    gen::pass_a_plane<T>(P, P.grids[g0 + g], P.scratch + (size_t)g * P.ng, blockIdx.x,
                         reinterpret_cast<cplx<T>*>(smem_raw));
}

// Pass B: slab ky of complex grid g: FFT along x, * K/Ng, inverse FFT along x.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_b_kernel(ConvArgs<T> P, int g0) {
    extern __shared__ unsigned char smem_raw[];
    gen::pass_b_slab<T>(P, P.scratch + (size_t)blockIdx.y * P.ng, blockIdx.x, reinterpret_cast<cplx<T>*>(smem_raw));
    (void)g0;
}

// Pass C: inverse 2D FFT of plane x, accumulate into W and pair energies.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_c_kernel(ConvArgs<T> P, int g0) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ double red[2 * 32];
    const int g = blockIdx.y, x = blockIdx.x;
    gen::pass_c_plane<T>(P, P.grids[g0 + g], P.scratch + (size_t)g * P.ng, x, reinterpret_cast<cplx<T>*>(smem_raw),
                         red, P.epart + ((size_t)g * gridDim.x + x) * 2);
}

// Sum the per-plane energies of each grid (fixed order) into the pair-energy
// matrix E[i][j] = E[j][i] = e_ij for occupied pairs.
__global__ void energy_collect_kernel(const double* epart, int nplanes, const PairGrid* grids, int g0, int ngr,
                                      int n_occ, double* E) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngr) return;
    const PairGrid d = grids[g0 + g];
    double sa = 0.0, sb = 0.0;
    for (int x = 0; x < nplanes; ++x) {
        sa += epart[((size_t)g * nplanes + x) * 2];
        sb += epart[((size_t)g * nplanes + x) * 2 + 1];
    }
    if (d.j1 < n_occ) {
        E[(size_t)d.i1 * n_occ + d.j1] = sa;
        E[(size_t)d.j1 * n_occ + d.i1] = sa;
    }
    if (d.j2 >= 0 && d.j2 < n_occ) {
        E[(size_t)d.i2 * n_occ + d.j2] = sb;
        E[(size_t)d.j2 * n_occ + d.i2] = sb;
    }
}

// The same for a merged launch: grid g of the round is refs[g0 + g] of its
// system; the energies go to that system's matrix.
__global__ void energy_collect_merged_kernel(const GridRef* __restrict__ refs, const MergedSys<float>* __restrict__ ms,
                                             int g0, int ngr, int nplanes) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngr) return;
    const GridRef r = refs[g0 + g];
    const MergedSys<float>& m = ms[r.sys];
    const PairGrid d = m.grids[r.g];
    const double* ep = m.epart + (size_t)(r.g - m.g0) * nplanes * 2;
    double sa = 0.0, sb = 0.0;
    for (int x = 0; x < nplanes; ++x) {
        sa += ep[2 * x];
        sb += ep[2 * x + 1];
    }
    const int n_occ = m.n_occ;
    if (d.j1 < n_occ) {
        m.E[(size_t)d.i1 * n_occ + d.j1] = sa;
        m.E[(size_t)d.j1 * n_occ + d.i1] = sa;
    }
    if (d.j2 >= 0 && d.j2 < n_occ) {
        m.E[(size_t)d.i2 * n_occ + d.j2] = sb;
        m.E[(size_t)d.j2 * n_occ + d.i2] = sb;
    }
}

}  // namespace

static const int kRadices[] = {16, 12, 10, 9, 8, 6, 5, 4, 3, 2};

static void search(int n, int depth, int maxdepth, std::vector<int>& cur, std::vector<int>& best, int& best_min) {
    if (n == 1) {
        int mn = 1 << 30;
        for (int r : cur) mn = std::min(mn, r);
        if (best.empty() || cur.size() < best.size() || (cur.size() == best.size() && mn > best_min)) {
            best = cur;
            best_min = mn;
        }
        return;
    }
    if (depth == maxdepth) return;
    for (int r : kRadices) {
        if (n % r == 0) {
            cur.push_back(r);
            search(n / r, depth + 1, maxdepth, cur, best, best_min);
            cur.pop_back();
        }
    }
}

bool plan_axis(int n, AxisPlan* out) {
    if (n < 2 || n > kMaxN) return false;
    std::vector<int> cur, best;
    int best_min = 0;
    for (int d = 1; d <= 4 && best.empty(); ++d) search(n, 0, d, cur, best, best_min);
    if (best.empty()) return false;
    out->n = n;
    out->nst = (int)best.size();
    for (int i = 0; i < 4; ++i) out->radix[i] = i < out->nst ? best[i] : 1;
    return true;
}

size_t pairconv_smem_bytes(const GridGeom& g, int eb, int pass) {
    const size_t c = 2 * (size_t)eb;
    if (pass == 1) return c * ((size_t)g.n[0] * g.n[2] + g.n[0]) + (size_t)eb * (g.n[0] + g.n[2]);
    return c * ((size_t)g.n[1] * g.n[2] + g.n[1] + g.n[2]);
}

template <typename T>
cudaError_t pairconv_run(const GridGeom& g, const FFTTables<T>& tb, const T* psi, int n_occ, T* W,
                         const PairGrid* d_grids, int n_grids, cplx<T>* scratch, int batch, double* epart,
                         double* d_pair_e, cudaStream_t s, int* launches, cudaEvent_t ev0, cudaEvent_t ev1) {
    ConvArgs<T> P;
    for (int a = 0; a < 3; ++a) {
        P.ax[a] = g.ax[a];
        P.tw[a] = tb.tw[a];
        P.g2[a] = tb.g2[a];
    }
    P.kscale = (T)(4.0 * M_PI / (double)g.ng);
    P.ktab = tb.ktab;
    P.psi = psi;
    P.n_occ = n_occ;
    P.W = W;
    P.grids = d_grids;
    P.scratch = scratch;
    P.epart = epart;
    P.ng = g.ng;
    P.dv = g.dv;
    const size_t sm_plane = pairconv_smem_bytes(g, sizeof(T), 0);
    const size_t sm_slab = pairconv_smem_bytes(g, sizeof(T), 1);
    cudaError_t e;
    // The dynamic shared-memory limit is a per-function attribute shared by
    // every thread and stream of the process: set it once per device to the
    // device's opt-in maximum (grids of different sizes can be in flight
    // together), never to one grid's need.
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if (dev >= 64 || !(attr_done.load() & (1ull << dev))) {
        int optin = 0;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
        const void* fns[3] = {(const void*)pass_a_kernel<T>, (const void*)pass_b_kernel<T>,
                              (const void*)pass_c_kernel<T>};
        for (const void* fn : fns) {
            cudaFuncAttributes fa{};
            if ((e = cudaFuncGetAttributes(&fa, fn))) return e;
            const int dyn = optin - (int)fa.sharedSizeBytes;  // static shared memory counts against the limit
            if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn))) return e;
        }
        if (dev < 64) attr_done.fetch_or(1ull << dev);
    }
    {
        // the out-of-place passes prefetch into L2 what the CTA two waves
        // later (at two CTAs per SM) will read
        int nsm = 0;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
        static const int per_sm = [] {
            const char* v = getenv("LACE_L2_PREFETCH_PER_SM");  // tuning: CTAs ahead per SM (0: off)
            return v ? atoi(v) : 2;
        }();
        P.pf_ahead = per_sm * nsm;
    }
    if (sm_plane > (size_t)INT32_MAX || sm_slab > (size_t)INT32_MAX) return cudaErrorInvalidValue;
    // size-specialised FP32 kernels for even cubic grids of the specialised
    // sizes (their planes start on 16-byte boundaries; LACE_GENERIC_FFT=1 to disable)
    const char* gen = getenv("LACE_GENERIC_FFT");
    const bool spec_ok = !(gen && gen[0] == '1') && g.n[0] == g.n[1] && g.n[1] == g.n[2] && g.n[0] % 2 == 0;
    if (ev0) cudaEventRecord(ev0, s);
    for (int g0 = 0; g0 < n_grids; g0 += batch) {
        const int nb = std::min(batch, n_grids - g0);
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (spec_ok) {
                for (int pass = 0; pass < 3; ++pass)
                    done = spec_launch_s(pass, g.n[0], nb, P, g0, s) || spec_launch_m(pass, g.n[0], nb, P, g0, s) ||
                           spec_launch_l(pass, g.n[0], nb, P, g0, s) || spec_launch_x(pass, g.n[0], nb, P, g0, s);
            }
        }
        if (!done) {
            pass_a_kernel<T><<<dim3(g.n[0], nb), kThreads, sm_plane, s>>>(P, g0);
            pass_b_kernel<T><<<dim3(g.n[1], nb), kThreads, sm_slab, s>>>(P, g0);
            pass_c_kernel<T><<<dim3(g.n[0], nb), kThreads, sm_plane, s>>>(P, g0);
        }
        energy_collect_kernel<<<(nb + 127) / 128, 128, 0, s>>>(epart, g.n[0], d_grids, g0, nb, n_occ, d_pair_e);
        *launches += 4;
        if ((e = cudaGetLastError())) return e;
    }
    if (ev1) cudaEventRecord(ev1, s);
    return cudaSuccess;
}

cudaError_t pairconv_run_merged(int n, const FFTTables<float>& tb, const std::vector<MergedSys<float>>& sys,
                                const std::vector<int>& n_grids, const std::vector<int>& cap, GridRef* d_refs,
                                MergedSys<float>* d_sys, cudaStream_t s, int* launches, int* rounds_out) {
    const int nsys = (int)sys.size();
    if (rounds_out) *rounds_out = 0;
    if (!spec_merge_ok(n) || nsys == 0 || (int)n_grids.size() != nsys || (int)cap.size() != nsys)
        return cudaErrorInvalidValue;
    // rounds: the next chunk of every system with grids left
    std::vector<GridRef> refs;
    std::vector<MergedSys<float>> per_round;
    std::vector<int> start;
    std::vector<int> next(nsys, 0);
    for (;;) {
        const int r0 = (int)refs.size();
        for (int q = 0; q < nsys; ++q) {
            MergedSys<float> m = sys[q];
            m.g0 = next[q];
            const int k = std::min(std::max(cap[q], 1), n_grids[q] - next[q]);
            for (int j = 0; j < k; ++j) refs.push_back(GridRef{q, next[q] + j});
            next[q] += std::max(k, 0);
            per_round.push_back(m);
        }
        if ((int)refs.size() == r0) {
            per_round.resize(per_round.size() - nsys);
            break;
        }
        start.push_back(r0);
    }
    start.push_back((int)refs.size());
    const int rounds = (int)start.size() - 1;
    if (rounds == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_refs, refs.data(), sizeof(GridRef) * refs.size(), cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(d_sys, per_round.data(), sizeof(MergedSys<float>) * per_round.size(),
                             cudaMemcpyHostToDevice, s)))
        return e;
    ConvArgs<float> P;
    for (int a = 0; a < 3; ++a) {
        P.tw[a] = tb.tw[a];
        P.g2[a] = tb.g2[a];
    }
    const size_t ng = (size_t)n * n * n;
    P.kscale = (float)(4.0 * M_PI / (double)ng);
    P.ktab = nullptr;
    P.psi = nullptr;
    P.W = nullptr;
    P.grids = nullptr;
    P.scratch = nullptr;
    P.epart = nullptr;
    P.n_occ = 0;
    P.ng = ng;
    P.dv = 0.0;
    P.refs = d_refs;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    P.pf_ahead = 2 * nsm;
    for (int r = 0; r < rounds; ++r) {
        const int g0 = start[r], nb = start[r + 1] - start[r];
        P.msys = d_sys + (size_t)r * nsys;
        for (int pass = 0; pass < 3; ++pass) {
            const bool ok = spec_launch_s(pass, n, nb, P, g0, s) || spec_launch_m(pass, n, nb, P, g0, s) ||
                            spec_launch_l(pass, n, nb, P, g0, s) || spec_launch_x(pass, n, nb, P, g0, s);
            if (!ok) return cudaErrorInvalidValue;
        }
        energy_collect_merged_kernel<<<(nb + 127) / 128, 128, 0, s>>>(d_refs, P.msys, g0, nb, n);
        *launches += 4;
        if ((e = cudaGetLastError())) return e;
    }
    if (rounds_out) *rounds_out = rounds;
    return cudaSuccess;
}

template cudaError_t pairconv_run<float>(const GridGeom&, const FFTTables<float>&, const float*, int, float*,
                                         const PairGrid*, int, cplx<float>*, int, double*, double*, cudaStream_t, int*,
                                         cudaEvent_t, cudaEvent_t);
template cudaError_t pairconv_run<double>(const GridGeom&, const FFTTables<double>&, const double*, int, double*,
                                          const PairGrid*, int, cplx<double>*, int, double*, double*, cudaStream_t,
                                          int*, cudaEvent_t, cudaEvent_t);

}  // namespace lace
