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

#include "lace_internal.cuh"

namespace lace {

namespace {

constexpr int kThreads = 256;

template <typename C>
__device__ __forceinline__ void load_tw(C* dst, const C* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Pass A: rho for plane x of complex grid g, forward FFT over z then y.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_a_kernel(ConvArgs<T> P, int g0) {
    using C = cplx<T>;
    extern __shared__ unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);
    const int n1 = P.ax[0].n, n2 = P.ax[1].n, n3 = P.ax[2].n;
    const int np = n2 * n3;
    C* tw2 = plane + np;
    C* tw3 = tw2 + n2;
    const int g = blockIdx.y, x = blockIdx.x;
    const PairGrid d = P.grids[g0 + g];
    load_tw(tw2, P.tw[1], n2);
    load_tw(tw3, P.tw[2], n3);
    const size_t off = (size_t)x * np;
    const T* a1 = P.psi + (size_t)d.i1 * P.ng + off;
    const T* b1 = P.psi + (size_t)d.j1 * P.ng + off;
    const bool two = d.j2 >= 0;
    const T* a2 = P.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off;
    const T* b2 = P.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        T ra = a1[e] * b1[e];
        T rb = two ? a2[e] * b2[e] : T(0);
        plane[e] = C{ra, rb};
    }
    __syncthreads();
    fft_lines<T, -1>(plane, P.ax[2], n2, n3, 1, false, tw3);  // z lines
    fft_lines<T, -1>(plane, P.ax[1], n3, 1, n3, true, tw2);   // y lines
    C* out = P.scratch + (size_t)g * P.ng + off;
    for (int e = threadIdx.x; e < np; e += blockDim.x) out[e] = plane[e];
    (void)n1;
}

// Pass B: slab ky of complex grid g: FFT along x, * K/Ng, inverse FFT along x.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_b_kernel(ConvArgs<T> P, int g0) {
    using C = cplx<T>;
    extern __shared__ unsigned char smem_raw[];
    C* slab = reinterpret_cast<C*>(smem_raw);
    const int n1 = P.ax[0].n, n2 = P.ax[1].n, n3 = P.ax[2].n;
    C* tw1 = slab + n1 * n3;
    T* gz2 = reinterpret_cast<T*>(tw1 + n1);
    T* gx2 = gz2 + n3;
    const int g = blockIdx.y, ky = blockIdx.x;
    load_tw(tw1, P.tw[0], n1);
    for (int i = threadIdx.x; i < n3; i += blockDim.x) gz2[i] = P.g2[2][i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) gx2[i] = P.g2[0][i];
    C* base = P.scratch + (size_t)g * P.ng + (size_t)ky * n3;
    const size_t xs = (size_t)n2 * n3;
    for (int e = threadIdx.x; e < n1 * n3; e += blockDim.x) {
        const int x = e / n3, z = e - x * n3;
        slab[e] = base[(size_t)x * xs + z];
    }
    __syncthreads();
    fft_lines<T, -1>(slab, P.ax[0], n3, 1, n3, true, tw1);
    const T gy2 = P.g2[1][ky];
    for (int e = threadIdx.x; e < n1 * n3; e += blockDim.x) {
        const int x = e / n3, z = e - x * n3;
        T k;
        if (P.ktab) {
            k = P.ktab[((size_t)x * n2 + ky) * n3 + z];
        } else {
            const T gg = gx2[x] + gy2 + gz2[z];
            k = gg > T(0) ? P.kscale / gg : T(0);
        }
        C v = slab[e];
        slab[e] = C{v.x * k, v.y * k};
    }
    __syncthreads();
    fft_lines<T, +1>(slab, P.ax[0], n3, 1, n3, true, tw1);
    for (int e = threadIdx.x; e < n1 * n3; e += blockDim.x) {
        const int x = e / n3, z = e - x * n3;
        base[(size_t)x * xs + z] = slab[e];
    }
    (void)g0;
}

template <typename T> __device__ __forceinline__ void red_add(T* p, T v) { atomicAdd(p, v); }

template <typename T> __device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Pass C: inverse 2D FFT of plane x, accumulate into W and pair energies.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_c_kernel(ConvArgs<T> P, int g0) {
    using C = cplx<T>;
    extern __shared__ unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);
    const int n2 = P.ax[1].n, n3 = P.ax[2].n;
    const int np = n2 * n3;
    C* tw2 = plane + np;
    C* tw3 = tw2 + n2;
    __shared__ double red[2][kThreads / 32];
    const int g = blockIdx.y, x = blockIdx.x;
    const PairGrid d = P.grids[g0 + g];
    load_tw(tw2, P.tw[1], n2);
    load_tw(tw3, P.tw[2], n3);
    const size_t off = (size_t)x * np;
    const C* in = P.scratch + (size_t)g * P.ng + off;
    for (int e = threadIdx.x; e < np; e += blockDim.x) plane[e] = in[e];
    __syncthreads();
    fft_lines<T, +1>(plane, P.ax[1], n3, 1, n3, true, tw2);
    fft_lines<T, +1>(plane, P.ax[2], n2, n3, 1, false, tw3);
    const bool two = d.j2 >= 0;
    const bool a_occ = d.j1 < P.n_occ, a_sym = a_occ && d.j1 != d.i1;
    const bool b_occ = two && d.j2 < P.n_occ, b_sym = b_occ && d.j2 != d.i2;
    const T* wi1 = P.psi + (size_t)d.i1 * P.ng + off;
    const T* pj1 = P.psi + (size_t)d.j1 * P.ng + off;
    T* Wj1 = P.W + (size_t)d.j1 * P.ng + off;
    T* Wi1 = P.W + (size_t)d.i1 * P.ng + off;
    const T* wi2 = P.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off;
    const T* pj2 = P.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off;
    T* Wj2 = P.W + (size_t)(two ? d.j2 : d.j1) * P.ng + off;
    T* Wi2 = P.W + (size_t)(two ? d.i2 : d.i1) * P.ng + off;
    // Per-thread energy sums in T with compensated (Kahan) addition; the
    // warp sums stay in T and only the per-warp totals go to FP64, so the
    // FP32 path issues no FP64 arithmetic per grid point.
    T sa = T(0), ca = T(0), sb = T(0), cb = T(0);
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        const C v = plane[e];
        const T x1 = wi1[e], y1 = pj1[e];
        red_add(Wj1 + e, -x1 * v.x);
        if (a_sym) red_add(Wi1 + e, -y1 * v.x);
        if (a_occ) kahan_add(sa, ca, x1 * y1 * v.x);
        if (two) {
            const T x2 = wi2[e], y2 = pj2[e];
            red_add(Wj2 + e, -x2 * v.y);
            if (b_sym) red_add(Wi2 + e, -y2 * v.y);
            if (b_occ) kahan_add(sb, cb, x2 * y2 * v.y);
        }
    }
    sa -= ca;
    sb -= cb;
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = (double)sa; red[1][warp] = (double)sb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tbb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ta += red[0][w]; tbb += red[1][w]; }
        double* ep = P.epart + ((size_t)g * gridDim.x + x) * 2;
        ep[0] = ta * P.dv;
        ep[1] = tbb * P.dv;
    }
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
    if (sm_plane > (size_t)INT32_MAX || sm_slab > (size_t)INT32_MAX) return cudaErrorInvalidValue;
    // size-specialised FP32 kernels for cubic grids with n % 4 == 0 (or LACE_GENERIC_FFT=1 to disable)
    const char* gen = getenv("LACE_GENERIC_FFT");
    const bool spec_ok = !(gen && gen[0] == '1') && g.n[0] == g.n[1] && g.n[1] == g.n[2] && g.n[0] % 4 == 0;
    if (ev0) cudaEventRecord(ev0, s);
    for (int g0 = 0; g0 < n_grids; g0 += batch) {
        const int nb = std::min(batch, n_grids - g0);
        bool done = false;
        if constexpr (std::is_same<T, float>::value) {
            if (spec_ok) {
                for (int pass = 0; pass < 3; ++pass)
                    done = spec_launch_s(pass, g.n[0], nb, P, g0, s) || spec_launch_m(pass, g.n[0], nb, P, g0, s) ||
                           spec_launch_l(pass, g.n[0], nb, P, g0, s);
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

template cudaError_t pairconv_run<float>(const GridGeom&, const FFTTables<float>&, const float*, int, float*,
                                         const PairGrid*, int, cplx<float>*, int, double*, double*, cudaStream_t, int*,
                                         cudaEvent_t, cudaEvent_t);
template cudaError_t pairconv_run<double>(const GridGeom&, const FFTTables<double>&, const double*, int, double*,
                                          const PairGrid*, int, cplx<double>*, int, double*, double*, cudaStream_t,
                                          int*, cudaEvent_t, cudaEvent_t);

}  // namespace lace
