// Size-specialised FP32 FFT passes of the pair convolutions for cubic grids
// n x n x n with n % 4 == 0.  Same three passes as pairconv.cu (Eq. 2 via
// FFTs, truncated by Eq. 5), but the radix plan, the thread count and every
// index are compile-time constants: each Stockham stage is one round of
// register-held butterflies, orbital reads and W updates are 16-byte vectors.
#pragma once

#include <atomic>
#include "lace_internal.cuh"

namespace lace {
namespace spec {

using C = float2;

struct Plan2 {
    int r1, r2;
};

__host__ __device__ constexpr bool radix_ok(int r) {
    return r == 2 || r == 3 || r == 4 || r == 5 || r == 6 || r == 8 || r == 9 || r == 10 || r == 12 || r == 16;
}

// Two register radices r1 * r2 = n with the largest smaller factor.
__host__ __device__ constexpr Plan2 plan2(int n) {
    Plan2 best{0, 0};
    int best_min = 0;
    for (int r1 = 16; r1 >= 2; --r1) {
        if (!radix_ok(r1) || n % r1) continue;
        const int r2 = n / r1;
        if (!radix_ok(r2)) continue;
        const int mn = r1 < r2 ? r1 : r2;
        if (mn > best_min) {
            best_min = mn;
            best = Plan2{r1, r2};
        }
    }
    return best;
}

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Threads per CTA: enough for one round of each stage with at most 16 complex
// values per thread held across the barrier.
__host__ __device__ constexpr int threads_for(int n) {
    const Plan2 p = plan2(n);
    const int a = n * (n / p.r1), b = n * (n / p.r2);
    const int ma = cmax(1, 16 / p.r1), mb = cmax(1, 16 / p.r2);
    int t = cmax((a + ma - 1) / ma, (b + mb - 1) / mb);
    t = (t + 31) / 32 * 32;
    return t > 1024 ? 1024 : t;
}

// One radix-R Stockham stage (same algorithm as fft_stage in common.cuh) on
// LINES lines of length N: line l, element e at buf[l*LP + e*ES].
template <int N, int R, int P, int DIR, int LINES, int LP, int ES, bool LF, int NT>
__device__ __forceinline__ void stage(C* __restrict__ buf, const C* __restrict__ tw) {
    constexpr int TN = N / R;
    constexpr int ITEMS = LINES * TN;
    constexpr int ROUNDS = (ITEMS + NT - 1) / NT;
    constexpr int TWSTEP = N / (P * R);
    C v[ROUNDS][R];
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int item = threadIdx.x + r * NT;
        if (ROUNDS * NT == ITEMS || item < ITEMS) {
            const int line = LF ? item % LINES : item / TN;
            const int i = LF ? item / LINES : item % TN;
            const C* src = buf + line * LP;
#pragma unroll
            for (int t = 0; t < R; ++t) v[r][t] = src[(i + t * TN) * ES];
            if (P > 1) {
                const int k = i % P;
#pragma unroll
                for (int t = 1; t < R; ++t) {
                    C w = tw[t * k * TWSTEP];
                    if (DIR > 0) w.y = -w.y;
                    v[r][t] = cmul(v[r][t], w);
                }
            }
            DFT<R, DIR>::run(v[r]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int item = threadIdx.x + r * NT;
        if (ROUNDS * NT == ITEMS || item < ITEMS) {
            const int line = LF ? item % LINES : item / TN;
            const int i = LF ? item / LINES : item % TN;
            const int k = i % P;
            C* dst = buf + line * LP;
            const int base = (i - k) * R + k;
#pragma unroll
            for (int s = 0; s < R; ++s) dst[(base + s * P) * ES] = v[r][s];
        }
    }
    __syncthreads();
}

// Full length-N FFT of LINES lines (two register stages).
template <int N, int DIR, int LINES, int LP, int ES, bool LF, int NT>
__device__ __forceinline__ void lines_fft(C* buf, const C* tw) {
    constexpr Plan2 pl = plan2(N);
    stage<N, pl.r1, 1, DIR, LINES, LP, ES, LF, NT>(buf, tw);
    stage<N, pl.r2, pl.r1, DIR, LINES, LP, ES, LF, NT>(buf, tw);
}

__device__ __forceinline__ void kahan(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Pass A: rho of plane x, forward FFT along z then y.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) spec_pass_a(ConvArgs<float> P, int g0) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    extern __shared__ float4 smem_v4[];
    C* plane = reinterpret_cast<C*>(smem_v4);
    C* tw = plane + NP;
    const int g = blockIdx.y, x = blockIdx.x;
    const PairGrid d = P.grids[g0 + g];
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = P.tw[2][i];
    const size_t off = (size_t)x * NP;
    const bool two = d.j2 >= 0;
    const float4* a1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.i1 * P.ng + off);
    const float4* b1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.j1 * P.ng + off);
    const float4* a2 = reinterpret_cast<const float4*>(P.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off);
    const float4* b2 = reinterpret_cast<const float4*>(P.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off);
    float4* pl4 = reinterpret_cast<float4*>(plane);
    const bool same_i = two && d.i1 == d.i2;
    for (int e = threadIdx.x; e < NP / 4; e += NT) {
        const float4 x1 = __ldg(a1 + e), y1 = __ldg(b1 + e);
        float4 x2 = make_float4(0.f, 0.f, 0.f, 0.f), y2 = x2;
        if (two) { x2 = same_i ? x1 : __ldg(a2 + e); y2 = __ldg(b2 + e); }
        pl4[2 * e] = make_float4(x1.x * y1.x, x2.x * y2.x, x1.y * y1.y, x2.y * y2.y);
        pl4[2 * e + 1] = make_float4(x1.z * y1.z, x2.z * y2.z, x1.w * y1.w, x2.w * y2.w);
    }
    __syncthreads();
    lines_fft<N, -1, N, N, 1, false, NT>(plane, tw);  // z
    lines_fft<N, -1, N, 1, N, true, NT>(plane, tw);   // y
    float4* out = reinterpret_cast<float4*>(P.scratch + (size_t)g * P.ng + off);
    for (int e = threadIdx.x; e < NP / 2; e += NT) out[e] = pl4[e];
}

// Pass B: slab ky: FFT along x, * K(G)/Ng, inverse FFT along x.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) spec_pass_b(ConvArgs<float> P, int g0) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    extern __shared__ float4 smem_v4[];
    C* slab = reinterpret_cast<C*>(smem_v4);
    C* tw = slab + NP;
    float* gx2 = reinterpret_cast<float*>(tw + N);
    float* gz2 = gx2 + N;
    const int g = blockIdx.y, ky = blockIdx.x;
    for (int i = threadIdx.x; i < N; i += NT) {
        tw[i] = P.tw[0][i];
        gx2[i] = P.g2[0][i];
        gz2[i] = P.g2[2][i];
    }
    C* base = P.scratch + (size_t)g * P.ng + (size_t)ky * N;
    float4* sl4 = reinterpret_cast<float4*>(slab);
    for (int e = threadIdx.x; e < NP / 2; e += NT) {
        const int xx = e / (N / 2), zz = e % (N / 2);
        sl4[e] = reinterpret_cast<const float4*>(base + (size_t)xx * NP)[zz];
    }
    __syncthreads();
    lines_fft<N, -1, N, 1, N, true, NT>(slab, tw);
    const float gy2 = P.g2[1][ky];
    for (int e = threadIdx.x; e < NP; e += NT) {
        const int xx = e / N, zz = e % N;
        float k;
        if (P.ktab) {
            k = __ldg(P.ktab + ((size_t)xx * N + ky) * N + zz);
        } else {
            const float gg = gx2[xx] + gy2 + gz2[zz];
            k = gg > 0.f ? P.kscale / gg : 0.f;
        }
        C v = slab[e];
        slab[e] = C{v.x * k, v.y * k};
    }
    __syncthreads();
    lines_fft<N, +1, N, 1, N, true, NT>(slab, tw);
    for (int e = threadIdx.x; e < NP / 2; e += NT) {
        const int xx = e / (N / 2), zz = e % (N / 2);
        reinterpret_cast<float4*>(base + (size_t)xx * NP)[zz] = sl4[e];
    }
    (void)g0;
}

// Pass C: inverse 2D FFT of plane x, W updates (16-byte vector reductions)
// and the real-space pair energies.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) spec_pass_c(ConvArgs<float> P, int g0) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    extern __shared__ float4 smem_v4[];
    C* plane = reinterpret_cast<C*>(smem_v4);
    C* tw = plane + NP;
    __shared__ double red[2][NT / 32];
    const int g = blockIdx.y, x = blockIdx.x;
    const PairGrid d = P.grids[g0 + g];
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = P.tw[2][i];
    const size_t off = (size_t)x * NP;
    const float4* in = reinterpret_cast<const float4*>(P.scratch + (size_t)g * P.ng + off);
    float4* pl4 = reinterpret_cast<float4*>(plane);
    for (int e = threadIdx.x; e < NP / 2; e += NT) pl4[e] = in[e];
    __syncthreads();
    lines_fft<N, +1, N, 1, N, true, NT>(plane, tw);   // y
    lines_fft<N, +1, N, N, 1, false, NT>(plane, tw);  // z
    const bool two = d.j2 >= 0;
    const bool a_occ = d.j1 < P.n_occ, a_sym = a_occ && d.j1 != d.i1;
    const bool b_occ = two && d.j2 < P.n_occ, b_sym = b_occ && d.j2 != d.i2;
    const float4* wi1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.i1 * P.ng + off);
    const float4* pj1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.j1 * P.ng + off);
    float4* Wj1 = reinterpret_cast<float4*>(P.W + (size_t)d.j1 * P.ng + off);
    float4* Wi1 = reinterpret_cast<float4*>(P.W + (size_t)d.i1 * P.ng + off);
    const float4* wi2 = reinterpret_cast<const float4*>(P.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off);
    const float4* pj2 = reinterpret_cast<const float4*>(P.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off);
    float4* Wj2 = reinterpret_cast<float4*>(P.W + (size_t)(two ? d.j2 : d.j1) * P.ng + off);
    float4* Wi2 = reinterpret_cast<float4*>(P.W + (size_t)(two ? d.i2 : d.i1) * P.ng + off);
    // both slots symmetric with the same occupied i: one reduction into W_i
    const bool merge_i = two && a_sym && b_sym && d.i1 == d.i2;
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    for (int e = threadIdx.x; e < NP / 4; e += NT) {
        const float4 v01 = pl4[2 * e], v23 = pl4[2 * e + 1];  // (re0, im0, re1, im1), (re2, im2, re3, im3)
        const float4 x1 = __ldg(wi1 + e), y1 = __ldg(pj1 + e);
        atomicAdd(Wj1 + e, make_float4(-x1.x * v01.x, -x1.y * v01.z, -x1.z * v23.x, -x1.w * v23.z));
        float4 wi_acc = make_float4(-y1.x * v01.x, -y1.y * v01.z, -y1.z * v23.x, -y1.w * v23.z);
        if (a_sym && !merge_i) atomicAdd(Wi1 + e, wi_acc);
        if (a_occ)
            kahan(sa, ca, x1.x * y1.x * v01.x + x1.y * y1.y * v01.z + x1.z * y1.z * v23.x + x1.w * y1.w * v23.z);
        if (two) {
            const float4 x2 = merge_i ? x1 : __ldg(wi2 + e);
            const float4 y2 = __ldg(pj2 + e);
            atomicAdd(Wj2 + e, make_float4(-x2.x * v01.y, -x2.y * v01.w, -x2.z * v23.y, -x2.w * v23.w));
            const float4 w2 = make_float4(-y2.x * v01.y, -y2.y * v01.w, -y2.z * v23.y, -y2.w * v23.w);
            if (merge_i) {
                atomicAdd(Wi1 + e, make_float4(wi_acc.x + w2.x, wi_acc.y + w2.y, wi_acc.z + w2.z, wi_acc.w + w2.w));
            } else if (b_sym) {
                atomicAdd(Wi2 + e, w2);
            }
            if (b_occ)
                kahan(sb, cb, x2.x * y2.x * v01.y + x2.y * y2.y * v01.w + x2.z * y2.z * v23.y + x2.w * y2.w * v23.w);
        }
    }
    sa -= ca;
    sb -= cb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = (double)sa; red[1][warp] = (double)sb; }
    __syncthreads();
    static_assert(NT / 32 <= 32, "one warp sums the warp partials");
    if (warp == 0) {
        // the warp partials in FP64 across the lanes of one warp (short chain)
        double ta = lane < NT / 32 ? red[0][lane] : 0.0, tbb = lane < NT / 32 ? red[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_xor_sync(0xffffffffu, ta, o);
            tbb += __shfl_xor_sync(0xffffffffu, tbb, o);
        }
        if (lane == 0) {
            double* ep = P.epart + ((size_t)g * gridDim.x + x) * 2;
            ep[0] = ta * P.dv;
            ep[1] = tbb * P.dv;
        }
    }
}

template <int N>
size_t spec_smem(int pass) {
    return sizeof(C) * ((size_t)N * N + N) + (pass == 1 ? 2 * sizeof(float) * N : 0);
}

template <int N>
bool spec_launch_one(int pass, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    static std::atomic<unsigned long long> attr_done{0};  // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !(attr_done.load() & (1ull << dev))) {
        cudaFuncSetAttribute(spec_pass_a<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem<N>(0));
        cudaFuncSetAttribute(spec_pass_b<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem<N>(1));
        cudaFuncSetAttribute(spec_pass_c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spec_smem<N>(2));
        attr_done.fetch_or(1ull << dev);
    }
    const size_t sm = spec_smem<N>(pass);
    const dim3 grid(N, nb);
    constexpr int NT = threads_for(N);
    if (pass == 0) spec_pass_a<N><<<grid, NT, sm, s>>>(P, g0);
    else if (pass == 1) spec_pass_b<N><<<grid, NT, sm, s>>>(P, g0);
    else spec_pass_c<N><<<grid, NT, sm, s>>>(P, g0);
    return true;
}

}  // namespace spec
}  // namespace lace
