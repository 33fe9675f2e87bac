// Size-specialised FP32 FFT passes of the pair convolutions, out-of-place
// form.  Same three passes and the same arithmetic as pairconv_spec.cuh
// (Eq. 2 evaluated with FFTs, Sec. 2; truncated by Eq. 5), laid out for
// fewer barriers and more memory-level parallelism:
//   * every radix stage reads one shared-memory plane and writes the other
//     (ping-pong), so a thread keeps one butterfly live and a stage ends in
//     one barrier instead of two;
//   * pass A forms rho = w_i psi_j with 16-byte loads into the second
//     plane buffer; the first stage of pass B loads its butterflies straight
//     from global memory, and the last stage of passes A and B stores
//     straight to global memory;
//   * pass B runs the forward x-FFT as decimation in time and the inverse as
//     decimation in frequency, so the second forward stage, the product
//     with K(G)/Ng and the first inverse stage act on the same registers:
//     for n = A*B (A = r2, B = r1), x index n1 + A n2 and k index k2 + B k1,
//       X[k2 + B k1] = sum_n1 w_A^{n1 k1} w_N^{n1 k2} sum_n2 w_B^{n2 k2} x[n1 + A n2]
//       x[n1 + A n2] = sum_k2 w_B^{-n2 k2} w_N^{-n1 k2} sum_k1 w_A^{-n1 k1} Y[k2 + B k1]
//     and a group of fixed k2 is one forward and one inverse butterfly.
//     Pass B needs two barriers; its slab of the K(G)/Ng table is staged in
//     shared memory by cp.async while the first stage runs;
//   * passes A and C launch plane-major (the CTAs in flight share one plane
//     of the orbitals and of W, which then stay in L2), and every CTA
//     prefetches into L2 what the CTA one wave ahead will read;
//   * each hand-off between two stages picks the row pitch (n or n + 1
//     complex values) that keeps the 8-byte accesses of a half-warp on
//     distinct banks for both stages, found with a bank model of every
//     stage's addresses;
//   * threads and the register cap are sized so that two CTAs share an SM
//     where shared memory allows (the register file is split over the SM's
//     four sub-partitions);
//   * the butterflies keep each complex value's real and imaginary parts in
//     one register pair, so complex additions and products with real
//     constants are single packed FP32 instructions (dft_packed.cuh).
#pragma once

#include <atomic>
#include <cstdlib>

#include "dft_packed.cuh"
#include "pairconv_spec.cuh"

namespace lace {
namespace spec2 {

using C = float2;
using spec::plan2;
using spec::Plan2;

// Dynamic shared memory: two complex planes (rows padded to n + 1 in passes
// A and C), the twiddle table and (pass B) the |G|^2 tables of x and z.
__host__ __device__ constexpr size_t smem_bytes_b(int n, bool kslab) {
    return sizeof(C) * (2 * (size_t)n * n + n) + 2 * sizeof(float) * n + (kslab ? sizeof(float) * n * n : 0);
}
// Pass B stages its slab of the K(G)/Ng table in shared memory (16-byte
// copies of table rows: n % 4 == 0) when two CTAs an SM still fit, or when
// the planes leave room for one CTA only and the slab fits beside them.
__host__ __device__ constexpr bool kslab_fits(int n) {
    if (n % 4 != 0) return false;
    const size_t plane_ac = sizeof(C) * (2 * (size_t)n * (n + 1) + n);
    const size_t without = plane_ac > smem_bytes_b(n, false) ? plane_ac : smem_bytes_b(n, false);
    const bool one_cta = 2 * (without + 1024) > 227 * 1024;
    return 2 * (smem_bytes_b(n, true) + 1024) <= 227 * 1024 || (one_cta && smem_bytes_b(n, true) + 1024 <= 227 * 1024);
}
__host__ __device__ constexpr size_t smem_bytes(int n, int pass) {
    return pass == 1 ? smem_bytes_b(n, kslab_fits(n)) : sizeof(C) * (2 * (size_t)n * (n + 1) + n);
}
__host__ __device__ constexpr size_t smem_max(int n) {
    return smem_bytes(n, 0) > smem_bytes(n, 1) ? smem_bytes(n, 0) : smem_bytes(n, 1);
}

// Registers a thread may use when m CTAs of nt threads share an SM: the
// register file is split over the SM's four sub-partitions (16K registers
// each), every warp takes its registers from one of them, and a thread's
// count is a multiple of 8.
__host__ __device__ constexpr int regs_at(int nt, int m) {
    const int warps = (nt + 31) / 32;
    const int per_part = (m * warps + 3) / 4;
    const int r = 16384 / (per_part * 32) / 8 * 8;
    return r > 255 ? 255 : r;
}

// CTAs of nt threads per SM with at least 48 registers a thread, within the
// shared memory (227 KB, 1 KB reserved per CTA) and 2048 threads of an SM.
__host__ __device__ constexpr int blocks_at(int n, int nt) {
    int m = (int)((227u * 1024u) / (smem_max(n) + 1024));
    const int by_thr = 2048 / ((nt + 31) / 32 * 32);
    if (m > by_thr) m = by_thr;
    while (m > 1 && regs_at(nt, m) < 48) --m;
    return m < 1 ? 1 : m;
}

// Threads per CTA: one butterfly per thread in the stage with the most
// butterflies, or in the one with the fewest when that is what lets two
// CTAs share an SM (the larger stage then takes a second round), or when one
// CTA fills the SM either way and the fewer threads take no more rounds (at
// 96^3: 768 threads, 2.5 % faster than 1024); at most 1024.
__host__ __device__ constexpr int threads_for(int n) {
    const Plan2 p = plan2(n);
    const int a = n * (n / p.r1), b = n * (n / p.r2);
    int hi = a > b ? a : b, lo = a > b ? b : a;
    hi = (hi + 31) / 32 * 32;
    lo = (lo + 31) / 32 * 32;
    if (hi > 1024) hi = 1024;
    if (lo > 1024) lo = 1024;
    if (blocks_at(n, hi) >= 2) return hi;
    if (blocks_at(n, lo) >= 2) return lo;
    const int r_hi = (a + hi - 1) / hi + (b + hi - 1) / hi, r_lo = (a + lo - 1) / lo + (b + lo - 1) / lo;
    return r_lo <= r_hi ? lo : hi;
}

// Register cap of the passes.
__host__ __device__ constexpr int max_regs(int n) { return regs_at(threads_for(n), blocks_at(n, threads_for(n))); }

// Row pitch (n or n + 1 complex values) of the shared-memory plane handed
// from one stage to the next: hand-offs 0-2 are pass A's stages 1->2, 2->3,
// 3->4, hand-offs 3-5 pass C's.  Chosen per size with a model of the 8-byte
// accesses of every stage (a half-warp's 16 addresses on 16 8-byte bank
// slots; a pitch that sends two of them to one slot costs a second
// wavefront): bit h set = pitch n + 1 for hand-off h.  Pass C's z stages run
// line-fast (consecutive threads on consecutive rows), so their rows need
// the odd pitch; line-fast y stages (consecutive threads along a row) want
// the plain one.
__host__ __device__ constexpr int pad_mask(int n) {
    switch (n) {
        case 24: case 36: case 50: case 54: case 60: return (1 << 4) | (1 << 5);
        case 72: return (1 << 1) | (1 << 4) | (1 << 5);
        case 100: return (1 << 0) | (1 << 1) | (1 << 4) | (1 << 5);
        default: return (1 << 0) | (1 << 4) | (1 << 5);  // 32, 40, 48, 64, 80, 96
    }
}
__host__ __device__ constexpr int pitch(int n, int h) { return (pad_mask(n) >> h) & 1 ? n + 1 : n; }

// The threads that run one pass body: the whole CTA (barrier 0), or one
// group of NT consecutive threads (whole warps) of a larger CTA with a named
// barrier of its own, so that several groups of one CTA work on different
// planes or slabs at once.  Every thread of a group takes the same sequence
// of barriers: the bodies' control flow around sync() is uniform.
struct Cta {
    __device__ __forceinline__ int tid() const { return (int)threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
template <int NT>
struct Sub {
    static_assert(NT % 32 == 0, "a group is whole warps");
    int t;   // thread index in the group
    int id;  // named barrier, 1..15
    __device__ __forceinline__ int tid() const { return t; }
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory"); }
};

// Hint: fetch bytes (a multiple of 16, 16-byte aligned) at p into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The CTA pf_ahead launch positions after this one, if any: its
// blockIdx.x (fast) and blockIdx.y (slow).
__device__ __forceinline__ bool ahead_cta(int pf_ahead, int& fast, int& slow) {
    if (pf_ahead <= 0) return false;
    const long lin = (long)blockIdx.y * gridDim.x + blockIdx.x + pf_ahead;
    if (lin >= (long)gridDim.x * gridDim.y) return false;
    fast = (int)(lin % gridDim.x);
    slow = (int)(lin / gridDim.x);
    return true;
}

// The buffers of grid g of a launch: its own system's in a merged launch
// (the request server), the launch's otherwise.
struct GridView {
    const float* psi;
    float* W;
    const float* ktab;
    C* scr;      // this grid's complex scratch grid
    double* ep;  // this grid's energy partials [n1][2]
    PairGrid d;
    int n_occ;
    double dv;
};
__device__ __forceinline__ GridView grid_view(const ConvArgs<float>& P, int g0, int g, int n1) {
    GridView v;
    if (P.refs) {
        const GridRef r = P.refs[g0 + g];
        const MergedSys<float>& m = P.msys[r.sys];
        v.psi = m.psi;
        v.W = m.W;
        v.ktab = m.ktab;
        v.d = m.grids[r.g];
        v.scr = m.scratch + (size_t)(r.g - m.g0) * P.ng;
        v.ep = m.epart + (size_t)(r.g - m.g0) * n1 * 2;
        v.n_occ = m.n_occ;
        v.dv = m.dv;
    } else {
        v.psi = P.psi;
        v.W = P.W;
        v.ktab = P.ktab;
        v.d = P.grids[g0 + g];
        v.scr = P.scratch + (size_t)g * P.ng;
        v.ep = P.epart + (size_t)g * n1 * 2;
        v.n_occ = P.n_occ;
        v.dv = P.dv;
    }
    return v;
}

// One radix-R Stockham stage over LINES lines of length N, out of place, on
// NT threads (tid: this thread's index among them): butterfly i of a line
// reads elements i + t N/R through ld(line, e), multiplies by w_{P R}^{t k}
// (k = i mod P), runs DFT_R and writes element (i - k) R + k + s P through
// st(line, e, v).  LF: consecutive threads take consecutive lines (else
// consecutive butterflies of one line).
template <int N, int R, int P, int DIR, int LINES, bool LF, int NT, class Ld, class St>
__device__ __forceinline__ void stage(int tid, const C* __restrict__ tw, Ld ld, St st) {
    constexpr int TN = N / R;
    constexpr int ITEMS = LINES * TN;
    constexpr int TWSTEP = N / (P * R);
#pragma unroll
    for (int item0 = 0; item0 < ITEMS; item0 += NT) {
        const int item = item0 + tid;
        if (item0 + NT <= ITEMS || item < ITEMS) {
            const int line = LF ? item % LINES : item / TN;
            const int i = LF ? item / LINES : item % TN;
            C v[R];
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = ld(line, i + t * TN);
            const int k = P > 1 ? i % P : 0;
            if (P > 1) {
#pragma unroll
                for (int t = 1; t < R; ++t) {
                    C w = tw[t * k * TWSTEP];
                    if (DIR > 0) w.y = -w.y;
                    v[t] = cmul(v[t], w);
                }
            }
            fx::FDFT<R, DIR>::run(v);
            const int base = (i - k) * R + k;
#pragma unroll
            for (int s = 0; s < R; ++s) st(line, base + s * P, v[s]);
        }
    }
}

// Pass A, one plane: rho of plane x of grid V, forward FFT along z then y,
// on the NT threads of grp (the thread block, or a group of it).  pf_plane: an orbital plane to fetch into
// L2 at the end (or null).
template <int N, int NT, class G = Cta>
__device__ __forceinline__ void body_a(const ConvArgs<float>& P, const GridView& V, int x, float4* smem_v4,
                                       const float* pf_plane, G grp = G()) {
    const int tid = grp.tid();
    static_assert(N % 2 == 0, "pass A reads orbital planes as 16-byte vectors");
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int LP = N + 1;  // buffer rows hold up to n + 1 complex values
    constexpr int P01 = pitch(N, 0), P12 = pitch(N, 1), P23 = pitch(N, 2);
    C* b0 = reinterpret_cast<C*>(smem_v4);
    C* b1 = b0 + N * LP;
    C* tw = b1 + N * LP;
    const PairGrid d = V.d;
    for (int i = tid; i < N; i += NT) tw[i] = P.tw[2][i];
    const size_t off = (size_t)x * NP;
    const bool two = d.j2 >= 0;
    const float* a1 = V.psi + (size_t)d.i1 * P.ng + off;
    const float* c1 = V.psi + (size_t)d.j1 * P.ng + off;
    const float* a2 = V.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off;
    const float* c2 = V.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off;
    // rho of the plane into b1 (pitch n) with 16-byte loads, four points a
    // thread (one load instruction per orbital per four points; n is even, so
    // every plane starts on a 16-byte boundary), then the z lines (line = y)
    {
        const float4* A1 = reinterpret_cast<const float4*>(a1);
        const float4* C1 = reinterpret_cast<const float4*>(c1);
        const float4* A2 = reinterpret_cast<const float4*>(a2);
        const float4* C2 = reinterpret_cast<const float4*>(c2);
        float4* r4 = reinterpret_cast<float4*>(b1);
        for (int e = tid; e < NP / 4; e += NT) {
            const float4 x1 = __ldg(A1 + e), y1 = __ldg(C1 + e);
            float4 x2 = make_float4(0.f, 0.f, 0.f, 0.f), y2 = x2;
            if (two) {
                x2 = __ldg(A2 + e);
                y2 = __ldg(C2 + e);
            }
            const float4 lo = make_float4(x1.x * y1.x, x2.x * y2.x, x1.y * y1.y, x2.y * y2.y);
            const float4 hi = make_float4(x1.z * y1.z, x2.z * y2.z, x1.w * y1.w, x2.w * y2.w);
            // each thread writes 32 bytes; threads 4-7 of every 8 write their
            // upper half first, so each store instruction's 8-thread phases
            // cover all eight 16-byte bank groups
            const bool sw = (tid >> 2) & 1;
            r4[2 * e + sw] = sw ? hi : lo;
            r4[2 * e + 1 - sw] = sw ? lo : hi;
        }
    }
    grp.sync();
    stage<N, pl.r1, 1, -1, N, false, NT>(
        tid, tw, [&](int y, int z) { return b1[y * N + z]; }, [&](int y, int z, C v) { b0[y * P01 + z] = v; });
    grp.sync();
    stage<N, pl.r2, pl.r1, -1, N, false, NT>(
        tid, tw, [&](int y, int z) { return b0[y * P01 + z]; }, [&](int y, int z, C v) { b1[y * P12 + z] = v; });
    grp.sync();
    // y lines (line = z)
    stage<N, pl.r1, 1, -1, N, true, NT>(
        tid, tw, [&](int z, int y) { return b1[y * P12 + z]; }, [&](int z, int y, C v) { b0[y * P23 + z] = v; });
    grp.sync();
    C* out = V.scr + off;
    stage<N, pl.r2, pl.r1, -1, N, true, NT>(
        tid, tw, [&](int z, int y) { return b0[y * P23 + z]; }, [&](int z, int y, C v) { out[y * N + z] = v; });
    if (pf_plane) prefetch_l2(pf_plane, NP * sizeof(float));
}

// Pass A: rho of plane x, forward FFT along z then y.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N)) pass_a(ConvArgs<float> P, int g0) {
    extern __shared__ float4 smem_v4[];
    const int g = blockIdx.x, x = blockIdx.y;  // plane-major: the CTAs in flight share plane x
    const GridView V = grid_view(P, g0, g, N);
    int xa = 0, ga = 0;
    const float* pf_plane = nullptr;  // orbital plane of the CTA ahead that this thread prefetches
    if (threadIdx.x < 4 && ahead_cta(P.pf_ahead, ga, xa)) {
        const GridView A = grid_view(P, g0, ga, N);
        const int o = threadIdx.x == 0 ? A.d.i1 : threadIdx.x == 1 ? A.d.j1 : threadIdx.x == 2 ? A.d.i2 : A.d.j2;
        if (o >= 0) pf_plane = A.psi + (size_t)o * P.ng + (size_t)xa * N * N;  // (j2 < 0: one pair)
    }
    body_a<N, threads_for(N)>(P, V, x, smem_v4, pf_plane);
}

// Pass B, one slab: slab ky of grid V: forward x-FFT (decimation in time),
// * K(G)/Ng, inverse x-FFT (decimation in frequency); the middle three steps
// share registers.  The NT threads of grp.
template <int N, int NT, class G = Cta>
__device__ __forceinline__ void body_b(const ConvArgs<float>& P, const GridView& V, int ky, float4* smem_v4,
                                       G grp = G()) {
    const int tid = grp.tid();
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int RB = pl.r2, RA = pl.r1;  // N = RA * RB; the middle (the heaviest step) takes the stage with fewer butterflies
    constexpr bool KS = kslab_fits(N);
    C* b0 = reinterpret_cast<C*>(smem_v4);
    C* b1 = b0 + NP;
    float* ks = reinterpret_cast<float*>(b1 + NP);  // K(G)/Ng of this slab, [x][z] (KS)
    C* tw = reinterpret_cast<C*>(ks + (KS ? NP : 0));
    float* gx2 = reinterpret_cast<float*>(tw + N);
    float* gz2 = gx2 + N;
    const float* ktab = V.ktab;
    const bool kstage = KS && ktab != nullptr;
    if (kstage) {
        // asynchronous 16-byte copies, waited for before the middle
        const unsigned ks_s = (unsigned)__cvta_generic_to_shared(ks);
        for (int q = tid; q < NP / 4; q += NT) {
            const int xx = q / (N / 4), z4 = q % (N / 4);
            const float* src = ktab + ((size_t)xx * N + ky) * N + 4 * z4;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ks_s + 16u * q), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = tid; i < N; i += NT) {
        tw[i] = P.tw[0][i];
        gx2[i] = P.g2[0][i];
        gz2[i] = P.g2[2][i];
    }
    C* base = V.scr + (size_t)ky * N;
    // forward stage 1 (line = z): DFT_RB over n2 of x[n1 + RA n2], to y[n1 RB + k2]
    stage<N, RB, 1, -1, N, true, NT>(
        tid, tw, [&](int z, int xx) { return base[(size_t)xx * NP + z]; },
        [&](int z, int xx, C v) { b0[xx * N + z] = v; });
    if (kstage) asm volatile("cp.async.wait_group 0;" ::: "memory");
    grp.sync();
    const float gy2 = P.g2[1][ky];
    // middle: for each (z, k2): twiddle, DFT_RA -> X[k2 + RB k1], * K, inverse
    // DFT_RA -> z[k2][n1], twiddle w_N^{-n1 k2}, stored at n1 RB + k2
    constexpr int MID = N * RB;
#pragma unroll
    for (int item0 = 0; item0 < MID; item0 += NT) {
        const int item = item0 + tid;
        if (item0 + NT <= MID || item < MID) {
            const int z = item % N, k2 = item / N;
            C v[RA];
#pragma unroll
            for (int t = 0; t < RA; ++t) {
                v[t] = b0[(k2 + t * RB) * N + z];
                if (t > 0) v[t] = cmul(v[t], tw[t * k2]);
            }
            fx::FDFT<RA, -1>::run(v);
#pragma unroll
            for (int s = 0; s < RA; ++s) {
                const int xx = k2 + s * RB;
                float k;
                if (kstage) {
                    k = ks[xx * N + z];
                } else if (ktab) {
                    k = __ldg(ktab + ((size_t)xx * N + ky) * N + z);
                } else {
                    const float gg = gx2[xx] + gy2 + gz2[z];
                    k = gg > 0.f ? P.kscale / gg : 0.f;
                }
                v[s] = C{v[s].x * k, v[s].y * k};
            }
            fx::FDFT<RA, +1>::run(v);
#pragma unroll
            for (int n1 = 0; n1 < RA; ++n1) {
                C w = tw[n1 * k2];
                w.y = -w.y;
                b1[(n1 * RB + k2) * N + z] = n1 > 0 ? cmul(v[n1], w) : v[n1];
            }
        }
    }
    grp.sync();
    // inverse stage 2 (line = z): for each n1, DFT_RB over k2 -> x[n1 + RA n2]
    constexpr int LAST = N * RA;
#pragma unroll
    for (int item0 = 0; item0 < LAST; item0 += NT) {
        const int item = item0 + tid;
        if (item0 + NT <= LAST || item < LAST) {
            const int z = item % N, n1 = item / N;
            C v[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) v[t] = b1[(n1 * RB + t) * N + z];
            fx::FDFT<RB, +1>::run(v);
#pragma unroll
            for (int s = 0; s < RB; ++s) base[(size_t)(n1 + RA * s) * NP + z] = v[s];
        }
    }
}

// Pass B: slab ky: forward x-FFT, * K(G)/Ng, inverse x-FFT.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N)) pass_b(ConvArgs<float> P, int g0) {
    extern __shared__ float4 smem_v4[];
    const int g = blockIdx.y, ky = blockIdx.x;
    const GridView V = grid_view(P, g0, g, N);
    {
        int ka = 0, ga = 0;
        if (threadIdx.x < N && ahead_cta(P.pf_ahead, ka, ga))
            prefetch_l2(grid_view(P, g0, ga, N).scr + (size_t)threadIdx.x * N * N + (size_t)ka * N, N * sizeof(C));
    }
    body_b<N, threads_for(N)>(P, V, ky, smem_v4);
}

// Pass C, one plane: inverse FFT along y then z of plane x of grid V, then
// the W updates (16-byte vector reductions) and the real-space pair
// energies.  The NT threads of grp; red: 2 x (NT / 32) doubles of shared
// memory of its own.
template <int N, int NT, class G = Cta>
__device__ __forceinline__ void body_c(const ConvArgs<float>& P, const GridView& V, int x, float4* smem_v4,
                                       double* red, G grp = G()) {
    const int tid = grp.tid();
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int LP = N + 1;  // buffer rows hold up to n + 1 complex values (the last stage writes pitch n)
    constexpr int P01 = pitch(N, 3), P12 = pitch(N, 4), P23 = pitch(N, 5);
    C* b0 = reinterpret_cast<C*>(smem_v4);
    C* b1 = b0 + N * LP;
    C* tw = b1 + N * LP;
    constexpr int NW = (NT + 31) / 32;
    const PairGrid d = V.d;
    for (int i = tid; i < N; i += NT) tw[i] = P.tw[2][i];
    const size_t off = (size_t)x * NP;
    const C* in = V.scr + off;
    stage<N, pl.r1, 1, +1, N, true, NT>(
        tid, tw, [&](int z, int y) { return in[y * N + z]; }, [&](int z, int y, C v) { b0[y * P01 + z] = v; });
    if (P.pf_ahead > 0 && tid < 8) {
        // the epilogue's orbital planes and W planes, fetched into L2 while
        // the FFT stages run
        const int q = tid & 3;
        const int o = q == 0 ? d.i1 : q == 1 ? d.j1 : q == 2 ? d.i2 : d.j2;
        if (o >= 0) {
            const float* src = (tid < 4 ? V.psi : V.W) + (size_t)o * P.ng + off;
            prefetch_l2(src, NP * sizeof(float));
        }
    }
    grp.sync();
    stage<N, pl.r2, pl.r1, +1, N, true, NT>(
        tid, tw, [&](int z, int y) { return b0[y * P01 + z]; }, [&](int z, int y, C v) { b1[y * P12 + z] = v; });
    grp.sync();
    // z lines (line = y)
    stage<N, pl.r1, 1, +1, N, true, NT>(
        tid, tw, [&](int y, int z) { return b1[y * P12 + z]; }, [&](int y, int z, C v) { b0[y * P23 + z] = v; });
    grp.sync();
    stage<N, pl.r2, pl.r1, +1, N, false, NT>(
        tid, tw, [&](int y, int z) { return b0[y * P23 + z]; }, [&](int y, int z, C v) { b1[y * N + z] = v; });
    grp.sync();
    const bool two = d.j2 >= 0;
    const bool a_occ = d.j1 < V.n_occ, a_sym = a_occ && d.j1 != d.i1;
    const bool b_occ = two && d.j2 < V.n_occ, b_sym = b_occ && d.j2 != d.i2;
    const float4* wi1 = reinterpret_cast<const float4*>(V.psi + (size_t)d.i1 * P.ng + off);
    const float4* pj1 = reinterpret_cast<const float4*>(V.psi + (size_t)d.j1 * P.ng + off);
    float4* Wj1 = reinterpret_cast<float4*>(V.W + (size_t)d.j1 * P.ng + off);
    float4* Wi1 = reinterpret_cast<float4*>(V.W + (size_t)d.i1 * P.ng + off);
    const float4* wi2 = reinterpret_cast<const float4*>(V.psi + (size_t)(two ? d.i2 : d.i1) * P.ng + off);
    const float4* pj2 = reinterpret_cast<const float4*>(V.psi + (size_t)(two ? d.j2 : d.j1) * P.ng + off);
    float4* Wj2 = reinterpret_cast<float4*>(V.W + (size_t)(two ? d.j2 : d.j1) * P.ng + off);
    float4* Wi2 = reinterpret_cast<float4*>(V.W + (size_t)(two ? d.i2 : d.i1) * P.ng + off);
    const bool merge_i = two && a_sym && b_sym && d.i1 == d.i2;
    const float4* pl4 = reinterpret_cast<const float4*>(b1);
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
#pragma unroll
    for (int e0 = 0; e0 < NP / 4; e0 += NT) {
        const int e = e0 + tid;
        if (e0 + NT <= NP / 4 || e < NP / 4) {
            // 32 bytes a thread, read in the bank-group order of pass A's rho stores
            const bool sw = (tid >> 2) & 1;
            const float4 p0 = pl4[2 * e + sw], p1 = pl4[2 * e + 1 - sw];
            const float4 v01 = sw ? p1 : p0, v23 = sw ? p0 : p1;
            const float4 x1 = __ldg(wi1 + e), y1 = __ldg(pj1 + e);
            atomicAdd(Wj1 + e, make_float4(-x1.x * v01.x, -x1.y * v01.z, -x1.z * v23.x, -x1.w * v23.z));
            const float4 wi_acc = make_float4(-y1.x * v01.x, -y1.y * v01.z, -y1.z * v23.x, -y1.w * v23.z);
            if (a_sym && !merge_i) atomicAdd(Wi1 + e, wi_acc);
            if (a_occ)
                spec::kahan(sa, ca,
                            x1.x * y1.x * v01.x + x1.y * y1.y * v01.z + x1.z * y1.z * v23.x + x1.w * y1.w * v23.z);
            if (two) {
                const float4 x2 = merge_i ? x1 : __ldg(wi2 + e);
                const float4 y2 = __ldg(pj2 + e);
                atomicAdd(Wj2 + e, make_float4(-x2.x * v01.y, -x2.y * v01.w, -x2.z * v23.y, -x2.w * v23.w));
                const float4 w2 = make_float4(-y2.x * v01.y, -y2.y * v01.w, -y2.z * v23.y, -y2.w * v23.w);
                if (merge_i) {
                    atomicAdd(Wi1 + e,
                              make_float4(wi_acc.x + w2.x, wi_acc.y + w2.y, wi_acc.z + w2.z, wi_acc.w + w2.w));
                } else if (b_sym) {
                    atomicAdd(Wi2 + e, w2);
                }
                if (b_occ)
                    spec::kahan(sb, cb,
                                x2.x * y2.x * v01.y + x2.y * y2.y * v01.w + x2.z * y2.z * v23.y + x2.w * y2.w * v23.w);
            }
        }
    }
    sa -= ca;
    sb -= cb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) { red[warp] = (double)sa; red[NW + warp] = (double)sb; }
    grp.sync();
    static_assert(NW <= 32, "one warp sums the warp partials");
    if (warp == 0) {
        // the warp partials in FP64 across the lanes of one warp (a short
        // chain: FP64 issues slowly, and one thread summing them serially
        // held the CTA's slot)
        double ta = lane < NW ? red[lane] : 0.0, tbb = lane < NW ? red[NW + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_xor_sync(0xffffffffu, ta, o);
            tbb += __shfl_xor_sync(0xffffffffu, tbb, o);
        }
        if (lane == 0) {
            double* ep = V.ep + (size_t)x * 2;
            ep[0] = ta * V.dv;
            ep[1] = tbb * V.dv;
        }
    }
}

// Pass C: inverse FFT along y then z of plane x, W updates and pair energies.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N)) pass_c(ConvArgs<float> P, int g0) {
    extern __shared__ float4 smem_v4[];
    __shared__ double red[2 * ((threads_for(N) + 31) / 32)];
    const int g = blockIdx.x, x = blockIdx.y;  // plane-major: the CTAs in flight share plane x
    const GridView V = grid_view(P, g0, g, N);
    {
        int xa = 0, ga = 0;
        if (threadIdx.x == 32 && ahead_cta(P.pf_ahead, ga, xa))
            prefetch_l2(grid_view(P, g0, ga, N).scr + (size_t)xa * N * N, N * N * sizeof(C));
    }
    body_c<N, threads_for(N)>(P, V, x, smem_v4, red);
}

// Launch pass 0/1/2 of a batch of nb complex grids.
template <int N>
bool launch_one(int pass, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    static std::atomic<unsigned long long> attr_done{0};  // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !(attr_done.load() & (1ull << dev))) {
        cudaFuncSetAttribute(pass_a<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(N, 0));
        cudaFuncSetAttribute(pass_b<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(N, 1));
        cudaFuncSetAttribute(pass_c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(N, 2));
        cudaFuncSetAttribute(pass_a<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(pass_b<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaFuncSetAttribute(pass_c<N>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        attr_done.fetch_or(1ull << dev);
    }
    const size_t sm = smem_bytes(N, pass);
    constexpr int NT = threads_for(N);
    if (pass == 0) pass_a<N><<<dim3(nb, N), NT, sm, s>>>(P, g0);
    else if (pass == 1) pass_b<N><<<dim3(N, nb), NT, sm, s>>>(P, g0);
    else pass_c<N><<<dim3(nb, N), NT, sm, s>>>(P, g0);
    return true;
}

// LACE_FFT_INPLACE=1 selects the in-place passes of pairconv_spec.cuh (kept
// for comparison and for grids whose two planes do not fit on chip).
inline bool enabled() {
    static const int on = [] {
        const char* e = getenv("LACE_FFT_INPLACE");
        return (e && e[0] == '1') ? 0 : 1;
    }();
    return on != 0;
}

}  // namespace spec2

namespace spec {

// The out-of-place passes where two planes fit in shared memory, else the
// in-place ones.  A merged launch (several systems, P.refs) takes the
// out-of-place passes or none.
template <int N>
bool launch_any(int pass, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s) {
    if constexpr (spec2::smem_max(N) <= 200 * 1024) {
        // merged launches (P.refs) exist only in the one-grid out-of-place passes
        if (spec2::enabled() || P.refs) return spec2::launch_one<N>(pass, nb, P, g0, s);
    }
    if (P.refs) return false;
    // the in-place passes read rows as 16-byte vectors: n % 4 == 0 only
    if constexpr (N % 4 == 0) return spec_launch_one<N>(pass, nb, P, g0, s);
    return false;
}

}  // namespace spec
}  // namespace lace
