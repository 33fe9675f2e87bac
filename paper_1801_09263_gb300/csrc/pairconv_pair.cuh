// Size-specialised FP32 FFT passes of the pair convolutions, two complex
// grids per CTA in packed FP32 pairs.
//
// Same three passes and the same arithmetic as pairconv_spec2.cuh (Eq. 2
// evaluated with FFTs, Sec. 2; truncated by Eq. 5): every complex grid still
// carries two real pair densities (rho_a + i rho_b).  What changes is the
// unit of work of a CTA: complex grids 2p and 2p + 1 of a batch run through
// the passes together.  Their transforms have the same indices, twiddles
// and K(G), so one thread does one butterfly for both, with every value held
// as a pair (grid 2p in the low lane, grid 2p + 1 in the high lane) and
// every addition, multiplication and fused multiply-add issued as one packed
// FP32 instruction of sm_100+ (add/sub/mul/fma .rn.f32x2): the butterfly
// arithmetic, the twiddle and K(G) loads, the shared-memory accesses
// (16-byte {re_a, re_b, im_a, im_b} elements) and the index arithmetic all
// cost half as many instructions per point as one grid at a time.
//
// The passes were instruction-issue bound (about 280 instructions a point
// against an HBM floor near half of that time), so halving the per-point
// instructions is what moves them toward the DRAM roofline.  The scratch
// grids of a pair are stored interleaved, [pair][x][y][z] of 16-byte
// elements, in the memory of grids 2p and 2p + 1.
//
// Layout choices otherwise as in pairconv_spec2.cuh: out-of-place ping-pong
// planes (one barrier a stage), global loads and stores fused into the first
// and last stages, pass B's forward stage / K(G) product / inverse stage in
// registers with its K slab staged by cp.async, plane-major launch order of
// passes A and C, L2 prefetch one wave ahead, odd row pitch for line-fast z
// stages.  Built where two paired planes fit in shared memory (n <= 80); off
// by default (see enabled(): slower than the one-grid passes as measured).
#pragma once

#include <atomic>
#include <cstdlib>

#include "f32x2.cuh"
#include "pairconv_spec2.cuh"

namespace lace {
namespace pair2 {

using spec::Plan2;
using spec::plan2;

// Two complex values: x = (re of grid a, re of grid b), y = (im a, im b).
struct P2 {
    f2 x, y;
};
__device__ __forceinline__ P2 ld2(const ulonglong2* p) {
    const ulonglong2 q = *p;
    return P2{f2{q.x}, f2{q.y}};
}
__device__ __forceinline__ void st2(ulonglong2* p, P2 v) { *p = make_ulonglong2(v.x.v, v.y.v); }
__device__ __forceinline__ P2 padd(P2 a, P2 b) { return P2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ P2 psub(P2 a, P2 b) { return P2{a.x - b.x, a.y - b.y}; }
// a + i S b and a - i S b (S = +-1) without a separate negation
template <int S> __device__ __forceinline__ P2 padd_i(P2 a, P2 b) {
    if constexpr (S > 0) return P2{a.x - b.y, a.y + b.x};
    else return P2{a.x + b.y, a.y - b.x};
}
template <int S> __device__ __forceinline__ P2 psub_i(P2 a, P2 b) { return padd_i<-S>(a, b); }

// Multiply by exp(DIR 2 pi i M / N), compile-time constant; the trivial
// cases need no multiplication and the odd multiples of pi/4 one constant
// product per component.
template <int N, int M, int DIR>
__device__ __forceinline__ P2 ptw_ct(P2 a) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == N) {
        return P2{neg2(a.x), neg2(a.y)};
    } else if constexpr (4 * m == N) {
        if constexpr (DIR > 0) return P2{neg2(a.y), a.x};
        else return P2{a.y, neg2(a.x)};
    } else if constexpr (4 * m == 3 * N) {
        if constexpr (DIR > 0) return P2{a.y, neg2(a.x)};
        else return P2{neg2(a.y), a.x};
    } else if constexpr ((8 * m) % N == 0) {
        // (cx + i ss) h with cx, ss = +-1, r = cx ss:
        // r = +1: (cx h (x - y), cx h (x + y)); r = -1: (cx h (x + y), -cx h (x - y))
        constexpr int e8 = 8 * m / N;
        constexpr int cx = (e8 == 1 || e8 == 7) ? 1 : -1;
        constexpr int ss = DIR * ((e8 == 1 || e8 == 3) ? 1 : -1);
        constexpr double h = 0.707106781186547524400844362104849039;
        const f2 s = a.x + a.y, d = a.x - a.y;
        if constexpr (cx * ss > 0) return P2{mulk2(d, cx * h), mulk2(s, cx * h)};
        else return P2{mulk2(s, cx * h), mulk2(d, -cx * h)};
    } else {
        constexpr double c = ct_cos2pi(m, N);
        constexpr double s = DIR * ct_sin2pi(m, N);
        // (x c - y s, x s + y c), each constant as hi + lo
        return P2{fmak2(a.x, c, mulk2(a.y, -s)), fmak2(a.x, s, mulk2(a.y, c))};
    }
}

// In-register DFTs of packed pairs: X_k = sum_t x_t exp(DIR 2 pi i t k / R).
template <int R, int DIR> struct PDFT;

template <int DIR> struct PDFT<2, DIR> {
    static __device__ __forceinline__ void run(P2* v) {
        const P2 a = v[0], b = v[1];
        v[0] = padd(a, b);
        v[1] = psub(a, b);
    }
};

template <int DIR> struct PDFT<3, DIR> {
    static __device__ __forceinline__ void run(P2* v) {
        constexpr double s3 = 0.866025403784438646763723170752936183;  // sin(2 pi/3)
        const P2 a = v[0], b = v[1], c = v[2];
        const P2 t1 = padd(b, c);
        const f2 mh = bc2(-0.5f);
        const P2 t2 = P2{fma2(t1.x, mh, a.x), fma2(t1.y, mh, a.y)};
        const P2 d = psub(b, c);
        const P2 e = P2{mulk2(d.x, s3), mulk2(d.y, s3)};
        v[0] = padd(a, t1);
        v[1] = padd_i<DIR>(t2, e);
        v[2] = psub_i<DIR>(t2, e);
    }
};

template <int DIR> struct PDFT<4, DIR> {
    static __device__ __forceinline__ void run(P2* v) {
        const P2 a = v[0], b = v[1], c = v[2], d = v[3];
        const P2 s0 = padd(a, c), d0 = psub(a, c);
        const P2 s1 = padd(b, d), e = psub(b, d);
        v[0] = padd(s0, s1);
        v[2] = psub(s0, s1);
        v[1] = padd_i<DIR>(d0, e);
        v[3] = psub_i<DIR>(d0, e);
    }
};

template <int DIR> struct PDFT<5, DIR> {
    static __device__ __forceinline__ void run(P2* v) {
        constexpr double c1 = ct_cos2pi(1, 5), c2 = ct_cos2pi(2, 5);
        constexpr double s1 = ct_sin2pi(1, 5), s2 = ct_sin2pi(2, 5);
        const P2 a = v[0];
        const P2 p1 = padd(v[1], v[4]), m1 = psub(v[1], v[4]);
        const P2 p2 = padd(v[2], v[3]), m2 = psub(v[2], v[3]);
        const P2 r1 = P2{fmak2(p1.x, c1, fmak2(p2.x, c2, a.x)), fmak2(p1.y, c1, fmak2(p2.y, c2, a.y))};
        const P2 r2 = P2{fmak2(p1.x, c2, fmak2(p2.x, c1, a.x)), fmak2(p1.y, c2, fmak2(p2.y, c1, a.y))};
        const P2 q1 = P2{fmak2(m1.x, s1, mulk2(m2.x, s2)), fmak2(m1.y, s1, mulk2(m2.y, s2))};
        const P2 q2 = P2{fmak2(m1.x, s2, mulk2(m2.x, -s1)), fmak2(m1.y, s2, mulk2(m2.y, -s1))};
        v[0] = padd(a, padd(p1, p2));
        v[1] = padd_i<DIR>(r1, q1);
        v[4] = psub_i<DIR>(r1, q1);
        v[2] = padd_i<DIR>(r2, q2);
        v[3] = psub_i<DIR>(r2, q2);
    }
};

// Composite R = A * B in registers (as DFTComposite in common.cuh):
// t = B ta + tb, k = ka + A kb.
template <int R, int A, int TB, int KA, int DIR> struct PCompTw {
    static __device__ __forceinline__ void run(const P2* u, P2* y) {
        y[TB * A + KA] = ptw_ct<R, TB * KA, DIR>(u[KA]);
        PCompTw<R, A, TB, KA + 1, DIR>::run(u, y);
    }
};
template <int R, int A, int TB, int DIR> struct PCompTw<R, A, TB, A, DIR> {
    static __device__ __forceinline__ void run(const P2*, P2*) {}
};
template <int A, int B, int TB, int DIR> struct PCompStep1 {
    static __device__ __forceinline__ void run(const P2* v, P2* y) {
        P2 u[A];
#pragma unroll
        for (int ta = 0; ta < A; ++ta) u[ta] = v[B * ta + TB];
        PDFT<A, DIR>::run(u);
        PCompTw<A * B, A, TB, 0, DIR>::run(u, y);
        PCompStep1<A, B, TB + 1, DIR>::run(v, y);
    }
};
template <int A, int B, int DIR> struct PCompStep1<A, B, B, DIR> {
    static __device__ __forceinline__ void run(const P2*, P2*) {}
};
template <int A, int B, int DIR> struct PDFTComposite {
    static __device__ __forceinline__ void run(P2* v) {
        P2 y[A * B];
        PCompStep1<A, B, 0, DIR>::run(v, y);
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
            P2 u[B];
#pragma unroll
            for (int tb = 0; tb < B; ++tb) u[tb] = y[tb * A + ka];
            PDFT<B, DIR>::run(u);
#pragma unroll
            for (int kb = 0; kb < B; ++kb) v[ka + A * kb] = u[kb];
        }
    }
};
template <int DIR> struct PDFT<6, DIR> : PDFTComposite<2, 3, DIR> {};
template <int DIR> struct PDFT<8, DIR> : PDFTComposite<2, 4, DIR> {};
template <int DIR> struct PDFT<9, DIR> : PDFTComposite<3, 3, DIR> {};
template <int DIR> struct PDFT<10, DIR> : PDFTComposite<2, 5, DIR> {};
template <int DIR> struct PDFT<12, DIR> : PDFTComposite<4, 3, DIR> {};
template <int DIR> struct PDFT<16, DIR> : PDFTComposite<4, 4, DIR> {};

// v * w for a table twiddle w = c + i s held as {c, c, s, s} (the same for
// both lanes); DIR > 0 multiplies by the conjugate.
template <int DIR>
__device__ __forceinline__ P2 pmul_tw(P2 v, P2 w) {
    const f2 ns = neg2(w.y);
    if constexpr (DIR < 0) return P2{fma2(v.y, ns, v.x * w.x), fma2(v.x, w.y, v.y * w.x)};
    else return P2{fma2(v.y, w.y, v.x * w.x), fma2(v.x, ns, v.y * w.x)};
}

// ---------------------------------------------------------------------------
// Launch geometry.
using C4 = ulonglong2;  // one paired complex element in memory

// Pass B stages its K(G)/Ng slab in shared memory where it fits beside the planes.
__host__ __device__ constexpr size_t smem_b(int n, bool kslab) {
    return sizeof(C4) * (2 * (size_t)n * n + n) + 2 * sizeof(float) * n + (kslab ? sizeof(float) * n * n : 0);
}
__host__ __device__ constexpr bool kslab_fits(int n) { return smem_b(n, true) + 1024 <= 227 * 1024; }
__host__ __device__ constexpr size_t smem_ac(int n) { return sizeof(C4) * (2 * (size_t)n * (n + 1) + n); }
__host__ __device__ constexpr size_t smem_bytes(int n, int pass) {
    return pass == 1 ? smem_b(n, kslab_fits(n)) : smem_ac(n);
}
__host__ __device__ constexpr size_t smem_max(int n) {
    return smem_bytes(n, 0) > smem_bytes(n, 1) ? smem_bytes(n, 0) : smem_bytes(n, 1);
}
// the paired passes exist where both planes fit one CTA's shared memory
__host__ __device__ constexpr bool fits(int n) { return smem_max(n) + 1024 <= 227 * 1024; }

// CTAs of nt threads per SM with at least 64 registers a thread (a paired
// radix-8/9 butterfly holds twice the values of an unpaired one).
__host__ __device__ constexpr int blocks_at(int n, int nt) {
    int m = (int)((227u * 1024u) / (smem_max(n) + 1024));
    const int by_thr = 2048 / ((nt + 31) / 32 * 32);
    if (m > by_thr) m = by_thr;
    while (m > 1 && spec2::regs_at(nt, m) < 64) --m;
    return m < 1 ? 1 : m;
}
// Threads per CTA: one butterfly per thread in the stage with the most
// butterflies, or in the one with the fewest when that is what lets two
// CTAs share an SM, or when it takes no more rounds; at most 1024.
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
    return r_lo < r_hi ? lo : hi;
}
__host__ __device__ constexpr int max_regs(int n) {
    return spec2::regs_at(threads_for(n), blocks_at(n, threads_for(n)));
}

// One radix-R Stockham stage over LINES lines of length N, out of place,
// on paired values (the stage of pairconv_spec2.cuh): butterfly i of a line
// reads elements i + t N/R through ld(line, e), multiplies by w_{P R}^{t k}
// (k = i mod P), runs DFT_R and writes element (i - k) R + k + s P through
// st(line, e, v).  LF: consecutive threads take consecutive lines.
template <int N, int R, int P, int DIR, int LINES, bool LF, int NT, class Ld, class St>
__device__ __forceinline__ void stage(const C4* __restrict__ tw, Ld ld, St st) {
    constexpr int TN = N / R;
    constexpr int ITEMS = LINES * TN;
    constexpr int TWSTEP = N / (P * R);
#pragma unroll
    for (int item0 = 0; item0 < ITEMS; item0 += NT) {
        const int item = item0 + (int)threadIdx.x;
        if (item0 + NT <= ITEMS || item < ITEMS) {
            const int line = LF ? item % LINES : item / TN;
            const int i = LF ? item / LINES : item % TN;
            P2 v[R];
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = ld(line, i + t * TN);
            const int k = P > 1 ? i % P : 0;
            if (P > 1) {
#pragma unroll
                for (int t = 1; t < R; ++t) v[t] = pmul_tw<DIR>(v[t], ld2(tw + t * k * TWSTEP));
            }
            PDFT<R, DIR>::run(v);
            const int base = (i - k) * R + k;
#pragma unroll
            for (int s = 0; s < R; ++s) st(line, base + s * P, v[s]);
        }
    }
}

// Twiddle table of one axis in shared memory as {c, c, s, s}.
__device__ __forceinline__ void load_tw(C4* tw, const float2* src, int n, int nt) {
    for (int i = threadIdx.x; i < n; i += nt) {
        const float2 w = src[i];
        tw[i] = make_ulonglong2(bc2(w.x).v, bc2(w.y).v);
    }
}

constexpr PairGrid kNoGrid{0, 0, -1, -1};

// ---------------------------------------------------------------------------
// Pass A: rho of plane x of both grids of pair pr, forward FFT along z then y.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N))
    pass_a(ConvArgs<float> P, int g0, int nb) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int LP = N + 1;  // odd row pitch: line-fast z stages are free of bank conflicts
    extern __shared__ float4 smem_v4[];
    C4* b0 = reinterpret_cast<C4*>(smem_v4);
    C4* b1 = b0 + N * LP;
    C4* tw = b1 + N * LP;
    const int pr = blockIdx.x, x = blockIdx.y;  // plane-major: the CTAs in flight share plane x
    const bool hb = 2 * pr + 1 < nb;
    const PairGrid da = P.grids[g0 + 2 * pr];
    const PairGrid db = hb ? P.grids[g0 + 2 * pr + 1] : kNoGrid;
    load_tw(tw, P.tw[2], N, NT);
    const size_t off = (size_t)x * NP;
    const bool two_a = da.j2 >= 0, two_b = db.j2 >= 0;
    const float* a1 = P.psi + (size_t)da.i1 * P.ng + off;
    const float* c1 = P.psi + (size_t)da.j1 * P.ng + off;
    const float* a2 = P.psi + (size_t)(two_a ? da.i2 : da.i1) * P.ng + off;
    const float* c2 = P.psi + (size_t)(two_a ? da.j2 : da.j1) * P.ng + off;
    const float* e1 = P.psi + (size_t)db.i1 * P.ng + off;
    const float* f1 = P.psi + (size_t)db.j1 * P.ng + off;
    const float* e2 = P.psi + (size_t)(two_b ? db.i2 : db.i1) * P.ng + off;
    const float* f2p = P.psi + (size_t)(two_b ? db.j2 : db.j1) * P.ng + off;
    int xa = 0, pa = 0;
    const bool pf = threadIdx.x < 8 && spec2::ahead_cta(P.pf_ahead, pa, xa);
    int pf_orb = -1;  // orbital plane of the CTA ahead that this thread prefetches
    if (pf) {
        const int gq = 2 * pa + (int)(threadIdx.x >> 2);
        if (gq < nb) pf_orb = __ldg(reinterpret_cast<const int*>(P.grids + g0 + gq) + (threadIdx.x & 3));
    }
    // z lines (line = y): rho straight from the orbitals
    stage<N, pl.r1, 1, -1, N, false, NT>(
        tw,
        [&](int y, int z) {
            const int q = y * N + z;
            const float ua = __ldg(a1 + q) * __ldg(c1 + q);
            const float va = two_a ? __ldg(a2 + q) * __ldg(c2 + q) : 0.f;
            const float ub = hb ? __ldg(e1 + q) * __ldg(f1 + q) : 0.f;
            const float vb = two_b ? __ldg(e2 + q) * __ldg(f2p + q) : 0.f;
            return P2{mk2(ua, ub), mk2(va, vb)};
        },
        [&](int y, int z, P2 v) { st2(b0 + y * N + z, v); });  // pitch N here: conflict-free stores
    __syncthreads();
    stage<N, pl.r2, pl.r1, -1, N, false, NT>(
        tw, [&](int y, int z) { return ld2(b0 + y * N + z); }, [&](int y, int z, P2 v) { st2(b1 + y * LP + z, v); });
    __syncthreads();
    // y lines (line = z)
    stage<N, pl.r1, 1, -1, N, true, NT>(
        tw, [&](int z, int y) { return ld2(b1 + y * LP + z); }, [&](int z, int y, P2 v) { st2(b0 + y * LP + z, v); });
    __syncthreads();
    C4* out = reinterpret_cast<C4*>(P.scratch) + (size_t)pr * P.ng + off;
    stage<N, pl.r2, pl.r1, -1, N, true, NT>(
        tw, [&](int z, int y) { return ld2(b0 + y * LP + z); }, [&](int z, int y, P2 v) { st2(out + y * N + z, v); });
    if (pf && pf_orb >= 0) spec2::prefetch_l2(P.psi + (size_t)pf_orb * P.ng + (size_t)xa * NP, NP * sizeof(float));
}

// Pass B: slab ky of pair pr: forward x-FFT (decimation in time), * K(G)/Ng,
// inverse x-FFT (decimation in frequency); the middle three steps share registers.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N))
    pass_b(ConvArgs<float> P, int g0, int nb) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int RB = pl.r2, RA = pl.r1;  // N = RA * RB
    constexpr bool KS = kslab_fits(N);
    extern __shared__ float4 smem_v4[];
    C4* b0 = reinterpret_cast<C4*>(smem_v4);
    C4* b1 = b0 + NP;
    C4* tw = b1 + NP;
    float* ks = reinterpret_cast<float*>(tw + N);  // K(G)/Ng of this slab, [x][z] (KS)
    float* gx2 = ks + (KS ? NP : 0);
    float* gz2 = gx2 + N;
    const int pr = blockIdx.y, ky = blockIdx.x;
    const bool kstage = KS && P.ktab != nullptr;
    if (kstage) {
        // asynchronous 16-byte copies, waited for before the middle
        const unsigned ks_s = (unsigned)__cvta_generic_to_shared(ks);
        for (int q = threadIdx.x; q < NP / 4; q += NT) {
            const int xx = q / (N / 4), z4 = q % (N / 4);
            const float* src = P.ktab + ((size_t)xx * N + ky) * N + 4 * z4;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ks_s + 16u * q), "l"(src) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    load_tw(tw, P.tw[0], N, NT);
    for (int i = threadIdx.x; i < N; i += NT) {
        gx2[i] = P.g2[0][i];
        gz2[i] = P.g2[2][i];
    }
    C4* base = reinterpret_cast<C4*>(P.scratch) + (size_t)pr * P.ng + (size_t)ky * N;
    {
        int ka = 0, pa = 0;
        if (threadIdx.x < N && spec2::ahead_cta(P.pf_ahead, ka, pa))
            spec2::prefetch_l2(reinterpret_cast<C4*>(P.scratch) + (size_t)pa * P.ng + (size_t)threadIdx.x * NP +
                                   (size_t)ka * N,
                               N * sizeof(C4));
    }
    // forward stage 1 (line = z): DFT_RB over n2 of x[n1 + RA n2], to y[n1 RB + k2]
    stage<N, RB, 1, -1, N, true, NT>(
        tw, [&](int z, int xx) { return ld2(base + (size_t)xx * NP + z); },
        [&](int z, int xx, P2 v) { st2(b0 + xx * N + z, v); });
    if (kstage) asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const float gy2 = P.g2[1][ky];
    // middle: for each (z, k2): twiddle, DFT_RA -> X[k2 + RB k1], * K, inverse
    // DFT_RA -> z[k2][n1], twiddle w_N^{-n1 k2}, stored at n1 RB + k2
    constexpr int MID = N * RB;
#pragma unroll
    for (int item0 = 0; item0 < MID; item0 += NT) {
        const int item = item0 + (int)threadIdx.x;
        if (item0 + NT <= MID || item < MID) {
            const int z = item % N, k2 = item / N;
            P2 v[RA];
#pragma unroll
            for (int t = 0; t < RA; ++t) {
                v[t] = ld2(b0 + (k2 + t * RB) * N + z);
                if (t > 0) v[t] = pmul_tw<-1>(v[t], ld2(tw + t * k2));
            }
            PDFT<RA, -1>::run(v);
#pragma unroll
            for (int s = 0; s < RA; ++s) {
                const int xx = k2 + s * RB;
                float k;
                if (kstage) {
                    k = ks[xx * N + z];
                } else if (P.ktab) {
                    k = __ldg(P.ktab + ((size_t)xx * N + ky) * N + z);
                } else {
                    const float gg = gx2[xx] + gy2 + gz2[z];
                    k = gg > 0.f ? P.kscale / gg : 0.f;
                }
                const f2 k2v = bc2(k);
                v[s] = P2{v[s].x * k2v, v[s].y * k2v};
            }
            PDFT<RA, +1>::run(v);
#pragma unroll
            for (int n1 = 0; n1 < RA; ++n1) {
                const P2 o = n1 > 0 ? pmul_tw<+1>(v[n1], ld2(tw + n1 * k2)) : v[n1];
                st2(b1 + (n1 * RB + k2) * N + z, o);
            }
        }
    }
    __syncthreads();
    // inverse stage 2 (line = z): for each n1, DFT_RB over k2 -> x[n1 + RA n2]
    constexpr int LAST = N * RA;
#pragma unroll
    for (int item0 = 0; item0 < LAST; item0 += NT) {
        const int item = item0 + (int)threadIdx.x;
        if (item0 + NT <= LAST || item < LAST) {
            const int z = item % N, n1 = item / N;
            P2 v[RB];
#pragma unroll
            for (int t = 0; t < RB; ++t) v[t] = ld2(b1 + (n1 * RB + t) * N + z);
            PDFT<RB, +1>::run(v);
#pragma unroll
            for (int s = 0; s < RB; ++s) st2(base + (size_t)(n1 + RA * s) * NP + z, v[s]);
        }
    }
    (void)g0;
    (void)nb;
}

// The W updates and real-space pair energies of one complex grid at four
// consecutive points e (16-byte vectors): va, vb = the potentials of its two
// real pairs (Re and Im of the inverse transform).
__device__ __forceinline__ void epilogue4(const ConvArgs<float>& P, const PairGrid& d, size_t off, int e, float4 va,
                                          float4 vb, float& sa, float& ca, float& sb, float& cb) {
    const bool two = d.j2 >= 0;
    const bool a_occ = d.j1 < P.n_occ, a_sym = a_occ && d.j1 != d.i1;
    const bool b_occ = two && d.j2 < P.n_occ, b_sym = b_occ && d.j2 != d.i2;
    const bool merge_i = two && a_sym && b_sym && d.i1 == d.i2;
    const float4* wi1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.i1 * P.ng + off);
    const float4* pj1 = reinterpret_cast<const float4*>(P.psi + (size_t)d.j1 * P.ng + off);
    float4* Wj1 = reinterpret_cast<float4*>(P.W + (size_t)d.j1 * P.ng + off);
    float4* Wi1 = reinterpret_cast<float4*>(P.W + (size_t)d.i1 * P.ng + off);
    const float4 x1 = __ldg(wi1 + e), y1 = __ldg(pj1 + e);
    atomicAdd(Wj1 + e, make_float4(-x1.x * va.x, -x1.y * va.y, -x1.z * va.z, -x1.w * va.w));
    const float4 wi_acc = make_float4(-y1.x * va.x, -y1.y * va.y, -y1.z * va.z, -y1.w * va.w);
    if (a_sym && !merge_i) atomicAdd(Wi1 + e, wi_acc);
    if (a_occ) spec::kahan(sa, ca, x1.x * y1.x * va.x + x1.y * y1.y * va.y + x1.z * y1.z * va.z + x1.w * y1.w * va.w);
    if (two) {
        const float4* wi2 = reinterpret_cast<const float4*>(P.psi + (size_t)d.i2 * P.ng + off);
        const float4* pj2 = reinterpret_cast<const float4*>(P.psi + (size_t)d.j2 * P.ng + off);
        float4* Wj2 = reinterpret_cast<float4*>(P.W + (size_t)d.j2 * P.ng + off);
        float4* Wi2 = reinterpret_cast<float4*>(P.W + (size_t)d.i2 * P.ng + off);
        const float4 x2 = merge_i ? x1 : __ldg(wi2 + e);
        const float4 y2 = __ldg(pj2 + e);
        atomicAdd(Wj2 + e, make_float4(-x2.x * vb.x, -x2.y * vb.y, -x2.z * vb.z, -x2.w * vb.w));
        const float4 w2 = make_float4(-y2.x * vb.x, -y2.y * vb.y, -y2.z * vb.z, -y2.w * vb.w);
        if (merge_i) {
            atomicAdd(Wi1 + e, make_float4(wi_acc.x + w2.x, wi_acc.y + w2.y, wi_acc.z + w2.z, wi_acc.w + w2.w));
        } else if (b_sym) {
            atomicAdd(Wi2 + e, w2);
        }
        if (b_occ)
            spec::kahan(sb, cb, x2.x * y2.x * vb.x + x2.y * y2.y * vb.y + x2.z * y2.z * vb.z + x2.w * y2.w * vb.w);
    }
}

// Pass C: inverse FFT along y then z of plane x of both grids of pair pr,
// then the W updates (16-byte vector reductions) and the pair energies.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) __maxnreg__(max_regs(N))
    pass_c(ConvArgs<float> P, int g0, int nb) {
    constexpr int NT = threads_for(N);
    constexpr int NP = N * N;
    constexpr Plan2 pl = plan2(N);
    constexpr int LP = N + 1;  // odd row pitch (the last stage writes pitch N for the epilogue)
    constexpr int NW = (NT + 31) / 32;
    extern __shared__ float4 smem_v4[];
    C4* b0 = reinterpret_cast<C4*>(smem_v4);
    C4* b1 = b0 + N * LP;
    C4* tw = b1 + N * LP;
    __shared__ double red[4][NW];
    const int pr = blockIdx.x, x = blockIdx.y;  // plane-major: the CTAs in flight share plane x
    const bool hb = 2 * pr + 1 < nb;
    const PairGrid da = P.grids[g0 + 2 * pr];
    const PairGrid db = hb ? P.grids[g0 + 2 * pr + 1] : kNoGrid;
    load_tw(tw, P.tw[2], N, NT);
    const size_t off = (size_t)x * NP;
    const C4* in = reinterpret_cast<const C4*>(P.scratch) + (size_t)pr * P.ng + off;
    {
        int xa = 0, pa = 0;
        if (threadIdx.x == 32 && spec2::ahead_cta(P.pf_ahead, pa, xa))
            spec2::prefetch_l2(reinterpret_cast<const C4*>(P.scratch) + (size_t)pa * P.ng + (size_t)xa * NP,
                               NP * sizeof(C4));
    }
    stage<N, pl.r1, 1, +1, N, true, NT>(
        tw, [&](int z, int y) { return ld2(in + y * N + z); }, [&](int z, int y, P2 v) { st2(b0 + y * LP + z, v); });
    if (P.pf_ahead > 0 && threadIdx.x < 16) {
        // the epilogue's orbital planes and W planes, fetched into L2 while
        // the FFT stages run
        const PairGrid& d = threadIdx.x < 8 ? da : db;
        const int q = threadIdx.x & 3;
        const int o = (threadIdx.x >= 8 && !hb) ? -1 : q == 0 ? d.i1 : q == 1 ? d.j1 : q == 2 ? d.i2 : d.j2;
        if (o >= 0) {
            const float* src = ((threadIdx.x & 4) ? P.W : P.psi) + (size_t)o * P.ng + off;
            spec2::prefetch_l2(src, NP * sizeof(float));
        }
    }
    __syncthreads();
    stage<N, pl.r2, pl.r1, +1, N, true, NT>(
        tw, [&](int z, int y) { return ld2(b0 + y * LP + z); }, [&](int z, int y, P2 v) { st2(b1 + y * LP + z, v); });
    __syncthreads();
    stage<N, pl.r1, 1, +1, N, true, NT>(
        tw, [&](int y, int z) { return ld2(b1 + y * LP + z); }, [&](int y, int z, P2 v) { st2(b0 + y * LP + z, v); });
    __syncthreads();
    stage<N, pl.r2, pl.r1, +1, N, false, NT>(
        tw, [&](int y, int z) { return ld2(b0 + y * LP + z); }, [&](int y, int z, P2 v) { st2(b1 + y * N + z, v); });
    __syncthreads();
    const float4* pl4 = reinterpret_cast<const float4*>(b1);  // per point {re_a, re_b, im_a, im_b}
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // (sum, compensation) x (a1, a2, b1, b2)
#pragma unroll 1
    for (int e = threadIdx.x; e < NP / 4; e += NT) {
        const float4 q0 = pl4[4 * e], q1 = pl4[4 * e + 1], q2 = pl4[4 * e + 2], q3 = pl4[4 * e + 3];
        epilogue4(P, da, off, e, make_float4(q0.x, q1.x, q2.x, q3.x), make_float4(q0.z, q1.z, q2.z, q3.z), s[0], s[1],
                  s[2], s[3]);
        if (hb)
            epilogue4(P, db, off, e, make_float4(q0.y, q1.y, q2.y, q3.y), make_float4(q0.w, q1.w, q2.w, q3.w), s[4],
                      s[5], s[6], s[7]);
    }
    float t[4] = {s[0] - s[1], s[2] - s[3], s[4] - s[5], s[6] - s[7]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k][warp] = (double)t[k];
    }
    __syncthreads();
    if (threadIdx.x < 4 && (threadIdx.x < 2 || hb)) {
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += red[threadIdx.x][w];
        const int gq = 2 * pr + (int)(threadIdx.x >> 1);
        P.epart[((size_t)gq * N + x) * 2 + (threadIdx.x & 1)] = tot * P.dv;
    }
}

// Launch pass 0/1/2 for a batch of nb complex grids (pairs of grids; the
// scratch must hold nb rounded up to even grids).
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
    const int npair = (nb + 1) / 2;
    if (pass == 0) pass_a<N><<<dim3(npair, N), NT, sm, s>>>(P, g0, nb);
    else if (pass == 1) pass_b<N><<<dim3(N, npair), NT, sm, s>>>(P, g0, nb);
    else pass_c<N><<<dim3(npair, N), NT, sm, s>>>(P, g0, nb);
    return true;
}

// Pairing halves the instructions a point but doubles the shared memory of
// a CTA, so fewer CTAs share an SM and their barriers are less hidden.
// Measured on GB300 against the one-grid passes (with packed real/imaginary
// butterflies): 72^3 3.31 vs 2.63 us per pair (one paired CTA an SM), 48^3
// 0.87 vs 0.78 (two).  So they are off unless LACE_FFT_PAIRED=1.
template <int N>
inline bool enabled() {
    static const int on = [] {
        const char* e = getenv("LACE_FFT_PAIRED");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return on != 0;
}

}  // namespace pair2

namespace spec {

// Paired out-of-place passes where two paired planes fit in shared memory
// (and the scratch holds an even number of grids), else the one-grid
// out-of-place passes where two planes fit, else in place.  A merged launch
// (several systems, P.refs) takes the one-grid out-of-place passes or none.
template <int N>
bool launch_any(int pass, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s, bool allow_pair) {
    if constexpr (pair2::fits(N)) {
        if (allow_pair && pair2::enabled<N>()) return pair2::launch_one<N>(pass, nb, P, g0, s);
    }
    if constexpr (spec2::smem_max(N) <= 200 * 1024) {
        // merged launches (P.refs) exist only in the one-grid out-of-place passes
        if (spec2::enabled() || P.refs) return spec2::launch_one<N>(pass, nb, P, g0, s);
    }
    if (P.refs) return false;
    return spec_launch_one<N>(pass, nb, P, g0, s);
}

}  // namespace spec
}  // namespace lace
