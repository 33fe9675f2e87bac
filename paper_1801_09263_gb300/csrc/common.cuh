// Shared device helpers of liblace: complex arithmetic, compile-time
// twiddle factors, register-resident small DFTs and the in-place
// shared-memory Stockham stage used by every FFT pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lace {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by i*s (s = +1 or -1)
template <int S, typename C> __device__ __forceinline__ C cmul_i(C a) {
    if constexpr (S > 0) return C{-a.y, a.x};
    else return C{a.y, -a.x};
}

// ---------------------------------------------------------------------------
// Compile-time trigonometry (Taylor series on a reduced argument), used only
// to produce the exact-to-rounding constants of the in-register DFTs.
constexpr double kPi = 3.141592653589793238462643383279502884;

__host__ __device__ constexpr double ct_sin_reduced(double x) {  // |x| <= pi/4
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_cos_reduced(double x) {  // |x| <= pi/4
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}
// cos and sin of 2*pi*m/n for integers (exact octant reduction).
__host__ __device__ constexpr double ct_cos2pi(long m, long n) {
    m %= n;
    if (m < 0) m += n;
    // angle = 2 pi m / n = (pi/4) * (8m/n); octant q = floor(8m/n), remainder
    long num = 8 * m;
    long q = num / n;
    double r = double(num - q * n) / double(n) * (kPi / 4.0);  // in [0, pi/4)
    switch (q) {
        case 0: return ct_cos_reduced(r);
        case 1: return ct_sin_reduced(kPi / 4.0 - r);
        case 2: return -ct_sin_reduced(r);
        case 3: return -ct_cos_reduced(kPi / 4.0 - r);
        case 4: return -ct_cos_reduced(r);
        case 5: return -ct_sin_reduced(kPi / 4.0 - r);
        case 6: return ct_sin_reduced(r);
        default: return ct_cos_reduced(kPi / 4.0 - r);
    }
}
__host__ __device__ constexpr double ct_sin2pi(long m, long n) { return ct_cos2pi(m * 4 - n, 4 * n); }  // sin(x) = cos(x - pi/2)

// x * c for a compile-time constant c.  In FP32 the constant is carried as
// hi + lo (two floats) and the product rounded once: rounding the irrational
// DFT constants (sqrt(1/2), sqrt(3)/2, cos/sin of 2 pi/5 ...) to a single
// float scales every butterfly that uses them the same way, and the pair
// energies inherit that bias (about -1e-7 relative per transform pair).
template <typename T> __device__ __forceinline__ T mulk(T x, double c) {
    if constexpr (sizeof(T) == 4) {
        const float hi = (float)c;
        const float lo = (float)(c - (double)hi);
        return fmaf(x, hi, x * lo);
    } else {
        return x * (T)c;
    }
}

// Multiply by exp(DIR * 2 pi i M / N), folding the trivial cases.
template <int N, int M, int DIR, typename C>
__device__ __forceinline__ C twiddle_ct(C a) {
    using T = decltype(a.x);
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == N) {
        return C{-a.x, -a.y};
    } else if constexpr (4 * m == N) {
        return cmul_i<DIR>(a);
    } else if constexpr (4 * m == 3 * N) {
        return cmul_i<-DIR>(a);
    } else if constexpr ((8 * m) % N == 0) {
        // odd multiple of pi/4: cos and sin are +-sqrt(1/2); add first,
        // then one constant product per component
        constexpr int e8 = 8 * m / N;
        constexpr int cx = (e8 == 1 || e8 == 7) ? 1 : -1;
        constexpr int ss = DIR * ((e8 == 1 || e8 == 3) ? 1 : -1);
        constexpr double h = 0.707106781186547524400844362104849039;
        const T u = cx > 0 ? (ss > 0 ? a.x - a.y : a.x + a.y) : (ss > 0 ? -a.x - a.y : a.y - a.x);
        const T w = cx > 0 ? (ss > 0 ? a.x + a.y : a.y - a.x) : (ss > 0 ? a.x - a.y : -a.x - a.y);
        return C{mulk(u, h), mulk(w, h)};
    } else {
        constexpr double c = ct_cos2pi(m, N);
        constexpr double s = DIR * ct_sin2pi(m, N);
        return C{mulk(a.x, c) - mulk(a.y, s), mulk(a.x, s) + mulk(a.y, c)};
    }
}

// ---------------------------------------------------------------------------
// In-register DFTs: X_k = sum_t x_t exp(DIR 2 pi i t k / R), natural order.
template <int R, int DIR> struct DFT;

template <int DIR> struct DFT<2, DIR> {
    template <typename C> static __device__ __forceinline__ void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR> struct DFT<3, DIR> {
    template <typename C> static __device__ __forceinline__ void run(C* v) {
        using T = decltype(v[0].x);
        constexpr double s3 = 0.866025403784438646763723170752936183;  // sin(2 pi/3)
        C a = v[0], b = v[1], c = v[2];
        C t1 = cadd(b, c);
        C t2 = C{a.x - T(0.5) * t1.x, a.y - T(0.5) * t1.y};
        C d = csub(b, c);
        C t3 = cmul_i<DIR>(C{mulk(d.x, s3), mulk(d.y, s3)});
        v[0] = cadd(a, t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};

template <int DIR> struct DFT<4, DIR> {
    template <typename C> static __device__ __forceinline__ void run(C* v) {
        C a = v[0], b = v[1], c = v[2], d = v[3];
        C s0 = cadd(a, c), d0 = csub(a, c);
        C s1 = cadd(b, d), d1 = cmul_i<DIR>(csub(b, d));
        v[0] = cadd(s0, s1);
        v[2] = csub(s0, s1);
        v[1] = cadd(d0, d1);
        v[3] = csub(d0, d1);
    }
};

template <int DIR> struct DFT<5, DIR> {
    template <typename C> static __device__ __forceinline__ void run(C* v) {
        using T = decltype(v[0].x);
        constexpr double c1 = ct_cos2pi(1, 5), c2 = ct_cos2pi(2, 5);
        constexpr double s1 = ct_sin2pi(1, 5), s2 = ct_sin2pi(2, 5);
        C a = v[0];
        C p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
        C p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
        C r1 = C{a.x + mulk(p1.x, c1) + mulk(p2.x, c2), a.y + mulk(p1.y, c1) + mulk(p2.y, c2)};
        C r2 = C{a.x + mulk(p1.x, c2) + mulk(p2.x, c1), a.y + mulk(p1.y, c2) + mulk(p2.y, c1)};
        C i1 = cmul_i<DIR>(C{mulk(m1.x, s1) + mulk(m2.x, s2), mulk(m1.y, s1) + mulk(m2.y, s2)});
        C i2 = cmul_i<DIR>(C{mulk(m1.x, s2) - mulk(m2.x, s1), mulk(m1.y, s2) - mulk(m2.y, s1)});
        v[0] = cadd(a, cadd(p1, p2));
        v[1] = cadd(r1, i1);
        v[4] = csub(r1, i1);
        v[2] = cadd(r2, i2);
        v[3] = csub(r2, i2);
    }
};

// Composite R = A * B (Cooley-Tukey in registers): t = B*ta + tb, k = ka + A*kb.
// Step 1 (for each tb): DFT_A over ta of v[B ta + tb], then twiddle
// w_R^{tb ka}, stored at y[tb A + ka].  Step 2 (for each ka): DFT_B over tb.
template <int R, int A, int TB, int KA, int DIR> struct CompTw {
    template <typename C> static __device__ __forceinline__ void run(const C* u, C* y) {
        y[TB * A + KA] = twiddle_ct<R, TB * KA, DIR>(u[KA]);
        CompTw<R, A, TB, KA + 1, DIR>::run(u, y);
    }
};
template <int R, int A, int TB, int DIR> struct CompTw<R, A, TB, A, DIR> {
    template <typename C> static __device__ __forceinline__ void run(const C*, C*) {}
};
template <int A, int B, int TB, int DIR> struct CompStep1 {
    template <typename C> static __device__ __forceinline__ void run(const C* v, C* y) {
        C u[A];
#pragma unroll
        for (int ta = 0; ta < A; ++ta) u[ta] = v[B * ta + TB];
        DFT<A, DIR>::run(u);
        CompTw<A * B, A, TB, 0, DIR>::run(u, y);
        CompStep1<A, B, TB + 1, DIR>::run(v, y);
    }
};
template <int A, int B, int DIR> struct CompStep1<A, B, B, DIR> {
    template <typename C> static __device__ __forceinline__ void run(const C*, C*) {}
};
template <int A, int B, int DIR> struct DFTComposite {
    template <typename C> static __device__ __forceinline__ void run(C* v) {
        C y[A * B];
        CompStep1<A, B, 0, DIR>::run(v, y);
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
            C u[B];
#pragma unroll
            for (int tb = 0; tb < B; ++tb) u[tb] = y[tb * A + ka];
            DFT<B, DIR>::run(u);
#pragma unroll
            for (int kb = 0; kb < B; ++kb) v[ka + A * kb] = u[kb];
        }
    }
};

template <int DIR> struct DFT<6, DIR> : DFTComposite<2, 3, DIR> {};
template <int DIR> struct DFT<8, DIR> : DFTComposite<2, 4, DIR> {};
template <int DIR> struct DFT<9, DIR> : DFTComposite<3, 3, DIR> {};
template <int DIR> struct DFT<10, DIR> : DFTComposite<2, 5, DIR> {};
template <int DIR> struct DFT<12, DIR> : DFTComposite<4, 3, DIR> {};
template <int DIR> struct DFT<16, DIR> : DFTComposite<4, 4, DIR> {};

// ---------------------------------------------------------------------------
// One radix-R Stockham stage over `nlines` lines of length n held in shared
// memory, in place.  Line l, element e lives at buf[l*lpitch + e*es].
// p = product of the radices of the earlier stages.  Butterfly i (0 <= i <
// n/R) reads x[i + t n/R] (t < R), multiplies by w_{pR}^{t k} (k = i mod p),
// runs DFT_R and writes y[(i-k) R + k + s p].  All butterflies of a chunk of
// whole lines are held in registers across a barrier, so the stage is safe
// in place.  tw holds exp(-2 pi i m/n), m < n (forward sign).
// lines_fast: consecutive threads take consecutive lines (use when es > 1).
//
// The radix is a runtime value; every radix shares one register array V
// (kStageElems complex values per thread) so that the live state across the
// barrier does not grow with the number of radices compiled in.
constexpr int kStageElems = 16;

struct StageGeom {
    int n, p, nlines, lpitch, es, tn, lc, nb, l0;
    bool lines_fast;
};

__device__ __forceinline__ void stage_index(const StageGeom& G, int idx, int& line, int& i) {
    if (G.lines_fast) { line = idx % G.lc; i = idx / G.lc; }
    else { line = idx / G.tn; i = idx - line * G.tn; }
}

template <typename T, int R, int DIR>
__device__ __forceinline__ void stage_compute(const cplx<T>* __restrict__ buf, const StageGeom& G,
                                              const cplx<T>* __restrict__ tw, cplx<T>* V) {
    using C = cplx<T>;
    constexpr int MAXB = kStageElems / R > 0 ? kStageElems / R : 1;
    const int twstep = G.n / (G.p * R);
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int idx = threadIdx.x + b * blockDim.x;
        if (idx < G.nb) {
            int line, i;
            stage_index(G, idx, line, i);
            const C* src = buf + (size_t)(G.l0 + line) * G.lpitch;
            C* v = V + b * R;
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = src[(i + t * G.tn) * G.es];
            if (G.p > 1) {
                const int k = i % G.p;
#pragma unroll
                for (int t = 1; t < R; ++t) {
                    C w = tw[t * k * twstep];
                    if (DIR > 0) w.y = -w.y;
                    v[t] = cmul(v[t], w);
                }
            }
            DFT<R, DIR>::run(v);
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void stage_store(cplx<T>* __restrict__ buf, const StageGeom& G, const cplx<T>* V) {
    using C = cplx<T>;
    constexpr int MAXB = kStageElems / R > 0 ? kStageElems / R : 1;
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int idx = threadIdx.x + b * blockDim.x;
        if (idx < G.nb) {
            int line, i;
            stage_index(G, idx, line, i);
            const int k = i % G.p;
            C* dst = buf + (size_t)(G.l0 + line) * G.lpitch;
            const int base = (i - k) * R + k;
            const C* v = V + b * R;
#pragma unroll
            for (int s = 0; s < R; ++s) dst[(base + s * G.p) * G.es] = v[s];
        }
    }
}

#define LACE_RADIX_SWITCH(R_, STMT) \
    switch (R_) {                   \
        case 2: { constexpr int RR = 2; STMT; } break;   \
        case 3: { constexpr int RR = 3; STMT; } break;   \
        case 4: { constexpr int RR = 4; STMT; } break;   \
        case 5: { constexpr int RR = 5; STMT; } break;   \
        case 6: { constexpr int RR = 6; STMT; } break;   \
        case 8: { constexpr int RR = 8; STMT; } break;   \
        case 9: { constexpr int RR = 9; STMT; } break;   \
        case 10: { constexpr int RR = 10; STMT; } break; \
        case 12: { constexpr int RR = 12; STMT; } break; \
        default: { constexpr int RR = 16; STMT; } break; \
    }

inline __host__ __device__ int stage_maxb(int r) { return kStageElems / r > 0 ? kStageElems / r : 1; }

// Axis plan: the radices of each stage (at most 4 stages).
struct AxisPlan {
    int n;
    int nst;
    int radix[4];
};

template <typename T, int DIR>
__device__ __forceinline__ void fft_lines(cplx<T>* buf, const AxisPlan& ap, int nlines, int lpitch, int es,
                                          bool lines_fast, const cplx<T>* tw) {
    using C = cplx<T>;
    StageGeom G;
    G.n = ap.n;
    G.nlines = nlines;
    G.lpitch = lpitch;
    G.es = es;
    G.lines_fast = lines_fast;
    G.p = 1;
#pragma unroll 1
    for (int s = 0; s < ap.nst; ++s) {
        const int r = ap.radix[s];
        G.tn = G.n / r;
        const int lines_per_chunk = max(1, (int)(blockDim.x * stage_maxb(r)) / G.tn);
#pragma unroll 1
        for (G.l0 = 0; G.l0 < nlines; G.l0 += lines_per_chunk) {
            G.lc = min(lines_per_chunk, nlines - G.l0);
            G.nb = G.lc * G.tn;
            C V[kStageElems];
            LACE_RADIX_SWITCH(r, (stage_compute<T, RR, DIR>(buf, G, tw, V)));
            __syncthreads();
            LACE_RADIX_SWITCH(r, (stage_store<T, RR>(buf, G, V)));
            __syncthreads();
        }
        G.p *= r;
    }
}

}  // namespace lace
