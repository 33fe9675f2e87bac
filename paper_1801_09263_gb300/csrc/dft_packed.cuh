// In-register DFTs of FP32 complex values with the real and imaginary parts
// packed in one register pair: every complex addition, subtraction and
// multiplication by a real constant is one packed FP32 instruction
// (add/sub/fma .rn.f32x2) instead of two.  Same transforms, same constants
// (hi + lo, product rounded once) and the same rounding of each operation as
// DFT<R, DIR> in common.cuh; the sums of constant products are fused
// (x c1 + y c2 + a as two chained FMAs per constant) instead of rounded after
// each product.  The multiplications by +-i and the final a +- i b of each
// small DFT mix the two parts and stay scalar.
#pragma once

#include "common.cuh"
#include "f32x2.cuh"

namespace lace {
namespace fx {

using C = float2;

__device__ __forceinline__ f2 pk(C a) { return mk2(a.x, a.y); }
__device__ __forceinline__ C upk(f2 a) {
    C r;
    unpk2(a, r.x, r.y);
    return r;
}
__device__ __forceinline__ C add(C a, C b) { return upk(pk(a) + pk(b)); }
__device__ __forceinline__ C sub(C a, C b) { return upk(pk(a) - pk(b)); }
// a + i S b (S = +-1)
template <int S> __device__ __forceinline__ C addi(C a, C b) {
    if constexpr (S > 0) return C{a.x - b.y, a.y + b.x};
    else return C{a.x + b.y, a.y - b.x};
}

// Multiply by exp(DIR 2 pi i M / N), compile-time constant.
template <int N, int M, int DIR>
__device__ __forceinline__ C tw_ct(C a) {
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == N) {
        return upk(neg2(pk(a)));
    } else if constexpr (4 * m == N) {
        return cmul_i<DIR>(a);
    } else if constexpr (4 * m == 3 * N) {
        return cmul_i<-DIR>(a);
    } else if constexpr ((8 * m) % N == 0) {
        // (cx + i ss) h, cx, ss = +-1, r = cx ss:
        // r = +1: (cx h (x - y), cx h (x + y)); r = -1: (cx h (x + y), -cx h (x - y))
        constexpr int e8 = 8 * m / N;
        constexpr int cx = (e8 == 1 || e8 == 7) ? 1 : -1;
        constexpr int ss = DIR * ((e8 == 1 || e8 == 3) ? 1 : -1);
        constexpr double h = 0.707106781186547524400844362104849039;
        const float s = a.x + a.y, d = a.x - a.y;
        if constexpr (cx * ss > 0) return upk(mulk2(mk2(d, s), cx * h));
        else return upk(mulk2v(mk2(s, d), cx * h, -cx * h));
    } else {
        constexpr double c = ct_cos2pi(m, N);
        constexpr double s = DIR * ct_sin2pi(m, N);
        // (x c - y s, x s + y c) = x (c, s) + y (-s, c)
        return upk(fmak2v(bc2(a.x), c, s, mulk2v(bc2(a.y), -s, c)));
    }
}

template <int R, int DIR> struct FDFT;

template <int DIR> struct FDFT<2, DIR> {
    static __device__ __forceinline__ void run(C* v) {
        const C a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    }
};

template <int DIR> struct FDFT<3, DIR> {
    static __device__ __forceinline__ void run(C* v) {
        constexpr double s3 = 0.866025403784438646763723170752936183;  // sin(2 pi/3)
        const C a = v[0], b = v[1], c = v[2];
        const C t1 = add(b, c);
        const C t2 = upk(fma2(pk(t1), bc2(-0.5f), pk(a)));
        const C e = upk(mulk2(pk(sub(b, c)), s3));
        v[0] = add(a, t1);
        v[1] = addi<DIR>(t2, e);
        v[2] = addi<-DIR>(t2, e);
    }
};

template <int DIR> struct FDFT<4, DIR> {
    static __device__ __forceinline__ void run(C* v) {
        const C a = v[0], b = v[1], c = v[2], d = v[3];
        const C s0 = add(a, c), d0 = sub(a, c);
        const C s1 = add(b, d), e = sub(b, d);
        v[0] = add(s0, s1);
        v[2] = sub(s0, s1);
        v[1] = addi<DIR>(d0, e);
        v[3] = addi<-DIR>(d0, e);
    }
};

template <int DIR> struct FDFT<5, DIR> {
    static __device__ __forceinline__ void run(C* v) {
        constexpr double c1 = ct_cos2pi(1, 5), c2 = ct_cos2pi(2, 5);
        constexpr double s1 = ct_sin2pi(1, 5), s2 = ct_sin2pi(2, 5);
        const C a = v[0];
        const f2 p1 = pk(add(v[1], v[4])), m1 = pk(sub(v[1], v[4]));
        const f2 p2 = pk(add(v[2], v[3])), m2 = pk(sub(v[2], v[3]));
        const C r1 = upk(fmak2(p1, c1, fmak2(p2, c2, pk(a))));
        const C r2 = upk(fmak2(p1, c2, fmak2(p2, c1, pk(a))));
        const C q1 = upk(fmak2(m1, s1, mulk2(m2, s2)));
        const C q2 = upk(fmak2(m1, s2, mulk2(m2, -s1)));
        v[0] = upk(pk(a) + (p1 + p2));
        v[1] = addi<DIR>(r1, q1);
        v[4] = addi<-DIR>(r1, q1);
        v[2] = addi<DIR>(r2, q2);
        v[3] = addi<-DIR>(r2, q2);
    }
};

// Composite R = A * B (as DFTComposite in common.cuh): t = B ta + tb, k = ka + A kb.
template <int R, int A, int TB, int KA, int DIR> struct FCompTw {
    static __device__ __forceinline__ void run(const C* u, C* y) {
        y[TB * A + KA] = tw_ct<R, TB * KA, DIR>(u[KA]);
        FCompTw<R, A, TB, KA + 1, DIR>::run(u, y);
    }
};
template <int R, int A, int TB, int DIR> struct FCompTw<R, A, TB, A, DIR> {
    static __device__ __forceinline__ void run(const C*, C*) {}
};
template <int A, int B, int TB, int DIR> struct FCompStep1 {
    static __device__ __forceinline__ void run(const C* v, C* y) {
        C u[A];
#pragma unroll
        for (int ta = 0; ta < A; ++ta) u[ta] = v[B * ta + TB];
        FDFT<A, DIR>::run(u);
        FCompTw<A * B, A, TB, 0, DIR>::run(u, y);
        FCompStep1<A, B, TB + 1, DIR>::run(v, y);
    }
};
template <int A, int B, int DIR> struct FCompStep1<A, B, B, DIR> {
    static __device__ __forceinline__ void run(const C*, C*) {}
};
template <int A, int B, int DIR> struct FDFTComposite {
    static __device__ __forceinline__ void run(C* v) {
        C y[A * B];
        FCompStep1<A, B, 0, DIR>::run(v, y);
#pragma unroll
        for (int ka = 0; ka < A; ++ka) {
            C u[B];
#pragma unroll
            for (int tb = 0; tb < B; ++tb) u[tb] = y[tb * A + ka];
            FDFT<B, DIR>::run(u);
#pragma unroll
            for (int kb = 0; kb < B; ++kb) v[ka + A * kb] = u[kb];
        }
    }
};
template <int DIR> struct FDFT<6, DIR> : FDFTComposite<2, 3, DIR> {};
template <int DIR> struct FDFT<8, DIR> : FDFTComposite<2, 4, DIR> {};
template <int DIR> struct FDFT<9, DIR> : FDFTComposite<3, 3, DIR> {};
template <int DIR> struct FDFT<10, DIR> : FDFTComposite<2, 5, DIR> {};
template <int DIR> struct FDFT<12, DIR> : FDFTComposite<4, 3, DIR> {};
template <int DIR> struct FDFT<16, DIR> : FDFTComposite<4, 4, DIR> {};

}  // namespace fx
}  // namespace lace
