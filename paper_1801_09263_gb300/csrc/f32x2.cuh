// Packed FP32 pairs: two FP32 values in one 64-bit register pair, operated
// on by the packed FP32 instructions of sm_100+ (add/sub/mul/fma .rn.f32x2):
// one instruction does the same operation on both lanes, each rounded as
// the scalar instruction would round it.
#pragma once

#include <cuda_runtime.h>

namespace lace {

struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 mk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f2 bc2(float a) { return mk2(a, a); }
__device__ __forceinline__ void unpk2(f2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
// a * b + c
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f2 neg2(f2 a) { return bc2(0.f) - a; }

// x * c for a compile-time constant c carried as hi + lo floats (the product
// rounded once: rounding the irrational DFT constants to one float would
// scale every butterfly that uses them the same way, a bias the pair
// energies inherit).
__device__ __forceinline__ f2 mulk2(f2 x, double c) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    return fma2(x, bc2(hi), x * bc2(lo));
}
// acc + x * c with c as hi + lo
__device__ __forceinline__ f2 fmak2(f2 x, double c, f2 acc) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    return fma2(x, bc2(hi), fma2(x, bc2(lo), acc));
}
// x * (c0, c1): a different constant in each lane, each as hi + lo
__device__ __forceinline__ f2 mulk2v(f2 x, double c0, double c1) {
    const float h0 = (float)c0, h1 = (float)c1;
    const float l0 = (float)(c0 - (double)h0), l1 = (float)(c1 - (double)h1);
    return fma2(x, mk2(h0, h1), x * mk2(l0, l1));
}
// acc + x * (c0, c1)
__device__ __forceinline__ f2 fmak2v(f2 x, double c0, double c1, f2 acc) {
    const float h0 = (float)c0, h1 = (float)c1;
    const float l0 = (float)(c0 - (double)h0), l1 = (float)(c1 - (double)h1);
    return fma2(x, mk2(h0, h1), fma2(x, mk2(l0, l1), acc));
}

}  // namespace lace
