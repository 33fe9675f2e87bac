// Generic-radix passes of the pair convolution (runtime axis plans) as
// device functions over one plane or slab of one complex grid, shared by the
// per-batch kernels (pairconv.cu) and the persistent multi-instance kernel
// (pairconv_multi.cu).  Eq. 2 evaluated with FFTs (Sec. 2): pass A forms
// rho = w_i psi_j (two real pairs per complex grid) and transforms over
// (y, z); pass B transforms along x, multiplies by K(G)/Ng and transforms
// back; pass C transforms back over (y, z), accumulates W -= w v and the
// real-space pair energies.  Every function ends with a block barrier, so the
// caller may reuse the shared memory for its next plane.
#pragma once

#include "lace_internal.cuh"

namespace lace {
namespace gen {

template <typename C>
__device__ __forceinline__ void load_tw(C* dst, const C* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Shared memory: plane [n2 n3] + tw2 [n2] + tw3 [n3] (complex).
template <typename T>
__device__ __forceinline__ void pass_a_plane(const ConvArgs<T>& P, const PairGrid d, cplx<T>* grid_out, int x,
                                             cplx<T>* plane) {
    using C = cplx<T>;
    const int n2 = P.ax[1].n, n3 = P.ax[2].n;
    const int np = n2 * n3;
    C* tw2 = plane + np;
    C* tw3 = tw2 + n2;
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
    C* out = grid_out + off;
    for (int e = threadIdx.x; e < np; e += blockDim.x) out[e] = plane[e];
    __syncthreads();
}

// Shared memory: slab [n1 n3] + tw1 [n1] (complex) + |G_z|^2 [n3] + |G_x|^2 [n1].
template <typename T>
__device__ __forceinline__ void pass_b_slab(const ConvArgs<T>& P, cplx<T>* grid, int ky, cplx<T>* slab) {
    using C = cplx<T>;
    const int n1 = P.ax[0].n, n2 = P.ax[1].n, n3 = P.ax[2].n;
    C* tw1 = slab + n1 * n3;
    T* gz2 = reinterpret_cast<T*>(tw1 + n1);
    T* gx2 = gz2 + n3;
    load_tw(tw1, P.tw[0], n1);
    for (int i = threadIdx.x; i < n3; i += blockDim.x) gz2[i] = P.g2[2][i];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) gx2[i] = P.g2[0][i];
    C* base = grid + (size_t)ky * n3;
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
    __syncthreads();
}

template <typename T> __device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Shared memory: as pass A; red holds 2 x 32 doubles.  Thread 0 writes the
// plane's two pair energies dV sum rho v to ep[0], ep[1].
template <typename T>
__device__ __forceinline__ void pass_c_plane(const ConvArgs<T>& P, const PairGrid d, const cplx<T>* grid_in, int x,
                                             cplx<T>* plane, double* red, double* ep) {
    using C = cplx<T>;
    const int n2 = P.ax[1].n, n3 = P.ax[2].n;
    const int np = n2 * n3;
    C* tw2 = plane + np;
    C* tw3 = tw2 + n2;
    load_tw(tw2, P.tw[1], n2);
    load_tw(tw3, P.tw[2], n3);
    const size_t off = (size_t)x * np;
    const C* in = grid_in + off;
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
        atomicAdd(Wj1 + e, -x1 * v.x);
        if (a_sym) atomicAdd(Wi1 + e, -y1 * v.x);
        if (a_occ) kahan_add(sa, ca, x1 * y1 * v.x);
        if (two) {
            const T x2 = wi2[e], y2 = pj2[e];
            atomicAdd(Wj2 + e, -x2 * v.y);
            if (b_sym) atomicAdd(Wi2 + e, -y2 * v.y);
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
    if (lane == 0) { red[warp] = (double)sa; red[32 + warp] = (double)sb; }
    __syncthreads();
    if (warp == 0) {
        // the warp partials in FP64 across the lanes of one warp (short chain)
        const int nw = (int)(blockDim.x >> 5);
        double ta = lane < nw ? red[lane] : 0.0, tbb = lane < nw ? red[32 + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_xor_sync(0xffffffffu, ta, o);
            tbb += __shfl_xor_sync(0xffffffffu, tbb, o);
        }
        if (lane == 0) {
            ep[0] = ta * P.dv;
            ep[1] = tbb * P.dv;
        }
    }
    __syncthreads();
}

}  // namespace gen
}  // namespace lace
