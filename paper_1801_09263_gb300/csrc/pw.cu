// Plane-wave front end: orbitals given as plane-wave coefficients (the
// basis in which the paper writes V_X, Sec. 2) are transformed to the
// real-space grid of the exchange, and results are transformed back.
//
// Basis (real Gamma-point orbitals): the half sphere of G = 2 pi (m1/a,
// m2/b, m3/c) with |G|^2/2 < ecut (the orbital cutoff of lace_set_cell),
// half-space m3 > 0, or m3 = 0 and m2 > 0, or m3 = m2 = 0 and m1 >= 0,
// ordered by |G|^2 then (m1, m2, m3).  phi(r) = c(0) + 2 Re sum c(G) e^{iG.r};
// c(G) = (1/Ng) sum_r phi(r) e^{-iG.r}.  Two real orbitals share one complex
// FP64 transform (phi_a + i phi_b), split by Hermitian symmetry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <tuple>
#include <vector>

#include "../../include/lace.h"
#include "lace_ctx.cuh"
#include "lace_internal.cuh"

using namespace lace;

namespace {

constexpr int PW_THREADS = 256;

// 2D FFT over (y, z) of plane x of grid g (direction DIR: -1 forward, +1 inverse).
template <int DIR>
__global__ void __launch_bounds__(PW_THREADS) pw_plane_kernel(double2* grids, size_t ng, AxisPlan a2, AxisPlan a3,
                                                              const double2* tw2, const double2* tw3) {
    extern __shared__ __align__(16) unsigned char pw_smem[];
    double2* plane = reinterpret_cast<double2*>(pw_smem);
    const int n2 = a2.n, n3 = a3.n, np = n2 * n3;
    double2* t2 = plane + np;
    double2* t3 = t2 + n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) t2[i] = tw2[i];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) t3[i] = tw3[i];
    double2* base = grids + (size_t)blockIdx.y * ng + (size_t)blockIdx.x * np;
    for (int e = threadIdx.x; e < np; e += blockDim.x) plane[e] = base[e];
    __syncthreads();
    fft_lines<double, DIR>(plane, a3, n2, n3, 1, false, t3);  // z lines
    fft_lines<double, DIR>(plane, a2, n3, 1, n3, true, t2);   // y lines
    for (int e = threadIdx.x; e < np; e += blockDim.x) base[e] = plane[e];
}

// FFT along x of slab y of grid g.
template <int DIR>
__global__ void __launch_bounds__(PW_THREADS) pw_xslab_kernel(double2* grids, size_t ng, AxisPlan a1, int n2, int n3,
                                                              const double2* tw1) {
    extern __shared__ __align__(16) unsigned char pw_smem[];
    double2* slab = reinterpret_cast<double2*>(pw_smem);
    const int n1 = a1.n;
    double2* t1 = slab + n1 * n3;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) t1[i] = tw1[i];
    double2* base = grids + (size_t)blockIdx.y * ng + (size_t)blockIdx.x * n3;
    const size_t xs = (size_t)n2 * n3;
    for (int e = threadIdx.x; e < n1 * n3; e += blockDim.x) {
        const int x = e / n3, z = e - x * n3;
        slab[e] = base[(size_t)x * xs + z];
    }
    __syncthreads();
    fft_lines<double, DIR>(slab, a1, n3, 1, n3, true, t1);
    for (int e = threadIdx.x; e < n1 * n3; e += blockDim.x) {
        const int x = e / n3, z = e - x * n3;
        base[(size_t)x * xs + z] = slab[e];
    }
}

// Complex grid of orbital pair (a, b) = (2p, 2p+1): F(G) = c_a(G) + i c_b(G),
// F(-G) = conj(c_a(G)) + i conj(c_b(G)).  coef [orb][n_pw] (re, im).
__global__ void pw_scatter_kernel(const double2* __restrict__ coef, long long n_pw, int n_orb, int p0,
                                  const int2* __restrict__ idx, double2* __restrict__ grids, size_t ng) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = p0 + blockIdx.y;
    if (k >= n_pw) return;
    const int a = 2 * p, b = 2 * p + 1;
    double2 ca = coef[(size_t)a * n_pw + k];
    double2 cb = b < n_orb ? coef[(size_t)b * n_pw + k] : make_double2(0.0, 0.0);
    const int2 ix = idx[k];
    double2* F = grids + (size_t)blockIdx.y * ng;
    if (ix.x == ix.y) {  // G = 0: the real parts
        F[ix.x] = make_double2(ca.x, cb.x);
        return;
    }
    F[ix.x] = make_double2(ca.x - cb.y, ca.y + cb.x);
    F[ix.y] = make_double2(ca.x + cb.y, cb.x - ca.y);
}

// real parts -> orbital a, imaginary parts -> orbital b (FP64 [orb][ng])
__global__ void pw_split_kernel(const double2* __restrict__ grids, size_t ng, int n_orb, int p0,
                                double* __restrict__ out) {
    const int p = p0 + blockIdx.y;
    const int a = 2 * p, b = 2 * p + 1;
    const double2* F = grids + (size_t)blockIdx.y * ng;
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (size_t)gridDim.x * blockDim.x) {
        const double2 v = F[r];
        out[(size_t)a * ng + r] = v.x;
        if (b < n_orb) out[(size_t)b * ng + r] = v.y;
    }
}

template <typename T>
__global__ void pw_pack_kernel(const T* __restrict__ src, size_t ng, int n_orb, int p0, double2* __restrict__ grids) {
    const int p = p0 + blockIdx.y;
    const int a = 2 * p, b = 2 * p + 1;
    double2* F = grids + (size_t)blockIdx.y * ng;
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < ng; r += (size_t)gridDim.x * blockDim.x) {
        const double va = (double)src[(size_t)a * ng + r];
        const double vb = b < n_orb ? (double)src[(size_t)b * ng + r] : 0.0;
        F[r] = make_double2(va, vb);
    }
}

// c_a = (F(G) + conj F(-G)) / (2 Ng), c_b = (F(G) - conj F(-G)) / (2 i Ng)
__global__ void pw_gather_kernel(const double2* __restrict__ grids, size_t ng, long long n_pw, int n_orb, int p0,
                                 const int2* __restrict__ idx, double2* __restrict__ coef) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = p0 + blockIdx.y;
    if (k >= n_pw) return;
    const int a = 2 * p, b = 2 * p + 1;
    const double2* F = grids + (size_t)blockIdx.y * ng;
    const int2 ix = idx[k];
    const double2 fp = F[ix.x], fm = F[ix.y];
    const double s = 0.5 / (double)ng;
    coef[(size_t)a * n_pw + k] = make_double2((fp.x + fm.x) * s, (fp.y - fm.y) * s);
    if (b < n_orb) coef[(size_t)b * n_pw + k] = make_double2((fp.y + fm.y) * s, (fm.x - fp.x) * s);
}

// The half-sphere basis, in its canonical order.
std::vector<std::tuple<int, int, int>> basis(const double cell[3], double ecut) {
    int mm[3];
    for (int a = 0; a < 3; ++a) mm[a] = (int)std::floor(std::sqrt(2.0 * ecut) * cell[a] / (2.0 * M_PI));
    std::vector<std::tuple<double, int, int, int>> v;
    for (int m1 = -mm[0]; m1 <= mm[0]; ++m1)
        for (int m2 = -mm[1]; m2 <= mm[1]; ++m2)
            for (int m3 = -mm[2]; m3 <= mm[2]; ++m3) {
                if (!(m3 > 0 || (m3 == 0 && m2 > 0) || (m3 == 0 && m2 == 0 && m1 >= 0))) continue;
                const double g1 = 2 * M_PI * m1 / cell[0], g2 = 2 * M_PI * m2 / cell[1], g3 = 2 * M_PI * m3 / cell[2];
                const double gg = g1 * g1 + g2 * g2 + g3 * g3;
                if (gg / 2.0 < ecut) v.emplace_back(gg, m1, m2, m3);
            }
    std::sort(v.begin(), v.end());
    std::vector<std::tuple<int, int, int>> out;
    out.reserve(v.size());
    for (auto& t : v) out.emplace_back(std::get<1>(t), std::get<2>(t), std::get<3>(t));
    return out;
}

int smooth235_at_least(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int k = m;
        for (int p : {2, 3, 5})
            while (k % p == 0) k /= p;
        if (k == 1) return m;
    }
}

// Index table (grid offsets of G and -G) of the context's basis; checks that
// the sphere fits the grid without folding.
lace_status pw_index(lace_ctx* c, std::vector<int2>& idx) {
    const auto b = basis(c->g.cell, c->ecut);
    for (const auto& t : b) {
        const int m[3] = {std::get<0>(t), std::get<1>(t), std::get<2>(t)};
        for (int a = 0; a < 3; ++a)
            if (2 * std::abs(m[a]) >= c->g.n[a])
                return ctx_fail(c, LACE_ERR_ARG, "the cutoff sphere does not fit the grid (|m| < n/2 on every axis)");
    }
    idx.resize(b.size());
    const int n1 = c->g.n[0], n2 = c->g.n[1], n3 = c->g.n[2];
    auto off = [&](int m1, int m2, int m3) {
        const int i1 = ((m1 % n1) + n1) % n1, i2 = ((m2 % n2) + n2) % n2, i3 = ((m3 % n3) + n3) % n3;
        return (i1 * n2 + i2) * n3 + i3;
    };
    for (size_t k = 0; k < b.size(); ++k) {
        const int m1 = std::get<0>(b[k]), m2 = std::get<1>(b[k]), m3 = std::get<2>(b[k]);
        idx[k] = make_int2(off(m1, m2, m3), off(-m1, -m2, -m3));
    }
    return LACE_OK;
}

size_t plane_smem(const GridGeom& g) { return sizeof(double2) * ((size_t)g.n[1] * g.n[2] + g.n[1] + g.n[2]); }
size_t slab_smem(const GridGeom& g) { return sizeof(double2) * ((size_t)g.n[0] * g.n[2] + g.n[0]); }

lace_status pw_prepare(lace_ctx* c, long long n_pw, int* batch) {
    if (!c->have_cell) return ctx_fail(c, LACE_ERR_STATE, "lace_set_cell must come first");
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    if (std::max(plane_smem(c->g), slab_smem(c->g)) > prop.sharedMemPerBlockOptin)
        return ctx_fail(c, LACE_ERR_UNSUPPORTED, "an FP64 grid plane does not fit in shared memory");
    std::vector<int2> idx;
    lace_status st = pw_index(c, idx);
    if (st) return st;
    if ((long long)idx.size() != n_pw) return ctx_fail(c, LACE_ERR_ARG, "coefficient count differs from the basis");
    if (c->pw_idx.ensure(sizeof(int2) * std::max<size_t>(idx.size(), 1)) != cudaSuccess ||
        cudaMemcpy(c->pw_idx.p, idx.data(), sizeof(int2) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, LACE_ERR_OOM, "plane-wave index table");
    }
    const int attrs[2] = {(int)plane_smem(c->g), (int)slab_smem(c->g)};
    cudaFuncSetAttribute(pw_plane_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, attrs[0]);
    cudaFuncSetAttribute(pw_plane_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, attrs[0]);
    cudaFuncSetAttribute(pw_xslab_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, attrs[1]);
    cudaFuncSetAttribute(pw_xslab_kernel<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, attrs[1]);
    *batch = (int)std::max<size_t>(1, std::min<size_t>(256, (512ull << 20) / (c->g.ng * sizeof(double2))));
    return LACE_OK;
}

}  // namespace

extern "C" {

lace_status lace_pw_basis(const double cell[3], double ecut_ha, int* m_out, long long cap, long long* n_pw_out) {
    if (!cell || !n_pw_out || !(cell[0] > 0) || !(cell[1] > 0) || !(cell[2] > 0) || !(ecut_ha > 0))
        return LACE_ERR_ARG;
    const auto b = basis(cell, ecut_ha);
    *n_pw_out = (long long)b.size();
    if (m_out)
        for (long long k = 0; k < std::min<long long>(cap, (long long)b.size()); ++k) {
            m_out[3 * k] = std::get<0>(b[k]);
            m_out[3 * k + 1] = std::get<1>(b[k]);
            m_out[3 * k + 2] = std::get<2>(b[k]);
        }
    return LACE_OK;
}

lace_status lace_grid_for_cutoff(const double cell[3], double ecut_ha, int dims_out[3]) {
    if (!cell || !dims_out || !(ecut_ha > 0)) return LACE_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (!(cell[a] > 0)) return LACE_ERR_ARG;
        const int mmax = (int)std::floor(std::sqrt(2.0 * ecut_ha) * cell[a] / (2.0 * M_PI));
        dims_out[a] = smooth235_at_least(2 * mmax + 1);
        if (dims_out[a] > kMaxN) return LACE_ERR_UNSUPPORTED;
    }
    return LACE_OK;
}

lace_status lace_load_orbitals_pw(lace_ctx* c, const double* coef, long long n_pw, int n_occ, int n_extra,
                                  int orthonormalize) {
    if (!c || !coef || n_occ < 1 || n_extra < 0) return LACE_ERR_ARG;
    cudaSetDevice(c->device);
    int batch = 0;
    lace_status st = pw_prepare(c, n_pw, &batch);
    if (st) return st;
    const int n_orb = n_occ + n_extra;
    const size_t ng = c->g.ng;
    const size_t cbytes = (size_t)n_orb * n_pw * sizeof(double2);
    // FP64 real-space orbitals go to a buffer of their own, read by the usual load
    if (c->pw_io.ensure(cbytes) != cudaSuccess || c->pw_real.ensure((size_t)n_orb * ng * sizeof(double)) != cudaSuccess ||
        c->scratch.ensure((size_t)batch * ng * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, LACE_ERR_OOM, "plane-wave buffers");
    }
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemcpyAsync(c->pw_io.p, coef, cbytes, cudaMemcpyHostToDevice, s);
    double2* grids = c->scratch.as<double2>();
    const int npairs = (n_orb + 1) / 2;
    for (int p0 = 0; p0 < npairs && e == cudaSuccess; p0 += batch) {
        const int nb = std::min(batch, npairs - p0);
        cudaMemsetAsync(grids, 0, (size_t)nb * ng * sizeof(double2), s);
        pw_scatter_kernel<<<dim3((unsigned)((n_pw + 255) / 256), nb), 256, 0, s>>>(
            c->pw_io.as<double2>(), n_pw, n_orb, p0, c->pw_idx.as<int2>(), grids, ng);
        pw_xslab_kernel<1><<<dim3(c->g.n[1], nb), PW_THREADS, slab_smem(c->g), s>>>(
            grids, ng, c->g.ax[0], c->g.n[1], c->g.n[2], c->tw_d[0].as<double2>());
        pw_plane_kernel<1><<<dim3(c->g.n[0], nb), PW_THREADS, plane_smem(c->g), s>>>(
            grids, ng, c->g.ax[1], c->g.ax[2], c->tw_d[1].as<double2>(), c->tw_d[2].as<double2>());
        pw_split_kernel<<<dim3(std::min<unsigned>(1024, (unsigned)((ng + 255) / 256)), nb), 256, 0, s>>>(
            grids, ng, n_orb, p0, c->pw_real.as<double>());
        c->launches += 4;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, LACE_ERR_CUDA, std::string("plane-wave transform: ") + cudaGetErrorString(e));
    }
    return ctx_load_dev64(c, c->pw_real.as<double>(), n_occ, n_extra, orthonormalize);
}

lace_status lace_get_orbitals_pw(lace_ctx* c, int which, double* coef_out, long long n_pw) {
    if (!c || !coef_out) return LACE_ERR_ARG;
    cudaSetDevice(c->device);
    const void* src = nullptr;
    lace_status st = ctx_orbitals(c, which, &src);
    if (st) return st;
    int batch = 0;
    if ((st = pw_prepare(c, n_pw, &batch))) return st;
    const int n_orb = c->n_p;
    const size_t ng = c->g.ng;
    const size_t cbytes = (size_t)n_orb * n_pw * sizeof(double2);
    if (c->pw_io.ensure(cbytes) != cudaSuccess || c->scratch.ensure((size_t)batch * ng * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, LACE_ERR_OOM, "plane-wave buffers");
    }
    cudaStream_t s = c->stream;
    double2* grids = c->scratch.as<double2>();
    const int npairs = (n_orb + 1) / 2;
    cudaError_t e = cudaSuccess;
    for (int p0 = 0; p0 < npairs && e == cudaSuccess; p0 += batch) {
        const int nb = std::min(batch, npairs - p0);
        const dim3 gp(std::min<unsigned>(1024, (unsigned)((ng + 255) / 256)), nb);
        if (c->prec == LACE_FP64)
            pw_pack_kernel<double><<<gp, 256, 0, s>>>(static_cast<const double*>(src), ng, n_orb, p0, grids);
        else
            pw_pack_kernel<float><<<gp, 256, 0, s>>>(static_cast<const float*>(src), ng, n_orb, p0, grids);
        pw_plane_kernel<-1><<<dim3(c->g.n[0], nb), PW_THREADS, plane_smem(c->g), s>>>(
            grids, ng, c->g.ax[1], c->g.ax[2], c->tw_d[1].as<double2>(), c->tw_d[2].as<double2>());
        pw_xslab_kernel<-1><<<dim3(c->g.n[1], nb), PW_THREADS, slab_smem(c->g), s>>>(
            grids, ng, c->g.ax[0], c->g.n[1], c->g.n[2], c->tw_d[0].as<double2>());
        pw_gather_kernel<<<dim3((unsigned)((n_pw + 255) / 256), nb), 256, 0, s>>>(grids, ng, n_pw, n_orb, p0,
                                                                                 c->pw_idx.as<int2>(),
                                                                                 c->pw_io.as<double2>());
        c->launches += 4;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(coef_out, c->pw_io.p, cbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(c, LACE_ERR_CUDA, std::string("plane-wave transform: ") + cudaGetErrorString(e));
    }
    return LACE_OK;
}

}  // extern "C"
