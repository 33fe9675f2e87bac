// C-ABI of liblace: context, state machine and orchestration of the
// exchange hot path of L-ACE (arXiv:1801.09263, Sec. 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lace.h"
#include "lace_internal.cuh"
#include "lace_ctx.cuh"

using namespace lace;

namespace {

lace_status fail(lace_ctx* c, lace_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

lace_status cuda_fail(lace_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(c, LACE_ERR_OOM, std::string(where) + ": out of device memory");
    }
    return fail(c, LACE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

lace_status ck_impl(lace_ctx* c, cudaError_t e, const char* where) {
    return e == cudaSuccess ? LACE_OK : cuda_fail(c, e, where);
}

// CK(expression, "where"): return a lace_status on a CUDA error.
#define CK(...)                                      \
    do {                                             \
        lace_status _st = ck_impl(c, __VA_ARGS__);   \
        if (_st != LACE_OK) return _st;              \
    } while (0)

bool good_size(int n) {
    if (n < 4 || n > kMaxN) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

size_t elem_bytes(const lace_ctx* c) { return c->prec == LACE_FP64 ? 8 : 4; }

void ev_begin(lace_ctx* c, int st) {
    cudaEventRecord(c->ev[2 * st], c->stream);
    c->ev_used[st] = true;
}
void ev_end(lace_ctx* c, int st) { cudaEventRecord(c->ev[2 * st + 1], c->stream); }

struct Launch {
    lace_ctx* c;
    int n = 0;
    ~Launch() { c->launches += n; }
};

// ------------------------------------------------------------------ tables
lace_status build_tables(lace_ctx* c) {
    for (int a = 0; a < 3; ++a) {
        const int n = c->g.n[a];
        std::vector<double2> twd(n);
        std::vector<float2> twf(n);
        std::vector<double> g2d(n);
        std::vector<float> g2f(n);
        for (int m = 0; m < n; ++m) {
            const double ang = -2.0 * M_PI * (double)m / (double)n;
            twd[m] = make_double2(std::cos(ang), std::sin(ang));
            twf[m] = make_float2((float)twd[m].x, (float)twd[m].y);
            const int mm = (m < (n + 1) / 2) ? m : m - n;
            const double gv = 2.0 * M_PI * (double)mm / c->g.cell[a];
            g2d[m] = gv * gv;
            g2f[m] = (float)g2d[m];
        }
        CK(c->tw_d[a].ensure(n * sizeof(double2)), "tables");
        CK(c->tw_f[a].ensure(n * sizeof(float2)), "tables");
        CK(c->g2_d[a].ensure(n * sizeof(double)), "tables");
        CK(c->g2_f[a].ensure(n * sizeof(float)), "tables");
        CK(cudaMemcpy(c->tw_d[a].p, twd.data(), n * sizeof(double2), cudaMemcpyHostToDevice), "tables");
        CK(cudaMemcpy(c->tw_f[a].p, twf.data(), n * sizeof(float2), cudaMemcpyHostToDevice), "tables");
        CK(cudaMemcpy(c->g2_d[a].p, g2d.data(), n * sizeof(double), cudaMemcpyHostToDevice), "tables");
        CK(cudaMemcpy(c->g2_f[a].p, g2f.data(), n * sizeof(float), cudaMemcpyHostToDevice), "tables");
    }
    // K(G)/Ng = 4 pi / (Ng |G|^2), K(0) = 0, evaluated in FP64 and rounded once:
    // rounding 4 pi/Ng and |G|^2 separately in FP32 biases every pair energy alike.
    const int n1 = c->g.n[0], n2 = c->g.n[1], n3 = c->g.n[2];
    std::vector<double> gx(n1), gy(n2), gz(n3);
    auto fill = [](std::vector<double>& v, int n, double len) {
        for (int m = 0; m < n; ++m) {
            const int mm = (m < (n + 1) / 2) ? m : m - n;
            const double gv = 2.0 * M_PI * (double)mm / len;
            v[m] = gv * gv;
        }
    };
    fill(gx, n1, c->g.cell[0]);
    fill(gy, n2, c->g.cell[1]);
    fill(gz, n3, c->g.cell[2]);
    // Kernels (scaled by the exchange fraction alpha):
    //   Coulomb:        4 pi / |G|^2, K(0) = 0;
    //   erfc-screened:  4 pi / |G|^2 (1 - exp(-|G|^2 / (4 omega^2))), the
    //                   short-range part of HSE, K(0) = pi / omega^2.
    std::vector<float> kt(c->g.ng);
    std::vector<double> ktd(c->g.ng);
    const double scale = 4.0 * M_PI / (double)c->g.ng;
    const bool erfc_k = c->kernel_kind == LACE_KERNEL_ERFC;
    const double w2 = c->kernel_omega * c->kernel_omega;
    for (int x = 0; x < n1; ++x)
        for (int y = 0; y < n2; ++y)
            for (int z = 0; z < n3; ++z) {
                const double gg = gx[x] + gy[y] + gz[z];
                double k;
                if (!erfc_k) k = gg > 0.0 ? scale / gg : 0.0;
                else k = gg > 0.0 ? scale / gg * -std::expm1(-gg / (4.0 * w2)) : M_PI / w2 / (double)c->g.ng;
                k *= c->kernel_alpha;
                const size_t i = ((size_t)x * n2 + y) * n3 + z;
                ktd[i] = k;
                kt[i] = (float)k;
            }
    CK(c->ktab_f.ensure(c->g.ng * sizeof(float)), "tables");
    CK(cudaMemcpy(c->ktab_f.p, kt.data(), c->g.ng * sizeof(float), cudaMemcpyHostToDevice), "tables");
    CK(c->ktab_d.ensure(c->g.ng * sizeof(double)), "tables");
    CK(cudaMemcpy(c->ktab_d.p, ktd.data(), c->g.ng * sizeof(double), cudaMemcpyHostToDevice), "tables");
    return LACE_OK;
}

template <typename T> FFTTables<T> tables(lace_ctx* c);
template <> FFTTables<double> tables<double>(lace_ctx* c) {
    FFTTables<double> t;
    for (int a = 0; a < 3; ++a) { t.tw[a] = c->tw_d[a].as<double2>(); t.g2[a] = c->g2_d[a].as<double>(); }
    t.ktab = c->ktab_d.as<double>();
    return t;
}
template <> FFTTables<float> tables<float>(lace_ctx* c) {
    FFTTables<float> t;
    for (int a = 0; a < 3; ++a) { t.tw[a] = c->tw_f[a].as<float2>(); t.g2[a] = c->g2_f[a].as<float>(); }
    t.ktab = c->ktab_f.as<float>();
    return t;
}

// ------------------------------------------------------------------ buffers
lace_status ensure_orbital_buffers(lace_ctx* c, int n_occ, int n_extra) {
    const int n_p = n_occ + n_extra;
    const size_t ng = c->g.ng, eb = elem_bytes(c);
    CK(c->psi.ensure((size_t)n_p * ng * eb), "alloc psi");
    CK(c->canon.ensure((size_t)n_occ * ng * eb), "alloc canon");
    CK(c->W.ensure((size_t)n_p * ng * eb), "alloc W");
    CK(c->stage64.ensure((size_t)n_p * ng * 8), "alloc staging");
    c->mslot = (size_t)n_p * n_p + 64 * (size_t)n_p + 64;
    CK(c->mat.ensure(c->mslot * kMatSlots * sizeof(double)), "alloc matrices");
    const size_t wk = std::max(gemm_rows_work_elems(n_p, n_p, ng), (size_t)1);
    CK(c->work.ensure(wk * sizeof(double)), "alloc work");
    CK(c->flag.ensure(64), "alloc flag");
    CK(c->exd.ensure((8 + 2 * kSumBlocks) * sizeof(double)), "alloc exd");  // [0] E_x, [1] ACE energy, sum scratch
    CK(c->counts.ensure(sizeof(int) * (2 * (size_t)n_occ + 2)), "alloc counts");
    return LACE_OK;
}

// Loewdin coefficients: X = S^{-1/2}, S = dV src src^T (FP64 Newton-Schulz;
// mixed path: FP32 Newton-Schulz and one FP64 first-order refinement).
template <typename T>
lace_status lowdin_coeffs(lace_ctx* c, const T* src, int n, double* X, Launch& L) {
    const size_t ng = c->g.ng;
    double* S = c->m(MS_A);
    CK(gemm_rows<T>(n, n, ng, src, ng, src, ng, c->g.dv, false, S, n, c->work.as<double>(),
                    c->work.bytes / sizeof(double), c->stream, &L.n),
       "loewdin overlap");
    int ok = 0;
    if (c->prec == LACE_FP64) {
        CK(inv_sqrt_spd(n, S, X, c->m(MS_NSWORK), c->flag.as<int>(), &ok, c->stream, &L.n), "loewdin inverse sqrt");
    } else {
        // FP32 Newton-Schulz, then one FP64 first-order Loewdin step on X^T S X
        CK(inv_sqrt_spd_mixed(n, S, X, c->m(MS_NSWORK), &ok, c->stream, &L.n), "loewdin inverse sqrt");
        if (ok) CK(lowdin_refine(n, X, S, c->m(MS_NSWORK), c->stream, &L.n), "loewdin refine");
    }
    if (!ok) return fail(c, LACE_ERR_NOT_PD, "overlap matrix is singular or ill-conditioned (inverse square root did not converge)");
    return LACE_OK;
}

// Loewdin: dst[n] = sum_k src[k] X[k][n], X = S^{-1/2}, S = dV src src^T.
template <typename T>
lace_status lowdin_rows(lace_ctx* c, const T* src, int n, T* dst, Launch& L) {
    double* X = c->m(MS_B);
    lace_status st = lowdin_coeffs<T>(c, src, n, X, L);
    if (st) return st;
    CK(gemm_combine<T>(n, c->g.ng, n, src, c->g.ng, X, n, 0.0, dst, c->g.ng, c->stream, &L.n), "loewdin combine");
    return LACE_OK;
}

// The occupied orbitals stay raw (canon buffer) with their Loewdin
// coefficients X: localisation folds X into its rotation (one combination
// over the grid instead of two), and psi is formed only when needed.
template <typename T>
lace_status load_impl(lace_ctx* c, const double* d_phi64, int n_occ, int n_extra, int ortho) {
    Launch L{c};
    const size_t ng = c->g.ng;
    T* psi = c->psi.as<T>();
    T* raw = c->canon.as<T>();
    double* X = c->m(MS_X);
    CK(convert<double, T>(d_phi64, raw, (size_t)n_occ * ng, c->stream, &L.n), "load convert");
    c->x_identity = !ortho;
    c->psi_occ_ready = false;
    if (ortho) {
        lace_status st = lowdin_coeffs<T>(c, raw, n_occ, X, L);
        if (st) return st;
    }
    if (n_extra > 0) {
        T* ex_raw = c->W.as<T>();  // staging
        CK(convert<double, T>(d_phi64 + (size_t)n_occ * ng, ex_raw, (size_t)n_extra * ng, c->stream, &L.n),
           "load convert");
        if (ortho) {
            // extra -= canon (dV canon^T extra), canon = raw X:  coefficients -X X^T G,
            // G = dV raw^T extra
            double* G = c->m(MS_A);
            double* T1 = c->m(MS_B);
            double* D = c->m(MS_LINV);
            CK(gemm_rows<T>(n_occ, n_extra, ng, raw, ng, ex_raw, ng, c->g.dv, false, G, n_extra, c->work.as<double>(),
                            c->work.bytes / sizeof(double), c->stream, &L.n),
               "extras projection");
            CK(small_gemm_f64(n_occ, n_extra, n_occ, X, n_occ, true, G, n_extra, false, 1.0, 0.0, T1, n_extra,
                              c->stream, &L.n),
               "extras projection");
            CK(small_gemm_f64(n_occ, n_extra, n_occ, X, n_occ, false, T1, n_extra, false, -1.0, 0.0, D, n_extra,
                              c->stream, &L.n),
               "extras projection");
            CK(gemm_combine<T>(n_extra, ng, n_occ, raw, ng, D, n_extra, 1.0, ex_raw, ng, c->stream, &L.n),
               "extras projection");
            lace_status st = lowdin_rows<T>(c, ex_raw, n_extra, psi + (size_t)n_occ * ng, L);
            if (st) return st;
        } else {
            CK(cudaMemcpyAsync(psi + (size_t)n_occ * ng, ex_raw, (size_t)n_extra * ng * sizeof(T),
                               cudaMemcpyDeviceToDevice, c->stream),
               "load");
        }
    }
    return LACE_OK;
}

// psi[0 .. n_occ) = canon X, the canonical orbitals (when not localised).
template <typename T>
lace_status materialize_impl(lace_ctx* c) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_occ;
    if (c->x_identity) {
        CK(cudaMemcpyAsync(c->psi.p, c->canon.p, (size_t)n * ng * sizeof(T), cudaMemcpyDeviceToDevice, c->stream),
           "orbitals");
    } else {
        CK(gemm_combine<T>(n, ng, n, c->canon.as<T>(), ng, c->m(MS_X), n, 0.0, c->psi.as<T>(), ng, c->stream, &L.n),
           "loewdin combine");
    }
    return LACE_OK;
}

lace_status materialize_psi(lace_ctx* c) {
    if (c->psi_occ_ready) return LACE_OK;
    lace_status st = c->prec == LACE_FP64 ? materialize_impl<double>(c) : materialize_impl<float>(c);
    if (st == LACE_OK) c->psi_occ_ready = true;
    return st;
}

lace_status load_common(lace_ctx* c, const double* phi, bool dev, int n_occ, int n_extra, int ortho) {
    if (!c) return LACE_ERR_ARG;
    if (!c->have_cell) return fail(c, LACE_ERR_STATE, "lace_set_cell must come first");
    if (!phi || n_occ < 1 || n_extra < 0 || n_occ > 1024 || n_occ + n_extra > 2048)
        return fail(c, LACE_ERR_ARG, "bad orbital pointer or counts (1 <= n_occ <= 1024, n_occ + n_extra <= 2048)");
    cudaSetDevice(c->device);
    // The ACE projector of the last successful build stays usable across new
    // orbitals of the same count (the inner loop of the paper's double loop
    // applies the previous outer iteration's ACE), until the next build.
    c->loaded = c->localized = c->screened = c->applied = false;
    if (n_occ + n_extra != c->n_p) c->ace = false;
    lace_status st = ensure_orbital_buffers(c, n_occ, n_extra);
    if (st) return st;
    c->n_occ = n_occ;
    c->n_extra = n_extra;
    c->n_p = n_occ + n_extra;
    ev_begin(c, ST_LOAD);
    const size_t bytes = (size_t)c->n_p * c->g.ng * sizeof(double);
    const double* src = phi;
    if (!dev) {
        CK(cudaMemcpyAsync(c->stage64.p, phi, bytes, cudaMemcpyHostToDevice, c->stream), "upload");
        src = c->stage64.as<double>();
    }
    st = c->prec == LACE_FP64 ? load_impl<double>(c, src, n_occ, n_extra, ortho)
                              : load_impl<float>(c, src, n_occ, n_extra, ortho);
    ev_end(c, ST_LOAD);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "load");
    c->loaded = true;
    return LACE_OK;
}

// ------------------------------------------------------------------ SCDM
template <typename T>
lace_status localize_impl(lace_ctx* c, int stride, const long long* imposed) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_occ;
    T* raw = c->canon.as<T>();
    const double* X = c->m(MS_X);
    CK(c->pivfull.ensure(sizeof(long long) * n), "alloc pivots");
    long long* d_full = c->pivfull.as<long long>();
    if (!imposed) {
        int ncol = 0;
        const int m1 = (c->g.n[0] + stride - 1) / stride, m2 = (c->g.n[1] + stride - 1) / stride,
                  m3 = (c->g.n[2] + stride - 1) / stride;
        const size_t ncol_sz = (size_t)m1 * m2 * m3;
        if (ncol_sz < (size_t)n) return fail(c, LACE_ERR_ARG, "subsample has fewer points than orbitals");
        const size_t need = (size_t)n * ncol_sz * sizeof(T);
        if (c->work.bytes < need) CK(c->work.ensure(need), "alloc qrcp");
        CK(c->aux.ensure(qrcp_aux_bytes(n, (int)ncol_sz)), "alloc qrcp aux");
        CK(c->piv.ensure(sizeof(int) * n), "alloc pivots");
        T* R = c->work.as<T>();
        // the canonical orbitals on the subsample: (raw on the subsample) X
        if (c->x_identity) {
            CK(gather_subsample<T>(c->g, stride, raw, n, R, &ncol, c->stream, &L.n), "subsample");
        } else {
            T* tmp = c->W.as<T>();
            CK(gather_subsample<T>(c->g, stride, raw, n, tmp, &ncol, c->stream, &L.n), "subsample");
            CK(gemm_combine<T>(n, (size_t)ncol, n, tmp, (size_t)ncol, X, n, 0.0, R, (size_t)ncol, c->stream, &L.n),
               "subsample");
        }
        int timeout = 0;
        CK(qrcp_pivots<T>(n, ncol, R, n, c->piv.as<int>(), c->aux.p, &timeout, c->wait_limit_ns, c->stream, &L.n),
           "qrcp");
        if (timeout) return fail(c, LACE_ERR_TIMEOUT, "pivoted QR: a grid barrier wait timed out");
        std::vector<int> hp(n);
        CK(cudaMemcpyAsync(hp.data(), c->piv.p, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream), "pivots");
        CK(cudaStreamSynchronize(c->stream), "pivots");
        c->pivots_host.resize(n);
        for (int k = 0; k < n; ++k) {
            const int cc = hp[k];
            const int kz = cc % m3, jy = (cc / m3) % m2, ix = cc / (m3 * m2);
            c->pivots_host[k] = ((long long)(ix * stride) * c->g.n[1] + (long long)(jy * stride)) * c->g.n[2] +
                                (long long)(kz * stride);
        }
    } else {
        c->pivots_host.assign(imposed, imposed + n);
    }
    CK(cudaMemcpyAsync(d_full, c->pivots_host.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, c->stream),
       "pivots");
    double* phic = c->m(MS_A);
    double* B = c->m(MS_B);
    double* Bmh = c->m(MS_LINV);
    double* U = c->m(MS_U);
    // phi_C = canonical orbitals at the pivot points = (raw at the points) X
    if (c->x_identity) {
        CK(gather_columns<T>(raw, ng, n, d_full, n, phic, c->stream, &L.n), "gather phi_C");
    } else {
        double* phir = c->m(MS_E);
        CK(gather_columns<T>(raw, ng, n, d_full, n, phir, c->stream, &L.n), "gather phi_C");
        CK(small_gemm_f64(n, n, n, phir, n, false, X, n, false, 1.0, 0.0, phic, n, c->stream, &L.n), "gather phi_C");
    }
    // B = phi_C phi_C^T  (points x points)
    CK(small_gemm_f64(n, n, n, phic, n, false, phic, n, true, 1.0, 0.0, B, n, c->stream, &L.n), "scdm B");
    int ok = 0;
    if (c->prec == LACE_FP64) {
        CK(inv_sqrt_spd(n, B, Bmh, c->m(MS_NSWORK), c->flag.as<int>(), &ok, c->stream, &L.n), "scdm inverse sqrt");
    } else {
        CK(inv_sqrt_spd_mixed(n, B, Bmh, c->m(MS_NSWORK), &ok, c->stream, &L.n), "scdm inverse sqrt");
    }
    if (!ok) return fail(c, LACE_ERR_NOT_PD, "selected columns are rank deficient");
    // U = phi_C^T B^{-1/2}  (orbitals x orbitals)
    CK(small_gemm_f64(n, n, n, phic, n, true, Bmh, n, false, 1.0, 0.0, U, n, c->stream, &L.n), "scdm U");
    // mixed path: restore exact orthogonality of U in FP64 (U <- U (I - (U^T U - I)/2))
    if (c->prec != LACE_FP64) CK(lowdin_refine(n, U, nullptr, c->m(MS_NSWORK), c->stream, &L.n), "scdm refine");
    // w = canon U = raw (X U): one combination over the grid
    const double* Cf = U;
    if (!c->x_identity) {
        double* XU = c->m(MS_LINVT);
        CK(small_gemm_f64(n, n, n, X, n, false, U, n, false, 1.0, 0.0, XU, n, c->stream, &L.n), "scdm rotate");
        Cf = XU;
    }
    CK(gemm_combine<T>(n, ng, n, raw, ng, Cf, n, 0.0, c->psi.as<T>(), ng, c->stream, &L.n), "scdm rotate");
    c->psi_occ_ready = true;
    return LACE_OK;
}

// ------------------------------------------------------------------ alignment
// w <- w Q, Q the polar factor of O = dV w ref^T (orthogonal Procrustes):
// Q = O (O^T O)^{-1/2}, the FP64 Newton-Schulz inverse square root.
template <typename T>
lace_status align_impl(lace_ctx* c) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_occ;
    T* w = c->psi.as<T>();
    T* ref = c->ref.as<T>();
    double* Om = c->m(MS_A);
    double* P = c->m(MS_B);
    double* Pmh = c->m(MS_LINV);
    double* Q = c->m(MS_LINVT);
    CK(gemm_rows<T>(n, n, ng, w, ng, ref, ng, c->g.dv, false, Om, n, c->work.as<double>(),
                    c->work.bytes / sizeof(double), c->stream, &L.n),
       "alignment overlap");
    CK(small_gemm_f64(n, n, n, Om, n, true, Om, n, false, 1.0, 0.0, P, n, c->stream, &L.n), "alignment");
    int ok = 0;
    CK(inv_sqrt_spd(n, P, Pmh, c->m(MS_NSWORK), c->flag.as<int>(), &ok, c->stream, &L.n), "alignment");
    if (!ok) return fail(c, LACE_ERR_NOT_PD, "the orbitals are nearly orthogonal to the previous ones (no alignment)");
    CK(small_gemm_f64(n, n, n, Om, n, false, Pmh, n, false, 1.0, 0.0, Q, n, c->stream, &L.n), "alignment");
    // the SCDM rotation now includes Q
    double* U = c->m(MS_U);
    double* UQ = c->m(MS_B);
    CK(small_gemm_f64(n, n, n, U, n, false, Q, n, false, 1.0, 0.0, UQ, n, c->stream, &L.n), "alignment");
    CK(cudaMemcpyAsync(U, UQ, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream), "alignment");
    T* tmp = c->W.as<T>();
    CK(gemm_combine<T>(n, ng, n, w, ng, Q, n, 0.0, tmp, ng, c->stream, &L.n), "alignment");
    CK(cudaMemcpyAsync(w, tmp, (size_t)n * ng * sizeof(T), cudaMemcpyDeviceToDevice, c->stream), "alignment");
    return LACE_OK;
}

// ------------------------------------------------------------------ screening
// Timeout flags of the tensor-core calls (see lace_ctx::hflags): a call
// takes slot s of the device flags (or, with none left, waits for its own,
// h_err != nullptr), and tc_flag_copy queues the slot's copy to the pinned
// host flags; tc_timed_out, after the API call's stream synchronisation,
// reports whether any of them gave up.
struct TcFlag {
    int* d = nullptr;  // device slot
    int* h = nullptr;  // host word to wait on (synchronous mode) or nullptr
    int s = -1;
    int herr = 0;
};
TcFlag tc_flag(lace_ctx* c) {
    TcFlag f;
    if (c->hflags && c->tc_next < kFlagSlots) {
        f.s = c->tc_next++;
        c->hflags[f.s] = 0;
        f.d = c->flag.as<int>() + f.s;
    } else {
        f.d = c->flag.as<int>() + 1;
        f.h = &f.herr;
    }
    return f;
}
cudaError_t tc_flag_copy(lace_ctx* c, const TcFlag& f) {
    if (f.s < 0) return cudaSuccess;
    return cudaMemcpyAsync(c->hflags + f.s, f.d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
}
bool tc_timed_out(lace_ctx* c) {
    bool any = false;
    for (int k = 2; k < c->tc_next; ++k) any |= c->hflags[k] != 0;
    c->tc_next = 2;
    return any;
}

// S_ik = dV sum_r |psi_i(r)| |psi_k(r)| (Eq. 4).  Mixed path: tcgen05 3xBF16
// (S only decides which pairs pass the threshold; the Gram's periodic
// compensated drains keep it ~1e-7 relative), symmetric tiles only; FP64 and
// grids whose point count is not a multiple of 4: the CUDA-core kernel.
template <typename T>
lace_status screen_impl(lace_ctx* c, double thr) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_occ;
    const T* psi = c->psi.as<T>();
    if constexpr (std::is_same<T, float>::value) {
        const char* notc = getenv("LACE_NO_TC");
        if (!(notc && notc[0] == '1') && ng % 4 == 0 && (uintptr_t)psi % 16 == 0) {
            CK(c->work.ensure(std::max(c->work.bytes, tc_gram_work_elems(n, n, ng, true) * sizeof(double))),
               "alloc work");
            TcFlag f = tc_flag(c);
            CK(tc_gram(n, n, ng, psi, ng, psi, ng, c->g.dv, c->m(MS_S), n, c->work.as<double>(),
                       c->work.bytes / sizeof(double), f.d, f.h, c->stream, &L.n, true, true),
               "overlap of moduli");
            if (f.herr) return fail(c, LACE_ERR_TIMEOUT, "overlap of moduli: an mbarrier wait timed out");
            CK(tc_flag_copy(c, f), "flags");
            return LACE_OK;
        }
    }
    CK(gemm_rows<T>(n, n, ng, psi, ng, psi, ng, c->g.dv, true, c->m(MS_S), n, c->work.as<double>(),
                    c->work.bytes / sizeof(double), c->stream, &L.n),
       "overlap of moduli");
    return LACE_OK;
}

lace_status make_pairs(lace_ctx* c, bool use_S, double thr, Launch& L) {
    const int n = c->n_occ, ne = c->n_extra;
    const size_t maxp = (size_t)n * (n + 1) / 2 + (size_t)n * ne;
    CK(c->pairs.ensure(sizeof(int2) * std::max<size_t>(maxp, 1)), "alloc pairs");
    CK(c->grids.ensure(sizeof(PairGrid) * std::max<size_t>((maxp + 1) / 2, 1)), "alloc grids");
    long long np = 0;
    CK(build_pair_list(n, ne, c->m(MS_S), thr, use_S, c->pairs.as<int2>(), c->counts.as<int>(), &np, c->stream, &L.n),
       "pair list");
    // Localised orbitals: order the pairs by the Z-order rank of their orbitals'
    // SCDM points, so consecutive FFT grids touch nearby orbitals and their W
    // and Psi planes stay in L2.  Each pair keeps (i, j) with i <= j.
    const char* noord = getenv("LACE_NO_PAIR_ORDER");
    if (c->localized && np > 1 && (int)c->pivots_host.size() == n && !(noord && noord[0] == '1')) {
        std::vector<int2> hp(np);
        CK(cudaMemcpyAsync(hp.data(), c->pairs.p, sizeof(int2) * np, cudaMemcpyDeviceToHost, c->stream), "pairs");
        CK(cudaStreamSynchronize(c->stream), "pairs");
        auto spread = [](uint64_t v) {  // interleave 21 bits with two zero bits
            v &= 0x1fffff;
            v = (v | v << 32) & 0x1f00000000ffffULL;
            v = (v | v << 16) & 0x1f0000ff0000ffULL;
            v = (v | v << 8) & 0x100f00f00f00f00fULL;
            v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
            v = (v | v << 2) & 0x1249249249249249ULL;
            return v;
        };
        std::vector<std::pair<uint64_t, int>> code(n);
        for (int i = 0; i < n; ++i) {
            const long long p = c->pivots_host[i];
            const uint64_t z = p % c->g.n[2], y = (p / c->g.n[2]) % c->g.n[1], x = p / ((long long)c->g.n[2] * c->g.n[1]);
            code[i] = {spread(x) << 2 | spread(y) << 1 | spread(z), i};
        }
        std::sort(code.begin(), code.end());
        std::vector<int> rank(n + ne);
        for (int r = 0; r < n; ++r) rank[code[r].second] = r;
        for (int e = 0; e < ne; ++e) rank[n + e] = n + e;
        std::stable_sort(hp.begin(), hp.end(), [&](const int2& a, const int2& b) {
            const int a0 = std::min(rank[a.x], rank[a.y]), a1 = std::max(rank[a.x], rank[a.y]);
            const int b0 = std::min(rank[b.x], rank[b.y]), b1 = std::max(rank[b.x], rank[b.y]);
            return a0 != b0 ? a0 < b0 : a1 < b1;
        });
        CK(cudaMemcpyAsync(c->pairs.p, hp.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, c->stream), "pairs");
        CK(cudaStreamSynchronize(c->stream), "pairs");
    }
    CK(pack_pair_grids(c->pairs.as<int2>(), np, c->grids.as<PairGrid>(), c->stream, &L.n), "pack pairs");
    c->n_pairs = np;
    return LACE_OK;
}

// Complex grids per batch of the FFT passes within a scratch budget (2 GiB by
// default: fewer, fuller launches; at 72^3 the pair convolutions ran 2.86,
// 2.75, 2.71 and 2.69 us per pair with 128, 256, 512 and 1024 grids a batch).
int batch_for_sizes(size_t ng, size_t eb, size_t budget) {
    const size_t per = ng * 2 * eb;
    const char* envb = getenv("LACE_BATCH");
    long long b = envb ? atoll(envb) : (long long)(budget / per);
    b = std::max<long long>(4, std::min<long long>(b, 1024));
    return (int)b;
}
int batch_for(lace_ctx* c) { return batch_for_sizes(c->g.ng, elem_bytes(c), c->fft_scratch_budget); }

// ------------------------------------------------------------------ exchange
template <typename T>
lace_status apply_impl(lace_ctx* c) {
    Launch L{c};
    const size_t ng = c->g.ng;
    if (!c->screened) {
        lace_status st = make_pairs(c, false, 0.0, L);
        if (st) return st;
        c->screened = true;
        c->s_thr = 0.0;
    }
    const long long n_grids = (c->n_pairs + 1) / 2;
    const int batch = (int)std::min<long long>(batch_for(c), std::max<long long>(n_grids, 1));
    CK(c->scratch.ensure((size_t)batch * ng * 2 * sizeof(T)), "alloc FFT scratch");
    CK(c->epart.ensure((size_t)batch * c->g.n[0] * 2 * sizeof(double)), "alloc energies");
    CK(cudaMemsetAsync(c->W.p, 0, (size_t)c->n_p * ng * sizeof(T), c->stream), "zero W");
    CK(fill_zero_f64(c->m(MS_E), (size_t)c->n_occ * c->n_occ, c->stream, &L.n), "zero E");
    CK(pairconv_run<T>(c->g, tables<T>(c), c->psi.as<T>(), c->n_occ, c->W.as<T>(), c->grids.as<PairGrid>(),
                       (int)n_grids, c->scratch.as<cplx<T>>(), batch, c->epart.as<double>(), c->m(MS_E), c->stream,
                       &L.n, c->ev[2 * ST_PAIRCONV], c->ev[2 * ST_PAIRCONV + 1]),
       "pair convolutions");
    c->ev_used[ST_PAIRCONV] = true;
    CK(exchange_energy_sum(c->n_occ, c->m(MS_E), c->exd.as<double>() + 8, c->exd.as<double>(), c->stream, &L.n),
       "energy");
    return LACE_OK;
}

// The exchange application split around its pair convolutions, for merged
// launches of the request server: the part before them (pair list, scratch,
// W and pair energies zeroed) and the part after (E_x from the pair
// energies).  Mixed precision only.
lace_status exchange_prepare_f(lace_ctx* c, MergedSys<float>* m, int* n_grids_out, int* cap_out) {
    Launch L{c};
    const size_t ng = c->g.ng;
    if (!c->screened) {
        lace_status st = make_pairs(c, false, 0.0, L);
        if (st) return st;
        c->screened = true;
        c->s_thr = 0.0;
    }
    const long long n_grids = (c->n_pairs + 1) / 2;
    const int batch = (int)std::min<long long>(batch_for(c), std::max<long long>(n_grids, 1));
    CK(c->scratch.ensure((size_t)batch * ng * 2 * sizeof(float)), "alloc FFT scratch");
    CK(c->epart.ensure((size_t)batch * c->g.n[0] * 2 * sizeof(double)), "alloc energies");
    CK(cudaMemsetAsync(c->W.p, 0, (size_t)c->n_p * ng * sizeof(float), c->stream), "zero W");
    CK(fill_zero_f64(c->m(MS_E), (size_t)c->n_occ * c->n_occ, c->stream, &L.n), "zero E");
    m->psi = c->psi.as<float>();
    m->W = c->W.as<float>();
    m->ktab = c->ktab_f.as<float>();
    m->grids = c->grids.as<PairGrid>();
    m->scratch = c->scratch.as<float2>();
    m->epart = c->epart.as<double>();
    m->E = c->m(MS_E);
    m->n_occ = c->n_occ;
    m->g0 = 0;
    m->dv = c->g.dv;
    *n_grids_out = (int)n_grids;
    *cap_out = batch;
    return LACE_OK;
}

lace_status exchange_finish(lace_ctx* c) {
    Launch L{c};
    CK(exchange_energy_sum(c->n_occ, c->m(MS_E), c->exd.as<double>() + 8, c->exd.as<double>(), c->stream, &L.n),
       "energy");
    return LACE_OK;
}

// ------------------------------------------------------------------ ACE
// Dense contraction over the grid for the ACE matrices: tcgen05 3xBF16 on the
// mixed path (LACE_NO_TC=1 selects the CUDA-core FP32 kernel), FP64 otherwise.
// The tensor-core kernel reads rows with 16-byte loads, so grids whose point
// count is not a multiple of 4 take the CUDA-core kernel.
template <typename T>
lace_status ace_contract(lace_ctx* c, int M, int N, const T* A, const T* B, double alpha, double* C, Launch& L) {
    const size_t ng = c->g.ng;
    if constexpr (std::is_same<T, float>::value) {
        const char* notc = getenv("LACE_NO_TC");
        const bool aligned = ng % 4 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0;
        if (!(notc && notc[0] == '1') && aligned) {
            CK(c->work.ensure(std::max(c->work.bytes, tc_gram_work_elems(M, N, ng) * sizeof(double))), "alloc work");
            TcFlag f = tc_flag(c);
            CK(tc_gram(M, N, ng, A, ng, B, ng, alpha, C, N, c->work.as<double>(), c->work.bytes / sizeof(double),
                       f.d, f.h, c->stream, &L.n),
               "tensor-core contraction");
            if (f.herr) return fail(c, LACE_ERR_TIMEOUT, "tensor-core contraction: an mbarrier wait timed out");
            CK(tc_flag_copy(c, f), "flags");
            return LACE_OK;
        }
    }
    CK(c->work.ensure(std::max(c->work.bytes, gemm_rows_work_elems(M, N, ng) * sizeof(double))), "alloc work");
    CK(gemm_rows<T>(M, N, ng, A, ng, B, ng, alpha, false, C, N, c->work.as<double>(), c->work.bytes / sizeof(double),
                    c->stream, &L.n),
       "contraction");
    return LACE_OK;
}

// Out[n] = sum_k Coef[k][n] A[k] over the grid for the ACE vectors: tcgen05
// 3xBF16 on the mixed path (LACE_NO_TC=1: CUDA-core FP32), FP64 otherwise.
// Out may be FP64 on the mixed path (the ACE apply's result, written by the
// tensor-core epilogue directly); the CUDA-core form then goes through an FP32
// buffer and a conversion.
template <typename T, typename TO>
lace_status ace_combine(lace_ctx* c, int N, int Kc, const T* A, const double* Coef, TO* Out, Launch& L) {
    const size_t ng = c->g.ng;
    if constexpr (std::is_same<T, float>::value) {
        const char* notc = getenv("LACE_NO_TC");
        if (!(notc && notc[0] == '1')) {
            CK(c->work.ensure(std::max(c->work.bytes, tc_combine_scratch_bytes(N, Kc))), "alloc work");
            TcFlag f = tc_flag(c);
            CK(tc_combine(N, ng, Kc, A, ng, Coef, N, 0.0, Out, ng, c->work.p, f.d, f.h, c->stream, &L.n),
               "tensor-core combination");
            if (f.herr) return fail(c, LACE_ERR_TIMEOUT, "tensor-core combination: an mbarrier wait timed out");
            CK(tc_flag_copy(c, f), "flags");
            return LACE_OK;
        }
    }
    if constexpr (std::is_same<T, TO>::value) {
        CK(gemm_combine<T>(N, ng, Kc, A, ng, Coef, N, 0.0, Out, ng, c->stream, &L.n), "combination");
    } else {
        CK(c->scratch.ensure((size_t)2 * N * ng * sizeof(T)), "alloc combination");
        T* tmp = c->scratch.as<T>() + (size_t)N * ng;  // past the staged input of the ACE apply
        CK(gemm_combine<T>(N, ng, Kc, A, ng, Coef, N, 0.0, tmp, ng, c->stream, &L.n), "combination");
        CK(convert<T, TO>(tmp, Out, (size_t)N * ng, c->stream, &L.n), "convert out");
    }
    return LACE_OK;
}

template <typename T>
lace_status build_ace_impl(lace_ctx* c, int sym) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_p;
    CK(c->xi.ensure((size_t)n * ng * sizeof(T)), "alloc xi");
    double* M = c->m(MS_M);
    double* A = c->m(MS_MSYM);
    double* Linv = c->m(MS_LINV);
    double* LinvT = c->m(MS_LINVT);
    {
        lace_status st = ace_contract<T>(c, n, n, c->psi.as<T>(), c->W.as<T>(), c->g.dv, M, L);
        if (st) return st;
    }
    CK(symmetrize(n, M, A, sym, true, c->stream, &L.n), "symmetrize");
    int ok = 0;
    CK(cholesky_lower(n, A, n, c->flag.as<int>(), &ok, c->stream, &L.n), "cholesky");
    // (the Cholesky's flag read synchronised the stream: the Gram's flag is in)
    if (c->hflags && tc_timed_out(c))
        return fail(c, LACE_ERR_TIMEOUT, "tensor-core contraction: an mbarrier wait timed out");
    if (!ok) return fail(c, LACE_ERR_NOT_PD, "-M' is not positive definite (Cholesky failed)");
    CK(cudaMemcpyAsync(c->m(MS_L), A, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, c->stream), "copy L");
    CK(trtri_lower(n, A, n, Linv, n, c->stream, &L.n), "trtri");
    CK(transpose_f64(n, Linv, LinvT, c->stream, &L.n), "transpose");
    // xi_k = sum_j W_j (L^{-T})_{jk} = sum_j W_j Linv[k][j]: Coef[j][k] = LinvT[j][k]
    {
        lace_status st = ace_combine<T, T>(c, n, n, c->W.as<T>(), LinvT, c->xi.as<T>(), L);
        if (st) return st;
    }
    return LACE_OK;
}

// chunk >= 0: one chunk of a pipelined host apply; its share of the ACE
// energy goes to exd[2 + chunk] (summed into exd[1] after the last chunk).
template <typename T>
lace_status apply_ace_impl(lace_ctx* c, const double* d_psi64, int nf, double* d_out64, int chunk = -1) {
    Launch L{c};
    const size_t ng = c->g.ng;
    const int n = c->n_p;
    // staging for psi and result in working precision: use the FFT scratch
    CK(c->scratch.ensure((size_t)2 * nf * ng * sizeof(T)), "alloc ace apply");
    T* f = c->scratch.as<T>();
    const T* in = nullptr;
    if (sizeof(T) == 8) {
        in = reinterpret_cast<const T*>(d_psi64);
    } else {
        CK(convert<double, T>(d_psi64, f, (size_t)nf * ng, c->stream, &L.n), "convert psi");
        in = f;
    }
    double* X = c->m(MS_A);
    if ((size_t)n * nf > c->mslot) return fail(c, LACE_ERR_ARG, "too many functions in one ACE apply");
    {
        lace_status st = ace_contract<T>(c, n, nf, c->xi.as<T>(), in, -c->g.dv, X, L);
        if (st) return st;
    }
    // the block's ACE energy sum_j <psi_j|K_ACE|psi_j> = dV psi^T xi X = -|X|^2
    CK(neg_sum_squares((size_t)n * nf, X, c->exd.as<double>() + 8 + kSumBlocks,
                       c->exd.as<double>() + (chunk < 0 ? 1 : 2 + chunk), c->stream, &L.n),
       "ace energy");
    // K_ACE psi straight into the FP64 result (mixed path: the tensor-core
    // epilogue widens its FP32 accumulators as it stores them)
    return ace_combine<T, double>(c, nf, n, c->xi.as<T>(), X, d_out64, L);
}

template <typename T>
lace_status copy_orbitals_out(lace_ctx* c, const T* src, size_t count, double* host) {
    Launch L{c};
    if (sizeof(T) == 8) {
        CK(cudaMemcpyAsync(host, src, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "download");
    } else {
        CK(c->stage64.ensure(count * sizeof(double)), "alloc staging");
        CK(convert<T, double>(src, c->stage64.as<double>(), count, c->stream, &L.n), "convert");
        CK(cudaMemcpyAsync(host, c->stage64.p, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "download");
    }
    CK(cudaStreamSynchronize(c->stream), "download");
    return LACE_OK;
}

}  // namespace

namespace lace {

lace_status ctx_fail(lace_ctx* c, lace_status st, const std::string& msg) { return fail(c, st, msg); }

bool ctx_mergeable(lace_ctx* c) {
    return c && c->prec == LACE_MIXED && c->loaded && c->g.n[0] == c->g.n[1] && c->g.n[1] == c->g.n[2] &&
           spec_merge_ok(c->g.n[0]);
}

lace_status ctx_exchange_prepare(lace_ctx* c, MergedSys<float>* m, int* n_grids, int* cap, cudaEvent_t ready) {
    if (!ctx_mergeable(c)) return fail(c, LACE_ERR_STATE, "not a mixed-precision context on a merged grid size");
    cudaSetDevice(c->device);
    c->applied = false;
    lace_status st = materialize_psi(c);
    if (st) return st;
    ev_begin(c, ST_EXCHANGE);
    st = exchange_prepare_f(c, m, n_grids, cap);
    if (st) return st;
    CK(cudaEventRecord(ready, c->stream), "exchange");
    return LACE_OK;
}

lace_status ctx_exchange_finish(lace_ctx* c, cudaEvent_t done, double* ex_out) {
    cudaSetDevice(c->device);
    CK(cudaStreamWaitEvent(c->stream, done, 0), "exchange");
    lace_status st = exchange_finish(c);
    ev_end(c, ST_EXCHANGE);
    c->ev_used[ST_PAIRCONV] = false;  // the merged passes ran on the server's stream
    if (st) return st;
    c->applied = true;
    if (ex_out) CK(cudaMemcpyAsync(ex_out, c->exd.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "energy");
    CK(cudaStreamSynchronize(c->stream), "apply exchange");
    return LACE_OK;
}

FFTTables<float> ctx_tables_f(lace_ctx* c) { return tables<float>(c); }
int ctx_device(lace_ctx* c) { return c->device; }

lace_status ctx_load_dev64(lace_ctx* c, const double* d_phi, int n_occ, int n_extra, int ortho) {
    return load_common(c, d_phi, true, n_occ, n_extra, ortho);
}

lace_status ctx_orbitals(lace_ctx* c, int which, const void** src) {
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals first");
    switch (which) {
        case LACE_ORB_PSI: {
            lace_status st = materialize_psi(c);
            if (st) return st;
            *src = c->psi.p;
            return LACE_OK;
        }
        case LACE_ORB_W:
            if (!c->applied) return fail(c, LACE_ERR_STATE, "apply the exchange first");
            *src = c->W.p;
            return LACE_OK;
        case LACE_ORB_XI:
            if (!c->ace) return fail(c, LACE_ERR_STATE, "build ACE first");
            *src = c->xi.p;
            return LACE_OK;
        default: return fail(c, LACE_ERR_ARG, "unknown orbital set");
    }
}

// Device bytes a context holds after loading n_occ + n_extra orbitals on an
// n[0] x n[1] x n[2] grid, localising them (stride 2), screening, applying the
// exchange, building ACE and applying it to n_apply host functions: the
// buffers of the calls above at their largest (the tables excepted, which
// are far smaller than one orbital).
size_t predict_ctx_bytes(int prec, const int n[3], int n_occ, int n_extra, int n_apply, size_t fft_budget) {
    const size_t ng = (size_t)n[0] * n[1] * n[2], eb = prec == LACE_FP64 ? 8 : 4;
    const size_t n_p = (size_t)n_occ + n_extra, na = (size_t)std::max(n_apply, 0);
    const size_t ncol = (size_t)((n[0] + 1) / 2) * ((n[1] + 1) / 2) * ((n[2] + 1) / 2);
    const size_t maxp = (size_t)n_occ * (n_occ + 1) / 2 + (size_t)n_occ * n_extra;
    const size_t batch = (size_t)std::min<long long>(batch_for_sizes(ng, eb, fft_budget), std::max<long long>((maxp + 1) / 2, 1));
    size_t work = gemm_rows_work_elems((int)n_p, (int)n_p, ng) * sizeof(double);
    work = std::max(work, (size_t)n_occ * ncol * eb);
    if (prec != LACE_FP64) {
        work = std::max(work, tc_gram_work_elems((int)n_p, (int)n_p, ng) * sizeof(double));
        work = std::max(work, tc_gram_work_elems(n_occ, n_occ, ng, true) * sizeof(double));
        work = std::max(work, tc_combine_scratch_bytes((int)n_p, (int)n_p));
        if (na) {
            work = std::max(work, tc_gram_work_elems((int)n_p, (int)na, ng) * sizeof(double));
            work = std::max(work, tc_combine_scratch_bytes((int)na, (int)n_p));
        }
    }
    if (na) work = std::max(work, gemm_rows_work_elems((int)n_p, (int)na, ng) * sizeof(double));
    const size_t mslot = n_p * n_p + 64 * n_p + 64;
    size_t b = 0;
    b += 3 * n_p * ng * eb;        // psi, W, xi
    b += (size_t)n_occ * ng * eb;  // canonical orbitals
    b += n_p * ng * 8;             // FP64 staging
    b += mslot * kMatSlots * sizeof(double) + work + qrcp_aux_bytes(n_occ, (int)ncol);
    b += maxp * 8 + (maxp + 1) / 2 * sizeof(PairGrid);
    b += std::max(batch * ng * 2 * eb, 2 * na * ng * eb) + batch * n[0] * 2 * sizeof(double);
    b += 2 * na * ng * sizeof(double) + ng * (sizeof(float) + sizeof(double));
    return b;
}

}  // namespace lace

// ============================================================================ C ABI

extern "C" {

const char* lace_status_string(lace_status s) {
    switch (s) {
        case LACE_OK: return "ok";
        case LACE_ERR_ARG: return "invalid argument";
        case LACE_ERR_STATE: return "call made out of order";
        case LACE_ERR_OOM: return "out of device memory";
        case LACE_ERR_CUDA: return "CUDA error";
        case LACE_ERR_NOT_PD: return "matrix not positive definite";
        case LACE_ERR_TIMEOUT: return "iteration did not converge";
        case LACE_ERR_UNSUPPORTED: return "unsupported size or option";
    }
    return "unknown status";
}

const char* lace_last_error(lace_ctx* c) { return c ? c->err.c_str() : "null context"; }

lace_status lace_create(lace_ctx** out, int device, int precision) {
    if (!out) return LACE_ERR_ARG;
    *out = nullptr;
    if (precision != LACE_FP64 && precision != LACE_MIXED) return LACE_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LACE_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LACE_ERR_CUDA;
    lace_ctx* c = new lace_ctx();
    c->device = device;
    c->prec = precision;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return LACE_ERR_CUDA;
    }
    c->stream = c->own_stream;
    for (auto& e : c->ev) cudaEventCreate(&e);
    void* hf = nullptr;  // pinned timeout flags (without them every tensor-core call waits for its own)
    if (cudaHostAlloc(&hf, kFlagSlots * sizeof(int), cudaHostAllocDefault) == cudaSuccess) {
        c->hflags = static_cast<int*>(hf);
    } else {
        cudaGetLastError();
    }
    *out = c;
    return LACE_OK;
}

lace_status lace_destroy(lace_ctx* c) {
    if (!c) return LACE_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->psi, &c->canon, &c->W, &c->xi, &c->stage64, &c->scratch, &c->work, &c->aux, &c->mat,
                      &c->pairs, &c->counts, &c->grids, &c->epart, &c->flag, &c->piv, &c->pivfull, &c->exd,
                      &c->aceio, &c->ref, &c->pw_idx, &c->pw_io, &c->pw_real};
    for (DevBuf* b : bufs) b->release();
    for (int a = 0; a < 3; ++a) { c->tw_d[a].release(); c->tw_f[a].release(); c->g2_d[a].release(); c->g2_f[a].release(); }
    c->ktab_f.release();
    c->ktab_d.release();
    for (auto& e : c->ev) if (e) cudaEventDestroy(e);
    if (c->io_in) {
        cudaStreamSynchronize(c->io_in);
        cudaStreamSynchronize(c->io_out);
        cudaStreamDestroy(c->io_in);
        cudaStreamDestroy(c->io_out);
    }
    for (auto& e : c->io_ev) if (e) cudaEventDestroy(e);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
    return LACE_OK;
}

lace_status lace_set_stream(lace_ctx* c, void* stream) {
    if (!c) return LACE_ERR_ARG;
    c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    return LACE_OK;
}

lace_status lace_set_wait_limit(lace_ctx* c, double seconds) {
    if (!c) return LACE_ERR_ARG;
    if (!(seconds >= 0.0 && seconds <= 3600.0)) return fail(c, LACE_ERR_ARG, "wait limit must be in [0, 3600] s");
    c->wait_limit_ns = (unsigned long long)(seconds * 1e9);
    return LACE_OK;
}

lace_status lace_set_cell(lace_ctx* c, const double cell[3], int n1, int n2, int n3, double ecut_ha) {
    if (!c) return LACE_ERR_ARG;
    if (!cell || !(cell[0] > 0) || !(cell[1] > 0) || !(cell[2] > 0) || !(ecut_ha > 0))
        return fail(c, LACE_ERR_ARG, "cell lengths and cutoff must be positive");
    const int ns[3] = {n1, n2, n3};
    for (int a = 0; a < 3; ++a)
        if (!good_size(ns[a])) return fail(c, LACE_ERR_UNSUPPORTED, "grid sizes must be 2^a 3^b 5^c within [4, 128]");
    GridGeom g{};
    for (int a = 0; a < 3; ++a) {
        g.n[a] = ns[a];
        g.cell[a] = cell[a];
        if (!plan_axis(ns[a], &g.ax[a])) return fail(c, LACE_ERR_UNSUPPORTED, "no FFT plan for this size");
    }
    g.ng = (size_t)n1 * n2 * n3;
    g.omega = cell[0] * cell[1] * cell[2];
    g.dv = g.omega / (double)g.ng;
    cudaSetDevice(c->device);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    const size_t eb = elem_bytes(c);
    const size_t need = std::max(pairconv_smem_bytes(g, (int)eb, 0), pairconv_smem_bytes(g, (int)eb, 1));
    if (need > prop.sharedMemPerBlockOptin)
        return fail(c, LACE_ERR_UNSUPPORTED, "grid plane does not fit in shared memory at this precision");
    c->g = g;
    c->ecut = ecut_ha;
    c->have_cell = true;
    c->have_ref = false;
    c->loaded = c->localized = c->screened = c->applied = c->ace = false;
    return build_tables(c);
}

lace_status lace_set_kernel(lace_ctx* c, int kind, double omega, double alpha) {
    if (!c) return LACE_ERR_ARG;
    if (kind != LACE_KERNEL_COULOMB && kind != LACE_KERNEL_ERFC) return fail(c, LACE_ERR_ARG, "unknown kernel");
    if (kind == LACE_KERNEL_ERFC && !(omega > 0.0)) return fail(c, LACE_ERR_ARG, "omega must be > 0");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(c, LACE_ERR_ARG, "alpha must be > 0");
    c->kernel_kind = kind;
    c->kernel_omega = omega;
    c->kernel_alpha = alpha;
    c->applied = c->ace = false;
    if (!c->have_cell) return LACE_OK;
    cudaSetDevice(c->device);
    return build_tables(c);
}

lace_status lace_load_orbitals(lace_ctx* c, const double* phi, int n_occ, int n_extra, int orthonormalize) {
    return load_common(c, phi, false, n_occ, n_extra, orthonormalize);
}

lace_status lace_load_orbitals_dev(lace_ctx* c, const double* d_phi, int n_occ, int n_extra, int orthonormalize) {
    return load_common(c, d_phi, true, n_occ, n_extra, orthonormalize);
}

static lace_status localize_common(lace_ctx* c, int stride, const long long* imposed, long long* pivots_out) {
    if (!c) return LACE_ERR_ARG;
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals before localising");
    if (!imposed && (stride < 1 || stride > 8)) return fail(c, LACE_ERR_ARG, "stride must be in [1, 8]");
    cudaSetDevice(c->device);
    c->localized = c->screened = c->applied = false;
    ev_begin(c, ST_LOCALIZE);
    lace_status st = c->prec == LACE_FP64 ? localize_impl<double>(c, stride, imposed)
                                          : localize_impl<float>(c, stride, imposed);
    ev_end(c, ST_LOCALIZE);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "localize");
    if (pivots_out) std::copy(c->pivots_host.begin(), c->pivots_host.end(), pivots_out);
    c->localized = true;
    return LACE_OK;
}

lace_status lace_localize(lace_ctx* c, int stride, long long* pivots_out) {
    return localize_common(c, stride, nullptr, pivots_out);
}

lace_status lace_set_pivots(lace_ctx* c, const long long* pivots, int n) {
    if (!c) return LACE_ERR_ARG;
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals before localising");
    if (!pivots || n != c->n_occ) return fail(c, LACE_ERR_ARG, "need exactly n_occ pivots");
    std::vector<long long> v(pivots, pivots + n);
    for (long long p : v)
        if (p < 0 || (size_t)p >= c->g.ng) return fail(c, LACE_ERR_ARG, "pivot outside the grid");
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end()) return fail(c, LACE_ERR_ARG, "pivots must be distinct");
    return localize_common(c, 0, pivots, nullptr);
}

lace_status lace_align_to_previous(lace_ctx* c, int* aligned_out) {
    if (!c) return LACE_ERR_ARG;
    if (!c->localized) return fail(c, LACE_ERR_STATE, "localise before aligning");
    cudaSetDevice(c->device);
    const size_t bytes = (size_t)c->n_occ * c->g.ng * elem_bytes(c);
    if (aligned_out) *aligned_out = 0;
    if (c->have_ref && c->ref_n == c->n_occ && c->ref.bytes >= bytes) {
        c->screened = c->applied = false;
        lace_status st = c->prec == LACE_FP64 ? align_impl<double>(c) : align_impl<float>(c);
        if (st) return st;
        if (aligned_out) *aligned_out = 1;
    }
    CK(c->ref.ensure(bytes), "alloc alignment reference");
    CK(cudaMemcpyAsync(c->ref.p, c->psi.p, bytes, cudaMemcpyDeviceToDevice, c->stream), "alignment");
    CK(cudaStreamSynchronize(c->stream), "alignment");
    c->have_ref = true;
    c->ref_n = c->n_occ;
    return LACE_OK;
}

lace_status lace_screen(lace_ctx* c, double s_thr, long long* n_pairs_out) {
    if (!c) return LACE_ERR_ARG;
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals before screening");
    if (!(s_thr >= 0.0)) return fail(c, LACE_ERR_ARG, "threshold must be >= 0");
    cudaSetDevice(c->device);
    c->screened = c->applied = false;
    {
        lace_status st = materialize_psi(c);
        if (st) return st;
    }
    ev_begin(c, ST_SCREEN);
    c->tc_next = 2;
    lace_status st = c->prec == LACE_FP64 ? screen_impl<double>(c, s_thr) : screen_impl<float>(c, s_thr);
    if (st) return st;
    Launch L{c};
    st = make_pairs(c, true, s_thr, L);  // reads the pair count back (stream synchronised)
    ev_end(c, ST_SCREEN);
    if (c->hflags && tc_timed_out(c))
        return fail(c, LACE_ERR_TIMEOUT, "overlap of moduli: an mbarrier wait timed out");
    if (st) return st;
    c->screened = true;
    c->s_thr = s_thr;
    if (n_pairs_out) *n_pairs_out = c->n_pairs;
    return LACE_OK;
}

lace_status lace_apply_exchange(lace_ctx* c, double* W_out, double* ex_out) {
    if (!c) return LACE_ERR_ARG;
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals before applying the exchange");
    cudaSetDevice(c->device);
    c->applied = false;
    {
        lace_status st = materialize_psi(c);
        if (st) return st;
    }
    ev_begin(c, ST_EXCHANGE);
    lace_status st = c->prec == LACE_FP64 ? apply_impl<double>(c) : apply_impl<float>(c);
    ev_end(c, ST_EXCHANGE);
    if (st) return st;
    c->applied = true;
    if (ex_out) {
        CK(cudaMemcpyAsync(ex_out, c->exd.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "energy");
    }
    if (W_out) {
        st = c->prec == LACE_FP64 ? copy_orbitals_out<double>(c, c->W.as<double>(), (size_t)c->n_p * c->g.ng, W_out)
                                  : copy_orbitals_out<float>(c, c->W.as<float>(), (size_t)c->n_p * c->g.ng, W_out);
        if (st) return st;
    }
    CK(cudaStreamSynchronize(c->stream), "apply exchange");
    return LACE_OK;
}

lace_status lace_exchange_energy(lace_ctx* c, double f_spin, double* ex_out) {
    if (!c || !ex_out) return LACE_ERR_ARG;
    if (!c->applied) return fail(c, LACE_ERR_STATE, "apply the exchange first");
    double ex = 0.0;
    CK(cudaMemcpyAsync(&ex, c->exd.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "energy");
    CK(cudaStreamSynchronize(c->stream), "energy");
    *ex_out = f_spin * ex;
    return LACE_OK;
}

lace_status lace_build_ace(lace_ctx* c, int sym) {
    if (!c) return LACE_ERR_ARG;
    if (!c->applied) return fail(c, LACE_ERR_STATE, "apply the exchange before building ACE");
    if (sym < 0 || sym > 2) return fail(c, LACE_ERR_ARG, "bad symmetrisation");
    cudaSetDevice(c->device);
    ev_begin(c, ST_ACE_BUILD);
    c->tc_next = 2;
    lace_status st = c->prec == LACE_FP64 ? build_ace_impl<double>(c, sym) : build_ace_impl<float>(c, sym);
    ev_end(c, ST_ACE_BUILD);
    if (st) {
        // a failed Cholesky stops the build before xi and L are written: the
        // previous projector stays; any other failure may have left xi half written
        if (st != LACE_ERR_NOT_PD) c->ace = false;
        return st;
    }
    CK(cudaStreamSynchronize(c->stream), "build ace");
    if (c->hflags && tc_timed_out(c)) {
        c->ace = false;
        return fail(c, LACE_ERR_TIMEOUT, "tensor-core combination: an mbarrier wait timed out");
    }
    c->ace = true;
    return LACE_OK;
}

__global__ void sum_chunks_kernel(int n, const double* __restrict__ in, double* __restrict__ out) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += in[i];  // fixed order
    *out = s;
}

// Mixed-precision ACE apply of host arrays in chunks of functions: chunk k's
// upload (io_in), its application (the context's stream) and chunk k - 1's
// download (io_out) overlap, so the two directions of the host link and the
// GPU work at once instead of one after the other.
static lace_status apply_ace_pipelined(lace_ctx* c, const double* psi, int n, double* out) {
    const size_t ng = c->g.ng, cnt = (size_t)n * ng;
    CK(c->aceio.ensure(2 * cnt * sizeof(double)), "alloc ace io");
    if (!c->io_in) {
        CK(cudaStreamCreateWithFlags(&c->io_in, cudaStreamNonBlocking), "streams");
        CK(cudaStreamCreateWithFlags(&c->io_out, cudaStreamNonBlocking), "streams");
        for (auto& e : c->io_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "events");
    }
    double* din = c->aceio.as<double>();
    double* dout = din + cnt;
    c->tc_next = 2;
    const int nch = std::min(kApplyChunks, n);
    const int per = (n + nch - 1) / nch;
    // uploads after whatever the context's stream holds
    CK(cudaEventRecord(c->io_ev[0], c->stream), "events");
    CK(cudaStreamWaitEvent(c->io_in, c->io_ev[0], 0), "events");
    for (int k = 0; k < nch; ++k) {
        const size_t off = (size_t)k * per * ng, m = (size_t)std::max(0, std::min(per, n - k * per));
        if (m) CK(cudaMemcpyAsync(din + off, psi + off, m * ng * sizeof(double), cudaMemcpyHostToDevice, c->io_in),
                  "upload");
        CK(cudaEventRecord(c->io_ev[1 + k], c->io_in), "events");
    }
    ev_begin(c, ST_ACE_APPLY);
    lace_status st = LACE_OK;
    for (int k = 0; k < nch && !st; ++k) {
        const int m = std::max(0, std::min(per, n - k * per));
        const size_t off = (size_t)k * per * ng;
        CK(cudaStreamWaitEvent(c->stream, c->io_ev[1 + k], 0), "events");
        if (m) st = apply_ace_impl<float>(c, din + off, m, dout + off, k);
        else CK(cudaMemsetAsync(c->exd.as<double>() + 2 + k, 0, sizeof(double), c->stream), "energy");
        if (st) break;
        CK(cudaEventRecord(c->io_ev[1 + kApplyChunks + k], c->stream), "events");
        CK(cudaStreamWaitEvent(c->io_out, c->io_ev[1 + kApplyChunks + k], 0), "events");
        if (m) CK(cudaMemcpyAsync(out + off, dout + off, (size_t)m * ng * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->io_out),
                  "download");
    }
    if (!st) {
        sum_chunks_kernel<<<1, 1, 0, c->stream>>>(nch, c->exd.as<double>() + 2, c->exd.as<double>() + 1);
        c->launches += 1;
    }
    ev_end(c, ST_ACE_APPLY);
    cudaError_t e1 = cudaStreamSynchronize(c->io_out), e2 = cudaStreamSynchronize(c->stream),
                e3 = cudaStreamSynchronize(c->io_in);
    const bool timed_out = c->hflags && tc_timed_out(c);
    if (st) return st;
    if (e1 || e2 || e3) return cuda_fail(c, e1 ? e1 : e2 ? e2 : e3, "apply ace");
    CK(cudaGetLastError(), "apply ace");
    if (timed_out) return fail(c, LACE_ERR_TIMEOUT, "ACE apply: a tensor-core mbarrier wait timed out");
    c->ace_applied = true;
    return LACE_OK;
}

static lace_status apply_ace_common(lace_ctx* c, const double* psi, int n, double* out, bool dev) {
    if (!c) return LACE_ERR_ARG;
    if (!c->ace) return fail(c, LACE_ERR_STATE, "build ACE before applying it");
    if (!psi || !out || n < 1) return fail(c, LACE_ERR_ARG, "bad pointers or count");
    cudaSetDevice(c->device);
    if (!dev && c->prec != LACE_FP64 && (size_t)n * c->n_p <= c->mslot) return apply_ace_pipelined(c, psi, n, out);
    c->tc_next = 2;
    const size_t cnt = (size_t)n * c->g.ng;
    const double* din = psi;
    double* dout = out;
    if (!dev) {
        CK(c->aceio.ensure(2 * cnt * sizeof(double)), "alloc ace io");
        CK(cudaMemcpyAsync(c->aceio.p, psi, cnt * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload");
        din = c->aceio.as<double>();
        dout = c->aceio.as<double>() + cnt;
    }
    ev_begin(c, ST_ACE_APPLY);
    lace_status st = c->prec == LACE_FP64 ? apply_ace_impl<double>(c, din, n, dout)
                                          : apply_ace_impl<float>(c, din, n, dout);
    ev_end(c, ST_ACE_APPLY);
    if (st == LACE_OK && !dev) {
        cudaError_t e = cudaMemcpyAsync(out, dout, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e) st = cuda_fail(c, e, "download");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    const bool timed_out = c->hflags && tc_timed_out(c);
    if (st) return st;
    if (e) return cuda_fail(c, e, "apply ace");
    if (timed_out) return fail(c, LACE_ERR_TIMEOUT, "ACE apply: a tensor-core mbarrier wait timed out");
    c->ace_applied = true;
    return LACE_OK;
}

lace_status lace_apply_ace(lace_ctx* c, const double* psi, int n, double* kpsi_out) {
    return apply_ace_common(c, psi, n, kpsi_out, false);
}

lace_status lace_apply_ace_dev(lace_ctx* c, const double* d_psi, int n, double* d_kpsi_out) {
    return apply_ace_common(c, d_psi, n, d_kpsi_out, true);
}

lace_status lace_get_matrix(lace_ctx* c, int which, double* out, long long count) {
    if (!c || !out) return LACE_ERR_ARG;
    const double* src = nullptr;
    long long need = 0;
    switch (which) {
        case LACE_MAT_OVERLAP_MODULI:
            if (!c->screened || !c->loaded) return fail(c, LACE_ERR_STATE, "screen first");
            src = c->m(MS_S);
            need = (long long)c->n_occ * c->n_occ;
            break;
        case LACE_MAT_EXCHANGE:
            if (!c->ace) return fail(c, LACE_ERR_STATE, "build ACE first");
            src = c->m(MS_M);
            need = (long long)c->n_p * c->n_p;
            break;
        case LACE_MAT_CHOLESKY:
            if (!c->ace) return fail(c, LACE_ERR_STATE, "build ACE first");
            src = c->m(MS_L);
            need = (long long)c->n_p * c->n_p;
            break;
        case LACE_MAT_PAIR_ENERGY:
            if (!c->applied) return fail(c, LACE_ERR_STATE, "apply the exchange first");
            src = c->m(MS_E);
            need = (long long)c->n_occ * c->n_occ;
            break;
        case LACE_MAT_SCDM_U:
            if (!c->localized) return fail(c, LACE_ERR_STATE, "localise first");
            src = c->m(MS_U);
            need = (long long)c->n_occ * c->n_occ;
            break;
        default: return fail(c, LACE_ERR_ARG, "unknown matrix");
    }
    if (count < need) return fail(c, LACE_ERR_ARG, "output buffer too small");
    CK(cudaMemcpyAsync(out, src, sizeof(double) * need, cudaMemcpyDeviceToHost, c->stream), "get matrix");
    CK(cudaStreamSynchronize(c->stream), "get matrix");
    return LACE_OK;
}

lace_status lace_get_orbitals(lace_ctx* c, int which, double* out, long long count) {
    if (!c || !out) return LACE_ERR_ARG;
    if (!c->loaded) return fail(c, LACE_ERR_STATE, "load orbitals first");
    const long long need = (long long)c->n_p * (long long)c->g.ng;
    if (count < need) return fail(c, LACE_ERR_ARG, "output buffer too small");
    const void* src = nullptr;
    switch (which) {
        case LACE_ORB_PSI: {
            cudaSetDevice(c->device);
            lace_status st = materialize_psi(c);
            if (st) return st;
            src = c->psi.p;
            break;
        }
        case LACE_ORB_W:
            if (!c->applied) return fail(c, LACE_ERR_STATE, "apply the exchange first");
            src = c->W.p;
            break;
        case LACE_ORB_XI:
            if (!c->ace) return fail(c, LACE_ERR_STATE, "build ACE first");
            src = c->xi.p;
            break;
        default: return fail(c, LACE_ERR_ARG, "unknown orbital set");
    }
    cudaSetDevice(c->device);
    return c->prec == LACE_FP64 ? copy_orbitals_out<double>(c, static_cast<const double*>(src), need, out)
                                : copy_orbitals_out<float>(c, static_cast<const float*>(src), need, out);
}

lace_status lace_get_pairs(lace_ctx* c, int* pairs_out, long long cap, long long* n_out) {
    if (!c || !n_out) return LACE_ERR_ARG;
    if (!c->screened) return fail(c, LACE_ERR_STATE, "screen (or apply the exchange) first");
    *n_out = c->n_pairs;
    if (pairs_out && cap > 0) {
        const long long k = std::min(cap, c->n_pairs);
        CK(cudaMemcpyAsync(pairs_out, c->pairs.p, sizeof(int2) * k, cudaMemcpyDeviceToHost, c->stream), "get pairs");
        CK(cudaStreamSynchronize(c->stream), "get pairs");
    }
    return LACE_OK;
}

lace_status lace_get_ace_energy(lace_ctx* c, double* e_out) {
    if (!c || !e_out) return LACE_ERR_ARG;
    if (!c->ace_applied) return fail(c, LACE_ERR_STATE, "apply ACE first");
    CK(cudaMemcpyAsync(e_out, c->exd.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "energy");
    CK(cudaStreamSynchronize(c->stream), "energy");
    return LACE_OK;
}

lace_status lace_get_pivots(lace_ctx* c, long long* pivots_out, int n) {
    if (!c || !pivots_out) return LACE_ERR_ARG;
    if (!c->localized) return fail(c, LACE_ERR_STATE, "localise first");
    if (n < c->n_occ) return fail(c, LACE_ERR_ARG, "output buffer too small");
    std::copy(c->pivots_host.begin(), c->pivots_host.end(), pivots_out);
    return LACE_OK;
}

lace_status lace_get_timings(lace_ctx* c, double* ms_out, int count) {
    if (!c || !ms_out) return LACE_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream), "timings");
    for (int i = 0; i < count && i < ST_COUNT; ++i) {
        float ms = 0.f;
        if (c->ev_used[i] && cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess)
            ms_out[i] = ms;
        else {
            cudaGetLastError();
            ms_out[i] = 0.0;
        }
    }
    return LACE_OK;
}

lace_status lace_get_device_bytes(lace_ctx* c, unsigned long long* bytes_out) {
    if (!c || !bytes_out) return LACE_ERR_ARG;
    const DevBuf* bufs[] = {&c->psi,   &c->canon, &c->W,      &c->xi,    &c->stage64, &c->scratch, &c->work,
                            &c->aux,   &c->mat,   &c->pairs,  &c->counts, &c->grids,  &c->epart,   &c->flag,
                            &c->piv,   &c->pivfull, &c->exd,  &c->aceio, &c->ktab_f, &c->ktab_d, &c->ref,
                            &c->pw_idx, &c->pw_io,  &c->pw_real};
    unsigned long long b = 0;
    for (const DevBuf* d : bufs) b += d->bytes;
    for (int a = 0; a < 3; ++a) b += c->tw_d[a].bytes + c->tw_f[a].bytes + c->g2_d[a].bytes + c->g2_f[a].bytes;
    *bytes_out = b;
    return LACE_OK;
}

lace_status lace_get_launch_count(lace_ctx* c, long long* count_out) {
    if (!c || !count_out) return LACE_ERR_ARG;
    *count_out = c->launches;
    return LACE_OK;
}

}  // extern "C"
