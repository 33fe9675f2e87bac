// The library context (private to liblace's translation units): device
// buffers, grid geometry, state flags and the stage events of one lace_ctx.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lace.h"
#include "lace_internal.cuh"

namespace lace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t b) {
        if (b <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (b == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

enum Stage { ST_LOAD = 0, ST_LOCALIZE, ST_SCREEN, ST_EXCHANGE, ST_ACE_BUILD, ST_ACE_APPLY, ST_PAIRCONV, ST_COUNT };

// Small-matrix slots inside lace_ctx::mat (each mslot doubles).
enum MatSlot { MS_S = 0, MS_M, MS_MSYM, MS_L, MS_LINV, MS_LINVT, MS_E, MS_U, MS_A, MS_B, MS_X, MS_NSWORK, MS_COUNT_BASE };
// MS_NSWORK takes 5 slots (Newton-Schulz work)
constexpr int kMatSlots = MS_NSWORK + 5 + 1;
// chunks of a host ACE apply (the chunk energies sit in exd[2 .. 2 + kApplyChunks))
constexpr int kApplyChunks = 4;
// int slots of a context's device flag buffer (64 bytes)
constexpr int kFlagSlots = 16;

}  // namespace lace

using lace::DevBuf;
using lace::GridGeom;

struct lace_ctx {
    int device = 0;
    int prec = LACE_FP64;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    std::string err;
    long long launches = 0;
    size_t fft_scratch_budget = lace::kFftScratchBudget;  // bytes of complex grids per batch of the FFT passes
    unsigned long long wait_limit_ns = 2000000000ull;     // bound of one grid-barrier wait (lace_set_wait_limit)

    bool have_cell = false;
    GridGeom g{};
    DevBuf tw_d[3], tw_f[3], g2_d[3], g2_f[3];
    DevBuf ktab_f;  // K(G)/Ng rounded once from FP64 (FP32 path)
    DevBuf ktab_d;  // K(G)/Ng (FP64 path)
    int kernel_kind = LACE_KERNEL_COULOMB;
    double kernel_omega = 0.0, kernel_alpha = 1.0;

    int n_occ = 0, n_extra = 0, n_p = 0;
    bool loaded = false, localized = false, screened = false, applied = false, ace = false;
    bool ace_applied = false;    // exd[1] holds the block ACE energy of the last ACE application
    bool x_identity = false;     // X = I (loaded without orthonormalisation)
    bool psi_occ_ready = false;  // psi[0 .. n_occ) holds canon X (or its SCDM rotation)
    double s_thr = 0.0;

    DevBuf psi;     // [n_p][ng] working precision: [w (localised occupied) ; extras]
    DevBuf canon;   // [n_occ][ng] the raw occupied orbitals; the canonical (Loewdin) ones are canon X, X in MS_X
    DevBuf W;       // [n_p][ng]
    DevBuf xi;      // [n_p][ng]
    DevBuf stage64; // [rows][ng] FP64 staging (uploads, conversions)
    DevBuf scratch; // complex FFT grids of one batch
    DevBuf work;    // GEMM partials and the QRCP matrix
    DevBuf aux;     // QRCP auxiliary
    DevBuf mat;     // small FP64 matrices (see offsets below)
    DevBuf pairs, counts, grids, epart, flag, piv, pivfull, exd;
    DevBuf aceio;   // FP64 device copies of a host ACE apply's input and output
    DevBuf ref;     // [n_occ][ng] localised orbitals of the previous alignment
    DevBuf pw_idx, pw_io, pw_real;  // plane-wave front end: G offsets, coefficients, FP64 orbitals
    double ecut = 0.0;              // orbital cutoff of lace_set_cell (Ha)
    bool have_ref = false;
    int ref_n = 0;
    long long n_pairs = 0;
    std::vector<long long> pivots_host;

    cudaEvent_t ev[2 * lace::ST_COUNT] = {};
    bool ev_used[lace::ST_COUNT] = {};
    // a host ACE apply's chunks: uploads on io_in, downloads on io_out (both
    // directions of the host link at once), made on first use
    cudaStream_t io_in = nullptr, io_out = nullptr;
    cudaEvent_t io_ev[1 + 2 * lace::kApplyChunks] = {};
    // timeout flags of the tensor-core calls of one API call: device slots
    // flag[2 .. tc_next), copied after each call into pinned hflags and read
    // at the API call's next synchronisation instead of one wait per call
    int* hflags = nullptr;  // pinned, kFlagSlots ints
    int tc_next = 2;

    // small-matrix slots inside `mat` (each n_p*n_p doubles, plus staging)
    size_t mslot = 0;
    double* m(int k) { return mat.as<double>() + (size_t)k * mslot; }
};

namespace lace {
// Shared with the other translation units (defined in lace_api.cu).
lace_status ctx_fail(lace_ctx* c, lace_status st, const std::string& msg);
// lace_load_orbitals from FP64 device memory (borrowed for the call)
lace_status ctx_load_dev64(lace_ctx* c, const double* d_phi, int n_occ, int n_extra, int ortho);
// device pointer of PSI / W / XI (working precision, [n_p][ng]) after the state checks
lace_status ctx_orbitals(lace_ctx* c, int which, const void** src);
// Merged pair convolutions of the request server: whether the context can
// take part (mixed precision, a cubic grid with merged passes); the exchange
// application before the pair convolutions (fills *m, the grid count and the
// grids its scratch holds; records `ready` on the context's stream) and after
// them (the context's stream waits for `done`; E_x into *ex_out, synchronous).
bool ctx_mergeable(lace_ctx* c);
lace_status ctx_exchange_prepare(lace_ctx* c, MergedSys<float>* m, int* n_grids, int* cap, cudaEvent_t ready);
lace_status ctx_exchange_finish(lace_ctx* c, cudaEvent_t done, double* ex_out);
FFTTables<float> ctx_tables_f(lace_ctx* c);
int ctx_device(lace_ctx* c);
}  // namespace lace
