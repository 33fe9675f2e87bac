// Internal interfaces between the translation units of liblace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace lace {

constexpr int kMaxN = 128;  // largest grid size per axis (FP32); FP64 is limited by shared memory

struct GridGeom {
    int n[3];
    double cell[3];
    size_t ng;
    double omega, dv;
    AxisPlan ax[3];
};

// Device tables of one grid, per precision.
template <typename T> struct FFTTables {
    cplx<T>* tw[3] = {nullptr, nullptr, nullptr};  // exp(-2 pi i m / n_a), m < n_a
    T* g2[3] = {nullptr, nullptr, nullptr};         // (2 pi m / L_a)^2 in FFT order
    T* ktab = nullptr;                              // optional K(G)/Ng table [n1][n2][n3]
};

// One complex FFT grid carries two real pair densities: slot a = (i1, j1),
// slot b = (i2, j2); j2 < 0 marks an empty slot.  i is an occupied orbital
// (row of Psi < n_occ), j any row of Psi.
struct PairGrid {
    int i1, j1, i2, j2;
};

// Merged launches (the request server): the complex grids of several
// systems on one grid size run through one launch of each pass.  Per grid of
// the launch, its system and its index in that system's grid list; per
// system, its buffers, with g0 = the first of its grids in this launch (its
// scratch and energy partials hold grids g0, g0 + 1, ...).
struct GridRef {
    int sys, g;
};
template <typename T> struct MergedSys {
    const T* psi;
    T* W;
    const T* ktab;
    const PairGrid* grids;
    cplx<T>* scratch;
    double* epart;
    double* E;  // pair-energy matrix [n_occ][n_occ]
    int n_occ, g0;
    double dv;
};

// Kernel arguments of the three FFT passes.
template <typename T> struct ConvArgs {
    AxisPlan ax[3];
    const cplx<T>* tw[3];
    const T* g2[3];
    T kscale;         // 4 pi / Ng
    const T* ktab;    // K(G)/Ng per grid point, rounded once from FP64 (null: computed in T)
    const T* psi;
    int n_occ;
    T* W;
    const PairGrid* grids;
    cplx<T>* scratch;
    double* epart;  // [batch][n1][2]
    size_t ng;
    double dv;
    int pf_ahead = 0;  // L2 prefetch distance in CTAs of the out-of-place passes (0: none)
    // merged launches (null otherwise): grid g of the launch is refs[g0 + g]
    // of system msys[refs[.].sys]; psi, W, ktab, grids, scratch, epart,
    // n_occ and dv above are then unused
    const GridRef* refs = nullptr;
    const MergedSys<T>* msys = nullptr;
};

// Size-specialised FP32 passes for cubic grids (pairconv_spec_*.cu): launch
// pass 0/1/2 (A/B/C) for grid size n if a specialisation exists.
bool spec_launch_s(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s);
bool spec_launch_m(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s);
bool spec_launch_l(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s);
bool spec_launch_x(int pass, int n, int nb, const ConvArgs<float>& P, int g0, cudaStream_t s);

// Grid sizes whose size-specialised passes take merged launches (one grid
// per CTA, out of place) (pairconv_spec_*.cu).
bool spec_merge_ok(int n);

// The pair convolutions of several systems on one cubic grid size (n in
// spec_merge_ok), merged: per round, the next chunk of every system's grids
// (at most cap[q] of system q, the grids its scratch holds) goes through one
// launch of each pass, then the pair energies of every grid of the round are
// collected into its system's E.  tb: the twiddle tables of the size;
// d_refs / d_sys: device space for n_grids_total GridRefs and rounds x nsys
// MergedSys (the host side uploads them); every launch runs on stream s.
cudaError_t pairconv_run_merged(int n, const FFTTables<float>& tb, const std::vector<MergedSys<float>>& sys,
                                const std::vector<int>& n_grids, const std::vector<int>& cap, GridRef* d_refs,
                                MergedSys<float>* d_sys, cudaStream_t s, int* launches, int* rounds_out);

// Persistent multi-instance pair convolutions (pairconv_multi.cu): the kept
// pairs of many independent systems in one cooperative launch.
struct MultiInst {
    ConvArgs<float> P;  // per-instance arguments (P.scratch, P.epart unused)
    double* E;          // pair-energy matrix [n_occ][n_occ]
    int n1, n2;         // planes of passes A/C, slabs of pass B
    int spec;           // cubic size with size-specialised pass bodies (multi_spec_size), else 0
};
struct MultiArgs {
    const MultiInst* inst;  // device array [n_inst]
    int n_inst;
    const int* n_grids;     // device: complex grids per instance, read at run time
    cplx<float>* pool;      // complex scratch of pool_elems elements (>= the largest grid)
    size_t pool_elems;
    double* epart;          // plane energies, epart_elems doubles (>= 2 n1 of any instance)
    size_t epart_elems;
    unsigned* bar;          // 4 unsigned: barrier counters and the timeout flag bar[2]
    size_t smem_cta;        // dynamic shared memory of a CTA (set by pairconv_multi_run)
};
size_t pairconv_multi_smem(int n1, int n2, int n3);
// Cubic sizes whose size-specialised pass bodies the persistent kernel runs
// (with 256 or 512 threads a CTA): n, else 0; their shared memory.
int multi_spec_size(int n1, int n2, int n3);
size_t multi_spec_smem(int n);
const void* multi_kernel_256();    // pairconv_multi_256.cu (two CTAs an SM)
const void* multi_kernel_512();    // pairconv_multi_512.cu (one CTA an SM)
const void* multi_kernel_512x2();  // pairconv_multi_512x2.cu (two CTAs an SM, 64 registers)
// Dynamic shared memory for ctas_per_sm CTAs of `threads` an SM: all that
// the SM shares out to each (at least need), or 0 when that launch shape
// does not fit.
size_t pairconv_multi_cta_smem(int threads, int ctas_per_sm, size_t need);
// n_chunks cooperative launches (chunk c in launch c; see pairconv_multi_chunks).
cudaError_t pairconv_multi_run(const MultiArgs& A, int n_chunks, size_t smem, int threads, int ctas_per_sm,
                               cudaStream_t s, int* launches);
// Host copy of the kernel's chunking: chunks needed for these grid counts.
int pairconv_multi_chunks(const std::vector<int>& n_grids, const std::vector<size_t>& ng, const std::vector<int>& n1,
                          size_t pool_elems, size_t epart_elems);

// Host planning helpers (pairconv.cu)
bool plan_axis(int n, AxisPlan* out);
size_t pairconv_smem_bytes(const GridGeom& g, int elem_bytes, int pass);

// batch: complex grids the scratch (and epart) hold; the grids are processed
// in chunks of at most that many.
template <typename T>
cudaError_t pairconv_run(const GridGeom& g, const FFTTables<T>& tb, const T* psi, int n_occ, T* W,
                         const PairGrid* d_grids, int n_grids, cplx<T>* scratch, int batch, double* epart,
                         double* d_pair_e, cudaStream_t s, int* launches, cudaEvent_t ev0, cudaEvent_t ev1);

// Dense linear algebra (linalg.cu).  Matrices are row-major.
// C[m][n] = alpha * sum_r op(A[m][r]) op(B[n][r]) over r < K (A, B rows of
// length K with leading dimension ld*), op = |.| when absval.  Accumulates
// per K-chunk in T, reduces the chunks in FP64 (deterministic).
template <typename T>
cudaError_t gemm_rows(int M, int N, size_t K, const T* A, size_t lda, const T* B, size_t ldb, double alpha,
                      bool absval, double* C, int ldc, double* work, size_t work_elems, cudaStream_t s, int* launches);
size_t gemm_rows_work_elems(int M, int N, size_t K);

// Out[n][r] = beta*Out[n][r] + sum_k Coef[k][n] * A[k][r]  (r < K, n < N, k < Kc)
// Coef is FP64 [Kc][ldcoef] on the device.
template <typename T>
cudaError_t gemm_combine(int N, size_t K, int Kc, const T* A, size_t lda, const double* Coef, int ldcoef, double beta,
                         T* Out, size_t ldo, cudaStream_t s, int* launches);

// Tensor-core (tcgen05) 3xBF16 contraction C = alpha * sum_r op(A[m][r]) op(B[n][r])
// (FP32 operands, rows 16-byte aligned; op = |.| if absval); sym: A = B and
// only the tiles on and above the diagonal are computed.  h_err (nullable)
// receives 1 if a bounded mbarrier wait gave up (the call then synchronises s).
cudaError_t tc_gram(int M, int N, size_t K, const float* A, size_t lda, const float* B, size_t ldb, double alpha,
                    double* C, int ldc, double* work, size_t work_elems, int* d_err, int* h_err, cudaStream_t s,
                    int* launches, bool absval = false, bool sym = false);
size_t tc_gram_work_elems(int M, int N, size_t K, bool sym = false);
// Tensor-core combination Out[n][r] = beta Out + sum_k Coef[k][n] A[k][r]
// (FP32 A, FP64 Coef, split 3xBF16, FP32 accumulation; Out FP32 or FP64);
// scratch of tc_combine_scratch_bytes.
template <typename TO>
cudaError_t tc_combine(int N, size_t K, int Kc, const float* A, size_t lda, const double* Coef, int ldcoef,
                       double beta, TO* Out, size_t ldo, void* scratch, int* d_err, int* h_err, cudaStream_t s,
                       int* launches);
size_t tc_combine_scratch_bytes(int N, int Kc);

// Small FP64 dense kernels (N x N).
cudaError_t small_gemm_f64(int M, int N, int K, const double* A, int lda, bool ta, const double* B, int ldb, bool tb,
                           double alpha, double beta, double* C, int ldc, cudaStream_t s, int* launches);
// X = A^{-1/2} of a symmetric positive definite A by the coupled Newton-Schulz
// iteration; returns cudaSuccess and *ok=0 if it does not converge.
cudaError_t inv_sqrt_spd(int N, const double* A, double* X, double* work, int* d_flag, int* ok, cudaStream_t s,
                         int* launches);
size_t inv_sqrt_work_elems(int N);
// Mixed-precision variant: FP32 Newton-Schulz to ~1e-7, returns X0 ~ A^{-1/2}
// (FP64, symmetric).  Pair it with lowdin_refine.
cudaError_t inv_sqrt_spd_mixed(int N, const double* A, double* X, double* work, int* ok, cudaStream_t s,
                               int* launches);
size_t inv_sqrt_mixed_work_elems(int N);
// F <- F (I - E/2), E = F^T G F - I (G = I when null): orthonormality to O(E^2).
cudaError_t lowdin_refine(int N, double* F, const double* G, double* work, cudaStream_t s, int* launches);
// In-place lower Cholesky of A (N x N, lda); *ok = 0 when not positive definite.
// With ok == nullptr nothing is read back (stream-capturable): d_flag != 0
// then marks failure.
cudaError_t cholesky_lower(int N, double* A, int lda, int* d_flag, int* ok, cudaStream_t s, int* launches);
// Linv = L^{-1} for lower triangular L.
cudaError_t trtri_lower(int N, const double* L, int ldl, double* Linv, int ldi, cudaStream_t s, int* launches);
// B = A^T (N x N)
cudaError_t transpose_f64(int N, const double* A, double* B, cudaStream_t s, int* launches);
// B = sym(A): 0 avg, 1 upper->lower, 2 lower->upper; also negates when neg.
cudaError_t symmetrize(int N, const double* A, double* B, int mode, bool neg, cudaStream_t s, int* launches);

// SCDM pivoted QR (scdm.cu): selects npiv columns of R (nrow x ncol,
// row-major, overwritten).  Pivots are column indices, ties to the lowest
// index.  aux: caller scratch of qrcp_aux_bytes(nrow, ncol) bytes.
// *h_timeout = 1 when a grid-barrier wait of the persistent kernel ran out of
// time (the pivots are then invalid); wait_limit_ns bounds each such wait.
// The persistent path waits for s.
template <typename T>
cudaError_t qrcp_pivots(int nrow, int ncol, T* R, int npiv, int* d_piv, void* aux, int* h_timeout,
                        unsigned long long wait_limit_ns, cudaStream_t s, int* launches);
size_t qrcp_aux_bytes(int nrow, int ncol);

// Subsample gather: out[o][c] = psi[o][full index of subsample point c]
template <typename T>
cudaError_t gather_subsample(const GridGeom& g, int stride, const T* psi, int norb, T* out, int* ncol_out,
                             cudaStream_t s, int* launches);
// Gather phi_C[point p][orbital o] = psi[o][pivot_full[p]] into FP64 (N x N).
template <typename T>
cudaError_t gather_columns(const T* psi, size_t ldpsi, int norb, const long long* d_full_idx, int npts, double* out,
                           cudaStream_t s, int* launches);

// Screening (screen.cu): keep mask from S and the pair list.
// Writes the kept (i, j) pairs, i <= j < n_occ with S_ij >= thr, row by row,
// followed by all (i, n_occ + e).  Returns the count in *n_pairs (host).
cudaError_t build_pair_list(int n_occ, int n_extra, const double* d_S, double thr, bool use_S, int2* d_pairs,
                            int* d_counts, long long* n_pairs, cudaStream_t s, int* launches);
// Pack pairs two by two into complex FFT grids.
cudaError_t pack_pair_grids(const int2* d_pairs, long long n_pairs, PairGrid* d_grids, cudaStream_t s, int* launches);
// Fixed-order FP64 sums over up to kSumBlocks blocks; part: kSumBlocks
// doubles of scratch (one caller at a time per scratch).
constexpr int kSumBlocks = 128;
// out[0] = -sum of the squares of the m entries of X (fixed order).
cudaError_t neg_sum_squares(size_t m, const double* d_X, double* d_part, double* d_out, cudaStream_t s,
                            int* launches);
// E_x = -1/2 sum_ij E[i][j] over the n_occ x n_occ pair-energy matrix.
cudaError_t exchange_energy_sum(int n_occ, const double* d_E, double* d_part, double* d_ex, cudaStream_t s,
                                int* launches);

// Precision conversions and small helpers (linalg.cu)
template <typename Tin, typename Tout>
cudaError_t convert(const Tin* in, Tout* out, size_t n, cudaStream_t s, int* launches);
cudaError_t fill_zero_f64(double* p, size_t n, cudaStream_t s, int* launches);

// Device bytes of a context after a full load / localise / screen / exchange /
// ACE build / ACE apply of n_apply host functions (lace_api.cu).
// FFT scratch per context: 2 GiB of complex grids a batch (fewer, fuller
// launches); contexts of the request server take 768 MiB: on the serving
// stream 2 GiB raised the peak resident memory from 111 to 134 GB at the same
// served throughput, leaving less room for admission.
constexpr size_t kFftScratchBudget = 2048ull << 20;
constexpr size_t kServeFftScratchBudget = 768ull << 20;
size_t predict_ctx_bytes(int prec, const int n[3], int n_occ, int n_extra, int n_apply,
                         size_t fft_budget = kFftScratchBudget);

}  // namespace lace
