/*
 * liblace -- GB300 (sm_103a) library for the exchange hot path of the L-ACE
 * method (localized Adaptively Compressed Exchange, Carnimeo, Baroni and
 * Giannozzi, arXiv:1801.09263).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Hartree atomic units, e^2 = 1; Gamma point; real orbitals; spin omitted
 *    (Sec. 2).  K = -V_X is the (negative semidefinite) exchange operator:
 *    the paper's V_X carries a minus sign to be positive definite (Sec. 2).
 *  - An orthorhombic cell a x b x c (bohr) with an n1 x n2 x n3 grid,
 *    Ng = n1 n2 n3, dV = abc / Ng.  Orbitals are real arrays laid out
 *    [orbital][n1][n2][n3], C order (n3 fastest), normalised so that
 *    dV * sum_r phi(r)^2 = 1.  Inner products carry dV.
 *  - Coulomb kernel K(G) = 4 pi / |G|^2 on every G of the grid, K(0) = 0.
 *  - Host pointers are owned by the caller and only read or written during
 *    the call.  "_dev" pointers are device pointers on the context's device,
 *    borrowed for the duration of the call (the call synchronises the
 *    context's stream before returning).  All outputs go to caller buffers.
 *  - Every call returns a lace_status; nothing throws across the ABI.  A call
 *    made out of order returns LACE_ERR_STATE; lace_last_error() then holds a
 *    one-line explanation.  A context is used by one host thread at a time.
 *  - Precision LACE_FP64: every step in FP64.  LACE_MIXED: pair FFTs and the
 *    accumulation of W in FP32 with FP64 pair energies; dense contractions
 *    over the grid in split-precision (3xBF16 products, FP32 accumulate)
 *    on tensor cores; FP64 for the small N x N factorisations (Cholesky,
 *    triangular inverse, inverse square roots).
 */
#ifndef LACE_H
#define LACE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lace_ctx lace_ctx; /* opaque; created and freed by the library */

/* Interaction kernels of lace_set_kernel. */
typedef enum { LACE_KERNEL_COULOMB = 0, LACE_KERNEL_ERFC = 1 } lace_kernel;

typedef enum {
    LACE_OK = 0,
    LACE_ERR_ARG = 1,         /* bad pointer, size or option value */
    LACE_ERR_STATE = 2,       /* call made out of order */
    LACE_ERR_OOM = 3,         /* device allocation failed; context unchanged */
    LACE_ERR_CUDA = 4,        /* a CUDA call failed; see lace_last_error */
    LACE_ERR_NOT_PD = 5,      /* -M' is not positive definite (Cholesky failed) */
    LACE_ERR_TIMEOUT = 6,     /* a bounded device-side iteration did not converge */
    LACE_ERR_UNSUPPORTED = 7  /* grid size or option this build does not handle */
} lace_status;

typedef enum { LACE_FP64 = 0, LACE_MIXED = 1 } lace_precision;

/* Symmetrisation of the truncated exchange matrix M' before its Cholesky
 * factorisation (Sec. 2, after Eq. 7): (M'+M'^T)/2, upper triangle copied
 * into the lower, or lower copied into the upper. */
typedef enum { LACE_SYM_AVG = 0, LACE_SYM_UPPER = 1, LACE_SYM_LOWER = 2 } lace_sym;

/* Matrices that lace_get_matrix can return (FP64, row-major). */
typedef enum {
    LACE_MAT_OVERLAP_MODULI = 0, /* S_ik = int |w_i||w_k| (Eq. 4), n_occ x n_occ */
    LACE_MAT_EXCHANGE = 1,       /* M' = dV Psi^T W before symmetrisation (Eq. 3/7), N_P x N_P */
    LACE_MAT_CHOLESKY = 2,       /* L with -M'_sym = L L^T, lower triangular, N_P x N_P */
    LACE_MAT_PAIR_ENERGY = 3,    /* e_ik = (ik|ki) for kept occupied pairs, 0 elsewhere, n_occ x n_occ */
    LACE_MAT_SCDM_U = 4          /* orthogonal SCDM rotation U, w = phi U, n_occ x n_occ */
} lace_matrix;

/* Orbital sets that lace_get_orbitals can return (FP64, [orbital][n1][n2][n3]). */
typedef enum {
    LACE_ORB_PSI = 0, /* projection set Psi = [w (localised occupied), extras], N_P orbitals */
    LACE_ORB_W = 1,   /* W = K' Psi from the last lace_apply_exchange, N_P orbitals */
    LACE_ORB_XI = 2   /* ACE vectors xi = W L^{-T}, N_P orbitals */
} lace_orbitals;

/* Create a context on CUDA device `device` computing in `precision`
 * (lace_precision).  *out receives the handle.  No device memory is
 * allocated until lace_set_cell. */
lace_status lace_create(lace_ctx** out, int device, int precision);

/* Free the context and all its device memory.  NULL is accepted. */
lace_status lace_destroy(lace_ctx* ctx);

/* Run the context's work on `stream` (a cudaStream_t, or NULL for the
 * context's own stream). */
lace_status lace_set_stream(lace_ctx* ctx, void* stream);

/* Time limit, in seconds (0 to 3600; default 2), of each bounded device
 * wait of this context's persistent pivoted-QR kernel (lace_localize): a
 * grid-barrier wait for the other CTAs of the launch.  A wait that runs out
 * sets an error flag and its CTA leaves the kernel (the others then run out
 * at their next barrier and leave too); lace_localize returns
 * LACE_ERR_TIMEOUT and the context stays usable, with its orbitals loaded
 * but not localised (localise again).  A short limit turns a stalled
 * launch into an error quickly; 0 makes every wait that has to wait at all
 * give up.
 * Returns LACE_ERR_ARG for a limit outside [0, 3600]. */
lace_status lace_set_wait_limit(lace_ctx* ctx, double seconds);

/* Cell, grid and orbital cutoff (Sec. 3: the exchange grid follows from the
 * cell and the cutoff; here the caller gives the grid).  cell = (a, b, c) in
 * bohr.  Every grid size must factor into 2, 3 and 5; this build handles
 * 4 <= n <= 128 (FP32) and 4 <= n <= 108 (FP64).  ecut_ha > 0 is kept for
 * the caller's records (the kernel uses every G of the grid).  Resets all
 * loaded state. */
lace_status lace_set_cell(lace_ctx* ctx, const double cell[3], int n1, int n2, int n3, double ecut_ha);

/* Interaction kernel of the exchange operator (default: LACE_KERNEL_COULOMB,
 * alpha = 1).  K(G) = alpha 4 pi/|G|^2 with K(0) = 0 (Coulomb, Eq. 2), or, for
 * range-separated hybrids such as HSE (Sec. 4), the erfc-screened short-range
 * kernel K(G) = alpha 4 pi/|G|^2 (1 - exp(-|G|^2/(4 omega^2))) with
 * K(0) = alpha pi/omega^2 (the paper cites HSE without its formula; this is
 * the standard one).  alpha is the exact-exchange fraction (0.25 for PBE0 and
 * HSE06): W and E_x scale with it.  omega (bohr^-1) must be > 0 for
 * LACE_KERNEL_ERFC.  Invalidates the exchange and ACE state; may come before
 * or after lace_set_cell.  The allocation-free call below always uses the
 * bare Coulomb kernel. */
lace_status lace_set_kernel(lace_ctx* ctx, int kind, double omega, double alpha);

/* Load n_occ occupied orbitals followed by n_extra extra (virtual) orbitals
 * from host FP64 memory phi[(n_occ+n_extra)][n1][n2][n3] (copied).  With
 * orthonormalize != 0 the occupied set is Loewdin-orthonormalised
 * (phi <- phi S^{-1/2}, S = dV phi^T phi) and the extras are projected out
 * of the occupied span and Loewdin-orthonormalised; otherwise the caller
 * guarantees orthonormality.  Until lace_localize, the occupied orbitals
 * used by the exchange are these (canonical) ones.  Resets localisation,
 * screening and exchange state; the ACE projector of the last successful
 * lace_build_ace stays usable by lace_apply_ace while n_occ + n_extra is
 * unchanged (the paper's inner loop applies the previous outer iteration's
 * ACE until the next build).  LACE_ERR_NOT_PD if an overlap matrix is
 * singular. */
lace_status lace_load_orbitals(lace_ctx* ctx, const double* phi, int n_occ, int n_extra, int orthonormalize);

/* As lace_load_orbitals, from a device FP64 buffer (borrowed). */
lace_status lace_load_orbitals_dev(lace_ctx* ctx, const double* d_phi, int n_occ, int n_extra, int orthonormalize);

/* SCDM localisation of the occupied orbitals (Sec. 2): pivoted QR of the
 * orbitals on the subsample of grid points whose three indices are
 * multiples of `stride` (2 = 1/8 of the grid) selects n_occ points; then
 * w = phi U with U = phi_C^T (phi_C phi_C^T)^{-1/2}.  pivots_out (nullable,
 * n_occ entries) receives the selected points as full-grid linear indices
 * in selection order.  Ties in the pivot choice go to the lowest index.
 * Resets screening and exchange state (not the ACE projector). */
lace_status lace_localize(lace_ctx* ctx, int stride, long long* pivots_out);

/* SCDM with imposed pivots (full-grid linear indices, n == n_occ, all
 * distinct): skips the pivoted QR.  Used to compare localised results with
 * another implementation on the same point selection. */
lace_status lace_set_pivots(lace_ctx* ctx, const long long* pivots, int n);

/* Align the localised orbitals to those of the previous call (end of Sec. 2:
 * aligning each iteration's orbitals to the previous step's lets the SCF
 * converge to arbitrary precision).  Reading: within their span, rotate them
 * to the orthonormal set closest to the previous one, w <- w Q with Q the
 * polar factor of O = dV w prev^T (orthogonal Procrustes); the SCDM rotation
 * returned by lace_get_matrix(LACE_MAT_SCDM_U) includes Q.  The first call
 * only records the reference (*aligned_out = 0); later calls rotate
 * (*aligned_out = 1, nullable) and record the rotated set.  Requires
 * lace_localize (LACE_ERR_STATE); LACE_ERR_NOT_PD when O is singular (the new
 * span is nearly orthogonal to the old one). */
lace_status lace_align_to_previous(lace_ctx* ctx, int* aligned_out);

/* Overlap-of-moduli screen (Eq. 4): an occupied pair (i, k) is dropped when
 * S_ik < s_thr (both u^(ik) and u^(ki) of Eq. 5 go); pairs with an extra
 * orbital are always kept (Sec. 4.1).  s_thr = 0 keeps everything.
 * *n_pairs_out (nullable) receives the number of pair convolutions one
 * exchange application will run (unique occupied pairs i <= k kept plus
 * n_occ * n_extra). */
lace_status lace_screen(lace_ctx* ctx, double s_thr, long long* n_pairs_out);

/* Apply the (truncated) exchange operator to the projection set Psi (Eq. 2
 * with Eq. 5): W_j = -sum_{i kept with j} w_i v_ij, v_ij the Coulomb
 * potential of w_i psi_j.  W stays on the device; W_out (nullable, host,
 * N_P x Ng FP64) receives a copy.  ex_out (nullable) receives E_x for
 * f_spin = 1: -1/2 sum over ordered kept occupied pairs of (ik|ki). */
lace_status lace_apply_exchange(lace_ctx* ctx, double* W_out, double* ex_out);

/* E_x of the last lace_apply_exchange, times f_spin (1 for the unit
 * occupations of Sec. 2, 2 for a closed shell). */
lace_status lace_exchange_energy(lace_ctx* ctx, double f_spin, double* ex_out);

/* Build the ACE projector from the last W (Eq. 3 and its Cholesky form):
 * M' = dV Psi^T W, symmetrised by `sym` (lace_sym), -M'_sym = L L^T in
 * FP64, xi = W L^{-T}.  LACE_ERR_NOT_PD (the Cholesky factorisation met a
 * pivot <= 0, e.g. M' = 0 when every pair was screened out) stops before L
 * and xi are written: the previous ACE projector, its L and lace_apply_ace
 * stay as they were (LACE_MAT_EXCHANGE then holds the failing M').  After
 * any other failure lace_apply_ace returns LACE_ERR_STATE until a build
 * succeeds. */
lace_status lace_build_ace(lace_ctx* ctx, int sym);

/* K_ACE psi = -xi (dV xi^T psi) for n functions psi (host FP64,
 * [n][n1][n2][n3]); kpsi_out (host FP64, same shape) receives the result.
 * In mixed precision the functions go in up to four chunks whose uploads,
 * applications and downloads overlap (two extra streams of the context,
 * made on first use); the call returns when all are done.  A tensor-core
 * wait that gave up (LACE_ERR_TIMEOUT) is reported when the call returns;
 * kpsi_out is then undefined. */
lace_status lace_apply_ace(lace_ctx* ctx, const double* psi, int n, double* kpsi_out);

/* The ACE energy of the block of the last lace_apply_ace(_dev):
 * sum_j <psi_j| K_ACE |psi_j> = dV sum_j psi_j . (K_ACE psi)_j = -|X|^2 with
 * X = dV xi^T psi (in Ha for dV-normalised psi_j), formed on the device from
 * the application's own N_P x n coefficients.  Its change between
 * consecutive applications of one projector measures how far the inner loop
 * of the paper's double loop (Sec. 2) still moves.  LACE_ERR_STATE before
 * the first application. */
lace_status lace_get_ace_energy(lace_ctx* ctx, double* e_out);

/* As lace_apply_ace with device FP64 buffers (borrowed). */
lace_status lace_apply_ace_dev(lace_ctx* ctx, const double* d_psi, int n, double* d_kpsi_out);

/* Copy a matrix (lace_matrix) to host FP64 memory `out` of `count` doubles;
 * LACE_ERR_ARG if count is smaller than the matrix. */
lace_status lace_get_matrix(lace_ctx* ctx, int which, double* out, long long count);

/* Copy an orbital set (lace_orbitals) to host FP64 memory `out` of `count`
 * doubles (N_P x Ng). */
lace_status lace_get_orbitals(lace_ctx* ctx, int which, double* out, long long count);

/* Copy the kept pair list: pairs_out[2*p], pairs_out[2*p+1] = (i, j) with i
 * occupied and i <= j for occupied j; up to `cap` pairs; *n_out = count. */
lace_status lace_get_pairs(lace_ctx* ctx, int* pairs_out, long long cap, long long* n_out);

/* The SCDM points of the last lace_localize or lace_set_pivots (Sec. 2):
 * n_occ full-grid linear indices in selection order, into pivots_out (n
 * entries, n >= n_occ).  LACE_ERR_STATE before localisation. */
lace_status lace_get_pivots(lace_ctx* ctx, long long* pivots_out, int n);

/* Device milliseconds of the stages of the last calls (CUDA events on the
 * context's stream): [0] load+orthonormalise, [1] localise, [2] screen,
 * [3] exchange (pair convolutions), [4] ACE build, [5] ACE apply,
 * [6] pair-convolution kernels alone (sum over their launches). */
lace_status lace_get_timings(lace_ctx* ctx, double* ms_out, int count);

/* Number of kernel launches the library made since the context was
 * created (all calls). */
lace_status lace_get_launch_count(lace_ctx* ctx, long long* count_out);

/* Device bytes the context's buffers hold now (they grow to the largest
 * request seen and are freed by lace_destroy). */
lace_status lace_get_device_bytes(lace_ctx* ctx, unsigned long long* bytes_out);

/* ------------------------------------------------------------------ plane waves
 * Front end for orbitals given as plane-wave coefficients, the basis of the
 * paper's V_X matrix (Sec. 2), with grids derived from cutoffs (Sec. 3).
 * Basis of real (Gamma-point) orbitals: the half sphere of
 * G = 2 pi (m1/a, m2/b, m3/c) with |G|^2/2 < ecut, half-space m3 > 0, or
 * m3 = 0 and m2 > 0, or m3 = m2 = 0 and m1 >= 0, ordered by |G|^2 and then
 * (m1, m2, m3); phi(r) = c(0) + 2 Re sum_{G != 0} c(G) exp(i G.r), so
 * c(G) = (1/Ng) sum_r phi(r) exp(-i G.r).  Coefficients are interleaved FP64
 * (re, im) [orbital][n_pw]; the imaginary part of c(0) is ignored.  The
 * transforms run on the device in FP64 (two orbitals per complex FFT). */

/* The basis of a cell and cutoff: *n_pw_out = its size; m_out (nullable)
 * receives up to cap triples (m1, m2, m3).  Host only. */
lace_status lace_pw_basis(const double cell[3], double ecut_ha, int* m_out, long long cap, long long* n_pw_out);

/* Smallest 2^a 3^b 5^c grid holding the sphere |G|^2/2 < ecut_ha without
 * folding (n >= 2 m_max + 1 on each axis).  For an exchange grid free of
 * aliasing pass the cutoff of the pair densities (4x the orbital cutoff).
 * LACE_ERR_UNSUPPORTED beyond 128 points.  Host only. */
lace_status lace_grid_for_cutoff(const double cell[3], double ecut_ha, int dims_out[3]);

/* lace_load_orbitals from coefficients in the basis of the context's cell and
 * cutoff (lace_set_cell).  coef: host, n_occ + n_extra rows of n_pw complex
 * values, copied.  LACE_ERR_ARG when n_pw is not the basis size or the sphere
 * does not fit the grid (|m| < n/2 on every axis); LACE_ERR_UNSUPPORTED when an
 * FP64 grid plane does not fit in shared memory. */
lace_status lace_load_orbitals_pw(lace_ctx* ctx, const double* coef, long long n_pw, int n_occ, int n_extra,
                                  int orthonormalize);

/* Orbitals (LACE_ORB_PSI / W / XI, as lace_get_orbitals) as coefficients of
 * the context's basis: coef_out host, n_p rows of n_pw complex values.  W in
 * this form is the V_X matrix applied to the orbitals, as plane-wave codes
 * use it (with the sign convention of lace_apply_exchange). */
lace_status lace_get_orbitals_pw(lace_ctx* ctx, int which, double* coef_out, long long n_pw);

/* ------------------------------------------------------------------ serving
 * A request server over resident systems (the paper's double SCF loop, Sec. 2,
 * rebuilds ACE once per outer iteration and applies it many times; a server
 * keeps each system's projector on the device between those requests).
 * Each system owns a context and CUDA stream (APPLY requests run on a
 * high-priority stream of their system); `slots` worker threads each run one
 * request at a time, taking the earliest queued request whose system is idle,
 * whose device memory fits the budget and, for a REBUILD, for which one of the
 * `rebuild_slots` is free, so requests for different systems overlap on the
 * GPU and short applications are not stuck behind long rebuilds.  Requests of one system run in submission
 * order; a request that does not fit yet waits while others run, and may be
 * overtaken by requests of other systems that do fit.  Memory is accounted
 * as the bytes every resident system holds plus, for each running request,
 * the predicted growth of its system.  Host buffers passed to a request must
 * stay valid until it completes.  All server calls are thread-safe. */
typedef struct lace_server lace_server;

typedef enum {
    LACE_REQ_REBUILD = 0, /* data = n_occ + n_extra raw orbitals (host FP64): orthonormalise,
                             localise (stride 2), screen at the system's S_thr, apply the
                             exchange and build ACE; the result is E_x (f_spin = 1) */
    LACE_REQ_APPLY = 1    /* data = n functions (host FP64): out = K_ACE data (host FP64) */
} lace_request_kind;

/* Server on `device` computing in `precision` with `slots` concurrent
 * requests (1..64), of which at most rebuild_slots (1..slots; 0 = slots) are
 * REBUILDs, and a device-memory budget of mem_bytes (0 = 90% of the free
 * memory at creation). */
lace_status lace_server_create(lace_server** out, int device, int precision, int slots, int rebuild_slots,
                               unsigned long long mem_bytes);

/* Wait for every queued request, then free all systems.  NULL is accepted. */
lace_status lace_server_destroy(lace_server* srv);

/* Flags of lace_server_add_system. */
#define LACE_SYSTEM_ALIGN 1 /* every REBUILD aligns its localised orbitals to the previous ones */

/* Register a resident system (cell, grid and cutoff as lace_set_cell; the
 * orbital counts and screening threshold of its rebuilds; flags).
 * *system_id_out receives its id.  Nothing is computed until its first
 * REBUILD. */
lace_status lace_server_add_system(lace_server* srv, const double cell[3], int n1, int n2, int n3, double ecut_ha,
                                   int n_occ, int n_extra, double s_thr, int flags, int* system_id_out);

/* Queue a request (lace_request_kind) for a system.  data (host, borrowed
 * until completion) holds n_occ + n_extra orbitals for a REBUILD or n
 * functions for an APPLY; out (host, n functions, APPLY only) receives
 * K_ACE data.  *request_id_out receives the request id.  LACE_ERR_ARG for an
 * unknown system or bad sizes (an APPLY takes 1 .. n_occ + n_extra + 64
 * functions); an APPLY before the system's first successful REBUILD
 * completes with LACE_ERR_STATE; a request that does not fit the memory
 * budget while no other request runs completes with LACE_ERR_OOM. */
lace_status lace_server_submit(lace_server* srv, int system_id, int kind, const double* data, int n, double* out,
                               long long* request_id_out);

/* Status of a request: *done_out = 1 once it has completed (wait != 0 blocks
 * until then).  On completion *result_out holds its lace_status, *latency_ms
 * the time from submission to completion, and for a REBUILD *ex_out its E_x
 * and *n_pairs_out the pair convolutions it ran.  Any output may be NULL;
 * LACE_ERR_ARG for an unknown request id. */
lace_status lace_server_poll(lace_server* srv, long long request_id, int wait, int* done_out, int* result_out,
                             double* latency_ms, double* ex_out, long long* n_pairs_out);

/* What made a completed request fail ("" when it succeeded); NULL for an
 * unknown or unfinished request.  The string lives as long as the server. */
const char* lace_server_request_error(lace_server* srv, long long request_id);

/* Rebuild cadence of a system (the double loop of Sec. 2: the projector of
 * an outer iteration serves the inner iterations until they converge, then
 * the outer loop rebuilds it).  With tol > 0, every completed APPLY of the
 * system reports rebuild_due = 1 (lace_server_apply_info) once its block's
 * ACE energy sum_j <data_j|K_ACE|data_j> differs by at most tol (relative)
 * from that of the system's previous APPLY of as many functions on the same
 * projector; the first APPLY after a REBUILD reports 0.  tol = 0 (default)
 * never reports a rebuild as due.  LACE_ERR_ARG for an unknown system or
 * tol < 0. */
lace_status lace_server_set_rebuild_tolerance(lace_server* srv, int system_id, double tol);

/* APPLY results of a completed request: *e_block_out its block's ACE energy
 * (lace_get_ace_energy) and *rebuild_due_out the cadence's decision.  Any
 * output may be NULL; LACE_ERR_ARG for an unknown or unfinished request. */
lace_status lace_server_apply_info(lace_server* srv, long long request_id, double* e_block_out,
                                   int* rebuild_due_out);

/* Free a system's device memory once its queued requests have completed
 * (blocks until then); later requests for it fail with LACE_ERR_ARG. */
lace_status lace_server_remove_system(lace_server* srv, int system_id);

/* Merged pair convolutions across requests (on by default, window 50 ms).
 * The REBUILDs of systems on one cubic grid size with size-specialised
 * passes (n in {24, 32, 36, 40, 48, 50, 54, 60, 64, 72, 80, 96, 100}, mixed
 * precision) that reach their exchange step together share every launch of
 * the FFT passes: one launch per pass covers the next chunk of complex grids
 * of every such system, each grid resolving its own system's orbitals, W,
 * kernel table and scratch.  The scheduler admits such REBUILDs in groups:
 * when one starts, up to 3 queued REBUILDs of other idle systems on the same
 * grid (each its system's oldest queued request, within the memory budget)
 * start with it, the group taking one rebuild slot and going ahead of
 * requests queued before its companions.  The first REBUILD of a size to
 * reach its exchange step waits at most window_ms (0..10000) for the others
 * of that size already started.  Results are those of the REBUILDs run alone
 * (the same arithmetic per grid).  enable = 0 turns off both the merging and
 * the groups.  Call while no request is queued or running (LACE_ERR_STATE
 * otherwise). */
lace_status lace_server_set_pair_merging(lace_server* srv, int enable, double window_ms);

/* Counters of the merged pair convolutions: launch batches queued, batches
 * that held more than one REBUILD, and the REBUILDs those held.  Any output
 * may be NULL. */
lace_status lace_server_merge_stats(lace_server* srv, long long* batches, long long* merged_batches,
                                    long long* merged_requests);

/* Snapshot: device bytes held by resident systems, requests running and
 * requests queued.  Any output may be NULL. */
lace_status lace_server_stats(lace_server* srv, unsigned long long* bytes_resident, int* running, int* queued);

/* ------------------------------------------------------------------ batches
 * Batched uneven instances: many independent systems (each its own cell,
 * grid, cutoff, orbital count and threshold) run the localised exchange and
 * the ACE build of Sec. 2 together, in the mixed precision of LACE_MIXED:
 * per instance orthonormalisation, SCDM (stride 2) and screening on host
 * worker threads; then the pair convolutions of every instance in one
 * persistent cooperative launch (one per scratch chunk of 16 GiB), E_x, and
 * the ACE builds on forked streams.  That second part runs eagerly on the
 * first lace_batch_run and is captured into a CUDA graph on the second;
 * later runs replay it.  The launch shape of the persistent kernel (threads
 * per CTA, CTAs per SM) is chosen by timing every candidate on the first
 * run, against a per-instance mode that runs each instance's pair
 * convolutions through the single-system (size-specialised) passes; the
 * faster is kept.  A graph of the per-instance mode is re-captured (and
 * updated in place) every run, since its launch sizes follow the pair
 * counts. */
typedef struct lace_batch lace_batch;

typedef struct {
    double cell[3];     /* orthorhombic a, b, c (bohr) */
    int n1, n2, n3;     /* grid, 2^a 3^b 5^c, 4 .. 128 */
    double ecut_ha;     /* orbital cutoff, as lace_set_cell */
    int n_occ;          /* occupied orbitals, 1 .. 1024 */
    double s_thr;       /* screening threshold (Eq. 5) */
} lace_instance;

/* A batch of n_inst (1 .. 4096) instances on `device`.  LACE_ERR_UNSUPPORTED
 * for a grid as lace_set_cell rejects it. */
lace_status lace_batch_create(lace_batch** out, int device, int n_inst, const lace_instance* inst);

/* Free the batch and its instances' contexts.  NULL is accepted. */
lace_status lace_batch_destroy(lace_batch* batch);

/* Raw orbitals of instance `inst` (host FP64 [n_occ][n1][n2][n3], borrowed:
 * read by every later lace_batch_run, so they must stay valid and may be
 * changed between runs). */
lace_status lace_batch_set_orbitals(lace_batch* batch, int inst, const double* phi);

/* Run every instance.  ex_out[q] (nullable) receives E_x of instance q
 * (f_spin = 1), status_out[q] (nullable) its status: LACE_ERR_NOT_PD for
 * a failed Cholesky, LACE_ERR_TIMEOUT for a bounded wait that gave up, or
 * the status of its setup.  The call returns LACE_OK when it ran, even if
 * some instances failed. */
lace_status lace_batch_run(lace_batch* batch, double* ex_out, int* status_out);

/* The context of instance `inst` (owned by the batch): after a run the
 * getters lace_get_matrix / lace_get_orbitals / lace_get_pairs and the ACE
 * applications work on it.  NULL for a bad index. */
lace_ctx* lace_batch_context(lace_batch* batch, int inst);

/* The chosen launch shape, the scratch chunks (launches of the persistent
 * kernel), graph replays so far, kernel launches so far (all instances),
 * milliseconds of the last run ([0] setup, host; [1] pair convolutions,
 * device, of the last eager run or of the autotuned shape; [2] pair
 * convolutions + energies + ACE builds, device; [3] the whole call, host) and the timed candidates
 * (-1: did not fit; eight persistent launch shapes 128x1, 128x2, 128x3,
 * 128x4, 256x1, 256x2, 512x1, 512x2, then the per-instance mode).  The shape
 * outputs name the best persistent shape even when the per-instance mode
 * was kept (it was when its time is the smallest).  The environment variable
 * LACE_BATCH_SHAPE=<threads>x<ctas> restricts the persistent kernel to one
 * shape and keeps it (for tests).  Any output may be NULL. */
lace_status lace_batch_info(lace_batch* batch, int* threads, int* ctas_per_sm, int* chunks, long long* graph_replays,
                            long long* launches, double* ms_out, double* tune_ms_out, int tune_count);

/* The mode the batch runs its pair convolutions in: *per_instance = 1 for
 * the per-instance single-system passes, 0 for the persistent kernel (before
 * the first run: 0).  LACE_ERR_ARG for a null argument. */
lace_status lace_batch_mode(lace_batch* batch, int* per_instance);

/* Message of the last failed batch call. */
const char* lace_batch_last_error(lace_batch* batch);

/* Allocation-free exchange application (the paper has no counterpart: this
 * call exists for callers that cannot allocate device memory where they need
 * the exchange, e.g. a latency-critical loop where cudaMalloc/cudaFree would
 * synchronise the device and stall other streams, or a program whose device
 * memory is owned end to end by its own pool allocator).
 *
 * Computes, in FP64 and without a context, what lace_apply_exchange computes
 * for a given pair list: W_j = -sum_i w_i v_ij over the pairs, with
 * W_i -= w_j v_ij as well for an occupied j != i, and the pair energies.
 *   cell      orthorhombic cell (a, b, c) in bohr (host, read during the call)
 *   n1..n3    grid; each 2^a 3^b 5^c in [4, 128] and small enough for the FP64
 *             passes' shared memory (n <= 108 on GB300)
 *   d_psi     device FP64 [n_p][n1][n2][n3]; rows < n_occ are the occupied w_i
 *   d_pairs   device int32 [n_pairs][2] of (i, j): i < n_occ, j < n_p, i <= j
 *             when j < n_occ, each pair at most once (the layout
 *             lace_get_pairs returns)
 *   d_W       device FP64 [n_p][n1][n2][n3], overwritten (cleared first)
 *   d_pair_e  device FP64 [n_occ][n_occ], overwritten: (ij|ji) of each pair,
 *             both (i, j) and (j, i), zero elsewhere; E_x = -1/2 sum
 *   stream    cudaStream_t the work is queued on (NULL = legacy default)
 * Memory: every call uses one fixed 32 MiB device array inside the library
 * (allocated when the library's device code is loaded, held until exit) and
 * calls no cudaMalloc/cudaFree.  The array keeps the last call's contents;
 * everything a call reads from it is rewritten by that call first.  Calls
 * that overlap on the GPU (different streams, or different host threads on
 * one device) share the array and race: serialise them.
 * Set-up: the first call on a device, and the first call after a
 * cudaDeviceReset of it, looks up the array's device address with that
 * device current (the reset gives the device code a new context, where the
 * array can sit at another address).  Each call synchronises `stream` once,
 * after checking the pair list on the device and before queueing the FFT
 * passes.
 * Returns LACE_ERR_ARG for null pointers, bad counts, a pair outside the
 * ranges above or a pair listed twice; LACE_ERR_UNSUPPORTED for a grid size
 * outside the list above or when one complex FFT grid (16 n1 n2 n3 bytes)
 * with its energy partials, the pair descriptors ((n_pairs+1)/2 x 16 bytes)
 * and a bitmap of n_occ x n_p bits do not fit in the 32 MiB array together;
 * LACE_ERR_CUDA on a CUDA error. */
lace_status lace_exchange_pairs_noalloc(const double cell[3], int n1, int n2, int n3, const double* d_psi,
                                        int n_occ, int n_p, const int* d_pairs, long long n_pairs, double* d_W,
                                        double* d_pair_e, void* stream);

/* Arithmetic peaks of device `device`, measured: rates_out[0] FP32 FLOP/s
 * of scalar fused multiply-adds, [1] FP32 FLOP/s of packed pair FMAs
 * (fma.rn.f32x2, two per instruction), [2] FP64 FLOP/s of fused
 * multiply-adds (2 FLOP per FMA; entries past [2] are set to 0).  Each is the
 * best of five CUDA-event-timed launches of independent dependent-FMA chains
 * filling every SM.  These are the ceilings the ALU-bound steps of the path
 * (FFT butterflies, FP32 Gram matrices, FP64 factorisations) are reported
 * against; the paper gives none (its timings are whole CPU runs, Sec. 4).
 * Takes about 0.3 s; allocates and frees a small device buffer. */
lace_status lace_probe_peak_rates(int device, double* rates_out, int count);

/* Static description of a status code. */
const char* lace_status_string(lace_status status);

/* One-line description of the last error on this context ("" if none). */
const char* lace_last_error(lace_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LACE_H */
