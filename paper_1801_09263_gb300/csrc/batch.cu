// Batched uneven instances (lace_batch_*): many independent systems, each
// with its own cell, grid and orbital count, run localised exchange and the
// ACE build (Sec. 2) together.
//
//   setup (per instance, host worker threads, one stream each):
//       orthonormalise (FP32 Newton-Schulz + FP64 refinement), SCDM, screen
//   hot part (one stream, forked for the ACE builds):
//       zero W and the pair energies of every instance
//       pair convolutions of every instance: one persistent cooperative
//           launch per scratch chunk (pairconv_multi.cu), launch shape
//           (threads per CTA, CTAs per SM) chosen by timing on first use
//       E_x per instance
//       ACE build per instance (tcgen05 3xBF16 M', FP64 Cholesky and L^{-1},
//           xi = W L^{-T}), spread over 8 forked streams
//
// The hot part runs eagerly on the first call and is captured into a CUDA
// graph on the second; later calls replay the graph.  Nothing in it reads
// back to the host: failures are flags in device memory, read after the
// graph (Cholesky, tensor-core waits, grid barriers).  It is re-captured
// when the set of instances that passed setup changes or when the pair
// counts need more scratch chunks than the captured graph has launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lace.h"
#include "lace_ctx.cuh"
#include "lace_internal.cuh"

using namespace lace;

namespace {

constexpr int kBranches = 8;
constexpr int kSetupThreads = 48;  // setup is latency-bound (host round trips): one thread per instance
constexpr size_t kPoolCap = 16ull << 30;  // complex scratch of the pair convolutions, bytes

size_t ace_work_bytes(int n, size_t ng) {
    size_t w = gemm_rows_work_elems(n, n, ng) * sizeof(double);
    w = std::max(w, tc_gram_work_elems(n, n, ng) * sizeof(double));
    w = std::max(w, tc_combine_scratch_bytes(n, n));
    return w;
}

// The ACE build of one instance with nothing read back (capturable).
// Flags: c->flag[0] tensor-core Gram timeout, [1] Cholesky failure,
// [2] tensor-core combination timeout.
cudaError_t ace_build_deferred(lace_ctx* c, cudaStream_t s, int* launches) {
    const int n = c->n_p;
    const size_t ng = c->g.ng;
    const float* psi = c->psi.as<float>();
    const float* W = c->W.as<float>();
    double* M = c->m(MS_M);
    double* A = c->m(MS_MSYM);
    double* Linv = c->m(MS_LINV);
    double* LinvT = c->m(MS_LINVT);
    int* f = c->flag.as<int>();
    cudaError_t e;
    const bool aligned = ng % 4 == 0 && (uintptr_t)psi % 16 == 0 && (uintptr_t)W % 16 == 0;
    if (aligned) {
        e = tc_gram(n, n, ng, psi, ng, W, ng, c->g.dv, M, n, c->work.as<double>(), c->work.bytes / sizeof(double),
                    f + 0, nullptr, s, launches);
    } else {
        if ((e = cudaMemsetAsync(f, 0, sizeof(int), s))) return e;
        e = gemm_rows<float>(n, n, ng, psi, ng, W, ng, c->g.dv, false, M, n, c->work.as<double>(),
                             c->work.bytes / sizeof(double), s, launches);
    }
    if (e) return e;
    if ((e = symmetrize(n, M, A, LACE_SYM_AVG, true, s, launches))) return e;
    if ((e = cholesky_lower(n, A, n, f + 1, nullptr, s, launches))) return e;
    if ((e = cudaMemcpyAsync(c->m(MS_L), A, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s))) return e;
    if ((e = trtri_lower(n, A, n, Linv, n, s, launches))) return e;
    if ((e = transpose_f64(n, Linv, LinvT, s, launches))) return e;
    return tc_combine(n, ng, n, W, ng, LinvT, n, 0.0, c->xi.as<float>(), ng, c->work.p, f + 2, nullptr, s, launches);
}

}  // namespace

struct lace_batch {
    int device = 0;
    int n = 0;
    std::vector<lace_instance> desc;
    std::vector<lace_ctx*> ctx;
    std::vector<const double*> phi;
    std::vector<int> status;
    std::vector<char> in_graph;  // instances of the prepared hot part
    cudaStream_t main = nullptr;
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kBranches] = {}, ev_pc0 = nullptr, ev_pc1 = nullptr, ev_h0 = nullptr,
                ev_h1 = nullptr;
    std::vector<cudaEvent_t> ev_ready;
    DevBuf inst, ngrids, pool, epart, bar;
    int* h_ngrids = nullptr;  // pinned
    size_t pool_elems = 0, epart_elems = 0, smem = 0;  // smem: what one item needs
    size_t smem_run = 0;                                 // dynamic shared memory of the chosen launch shape
    int threads = 0, ctas = 0, chunks = 0;
    int mode = 0;  // 0: one persistent multi-instance launch per chunk; 1: per-instance specialised passes
    bool prepared = false;
    cudaGraphExec_t exec = nullptr;
    long long runs = 0, replays = 0, launches = 0, hot_launches = 0;
    bool graph_ok = true;  // false once a capture has failed: the hot part then runs eagerly
    double ms[4] = {};  // setup (host), pair convolutions (device), hot part (device), whole call (host)
    double pc_eager_ms = 0.0;  // pair convolutions of the last eager run (events are not recorded in the graph)
    std::vector<double> tune;  // ms per candidate launch shape; the last entry: the per-instance mode
    std::string err;
};

namespace {

lace_status bfail(lace_batch* b, lace_status st, const std::string& m) {
    b->err = m;
    return st;
}

lace_status bcuda(lace_batch* b, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LACE_OK;
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? LACE_ERR_OOM : LACE_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCK(expr, where)                                  \
    do {                                                  \
        lace_status _st = bcuda(b, (expr), (where));      \
        if (_st != LACE_OK) return _st;                   \
    } while (0)

MultiArgs multi_args(lace_batch* b) {
    MultiArgs A{};
    A.inst = b->inst.as<MultiInst>();
    A.n_inst = b->n;
    A.n_grids = b->ngrids.as<int>();
    A.pool = b->pool.as<cplx<float>>();
    A.pool_elems = b->pool_elems;
    A.epart = b->epart.as<double>();
    A.epart_elems = b->epart_elems;
    A.bar = b->bar.as<unsigned>();
    return A;
}

int chunks_for(lace_batch* b) {
    std::vector<int> ngr(b->n), n1(b->n);
    std::vector<size_t> ng(b->n);
    for (int q = 0; q < b->n; ++q) {
        ngr[q] = b->h_ngrids[q];
        ng[q] = b->ctx[q]->g.ng;
        n1[q] = b->ctx[q]->g.n[0];
    }
    return pairconv_multi_chunks(ngr, ng, n1, b->pool_elems, b->epart_elems);
}

// Buffers, instance table and launch shape for the instances that passed
// setup (eager, before any capture).
lace_status prepare(lace_batch* b) {
    cudaSetDevice(b->device);
    size_t need_pool = 0, max_ng = 0, min_ng = SIZE_MAX;
    int max_n1 = 0, max_n2 = 0, max_n3 = 0;
    std::vector<MultiInst> hi(b->n);
    size_t spec_smem = 0;
    for (int q = 0; q < b->n; ++q) {
        lace_ctx* c = b->ctx[q];
        const size_t ng = c->g.ng;
        const int np = c->n_p;
        max_ng = std::max(max_ng, ng);
        min_ng = std::min(min_ng, ng);
        max_n1 = std::max(max_n1, c->g.n[0]);
        max_n2 = std::max(max_n2, c->g.n[1]);
        max_n3 = std::max(max_n3, c->g.n[2]);
        const size_t max_grids = ((size_t)np * (np + 1) / 2 + 1) / 2;
        need_pool += max_grids * ng;
        MultiInst& I = hi[q];
        std::memset(&I, 0, sizeof(I));
        if (!b->in_graph[q]) continue;  // n_grids = 0: the kernel never reads it
        // ACE buffers (sized before any capture)
        if (c->xi.ensure((size_t)np * ng * sizeof(float)) != cudaSuccess ||
            c->work.ensure(std::max(c->work.bytes, ace_work_bytes(np, ng))) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, LACE_ERR_OOM, "out of device memory for the ACE buffers");
        }
        for (int a = 0; a < 3; ++a) {
            I.P.ax[a] = c->g.ax[a];
            I.P.tw[a] = c->tw_f[a].as<cplx<float>>();
            I.P.g2[a] = c->g2_f[a].as<float>();
        }
        I.P.kscale = (float)(4.0 * M_PI / (double)ng);
        I.P.ktab = c->ktab_f.as<float>();
        I.P.psi = c->psi.as<float>();
        I.P.n_occ = c->n_occ;
        I.P.W = c->W.as<float>();
        I.P.grids = c->grids.as<PairGrid>();
        I.P.ng = ng;
        I.P.dv = c->g.dv;
        I.E = c->m(MS_E);
        I.n1 = c->g.n[0];
        I.n2 = c->g.n[1];
        I.spec = multi_spec_size(c->g.n[0], c->g.n[1], c->g.n[2]);
        spec_smem = std::max(spec_smem, multi_spec_smem(I.spec));
    }
    size_t cap = kPoolCap;
    if (const char* env = getenv("LACE_BATCH_POOL_MB")) cap = (size_t)std::max(1, atoi(env)) << 20;  // testing chunking
    b->pool_elems = std::max(std::min(need_pool, cap / sizeof(cplx<float>)), max_ng);
    b->epart_elems = 2 * (size_t)max_n1 * (b->pool_elems / min_ng + 1);
    b->smem = std::max(pairconv_multi_smem(max_n1, max_n2, max_n3), spec_smem);
    BCK(b->inst.ensure(sizeof(MultiInst) * b->n), "batch tables");
    BCK(b->ngrids.ensure(sizeof(int) * b->n), "batch tables");
    BCK(b->pool.ensure(b->pool_elems * sizeof(cplx<float>)), "batch scratch");
    BCK(b->epart.ensure(b->epart_elems * sizeof(double)), "batch scratch");
    BCK(b->bar.ensure(64), "batch barrier");
    BCK(cudaMemcpy(b->inst.p, hi.data(), sizeof(MultiInst) * b->n, cudaMemcpyHostToDevice), "batch tables");
    b->prepared = true;
    return LACE_OK;
}

// Per-instance mode: each instance's pair convolutions through the
// single-system passes (size-specialised where they exist).  The instances
// are spread over the branch streams (largest first, each to the least
// loaded stream), each stream with its own slice of the scratch pool, so
// small instances overlap.  The launch sizes follow the current pair counts,
// so a graph of this mode is re-captured every run.
lace_status pairconv_per_instance(lace_batch* b, cudaStream_t s, int* launches) {
    std::vector<int> act;
    size_t max_ng = 1;
    int max_n1 = 1;
    for (int q = 0; q < b->n; ++q) {
        if (!b->in_graph[q] || b->h_ngrids[q] == 0) continue;
        act.push_back(q);
        max_ng = std::max(max_ng, b->ctx[q]->g.ng);
        max_n1 = std::max(max_n1, b->ctx[q]->g.n[0]);
    }
    if (act.empty()) return LACE_OK;
    const auto work = [&](int q) { return (double)b->h_ngrids[q] * (double)b->ctx[q]->g.ng; };
    std::sort(act.begin(), act.end(), [&](int x, int y) { return work(x) > work(y); });
    int P = std::min<int>(kBranches, (int)act.size());
    P = (int)std::max<size_t>(1, std::min<size_t>({(size_t)P, b->pool_elems / (max_ng + 256),
                                                   b->epart_elems / (2 * (size_t)max_n1 + 256)}));
    // slices start on 2 KB boundaries (the FFT passes use vector accesses);
    // P was bounded so that a rounded slice still holds the largest grid
    const size_t part = P > 1 ? b->pool_elems / P / 256 * 256 : b->pool_elems;
    const size_t epart = P > 1 ? b->epart_elems / P / 256 * 256 : b->epart_elems;
    std::vector<double> load(P, 0.0);
    std::vector<std::vector<int>> lanes(P);
    for (int q : act) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lanes[k].push_back(q);
        load[k] += work(q);
    }
    if (P > 1) {
        BCK(cudaEventRecord(b->ev_fork, s), "batch");
        for (int k = 0; k < P; ++k) BCK(cudaStreamWaitEvent(b->branch[k], b->ev_fork, 0), "batch");
    }
    for (int k = 0; k < P; ++k) {
        cudaStream_t sk = P > 1 ? b->branch[k] : s;
        cplx<float>* pool = b->pool.as<cplx<float>>() + k * part;
        double* ep = b->epart.as<double>() + k * epart;
        for (int q : lanes[k]) {
            lace_ctx* c = b->ctx[q];
            FFTTables<float> tb;
            for (int a = 0; a < 3; ++a) {
                tb.tw[a] = c->tw_f[a].as<cplx<float>>();
                tb.g2[a] = c->g2_f[a].as<float>();
            }
            tb.ktab = c->ktab_f.as<float>();
            const size_t ng = c->g.ng;
            const int batch = (int)std::max<size_t>(
                1, std::min<size_t>({(size_t)b->h_ngrids[q], part / ng, epart / (2 * (size_t)c->g.n[0]), (size_t)1024}));
            BCK(pairconv_run<float>(c->g, tb, c->psi.as<float>(), c->n_occ, c->W.as<float>(), c->grids.as<PairGrid>(),
                                    b->h_ngrids[q], pool, batch, ep, c->m(MS_E), sk, launches, nullptr, nullptr),
                "per-instance pair convolutions");
        }
    }
    if (P > 1) {
        for (int k = 0; k < P; ++k) {
            BCK(cudaEventRecord(b->ev_join[k], b->branch[k]), "batch");
            BCK(cudaStreamWaitEvent(s, b->ev_join[k], 0), "batch");
        }
    }
    return LACE_OK;
}

// Time every launch shape once on the real batch, and the per-instance mode
// (W and E are zeroed by the hot part afterwards).
lace_status autotune(lace_batch* b) {
    const int cand[][2] = {{128, 1}, {128, 2}, {128, 3}, {128, 4}, {256, 1}, {256, 2}, {512, 1}, {512, 2}};
    const MultiArgs A = multi_args(b);
    const int chunks = std::max(1, chunks_for(b));
    float best = 1e30f;
    b->tune.clear();
    // LACE_BATCH_SHAPE=<threads>x<ctas per SM> keeps only that persistent shape
    int force_t = 0, force_c = 0;
    if (const char* fs = getenv("LACE_BATCH_SHAPE")) {
        if (sscanf(fs, "%dx%d", &force_t, &force_c) != 2) force_t = force_c = 0;
    }
    for (const auto& cd : cand) {
        const bool skip = force_t && (cd[0] != force_t || cd[1] != force_c);
        const size_t smem = skip ? 0 : pairconv_multi_cta_smem(cd[0], cd[1], b->smem);
        if (!smem) {
            b->tune.push_back(-1.0);
            continue;
        }
        int l = 0;
        BCK(pairconv_multi_run(A, chunks, smem, cd[0], cd[1], b->main, &l), "autotune");  // warm-up
        BCK(cudaEventRecord(b->ev_pc0, b->main), "autotune");
        BCK(pairconv_multi_run(A, chunks, smem, cd[0], cd[1], b->main, &l), "autotune");
        BCK(cudaEventRecord(b->ev_pc1, b->main), "autotune");
        BCK(cudaEventSynchronize(b->ev_pc1), "autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev_pc0, b->ev_pc1);
        b->tune.push_back(ms);
        b->launches += l;
        if (ms < best) {
            best = ms;
            b->threads = cd[0];
            b->ctas = cd[1];
            b->smem_run = smem;
        }
    }
    if (!b->threads) return bfail(b, LACE_ERR_UNSUPPORTED, "no launch shape of the batched pair convolutions fits");
    {
        int l = 0;
        lace_status st = pairconv_per_instance(b, b->main, &l);  // warm-up
        if (st) return st;
        BCK(cudaEventRecord(b->ev_pc0, b->main), "autotune");
        if ((st = pairconv_per_instance(b, b->main, &l))) return st;
        BCK(cudaEventRecord(b->ev_pc1, b->main), "autotune");
        BCK(cudaEventSynchronize(b->ev_pc1), "autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev_pc0, b->ev_pc1);
        b->tune.push_back(ms);
        b->launches += l;
        b->mode = ms < best ? 1 : 0;
        // LACE_BATCH_MODE=persistent | per_instance overrides the timing
        const char* fm = getenv("LACE_BATCH_MODE");
        if ((fm && !strcmp(fm, "persistent")) || force_t) b->mode = 0;
        if (fm && !strcmp(fm, "per_instance")) b->mode = 1;
        if (b->mode == 1) best = ms;
    }
    b->pc_eager_ms = best;
    return LACE_OK;
}

// The hot part on b->main (eager, or while capturing: the pair-convolution
// events are recorded in eager runs only).
lace_status enqueue_hot(lace_batch* b, bool capturing) {
    int l = 0;
    for (int q = 0; q < b->n; ++q) {
        if (!b->in_graph[q]) continue;
        lace_ctx* c = b->ctx[q];
        BCK(cudaMemsetAsync(c->W.p, 0, (size_t)c->n_p * c->g.ng * sizeof(float), b->main), "zero W");
        BCK(fill_zero_f64(c->m(MS_E), (size_t)c->n_occ * c->n_occ, b->main, &l), "zero E");
    }
    if (!capturing) BCK(cudaEventRecord(b->ev_pc0, b->main), "batch");
    if (b->mode == 1) {
        lace_status st = pairconv_per_instance(b, b->main, &l);
        if (st) return st;
    } else {
        BCK(pairconv_multi_run(multi_args(b), b->chunks, b->smem_run, b->threads, b->ctas, b->main, &l),
            "batched pair convolutions");
    }
    if (!capturing) BCK(cudaEventRecord(b->ev_pc1, b->main), "batch");
    for (int q = 0; q < b->n; ++q) {
        if (!b->in_graph[q]) continue;
        lace_ctx* c = b->ctx[q];
        BCK(exchange_energy_sum(c->n_occ, c->m(MS_E), c->exd.as<double>() + 8, c->exd.as<double>(), b->main, &l),
            "energy");
    }
    BCK(cudaEventRecord(b->ev_fork, b->main), "batch");
    for (int k = 0; k < kBranches; ++k) BCK(cudaStreamWaitEvent(b->branch[k], b->ev_fork, 0), "batch");
    int k = 0;
    for (int q = 0; q < b->n; ++q) {
        if (!b->in_graph[q]) continue;
        BCK(ace_build_deferred(b->ctx[q], b->branch[k], &l), "ACE build");
        k = (k + 1) % kBranches;
    }
    for (int j = 0; j < kBranches; ++j) {
        BCK(cudaEventRecord(b->ev_join[j], b->branch[j]), "batch");
        BCK(cudaStreamWaitEvent(b->main, b->ev_join[j], 0), "batch");
    }
    b->hot_launches = l;
    return LACE_OK;
}

// Capture the hot part; an existing executable graph is updated in place
// when the new capture has its topology (the per-instance mode re-captures
// every run with new launch sizes), else rebuilt.
lace_status capture(lace_batch* b) {
    BCK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal), "graph capture");
    lace_status st = enqueue_hot(b, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->main, &g);
    if (st != LACE_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    BCK(e, "graph capture");
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess) {
            cudaGraphDestroy(g);
            return LACE_OK;
        }
        cudaGetLastError();
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    BCK(ei, "graph instantiate");
    return LACE_OK;
}

}  // namespace

extern "C" {

lace_status lace_batch_create(lace_batch** out, int device, int n_inst, const lace_instance* inst) {
    if (!out) return LACE_ERR_ARG;
    *out = nullptr;
    if (n_inst < 1 || n_inst > 4096 || !inst) return LACE_ERR_ARG;
    lace_batch* b = new lace_batch();
    b->device = device;
    b->n = n_inst;
    b->desc.assign(inst, inst + n_inst);
    b->ctx.assign(n_inst, nullptr);
    b->phi.assign(n_inst, nullptr);
    b->status.assign(n_inst, LACE_ERR_STATE);
    b->in_graph.assign(n_inst, 0);
    lace_status st = LACE_OK;
    for (int q = 0; q < n_inst && st == LACE_OK; ++q) {
        const lace_instance& d = inst[q];
        if (d.n_occ < 1 || d.n_occ > 1024 || !(d.s_thr >= 0)) {
            st = LACE_ERR_ARG;
            break;
        }
        if ((st = lace_create(&b->ctx[q], device, LACE_MIXED))) break;
        st = lace_set_cell(b->ctx[q], d.cell, d.n1, d.n2, d.n3, d.ecut_ha);
    }
    if (st == LACE_OK) {
        cudaSetDevice(device);
        bool ok = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) == cudaSuccess;
        for (int k = 0; k < kBranches && ok; ++k) {
            ok = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
        }
        ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&b->ev_pc0) == cudaSuccess && cudaEventCreate(&b->ev_pc1) == cudaSuccess &&
             cudaEventCreate(&b->ev_h0) == cudaSuccess && cudaEventCreate(&b->ev_h1) == cudaSuccess &&
             cudaMallocHost(&b->h_ngrids, sizeof(int) * n_inst) == cudaSuccess;
        b->ev_ready.assign(n_inst, nullptr);
        for (int q = 0; q < n_inst && ok; ++q)
            ok = cudaEventCreateWithFlags(&b->ev_ready[q], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            st = LACE_ERR_CUDA;
        }
    }
    if (st != LACE_OK) {
        lace_batch_destroy(b);
        return st;
    }
    *out = b;
    return LACE_OK;
}

lace_status lace_batch_destroy(lace_batch* b) {
    if (!b) return LACE_OK;
    cudaSetDevice(b->device);
    if (b->main) cudaStreamSynchronize(b->main);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (lace_ctx* c : b->ctx) lace_destroy(c);
    DevBuf* bufs[] = {&b->inst, &b->ngrids, &b->pool, &b->epart, &b->bar};
    for (DevBuf* d : bufs) d->release();
    for (int k = 0; k < kBranches; ++k) {
        if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    for (cudaEvent_t e : {b->ev_fork, b->ev_pc0, b->ev_pc1, b->ev_h0, b->ev_h1})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_ready)
        if (e) cudaEventDestroy(e);
    if (b->main) cudaStreamDestroy(b->main);
    if (b->h_ngrids) cudaFreeHost(b->h_ngrids);
    delete b;
    return LACE_OK;
}

lace_status lace_batch_set_orbitals(lace_batch* b, int inst, const double* phi) {
    if (!b || inst < 0 || inst >= b->n || !phi) return LACE_ERR_ARG;
    b->phi[inst] = phi;
    return LACE_OK;
}

lace_status lace_batch_run(lace_batch* b, double* ex_out, int* status_out) {
    if (!b) return LACE_ERR_ARG;
    for (int q = 0; q < b->n; ++q)
        if (!b->phi[q]) return bfail(b, LACE_ERR_STATE, "orbitals of an instance were not set");
    const auto t0 = std::chrono::steady_clock::now();
    // setup: orthonormalise, SCDM, screen (host worker threads, one stream per instance)
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int q = next++; q < b->n; q = next++) {
            lace_ctx* c = b->ctx[q];
            const lace_instance& d = b->desc[q];
            lace_status st = lace_load_orbitals(c, b->phi[q], d.n_occ, 0, 1);
            if (!st) st = lace_localize(c, 2, nullptr);
            if (!st) st = lace_screen(c, d.s_thr, nullptr);
            b->status[q] = st;
        }
    };
    {
        std::vector<std::thread> pool;
        const int nt = std::min(kSetupThreads, b->n);
        for (int k = 0; k < nt; ++k) pool.emplace_back(worker);
        for (auto& t : pool) t.join();
    }
    const auto t1 = std::chrono::steady_clock::now();
    cudaSetDevice(b->device);
    bool same = b->prepared;
    for (int q = 0; q < b->n; ++q) {
        const bool ok = b->status[q] == LACE_OK;
        same = same && (ok == (b->in_graph[q] != 0));
        b->h_ngrids[q] = ok ? (int)((b->ctx[q]->n_pairs + 1) / 2) : 0;
        if (ok) {
            BCK(cudaEventRecord(b->ev_ready[q], b->ctx[q]->stream), "batch");
            BCK(cudaStreamWaitEvent(b->main, b->ev_ready[q], 0), "batch");
        }
    }
    if (!same) {
        for (int q = 0; q < b->n; ++q) b->in_graph[q] = b->status[q] == LACE_OK;
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        lace_status st = prepare(b);
        if (st) return st;
    }
    BCK(cudaMemcpyAsync(b->ngrids.p, b->h_ngrids, sizeof(int) * b->n, cudaMemcpyHostToDevice, b->main), "batch");
    const int need = std::max(1, chunks_for(b));
    lace_status st = LACE_OK;
    if (!b->threads) {
        if ((st = autotune(b))) return st;
    }
    bool eager = b->runs == 0 || !b->graph_ok;  // first call: eager (sets kernel attributes, checks the path)
    if (!eager && (!b->exec || need > b->chunks || b->mode == 1)) {
        b->chunks = std::max(need, b->chunks);
        if (capture(b) != LACE_OK) {
            // capture unsupported here: run eagerly from now on
            cudaGetLastError();
            b->graph_ok = false;
            eager = true;
        }
    }
    BCK(cudaEventRecord(b->ev_h0, b->main), "batch");
    if (eager) {
        b->chunks = std::max(need, b->chunks);
        if ((st = enqueue_hot(b, false))) return st;
    } else {
        BCK(cudaGraphLaunch(b->exec, b->main), "graph launch");
        b->replays++;
    }
    BCK(cudaEventRecord(b->ev_h1, b->main), "batch");
    b->launches += b->hot_launches;
    BCK(cudaStreamSynchronize(b->main), "batch");
    b->runs++;
    unsigned barflag = 0;
    BCK(cudaMemcpy(&barflag, b->bar.as<unsigned>() + 2, sizeof(unsigned), cudaMemcpyDeviceToHost), "batch");
    for (int q = 0; q < b->n; ++q) {
        lace_ctx* c = b->ctx[q];
        if (ex_out) ex_out[q] = 0.0;
        if (!b->in_graph[q]) continue;
        int f[3] = {0, 0, 0};
        double ex = 0.0;
        BCK(cudaMemcpy(f, c->flag.p, sizeof(f), cudaMemcpyDeviceToHost), "batch");
        BCK(cudaMemcpy(&ex, c->exd.p, sizeof(double), cudaMemcpyDeviceToHost), "batch");
        int s = LACE_OK;
        if (barflag || f[0] || f[2]) s = LACE_ERR_TIMEOUT;
        else if (f[1]) s = LACE_ERR_NOT_PD;
        b->status[q] = s;
        c->applied = true;
        c->ace = s == LACE_OK;
        if (ex_out) ex_out[q] = ex;
    }
    if (status_out) std::copy(b->status.begin(), b->status.end(), status_out);
    float pc = 0.f, hot = 0.f;
    if (eager && cudaEventElapsedTime(&pc, b->ev_pc0, b->ev_pc1) == cudaSuccess) b->pc_eager_ms = pc;
    cudaEventElapsedTime(&hot, b->ev_h0, b->ev_h1);
    cudaGetLastError();
    const auto t2 = std::chrono::steady_clock::now();
    b->ms[0] = std::chrono::duration<double, std::milli>(t1 - t0).count();
    b->ms[1] = b->pc_eager_ms;
    b->ms[2] = hot;
    b->ms[3] = std::chrono::duration<double, std::milli>(t2 - t0).count();
    return LACE_OK;
}

lace_ctx* lace_batch_context(lace_batch* b, int inst) {
    if (!b || inst < 0 || inst >= b->n) return nullptr;
    return b->ctx[inst];
}

lace_status lace_batch_info(lace_batch* b, int* threads, int* ctas_per_sm, int* chunks, long long* graph_replays,
                            long long* launches, double* ms_out, double* tune_ms_out, int tune_count) {
    if (!b) return LACE_ERR_ARG;
    if (launches) {
        long long l = b->launches;
        for (lace_ctx* c : b->ctx) l += c->launches;
        *launches = l;
    }
    if (threads) *threads = b->threads;
    if (ctas_per_sm) *ctas_per_sm = b->ctas;
    if (chunks) *chunks = b->chunks;
    if (graph_replays) *graph_replays = b->replays;
    if (ms_out) std::copy(b->ms, b->ms + 4, ms_out);
    if (tune_ms_out)
        for (int k = 0; k < tune_count; ++k) tune_ms_out[k] = k < (int)b->tune.size() ? b->tune[k] : -1.0;
    return LACE_OK;
}

lace_status lace_batch_mode(lace_batch* b, int* per_instance) {
    if (!b || !per_instance) return LACE_ERR_ARG;
    *per_instance = b->mode == 1 ? 1 : 0;
    return LACE_OK;
}

const char* lace_batch_last_error(lace_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
