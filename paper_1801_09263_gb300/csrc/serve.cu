// C-ABI of the exchange server (lace_server_*): the scheduler of
// serve_core.h over one context per resident system.  A REBUILD runs the
// outer-loop step of Sec. 2 (orthonormalise, SCDM, screening, exchange, ACE
// build); an APPLY is the inner-loop K_ACE application.  Each context owns its
// stream, so the requests of different systems run concurrently on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <vector>
#include <new>
#include <string>

#include "../../include/lace.h"
#include "lace_ctx.cuh"
#include "lace_internal.cuh"
#include "serve_core.h"

namespace {

// A resident system: its context, a high-priority stream for the short
// inner-loop applications (so that the block scheduler runs their kernels
// ahead of the CTAs of long rebuilds of other systems), and the two events
// that order its merged pair convolutions.
struct SysState {
    lace_ctx* ctx = nullptr;
    cudaStream_t hi = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
};

// Merged pair convolutions across requests.  The REBUILDs of systems on one
// grid size that reach their exchange step together share every launch of
// the FFT passes: each prepares its pair list and buffers on its own
// stream, then joins the merger.  The first to join leads: while other
// REBUILDs of that size are still on their way to the exchange step it
// waits for them (at most window_ms), then queues the passes of everything
// that joined on the merger's stream, one launch per pass for the next chunk
// of every system; the others wait until that is queued.  The systems'
// streams wait for the passes, then go on with E_x and the ACE build.
class PairMerger {
  public:
    struct Entry {
        lace_ctx* ctx = nullptr;
        lace::MergedSys<float> m{};
        int n_grids = 0, cap = 0;
        cudaEvent_t ready = nullptr, done = nullptr;
        bool launched = false;
        lace_status status = LACE_OK;
    };

    bool enabled = true;
    double window_ms = 50.0;
    int device = 0;

    ~PairMerger() {
        for (auto& kv : keys_) {
            Key& k = kv.second;
            if (k.s) {
                cudaSetDevice(device);
                cudaStreamSynchronize(k.s);
                cudaStreamDestroy(k.s);
            }
            k.refs.release();
            k.sys.release();
        }
    }

    // A REBUILD of grid size n started / left before its exchange step.
    void starting(int n) {
        std::lock_guard<std::mutex> lk(mu_);
        keys_[n].expected++;
    }
    void abandoned(int n) {
        std::lock_guard<std::mutex> lk(mu_);
        keys_[n].expected--;
        cv_.notify_all();
    }

    // Join with a prepared entry; returns once its passes are queued.
    lace_status run(int n, Entry* e) {
        std::unique_lock<std::mutex> lk(mu_);
        Key& k = keys_[n];
        k.expected--;
        k.pending.push_back(e);
        cv_.notify_all();
        if (k.leading) {
            cv_.wait(lk, [&] { return e->launched; });
            return e->status;
        }
        k.leading = true;
        const auto deadline = std::chrono::steady_clock::now() +
                              std::chrono::microseconds((long long)(1000.0 * std::max(0.0, window_ms)));
        while (k.expected > 0 && cv_.wait_until(lk, deadline) != std::cv_status::timeout) {
        }
        std::vector<Entry*> batch;
        batch.swap(k.pending);
        k.leading = false;
        std::unique_lock<std::mutex> launch_lk(k.launch_mu);  // one batch of this size queued at a time
        lk.unlock();
        const lace_status st = launch(n, k, batch);
        launch_lk.unlock();
        lk.lock();
        batches_++;
        if (batch.size() > 1) {
            merged_batches_++;
            merged_requests_ += (long long)batch.size();
        }
        for (Entry* b : batch) {
            b->status = st;
            b->launched = true;
        }
        cv_.notify_all();
        return e->status;
    }

    void stats(long long* batches, long long* merged_batches, long long* merged_requests) {
        std::lock_guard<std::mutex> lk(mu_);
        if (batches) *batches = batches_;
        if (merged_batches) *merged_batches = merged_batches_;
        if (merged_requests) *merged_requests = merged_requests_;
    }

  private:
    struct Key {
        std::vector<Entry*> pending;
        bool leading = false;
        int expected = 0;  // REBUILDs of this size started and not yet joined
        std::mutex launch_mu;
        cudaStream_t s = nullptr;
        DevBuf refs, sys;
    };

    lace_status launch(int n, Key& k, std::vector<Entry*>& batch) {
        cudaSetDevice(device);
        if (!k.s && cudaStreamCreateWithFlags(&k.s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return LACE_ERR_CUDA;
        }
        std::vector<lace::MergedSys<float>> sys;
        std::vector<int> ng, cap;
        size_t total = 0, rounds = 1;
        for (Entry* b : batch) {
            sys.push_back(b->m);
            ng.push_back(b->n_grids);
            cap.push_back(b->cap);
            total += (size_t)b->n_grids;
            rounds = std::max(rounds, (size_t)((b->n_grids + std::max(b->cap, 1) - 1) / std::max(b->cap, 1)));
        }
        // device space for the grid map and the per-round system table; the
        // previous batch of this size must be done before it is reallocated
        const size_t refs_bytes = std::max<size_t>(total, 1) * sizeof(lace::GridRef);
        const size_t sys_bytes = rounds * sys.size() * sizeof(lace::MergedSys<float>);
        if (refs_bytes > k.refs.bytes || sys_bytes > k.sys.bytes) {
            if (cudaStreamSynchronize(k.s) != cudaSuccess) return LACE_ERR_CUDA;
            if (k.refs.ensure(std::max(refs_bytes, (size_t)1 << 19)) != cudaSuccess ||
                k.sys.ensure(std::max(sys_bytes, (size_t)1 << 16)) != cudaSuccess) {
                cudaGetLastError();
                return LACE_ERR_OOM;
            }
        }
        for (Entry* b : batch)
            if (cudaStreamWaitEvent(k.s, b->ready, 0) != cudaSuccess) return LACE_ERR_CUDA;
        int launches = 0, nr = 0;
        const cudaError_t e = lace::pairconv_run_merged(n, lace::ctx_tables_f(batch[0]->ctx), sys, ng, cap,
                                                        k.refs.as<lace::GridRef>(),
                                                        k.sys.as<lace::MergedSys<float>>(), k.s, &launches, &nr);
        for (Entry* b : batch) {
            b->ctx->launches += launches;
            if (cudaEventRecord(b->done, k.s) != cudaSuccess) return LACE_ERR_CUDA;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return LACE_ERR_CUDA;
        }
        return LACE_OK;
    }

    std::mutex mu_;
    std::condition_variable cv_;
    std::map<int, Key> keys_;
    long long batches_ = 0, merged_batches_ = 0, merged_requests_ = 0;
};

struct GpuExec {
    using Handle = SysState*;
    int device = 0, prec = LACE_MIXED;
    PairMerger* merger = nullptr;

    // the grid size whose merged launches a REBUILD of d can join (0: none)
    int merge_key(const lace_serve::SystemDesc& d) const {
        if (!merger || !merger->enabled || prec != LACE_MIXED) return 0;
        if (d.n[0] != d.n[1] || d.n[1] != d.n[2] || !lace::spec_merge_ok(d.n[0])) return 0;
        return d.n[0];
    }

    size_t predict(const lace_serve::SystemDesc& d, const Handle& h, int kind, int n) const {
        const size_t now = held(h);
        if (kind == lace_serve::REQ_APPLY && !(h && h->ctx)) return now;  // fails with LACE_ERR_STATE
        const size_t full = lace::predict_ctx_bytes(prec, d.n, d.n_occ, d.n_extra,
                                                    kind == lace_serve::REQ_APPLY ? n : 0,
                                                    lace::kServeFftScratchBudget);
        return std::max(now, full);
    }

    size_t held(const Handle& h) const {
        unsigned long long b = 0;
        if (h && h->ctx) lace_get_device_bytes(h->ctx, &b);
        return (size_t)b;
    }

    int run(const lace_serve::SystemDesc& d, Handle& h, lace_serve::Request& r) {
        const lace_status st = run_calls(d, h, r);
        if (st != LACE_OK) {
            const char* m = h && h->ctx ? lace_last_error(h->ctx) : nullptr;
            r.err = std::string(lace_status_string(st)) + (m && *m ? std::string(": ") + m : std::string());
        }
        return st;
    }

    lace_status run_calls(const lace_serve::SystemDesc& d, Handle& h, lace_serve::Request& r) {
        if (r.kind == lace_serve::REQ_APPLY) {
            if (!h || !h->ctx) return LACE_ERR_STATE;
            lace_set_stream(h->ctx, h->hi);
            lace_status st = lace_apply_ace(h->ctx, r.data, r.n, r.out);
            if (st == LACE_OK) st = lace_get_ace_energy(h->ctx, &r.e_block);
            lace_set_stream(h->ctx, nullptr);
            return st;
        }
        // a REBUILD that can join merged launches counts as expected there
        // until it joins (or leaves before its exchange step)
        struct Expect {
            PairMerger* m;
            int key;
            bool joined = false;
            ~Expect() {
                if (key && !joined) m->abandoned(key);
            }
        } expect{merger, merge_key(d)};
        if (expect.key) merger->starting(expect.key);
        lace_status st = LACE_OK;
        if (!h) h = new SysState();
        if (!h->ctx) {
            if ((st = lace_create(&h->ctx, device, prec))) return st;
            h->ctx->fft_scratch_budget = lace::kServeFftScratchBudget;
            if ((st = lace_set_cell(h->ctx, d.cell, d.n[0], d.n[1], d.n[2], d.ecut))) return st;
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            if (cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest) != cudaSuccess) {
                cudaGetLastError();
                h->hi = nullptr;  // the context's own stream serves the applications too
            }
        }
        lace_ctx* c = h->ctx;
        if ((st = lace_load_orbitals(c, r.data, d.n_occ, d.n_extra, 1))) return st;
        if ((st = lace_localize(c, 2, nullptr))) return st;
        if ((d.flags & LACE_SYSTEM_ALIGN) && (st = lace_align_to_previous(c, nullptr))) return st;
        if ((st = lace_screen(c, d.s_thr, &r.n_pairs))) return st;
        if (expect.key && lace::ctx_mergeable(c)) {
            if (!h->ready && (cudaEventCreateWithFlags(&h->ready, cudaEventDisableTiming) != cudaSuccess ||
                              cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess)) {
                cudaGetLastError();
                return LACE_ERR_CUDA;
            }
            PairMerger::Entry e;
            e.ctx = c;
            e.ready = h->ready;
            e.done = h->done;
            if ((st = lace::ctx_exchange_prepare(c, &e.m, &e.n_grids, &e.cap, h->ready))) return st;
            expect.joined = true;
            if ((st = merger->run(expect.key, &e))) return st;
            if ((st = lace::ctx_exchange_finish(c, h->done, &r.ex))) return st;
        } else if ((st = lace_apply_exchange(c, nullptr, &r.ex))) {
            return st;
        }
        return lace_build_ace(c, LACE_SYM_AVG);
    }

    void release(Handle& h) {
        if (!h) return;
        if (h->ctx) lace_destroy(h->ctx);
        cudaSetDevice(device);
        if (h->hi) cudaStreamDestroy(h->hi);
        if (h->ready) cudaEventDestroy(h->ready);
        if (h->done) cudaEventDestroy(h->done);
        delete h;
        h = nullptr;
    }
};

}  // namespace

// REBUILDs of one grid size admitted together when pair merging is on.
constexpr int kRebuildGroup = 4;

struct lace_server {
    GpuExec exec;
    PairMerger merger;
    lace_serve::Scheduler<GpuExec>* sched = nullptr;
};

extern "C" {

lace_status lace_server_create(lace_server** out, int device, int precision, int slots, int rebuild_slots,
                               unsigned long long mem_bytes) {
    if (!out) return LACE_ERR_ARG;
    *out = nullptr;
    if ((precision != LACE_FP64 && precision != LACE_MIXED) || slots < 1 || slots > 64) return LACE_ERR_ARG;
    if (rebuild_slots < 0 || rebuild_slots > slots) return LACE_ERR_ARG;
    if (rebuild_slots == 0) rebuild_slots = slots;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LACE_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LACE_ERR_CUDA;
    if (mem_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return LACE_ERR_CUDA;
        mem_bytes = (unsigned long long)(0.9 * (double)fr);
    }
    lace_server* s = new (std::nothrow) lace_server();
    if (!s) return LACE_ERR_OOM;
    s->exec.device = device;
    s->exec.prec = precision;
    s->merger.device = device;
    s->exec.merger = &s->merger;
    s->sched = new lace_serve::Scheduler<GpuExec>(s->exec, slots, rebuild_slots, (size_t)mem_bytes);
    s->sched->set_rebuild_group(kRebuildGroup);
    *out = s;
    return LACE_OK;
}

lace_status lace_server_destroy(lace_server* s) {
    if (!s) return LACE_OK;
    delete s->sched;
    delete s;
    return LACE_OK;
}

lace_status lace_server_add_system(lace_server* s, const double cell[3], int n1, int n2, int n3, double ecut_ha,
                                   int n_occ, int n_extra, double s_thr, int flags, int* id_out) {
    if (!s || !cell || !id_out) return LACE_ERR_ARG;
    if (!(cell[0] > 0) || !(cell[1] > 0) || !(cell[2] > 0) || !(ecut_ha > 0) || !(s_thr >= 0)) return LACE_ERR_ARG;
    if (n1 < 4 || n2 < 4 || n3 < 4 || n1 > lace::kMaxN || n2 > lace::kMaxN || n3 > lace::kMaxN)
        return LACE_ERR_UNSUPPORTED;
    if (n_occ < 1 || n_extra < 0 || n_occ > 1024 || n_occ + n_extra > 2048) return LACE_ERR_ARG;
    if (flags & ~LACE_SYSTEM_ALIGN) return LACE_ERR_ARG;
    lace_serve::SystemDesc d{{cell[0], cell[1], cell[2]}, {n1, n2, n3}, ecut_ha, n_occ, n_extra, s_thr, flags};
    *id_out = s->sched->add_system(d);
    return LACE_OK;
}

lace_status lace_server_submit(lace_server* s, int sys, int kind, const double* data, int n, double* out,
                               long long* id_out) {
    if (!s || !id_out || !data) return LACE_ERR_ARG;
    const lace_serve::SystemDesc* d = s->sched->desc(sys);
    if (!d) return LACE_ERR_ARG;
    if (kind == LACE_REQ_REBUILD) {
        if (n != d->n_occ + d->n_extra) return LACE_ERR_ARG;
    } else if (kind == LACE_REQ_APPLY) {
        if (n < 1 || !out || n > d->n_occ + d->n_extra + 64) return LACE_ERR_ARG;
    } else {
        return LACE_ERR_ARG;
    }
    return (lace_status)s->sched->submit(sys, kind, data, n, out, id_out);
}

lace_status lace_server_poll(lace_server* s, long long id, int wait, int* done, int* result, double* lat_ms,
                             double* ex, long long* n_pairs) {
    if (!s) return LACE_ERR_ARG;
    return (lace_status)s->sched->poll(id, wait != 0, done, result, lat_ms, ex, n_pairs);
}

const char* lace_server_request_error(lace_server* s, long long id) {
    if (!s) return nullptr;
    return s->sched->error(id);
}

lace_status lace_server_remove_system(lace_server* s, int sys) {
    if (!s) return LACE_ERR_ARG;
    return (lace_status)s->sched->remove_system(sys);
}

lace_status lace_server_set_pair_merging(lace_server* s, int enable, double window_ms) {
    if (!s || !(window_ms >= 0.0 && window_ms <= 10000.0)) return LACE_ERR_ARG;
    int running = 0, queued = 0;
    s->sched->stats(nullptr, &running, &queued);
    if (running || queued) return LACE_ERR_STATE;
    s->merger.enabled = enable != 0;
    s->merger.window_ms = window_ms;
    s->sched->set_rebuild_group(enable ? kRebuildGroup : 1);
    return LACE_OK;
}

lace_status lace_server_set_rebuild_tolerance(lace_server* s, int sys, double tol) {
    if (!s || !(tol >= 0.0)) return LACE_ERR_ARG;
    return (lace_status)s->sched->set_rebuild_tolerance(sys, tol);
}

lace_status lace_server_apply_info(lace_server* s, long long id, double* e_block, int* rebuild_due) {
    if (!s) return LACE_ERR_ARG;
    return (lace_status)s->sched->apply_info(id, e_block, rebuild_due);
}

lace_status lace_server_merge_stats(lace_server* s, long long* batches, long long* merged_batches,
                                    long long* merged_requests) {
    if (!s) return LACE_ERR_ARG;
    s->merger.stats(batches, merged_batches, merged_requests);
    return LACE_OK;
}

lace_status lace_server_stats(lace_server* s, unsigned long long* bytes, int* running, int* queued) {
    if (!s) return LACE_ERR_ARG;
    size_t b = 0;
    s->sched->stats(&b, running, queued);
    if (bytes) *bytes = b;
    return LACE_OK;
}

}  // extern "C"
