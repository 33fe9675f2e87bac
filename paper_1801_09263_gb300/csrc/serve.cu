// C-ABI of the exchange server (lace_server_*): the scheduler of
// serve_core.h over one context per resident system.  A REBUILD runs the
// outer-loop step of Sec. 2 (orthonormalise, SCDM, screening, exchange, ACE
// build); an APPLY is the inner-loop K_ACE application.  Each context owns its
// stream, so the requests of different systems run concurrently on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/lace.h"
#include "lace_ctx.cuh"
#include "lace_internal.cuh"
#include "serve_core.h"

namespace {

// A resident system: its context, and a high-priority stream for the short
// inner-loop applications, so that the block scheduler runs their kernels
// ahead of the CTAs of long rebuilds of other systems.
struct SysState {
    lace_ctx* ctx = nullptr;
    cudaStream_t hi = nullptr;
};

struct GpuExec {
    using Handle = SysState*;
    int device = 0, prec = LACE_MIXED;

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
            const lace_status st = lace_apply_ace(h->ctx, r.data, r.n, r.out);
            lace_set_stream(h->ctx, nullptr);
            return st;
        }
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
        if ((st = lace_apply_exchange(c, nullptr, &r.ex))) return st;
        return lace_build_ace(c, LACE_SYM_AVG);
    }

    void release(Handle& h) {
        if (!h) return;
        if (h->ctx) lace_destroy(h->ctx);
        if (h->hi) {
            cudaSetDevice(device);
            cudaStreamDestroy(h->hi);
        }
        delete h;
        h = nullptr;
    }
};

}  // namespace

struct lace_server {
    GpuExec exec;
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
    s->sched = new lace_serve::Scheduler<GpuExec>(s->exec, slots, rebuild_slots, (size_t)mem_bytes);
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

lace_status lace_server_stats(lace_server* s, unsigned long long* bytes, int* running, int* queued) {
    if (!s) return LACE_ERR_ARG;
    size_t b = 0;
    s->sched->stats(&b, running, queued);
    if (bytes) *bytes = b;
    return LACE_OK;
}

}  // extern "C"
