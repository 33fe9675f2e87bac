// Drives the exchange server's scheduler (serve_core.h) with a fake executor
// that sleeps instead of computing, and prints one JSON object per scenario:
// per request its status and start / end times (ms from the scenario start),
// and the largest number of requests seen running at once.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "serve_core.h"

using namespace lace_serve;

constexpr int kMergeable = 1 << 8;  // a flag of the fake executor's systems

struct FakeExec {
    // a system holds n_occ units once built; a REBUILD needs n_occ + n_extra
    // units while it runs; s_thr is the request's duration in seconds.
    struct Handle {
        bool built = false;
        size_t held = 0;
    };
    std::mutex mu;
    std::atomic<int> running{0}, max_running{0}, rebuilding{0}, max_rebuilding{0};
    Clock::time_point t0 = Clock::now();
    struct Rec {
        long long id;
        int sys, kind, status;
        double start, end;
    };
    std::vector<Rec> log;

    size_t predict(const SystemDesc& d, const Handle& h, int kind, int) {
        if (kind == REQ_APPLY) return h.held;
        return std::max(h.held, (size_t)(d.n_occ + d.n_extra));
    }
    size_t held(const Handle& h) { return h.held; }
    int run(const SystemDesc& d, Handle& h, Request& r) {
        const int now = ++running;
        int m = max_running.load();
        while (now > m && !max_running.compare_exchange_weak(m, now)) {}
        if (r.kind == REQ_REBUILD) {
            const int nr = ++rebuilding;
            int mr = max_rebuilding.load();
            while (nr > mr && !max_rebuilding.compare_exchange_weak(mr, nr)) {}
        }
        const double t_start = ms();
        int st = S_OK;
        if (r.kind == REQ_APPLY && !h.built) {
            st = S_ERR_STATE;
        } else {
            std::this_thread::sleep_for(std::chrono::microseconds((long long)(d.s_thr * 1e6)));
            if (r.kind == REQ_REBUILD) {
                h.built = true;
                h.held = (size_t)d.n_occ;
                r.ex = -1.0 * (r.sys + 1);
                r.n_pairs = 10 * (r.sys + 1);
            } else {
                double e = 0.0;
                for (int k = 0; k < r.n; ++k) {
                    r.out[k] = 2.0 * r.data[k];
                    e -= r.data[k] * r.data[k];
                }
                r.e_block = e;
            }
        }
        if (r.kind == REQ_REBUILD) --rebuilding;
        --running;
        std::lock_guard<std::mutex> lk(mu);
        log.push_back({r.id, r.sys, r.kind, st, t_start, ms()});
        return st;
    }
    void release(Handle& h) { h = Handle{}; }
    // systems flagged kMergeable share a key per grid size
    int merge_key(const SystemDesc& d) const { return (d.flags & kMergeable) ? d.n[0] : 0; }
    double ms() { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

static SystemDesc sys_desc(int base, int transient, double seconds, int grid = 16, bool mergeable = false) {
    return SystemDesc{{10, 10, 10}, {grid, grid, grid}, 10.0, base, transient, seconds, mergeable ? kMergeable : 0};
}

struct Sub {
    int sys, kind;
};

// scales: per submission, the factor of its 8 input values (1.5 each by
// default); cadence_tol: the rebuild-cadence tolerance of every system.
static void scenario(const char* name, int slots, size_t budget, const std::vector<SystemDesc>& systems,
                     const std::vector<Sub>& subs, int remove_after = -1, int remove_sys = -1,
                     int rebuild_slots = 0, const std::vector<double>& scales = {}, double cadence_tol = 0.0) {
    FakeExec ex;
    std::vector<double> in(8 * subs.size(), 1.5), out(8 * subs.size(), 0.0);
    for (size_t k = 0; k < scales.size() && k < subs.size(); ++k)
        for (int j = 0; j < 8; ++j) in[8 * k + j] = 1.5 * scales[k];
    std::vector<long long> ids;
    std::vector<int> res, done_flags, dues;
    std::vector<double> exs, lat, eblocks;
    std::vector<long long> npairs;
    {
        Scheduler<FakeExec> s(ex, slots, rebuild_slots > 0 ? rebuild_slots : slots, budget);
        for (auto& d : systems) {
            const int id = s.add_system(d);
            if (cadence_tol > 0.0) s.set_rebuild_tolerance(id, cadence_tol);
        }
        for (size_t k = 0; k < subs.size(); ++k) {
            long long id = -1;
            const int st = s.submit(subs[k].sys, subs[k].kind, in.data() + 8 * k, 8, out.data() + 8 * k, &id);
            ids.push_back(st == S_OK ? id : -st);
            if ((int)k == remove_after) s.remove_system(remove_sys);
        }
        for (long long id : ids) {
            int d = 0, r = -1, due = 0;
            double l = 0, e = 0, eb = 0;
            long long np = 0;
            if (id > 0) {
                s.poll(id, true, &d, &r, &l, &e, &np);
                s.apply_info(id, &eb, &due);
            }
            done_flags.push_back(d);
            res.push_back(id > 0 ? r : (int)id);
            exs.push_back(e);
            lat.push_back(l);
            npairs.push_back(np);
            eblocks.push_back(eb);
            dues.push_back(due);
        }
    }
    std::string o = std::string("{\"name\": \"") + name + "\", \"max_running\": " + std::to_string(ex.max_running.load()) +
                    ", \"max_rebuilding\": " + std::to_string(ex.max_rebuilding.load());
    o += ", \"requests\": [";
    for (size_t k = 0; k < ids.size(); ++k) {
        double st = -1, en = -1;
        for (auto& r : ex.log)
            if (r.id == ids[k]) { st = r.start; en = r.end; }
        char buf[640];
        snprintf(buf, sizeof buf,
                 "%s{\"id\": %lld, \"sys\": %d, \"kind\": %d, \"status\": %d, \"done\": %d, \"start\": %.3f, "
                 "\"end\": %.3f, \"latency\": %.3f, \"ex\": %.1f, \"n_pairs\": %lld, \"out0\": %.2f, "
                 "\"e_block\": %.17g, \"rebuild_due\": %d}",
                 k ? ", " : "", ids[k], subs[k].sys, subs[k].kind, res[k], done_flags[k], st, en, lat[k], exs[k],
                 npairs[k], subs[k].kind == REQ_APPLY ? out[8 * k] : 0.0, eblocks[k], dues[k]);
        o += buf;
    }
    o += "]}";
    printf("%s\n", o.c_str());
    fflush(stdout);
}

int main() {
    const double T = 0.05;  // 50 ms per request
    // four systems, one rebuild + two applies each, four slots, ample memory
    {
        std::vector<SystemDesc> sys;
        std::vector<Sub> subs;
        for (int k = 0; k < 4; ++k) sys.push_back(sys_desc(10, 10, T));
        for (int it = 0; it < 3; ++it)
            for (int k = 0; k < 4; ++k) subs.push_back({k, it == 0 ? REQ_REBUILD : REQ_APPLY});
        scenario("overlap", 4, 1000, sys, subs);
    }
    // one slot: strictly one request at a time, in submission order
    {
        std::vector<SystemDesc> sys{sys_desc(10, 10, 0.01), sys_desc(10, 10, 0.01)};
        std::vector<Sub> subs{{0, REQ_REBUILD}, {1, REQ_REBUILD}, {0, REQ_APPLY}, {1, REQ_APPLY}};
        scenario("serial", 1, 1000, sys, subs);
    }
    // an apply before any rebuild fails; an apply after it succeeds
    {
        std::vector<SystemDesc> sys{sys_desc(10, 10, 0.01)};
        std::vector<Sub> subs{{0, REQ_APPLY}, {0, REQ_REBUILD}, {0, REQ_APPLY}};
        scenario("state", 2, 1000, sys, subs);
    }
    // transient memory: each rebuild needs 70 of 100 while it runs and keeps
    // 30, so B waits for A, then fits; C's rebuild (needs 70 beside 60 held)
    // never fits: OOM.  The applies need nothing more and run.
    {
        std::vector<SystemDesc> sys{sys_desc(30, 40, T), sys_desc(30, 40, T), sys_desc(30, 40, T)};
        std::vector<Sub> subs{{0, REQ_REBUILD}, {1, REQ_REBUILD}, {0, REQ_APPLY}, {1, REQ_APPLY}, {2, REQ_REBUILD}};
        scenario("memory", 4, 100, sys, subs);
    }
    // removing a system frees its memory for another one's rebuild
    {
        std::vector<SystemDesc> sys{sys_desc(60, 0, T), sys_desc(60, 0, T)};
        std::vector<Sub> subs{{0, REQ_REBUILD}, {0, REQ_APPLY}, {1, REQ_REBUILD}, {0, REQ_APPLY}};
        scenario("remove", 2, 100, sys, subs, /*remove_after=*/1, /*remove_sys=*/0);
    }
    // one rebuild slot of four: rebuilds run one at a time while the applies of
    // the built system use the other slots
    {
        std::vector<SystemDesc> sys{sys_desc(10, 10, 0.03), sys_desc(10, 10, 0.1), sys_desc(10, 10, 0.1)};
        std::vector<Sub> subs{{0, REQ_REBUILD}, {1, REQ_REBUILD}, {2, REQ_REBUILD}, {0, REQ_APPLY}, {0, REQ_APPLY}};
        scenario("rebuild_slots", 4, 1000, sys, subs, -1, -1, /*rebuild_slots=*/1);
    }
    // REBUILD groups: one rebuild slot, first held by system 3 (another grid)
    // while the others queue; systems 0 and 2 share a grid and can merge,
    // system 1 is on another grid.  When the slot frees, 0 and 2 start
    // together as one group ahead of 1, which waits for the group's slot.
    {
        std::vector<SystemDesc> sys{sys_desc(10, 10, T, 16, true), sys_desc(10, 10, T, 24, true),
                                    sys_desc(10, 10, T, 16, true), sys_desc(10, 10, T, 32, false)};
        std::vector<Sub> subs{{3, REQ_REBUILD}, {0, REQ_REBUILD}, {1, REQ_REBUILD}, {2, REQ_REBUILD}};
        scenario("group", 4, 1000, sys, subs, -1, -1, /*rebuild_slots=*/1);
    }
    // a group only within the memory budget: each rebuild needs 70 of 100
    // while it runs, so 0 and 1 (same grid) run one after the other
    {
        std::vector<SystemDesc> sys{sys_desc(30, 40, T, 16, true), sys_desc(30, 40, T, 16, true)};
        std::vector<Sub> subs{{0, REQ_REBUILD}, {1, REQ_REBUILD}};
        scenario("group_memory", 4, 100, sys, subs);
    }
    // rebuild cadence: the inputs of an inner loop converge geometrically
    // (factor 1 + 0.5^k); a REBUILD resets the comparison
    {
        std::vector<SystemDesc> sys{sys_desc(10, 10, 0.001)};
        std::vector<Sub> subs{{0, REQ_REBUILD}};
        std::vector<double> scales{1.0};
        for (int k = 0; k < 14; ++k) {
            subs.push_back({0, REQ_APPLY});
            scales.push_back(1.0 + std::pow(0.5, k));
        }
        subs.push_back({0, REQ_REBUILD});
        scales.push_back(1.0);
        for (int k = 0; k < 2; ++k) {
            subs.push_back({0, REQ_APPLY});
            scales.push_back(1.25);
        }
        scenario("cadence", 1, 1000, sys, subs, -1, -1, 0, scales, 1e-3);
    }
    return 0;
}
