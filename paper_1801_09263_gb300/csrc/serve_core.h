// Request scheduling of the exchange server: requests against resident
// systems are admitted continuously as worker slots and device memory free
// up, so the work of requests for different systems overlaps on the device.
// The paper's double loop (Sec. 2) rebuilds the ACE projector once per outer
// SCF iteration and applies it many times in the inner loop; the server keeps
// each system's projector resident between those requests.
//
// Plain C++17 (no CUDA): the executor that runs a request on a system is a
// template parameter, so the scheduling is testable without a device.
//
// Executor interface (all calls from worker threads; calls for one system are
// never concurrent):
//   using Handle = ...;                                   // per-system state, default-constructible
//   size_t predict(const SystemDesc&, const Handle&, int kind, int n);  // bytes the system holds after the request
//   size_t held(const Handle&);                           // bytes the system holds now
//   int run(const SystemDesc&, Handle&, Request&);        // status code (0 = ok); fills ex / n_pairs /
//                                                         // e_block (APPLY) / err
//   void release(Handle&);                                // free the system's memory
//   int merge_key(const SystemDesc&);                     // REBUILDs of systems with one nonzero key can
//                                                         // share their pair-convolution launches (0: never)
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace lace_serve {

// Status codes (the values of lace_status).
enum { S_OK = 0, S_ERR_ARG = 1, S_ERR_STATE = 2, S_ERR_OOM = 3 };
enum { REQ_REBUILD = 0, REQ_APPLY = 1 };

using Clock = std::chrono::steady_clock;

struct SystemDesc {
    double cell[3];
    int n[3];
    double ecut;
    int n_occ, n_extra;
    double s_thr;
    int flags;
};

struct Request {
    long long id = 0;
    int sys = 0, kind = 0, n = 0;
    const double* data = nullptr;
    double* out = nullptr;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int result = 0;
    double ex = 0.0;
    long long n_pairs = 0;
    double e_block = 0.0;  // APPLY: sum_j <data_j| K_ACE |data_j> (set by the executor)
    int rebuild_due = 0;   // APPLY: the inner loop has converged on this projector (see Scheduler)
    std::string err;       // what failed (empty when result == 0)
};

// The rebuild cadence of the paper's double loop (Sec. 2): the ACE projector
// built in an outer iteration serves the inner iterations until they have
// converged, then the outer loop rebuilds it.  The inner loop is seen through
// the APPLY requests of a system: consecutive applications of one projector
// to the evolving block of functions; once the block's ACE energy changes by
// at most tol (relative) from one application to the next, the inner loop has
// converged and a rebuild is due.  The first application after a rebuild
// has nothing to compare with.
struct RebuildCadence {
    double tol = 0.0;  // 0: never report a rebuild as due
    bool have_prev = false;
    int prev_n = 0;
    double prev_e = 0.0;

    void rebuilt() { have_prev = false; }
    // after a successful APPLY of n functions with block energy e
    int applied(int n, double e) {
        int due = 0;
        if (tol > 0.0 && have_prev && prev_n == n) {
            const double scale = std::max(std::abs(e), 1e-300);
            due = std::abs(e - prev_e) <= tol * scale ? 1 : 0;
        }
        have_prev = true;
        prev_n = n;
        prev_e = e;
        return due;
    }
};

template <class Exec>
class Scheduler {
  public:
    // slots worker threads run requests; at most rebuild_slots of them run a
    // REBUILD at once, so short APPLY requests find a free slot while long
    // rebuilds run.
    Scheduler(Exec& exec, int slots, int rebuild_slots, size_t budget)
        : exec_(exec), budget_(budget), rebuild_slots_(std::max(1, std::min(rebuild_slots, slots))) {
        for (int k = 0; k < slots; ++k) workers_.emplace_back([this] { work(); });
    }

    ~Scheduler() {
        {
            std::unique_lock<std::mutex> lk(mu_);
            idle_cv_.wait(lk, [&] { return pending_.empty() && running_ == 0; });
            stop_ = true;
        }
        work_cv_.notify_all();
        for (auto& t : workers_) t.join();
        for (auto& s : systems_)
            if (s && s->alive) exec_.release(s->h);
    }

    int add_system(const SystemDesc& d) {
        std::lock_guard<std::mutex> lk(mu_);
        systems_.emplace_back(new Sys{d});
        return (int)systems_.size() - 1;
    }

    const SystemDesc* desc(int sys) {
        std::lock_guard<std::mutex> lk(mu_);
        return valid(sys) ? &systems_[sys]->d : nullptr;
    }

    // Queue a request; the caller validated its sizes against desc().
    int submit(int sys, int kind, const double* data, int n, double* out, long long* id_out) {
        std::lock_guard<std::mutex> lk(mu_);
        if (!valid(sys) || systems_[sys]->removing) return S_ERR_ARG;
        auto r = std::make_shared<Request>();
        r->id = next_id_++;
        r->sys = sys;
        r->kind = kind;
        r->data = data;
        r->n = n;
        r->out = out;
        r->t_submit = Clock::now();
        reqs_[r->id] = r;
        pending_.push_back(r);
        systems_[sys]->queued++;
        *id_out = r->id;
        work_cv_.notify_one();
        return S_OK;
    }

    int poll(long long id, bool wait, int* done, int* result, double* lat_ms, double* ex, long long* n_pairs) {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = reqs_.find(id);
        if (it == reqs_.end()) return S_ERR_ARG;
        std::shared_ptr<Request> r = it->second;
        if (wait) done_cv_.wait(lk, [&] { return r->done; });
        if (done) *done = r->done ? 1 : 0;
        if (r->done) {
            if (result) *result = r->result;
            if (lat_ms) *lat_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
            if (ex) *ex = r->ex;
            if (n_pairs) *n_pairs = r->n_pairs;
        }
        return S_OK;
    }

    // APPLY results of a completed request: block energy and whether a
    // rebuild is due.
    int apply_info(long long id, double* e_block, int* rebuild_due) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = reqs_.find(id);
        if (it == reqs_.end() || !it->second->done) return S_ERR_ARG;
        if (e_block) *e_block = it->second->e_block;
        if (rebuild_due) *rebuild_due = it->second->rebuild_due;
        return S_OK;
    }

    // Largest group of REBUILDs admitted together (see pick); 1: none.
    void set_rebuild_group(int max_group) {
        std::lock_guard<std::mutex> lk(mu_);
        group_max_ = std::max(1, std::min(max_group, kMaxGroup));
    }

    // Relative tolerance of a system's rebuild cadence (0: off).
    int set_rebuild_tolerance(int sys, double tol) {
        std::lock_guard<std::mutex> lk(mu_);
        if (!valid(sys) || !(tol >= 0.0)) return S_ERR_ARG;
        systems_[sys]->cadence.tol = tol;
        return S_OK;
    }

    // The failure message of a completed request ("" if none); the storage
    // lives as long as the scheduler.
    const char* error(long long id) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = reqs_.find(id);
        if (it == reqs_.end() || !it->second->done) return nullptr;
        return it->second->err.c_str();
    }

    int remove_system(int sys) {
        std::unique_lock<std::mutex> lk(mu_);
        if (!valid(sys) || systems_[sys]->removing) return S_ERR_ARG;
        Sys& s = *systems_[sys];
        s.removing = true;
        done_cv_.wait(lk, [&] { return s.queued == 0 && !s.busy; });
        exec_.release(s.h);
        s.held = 0;
        s.alive = false;
        work_cv_.notify_all();
        return S_OK;
    }

    // REBUILD groups admitted so far (more than one request) and their requests.
    void group_stats(long long* groups, long long* requests) {
        std::lock_guard<std::mutex> lk(mu_);
        if (groups) *groups = groups_;
        if (requests) *requests = grouped_;
    }

    void stats(size_t* held, int* running, int* queued) {
        std::lock_guard<std::mutex> lk(mu_);
        size_t h = 0;
        for (auto& s : systems_) h += s->held;
        if (held) *held = h;
        if (running) *running = running_;
        if (queued) *queued = (int)pending_.size();
    }

  private:
    struct Sys {
        SystemDesc d;
        typename Exec::Handle h{};
        size_t held = 0;     // bytes the system holds (updated after each request)
        size_t growth = 0;   // predicted growth of the running request
        int queued = 0;      // requests submitted and not yet completed
        bool busy = false, removing = false, alive = true;
        RebuildCadence cadence;
    };

    bool valid(int sys) const { return sys >= 0 && sys < (int)systems_.size() && systems_[sys]->alive; }

    static constexpr int kMaxGroup = 8;

    struct Pick {
        std::shared_ptr<Request> r;
        size_t growth;
    };

    size_t committed() const {
        size_t b = 0;
        for (auto& s : systems_) b += s->held + (s->busy ? s->growth : 0);
        return b;
    }

    // Under mu_: the earliest pending request whose system is idle, that is
    // its system's oldest pending request, whose growth fits the budget and,
    // for a REBUILD, for which a rebuild slot is free.  A request that cannot
    // fit even with nothing running completes with S_ERR_OOM (growth -1).
    // A REBUILD whose system has a merge key takes with it, as one group in
    // one rebuild slot, up to group_max_ - 1 REBUILDs of other idle systems
    // with the same key that are their systems' oldest pending requests and
    // fit the budget beside it: the group runs at once, so its members reach
    // their pair convolutions together and the executor can merge their
    // launches.  Companions go ahead of requests queued before them.
    std::vector<Pick> pick() {
        std::vector<char> seen(systems_.size(), 0);
        const size_t used = committed();
        for (auto it = pending_.begin(); it != pending_.end(); ++it) {
            auto r = *it;
            Sys& s = *systems_[r->sys];
            if (seen[r->sys]) continue;
            seen[r->sys] = 1;
            if (s.busy) continue;
            if (r->kind == REQ_REBUILD && rebuilds_running_ >= rebuild_slots_) continue;
            const size_t after = exec_.predict(s.d, s.h, r->kind, r->n);
            const size_t growth = after > s.held ? after - s.held : 0;
            if (used + growth <= budget_) {
                std::vector<Pick> group{{r, growth}};
                pending_.erase(it);
                const int key = r->kind == REQ_REBUILD && group_max_ > 1 ? exec_.merge_key(s.d) : 0;
                if (key) add_companions(r->sys, key, used + growth, group);
                return group;
            }
            // nothing else can release memory: this request never fits
            if (running_ == 0 && used - s.held + after > budget_) {
                pending_.erase(it);
                return {{r, (size_t)-1}};
            }
        }
        return {};
    }

    void add_companions(int first_sys, int key, size_t used, std::vector<Pick>& group) {
        std::vector<char> seen(systems_.size(), 0);
        seen[first_sys] = 1;
        for (auto it = pending_.begin(); it != pending_.end() && (int)group.size() < group_max_;) {
            auto r = *it;
            Sys& s = *systems_[r->sys];
            if (seen[r->sys]) {
                ++it;
                continue;
            }
            seen[r->sys] = 1;  // only a system's oldest pending request may run
            if (s.busy || r->kind != REQ_REBUILD || exec_.merge_key(s.d) != key) {
                ++it;
                continue;
            }
            const size_t after = exec_.predict(s.d, s.h, r->kind, r->n);
            const size_t growth = after > s.held ? after - s.held : 0;
            if (used + growth > budget_) {
                ++it;
                continue;
            }
            used += growth;
            group.push_back({r, growth});
            it = pending_.erase(it);
        }
    }

    void work() {
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            std::vector<Pick> group;
            work_cv_.wait(lk, [&] { return stop_ || !(group = pick()).empty(); });
            if (group.empty()) return;  // stop_ with nothing runnable
            if (group[0].growth == (size_t)-1) {
                Request& r = *group[0].r;
                r.err = "the request does not fit the device-memory budget beside the resident systems";
                finish(*systems_[r.sys], r, S_ERR_OOM);
                continue;
            }
            const bool rebuild = group[0].r->kind == REQ_REBUILD;
            std::vector<Sys*> sys;  // taken under mu_ (add_system may grow systems_)
            for (auto& g : group) {
                Sys* s = systems_[g.r->sys].get();
                s->busy = true;
                s->growth = g.growth;
                sys.push_back(s);
            }
            running_ += (int)group.size();
            rebuilds_running_ += rebuild;  // a group takes one rebuild slot
            if (group.size() > 1) groups_++, grouped_ += (long long)group.size();
            lk.unlock();
            // the companions on threads of their own, the first request here
            std::vector<int> st(group.size(), S_OK);
            std::vector<size_t> held(group.size(), 0);
            auto run_one = [&](size_t k) {
                st[k] = exec_.run(sys[k]->d, sys[k]->h, *group[k].r);
                held[k] = exec_.held(sys[k]->h);
            };
            std::vector<std::thread> helpers;
            for (size_t k = 1; k < group.size(); ++k) {
                try {
                    helpers.emplace_back(run_one, k);
                } catch (...) {
                    run_one(k);  // no thread to be had: one after the other (the merge is then skipped)
                }
            }
            run_one(0);
            for (auto& t : helpers) t.join();
            lk.lock();
            for (size_t k = 0; k < group.size(); ++k) {
                Request& r = *group[k].r;
                Sys& s = *sys[k];
                s.held = held[k];
                s.busy = false;
                s.growth = 0;
                if (st[k] == S_OK) {
                    if (rebuild) s.cadence.rebuilt();
                    else r.rebuild_due = s.cadence.applied(r.n, r.e_block);
                }
            }
            running_ -= (int)group.size();
            rebuilds_running_ -= rebuild;
            for (size_t k = 0; k < group.size(); ++k) finish(*sys[k], *group[k].r, st[k]);
            work_cv_.notify_all();  // memory and the systems are free again
        }
    }

    void finish(Sys& s, Request& r, int st) {
        r.result = st;
        r.t_done = Clock::now();
        r.done = true;
        s.queued--;
        done_cv_.notify_all();
        if (pending_.empty() && running_ == 0) idle_cv_.notify_all();
    }

    Exec& exec_;
    const size_t budget_;
    std::mutex mu_;
    std::condition_variable work_cv_, done_cv_, idle_cv_;
    std::vector<std::unique_ptr<Sys>> systems_;
    std::deque<std::shared_ptr<Request>> pending_;
    std::map<long long, std::shared_ptr<Request>> reqs_;
    std::vector<std::thread> workers_;
    const int rebuild_slots_;
    long long next_id_ = 1;
    int running_ = 0, rebuilds_running_ = 0;
    bool stop_ = false;
    int group_max_ = 4;
    long long groups_ = 0, grouped_ = 0;
};

}  // namespace lace_serve
