// Request scheduler of the serving loop: host C++ only (no CUDA), so that its
// queueing, admission and accounting logic is tested on its own.
//
// Requests carry a key (the catalog basis they run on) and an estimated device
// working set in bytes.  Every key has one queue and one worker thread (the executor
// of a key is not re-entrant: one library context per basis), so work of different
// keys runs concurrently.  When a worker takes the head of its queue it also takes
// every later queued request that can share the head's batch (the merge predicate)
// and fits, up to max_merge requests: they run as ONE batched execution (continuous
// batching -- requests that arrived while the previous batch was on the device join
// the next one as soon as it starts).  A batch starts only while the working sets of
// the running batches plus its own stay within the byte budget (admission control);
// a request larger than the whole budget is refused at submission.  Requests that
// cannot merge keep their arrival order.  Latency is measured from submission to
// completion.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace pwqt {

template <class Req>
class Scheduler {
public:
    using Clock = std::chrono::steady_clock;
    // exec(key, batch, rcs) runs a batch of requests on the key's worker thread and sets
    // one status code per request
    using Exec = std::function<void(int, std::vector<Req*>&, std::vector<int>&)>;
    // merge(head, other): may `other` run in the same batch as `head`
    using Merge = std::function<bool(const Req&, const Req&)>;

    enum : int { OK = 0, ERR_ARG = -1, ERR_STATE = -5, ERR_BUSY = -8, WAIT_TIMEOUT = 1 };

    Scheduler(size_t budget_bytes, size_t queue_capacity, Exec exec, Merge merge = nullptr, size_t max_merge = 1)
        : budget_(budget_bytes), capacity_(queue_capacity), exec_(std::move(exec)), merge_(std::move(merge)),
          max_merge_(std::max<size_t>(1, max_merge)) {}

    ~Scheduler() { shutdown(); }

    // a new key gets its queue and worker; adding a key twice is an error
    int add_key(int key) {
        std::lock_guard<std::mutex> g(m_);
        if (stopping_ || lanes_.count(key)) return ERR_STATE;
        auto lane = std::make_unique<Lane>();
        Lane* L = lane.get();
        lanes_[key] = std::move(lane);
        L->worker = std::thread([this, key, L] { run(key, L); });
        return OK;
    }

    // queue a request; ticket receives its id
    int submit(int key, Req r, size_t bytes, long long* ticket) {
        std::lock_guard<std::mutex> g(m_);
        if (stopping_) return ERR_STATE;
        auto it = lanes_.find(key);
        if (it == lanes_.end()) return ERR_ARG;
        if (bytes > budget_) return ERR_ARG;
        if (queued_ >= capacity_) return ERR_BUSY;
        const long long id = ++next_id_;
        Job& j = jobs_[id];
        j.req = std::move(r);
        j.bytes = bytes;
        j.submitted = Clock::now();
        it->second->queue.push_back(id);
        ++queued_;
        if (ticket) *ticket = id;
        cv_work_.notify_all();
        return OK;
    }

    // wait for a request; rc receives the executor's status, latency its seconds.
    // Returns OK, WAIT_TIMEOUT (still running; ask again) or ERR_ARG (unknown or
    // already collected ticket).  A collected ticket is forgotten.
    int wait(long long ticket, double timeout_s, int* rc, double* latency_s) {
        std::unique_lock<std::mutex> g(m_);
        auto it = jobs_.find(ticket);
        if (it == jobs_.end()) return ERR_ARG;
        auto done = [&] { auto k = jobs_.find(ticket); return k == jobs_.end() || k->second.done; };
        if (timeout_s < 0) cv_done_.wait(g, done);
        else if (!cv_done_.wait_for(g, std::chrono::duration<double>(timeout_s), done)) return WAIT_TIMEOUT;
        it = jobs_.find(ticket);
        if (it == jobs_.end()) return ERR_ARG;
        if (rc) *rc = it->second.rc;
        if (latency_s) *latency_s = it->second.latency;
        jobs_.erase(it);
        return OK;
    }

    // completed requests, latency percentiles (nearest rank) over them, peak admitted bytes
    void stats(long long* completed, double* p50, double* p99, size_t* peak_bytes) {
        std::lock_guard<std::mutex> g(m_);
        std::vector<double> l = latencies_;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            if (l.empty()) return 0.0;
            size_t k = (size_t)std::max(0.0, std::ceil(q * l.size()) - 1.0);
            return l[std::min(k, l.size() - 1)];
        };
        if (completed) *completed = (long long)l.size();
        if (p50) *p50 = pct(0.50);
        if (p99) *p99 = pct(0.99);
        if (peak_bytes) *peak_bytes = peak_;
    }

    // batches executed and the requests they held (requests / batches = mean batch size)
    void batch_stats(long long* batches, long long* requests, long long* largest) {
        std::lock_guard<std::mutex> g(m_);
        if (batches) *batches = batches_;
        if (requests) *requests = batched_;
        if (largest) *largest = largest_;
    }

    void reset_stats() {
        std::lock_guard<std::mutex> g(m_);
        latencies_.clear();
        peak_ = in_use_;
        batches_ = batched_ = largest_ = 0;
    }

    // finish the queued work, then stop the workers
    void shutdown() {
        {
            std::lock_guard<std::mutex> g(m_);
            if (stopping_) return;
            stopping_ = true;
            cv_work_.notify_all();
        }
        for (auto& kv : lanes_)
            if (kv.second->worker.joinable()) kv.second->worker.join();
    }

private:
    struct Job {
        Req req{};
        size_t bytes = 0;
        Clock::time_point submitted;
        bool done = false;
        int rc = 0;
        double latency = 0;
    };
    struct Lane {
        std::deque<long long> queue;
        std::thread worker;
    };

    void run(int key, Lane* L) {
        std::unique_lock<std::mutex> g(m_);
        for (;;) {
            // the head of this key's queue starts when its bytes fit beside the running work
            cv_work_.wait(g, [&] {
                if (L->queue.empty()) return stopping_;
                return in_use_ + jobs_[L->queue.front()].bytes <= budget_;
            });
            if (L->queue.empty()) return;   // stopping and drained
            std::vector<long long> ids{L->queue.front()};
            L->queue.pop_front();
            size_t bytes = jobs_[ids[0]].bytes;
            // later requests that can share the head's batch and still fit join it
            if (merge_)
                for (auto it = L->queue.begin(); it != L->queue.end() && ids.size() < max_merge_;) {
                    const Job& j = jobs_[*it];
                    if (merge_(jobs_[ids[0]].req, j.req) && in_use_ + bytes + j.bytes <= budget_) {
                        ids.push_back(*it);
                        bytes += j.bytes;
                        it = L->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            queued_ -= ids.size();
            in_use_ += bytes;
            peak_ = std::max(peak_, in_use_);
            ++batches_;
            batched_ += (long long)ids.size();
            largest_ = std::max(largest_, (long long)ids.size());
            std::vector<Req> reqs;
            reqs.reserve(ids.size());
            for (long long id : ids) reqs.push_back(jobs_[id].req);
            g.unlock();
            std::vector<Req*> ptrs;
            for (auto& r : reqs) ptrs.push_back(&r);
            std::vector<int> rcs(ids.size(), 0);
            exec_(key, ptrs, rcs);
            g.lock();
            for (size_t q = 0; q < ids.size(); ++q) {
                Job& jd = jobs_[ids[q]];
                jd.rc = rcs[q];
                jd.done = true;
                jd.latency = std::chrono::duration<double>(Clock::now() - jd.submitted).count();
                latencies_.push_back(jd.latency);
            }
            in_use_ -= bytes;
            cv_done_.notify_all();
            cv_work_.notify_all();
        }
    }

    const size_t budget_, capacity_;
    Exec exec_;
    Merge merge_;
    const size_t max_merge_;
    long long batches_ = 0, batched_ = 0, largest_ = 0;
    std::mutex m_;
    std::condition_variable cv_work_, cv_done_;
    std::map<int, std::unique_ptr<Lane>> lanes_;
    std::map<long long, Job> jobs_;
    std::vector<double> latencies_;
    size_t in_use_ = 0, peak_ = 0, queued_ = 0;
    long long next_id_ = 0;
    bool stopping_ = false;
};

}  // namespace pwqt
