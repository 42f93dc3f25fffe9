// Host-only checks of the serving scheduler (paper_1903_00548_gb300/csrc/scheduler.h)
// with a fake executor: per-key order, concurrency across keys, admission by the
// byte budget, refusal of oversized requests, latency accounting, draining, and
// continuous batching (requests queued behind a running batch merge into the next
// one when the predicate allows and the budget holds).
#include <atomic>
#include <chrono>
#include <cstdio>
#include <mutex>
#include <thread>
#include <vector>

#include "scheduler.h"

struct Req {
    int seq = 0;
    int sleep_ms = 0;
    size_t bytes = 0;
    int cls = 0;          // requests of one class may share a batch
};

#define CHECK(c)                                                       \
    do {                                                               \
        if (!(c)) {                                                    \
            std::fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
            return 1;                                                  \
        }                                                              \
    } while (0)

int main() {
    using S = pwqt::Scheduler<Req>;
    std::mutex mu;
    std::vector<std::vector<int>> order(3);
    std::atomic<long long> in_use{0}, peak{0};
    std::atomic<int> running{0}, max_running{0};
    {
        auto one = [&](int key, Req& r) {
            long long u = in_use += (long long)r.bytes;
            long long p = peak.load();
            while (u > p && !peak.compare_exchange_weak(p, u)) {}
            int k = ++running;
            int mr = max_running.load();
            while (k > mr && !max_running.compare_exchange_weak(mr, k)) {}
            std::this_thread::sleep_for(std::chrono::milliseconds(r.sleep_ms));
            {
                std::lock_guard<std::mutex> g(mu);
                order[key].push_back(r.seq);
            }
            --running;
            in_use -= (long long)r.bytes;
            return r.seq == 7 ? -3 : 0;   // one request reports a failure code
        };
        S sched(100, 1000, [&](int key, std::vector<Req*>& b, std::vector<int>& rcs) {
            for (size_t q = 0; q < b.size(); ++q) rcs[q] = one(key, *b[q]);
        });
        CHECK(sched.add_key(0) == S::OK);
        CHECK(sched.add_key(1) == S::OK);
        CHECK(sched.add_key(2) == S::OK);
        CHECK(sched.add_key(1) == S::ERR_STATE);
        long long t;
        CHECK(sched.submit(5, Req{}, 1, &t) == S::ERR_ARG);        // unknown key
        CHECK(sched.submit(0, Req{}, 101, &t) == S::ERR_ARG);      // larger than the budget
        std::vector<long long> tickets;
        for (int q = 0; q < 12; ++q) {
            const int key = q % 3;
            Req r{q, 20, (size_t)(key == 2 ? 60 : 30)};
            CHECK(sched.submit(key, r, r.bytes, &t) == S::OK);
            tickets.push_back(t);
        }
        int failed = 0;
        for (long long tk : tickets) {
            int rc = 0;
            double lat = 0;
            CHECK(sched.wait(tk, -1.0, &rc, &lat) == S::OK);
            CHECK(lat > 0.015);
            if (rc != 0) ++failed;
        }
        CHECK(failed == 1);
        CHECK(sched.wait(tickets[0], 0.0, nullptr, nullptr) == S::ERR_ARG);   // collected already
        long long done = 0;
        double p50 = 0, p99 = 0;
        size_t pk = 0;
        sched.stats(&done, &p50, &p99, &pk);
        CHECK(done == 12);
        CHECK(p50 > 0.015 && p99 >= p50);
        CHECK(pk <= 100);
        // a long request, then a timed wait that returns before it finishes
        CHECK(sched.submit(0, Req{100, 200, 10}, 10, &t) == S::OK);
        int rc = 0;
        CHECK(sched.wait(t, 0.01, &rc, nullptr) == S::WAIT_TIMEOUT);
        CHECK(sched.wait(t, -1.0, &rc, nullptr) == S::OK);
        // queued work is finished by shutdown (destructor)
        for (int q = 0; q < 4; ++q) CHECK(sched.submit(1, Req{200 + q, 5, 10}, 10, &t) == S::OK);
    }
    // per key, requests ran in submission order
    for (int k = 0; k < 3; ++k)
        for (size_t q = 1; q < order[k].size(); ++q) CHECK(order[k][q] > order[k][q - 1]);
    CHECK(order[1].size() == 4 + 4);   // 4 from the first wave, 4 drained at shutdown
    // keys ran concurrently, and the admitted bytes never exceeded the budget
    CHECK(max_running.load() >= 2);
    CHECK(peak.load() <= 100);
    // ---- continuous batching: a slow request holds key 0; meanwhile six requests of two
    // classes queue behind it.  The next batch takes the head (class 1) and the other
    // class-1 requests that fit (budget 100, 30 bytes each: three in all), in arrival
    // order; the class-2 requests keep their order and batch after it.
    std::vector<std::vector<int>> batches;
    {
        S sched(100, 1000,
                [&](int, std::vector<Req*>& b, std::vector<int>& rcs) {
                    std::vector<int> seqs;
                    for (auto* r : b) seqs.push_back(r->seq);
                    std::this_thread::sleep_for(std::chrono::milliseconds(b[0]->sleep_ms));
                    {
                        std::lock_guard<std::mutex> g(mu);
                        batches.push_back(seqs);
                    }
                    for (size_t q = 0; q < b.size(); ++q) rcs[q] = b[q]->seq;   // echo
                },
                [](const Req& a, const Req& b) { return a.cls == b.cls; }, 8);
        CHECK(sched.add_key(0) == S::OK);
        long long t;
        std::vector<long long> tk;
        CHECK(sched.submit(0, Req{0, 150, 10, 0}, 10, &t) == S::OK);
        tk.push_back(t);
        std::this_thread::sleep_for(std::chrono::milliseconds(40));    // the slow one is running
        const int cls[6] = {1, 2, 1, 1, 2, 1};
        for (int q = 1; q <= 6; ++q) {
            CHECK(sched.submit(0, Req{q, 10, 30, cls[q - 1]}, 30, &t) == S::OK);
            tk.push_back(t);
        }
        for (size_t q = 0; q < tk.size(); ++q) {
            int rc = -1;
            CHECK(sched.wait(tk[q], -1.0, &rc, nullptr) == S::OK);
            CHECK(rc == (int)q);                       // every request got its own result
        }
        long long nb = 0, nreq = 0, largest = 0;
        sched.batch_stats(&nb, &nreq, &largest);
        CHECK(nreq == 7 && largest == 3);
    }
    // [0] alone; then class 1 {1, 3, 4} (budget: 3 x 30 with the 10 of [0] gone), class 2
    // {2, 5}, and class 1 {6}
    CHECK(batches.size() == 4);
    CHECK(batches[0] == std::vector<int>({0}));
    CHECK(batches[1] == std::vector<int>({1, 3, 4}));
    CHECK(batches[2] == std::vector<int>({2, 5}));
    CHECK(batches[3] == std::vector<int>({6}));
    std::printf("scheduler host checks passed (max concurrent %d, peak bytes %lld, batches %zu)\n", max_running.load(),
                peak.load(), batches.size());
    return 0;
}
