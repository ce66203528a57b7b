// Host worker pool of the library (plain C++, no CUDA): run(n, f) calls
// f(0) ... f(n - 1) across the pool's workers and the calling thread and returns
// when all have returned. One call runs at a time; a call made while another is
// running (from another host thread) runs its jobs on the caller alone, so that
// callers never wait on each other's jobs. The workers block on a condition
// variable between calls; the destructor stops and joins them.
#pragma once

#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace pb {

struct HostPool {
    std::vector<std::thread> workers;
    std::mutex run_mu;  // one parallel call at a time
    std::mutex mu;
    std::condition_variable cv, done_cv;
    const std::function<void(int)>* job = nullptr;
    int njobs = 0, next = 0, remaining = 0;
    uint64_t gen = 0;
    bool stop = false;

    explicit HostPool(int nworkers) {
        for (int w = 0; w < nworkers; ++w) workers.emplace_back([this] { loop(); });
    }
    // stops and joins the workers (no call may be running)
    ~HostPool() {
        {
            std::lock_guard<std::mutex> lk(mu);
            stop = true;
            ++gen;
        }
        cv.notify_all();
        for (auto& t : workers) t.join();
    }
    HostPool(const HostPool&) = delete;
    HostPool& operator=(const HostPool&) = delete;
    // take jobs of the current call until none is left (mu held on entry and exit)
    void drain(std::unique_lock<std::mutex>& lk) {
        while (job && next < njobs) {
            const int i = next++;
            const std::function<void(int)>* f = job;
            lk.unlock();
            (*f)(i);
            lk.lock();
            if (--remaining == 0) done_cv.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv.wait(lk, [&] { return gen != seen; });
            if (stop) return;
            seen = gen;
            drain(lk);
        }
    }
    void run(int n, const std::function<void(int)>& f) {
        std::unique_lock<std::mutex> busy(run_mu, std::try_to_lock);
        if (!busy.owns_lock() || workers.empty() || n <= 1) {
            for (int i = 0; i < n; ++i) f(i);
            return;
        }
        std::unique_lock<std::mutex> lk(mu);
        job = &f;
        njobs = n;
        next = 0;
        remaining = n;
        ++gen;
        cv.notify_all();
        drain(lk);
        done_cv.wait(lk, [&] { return remaining == 0; });
        job = nullptr;
    }
};

}  // namespace pb
