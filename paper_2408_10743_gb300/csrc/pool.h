// pool.h -- the host threads the batch engine plans and post-processes
// slices on: a process-wide pool created on first use, one worker per
// hardware thread beyond the caller's (at most 15).  A parallel region hands
// out ranges of `grain` items from an atomic counter, so that uneven items
// (codes of different sizes) spread evenly; the caller works too.  Waking a
// sleeping thread takes from a few to tens of microseconds, so workers spin
// for kIdleSpin after each region before they sleep (the slices of a batch
// follow one another).  One region runs at a time; a caller that finds one
// running, or that runs in a child process made by fork() (which has none of
// the workers), does its items itself.
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include <unistd.h>

namespace dist {

class HostPool {
   public:
    static HostPool& get() {
        static HostPool* p = new HostPool();  // never destroyed: its threads run until exit
        return *p;
    }

    // fn(a, b) over [0, n), every item in exactly one call.
    template <class F>
    void run(size_t n, size_t grain, const F& fn) {
        grain = std::max<size_t>(1, grain);
        if (getpid() != owner_ || workers_.empty() || n <= grain) {
            fn((size_t)0, n);
            return;
        }
        std::unique_lock<std::mutex> region(region_mu_, std::try_to_lock);
        if (!region.owns_lock()) {
            fn((size_t)0, n);
            return;
        }
        const std::function<void(size_t, size_t)> job = fn;
        job_ = &job;
        n_ = n;
        grain_ = grain;
        next_.store(0, std::memory_order_relaxed);
        pending_.store((int)workers_.size(), std::memory_order_relaxed);
        {
            std::lock_guard<std::mutex> lk(mu_);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        work();
        // every worker takes part in every region, so none can still be
        // reading this region's job once pending_ is 0
        if (!spin_until([this] { return pending_.load(std::memory_order_acquire) == 0; }, kIdleSpin)) {
            std::unique_lock<std::mutex> lk(mu_);
            done_.wait(lk, [this] { return pending_.load(std::memory_order_acquire) == 0; });
        }
        job_ = nullptr;
    }

    size_t threads() const { return workers_.size() + 1; }

   private:
    static constexpr double kIdleSpin = 2e-3;  // seconds
    template <class Pred>
    static bool spin_until(Pred pred, double seconds) {
        const auto t0 = std::chrono::steady_clock::now();
        for (unsigned it = 0;; it++) {
            if (pred()) return true;
            if ((it & 255u) == 255u &&
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > seconds)
                return false;
        }
    }
    HostPool() : owner_(getpid()) {
        const unsigned hw = std::thread::hardware_concurrency();
        const unsigned nw = hw > 1 ? std::min(hw - 1, 15u) : 0u;
        for (unsigned t = 0; t < nw; t++) workers_.emplace_back([this] { loop(); });
        for (std::thread& th : workers_) th.detach();
    }
    void work() {
        for (;;) {
            const size_t a = next_.fetch_add(grain_, std::memory_order_relaxed);
            if (a >= n_) break;
            (*job_)(a, std::min(n_, a + grain_));
        }
    }
    void loop() {
        unsigned long long seen = 0;
        for (;;) {
            if (!spin_until([&] { return gen_.load(std::memory_order_acquire) != seen; }, kIdleSpin)) {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
            }
            seen = gen_.load(std::memory_order_acquire);
            work();
            if (pending_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
                std::lock_guard<std::mutex> lk(mu_);
                done_.notify_all();
            }
        }
    }

    std::vector<std::thread> workers_;
    std::mutex region_mu_, mu_;
    std::condition_variable cv_, done_;
    std::atomic<unsigned long long> gen_{0};
    std::atomic<size_t> next_{0};
    std::atomic<int> pending_{0};
    const std::function<void(size_t, size_t)>* job_ = nullptr;
    size_t n_ = 0, grain_ = 1;
    const pid_t owner_;
};

}  // namespace dist
