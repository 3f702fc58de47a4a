// A fixed pool of host worker threads running queued tasks in FIFO order
// (ring and server copies between pinned slots and pageable images).
#pragma once
#include <pthread.h>
#include <sched.h>

#include <condition_variable>
#include <cstdlib>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace snapk {

class Pool {
public:
    explicit Pool(int n)
    {
        // SNAP_PIN_WORKERS=1 pins worker i to host CPU i modulo the CPU count
        // (for measurements; by default the scheduler places them)
        const char *pin = std::getenv("SNAP_PIN_WORKERS");
        const int ncpu = (int)std::thread::hardware_concurrency();
        for (int i = 0; i < n; ++i) {
            th_.emplace_back([this] { run(); });
            if (pin && pin[0] == '1' && ncpu > 0) {
                cpu_set_t set;
                CPU_ZERO(&set);
                CPU_SET(i % ncpu, &set);
                pthread_setaffinity_np(th_.back().native_handle(), sizeof set, &set);
            }
        }
    }
    ~Pool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    void push(std::function<void()> f)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            q_.push_back(std::move(f));
        }
        cv_.notify_one();
    }
    int size() const { return (int)th_.size(); }

private:
    void run()
    {
        for (;;) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return stop_ || !q_.empty(); });
                if (q_.empty()) return;
                f = std::move(q_.front());
                q_.pop_front();
            }
            f();
        }
    }
    std::vector<std::thread> th_;
    std::deque<std::function<void()>> q_;
    std::mutex mu_;
    std::condition_variable cv_;
    bool stop_ = false;
};

}  // namespace snapk
