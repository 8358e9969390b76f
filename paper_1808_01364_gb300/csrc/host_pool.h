// A small pool of host threads for the level planner: parallel_for(n, fn)
// runs fn(i) for i in [0, n) on the workers and the calling thread and
// returns when all are done.  The planner issues its parallel loops back to
// back, so a worker that finishes one keeps polling for the next for a short
// while (kSpin) before it sleeps on a condition variable; the caller likewise
// polls for the workers' completion before it sleeps.  The pool is created on
// first use; a child created by fork() gets a fresh pool (the parent's
// workers do not exist there).
#pragma once
#include <pthread.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

namespace rhif {

class HostPool {
 public:
  static HostPool& get() {
    static std::mutex mu;
    static HostPool* pool = nullptr;
    static pid_t owner = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!pool || owner != getpid()) {   // first use, or a forked child: (re)create
      pool = new HostPool();            // a parent's pool object is left as is in the child
      owner = getpid();
    }
    return *pool;
  }

  int threads() const { return (int)workers_.size() + 1; }

  // fn(i) for every i in [0, n); chunks of `grain` indices are handed out in order.
  void parallel_for(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn) {
    if (n <= 0) return;
    grain = std::max<int64_t>(grain, 1);
    if (workers_.empty() || n <= grain) {
      fn(0, n);
      return;
    }
    // one parallel_for at a time: a caller that finds the pool busy (another
    // host thread planning another problem) runs its loop itself
    std::unique_lock<std::mutex> call(call_mu_, std::try_to_lock);
    if (!call.owns_lock()) {
      fn(0, n);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      n_ = n;
      grain_ = grain;
      next_.store(0);
      active_.store((int)workers_.size());
      gen_.fetch_add(1, std::memory_order_release);   // publishes the fields above
    }
    cv_.notify_all();
    work();
    if (!poll([&] { return active_.load(std::memory_order_acquire) == 0; })) {
      std::unique_lock<std::mutex> lk(mu_);
      done_cv_.wait(lk, [&] { return active_.load(std::memory_order_acquire) == 0; });
    }
    fn_ = nullptr;
  }

 private:
  HostPool() {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nw = (int)std::min<unsigned>(hw > 1 ? hw / 2 : 0, 7);
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
    for (auto& t : workers_) t.detach();
  }

  void work() {
    for (;;) {
      const int64_t b = next_.fetch_add(grain_);
      if (b >= n_) break;
      (*fn_)(b, std::min(n_, b + grain_));
    }
  }

  // Polls `ready` for about kSpin; false if it did not become true.
  template <typename Pred>
  static bool poll(Pred ready) {
    constexpr auto kSpin = std::chrono::microseconds(200);
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0;; ++i) {
      if (ready()) return true;
      if ((i & 255) == 255 && std::chrono::steady_clock::now() - t0 > kSpin) return false;
    }
  }

  void loop() {
    uint64_t seen = 0;
    for (;;) {
      auto fresh = [&] { return gen_.load(std::memory_order_acquire) != seen; };
      if (!poll(fresh)) {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, fresh);
      }
      seen = gen_.load(std::memory_order_acquire);
      work();
      if (active_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        std::lock_guard<std::mutex> lk(mu_);   // the caller may be about to wait
        done_cv_.notify_one();
      }
    }
  }

  std::vector<std::thread> workers_;
  std::mutex mu_, call_mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int64_t, int64_t)>* fn_ = nullptr;
  int64_t n_ = 0, grain_ = 1;
  std::atomic<int64_t> next_{0};
  std::atomic<int> active_{0};
  std::atomic<uint64_t> gen_{0};
};

}  // namespace rhif
