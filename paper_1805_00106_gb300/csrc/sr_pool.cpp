// sr_pool.cpp -- a fork-join pool of host threads for the library's parallel
// host stages (batch validation, index building, SAM formatting).  Creating
// threads per call costs tens of microseconds each; the pool keeps them.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "sr_host.h"

namespace sr {
namespace {

class Pool {
 public:
  explicit Pool(unsigned workers) : pid_(getpid()) {
    for (unsigned i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  unsigned size() const { return static_cast<unsigned>(th_.size()) + 1; }
  bool usable() const { return getpid() == pid_; }  // a forked child has no workers

  // fn(0) .. fn(n - 1) on the workers and the caller; returns when all are done
  void run(uint32_t n, const std::function<void(uint32_t)>& fn) {
    std::lock_guard<std::mutex> one(run_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &fn;
      n_ = n;
      next_.store(0);
      finished_ = 0;
      ++gen_;
    }
    cv_.notify_all();
    work(fn, n);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return finished_ == th_.size(); });
    job_ = nullptr;
  }

 private:
  void work(const std::function<void(uint32_t)>& fn, uint32_t n) {
    for (uint32_t t; (t = next_.fetch_add(1)) < n;) fn(t);
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(uint32_t)>* f;
      uint32_t n;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        f = job_;
        n = n_;
      }
      work(*f, n);
      {
        std::lock_guard<std::mutex> lk(mu_);
        ++finished_;
      }
      done_.notify_all();
    }
  }
  const pid_t pid_;
  std::vector<std::thread> th_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_;
  const std::function<void(uint32_t)>* job_ = nullptr;
  uint32_t n_ = 0;
  std::atomic<uint32_t> next_{0};
  size_t finished_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

Pool& pool() {
  static Pool p(std::max(1u, std::min(16u, std::thread::hardware_concurrency())) - 1u);
  return p;
}

}  // namespace

unsigned host_threads() { return pool().size(); }

void parallel_for(uint32_t n, const std::function<void(uint32_t)>& fn) {
  if (n <= 1 || !pool().usable()) {
    for (uint32_t t = 0; t < n; ++t) fn(t);
    return;
  }
  pool().run(n, fn);
}

}  // namespace sr
