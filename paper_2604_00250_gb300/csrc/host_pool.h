// Host worker threads for the plan's parallel passes (plain C++, no CUDA).
#pragma once

#include <pthread.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <system_error>
#include <thread>
#include <vector>

namespace prism {

// A fixed set of worker threads, started on first use and kept for the life of the process:
// starting threads anew for every pass of the plan costs more than the passes themselves on
// the small volumes of a slab batch (the plan calls four passes per volume). One job runs at a
// time. A caller that finds the pool busy (another thread building another plan), or that runs
// in a child forked after the pool started (its workers do not exist there), gets `false` from
// run() and runs the job itself.
class HostPool {
 public:
  using Fn = std::function<void(int64_t, int64_t)>;

  // The process's pool, or nullptr where no worker could be started or after a fork.
  static HostPool* get() {
    static std::once_flag once;
    static HostPool* pool = nullptr;
    std::call_once(once, [] {
      pthread_atfork(nullptr, nullptr, &HostPool::forked_child);
      unsigned hc = std::thread::hardware_concurrency();
      const int want = static_cast<int>(std::min<unsigned>(hc ? hc : 1, 16)) - 1;
      if (want < 1) return;
      auto* p = new HostPool();   // kept until the process exits (workers never stop)
      for (int i = 0; i < want; ++i) {
        try {
          std::thread([p] { p->worker(); }).detach();
          ++p->nworkers_;
        } catch (const std::system_error&) {
          break;
        }
      }
      if (p->nworkers_ > 0) pool = p;
    });
    return in_forked_child().load() ? nullptr : pool;
  }

  // Threads a job can use: the workers and the caller.
  int threads() const { return nworkers_ + 1; }

  // Runs fn(n * i / nt, n * (i + 1) / nt) for i in [0, nt) on the workers and the calling
  // thread; returns after every chunk has run. false (nothing run) when the pool is busy.
  bool run(int64_t n, int nt, const Fn& fn) {
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_.store(&fn, std::memory_order_relaxed);
      n_.store(n, std::memory_order_relaxed);
      nt_.store(nt, std::memory_order_relaxed);
      left_.store(nt, std::memory_order_relaxed);
      next_.store(0, std::memory_order_release);
      ++seq_;
    }
    cv_.notify_all();
    drain();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return left_.load(std::memory_order_acquire) == 0; });
    return true;
  }

 private:
  HostPool() = default;

  static std::atomic<bool>& in_forked_child() {
    static std::atomic<bool> f{false};
    return f;
  }
  static void forked_child() { in_forked_child().store(true); }

  // Takes chunks of the current job until none is left.
  void drain() {
    for (;;) {
      const int i = next_.fetch_add(1, std::memory_order_acq_rel);
      const int nt = nt_.load(std::memory_order_relaxed);
      if (i >= nt) break;
      const int64_t n = n_.load(std::memory_order_relaxed);
      (*fn_.load(std::memory_order_relaxed))(n * i / nt, n * (i + 1) / nt);
      if (left_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        std::lock_guard<std::mutex> lk(mu_);
        done_cv_.notify_all();
      }
    }
  }

  void worker() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return seq_ != seen; });
        seen = seq_;
      }
      drain();
    }
  }

  int nworkers_ = 0;
  std::mutex busy_;                // held by the caller of the running job
  std::mutex mu_;                  // guards seq_ and the wake-ups
  std::condition_variable cv_, done_cv_;
  uint64_t seq_ = 0;               // job counter
  std::atomic<const Fn*> fn_{nullptr};
  std::atomic<int64_t> n_{0};
  std::atomic<int> nt_{0}, next_{0}, left_{0};
};

}  // namespace prism
