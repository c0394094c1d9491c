// Checks of the host worker pool (paper_2604_00250_gb300/csrc/host_pool.h), built with g++ by
// tests/test_host_pool.py: every chunk of a job runs exactly once and covers [0, n) without
// overlap; two threads that submit jobs at once both get their work done (the loser of the
// race runs its job itself); a child forked after the pool started gets no pool and must run
// its jobs itself. Prints "ok" and exits 0, or names the failed check and exits 1.
#include <sys/wait.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "host_pool.h"

using prism::HostPool;

static bool cover(HostPool* pool, int64_t n, int nt) {
  std::vector<std::atomic<int>> hit(static_cast<size_t>(n));
  for (auto& h : hit) h.store(0);
  const bool ran = pool->run(n, nt, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) hit[static_cast<size_t>(i)].fetch_add(1);
  });
  if (!ran) return true;   // busy: the caller would run it itself
  for (auto& h : hit)
    if (h.load() != 1) return false;
  return true;
}

int main() {
  HostPool* pool = HostPool::get();
  if (!pool) {
    std::printf("ok (no pool: jobs run on the calling thread)\n");
    return 0;
  }
  if (pool->threads() < 2 || pool->threads() > 16) {
    std::printf("threads %d outside 2..16\n", pool->threads());
    return 1;
  }
  for (int rep = 0; rep < 200; ++rep) {
    const int64_t n = 1 + (rep * 7919) % 5000;
    const int nt = 1 + rep % pool->threads();
    if (!cover(pool, n, nt)) {
      std::printf("chunks of n=%lld nt=%d did not cover [0, n) exactly once\n", static_cast<long long>(n), nt);
      return 1;
    }
  }
  // two submitters at once: each job must run completely, by the pool or by its caller
  std::atomic<int64_t> sum{0};
  auto submit = [&](int64_t base) {
    for (int rep = 0; rep < 100; ++rep) {
      const int64_t n = 1000;
      auto fn = [&](int64_t b, int64_t e) {
        int64_t s = 0;
        for (int64_t i = b; i < e; ++i) s += base + i;
        sum.fetch_add(s);
      };
      if (!pool->run(n, pool->threads(), fn)) fn(0, n);
    }
  };
  std::thread t1(submit, 0), t2(submit, 1000000);
  t1.join();
  t2.join();
  const int64_t want = 100 * (999 * 1000 / 2) + 100 * (1000000LL * 1000 + 999 * 1000 / 2);
  if (sum.load() != want) {
    std::printf("concurrent jobs summed %lld, want %lld\n", static_cast<long long>(sum.load()),
                static_cast<long long>(want));
    return 1;
  }
  // a forked child has no workers: get() must return nullptr there
  const pid_t pid = fork();
  if (pid == 0) _exit(HostPool::get() == nullptr ? 0 : 3);
  int st = 0;
  if (pid < 0 || waitpid(pid, &st, 0) != pid || !WIFEXITED(st) || WEXITSTATUS(st) != 0) {
    std::printf("the forked child still saw the pool\n");
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
