// Host-side check of the library's worker pool (parallel_for, parallel_items, run_parts in
// gn_internal.cuh / gn_graph.cu), linked against libgn.so.  No GPU is used.  Prints "ok" and
// returns 0 when every check passes; prints what failed and returns 1 otherwise.
#include <sys/wait.h>
#include <unistd.h>

#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "gn_internal.cuh"

static int failures = 0;
#define CHECK(cond, what)                       \
  do {                                          \
    if (!(cond)) {                              \
      std::printf("FAILED: %s\n", what);        \
      ++failures;                               \
    }                                           \
  } while (0)

// every index of [0, n) once, in contiguous blocks with in-range thread ids
static bool covers_once(int n, int grain) {
  std::vector<std::atomic<int>> hits(n);
  for (auto& h : hits) h.store(0);
  std::atomic<bool> ok{true};
  gn::parallel_for(n, grain, [&](int lo, int hi, int t) {
    if (lo > hi || lo < 0 || hi > n || t < 0 || t >= gn::host_threads()) ok = false;
    for (int i = lo; i < hi; ++i) hits[i].fetch_add(1);
  });
  for (int i = 0; i < n; ++i)
    if (hits[i].load() != 1) ok = false;
  return ok;
}

static bool items_once(int n) {
  std::vector<std::atomic<int>> hits(n);
  for (auto& h : hits) h.store(0);
  std::atomic<bool> ok{true};
  gn::parallel_items(n, [&](int i, int t) {
    if (i < 0 || i >= n || t < 0 || t >= gn::host_threads()) ok = false;
    hits[i].fetch_add(1);
  });
  for (int i = 0; i < n; ++i)
    if (hits[i].load() != 1) ok = false;
  return ok;
}

int main() {
  CHECK(gn::host_threads() >= 1 && gn::host_threads() <= 64, "host_threads in [1, 64]");
  for (int n : {0, 1, 7, 1000, 100003})
    for (int grain : {1, 16, 4096}) CHECK(covers_once(n, grain), "parallel_for covers [0, n) once");
  for (int n : {0, 1, 152, 10007}) CHECK(items_once(n), "parallel_items runs each item once");

  // a job posted from inside a job runs inline (no deadlock), from block 0 and from the workers
  {
    std::atomic<long> sum{0};
    gn::parallel_for(64, 1, [&](int lo, int hi, int) {
      for (int i = lo; i < hi; ++i)
        gn::parallel_for(100, 1, [&](int a, int b, int) { sum.fetch_add(b - a); });
    });
    CHECK(sum.load() == 64L * 100, "nested parallel_for");
  }

  // jobs posted from several threads at once are serialised, each complete
  {
    std::atomic<long> sum{0};
    std::vector<std::thread> th;
    for (int c = 0; c < 4; ++c)
      th.emplace_back([&] {
        for (int r = 0; r < 200; ++r)
          gn::parallel_items(50, [&](int i, int) { sum.fetch_add(i); });
      });
    for (auto& t : th) t.join();
    CHECK(sum.load() == 4L * 200 * (49 * 50 / 2), "concurrent callers");
  }

  // a forked child starts its own workers (the parent's do not exist there)
  {
    std::fflush(stdout);
    const pid_t pid = fork();
    if (pid == 0) {
      alarm(20);  // a hang here ends the child, and the check below fails
      _exit(covers_once(100000, 16) && items_once(500) ? 0 : 3);
    }
    int status = 0;
    CHECK(pid > 0 && waitpid(pid, &status, 0) == pid && WIFEXITED(status) && WEXITSTATUS(status) == 0,
          "pool in a forked child");
  }

  if (failures == 0) std::printf("ok\n");
  return failures == 0 ? 0 : 1;
}
