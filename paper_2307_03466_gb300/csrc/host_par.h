// Host-side parallel helpers of the set-up path: a fork-join on a small pool of
// std::thread workers, and the stable CSR transpose (counting sort) that the
// set-up needs twice (the stored transpose A^T of the device path, and the
// column structure of the host propagation).
#pragma once

#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include <unistd.h>

namespace scylla {

// worker threads for host set-up work: the hardware threads, at most 16
inline int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return int(std::max(1u, std::min(h, 16u)));
}

// A fixed pool of host_threads() - 1 workers, created on first use (per process)
// and never torn down (its threads sleep between jobs and end with the process).  run(T, f) calls
// f(t) for t = 0 .. T-1 on the workers and the calling thread, and returns when all
// calls have returned; concurrent callers take turns.
class HostPool {
 public:
  static HostPool& get() {
    // a forked child has none of its parent's workers: it starts a pool of its own
    static HostPool* pool = nullptr;
    static pid_t owner = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!pool || owner != getpid()) {
      pool = new HostPool(host_threads() - 1);
      owner = getpid();
    }
    return *pool;
  }
  void run(int T, const std::function<void(int)>& f) {
    std::lock_guard<std::mutex> turn(run_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &f;
      next_ = 0;
      total_ = T;
      pending_ = T;
      ++gen_;
    }
    cv_work_.notify_all();
    std::unique_lock<std::mutex> lk(mu_);
    drain(lk);
    cv_done_.wait(lk, [&] { return pending_ == 0; });
    job_ = nullptr;
  }

 private:
  explicit HostPool(int workers) {
    for (int w = 0; w < workers; ++w) th_.emplace_back([this] { loop(); });
  }
  // claim and run tasks of the current job until none is left (lock held on entry
  // and exit, released around each task)
  void drain(std::unique_lock<std::mutex>& lk) {
    while (job_ && next_ < total_) {
      const int t = next_++;
      const std::function<void(int)>* f = job_;
      lk.unlock();
      (*f)(t);
      lk.lock();
      if (--pending_ == 0) cv_done_.notify_all();
    }
  }
  void loop() {
    std::unique_lock<std::mutex> lk(mu_);
    unsigned long long seen = 0;
    for (;;) {
      cv_work_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      drain(lk);
    }
  }
  std::mutex run_mu_, mu_;
  std::condition_variable cv_work_, cv_done_;
  const std::function<void(int)>* job_ = nullptr;
  int next_ = 0, total_ = 0, pending_ = 0;
  unsigned long long gen_ = 0;
  std::vector<std::thread> th_;
};

// f(t) for t = 0 .. T-1 on the host pool
template <typename F>
void fork_join(int T, F&& f) {
  if (T <= 1) {
    f(0);
    return;
  }
  const std::function<void(int)> g = [&f](int t) { f(t); };
  HostPool::get().run(T, g);
}

// threads worth using for `work` elementary steps (about 64k steps per thread)
inline int threads_for(int64_t work) {
  return int(std::max<int64_t>(1, std::min<int64_t>(host_threads(), work / 65536)));
}

// Stable transpose of an m x n CSR matrix: column j of the result lists the rows
// of the nonzeros of column j in ascending order (with their values when vals is
// given).  Parallel counting sort: thread t takes the rows of the t-th slice of the
// nonzeros, counts its entries per column, the counts are turned into per-thread
// write positions (thread t after threads 0..t-1 within every column), and each
// thread scatters its rows in order.  The per-thread counts take T * n * 4 bytes;
// T is capped to keep them under 256 MB.
template <typename IP, typename IQ>
void transpose_csr(int64_t m, int64_t n, const IP* rowptr, const int32_t* cols, const double* vals,
                   std::vector<IQ>& colptr, std::vector<int32_t>& rows, std::vector<double>* tvals) {
  const int64_t nnz = int64_t(rowptr[m]);
  colptr.assign(size_t(n) + 1, IQ(0));
  rows.assign(size_t(nnz), 0);
  if (tvals) tvals->assign(size_t(nnz), 0.0);
  int T = threads_for(nnz);
  const int64_t cap = (int64_t(256) << 20) / (4 * std::max<int64_t>(n, 1));
  T = int(std::max<int64_t>(1, std::min<int64_t>(T, cap)));
  // row slices with about nnz / T nonzeros each
  std::vector<int64_t> r(size_t(T) + 1, 0);
  for (int t = 1; t < T; ++t) {
    const int64_t target = nnz * t / T;
    r[t] = int64_t(std::lower_bound(rowptr, rowptr + m + 1, IP(target)) - rowptr);
    r[t] = std::max(r[t], r[t - 1]);
  }
  r[T] = m;
  std::vector<int32_t> cnt(size_t(T) * size_t(n), 0);
  fork_join(T, [&](int t) {
    int32_t* c = cnt.data() + size_t(t) * size_t(n);
    for (int64_t p = int64_t(rowptr[r[t]]); p < int64_t(rowptr[r[t + 1]]); ++p) c[cols[p]]++;
  });
  // column totals and their prefix, by column ranges
  std::vector<int64_t> part(size_t(T) + 1, 0);
  auto crange = [&](int t, int64_t& j0, int64_t& j1) {
    j0 = n * t / T;
    j1 = n * (t + 1) / T;
  };
  fork_join(T, [&](int t) {
    int64_t j0, j1, s = 0;
    crange(t, j0, j1);
    for (int64_t j = j0; j < j1; ++j)
      for (int u = 0; u < T; ++u) s += cnt[size_t(u) * size_t(n) + size_t(j)];
    part[t + 1] = s;
  });
  for (int t = 0; t < T; ++t) part[t + 1] += part[t];
  fork_join(T, [&](int t) {
    int64_t j0, j1;
    crange(t, j0, j1);
    int64_t run = part[t];
    for (int64_t j = j0; j < j1; ++j) {
      colptr[size_t(j)] = IQ(run);
      for (int u = 0; u < T; ++u) {
        int32_t& c = cnt[size_t(u) * size_t(n) + size_t(j)];
        const int32_t k = c;
        c = int32_t(run);
        run += k;
      }
    }
  });
  colptr[size_t(n)] = IQ(nnz);
  fork_join(T, [&](int t) {
    int32_t* c = cnt.data() + size_t(t) * size_t(n);
    for (int64_t i = r[t]; i < r[t + 1]; ++i)
      for (int64_t p = int64_t(rowptr[i]); p < int64_t(rowptr[i + 1]); ++p) {
        const int32_t q = c[cols[p]]++;
        rows[size_t(q)] = int32_t(i);
        if (tvals) (*tvals)[size_t(q)] = vals[p];
      }
  });
}

}  // namespace scylla
