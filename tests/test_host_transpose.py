"""The host set-up's parallel stable CSR transpose (a counting sort over slices of
rows on a worker pool) against a serial counting sort, on random matrices that
give the pool one to many slices; compiled from the library's own header."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2307_03466_gb300", "csrc")

HARNESS = r"""
#include "host_par.h"
#include <cstdio>
#include <random>
int main() {
  std::mt19937 g(12345);
  for (int trial = 0; trial < 40; ++trial) {
    const int m = 1 + int(g() % 40000), n = 1 + int(g() % 5000);
    const int maxk = trial % 4 == 0 ? 300 : 30;
    std::vector<int> rp(m + 1, 0), ci;
    std::vector<double> va;
    for (int i = 0; i < m; ++i) {
      std::vector<int> cs;
      const int k = int(g() % maxk);
      for (int q = 0; q < k; ++q) cs.push_back(int(g() % n));
      std::sort(cs.begin(), cs.end());
      cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
      for (int c : cs) { ci.push_back(c); va.push_back(double(g() % 1000) - 500.0); }
      rp[i + 1] = int(ci.size());
    }
    std::vector<int> tp, tr;
    std::vector<double> tv;
    scylla::transpose_csr(m, n, rp.data(), ci.data(), va.data(), tp, tr, &tv);
    std::vector<int64_t> tp64;
    std::vector<int> tr2;
    scylla::transpose_csr(m, n, rp.data(), ci.data(), nullptr, tp64, tr2, nullptr);
    std::vector<int> cp(n + 1, 0), rr(ci.size());
    std::vector<double> vv(ci.size());
    for (int c : ci) cp[c + 1]++;
    for (int j = 0; j < n; ++j) cp[j + 1] += cp[j];
    std::vector<int> cur(cp.begin(), cp.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int p = rp[i]; p < rp[i + 1]; ++p) { const int q = cur[ci[p]]++; rr[q] = i; vv[q] = va[p]; }
    bool ok = cp == tp && rr == tr && vv == tv && rr == tr2;
    for (int j = 0; j <= n; ++j) ok = ok && tp64[j] == cp[j];
    if (!ok) { printf("mismatch in trial %d (m %d, n %d, nnz %zu)\n", trial, m, n, ci.size()); return 1; }
  }
  printf("ok\n");
  return 0;
}
"""


def test_parallel_transpose_matches_serial_counting_sort(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "t.cpp"
    exe = tmp_path / "t"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
