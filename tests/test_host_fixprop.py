"""The library's host rounding steps, run on the CPU through the built library on a
handle whose host copies are filled directly (no device work is involved), against
the oracle: fix-and-propagate (Section 2.3) bit for bit (the rounded point, the
final domains, the fixed columns in fixing order and the ignored rows), the exact
MIP-feasibility test, the cycle perturbation and the test of an infeasibility
certificate (scylla_farkas_gap, through its C entry point).  The instances include rows
long enough, and slack enough, for the propagation's slack screen and row-activity
caches to end most visits early, so these check that the shortcuts change nothing."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fixprop as F
from paper_2307_03466_gb300 import build as B
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import long_row_instance

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2307_03466_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

HARNESS = r"""
#include <cstdio>
#include <string>
#include <vector>
#include "lp_handle.h"
namespace scylla {
int fix_and_propagate_host(const scylla_lp& lp, const double* xbar, double* xhat, double* dom_lo, double* dom_hi,
                           int32_t* fixed_cols, int64_t* n_fixed, uint8_t* ignored_rows);
int64_t perturb_host(const scylla_lp& lp, double* x, const double* xbar, int kind, int64_t K, uint64_t seed);
}
template <typename T> static std::vector<T> rd(const char* dir, const char* name, size_t n) {
  char f[1024]; snprintf(f, sizeof f, "%s/%s", dir, name);
  std::vector<T> v(n); FILE* fp = fopen(f, "rb");
  if (!fp || fread(v.data(), sizeof(T), n, fp) != n) { fprintf(stderr, "read %s\n", f); exit(2); }
  fclose(fp); return v;
}
template <typename T> static void wr(const char* dir, const char* name, const T* p, size_t n) {
  char f[1024]; snprintf(f, sizeof f, "%s/%s", dir, name);
  FILE* fp = fopen(f, "wb"); fwrite(p, sizeof(T), n, fp); fclose(fp);
}
int main(int argc, char** argv) {
  const char* d = argv[1];
  auto dims = rd<int64_t>(d, "dims", 3);
  scylla_lp lp;
  lp.m0 = dims[0]; lp.n0 = dims[1]; lp.nnz0 = dims[2];
  lp.rowptr0 = rd<int64_t>(d, "rowptr", size_t(lp.m0 + 1));
  lp.cols0 = rd<int32_t>(d, "cols", size_t(lp.nnz0));
  lp.vals0 = rd<double>(d, "vals", size_t(lp.nnz0));
  lp.host_matrix_ready = true;
  lp.c0.assign(size_t(lp.n0), 0.0);
  lp.lo0 = rd<double>(d, "lo", size_t(lp.m0)); lp.hi0 = rd<double>(d, "hi", size_t(lp.m0));
  lp.l0 = rd<double>(d, "l", size_t(lp.n0)); lp.u0 = rd<double>(d, "u", size_t(lp.n0));
  lp.int0 = rd<uint8_t>(d, "int", size_t(lp.n0));
  lp.host_vectors_ready = true;
  lp.n_int = 0; for (auto v : lp.int0) lp.n_int += v;
  auto xbar = rd<double>(d, "xbar", size_t(lp.n0));
  const std::string mode = argc > 2 ? argv[2] : "fixprop";
  if (mode == "check") {
    // points in "pts" (npts x n): one verdict byte each
    auto np_ = rd<int64_t>(d, "npts", 1);
    auto pts = rd<double>(d, "pts", size_t(np_[0] * lp.n0));
    std::vector<uint8_t> v(static_cast<size_t>(np_[0]));
    for (int64_t k = 0; k < np_[0]; ++k) v[size_t(k)] = scylla::check_feasible_host(lp, pts.data() + k * lp.n0) ? 1 : 0;
    wr(d, "o_check", v.data(), v.size());
    return 0;
  }
  if (mode == "many") {
    // points in "pts" (npts x n) through scylla_fix_and_propagate_many: xhat, domains
    // and fixed counts of all points
    auto np_ = rd<int64_t>(d, "npts", 1);
    const size_t K = size_t(np_[0]), n = size_t(lp.n0);
    auto pts = rd<double>(d, "pts", K * n);
    std::vector<double> xh(K * n), dlo(K * n), dhi(K * n);
    std::vector<int64_t> nfs(K);
    const int rc = scylla_fix_and_propagate_many(&lp, int32_t(K), pts.data(), xh.data(), dlo.data(), dhi.data(),
                                                 nfs.data());
    if (rc != 0) { fprintf(stderr, "rc %d\n", rc); return 3; }
    wr(d, "m_xhat", xh.data(), xh.size()); wr(d, "m_dl", dlo.data(), dlo.size());
    wr(d, "m_du", dhi.data(), dhi.size()); wr(d, "m_nf", nfs.data(), nfs.size());
    return 0;
  }
  if (mode == "farkas") {
    // multipliers in "ys" (ny x m): D(y) of each
    auto ny = rd<int64_t>(d, "ny", 1);
    auto ys = rd<double>(d, "ys", size_t(ny[0] * lp.m0));
    std::vector<double> g(static_cast<size_t>(ny[0]));
    std::vector<int32_t> rcs(static_cast<size_t>(ny[0]));
    for (int64_t k = 0; k < ny[0]; ++k) rcs[size_t(k)] = scylla_farkas_gap(&lp, ys.data() + k * lp.m0, &g[size_t(k)]);
    wr(d, "o_gap", g.data(), g.size());
    wr(d, "o_rc", rcs.data(), rcs.size());
    return 0;
  }
  if (mode == "perturb") {
    auto args = rd<int64_t>(d, "pargs", 3);  // kind, K, seed
    auto x = rd<double>(d, "xhat", size_t(lp.n0));
    const int64_t fl = scylla::perturb_host(lp, x.data(), xbar.data(), int(args[0]), args[1], uint64_t(args[2]));
    wr(d, "o_pert", x.data(), x.size());
    wr(d, "o_flipped", &fl, 1);
    return 0;
  }
  std::vector<double> xhat(lp.n0), dl(lp.n0), du(lp.n0);
  std::vector<int32_t> fixed(lp.n0);
  std::vector<uint8_t> ign(lp.m0 > 0 ? lp.m0 : 1);
  int64_t nf = 0;
  if (mode == "multi") {
    // points in "pts" (npts x n), one call each on the same handle; outputs o<k>_*
    auto np_ = rd<int64_t>(d, "npts", 1);
    auto pts = rd<double>(d, "pts", size_t(np_[0] * lp.n0));
    for (int64_t k = 0; k < np_[0]; ++k) {
      const int rck = scylla::fix_and_propagate_host(lp, pts.data() + k * lp.n0, xhat.data(), dl.data(), du.data(),
                                                     fixed.data(), &nf, ign.data());
      if (rck != 0) { fprintf(stderr, "rc %d\n", rck); return 3; }
      char pre[32];
      auto name = [&](const char* s) { snprintf(pre, sizeof pre, "o%lld_%s", (long long)k, s); return pre; };
      wr(d, name("xhat"), xhat.data(), xhat.size()); wr(d, name("dl"), dl.data(), dl.size());
      wr(d, name("du"), du.data(), du.size()); wr(d, name("fixed"), fixed.data(), size_t(nf));
      wr(d, name("ign"), ign.data(), size_t(lp.m0)); wr(d, name("nf"), &nf, 1);
    }
    return 0;
  }
  const int rc = scylla::fix_and_propagate_host(lp, xbar.data(), xhat.data(), dl.data(), du.data(), fixed.data(), &nf,
                                                ign.data());
  if (rc != 0) { fprintf(stderr, "rc %d\n", rc); return 3; }
  wr(d, "o_xhat", xhat.data(), xhat.size()); wr(d, "o_dl", dl.data(), dl.size()); wr(d, "o_du", du.data(), du.size());
  wr(d, "o_fixed", fixed.data(), size_t(nf)); wr(d, "o_ign", ign.data(), size_t(lp.m0));
  wr(d, "o_nf", &nf, 1);
  if (mode == "twice") {
    // a second call on the same handle (it reuses the first propagation's end state)
    auto xbar2 = rd<double>(d, "xbar2", size_t(lp.n0));
    const int rc2 = scylla::fix_and_propagate_host(lp, xbar2.data(), xhat.data(), dl.data(), du.data(), fixed.data(),
                                                   &nf, ign.data());
    if (rc2 != 0) { fprintf(stderr, "rc %d\n", rc2); return 3; }
    wr(d, "o2_xhat", xhat.data(), xhat.size()); wr(d, "o2_dl", dl.data(), dl.size());
    wr(d, "o2_du", du.data(), du.size()); wr(d, "o2_fixed", fixed.data(), size_t(nf));
    wr(d, "o2_ign", ign.data(), size_t(lp.m0)); wr(d, "o2_nf", &nf, 1);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    lib = B.build()
    d = tmp_path_factory.mktemp("fp")
    src = d / "h.cpp"
    exe = d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE, "-I", CUDA_INC, str(src), "-o", str(exe),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    return str(exe)


def write_instance(inst, xbar, d):
    os.makedirs(d, exist_ok=True)
    np.asarray([inst.m, inst.n, len(inst.vals)], np.int64).tofile(os.path.join(d, "dims"))
    np.asarray(inst.rowptr, np.int64).tofile(os.path.join(d, "rowptr"))
    np.asarray(inst.cols, np.int32).tofile(os.path.join(d, "cols"))
    np.asarray(inst.vals, np.float64).tofile(os.path.join(d, "vals"))
    for k in ("lo", "hi", "l", "u"):
        np.asarray(getattr(inst, k), np.float64).tofile(os.path.join(d, k))
    np.asarray(inst.is_int, np.uint8).tofile(os.path.join(d, "int"))
    np.asarray(xbar, np.float64).tofile(os.path.join(d, "xbar"))


def read_outputs(d, prefix="o_"):
    f = lambda k: os.path.join(d, prefix + k)
    nf = int(np.fromfile(f("nf"), np.int64)[0])
    return (np.fromfile(f("xhat")), np.fromfile(f("dl")), np.fromfile(f("du")),
            np.fromfile(f("fixed"), np.int32)[:nf], np.fromfile(f("ign"), np.uint8).astype(bool))


def run_harness(exe, inst, xbar, d):
    write_instance(inst, xbar, d)
    r = subprocess.run([exe, d], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return read_outputs(d)


def ping_pong_instance():
    """x - y >= 1 and y - x >= 1 over integers in [0, 1e9] plus a free integer column:
    the first propagation stops at its visit cap (20 m + 1000) long before the domains
    cross, and fixing x then sends the pair around again."""
    inf = np.inf
    return I.Instance("ping_pong", 2, 3, np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.int32),
                      np.array([1.0, -1.0, -1.0, 1.0]), np.zeros(3), np.array([1.0, 1.0]), np.array([inf, inf]),
                      np.zeros(3), np.array([1e9, 1e9, 5.0]), np.ones(3, np.uint8))


INSTANCES = {
    "setcover": lambda: I.set_cover(),
    "knapcover": lambda: I.knapsack_cover(300, seed=8),
    "packcover_gen_int": lambda: I.packing_covering(m=300, n=600, per_col=4, seed=21),
    "packcover_2kx4k": lambda: I.packing_covering(m=2000, n=4000, per_col=10, seed=11),
    "mcf_small": lambda: I.mcf(nodes=20, avg_degree=4, commodities=6, seed=2),
    "long_rows": lambda: long_row_instance(),
    "ping_pong": lambda: ping_pong_instance(),
    "no_rows": lambda: I.Instance("no_rows", 0, 4, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                                  np.zeros(4), np.zeros(0), np.zeros(0), np.array([0.0, -3.0, 0.0, -np.inf]),
                                  np.array([1.0, 3.0, 2.5, np.inf]), np.array([1, 1, 0, 1], np.uint8)),
    "no_integers": lambda: I.Instance("no_integers", 2, 3, np.array([0, 2, 3], np.int64),
                                      np.array([0, 2, 1], np.int32), np.array([1.0, 2.0, -1.0]), np.zeros(3),
                                      np.array([1.0, -np.inf]), np.array([np.inf, 0.5]), np.zeros(3),
                                      np.full(3, 4.0), np.zeros(3, np.uint8)),
}


@pytest.mark.parametrize("name", list(INSTANCES))
def test_host_fix_and_propagate_equals_oracle(harness, tmp_path, name):
    inst = INSTANCES[name]()
    rng = np.random.default_rng(17)
    lo_b = np.where(np.isfinite(inst.l), inst.l, -5.0)
    hi_b = np.where(np.isfinite(inst.u), inst.u, lo_b + 10.0)
    xbar = rng.uniform(lo_b, hi_b)
    xhat, dl, du, fixed, ign = run_harness(harness, inst, xbar, str(tmp_path / name))
    oxhat, odl, odu, ofixed, oign = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                        inst.l, inst.u, inst.is_int, xbar)
    assert np.array_equal(xhat, oxhat) and np.array_equal(dl, odl) and np.array_equal(du, odu)
    assert np.array_equal(fixed, ofixed) and np.array_equal(ign, oign)


def assert_equals_oracle(inst, xbar, got):
    want = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, xbar)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("name", ["setcover", "packcover_2kx4k", "long_rows"])
def test_host_second_call_reuses_first_propagation(harness, tmp_path, name):
    """The first propagation (bounds alone) is kept in the handle; a second call with
    another point starts from it and still equals the oracle's fresh run."""
    inst = INSTANCES[name]()
    rng = np.random.default_rng(23)
    lo_b = np.where(np.isfinite(inst.l), inst.l, -5.0)
    hi_b = np.where(np.isfinite(inst.u), inst.u, lo_b + 10.0)
    xbar, xbar2 = rng.uniform(lo_b, hi_b), rng.uniform(lo_b, hi_b)
    d = str(tmp_path / name)
    write_instance(inst, xbar, d)
    np.asarray(xbar2, np.float64).tofile(os.path.join(d, "xbar2"))
    r = subprocess.run([harness, d, "twice"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert_equals_oracle(inst, xbar, read_outputs(d))
    assert_equals_oracle(inst, xbar2, read_outputs(d, "o2_"))


@pytest.mark.parametrize("name", ["setcover", "knapcover", "packcover_gen_int", "mcf_small", "long_rows"])
def test_host_consecutive_calls_on_the_gpu_tests_points(harness, tmp_path, name):
    """The points of the GPU rounding test (a random point, an oracle LP point, exact
    halves), one call after another on one handle as that test makes them."""
    from tests.test_gpu_rounding import xbar_points
    inst = INSTANCES[name]()
    pts = xbar_points(inst, 5)
    d = str(tmp_path / name)
    write_instance(inst, np.zeros(inst.n), d)
    np.asarray([len(pts)], np.int64).tofile(os.path.join(d, "npts"))
    np.asarray(pts, np.float64).tofile(os.path.join(d, "pts"))
    r = subprocess.run([harness, d, "multi"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    for k, xb in enumerate(pts):
        assert_equals_oracle(inst, xb, read_outputs(d, f"o{k}_"))


@pytest.mark.parametrize("name", ["setcover", "knapcover", "packcover_gen_int", "mcf_small", "long_rows"])
def test_host_feasibility_check_equals_oracle(harness, tmp_path, name):
    """The exact MIP-feasibility test (Algorithm 1's two tests) on random integral
    points, the all-zero and all-one points and the generator's interior point."""
    from oracle import pump as P
    inst = INSTANCES[name]()
    rng = np.random.default_rng(1)
    hi_b = np.where(np.isfinite(inst.u), inst.u, inst.l + 10)
    pts = [np.ones(inst.n), np.zeros(inst.n)]
    for _ in range(20):
        x = rng.uniform(inst.l, np.minimum(hi_b, inst.l + 10))
        x[inst.is_int == 1] = np.round(x[inst.is_int == 1])
        pts.append(x)
    if "x0" in inst.meta:
        pts.append(inst.meta["x0"])
    d = str(tmp_path / name)
    write_instance(inst, np.zeros(inst.n), d)
    np.asarray([len(pts)], np.int64).tofile(os.path.join(d, "npts"))
    np.asarray(pts, np.float64).tofile(os.path.join(d, "pts"))
    r = subprocess.run([harness, d, "check"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(os.path.join(d, "o_check"), np.uint8).astype(bool)
    want = [P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, x)
            for x in pts]
    assert list(got) == want


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("K", [1, 2, 17])
def test_host_perturbation_equals_oracle(harness, tmp_path, kind, K):
    """Cycle handling (Section 2.3): the short- and long-cycle flips with the
    SplitMix64 stream of the round."""
    from oracle import pump as P
    inst = I.packing_covering(m=200, n=400, per_col=3, seed=4)
    rng = np.random.default_rng(K)
    xbar = rng.uniform(inst.l, np.minimum(inst.u, 10))
    xhat = xbar.copy()
    ic = np.nonzero(inst.is_int)[0]
    xhat[ic] = np.floor(xbar[ic] + 0.5)
    key = tuple(float(xhat[j]) for j in ic)
    hist = [key] if kind == 1 else [key, tuple(v + 1 for v in key)]
    xo, _ = P.perturb(xhat, xbar, hist, K, 12345, list(ic), inst.l, inst.u)
    d = str(tmp_path / f"p{kind}_{K}")
    write_instance(inst, xbar, d)
    np.asarray(xhat, np.float64).tofile(os.path.join(d, "xhat"))
    np.asarray([kind, K, 12345], np.int64).tofile(os.path.join(d, "pargs"))
    r = subprocess.run([harness, d, "perturb"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    xg = np.fromfile(os.path.join(d, "o_pert"))
    assert np.array_equal(xg, xo)
    assert int(np.fromfile(os.path.join(d, "o_flipped"), np.int64)[0]) == int(np.sum(xg != xhat))


def _farkas(harness, d, inst, ys):
    write_instance(inst, np.zeros(inst.n), d)
    np.asarray([len(ys)], np.int64).tofile(os.path.join(d, "ny"))
    np.asarray(ys, np.float64).tofile(os.path.join(d, "ys"))
    r = subprocess.run([harness, d, "farkas"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rc = np.fromfile(os.path.join(d, "o_rc"), np.int32)
    g = np.fromfile(os.path.join(d, "o_gap"))
    return np.where(rc == 0, g, np.nan) if np.any(rc != 0) else g


def test_host_farkas_gap_equals_oracle(harness, tmp_path):
    """The library's certificate test (scylla_farkas_gap) against oracle/infeas.py: the
    same -inf verdicts, equal values on exactly representable cases, and values within
    the rounding of the oracle's uncompensated A^T y elsewhere (LPs with a known
    feasible point, and the same LPs with a row added that makes them infeasible)."""
    from oracle import infeas as X
    from tests.test_oracle_infeas import _admissible_y
    inf = np.inf
    # hand cases: x >= 1 and x <= 0 on a free x; a row against a box
    two = I.Instance("two", 2, 1, np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), np.array([1.0, 1.0]),
                     np.zeros(1), np.array([1.0, -inf]), np.array([inf, 0.0]), np.array([-inf]), np.array([inf]),
                     np.zeros(1, np.uint8))
    g = _farkas(harness, str(tmp_path / "two"), two, [[1.0, -1.0], [3.0, -3.0], [1.0, 0.0], [-1.0, 1.0], [0.0, 0.0]])
    assert list(g) == [1.0, 3.0, -inf, -inf, 0.0]
    # a NaN multiplier is rejected by the entry point (INVALID_ARG, no value)
    assert np.isnan(_farkas(harness, str(tmp_path / "two_nan"), two, [[np.nan, 1.0]])[0])
    for seed in range(3):
        inst = I.packing_covering(m=50, n=100, per_col=4, seed=200 + seed)
        rng = np.random.default_rng(seed)
        ys = [_admissible_y(inst, rng) for _ in range(20)]
        ys.append(rng.normal(size=inst.m))  # leans on infinite sides
        got = _farkas(harness, str(tmp_path / f"pc{seed}"), inst, ys)
        A = inst.csr()
        for y, gl in zip(ys, got):
            go = X.farkas_gap(A, inst.lo, inst.hi, inst.l, inst.u, y)
            if go == -inf:
                assert gl == -inf
                continue
            scale = 1.0 + float(np.abs(A).T @ np.abs(y) @ np.abs(inst.u)) + float(
                np.abs(y) @ np.where(y > 0, np.abs(np.nan_to_num(inst.lo, neginf=0)), np.abs(np.nan_to_num(inst.hi, posinf=0))))
            assert abs(gl - go) <= 1e-13 * scale
            assert gl <= 1e-9 * scale  # weak duality on a feasible LP
        # the infeasible extension of the oracle pins: D = 1 up to rounding
        y0 = ys[0]
        a = A.T @ y0
        L = X._side_min(y0, inst.lo, inst.hi)
        A2 = sp.vstack([A, sp.csr_matrix(a)]).tocsr()
        inf_inst = I.Instance("ext", inst.m + 1, inst.n, A2.indptr.astype(np.int64), A2.indices.astype(np.int32),
                              A2.data, inst.c, np.append(inst.lo, -inf), np.append(inst.hi, L - 1.0), inst.l, inst.u,
                              inst.is_int)
        y2 = np.append(y0, -1.0)
        g2 = _farkas(harness, str(tmp_path / f"ext{seed}"), inf_inst, [y2])[0]
        assert abs(g2 - 1.0) <= 1e-9 * (1.0 + abs(L))


@pytest.mark.parametrize("name", ["setcover", "packcover_2kx4k", "mcf_small", "long_rows", "ping_pong", "no_rows"])
def test_host_many_points_at_once_equal_the_oracle(harness, tmp_path, name):
    """scylla_fix_and_propagate_many (the points dealt to the host threads, each from
    the kept first propagation) gives every point exactly the oracle's result."""
    inst = INSTANCES[name]()
    rng = np.random.default_rng(31)
    lo_b = np.where(np.isfinite(inst.l), inst.l, -5.0)
    hi_b = np.where(np.isfinite(inst.u), inst.u, lo_b + 10.0)
    pts = [rng.uniform(lo_b, hi_b) for _ in range(11)]
    pts.append(np.clip(np.floor(pts[0]) + 0.5, inst.l, inst.u))
    d = str(tmp_path / name)
    write_instance(inst, np.zeros(inst.n), d)
    np.asarray([len(pts)], np.int64).tofile(os.path.join(d, "npts"))
    np.asarray(pts, np.float64).tofile(os.path.join(d, "pts"))
    r = subprocess.run([harness, d, "many"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    K, n = len(pts), inst.n
    xh = np.fromfile(os.path.join(d, "m_xhat")).reshape(K, n)
    dl = np.fromfile(os.path.join(d, "m_dl")).reshape(K, n)
    du = np.fromfile(os.path.join(d, "m_du")).reshape(K, n)
    nf = np.fromfile(os.path.join(d, "m_nf"), np.int64)
    for k, xb in enumerate(pts):
        oxhat, odl, odu, ofixed, _ = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                         inst.l, inst.u, inst.is_int, xb)
        assert np.array_equal(xh[k], oxhat) and np.array_equal(dl[k], odl) and np.array_equal(du[k], odu)
        assert nf[k] == len(ofixed)


def test_host_many_with_no_points_and_a_nan(harness, tmp_path):
    inst = I.set_cover(m=20, n=30, seed=1)
    d = str(tmp_path / "k0")
    write_instance(inst, np.zeros(inst.n), d)
    np.asarray([0], np.int64).tofile(os.path.join(d, "npts"))
    np.zeros(0).tofile(os.path.join(d, "pts"))
    r = subprocess.run([harness, d, "many"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    pts = np.zeros((2, inst.n))
    pts[1, 3] = np.nan
    np.asarray([2], np.int64).tofile(os.path.join(d, "npts"))
    pts.tofile(os.path.join(d, "pts"))
    r = subprocess.run([harness, d, "many"], capture_output=True, text=True, timeout=60)
    assert r.returncode == 3 and "rc -1" in r.stderr  # INVALID_ARG, nothing computed
