"""The device More-Thuente search (Step III, Section 2.1; Section 2.4),
compiled for the host, against the oracle's search on thousands of random
polynomial lines.

The GPU line search evaluates phi(beta) = f(x + beta d), a polynomial of
degree 2N, from its coefficients and advances the search one trial at a time
with mt_init / mt_advance of csrc/mt_device.cuh.  Here those two functions
(and the Newton-refined FP64 helpers they call) are compiled with the host
C++ compiler, unchanged: the FP32 seeds of the Newton steps come from IEEE
host operations, and floating-point contraction is off, so values can differ
from the device's in the last bits only.  Each search runs on a random
polynomial of degree 4, 6 or 8 (with phi'(0) < 0 but for a few) under varied
options (ftol, gtol, xtol, smallest, largest and first step, maxfev) so that
every exit code occurs, and the two searches must make the same
trials (within 1e-9 relative), the same number of them, and end with the same
exit code.  Trials are compared relative to the largest step the search has
tried so far: a trial near 0 reached from steps of size ~100 is an
interpolant's minimiser computed with cancellation, and the two sides form
the interpolants in different (algebraically equal) ways.  A decision taken
at the rounding limit (a bracket a few ulps wide) can go either way under a
last-bit difference, so a small share of searches (at most 0.2 %) may end
differently; each is printed."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cp_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1105_5331_gb300", "csrc")
MAX_TRIALS = 64

HARNESS = r"""
#include <cmath>
#include <cstdio>
#define __device__
#define __forceinline__ inline
static inline float __frcp_rn(float x) { return 1.0f / x; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
using std::fabs; using std::fma; using std::fmax; using std::fmin; using std::isfinite; using std::sqrt;
#include "mt_device.cuh"

// phi = sum_k c[k] b^k and phi' = sum_k dc[k] b^k by Horner's rule
static double horner(const double* c, int deg, double b) {
  double v = c[deg];
  for (int k = deg - 1; k >= 0; --k) v = v * b + c[k];
  return v;
}

int main() {
  int n;
  if (std::scanf("%d", &n) != 1) return 1;
  for (int p = 0; p < n; ++p) {
    int deg;
    double c[16], dc[16];
    cp_ls_opts o;
    std::scanf("%d", &deg);
    for (int k = 0; k <= deg; ++k) std::scanf("%lf", &c[k]);
    for (int k = 0; k < deg; ++k) std::scanf("%lf", &dc[k]);
    std::scanf("%lf %lf %lf %lf %lf %lf %d", &o.ftol, &o.gtol, &o.xtol, &o.stpmin, &o.stpmax, &o.stp0,
               &o.maxfev);
    const double f0 = horner(c, deg, 0.0), g0 = horner(dc, deg - 1, 0.0);
    cpg::MTState s;
    cpg::mtdev::mt_init(s, f0, g0, o);
    double trials[MAXT];
    int nt = 0;
    while (!s.done && nt < MAXT) {
      trials[nt++] = s.stp;
      const double f = horner(c, deg, s.stp), g = horner(dc, deg - 1, s.stp);
      cpg::mtdev::mt_advance(&s, &f, &g);
    }
    std::printf("%d %d %.17g", s.nfev, s.info, s.stp_eval);
    for (int k = 0; k < nt; ++k) std::printf(" %.17g", trials[k]);
    std::printf("\n");
  }
  return 0;
}
""".replace("MAXT", str(MAX_TRIALS))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("mt_host")
    # The search's state struct, taken from the library's header; the rest of
    # that header (launch plumbing, CUDA runtime types) is not needed here.
    src = open(os.path.join(CSRC, "linesearch.cuh")).read()
    m = re.search(r"struct MTState \{.*?\};", src, re.S)
    assert m, "MTState not found"
    with open(d / "linesearch.cuh", "w") as fh:
        fh.write('#pragma once\n#include "cp.h"\nnamespace cpg {\n' + m.group(0) + "\n}\n")
    for name in ("mt_device.cuh", "newton.cuh"):
        shutil.copy(os.path.join(CSRC, name), d / name)
    with open(d / "harness.cpp", "w") as fh:
        fh.write(HARNESS)
    exe = d / "mt_host"
    out = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(d),
                          "-I", os.path.join(ROOT, "include"), str(d / "harness.cpp"), "-o", str(exe)],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-3000:]
    return str(exe)


def random_searches(n, seed=20240605):
    """Polynomial lines of degree 2N (N = 2, 3, 4) with phi'(0) < 0 and a
    positive leading coefficient, scaled over several decades, with options
    drawn to reach the search's rules (tight and loose tolerances, first steps
    far too short or too long, a few trials only)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        deg = int(rng.choice([4, 6, 8]))
        c = rng.standard_normal(deg + 1) * 10.0 ** rng.uniform(-2, 2, deg + 1)
        # a few lines that do not descend (both sides stop at once, info -1)
        c[1] = -abs(c[1]) - 1e-3 if rng.uniform() > 0.01 else abs(c[1])
        c[deg] = abs(c[deg]) + 1e-3
        opts = O.LSOpts(ftol=float(rng.choice([1e-4, 1e-3, 0.1, 0.3])),
                        gtol=float(rng.choice([1e-2, 0.1, 0.5, 0.9])),
                        xtol=float(rng.choice([1e-15, 1e-15, 1e-8, 1e-3, 0.1, 0.8])),
                        # a smallest step above the minimiser now and then (info 4)
                        stpmin=float(rng.choice([1e-15] * 19 + [0.3])),
                        stpmax=float(rng.choice([1e15, 1e15, 2.0, 10.0])),
                        stp0=float(10.0 ** rng.uniform(-4, 3)),
                        maxfev=int(rng.choice([20, 20, 6, 3])))
        if opts.ftol >= opts.gtol:
            opts.ftol = opts.gtol / 10.0
        out.append((c, opts))
    return out


def horner(c, b):
    v = c[-1]
    for x in reversed(c[:-1]):
        v = v * b + x
    return v


def derivative(c):
    return [k * float(c[k]) for k in range(1, len(c))]


def oracle_search(c, opts):
    trials = []
    c = [float(x) for x in c]
    dc = derivative(c)

    def phi(b):
        trials.append(b)
        return horner(c, b), horner(dc, b), None

    f0 = float(c[0])
    g0 = float(c[1])
    stp, _, _, _, nfev, info = O.more_thuente(phi, f0, g0, opts)
    return nfev, info, stp, trials


def test_device_search_matches_the_oracle_on_random_lines(harness):
    cases = random_searches(10000)
    lines = [str(len(cases))]
    for c, o in cases:
        lines.append(f"{len(c) - 1} " + " ".join(repr(float(x)) for x in list(c) + derivative(c)))
        lines.append(f"{o.ftol!r} {o.gtol!r} {o.xtol!r} {o.stpmin!r} {o.stpmax!r} {o.stp0!r} {o.maxfev}")
    out = subprocess.run([harness], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = out.stdout.strip().splitlines()
    assert len(rows) == len(cases)
    differ, infos = [], {}
    for k, ((c, o), row) in enumerate(zip(cases, rows)):
        v = row.split()
        nfev, info, stp = int(v[0]), int(v[1]), float(v[2])
        trials = [float(x) for x in v[3:]]
        nfo, info_o, stp_o, trials_o = oracle_search(c, o)
        infos[info_o] = infos.get(info_o, 0) + 1
        same = (nfev, info) == (nfo, info_o) and len(trials) == len(trials_o) and all(
            abs(a - b) <= 1e-9 * max(abs(x) for x in trials_o[:j + 1]) for j, (a, b) in enumerate(zip(trials, trials_o)))
        if not same:
            differ.append((k, (nfev, info, trials), (nfo, info_o, trials_o)))
    print("exit codes over the searches (oracle):", dict(sorted(infos.items())))
    for k, got, want in differ:
        print("search", k, "host build", got, "oracle", want)
    # every exit code the polynomial lines can produce is reached
    assert {-1, 1, 2, 3, 4, 5, 6}.issubset(infos), infos
    assert len(differ) <= 0.002 * len(cases), f"{len(differ)} of {len(cases)} searches differ"
