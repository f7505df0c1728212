"""Each plausible mistake below, planted in a copy of the oracle, must fail at
least one pin of tests/test_oracle_pins.py: a check that the pins are strong
enough to tell a right oracle from a nearly right one.  CPU only; nothing is
changed in the real oracle."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text in oracle/cp_oracle.py, planted replacement)
MUTATIONS = [
    ("f drops the factor 2 of the cross term",
     "f = 0.5 * (X.norm2 - 2.0 * inner + model2)", "f = 0.5 * (X.norm2 - inner + model2)"),
    ("gradient sign",
     "g = pack([-Ms[n] + factors[n] @ gamma_bar(factors, n) for n in range(N)])",
     "g = pack([Ms[n] - factors[n] @ gamma_bar(factors, n) for n in range(N)])"),
    ("Gammabar keeps mode n",
     "        if m != n:\n            out = out * (A.T @ A)", "        out = out * (A.T @ A)"),
    ("ALS as Jacobi (old factors in every mode)",
     "        M = X.mttkrp(factors, n)\n        factors[n] = als_mode_solve",
     "        M = X.mttkrp(unpack(np.array(u, dtype=np.float64), X.dims, R), n)\n        factors[n] = als_mode_solve"),
    ("dense MTTKRP pairs the factors with the wrong modes",
     'expr = letters + "," + ",".join(letters[m] + "z" for m in others)',
     'expr = letters + "," + ",".join(letters[m] + "z" for m in reversed(others))'),
    ("COO sort key in the wrong order",
     "perm = np.lexsort(tuple(coords[:, m] for m in reversed(key_modes))).astype(np.int64)",
     "perm = np.lexsort(tuple(coords[:, m] for m in key_modes)).astype(np.int64)"),
    ("COO segment pointers end one short",
     "seg_ptr = np.concatenate([starts, [rows.size]]).astype(np.int64)",
     "seg_ptr = np.concatenate([starts, [rows.size - 1]]).astype(np.int64)"),
    ("Gamma leaves out the last mode",
     "    for G in grams(factors):\n        out = out * G",
     "    for G in grams(factors)[:-1]:\n        out = out * G"),
    ("sparse MTTKRP gathers the output mode",
     "w = w * factors[m][coords[:, m]]", "w = w * factors[m][coords[:, n]]"),
    ("normalisation orders by increasing lambda",
     'order = np.argsort(-lam, kind="stable")', 'order = np.argsort(lam, kind="stable")'),
    ("gradient scaled like the factor",
     "grads[n][:, r] /= s", "grads[n][:, r] *= s"),
    ("lambda root 1/(N-1)",
     "root = pow(float(lam[r]), 1.0 / N)", "root = pow(float(lam[r]), 1.0 / max(N - 1, 1))"),
    ("N-GMRES right-hand side sign", "rhs = -(Pm @ gbar)", "rhs = (Pm @ gbar)"),
    ("N-GMRES step along u_j - ubar", "(ubar[None, :] - U)", "(U - ubar[None, :])"),
    ("N-GMRES ridge not relative", "H + eps * dmax * np.eye", "H + 1e-6 * np.eye"),
    ("ALS iterate not normalised",
     "ubar, _, _ = normalize(als_sweep(X, u, R), dims, R)", "ubar = als_sweep(X, u, R)"),
    ("accelerated iterate not normalised (R6)",
     "uhat, _, _ = normalize(uhat, dims, R)               # R6", "pass"),
    ("line-search point not normalised (R8)",
     "u, g, _ = normalize(x, dims, R, gx)        # R8", "u, g = x, gx"),
    ("failed search keeps any point (R10)",
     "if info == 1 or (extra is not None and fb <= fbar + opts.ls.ftol * beta * s):",
     "if extra is not None:"),
    ("window drops the newest point",
     "                Wu.pop(0)\n                Wg.pop(0)", "                Wu.pop()\n                Wg.pop()"),
    ("window stores the ALS iterate",
     "            Wu.append(u)\n            Wg.append(g)", "            Wu.append(ubar)\n            Wg.append(gbar)"),
    ("trial selection: cubic and quadratic exchanged (case 1)",
     "        ac = _cubic_min(al, fl, gl, at, ft, gt)\n        aq = _quad_min(al, fl, gl, at, ft)",
     "        aq = _cubic_min(al, fl, gl, at, ft, gt)\n        ac = _quad_min(al, fl, gl, at, ft)"),
    ("trial selection: quadratic instead of midpoint (case 1)",
     "nxt = ac if abs(ac - al) < abs(aq - al) else ac + 0.5 * (aq - ac)",
     "nxt = ac if abs(ac - al) < abs(aq - al) else aq"),
    ("trial selection: nearer step (case 2)",
     "nxt = ac if abs(ac - at) >= abs(asec - at) else asec",
     "nxt = ac if abs(ac - at) < abs(asec - at) else asec"),
    ("trial selection: no 0.66 limit (case 3)",
     "nxt = min(at + 0.66 * (au - at), nxt)", "nxt = nxt"),
    ("trial selection: wrong bound (case 3)",
     "ac = stmax if at > al else stmin", "ac = stmin if at > al else stmax"),
    ("trial selection: cubic from the lower end (case 4)",
     "ac = _cubic_min(at, ft, gt, au, fu, gu)", "ac = _cubic_min(al, fl, gl, au, fu, gu)"),
    ("interval update sign",
     "if gt * (al - at) < 0.0:", "if gt * (al - at) > 0.0:"),
    ("line search without the psi stage",
     "if stage == 1 and f <= lo[1] and f > ftest:", "if False:"),
    ("sufficient decrease with the wrong sign",
     "ftest = f0 + stp * ftol * g0", "ftest = f0 - stp * ftol * g0"),
    ("curvature condition without the absolute value",
     "if f <= ftest and abs(g) <= gtol * (-g0):", "if f <= ftest and g <= gtol * (-g0):"),
    ("extrapolation upper limit of 2 steps",
     "xhi = stp + 4.0 * (stp - lo[0])", "xhi = stp + 2.0 * (stp - lo[0])"),
    ("extrapolation lower limit of 1 step",
     "xlo = stp + 1.1 * (stp - lo[0])", "xlo = stp + 1.0 * (stp - lo[0])"),
    ("one evaluation more than maxfev",
     "if nfev >= opts.maxfev:", "if nfev > opts.maxfev:"),
    ("lower end mapped back from psi without the ftol term",
     "lo = (lo_m[0], lo_m[1] + f0 + lo_m[0] * ftol * g0, lo_m[2] + ftol * g0)",
     "lo = (lo_m[0], lo_m[1] + f0, lo_m[2] + ftol * g0)"),
    ("no bisection of a bracket that shrinks too slowly",
     "if abs(hi[0] - lo[0]) >= 0.66 * width1:", "if False:"),
    ("no fall-back to the best point when no progress is possible",
     "or imax - imin <= xtol * imax):\n            stp = lo[0]",
     "or imax - imin <= xtol * imax):\n            pass"),
    ("second stage entered without the slope condition",
     "if stage == 1 and f <= ftest and g >= min(ftol, gtol) * g0:", "if stage == 1 and f <= ftest:"),
]
# Removing the switch to the second stage altogether is an equivalent
# mistake, not planted here: after the first trial with psi <= 0 and
# phi' >= min(ftol, gtol) phi'(0) no later trial can be both no higher than
# the best point and above the sufficient-decrease line, so the first stage's
# step on psi is never taken again (test_linesearch_first_stage_cannot_return_after_the_switch).


@pytest.mark.slow
@pytest.mark.parametrize("name,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, orig, planted):
    src = open(os.path.join(ROOT, "oracle", "cp_oracle.py")).read()
    assert src.count(orig) == 1, f"mutation site not unique or missing: {name}"
    (tmp_path / "oracle").mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), tmp_path / "oracle" / "__init__.py")
    (tmp_path / "oracle" / "cp_oracle.py").write_text(src.replace(orig, planted))
    shutil.copytree(os.path.join(ROOT, "synth"), tmp_path / "synth",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (tmp_path / "tests").mkdir()
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=tmp_path, capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 1, f"no pin fails with '{name}':\n{r.stdout[-1500:]}"
