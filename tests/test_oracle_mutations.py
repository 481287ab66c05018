"""Planted mistakes in the oracle, on the CPU: each mutation below is applied
to a temporary copy of oracle/ (with tests/ and workloads/ beside it) and the
pins that guard that part must then fail, while the unchanged copy passes
them.  This is what shows that the pins of test_oracle_pins.py,
test_kpoint_pins.py and test_lrdma_pins.py would catch a dropped term, a
wrong constant, a wrong sign, index or conjugate in the oracle -- not only
that the oracle agrees with itself."""

import concurrent.futures
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join("oracle", "lrdm_oracle.py")

CORE = "tests/test_oracle_pins.py"
KPOINT = "tests/test_kpoint_pins.py"
LRDMA = "tests/test_lrdma_pins.py"

# name: (text in the oracle, replacement, pin file)
MUTATIONS = {
    # the response and its inputs (§II.C, Eqs. jacobian, densityResponse, subspaceDensityMatResponse)
    "dropped mu'": ("dmu[k] = dmu_shift(L, X)", "dmu[k] = 0.0", CORE),
    "f_x constant 1/2": ("return -(c / 3.0) * r ** (-2.0 / 3.0)", "return -(c / 2.0) * r ** (-2.0 / 3.0)", CORE),
    "Hartree 2 pi": ("sym = np.where(g2 > 0.0, 4.0 * np.pi / np.where(g2 > 0.0, g2, 1.0), 0.0)",
                     "sym = np.where(g2 > 0.0, 2.0 * np.pi / np.where(g2 > 0.0, g2, 1.0), 0.0)", CORE),
    "Loewner 2 kT": ("val_direct = -sinhc / (4.0 * kT * np.cosh", "val_direct = -sinhc / (2.0 * kT * np.cosh", CORE),
    "sinhc argument": ("u = 0.5 * (xi - xj)", "u = (xi - xj)", CORE),
    "dropped g": ('return g * np.einsum("ri,ri->r", psi @ Xp, psi)', 'return np.einsum("ri,ri->r", psi @ Xp, psi)',
                  CORE),
    "spin Hartree of one channel": (
        "vh = hartree(sum(np.asarray(v, dtype=np.float64) for v in v_channels), n, h, kind)",
        "vh = hartree(np.asarray(v_channels[0], dtype=np.float64), n, h, kind)", CORE),
    # least squares (Eqs. plowrank, relativeError)
    "LS Gram without w": ("S = w * (Fm @ Fm.T)", "S = (Fm @ Fm.T)", CORE),
    # adjoint
    "adjoint without the mu' term": ("Ybar = L[s] * Gbar[s] - np.diag(np.diag(L[s])) * (T / s_sum)",
                                     "Ybar = L[s] * Gbar[s]", CORE),
    "Lbar without the trace term": ("Lbar[s] -= np.diag((T / s_sum) * (np.diag(X) - dmu))", "Lbar[s] -= 0.0", CORE),
    "eps_bar sign": ("eb = np.sum(np.where(far, sym * (-L[s] * inv), 0.0), axis=1)",
                     "eb = np.sum(np.where(far, sym * (L[s] * inv), 0.0), axis=1)", CORE),
    "occ_bar sign": ("ob = np.sum(np.where(far, sym * inv, 0.0), axis=1)",
                     "ob = np.sum(np.where(far, -sym * inv, 0.0), axis=1)", CORE),
    # Brillouin-zone sampling (§II.C closing paragraphs, Eq. tracelessCondition)
    "k-points: conjugate on the wrong side": ('np.einsum("ri,ri->r", psi @ G, psi.conj())',
                                              'np.einsum("ri,ri->r", psi.conj() @ G, psi)', KPOINT),
    "k-points: mu' per point": (
        "G = Lk * (Xk - dmu[k] * np.eye(Xk.shape[0]))",
        "G = Lk * (Xk - float(np.dot(np.diag(Lk), np.diag(Xk).real) / np.sum(np.diag(Lk))) * np.eye(Xk.shape[0]))",
        KPOINT),
    "k-points: unweighted mu' numerator": ("num = sum(wk * float", "num = sum(1.0 * float", KPOINT),
    "k-points: transposed X": ("Xk = psi.conj().T @ ((w * dVk)[:, None] * psi)",
                               "Xk = psi.T @ ((w * dVk)[:, None] * psi.conj())", KPOINT),
    # the accumulated step's decisions (§II.B.1, Eqs. linearapprox, linearityIndicator, accum)
    "LRDMA: inverted beta ratio": (
        "beta = abs(float(np.sqrt(w * np.sum(state.R_lin * state.R_lin))) / r_norm - 1.0)",
        "beta = abs(r_norm / float(np.sqrt(w * np.sum(state.R_lin * state.R_lin))) - 1.0)", LRDMA),
    "LRDMA: R_lin without alpha": ("state.R_lin = Rm - alpha * np.tensordot", "state.R_lin = Rm - 1.0 * np.tensordot",
                                   LRDMA),
    "LRDMA: first new direction from t": (
        "u = Rm / r_norm if fresh else _orthonormalise(Rm, state.U, w)",
        "u = Rm / r_norm if fresh else _orthonormalise(state.T[-1], state.U, w)", LRDMA),
    "LRDMA: orthogonal to the new directions only": (
        "u = _orthonormalise(state.T[-1], state.U, w)",
        "u = _orthonormalise(state.T[-1], state.U[len(state.U) - n_new:], w)", LRDMA),
    "LRDMA: no CT flag": ("            state.clear_next = True\n", "            state.clear_next = False\n", LRDMA),
    "LRDMA: inverted reuse test": ("if s_hist < s_tol:", "if s_hist > s_tol:", LRDMA),
    "LRDMA: r_max_iter off by one": ("max(1, min(r_max_iter, r_max - len(state.U)))",
                                     "max(1, min(r_max_iter + 1, r_max - len(state.U)))", LRDMA),
    "LRDMA: inverted CR test": ("elif r_norm > r_norm_clear:", "elif r_norm < r_norm_clear:", LRDMA),
    "LRDMA: history kept on CL": ('if event in ("CT", "CL", "CR"):', 'if event in ("CT", "CR"):', LRDMA),
    "LRDMA: fit over the new derivatives only": (
        "ls = lrdm_apply(Rm, np.stack(state.U), np.stack(state.T), w, alpha, rcond=rcond,",
        "ls = lrdm_apply(Rm, np.stack(state.U[-max(n_new, 1):] if event == 'accumulate' else state.U), "
        "np.stack(state.T[-max(n_new, 1):] if event == 'accumulate' else state.T), w, alpha, rcond=rcond,",
        LRDMA),
}


def _copy(dst, source=None):
    for sub in ("oracle", "workloads", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(dst, sub),
                        ignore=shutil.ignore_patterns("__pycache__", "*.pyc"))
    if source is not None:
        with open(os.path.join(dst, ORACLE), "w") as fh:
            fh.write(source)


def _run_pins(cwd, pin_file):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
           pin_file]
    if pin_file == CORE:
        cmd += ["-k", "not mpmath"]          # the 50-digit Loewner pin is slow; the others suffice
    r = subprocess.run(cmd, cwd=cwd, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-1500:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(os.path.join(ROOT, ORACLE)) as fh:
        src = fh.read()
    for name, (old, new, _) in MUTATIONS.items():
        assert src.count(old) == 1, f"mutation '{name}' no longer matches the oracle's text"

    jobs = {}
    control = tmp_path / "control"
    _copy(str(control))
    for i, (name, (old, new, pins)) in enumerate(MUTATIONS.items()):
        d = tmp_path / f"m{i}"
        _copy(str(d), src.replace(old, new, 1))
        jobs[name] = (str(d), pins)
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        ctrl = {p: ex.submit(_run_pins, str(control), p) for p in (CORE, KPOINT, LRDMA)}
        futs = {name: ex.submit(_run_pins, d, p) for name, (d, p) in jobs.items()}
        for p, f in ctrl.items():
            rc, out = f.result()
            assert rc == 0, f"unchanged oracle fails {p}:\n{out}"
        survivors = []
        for name, f in futs.items():
            rc, out = f.result()
            # 1 = some pin failed; anything else (2+: the copy did not even collect) is not a catch
            if rc != 1:
                survivors.append(f"{name} (pytest exit {rc}):\n{out}")
    assert not survivors, "planted mistakes not caught:\n" + "\n".join(survivors)
