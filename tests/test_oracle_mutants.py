"""Mutation check of the oracle's pins.

Each case plants one plausible mistake (a dropped term, a wrong sign, index,
order or conjugate) in a copy of oracle/oracle.c, builds that copy with gcc
and runs the pin file that covers the mutated function against it: at least
one pin must fail.  An unmodified copy must pass the same files (the control).
CPU only; nothing here touches the CUDA library.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DIRAC, SAP, SOLVER, SEC22 = ("test_oracle_dirac.py", "test_oracle_sap.py", "test_oracle_solver.py",
                             "test_oracle_clover_ssor.py")

# (name, text in oracle.c, replacement (first occurrence), pin file)
MUTANTS = [
    # Wilson-Dirac operator, Sec. 2.1
    ("D: spin projector signs swapped", "const double sgn = (dir > 0) ? -1.0 : 1.0;",
     "const double sgn = (dir > 0) ? 1.0 : -1.0;", DIRAC),
    ("D: backward link not daggered", "(dir > 0) ? Ulink[a * 3 + b] : conj(Ulink[b * 3 + a])",
     "(dir > 0) ? Ulink[a * 3 + b] : conj(Ulink[a * 3 + b])", DIRAC),
    ("D: backward link taken at x", ": U + (nb * 4 + mu) * 9;", ": U + (s * 4 + mu) * 9;", DIRAC),
    ("D: no phase on the forward t wrap", "if (n[mu] == d[mu]) { n[mu] = 0; if (mu == 3) *phase = -1.0; }",
     "if (n[mu] == d[mu]) { n[mu] = 0; }", DIRAC),
    ("D: sign of kappa", "o[k] = phis[k] - kappa * eta[k];", "o[k] = phis[k] + kappa * eta[k];", DIRAC),
    # SAP with MR domain solves, Sec. 2.2
    ("SAP: MR numerator not conjugated", "num[(long)dd * L + i] += conj(q[k]) * r[k];",
     "num[(long)dd * L + i] += q[k] * r[k];", SAP),
    ("SAP: MR solution updated with q", "x[k] += om * r[k];", "x[k] += om * q[k];", SAP),
    ("SAP: residual of the other colour", "mask_colour(dims, block, colour, r, L);",
     "mask_colour(dims, block, 1 - colour, r, L);", SAP),
    ("SAP: one cycle too many", "for (int cyc = 0; cyc < ncycle; ++cyc) {",
     "for (int cyc = 0; cyc <= ncycle; ++cyc) {", SAP),
    # the frozen step-length table (the stationary preconditioner of Sec. 2.1)
    ("SAP frozen: one table entry for every cycle", "table + (((long)cyc * 2 + colour) * nmr + it) * nd + dd",
     "table + (((long)0 * 2 + colour) * nmr + it) * nd + dd", SAP),
    ("SAP frozen: one table entry for every MR step", "table + (((long)cyc * 2 + colour) * nmr + it) * nd + dd",
     "table + (((long)cyc * 2 + colour) * nmr + 0) * nd + dd", SAP),
    ("SAP frozen: recorded where the residual is zero", "if (mr_mode == 2 && d_sum > 0) *tab = om;",
     "if (mr_mode == 2) *tab = om;", SAP),
    ("SAP frozen: the replay ignores the table", "if (mr_mode == 2 && !isnan(creal(*tab))) {",
     "if (0 && mr_mode == 2 && !isnan(creal(*tab))) {", SAP),
    # QR and L x L solves, Sec. 2.1
    ("QR: projection conjugated on the wrong side", "s += conj(A[n * L + i]) * A[n * L + j];",
     "s += A[n * L + i] * conj(A[n * L + j]);", SOLVER),
    ("QR: columns not normalised", "P[n * L + j] /= nrm;", "P[n * L + j] /= 1.0;", SOLVER),
    ("QR: gamma diagonal not stored", "if (gm) gm[j * L + j] = nrm;", "if (gm) gm[j * L + j] = 1.0;",
     SOLVER),
    ("LU: no pivot search", "if (cabs(A[r * L + k]) > best)", "if (0 && cabs(A[r * L + k]) > best)",
     SOLVER),
    ("LU: back substitution sign", "s -= A[k * L + j] * C[j * M + c];", "s += A[k * L + j] * C[j * M + c];",
     SOLVER),
    # Algorithm 1
    ("Alg 1: sign of V alpha", "T[n] = R[n] - W[n];", "T[n] = R[n] + W[n];", SOLVER),
    ("Alg 1: zeta conjugated", "block_gram(Z, T, N, L, gzt);", "block_gram(T, Z, N, L, gzt);", SOLVER),
    ("Alg 1: sign of beta", "for (int q = 0; q < L * L; ++q) beta[q] = -beta[q];",
     "for (int q = 0; q < L * L; ++q) beta[q] = beta[q];", SOLVER),
    ("Alg 1: sign of zeta V in P", "T[n] = P[n] - zeta * Vb[n];", "T[n] = P[n] + zeta * Vb[n];", SOLVER),
    ("Alg 1: zeta S missing from X", "X[n] += W[n] + zeta * S[n];", "X[n] += W[n];", SOLVER),
    ("Alg 1: no preconditioner on T", "apply_M(dims, Ud, kappa, &pc, T, S, L, NL);",
     "memcpy(S, T, sizeof(cplx) * NL);", SOLVER),
    ("Alg 1: no QR of P", "if (oracle_qr_mgs((double*)P, N, L, NULL) != 0) { status = 2; break; }",
     "", SOLVER),
    # SSOR, clover, Jacobi preconditioning, Sec. 2.2
    ("SSOR: L substituted in increasing order", "sites[which == 1 ? n - 1 - m : m]", "sites[m]", SEC22),
    ("SSOR: U substituted in decreasing order", "sites[which == 1 ? n - 1 - m : m]", "sites[n - 1 - m]", SEC22),
    ("SSOR: sign of omega - 2", "(c->omega - 2.0) * pqv[e]", "(c->omega + 2.0) * pqv[e]", SEC22),
    ("SSOR: product of inverses in the wrong order",
     "ssor_triangular(c, sites, n, 1, qv, pqv, h, w, th);",
     "ssor_triangular(c, sites, n, 2, pv, pqv, h, w, th);", SEC22),
    ("SSOR: one term short", "for (int j = 1; j <= nssor; ++j) {", "for (int j = 1; j < nssor; ++j) {", SEC22),
    ("SSOR: final U substitution missing", "ssor_triangular(c, sites, n, 2, acc, out, h, w, th);",
     "for (long m = 0; m < n; ++m) for (long k = 0; k < len; ++k) out[sites[m] * len + k] = acc[sites[m] * len + k];",
     SEC22),
    ("SSOR: T^{-1} ignored", "if (c->Tinv) { site_matrix_apply", "if (0) { site_matrix_apply", SEC22),
    ("SSOR: omega missing in the substitution", "y[s * len + k] + c->omega * c->kappa * hh[k]",
     "y[s * len + k] + c->kappa * hh[k]", SEC22),
    ("SAP-SSOR: residual not updated", "for (long k = 0; k < NL; ++k) r[k] = eta[k] - r[k];\n      ssor_colour",
     "for (long k = 0; k < NL; ++k) r[k] = eta[k];\n      ssor_colour", SEC22),
    ("clover: Q + Q^dagger", "(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0", "(Q[a * 3 + b] + conj(Q[b * 3 + a])) / 8.0",
     SEC22),
    ("clover: dagger without transpose", "(Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0",
     "(Q[a * 3 + b] - conj(Q[a * 3 + b])) / 8.0", SEC22),
    ("clover: 1/4 instead of 1/8", "/ 8.0;", "/ 4.0;", SEC22),
    ("clover: sign of sigma", "sigma[mu][nu][r][c] = 0.5 * I * comm;", "sigma[mu][nu][r][c] = -0.5 * I * comm;",
     SEC22),
    ("clover: leaf 2 link not daggered", "const int d2[4] = {0, 1, 1, 0};", "const int d2[4] = {0, 0, 1, 0};", SEC22),
    ("clover: leaf 3 links swapped", "const cplx* l3[4] = {U + (xm * 4 + mu) * 9, U + (xmn * 4 + nu) * 9,",
     "const cplx* l3[4] = {U + (xmn * 4 + nu) * 9, U + (xm * 4 + mu) * 9,", SEC22),
    ("clover: leaf 4 link at the wrong site", "U + (xpd * 4 + nu) * 9, U + (s * 4 + mu) * 9}",
     "U + (xp * 4 + nu) * 9, U + (s * 4 + mu) * 9}", SEC22),
    ("clover: leaf 4 dropped", "loop4(l4, d4, w); for (int k = 0; k < 9; ++k) Q[k] += w[k];", "loop4(l4, d4, w);",
     SEC22),
    ("clover: factor i missing", "+= I * kappa * csw * sg", "+= kappa * csw * sg", SEC22),
    ("Jacobi: T^{-1} not applied", "site_matrix_apply(Ti + s * 144, eta, L, h);",
     "memcpy(h, eta, sizeof(cplx) * 12 * L);", SEC22),
    ("clover D: T missing", "out[s * 12L * L + k] = tp[k] - kappa * eta[k];",
     "out[s * 12L * L + k] = in[s * 12L * L + k] - kappa * eta[k];", SEC22),
]


def _run_copy(workdir, source, pin_file, threads):
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(workdir, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutants.py"))
    for d in ("synth", "oracle"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(workdir, d),
                        ignore=shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__"))
    with open(os.path.join(workdir, "oracle", "oracle.c"), "w") as f:
        f.write(source)
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", os.path.join("tests", pin_file)],
                       cwd=workdir, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(os.path.join(ROOT, "oracle", "oracle.c")) as f:
        src = f.read()
    for name, old, _new, _pin in MUTANTS:
        assert old in src, f"mutation pattern no longer in oracle.c: {name}"
    workers = max(4, os.cpu_count() or 4)
    threads = max(1, (os.cpu_count() or 4) // workers)

    # the controls (the unmodified oracle on every pin file used below) and the
    # mutants in one pool
    pins = sorted({m[3] for m in MUTANTS})
    jobs = [("control " + pin, src, pin) for pin in pins] + \
           [(name, src.replace(old, new, 1), pin) for name, old, new, pin in MUTANTS]

    def one(k):
        name, source, pin = jobs[k]
        rc, out = _run_copy(str(tmp_path / f"j{k:02d}"), source, pin, threads)
        return name, rc, out

    with ThreadPoolExecutor(workers) as ex:
        done = list(ex.map(one, range(len(jobs))))
    for name, rc, out in done[:len(pins)]:
        assert rc == 0, f"unmodified oracle fails its pins ({name}):\n{out}"
    results = done[len(pins):]
    missed = [n for n, rc, _ in results if rc == 0]
    broken = [(n, out) for n, rc, out in results if rc not in (0, 1)]
    assert not broken, f"mutants that did not build or collect: {broken}"
    assert not missed, f"planted mistakes no pin catches: {missed}"
