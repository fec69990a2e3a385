"""The FP32 factor check of ``parity.fp32_factor_check`` on the CPU: the FP64
oracle's factors rounded to FP32 pass it (they are an FP32 factorization with
one rounding per entry); a factor entry perturbed far beyond FP32 rounding, or
an update left out, fails it."""
import numpy as np

import oracle
import synth
from parity import fp32_factor_check, update_counts


def _case():
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    v = m.values(5)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    return m, v, f


def test_rounded_oracle_factors_pass():
    m, v, f = _case()
    r = fp32_factor_check(m.n, m.colptr, m.rowidx, v, m.perm, f.lu_colptr, f.lu_rowidx,
                          f.lu_val.astype(np.float32).astype(np.float64), f.lu_val)
    assert r["backward_worst"] <= 1.0 and r["forward_within"] == 1.0, r
    assert r["forward_worst_rel"] <= 2.0 ** -24 and r["clean_entries"] >= 0.75 * r["entries"]


def test_planted_mistakes_fail():
    m, v, f = _case()
    got = f.lu_val.astype(np.float32).astype(np.float64)
    # an entry with few updates (a tight bound) and the largest magnitude among them
    c = update_counts(f.lu_colptr, f.lu_rowidx)
    few = np.nonzero(c <= 4)[0]
    q = int(few[np.argmax(np.abs(f.lu_val[few]))])
    bad = got.copy()
    bad[q] *= 1.0 + 1e-4
    r = fp32_factor_check(m.n, m.colptr, m.rowidx, v, m.perm, f.lu_colptr, f.lu_rowidx, bad, f.lu_val)
    assert r["backward_worst"] > 1.0 and r["forward_within"] < 1.0, r
    # the factors of other values (a whole refactorization missed) fail too
    other = f.factor(m.values(6)).astype(np.float32).astype(np.float64)
    r = fp32_factor_check(m.n, m.colptr, m.rowidx, v, m.perm, f.lu_colptr, f.lu_rowidx, other, f.lu_val)
    assert r["backward_worst"] > 1.0, r
