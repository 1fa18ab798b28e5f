"""The prediction-setting split generator (Sec. 2: settings 1-4) on the CPU.

* setting 1 holds out random pairs, and every object is seen in training;
* setting 2 (3) holds out drugs (targets): no test drug (target) is a training one, and the
  other side is shared;
* setting 4 holds out both: a test pair has a new drug and a new target, and no training pair
  touches either;
* ids are dense on both sides, and every test pair maps back to an original pair.
"""
import numpy as np
import pytest

from paper_2009_01054_gb300 import synth


def _rows(X):
    return {tuple(np.round(r, 12)) for r in X}


@pytest.mark.parametrize("setting", [1, 2, 3, 4])
def test_setting_split_semantics(setting):
    p = synth.merget(0, m=120, q=50, dim=6, n=2400)
    sp = synth.setting_split(p, setting, test_frac=0.3, seed=1)
    assert sp.d.max() < len(sp.Xd_train) and sp.t.max() < len(sp.Xt_train)
    assert sp.d_test.max() < len(sp.Xd_test) and sp.t_test.max() < len(sp.Xt_test)
    orig = {(tuple(np.round(p.Xd[a], 12)), tuple(np.round(p.Xt[b], 12))) for a, b in zip(p.d, p.t)}
    train = {(tuple(np.round(sp.Xd_train[a], 12)), tuple(np.round(sp.Xt_train[b], 12))) for a, b in zip(sp.d, sp.t)}
    test = {(tuple(np.round(sp.Xd_test[a], 12)), tuple(np.round(sp.Xt_test[b], 12)))
            for a, b in zip(sp.d_test, sp.t_test)}
    assert train <= orig and test <= orig and not (train & test)
    dtr, ttr = _rows(sp.Xd_train), _rows(sp.Xt_train)
    dte, tte = _rows(sp.Xd_test), _rows(sp.Xt_test)
    if setting == 1:
        assert len(train) + len(test) == p.n and dte == dtr and tte == ttr
    if setting == 2:
        assert not (dte & dtr) and tte == ttr and len(train) + len(test) == p.n
    if setting == 3:
        assert not (tte & ttr) and dte == dtr and len(train) + len(test) == p.n
    if setting == 4:
        assert not (dte & dtr) and not (tte & ttr) and len(train) + len(test) < p.n
    assert len(test) > 0 and len(train) > 0
