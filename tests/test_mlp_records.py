"""The MLP's training records and instance families (host logic, no GPU):
the families' instances follow their documented ranges and are reproducible
from their seeds, the committed records are the method's runs on exactly
those instances, and the training set built from them has one label per
instance with a complete run."""
import glob
import os

import numpy as np
import pytest

from paper_1510_04895_gb300 import mlp_train

DATA = os.path.join(os.path.dirname(mlp_train.__file__), "data")


@pytest.mark.parametrize("family", mlp_train.FAMILIES)
def test_instance_families_follow_their_ranges(family):
    for k in range(40):
        a, b = mlp_train.instance(k, family), mlp_train.instance(k, family)
        assert a == b                                    # reproducible
        if family == "small":
            assert 6 <= a["L"] <= 8 and 4 <= a["Lz"] <= 8 and 0.3 <= a["W"] <= 2.5
            assert 6 <= a["NT"] <= 30 and a["seed"] == 7000 + k
        elif family == "ensemble":
            assert 10 <= a["L"] <= 12 and a["Lz"] == a["L"] and 0.2 <= a["W"] <= 2.0
            assert a["delta"] == 0.05 and a["seed"] == 20000 + k
        else:
            assert a["L"] == 2 * a["Lz"] and 5 <= a["Lz"] <= 7 and 10 <= a["NT"] <= 60
            assert a["W"] == (1.0 if family == "medium_shape" else 0.5)
    seeds = {mlp_train.instance(k, f)["seed"] for f in mlp_train.FAMILIES for k in range(40)}
    assert len(seeds) == 4 * 40                          # no instance shared by two families


def test_window_of_fixed_or_sized():
    eigs = np.concatenate([-np.arange(1, 41) * 0.01, np.arange(1, 41) * 0.01])
    assert mlp_train.window_of({"delta": 0.05, "NT": 0}, eigs) == 0.05
    d = mlp_train.window_of({"NT": 20}, eigs)
    assert 16 <= np.sum(np.abs(eigs) <= d) <= 28


def test_committed_records_match_their_instances():
    paths = sorted(glob.glob(os.path.join(DATA, "mlp_records*.jsonl")))
    assert len(paths) == 4
    total = 0
    for p in paths:
        recs = mlp_train.load_records(p)
        total += len(recs)
        for rec in recs:
            inst = rec["instance"]
            fam = inst.get("family", "small")
            assert inst == mlp_train.instance(inst["k"], fam)
            assert len(rec["features"]) == mlp_train.N_IN
            assert len(rec["runs"]) == len(mlp_train.NP_FACTORS) * len(mlp_train.NS_FACTORS) * \
                len(mlp_train.KERNELS)
            assert rec["n_target_exact"] >= 1
            for run in rec["runs"]:
                assert run["cost"] == mlp_train.cost_of(run["iterations"], run["ns"], run["Np"])
                assert not run["correct"] or run["converged"]
    assert total == 240
    X, T = mlp_train.dataset([r for p in paths for r in mlp_train.load_records(p)])
    assert X.shape[1] == mlp_train.N_IN and T.shape[1] == 3 and 200 <= len(X) <= 240
    assert set(np.unique(T[:, 2])) <= {0.0, 1.0}
