"""The batched workloads' templates: the table that tests/golden/make_templates.py
wrote with the oracle still describes the spaces that ffg_inputs builds, and
every template meets the workload's shape (3-10 parameters, valid size within
+-20 % of its log-uniform target, targets inside the family's range)."""
import json

import numpy as np
import pytest

import ffg_inputs as fi
import oracle


@pytest.fixture(scope="module")
def table():
    oracle.compile_oracle()
    with open(fi.TEMPLATE_TABLE) as fh:
        return json.load(fh)


@pytest.mark.parametrize("family", sorted(fi.TEMPLATE_FAMILIES))
def test_template_table_matches_oracle(table, family):
    seed, count, lo, hi = fi.TEMPLATE_FAMILIES[family]
    rows = table[family]
    targets = fi.valid_targets(family)
    assert len(rows) == count == len(targets)
    assert np.all((targets >= lo) & (targets <= hi))
    prefix = "template" if family == "batch" else "sweep"
    specs = fi.family_templates(family, prefix)
    for t, (row, sp, target) in enumerate(zip(rows, specs, targets)):
        assert 3 <= sp.n_params <= 10, (family, t)
        assert sp.n_raw == row["n_raw"], (family, t)
        n = int(oracle.valid_mask(sp).sum())
        assert n == row["n_valid"], (family, t, n, row["n_valid"])
        assert abs(n - target) <= fi.VALID_TOL * target, (family, t, n, target)


def test_targets_are_stratified_log_uniform():
    """One target per equal slice of the log range (so the batch's total size
    is near its expectation)."""
    for family, (seed, count, lo, hi) in fi.TEMPLATE_FAMILIES.items():
        u = np.log(fi.valid_targets(family) / lo) / np.log(hi / lo)
        assert sorted(np.floor(u * count).astype(int).tolist()) == list(range(count))


def test_batch_workload_shape():
    work = fi.batch_workload()
    assert len(work) == 26 * 9
    names = [sp.name for sp, _, _ in work]
    assert names[0] == "convolution" and names[9] == "gemm" and names[18] == "pnpoly"
    assert sorted({f for _, _, f in work}) == [0.03, 0.30, 0.70]
    assert len({(sp.name, s) for sp, s, _ in work}) == 234
    kinds = {c.kind for sp in fi.batch_templates() for c in sp.clauses}
    assert {"prod_le", "prod_ge", "divides"} <= kinds
