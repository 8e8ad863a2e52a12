"""Writes tests/golden/templates.json: the random tuning-space templates of
the batched workloads, chosen by rejection sampling on their number of VALID
configurations.

For every random template t of a family (``ffg_inputs.TEMPLATE_FAMILIES``),
candidates k = 0, 1, ... are drawn with ``ffg_inputs.template_candidate``
at a raw size of target / (valid fraction seen so far); a candidate is
accepted when it has 3 to 10 parameters and its valid count, computed by the
CPU oracle's constraint mask, lies within +-20 % of the template's
log-uniform target.  The table records the accepted candidate index, its
raw-size target and its valid count.  Only the oracle decides validity; the
CUDA library is not used.

    python tests/golden/make_templates.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ffg_inputs as fi  # noqa: E402
import oracle  # noqa: E402

MAX_RAW = (1 << 31) - 1


def choose(family: str, t: int, target: float):
    frac = 0.5
    for k in range(10000):
        raw = max(2, int(round(target / frac)))
        sp = fi.template_candidate(family, t, k, raw)
        if not 3 <= sp.n_params <= 10 or sp.n_raw > MAX_RAW:
            continue
        n = int(oracle.valid_mask(sp).sum())
        if n > 0:
            frac = min(1.0, 0.5 * frac + 0.5 * n / sp.n_raw)
        if abs(n - target) <= fi.VALID_TOL * target:
            return {"k": k, "raw_target": raw, "n_raw": sp.n_raw, "n_valid": n,
                    "target": round(float(target), 3)}
    raise RuntimeError(f"{family} template {t}: no candidate within the tolerance")


def main():
    oracle.compile_oracle()
    table = {}
    for family in fi.TEMPLATE_FAMILIES:
        rows = []
        for t, target in enumerate(fi.valid_targets(family)):
            rows.append(choose(family, t, float(target)))
            print(family, t, rows[-1], flush=True)
        table[family] = rows
    with open(fi.TEMPLATE_TABLE, "w") as fh:
        json.dump(table, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
