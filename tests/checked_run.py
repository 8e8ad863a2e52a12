"""Child process of test_gpu_checked.py: runs the library's paths on a few
seeded spaces and prints their results as one JSON line.

With FFG_LIB=checked it loads the bounds-checked build and also reports the
failed-check record, first after the clean runs (expected empty), then after
runs on graphs with planted out-of-range indices (expected: counted, first
site code reported, no fault)."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import ffg_inputs as fi  # noqa: E402
import paper_2210_01465_gb300 as ffg  # noqa: E402

P = [0.01, 0.05, 0.1]


def _digest(t):
    a = t.detach().cpu().numpy()
    return [float(np.asarray(a, dtype=np.float64).sum()), hashlib.sha256(a.tobytes()).hexdigest()]


def clean_runs(dev):
    out = {}
    specs = [fi.single_small(), fi.conv_space(), fi.gemm_space(), fi.pnpoly_space()]
    fits = [fi.runtimes_torch(sp, 31 + i, 0.05, device=dev) for i, sp in enumerate(specs)]
    graphs = []
    for sp, f in zip(specs, fits):
        s = ffg.Space.from_spec(sp)
        for nbh in (ffg.HAMMING, ffg.ADJACENT):
            g = ffg.build_graph(s, f, nbh)
            graphs.append((g, f))
            key = f"{sp.name}/{nbh}"
            out[key + "/graph"] = [g.n_nodes, g.n_edges, g.n_minima,
                                   _digest(g.in_idx[:g.n_edges]), _digest(g.out_idx[:g.n_edges])]
            for prec in (ffg.F64, ffg.F32):
                x, it, _, _ = ffg.pagerank(g, 0.85, 1e-12, 10000, prec)
                out[f"{key}/pr{prec}"] = [it, _digest(x),
                                          ffg.centrality(g, f, x, P).tolist()]
            xd, lv = ffg.dag(g, 0.85)
            out[key + "/dag"] = [lv, _digest(xd)]
            c, steps = ffg.walks(g, 7, 4096)
            out[key + "/walks"] = [steps, _digest(c)]
            fr, nd = ffg.minima_fraction(g, f)
            out[key + "/minima"] = [_digest(fr), _digest(nd)]
    bb = ffg.BuildBatch([(ffg.Space.from_spec(sp), f, ffg.HAMMING) for sp, f in zip(specs, fits)])
    pb = ffg.PageRankBatch([(g, 0.85) for g in bb.graphs], prec=ffg.F32, tol=1e-12)
    cb = ffg.CentralityBatch([(g, f, x) for g, f, x in zip(bb.graphs, fits, pb.ranks)], P)
    sb = ffg.SpaceBatch(pb, bb, cb)
    for _ in range(2):
        sb.run()
    it, _, st = pb.query()
    cp, _ = cb.query()
    out["batch"] = [it.tolist(), st.tolist(), np.asarray(cp).tolist(),
                    [_digest(x) for x in pb.ranks]]
    torch.cuda.synchronize(dev)
    return out, graphs


def planted_runs(graphs):
    """Out-of-range indices planted in copies of the graphs' arrays: each
    guarded access must be skipped and counted with its site code."""
    rec = {}
    g, f = graphs[0]
    n, e = g.n_nodes, g.n_edges
    # PageRank: in-neighbours past the end of w and below its start
    saved = g.in_idx.clone()
    g.in_idx[e // 3] = n + 1000
    g.in_idx[e // 2] = -7
    ffg.ffg_checked_failures(reset=True)
    x, it, _, _ = ffg.pagerank(g, 0.85, 1e-12, 200, ffg.F32)
    torch.cuda.synchronize()
    rec["pagerank"] = ffg.ffg_checked_failures(reset=True)
    rec["pagerank_finite"] = bool(torch.isfinite(x).all())
    g.in_idx.copy_(saved)
    # C_p: a minimum whose raw point lies past the fitness vector
    saved = g.node_raw.clone()
    mins = torch.nonzero(g.is_min).flatten()
    g.node_raw[mins[0]] = g.n_raw + 5
    x, _, _, _ = ffg.pagerank(g, 0.85, 1e-12, 10000, ffg.F64)
    try:        # with the only minimum skipped the space holds no minimum mass
        ffg.centrality(g, f, x, P)
    except ffg.FFGError:
        pass
    torch.cuda.synchronize()
    rec["centrality"] = ffg.ffg_checked_failures(reset=True)
    g.node_raw.copy_(saved)
    # walks: every out-neighbour past the last node
    saved = g.out_idx.clone()
    g.out_idx[:e] = n + 3
    try:
        ffg.walks(g, 7, 256)
        rec["walks_status"] = "ok"
    except ffg.FFGError as exc:
        rec["walks_status"] = str(exc)[:80]
    torch.cuda.synchronize()
    rec["walks"] = ffg.ffg_checked_failures(reset=True)
    g.out_idx.copy_(saved)
    rec["after"] = ffg.ffg_checked_failures()
    return rec


def main():
    dev = torch.device("cuda:0")
    ffg.build(checked=os.environ.get("FFG_LIB") == "checked")
    checked = ffg.ffg_checked_build()
    if checked:
        ffg.ffg_checked_failures(reset=True)
    out, graphs = clean_runs(dev)
    res = {"checked": checked, "results": out}
    if checked:
        res["clean_failures"] = ffg.ffg_checked_failures()
        res["planted"] = planted_runs(graphs)
    print("RESULT " + json.dumps(res))


if __name__ == "__main__":
    main()
