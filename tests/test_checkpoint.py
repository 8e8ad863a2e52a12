"""Graph checkpoints: an FFG saved as a CSR .npz and loaded back is the same
graph (host tensors here; the GPU round trip is in the parity tests)."""
import numpy as np
import pytest

import ffg_inputs as fi
import oracle

torch = pytest.importorskip("torch")
ffg = pytest.importorskip("paper_2210_01465_gb300")


def _host_graph(og):
    g = ffg.Graph(og.n_raw, og.n_nodes, og.n_edges, int(og.is_min.sum()), og.f_opt, "cpu")
    e = og.n_edges
    g.out_ptr.copy_(torch.from_numpy(og.out_ptr.astype(np.int64)))
    g.in_ptr.copy_(torch.from_numpy(og.in_ptr.astype(np.int64)))
    g.out_idx[:e].copy_(torch.from_numpy(og.out_idx.astype(np.int32)))
    g.in_idx[:e].copy_(torch.from_numpy(og.in_idx.astype(np.int32)))
    g.outdeg.copy_(torch.from_numpy(og.outdeg.astype(np.int32)))
    g.node_raw.copy_(torch.from_numpy(og.node_raw.astype(np.int64)))
    g.is_min.copy_(torch.from_numpy(og.is_min.astype(np.uint8)))
    return g


@pytest.mark.parametrize("nbh", [oracle.HAMMING, oracle.ADJACENT])
def test_graph_checkpoint_round_trip(tmp_path, nbh):
    spec = fi.pnpoly_space()
    og = oracle.build(spec, fi.runtimes(spec, 4, fail_frac=0.3), nbh)
    g = _host_graph(og)
    g.nbh = nbh
    path = tmp_path / "ffg.npz"
    g.save(path)
    h = ffg.load_graph(path, device="cpu")
    assert (h.n_raw, h.n_nodes, h.n_edges, h.n_minima, h.f_opt, h.nbh) == \
        (og.n_raw, og.n_nodes, og.n_edges, int(og.is_min.sum()), og.f_opt, nbh)
    e = og.n_edges
    np.testing.assert_array_equal(h.out_ptr.numpy(), og.out_ptr)
    np.testing.assert_array_equal(h.in_ptr.numpy(), og.in_ptr)
    np.testing.assert_array_equal(h.out_idx[:e].numpy(), og.out_idx)
    np.testing.assert_array_equal(h.in_idx[:e].numpy(), og.in_idx)
    np.testing.assert_array_equal(h.outdeg.numpy(), og.outdeg)
    np.testing.assert_array_equal(h.node_raw.numpy(), og.node_raw)
    np.testing.assert_array_equal(h.is_min.numpy().astype(bool), og.is_min)
    # the struct handed to the library points at the loaded tensors
    assert h.c.out_ptr == h.out_ptr.data_ptr() and h.c.in_idx == h.in_idx.data_ptr()


def test_graph_checkpoint_refuses_mismatched_arrays(tmp_path):
    spec = fi.single_small()
    og = oracle.build(spec, fi.runtimes(spec, 2), oracle.HAMMING)
    g = _host_graph(og)
    path = tmp_path / "ffg.npz"
    g.save(path)
    with np.load(path) as z:
        d = {k: z[k] for k in z.files}
    d["outdeg"] = d["outdeg"][:-1]          # one out-degree short
    bad = tmp_path / "bad.npz"
    np.savez(bad, **d)
    with pytest.raises(ValueError):
        ffg.load_graph(bad, device="cpu")
