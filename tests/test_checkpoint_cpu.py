"""Checkpoint bookkeeping (CPU): finished replication ranges, the missing
ones, overlap and count checks, a JSON round trip, and the merge of the
recorded triples in replication order (the engine's host merge, checked
against a two-pass computation)."""
import numpy as np
import pytest


def _engine():
    import paper_1501_01405_gb300 as eng
    try:
        eng.lib()
    except eng.MripLibraryMissing:
        from paper_1501_01405_gb300 import build
        build.build()
        eng.lib()
    return eng


def _triples(x):
    return np.array([[r.size, r.mean(), ((r - r.mean()) ** 2).sum()] for r in x])


def test_ranges_missing_merge_and_round_trip(tmp_path):
    eng = _engine()
    from paper_1501_01405_gb300.checkpoint import Checkpoint
    rng = np.random.default_rng(3)
    data = rng.normal(2.0, 1.5, size=(3, 100))  # stand-in outputs of 3 design points
    c = Checkpoint(eng.MRIP_MM1, {"n_clients": 10}, [[0.5, 1.0]] * 3, 100, 42)
    assert c.missing() == [(0, 100)] and not c.complete()
    c.add(30, 55, _triples(data[:, 30:55]))
    c.add(0, 10, _triples(data[:, 0:10]))
    assert c.missing() == [(10, 30), (55, 100)]
    with pytest.raises(ValueError):
        c.add(50, 60, _triples(data[:, 50:60]))  # overlaps [30, 55)
    with pytest.raises(ValueError):
        c.add(60, 70, _triples(data[:, 60:69]))  # 9 replications counted for a range of 10
    with pytest.raises(ValueError):
        c.add(90, 101, _triples(data[:, 90:100]))
    path = str(tmp_path / "ck.json")
    c.save(path)
    d = Checkpoint.load(path)
    assert d.missing() == c.missing() and d.seed == 42 and d.params == {"n_clients": 10}
    d.add(10, 30, _triples(data[:, 10:30]))
    d.add(55, 100, _triples(data[:, 55:100]))
    assert d.complete() and d.missing() == []
    m = d.merged()
    ref = _triples(data)
    assert np.array_equal(m[:, 0], ref[:, 0])
    np.testing.assert_allclose(m[:, 1:], ref[:, 1:], rtol=1e-13)
