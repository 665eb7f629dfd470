"""Store of tile colourings (Sec. 3.5): round trips, canonical keys, damaged
or mismatched files refused, invalid colourings refused, atomic writes, and
the lookup glue (tile, hit or colour-and-store, repetition) against a fake
binding whose colourings come from the oracle.  No GPU needed."""
import os
import types

import numpy as np
import pytest

from oracle.colouring import greedy_colour
from oracle import tiles as OT
from paper_2106_01275_gb300 import colour_db as cdb


def _tile_colouring(tile, mu, ps, k, order=0):
    return greedy_colour(tile, mu, ps, k, order)


def test_round_trip_and_canonical_key(tmp_path):
    db = cdb.ColourDB(tmp_path)
    tile, mu, k = [4, 4, 8, 4], 2, 1
    col, m = _tile_colouring(tile, mu, [1, 2], k)
    assert db.get(tile, mu, [1, 2], k, "natural") is None
    path = db.put(tile, mu, [2, 1, 2], k, "natural", col, m)
    for ps in ([1, 2], [2, 1], [-1, 2], [2, 2, 1, -2]):          # one neighbourhood, one key
        got = db.get(tile, mu, ps, k, 0)
        assert got is not None and got[1] == m and np.array_equal(got[0], col)
    assert db.path(tile, mu, [1, 2], k, "natural") == path
    assert db.get(tile, mu, [1, 2], k, "redblack") is None        # other order, other key
    assert db.get(tile, mu, [1], k, "natural") is None
    assert db.get(tile, 1, [1, 2], k, "natural") is None
    assert [f for f in os.listdir(tmp_path) if f.startswith(".tmp_")] == []


def test_damaged_files_are_refused(tmp_path):
    db = cdb.ColourDB(tmp_path)
    tile, mu, k = [4, 4, 4, 6], 3, 1
    col, m = _tile_colouring(tile, mu, [1], k)
    path = db.put(tile, mu, [1], k, "natural", col, m)
    raw = bytearray(open(path, "rb").read())
    bad = bytearray(raw)
    bad[-3] ^= 0x01                                               # one payload bit
    open(path, "wb").write(bytes(bad))
    with pytest.raises(cdb.ColourDBError, match="CRC"):
        db.get(tile, mu, [1], k, "natural")
    open(path, "wb").write(bytes(raw[:-4]))                       # truncated payload
    with pytest.raises(cdb.ColourDBError, match="payload"):
        db.get(tile, mu, [1], k, "natural")
    open(path, "wb").write(bytes(raw[:10]))                       # truncated header
    with pytest.raises(cdb.ColourDBError, match="header"):
        db.get(tile, mu, [1], k, "natural")
    bad = bytearray(raw)
    bad[0:8] = b"NOTACOLR"
    open(path, "wb").write(bytes(bad))
    with pytest.raises(cdb.ColourDBError, match="not a colour store"):
        db.get(tile, mu, [1], k, "natural")
    # a whole file under another key's name
    open(path, "wb").write(bytes(raw))
    other = db.path(tile, mu, [1], 2, "natural")
    os.replace(path, other)
    with pytest.raises(cdb.ColourDBError, match="differs"):
        db.get(tile, mu, [1], 2, "natural")


def test_invalid_colourings_are_not_stored(tmp_path):
    db = cdb.ColourDB(tmp_path)
    tile = [2, 2, 2, 2]
    with pytest.raises(ValueError):
        db.put(tile, 0, [1], 1, "natural", np.zeros(15, np.int32), 1)          # wrong size
    with pytest.raises(ValueError):
        db.put(tile, 0, [1], 1, "natural", np.full(16, 3, np.int32), 3)        # colour >= m
    with pytest.raises(ValueError):
        db.put(tile, 0, [1], 1, "natural", np.full(16, -1, np.int32), 2)       # negative
    with pytest.raises(ValueError):
        db.put(tile, 0, [], 1, "natural", np.zeros(16, np.int32), 1)           # no displacement
    with pytest.raises(ValueError):
        db.put(tile, 0, [1], 1, "diagonal", np.zeros(16, np.int32), 1)         # unknown order
    assert os.listdir(tmp_path) == []


def _fake_binding(calls):
    """ptrace stand-in on the CPU: the oracle's tile policy, greedy colouring
    and tile repetition, numpy arrays for device buffers."""
    def _ps(name, p_list):                    # the library's range check (0 <= p <= 4096)
        if not 1 <= len(p_list) <= 64 or any(not 0 <= int(p) <= 4096 for p in p_list):
            raise RuntimeError("%s: displacement out of range" % name)

    def tile_dims(dims, mu, p_list, k):
        _ps("pt_tile_dims", p_list)
        return list(OT.tile_dims(dims, mu, p_list, k))

    def colour(ctx, dims, mu, p_list, k, order):
        _ps("pt_colour", p_list)
        calls.append(("colour", list(dims), list(p_list), k, order))
        import torch
        c, m = greedy_colour(dims, mu, p_list, k, {"natural": 0, "redblack": 1}.get(order, order))
        return torch.as_tensor(c), m

    def tile_replicate(ctx, tile, tcol, dims, out=None):
        t = np.asarray(tcol).reshape(tile[::-1])
        reps = [d // s for d, s in zip(dims[::-1], tile[::-1])]
        return np.tile(t, reps).reshape(-1)

    return types.SimpleNamespace(tile_dims=tile_dims, colour=colour, tile_replicate=tile_replicate)


def test_lookup_glue_miss_then_hit(tmp_path, monkeypatch):
    import sys
    import torch
    calls = []
    fake = _fake_binding(calls)
    monkeypatch.setitem(sys.modules, "paper_2106_01275_gb300.ptrace", fake)
    import paper_2106_01275_gb300 as pkg
    monkeypatch.setattr(pkg, "ptrace", fake, raising=False)
    monkeypatch.setattr(torch.Tensor, "to", lambda self, *a, **k: self.numpy())
    db = cdb.ColourDB(tmp_path)
    ctx = types.SimpleNamespace(device=0)
    dims, mu, ps, k = [8, 8, 16, 8], 2, [2], 1
    col, m, tile, hit = db.colour(ctx, dims, mu, ps, k, "natural")
    assert not hit and len(calls) == 1 and calls[0][1] == tile
    want_t, want_m = greedy_colour(tile, mu, ps, k, 0)
    assert m == want_m
    assert np.array_equal(col, fake.tile_replicate(ctx, tile, want_t, dims))
    col2, m2, tile2, hit2 = db.colour(ctx, dims, mu, [-2, 2], k, "natural")
    assert hit2 and len(calls) == 1 and m2 == m and tile2 == tile and np.array_equal(col2, col)
