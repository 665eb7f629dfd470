"""Store of precomputed tile colourings (Sec. 3.5).

The paper colours a small torus (the tile) once and repeats it over every
lattice that the tile divides, keeping the tiles it has coloured for reuse.
Here a tile colouring is one file per key

    (tile dims, displacement dimension mu, displacements, distance k, order),

with the displacements reduced to the sorted set of |p| (the neighbourhood
of Eq. (8), and so the greedy colouring, depends on nothing else).  A file is
a fixed little-endian header (magic, version, the key, the colour count m,
the node count, a CRC-32 of the payload) followed by the int32 colours in
storage order.  Reads check every field against the key asked for and the
CRC against the payload; writes go to a temporary file in the same folder
and are renamed into place, so a reader sees either no file or a whole one.

`ColourDB.colour` is the lookup the estimator uses: the tile of Sec. 3.5
(`pt_tile_dims`), its colouring from the store or, on a miss, from the GPU
walk (`pt_colour`, then stored), and the repetition over the lattice
(`pt_tile_replicate`).
"""
import os
import struct
import tempfile
import zlib

import numpy as np

MAGIC = b"PTCOLDB1"
VERSION = 1
MAX_P = 16
ORDERS = {"natural": 0, "redblack": 1}
_HEAD = struct.Struct("<8sI4iiiiI%diiqI" % MAX_P)     # magic, version, dims, mu, k, order, n_p, p[16], m, N, crc


class ColourDBError(RuntimeError):
    """A stored colouring that is damaged or does not match its key."""


def canonical_p(p_list):
    ps = sorted({abs(int(p)) for p in p_list})
    if not ps or len(ps) > MAX_P:
        raise ValueError("1 to %d distinct displacements" % MAX_P)
    return ps


def _order(order):
    if isinstance(order, str):
        if order not in ORDERS:
            raise ValueError("order: natural (0) or redblack (1)")
        return ORDERS[order]
    if int(order) not in ORDERS.values():
        raise ValueError("order: natural (0) or redblack (1)")
    return int(order)


class ColourDB:
    def __init__(self, root):
        self.root = str(root)
        os.makedirs(self.root, exist_ok=True)

    def path(self, tile, mu, p_list, k, order):
        t = "x".join(str(int(d)) for d in tile)
        ps = "-".join(str(p) for p in canonical_p(p_list))
        name = "tile_%s_mu%d_p%s_k%d_%s.ptcol" % (t, int(mu), ps, int(k),
                                                 "rb" if _order(order) else "nat")
        return os.path.join(self.root, name)

    def put(self, tile, mu, p_list, k, order, col, m):
        """Store a tile colouring (int32 [prod(tile)], colours 0..m-1)."""
        tile = [int(d) for d in tile]
        if len(tile) != 4 or min(tile) < 1:
            raise ValueError("tile: four positive sides")
        col = np.ascontiguousarray(np.asarray(col).reshape(-1), dtype="<i4")
        N = int(np.prod(tile))
        if col.size != N:
            raise ValueError("colouring has %d entries, the tile %d" % (col.size, N))
        if m < 1 or col.min() < 0 or col.max() >= m:
            raise ValueError("colours must lie in 0..m-1")
        ps = canonical_p(p_list)
        payload = col.tobytes()
        head = _HEAD.pack(MAGIC, VERSION, *tile, int(mu), int(k), _order(order), len(ps),
                          *(ps + [0] * (MAX_P - len(ps))), int(m), N, zlib.crc32(payload))
        path = self.path(tile, mu, ps, k, order)
        fd, tmp = tempfile.mkstemp(dir=self.root, prefix=".tmp_", suffix=".ptcol")
        try:
            with os.fdopen(fd, "wb") as f:
                f.write(head)
                f.write(payload)
            os.replace(tmp, path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise
        return path

    def get(self, tile, mu, p_list, k, order):
        """(col int32 [prod(tile)], m), or None if the key is not stored."""
        path = self.path(tile, mu, p_list, k, order)
        if not os.path.exists(path):
            return None
        with open(path, "rb") as f:
            raw = f.read()
        if len(raw) < _HEAD.size:
            raise ColourDBError("%s: truncated header" % path)
        h = _HEAD.unpack_from(raw)
        magic, version, dims, mu_f, k_f, order_f, n_p = h[0], h[1], list(h[2:6]), h[6], h[7], h[8], h[9]
        p_f = list(h[10:10 + n_p]) if 0 < n_p <= MAX_P else None
        m, N, crc = h[10 + MAX_P], h[11 + MAX_P], h[12 + MAX_P]
        if magic != MAGIC or version != VERSION:
            raise ColourDBError("%s: not a colour store file (version %r)" % (path, version))
        want = ([int(d) for d in tile], int(mu), int(k), _order(order), canonical_p(p_list))
        if (dims, mu_f, k_f, order_f, p_f) != want:
            raise ColourDBError("%s: stored key %r differs from %r" % (path, (dims, mu_f, k_f, order_f, p_f), want))
        if N != int(np.prod(dims)) or len(raw) != _HEAD.size + 4 * N:
            raise ColourDBError("%s: payload size does not match %d nodes" % (path, N))
        payload = raw[_HEAD.size:]
        if zlib.crc32(payload) != crc:
            raise ColourDBError("%s: CRC mismatch" % path)
        col = np.frombuffer(payload, dtype="<i4").astype(np.int32)
        if m < 1 or col.min() < 0 or col.max() >= m:
            raise ColourDBError("%s: colours outside 0..m-1" % path)
        return col, int(m)

    def colour(self, ctx, dims, mu, p_list, k, order="natural", out=None):
        """The Sec. 3.5 colouring of `dims` through the store: (col on the
        device, m, tile, hit).  A miss colours the tile on the GPU and stores it."""
        import torch
        from . import ptrace as pt
        ps = canonical_p(p_list)          # the library takes |p|: the neighbourhood is symmetric in p
        tile = pt.tile_dims(dims, mu, ps, k)
        got = self.get(tile, mu, ps, k, order)
        hit = got is not None
        if hit:
            tcol, m = got
            tdev = torch.as_tensor(tcol).to("cuda:%d" % ctx.device)
        else:
            tdev, m = pt.colour(ctx, tile, mu, ps, k, order)
            self.put(tile, mu, ps, k, order, tdev.cpu().numpy(), m)
        col = pt.tile_replicate(ctx, tile, tdev, dims, out)
        return col, m, tile, hit
