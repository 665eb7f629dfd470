"""Resumable probed trace estimation: per-set estimates kept on disk.

The estimate of each noise set (Eqs. (1), (5): the sum over colours and
dilution components of v^H P_n A^{-1} v, for every displacement p_n) is
independent of the others, so a long run can stop after any set and be
continued, or extended to more sets later, without redoing solves.  The log
is a JSON-lines file: a header line with the run's key (operator, a CRC-32 of
the colouring and, for Wilson, of the links, the displacements, the noise,
the seed, dilution, precision and tolerance), then one line per completed
set with its estimates (doubles written with round-trip precision).  Lines
are appended and flushed to disk a chunk at a time; a line cut short by a
crash is ignored on reading, any other damage is an error, and a key that
differs from the header is refused.
"""
import json
import os
import zlib

import numpy as np

VERSION = 1


class CheckpointError(RuntimeError):
    """A log that is damaged or belongs to another run."""


def _crc(a):
    if a is None:
        return None
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return zlib.crc32(np.ascontiguousarray(a).tobytes())


def run_key(op, col, mu, p_list, noise, seed, dilute, prec, tol, links=None):
    return {"dims": [int(d) for d in op.dims], "dof": int(op.dof),
            "m2": getattr(op, "m2", None), "kappa": getattr(op, "kappa", None),
            "links_crc32": _crc(links), "colouring_crc32": _crc(col), "mu": int(mu),
            "p_list": [int(p) for p in p_list], "noise": str(noise), "seed": int(seed),
            "dilute": bool(dilute), "prec": str(prec), "tol": float(tol)}


def _complete_lines(path):
    """The lines that end in a newline (text after the last one was cut short)."""
    with open(path, "r") as f:
        return f.read().split("\n")[:-1]


def read_log(path, key):
    """Estimates of the sets already in the log, est[s, n] (complex), s = 0..done-1."""
    n_p = len(key["p_list"])
    if not os.path.exists(path):
        return np.zeros((0, n_p), dtype=np.complex128)
    complete = _complete_lines(path)
    if not complete:                            # the header itself was cut short
        return np.zeros((0, n_p), dtype=np.complex128)
    try:
        head = json.loads(complete[0])
    except ValueError:
        raise CheckpointError("%s: damaged header" % path)
    if head.get("version") != VERSION or head.get("key") != key:
        raise CheckpointError("%s: the log belongs to another run (%r)" % (path, head.get("key")))
    rows = []
    for i, line in enumerate(complete[1:]):
        try:
            r = json.loads(line)
            s, est = int(r["set"]), r["est"]
            row = [complex(float(re), float(im)) for re, im in est]
        except (ValueError, KeyError, TypeError):
            raise CheckpointError("%s: damaged line %d" % (path, i + 2))
        if s != len(rows) or len(row) != n_p:
            raise CheckpointError("%s: line %d holds set %d, expected set %d" % (path, i + 2, s, len(rows)))
        rows.append(row)
    return np.array(rows, dtype=np.complex128).reshape(len(rows), n_p)


def _trim(path):
    """Drop a line cut short; remove a log whose header was cut short."""
    if not os.path.exists(path):
        return
    complete = _complete_lines(path)
    with open(path, "r") as f:
        whole = f.read()
    text = "".join(l + "\n" for l in complete)
    if not complete:
        os.unlink(path)
    elif text != whole:
        with open(path, "w") as f:
            f.write(text)
            f.flush()
            os.fsync(f.fileno())


def _append(path, key, first_set, est):
    new = not os.path.exists(path)
    with open(path, "a") as f:
        if new:
            f.write(json.dumps({"version": VERSION, "key": key}) + "\n")
        for i, row in enumerate(est):
            f.write(json.dumps({"set": first_set + i,
                                "est": [[float(z.real), float(z.imag)] for z in row]}) + "\n")
        f.flush()
        os.fsync(f.fileno())


def trace_resumable(op, col, n_colours, mu, p_list, noise, seed, n_sets, log_path, chunk=1, dilute=True,
                    prec="mixed_fp32", tol=1e-10, maxit=20000, links=None):
    """est[s, n] for sets 0..n_sets-1: the sets in the log are read back, the
    rest computed `chunk` sets per call of pt_trace_PAinv and appended."""
    from . import ptrace as pt
    key = run_key(op, col, mu, p_list, noise, seed, dilute, prec, tol, links)
    have = read_log(log_path, key)
    _trim(log_path)
    done = have.shape[0]
    parts = [have[:n_sets]]
    while done < n_sets:
        n = min(chunk, n_sets - done)
        est, _, _, _ = pt.trace(op, col, n_colours, mu, p_list, noise, seed, done, n, dilute, prec, tol, maxit)
        est = np.asarray(est, dtype=np.complex128).reshape(n, len(p_list))
        _append(log_path, key, done, est)
        parts.append(est)
        done += n
    return np.concatenate(parts, axis=0)
