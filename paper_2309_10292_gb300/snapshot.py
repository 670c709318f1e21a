"""Readers for the snapshot and checkpoint files libgs writes, and a headless
image writer for slices.

The paper stores U and V with a provenance record (the run's parameters and
each field's min/max, Section 3.4, Listing 1) and inspects 2D slices of them
(Section 3.4).  File layout (little-endian; the C side is gs_io.cu):

  header : 8-byte magic b"GSSNAP01" (snapshots) or b"GSCKPT01" (checkpoint),
           uint32 n, n bytes of JSON provenance
  record : 8-byte magic b"GSREC001", int64 step, float64 U min, U max,
           V min, V max, then U and V (L^3 elements each, [z][y][x], x
           fastest, float32 or float64 as the header's "dtype")
"""
from __future__ import annotations

import json
import struct
from typing import Iterator

import numpy as np

MAGICS = {b"GSSNAP01": "snapshot", b"GSCKPT01": "checkpoint"}
RECORD_MAGIC = b"GSREC001"


def read_header(f) -> dict:
    """Parse the header of an open file; returns the provenance dict plus 'kind'."""
    magic = f.read(8)
    if magic not in MAGICS:
        raise ValueError(f"not a libgs snapshot or checkpoint (magic {magic!r})")
    (n,) = struct.unpack("<I", f.read(4))
    prov = json.loads(f.read(n).decode("utf-8"))
    prov["kind"] = MAGICS[magic]
    return prov


def iter_records(path: str, load_fields: bool = True) -> Iterator[dict]:
    """Yield {'step', 'u_min', 'u_max', 'v_min', 'v_max', 'u', 'v'} per record
    (u, v: numpy arrays [L, L, L], or None when load_fields is False)."""
    with open(path, "rb") as f:
        prov = read_header(f)
        L = int(prov["L"])
        dt = np.dtype("<f4") if prov["dtype"] == "f32" else np.dtype("<f8")
        nbytes = L ** 3 * dt.itemsize
        while True:
            magic = f.read(8)
            if not magic:
                return
            if magic != RECORD_MAGIC:
                raise ValueError(f"bad record magic {magic!r}")
            (step,) = struct.unpack("<q", f.read(8))
            mm = struct.unpack("<4d", f.read(32))
            rec = {"step": step, "u_min": mm[0], "u_max": mm[1], "v_min": mm[2], "v_max": mm[3]}
            if load_fields:
                rec["u"] = np.frombuffer(f.read(nbytes), dtype=dt).reshape(L, L, L)
                rec["v"] = np.frombuffer(f.read(nbytes), dtype=dt).reshape(L, L, L)
                if rec["u"].size != L ** 3 or rec["v"].size != L ** 3:
                    raise ValueError("truncated record")
            else:
                f.seek(2 * nbytes, 1)
                rec["u"] = rec["v"] = None
            yield rec


def read(path: str, load_fields: bool = True):
    """(provenance dict, list of records) of a snapshot or checkpoint file."""
    with open(path, "rb") as f:
        prov = read_header(f)
    return prov, list(iter_records(path, load_fields))


def write_pgm(path: str, plane: np.ndarray, lo: float | None = None, hi: float | None = None) -> None:
    """Write a 2D array as an 8-bit greyscale binary PGM image (lo -> black,
    hi -> white; default: the array's range)."""
    a = np.asarray(plane, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("plane must be 2D")
    lo = float(np.nanmin(a)) if lo is None else float(lo)
    hi = float(np.nanmax(a)) if hi is None else float(hi)
    scale = 255.0 / (hi - lo) if hi > lo else 0.0
    img = np.clip(np.nan_to_num((a - lo) * scale, nan=0.0), 0, 255).round().astype(np.uint8)
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())
