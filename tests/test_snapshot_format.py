"""CPU tests of the snapshot/checkpoint reader and the slice image writer.

The file is assembled here byte by byte from the documented layout (magic,
uint32 JSON length, JSON provenance, records of magic, int64 step, four
float64 min/max values, U, V), independently of the library that writes it.
"""
import json
import struct

import numpy as np
import pytest

from paper_2309_10292_gb300 import snapshot


def _file(tmp_path, magic=b"GSSNAP01", L=3, dtype="f32", steps=(0, 20)):
    prov = {"format": "gs-snapshot", "version": 1, "L": L, "dtype": dtype, "Du": 0.2, "Dv": 0.1,
            "F": 0.02, "k": 0.048, "dt": 1.0, "noise": 0.1, "seed": 42}
    js = json.dumps(prov).encode()
    npdt = np.float32 if dtype == "f32" else np.float64
    rng = np.random.default_rng(0)
    fields = []
    buf = magic + struct.pack("<I", len(js)) + js
    for st in steps:
        u = rng.uniform(-0.1, 1.5, (L, L, L)).astype(npdt)
        v = rng.uniform(0, 1, (L, L, L)).astype(npdt)
        buf += b"GSREC001" + struct.pack("<q", st) + struct.pack("<4d", u.min(), u.max(), v.min(), v.max())
        buf += u.tobytes() + v.tobytes()
        fields.append((st, u, v))
    p = tmp_path / "x.gs"
    p.write_bytes(buf)
    return p, prov, fields


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_reader_round_trip(tmp_path, dtype):
    p, prov, fields = _file(tmp_path, dtype=dtype)
    hdr, recs = snapshot.read(str(p))
    assert hdr["kind"] == "snapshot" and hdr["L"] == 3 and hdr["F"] == prov["F"] and hdr["seed"] == 42
    assert [r["step"] for r in recs] == [0, 20]
    for r, (st, u, v) in zip(recs, fields):
        np.testing.assert_array_equal(r["u"], u)
        np.testing.assert_array_equal(r["v"], v)
        assert r["u_min"] == u.min() and r["v_max"] == v.max()
    # headers only
    _, light = snapshot.read(str(p), load_fields=False)
    assert [r["step"] for r in light] == [0, 20] and light[0]["u"] is None


def test_reader_rejects_foreign_and_truncated_files(tmp_path):
    bad = tmp_path / "bad.gs"
    bad.write_bytes(b"NOTGSNAP" + b"\0" * 16)
    with pytest.raises(ValueError):
        snapshot.read(str(bad))
    p, _, _ = _file(tmp_path, magic=b"GSCKPT01", steps=(7,))
    hdr, recs = snapshot.read(str(p))
    assert hdr["kind"] == "checkpoint" and recs[0]["step"] == 7
    data = p.read_bytes()
    p.write_bytes(data[:-5])
    with pytest.raises(ValueError):
        snapshot.read(str(p))


def test_pgm_image(tmp_path):
    a = np.array([[0.0, 0.5], [1.0, 0.25]])
    out = tmp_path / "s.pgm"
    snapshot.write_pgm(str(out), a)
    raw = out.read_bytes()
    assert raw.startswith(b"P5\n2 2\n255\n")
    assert list(raw[-4:]) == [0, 128, 255, 64]
