"""Host-side snapshots (checkpoint / resume): exact round trip of the step,
time and caller-order bodies; corrupted, truncated and foreign files are
refused.  No GPU."""
import numpy as np
import pytest

from paper_1204_2280_gb300 import snapshot as S
from paper_1204_2280_gb300 import workloads as W


def test_round_trip_is_exact(tmp_path):
    b = W.plummer(5000, 11)
    ids = np.random.default_rng(1).permutation(5000).astype(np.int64) * 7
    p = tmp_path / "s.bin"
    S.save(str(p), b.pos, b.vel, b.mass, ids, step=123, t=0.9609375)
    r = S.load(str(p))
    assert r["n"] == 5000 and r["step"] == 123 and r["t"] == 0.9609375
    for k, v in (("pos", b.pos), ("vel", b.vel), ("mass", b.mass), ("ids", ids)):
        assert r[k].dtype == np.asarray(v).dtype and np.array_equal(r[k], v)
    assert p.stat().st_size == 8 + 16 + 8 + 5000 * 36 + 8


def test_default_ids_and_single_body(tmp_path):
    p = tmp_path / "one.bin"
    S.save(str(p), [[1.0, 2.0, 3.0]], [[0.0, 0.5, 0.0]], [2.5])
    r = S.load(str(p))
    assert r["n"] == 1 and r["ids"].tolist() == [0] and r["mass"].tolist() == [2.5]
    with pytest.raises(ValueError):
        S.save(str(p), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))


def test_damaged_files_are_refused(tmp_path):
    b = W.plummer(300, 12)
    p = tmp_path / "s.bin"
    S.save(str(p), b.pos, b.vel, b.mass, step=5, t=0.1)
    raw = p.read_bytes()
    flip = bytearray(raw)
    flip[100] ^= 0x01                       # one bit of a position
    (tmp_path / "flip.bin").write_bytes(bytes(flip))
    (tmp_path / "short.bin").write_bytes(raw[:-9])
    (tmp_path / "foreign.bin").write_bytes(b"NOTASNAP" + raw[8:])
    for name, what in (("flip.bin", "checksum"), ("short.bin", "truncated"), ("foreign.bin", "not a snapshot")):
        with pytest.raises(ValueError, match=what):
            S.load(str(tmp_path / name))
