"""Checkpoint files on the host (no GPU): the format layer of algdock_checkpoint_save / _load with
host arrays and no context.  A checkpoint stores a run's state between cycles, as the paper's
stages store their data so that an interrupted calculation restarts ("Stages").

Pins: the trailer is the standard CRC-32 of the preceding bytes (checked with zlib, an independent
implementation); a round trip returns every array, the seed and the cycle unchanged; any corrupted,
truncated or foreign file, and any missing or mistyped array, is rejected with ALGDOCK_E_INVALID
and leaves the destination buffers untouched."""
import struct
import zlib

import numpy as np
import pytest

from paper_1507_03703_gb300 import algdock as A


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1507_03703_gb300 import build
    build.build()
    A.load_library()


def _arrays(seed=0):
    rng = np.random.default_rng(seed)
    return {"x": rng.normal(size=(7, 5, 3)).astype(np.float32), "comps": rng.normal(size=(7, 4)),
            "state_of": rng.integers(0, 9, size=7).astype(np.int32), "counters": np.arange(4, dtype=np.int64),
            "acc": rng.integers(0, 2, size=7).astype(np.uint8), "empty": np.zeros(0)}


def _blank(a):
    return {k: np.full_like(v, 7 if v.dtype.kind in "iu" else np.nan) for k, v in a.items()}


def test_round_trip_and_crc(tmp_path):
    p = tmp_path / "run.ckpt"
    a = _arrays(1)
    A.checkpoint_save(None, p, seed=0xDEADBEEF12345, cycle=4242, arrays=a)
    raw = p.read_bytes()
    assert raw[:8] == b"ALGDCKPT"
    assert struct.unpack("<I", raw[-4:])[0] == zlib.crc32(raw[:-4])
    b = _blank(a)
    seed, cycle = A.checkpoint_load(None, p, b)
    assert (seed, cycle) == (0xDEADBEEF12345, 4242)
    for k in a:
        assert np.array_equal(a[k], b[k]) and a[k].dtype == b[k].dtype, k
    q = A.checkpoint_query(None, p, ["x", "acc", "absent"])
    assert q["x"] == (A.F32, 105) and q["acc"] == (A.U8, 7) and q["absent"][1] == -1


def _expect_invalid(p, arrays):
    b = _blank(arrays)
    before = {k: v.copy() for k, v in b.items()}
    with pytest.raises(A.AlgdockError) as ei:
        A.checkpoint_load(None, p, b)
    assert ei.value.status == A.E_INVALID
    for k in b:
        assert np.array_equal(b[k], before[k], equal_nan=True), k


@pytest.mark.parametrize("where", [0, 9, 20, 60, -30, -5, -1])
def test_corrupt_byte_is_rejected(tmp_path, where):
    p = tmp_path / "run.ckpt"
    a = _arrays(2)
    A.checkpoint_save(None, p, 1, 2, a)
    raw = bytearray(p.read_bytes())
    raw[where] ^= 0x40
    p.write_bytes(bytes(raw))
    _expect_invalid(p, a)


@pytest.mark.parametrize("keep", [0, 3, 40, -1, -4, -50])
def test_truncated_file_is_rejected(tmp_path, keep):
    p = tmp_path / "run.ckpt"
    a = _arrays(3)
    A.checkpoint_save(None, p, 1, 2, a)
    raw = p.read_bytes()
    p.write_bytes(raw[:keep] if keep >= 0 else raw[:len(raw) + keep])
    _expect_invalid(p, a)


def test_foreign_file_and_wrong_requests_are_rejected(tmp_path):
    p = tmp_path / "other.bin"
    body = b"not a checkpoint, but long enough to hold a header" * 4
    p.write_bytes(body + struct.pack("<I", zlib.crc32(body)))  # a valid CRC does not make it one
    _expect_invalid(p, _arrays(4))
    q = tmp_path / "run.ckpt"
    a = _arrays(5)
    A.checkpoint_save(None, q, 1, 2, a)
    _expect_invalid(q, {"x": a["x"], "missing": np.zeros(3)})       # absent name
    _expect_invalid(q, {"comps": a["comps"].astype(np.float32)})   # other dtype
    _expect_invalid(q, {"state_of": a["state_of"][:5].copy()})     # other count
    assert not (tmp_path / "missing").exists()
    with pytest.raises(A.AlgdockError):
        A.checkpoint_load(None, tmp_path / "does_not_exist.ckpt", {"x": a["x"]})


def test_save_rejects_duplicate_or_bad_names(tmp_path):
    x = np.zeros(3)
    L = A.load_library()
    arr = (A.ArrayC * 2)(A._array_c("x", x), A._array_c("x", x))
    assert L.algdock_checkpoint_save(None, str(tmp_path / "d.ckpt").encode(), 0, 0, 2, arr) == A.E_INVALID
    bad = A._array_c("y", x)
    bad.dtype = 99
    arr = (A.ArrayC * 1)(bad)
    assert L.algdock_checkpoint_save(None, str(tmp_path / "e.ckpt").encode(), 0, 0, 1, arr) == A.E_INVALID
    assert not (tmp_path / "d.ckpt").exists() and not (tmp_path / "e.ckpt").exists()
