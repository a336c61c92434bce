"""Network checkpoints: a saved file loads back bit for bit with its
metadata, and damaged, truncated or foreign files are refused."""
import numpy as np
import pytest

from paper_2312_13094_gb300 import checkpoint as ck


def test_roundtrip(tmp_path):
    p = np.random.default_rng(0).standard_normal(5000).astype(np.float32)
    path = str(tmp_path / "net.fdck")
    ck.save(path, p, {"epochs": 20, "loss": 2.7e-6})
    q, meta = ck.load(path)
    assert q.dtype == np.float32 and np.array_equal(p, q)
    assert meta == {"epochs": 20, "loss": 2.7e-6}


@pytest.mark.parametrize("damage", ["flip", "truncate", "magic", "version"])
def test_damaged_files_are_refused(tmp_path, damage):
    path = str(tmp_path / "net.fdck")
    ck.save(path, np.arange(100, dtype=np.float32), {"a": 1})
    b = bytearray(open(path, "rb").read())
    if damage == "flip":
        b[60] ^= 0x10
    elif damage == "truncate":
        b = b[:-9]
    elif damage == "magic":
        b[0:2] = b"XX"
    else:
        b[8] = 2
    open(path, "wb").write(bytes(b))
    with pytest.raises(ValueError):
        ck.load(path)
