"""Versioned checkpoints of the learned-weight network's parameters.

File layout (little-endian): the 8-byte magic b"FDMLPCK\\0", a uint32 format
version (1), the uint32 parameter count, the uint32 length of a UTF-8 JSON
metadata block (training settings, losses, ...), the metadata, the float32
parameters, and a uint32 CRC-32 (zlib) of every byte before it.  A file with a
wrong magic, version, length or checksum is refused, so a truncated or
damaged checkpoint cannot be loaded silently.
"""
from __future__ import annotations

import json
import struct
import zlib

import numpy as np

MAGIC = b"FDMLPCK\0"
VERSION = 1


def save(path: str, params, meta: dict | None = None) -> None:
    p = np.ascontiguousarray(params, dtype="<f4").reshape(-1)
    m = json.dumps(meta or {}, sort_keys=True).encode()
    body = MAGIC + struct.pack("<III", VERSION, p.size, len(m)) + m + p.tobytes()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))
    import os
    os.replace(tmp, path)


def load(path: str):
    """(params float32 array, metadata dict); ValueError on any damage."""
    with open(path, "rb") as f:
        data = f.read()
    head = len(MAGIC) + 12
    if len(data) < head + 4 or data[:len(MAGIC)] != MAGIC:
        raise ValueError(f"{path}: not a network checkpoint")
    version, n, mlen = struct.unpack("<III", data[len(MAGIC):head])
    if version != VERSION:
        raise ValueError(f"{path}: checkpoint format {version}, this build reads {VERSION}")
    end = head + mlen + 4 * n
    if len(data) != end + 4:
        raise ValueError(f"{path}: checkpoint is {len(data)} bytes, expected {end + 4}")
    (crc,) = struct.unpack("<I", data[end:])
    if zlib.crc32(data[:end]) & 0xFFFFFFFF != crc:
        raise ValueError(f"{path}: checksum mismatch")
    meta = json.loads(data[head:head + mlen].decode())
    params = np.frombuffer(data[head + mlen:end], dtype="<f4").astype(np.float32)
    return params, meta
