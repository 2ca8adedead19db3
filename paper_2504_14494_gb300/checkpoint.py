"""Checkpoint / resume of simulation and training state.

A checkpoint is one file: a fixed header (magic b"LBMGNNCK", format version,
number of records), then per record a name, dtype, shape, byte count and
CRC32, followed by the raw little-endian bytes.  Device tensors are copied to
the host on save and back to their device on load; a CRC mismatch, a wrong
magic or version, or a shape/dtype mismatch with the destination raises.
Resuming a run from a checkpoint reproduces the uninterrupted run bit for
bit, since every kernel of the library is deterministic.
"""
import struct
import zlib

import numpy as np

MAGIC = b"LBMGNNCK"
VERSION = 1
_DT = {"float32": 0, "float64": 1, "int64": 2, "uint8": 3, "int32": 4}
_DT_INV = {v: k for k, v in _DT.items()}


def _to_numpy(x):
    if isinstance(x, (np.ndarray, np.generic, int, float)):
        return np.array(x, order="C")
    return x.detach().contiguous().cpu().numpy()


def save(path, records):
    """records: dict name -> torch tensor or numpy array (or python scalar)."""
    items = []
    for name, v in records.items():
        a = _to_numpy(v)
        a = a.astype(a.dtype.newbyteorder("<"), copy=False)
        if a.dtype.name not in _DT:
            raise TypeError(f"unsupported dtype {a.dtype} for {name}")
        items.append((name, a))
    with open(path, "wb") as fh:
        fh.write(MAGIC + struct.pack("<II", VERSION, len(items)))
        for name, a in items:
            raw = a.tobytes()
            nb = name.encode()
            fh.write(struct.pack("<H", len(nb)) + nb)
            fh.write(struct.pack("<BB", _DT[a.dtype.name], a.ndim))
            fh.write(struct.pack(f"<{a.ndim}q", *a.shape))
            fh.write(struct.pack("<QI", len(raw), zlib.crc32(raw) & 0xFFFFFFFF))
            fh.write(raw)


def load(path):
    """Returns dict name -> numpy array (CRC-checked)."""
    out = {}
    with open(path, "rb") as fh:
        if fh.read(8) != MAGIC:
            raise ValueError("not a checkpoint (bad magic)")
        version, n = struct.unpack("<II", fh.read(8))
        if version != VERSION:
            raise ValueError(f"checkpoint version {version}, expected {VERSION}")
        for _ in range(n):
            (ln,) = struct.unpack("<H", fh.read(2))
            name = fh.read(ln).decode()
            dt, nd = struct.unpack("<BB", fh.read(2))
            shape = struct.unpack(f"<{nd}q", fh.read(8 * nd))
            nbytes, crc = struct.unpack("<QI", fh.read(12))
            raw = fh.read(nbytes)
            if len(raw) != nbytes or (zlib.crc32(raw) & 0xFFFFFFFF) != crc:
                raise ValueError(f"checkpoint record {name!r} is truncated or corrupt")
            out[name] = np.frombuffer(raw, dtype=np.dtype(_DT_INV[dt]).newbyteorder("<")).reshape(shape).copy()
    return out


def restore(path, destinations):
    """Loads a checkpoint into existing tensors/arrays (same shape and dtype);
    returns the records that have no destination."""
    data = load(path)
    for name, dst in destinations.items():
        a = data.pop(name)
        if tuple(a.shape) != tuple(dst.shape) or a.dtype.name != str(dst.dtype).replace("torch.", ""):
            raise ValueError(f"record {name!r}: {a.dtype}{a.shape} does not fit the destination")
        if isinstance(dst, np.ndarray):
            dst[...] = a
        else:
            import torch
            dst.copy_(torch.from_numpy(a))
    return data
