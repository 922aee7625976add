"""Save and reload a built hierarchy level (checkpoint / resume).

A level's outputs -- the prolongator P, the coarse operator X, Y, the retained
singular values sigma and, optionally, anything else the caller names -- are
written to one binary file:

  8 bytes     magic b"MGHIER01"
  8 bytes     header length L (little-endian uint64)
  L bytes     JSON header: format version, the problem (mg.Problem or
              mg.CoarseProblem fields), free-form metadata, and per array its
              name, dtype, shape, byte offset and size in the payload, plus the
              SHA-256 of the payload
  payload     the arrays' bytes, C order, little-endian, each starting at a
              multiple of 64 bytes

Reloading returns the same arrays bit for bit (on the device asked for), so a
reloaded level gives bitwise the coarse applies of the level that was saved.
Files are checked on load: magic, version, sizes and checksum.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import struct

import numpy as np

MAGIC = b"MGHIER01"
VERSION = 1
_ALIGN = 64
_DTYPES = {"complex64": "<c8", "complex128": "<c16", "float32": "<f4", "float64": "<f8",
           "int32": "<i4", "int64": "<i8", "uint8": "|u1"}


class CheckpointError(RuntimeError):
    pass


def _to_numpy(t):
    if hasattr(t, "detach"):  # torch tensor (any device)
        t = t.detach().cpu().numpy()
    return np.ascontiguousarray(t)


def save(path: str, problem, arrays: dict, meta: dict | None = None) -> None:
    """Write `arrays` (name -> torch tensor or numpy array) with the problem they
    belong to (a dataclass or a dict) and free-form metadata."""
    prob = dataclasses.asdict(problem) if dataclasses.is_dataclass(problem) else dict(problem)
    entries, blobs, off = [], [], 0
    for name, a in arrays.items():
        a = _to_numpy(a)
        kind = str(a.dtype)
        if kind not in _DTYPES:
            raise CheckpointError(f"{name}: dtype {kind} not supported")
        raw = a.astype(_DTYPES[kind], copy=False).tobytes(order="C")
        pad = (-off) % _ALIGN
        off += pad
        blobs.append(b"\0" * pad)
        entries.append({"name": name, "dtype": kind, "shape": list(a.shape), "offset": off,
                        "nbytes": len(raw)})
        blobs.append(raw)
        off += len(raw)
    payload = b"".join(blobs)
    header = {"format": VERSION, "problem": prob, "meta": meta or {}, "arrays": entries,
              "payload_bytes": len(payload), "sha256": hashlib.sha256(payload).hexdigest()}
    hb = json.dumps(header, sort_keys=True).encode()
    with open(path, "wb") as fh:
        fh.write(MAGIC)
        fh.write(struct.pack("<Q", len(hb)))
        fh.write(hb)
        fh.write(payload)


def load(path: str, device: str | None = None):
    """Read a file written by save(): returns (problem dict, {name: array},
    meta).  Arrays are torch tensors on `device` when it is given, else numpy."""
    with open(path, "rb") as fh:
        data = fh.read()
    if len(data) < 16 or data[:8] != MAGIC:
        raise CheckpointError("not a hierarchy checkpoint (bad magic)")
    (hl,) = struct.unpack("<Q", data[8:16])
    if 16 + hl > len(data):
        raise CheckpointError("truncated header")
    header = json.loads(data[16:16 + hl].decode())
    if header.get("format") != VERSION:
        raise CheckpointError(f"unsupported format {header.get('format')}")
    payload = data[16 + hl:]
    if len(payload) != header["payload_bytes"]:
        raise CheckpointError("truncated or oversized payload")
    if hashlib.sha256(payload).hexdigest() != header["sha256"]:
        raise CheckpointError("payload checksum mismatch")
    arrays = {}
    for e in header["arrays"]:
        raw = payload[e["offset"]:e["offset"] + e["nbytes"]]
        a = np.frombuffer(raw, dtype=_DTYPES[e["dtype"]]).reshape(e["shape"]).copy()
        if device is not None:
            import torch
            a = torch.from_numpy(a).to(device)
        arrays[e["name"]] = a
    return header["problem"], arrays, header["meta"]


def save_level(path: str, level, meta: dict | None = None) -> None:
    """A built mg.Level (P, X, Y, sigma) or mg.CoarseLevel (P, X2, Y2, sigma)."""
    if hasattr(level, "X2"):
        arrays = {"P": level.P, "X": level.X2, "Y": level.Y2, "sigma": level.sigma}
    else:
        arrays = {"P": level.P, "X": level.X, "Y": level.Y, "sigma": level.sigma}
    save(path, level.prob, arrays, meta)
