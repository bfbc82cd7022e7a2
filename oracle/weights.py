"""Classifier weights file: reader and writer (oracle side).

Test infrastructure.  The file carries the parameters (w^l, b^l), l = 1..L, of
the classifier of Sec. 3.1, Eq. (reconstuction), in FP64:

    bytes 0..7    magic "NENO6W01"
    int32         n_layers L
    int32 x (L+1) widths (inputs first, outputs last)
    per layer     W[out][in] row-major float64 little-endian, then b[out]
    uint64        FNV-1a 64-bit hash of the payload bytes (everything above
                  after the magic)

The CUDA library has its own, independent reader of the same format.
"""
import hashlib
import struct

import numpy as np

MAGIC = b"NENO6W01"
FNV_OFFSET = 0xCBF29CE484222325
FNV_PRIME = 0x100000001B3


def fnv1a64(data: bytes) -> int:
    h = FNV_OFFSET
    for byte in data:
        h ^= byte
        h = (h * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


class Net:
    """Layers as a list of (W [out, in], b [out]) float64 arrays."""

    def __init__(self, layers):
        self.layers = [(np.ascontiguousarray(W, dtype=np.float64),
                        np.ascontiguousarray(b, dtype=np.float64)) for W, b in layers]
        for (W, b) in self.layers:
            assert W.ndim == 2 and b.shape == (W.shape[0],)
        for (W0, _), (W1, _) in zip(self.layers, self.layers[1:]):
            assert W1.shape[1] == W0.shape[0]

    @property
    def widths(self):
        return [self.layers[0][0].shape[1]] + [W.shape[0] for W, _ in self.layers]

    def packed(self):
        return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in self.layers])

    def payload(self) -> bytes:
        w = self.widths
        head = struct.pack("<i", len(self.layers)) + struct.pack("<%di" % len(w), *w)
        return head + self.packed().astype("<f8").tobytes()

    def sha256(self) -> str:
        return hashlib.sha256(self.payload()).hexdigest()

    def save(self, path):
        pl = self.payload()
        with open(path, "wb") as f:
            f.write(MAGIC + pl + struct.pack("<Q", fnv1a64(pl)))

    @classmethod
    def load(cls, path):
        data = open(path, "rb").read()
        if data[:8] != MAGIC:
            raise ValueError("bad magic")
        pl, tail = data[8:-8], data[-8:]
        if struct.unpack("<Q", tail)[0] != fnv1a64(pl):
            raise ValueError("checksum mismatch")
        (nl,) = struct.unpack_from("<i", pl, 0)
        widths = struct.unpack_from("<%di" % (nl + 1), pl, 4)
        off = 4 + 4 * (nl + 1)
        vals = np.frombuffer(pl[off:], dtype="<f8")
        layers, p = [], 0
        for l in range(nl):
            nin, nout = widths[l], widths[l + 1]
            W = vals[p:p + nout * nin].reshape(nout, nin)
            p += nout * nin
            b = vals[p:p + nout]
            p += nout
            layers.append((W.copy(), b.copy()))
        if p != vals.size:
            raise ValueError("trailing data")
        return cls(layers)

    @classmethod
    def random(cls, widths=(6, 64, 32, 16, 8, 4), seed=0, scale=1.0):
        """He-style random network (parity tests do not need trained weights)."""
        rng = np.random.default_rng(seed)
        layers = []
        for nin, nout in zip(widths[:-1], widths[1:]):
            W = rng.normal(0.0, scale * np.sqrt(2.0 / nin), size=(nout, nin))
            b = rng.normal(0.0, 0.1, size=nout)
            layers.append((W, b))
        return cls(layers)
