"""The network checkpoint format of include/plo.h written and read in plain
Python (test helper): magic "PLOMLP01", a uint64 header length, a flat JSON
header, then 64-byte-aligned little-endian blobs master / adam_m / adam_v
(float32) and weights_bf16 (bfloat16 bits as uint16)."""
from __future__ import annotations

import json
import struct

import numpy as np

MAGIC = b"PLOMLP01"
BLOBS = ("master", "adam_m", "adam_v", "weights_bf16")


def write(path, desc: dict, step: int, master, adam_m, adam_v, weights_bf16_bits):
    arrays = [np.asarray(master, "<f4"), np.asarray(adam_m, "<f4"), np.asarray(adam_v, "<f4"),
              np.asarray(weights_bf16_bits, "<u2")]
    head = dict(format="plo-mlp", version=1, **{k: desc[k] for k in (
        "arch", "sh_degree", "transmittance", "loss", "total_steps", "l_max", "eps", "lr0", "lr1", "init_radiance")},
        seed=str(desc["seed"]), step=step, n_params=int(arrays[0].size))
    offs = [0] * 4
    for _ in range(2):  # the offsets depend on the header's own length
        text = json.dumps(dict(head, **{f"{b}_offset": o for b, o in zip(BLOBS, offs)}))
        pos = (16 + len(text) + 63) // 64 * 64
        for k, a in enumerate(arrays):
            offs[k] = pos
            pos = (pos + a.nbytes + 63) // 64 * 64
    text = json.dumps(dict(head, **{f"{b}_offset": o for b, o in zip(BLOBS, offs)}))
    assert (16 + len(text) + 63) // 64 * 64 <= offs[0]
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<Q", len(text)) + text.encode())
        for o, a in zip(offs, arrays):
            f.write(b"\0" * (o - f.tell()))
            f.write(a.tobytes())


def read(path):
    """(header dict, {blob name: array})."""
    with open(path, "rb") as f:
        data = f.read()
    assert data[:8] == MAGIC
    (hl,) = struct.unpack("<Q", data[8:16])
    head = json.loads(data[16:16 + hl])
    n = head["n_params"]
    out = {}
    for b in BLOBS[:3]:
        o = head[f"{b}_offset"]
        out[b] = np.frombuffer(data[o:o + 4 * n], "<f4")
    o = head["weights_bf16_offset"]
    out["weights_bf16"] = np.frombuffer(data[o:], "<u2")
    return head, out
