"""Reader for the hand-derived golden stream fixtures in tests/golden/.

Each fixture lists the input field, the bound, and the expected stream as
hand-worked header fields, flag words, payload blocks and outliers.  This
module only assembles those numbers into bytes with the stream layout
(64-byte header, flags, payload, outliers); it computes none of the method.
"""
import os
import struct

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    rec = {"flags": [], "blocks": [], "outliers": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "ndim":
                rec["ndim"] = int(vals[0])
            elif key == "mode":
                rec["mode"] = {"abs": 0, "rel": 1}[vals[0]]
            elif key == "eb":
                rec["eb"] = float(vals[0])
            elif key == "dims":
                rec["dims"] = [int(v) for v in vals]
            elif key == "x":
                rec["x"] = np.array([float(v) for v in vals], np.float32)
            elif key == "header":
                rec["header"] = {k: v for k, v in (kv.split("=") for kv in vals)}
            elif key == "flag":
                rec["flags"].append(tuple(int(v, 0) for v in vals))
            elif key == "block":
                rec["blocks"].append([int(v, 0) for v in vals])
            elif key == "outlier":
                rec["outliers"].append((int(vals[0]), int(vals[1])))
            elif key == "size":
                rec["size"] = int(vals[0])
    d = rec["dims"]
    x = rec["x"].reshape(d[2], d[1], d[0])
    if rec["ndim"] == 2:
        x = x[0]
    elif rec["ndim"] == 1:
        x = x[0, 0]
    rec["x"] = x
    return rec


def expected_bytes(rec):
    h = rec["header"]
    nt = int(h["n_tiles"])
    hdr = b"FZG1" + bytes([1, rec["ndim"], rec["mode"], 0])
    hdr += struct.pack("<3I", *rec["dims"])
    hdr += struct.pack("<I", nt)
    hdr += struct.pack("<d", rec["eb"])
    hdr += struct.pack("<3f", float(h["eb_f"]), float(h["ebx2"]),
                       float(h["ebx2_r"]))
    hdr += struct.pack("<2I", int(h["nnz"]), int(h["n_out"]))
    hdr += struct.pack("<2f", float(h["min"]), float(h["max"]))
    hdr += struct.pack("<I", 0)
    assert len(hdr) == 64
    flags = np.zeros((nt, 8), np.uint32)
    for tile, word, val in rec["flags"]:
        flags[tile, word] = val
    body = flags.astype("<u4").tobytes()
    for b in rec["blocks"]:
        body += struct.pack("<4I", *b)
    for idx, val in rec["outliers"]:
        body += struct.pack("<Ii", idx, val)
    out = hdr + body
    assert len(out) == rec["size"], (len(out), rec["size"])
    return out
