"""Reader for the stored full-size orderings (tests/golden/*_order.txt, written by
tests/golden/make_order_golden.py from the oracle alone) and the digest convention they
use: SHA-256 of the little-endian bytes of key u64, perm u32, rad2 i64, radius f32 bits."""
import hashlib
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def sha(a: np.ndarray) -> str:
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def read(name: str) -> list[dict]:
    """Records of a golden file: dict(name, id, n, start, scale, key/perm/rad2/radius
    digests, at = {index: (perm, rad2)})."""
    recs = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            if w[0] == "part":
                recs.append(dict(name=w[1], id=int(w[3]), n=int(w[5]), start=int(w[7]), scale=float(w[9]), at={}))
            elif w[0].endswith("_sha256"):
                recs[-1][w[0][:-7]] = w[1]
            elif w[0] == "at":
                recs[-1]["at"][int(w[1])] = (int(w[3]), int(w[5]))
    return recs


def check(rec: dict, key: np.ndarray, perm: np.ndarray, rad2: np.ndarray, radius: np.ndarray | None) -> None:
    """Asserts that a full ordering equals the stored one (inputs first, then outputs)."""
    assert len(key) == rec["n"], (rec["name"], len(key), rec["n"])
    assert sha(key.view(np.uint64)) == rec["key"], rec["name"] + ": surfel keys differ from the oracle's"
    for i, (p, r) in rec["at"].items():
        assert int(perm[i]) == p and int(rad2[i]) == r, (rec["name"], i, int(perm[i]), int(rad2[i]), p, r)
    assert sha(perm.view(np.uint32)) == rec["perm"], rec["name"] + ": permutation differs from the oracle's"
    assert sha(rad2.view(np.int64)) == rec["rad2"], rec["name"] + ": squared radii differ from the oracle's"
    if radius is not None:
        assert sha(radius.view(np.uint32)) == rec["radius"], rec["name"] + ": radii differ from the oracle's"
