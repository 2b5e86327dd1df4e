"""Write the oracle's reduced He-4 term table to tests/golden/ (oracle only).

    python tests/golden/make_tables.py

The He-4 (p up, p down, n up, n down; upper components) table is checked here
exactly modulo 2^61 - 1 at a fresh random point (Theorem 1, App. C) against the
plain Wick sum over all 1.07e10 (sink, source tuple, sigma_u, sigma_d) terms --
minutes of CPU time, too slow for every test run -- and stored with a SHA-256
digest of its canonical bytes (rep int64, w int64, ids uint16, little endian,
in that order).  It imports nothing but `oracle/`.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import operators as ops  # noqa: E402
from oracle import oracle as O  # noqa: E402


def digest(rep, w, ids) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(rep, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(w, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(ids, dtype="<u2").tobytes())
    return h.hexdigest()


def main(name="he4", check_point=True):
    nuc = ops.nucleus(name)
    t0 = time.time()
    tab = O.dedup(nuc, seed=0x5EED)
    t1 = time.time()
    info = dict(nucleus=name, form="upper", stats=list(tab["stats"]), U=len(tab["w"]),
                sha256=digest(tab["rep"], tab["w"], tab["ids"]), oracle_seconds=round(t1 - t0, 1),
                oracle_threads=O.num_threads())
    if check_point:
        seed = 0xC0FFEE
        a = O.modp_table(nuc, tab, seed)
        b = O.modp_raw(nuc, seed)
        assert a == b, "reduced table disagrees with the raw Wick sum mod p"
        info["modp_check"] = dict(seed=seed, value=a)
    np.savez_compressed(os.path.join(HERE, f"{name}_upper_table.npz"),
                        rep_delta=np.diff(tab["rep"], prepend=0), w=tab["w"].astype(np.int32), ids=tab["ids"])
    with open(os.path.join(HERE, f"{name}_upper_table.json"), "w") as f:
        json.dump(info, f, indent=1)
    print(json.dumps(info))


def load(name="he4"):
    d = np.load(os.path.join(HERE, f"{name}_upper_table.npz"))
    info = json.load(open(os.path.join(HERE, f"{name}_upper_table.json")))
    tab = dict(rep=np.cumsum(d["rep_delta"]).astype(np.int64), w=d["w"].astype(np.int64),
               ids=d["ids"].astype(np.uint16))
    assert digest(tab["rep"], tab["w"], tab["ids"]) == info["sha256"]
    return tab, info


if __name__ == "__main__":
    main(*(sys.argv[1:2] or ["he4"]))
