"""Write tests/golden/exact_tau.json: the exact triangle count and maximum
degree of the named single-stream workloads, for the relative-error report
and the Theorem 3.2 sample bound, with a hash of the generated edge stream
(a reader uses the values only for the same stream).  Calls only oracle/ (the forward-algorithm
counter) on the synth/ generators' output.

    python tests/golden/make_exact_tau.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import exact  # noqa: E402


def main():
    out = {}
    for name, gen in (("tiny", synth.tiny_chung_lu), ("rmat20", synth.rmat20_single)):
        keys = gen()
        n = synth.WORKLOADS[name]["n"]
        u, v = synth.unpack(keys)
        deg = np.bincount(np.concatenate([u, v]).astype(np.int64), minlength=n)
        out[name] = {"m": int(keys.size), "tau": int(exact.count(keys, n)),
                     "max_degree": int(deg.max()),
                     "keys_sha256": hashlib.sha256(keys.astype("<u8").tobytes()).hexdigest()}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "exact_tau.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
