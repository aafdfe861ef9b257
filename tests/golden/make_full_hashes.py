"""Writes tests/golden/full_hashes.json: for every full-size case of
tests/full_cases.py, the SHA-256 of the seeded field, of the oracle's stream and of
the oracle's reconstruction.

Only the seeded generator (``paper_2603_26968_b300.synth``) and the CPU oracle
(``oracle/``, its OpenMP build: the same bytes as the single-threaded one) run
here; nothing of the CUDA path.  A full run takes tens of minutes on a few cores:

    python tests/golden/make_full_hashes.py [--workers 4] [--only c2_]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor, as_completed
from pathlib import Path

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent.parent
OUT = HERE / "full_hashes.json"


def _sha(b) -> str:
    return hashlib.sha256(b).hexdigest()


def _one(name, group, spec, threads):
    os.environ["OMP_NUM_THREADS"] = str(threads)
    sys.path.insert(0, str(ROOT))
    import oracle
    from paper_2603_26968_b300 import synth
    t0 = time.time()
    x = synth.make_field(spec)
    st = oracle.compress(x, 1, spec.eb, openmp=True)
    y = oracle.decompress(st, openmp=True)
    return name, {
        "group": group, "shape": list(x.shape), "dtype": spec.dtype, "mode": "NOA", "eb": spec.eb,
        "field_sha256": _sha(x.tobytes()), "stream_bytes": len(st), "stream_sha256": _sha(st),
        "xhat_sha256": _sha(y.tobytes()), "oracle_s": round(time.time() - t0, 1),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--only", default="", help="prefix of the case names to (re)compute")
    a = ap.parse_args()
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    import oracle
    from full_cases import cases
    oracle.build(openmp=True)
    todo = [c for c in cases() if c[0].startswith(a.only)]
    todo.sort(key=lambda c: -c[2].nbytes)  # largest first
    have = json.loads(OUT.read_text())["cases"] if OUT.exists() else {}
    threads = max(1, (os.cpu_count() or 1) // a.workers)
    with ProcessPoolExecutor(a.workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_one, n, g, s, threads) for n, g, s in todo]
        for f in as_completed(futs):
            name, rec = f.result()
            have[name] = rec
            print(f"{name}: {rec['stream_bytes']} bytes, {rec['oracle_s']} s", flush=True)
            OUT.write_text(json.dumps({"generator": "paper_2603_26968_b300.synth", "writer": "oracle",
                                       "cases": dict(sorted(have.items()))}, indent=1) + "\n")


if __name__ == "__main__":
    main()
