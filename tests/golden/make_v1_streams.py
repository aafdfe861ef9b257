"""Writes the format-1 stream fixtures: seeded fields compressed by the oracle while
it wrote format 1 (bin records DIFFNB.BIT.RZE_1 only), with the oracle's
reconstruction of each.  Readers must keep decoding these streams.  Run from the
repository root: python tests/golden/make_v1_streams.py"""
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))
import oracle  # noqa: E402
from paper_2603_26968_b300 import synth as S  # noqa: E402

HERE = Path(__file__).resolve().parent

FIELDS = {
    # name: (shape, dtype, mode, eb, seed)
    "v1_2d_f32": ((70, 90), "f32", 1, 1e-3, 3),
    "v1_3d_f64": ((11, 21, 34), "f64", 1, 1e-3, 4),
    "v1_3d_f32_abs": ((17, 19, 23), "f32", 0, 2e-3, 5),
}


def field(shape, dtype, seed):
    f = np.zeros(shape, np.float64)
    S.add_bumps(f, 12, max(shape) / 20.0, max(shape) / 4.0, seed)
    S.add_uniform_noise(f, 1e-4, seed)
    return f.astype(np.float32 if dtype == "f32" else np.float64)


def main():
    for name, (shape, dt, mode, eb, seed) in FIELDS.items():
        x = field(shape, dt, seed)
        st = oracle.compress(x, mode, eb)
        assert int.from_bytes(st[4:6], "little") == 1, "the oracle no longer writes format 1"
        (HERE / f"{name}.lopc").write_bytes(st)
        np.save(HERE / f"{name}_xhat.npy", oracle.decompress(st))
        print(name, len(st), "bytes")


if __name__ == "__main__":
    main()
