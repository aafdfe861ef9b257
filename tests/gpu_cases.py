"""Seeded fields shared by the GPU test files: several tiles with ragged edges, very tight
bounds, degenerate shapes, heavy ties, deep repair chains, signed zeros and denormals."""
import numpy as np

from paper_2603_26968_b300 import synth as S


def bumps(shape, dtype, seed=1, n=24, noise=1e-4):
    f = np.zeros(shape, np.float64)
    S.add_bumps(f, n, max(shape) / 40.0, max(shape) / 5.0, seed)
    if noise:
        S.add_uniform_noise(f, noise, seed)
    return f.astype(dtype)


CASES = [
    ("2d_f32_c1", lambda: S.make_field(S.spec_2d_small()), 1, 1e-3),
    ("2d_f32_c1_loose", lambda: S.make_field(S.spec_2d_small()), 1, 1e-2),
    ("2d_f32_c1_tight", lambda: S.make_field(S.spec_2d_small()), 1, 1e-4),
    ("2d_f32_ragged", lambda: bumps((130, 200), np.float32), 1, 1e-2),
    ("2d_f64_ragged", lambda: bumps((100, 150), np.float64), 1, 1e-3),
    ("2d_f64_abs", lambda: bumps((70, 65), np.float64), 0, 2e-3),
    ("3d_f32_ragged", lambda: S.make_field(S.spec_3d_f32(n=48))[:45, :40, :37].copy(), 1, 1e-3),
    ("3d_f32_loose", lambda: S.make_field(S.spec_3d_f32(n=48)), 1, 1e-2),
    ("3d_f32_tight", lambda: S.make_field(S.spec_3d_f32(n=40)), 1, 1e-4),
    ("3d_f64_ties", lambda: S.make_field(S.spec_3d_f64_ties(shape=(24, 36, 36))), 1, 5e-4),
    ("3d_f64_ties_ragged", lambda: S.make_field(S.spec_3d_f64_ties(shape=(24, 36, 36)))[:19, :35, :33].copy(), 1, 5e-4),
    ("3d_f64_abs", lambda: bumps((17, 20, 23), np.float64), 0, 1e-3),
    # very tight bounds: bin residuals reach 14-40 bit planes (the transposes' packed,
    # 32-plane and 64-bit paths)
    ("3d_f32_eb1e-6", lambda: S.make_field(S.spec_3d_f32(n=40)), 1, 1e-6),
    ("2d_f32_eb1e-6", lambda: bumps((130, 200), np.float32), 1, 1e-6),
    ("2d_f64_eb1e-10", lambda: bumps((100, 150), np.float64), 1, 1e-10),
    ("3d_f64_eb1e-12", lambda: bumps((17, 20, 23), np.float64, noise=0), 1, 1e-12),
    ("row_1xN", lambda: bumps((1, 777), np.float32), 1, 1e-2),
    ("col_Nx1", lambda: bumps((300, 1), np.float64), 1, 1e-2),
    ("3d_thin_z", lambda: bumps((1, 40, 50), np.float32), 1, 1e-2),
    ("3d_two_z", lambda: bumps((2, 33, 17), np.float64), 1, 1e-2),
    ("3d_line", lambda: bumps((70, 1, 1), np.float32), 1, 1e-2),
    ("tiny_2x2", lambda: np.array([[0.0, 1.0], [1.0, 0.0]], np.float32), 1, 0.6),
    ("single_point", lambda: np.array([[3.5]], np.float64), 0, 1e-3),
    ("constant_noa", lambda: np.full((20, 30, 40), -1.25, np.float32), 1, 1e-3),
    ("integer_plateaus", lambda: np.floor(bumps((40, 40, 40), np.float32, noise=0) * 3), 1, 0.3),
    ("long_chain_2d", lambda: np.linspace(1.0, 0.0, 2000, dtype=np.float32).reshape(1, 2000), 0, 10.0),
    ("long_chain_3d", lambda: (-np.arange(30 * 31 * 32, dtype=np.float64)).reshape(30, 31, 32), 0, 1e9),
    ("neg_zero_mix", lambda: np.array([[0.0, -0.0, 0.0, -0.0], [1e-30, -1e-30, 0.0, -0.0]], np.float32), 0, 0.5),
    ("denormals", lambda: (np.arange(64, dtype=np.float32).reshape(8, 8) * np.float32(1e-44)), 0, 1e-44),
]
