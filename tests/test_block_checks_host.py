"""The per-(m, parity) checks of the split-path tests, exercised on the CPU
with mistakes planted in oracle outputs: a missing tile of one high-m
Legendre problem slips under the whole-output relative L2 bound of the
split path (1e-6) on the steep spectra of the workloads, and the block
checks catch it, while split-sized rounding passes both."""
import numpy as np

import oracle as O
from paper_1711_11296_gb300 import workloads as W
from sht_testutil import grid_block_errors, rel_l2, spec_block_errors, worst

N, J, I, F = 63, 129, 256, 2
JH = (J + 1) // 2


def _synthesis_without_tile(a, m_drop, q_drop, rows):
    """The oracle's synthesis with the contribution of problem (m_drop,
    q_drop) removed at the northern latitudes ``rows`` (0-based): what an
    inverse contraction that skipped one row tile of that problem would
    leave (its hemisphere-mirrored rows lose the same S or A part)."""
    g = O.synthesis(a, N, J, I)
    r0 = O.coef_offset(N, m_drop)
    part = np.zeros_like(a)
    sl = slice(r0 + q_drop, r0 + N - m_drop + 1, 2)
    part[sl] = a[sl]
    gp = O.synthesis(part, N, J, I)
    rows = np.asarray(rows)
    g[:, rows] -= gp[:, rows]
    g[:, J - 1 - rows] -= gp[:, J - 1 - rows]
    return g


def _rounding(x, eps, seed):
    g = np.random.default_rng(seed)
    return x * (1 + eps * g.standard_normal(x.shape))


def test_dropped_inverse_tile_escapes_global_bound_but_not_block_check():
    rows = np.arange(20, 36)                       # a 16-row mid-latitude tile
    steep = W.random_spectrum(N, F, "n^-1.5", seed=5)
    ref = O.synthesis(steep, N, J, I)
    bad = _synthesis_without_tile(steep, 58, 1, rows)
    assert rel_l2(bad, ref) < 1e-6                 # the global bound misses it
    flat = W.random_spectrum(N, F, "flat", seed=6)
    ref = O.synthesis(flat, N, J, I)
    bad = _synthesis_without_tile(flat, 58, 1, rows)
    north, south = np.arange(JH), J - 1 - np.arange(JH)
    errs = grid_block_errors(bad[:, north], bad[:, south], ref[:, north], ref[:, south], N,
                             floor=0.1)
    e, k = worst(errs)
    assert k == (58, 1) and e > 1e-5
    ok = _rounding(ref, 1e-7, 7)
    errs = grid_block_errors(ok[:, north], ok[:, south], ref[:, north], ref[:, south], N,
                             floor=0.1)
    assert worst(errs)[0] < 4e-6


def test_dropped_forward_rows_caught_by_block_check():
    x = W.random_grid(F, J, I, seed=8)
    ref = O.analysis(x, N)
    bad = ref.copy()
    r0 = O.coef_offset(N, 61)
    bad[r0 + 1:r0 + 3:2] = 0.0                     # problem (61, odd) lost
    errs = spec_block_errors(bad, ref, N)
    assert worst(errs)[1] == (61, 1) and worst(errs)[0] == 1.0
    assert worst(spec_block_errors(_rounding(ref, 1e-7, 9), ref, N))[0] < 4e-6
