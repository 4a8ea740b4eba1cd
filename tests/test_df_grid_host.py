"""The frame and transform grid the library picks for each darkfield solve (an
implementation choice, Eq. 13 unchanged) keep the two correlations of the solve
exact.

For every used image the library reports whether it solves with x and y swapped
and the row x column grid of its register-FFT solve. On that circular grid the
FFT correlations must equal the correlations without wrap-around:
  C u   (k in Q) = sum_q u(q) conj P(q - k)      (Eq. 12-13, q in U)
  C^H r (q in U) = sum_k P(q - k) r(k)           (k in Q)
whose reference is the same correlation on a 1024 x 1024 grid, larger than any
difference of the sets' coordinates (|c| < 256), so nothing can wrap there. A
grid half the chosen size must alias (the check is not vacuous). Host-only
plans; numpy float64.
"""
import numpy as np
import pytest

from paper_2407_20469_gb300 import apic, synth

BIG = 1024
# register-FFT grid 16 B >= 4 R + 1 of these geometries (R = 21.2 and 42.5 pixels)
REGISTER_GRID = {128: 96, 256: 192}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2407_20469_gb300 import build
    build.build()


def _grid(points, values, L, M):
    """values at (x, y) points on an M-row, L-column circular grid (x along the rows)."""
    g = np.zeros((M, L), dtype=np.complex128)
    np.add.at(g, (points[:, 1] % M, points[:, 0] % L), values)
    return g


def _correlations(U, P, Q, u, pv, r, L, M):
    """(C u on Q, C^H r on U) by FFT correlation on an L x M grid."""
    gu, gp, gr = _grid(U, u, L, M), _grid(P, pv, L, M), _grid(Q, r, L, M)
    a, b = np.fft.ifft2(gu), np.fft.ifft2(gp)
    cu = np.fft.fft2(a * np.conj(b)) * (L * M)
    chr_ = np.fft.fft2(np.fft.ifft2(gr) * b) * (L * M)
    return cu[Q[:, 1] % M, Q[:, 0] % L], chr_[U[:, 1] % M, U[:, 0] % L]


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n,ill", [(256, synth.illumination()), (128, synth.illumination()),
                                   (128, synth.illumination_8_24()), (256, synth.illumination_12_22())])
def test_solve_grid_keeps_the_correlations_exact(n, ill):
    plan = apic.Plan.from_illumination(n, ill, flags=apic.APIC_HOST_ONLY)
    rng = np.random.default_rng(11)
    mr = REGISTER_GRID[n]
    checked, grids = 0, set()
    for idx in range(plan.info.n_df):
        U, meta = plan.df_set(idx, 0)
        P, _ = plan.df_set(idx, 1)
        Q, _ = plan.df_set(idx, 2)
        tr, mx, my = plan.df_grid(idx)
        if not meta[1]:
            assert (tr, mx, my) == (0, 0, 0)
            continue
        ext = lambda v: int(v.max() - v.min() + 1)
        assert tr == int(ext(Q[:, 0]) < ext(Q[:, 1]))          # rows along the narrower lag band
        assert mx % 16 == 0 and my % 16 == 0 and 0 < mx <= mr and 0 < my <= mr
        if tr:                                                 # solve frame: x <-> y
            U, P, Q = U[:, ::-1], P[:, ::-1], Q[:, ::-1]
        assert max(np.abs(U).max(), np.abs(P).max(), np.abs(Q).max()) < BIG // 4
        u = rng.standard_normal(len(U)) + 1j * rng.standard_normal(len(U))
        pv = rng.standard_normal(len(P)) + 1j * rng.standard_normal(len(P))
        r = rng.standard_normal(len(Q)) + 1j * rng.standard_normal(len(Q))
        cu_ref, chr_ref = _correlations(U, P, Q, u, pv, r, BIG, BIG)
        cu, chr_ = _correlations(U, P, Q, u, pv, r, mx, my)
        assert _rel(cu, cu_ref) < 1e-10 and _rel(chr_, chr_ref) < 1e-10, (idx, mx, my)
        cu_half, chr_half = _correlations(U, P, Q, u, pv, r, mx // 2, my // 2)
        assert max(_rel(cu_half, cu_ref), _rel(chr_half, chr_ref)) > 1e-3, (idx, mx, my)
        checked += 1
        grids.add((mx, my))
    assert checked == plan.info.n_df_used > 0
    if mr == 192:              # the 256-pixel tiles use grids shorter than 192 on both axes
        assert any(g[0] < mr for g in grids) and any(g[1] < mr for g in grids)


DF_GRIDS = [(192, 192), (192, 144), (192, 128), (192, 96), (160, 128), (160, 96), (144, 144)]


def test_every_accepted_grid_override_is_exact():
    """apic_plan_set_df_grid accepts a supported grid for an image only if it keeps
    the image's correlations exact (same FFT-vs-wrap-free check as above), refuses
    unsupported pairs, and refuses at least one supported pair on these images."""
    n = 256
    plan = apic.Plan.from_illumination(n, synth.illumination(), flags=apic.APIC_HOST_ONLY)
    rng = np.random.default_rng(5)
    accepted = refused = 0
    for idx in range(plan.info.n_df):
        U, meta = plan.df_set(idx, 0)
        if not meta[1]:
            with pytest.raises(apic.ApicError):
                plan.set_df_grid(idx, 192, 192)
            continue
        P, _ = plan.df_set(idx, 1)
        Q, _ = plan.df_set(idx, 2)
        tr = plan.df_grid(idx)[0]
        if tr:
            U, P, Q = U[:, ::-1], P[:, ::-1], Q[:, ::-1]
        u = rng.standard_normal(len(U)) + 1j * rng.standard_normal(len(U))
        pv = rng.standard_normal(len(P)) + 1j * rng.standard_normal(len(P))
        r = rng.standard_normal(len(Q)) + 1j * rng.standard_normal(len(Q))
        cu_ref, chr_ref = _correlations(U, P, Q, u, pv, r, BIG, BIG)
        for mx, my in DF_GRIDS:
            try:
                plan.set_df_grid(idx, mx, my)
            except apic.ApicError as e:
                assert "aliases" in str(e)
                refused += 1
                continue
            assert plan.df_grid(idx) == (tr, mx, my)
            cu, chr_ = _correlations(U, P, Q, u, pv, r, mx, my)
            assert _rel(cu, cu_ref) < 1e-10 and _rel(chr_, chr_ref) < 1e-10, (idx, mx, my)
            accepted += 1
        with pytest.raises(apic.ApicError):
            plan.set_df_grid(idx, 176, 128)
    assert accepted > 0 and refused > 0
