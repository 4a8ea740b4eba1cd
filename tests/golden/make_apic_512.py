"""Writes apic_512_8x24.npz: the float64 checker's reconstruction of one seeded
512 x 512 tile with 8 NA-matching + 24 darkfield images (the mixed-precision
workload's tile; inputs from tests/helpers.golden_512_inputs).

Only the checker (oracle/) computes the stored values. Stored: the known
spectrum after the brightfield stitch and after the darkfield extension (masks
packed by np.packbits over the 1024 x 1024 output grid, values complex64 in
row-major order of the final mask), the 15 Noll coefficients, the per-image
float64 sums of the inputs (to catch an input recipe that drifted), the
darkfield sets' sizes.

    python tests/golden/make_apic_512.py      # about 10 minutes on 8 cores
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from helpers import GOLDEN_512_SEED, golden_512_inputs  # noqa: E402
from oracle import apic as oapic  # noqa: E402

OUT = os.path.join(HERE, "apic_512_8x24.npz")


def main():
    t0 = time.time()
    I, c_true, g, k, ill = golden_512_inputs()
    I64 = I.astype(np.float64)
    n_bf = ill.n_bf
    X = [oapic.kk_spectrum(I64[i], k[i], g) for i in range(n_bf)]
    rows = oapic.overlap_rows(g, k[:n_bf])
    c15 = oapic.aberration_solve(oapic.phase_differences(X, rows), rows)
    spec = oapic.stitch_brightfield(X, g, k[:n_bf], c15)
    bf_known = spec.known.copy()
    log = oapic.darkfield_extend(spec, I64[n_bf:], g, k[n_bf:], c15)
    known = spec.known
    np.savez_compressed(
        OUT,
        seed=np.int64(GOLDEN_512_SEED),
        shape=np.array(known.shape, np.int64),
        known=np.packbits(known.ravel()),
        bf_known=np.packbits(bf_known.ravel()),
        values=spec.values[known].astype(np.complex64),
        c15=c15,
        c_true=c_true,
        input_sums=I64.sum(axis=(1, 2)),
        df_sizes=np.array([[len(s.U), len(s.P), len(s.Q), int(s.used)] for s in log], np.int64),
    )
    print(f"wrote {OUT} in {time.time() - t0:.0f} s; pupil error vs truth "
          f"{np.sqrt(np.sum((c15[3:] - c_true[3:]) ** 2)):.3e} rad")


if __name__ == "__main__":
    main()
