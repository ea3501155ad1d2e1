"""Shared comparison rules of the GPU parity tests (CUDA path vs the FP64 oracle).

Tolerances:
* integer work (shift table, segment counts, event / pulse indices): bit-exact;
* FP32 amplitudes |G|: relative 1e-4 (the FP32 transform's error is ~1e-6 relative);
* argmax cell: exact, except where the oracle's own runner-up is within 1e-5 of the
  maximum (then the GPU's cell must hold an oracle value within 1e-5 of the maximum);
* normalised power P: absolute 1e-4 * (1 + |P| + mean/std), the propagation of the
  amplitude tolerance through Eq. 6; crossings with |P - threshold| below that band
  may fall on either side and are compared separately.
"""
import numpy as np

from oracle import reference as R

AMP_RTOL = 1e-4
TIE_RTOL = 1e-5


def assert_fit_match(st, vis, dk, segs, gpu, ref, allow=(None, None)):
    """gpu: frbx_seg records; ref: (amp, m, q, amp2) of the oracle for the same segs."""
    a, m, q, a2 = ref[:4]
    ga = gpu["amp"].astype(np.float64)
    gm = gpu["sbd_idx"].astype(np.int64)
    gq = gpu["mbd_idx"].astype(np.int64)
    np.testing.assert_allclose(ga, a, rtol=AMP_RTOL, atol=1e-6 * max(1.0, float(np.max(a, initial=1.0))))
    diff = np.flatnonzero((gm != m) | (gq != q))
    if diff.size:
        near = (a[diff] - a2[diff]) <= TIE_RTOL * a[diff]
        assert near.all(), f"argmax differs off a near tie at rows {diff[~near][:10]}"
        _, _, _, _, grid = R.fit_segments(st, vis, dk, segs[diff], allow[0], allow[1], want_grid=True)
        for k, i in enumerate(diff):
            v = abs(grid[k][gm[i], gq[i]])
            assert v >= (1 - TIE_RTOL) * a[i], (i, v, a[i])
    return diff.size


def p_band(P_or, mean_over_std):
    return 1e-4 * (1.0 + np.abs(P_or) + mean_over_std)
