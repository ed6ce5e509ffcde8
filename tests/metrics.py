"""Error metric of Sec. 3.1: per-particle |F_alg - F_ref| / |F_ref|.

The paper's metric has no floor; particles whose reference force is below
1e-6 of the rms reference force are excluded (their relative error is not
meaningful) and counted separately."""
import numpy as np


def rel_err(a, ref, floor=1e-6):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    mag = np.linalg.norm(ref, axis=0)
    rms = np.sqrt(np.mean(mag ** 2)) if mag.size else 0.0
    keep = mag >= floor * rms
    keep &= mag > 0
    err = np.linalg.norm(a - ref, axis=0)[keep] / mag[keep]
    return err, int((~keep).sum())
