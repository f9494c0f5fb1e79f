"""FP64 numpy statements of the flow metrics of the paper's comparisons (oracle side).

TEST INFRASTRUCTURE ONLY (imported by tests/ and never by the library); shares no code with the
CUDA path.

  similarity_index: the similarity index of Sec. 3.4 between a high- and a low-resolution
    velocity field on a set of points, read with the factor 1/2 that bounds it by 1 (the printed
    form ranges over [0, 2]): SI = mean_p 1/2 (1 + cos theta_p)(1 - | |u_a|/max|u_a| - |u_b|/max|u_b| |),
    the maxima over the same point set; a point where either vector is zero has cos theta = 0.
  time_mean: the running mean of sampled fields (the time averaging of Sec. 3.3).
"""
import numpy as np


def similarity_index(u_a, u_b, mask):
    """u_a, u_b: (3, ...) velocity fields; mask: (...) nonzero at the points compared."""
    sel = np.asarray(mask) != 0
    a = np.asarray(u_a, dtype=np.float64)[:, sel]
    b = np.asarray(u_b, dtype=np.float64)[:, sel]
    if a.shape[1] == 0:
        return 0.0
    na = np.sqrt((a * a).sum(0))
    nb = np.sqrt((b * b).sum(0))
    dot = (a * b).sum(0)
    both = (na > 0) & (nb > 0)
    cos = np.zeros_like(na)
    cos[both] = dot[both] / (na[both] * nb[both])
    ma, mb = na.max(), nb.max()
    ra = na / ma if ma > 0 else np.zeros_like(na)
    rb = nb / mb if mb > 0 else np.zeros_like(nb)
    return float(np.mean(0.5 * (1.0 + cos) * (1.0 - np.abs(ra - rb))))


def time_mean(samples):
    """Mean of a sequence of equally shaped arrays, accumulated in FP64 in order."""
    acc = None
    n = 0
    for s in samples:
        s = np.asarray(s, dtype=np.float64)
        acc = s.copy() if acc is None else acc + s
        n += 1
    return acc / n
