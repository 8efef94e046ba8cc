"""Plan-quality figures from the GPU dose-volume histogram counts
(vmat_dvh): host-side arithmetic on a few thousand bins, for reports."""
import numpy as np


def dvh_metrics(counts, dose_max, names, rx):
    """Cumulative DVH per structure and a few plan-quality figures from the
    counts: mean dose (bin centres), D95 / D5 (dose received by 95% / 5% of
    the volume, lower bin edge), V(rx) (fraction at or above the
    prescription rx)."""
    n_bins = counts.shape[1]
    w = dose_max / n_bins
    out = {}
    for s, name in enumerate(names):
        c = counts[s]
        n = int(c.sum())
        if n == 0:
            continue
        cum = np.cumsum(c[::-1])[::-1] / n  # fraction receiving >= bin lower edge
        centres = (np.arange(n_bins) + 0.5) * w

        def dq(q):
            idx = np.flatnonzero(cum >= q)
            return float(idx[-1] * w) if idx.size else 0.0
        out[name] = {"voxels": n, "mean": float((c * centres).sum() / n), "D95": dq(0.95),
                     "D5": dq(0.05), "V_rx": float(cum[min(n_bins - 1, int(rx / w))])}
    return out
