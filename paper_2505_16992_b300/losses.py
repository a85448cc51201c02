"""User-side loss code built on the library's differentiable statistics.

The statistics loss of Sec. 3.3 (Eq. TCFstatsLossGeneric) is not part of the
solver: it is the kind of objective a user writes in PyTorch on top of the
records the CUDA library produces (``solver.frame_record`` and
``solver.time_averaged_record``, whose backward passes run the library's
record-adjoint kernels).  The few elementwise tensor operations below are
that user-side composition; every statistic they read comes from the library.
"""
from __future__ import annotations

from .solver import PlaneStats, frame_record, time_averaged_record


def stats_loss(stats: PlaneStats, qs, ref_mean, ref_m2, lam_U=1.0, lam_uu=1.0, lam_frame=1.0):
    """L_stats of Eq. TCFstatsLossGeneric (Sec. 3.3) with one weight per kind:
    squared errors of the mean profiles and second-order statistics per plane
    (averaged over the planes) for the time-averaged record of all frames plus
    lam_frame times the same terms of every frame's own record."""
    def terms(rec):
        _, mean, m2, _ = stats.split(rec)
        ny = mean.shape[0]
        return (lam_U * ((mean - ref_mean) ** 2).sum() + lam_uu * ((m2 - ref_m2) ** 2).sum()) / ny
    total = terms(time_averaged_record(stats, qs))
    for q in qs:
        total = total + lam_frame * terms(frame_record(stats, q))
    return total
