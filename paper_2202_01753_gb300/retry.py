"""Calls per iteration for the retry of an integral that ended unconverged.

The accuracy protocol of Sec. 5.1 raises the number of samples for tighter
tolerances without a rule; this is the library's, the same as the server's
(mcubes_server_set_escalation / mcubes_server_set_retry_sized in
include/mcubes.h), for host loops over batches.
"""
from __future__ import annotations

import math


def retry_ncall(ncall: int, estimate: float, sigma: float, rel_tol: float, abs_tol: float,
                min_factor: float, max_factor: float, ncall_max: int) -> int:
    """Fixed rule (max_factor <= 0): ncall x min_factor while that stays
    <= ncall_max, else ncall (no retry).  Sized rule: sigma falls as
    (calls x iterations)^-1/2, so ncall x 2 (sigma/tau)^2 calls reach the
    tolerance tau = max(abs_tol, rel_tol |estimate|); the factor is clamped
    to [min_factor, max_factor] (max_factor when tau is not positive) and
    the calls to ncall_max."""
    if max_factor <= 0.0:
        more = ncall * min_factor
        return int(more) if more <= ncall_max else ncall
    tau = max(abs_tol, rel_tol * abs(estimate))
    k = max_factor
    if tau > 0.0 and math.isfinite(sigma):
        q = sigma / tau
        k = min(max_factor, max(min_factor, 2.0 * q * q))
    return int(min(ncall * k, float(ncall_max)))
