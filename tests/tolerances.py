"""Parity tolerances of the CUDA path against the oracle, one rule for every GPU test.

Per precision mode: (readout bound, degenerate-cut threshold, unit roundoff of the contractions,
unit roundoff of the eigensolvers).

* Readouts (normalised expectations, density-matrix entries, probabilities): the bound the target
  states per result, 1e-6 absolute in MIXED (complex64 contractions, FP64 truncation eigensolvers)
  and 1e-10 in FP64, on the readouts of the unnormalised state Tr(rho O), whose norm starts at 1.
  Every rounding error is committed relative to the norm of the state at that time, and nothing is
  renormalised (Sec. II.D truncations only discard weight, the channels preserve the trace), so on
  a normalised readout Tr(rho O) / Tr(rho) the bound becomes bound / Tr(rho) of the final state.  FP32 mode (complex64 with FP32 eigensolvers) is not one of the target's
  modes: its eigensolvers add a backward error of about sqrt(n) u32 ||G|| per truncation, up to
  sqrt(256) = 16 times the complex64 Gram's own 2 u32, so its readouts are held to 3e-6.  The only
  addition is the oracle's cut_allowance(threshold): truncations whose relative eigenvalue gap at
  the cut is below the threshold (1e-5 complex64, 1e-9 FP64) cut inside a near-degenerate cluster,
  where the truncation of Sec. II.D is not unique; cuts above it add nothing.
* Cumulative discarded weights: per truncation the weight 1 - kept / total is read off the
  eigenvalues of a Gram matrix G whose entries carry a relative error of at most gamma = 2u (one
  rounding of the stored elements, compensated sums), i.e. ||dG||_F <= gamma tr G.  By Ky Fan's
  inequality the sum of the k kept eigenvalues then moves by at most sqrt(k) gamma tr G and the
  trace by gamma tr G; the eigensolver adds its backward error, about sqrt(n) u_eig ||G|| per
  eigenvalue (n = order of G), to the k kept eigenvalues and to the n diagonal entries whose sum is
  the trace.  So |dw_t| <= (sqrt(k) + 1) 2u + (k + n) sqrt(n) u_eig, summed over the truncations of
  that kind; a near-degenerate cut can change every later truncation, so the readout allowance is
  added once per truncation.
"""
import math

MODES = {
    "fp64": (1e-10, 1e-9, 2.0 ** -53, 2.0 ** -53),
    "mixed": (1e-6, 1e-5, 2.0 ** -24, 2.0 ** -53),
    "fp32": (3e-6, 1e-5, 2.0 ** -24, 2.0 ** -24),
}


def allowance(orc, prec: str) -> float:
    return orc.cut_allowance(MODES[prec][1])


def readout_limit(orc, prec: str, scale: float = 1.0) -> float:
    """Bound on |GPU - oracle| for a normalised readout of an operator of norm `scale`."""
    return scale * (MODES[prec][0] / min(1.0, orc.trace()) + allowance(orc, prec))


def discarded_limit(orc, prec: str, kind: str) -> float:
    """Bound on the cumulative discarded weight of the bond ("chi") or Kraus-leg ("kappa") cuts."""
    _, _, u, ue = MODES[prec]
    b = sum((math.sqrt(kept) + 1) * 2 * u + (kept + avail) * math.sqrt(avail) * ue
            for k, _, kept, avail, _ in orc.log if k == kind)
    return b + len(orc.log) * allowance(orc, prec)
