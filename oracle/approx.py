"""CPU oracle for subband dedispersion, the thesis's two-step approximation of
the brute-force sum (Sec. 2.1.3, subband dedispersion), for time binning past
the diagonal DM (Sec. 2.1.1 and the downfactoring procedure of Sec. 2.1.2),
and the analytic S/N loss of a pulse dedispersed at a wrong DM (Sec. 3.6,
candidate classification after Cordes & McLaughlin).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.  Both steps are plain
brute-force sums over delay tables, so each runs through ``oracle.dedisperse``
(the C oracle) on tables built here from the brute-force table T[c][d]:

* the trial DMs fall into groups of ``dms_per_group`` consecutive trials; each
  group is represented by one nominal trial (its middle one, the lower of the
  two middle ones for an even group);
* step 1 dedisperses each subband of ``chans_per_subband`` adjacent channels
  (first channel c_s) at the nominal trials only, with delays relative to the
  subband's first channel:  d1[c][n] = T[c][n] - T[c_s][n];
* step 2 treats the subband series as channels and dedisperses them at every
  trial of the nominal's group with the delays of the subbands' first
  channels:  d2[s][d] = T[c_s][d].

Hence at a nominal trial the result equals the brute-force sum exactly, and
elsewhere each subband is summed with its nominal trial's internal delays.
Output length: nsamp_in - (D1 + D2), D1 = largest step-1 delay over all
subbands, D2 = largest step-2 delay over all groups.  Readings where the
thesis is silent (group representative, delays as differences of the
brute-force table, common lengths) are listed in the design notes.
"""
from __future__ import annotations

import math

import numpy as np

from . import dedisperse


class SubbandTables:
    """Delay tables of the two steps for a brute-force table T[nchan][ndm]."""

    def __init__(self, delays: np.ndarray, chans_per_subband: int, dms_per_group: int):
        T = np.asarray(delays, dtype=np.int64)
        nchan, ndm = T.shape
        if chans_per_subband < 1 or dms_per_group < 1:
            raise ValueError("subband and group sizes must be >= 1")
        self.nchan, self.ndm = nchan, ndm
        self.first = list(range(0, nchan, chans_per_subband))  # c_s
        self.nsub = len(self.first)
        self.groups = [(g0, min(ndm, g0 + dms_per_group)) for g0 in range(0, ndm, dms_per_group)]
        self.nominal = [g0 + (g1 - g0 - 1) // 2 for g0, g1 in self.groups]
        # step 1: per subband [channels of s][nominal]
        self.d1 = []
        for s, c0 in enumerate(self.first):
            c1 = min(nchan, c0 + chans_per_subband)
            self.d1.append((T[c0:c1][:, self.nominal] - T[c0][self.nominal]).astype(np.int32))
        # step 2: per group [subband][trial of the group]
        self.d2 = [T[self.first][:, g0:g1].astype(np.int32) for g0, g1 in self.groups]
        self.D1 = max(int(t.max()) for t in self.d1)
        self.D2 = max(int(t.max()) for t in self.d2)
        self.maxshift = self.D1 + self.D2


def subband_dedisperse(block: np.ndarray, delays: np.ndarray, chans_per_subband: int,
                       dms_per_group: int, nsamp_in: int | None = None) -> np.ndarray:
    """Two-step subband dedispersion of block[nchan][>= nsamp_in].

    uint8 input: step-1 sums are exact integers, carried into step 2 as
    float32 (exact below 2^24) and the result returned as int32 (exact).
    Float input: step 1 sums in double, its series are stored as float32
    (the device keeps them in float), step 2 sums in double; float64 result.
    """
    tb = SubbandTables(delays, chans_per_subband, dms_per_group)
    if nsamp_in is None:
        nsamp_in = block.shape[1]
    L1 = nsamp_in - tb.D1
    nsamp_out = L1 - tb.D2
    if nsamp_out < 1:
        raise ValueError("block shorter than the subband plan's delays")
    nnom = len(tb.nominal)
    sb = np.empty((nnom, tb.nsub, L1), dtype=np.float32)
    for s, c0 in enumerate(tb.first):
        c1 = c0 + tb.d1[s].shape[0]
        part = dedisperse(np.ascontiguousarray(block[c0:c1]), tb.d1[s], nsamp_out=L1,
                          nsamp_in=nsamp_in)
        sb[:, s, :] = part.astype(np.float32)
    out = np.empty((tb.ndm, nsamp_out), dtype=np.int32 if block.dtype == np.uint8 else np.float64)
    for g, (g0, g1) in enumerate(tb.groups):
        D = dedisperse(np.ascontiguousarray(sb[g]), tb.d2[g], nsamp_out=nsamp_out, nsamp_in=L1)
        out[g0:g1] = D if block.dtype != np.uint8 else np.rint(D).astype(np.int32)
    return out


def smearing_peak_ratio(ddm: float, bandwidth_mhz: float, f_centre_ghz: float,
                        width_ms: float) -> float:
    """Peak of a Gaussian pulse (FWHM ``width_ms``) dedispersed with a DM error
    ``ddm`` over a flat band of ``bandwidth_mhz`` centred at ``f_centre_ghz``,
    relative to its peak at the true DM (Sec. 3.6):
        S(dDM)/S = sqrt(pi)/2 * erf(zeta) / zeta,
        zeta = 6.91e-3 dDM bandwidth_MHz / (W_ms f_GHz^3)."""
    zeta = 6.91e-3 * abs(ddm) * bandwidth_mhz / (width_ms * f_centre_ghz ** 3)
    if zeta == 0:
        return 1.0
    return math.sqrt(math.pi) / 2 * math.erf(zeta) / zeta


# ---------------------------------------------------------------- time binning
#
# Above the diagonal DM a channel's dispersion sweep is wider than a sample, so
# the thesis dedisperses the higher DM ranges from a time series downfactored
# by 2 (adjacent samples summed), 4, ...: trials below twice the diagonal DM
# at full resolution, trials in [2^k, 2^(k+1)) x DM_diag from the series
# binned by 2^k (capped at max_factor), with delays at 2^k sampling times.
# The 8-bit variant keeps uint8 binned series (rounded means instead of sums,
# which need 9 or more bits), at the cost of a rounding error of at most half
# a count per halving; it is not in the thesis.


def diagonal_dm(nchan: int, f_top_mhz: float, chan_width_mhz: float, t_samp_s: float,
                k_dm: float = 4.148808e3) -> float:
    """DM at which the dispersion delay across one channel at the bottom of the
    band equals one sample: d/dc [K DM (f_c^-2 - f_top^-2)] = t_samp with
    f_c = f_top - c df, i.e. DM_diag = t_samp f_bot^3 / (2 K df)."""
    f_bot = f_top_mhz - (nchan - 1) * chan_width_mhz
    return t_samp_s * (f_bot * f_bot * f_bot) / (2.0 * k_dm * chan_width_mhz)


def binning_factors(dms: np.ndarray, dm_diag: float, max_factor: int) -> np.ndarray:
    """Downfactor per trial: 1 below 2 DM_diag, else 2^floor(log2(DM/DM_diag)),
    at most max_factor (a power of two)."""
    f = np.ones(len(dms), dtype=np.int32)
    for i, dm in enumerate(np.asarray(dms, dtype=np.float64)):
        k = 1
        while 2 * k <= max_factor and dm >= 2 * k * dm_diag:
            k *= 2
        f[i] = k
    return f


def decimate(block: np.ndarray, nsamp_in: int, factor: int) -> np.ndarray:
    """Sum adjacent samples pairwise, log2(factor) times: b[c][t] = a[c][2t] +
    a[c][2t+1].  Integers for uint8 input (exact), float32 otherwise (in this
    order).  Length nsamp_in // factor."""
    x = block[:, :nsamp_in].astype(np.int64 if block.dtype == np.uint8 else np.float32)
    while factor > 1:
        n = x.shape[1] // 2
        x = x[:, 0:2 * n:2] + x[:, 1:2 * n:2]
        factor //= 2
    return x


def decimate_mean8(block: np.ndarray, nsamp_in: int, factor: int) -> np.ndarray:
    """8-bit binned series of uint8 input (a variant; the thesis sums): each
    halving takes the mean of two adjacent samples rounded half up,
    b[c][t] = floor((a[c][2t] + a[c][2t+1] + 1) / 2), log2(factor) times.
    Length nsamp_in // factor, uint8."""
    if block.dtype != np.uint8:
        raise ValueError("8-bit means need uint8 input")
    x = block[:, :nsamp_in].astype(np.int64)
    while factor > 1:
        n = x.shape[1] // 2
        x = (x[:, 0:2 * n:2] + x[:, 1:2 * n:2] + 1) // 2
        factor //= 2
    return x.astype(np.uint8)


def binned_dedisperse(block: np.ndarray, nchan: int, f_top_mhz: float, chan_width_mhz: float,
                      t_samp_s: float, dms: np.ndarray, max_factor: int,
                      nsamp_in: int | None = None, mode: str = "sum"):
    """Time-binned dedispersion.  Returns (rows, factors, lengths): rows[d] is
    the dedispersed series of trial d at 1/factor[d] of the sampling rate,
    lengths[d] its length (nsamp_in // f - maxshift of its factor's trials at
    f t_samp); int32 for uint8 input, float64 otherwise.  mode "sum" bins by
    summing (the thesis's downfactoring); "mean8" (uint8 input only) bins
    into 8-bit rounded means (decimate_mean8) and dedisperses those."""
    from . import delay_table

    if mode not in ("sum", "mean8"):
        raise ValueError(f"unknown binning mode {mode!r}")
    if mode == "mean8" and block.dtype != np.uint8:
        raise ValueError("8-bit means need uint8 input")
    dms = np.asarray(dms, dtype=np.float64)
    if nsamp_in is None:
        nsamp_in = block.shape[1]
    fac = binning_factors(dms, diagonal_dm(nchan, f_top_mhz, chan_width_mhz, t_samp_s),
                          max_factor)
    rows = [None] * len(dms)
    for f in sorted(set(fac.tolist())):
        idx = np.nonzero(fac == f)[0]
        delays, _ = delay_table(nchan, f_top_mhz, chan_width_mhz, t_samp_s * f, dms[idx])
        if f == 1:
            src, n_in = block, nsamp_in
        elif mode == "mean8":
            src = decimate_mean8(block, nsamp_in, f)
            n_in = src.shape[1]
        else:
            d = decimate(block, nsamp_in, f)
            src = d.astype(np.float32)  # exact for the integer sums of uint8 input
            n_in = d.shape[1]
        D = dedisperse(np.ascontiguousarray(src), delays, nsamp_in=n_in)
        if block.dtype == np.uint8 and D.dtype != np.int32:
            D = np.rint(D).astype(np.int32)
        for j, i in enumerate(idx):
            rows[i] = D[j]
    return rows, fac, np.array([len(r) for r in rows])
