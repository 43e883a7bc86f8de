"""Comparison of CUDA-path patterns with oracle patterns (test helper).

Bar (see the tolerance table of the design notes):
* peak positions: |d 2theta| <= 1e-6 deg; d spacings to 1e-12 relative;
* hkl families and multiplicities: identical;
* intensities: |dI| <= tol * I_max for every peak (tol = 1e-5 for the FP32
  variants, 1e-9 for FP64), i.e. relative to the largest peak, the scale on
  which the paper quotes its intensity agreement (Sec. 3); FP64 is also held to
  1e-8 relative elementwise on peaks above 1e-6 I_max;
* with a cutoff, a peak present on one side only is allowed solely when its
  intensity lies within tol of the cutoff threshold (and is reported).
"""
import numpy as np

TT_TOL = 1e-6
I_TOL = {"fp64": 1e-9, "fp32_phase64": 1e-5, "fp32_phasefix": 1e-5}


def families(res, s, p):
    fo = res["peak_fam_off"][s]
    return [(tuple(int(x) for x in res["fam_hkl"][s][f]), int(res["fam_mult"][s][f])) for f in range(fo[p], fo[p + 1])]


def compare_structure(got, ref, s, prec, cutoff, scaled, imax_ref=None):
    """Returns a dict of findings; raises AssertionError on a parity failure."""
    tol = I_TOL[prec]
    gt, rt = np.asarray(got["peak_tt"][s]), np.asarray(ref["peak_tt"][s])
    gI, rI = np.asarray(got["peak_I"][s]), np.asarray(ref["peak_I"][s])
    if scaled:
        imax = 100.0
    else:
        imax = imax_ref if imax_ref is not None else (rI.max() if len(rI) else 0.0)
    i = j = 0
    pairs, xg, xr = [], [], []
    while i < len(gt) and j < len(rt):
        if abs(gt[i] - rt[j]) <= TT_TOL:
            pairs.append((i, j))
            i += 1
            j += 1
        elif gt[i] < rt[j]:
            xg.append(i)
            i += 1
        else:
            xr.append(j)
            j += 1
    xg += list(range(i, len(gt)))
    xr += list(range(j, len(rt)))
    thr = cutoff * imax
    for k in xg:
        assert cutoff > 0 and abs(gI[k] - thr) <= 2 * tol * imax, \
            ("extra GPU peak", s, k, gt[k], gI[k], thr)
    for k in xr:
        assert cutoff > 0 and abs(rI[k] - thr) <= 2 * tol * imax, \
            ("missing GPU peak", s, k, rt[k], rI[k], thr)
    worst_abs = 0.0
    worst_rel = 0.0
    gd, rd = np.asarray(got["peak_d"][s]), np.asarray(ref["peak_d"][s])
    for a, b in pairs:
        assert families(got, s, a) == families(ref, s, b), ("families", s, a, families(got, s, a), families(ref, s, b))
        assert abs(gd[a] - rd[b]) <= 1e-12 * rd[b], ("d spacing", s, a, gd[a], rd[b])
        d = abs(gI[a] - rI[b])
        worst_abs = max(worst_abs, d / imax if imax > 0 else d)
        if rI[b] > 1e-6 * imax:
            worst_rel = max(worst_rel, d / rI[b])
        assert d <= tol * imax + 1e-300, ("intensity", s, a, gt[a], gI[a], rI[b], d / imax)
    if prec == "fp64":
        assert worst_rel <= 1e-8, ("fp64 elementwise", s, worst_rel)
    return {"pairs": len(pairs), "boundary": len(xg) + len(xr), "max_abs_rel_to_max": worst_abs,
            "max_rel": worst_rel}


def compare_batch(got, ref, prec, cutoff, scaled):
    n = len(ref["peak_tt"])
    assert len(got["peak_tt"]) == n
    stats = {"pairs": 0, "boundary": 0, "max_abs_rel_to_max": 0.0, "max_rel": 0.0}
    for s in range(n):
        assert int(got["status"][s]) == int(ref["status"][s]), ("status", s, got["status"][s], ref["status"][s])
        r = compare_structure(got, ref, s, prec, cutoff, scaled)
        stats["pairs"] += r["pairs"]
        stats["boundary"] += r["boundary"]
        stats["max_abs_rel_to_max"] = max(stats["max_abs_rel_to_max"], r["max_abs_rel_to_max"])
        stats["max_rel"] = max(stats["max_rel"], r["max_rel"])
    return stats
