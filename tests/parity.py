"""Comparison of CUDA-path patterns with oracle patterns (test helper).

Bar (see the tolerance table of the design notes):
* peak positions: |d 2theta| <= 1e-6 deg; d spacings to 1e-12 relative;
* hkl families and multiplicities: identical;
* intensities, every peak: |dI| <= tol * I_max (tol = 1e-5 for the FP32
  variants, 1e-9 for FP64), relative to the largest peak, the scale on which
  the paper quotes its intensity agreement (Sec. 3);
* intensities, elementwise: |dI| / I <= 1e-5 (FP32) on every peak above
  1e-3 I_max -- every kept peak at the default cutoff, and the same floor on
  an uncut list; FP64: 1e-8 on every peak above 1e-6 I_max;
* with a cutoff, a peak present on one side only is allowed solely when its
  intensity lies within tol of the cutoff threshold (and is reported).
"""
import numpy as np

TT_TOL = 1e-6
I_TOL = {"fp64": 1e-9, "fp32_phase64": 1e-5, "fp32_phasefix": 1e-5}
# elementwise relative bar and the floor (fraction of the largest peak) above which it applies
REL_TOL = {"fp64": 1e-8, "fp32_phase64": 1e-5, "fp32_phasefix": 1e-5}
REL_FLOOR = {"fp64": 1e-6, "fp32_phase64": 1e-3, "fp32_phasefix": 1e-3}


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
        assert d <= tol * imax + 1e-300, ("intensity", s, a, gt[a], gI[a], rI[b], d / imax)
        if rI[b] > REL_FLOOR[prec] * imax:
            worst_rel = max(worst_rel, d / rI[b])
            assert d <= REL_TOL[prec] * rI[b], ("elementwise intensity", prec, s, a, gt[a], gI[a], rI[b], d / rI[b])
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


def half_space(hkl):
    """Rows of a full-sphere hkl list in the Friedel half-space (first nonzero index positive)."""
    h, k, l = hkl[:, 0], hkl[:, 1], hkl[:, 2]
    return (h > 0) | ((h == 0) & (k > 0)) | ((h == 0) & (k == 0) & (l > 0))


def compare_reflections(got, ref, s, prec, q_of=None, r2=None):
    """Per-reflection list of structure s (GPU: Friedel-unique) against the oracle's full sphere.

    * hkl set identical (bit-exact), except a reflection whose oracle |g|^2 lies within 4 ulp of a
      sphere radius^2 (boundary-ambiguous: reported, not failed). q_of(hkl) gives the oracle's |g|^2
      and r2 = (r_min^2, r_max^2) for that check;
    * 2-theta to 1e-6 degrees; the GPU list ascends in 2-theta;
    * intensity of each reflection: |dI| <= 1e-5 max(I, 1e-3 M) (FP32; M the largest reflection
      intensity), 1e-9 max(I, 1e-6 M) (FP64) -- the per-reflection form of the peak bar.
    Returns a dict of counts and the largest errors."""
    gh = np.asarray(got["refl_hkl"][s]).reshape(-1, 3)
    rh = np.asarray(ref["refl_hkl"])
    sel = half_space(rh)
    rh, rtt, rI = rh[sel], np.asarray(ref["refl_tt"])[sel], np.asarray(ref["refl_I"])[sel]
    gk = {tuple(v): i for i, v in enumerate(gh.tolist())}
    rk = {tuple(v): i for i, v in enumerate(rh.tolist())}
    only_g = [k for k in gk if k not in rk]
    only_r = [k for k in rk if k not in gk]
    ambiguous = 0
    for k in only_g + only_r:
        assert q_of is not None and r2 is not None, ("hkl sets differ", s, k)
        q = q_of(k)
        near = min(abs(q - r2[0]), abs(q - r2[1]))
        assert near <= 4 * np.spacing(max(r2[1], 1e-300)), ("hkl sets differ off the boundary", s, k, q, r2)
        ambiguous += 1
    gtt, gI = np.asarray(got["refl_tt"][s]), np.asarray(got["refl_I"][s])
    assert np.all(np.diff(gtt) >= -1e-9), ("GPU list not ascending in 2-theta", s)  # up to 2-theta's rounding
    common = [k for k in gk if k in rk]
    gi = np.array([gk[k] for k in common], dtype=np.int64)
    ri = np.array([rk[k] for k in common], dtype=np.int64)
    if len(common) == 0:
        return {"refl": 0, "ambiguous": ambiguous, "max_tt": 0.0, "max_rel": 0.0}
    dtt = np.abs(gtt[gi] - rtt[ri])
    assert dtt.max() <= TT_TOL, ("reflection 2-theta", s, dtt.max())
    M = rI.max()
    tol, floor = (1e-9, 1e-6) if prec == "fp64" else (1e-5, 1e-3)
    dI = np.abs(gI[gi] - rI[ri])
    bound = tol * np.maximum(rI[ri], floor * M)
    bad = np.nonzero(dI > bound)[0]
    assert len(bad) == 0, ("reflection intensity", prec, s, [(common[j], gI[gi[j]], rI[ri[j]]) for j in bad[:5]])
    strong = rI[ri] > floor * M
    rel = float((dI[strong] / rI[ri][strong]).max()) if strong.any() else 0.0
    return {"refl": len(common), "ambiguous": ambiguous, "max_tt": float(dtt.max()), "max_rel": rel}
