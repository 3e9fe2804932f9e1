"""Solidification kinetics: the paper's Table I, its rate fit, and comparisons of quench ensembles.

Host analysis of the output of ``quench.py`` (no GPU work). It covers:

- ``TABLE_I``: the lifetimes of the supercooled liquid that the paper lists for Ni2057 at 780-835 K
  (Sec. III D, Table I), in ps, one list per temperature.
- ``kappa_fit``: the paper's fit of the escape rate against temperature (Eq. rate3) with its printed
  constants a = 1.24, b = 31053 eV K^2, T0 = 1029 K. The paper writes the left side as ln(kappa * 1 fs);
  with those constants only ln(kappa * 1 ps) reproduces its own table (780 K: 2.01e-3 against the listed
  1.99e-3 ps^-1) and its precursor frequency e^a = 3.5 ps^-1, so kappa is in ps^-1 here.
- ``temperature_for_kappa``: the inverse of that fit on the supercooled branch T0/3 < T < T0.
- ``rate_mle``: the exponential escape rate from lifetimes with right censoring (events / time at risk).
- ``rate_ratio``: a ratio of two such rates with its confidence interval. For exponential lifetimes,
  2 kappa (total time at risk) follows chi^2 with 2 d degrees of freedom for d events (exact without
  censoring, the usual approximation with it). The estimate of kappa_a / kappa_b over its true value is
  then [chi^2(2 d_b) / 2 d_b] / [chi^2(2 d_a) / 2 d_a], an F variable with (2 d_b, 2 d_a) degrees of
  freedom.
- ``compare_with_table1`` and ``compare_ensembles``: the statistics quoted for the Table I comparison
  and for the MIXED-against-FP64 ensembles (two-sample Kolmogorov-Smirnov, Fisher's exact test on the
  solidified counts, Mann-Whitney on per-cluster quantities).

- ``fit_rate3``: Eq. rate3 fitted to escape rates measured at several temperatures, free or with T0 fixed.

Usage: python -m paper_1210_3559_gb300.kinetics --table1 780 run_780.json
       python -m paper_1210_3559_gb300.kinetics --compare run_mixed.json run_fp64.json
       python -m paper_1210_3559_gb300.kinetics --fit run_780.json run_800.json run_820.json ...
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

# Table I (Sec. III D): lifetimes in ps of the supercooled liquid of Ni2057, per trajectory.
TABLE_I = {
    780: [80, 170, 230, 240, 280, 310, 360, 370, 380, 530, 540, 570, 740, 750, 2000],
    800: [110, 170, 180, 550, 820, 890, 1260, 1320, 1390, 1600, 1830, 1930, 2210, 2800, 3610],
    820: [100, 1740, 2260, 3600, 5020, 5130, 6670, 7430, 7800, 9450, 11620, 23400],
    830: [3610, 3730, 9340, 18130, 19080, 19760, 22640, 26670, 27670, 36380],
    835: [1160, 3320, 5890, 14680, 20008, 22240, 28640, 30230, 41670, 63180],
}
# The table's own summary rows: mean lifetime (ps) and kappa (1e-5 ps^-1), as printed.
TABLE_I_MEAN_PS = {780: 503, 800: 1378, 820: 6440, 830: 18731, 835: 23102}
TABLE_I_KAPPA_1E5 = {780: 199, 800: 72.6, 820: 15.5, 830: 5.34, 835: 4.33}

KB_EV_PER_K = 8.617333262e-5
FIT_A, FIT_B_EV_K2, FIT_T0_K = 1.24, 31053.0, 1029.0


def kappa_fit(T, a: float = FIT_A, b: float = FIT_B_EV_K2, T0: float = FIT_T0_K):
    """Escape rate (ps^-1) of the paper's fit (Eq. rate3): ln(kappa ps) = a - b / (k_B T (T - T0)^2)."""
    T = np.asarray(T, dtype=np.float64)
    return np.exp(a - b / (KB_EV_PER_K * T * (T - T0) ** 2))


def temperature_for_kappa(kappa: float, a: float = FIT_A, b: float = FIT_B_EV_K2, T0: float = FIT_T0_K) -> float:
    """The temperature on the supercooled branch (T0/3, T0) at which the fit gives kappa (ps^-1).

    T (T0 - T)^2 falls monotonically from T0/3 to T0, so the fitted rate does too; bisection."""
    lo, hi = T0 / 3.0, T0
    target = math.log(kappa)
    if not (a - b / (KB_EV_PER_K * lo * (lo - T0) ** 2) > target):
        raise ValueError(f"kappa {kappa} exceeds the fit's maximum on the supercooled branch")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if a - b / (KB_EV_PER_K * mid * (mid - T0) ** 2) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def rate_mle(lifetimes_ps, n_censored: int = 0, horizon_ps: float = 0.0):
    """(kappa, events, time at risk): events / time at risk for exponential lifetimes, the censored runs
    counted as liquid up to the horizon."""
    t = np.asarray(lifetimes_ps, dtype=np.float64)
    at_risk = float(t.sum() + n_censored * horizon_ps)
    d = int(t.size)
    return (d / at_risk if at_risk > 0 else float("nan")), d, at_risk


def rate_ratio(d_a: int, at_risk_a: float, d_b: int, at_risk_b: float, level: float = 0.95):
    """Ratio kappa_a / kappa_b of two exponential escape rates and its confidence interval.

    (kappa_a_hat / kappa_b_hat) / (kappa_a / kappa_b) ~ F(2 d_b, 2 d_a), so with q the F quantiles the
    interval is [r_hat / q_hi, r_hat / q_lo]."""
    from scipy.stats import f as fdist
    r = (d_a / at_risk_a) / (d_b / at_risk_b)
    alpha = 1.0 - level
    q_lo = fdist.ppf(alpha / 2, 2 * d_b, 2 * d_a)
    q_hi = fdist.ppf(1 - alpha / 2, 2 * d_b, 2 * d_a)
    return r, float(r / q_hi), float(r / q_lo)


def compare_with_table1(T: int, lifetimes_ps, n_censored: int = 0, horizon_ps: float = 0.0) -> dict:
    """Measured lifetimes at temperature T (runs still liquid at the horizon counted as censored) against the
    paper's Table I column for T."""
    from scipy.stats import ks_2samp
    paper = np.asarray(TABLE_I[T], dtype=np.float64)
    ours = np.asarray(lifetimes_ps, dtype=np.float64)
    k_ours, d_ours, risk_ours = rate_mle(ours, n_censored, horizon_ps)
    k_paper, d_paper, risk_paper = rate_mle(paper)
    r, lo, hi = rate_ratio(d_ours, risk_ours, d_paper, risk_paper)
    T_fit = temperature_for_kappa(k_ours)
    return {
        "T_K": T, "runs": int(ours.size + n_censored), "solidified": int(ours.size),
        "mean_ps": float(ours.mean()) if ours.size else None,
        "sem_ps": float(ours.std(ddof=1) / math.sqrt(ours.size)) if ours.size > 1 else None,
        "paper_mean_ps": float(paper.mean()), "paper_sem_ps": float(paper.std(ddof=1) / math.sqrt(paper.size)),
        "kappa_per_ps": k_ours, "paper_kappa_per_ps": k_paper, "paper_fit_kappa_per_ps": float(kappa_fit(T)),
        "rate_ratio": r, "rate_ratio_ci95": [lo, hi],
        "ks_p": float(ks_2samp(ours, paper).pvalue),
        "fit_temperature_for_our_kappa_K": T_fit, "fit_offset_K": T_fit - T,
    }


def fit_rate3(T, kappa, events=None, T0: float | None = None) -> dict:
    """Least-squares fit of Eq. rate3, ln(kappa ps) = a - b / (k_B T (T - T0)^2), to escape rates kappa (ps^-1)
    measured at temperatures T (K). With `events` (solidified runs per temperature), each ln(kappa) is
    weighted by its standard error 1/sqrt(events) (exponential lifetimes). T0=None fits (a, b, T0); a given
    T0 (e.g. the paper's 1029 K) fits (a, b) alone, which stays well conditioned with few temperatures.
    Returns the parameters, their standard errors, and the residuals of ln(kappa)."""
    from scipy.optimize import curve_fit
    T = np.asarray(T, dtype=np.float64)
    y = np.log(np.asarray(kappa, dtype=np.float64))
    sig = None if events is None else 1.0 / np.sqrt(np.asarray(events, dtype=np.float64))
    if T0 is None:
        def f(t, a, b, t0):
            return a - b / (KB_EV_PER_K * t * (t - t0) ** 2)
        p, c = curve_fit(f, T, y, p0=[FIT_A, FIT_B_EV_K2, FIT_T0_K], sigma=sig, absolute_sigma=sig is not None,
                         maxfev=20000)
        res = y - f(T, *p)
        names = ["a", "b_eV_K2", "T0_K"]
    else:
        def f(t, a, b):
            return a - b / (KB_EV_PER_K * t * (t - T0) ** 2)
        p, c = curve_fit(f, T, y, p0=[FIT_A, FIT_B_EV_K2], sigma=sig, absolute_sigma=sig is not None, maxfev=20000)
        res = y - f(T, *p)
        names = ["a", "b_eV_K2"]
    err = np.sqrt(np.diag(c))
    out = {k: float(v) for k, v in zip(names, p)}
    out.update({k + "_se": float(v) for k, v in zip(names, err)})
    if T0 is not None:
        out["T0_K"] = float(T0)
        out["T0_fixed"] = True
    out["residuals_ln_kappa"] = [float(r) for r in res]
    return out


def compare_ensembles(a: dict, b: dict) -> dict:
    """Two quench ensembles (outputs of quench.run with the same clusters and schedule), e.g. MIXED against
    FP64: solidified counts, lifetimes, censored rates, final crystalline fractions, and (when both carry
    energy traces) the energy drop from the first to the last 20 ps of each trace."""
    from scipy.stats import fisher_exact, ks_2samp, mannwhitneyu
    out = {}
    ta = np.array([c["t_nuc_ps"] for c in a["per_cluster"] if c["t_nuc_ps"] is not None])
    tb = np.array([c["t_nuc_ps"] for c in b["per_cluster"] if c["t_nuc_ps"] is not None])
    na, nb = len(a["per_cluster"]), len(b["per_cluster"])
    out["solidified"] = [int(ta.size), int(tb.size)]
    out["clusters"] = [na, nb]
    out["fisher_p"] = float(fisher_exact([[ta.size, na - ta.size], [tb.size, nb - tb.size]]).pvalue)
    if ta.size and tb.size:
        out["mean_lifetime_ps"] = [float(ta.mean()), float(tb.mean())]
        out["median_lifetime_ps"] = [float(np.median(ta)), float(np.median(tb))]
        out["ks_p"] = float(ks_2samp(ta, tb).pvalue)
        ka, da, ra = rate_mle(ta, na - ta.size, a["horizon_ps"])
        kb, db, rb = rate_mle(tb, nb - tb.size, b["horizon_ps"])
        r, lo, hi = rate_ratio(da, ra, db, rb)
        out["kappa_mle_per_ps"] = [ka, kb]
        out["rate_ratio"], out["rate_ratio_ci95"] = r, [lo, hi]
    ca = np.array([c["crystalline_end"] for c in a["per_cluster"]])
    cb = np.array([c["crystalline_end"] for c in b["per_cluster"]])
    out["crystalline_end_mean"] = [float(ca.mean()), float(cb.mean())]
    out["crystalline_end_mannwhitney_p"] = float(mannwhitneyu(ca, cb).pvalue)
    if "traces_eV_per_atom" in a and "traces_eV_per_atom" in b:
        def drop(res):
            e = np.asarray(res["traces_eV_per_atom"])
            w = max(1, int(round(20.0 / (res["horizon_ps"] / (e.shape[1] - 1)))))
            return e[:, -w:].mean(1) - e[:, :w].mean(1)
        da_, db_ = drop(a), drop(b)
        out["energy_drop_mean_eV_per_atom"] = [float(da_.mean()), float(db_.mean())]
        out["energy_drop_mannwhitney_p"] = float(mannwhitneyu(da_, db_).pvalue)
    return out


def _censored(res: dict) -> int:
    return sum(c["t_nuc_ps"] is None for c in res["per_cluster"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--table1", type=int, default=None, choices=sorted(TABLE_I), help="temperature (K)")
    ap.add_argument("--compare", action="store_true", help="compare two quench outputs")
    ap.add_argument("--fit", action="store_true",
                    help="fit Eq. rate3 to the censored escape rates of quench outputs at several temperatures")
    ap.add_argument("files", nargs="+", help="quench.py --out JSON files")
    a = ap.parse_args()
    runs = [json.load(open(p)) for p in a.files]
    if a.compare:
        if len(runs) != 2:
            raise SystemExit("--compare takes two files")
        print(json.dumps(compare_ensembles(runs[0], runs[1])))
    elif a.fit:
        by_T = {}
        for r in runs:
            by_T.setdefault(float(r["T_K"]), []).append(r)
        T, kap, ev, rows = [], [], [], []
        for t in sorted(by_T):
            lt = [c["t_nuc_ps"] for r in by_T[t] for c in r["per_cluster"] if c["t_nuc_ps"] is not None]
            nc = sum(_censored(r) for r in by_T[t])
            k, d, risk = rate_mle(lt, nc, max(r["horizon_ps"] for r in by_T[t]))
            T.append(t)
            kap.append(k)
            ev.append(d)
            row = {"T_K": t, "runs": len(lt) + nc, "solidified": d, "kappa_per_ps": k,
                   "paper_fit_kappa_per_ps": float(kappa_fit(t)), "fit_offset_K": temperature_for_kappa(k) - t}
            if int(t) in TABLE_I and float(int(t)) == t:
                row["table1"] = compare_with_table1(int(t), lt, nc, max(r["horizon_ps"] for r in by_T[t]))
            rows.append(row)
        out = {"temperatures": rows}
        if len(T) >= 2:
            out["fit_T0_paper"] = fit_rate3(T, kap, ev, T0=FIT_T0_K)
        if len(T) >= 4:
            out["fit_free"] = fit_rate3(T, kap, ev)
        print(json.dumps(out))
    elif a.table1 is not None:
        t = [c["t_nuc_ps"] for r in runs for c in r["per_cluster"] if c["t_nuc_ps"] is not None]
        nc = sum(_censored(r) for r in runs)
        horizon = max(r["horizon_ps"] for r in runs)
        print(json.dumps(compare_with_table1(a.table1, t, nc, horizon)))
    else:
        raise SystemExit("give --table1 T, --compare or --fit")


if __name__ == "__main__":
    main()
