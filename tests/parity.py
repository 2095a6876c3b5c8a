"""Comparison of GPU solver outputs with the FP64 oracle.

The rules (tolerances are written here and nowhere else):
  * supports must be identical, in selection order;
  * relative l2 error of the coefficients ||c_gpu - c_ora|| / ||c_ora||
    <= COEF_RTOL (1e-5) for every signal whose support matches;
  * a support that differs from the oracle's is an "ambiguous tie" only when
    the oracle's own top-2 margin at the first differing pick,
    (|c|_(1) - |c|_(2)) / |c|_(1), is below AMBIGUOUS_MARGIN -- i.e. when the
    two atoms' correlations agree to the accuracy float32 arithmetic can
    resolve.  Any other difference is a failure.  Ambiguous signals are
    counted and must stay rare (MAX_AMBIGUOUS_FRAC).
"""
from __future__ import annotations

import numpy as np

COEF_RTOL = 1e-5
AMBIGUOUS_MARGIN = 2e-5
MAX_AMBIGUOUS_FRAC = 0.01


def f32_problem(A, Y):
    """The problem the GPU actually solves: inputs rounded to float32."""
    A32 = np.asfortranarray(A, dtype=np.float32)
    Y32 = np.asfortranarray(Y, dtype=np.float32)
    return A32, Y32, A32.astype(np.float64, order="F"), Y32.astype(np.float64, order="F")


def f32(x):
    return float(np.float32(x))


def compare(gpu, ora, idx=None, coef_rtol=COEF_RTOL, margin=AMBIGUOUS_MARGIN,
            check_status=True, status_equiv=None):
    """gpu: dict of numpy arrays over the full batch; ora: oracle dict over the
    signals `idx` (default: all).  Returns a summary dict; raises
    AssertionError on any non-ambiguous difference."""
    summary, fails = summarize(gpu, ora, idx, coef_rtol, margin, check_status, status_equiv)
    assert not fails, "\n".join(fails[:20]) + f"\n({len(fails)} failures) {summary}"
    assert summary["ambiguous"] <= max(1, int(MAX_AMBIGUOUS_FRAC * summary["signals"])), summary
    return summary


def summarize(gpu, ora, idx=None, coef_rtol=COEF_RTOL, margin=AMBIGUOUS_MARGIN,
              check_status=True, status_equiv=None):
    """The comparison of compare() without raising: (summary, failures)."""
    B = ora["support"].shape[0]
    idx = np.arange(B) if idx is None else np.asarray(idx)
    ambiguous, worst, fails = [], 0.0, []
    for r, b in enumerate(idx):
        sg, so = gpu["support"][b], ora["support"][r]
        if not np.array_equal(sg, so):
            p = int(np.nonzero(sg != so)[0][0])
            t1, t2 = ora["top1"][r, p], ora["top2"][r, p]
            rel = (t1 - t2) / t1 if t1 > 0 else 0.0
            if rel < margin:
                ambiguous.append((int(b), p, float(rel)))
                continue
            fails.append(f"signal {b}: support differs at pick {p} (oracle margin {rel:.3e}) "
                         f"gpu={sg.tolist()} oracle={so.tolist()}")
            continue
        co = ora["coef"][r]
        cg = gpu["coef"][b].astype(np.float64)
        nrm = np.linalg.norm(co)
        err = np.linalg.norm(cg - co) / (nrm if nrm > 0 else 1.0)
        worst = max(worst, err)
        if not err <= coef_rtol:
            fails.append(f"signal {b}: coefficient rel err {err:.3e} > {coef_rtol}")
        if check_status:
            gs, os_ = int(gpu["status"][b]), int(ora["status"][r])
            ok = gs == os_ or (status_equiv is not None and (gs, os_) in status_equiv)
            if not ok:
                fails.append(f"signal {b}: status gpu={gs} oracle={os_}")
            if int(gpu["n_iter"][b]) != int(ora["n_iter"][r]):
                fails.append(f"signal {b}: n_iter gpu={gpu['n_iter'][b]} oracle={ora['n_iter'][r]}")
    summary = dict(signals=len(idx), ambiguous=len(ambiguous), max_coef_rel_err=worst,
                   failures=len(fails), ambiguous_list=ambiguous[:10])
    return summary, fails


def to_numpy(res):
    return dict(support=res.support.cpu().numpy(), coef=res.coef.cpu().numpy(),
                n_iter=res.n_iter.cpu().numpy(), res_norm=res.res_norm.cpu().numpy(),
                status=res.status.cpu().numpy())
