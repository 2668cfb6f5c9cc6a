"""Error measures of GPU results against the oracle (test infrastructure; the
readings are stated once here).

* b: per-SNP normwise relative error ||b - b_ref||_2 / ||b_ref||_2, max over
  SNPs, plus the SE-scaled error max_j |b_j - b_ref_j| / se_ref_j (a
  component-wise relative error is ill-posed for null SNPs whose effect is ~0);
* se: component-wise relative error (se is never 0);
* status: must agree exactly; SNPs flagged singular by both sides carry NaN.
"""
import numpy as np


def compare(b, se, st, b_ref, se_ref, st_ref):
    b, se, b_ref, se_ref = (np.asarray(a, dtype=np.float64) for a in (b, se, b_ref, se_ref))
    st, st_ref = np.asarray(st), np.asarray(st_ref)
    assert st.shape == st_ref.shape
    mism = np.nonzero(st != st_ref)[0]
    assert mism.size == 0, f"status differs at SNPs {mism[:10]} (got {st[mism[:10]]}, want {st_ref[mism[:10]]})"
    ok = st_ref == 0
    if (~ok).any():
        assert np.isnan(b[:, ~ok]).all() and np.isnan(se[:, ~ok]).all()
    if not ok.any():
        return dict(b_norm=0.0, b_se_scaled=0.0, se_rel=0.0, b_comp_median=0.0)
    d = b[:, ok] - b_ref[:, ok]
    b_norm = (np.linalg.norm(d, axis=0) / np.linalg.norm(b_ref[:, ok], axis=0)).max()
    b_se = (np.abs(d) / se_ref[:, ok]).max()
    se_rel = (np.abs(se[:, ok] - se_ref[:, ok]) / se_ref[:, ok]).max()
    big = np.abs(b_ref[:, ok]) >= se_ref[:, ok]
    comp = np.abs(d)[big] / np.abs(b_ref[:, ok])[big]
    return dict(b_norm=float(b_norm), b_se_scaled=float(b_se), se_rel=float(se_rel),
                b_comp_max=float(comp.max()) if comp.size else 0.0,
                b_comp_median=float(np.median(comp)) if comp.size else 0.0)
