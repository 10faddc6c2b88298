"""Shared comparison helpers for the GPU parity tests (test code only)."""

import numpy as np

import oracle

# per-query relative tolerance of the FP32 path against the FP64 oracle
RTOL = 1e-4


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    out = np.zeros_like(ref)
    nz = ref != 0
    out[nz] = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
    out[~nz] = np.where(got[~nz] == 0, 0.0, np.inf)
    return out


def check_pndf(D_gpu, oracle_out, rtol=RTOL, hits_gpu=None, hash_gpu=None, label=""):
    """Compare GPU densities (and optionally hit counts / hit-set hashes) with
    the oracle on every query the oracle does not flag as a tie.  Returns a
    summary dict with the counts of compared and excluded queries."""
    Do, fo, ho, hho = oracle_out
    ok = (fo & oracle.F_EXCLUDE) == 0
    r = rel_err(D_gpu[ok], Do[ok])
    worst = int(np.argmax(r)) if r.size else -1
    assert r.size == 0 or r.max() <= rtol, (
        f"{label}: max rel err {r.max():.3e} at query {np.flatnonzero(ok)[worst]} "
        f"(gpu {D_gpu[ok][worst]!r}, oracle {Do[ok][worst]!r}); {int((r > rtol).sum())} over tolerance")
    if hits_gpu is not None:
        bad = np.flatnonzero(hits_gpu[ok] != ho[ok])
        assert bad.size == 0, f"{label}: hit counts differ on {bad.size} queries, e.g. {np.flatnonzero(ok)[bad[:5]]}"
    if hash_gpu is not None:
        bad = np.flatnonzero(hash_gpu[ok].astype(np.uint32) != hho[ok])
        assert bad.size == 0, f"{label}: hit sets differ on {bad.size} queries"
    return {"compared": int(ok.sum()), "excluded": int((~ok).sum()), "max_rel": float(r.max()) if r.size else 0.0,
            "nonzero": int((Do[ok] != 0).sum())}
