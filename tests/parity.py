"""Parity checks of the CUDA path against the oracle, shared by the GPU tests.

Tolerances (FP32 kernels against the oracle's FP64 smooth values and FP64
sums; discrete decisions identical on both sides):

  pixels     |I_gpu - I_or| <= 1e-4 |I_or| + 1e-7
  gradients  |g_gpu - g_or| <= 1e-4 |g_or| + 1e-6 A

A is the oracle's per-entry magnitude of the terms summed into the entry,
carried through every operation by the chain rule with absolute values (and
|f_u| + |f_l| in place of |f_u - f_l| for an edge sample's radiance
difference).  An FP32 evaluation of a contribution that is small by
cancellation errs by about u A, not u |g|.

Every gradient check also reports, per call:
  - the fraction of entries within the pure relative bound 1e-4 |g_or|;
  - the largest error over the bound used (1.0 = at the bound);
  - the same two figures with the plain scale C = sum_k |c_k| over the
    samples' whole contributions in place of A (when the caller passes C),
    which shows how much of the bound the chain-rule scale A supplies.
Records go to stdout and, if the environment variable DRT_PARITY_REPORT
names a file, are appended to it as JSON lines.
"""
from __future__ import annotations

import json
import os

import numpy as np

REL = 1e-4
ABS_SCALE = 1e-6


def _record(rec: dict) -> None:
    line = json.dumps(rec)
    print("parity " + line)
    path = os.environ.get("DRT_PARITY_REPORT")
    if path:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "a") as f:
            f.write(line + "\n")


def grad_stats(got, want, absum, contrib=None) -> dict:
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    bound = REL * np.abs(want) + ABS_SCALE * absum + 1e-12
    out = {"entries": int(err.size), "nonzero": int(np.count_nonzero(want)),
           "pass_frac": float(np.mean(err <= bound)) if err.size else 1.0,
           "pure_rel_frac": float(np.mean(err <= REL * np.abs(want))) if err.size else 1.0,
           "max_norm_err": float(np.max(err / bound)) if err.size else 0.0}
    if contrib is not None:
        bc = REL * np.abs(want) + ABS_SCALE * np.asarray(contrib, np.float64) + 1e-12
        out["sum_abs_c_pass_frac"] = float(np.mean(err <= bc)) if err.size else 1.0
        out["sum_abs_c_max_norm_err"] = float(np.max(err / bc)) if err.size else 0.0
    return out


def assert_grads(got, want, absum, label="", contrib=None):
    """Gradient parity within 1e-4 |g| + 1e-6 A, with the report above."""
    got = np.asarray(got, np.float64)
    st = grad_stats(got, want, absum, contrib)
    st["label"] = label
    _record(st)
    err = np.abs(got - want)
    bound = REL * np.abs(want) + ABS_SCALE * absum + 1e-12
    bad = err > bound
    i = int(np.argmax(err / bound)) if err.size else 0
    assert not bad.any(), "%s: %d/%d entries off; worst entry %d got %g want %g (A=%g)" % (
        label, bad.sum(), bad.size, i, got[i], want[i], absum[i])


def assert_pixels(got, want, label=""):
    """Pixel parity within 1e-4 |I| + 1e-7."""
    got = np.asarray(got, np.float64)
    err = np.abs(got - want)
    bound = REL * np.abs(want) + 1e-7
    bad = err > bound
    if label:
        _record({"label": label, "pixels": int(err.size), "max_norm_err": float(np.max(err / bound)),
                 "pure_rel_frac": float(np.mean(err <= REL * np.abs(want)))})
    assert not bad.any(), "%d/%d pixels off; worst err %g at %s (want %g)" % (
        bad.sum(), bad.size, err.max(), np.unravel_index(err.argmax(), err.shape), want.flat[err.argmax()])
