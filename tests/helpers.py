"""Test helpers: error metrics and small conversions (no method arithmetic).

Error metrics per result (acceleration-like vectors a_i against a reference):
  rms_rel = sqrt(sum_i |a_i - ref_i|^2 / sum_i |ref_i|^2)
  max_rel = max_i |a_i - ref_i| / (|ref_i| + 0.01 * rms(|ref|))
The 1% floor keeps particles where |a| vanishes by symmetry (halo centres)
from dominating the maximum; it makes the maximum looser than a plain
max_i |a_i - ref_i| / |ref_i| for the smallest accelerations, so the tests
print the plain figure (max_plain) beside it.
"""
import numpy as np
import pytest

# tolerance stated for accelerations against the FP64 oracle
RMS_TOL = 1e-6
MAX_TOL = 1e-4


def err(a, ref):
    a = np.asarray(a, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    d = np.linalg.norm(a - ref, axis=1)
    nr = np.linalg.norm(ref, axis=1)
    rms_ref = np.sqrt(np.mean(nr ** 2))
    rms = np.sqrt(np.sum(d ** 2) / max(np.sum(nr ** 2), 1e-300))
    mx = float(np.max(d / (nr + 0.01 * rms_ref))) if len(d) else 0.0
    return float(rms), mx


def max_plain(a, ref):
    """max_i |a_i - ref_i| / |ref_i| without the floor (rows with ref_i = 0
    are left out): reported beside the floored figure."""
    a = np.asarray(a, np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    d = np.linalg.norm(a - ref, axis=1)
    nr = np.linalg.norm(ref, axis=1)
    ok = nr > 0
    return float(np.max(d[ok] / nr[ok])) if ok.any() else 0.0


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1807_08116_gb300 import native
    native.lib()
    return torch


def pos_h_of(r, h):
    ph = np.empty((len(r), 4), np.float32)
    ph[:, :3] = r
    ph[:, 3] = h
    return ph


def pos_m_of(r, m):
    pm = np.empty((len(r), 4), np.float32)
    pm[:, :3] = r
    pm[:, 3] = m
    return pm
