"""Helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def l1_rel(got, want) -> float:
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    den = np.abs(want).sum()
    return float(np.abs(got - want).sum() / (den if den > 0 else 1.0))


def to_dev(g):
    return g.rowptr.cuda(), g.colidx.cuda()
