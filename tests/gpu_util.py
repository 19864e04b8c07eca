"""Tolerances for the GPU parity tests (no method arithmetic here).

Every tolerance is a rounding bound built from the oracle's per-row terms
(E, G, Gd) = oracle Problem.bound(X) (see orc_eval_bound):
  E  first-order rounding magnitude of the plain FP64 body arithmetic of two
     implementations, in units of u = 2^-53;
  G  sum_i |dg/dz_i| * sum_j |M_ij d_j|  (sensitivity to errors in z that
     scale with the products of the rotation);
  Gd sum_i |dg/dz_i| * ||d||_2           (sensitivity to an error in M),
and from dM = ||M_library - M_oracle||_2, the measured difference of the two
sides' rotations of the instance (both are the Q of the same seeded matrix:
Householder in the oracle, Gram-Schmidt twice in the library; they differ by
round-off amplified by the matrix's condition number).
"""
import numpy as np

U64 = 2.0 ** -53


def eps_z(prec, D):
    """Error in z per unit of sum_j |M_ij d_j| for a rotation precision on
    the GPU, the oracle's own FP64 dot products included: operand rounding
    of d and M (TF32: 2^-11 each, round to nearest; split BF16: 3 * 2^-16
    for hi*hi + hi*lo + lo*hi with lo*lo dropped; FP32: 2^-24 each plus the
    product), d rounded to FP32 (2^-24), and an FP32 accumulation of D
    products allowed one FP32 ulp (2^-23) per add."""
    acc = D * 2.0 ** -23 + 2 * D * U64
    if prec == "TF32":
        return 2 * 2.0 ** -11 + 2.0 ** -24 + acc
    if prec == "BF16X3":
        return 3 * 2.0 ** -16 + 2.0 ** -24 + acc
    if prec == "FP32":
        return 3 * 2.0 ** -24 + acc
    raise ValueError(prec)


def rot_diff(p, q):
    """max over components of ||M_library - M_oracle||_2 (cached on p)."""
    dM = getattr(p, "_rot_diff", None)
    if dM is None:
        dM = 0.0
        for c in range(q.ncomp):
            d = p.export(c)["M"] - q.rotation(c)
            dM = max(dM, float(np.linalg.norm(d, 2) if q.D <= 2000 else np.linalg.norm(d)))
        p._rot_diff = dM
    return dM


def bound(p, q, X):
    """(E, G, Gd, dM, D) for the rows of X on library problem p and oracle
    problem q of the same instance."""
    E, G, Gd = q.bound(X)
    return E, G, Gd, rot_diff(p, q), q.D


def sel(bnd, idx):
    """The bound terms of a subset of rows."""
    E, G, Gd, dM, D = bnd
    return E[idx], G[idx], Gd[idx], dM, D


def tol64(want, bnd, rel=1e-12):
    """FP64 GPU path against the oracle: the larger of rel * |f| and the
    rounding bound u * (E + 2 D G) + dM * Gd -- both sides' body arithmetic
    (E), both sides' D-term dot products for z (D u sum_j |M_ij d_j| each),
    and the two sides' rotations differing by dM."""
    E, G, Gd, dM, D = bnd
    return np.maximum(rel * np.abs(want), U64 * (E + 2.0 * D * G) + dM * Gd)


def tol_mixed(prec, want, bnd):
    """Mixed path (rotation in TF32 / split BF16 / FP32, FP32 bodies) against
    the oracle: eps_z * G for the rotation, 2^-23 * E for the FP32 body
    arithmetic (each IEEE operation allowed 4 FP32 ulps, each transcendental
    12), plus the FP64 tolerance."""
    E, G, Gd, dM, D = bnd
    return eps_z(prec, D) * G + 2.0 ** -23 * E + tol64(want, bnd)


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
