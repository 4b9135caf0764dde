"""Error measures shared by the GPU parity tests (oracle values vs the CUDA path)."""

import numpy as np


def normal_angle(a, b):
    """Angle between row vectors by atan2(|a x b|, a . b) (accurate at small angles)."""
    a = np.asarray(a, dtype=np.float64)[:, :3]
    b = np.asarray(b, dtype=np.float64)[:, :3]
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.einsum("ij,ij->i", a, b))


def decision_agreement(f_ref, hit_gpu, eps, margin):
    """Fraction of points with |f_ref| > margin whose collision decision matches."""
    sel = np.abs(f_ref) > margin
    return float(np.mean((f_ref[sel] < eps) == hit_gpu[sel])) if sel.any() else 1.0


def report(f_ref, n_ref, f_gpu, n_gpu):
    ds = np.abs(np.asarray(f_gpu, np.float64) - f_ref)
    ang = normal_angle(n_ref, n_gpu)
    return {"sdf_max": float(ds.max()), "sdf_p99": float(np.percentile(ds, 99)),
            "angle_max": float(ang.max()), "angle_p99": float(np.percentile(ang, 99))}
