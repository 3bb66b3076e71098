"""Cyclic-by-row Jacobi eigensolver for small dense symmetric matrices.

A brute-force reference used to pin the oracle on tiny inputs: it shares no
code with numpy.linalg and is checked on its own against closed-form spectra.
Each rotation zeroes A[i, j] with the classical choice of angle
(tan 2 theta = 2 a_ij / (a_jj - a_ii), smaller root for t = tan theta).
"""
import math

import numpy as np


def jacobi_eigh(A, sweeps=60, tol=1e-15):
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = math.sqrt(max(0.0, float(np.sum(A * A) - np.sum(np.diag(A) ** 2))))
        if off <= tol * math.sqrt(float(np.sum(A * A))):
            break
        for i in range(n - 1):
            for j in range(i + 1, n):
                aij = A[i, j]
                if aij == 0.0:
                    continue
                d = A[j, j] - A[i, i]
                if abs(d) > 1e150 * abs(aij):
                    # theta = d / (2 a_ij) (or theta^2) would overflow; then
                    # t = 1/(|theta| + sqrt(theta^2 + 1)) = 1/(2 theta) = a_ij / d
                    t = aij / d
                else:
                    theta = d / (2.0 * aij)
                    t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                # A <- J^T A J on rows/columns i, j
                ai = A[:, i].copy()
                aj = A[:, j].copy()
                A[:, i] = c * ai - s * aj
                A[:, j] = s * ai + c * aj
                ai = A[i, :].copy()
                aj = A[j, :].copy()
                A[i, :] = c * ai - s * aj
                A[j, :] = s * ai + c * aj
                vi = V[:, i].copy()
                vj = V[:, j].copy()
                V[:, i] = c * vi - s * vj
                V[:, j] = s * vi + c * vj
    w = np.diag(A).copy()
    order = np.argsort(w)[::-1]
    return w[order], V[:, order]
