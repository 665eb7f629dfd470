"""Seeded synthetic inputs shared by the tests, the bench and the oracle calls.

Holds no arithmetic of the estimator itself: only the gauge field, which is
input data.  The paper's gauge ensemble (a 32^3 x 64 clover configuration,
Sec. 4.2) is not available; it is replaced by links

    U_mu(x) = exp(i eps H),   H = (G + G^dagger)/2 - tr(.)/3 I,

with G a 3 x 3 complex matrix whose real and imaginary parts are standard
normal draws from numpy's default_rng(seed), eps = 0.3.  U is in SU(3)
(unitary, det 1).  Exponentiated in FP64 through the Hermitian eigensystem.
Layout: complex128 [N, 4, 3, 3] (site in storage order x_0 fastest,
direction mu, row, column).  Imports numpy only.
"""
import numpy as np


def volume(dims):
    n = 1
    for D in dims:
        n *= int(D)
    return n


def gauge_links(dims, seed, eps=0.3):
    N = volume(dims)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, 4, 3, 3)) + 1j * rng.standard_normal((N, 4, 3, 3))
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, V = np.linalg.eigh(H)
    U = np.einsum('...ab,...b,...cb->...ac', V, np.exp(1j * eps * w), np.conj(V))
    return np.ascontiguousarray(U, dtype=np.complex128)


def unit_links(dims):
    """Free field U = 1."""
    N = volume(dims)
    return np.ascontiguousarray(np.broadcast_to(np.eye(3, dtype=np.complex128), (N, 4, 3, 3)))


def random_su3(n, seed):
    """n Haar-ish random SU(3) matrices (QR of complex Gaussians, det fixed)."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]
