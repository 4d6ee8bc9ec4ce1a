"""Naive azimuthal DFT (Sec. 2.2).

Forward: rho^m = (1/N) sum_{k=0}^{N-1} rho_k exp(-2 pi i m k / N), m = 0..N/2,
the inverse of the synthesis in Eq. fourier_decomposition (whose index range
1..N is read as 0..N-1).  Inverse: the synthesis over all N modes with the
upper half rebuilt from Hermitian symmetry (Eq. Hermitian_symmetry):

    Phi_k = Re Phi^0 + 2 Re sum_{m=1}^{N/2-1} Phi^m exp(2 pi i m k / N)
            + Re Phi^{N/2} (-1)^k.

Both are O(N^2) per row, written as products with the explicit matrix.
"""
import numpy as np


def forward(rho):
    """rho (..., N) real -> (..., N/2+1) complex."""
    N = rho.shape[-1]
    m = np.arange(N // 2 + 1)[:, None]
    k = np.arange(N)[None, :]
    E = np.exp(-2j * np.pi * ((m * k) % N) / N) / N
    return rho @ E.T


def inverse(phi_hat, N):
    """(..., N/2+1) complex -> (..., N) real."""
    M = N // 2 + 1
    assert phi_hat.shape[-1] == M
    m = np.arange(M)[:, None]
    k = np.arange(N)[None, :]
    w = np.full((M, 1), 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    E = w * np.exp(2j * np.pi * ((m * k) % N) / N)
    return (phi_hat @ E).real
