"""The seeded inputs against independent constructions of what they stand for
(CPU only).  The MRI problem of the paper: its coupling (Eq. MRIJMatrix1) and
Zeeman term (Eq. MRIzeeman, read as A^T y) built here from dense operators on an
8 x 8 image, against the Gram data of the augmented real system that
mri_full_instance returns."""
import math

import numpy as np

import cs_inputs


def test_mri_full_gram_is_the_papers_coupling():
    n, gamma = 8, 0.01
    inst = cs_inputs.mri_full_instance(n, 0.2, 0.3, gamma, 0.01, seed=5)
    N = n * n
    M = int(round(0.3 * N))
    A, y = inst.A, inst.y
    assert A.shape == (2 * M + 2 * N, N)
    # dense operators: orthonormal 1-D DFT and Haar, 2-D by Kronecker products over
    # the row-major image, zero-padded second differences
    u = np.arange(n)
    F1 = np.exp(-2j * math.pi * np.outer(u, u) / n) / math.sqrt(n)
    F2 = np.kron(F1, F1)
    H1 = cs_inputs.haar_1d_matrix(n)
    Psi = np.kron(H1, H1)
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = -2.0
        if i > 0:
            D[i, i - 1] = 1.0
        if i + 1 < n:
            D[i, i + 1] = 1.0
    Dv, Dh = np.kron(D, np.eye(n)), np.kron(np.eye(n), D)
    # the sampled frequencies are the rows whose DFT reproduces the complex rows of A
    Ac = A[:M] + 1j * A[M:2 * M]
    SF = F2 @ Psi.T
    rows = [int(np.argmin(np.abs(SF - a[None, :]).max(axis=1))) for a in Ac]
    np.testing.assert_allclose(SF[rows], Ac, rtol=0, atol=1e-13)
    assert rows[0] == 0 and len(set(rows)) == M  # DC kept, no frequency twice
    S = np.zeros((M, N))
    S[np.arange(M), rows] = 1.0
    J = Psi @ F2.conj().T @ S.T @ S @ F2 @ Psi.T + gamma * Psi @ Dv.T @ Dv @ Psi.T + gamma * Psi @ Dh.T @ Dh @ Psi.T
    np.testing.assert_allclose(A.T @ A, J.real, rtol=0, atol=1e-12)
    # J is Hermitian: its imaginary part is antisymmetric and drops out of x^T J x
    # for the real coefficient vector, so the real part is the whole coupling
    np.testing.assert_allclose(J.imag, -J.imag.T, rtol=0, atol=1e-12)
    yc = S @ F2 @ Psi.T @ inst.x0
    np.testing.assert_allclose(A.T @ y, (Psi @ F2.conj().T @ S.T @ yc).real, rtol=0, atol=1e-12)
    # the image is sparse in the Haar domain as asked
    assert inst.xi.sum() == int(round(0.2 * N)) and np.all((inst.x0 != 0) == (inst.xi == 1))
