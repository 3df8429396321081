"""Euclidean Dirac matrices (Sec. 2, Eq. 2).

The paper prints only (1 - gamma_1) (Eq. 2). The representation used here is
the Dirac one: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] for k = 1, 2, 3 and
gamma_4 = diag(1, 1, -1, -1); it reproduces the printed (1 - gamma_1) exactly.
Index 0..3 of the returned stack is the direction x, y, z, t.
"""

import torch

CDT = torch.complex128


def pauli() -> torch.Tensor:
    s = torch.zeros((3, 2, 2), dtype=CDT)
    s[0] = torch.tensor([[0, 1], [1, 0]], dtype=CDT)
    s[1] = torch.tensor([[0, -1j], [1j, 0]], dtype=CDT)
    s[2] = torch.tensor([[1, 0], [0, -1]], dtype=CDT)
    return s


def gammas() -> torch.Tensor:
    """gamma_mu for mu = x, y, z, t; shape [4, 4, 4]."""
    g = torch.zeros((4, 4, 4), dtype=CDT)
    sig = pauli()
    for k in range(3):
        g[k, 0:2, 2:4] = -1j * sig[k]
        g[k, 2:4, 0:2] = 1j * sig[k]
    g[3] = torch.diag(torch.tensor([1, 1, -1, -1], dtype=CDT))
    return g


def gamma5() -> torch.Tensor:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def projectors():
    """(1 - gamma_mu) and (1 + gamma_mu), each [4, 4, 4]: the spin factors of Eq. 1."""
    g = gammas()
    eye = torch.eye(4, dtype=CDT)
    return eye - g, eye + g
