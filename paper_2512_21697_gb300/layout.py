"""Index maps between the library's vector order and the paper's order (pure permutations).

Library order: channel (library enumeration) -> radial slot r -> DKB type t: index 2 r + t.
Paper order:   channel (kappa = -1, 1, -2, 2, ..., then 2mu ascending) -> type t -> slot r:
               index t (N + 1) + r.
"""
import numpy as np


def paper_channels(kappa_max, two_mu_max=0):
    out = []
    for ak in range(1, kappa_max + 1):
        for kappa in (-ak, ak):
            for tm in range(-(2 * ak - 1), 2 * ak, 2):
                if two_mu_max <= 0 or abs(tm) <= two_mu_max:
                    out.append((kappa, tm))
    return out


def lib_to_paper_perm(lib_kappa, lib_two_mu, kappa_max, two_mu_max, N):
    """perm such that v_paper = v_lib[perm] (whole vectors)."""
    nb = 2 * (N + 1)
    where = {(int(k), int(m)): i for i, (k, m) in enumerate(zip(lib_kappa, lib_two_mu))}
    inner = np.empty(nb, np.int64)
    for t in range(2):
        for r in range(N + 1):
            inner[t * (N + 1) + r] = 2 * r + t
    perm = []
    for ch in paper_channels(kappa_max, two_mu_max):
        perm.append(where[ch] * nb + inner)
    return np.concatenate(perm)


def block_perm(N):
    """p such that M_paper = M_lib[np.ix_(p, p)] for one channel block."""
    nb = 2 * (N + 1)
    p = np.empty(nb, np.int64)
    for t in range(2):
        for r in range(N + 1):
            p[t * (N + 1) + r] = 2 * r + t
    return p
