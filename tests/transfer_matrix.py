"""Exact partition functions of small +-J lattices by transfer matrices (test helper).

An independent route to Z(beta) = sum_E g(E) exp(-beta E): rows (2D) or planes (3D) of
spins are the transfer states, and Z is the trace of the product of the row-to-row (or
plane-to-plane) Boltzmann matrices around the periodic direction.  Used to pin the oracle's
brute-force density of states.  Couplings use the layout J[i*dim + d], site i = x + L y
(+ L^2 z), bond (i, d) joins i and i + e_d.
"""
import itertools

import numpy as np


def _layer_states(n):
    # rows of +-1 spins, state index bit k <-> spin k (bit set = -1)
    s = np.array(list(itertools.product([1, -1], repeat=n)), dtype=np.float64)[:, ::-1]
    return s


def partition_function(dim, L, J, beta):
    J = np.asarray(J, dtype=np.float64)
    if dim == 2:
        n = L                       # spins per row (x), rows along y
        layer_sites = lambda layer: [x + L * layer for x in range(L)]
        in_layer = [(x, (x + 1) % L, 0) for x in range(L)]   # (a, b, direction)
        nd = 2
        inter_dir = 1
    else:
        n = L * L                   # spins per plane (x, y), planes along z
        layer_sites = lambda layer: [x + L * y + L * L * layer for y in range(L) for x in range(L)]
        in_layer = []
        for y in range(L):
            for x in range(L):
                a = x + L * y
                in_layer.append((a, (x + 1) % L + L * y, 0))
                in_layer.append((a, x + L * ((y + 1) % L), 1))
        nd = 3
        inter_dir = 2
    S = _layer_states(n)
    T = np.eye(S.shape[0])
    for layer in range(L):
        sites = layer_sites(layer)
        e_in = np.zeros(S.shape[0])
        for a, b, d in in_layer:
            e_in += J[sites[a] * nd + d] * S[:, a] * S[:, b]
        jz = np.array([J[sites[a] * nd + inter_dir] for a in range(n)])
        e_between = (S * jz) @ S.T            # sum_a J_a s_a s'_a
        A = np.exp(beta * (e_in[:, None] + e_between))
        T = T @ A
    return float(np.trace(T))


def z_from_dos(g, nb, beta):
    u = np.arange(len(g), dtype=np.float64)
    E = 2 * u - nb
    return float(np.sum(np.asarray(g, dtype=np.float64) * np.exp(-beta * E)))
