"""Closed forms of the per-antenna blocks of J^H J and J^H r, FP64.

Test infrastructure only (see the package header).

All sums run over the directed rows [pq s] with p != q (Sect. 2.1 eq. JJ:di and Sect. 2.3):
every stored baseline (p, q) also stands for its conjugate row (q, p) with
d_qp = conj(d_pq), m_qp = conj(m_pq) (scalar) or D_qp = D_pq^H, M_qp = M_pq^H (2x2, Sect. 4).
``np.add.at`` (and, for the N_d x N_d blocks, one matrix product per antenna) sums rows into antennas.
"""
from __future__ import annotations

import numpy as np


def directed_rows(vis, model, a1, a2, kind):
    """Rows of both orientations: (i, j, d_ij, m_ij) flattened over samples.

    vis/model arrive as [N_s, N_bl(, 2, 2)] (dd: model [Nd, N_s, N_bl]).
    """
    a1 = np.asarray(a1, np.int64); a2 = np.asarray(a2, np.int64)
    vis = np.asarray(vis, np.complex128); model = np.asarray(model, np.complex128)
    ns = vis.shape[0]
    i = np.concatenate([np.tile(a1, ns), np.tile(a2, ns)])
    j = np.concatenate([np.tile(a2, ns), np.tile(a1, ns)])
    if kind == 'jones':
        d = vis.reshape(-1, 2, 2); m = model.reshape(-1, 2, 2)
        dH = np.conj(np.swapaxes(d, -1, -2)); mH = np.conj(np.swapaxes(m, -1, -2))
        return i, j, np.concatenate([d, dH]), np.concatenate([m, mH])
    if kind == 'dd':
        d = vis.reshape(-1); m = model.reshape(model.shape[0], -1)
        return i, j, np.concatenate([d, np.conj(d)]), np.concatenate([m, np.conj(m)], axis=1)
    d = vis.reshape(-1); m = model.reshape(-1)
    return i, j, np.concatenate([d, np.conj(d)]), np.concatenate([m, np.conj(m)])


def scalar_blocks(g, vis, model, a1, a2, n_ant):
    """Scalar DI with intervals (eqs. JHJ:DI:tf, JHR:DI:tf) and the data form (eq. ghat).

    Returns dict with
      A    [n]      diag of the top-left block: sum_{q!=i,s} |y_iqs|^2, y_iqs = m_iqs conj(g_q)
      B    [n, n]   top-right block: B_ij = sum_s conj(y_ijs) conj(y_jis) (i != j)
      c    [n]      top half of J^H r:  sum conj(y_iqs) r_iqs
      cd   [n]      top half of J^H d:  sum conj(y_iqs) d_iqs
    """
    g = np.asarray(g, np.complex128)
    i, j, d, m = directed_rows(vis, model, a1, a2, 'scalar')
    y = m * np.conj(g[j])
    r = d - g[i] * y
    A = np.zeros(n_ant); c = np.zeros(n_ant, np.complex128); cd = np.zeros(n_ant, np.complex128)
    np.add.at(A, i, np.abs(y) ** 2)
    np.add.at(c, i, np.conj(y) * r)
    np.add.at(cd, i, np.conj(y) * d)
    # off-diagonal block: pair each directed row ij s with its mirror ji s
    half = y.shape[0] // 2
    y_ij, y_ji = y[:half], y[half:]
    B = np.zeros((n_ant, n_ant), np.complex128)
    np.add.at(B, (i[:half], j[:half]), np.conj(y_ij) * np.conj(y_ji))
    np.add.at(B, (j[:half], i[:half]), np.conj(y_ij) * np.conj(y_ji))
    return dict(A=A, B=B, c=c, cd=cd)


def jones_blocks(G, vis, model, a1, a2, n_ant):
    """2x2 DI: the diagonal operator blocks of eq. JHJ:pol and the top half of J^H R.

    Y_iq = M_iq G_q^H, R_iq = D_iq - G_i Y_iq.
      H    [n, 2, 2]  sum_q Y_iq Y_iq^H        (top-left block is R_H, i.e. H^T kron I)
      C    [n, 2, 2]  sum_q R_iq Y_iq^H        (J^H R; product order read from R_A X = X A)
      CD   [n, 2, 2]  sum_q D_iq Y_iq^H        (J^H D, the data form of eq. ghat:matrix)
    """
    G = np.asarray(G, np.complex128)
    i, j, D, M = directed_rows(vis, model, a1, a2, 'jones')
    Y = M @ np.conj(np.swapaxes(G[j], -1, -2))
    YH = np.conj(np.swapaxes(Y, -1, -2))
    R = D - G[i] @ Y
    H = np.zeros((n_ant, 2, 2), np.complex128)
    C = np.zeros((n_ant, 2, 2), np.complex128)
    CD = np.zeros((n_ant, 2, 2), np.complex128)
    np.add.at(H, i, Y @ YH)
    np.add.at(C, i, R @ YH)
    np.add.at(CD, i, D @ YH)
    return dict(H=H, C=C, CD=CD)


def dd_blocks(g, vis, model, a1, a2, n_ant):
    """Scalar DD (eqs. JHJ:DD:unpol, JHR:DD:unpol): the N_d x N_d antenna blocks of CohJones.

    y^(d)_iqs = m^(d)_iqs conj(g_q^(d)).
      A   [n, Nd, Nd]  A_i[c, d] = sum conj(y^(c)) y^(d)
      c   [n, Nd]      sum conj(y^(d)) r
      cd  [n, Nd]      sum conj(y^(d)) d
    """
    g = np.asarray(g, np.complex128)
    i, j, d, m = directed_rows(vis, model, a1, a2, 'dd')
    y = m * np.conj(g[j]).T                       # [Nd, rows]
    v = np.sum(g[i].T * y, axis=0)
    r = d - v
    nd = g.shape[1]
    A = np.zeros((n_ant, nd, nd), np.complex128)
    c = np.zeros((n_ant, nd), np.complex128)
    cd = np.zeros((n_ant, nd), np.complex128)
    for p in range(n_ant):                        # rows whose first antenna is p: Y_p^H Y_p etc.
        sel = i == p
        Yp = y[:, sel].T                          # [rows_p, Nd]
        A[p] = np.conj(Yp).T @ Yp
        c[p] = np.conj(Yp).T @ r[sel]
        cd[p] = np.conj(Yp).T @ d[sel]
    return dict(A=A, c=c, cd=cd)
