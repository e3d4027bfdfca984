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
    if kind == 'dd_jones':
        d = vis.reshape(-1, 2, 2); m = model.reshape(model.shape[0], -1, 2, 2)
        dH = np.conj(np.swapaxes(d, -1, -2)); mH = np.conj(np.swapaxes(m, -1, -2))
        return i, j, np.concatenate([d, dH]), np.concatenate([m, mH], axis=1)
    d = vis.reshape(-1); m = model.reshape(-1)
    return i, j, np.concatenate([d, np.conj(d)]), np.concatenate([m, np.conj(m)])


def directed_weights(weights, n_dir_rows):
    """Per-row weights w_pqs (Sect. 2.4, a diagonal W in eq. LSmin:w) for the directed rows of
    ``directed_rows``: a stored row and its conjugate row share one weight.  None: unit weights."""
    if weights is None:
        return np.ones(n_dir_rows)
    w = np.asarray(weights, np.float64).reshape(-1)
    return np.concatenate([w, w])


def scalar_blocks(g, vis, model, a1, a2, n_ant, weights=None):
    """Scalar DI with intervals (eqs. JHJ:DI:tf, JHR:DI:tf) and the data form (eq. ghat); with
    per-row weights, eqs. JHJ:DI:tfw and JHR:DI:tfw (each sum over rows carries w_iqs).

    Returns dict with
      A    [n]      diag of the top-left block: sum_{q!=i,s} |y_iqs|^2, y_iqs = m_iqs conj(g_q)
      B    [n, n]   top-right block: B_ij = sum_s conj(y_ijs) conj(y_jis) (i != j)
      c    [n]      top half of J^H r:  sum conj(y_iqs) r_iqs
      cd   [n]      top half of J^H d:  sum conj(y_iqs) d_iqs
    """
    g = np.asarray(g, np.complex128)
    i, j, d, m = directed_rows(vis, model, a1, a2, 'scalar')
    w = directed_weights(weights, i.shape[0])
    y = m * np.conj(g[j])
    r = d - g[i] * y
    A = np.zeros(n_ant); c = np.zeros(n_ant, np.complex128); cd = np.zeros(n_ant, np.complex128)
    np.add.at(A, i, w * np.abs(y) ** 2)
    np.add.at(c, i, w * np.conj(y) * r)
    np.add.at(cd, i, w * np.conj(y) * d)
    # off-diagonal block: pair each directed row ij s with its mirror ji s
    half = y.shape[0] // 2
    y_ij, y_ji = y[:half], y[half:]
    B = np.zeros((n_ant, n_ant), np.complex128)
    np.add.at(B, (i[:half], j[:half]), w[:half] * np.conj(y_ij) * np.conj(y_ji))
    np.add.at(B, (j[:half], i[:half]), w[:half] * np.conj(y_ij) * np.conj(y_ji))
    return dict(A=A, B=B, c=c, cd=cd)


def jones_blocks(G, vis, model, a1, a2, n_ant, weights=None):
    """2x2 DI: the diagonal operator blocks of eq. JHJ:pol and the top half of J^H R.

    Y_iq = M_iq G_q^H, R_iq = D_iq - G_i Y_iq.
      H    [n, 2, 2]  sum_q Y_iq Y_iq^H        (top-left block is R_H, i.e. H^T kron I)
      C    [n, 2, 2]  sum_q R_iq Y_iq^H        (J^H R; product order read from R_A X = X A)
      CD   [n, 2, 2]  sum_q D_iq Y_iq^H        (J^H D, the data form of eq. ghat:matrix)
    """
    G = np.asarray(G, np.complex128)
    i, j, D, M = directed_rows(vis, model, a1, a2, 'jones')
    w = directed_weights(weights, i.shape[0])[:, None, None]
    Y = M @ np.conj(np.swapaxes(G[j], -1, -2))
    YH = np.conj(np.swapaxes(Y, -1, -2))
    R = D - G[i] @ Y
    H = np.zeros((n_ant, 2, 2), np.complex128)
    C = np.zeros((n_ant, 2, 2), np.complex128)
    CD = np.zeros((n_ant, 2, 2), np.complex128)
    np.add.at(H, i, w * (Y @ YH))
    np.add.at(C, i, w * (R @ YH))
    np.add.at(CD, i, w * (D @ YH))
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


def dd_jones_blocks(G, vis, model, a1, a2, n_ant):
    """2x2 DD (Sect. 4.4, eqs. JHJ:DD:pol and JHR:DD:pol, product order as for the DI case):
    Y^(d)_iqs = M^(d)_iqs G_q^(d)H, R_iqs = D_iqs - sum_d G_i^(d) Y^(d)_iqs.

      H   [n, 2Nd, 2Nd]  block (c, d) = sum_{q,s} Y^(c) Y^(d)H: the operator form of the top-left
                         antenna block is X -> X H (R_H of App. B), so the antenna's normal
                         equations read [G^(1) .. G^(Nd)] H = [C^(1) .. C^(Nd)]
      C   [n, 2, 2Nd]    [.. sum R Y^(d)H ..]  (J^H R, direction d in columns 2d, 2d+1)
      CD  [n, 2, 2Nd]    [.. sum D Y^(d)H ..]  (J^H D)
    """
    G = np.asarray(G, np.complex128)
    nd = G.shape[1]
    i, j, D, M = directed_rows(vis, model, a1, a2, 'dd_jones')
    Y = M @ np.conj(np.swapaxes(G[j], -1, -2)).transpose(1, 0, 2, 3)          # [Nd, rows, 2, 2]
    V = np.sum(G[i].transpose(1, 0, 2, 3) @ Y, axis=0)
    R = D - V
    H = np.zeros((n_ant, 2 * nd, 2 * nd), np.complex128)
    C = np.zeros((n_ant, 2, 2 * nd), np.complex128)
    CD = np.zeros((n_ant, 2, 2 * nd), np.complex128)
    for p in range(n_ant):                    # rows whose first antenna is p, summed as one product
        sel = i == p
        A = Y[:, sel].transpose(0, 2, 1, 3).reshape(2 * nd, -1)   # [Y^(1); ..; Y^(Nd)] side by side over rows
        H[p] = A @ A.conj().T
        C[p] = R[sel].transpose(1, 0, 2).reshape(2, -1) @ A.conj().T
        CD[p] = D[sel].transpose(1, 0, 2).reshape(2, -1) @ A.conj().T
    return dict(H=H, C=C, CD=CD)


# ----------------------------------------------------------------------------- full J^H J (exact GN / LM)

def op_R4(A):
    """W R_A of App. B eq. RA4x4: the 4x4 matrix of X -> X A acting on vec X (stacked columns)."""
    A = np.asarray(A, np.complex128)
    W = np.zeros(A.shape[:-2] + (4, 4), np.complex128)
    W[..., 0, 0] = A[..., 0, 0]; W[..., 0, 2] = A[..., 1, 0]
    W[..., 1, 1] = A[..., 0, 0]; W[..., 1, 3] = A[..., 1, 0]
    W[..., 2, 0] = A[..., 0, 1]; W[..., 2, 2] = A[..., 1, 1]
    W[..., 3, 1] = A[..., 0, 1]; W[..., 3, 3] = A[..., 1, 1]
    return W


def op_L4(A):
    """W L_A of App. B eq. LA4x4: the 4x4 matrix of X -> A X acting on vec X."""
    A = np.asarray(A, np.complex128)
    W = np.zeros(A.shape[:-2] + (4, 4), np.complex128)
    W[..., 0:2, 0:2] = A
    W[..., 2:4, 2:4] = A
    return W


def _vec(X):
    return np.stack([X[..., 0, 0], X[..., 1, 0], X[..., 0, 1], X[..., 1, 1]], axis=-1)


def jones_jhj_full(G, vis, model, a1, a2, n_ant, weights=None):
    """The whole J^H J and J^H R of the 2x2 DI problem, off-diagonal antenna blocks included.

    Sect. 4.2 eq. JHJ:pol with the 4x4 operator forms of App. B, over the directed rows [pq],
    p != q (eq. JJ:pol) and the samples of the interval (Sect. 2.3).  The augmented parameter
    vector is eq. GGvec, [vec G_1 .. vec G_n, vec G_1^H .. vec G_n^H]; with Y_ij = M_ij G_j^H:
      top-left  (i, i)   sum_{q != i} R_{Y_iq Y_iq^H}        (zero for i != j)
      top-right (i, j)   sum R_{Y_ij^H} L_{Y_ji^H}, i != j   (zero for i == j)
      bottom-left (i, j) sum L_{Y_ij} R_{Y_ji}, i != j
      bottom-right (i,i) sum_{q != i} L_{Y_iq Y_iq^H}
    J^H R: top vec(sum_q R_iq Y_iq^H) (the product order read from R_A X = X A), bottom
    vec((sum_q R_iq Y_iq^H)^H).  With per-row weights every sum carries w_iqs (J^H W J, J^H W R).
    Returns (JHJ [8n, 8n], JHR [8n]) as complex128.
    """
    G = np.asarray(G, np.complex128)
    i, j, D, M = directed_rows(vis, model, a1, a2, 'jones')
    w = directed_weights(weights, i.shape[0])[:, None, None]
    half = i.shape[0] // 2
    mirror = np.concatenate([np.arange(half, 2 * half), np.arange(0, half)])   # row (j, i) of row (i, j)
    Y = M @ np.conj(np.swapaxes(G[j], -1, -2))
    YH = np.conj(np.swapaxes(Y, -1, -2))
    R = D - G[i] @ Y
    n = int(n_ant)
    TL = np.zeros((n, 4, 4), np.complex128)
    BR = np.zeros((n, 4, 4), np.complex128)
    TR = np.zeros((n, n, 4, 4), np.complex128)
    BL = np.zeros((n, n, 4, 4), np.complex128)
    np.add.at(TL, i, w * op_R4(Y @ YH))
    np.add.at(BR, i, w * op_L4(Y @ YH))
    np.add.at(TR, (i, j), w * (op_R4(YH) @ op_L4(YH[mirror])))
    np.add.at(BL, (i, j), w * (op_L4(Y) @ op_R4(Y[mirror])))
    C = np.zeros((n, 2, 2), np.complex128)
    np.add.at(C, i, w * (R @ YH))
    H = np.zeros((8 * n, 8 * n), np.complex128)
    for p in range(n):
        H[4 * p:4 * p + 4, 4 * p:4 * p + 4] = TL[p]
        H[4 * n + 4 * p:4 * n + 4 * p + 4, 4 * n + 4 * p:4 * n + 4 * p + 4] = BR[p]
        for q in range(n):
            H[4 * p:4 * p + 4, 4 * n + 4 * q:4 * n + 4 * q + 4] = TR[p, q]
            H[4 * n + 4 * p:4 * n + 4 * p + 4, 4 * q:4 * q + 4] = BL[p, q]
    b = np.concatenate([_vec(C).reshape(-1), _vec(np.conj(np.swapaxes(C, -1, -2))).reshape(-1)])
    return H, b


def scalar_jhj_full(g, vis, model, a1, a2, n_ant, weights=None):
    """The whole J^H J and J^H r of the scalar DI problem (eq. JHJ:DI:ABCD / eq. JHJ:DI with the
    sample sums of eq. JHJ:DI:tf, and eq. JHR:DI), ordering [g; conj g].  Returns (JHJ [2n, 2n],
    JHR [2n])."""
    blk = scalar_blocks(g, vis, model, a1, a2, n_ant, weights)
    A = np.diag(blk['A']).astype(np.complex128)
    B = blk['B']
    H = np.block([[A, B], [np.conj(B), A]])
    return H, np.concatenate([blk['c'], np.conj(blk['c'])])
