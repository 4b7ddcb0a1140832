"""Oracle: discrete trigonometric / Fourier transforms of nodal fields, written as
plain O(n^2) trigonometric sums in float64.

Test infrastructure only (see oracle/__init__.py).

Paper passages followed:
  * Section 3.2.2, Table 2 -- symmetry pair on the two faces of an axis -> transform
    type of a nodal field: SS -> DCT1, SA -> DCT3, AA -> DST1, AS -> DST3, periodic -> DFT.
  * Section 3.2.2, Eq. 7 and Table 3 -- real-space selection S_R of the nodes a
    transform acts on (DCT1 [0:n], DCT3 [0:n-1], DST1 [1:n-1], DST3 [1:n]) and the
    frequencies of the 4n-extended DFT they correspond to.  Table 3's parenthesised
    index lists are swapped between the DST1 and DST3 rows; the "2x[...]" formulas are
    the consistent ones and are used here: DST1 keeps the even frequencies 2k
    (k=1..n-1), DST3 the odd ones 2k+1 (k=0..n-1).  In units of the n-voxel axis the
    wave numbers are q_k = pi*k/n (DCT1, DST1) and q_k = pi*(2k+1)/(2n) (DCT3, DST3),
    and q_k = 2*pi*k/n for the periodic DFT.
  * The factor alpha of Table 3 only rescales the spectrum; the Green step is
    forward -> diagonal -> inverse, so the pair used here is normalised to be an
    exact inverse pair and alpha does not enter.

Boundary-condition codes: 0 periodic, 1 Dirichlet (A extension of the displacement
component), 2 Neumann (S extension), Table 1.
"""
import numpy as np

BC_P, BC_D, BC_N = 0, 1, 2

DCT1, DCT3, DST1, DST3, DFT = "DCT1", "DCT3", "DST1", "DST3", "DFT"


def transform_type(bc0, bc1):
    """Table 1 + Table 2: (face-0 BC, face-1 BC) of one component on one axis -> type."""
    if bc0 == BC_P or bc1 == BC_P:
        if not (bc0 == BC_P and bc1 == BC_P):
            raise ValueError("periodic must be set on both faces of an axis")
        return DFT
    table = {(BC_N, BC_N): DCT1, (BC_N, BC_D): DCT3, (BC_D, BC_D): DST1, (BC_D, BC_N): DST3}
    return table[(bc0, bc1)]


def selection(ttype, n):
    """Table 3: real-space node indices S_R and wave numbers q_k for an axis of n voxels.

    Returns (sel_nodes, k_index, q): k_index are the spectral indices kept, q the
    corresponding wave numbers (radians per voxel).
    """
    if ttype == DCT1:
        j = np.arange(0, n + 1)
        k = np.arange(0, n + 1)
        q = np.pi * k / n
    elif ttype == DCT3:
        j = np.arange(0, n)
        k = np.arange(0, n)
        q = np.pi * (2 * k + 1) / (2 * n)
    elif ttype == DST1:
        j = np.arange(1, n)
        k = np.arange(1, n)
        q = np.pi * k / n
    elif ttype == DST3:
        j = np.arange(1, n + 1)
        k = np.arange(0, n)
        q = np.pi * (2 * k + 1) / (2 * n)
    elif ttype == DFT:
        j = np.arange(0, n)
        k = np.arange(0, n)
        q = 2.0 * np.pi * k / n
    else:
        raise ValueError(ttype)
    return j, k, q


def node_count(ttype, n):
    """Nodes stored along an axis of n voxels: n for a periodic axis, else n+1."""
    return n if ttype == DFT else n + 1


def forward_matrix(ttype, n):
    """Forward transform as an explicit (N_sel x n_nodes) matrix of trigonometric sums.

    Row k, column j (a node index along the axis):
      DCT1  X_k = sum_{j=0..n}   w_j x_j cos(pi j k / n),           w_0 = w_n = 1/2
      DCT3  X_k = sum_{j=0..n-1} w_j x_j cos(pi j (2k+1) / (2n)),   w_0 = 1/2
      DST1  X_k = sum_{j=1..n-1}     x_j sin(pi j k / n)
      DST3  X_k = sum_{j=1..n}   w_j x_j sin(pi j (2k+1) / (2n)),   w_n = 1/2
      DFT   X_k = sum_{j=0..n-1}     x_j exp(-2 pi i j k / n)
    The end-node weights 1/2 are those of the symmetric extension (a node lying on a
    mirror plane is counted once in a period of length 2n).
    """
    sel, _, q = selection(ttype, n)
    nn = node_count(ttype, n)
    if ttype == DFT:
        F = np.zeros((len(q), nn), dtype=np.complex128)
        for a, qk in enumerate(q):
            for j in sel:
                F[a, j] = np.exp(-1j * qk * j)
        return F
    F = np.zeros((len(q), nn))
    for a, qk in enumerate(q):
        for j in sel:
            w = 1.0
            if ttype == DCT1 and (j == 0 or j == n):
                w = 0.5
            if ttype == DCT3 and j == 0:
                w = 0.5
            if ttype == DST3 and j == n:
                w = 0.5
            trig = np.cos(qk * j) if ttype in (DCT1, DCT3) else np.sin(qk * j)
            F[a, j] = w * trig
    return F


def inverse_matrix(ttype, n):
    """Inverse transform as an explicit (n_nodes x N_sel) matrix (synthesis).

      DCT1  x_j = (2/n) sum_{k=0..n}   w_k X_k cos(pi j k / n),         w_0 = w_n = 1/2
      DCT3  x_j = (2/n) sum_{k=0..n-1}     X_k cos(pi j (2k+1) / (2n))
      DST1  x_j = (2/n) sum_{k=1..n-1}     X_k sin(pi j k / n)
      DST3  x_j = (2/n) sum_{k=0..n-1}     X_k sin(pi j (2k+1) / (2n))
      DFT   x_j = (1/n) sum_{k=0..n-1}     X_k exp(+2 pi i j k / n)
    Rows of nodes outside S_R (antisymmetry nodes) are zero.
    """
    sel, kidx, q = selection(ttype, n)
    nn = node_count(ttype, n)
    if ttype == DFT:
        B = np.zeros((nn, len(q)), dtype=np.complex128)
        for j in sel:
            for a, qk in enumerate(q):
                B[j, a] = np.exp(1j * qk * j) / n
        return B
    B = np.zeros((nn, len(q)))
    for j in sel:
        for a, qk in enumerate(q):
            w = 1.0
            if ttype == DCT1 and (kidx[a] == 0 or kidx[a] == n):
                w = 0.5
            trig = np.cos(qk * j) if ttype in (DCT1, DCT3) else np.sin(qk * j)
            B[j, a] = (2.0 / n) * w * trig
    return B


def apply_along(M, x, axis):
    """Apply matrix M (out x in) along one axis of array x (plain contraction)."""
    y = np.tensordot(M, x, axes=([1], [axis]))
    return np.moveaxis(y, 0, axis)


def forward_3d(x, types, nvox):
    """Forward transform of one nodal component; x has shape (nnz, nny, nnx).

    types = (type_x, type_y, type_z); axis 0 of x is z, axis 2 is x.
    """
    y = x.astype(np.complex128) if DFT in types else x.astype(np.float64)
    for d, arr_axis in ((0, 2), (1, 1), (2, 0)):
        y = apply_along(forward_matrix(types[d], nvox[d]), y, arr_axis)
    return y


def inverse_3d(X, types, nvox):
    """Inverse of forward_3d, back to the nodal grid (shape (nnz, nny, nnx))."""
    y = X
    for d, arr_axis in ((2, 0), (1, 1), (0, 2)):
        y = apply_along(inverse_matrix(types[d], nvox[d]), y, arr_axis)
    if np.iscomplexobj(y):
        y = y.real
    return np.ascontiguousarray(y)


def wave_numbers(types, nvox):
    """Per-axis wave-number vectors (qx, qy, qz) of the kept spectral points."""
    return tuple(selection(types[d], nvox[d])[2] for d in range(3))
