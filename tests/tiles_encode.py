"""Test-side encoder of the Section 3.2 tile format (SCSR + COO), written from
the format's description: per tile, rows with >= 2 entries as a header word
(0x8000 | row) followed by column words, then single-entry rows as
(row, column) pairs; values in the same order."""
import numpy as np


def encode(A, tile):
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    cols = A.col_idx.astype(np.int64)
    vals = None if A.values is None else A.values
    tr, tc = rows // tile, cols // tile
    order = np.lexsort((np.arange(A.nnz), tc, tr))          # tile-major, storage order inside
    tiles = []
    key = tr[order] * (A.n_cols // tile + 2) + tc[order]
    bounds = np.flatnonzero(np.diff(key)) + 1
    for seg in np.split(order, bounds):
        if len(seg) == 0:
            continue
        lr, lc = rows[seg] % tile, cols[seg] % tile
        scsr, coo, v_scsr, v_coo = [], [], [], []
        for r in np.unique(lr):
            m = lr == r
            if m.sum() >= 2:
                scsr.append(0x8000 | int(r))
                scsr.extend(int(c) for c in lc[m])
                if vals is not None:
                    v_scsr.extend(vals[seg[m]])
            else:
                coo.append((int(r), int(lc[m][0])))
                if vals is not None:
                    v_coo.extend(vals[seg[m]])
        v = None if vals is None else np.array(v_scsr + v_coo, dtype=np.float32)
        tiles.append((int(tr[seg[0]]), int(tc[seg[0]]), np.array(scsr, np.uint16),
                      np.array(coo, np.uint16).reshape(-1, 2), v))
    return tiles


def storage_bytes(tiles, value_bytes):
    return sum(2 * len(s) + 4 * len(c) + value_bytes * (len(s) - int(np.sum(np.asarray(s) >= 0x8000)) + len(c))
               for _, _, s, c, _ in tiles)
