"""Element-wise comparison helpers for the GPU-vs-oracle parity tests.

Besides the whole-array relative L2 error (the tolerance the method is specified at), every field
is checked for its largest local error, and on thin regions where a localised mistake would hide
under the whole-grid norm: the CPML slabs, the PEC walls, the two x columns either side of the
TF/SF plane, the cells next to the design-box faces (inside and outside), the gap with its
neighbours, and the point source's neighbourhood.
"""
import numpy as np

TOL = {32: 1e-4, 64: 1e-10}
REGION_FACTOR = 10.0      # a region's error against max(its norm, 1% of the whole array's norm)


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0)


def _grow(box, n, by):
    """Box (i0,i1,j0,j1,k0,k1) grown by `by` cells on every face, clipped to the grid n = (nx,ny,nz)."""
    return [max(box[0] - by, 0), min(box[1] + by, n[0]), max(box[2] - by, 0), min(box[3] + by, n[1]),
            max(box[4] - by, 0), min(box[5] + by, n[2])]


def _box_mask(shape_zyx, box):
    m = np.zeros(shape_zyx, dtype=bool)
    if box[1] > box[0] and box[3] > box[2] and box[5] > box[4]:
        m[box[4]:box[5], box[2]:box[3], box[0]:box[1]] = True
    return m


def field_regions(desc):
    """(name, mask) pairs over the (nz, ny, nx) grid of a description."""
    nx, ny, nz = desc["nx"], desc["ny"], desc["nz"]
    n = (nx, ny, nz)
    shape = (nz, ny, nx)
    cp = desc["cpml"]
    out = []
    cpml = np.zeros(shape, dtype=bool)
    for a, (lo, hi) in enumerate(((cp[0], cp[1]), (cp[2], cp[3]), (cp[4], cp[5]))):
        idx = [slice(None)] * 3
        ax = 2 - a
        if lo:
            idx[ax] = slice(0, lo)
            cpml[tuple(idx)] = True
        if hi:
            idx[ax] = slice(n[a] - hi, n[a])
            cpml[tuple(idx)] = True
    out.append(("cpml", cpml))
    walls = np.zeros(shape, dtype=bool)
    walls[0], walls[-1], walls[:, 0], walls[:, -1], walls[:, :, 0], walls[:, :, -1] = (True,) * 6
    out.append(("pec walls", walls))
    if desc["src_kind"] == 1:
        i0 = desc["src_pos"][0]
        m = np.zeros(shape, dtype=bool)
        m[:, :, max(i0 - 1, 0):i0 + 1] = True
        out.append(("tf/sf plane", m))
    else:
        s = desc["src_pos"]
        out.append(("source", _box_mask(shape, _grow([s[0], s[0] + 1, s[1], s[1] + 1, s[2], s[2] + 1], n, 2))))
    db = list(desc["design_box"])
    if db[1] > db[0]:
        rim = _box_mask(shape, _grow(db, n, 1)) & ~_box_mask(shape, [db[0] + 1, db[1] - 1, db[2] + 1, db[3] - 1,
                                                                     db[4] + 1, db[5] - 1])
        out.append(("design-box rim", rim))
    gb = list(desc["gap_box"])
    if gb[1] > gb[0]:
        out.append(("gap", _box_mask(shape, _grow(gb, n, 1))))
    return out


def box_rim(shape_zyx):
    """Cells on the faces of an array (the design box's outermost voxel layer)."""
    m = np.zeros(shape_zyx, dtype=bool)
    m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (True,) * 6
    return m


def check_array(name, g, o, tol, regions=()):
    """Whole-array relative L2 <= tol, largest local error <= tol x the largest value, and on each
    region (a mask over the trailing axes) the error norm <= REGION_FACTOR tol x max(the region's
    norm, 1% of the whole array's norm)."""
    g = np.asarray(g)
    o = np.asarray(o)
    e = rel(g, o)
    assert e <= tol, f"{name}: relative L2 {e:.3e}"
    d = np.abs(g - o)
    omax = np.abs(o).max() if o.size else 0.0
    assert d.max(initial=0.0) <= tol * omax, f"{name}: max abs error {d.max():.3e} vs max |value| {omax:.3e}"
    onorm = np.linalg.norm(o.ravel())
    for rname, mask in regions:
        if not mask.any():
            continue
        dr = np.linalg.norm(d[..., mask])
        orr = np.linalg.norm(o[..., mask])
        bound = REGION_FACTOR * tol * max(orr, 1e-2 * onorm)
        assert dr <= bound, f"{name} on {rname}: error {dr:.3e} vs bound {bound:.3e} (region norm {orr:.3e})"
