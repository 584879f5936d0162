"""Pins of the oracle's AMR refinement rule (oracle/amr.py, Sec. 2.5): counts
that follow from the rule by hand, translation covariance, and a cell-by-cell
loop on a small grid."""
import numpy as np

from oracle import amr


def test_one_node_of_the_other_colour_refines_a_4x4x4_block():
    """One node of colour 1 is a corner of 8 cells (2x2x2), all interfacial;
    their 3x3x3 neighbourhoods cover a 4x4x4 block."""
    cb = np.zeros((12, 11, 10), np.uint8)
    cb[5, 6, 7] = 1
    f = amr.interfacial_cells(cb)
    assert f.sum() == 8 and f[4:6, 5:7, 6:8].all()
    m = amr.refine_mask(cb)
    assert m.sum() == 64 and m[3:7, 4:8, 5:9].all()


def test_plane_interface_refines_three_layers_per_crossing():
    """Colours x >= 6 on a periodic 16-cell axis change between nodes 5|6 and
    15|0: two layers of interfacial cells (i = 5, i = 15), six refined layers."""
    nz, ny, nx = 8, 9, 16
    cb = np.zeros((nz, ny, nx), np.uint8)
    cb[:, :, 6:] = 1
    f = amr.interfacial_cells(cb)
    assert f.sum() == 2 * ny * nz and f[:, :, 5].all() and f[:, :, 15].all()
    m = amr.refine_mask(cb)
    assert m.sum() == 6 * ny * nz
    assert m[:, :, [4, 5, 6, 14, 15, 0]].all()


def test_uniform_fields_refine_nothing():
    for v in (0, 1):
        cb = np.full((8, 8, 8), v, np.uint8)
        assert not amr.refine_mask(cb).any()
        assert len(amr.brick_tiles(cb)) == 0


def test_face_bits_do_not_count():
    """Only bit 0 (the node colour) decides; face colour bits are ignored."""
    rng = np.random.default_rng(4)
    cb = rng.integers(0, 2, (9, 10, 11)).astype(np.uint8)
    noisy = cb | (rng.integers(0, 8, cb.shape).astype(np.uint8) << 1)
    assert np.array_equal(amr.refine_mask(cb), amr.refine_mask(noisy))


def test_translation_covariance_and_a_cell_by_cell_loop():
    rng = np.random.default_rng(9)
    n3 = (7, 9, 8)
    cb = (rng.random(n3) < 0.15).astype(np.uint8)
    m = amr.refine_mask(cb)
    # the mask moves with the colours
    sh = (2, -3, 5)
    assert np.array_equal(amr.refine_mask(np.roll(cb, sh, axis=(0, 1, 2))), np.roll(m, sh, axis=(0, 1, 2)))
    # the rule written cell by cell with explicit modular indices
    nz, ny, nx = n3
    inter = np.zeros(n3, bool)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                cs = {int(cb[(k + a) % nz, (j + b) % ny, (i + c) % nx]) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
                inter[k, j, i] = len(cs) == 2
    ref = np.zeros(n3, bool)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ref[k, j, i] = any(inter[(k + a) % nz, (j + b) % ny, (i + c) % nx]
                                   for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    assert np.array_equal(m, ref)


def test_brick_tiles_of_a_ragged_grid():
    """A single node of colour 1 near the upper corner of a 20 x 12 x 10 grid
    (tiles 3 x 2 x 2, the last ones partial): the refined 4x4x4 block spans
    two tiles along each axis."""
    cb = np.zeros((10, 12, 20), np.uint8)  # nz, ny, nx
    cb[8, 7, 17] = 1  # interfacial cells x 16..17, y 6..7, z 7..8; refined x 15..18, y 5..8, z 6..9
    ids = amr.brick_tiles(cb)
    tx, ty = 3, 2
    expect = sorted({(bz * ty + by) * tx + bx for bz in (0, 1) for by in (0, 1) for bx in (1, 2)})
    assert list(ids) == expect
