"""The batch builder: replica meshes concatenated with index offsets.  Each
replica's slice of the union, shifted back by its offsets, is its own mesh;
no index of one replica reaches into another; boundary codes are kept."""
import numpy as np

from paper_1906_08125_gb300 import inputs


def test_batch_slices_are_the_members(plate_small, tip_small):
    members = [tip_small, plate_small, tip_small]
    b = inputs.batch_meshes(members, [1e10, 9e9, 1.1e10])
    m = b.mesh
    assert b.n_rep == 3 and m.n_tets == sum(x.n_tets for x in members)
    assert list(b.node_off) == [0, tip_small.n_nodes, tip_small.n_nodes + plate_small.n_nodes,
                                m.n_nodes]
    for r, x in enumerate(members):
        n0, n1 = b.node_off[r], b.node_off[r + 1]
        t0, t1 = b.tet_off[r], b.tet_off[r + 1]
        f0, f1 = b.face_off[r], b.face_off[r + 1]
        assert np.array_equal(m.xyz[n0:n1], x.xyz)
        assert np.array_equal(m.tet[t0:t1] - n0, x.tet)
        nb = m.nbr[t0:t1]
        assert np.array_equal(np.where(nb >= 0, nb - t0, nb), x.nbr)
        assert np.all((nb < 0) | ((nb >= t0) & (nb < t1)))
        pn = m.periodic_nbr[t0:t1]
        assert np.array_equal(np.where(pn >= 0, pn - t0, pn), x.periodic_nbr)
        assert np.array_equal(m.face_nodes[f0:f1] - n0, x.face_nodes)
        assert np.array_equal(m.face_tet[f0:f1] - t0, x.face_tet)
        assert np.array_equal(m.dirichlet[n0:n1], x.dirichlet)
        assert np.array_equal(m.work_function[f0:f1], x.work_function)
    assert np.allclose(m.box_hi, np.max([x.box_hi for x in members], axis=0))


def test_ensemble_recipe_is_seeded_and_in_range():
    scales = {3: (4.0,), 6: (4.0,)}
    a = inputs.ensemble(n_rep=6, seed=5, scales=scales)
    b = inputs.ensemble(n_rep=6, seed=5, scales=scales)
    assert np.array_equal(a.E0, b.E0) and [x.name for x in a.members] == [x.name for x in b.members]
    assert np.all((a.E0 >= 8e9) & (a.E0 <= 12e9))
    assert {x.name for x in a.members} <= {"tip_r3_s4.0", "tip_r6_s4.0"}
    assert all(5e4 <= x.n_tets <= 1.1e6 for x in a.members)
