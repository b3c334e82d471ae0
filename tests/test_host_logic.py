"""CPU checks of the library's host logic through its host-only test hooks
(no GPU needed): the mesh builder's tables (Sec. 4: leaves, refined base
cells, hanging faces) against the oracle's independently built tables, bit
for bit, and the face lists' structure; the Runge-Kutta stage programs
derived from the SSP tableaux (Appendix D) against the Butcher form of the
step with the printed tableaux (tests/golden/), unlimited and with a limiter
pass on every stage state."""
import numpy as np
import pytest

import golden_values
from oracle import pyoracle as O
from paper_1506_06140_gb300 import workloads as wl

PER, TRN = 0, 1


@pytest.fixture(scope="module")
def dg():
    from paper_1506_06140_gb300 import build, dg as mod
    build.build()
    return mod


MESHES = {
    "u2_periodic": wl.mesh_uniform(2, [7, 5], [0.0, 0.0], [7 / 5.0, 1.0]),
    "u2_transmissive": wl.mesh_uniform(2, [6, 3], [0.0, 0.0], [2.0, 1.0], bc=[TRN, PER]),
    "amr2": dict(wl.mesh_uniform(2, [16, 12], [0.0, 0.0], [4 / 3.0, 1.0]),
                 refine_boxes=[[4, 3, 9, 7], [13, 0, 15, 1]]),
    "amr2_edge_transmissive": dict(wl.mesh_uniform(2, [8, 8], [0.0, 0.0], [1.0, 1.0], bc=[TRN, TRN]),
                                   refine_boxes=[[0, 0, 2, 3], [6, 6, 7, 7]]),
    "u3": wl.mesh_uniform(3, [4, 3, 5], [0.0, 0.0, 0.0], [4 / 3.0, 1.0, 5 / 3.0]),
    "amr3": dict(wl.mesh_uniform(3, [6, 6, 6], [0.0] * 3, [1.0] * 3, bc=[PER, TRN, PER]),
                 refine_boxes=[[1, 1, 1, 3, 3, 2], [5, 0, 0, 5, 0, 5]]),
    "sedov_like": wl.mesh_two_level_3d(8, 2, 5),
    # degenerate: one cell (its own neighbour on every side), one row, one open column
    "one_cell_2d": wl.mesh_uniform(2, [1, 1], [0.0, 0.0], [1.0, 1.0]),
    "one_cell_3d": wl.mesh_uniform(3, [1, 1, 1], [0.0] * 3, [1.0] * 3),
    "one_row_open": wl.mesh_uniform(2, [6, 1], [0.0, 0.0], [6.0, 1.0], bc=[TRN, TRN]),
    "one_refined_cell": dict(wl.mesh_uniform(2, [1, 1], [0.0, 0.0], [1.0, 1.0]), refine_boxes=[[0, 0, 0, 0]]),
}


def oracle_for(m):
    return O.Oracle(m["dim"], m["n"], m["lo"], m["hi"], 1, 1.4, bc=m["bc"],
                    refine_boxes=m["refine_boxes"])


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_tables_match_the_oracle(dg, name):
    m = MESHES[name]
    t = dg.mesh_tables(m)
    o = oracle_for(m)
    assert t["nbr"].shape[1] == o.n_cells
    np.testing.assert_array_equal(t["nbr"], o.neighbor_table())
    np.testing.assert_array_equal(t["levels"], o.levels())
    assert t["n_nodes"] == o.n_nodes


@pytest.mark.parametrize("name", list(MESHES))
def test_face_lists(dg, name):
    """Every face joins the cells the neighbour table says it joins; every
    cell side maps to its face(s); every face is some side's face; the
    conforming and boundary faces come first, grouped by axis in cell order,
    then the hanging sub-faces in quadrant order per coarse side."""
    m = MESHES[name]
    t = dg.mesh_tables(m)
    d = m["dim"]
    nbr, lev, faces, sface = t["nbr"], t["levels"], t["faces"], t["sface"]
    nc, nf = nbr.shape[1], faces.shape[1]
    nsub = 2 ** (d - 1)
    fm, fp, info = faces
    axis, vm, vp = info & 3, (info >> 2) & 7, (info >> 5) & 7
    assert np.all(axis < d) and np.all((vm == 0) | (vp == 0))
    seen = np.zeros(nf, bool)
    for c in range(nc):
        for a in range(d):
            for s in range(2):
                side = 2 * a + s
                f = sface[side, c]
                assert 0 <= f < nf
                nb = nbr[side, c]
                mine, other = (fm, fp) if s == 1 else (fp, fm)
                if nb <= -2:
                    # coarse side of a hanging face: nsub consecutive sub-faces
                    for q in range(nsub):
                        g = f + q
                        assert mine[g] == c and axis[g] == a
                        assert (vm[g] if s == 1 else vp[g]) == 1 + q
                        fine = other[g]
                        assert lev[fine] == lev[c] + 1
                        assert sface[2 * a + (1 - s), fine] == g
                        seen[g] = True
                else:
                    assert mine[f] == c and axis[f] == a
                    var_mine, var_other = (vp[f], vm[f]) if s == 0 else (vm[f], vp[f])
                    assert var_mine == 0
                    assert other[f] == nb  # -1 beyond a transmissive boundary
                    if var_other > 0:
                        # c is the fine side of a hanging face
                        assert lev[c] == 1 and lev[nb] == 0
                    elif nb >= 0:
                        assert lev[nb] == lev[c]
                    else:
                        assert m["bc"][a] == TRN
                    seen[f] = True
    assert seen.all()
    # ordering: whole faces first (by axis, owner cell non-decreasing), then sub-faces
    whole = (vm == 0) & (vp == 0)
    n_whole = int(whole.sum())
    assert whole[:n_whole].all() and not whole[n_whole:].any()
    owner = np.where(fm[:n_whole] >= 0, fm[:n_whole], fp[:n_whole])
    ax = axis[:n_whole]
    assert np.all(np.diff(ax) >= 0)
    for a in range(d):
        assert np.all(np.diff(owner[ax == a]) >= 0)
    # hanging: the number of sub-faces is nsub per coarse side
    assert nf - n_whole == nsub * int((nbr <= -2).sum())


def test_batch_tables_concatenate_the_problems(dg):
    """An ensemble's tables are its problems' own tables in problem order,
    cell and face indices shifted by the offsets (node and boundary codes
    unchanged), with each cell's problem index."""
    meshes = [wl.mesh_uniform(2, [n, n], [-5.0, -5.0], [5.0, 5.0]) for n in (5, 3, 8)]
    meshes.append(wl.mesh_uniform(2, [4, 2], [0.0, 0.0], [2.0, 1.0], bc=[TRN, PER]))
    b = dg.mesh_tables(meshes)
    c0 = f0 = 0
    for p, m in enumerate(meshes):
        t = dg.mesh_tables(m)
        nc, nf = t["nbr"].shape[1], t["faces"].shape[1]
        sl = slice(c0, c0 + nc)
        np.testing.assert_array_equal(b["nbr"][:, sl], np.where(t["nbr"] >= 0, t["nbr"] + c0, t["nbr"]))
        np.testing.assert_array_equal(b["levels"][sl], t["levels"])
        np.testing.assert_array_equal(b["sface"][:, sl], t["sface"] + f0)
        np.testing.assert_array_equal(b["prob"][sl], p)
        fb = b["faces"][:, f0:f0 + nf]
        np.testing.assert_array_equal(fb[:2], np.where(t["faces"][:2] >= 0, t["faces"][:2] + c0, -1))
        np.testing.assert_array_equal(fb[2], t["faces"][2])
        c0 += nc
        f0 += nf
    assert c0 == b["nbr"].shape[1] and f0 == b["faces"].shape[1]
    # ensembles are uniform meshes of one dimension
    with pytest.raises(dg.DGError) as ei:
        dg.mesh_tables([meshes[0], MESHES["amr2"]])
    assert ei.value.code == dg.DG_ERR_UNSUPPORTED
    with pytest.raises(dg.DGError) as ei:
        dg.mesh_tables([meshes[0], MESHES["u3"]])
    assert ei.value.code == dg.DG_ERR_ARG


def test_mesh_tables_reject_bad_meshes(dg):
    for bad in (dict(wl.mesh_uniform(2, [4, 4], [0.0, 0.0], [1.0, 2.0])),  # non-cubical cells
                dict(wl.mesh_uniform(2, [0, 4], [0.0, 0.0], [1.0, 1.0]))):
        with pytest.raises(dg.DGError) as ei:
            dg.mesh_tables(bad)
        assert ei.value.code == dg.DG_ERR_ARG


def run_program(ops, n_regs, f, lim, w, dt):
    """One step of a stage program: registers R[0] = w, R[1..n_regs]."""
    R = [w.copy()] + [np.full_like(w, np.nan) for _ in range(n_regs)]
    for op in ops:
        U = R[op["in_reg"]].copy()
        K = f(U)
        for o, dst in enumerate(op["outs"]):
            val = op["ck"][o] * dt * K
            for r, src in enumerate(op["ins"]):
                val = val + op["C"][o][r] * (U if src == op["in_reg"] else R[src])
            R[dst] = val
        if op["lim_src"] >= 0:
            R[op["lim_dst"]] = lim(R[op["lim_src"]])
    return R[0]


def butcher_step(order, f, lim, w, dt):
    """The Butcher form with the tableau as printed (Appendix D; forward
    Euler for order 1): stage states U_1 = w and U_i = lim(w + dt sum_j a_ij
    k_j), k_i = f(U_i); new state lim(w + dt sum_j b_j k_j)."""
    A, b = (np.zeros((1, 1)), np.ones(1)) if order == 1 else golden_values.rk_tableaux()[order][:2]
    s = len(b)
    k = []
    for i in range(s):
        U = w if i == 0 else lim(w + dt * sum(A[i, j] * k[j] for j in range(i)))
        k.append(f(U))
    return lim(w + dt * sum(b[j] * k[j] for j in range(s)))


@pytest.mark.parametrize("limited", [0, 1])
@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_stage_program_is_the_butcher_step(dg, order, limited):
    rng = np.random.default_rng(70 + order + 10 * limited)
    n = 6
    M = rng.normal(size=(n, n))

    def f(y):
        return M @ y + 0.3 * np.sin(y) - 0.1 * y ** 3

    ident = lambda y: y
    lim = (lambda y: y - 0.05 * np.tanh(3.0 * y)) if limited else ident
    ops, n_regs = dg.stage_program(order, limited)
    assert len(ops) == (1 if order == 1 else len(golden_values.rk_tableaux()[order][1]))
    for _ in range(3):
        w = rng.normal(size=n)
        dt = 0.05
        got = run_program(ops, n_regs, f, lim, w, dt)
        ref = butcher_step(order, f, lim, w, dt)
        # unlimited RK4: the printed tableau's near-identities taken as exact
        # (coefficients matched to 1e-9 relative); otherwise exact to rounding
        tol = 1e-9 if (order == 4 and not limited) else 1e-13
        assert np.max(np.abs(got - ref)) < tol * (1.0 + np.max(np.abs(ref))), (order, limited)
    # with the identity limiter the limited program takes the same step
    if limited:
        w = rng.normal(size=n)
        ref = butcher_step(order, f, ident, w, 0.05)
        got = run_program(ops, n_regs, f, ident, w, 0.05)
        assert np.max(np.abs(got - ref)) < 1e-13 * (1.0 + np.max(np.abs(ref)))


@pytest.mark.parametrize("order", [2, 3, 4])
def test_unlimited_programs_move_three_arrays_per_stage(dg, order):
    """Unlimited, every stage reads its stage state and at most w^n and writes
    one state (3 arrays), except the last stage of the five-stage RK4, which
    also reads U_3; no limiter passes; register 0 ends as the new state."""
    ops, n_regs = dg.stage_program(order, 0)
    for i, op in enumerate(ops):
        assert len(op["outs"]) == 1 and op["lim_src"] < 0
        others = [r for r in op["ins"] if r != op["in_reg"]]
        extra = 1 if (order == 4 and i == len(ops) - 1) else 0
        assert len(others) <= 1 + extra, (i, op)
        assert 0 in op["ins"] or op["in_reg"] == 0
    assert ops[-1]["outs"] == [0]
    assert n_regs <= 3


def test_stage_program_rejects_bad_arguments(dg):
    with pytest.raises(dg.DGError):
        dg.stage_program(5, 0)
    with pytest.raises(dg.DGError):
        dg.stage_program(3, 2)


def test_checkpoint_version_is_checked_before_any_device_work(dg, tmp_path):
    """A checkpoint of another format version is refused while reading the
    file, before a handle is built."""
    import json
    path = tmp_path / "old.npz"
    with open(path, "wb") as f:
        np.savez(f, version=np.int64(dg.CHECKPOINT_VERSION + 1), config=np.array(json.dumps({})),
                 refinement=np.zeros(0, np.int32), W=np.zeros((4, 3, 1)), meta=np.array("{}"))
    with pytest.raises(ValueError, match="version"):
        dg.Solver.from_checkpoint(path)
    m = dict(wl.mesh_uniform(2, [3, 2], [0.0, 0.0], [1.5, 1.0], bc=[TRN, PER]), refine_boxes=[(1, 0, 2, 1)])
    plain = dg._plain_mesh(m)
    assert plain == json.loads(json.dumps(plain))
    assert plain["refine_boxes"] == [[1, 0, 2, 1]] and plain["bc"] == [TRN, PER]
