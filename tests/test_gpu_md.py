"""Molecular dynamics on the device (mtp_md_*) against the oracle's
velocity-Verlet integrator (oracle.mtp.velocity_verlet, a fresh neighbour list
every step), through the C-ABI.

Tolerances:
  neighbour lists: bit-exact (the per-step exact list equals a fresh build);
  FP64 trajectories (12 steps of 1 fs): positions within 1e-9 A, velocities
    within 1e-7 A/ps, forces within 1e-8 eV/A, energies within 1e-10 relative
    (per-step force differences of ~1e-12 relative, integrated over the run);
  mixed trajectories against the FP64 device trajectory (4 steps of 1 fs):
    the mixed force error (<= 1e-4 eV/A RMS, max below 1e-3) gives
    acceleration errors below 1e-3 / (m 1.0364e-4) A/ps^2, i.e. below 0.2 A/ps^2
    for m >= 50 amu, so after t = 4 fs positions agree within 0.5 a t^2 < 2e-6 A
    and velocities within a t < 1e-3 A/ps; potential energy within 1e-5 eV/atom.
"""
import types

import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import oracle_model, oracle_sampled, pot_dict

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KB = 8.617333e-5   # eV/K


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def start(st, masses, temperature, seed):
    m = np.asarray(masses)[st.z]
    sd = np.sqrt(KB * temperature / (m * O.AMU_A2_PS2_IN_EV))
    v = synth.rng(seed, 7).normal(size=(st.n, 3)) * sd[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return v


def device_run(P, pot, st, v0, masses, dt, n_steps, precision, skin=0.3, rebuild_every=5):
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    v = torch.tensor(v0, device="cuda")
    md = P.MD(pot, x, st.cell, st.pbc, skin=skin)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=precision)["forces"]
    e_pot = torch.empty(n_steps, dtype=torch.float64, device="cuda")
    e_kin = torch.empty(n_steps, dtype=torch.float64, device="cuda")
    md.run(x, v, z, masses, dt, n_steps, f, rebuild_every=rebuild_every, precision=precision, e_pot=e_pot,
           e_kin=e_kin)
    torch.cuda.synchronize()
    return md, x, v, z, f, e_pot.cpu().numpy(), e_kin.cpu().numpy()


def list_arrays(nl):
    off, j, img = nl.to_tensors()
    torch.cuda.synchronize()
    return off.cpu().numpy(), j.cpu().numpy(), img.cpu().numpy()


@pytest.mark.parametrize("name,recipe,masses,n_steps", [
    ("bcc-l8-s1", ("bcc", (4, 4, 4), 3.16, 0.05, 1, 1), [183.84], 12),
    ("bcc-l16-s3", ("bcc", (4, 4, 4), 3.16, 0.08, 3, 2), [183.84, 95.95, 50.94], 4),
])
def test_md_fp64_trajectory_matches_oracle(P, name, recipe, masses, n_steps):
    st = synth.crystal(*recipe)
    pot = P.Potential.from_dict(pot_dict(name))
    v0 = start(st, masses, 300.0, 11)
    dt = 1e-3
    md, x, v, z, f, e_pot, e_kin = device_run(P, pot, st, v0, masses, dt, n_steps, P.MTP_FP64, rebuild_every=5)
    xo, vo, fo, epo, eko = O.velocity_verlet(oracle_model(name), st.x, v0, st.z, st.cell, st.pbc, masses, dt,
                                             n_steps)
    assert np.abs(xo - st.x).max() > 1e-3
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-7
    assert np.abs(f.cpu().numpy() - fo).max() <= 1e-8
    assert np.allclose(e_pot, epo, rtol=1e-10, atol=1e-10)
    assert np.allclose(e_kin, eko, rtol=1e-10, atol=1e-12)
    assert md.status() == n_steps - 5 * ((n_steps - 1) // 5)   # steps since the last rebuild


def test_md_exact_list_equals_fresh_build_and_oracle(P):
    st = synth.crystal("bcc", (5, 4, 3), 3.16, 0.08, 3, 2)
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    masses = [183.84, 95.95, 50.94]
    # hot (1000 K) and the random potential's forces (4 eV/A RMS, 21 max here)
    # move atoms up to ~0.4 A in 10 fs, so pairs cross the cutoff; skin 1.5 A
    v0 = start(st, masses, 1000.0, 12)
    md, x, v, z, f, _, _ = device_run(P, pot, st, v0, masses, 1e-3, 10, P.MTP_FP64, skin=1.5, rebuild_every=0)
    md.status()   # no atom moved more than skin/2: the list is complete
    mine = list_arrays(md.nlist())
    fresh = list_arrays(P.mtp_build_neighbors(pot, x, st.cell, st.pbc))
    for a, b in zip(mine, fresh):
        assert np.array_equal(a, b)
    xn = x.cpu().numpy()
    i, j, n = O.neighbor_list(xn, st.cell, st.pbc, pot.r_cut)
    assert np.array_equal(mine[1], j) and np.array_equal(mine[2], n)
    assert np.array_equal(mine[0], np.searchsorted(i, np.arange(st.n + 1)))
    # the list changed during the run (pairs entered or left the cutoff)
    i0, j0, _ = O.neighbor_list(st.x, st.cell, st.pbc, pot.r_cut)
    assert len(i0) != len(i) or not np.array_equal(j0, j)


def test_md_mixed_trajectory_against_fp64(P):
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.08, 3, 2)
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    masses = [183.84, 95.95, 50.94]
    v0 = start(st, masses, 300.0, 13)
    ref = device_run(P, pot, st, v0, masses, 1e-3, 4, P.MTP_FP64)
    mix = device_run(P, pot, st, v0, masses, 1e-3, 4, P.MTP_MIXED)
    assert np.abs(mix[1].cpu().numpy() - ref[1].cpu().numpy()).max() <= 2e-6
    assert np.abs(mix[2].cpu().numpy() - ref[2].cpu().numpy()).max() <= 1e-3
    assert np.abs(mix[5] - ref[5]).max() <= 1e-5 * st.n


def test_md_checked_rebuilds_keep_the_oracle_trajectory(P):
    """Displacements checked every step with a skin so small that the list is
    rebuilt during the run: the trajectory still equals the oracle's."""
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)
    pot = P.Potential.from_dict(pot_dict("bcc-l8-s1"))
    v0 = start(st, [183.84], 300.0, 17)
    md, x, v, z, f, e_pot, _ = device_run(P, pot, st, v0, [183.84], 1e-3, 8, P.MTP_FP64, skin=0.01,
                                          rebuild_every=-1)
    assert md.rebuilds() >= 3
    md.status()
    xo, vo, _, epo, _ = O.velocity_verlet(oracle_model("bcc-l8-s1"), st.x, v0, st.z, st.cell, st.pbc, [183.84],
                                          1e-3, 8)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-7
    assert np.allclose(e_pot, epo, rtol=1e-10, atol=1e-10)


def test_md_stale_list_is_reported(P):
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)
    pot = P.Potential.from_dict(pot_dict("bcc-l8-s1"))
    v0 = start(st, [183.84], 300.0, 14)
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    v = torch.tensor(v0, device="cuda")
    md = P.MD(pot, x, st.cell, st.pbc, skin=1e-4)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_FP64)["forces"]
    md.run(x, v, z, [183.84], 1e-3, 3, f, rebuild_every=0, precision=P.MTP_FP64)
    with pytest.raises(P.MtpError) as err:
        md.status()
    assert err.value.code == P._lib.MTP_ERR_STALE_LIST
    md.rebuild(x)
    assert md.status() == 0
    with pytest.raises(P.MtpError) as err:
        md.run(x, v, z, [183.84], 1e-3, 6, f, rebuild_every=4, precision=P.MTP_FP64)
    assert err.value.code == P._lib.MTP_ERR_STALE_LIST


def test_md_graph_replay_matches_direct_steps(P):
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)
    pot = P.Potential.from_dict(pot_dict("bcc-l8-s1"))
    masses = [183.84]
    v0 = start(st, masses, 300.0, 15)
    runs = []
    for use_graph in (False, True):
        x = torch.tensor(st.x, device="cuda")
        z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
        v = torch.tensor(v0, device="cuda")
        md = P.MD(pot, x, st.cell, st.pbc, skin=0.5)
        f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_FP64)["forces"]
        md.run(x, v, z, masses, 1e-3, 1, f, precision=P.MTP_FP64)   # sizes every scratch buffer
        torch.cuda.synchronize()
        if use_graph:
            s = torch.cuda.Stream()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                md.run(x, v, z, masses, 1e-3, 1, f, precision=P.MTP_FP64)
            for _ in range(6):
                g.replay()
        else:
            md.run(x, v, z, masses, 1e-3, 6, f, precision=P.MTP_FP64)
        torch.cuda.synchronize()
        md.status()
        runs.append((x.cpu().numpy(), v.cpu().numpy()))
    assert np.abs(runs[0][0] - st.x).max() > 1e-3
    # identical up to the order of the FP64 force atomics
    assert np.abs(runs[0][0] - runs[1][0]).max() <= 1e-11
    assert np.abs(runs[0][1] - runs[1][1]).max() <= 1e-9


def test_md_full_size_list_and_sampled_forces(P):
    """The 1,024,000-atom level-16 workload as the MD section of bench.py runs
    it (mixed, dt 0.01 fs, skin 0.3 A, displacements checked every step):
    after 50 steps the exact list equals a fresh build and sampled forces
    match the oracle at the final positions."""
    st = synth.crystal("bcc", (80, 80, 80), 3.16, 0.08, 3, 2)
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    masses = [183.84, 95.95, 50.94]
    v0 = start(st, masses, 300.0, 16)
    md, x, v, z, f, e_pot, e_kin = device_run(P, pot, st, v0, masses, 1e-5, 50, P.MTP_MIXED, skin=0.3,
                                              rebuild_every=-1)
    md.status()
    # the oracle below needs a compact structure (no atom far from its site)
    assert float((x.cpu() - torch.tensor(st.x)).abs().max()) < 0.5
    assert np.all(np.isfinite(e_pot)) and np.all(np.isfinite(e_kin))
    mine = list_arrays(md.nlist())
    fresh = list_arrays(P.mtp_build_neighbors(pot, x, st.cell, st.pbc))
    for a, b in zip(mine, fresh):
        assert np.array_equal(a, b)
    fin = types.SimpleNamespace(x=x.cpu().numpy(), z=st.z, cell=st.cell, pbc=st.pbc, n=st.n)
    atoms = [0, 123457, 1023999]
    ref = oracle_sampled(oracle_model("bcc-l16-s3"), fin, pot.r_cut, atoms, force_atoms=atoms)
    got = f.cpu().numpy()[atoms]
    assert np.sqrt(((got - ref["forces"]) ** 2).mean()) <= 1e-4


def test_md_npt_fp64_matches_oracle(P):
    """Berendsen NPT (isotropic, strong coupling so that the cell moves by
    ~1e-4 per step) against the oracle's berendsen_npt: positions, velocities,
    cell and pressure after 6 steps of 1 fs (FP64 forces)."""
    name = "bcc-l8-s1"
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)
    pot = P.Potential.from_dict(pot_dict(name))
    masses = [183.84]
    v0 = start(st, masses, 300.0, 13)
    dt, n_steps, p0, tau, bulk = 1e-3, 6, 0.0, 1e-2, 1e7
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    v = torch.tensor(v0, device="cuda")
    md = P.MD(pot, x, st.cell, st.pbc, skin=0.3)
    md.set_barostat(p0, tau, bulk)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_FP64)["forces"]
    assert md.run(x, v, z, masses, dt, n_steps, f, rebuild_every=-1, precision=P.MTP_FP64) == 0
    info = md.info()
    xo, vo, fo, cello, pro = O.berendsen_npt(oracle_model(name), st.x, v0, st.z, st.cell, st.pbc, masses, dt,
                                             n_steps, p0, tau, bulk)
    assert abs(np.linalg.det(cello) / np.linalg.det(st.cell) - 1) > 1e-5   # the cell moved
    assert np.abs(info["cell"] - cello).max() <= 1e-12 * np.abs(cello).max()
    assert info["pressure_bar"] == pytest.approx(pro[-1], rel=1e-8, abs=1e-6)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9
    assert np.abs(v.cpu().numpy() - vo).max() <= 1e-7
    assert np.abs(f.cpu().numpy() - fo).max() <= 1e-8
    # the exact list at the final (scaled) positions equals a fresh build in the final cell
    mine = list_arrays(md.nlist())
    fresh = list_arrays(P.mtp_build_neighbors(pot, x, info["cell"], st.pbc))
    for a, b in zip(mine, fresh):
        assert np.array_equal(a, b)


def _active(P):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "potentials",
                           "bcc-l16-s1-active.json")) as fh:
        act = json.load(fh)
    m = act["m"]
    return np.asarray(act["a_inv"]).reshape(m, m)


def test_md_grade_every_x_steps_matches_oracle(P):
    """The grade evaluated inside the run every 2 steps (paper: every X steps
    of the MD): the largest grade of the last evaluation and the selection
    flags accumulated over the run equal the oracle's grades of the oracle
    trajectory at steps 2, 4 and 6 (FP64 forces, level 16, 128 atoms)."""
    name = "bcc-l16-s1"
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.12, 1, 5)
    pot = P.Potential.from_dict(pot_dict(name))
    masses = [183.84]
    v0 = start(st, masses, 300.0, 14)
    a_inv = _active(P)
    dt, every, n_steps = 1e-3, 2, 6
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    v = torch.tensor(v0, device="cuda")
    md = P.MD(pot, x, st.cell, st.pbc, skin=0.3)
    model = oracle_model(name)
    # oracle trajectory and grades at the evaluation steps
    xo, vo, fo = st.x, v0, None
    gam = []
    for _ in range(n_steps // every):
        xo, vo, fo, _, _ = O.velocity_verlet(model, xo, vo, st.z, st.cell, st.pbc, masses, dt, every, f=fo)
        b = O.basis_matrix(model, xo, st.z, st.cell, O.neighbor_list(xo, st.cell, st.pbc, pot.r_cut))
        gam.append(O.grade(b, a_inv))
    gam = np.array(gam)
    tau_sel = float(np.median(gam))          # about half the atoms selected at some step
    tau_brk = float(gam.max()) * 10.0
    flags_ref = np.zeros(st.n, dtype=np.uint8)
    for g in gam:
        flags_ref |= O.grade_flags(g, tau_sel, tau_brk).astype(np.uint8)
    sel = torch.zeros(st.n, dtype=torch.uint8, device="cuda")
    a_inv_d = torch.tensor(a_inv, device="cuda")
    md.set_grade(a_inv_d, every, tau_sel, tau_brk, P.MTP_GRADE_TENSOR, sel)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_FP64)["forces"]
    assert md.run(x, v, z, masses, dt, n_steps, f, rebuild_every=-1, precision=P.MTP_FP64) == 0
    info = md.info()
    assert info["grade_evals"] == n_steps // every
    assert info["gamma_max_last"] == pytest.approx(gam[-1].max(), rel=1e-7)
    assert info["n_selected_last"] == int((gam[-1] > tau_sel).sum())
    assert np.array_equal(sel.cpu().numpy(), flags_ref)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9


def test_md_grade_break_stops_the_run(P):
    """A break threshold below the grades stops mtp_md_run with
    MTP_STATUS_BREAK right after the first evaluation step; the completed
    step's state is kept and the run can continue after the grade is off."""
    name = "bcc-l16-s1"
    st = synth.crystal("bcc", (4, 4, 4), 3.16, 0.12, 1, 5)
    pot = P.Potential.from_dict(pot_dict(name))
    masses = [183.84]
    v0 = start(st, masses, 300.0, 14)
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    v = torch.tensor(v0, device="cuda")
    md = P.MD(pot, x, st.cell, st.pbc, skin=0.3)
    md.set_grade(torch.tensor(_active(P), device="cuda"), 3, 1e-3, 1e-3, P.MTP_GRADE_FP64)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_MIXED)["forces"]
    assert md.run(x, v, z, masses, 1e-3, 10, f, rebuild_every=-1, precision=P.MTP_MIXED) == P.MTP_STATUS_BREAK
    info = md.info()
    assert info["steps"] == 3 and info["grade_evals"] == 1
    assert info["n_selected_last"] == st.n
    md.set_grade(None, 0)
    assert md.run(x, v, z, masses, 1e-3, 2, f, rebuild_every=-1, precision=P.MTP_MIXED) == 0
    assert md.info()["steps"] == 5
