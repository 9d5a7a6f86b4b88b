"""Parity of the CUDA path with the oracle, through the C-ABI.

Tolerances (float64 outputs in every mode):
  neighbour lists: bit-exact (offsets, j, images, order);
  FP64 path: site energies within 1e-12 relative (|dE_i| <= 1e-12 max(1, |E_i|)),
             total energy within 1e-12 of sum |E_i|, forces within 1e-10 eV/A,
             virial within 1e-10 of max |W| (and 1e-10 eV absolute);
  mixed path: |dE_i| <= 1e-5 eV/atom and force RMS error <= 1e-4 eV/A (the
             stated target of the level-16 workloads); for the level-20
             workload, which states no mixed target, the mixed-precision bound
             of tests/test_gpu_mixed_bound.py: |dE_i| <= 1e-5 eV + 64 u a_i with
             u = 2^-24 and a_i = sum_alpha |xi_alpha B_alpha(i)| (first-order
             FP32 rounding of products of up to ten moment contractions).
The energy/force calls here take the library's default kernel for these small
boxes; tests/test_gpu_team.py runs both kernels explicitly.
"""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import oracle_model, oracle_sampled, pot_dict, structure

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


_POTS = {}


def gpu_pot(P, name):
    if name not in _POTS:
        if name.startswith("rc"):
            # list-only cases: any level-8 potential with this cutoff
            d = dict(pot_dict("bcc-l8-s1"))
            d["r_cut"] = float(name[2:])
            _POTS[name] = P.Potential.from_dict(d)
        else:
            _POTS[name] = P.Potential.from_dict(pot_dict(name))
    return _POTS[name]


def dev(st):
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    return x, z


def gpu_list(P, pot, st):
    x, _ = dev(st)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    off, j, img = nl.to_tensors()
    torch.cuda.synchronize()
    return nl, off.cpu().numpy(), j.cpu().numpy(), img.cpu().numpy()


NEIGHBOR_CASES = {
    "bcc-4x4x4": ("bcc-l8-s1", ("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)),
    "bcc-5x4x3-s3": ("bcc-l16-s3", ("bcc", (5, 4, 3), 3.16, 0.08, 3, 2)),
    "fcc-3x3x2": ("rc5.5", ("fcc", (3, 3, 2), 3.6, 0.1, 4, 3)),
    "gas-8": ("gas-l16-s2", ("gas", 8, 0, 0, 2, 4)),
    "gas-37": ("gas-l16-s2", ("gas", 37, 0, 0, 2, 4)),
}


@pytest.mark.parametrize("case", sorted(NEIGHBOR_CASES))
def test_neighbor_list_bit_exact(P, case):
    name, rec = NEIGHBOR_CASES[case]
    st = structure(*rec)
    pot = gpu_pot(P, name)
    _, off, j, img = gpu_list(P, pot, st)
    i0, j0, n0 = O.neighbor_list(st.x, st.cell, st.pbc, pot.r_cut)
    assert off[-1] == len(j0)
    assert np.array_equal(np.repeat(np.arange(st.n), np.diff(off)), i0)
    assert np.array_equal(j, j0)
    assert np.array_equal(img, n0)


def test_neighbor_list_unwrapped_positions_and_open_axes(P):
    pot = gpu_pot(P, "bcc-l8-s1")
    st = structure("bcc", (3, 4, 4), 3.16, 0.05, 1, 1)
    st.x = st.x + np.array([[1, -2, 0]]) @ st.cell * (np.arange(st.n)[:, None] % 3 == 0)
    for pbc in [(1, 1, 1), (0, 1, 1), (0, 0, 0)]:
        st.pbc = pbc
        _, off, j, img = gpu_list(P, pot, st)
        i0, j0, n0 = O.neighbor_list(st.x, st.cell, pbc, pot.r_cut)
        assert np.array_equal(np.repeat(np.arange(st.n), np.diff(off)), i0)
        assert np.array_equal(j, j0) and np.array_equal(img, n0)


EFV_CASES = {
    # config 1 exactly: 128-atom BCC, level 8, one species
    "cfg1-bcc-l8": ("bcc-l8-s1", ("bcc", (4, 4, 4), 3.16, 0.05, 1, 1)),
    # configs 2 and 5 shapes, reduced: several 128-thread blocks and a ragged tail
    "cfg2-bcc-l16-s3": ("bcc-l16-s3", ("bcc", (5, 4, 4), 3.16, 0.08, 3, 2)),
    "cfg2-bcc-l16-s3-rc5.6": ("bcc-l16-s3-rc5.6", ("bcc", (4, 4, 3), 3.16, 0.08, 3, 2)),
    "cfg5-bcc-l16-s1": ("bcc-l16-s1", ("bcc", (5, 4, 4), 3.16, 0.15, 1, 5)),
    "cfg4-gas-l16-s2": ("gas-l16-s2", ("gas", 45, 0, 0, 2, 4)),
    # config 3 shape, reduced: level 20, four species, FCC, 54 neighbours
    "cfg3-fcc-l20-s4": ("fcc-l20-s4", ("fcc", (2, 2, 2), 3.6, 0.1, 4, 3)),
}

_ORACLE_CACHE = {}


def oracle_efv(case):
    if case not in _ORACLE_CACHE:
        name, rec = EFV_CASES[case]
        st = structure(*rec)
        model = oracle_model(name)
        nl = O.neighbor_list(st.x, st.cell, st.pbc, pot_dict(name)["r_cut"])
        out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "f", "w", "dtheta"))
        out["abs_terms"] = np.abs(O.basis_matrix(model, st.x, st.z, st.cell, nl)) @ np.abs(model.xi.numpy())
        _ORACLE_CACHE[case] = (st, out)
    return _ORACLE_CACHE[case]


def run_gpu(P, name, st, precision, dtheta=False, chunk=0):
    pot = gpu_pot(P, name)
    x, z = dev(st)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision, dtheta=dtheta, chunk_atoms=chunk)
    torch.cuda.synchronize()
    assert P.mtp_device_status(pot) == 0
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


@pytest.mark.parametrize("case", sorted(EFV_CASES))
def test_efv_fp64_matches_oracle(P, case):
    name = EFV_CASES[case][0]
    st, ref = oracle_efv(case)
    got = run_gpu(P, name, st, P.MTP_FP64, dtheta=True)
    e_ref = ref["e_atom"]
    assert np.all(np.abs(got["e_atom"] - e_ref) <= 1e-12 * np.maximum(1.0, np.abs(e_ref)))
    assert abs(got["e_total"][0] - ref["e"]) <= 1e-12 * np.abs(e_ref).sum()
    assert np.abs(got["forces"] - ref["f"]).max() <= 1e-10
    assert np.abs(got["virial"] - ref["w"]).max() <= max(1e-10, 1e-10 * np.abs(ref["w"]).max())
    theta_ref = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
    scale = np.maximum(1.0, np.abs(theta_ref))
    assert np.all(np.abs(got["dtheta"] - theta_ref) <= 1e-10 * scale)


@pytest.mark.parametrize("case", sorted(EFV_CASES))
def test_efv_mixed_within_stated_error(P, case):
    name = EFV_CASES[case][0]
    st, ref = oracle_efv(case)
    got = run_gpu(P, name, st, P.MTP_MIXED, dtheta=True)
    tol = 1e-5 + (64 * 2.0 ** -24 * ref["abs_terms"] if pot_dict(name)["level"] > 16 else 0.0)
    assert np.all(np.abs(got["e_atom"] - ref["e_atom"]) <= tol)
    assert np.sqrt(np.mean((got["forces"] - ref["f"]) ** 2)) <= 1e-4
    assert abs(got["e_total"][0] - ref["e"]) / st.n <= np.max(tol)
    assert np.abs(got["virial"] - ref["w"]).max() <= 1e-4 * max(1.0, np.abs(ref["w"]).max())
    theta_ref = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
    assert np.abs(got["dtheta"] - theta_ref).max() <= 1e-4 * max(1.0, np.abs(theta_ref).max())


def test_chunked_launches_match_single_launch(P):
    name, rec = EFV_CASES["cfg2-bcc-l16-s3"]
    st = structure(*rec)
    a = run_gpu(P, name, st, P.MTP_FP64)
    b = run_gpu(P, name, st, P.MTP_FP64, chunk=37)
    assert np.abs(a["e_atom"] - b["e_atom"]).max() <= 1e-13
    assert np.abs(a["forces"] - b["forces"]).max() <= 1e-12


def test_level20_split_kernels_in_chunks_match_oracle(P):
    """Level 20 runs as three kernels (moment sweep, contraction, adjoint
    sweep) through a scratch of the chunk's moments: 108-atom FCC (4 species)
    in one chunk, in chunks of 37 (a ragged last chunk) and of one atom, FP64
    with dE/dtheta against the oracle; mixed chunked against unchunked."""
    name = "fcc-l20-s4"
    st = structure("fcc", (3, 3, 3), 3.6, 0.1, 4, 3)
    model = oracle_model(name)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, pot_dict(name)["r_cut"])
    ref = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "f", "w", "dtheta"))
    theta_ref = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
    for chunk in (0, 37, 1):
        got = run_gpu(P, name, st, P.MTP_FP64, dtheta=True, chunk=chunk)
        assert np.all(np.abs(got["e_atom"] - ref["e_atom"]) <= 1e-12 * np.maximum(1.0, np.abs(ref["e_atom"]))), chunk
        assert np.abs(got["forces"] - ref["f"]).max() <= 1e-10, chunk
        assert np.abs(got["virial"] - ref["w"]).max() <= max(1e-10, 1e-10 * np.abs(ref["w"]).max()), chunk
        assert np.all(np.abs(got["dtheta"] - theta_ref) <= 1e-10 * np.maximum(1.0, np.abs(theta_ref))), chunk
    a = run_gpu(P, name, st, P.MTP_MIXED, dtheta=True)
    b = run_gpu(P, name, st, P.MTP_MIXED, dtheta=True, chunk=37)
    assert np.abs(a["e_atom"] - b["e_atom"]).max() <= 1e-9
    # FP32 force atomics add each atom's ~2 x 54 pair terms in an order that
    # depends on the launch: a few units in the last place of the largest force
    assert np.abs(a["forces"] - b["forces"]).max() <= 2.0 ** -17 * max(1.0, np.abs(a["forces"]).max())


def test_empty_and_isolated_atoms(P):
    pot = gpu_pot(P, "bcc-l8-s1")
    st = synth.Structure(np.array([[1.0, 1.0, 1.0], [30.0, 30.0, 30.0]]), np.zeros(2, np.int32), np.eye(3) * 60.0,
                         (1, 1, 1))
    got = run_gpu(P, "bcc-l8-s1", st, P.MTP_FP64)
    assert np.allclose(got["e_atom"], pot_dict("bcc-l8-s1")["species_energy"][0], rtol=0, atol=1e-15)
    assert np.all(got["forces"] == 0.0)


@pytest.mark.slow
def test_full_size_config2_sampled_parity(P):
    """1,024,000-atom BCC, 3 species, level 16: sampled site energies and forces
    against the oracle, neighbour counts, and sum of forces = 0."""
    name = "bcc-l16-s3"
    st = synth.crystal("bcc", (80, 80, 80), 3.16, 0.08, 3, 2)
    model = oracle_model(name)
    g = synth.rng(2, 77)
    centres = np.sort(g.choice(st.n, 24, replace=False))
    force_atoms = centres[:4]
    ref = oracle_sampled(model, st, 5.0, centres, force_atoms)
    for precision, e_tol, f_tol in [(P.MTP_FP64, 1e-12, 1e-10), (P.MTP_MIXED, 1e-5, 1e-4)]:
        pot = gpu_pot(P, name)
        x, z = dev(st)
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        off, _, _ = nl.to_tensors()
        off = off.cpu().numpy()
        assert np.array_equal(np.diff(off)[centres], ref["nbr_count"])
        out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision)
        e = out["e_atom"].cpu().numpy()
        f = out["forces"].cpu().numpy()
        assert np.all(np.abs(e[centres] - ref["e_atom"]) <= e_tol * np.maximum(1, np.abs(ref["e_atom"])))
        assert np.abs(f[force_atoms] - ref["forces"]).max() <= f_tol * (1 if precision == P.MTP_FP64 else 10)
        assert np.abs(f.sum(axis=0)).max() <= (1e-8 if precision == P.MTP_FP64 else 1e-2)
        assert abs(out["e_total"].item() - e.sum()) <= 1e-9 * np.abs(e).sum()


@pytest.mark.slow
def test_full_size_config3_sampled_parity(P):
    """256,000-atom FCC (40^3 cells, a = 3.6 A, sigma 0.1 A), 4 species, level 20:
    sampled site energies and forces against the oracle (FP64)."""
    name = "fcc-l20-s4"
    st = synth.crystal("fcc", (40, 40, 40), 3.6, 0.1, 4, 3)
    model = oracle_model(name)
    centres = np.sort(synth.rng(3, 77).choice(st.n, 8, replace=False))
    ref = oracle_sampled(model, st, 5.5, centres, centres[:2])
    pot = gpu_pot(P, name)
    x, z = dev(st)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_FP64)
    e = out["e_atom"].cpu().numpy()
    f = out["forces"].cpu().numpy()
    assert np.all(np.abs(e[centres] - ref["e_atom"]) <= 1e-12 * np.maximum(1, np.abs(ref["e_atom"])))
    assert np.abs(f[centres[:2]] - ref["forces"]).max() <= 1e-10
    assert np.abs(f.sum(axis=0)).max() <= 1e-8
