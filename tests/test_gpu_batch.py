"""Batched evaluation of many small periodic configurations: neighbour lists
bit-exact per configuration, FP64 energies/forces/virials/dE-dtheta against
the oracle (same tolerances as the single-configuration parity tests), the
mixed path, agreement with per-configuration launches, tuning, and replay
under a CUDA graph.

Mixed-path tolerance for these random gases (the workload states none):
|dE_i| <= 1e-5 eV + 1e-6 sum_alpha |xi_alpha B_alpha(i)| and force RMS
<= 1e-4 eV/A.  The second term is FP32 rounding (6e-8) times a cancellation
allowance of ~16 on the sum of basis contributions: contacts down to 1.9 A
fall below R_min = 2.0 A, where the Chebyshev polynomials are extrapolated and
individual terms grow."""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import oracle_model, pot_dict

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NAME = "gas-l16-s2"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def concat(structs):
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])]).astype(np.int64)
    x = np.concatenate([s.x for s in structs])
    z = np.concatenate([s.z for s in structs]).astype(np.int32)
    cells = np.stack([s.cell for s in structs])
    return off, x, z, cells


@pytest.fixture(scope="module")
def small_batch():
    structs = synth.random_gas_batch(20, 8, 256, 0.085, 1.9, 2, 4, workers=1)
    return structs, concat(structs)


@pytest.fixture(scope="module")
def oracle_results(small_batch):
    structs, _ = small_batch
    model = oracle_model(NAME)
    xi = np.abs(model.xi.numpy())
    res = []
    for st in structs:
        nl = O.neighbor_list(st.x, st.cell, st.pbc, 5.0)
        out = O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "f", "w", "dtheta"))
        out["abs_terms"] = np.abs(O.basis_matrix(model, st.x, st.z, st.cell, nl)) @ xi
        res.append((nl, out))
    return res


def gpu_batch(P, small_batch, precision, dtheta=True, tune=False):
    structs, (off, x, z, cells) = small_batch
    pot = P.Potential.from_dict(pot_dict(NAME))
    xd = torch.tensor(x, device="cuda")
    zd = torch.tensor(z, device="cuda")
    b = P.Batch(pot, off, cells, xd)
    chosen = P.mtp_batch_tune(pot, b, xd, zd, precision, dtheta) if tune else None
    out = P.mtp_compute_batch(pot, b, xd, zd, precision=precision, dtheta=dtheta)
    torch.cuda.synchronize()
    assert P.mtp_device_status(pot) == 0
    return pot, b, xd, zd, {k: v.cpu().numpy() for k, v in out.items() if v is not None}, chosen


def test_batch_neighbor_lists_bit_exact(P, small_batch, oracle_results):
    structs, (off, _, _, _) = small_batch
    _, b, _, _, _, _ = gpu_batch(P, small_batch, P.MTP_FP64, dtheta=False)
    o, j, img = (t.cpu().numpy() for t in b.nlist_tensors())
    for c, (st, (nl, _)) in enumerate(zip(structs, oracle_results)):
        seg = slice(o[off[c]], o[off[c + 1]])
        counts = np.diff(o[off[c]:off[c + 1] + 1])
        assert np.array_equal(np.repeat(np.arange(st.n), counts), nl[0])
        assert np.array_equal(j[seg] - off[c], nl[1])
        assert np.array_equal(img[seg], nl[2])


def test_batch_fp64_matches_oracle(P, small_batch, oracle_results):
    structs, (off, _, _, _) = small_batch
    _, _, _, _, got, _ = gpu_batch(P, small_batch, P.MTP_FP64)
    for c, (st, (_, ref)) in enumerate(zip(structs, oracle_results)):
        e = ref["e_atom"]
        assert np.all(np.abs(got["e_atom"][off[c]:off[c + 1]] - e) <= 1e-12 * np.maximum(1, np.abs(e)))
        assert abs(got["e_cfg"][c] - ref["e"]) <= 1e-12 * np.abs(e).sum()
        assert np.abs(got["forces"][off[c]:off[c + 1]] - ref["f"]).max() <= 1e-10
        assert np.abs(got["virial"][c] - ref["w"]).max() <= max(1e-10, 1e-10 * np.abs(ref["w"]).max())
        th = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
        assert np.all(np.abs(got["dtheta"][c] - th) <= 1e-10 * np.maximum(1, np.abs(th)))


def test_batch_mixed_within_stated_error(P, small_batch, oracle_results):
    structs, (off, _, _, _) = small_batch
    _, _, _, _, got, chosen = gpu_batch(P, small_batch, P.MTP_MIXED, tune=True)
    assert chosen in (32, 64, 128, 256)
    for c, (st, (_, ref)) in enumerate(zip(structs, oracle_results)):
        tol = 1e-5 + 1e-6 * ref["abs_terms"]
        assert np.all(np.abs(got["e_atom"][off[c]:off[c + 1]] - ref["e_atom"]) <= tol)
        assert np.sqrt(np.mean((got["forces"][off[c]:off[c + 1]] - ref["f"]) ** 2)) <= 1e-4
        th = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
        assert np.abs(got["dtheta"][c] - th).max() <= 1e-4 * max(1.0, np.abs(th).max())


def test_batch_equals_per_configuration_launches(P, small_batch):
    structs, (off, _, _, _) = small_batch
    pot, _, _, _, got, _ = gpu_batch(P, small_batch, P.MTP_FP64, dtheta=False)
    for c, st in enumerate(structs[:6]):
        x = torch.tensor(st.x, device="cuda")
        z = torch.tensor(st.z, device="cuda")
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        one = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_FP64)
        assert abs(one["e_total"].item() - got["e_cfg"][c]) <= 1e-11 * max(1, abs(got["e_cfg"][c]))
        assert np.abs(one["forces"].cpu().numpy() - got["forces"][off[c]:off[c + 1]]).max() <= 1e-11


def test_batch_replays_under_a_cuda_graph(P, small_batch):
    structs, (off, x, z, cells) = small_batch
    pot = P.Potential.from_dict(pot_dict(NAME))
    xd = torch.tensor(x, device="cuda")
    zd = torch.tensor(z, device="cuda")
    b = P.Batch(pot, off, cells, xd)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = P.mtp_compute_batch(pot, b, xd, zd, precision=P.MTP_MIXED, dtheta=True, stream=s)
        ref = {k: v.clone() for k, v in out.items() if v is not None}
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.mtp_compute_batch(pot, b, xd, zd, precision=P.MTP_MIXED, dtheta=True, out=out, stream=s)
    for k in out:
        if out[k] is not None:
            out[k].zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.allclose(out["e_cfg"], ref["e_cfg"], rtol=0, atol=1e-9)
    # forces: FP32 atomics from every pair in an order that differs between
    # runs; a force is a sum of ~50 pair terms, so replays agree to a few units
    # of 2^-24 times the largest force, not to an absolute 1e-5 (the random
    # gases have forces of tens of eV/A at their closest contacts)
    fscale = max(1.0, ref["forces"].abs().max().item())
    assert (out["forces"] - ref["forces"]).abs().max().item() <= 2.0 ** -17 * fscale
    # FP32 shared-memory atomics: the order of the additions differs between runs
    scale = ref["dtheta"].abs().max().item()
    assert (out["dtheta"] - ref["dtheta"]).abs().max().item() <= 1e-5 * scale


@pytest.mark.slow
def test_full_size_config4_sampled(P):
    """4096 configurations of 8..256 atoms: sampled configurations against the
    oracle and per-configuration sums."""
    structs = synth.random_gas_batch(4096, 8, 256, 0.085, 1.9, 2, 4)
    off, x, z, cells = concat(structs)
    pot = P.Potential.from_dict(pot_dict(NAME))
    xd = torch.tensor(x, device="cuda")
    zd = torch.tensor(z, device="cuda")
    b = P.Batch(pot, off, cells, xd)
    P.mtp_batch_tune(pot, b, xd, zd, P.MTP_MIXED, True)
    out = {k: v.cpu().numpy() for k, v in P.mtp_compute_batch(pot, b, xd, zd, precision=P.MTP_FP64,
                                                               dtheta=True).items() if v is not None}
    model = oracle_model(NAME)
    for c in [0, 1000, 2047, 4095]:
        st = structs[c]
        ref = O.evaluate(model, st.x, st.z, st.cell, O.neighbor_list(st.x, st.cell, st.pbc, 5.0),
                         want=("e", "f", "dtheta"))
        assert abs(out["e_cfg"][c] - ref["e"]) <= 1e-12 * np.abs(ref["e_atom"]).sum()
        assert np.abs(out["forces"][off[c]:off[c + 1]] - ref["f"]).max() <= 1e-10
        th = np.concatenate([ref["dE_ds"], ref["dE_dc"].ravel(), ref["dE_dxi"]])
        assert np.all(np.abs(out["dtheta"][c] - th) <= 1e-10 * np.maximum(1, np.abs(th)))
    e_atom_sum = np.add.reduceat(out["e_atom"], off[:-1])
    assert np.allclose(e_atom_sum, out["e_cfg"], rtol=1e-12, atol=1e-10)
    f_sum = np.add.reduceat(out["forces"], off[:-1], axis=0)
    assert np.abs(f_sum).max() <= 1e-9
