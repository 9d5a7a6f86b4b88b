"""Force-matching double backward through torch.autograd over the C-ABI:
d loss / d theta with loss = (1/3N) sum |F - F_t|^2, F = -dE/dx, against the
oracle's double backward (FP64, 1e-8 relative to the largest entry), the
Hessian-vector product against central differences of the GPU forces, and
the mixed-precision path with its error stated against the FP64 result."""
import numpy as np
import pytest

import synth
from oracle import mtp as O
from tests.helpers import oracle_model, pot_dict, structure

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


CASES = {
    "bcc-l8-s1": ("bcc", (3, 3, 3), 3.16, 0.1, 1, 1),
    "bcc-l16-s3": ("bcc", (3, 3, 2), 3.16, 0.1, 3, 2),
    # config 3 recipe on a 2-cell, 32-atom FCC box (level 20, 4 species)
    "fcc-l20-s4": ("fcc", (2, 2, 2), 3.6, 0.1, 4, 3),
}


def gpu_loss_grad(P, name, st, ft, precision):
    from paper_2510_00193_gb300.autograd import energy
    pot = P.Potential.from_dict(pot_dict(name))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda", requires_grad=True)
    z = torch.tensor(st.z, device="cuda")
    nl = P.mtp_build_neighbors(pot, x.detach(), st.cell, st.pbc)
    theta = pot.initial_theta().requires_grad_(True)
    e = energy(pot, nl, x, z, st.cell, theta, precision)
    (gx,) = torch.autograd.grad(e, x, create_graph=True)
    f = -gx
    loss = ((f - torch.tensor(ft, device="cuda")) ** 2).sum() / (3 * st.n)
    loss.backward()
    return loss.item(), theta.grad.cpu().numpy(), pot, nl, x, z


@pytest.mark.parametrize("name", sorted(CASES))
def test_force_matching_gradient_matches_oracle(P, name):
    st = structure(*CASES[name])
    ft = synth.target_forces(st.n, 9)
    loss, g, *_ = gpu_loss_grad(P, name, st, ft, P.MTP_FP64)
    model = oracle_model(name)
    nl = O.neighbor_list(st.x, st.cell, st.pbc, pot_dict(name)["r_cut"])
    loss_ref, grads = O.force_matching_grad(model, st.x, st.z, st.cell, nl, ft)
    ref = np.concatenate([grads[0], grads[1].ravel(), grads[2]])
    assert loss == pytest.approx(loss_ref, rel=1e-10)
    assert np.abs(g - ref).max() <= 1e-8 * np.abs(ref).max()
    # mixed precision: same gradient within 1e-4 of the largest entry
    _, gm, *_ = gpu_loss_grad(P, name, st, ft, P.MTP_MIXED)
    assert np.abs(gm - ref).max() <= 1e-4 * np.abs(ref).max()


def test_hessian_vector_product_matches_finite_differences(P):
    name = "bcc-l16-s3"
    st = structure(*CASES[name])
    pot = P.Potential.from_dict(pot_dict(name))
    z = torch.tensor(st.z, device="cuda")
    v = synth.rng(3, 9).normal(size=st.x.shape)
    x = torch.tensor(st.x, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    tan = P.mtp_compute_efv_tangent(pot, nl, x, z, st.cell, torch.tensor(v, device="cuda"), precision=P.MTP_FP64)
    h = 1e-5
    fp = P.mtp_compute_efv(pot, nl, torch.tensor(st.x + h * v, device="cuda"), z, st.cell, precision=P.MTP_FP64,
                           dtheta=True)
    fm = P.mtp_compute_efv(pot, nl, torch.tensor(st.x - h * v, device="cuda"), z, st.cell, precision=P.MTP_FP64,
                           dtheta=True)
    fd_f = (fp["forces"] - fm["forces"]).cpu().numpy() / (2 * h)
    fd_t = (fp["dtheta"] - fm["dtheta"]).cpu().numpy() / (2 * h)
    got_f = tan["force_tan"].cpu().numpy()
    got_t = tan["dtheta_tan"].cpu().numpy()
    assert np.abs(got_f - fd_f).max() <= 1e-5 * max(1.0, np.abs(fd_f).max())
    assert np.abs(got_t - fd_t).max() <= 1e-5 * max(1.0, np.abs(fd_t).max())


@pytest.mark.slow
def test_full_size_config3_directional_derivatives(P):
    """256,000-atom FCC, level 20: the tangent of dE/dtheta and of the forces
    along a random direction equals central differences of the FP64 results
    (a property that holds at any size)."""
    name = "fcc-l20-s4"
    st = synth.crystal("fcc", (40, 40, 40), 3.6, 0.1, 4, 3)
    pot = P.Potential.from_dict(pot_dict(name))
    z = torch.tensor(st.z, device="cuda")
    v = synth.rng(3, 10).normal(size=st.x.shape)
    x = torch.tensor(st.x, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    tan = P.mtp_compute_efv_tangent(pot, nl, x, z, st.cell, torch.tensor(v, device="cuda"), precision=P.MTP_FP64)
    # fourth-order central differences: close contacts make some Hessian
    # entries ~1e7, where the second-order stencil's truncation error shows
    h = 1e-5
    vals = {}
    for k in (-2, -1, 1, 2):
        o = P.mtp_compute_efv(pot, nl, torch.tensor(st.x + k * h * v, device="cuda"), z, st.cell,
                              precision=P.MTP_FP64, dtheta=True)
        vals[k] = (o["dtheta"].cpu().numpy(), o["forces"].cpu().numpy())
    fd_t = (-vals[2][0] + 8 * vals[1][0] - 8 * vals[-1][0] + vals[-2][0]) / (12 * h)
    fd_f = (-vals[2][1] + 8 * vals[1][1] - 8 * vals[-1][1] + vals[-2][1]) / (12 * h)
    assert np.abs(tan["dtheta_tan"].cpu().numpy() - fd_t).max() <= 1e-5 * np.abs(fd_t).max()
    assert np.abs(tan["force_tan"].cpu().numpy() - fd_f).max() <= 1e-5 * np.abs(fd_f).max()


def test_theta_drives_the_potential(P):
    """theta passed to the autograd energy is uploaded into the handle: with
    every xi doubled and the species energies shifted, the energy, forces and
    force-matching gradient equal those of a potential loaded with those
    parameters, and the original theta gives the original energy back."""
    from paper_2510_00193_gb300.autograd import energy
    name = "bcc-l16-s3"
    st = structure(*CASES[name])
    d = pot_dict(name)
    pot = P.Potential.from_dict(d)
    d2 = dict(d)
    d2["xi"] = [2.0 * v for v in d["xi"]]
    d2["species_energy"] = [v + 0.25 for v in d["species_energy"]]
    pot2 = P.Potential.from_dict(d2)
    z = torch.tensor(st.z, device="cuda")
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda", requires_grad=True)
    nl = P.mtp_build_neighbors(pot, x.detach(), st.cell, st.pbc)
    theta2 = pot2.initial_theta().requires_grad_(True)
    e = energy(pot, nl, x, z, st.cell, theta2, P.MTP_FP64)
    (gx,) = torch.autograd.grad(e, x, create_graph=True)
    ft = torch.tensor(synth.target_forces(st.n, 9), device="cuda")
    loss = ((-gx - ft) ** 2).sum() / (3 * st.n)
    loss.backward()
    ref = P.mtp_compute_efv(pot2, nl, x.detach(), z, st.cell, precision=P.MTP_FP64, dtheta=True)
    assert abs(e.item() - ref["e_total"].item()) <= 1e-12 * abs(ref["e_total"].item())
    assert torch.allclose(-gx.detach(), ref["forces"], rtol=0, atol=1e-10)
    tan = P.mtp_compute_efv_tangent(pot2, nl, x.detach(), z, st.cell, (ref["forces"] - ft).contiguous(),
                                    precision=P.MTP_FP64)
    want = -2.0 / (3 * st.n) * tan["dtheta_tan"]
    assert torch.allclose(theta2.grad, want, rtol=0, atol=1e-10 * want.abs().max().item())
    e0 = energy(pot, nl, x.detach(), z, st.cell, pot.initial_theta(), P.MTP_FP64)
    ref0 = P.mtp_compute_efv(P.Potential.from_dict(d), nl, x.detach(), z, st.cell, precision=P.MTP_FP64)
    assert abs(e0.item() - ref0["e_total"].item()) <= 1e-12 * abs(ref0["e_total"].item())
