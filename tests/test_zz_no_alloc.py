"""mtp_compute_efv_noalloc against mtp_compute_efv (mixed precision).

The no-allocation entry point is for callers that cannot let the library
allocate device memory during a step (a fixed device-memory budget laid out at
start-up, or loops where cudaMalloc's device-wide synchronisation is not
acceptable).  Its results must equal the regular entry point's within the
mixed-precision tolerance used elsewhere in these tests (site energies 1e-5 eV,
forces 1e-4 eV/A), on two calls in a row that reuse the shared scratch array.
This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from tests.helpers import pot_dict, structure

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


def _alloc(n):
    dev = "cuda"
    return {"e_atom": torch.full((n,), np.nan, dtype=torch.float64, device=dev),
            "forces": torch.full((n, 3), np.nan, dtype=torch.float64, device=dev),
            "virial": torch.full((6,), np.nan, dtype=torch.float64, device=dev),
            "e_total": torch.full((1,), np.nan, dtype=torch.float64, device=dev)}


def test_noalloc_matches_regular_entry_point_on_two_calls(P):
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    # a larger configuration first, then a smaller one: the second call runs on
    # scratch that still holds the first call's positions
    for rec in [("bcc", (6, 5, 5), 3.16, 0.08, 3, 2), ("bcc", (4, 4, 3), 3.16, 0.08, 3, 2, 1)]:
        st = structure(*rec)
        x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
        z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        ref = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
        got = P.mtp_compute_efv_noalloc(pot, nl, x, z, st.cell, _alloc(st.n))
        torch.cuda.synchronize()
        assert P.mtp_device_status(pot) == 0
        r = {k: v.cpu().numpy() for k, v in ref.items() if v is not None}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        assert np.abs(g["e_atom"] - r["e_atom"]).max() <= 1e-5
        assert np.abs(g["forces"] - r["forces"]).max() <= 1e-4
        assert np.abs(g["virial"] - r["virial"]).max() <= 1e-4 * max(1.0, np.abs(r["virial"]).max())
        assert abs(g["e_total"][0] - r["e_total"][0]) <= 1e-5 * st.n


def test_noalloc_rejects_configurations_beyond_its_scratch(P):
    from paper_2510_00193_gb300 import _lib
    pot = P.Potential.from_dict(pot_dict("bcc-l16-s3"))
    st = structure("bcc", (3, 3, 3), 3.16, 0.08, 3, 2)
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    so = _lib.load()
    cell = np.ascontiguousarray(st.cell.reshape(-1), dtype=np.float64)
    dummy = ctypes.c_void_p(x.data_ptr())
    rc = so.mtp_compute_efv_noalloc(pot.handle, nl.handle, dummy, dummy, 65537,
                                    cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, dummy, dummy, dummy,
                                    dummy, None)
    assert rc == -1
    assert b"at most 65536" in so.mtp_last_error()
