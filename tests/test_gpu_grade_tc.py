"""Tensor-core arithmetic of the grade product, bit for bit.

The grade kernel multiplies BF16 "slices" (small integers) on the tensor cores
with FP32 accumulation and combines the slice groups exactly in int64.  Its
accuracy claim rests on two facts checked here through the C-ABI verification
hook, on random slices at the largest magnitudes the splitting produces:
every slice-group sum G_d = sum_{s+t=d} X_s Y_t with d <= 7 is exact (it stays
below 2^24), and the grade equals max_k |T_k| 2^(f_k + e_i - 56) with
T = sum_d G_d 2^(56 - 8d), computed here in exact integer arithmetic.
Three tiles of rows, the last one ragged."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_SLICES, K = 7, 128


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00193_gb300 import build as B
    B.build()
    import paper_2510_00193_gb300 as P
    return P


def bf16_bits(q):
    """BF16 encodings of small integers (at most 8 significant bits: exact)."""
    return (np.asarray(q, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def pack_x(X):
    """[rows, S, 128] integer slices -> the kernel's X operand layout, per tile
    [S][128 x 128]: element (i, j) at (j/8)*1024 + (i/8)*64 + (i%8)*8 + j%8."""
    n = X.shape[0]
    tiles = (n + 127) // 128
    out = np.zeros((tiles, N_SLICES, 128 * K), dtype=np.uint16)
    i = np.arange(128)[:, None]
    j = np.arange(K)[None, :]
    pos = (j // 8) * 1024 + (i // 8) * 64 + (i % 8) * 8 + j % 8
    for t in range(tiles):
        blk = np.zeros((128, N_SLICES, K))
        rows = X[t * 128:(t + 1) * 128]
        blk[:len(rows)] = rows
        for s in range(N_SLICES):
            out[t, s, pos.ravel()] = bf16_bits(blk[:, s, :]).ravel()
    return out


def pack_y(Y):
    """[S, 128 (j), 128 (k)] -> [2 halves][S * 64 x 128]: per half one operand
    whose row kg = 64 s + k is column k of slice s; element (kg, j) at
    (j/8)*(8 * 64 S) + (kg/8)*64 + (kg%8)*8 + j%8."""
    rows = N_SLICES * 64
    out = np.zeros((2, rows * K), dtype=np.uint16)
    kg = np.arange(rows)[:, None]
    j = np.arange(K)[None, :]
    pos = (j // 8) * (8 * rows) + (kg // 8) * 64 + (kg % 8) * 8 + j % 8
    for h in range(2):
        blk = np.concatenate([Y[s][:, h * 64:(h + 1) * 64].T for s in range(N_SLICES)], axis=0)   # [rows, K]
        out[h, pos.ravel()] = bf16_bits(blk).ravel()
    return out


def random_slices(g, shape_first, shape_rest):
    """Slice 1 in [-256, 256], slices 2..7 in [-128, 128] (the ranges that
    round-to-nearest splitting produces)."""
    out = [g.integers(-256, 257, size=shape_rest)]
    out += [g.integers(-128, 129, size=shape_rest) for _ in range(N_SLICES - 1)]
    return np.stack(out, axis=shape_first)


def test_slice_groups_are_exact_and_grade_is_exact(P):
    g = np.random.default_rng(20251007)
    n = 300
    X = random_slices(g, 1, (n, K))             # [n, S, K]
    Y = random_slices(g, 0, (K, K))             # [S, K(j), K(k)]
    fexp = g.integers(-20, 21, size=K).astype(np.int32)
    erow = g.integers(-30, 31, size=n).astype(np.int32)
    xs = torch.tensor(pack_x(X).view(np.int16).ravel(), device="cuda")
    ys = torch.tensor(pack_y(Y).view(np.int16).ravel(), device="cuda")
    acc = torch.zeros((n, 2, 7, 64), dtype=torch.float32, device="cuda")
    gam = P.mtp_grade_tc_selftest(xs, ys, torch.tensor(fexp, device="cuda"), torch.tensor(erow, device="cuda"), n,
                                  acc=acc)
    acc = acc.cpu().numpy().astype(np.float64)
    got = np.concatenate([acc[:, 0], acc[:, 1]], axis=2)   # [n, 7 (d = 2..8), 128]
    Xi = X.astype(np.int64)
    Yi = Y.astype(np.int64)
    G = np.zeros((n, 7, K), dtype=np.int64)
    for s in range(N_SLICES):
        for t in range(N_SLICES):
            if s + t <= 6:
                G[:, s + t] += Xi[:, s] @ Yi[t]
    assert np.abs(G[:, :6]).max() <= 2 ** 24
    np.testing.assert_array_equal(got[:, :6], G[:, :6].astype(np.float64))
    # G_8 may exceed 2^24 and round in the accumulator: a few units at most
    assert np.abs(got[:, 6] - G[:, 6]).max() <= 64
    # exact grade from the exact groups (Python integers, no overflow)
    gam = gam.cpu().numpy()
    for i in range(n):
        best = 0.0
        for k in range(K):
            T = sum(int(G[i, a, k]) << (40 - 8 * a) for a in range(6)) + (int(G[i, 6, k]) >> 8)
            best = max(best, abs(float(T)) * 2.0 ** (int(fexp[k]) + int(erow[i]) - 56))
        # the kernel's G_8 may differ by a few units of 2^-64, i.e. below 1 unit of T
        tol = 2.0 ** (int(fexp.max()) + int(erow[i]) - 56) + 2.0 ** -50 * best
        assert abs(gam[i] - best) <= tol, (i, gam[i], best)
