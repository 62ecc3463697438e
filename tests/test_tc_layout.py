"""The operand layouts of the tensor-core forward pass, checked on the CPU.

The tcgen05 shared-memory descriptors of the kernel (no swizzle, K-major) place
element (row n, column k) of an operand at byte
    start + (n // 8) * SBO + (k // 8) * LBO + (n % 8) * 16 + (k % 8) * 2.
With the kernel's arrays (the column-major R window T[y/8][x][y%8] and the
Hankel arrays Zk_b[c][t][e] = K[8c + t + e - 31][b]) and its start offsets and
strides, the sum over kernel columns b and K steps of A_b B_b^T must be the
correlation of Eq. 2 for every kernel side; this test rebuilds the operands
through that address formula and compares."""
import numpy as np
import pytest

NO, MT, XT, YT, KC = 32, 128, 160, 64, 12   # the kernel's tile constants


def _operand(buf, start, lbo, sbo, rows, cols):
    """Gather a rows x cols operand through the descriptor address formula
    (offsets in bf16 elements: 16-byte rows are 8 elements)."""
    n = np.arange(rows)[:, None]
    k = np.arange(cols)[None, :]
    idx = start + (n // 8) * sbo + (k // 8) * lbo + (n % 8) * 8 + (k % 8)
    return buf[idx]


@pytest.mark.parametrize("m", [1, 3, 5, 9, 17, 25, 31])
def test_window_and_hankel_operands_give_the_correlation(m):
    rng = np.random.default_rng(m)
    H, W = NO + m - 1 + 2, MT + m - 1 + 3
    R = rng.normal(size=(H, W))
    K = rng.normal(size=(m, m))
    # T[yc][x][e] = R[8 yc + e][x] (zero outside the image)
    T = np.zeros((YT // 8, XT, 8))
    for yc in range(YT // 8):
        for e in range(8):
            y = 8 * yc + e
            if y < H:
                T[yc, :min(XT, W), e] = R[y, :min(XT, W)]
    T = T.ravel()
    # Zk_b[c][t][e] = K[8c + t + e - (NO - 1)][b]
    s = (8 * np.arange(KC)[:, None, None] + np.arange(8)[None, :, None] +
         np.arange(8)[None, None, :]) - (NO - 1)
    nks = (NO + m - 1 + 15) // 16
    D = np.zeros((MT, NO))
    for b in range(m):
        kb = np.where((s >= 0) & (s < m), K[np.clip(s, 0, m - 1), b], 0.0).ravel()
        for ks in range(nks):
            # A_b: start (2 ks) XT + b chunks of 16 bytes, LBO = XT chunks, SBO = 8 chunks
            A = _operand(T, (2 * ks * XT + b) * 8, XT * 8, 64, MT, 16)
            # B_b: start 2 ks blocks of 128 bytes, LBO = SBO = 128 bytes
            B = _operand(kb, 2 * ks * 64, 64, 64, NO, 16)
            D += A @ B.T
    for ip in range(NO):
        i = NO - 1 - ip                     # output rows in reverse order
        if i + m <= H:
            ref = np.array([np.sum(K * R[i:i + m, j:j + m]) for j in range(MT) if j + m <= W])
            np.testing.assert_allclose(D[:len(ref), ip], ref, rtol=0, atol=1e-10)


def test_descriptor_offsets_stay_in_their_arrays():
    """Largest element any descriptor of the kernel reaches: the window rows of
    the last K step and the last column shift stay inside T; the Hankel blocks
    I + Y stay inside Zk_b."""
    for m in (1, 31):
        nks = (NO + m - 1 + 15) // 16
        last_a = (2 * (nks - 1) * XT + (m - 1)) * 8 + (MT // 8 - 1) * 64 + (16 // 8 - 1) * XT * 8 + 63
        assert last_a < (YT // 8) * XT * 8
        last_b = 2 * (nks - 1) * 64 + (NO // 8 - 1) * 64 + (16 // 8 - 1) * 64 + 63
        assert last_b < KC * 64


# ---------------------------------------------------------------------------
# The weight-gradient kernel (dia_tc_grad.cu): tiles of GI x GJ of g as the
# K-major A operand, the R window (GWY rows x GWX columns, chunks of 8 rows)
# as the MN-major B operand whose start moves by one column per kernel column
# b, and the epilogue's diagonal sums by warp shuffles.
GI, GJ, GWY, GWX = 128, 64, 160, 96


def _operand_mn(buf, start, lbo, sbo, rows, cols):
    """An MN-major operand (rows = M or N, cols = K): core matrices of 8 K
    rows of 16 bytes, each row holding 8 consecutive M / N elements; element
    (n, k) at start + (n // 8) SBO + (k // 8) LBO + (k % 8) 16 B + (n % 8) 2 B."""
    n = np.arange(rows)[:, None]
    k = np.arange(cols)[None, :]
    idx = start + (n // 8) * sbo + (k // 8) * lbo + (k % 8) * 8 + (n % 8)
    return buf[idx]


def _grad_operands(Wwin, g):
    """The two stage arrays in float16-element units: the window T[y/8][x][y%8]
    and the g tile [i/8][j/8][i%8][j%8]."""
    T = Wwin.reshape(GWY // 8, 8, GWX).transpose(0, 2, 1).ravel()
    Gs = g.reshape(GI // 8, 8, GJ // 8, 8).transpose(0, 2, 1, 3).ravel()
    return T, Gs


def _epilogue_diagonals(P, m):
    """The epilogue warps' sums: warp w, lane L holds v[c] = P[32w + L][32w + c]
    (c < 64); lane a adds, in order of c, the value lane c - a holds at c when
    0 <= c - a < 32.  Returns the per-warp sums [w][a] for a < m."""
    out = np.zeros((4, m))
    for w in range(4):
        v = P[32 * w:32 * w + 32, 32 * w:32 * w + 64]
        for a in range(m):
            for c in range(64):
                src = c - a
                if 0 <= src < 32:
                    out[w, a] += v[src, c]
    return out


@pytest.mark.parametrize("m", [1, 3, 7, 13, 25, 31])
def test_gradient_operands_and_diagonal_sums_give_the_correlation(m):
    """dK[a][b] = sum_{i,j} g[i][j] W[i + a][j + b] from the kernel's operands:
    P_b = A B_b^T with A the K-major g tile and B_b the MN-major window moved
    by b columns (16 b bytes), summed over K steps of 16; then the epilogue's
    shuffle sums along the diagonals y - i = a of each warp's 32 rows."""
    rng = np.random.default_rng(m)
    Wwin = rng.normal(size=(GWY, GWX))
    g = rng.normal(size=(GI, GJ))
    T, Gs = _grad_operands(Wwin, g)
    dK = np.zeros((m, m))
    for b in range(m):
        P = np.zeros((GI, GWY))
        for ks in range(GJ // 16):
            A = _operand(Gs, ks * 128, 64, (GJ // 8) * 64, GI, 16)              # (i, j)
            B = _operand_mn(T, (16 * ks + b) * 8, 64, GWX * 8, GWY, 16)          # (y, x)
            P += A @ B.T
        dK[:, b] = _epilogue_diagonals(P, m).sum(axis=0)
    ref = np.array([[np.sum(g * Wwin[a:a + GI, b:b + GJ]) for b in range(m)] for a in range(m)])
    np.testing.assert_allclose(dK, ref, rtol=1e-12, atol=1e-9)


def test_gradient_descriptors_and_accumulators_stay_in_bounds():
    """Every element the gradient kernel's descriptors reach lies inside its
    own split array, every window row a diagonal needs is multiplied, and the
    epilogue's tensor-memory columns stay inside their accumulator buffer."""
    m = 31
    nks = GJ // 16
    last_b = (16 * (nks - 1) + (m - 1)) * 8 + (GWY // 8 - 1) * GWX * 8 + 64 + 7 * 8 + 7
    assert last_b < (GWY // 8) * GWX * 8
    last_a = (nks - 1) * 128 + (GI // 8 - 1) * (GJ // 8) * 64 + 64 + 7 * 8 + 7
    assert last_a < GI * GJ
    assert GI - 1 + m - 1 < GWY and GJ - 1 + m - 1 < GWX
    # lane rows 32w .. 32w + 31 need columns up to 32w + 31 + m - 1 < 32w + 64
    assert 31 + m - 1 < 64 and 32 * 3 + 63 < GWY
    # three accumulator buffers of 160 columns at 0, 160, 320 (512 allocated);
    # the epilogue's loads reach column 160 b + 32 w + 63
    assert 3 * GWY <= 512 and 2 * GWY + 32 * 3 + 63 < 512
    # shared memory: two stages of (g hi/lo, window hi/lo) + float64 sums
    stage = 2 * GI * GJ * 2 + 2 * GWY * GWX * 2
    assert 2 * stage + 4 * 31 * 32 * 8 + 2 * 4 * 32 * 4 + 128 <= 232448
