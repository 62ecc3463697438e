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
# The weight-gradient kernel (dia_tc_grad.cu): tiles of GI x GJ of g, the R
# window in the same chunked layout (GYC chunks of 8 rows, GXT columns) read
# as an MN-major A operand, the g tile as a K-major B operand.
GI, GJ, GXT, GYC = 64, 128, 160, 12


def _operand_mn(buf, start, lbo, sbo, rows, cols):
    """An MN-major operand (rows = M or N, cols = K): core matrices of 8 K
    rows of 16 bytes, each row holding 8 consecutive M elements; element
    (n, k) at start + (n // 8) SBO + (k // 8) LBO + (k % 8) 16 B + (n % 8) 2 B."""
    n = np.arange(rows)[:, None]
    k = np.arange(cols)[None, :]
    idx = start + (n // 8) * sbo + (k // 8) * lbo + (k % 8) * 8 + (n % 8)
    return buf[idx]


@pytest.mark.parametrize("m", [1, 3, 7, 13, 25, 31])
def test_gradient_operands_and_diagonal_sums_give_the_correlation(m):
    """dK[a][b] = sum_{i,j} g[i][j] W[i + a][j + b] from the kernel's operands:
    P_b = A_b B^T with A_b the MN-major window shifted by b columns (16 b
    bytes) and B the K-major g tile, summed over K steps of 16; then
    dK[a][b] = sum_i P_b[i + a][i]."""
    rng = np.random.default_rng(m)
    Wwin = rng.normal(size=(GYC * 8, GXT))           # the window W[y][x]
    g = rng.normal(size=(GI, GJ))
    # T[yc][x][e] = W[8 yc + e][x] (one split), followed by the other split and
    # the g tile so that rows of A beyond the window stay in the buffer
    T = np.zeros((GYC, GXT, 8))
    for yc in range(GYC):
        for e in range(8):
            T[yc, :, e] = Wwin[8 * yc + e]
    # g tile K-major: [i / 8][j / 8][i % 8][j % 8]
    Gs = np.zeros((GI // 8, GJ // 8, 8, 8))
    for i in range(GI):
        for j in range(GJ):
            Gs[i // 8, j // 8, i % 8, j % 8] = g[i, j]
    buf = np.concatenate([T.ravel(), np.full(T.size, np.nan), Gs.ravel(), Gs.ravel()])
    gbase = 2 * T.size
    dK = np.zeros((m, m))
    for b in range(m):
        P = np.zeros((128, GI))
        for ks in range(GJ // 16):
            A = _operand_mn(buf, b * 8 + ks * 128, 64, GXT * 8, 128, 16)   # (y, j)
            B = _operand(buf, gbase + ks * 128, 64, (GJ // 8) * 64, GI, 16)   # (i, j)
            P += np.nan_to_num(A) @ B.T
        for a in range(m):
            dK[a, b] = sum(P[i + a, i] for i in range(GI))
    ref = np.array([[np.sum(g * Wwin[a:a + GI, b:b + GJ]) for b in range(m)] for a in range(m)])
    np.testing.assert_allclose(dK, ref, rtol=1e-12, atol=1e-9)


def test_gradient_descriptors_stay_in_shared_memory():
    """Every byte the gradient kernel's descriptors reach lies inside its
    operand arrays: A rows 96..127 of the second split run into the g tile
    (ignored rows), the last column shift and K step stay inside a row."""
    t_split = GYC * GXT * 16                       # bytes of one window split
    g_bytes = 2 * GI * GJ * 2
    m = 31
    last_a = t_split + (m - 1) * 16 + (GJ // 16 - 1) * 256 + 15 * GXT * 16 + 128 + 127
    assert last_a < 2 * t_split + g_bytes
    last_b = g_bytes // 2 + (GJ // 16 - 1) * 256 + (GI // 8 - 1) * (GJ // 8) * 128 + 128 + 127
    assert last_b < g_bytes
    # the columns a K step reads: b + 16 ks + 15 < GXT
    assert (m - 1) + 16 * (GJ // 16 - 1) + 15 < GXT
