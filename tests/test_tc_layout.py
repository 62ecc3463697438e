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
