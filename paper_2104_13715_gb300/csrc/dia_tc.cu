// Tensor-core form of the forward model image (Sec. 2.1, Eq. 2) for sm_103a:
// tcgen05.mma with bf16 operands in shared memory, float32 accumulators in
// tensor memory, three split-precision products per contraction.
//
// The correlation as a GEMM.  For an output tile of NO rows (i) x 128 columns
// (j) starting at valid-region pixel (y0, x0), and each R row r of the tile's
// NO + m - 1 input rows (R row y0 + r),
//   D[j][i] += sum_b A_r[j][b] B_r[i][b],   A_r[j][b] = R[y0 + r][x0 + j + b],
//                                           B_r[i][b] = K[r - i][b] (0 outside [0, m)),
// so that after all input rows D[j][i] = M[y0 + i][x0 + j] - B0.  A_r is a Hankel
// matrix: in the no-swizzle K-major operand layout a core matrix (8 rows x 8
// bf16) of A_r starting at row 8J and column 8k is R[8(J+k) + t + e] (t the row,
// e the column in the core matrix), so one array Z[c][t][e] = R[8c + t + e] holds
// every core matrix and both descriptor strides are 128 bytes (the hardware
// reads overlapping core matrices).  B_r is a window of the row-reversed kernel
// stored with its rows contiguous per 16-byte column chunk, so a window may start
// at any row: B_r starts at row m - 1 - r + NO of the zero-padded reversed K.
//
// Precision: x = hi + lo with hi = bf16(x), lo = bf16(x - hi) for R and K; the
// three products hi*hi + hi*lo + lo*hi are accumulated in float32 (the omitted
// lo*lo term is below 2^-16 of each product).
//
// One CTA (4 warps) per output tile, up to four CTAs per SM.  The input rows are
// staged RB at a time (Z_hi, Z_lo), one thread issues their 6 MMAs each (two
// K steps of 16 x three products) and commits them to an mbarrier that every
// thread waits on (bounded) before the buffers are refilled; the accumulators
// are read back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
// columns j) and D = I - M is written over the valid region.
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/dia.h"
#include "dia_ops.cuh"

namespace dia {

namespace {

constexpr int kTcNO = 32;                  // output rows per tile (MMA N)
constexpr int kTcW = 128;                  // output columns per tile (MMA M)
constexpr int kTcRB = 8;                   // input rows staged per round
constexpr int kTcChunks = (kTcW + 32) / 8; // 16-byte chunks of one Hankel row array
constexpr int kTcZBytes = kTcChunks * 128; // one input row's Z array (bf16)
constexpr int kTcKRows = 96;               // >= 31 + 2 * kTcNO, multiple of 8
constexpr int kTcKBytes = 4 * kTcKRows * 16;
constexpr int kTcThreads = 128;
constexpr long long kTcWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

struct TcSmem {
    __nv_bfloat16 z[2][kTcRB][kTcZBytes / 2];   // [hi|lo][row][Z]
    __nv_bfloat16 k[2][kTcKBytes / 2];          // [hi|lo][kc][row][8]
    unsigned long long mbar;
    uint32_t tslot;
    int fail;
};

__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// no-swizzle K-major shared-memory matrix descriptor (start, leading = K-direction
// core-matrix stride, stride = M/N-direction 8-row stride; version 1)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: f32 accumulators, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t a, uint64_t b, uint32_t idesc,
                                       int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(taddr), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Wait for the phase with parity `ph` of the mbarrier; false after kTcWaitCycles.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t ph) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(ph));
        if (done) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

struct TcArgs {
    const float *R, *I;
    int H, W, ld, m;
    int Hv, Wv, tiles_x;
    const float *Kpad;   // m rows of kp floats, then B0
    int kp;
    float *diff_out;     // (Hv x Wv) D = I - M
    int *status;         // set to 1 if a wait ran out
};

__global__ void __launch_bounds__(kTcThreads, 4) tc_forward_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    const int y0 = (blockIdx.x / a.tiles_x) * kTcNO, x0 = (blockIdx.x % a.tiles_x) * kTcW;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(32));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(&S.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        S.fail = 0;
    }
    // reversed, zero-padded kernel: row t holds K[m - 1 - (t - NO)][b] for
    // t - NO in [0, m), as [kc][t][e] with b = 8 kc + e
    for (int i = tid; i < 4 * kTcKRows * 8; i += kTcThreads) {
        const int kc = i / (kTcKRows * 8), t = (i / 8) % kTcKRows, e = i % 8;
        const int ar = m - 1 - (t - kTcNO), b = 8 * kc + e;
        const float v = (ar >= 0 && ar < m && b < m) ? a.Kpad[ar * a.kp + b] : 0.f;
        split_bf16(v, S.k[0][i], S.k[1][i]);
    }
    const float B0 = a.Kpad[m * a.kp];
    const int nrows = kTcNO + m - 1;
    const uint32_t idesc = tc_idesc(kTcW, kTcNO);
    const uint32_t mb = su32(&S.mbar);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = S.tslot;

    bool ok = true;
    int round = 0;
    for (int r0 = 0; r0 < nrows; r0 += kTcRB, ++round) {
        const int nr = min(kTcRB, nrows - r0);
        // Z arrays of input rows r0 .. r0 + nr - 1: window s = 8c + t holds
        // R[y0 + r][x0 + s .. x0 + s + 7] (zero beyond the image)
        for (int i = tid; i < nr * kTcChunks * 8; i += kTcThreads) {
            const int rr = i / (kTcChunks * 8), s = i % (kTcChunks * 8);
            const int gy = y0 + r0 + rr;
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int gx = x0 + s + e;
                const float v = (gy < a.H && gx < a.W) ? __ldg(a.R + (size_t)gy * a.ld + gx) : 0.f;
                split_bf16(v, hi[e], lo[e]);
            }
            *reinterpret_cast<uint4 *>(&S.z[0][rr][s * 8]) = *reinterpret_cast<const uint4 *>(hi);
            *reinterpret_cast<uint4 *>(&S.z[1][rr][s * 8]) = *reinterpret_cast<const uint4 *>(lo);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int rr = 0; rr < nr; ++rr) {
                const int r = r0 + rr;
                const uint32_t brow = (uint32_t)(m - 1 - r + kTcNO) * 16;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ahi = tc_desc(su32(&S.z[0][rr][0]) + ks * 256, 128, 128);
                    const uint64_t alo = tc_desc(su32(&S.z[1][rr][0]) + ks * 256, 128, 128);
                    const uint32_t koff = (uint32_t)(2 * ks) * kTcKRows * 16 + brow;
                    const uint64_t bhi = tc_desc(su32(&S.k[0][0]) + koff, kTcKRows * 16, 128);
                    const uint64_t blo = tc_desc(su32(&S.k[1][0]) + koff, kTcKRows * 16, 128);
                    tc_mma(taddr, ahi, bhi, idesc, (r > 0 || ks > 0) ? 1 : 0);
                    tc_mma(taddr, ahi, blo, idesc, 1);
                    tc_mma(taddr, alo, bhi, idesc, 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mb));
        }
        // the MMAs of this round have read the buffers (and written D) when the
        // phase completes
        if (ok && !tc_wait(mb, (uint32_t)(round & 1))) {
            ok = false;
            S.fail = 1;
        }
        __syncthreads();
        ok = ok && (S.fail == 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        uint32_t v[kTcNO];
        const uint32_t ta = taddr + ((uint32_t)(32 * warp) << 16);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                       "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                       "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                       "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                       "=r"(v[30]), "=r"(v[31])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int h = m / 2, x = x0 + 32 * warp + lane;
        if (x < a.Wv) {
#pragma unroll
            for (int i = 0; i < kTcNO; ++i) {
                const int y = y0 + i;
                if (y < a.Hv) {
                    const float Iv = __ldg(a.I + (size_t)(y + h) * a.ld + (x + h));
                    a.diff_out[(size_t)y * a.Wv + x] = Iv - (__uint_as_float(v[i]) + B0);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(a.status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(32));
}

}  // namespace

int tc_smem_bytes() { return (int)sizeof(TcSmem); }

cudaError_t launch_tc_forward(const float *R, const float *I, int H, int W, int ld, int m,
                              const float *Kpad, int kp, float *diff_out, int *status,
                              cudaStream_t s) {
    if (m < 1 || m > 31 || (m & 1) == 0) return cudaErrorInvalidValue;
    TcArgs a;
    a.R = R;
    a.I = I;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.m = m;
    a.Hv = H - 2 * (m / 2);
    a.Wv = W - 2 * (m / 2);
    a.tiles_x = (a.Wv + kTcW - 1) / kTcW;
    a.Kpad = Kpad;
    a.kp = kp;
    a.diff_out = diff_out;
    a.status = status;
    const int tiles = a.tiles_x * ((a.Hv + kTcNO - 1) / kTcNO);
    const int smem = tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tc_forward_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc_forward_kernel<<<tiles, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dia
