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
// One CTA (4 warps) per output tile, up to three CTAs per SM.  Per round of RB
// input rows the threads load the rows once (coalesced), split them into bf16
// halves, build the Hankel arrays Z_hi, Z_lo from aligned 16-byte loads and a
// funnel shift, and one thread issues the rows' 6 MMAs each (two K steps of 16
// x three products) and commits them to the mbarrier of that Z buffer; the two
// Z buffers alternate, so a round's staging overlaps the previous round's MMAs,
// and a buffer is refilled only after its commit (bounded waits).  The
// accumulators are read back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31, i.e. columns j) and D = I - M is written over the valid region.
#include <cuda_bf16.h>
#include <cstdint>

#include "../../include/dia.h"
#include "dia_ops.cuh"

namespace dia {

namespace {

constexpr int kTcNO = 32;                  // output rows per tile (MMA N)
constexpr int kTcW = 128;                  // output columns per tile (MMA M)
constexpr int kTcRB = 4;                   // input rows per round
constexpr int kTcChunks = (kTcW + 32) / 8; // 16-byte chunks of one Hankel row array
constexpr int kTcZBytes = kTcChunks * 128; // one input row's Z array (bf16)
constexpr uint32_t kZBytesRow = kTcZBytes;
constexpr int kTcRaw = kTcW + 48;          // raw row segment (bf16), >= 8 * kTcChunks + 8
constexpr int kTcKRows = 96;               // >= 31 + 2 * kTcNO, multiple of 8
constexpr int kTcKBytes = 4 * kTcKRows * 16;
constexpr int kTcProducers = 128;           // warps 0-3: staging and epilogue
constexpr int kTcThreads = kTcProducers + 32;  // warp 4: TMEM owner and MMA issuer
constexpr long long kTcWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

struct TcSmem {
    __nv_bfloat16 z[2][2][kTcRB][kTcZBytes / 2];   // [buffer][hi|lo][row][Z]
    __nv_bfloat16 raw[2][kTcRB][kTcRaw];           // [hi|lo][row][x]: the round's R rows
    float rawf[2][kTcRB][kTcRaw];                  // [buffer][row][x]: prefetched R rows
    __nv_bfloat16 k[2][kTcKBytes / 2];             // [hi|lo][kc][row][8]
    uint64_t full[2];    // Z buffer written (128 producer arrivals)
    uint64_t empty[2];   // Z buffer read by its MMAs (tcgen05.commit)
    uint64_t done;       // every MMA of the tile finished (tcgen05.commit)
    uint32_t tslot;
    int fail;            // producers only: written before and read after their barrier
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

// Wait for the phase with parity `ph` of the mbarrier (try_wait suspends the
// thread for a while between checks); false after kTcWaitCycles.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t ph) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(ph));
        if (done) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

// cp.async of R rows r0 .. r0 + nr - 1 of the tile into rawf (zeros outside the
// image); 16-byte copies when rows are 16-byte aligned
__device__ __forceinline__ void tc_prefetch(float (*dst)[kTcRaw], const float *R, int H, int W,
                                            int ld, int gy0, int x0, int nr, bool vec) {
    if (vec) {
        for (int i = threadIdx.x; i < nr * (kTcRaw / 4); i += kTcProducers) {
            const int rr = i / (kTcRaw / 4), c4 = i % (kTcRaw / 4);
            const int gy = gy0 + rr, gx = x0 + 4 * c4;
            int bytes = 0;
            const float *src = R;
            if (gy < H && gx < W) {
                bytes = (W - gx >= 4) ? 16 : 4 * (W - gx);
                src = R + (size_t)gy * ld + gx;
            }
            cp_async16(&dst[rr][4 * c4], src, bytes);
        }
    } else {
        for (int i = threadIdx.x; i < nr * kTcRaw; i += kTcProducers) {
            const int rr = i / kTcRaw, x = i % kTcRaw;
            const int gy = gy0 + rr, gx = x0 + x;
            const bool in = gy < H && gx < W;
            cp_async4(&dst[rr][x], in ? R + (size_t)gy * ld + gx : R, in ? 4 : 0);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// 8 consecutive bf16 starting at element t (0..7) of the 16 held in (a, b)
// (word selection by predicated moves, so the words stay in registers)
__device__ __forceinline__ uint4 shift8(const uint4 a, const uint4 b, int t) {
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const int q = t >> 1;
    uint32_t s[5];   // words q .. q + 4
#pragma unroll
    for (int k = 0; k < 5; ++k)
        s[k] = q == 0 ? w[k] : q == 1 ? w[k + 1] : q == 2 ? w[k + 2] : w[k + 3];
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = (t & 1) ? __funnelshift_r(s[k], s[k + 1], 16) : s[k];
    return make_uint4(o[0], o[1], o[2], o[3]);
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

__device__ __forceinline__ void mbar_init(uint64_t *b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(su32(b)));
}
__device__ __forceinline__ bool failed(const TcSmem &S) {
    return *reinterpret_cast<const volatile int *>(&S.fail) != 0;
}
// (the MMA warp reports a failed wait through the global status word only, so
// that the producers' flag is never written while they read it)

// Warp-specialised: warps 0-3 stage the rounds' rows (named barrier 1 among
// them) and signal full[buf]; warp 4 (one lane) waits on full[buf], issues the
// round's MMAs and commits them to empty[buf], which the producers wait on
// before refilling that buffer; after the last round it commits to `done`, on
// which the producers wait before reading the accumulators.
__global__ void __launch_bounds__(kTcThreads, 3) tc_forward_kernel(const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    const int y0 = (blockIdx.x / a.tiles_x) * kTcNO, x0 = (blockIdx.x % a.tiles_x) * kTcW;

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(32));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&S.full[0], kTcProducers);
        mbar_init(&S.full[1], kTcProducers);
        mbar_init(&S.empty[0], 1);
        mbar_init(&S.empty[1], 1);
        mbar_init(&S.done, 1);
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
    const int nrows = kTcNO + m - 1, nrounds = (nrows + kTcRB - 1) / kTcRB;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = S.tslot;

    if (warp == 4) {
        if (lane == 0) {
            // descriptors of a round's first row; rows and K steps add byte
            // offsets >> 4 to the start-address field
            const uint32_t idesc = tc_idesc(kTcW, kTcNO);
            const uint64_t dz0 = tc_desc(su32(&S.z[0][0][0][0]), 128, 128);
            const uint64_t dk0 = tc_desc(su32(&S.k[0][0]), kTcKRows * 16, 128);
            constexpr uint32_t kZsplit = sizeof(S.z[0][0]), kZbuf = sizeof(S.z[0]);
            constexpr uint32_t kKsplit = sizeof(S.k[0]);
            bool ok = true;
            for (int k = 0; k < nrounds && ok; ++k) {
                const int buf = k & 1, r0 = k * kTcRB, nr = min(kTcRB, nrows - r0);
                if (!tc_wait(su32(&S.full[buf]), (uint32_t)((k >> 1) & 1))) {
                    atomicExch(a.status, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int rr = 0; rr < nr; ++rr) {
                    const int r = r0 + rr;
                    const uint64_t zrow = dz0 + ((buf * kZbuf + rr * kZBytesRow) >> 4);
                    const uint64_t krow = dk0 + (((uint32_t)(m - 1 - r + kTcNO) * 16) >> 4);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint64_t ahi = zrow + (ks * 256 >> 4), alo = ahi + (kZsplit >> 4);
                        const uint64_t bhi = krow + ((2 * ks * kTcKRows * 16) >> 4),
                                       blo = bhi + (kKsplit >> 4);
                        tc_mma(taddr, ahi, bhi, idesc, (r > 0 || ks > 0) ? 1 : 0);
                        tc_mma(taddr, ahi, blo, idesc, 1);
                        tc_mma(taddr, alo, bhi, idesc, 1);
                    }
                }
                tc_commit(&S.empty[buf]);
            }
            tc_commit(&S.done);   // arrives when every MMA issued above has finished
        }
        __syncwarp();
    } else {
        bool ok = true;
        const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.R) & 15) == 0);
        tc_prefetch(S.rawf[0], a.R, a.H, a.W, a.ld, y0, x0, min(kTcRB, nrows), vec);
        for (int k = 0; k < nrounds; ++k) {
            const int buf = k & 1, r0 = k * kTcRB, nr = min(kTcRB, nrows - r0);
            // this round's R rows have landed; the next round's are requested
            cp_async_wait<0>();
            asm volatile("bar.sync 1, %0;" :: "n"(kTcProducers));
            if (k + 1 < nrounds)
                tc_prefetch(S.rawf[buf ^ 1], a.R, a.H, a.W, a.ld, y0 + r0 + kTcRB, x0,
                            min(kTcRB, nrows - r0 - kTcRB), vec);
            // split once: raw[.][rr][x] = R[y0 + r0 + rr][x0 + x]
            for (int i = tid; i < nr * kTcRaw; i += kTcProducers) {
                const int rr = i / kTcRaw, x = i % kTcRaw;
                split_bf16(S.rawf[buf][rr][x], S.raw[0][rr][x], S.raw[1][rr][x]);
            }
            // the MMAs of round k - 2 read this Z buffer: wait for their commit
            if (k >= 2 && ok && !tc_wait(su32(&S.empty[buf]), (uint32_t)(((k - 2) >> 1) & 1)))
                S.fail = 1;
            asm volatile("bar.sync 1, %0;" :: "n"(kTcProducers));
            ok = ok && !failed(S);
            if (!ok) break;
            // Hankel arrays: window s = 8c + t is raw[s .. s + 7]
            for (int i = tid; i < 2 * nr * kTcChunks * 8; i += kTcProducers) {
                const int sp = i / (nr * kTcChunks * 8), rem = i % (nr * kTcChunks * 8);
                const int rr = rem / (kTcChunks * 8), s = rem % (kTcChunks * 8);
                const uint4 *src = reinterpret_cast<const uint4 *>(&S.raw[sp][rr][0]) + (s >> 3);
                *reinterpret_cast<uint4 *>(&S.z[buf][sp][rr][s * 8]) = shift8(src[0], src[1], s & 7);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&S.full[buf]);
        }
        cp_async_wait<0>();
        if (ok && !tc_wait(su32(&S.done), 0)) S.fail = 1;
        asm volatile("bar.sync 1, %0;" :: "n"(kTcProducers));
        ok = ok && !failed(S);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            uint32_t v[kTcNO];
            const uint32_t ta = taddr + ((uint32_t)(32 * warp) << 16);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                           "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                           "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                           "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                           "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                           "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 4)
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
