// Tensor-core form of the weight gradient (the correlation of dl/dM with R,
// Sec. 2.3) for sm_103a.
//
// With g = dl/dM over the valid region (0 where masked or outside it), for a
// tile of 128 rows (i) x 64 columns (j) of g at valid-region pixel (y0, x0)
// and its R window W[y][x] = R[y0 + y][x0 + x] (full-image coordinates,
// 160 x 96):
//   dL/dK[a][b] = sum_{i,j} g[y0+i][x0+j] W[i+a][j+b] = sum_i P_b[i][i+a],
//   P_b[i][y]   = sum_j g[i][j] W[y][j+b],
// one GEMM per kernel column b (M = tile row i, N = window row y, K = tile
// column j) followed by sums along the diagonals y - i = a.  The g tile is a
// K-major A operand; the window is stored in 8-row chunks, T[y/8][x][y%8], so
// B_b = W[.][. + b] is an MN-major operand whose start moves by b * 16 bytes
// (no copy per b).  N = 160 >= 128 + m - 1 window rows are multiplied.
//
// Precision: g and R are scaled by powers of two (from their largest
// magnitudes, which the forward pass reduces) into the range of float16 and
// split x = hi + lo in float16 (22 significant bits together); the products
// hi*hi + hi*lo + lo*hi are accumulated in float32 in tensor memory (the
// dropped lo*lo term and the split leave about 2^-21 of each product), the
// diagonal sums of one tile and kernel column in float32, and everything
// across tiles in float64.
//
// Persistent CTAs (one per SM), warp-specialised, every wait bounded:
//   warps 9-12 stage tile k's operands (scaled, split) into stage k & 1 and
//              arrive on full[k & 1]; they wait on empty[] before reuse;
//   warp 8     owns the tensor memory and, on one lane, issues per kernel
//              column b the 4 K steps x 3 split products into accumulator
//              buffer (round % 3) (128 lanes x 160 columns; three buffers so
//              that the products run up to two columns ahead of the read-back),
//              commits it to afull[], and after the tile's last column
//              commits empty[];
//   warps 0-7  read each accumulator buffer back (warps q and q + 4: lanes
//              32q .. 32q + 31 = tile rows, columns 32q .. 32q + 31 and
//              32q + 32 .. 32q + 63), release it on aempty[], and form the
//              diagonal sums with warp shuffles: lane a of a warp collects
//              diagonal a; warp q hands its sums to warp q + 4 through shared
//              memory at a named barrier of the pair, so every sum has a fixed
//              order and the result does not depend on timing.
#include <cuda_fp16.h>
#include <atomic>
#include <cstdint>
#include <cstring>

#include "../../include/dia.h"
#include "dia_ops.cuh"
#include "dia_tc_ptx.cuh"
#include "dia_tc_grad.h"

namespace dia {

namespace {

constexpr int kGI = kTcGradTileRows;   // tile rows (MMA M)
constexpr int kGJ = kTcGradTileCols;   // tile columns (MMA K: 4 steps of 16)
constexpr int kGWY = kGI + 32;         // window rows (MMA N): 128 + m - 1 <= 160
constexpr int kGWX = kGJ + 32;         // window columns
constexpr int kGYC = kGWY / 8;
constexpr int kGMaxM = kTcGradMaxM;
constexpr int kGEpi = 256;             // warps 0-7: warps q and q + 4 share lanes 32q .. 32q + 31
constexpr int kGMmaWarp = 8;
constexpr int kGProd = 128;            // warps 9-12
constexpr int kGProd0 = kGEpi + 32;
constexpr int kGThreads = kGProd0 + kGProd;
constexpr int kGAcc = kGWY;            // tensor-memory columns per accumulator buffer
constexpr int kGBufs = 3;              // accumulator buffers (3 x 160 of the 512 columns)

struct GradStage {
    __half g[2][kGI / 8][kGJ / 8][8][8];   // [hi|lo][i/8][j/8][i%8][j%8]
    __half t[2][kGYC][kGWX][8];            // [hi|lo][y/8][x][y%8]
};

struct GradSmem {
    GradStage st[2];
    double s64[4][kGMaxM][32];   // per lane quarter: [b][a] float64 totals
    float spart[2][4][32];       // warp q's partial diagonal sums for warp q + 4 (by round parity)
    uint64_t full[2];            // stage staged (kGProd arrivals)
    uint64_t empty[2];           // stage read by its MMAs (tcgen05.commit)
    uint64_t afull[kGBufs];      // accumulator buffer final (tcgen05.commit)
    uint64_t aempty[kGBufs];     // accumulator buffer read back (kGEpi arrivals)
    uint64_t drain;              // every MMA issued has completed
    uint32_t tslot;
    int abort;                   // set by any role whose wait ran out
};

// 2^e with |x| 2^e in [2^13, 2^14) for the largest magnitude x (1 if x == 0)
__device__ __forceinline__ float pow2_scale(float amax) {
    if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
    int e;
    frexpf(amax, &e);   // amax = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ void split_f16(float x, __half &hi, __half &lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

struct GradArgs {
    const float *R;
    int H, W, ld, m;
    const float *G;        // g over the padded valid region, pitch gld (multiple of 4)
    int gld, tiles_x, n_tiles;
    const unsigned *amax;  // [0] max |R| bits, [1] max |g| bits
    double *partials;      // per CTA: np doubles (dK at 1 .. m*m, the rest 0)
    int np;
    int *status;           // [0] 1 if a wait ran out, 3 if a bounds check failed; [1] its index
    long long wait_cycles;
    size_t n_img, n_g;     // elements addressable in R and in G (bounds checks)
    int rows;              // partial rows
    const int *done;       // nullable: nonzero -> return at once (a converged fit's graph)
};

// Named barrier 1 + q over the 64 threads of epilogue warps q and q + 4 with an
// OR reduction of `pred` (the pair leaves its loop together), and the plain
// barrier of the pair.
__device__ __forceinline__ bool pair_any(int q, bool pred) {
    uint32_t any;
    asm volatile("{\n\t.reg .pred c, p;\n\tsetp.ne.u32 c, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, 64, c;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(any) : "r"((uint32_t)pred), "r"(1 + q) : "memory");
    return any != 0;
}
__device__ __forceinline__ void pair_sync(int q) {
    asm volatile("bar.sync %0, 64;" :: "r"(1 + q) : "memory");
}

__device__ __forceinline__ void set_abort(GradSmem &S, int *status) {
    *reinterpret_cast<volatile int *>(&S.abort) = 1;
    atomicExch(status, 1);
}

__global__ void __launch_bounds__(kGThreads, 1) tc_grad_kernel(const GradArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(smem_raw);
    if (a.done != nullptr && *reinterpret_cast<const volatile int *>(a.done) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    if (warp == kGMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.full[i], kGProd);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < kGBufs; ++i) {
            mbar_init(&S.afull[i], 1);
            mbar_init(&S.aempty[i], kGEpi);
        }
        mbar_init(&S.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        S.abort = 0;
    }
    for (int i = tid; i < 4 * kGMaxM * 32; i += kGThreads) (&S.s64[0][0][0])[i] = 0.0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tslot;

    if (warp < 8) {
        // ---- epilogue: diagonal sums of P_b, lane a <- diagonal a ----
        const double unscale = 1.0 / ((double)pow2_scale(__uint_as_float(a.amax[0])) *
                                      (double)pow2_scale(__uint_as_float(a.amax[1])));
        const int q = warp & 3, half = warp >> 2;   // lane quarter, column half
        uint32_t rc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < a.n_tiles && ok; tile += gridDim.x) {
            for (int b = 0; b < m; ++b, ++rc) {
                const uint32_t hb = rc % kGBufs, use = rc / kGBufs;
                ok = tc_wait(&S.afull[hb], use & 1u, &S.abort, a.wait_cycles);
                // both warps of the pair take the same decision (barrier 1 + q)
                ok = !pair_any(q, !ok);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                // columns 32q + 32 half + c (c < 32) of this warp's rows 32q + lane
                uint32_t v[32];
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + hb * (uint32_t)kGAcc +
                                    (uint32_t)(32 * q + 32 * half);
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
                asm volatile("tcgen05.fence::before_thread_sync;");
                mbar_arrive(&S.aempty[hb]);
                // v[c] = P_b[32q + lane][32q + 32 half + c]; lane a takes from lane
                // 32 half + c - a the value of column c (its diagonal is a); four
                // partial sums (c mod 4) keep the dependent adds short, combined in
                // a fixed order
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int src = 32 * half + c - lane;
                    const float t = __shfl_sync(0xffffffffu, __uint_as_float(v[c]), src & 31);
                    if ((unsigned)src < 32u) acc[c & 3] += t;
                }
                const float accs = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                float* const slot = &S.spart[rc & 1][q][lane];
                if (half == 0) {
                    *slot = accs;
                    pair_sync(q);
                } else {
                    pair_sync(q);
                    if (lane < m) S.s64[q][b][lane] += (double)(*slot + accs) * unscale;
                }
            }
        }
        if (!ok && lane == 0) set_abort(S, a.status);
    } else if (warp == kGMmaWarp) {
        // ---- MMA issue (one lane) ----
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(kGI, kGWY, /*a_mn=*/0, /*b_mn=*/1, /*f16=*/1);
            constexpr uint32_t kGs = sizeof(S.st[0].g[0]), kTs = sizeof(S.st[0].t[0]);
            uint32_t rc = 0;
            int k = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
                const int s = k & 1;
                if (!tc_wait(&S.full[s], (uint32_t)((k >> 1) & 1), &S.abort, a.wait_cycles)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                // descriptor bases of this stage; per (b, ks) only the encoded
                // start address advances (by adds: ks 256 B of g, 16 ks + b
                // window columns of 16 B)
                const uint64_t dahi = tc_desc(su32(&S.st[s].g[0][0][0][0][0]), 128, (kGJ / 8) * 128);
                const uint64_t dalo = dahi + (uint64_t)(kGs >> 4);
                const uint64_t dbhi = tc_desc(su32(&S.st[s].t[0][0][0][0]), 128, kGWX * 16);
                const uint64_t dblo = dbhi + (uint64_t)(kTs >> 4);
                for (int b = 0; b < m; ++b, ++rc) {
                    const uint32_t hb = rc % kGBufs, use = rc / kGBufs;
                    if (!tc_wait(&S.aempty[hb], (use & 1u) ^ 1u, &S.abort, a.wait_cycles)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t acc = tmem + hb * (uint32_t)kGAcc;
#pragma unroll
                    for (int ks = 0; ks < kGJ / 16; ++ks) {
                        // A: g tile K-major, K core step 128 B, 8-row step (kGJ / 8) 128 B;
                        // B: window MN-major, K core step 8 columns = 128 B, 8-row step kGWX 16 B
                        const uint64_t ao = (uint64_t)(ks * 16), bo = (uint64_t)(16 * ks + b);
                        if (ks == 0)
                            tc_mma(acc, dahi, dbhi + bo, idesc, 0);
                        else
                            tc_mma_acc(acc, dahi + ao, dbhi + bo, idesc);
                        tc_mma_acc(acc, dahi + ao, dblo + bo, idesc);
                        tc_mma_acc(acc, dalo + ao, dbhi + bo, idesc);
                    }
                    tc_commit(&S.afull[hb]);
                }
                if (!ok) break;
                tc_commit(&S.empty[s]);
            }
            if (!ok) set_abort(S, a.status);
            // every MMA issued completes before the shared and tensor memory go
            tc_commit(&S.drain);
            const int never = 0;
            tc_wait(&S.drain, 0, &never);
        }
        __syncwarp();
    } else {
        // ---- producers: scale, split and stage the operands ----
        const int p = tid - kGProd0;
        const float sR = pow2_scale(__uint_as_float(a.amax[0]));
        const float sG = pow2_scale(__uint_as_float(a.amax[1]));
        int k = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
            const int s = k & 1;
            ok = tc_wait(&S.empty[s], (uint32_t)(((k >> 1) & 1) ^ 1), &S.abort, a.wait_cycles);
            if (!ok) break;
            const int y0 = (tile / a.tiles_x) * kGI, x0 = (tile % a.tiles_x) * kGJ;
            GradStage &st = S.st[s];
            // g tile: unit (i, jc) = 8 columns of row i, i % 8 fastest (the
            // 16-byte stores of a warp fill 512 contiguous bytes)
#pragma unroll 1
            for (int q0 = 0; q0 < 8; q0 += 4) {
                float4 gv[4][2];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const int q = q0 + qq, u = p + kGProd * q;
                    const int i = 8 * (u >> 6) + (u & 7), jc = (u >> 3) & 7;
                    const size_t gi = (size_t)(y0 + i) * a.gld + x0 + 8 * jc;
                    if (gi + 8 <= a.n_g) {
                        const float4 *src = reinterpret_cast<const float4 *>(a.G + gi);
                        gv[qq][0] = __ldg(src);
                        gv[qq][1] = __ldg(src + 1);
                    } else {
                        tc_report_bad(a.status, 3, gi);
                        gv[qq][0] = gv[qq][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const int q = q0 + qq, u = p + kGProd * q;
                    const int i = 8 * (u >> 6) + (u & 7), jc = (u >> 3) & 7;
                    const float f[8] = {gv[qq][0].x, gv[qq][0].y, gv[qq][0].z, gv[qq][0].w,
                                        gv[qq][1].x, gv[qq][1].y, gv[qq][1].z, gv[qq][1].w};
                    __align__(16) __half hi[8], lo[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) split_f16(f[e] * sG, hi[e], lo[e]);
                    *reinterpret_cast<uint4 *>(&st.g[0][i >> 3][jc][i & 7][0]) =
                        *reinterpret_cast<const uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(&st.g[1][i >> 3][jc][i & 7][0]) =
                        *reinterpret_cast<const uint4 *>(lo);
                }
            }
            // window: unit (yc, x) = rows 8 yc .. 8 yc + 7 of column x, three
            // units in flight per thread
            constexpr int kUnits = kGYC * kGWX / kGProd;   // 15
            static_assert(kUnits * kGProd == kGYC * kGWX && kUnits % 3 == 0, "window units");
#pragma unroll 1
            for (int q0 = 0; q0 < kUnits; q0 += 3) {
                float v[3][8];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int u = p + kGProd * (q0 + q);
                    const int yc = u / kGWX, x = u % kGWX;
                    const int gx = x0 + x;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int gy = y0 + 8 * yc + e;
                        const size_t ri = (size_t)gy * a.ld + gx;
                        v[q][e] = (gy < a.H && gx < a.W && ri < a.n_img) ? __ldg(a.R + ri) : 0.f;
                    }
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const int u = p + kGProd * (q0 + q);
                    const int yc = u / kGWX, x = u % kGWX;
                    __align__(16) __half hi[8], lo[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) split_f16(v[q][e] * sR, hi[e], lo[e]);
                    *reinterpret_cast<uint4 *>(&st.t[0][yc][x][0]) = *reinterpret_cast<const uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(&st.t[1][yc][x][0]) = *reinterpret_cast<const uint4 *>(lo);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&S.full[s]);
        }
        if (!ok) set_abort(S, a.status);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * a.np;
    for (int k = tid; k < a.np && (int)blockIdx.x < a.rows; k += kGThreads) {
        double t = 0.0;
        if (k >= 1 && k <= m * m) {
            const int aa = (k - 1) / m, b = (k - 1) % m;
#pragma unroll
            for (int w = 0; w < 4; ++w) t += S.s64[w][b][aa];
        }
        out[k] = t;
    }
    if (warp == kGMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

}  // namespace

int tc_grad_smem_bytes() { return (int)sizeof(GradSmem); }

cudaError_t tc_grad_prepare() {
    static std::atomic<int> done{0};
    if (done.load()) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(tc_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc_grad_smem_bytes());
    if (e == cudaSuccess) done.store(1);
    return e;
}

cudaError_t launch_tc_grad(const float *R, int H, int W, int ld, int m, const float *G, int gld,
                           int Hp, int Wp, const unsigned *amax, double *partials, int np,
                           int rows, int *status, long long wait_cycles, cudaStream_t s,
                           const int *done) {
    if (m < 1 || m > kGMaxM || (m & 1) == 0 || (gld & 3) != 0 || Hp % kGI != 0 ||
        Wp % kGJ != 0 || gld < Wp || (reinterpret_cast<uintptr_t>(G) & 15) != 0 || rows < 1)
        return cudaErrorInvalidValue;
    GradArgs a;
    a.R = R;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.m = m;
    a.G = G;
    a.gld = gld;
    a.tiles_x = Wp / kGJ;
    a.n_tiles = a.tiles_x * (Hp / kGI);
    a.amax = amax;
    a.partials = partials;
    a.np = np;
    a.status = status;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    a.n_img = (size_t)(H - 1) * ld + W;
    a.n_g = (size_t)Hp * gld;
    a.rows = rows;
    a.done = done;
    const int smem = tc_grad_smem_bytes();
    cudaError_t e = tc_grad_prepare();
    if (e != cudaSuccess) return e;
    const int grid = a.n_tiles < rows ? a.n_tiles : rows;
    tc_grad_kernel<<<grid, kGThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the grid may be smaller than its partial rows: clear the rest
    if (grid < rows)
        e = cudaMemsetAsync(partials + (size_t)grid * np, 0, (size_t)(rows - grid) * np * 8, s);
    return e;
}

}  // namespace dia
