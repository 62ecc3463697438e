// Observed Fisher information (Sec. 2.5, Eq. 15): F = d^2 L / d theta^2 at
// theta.  M is linear in theta = [K, B0] (Eq. 2), so
//   F = sum_p l''(M_p) phi_p phi_p^T,  phi_p = [R window of p, 1],
// the same sum as the preconditioner's Gauss-Newton Hessian with the exact
// per-pixel curvature l'' as the weight, taken over every valid pixel.  This
// file holds the curvature pass and the summary of the factorisation; the
// sum, the Cholesky factorisation (the positive-definiteness test of Sec. 2.5)
// and the inverse (the covariance estimate, Eq. 16) are those of
// dia_precond.cu.
#include <cmath>

#include "dia_eval.cuh"
#include "dia_ops.cuh"

namespace dia {

namespace {

// d^2 l / dM^2 of one pixel (float32), l = rho(z) + ln(v)/2 (the last term
// only for a model-dependent variance), z = (I - M) v^-1/2, v linear in M:
//   z'  = -v^-1/2 - z v' / (2 v)
//   z'' =  v' / (v^3/2) + 3 z v'^2 / (4 v^2)
//   l'' = rho''(z) z'^2 + rho'(z) z'' - v'^2 / (2 v^2).
__device__ __forceinline__ float pixel_curvature(const LossParams &lp, float I, float M,
                                                 float vmap, float F) {
    float v, dv;
    if (lp.var_model == 0) {
        v = vmap;
        dv = 0.f;
    } else {
        const float invGF = lp.inv_gain / F;
        if (lp.var_model == 1) {
            v = lp.s0sq / (F * F) + M * invGF;
            dv = invGF;
        } else {
            v = lp.excess * M * invGF;
            dv = lp.excess * invGF;
        }
        if (v < lp.var_floor) {
            v = lp.var_floor;
            dv = 0.f;
        }
    }
    const float inv_v = 1.0f / v, inv_s = sqrtf(inv_v);
    const float z = (I - M) * inv_s;
    const float q = dv * inv_v;                       // v'/v
    const float z1 = -inv_s - 0.5f * z * q;
    const float z2 = q * inv_s + 0.75f * z * q * q;
    float r1, r2;                                     // rho'(z), rho''(z)
    if (lp.rho == 0) {
        r1 = z;
        r2 = 1.f;
    } else if (lp.rho == 1) {
        const float c = lp.huber_c;
        if (fabsf(z) <= c) {
            r1 = z;
            r2 = 1.f;
        } else {
            r1 = copysignf(c, z);
            r2 = 0.f;
        }
    } else {   // rho = ln(1 + z^2)
        const float t = 1.f + z * z;
        r1 = 2.f * z / t;
        r2 = 2.f * (1.f - z * z) / (t * t);
    }
    float d2 = r2 * z1 * z1 + r1 * z2;
    if (lp.var_model != 0) d2 -= 0.5f * q * q;
    return d2;
}

__global__ void __launch_bounds__(256) fisher_weights_kernel(const EvalArgs a, float *w,
                                                             unsigned long long *count) {
    __shared__ unsigned int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    unsigned int cnt = 0;
    const int h = (a.H - a.Hv) / 2;
    const long long total = (long long)a.Hv * a.Wv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / a.Wv), x = (int)(i % a.Wv);
        const size_t off = (size_t)(y + h) * a.ld + (x + h);
        float out = 0.f;
        if (a.mask == nullptr || a.mask[off] != 0) {
            const float Iv = a.I[off];
            const float M = Iv - w[i];   // w holds D = I - M on entry
            const float vm = a.var ? a.var[off] : a.lp.var_scalar;
            const float F = a.flat ? a.flat[off] : 1.f;
            out = pixel_curvature(a.lp, Iv, M, vm, F);
            ++cnt;
        }
        w[i] = out;
    }
    atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(count, (unsigned long long)s_cnt);
}

// One CTA: log det of the factored H (2 sum ln L_kk over k < n) and the
// smallest squared pivot.
__global__ void fisher_finish_kernel(const double *A64, int n, int np, double *res) {
    __shared__ double s_sum[256], s_min[256];
    double sum = 0.0, mn = INFINITY;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double l = A64[(size_t)k * np + k];
        sum += 2.0 * log(l);
        mn = fmin(mn, l * l);
    }
    s_sum[threadIdx.x] = sum;
    s_min[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
            s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        res[0] = s_sum[0];
        res[1] = s_min[0];
    }
}

}  // namespace

cudaError_t launch_fisher_weights(const EvalArgs &ea, float *w, unsigned long long *count,
                                  cudaStream_t s) {
    fisher_weights_kernel<<<1024, 256, 0, s>>>(ea, w, count);
    return cudaGetLastError();
}

cudaError_t launch_fisher_finish(const double *A64, int n, int np, double *res, cudaStream_t s) {
    fisher_finish_kernel<<<1, 256, 0, s>>>(A64, n, np, res);
    return cudaGetLastError();
}

}  // namespace dia
