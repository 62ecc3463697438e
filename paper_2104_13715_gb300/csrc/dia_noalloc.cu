// dia_loss_grad_noalloc: one loss + gradient evaluation that needs no
// workspace from the caller and allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc, or cannot own a
// workspace buffer -- for example code running inside a host application
// whose device memory is entirely managed by that application's own pool
// (raw allocations are forbidden there), or a pipeline that must not
// allocate after start-up.  Such a caller still passes its own input and
// output buffers; only the scratch moves into this library.
//
// The scratch (per-CTA float64 partial sums, the float32 copy of theta and
// the reduced sums) lives in one file-scope __device__ array of fixed size.
// Every GPU that loads this library keeps that array for the life of the
// process.  Host code cannot use the array's name as a device address, so
// the address is looked up once per device with cudaGetSymbolAddress.
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "../../include/dia.h"
#include "dia_checks.h"
#include "dia_dispatch.h"
#include "dia_eval.cuh"
#include "dia_ops.cuh"

namespace {

using namespace dia;

constexpr size_t kScratchBytes = DIA_NOALLOC_SCRATCH_BYTES;
constexpr size_t kKpadOff = 0;                       // (31*32 + kBgMax + 1) floats
constexpr size_t kRedOff = 4096;                     // up to 31*31 + kBgMax + 4 doubles
constexpr size_t kPartOff = 16384;                   // per-CTA partials
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
std::set<std::pair<int, const void *>> g_attr_set;   // (device, kernel) with the smem attribute

// Device address of the scratch array for the current device (looked up on
// the first call on that device, with the device current).
cudaError_t scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

cudaError_t set_smem_attr(const KernelInfo &ki, int *occ) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_attr_set.count({dev, ki.fn[kModeGrad]})) {
            e = cudaFuncSetAttribute(ki.fn[kModeGrad], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     ki.smem);
            if (e != cudaSuccess) return e;
            g_attr_set.insert({dev, ki.fn[kModeGrad]});
        }
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, ki.fn[kModeGrad], ki.nt, ki.smem);
}

}  // namespace

#define NA_CK(expr)                        \
    do {                                   \
        if ((expr) != cudaSuccess) return DIA_ERR_CUDA; \
    } while (0)

extern "C" dia_status dia_loss_grad_noalloc(const dia_pair *pair, const dia_loss_spec *loss,
                                            const double *theta, double *loss_out,
                                            double *grad_out, void *stream) {
    if (!pair || !loss || !theta || !loss_out || !grad_out || !pair->ref || !pair->img)
        return DIA_ERR_ARG;
    if (pair->mem != DIA_MEM_DEVICE) return DIA_ERR_ARG;
    dia_status rc = check_pair(pair);
    if (rc != DIA_OK) return rc;
    if (pair->kernel_degree != 0) return DIA_ERR_UNSUPPORTED;   // one kernel per image only
    rc = check_loss(loss, pair);
    if (rc != DIA_OK) return rc;
    const int H = pair->H, W = pair->W, ld = pair->ld, m = pair->m;

    KernelInfo ki;
    if (!kernel_info(m, &ki)) return DIA_ERR_UNSUPPORTED;
    if (pair->bg_degree > 0) {   // the kernels with the polynomial background
        ki.fn[kModeGrad] = ki.fn_bg[kModeGrad];
        ki.fn[kModeForward] = ki.fn_bg[kModeForward];
    }
    const size_t part_bytes_per_cta = (size_t)ki.np * sizeof(double);
    const size_t max_ctas = (kScratchBytes - kPartOff) / part_bytes_per_cta;
    // sizes the fixed scratch cannot hold are refused (cannot happen for m <= DIA_MAX_M)
    if ((size_t)(m * ki.kp + kBgMax + 1) * 4 > kRedOff - kKpadOff || (size_t)ki.np * 8 > kPartOff - kRedOff ||
        max_ctas < 1)
        return DIA_ERR_WORKSPACE;

    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    NA_CK(scratch_for_current_device(&scratch));
    int occ = 1;
    NA_CK(set_smem_attr(ki, &occ));
    int dev = 0, sms = 1;
    NA_CK(cudaGetDevice(&dev));
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    const int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h;
    const int tiles_x = (Wv + kTW - 1) / kTW;
    const int n_tiles = tiles_x * ((Hv + ki.th - 1) / ki.th);
    long long grid = (long long)sms * (occ < 1 ? 1 : occ);
    if (grid > n_tiles) grid = n_tiles;
    if (grid > (long long)max_ctas) grid = (long long)max_ctas;   // the kernel loops over tiles

    char *base = (char *)scratch;
    float *kpad = (float *)(base + kKpadOff);
    double *red = (double *)(base + kRedOff);
    double *partials = (double *)(base + kPartOff);

    EvalArgs a;
    memset(&a, 0, sizeof(a));
    a.R = pair->ref;
    a.I = pair->img;
    a.mask = pair->mask;
    a.var = pair->var;
    a.flat = pair->flat;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.Hv = Hv;
    a.Wv = Wv;
    a.tiles_x = tiles_x;
    a.n_tiles = n_tiles;
    a.Kpad = kpad;
    a.partials = partials;
    a.clip_kappa = 5.0f;
    a.lp = to_params(loss);
    set_background(a, pair->bg_degree, H, W, h);
    const int nb = n_background(pair->bg_degree);

    // Every CTA writes all of its partials and the reduction writes every
    // reduced entry, so nothing left in the array by an earlier call is read.
    NA_CK(launch_prep_kpad(theta, m, ki.kp, nb, kpad, s));
    void *params[] = {(void *)&a};
    NA_CK(cudaLaunchKernel(ki.fn[kModeGrad], dim3((unsigned)grid), dim3(ki.nt), params, ki.smem, s));
    NA_CK(launch_reduce(partials, (int)grid, ki.np, red, nullptr, s));
    NA_CK(launch_emit_loss_grad(red, m, nb, loss_out, grad_out, s));
    return DIA_OK;
}
