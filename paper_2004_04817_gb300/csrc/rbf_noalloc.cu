// rbf_noalloc.cu -- volume displacement sum for callers that cannot allocate
// device memory.
//
// Some callers of this library cannot call cudaMalloc (or any routine that
// allocates device memory): for example a solver plug-in whose host
// application owns every byte of device memory through its own pool and
// forbids libraries from allocating, or a time-critical loop that must not
// pay for the implicit synchronisation an allocation can cause.  Such
// callers can still pass inputs and outputs, but cannot provide the
// workspace that rbf_deform_volume needs.  rbf_deform_volume_noalloc keeps
// its only scratch -- the packed (centre, weight) table -- in a fixed-size
// array in device global memory that belongs to this library's module.
// Under CUDA's default lazy module loading the driver loads the module, and
// so reserves the array, during the first call on each device (at the
// cudaGetSymbolAddress of the set-up); that call may synchronise the device
// and must stay outside time-critical loops and stream captures.
//
// The FP32 arithmetic is the same as rbf_deform_volume with RBF_PREC_F32;
// volume points are read straight from the caller's FP64 array instead of a
// packed copy.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocQ = 4;
constexpr int kNoAllocTile = 2048;    // centres per shared-memory tile

// The scratch: (centre / R, weight) float4 pairs for up to
// RBF_NOALLOC_MAX_CENTRES centres (256 KiB).  Every GPU that loads the
// library holds it until the process exits.  Host code may not use this name
// as a device address; it uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) float4 g_noalloc_cw[2 * RBF_NOALLOC_MAX_CENTRES];

__global__ void k_noalloc_pack(const double *__restrict__ xb, const int32_t *__restrict__ sel,
                               const double *__restrict__ w, int nc, double inv_r,
                               float4 *__restrict__ cw)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        const int64_t n = sel[j];
        cw[2 * j] = make_float4((float)(xb[3 * n] * inv_r), (float)(xb[3 * n + 1] * inv_r),
                                (float)(xb[3 * n + 2] * inv_r), 0.0f);
        cw[2 * j + 1] = make_float4((float)w[3 * j], (float)w[3 * j + 1], (float)w[3 * j + 2], 0.0f);
    }
}

template <int Q>
__global__ void __launch_bounds__(kNoAllocThreads)
k_noalloc_volume(const double *__restrict__ xv, int64_t nv, double inv_r,
                 const float4 *__restrict__ cw, int nc, double *__restrict__ out)
{
    extern __shared__ float4 s_tab[];
    const int tid = threadIdx.x;
    const int64_t per_block = (int64_t)kNoAllocThreads * Q;
    const bool one_tile = nc <= kNoAllocTile;
    if (one_tile) {
        for (int j = tid; j < 2 * nc; j += kNoAllocThreads)
            s_tab[j] = cw[j];
        __syncthreads();
    }
    for (int64_t base = blockIdx.x * per_block; base < nv; base += (int64_t)gridDim.x * per_block) {
        float qx[Q], qy[Q], qz[Q], ax[Q], ay[Q], az[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int64_t v = base + (int64_t)i * kNoAllocThreads + tid;
            v = v < nv ? v : nv - 1;
            qx[i] = (float)(xv[3 * v] * inv_r);
            qy[i] = (float)(xv[3 * v + 1] * inv_r);
            qz[i] = (float)(xv[3 * v + 2] * inv_r);
            ax[i] = 0.0f;
            ay[i] = 0.0f;
            az[i] = 0.0f;
        }
        for (int t0 = 0; t0 < nc; t0 += kNoAllocTile) {
            const int nt = min(kNoAllocTile, nc - t0);
            if (!one_tile) {
                __syncthreads();
                for (int j = tid; j < 2 * nt; j += kNoAllocThreads)
                    s_tab[j] = cw[2 * t0 + j];
                __syncthreads();
            }
#pragma unroll 2
            for (int j = 0; j < nt; ++j) {
                const float4 c = s_tab[2 * j];
                const float4 w = s_tab[2 * j + 1];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float dx = qx[i] - c.x, dy = qy[i] - c.y, dz = qz[i] - c.z;
                    const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    const float ph = phi_f32_s(s);
                    ax[i] = fmaf(w.x, ph, ax[i]);
                    ay[i] = fmaf(w.y, ph, ay[i]);
                    az[i] = fmaf(w.z, ph, az[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int64_t v = base + (int64_t)i * kNoAllocThreads + tid;
            if (v < nv) {
                out[3 * v] = (double)ax[i];
                out[3 * v + 1] = (double)ay[i];
                out[3 * v + 2] = (double)az[i];
            }
        }
    }
}

// Device address of the scratch array, looked up once per device with that
// device current.
struct NoAllocDev {
    float4 *cw = nullptr;
    int occ = 0;
    bool ready = false;
};

static bool noalloc_setup(int dev, NoAllocDev *out)
{
    static std::mutex mu;
    static std::vector<NoAllocDev> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev)
        cache.resize(dev + 1);
    NoAllocDev &d = cache[dev];
    if (!d.ready) {
        float4 *ptr = nullptr;
        if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_cw) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return false;
        }
        const int smem = (int)(sizeof(float4) * 2 * kNoAllocTile);
        if (cudaFuncSetAttribute(k_noalloc_volume<kNoAllocQ>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_noalloc_volume<kNoAllocQ>,
                                                          kNoAllocThreads, smem) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        d.cw = ptr;
        d.occ = std::max(occ, 1);
        d.ready = true;
    }
    *out = d;
    return true;
}

}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_deform_volume_noalloc(const double *d_xv, int64_t nv, const double *d_xb,
                                                const int32_t *d_sel_idx, int64_t nc,
                                                const double *d_w, const rbf_params *p,
                                                double *d_dv, void *stream)
{
    if (!p || nv < 0 || nc < 0 || nc > RBF_NOALLOC_MAX_CENTRES || !(p->radius > 0.0) ||
        p->eval_prec != RBF_PREC_F32 || nv > (int64_t)1 << 40)
        return RBF_E_ARG;
    if (nv > 0 && (!d_xv || !d_dv || (nc > 0 && (!d_xb || !d_sel_idx || !d_w))))
        return RBF_E_ARG;
    // The per-device set-up runs before the empty-input shortcut, so that a
    // call with nv = 0 prepares the device like any other first call.
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    NoAllocDev nd;
    if (!noalloc_setup(dev.device, &nd))
        return RBF_E_CUDA;
    if (nv == 0)
        return RBF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (nc == 0) {
        if (cudaMemsetAsync(d_dv, 0, sizeof(double) * 3 * (size_t)nv, st) != cudaSuccess)
            return RBF_E_CUDA;
        return RBF_OK;
    }
    const double inv_r = 1.0 / p->radius;
    // every entry the volume kernel reads ([0, 2 nc)) is rewritten here, so
    // nothing left from an earlier call is used
    const int cb = (int)std::min<int64_t>((nc + 255) / 256, (int64_t)dev.sms * 4);
    k_noalloc_pack<<<cb, 256, 0, st>>>(d_xb, d_sel_idx, d_w, (int)nc, inv_r, nd.cw);
    const size_t smem = sizeof(float4) * 2 * (size_t)std::min<int64_t>(nc, kNoAllocTile);
    const int64_t want =
        (nv + (int64_t)kNoAllocThreads * kNoAllocQ - 1) / ((int64_t)kNoAllocThreads * kNoAllocQ);
    const int grid = (int)std::min<int64_t>(want, (int64_t)dev.sms * nd.occ);
    k_noalloc_volume<kNoAllocQ><<<grid, kNoAllocThreads, smem, st>>>(d_xv, nv, inv_r, nd.cw,
                                                                     (int)nc, d_dv);
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}
