// rbf_kl.cu -- Kullback-Leibler divergence between two support sets
// (Sec. 4.1 of arXiv:2004.04817):
//     KL(S1 || S2) = sum_{i=1..N_b} d1_i log(d1_i / d2_i),
//     dk_i = min over j in Sk of |r_i - r_j|  for every boundary node i.
// Terms with d1_i = 0 or d2_i = 0 (node i belongs to a set) have no finite
// logarithm and are left out.
//
// Nearest-support distances: one thread per boundary node, support
// coordinates staged in shared memory in chunks, squared distances in FP64
// (a diagnostic: N_b x N_c pairs, 7 FP64 instructions each) with the minimum
// taken on the integer pipe (non-negative doubles order as their bit
// patterns).  The sum: FP64 terms, a fixed tree per CTA and the CTA partials
// added in index order by one thread (deterministic).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "rbf_device.cuh"
#include "rbf_host.h"

namespace rbf {

constexpr int kKlThreads = 256;
constexpr int kKlChunk = 2048;   // support nodes per shared-memory chunk (48 KB)
constexpr int kKlBlocks = 1024;  // CTAs of the sum

__global__ void __launch_bounds__(kKlThreads)
k_nearest_support(const double *__restrict__ xb, int64_t nb, const int32_t *__restrict__ sel,
                  int nc, double *__restrict__ dist)
{
    __shared__ double s_c[3 * kKlChunk];
    for (int64_t base = blockIdx.x * (int64_t)kKlThreads; base < nb;
         base += (int64_t)gridDim.x * kKlThreads) {
        const int64_t i = base + threadIdx.x;
        const int64_t ic = i < nb ? i : nb - 1;
        const double x = xb[3 * ic], y = xb[3 * ic + 1], z = xb[3 * ic + 2];
        unsigned long long best = 0x7FF0000000000000ull;   // +inf
        for (int c0 = 0; c0 < nc; c0 += kKlChunk) {
            const int nt = min(kKlChunk, nc - c0);
            __syncthreads();
            for (int t = threadIdx.x; t < nt; t += kKlThreads) {
                const int64_t n = sel[c0 + t];
                s_c[3 * t] = xb[3 * n];
                s_c[3 * t + 1] = xb[3 * n + 1];
                s_c[3 * t + 2] = xb[3 * n + 2];
            }
            __syncthreads();
            for (int t = 0; t < nt; ++t) {
                const double dx = x - s_c[3 * t], dy = y - s_c[3 * t + 1],
                             dz = z - s_c[3 * t + 2];
                const unsigned long long b = dbits(fma(dz, dz, fma(dy, dy, dx * dx)));
                best = b < best ? b : best;
            }
        }
        if (i < nb)
            dist[i] = sqrt(bitsd(best));
    }
}

// Per-CTA partial sums of d1 log(d1 / d2) over the nodes with d1, d2 > 0.
__global__ void __launch_bounds__(kKlThreads)
k_kl_partial(const double *__restrict__ d1, const double *__restrict__ d2, int64_t nb,
             double *__restrict__ part)
{
    __shared__ double s_w[kKlThreads / kWarp];
    double t = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kKlThreads + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * kKlThreads) {
        const double a = d1[i], b = d2[i];
        if (a > 0.0 && b > 0.0)
            t += a * log(a / b);
    }
    t = warp_sum_f64(t);
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kKlThreads / kWarp; ++w)
            s += s_w[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_kl_final(const double *__restrict__ part, int n, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b)
            s += part[b];
        out[0] = s;
    }
}

}  // namespace rbf

using namespace rbf;

extern "C" size_t rbf_support_kl_workspace_bytes(int64_t nb)
{
    if (nb < 1)
        return 0;
    return align_up(sizeof(double) * 2 * (size_t)nb, 256) +
           align_up(sizeof(double) * (kKlBlocks + 1), 256);
}

extern "C" rbf_status rbf_nearest_support(const double *d_xb, int64_t nb, const int32_t *d_sel_idx,
                                          int64_t nc, double *d_dist, void *stream)
{
    if (nb < 1 || nc < 1 || nc > INT32_MAX || !d_xb || !d_sel_idx || !d_dist)
        return RBF_E_ARG;
    DeviceInfo dev;
    if (!device_info(&dev))
        return RBF_E_CUDA;
    const int grid = (int)std::min<int64_t>((nb + kKlThreads - 1) / kKlThreads, (int64_t)dev.sms * 8);
    k_nearest_support<<<grid, kKlThreads, 0, (cudaStream_t)stream>>>(d_xb, nb, d_sel_idx, (int)nc,
                                                                     d_dist);
    return cudaGetLastError() == cudaSuccess ? RBF_OK : RBF_E_CUDA;
}

extern "C" rbf_status rbf_support_kl(const double *d_xb, int64_t nb, const int32_t *d_sel1,
                                     int64_t nc1, const int32_t *d_sel2, int64_t nc2,
                                     double *h_kl, void *d_ws, size_t ws_bytes, void *stream)
{
    if (nb < 1 || nc1 < 1 || nc2 < 1 || !d_xb || !d_sel1 || !d_sel2 || !h_kl)
        return RBF_E_ARG;
    const size_t need = rbf_support_kl_workspace_bytes(nb);
    if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255) != 0)
        return RBF_E_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    double *d1 = (double *)d_ws, *d2 = d1 + nb;
    double *part = (double *)((char *)d_ws + align_up(sizeof(double) * 2 * (size_t)nb, 256));
    rbf_status s = rbf_nearest_support(d_xb, nb, d_sel1, nc1, d1, stream);
    if (s != RBF_OK)
        return s;
    s = rbf_nearest_support(d_xb, nb, d_sel2, nc2, d2, stream);
    if (s != RBF_OK)
        return s;
    const int nblk = (int)std::min<int64_t>((nb + kKlThreads - 1) / kKlThreads, kKlBlocks);
    k_kl_partial<<<nblk, kKlThreads, 0, st>>>(d1, d2, nb, part);
    k_kl_final<<<1, 32, 0, st>>>(part, nblk, part + kKlBlocks);
    if (cudaGetLastError() != cudaSuccess)
        return RBF_E_CUDA;
    if (cudaMemcpyAsync(h_kl, part + kKlBlocks, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RBF_E_CUDA;
    return RBF_OK;
}
