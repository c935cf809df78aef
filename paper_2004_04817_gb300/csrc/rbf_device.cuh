// rbf_device.cuh -- device helpers shared by the librbfgcb kernels.
//
// Wendland C2 basis (Eq. 2 of arXiv:2004.04817) in FP32 and FP64, argmax key
// packing, and the bounded grid barrier used by the persistent kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rbfgcb.h"

namespace rbf {

constexpr int kWarp = 32;

// ----------------------------------------------------------------------------
// Eq. 2: phi(eta) = (1 - eta)^4 (4 eta + 1) for eta < 1, else 0.  The callers
// pass s = eta^2 (coordinates are pre-scaled by 1/R), so a pair costs one
// square root.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float sqrt_approx(float s)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(s));   // sqrt(0) = 0
    return r;
}

__device__ __forceinline__ float phi_f32_s(float s)
{
    const float eta = sqrt_approx(s);
    const float t = fmaxf(1.0f - eta, 0.0f);
    const float t2 = t * t;
    return (t2 * t2) * fmaf(4.0f, eta, 1.0f);
}

__device__ __forceinline__ double phi_f64_s(double s)
{
    const double eta = sqrt(s);
    const double t = fmax(1.0 - eta, 0.0);
    const double t2 = t * t;
    return (t2 * t2) * fma(4.0, eta, 1.0);
}

// ----------------------------------------------------------------------------
// Argmax keys.  Larger key = larger error; among equal errors the lowest node
// index wins.  Key 0 means "no candidate".
//  - FP64 errors: the top 40 bits of the (non-negative) double's bit pattern,
//    then 24 bits of (0xFFFFFF - node).  Truncation keeps the order of errors
//    that differ by more than 2^-28 relative; the exact FP64 value of the
//    winner is read back from the per-node error buffer.
// ----------------------------------------------------------------------------
constexpr uint64_t kIdxBits = 24;
constexpr uint64_t kIdxMask = (1ull << kIdxBits) - 1;
constexpr int64_t kMaxNodes = (int64_t)kIdxMask;   // node < 2^24 - 1

__device__ __forceinline__ uint64_t key_f64(double e, int node)
{
    const uint64_t b = (uint64_t)__double_as_longlong(e);
    return (b & ~kIdxMask) | (kIdxMask - (uint64_t)node);
}

__device__ __forceinline__ int key_node(uint64_t key)
{
    return (int)(kIdxMask - (key & kIdxMask));
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f32(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Four doubles on a 32-byte boundary (one point: x, y, z and a spare slot).
struct __align__(32) D4 {
    double x, y, z, w;
};

__host__ __device__ __forceinline__ D4 mk4(double x, double y, double z, double w)
{
    D4 r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.w = w;
    return r;
}

// L2-coherent loads for data that other CTAs of a persistent kernel write
// (never served from a possibly stale L1 line).
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ D4 ldcg(const D4 *p)
{
    D4 r;
    asm volatile("ld.global.cg.v2.f64 {%0, %1}, [%2];"
                 : "=d"(r.x), "=d"(r.y) : "l"(p) : "memory");
    asm volatile("ld.global.cg.v2.f64 {%0, %1}, [%2+16];"
                 : "=d"(r.z), "=d"(r.w) : "l"(p) : "memory");
    return r;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ----------------------------------------------------------------------------
// Grid barrier for cooperative launches (all CTAs co-resident).  Every wait is
// bounded: after `limit_ns` the waiting CTA latches RBF_E_TIMEOUT into
// *status and returns false; callers then leave the kernel.
// ----------------------------------------------------------------------------
struct GridBar {
    unsigned int count;
    unsigned int gen;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(GridBar *bar, int *status, unsigned int nblocks,
                                             uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int gen = ld_acquire_u32(&bar->gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(&bar->gen) == gen) {
                __nanosleep(64);
                if (*(volatile int *)status == (int)RBF_E_TIMEOUT) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicExch(status, (int)RBF_E_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (ok && *(volatile int *)status == (int)RBF_E_TIMEOUT)
            ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace rbf
